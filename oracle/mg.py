"""Multigrid pieces of the domain-wall method, FP64, following Sec. 2.3 and Sec. 3.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings of points the paper leaves open:
  * chiral doubling ("1/2(1+P_pm)" in Sec. 3 is garbled): every relaxed vector
    v is split into P_+ v and P_- v, giving 2*Nvec coarse dof per aggregate,
    ordered [chirality (+, -)][vector]; sigma_3 = diag(+1 x Nvec, -1 x Nvec).
  * block orthonormalisation = Gram-Schmidt of each aggregate's vectors of one
    chirality, in vector order; written here as the Q factor of a QR
    factorisation with a positive real diagonal of R (the same result).
  * "r_1" of Eq. TruncProjectInterpolate is the wall field of the permuted
    basis: (P^dag r)_1 = P_- r_1 + P_+ r_Ls.  Restriction puts
    Phat_- P^dag P_- r_1 on coarse slice 1 and Phat_+ P^dag P_+ r_Ls on slice
    Lhat_s; prolongation is the mirror image onto fine slices 1 and Ls.
  * the setup operator is D_W(m_setup) D_W(m_setup)^dag (Table kcycle) at a
    caller-chosen Wilson mass m_setup; relaxation is CG on the homogeneous
    system from a Gaussian start, at most 250 iterations or a residual
    reduction of 1e-4.
  * the coarse kernel is always P^dag D_W(-M5) P, so the coarse D_DW / D_PV
    of Eq. coarsenDW follow by linearity.
  * post-smoothing: 8 GCR iterations on A z = r starting from the prolonged
    coarse correction (0 pre-smoothing), A = D_PV^dag D_DW (Table kcycle).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import dirac
from .solvers import cgnr_fixed, gcr, norm


def relax_null_vector(Dw, v0, maxiter=250, tol=1e-4):
    """CG on the homogeneous system (D_W D_W^dag) v = 0 from the start v0.

    Returns (v, iterations).  The iterate's residual is -(D_W D_W^dag) v;
    CG stops once it has fallen by `tol` relative to the start or after
    `maxiter` steps (Table kcycle).
    """
    Dd = Dw.conj().T.tocsr()

    def A(v):
        return Dw @ (Dd @ v)

    x = np.array(v0, dtype=complex).ravel()
    r = -A(x)
    r0 = norm(r)
    p = r.copy()
    rr = np.vdot(r, r).real
    it = 0
    while it < maxiter and np.sqrt(rr) > tol * r0:
        Ap = A(p)
        alpha = rr / np.vdot(p, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = np.vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it


def aggregate_map(dims, block):
    """Coarse site of every fine site, and the coarse lattice dims."""
    cdims = tuple(L // b for L, b in zip(dims, block))
    for L, b in zip(dims, block):
        if L % b:
            raise ValueError("block must divide the lattice")
    c = dirac.site_coords(dims)
    cc = c // np.asarray(block)[None, :]
    return dirac.site_index(cc, cdims), cdims


def build_prolongator(vecs, dims, block, nd, nc):
    """Block-orthonormal, chirality-preserving prolongator P (Sec. 2.3).

    vecs: list of Nvec d-dim vectors ([site][spin][color]).  Returns
    (P sparse of shape (V*ns*nc, Vc*2*Nvec), coarse dims).  Columns are
    ordered [coarse site][chirality +,-][vector].
    """
    _, g5 = dirac.gammas(nd)
    chir = np.kron(np.diag(g5).real, np.ones(nc))          # +1 / -1 per site dof
    return build_prolongator_chiral(vecs, dims, block, chir)


def build_prolongator_chiral(vecs, dims, block, chir):
    """The prolongator of build_prolongator for vectors with any per-site dof
    layout: chir[d] = +1 / -1 is the chirality (the gamma_5, or on a coarse
    level the sigma_3, eigenvalue) of site dof d.  Each vector's chiral halves
    are orthonormalised per aggregate, in vector order."""
    chir = np.asarray(chir, dtype=float)
    dof = len(chir)
    V = int(np.prod(dims))
    nvec = len(vecs)
    agg, cdims = aggregate_map(dims, block)
    Vc = int(np.prod(cdims))
    Vm = np.stack([np.asarray(v).reshape(V, dof) for v in vecs], axis=-1)   # (V, dof, nvec)
    rows, cols, vals = [], [], []
    for a in range(Vc):
        sites = np.nonzero(agg == a)[0]
        for ci, sign in enumerate((+1.0, -1.0)):
            d_idx = np.nonzero(chir == sign)[0]
            M = Vm[np.ix_(sites, d_idx)].reshape(len(sites) * len(d_idx), nvec)
            Q, R = np.linalg.qr(M)
            ph = np.diag(R) / np.abs(np.diag(R))
            Q = Q * ph[None, :]
            fine = (sites[:, None] * dof + d_idx[None, :]).reshape(-1)
            for k in range(nvec):
                rows.append(fine)
                cols.append(np.full(fine.shape, (a * 2 + ci) * nvec + k))
                vals.append(Q[:, k])
    P = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(V * dof, Vc * 2 * nvec))
    return P, cdims


def coarse_projectors(Vc, nvec):
    """(Phat_+, Phat_-) = (1 pm sigma_3)/2 on the coarse d-dim space."""
    plus = np.concatenate([np.ones(nvec), np.zeros(nvec)])
    Pp = sp.kron(sp.identity(Vc), sp.diags(plus))
    Pm = sp.kron(sp.identity(Vc), sp.diags(1.0 - plus))
    return Pp.tocsr(), Pm.tocsr()


def galerkin_kernel(P, Dw):
    """Dhat_W = P^dag D_W P, the explicit sparse triple product (Sec. 2.3)."""
    return (P.conj().T @ Dw @ P).tocsr()


def coarse_dwf(Dhat_w, Ls_c, mf, nvec):
    """Coarse Dhat_DW(m) of Eq. coarsenDW: Eq. DWoperator around Dhat_W with Phat_pm."""
    Vc = Dhat_w.shape[0] // (2 * nvec)
    Pp, Pm = coarse_projectors(Vc, nvec)
    return dirac.dwf_from_kernel(Dhat_w, Ls_c, mf, Pp, Pm)


def sigma3(Vc, nvec):
    """sigma_3 = diag(+1 x nvec, -1 x nvec) on every coarse site (the coarse gamma_5)."""
    return sp.kron(sp.identity(Vc), sp.diags(np.concatenate([np.ones(nvec), -np.ones(nvec)]))).tocsr()


def coarse_dwf_dagger_g5(Dhat_w, Ls_c, mf, nvec):
    """Dhat_DW(m)^dag of Eq. coarsenDW with the kernel's adjoint written as
    sigma_3 Dhat_W sigma_3.

    The chirality-preserving prolongator (gamma_5 P = P sigma_3) makes the
    Galerkin kernel gamma_5-hermitian, Dhat_W^dag = sigma_3 Dhat_W sigma_3, so
    for an exact kernel this is the plain adjoint.  For a kernel whose blocks
    were rounded one by one (FP16 storage) the two differ by the rounding, and
    this form is the adjoint that uses one stored copy of the blocks.
    """
    Vc = Dhat_w.shape[0] // (2 * nvec)
    S3 = sigma3(Vc, nvec)
    # a kernel K with K^dag = sigma_3 Dhat_W sigma_3
    K = (S3 @ Dhat_w.conj().T @ S3).tocsr()
    return dirac.dagger(coarse_dwf(K, Ls_c, mf, nvec))


def kernel_blocks(Dhat_w, cdims, ncd):
    """Per-site blocks of a nearest-neighbour coarse kernel: Y[xc][dir] = block
    (xc, neighbour(xc, dir)), dir 0 = self, then +mu, -mu for mu = 0..d-1.
    Every coarse extent must be >= 3 (with extent 2 the two hops land on one
    neighbour and their blocks cannot be told apart)."""
    if min(cdims) < 3:
        raise ValueError("kernel_blocks needs coarse extents >= 3")
    Vc = int(np.prod(cdims))
    nd = len(cdims)
    D = Dhat_w.tocsr()
    Y = np.zeros((Vc, 2 * nd + 1, ncd, ncd), dtype=complex)
    nbrs = [np.arange(Vc)]
    for mu in range(nd):
        nbrs.append(dirac.neighbour(cdims, mu, +1)[0])
        nbrs.append(dirac.neighbour(cdims, mu, -1)[0])
    for xc in range(Vc):
        rows = D[xc * ncd:(xc + 1) * ncd]
        for d, nb in enumerate(nbrs):
            Y[xc, d] = rows[:, nb[xc] * ncd:(nb[xc] + 1) * ncd].toarray()
    return Y


def kernel_from_blocks(Y, cdims):
    """Assemble the sparse coarse kernel from per-site blocks Y[xc][dir] (the
    layout of kernel_blocks).  On lattices with extent 2 the +mu and -mu
    neighbours coincide and their blocks add, as in the operator."""
    Y = np.asarray(Y)
    Vc, ndir, ncd, _ = Y.shape
    nd = (ndir - 1) // 2
    nbrs = [np.arange(Vc)]
    for mu in range(nd):
        nbrs.append(dirac.neighbour(cdims, mu, +1)[0])
        nbrs.append(dirac.neighbour(cdims, mu, -1)[0])
    a = np.arange(ncd)
    rows, cols, vals = [], [], []
    for d, nb in enumerate(nbrs):
        r = (np.arange(Vc)[:, None, None] * ncd + a[None, :, None]) + 0 * a[None, None, :]
        c = (nb[:, None, None] * ncd + a[None, None, :]) + 0 * a[None, :, None]
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(Y[:, d].ravel())
    n = Vc * ncd
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def restrict(r, P, Ls, Ls_c, nd, nc, nvec):
    """Truncated restriction onto the coarse walls (Eq. TruncProjectInterpolate)."""
    V = P.shape[0] // (dirac.n_spin(nd) * nc)
    Pp, Pm = dirac.site_projectors(V, nd, nc)
    Cp, Cm = coarse_projectors(P.shape[1] // (2 * nvec), nvec)
    return restrict_walls(r, P, Ls, Ls_c, Pp, Pm, Cp, Cm)


def prolong(e_c, P, Ls, Ls_c, nd, nc, nvec):
    """Truncated prolongation from the coarse walls (Eq. TruncProjectInterpolate)."""
    V = P.shape[0] // (dirac.n_spin(nd) * nc)
    Pp, Pm = dirac.site_projectors(V, nd, nc)
    Cp, Cm = coarse_projectors(P.shape[1] // (2 * nvec), nvec)
    return prolong_walls(e_c, P, Ls, Ls_c, Pp, Pm, Cp, Cm)


def restrict_walls(r, P, Ls, Ls_c, Pp, Pm, Cp, Cm):
    """Eq. TruncProjectInterpolate between any two levels: Cm P^dag Pm r_1 on coarse
    slice 1 and Cp P^dag Pp r_Ls on coarse slice Ls_c (zero elsewhere); (Pp, Pm) and
    (Cp, Cm) are the chirality projectors of the finer and the coarser level."""
    nf = P.shape[0]
    r = np.asarray(r).reshape(Ls, nf)
    rho = P.conj().T @ (Pm @ r[0] + Pp @ r[Ls - 1])
    out = np.zeros((Ls_c, P.shape[1]), dtype=complex)
    out[0] = Cm @ rho
    out[Ls_c - 1] += Cp @ rho
    return out.reshape(-1)


def prolong_walls(e_c, P, Ls, Ls_c, Pp, Pm, Cp, Cm):
    """The mirror of restrict_walls: Pm P e_1 on slice 1 and Pp P e_{Ls_c} on slice Ls."""
    nf = P.shape[0]
    e_c = np.asarray(e_c).reshape(Ls_c, P.shape[1])
    eta = P @ (Cm @ e_c[0] + Cp @ e_c[Ls_c - 1])
    out = np.zeros((Ls, nf), dtype=complex)
    out[0] = Pm @ eta
    out[Ls - 1] += Pp @ eta
    return out.reshape(-1)


class TwoLevel:
    """Two-level PV-preconditioned K-cycle of Sec. 2.3 with the Table kcycle parameters."""

    def __init__(self, U, dims, Ls, M5, mf, P, nvec, Ls_c=4, group="u1", antiperiodic=None,
                 coarse_tol=0.05, coarse_maxiter=1024, post_smooth=8, restart=16):
        nd = len(dims)
        self.nd, self.nc = nd, (1 if group == "u1" else 3)
        self.Ls, self.Ls_c, self.nvec, self.P = Ls, Ls_c, nvec, P
        self.Ddw = dirac.dwf_matrix(U, dims, Ls, M5, mf, group, antiperiodic)
        Dpv = dirac.pv_matrix(U, dims, Ls, M5, group, antiperiodic)
        self.Dpv_dag = dirac.dagger(Dpv)
        self.A = (self.Dpv_dag @ self.Ddw).tocsr()
        Dw = dirac.wilson_matrix(U, dims, -M5, group, antiperiodic)
        self.Dhat_w = galerkin_kernel(P, Dw)
        Ddw_c = coarse_dwf(self.Dhat_w, Ls_c, mf, nvec)
        Dpv_c = coarse_dwf(self.Dhat_w, Ls_c, 1.0, nvec)
        self.Ac = (dirac.dagger(Dpv_c) @ Ddw_c).tocsr()
        self.coarse_tol, self.coarse_maxiter = coarse_tol, coarse_maxiter
        self.post_smooth, self.restart = post_smooth, restart
        self.coarse_iters = []

    def precondition(self, r):
        """One K-cycle preconditioner application z = M(r)."""
        rc = restrict(r, self.P, self.Ls, self.Ls_c, self.nd, self.nc, self.nvec)
        ec, it = cgnr_fixed(self.Ac, rc, self.coarse_tol, self.coarse_maxiter)
        self.coarse_iters.append(it)
        e0 = prolong(ec, self.P, self.Ls, self.Ls_c, self.nd, self.nc, self.nvec)
        z, _, _ = gcr(lambda v: self.A @ v, r, x0=e0, maxiter=self.post_smooth)
        return z

    def solve(self, b, tol=1e-10, max_restarts=200):
        """Outer flexible GCR(restart) on D_PV^dag D_DW x = D_PV^dag b.

        Stops on the true residual ||b - D_DW x|| / ||b|| <= tol.
        Returns (x, outer iterations, true relative residual).
        """
        b = np.asarray(b, dtype=complex).ravel()
        bn = norm(b)
        x = np.zeros_like(b)
        outer = 0
        for _ in range(max_restarts):
            rt = b - self.Ddw @ x
            if norm(rt) <= tol * bn:
                break
            rA = self.Dpv_dag @ rt
            # one restart cycle; stop early once the true residual is met
            Z, AZ = [], []
            r = rA.copy()
            for _k in range(self.restart):
                z = self.precondition(r)
                w = self.A @ z
                for zj, wj in zip(Z, AZ):
                    beta = np.vdot(wj, w)
                    w = w - beta * wj
                    z = z - beta * zj
                wn = norm(w)
                w, z = w / wn, z / wn
                alpha = np.vdot(w, r)
                x = x + alpha * z
                r = r - alpha * w
                Z.append(z)
                AZ.append(w)
                outer += 1
                if norm(b - self.Ddw @ x) <= tol * bn:
                    break
        return x, outer, norm(b - self.Ddw @ x) / bn


# ----------------------------------------------------------------------------
# Third level (Table kcycle: level l > 1 has 12 null vectors, 2^2 aggregates)
# ----------------------------------------------------------------------------

def coarse_setup_operator(Dhat_w, M5, m_setup):
    """Dhat_W(m_setup) = P^dag D_W(m_setup) P = Dhat_W + (m_setup + M5) 1: with
    P^dag P = 1 the Wilson mass shift passes through the Galerkin product, so the
    level-2 setup relaxes on the coarse kernel shifted to the setup mass."""
    return (Dhat_w + (m_setup + M5) * sp.identity(Dhat_w.shape[0], format="csr")).tocsr()


def coarse_chirality(nvec):
    """sigma_3 eigenvalue of each coarse site dof [chirality +, -][vector]."""
    return np.concatenate([np.ones(nvec), -np.ones(nvec)])


class ThreeLevel:
    """Three-level PV-preconditioned K-cycle (Sec. 2.3 Summary, Table kcycle), with
    optional deflation of the coarsest level (Table zerospacing).

    Level 1: outer FGCR(restart) on A = D_PV^dag D_DW, post_smooth GCR steps.
    Level 2: Dhat_W = P^dag D_W P on Ls_c slices; the coarse system
      Ahat = Dhat_PV^dag Dhat_DW is solved by flexible GCR to l2_tol (at most
      l2_maxiter steps), preconditioned by the wall restriction to level 3, the
      level-3 solve, the prolongation and l2_post_smooth GCR steps on Ahat.
    Level 3: Dhat2_W = P2^dag Dhat_W P2 on Ls_cc slices; CGNR on
      (Ahat2)^dag Ahat2, Ahat2 = Dhat2_PV^dag Dhat2_DW, to coarsest_tol; with
      n_deflate > 0 it starts from the exact solution of the normal equations on
      the span of the n_deflate lowest eigenvectors of (Ahat2)^dag Ahat2.
    """

    def __init__(self, U, dims, Ls, M5, mf, P, nvec, P2, nvec2, Ls_c=4, Ls_cc=4, group="u1", antiperiodic=None,
                 l2_tol=0.25, l2_maxiter=16, l2_post_smooth=8, coarsest_tol=0.05, coarsest_maxiter=1024,
                 post_smooth=8, restart=16, n_deflate=0):
        nd = len(dims)
        self.nd, self.nc = nd, (1 if group == "u1" else 3)
        self.Ls, self.Ls_c, self.Ls_cc = Ls, Ls_c, Ls_cc
        self.nvec, self.nvec2, self.P, self.P2 = nvec, nvec2, P, P2
        self.Ddw = dirac.dwf_matrix(U, dims, Ls, M5, mf, group, antiperiodic)
        self.Dpv_dag = dirac.dagger(dirac.pv_matrix(U, dims, Ls, M5, group, antiperiodic))
        self.A = (self.Dpv_dag @ self.Ddw).tocsr()
        Dw = dirac.wilson_matrix(U, dims, -M5, group, antiperiodic)
        self.Dhat_w = galerkin_kernel(P, Dw)
        self.A2 = (dirac.dagger(coarse_dwf(self.Dhat_w, Ls_c, 1.0, nvec)) @ coarse_dwf(self.Dhat_w, Ls_c, mf, nvec)).tocsr()
        self.Dhat2_w = galerkin_kernel(P2, self.Dhat_w)
        self.A3 = (dirac.dagger(coarse_dwf(self.Dhat2_w, Ls_cc, 1.0, nvec2))
                   @ coarse_dwf(self.Dhat2_w, Ls_cc, mf, nvec2)).tocsr()
        self.A3dag = dirac.dagger(self.A3)
        Vc = P.shape[1] // (2 * nvec)
        Vc2 = P2.shape[1] // (2 * nvec2)
        self.proj1 = dirac.site_projectors(P.shape[0] // (dirac.n_spin(nd) * self.nc), nd, self.nc)
        self.proj2 = coarse_projectors(Vc, nvec)
        self.proj3 = coarse_projectors(Vc2, nvec2)
        self.l2_tol, self.l2_maxiter, self.l2_post_smooth = l2_tol, l2_maxiter, l2_post_smooth
        self.coarsest_tol, self.coarsest_maxiter = coarsest_tol, coarsest_maxiter
        self.post_smooth, self.restart = post_smooth, restart
        self.defl = None
        if n_deflate > 0:
            from .solvers import low_modes
            self.defl = low_modes((self.A3dag @ self.A3).tocsr(), n_deflate)
        self.l2_iters, self.l3_iters = [], []

    def solve3(self, r3):
        from .solvers import cgnr_deflated
        if self.defl is None:
            e3, it = cgnr_fixed(self.A3, r3, self.coarsest_tol, self.coarsest_maxiter, Ddag=self.A3dag)
        else:
            lam, V = self.defl
            e3, it = cgnr_deflated(self.A3, r3, self.coarsest_tol, self.coarsest_maxiter, V, lam, Adag=self.A3dag)
        self.l3_iters.append(it)
        return e3

    def precondition2(self, r2):
        """Level-2 preconditioner: restrict to level 3, solve, prolong, post-smooth on Ahat."""
        r3 = restrict_walls(r2, self.P2, self.Ls_c, self.Ls_cc, self.proj2[0], self.proj2[1], *self.proj3)
        e3 = self.solve3(r3)
        e0 = prolong_walls(e3, self.P2, self.Ls_c, self.Ls_cc, self.proj2[0], self.proj2[1], *self.proj3)
        z, _, _ = gcr(lambda v: self.A2 @ v, r2, x0=e0, maxiter=self.l2_post_smooth)
        return z

    def solve2(self, r2):
        e2, _, k = gcr(lambda v: self.A2 @ v, r2, tol=self.l2_tol, maxiter=self.l2_maxiter,
                       precond=self.precondition2)
        self.l2_iters.append(k)
        return e2

    def precondition(self, r):
        """Level-1 preconditioner z = M(r): restrict, level-2 solve, prolong, post-smooth on A."""
        r2 = restrict_walls(r, self.P, self.Ls, self.Ls_c, self.proj1[0], self.proj1[1], *self.proj2)
        e2 = self.solve2(r2)
        e0 = prolong_walls(e2, self.P, self.Ls, self.Ls_c, self.proj1[0], self.proj1[1], *self.proj2)
        z, _, _ = gcr(lambda v: self.A @ v, r, x0=e0, maxiter=self.post_smooth)
        return z

    def solve(self, b, tol=1e-10, max_restarts=200):
        """Outer flexible GCR(restart) on D_PV^dag D_DW x = D_PV^dag b, stopped on
        ||b - D_DW x|| / ||b|| <= tol.  Returns (x, outer iterations, true residual)."""
        b = np.asarray(b, dtype=complex).ravel()
        bn = norm(b)
        x = np.zeros_like(b)
        outer = 0
        for _ in range(max_restarts):
            rt = b - self.Ddw @ x
            if norm(rt) <= tol * bn:
                break
            xc, _, k = gcr(lambda v: self.A @ v, self.Dpv_dag @ rt, maxiter=self.restart, precond=self.precondition,
                           tol=tol * bn / max(norm(self.Dpv_dag @ rt), 1e-300) * 0.5)
            x = x + xc
            outer += k
        return x, outer, norm(b - self.Ddw @ x) / bn


# ----------------------------------------------------------------------------
# Transfer-operator study (the paper's discussion section: boundary-only versus
# bulk transfers, local colinearity and the oblique projector)
# ----------------------------------------------------------------------------

def restrict_bulk(r, P, Ls):
    """The bulk alternative to Eq. TruncProjectInterpolate: P^dag on every slice (Lhat_s = Ls)."""
    return (sp.kron(sp.identity(Ls), P.conj().T) @ np.asarray(r).reshape(-1))


def prolong_bulk(e_c, P, Ls):
    """P on every slice (the adjoint of restrict_bulk)."""
    return (sp.kron(sp.identity(Ls), P) @ np.asarray(e_c).reshape(-1))


def colinearity(v, restrict_fn, prolong_fn):
    """||(1 - P R) v|| for a normalised vector v: how well the transfer keeps v."""
    v = np.asarray(v).reshape(-1)
    return norm(v - prolong_fn(restrict_fn(v))) / norm(v)


def oblique(v, A, Ac, restrict_fn, prolong_fn):
    """||(1 - P Ac^-1 R A) v|| / ||v||: the error left in the direction v by one exact coarse-grid
    correction with the coarse operator Ac (dense solve)."""
    v = np.asarray(v).reshape(-1)
    rc = restrict_fn(A @ v)
    ec = np.linalg.solve(Ac.toarray() if hasattr(Ac, "toarray") else Ac, rc)
    return norm(v - prolong_fn(ec)) / norm(v)

"""Fine-level operators of the domain-wall method, assembled as sparse FP64 matrices.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Conventions (readings of points the paper leaves open):
  * gamma basis: d = 2: gamma_1 = sigma_1, gamma_2 = sigma_2, gamma_5 = sigma_3;
    d = 4: chiral basis with gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 =
    diag(1, 1, -1, -1).  P_pm = (1 pm gamma_5)/2 then select spin components.
  * lattice: periodic in every direction unless `antiperiodic[mu]` is set, in
    which case a hop across the mu boundary picks up a factor -1.
  * M5 is the domain-wall height (positive); the kernel is the paper's
    D_W(M5_paper) with M5_paper = -M5, so its diagonal is d - M5 (Sec. 2).
  * the s-hops carry the paper's literal signs: +P_- on block (s, s+1),
    +P_+ on (s+1, s), -m P_+ on (1, Ls), -m P_- on (Ls, 1) (Eq. DWoperator).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


# ----------------------------------------------------------------------------
# gamma matrices and lattice geometry
# ----------------------------------------------------------------------------

def gammas(nd: int):
    """Return ([gamma_1..gamma_nd], gamma_5) for d = 2 or 4 (Hermitian, Euclidean)."""
    s1 = np.array([[0, 1], [1, 0]], dtype=complex)
    s2 = np.array([[0, -1j], [1j, 0]], dtype=complex)
    s3 = np.array([[1, 0], [0, -1]], dtype=complex)
    if nd == 2:
        return [s1, s2], s3
    if nd == 4:
        Z = np.zeros((2, 2), dtype=complex)
        I2 = np.eye(2, dtype=complex)
        g = [np.block([[Z, -1j * sk], [1j * sk, Z]]) for sk in (s1, s2, s3)]
        g.append(np.block([[Z, I2], [I2, Z]]))
        g5 = g[0] @ g[1] @ g[2] @ g[3]
        return g, g5
    raise ValueError("nd must be 2 or 4")


def n_spin(nd: int) -> int:
    return 2 if nd == 2 else 4


def site_coords(dims):
    """Coordinates of every site, shape (V, nd), x0 fastest."""
    V = int(np.prod(dims))
    idx = np.arange(V)
    out = np.empty((V, len(dims)), dtype=np.int64)
    for mu, L in enumerate(dims):
        out[:, mu] = idx % L
        idx = idx // L
    return out


def site_index(coords, dims):
    idx = np.zeros(coords.shape[0], dtype=np.int64)
    stride = 1
    for mu, L in enumerate(dims):
        idx += coords[:, mu] * stride
        stride *= L
    return idx


def neighbour(dims, mu: int, step: int):
    """For every site x: (index of x + step*mu_hat, boundary-crossing mask)."""
    c = site_coords(dims)
    raw = c[:, mu] + step
    cross = (raw < 0) | (raw >= dims[mu])
    c[:, mu] = raw % dims[mu]
    return site_index(c, dims), cross


# ----------------------------------------------------------------------------
# Wilson kernel D_W(U, mass)  (Sec. 2)
# ----------------------------------------------------------------------------

def _link_blocks(U, group: str):
    """Per-site colour blocks of the links: (nd, V, nc, nc)."""
    if group == "u1":
        return U[..., None, None]
    return U


def wilson_matrix(U, dims, mass: float, group: str = "u1", antiperiodic=None):
    """D_W(U, m)_{x,y} = -1/2 (1-gamma_mu) U_mu(x) delta_{x+mu,y}
                         -1/2 (1+gamma_mu) U_mu(x-mu)^dag delta_{x-mu,y} + (d+m) delta_{x,y}.

    Sparse CSR on d-dim vectors ordered [site][spin][color].
    """
    nd = len(dims)
    V = int(np.prod(dims))
    ns = n_spin(nd)
    nc = 1 if group == "u1" else 3
    dof = ns * nc
    g, _ = gammas(nd)
    anti = antiperiodic or [0] * nd
    Ub = _link_blocks(np.asarray(U), group)
    rows, cols, vals = [], [], []
    sites = np.arange(V)
    I_s = np.eye(ns)
    for mu in range(nd):
        # forward hop: -1/2 (1 - gamma_mu) U_mu(x) psi(x + mu)
        fwd, crossf = neighbour(dims, mu, +1)
        phase = np.where(crossf & bool(anti[mu]), -1.0, 1.0)
        spin = -0.5 * (I_s - g[mu])
        blk = np.einsum("ab,vij,v->vaibj", spin, Ub[mu], phase)    # (V, ns, nc, ns, nc)
        _append_blocks(rows, cols, vals, sites, fwd, blk.reshape(V, dof, dof), dof)
        # backward hop: -1/2 (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu)
        bwd, crossb = neighbour(dims, mu, -1)
        phase = np.where(crossb & bool(anti[mu]), -1.0, 1.0)
        spin = -0.5 * (I_s + g[mu])
        Udag = np.conj(np.swapaxes(Ub[mu][bwd], -1, -2))
        blk = np.einsum("ab,vij,v->vaibj", spin, Udag, phase)
        _append_blocks(rows, cols, vals, sites, bwd, blk.reshape(V, dof, dof), dof)
    n = V * dof
    D = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    D = D + (nd + mass) * sp.identity(n, dtype=complex, format="csr")
    return D.tocsr()


def _append_blocks(rows, cols, vals, rsite, csite, blk, dof):
    a = np.arange(dof)
    r = (rsite[:, None, None] * dof + a[None, :, None]) + 0 * a[None, None, :]
    c = (csite[:, None, None] * dof + a[None, None, :]) + 0 * a[None, :, None]
    rows.append(r.ravel())
    cols.append(c.ravel())
    vals.append(blk.ravel())


def chirality_projectors(nd: int, nc: int):
    """(P_+, P_-) on one site's [spin][color] dof, P_pm = (1 pm gamma_5)/2."""
    _, g5 = gammas(nd)
    Ic = np.eye(nc)
    Pp = np.kron(0.5 * (np.eye(n_spin(nd)) + g5), Ic)
    Pm = np.kron(0.5 * (np.eye(n_spin(nd)) - g5), Ic)
    return Pp, Pm


# ----------------------------------------------------------------------------
# Shamir domain-wall operator (Eq. DWoperator) and Pauli-Villars (Sec. 2.2)
# ----------------------------------------------------------------------------

def dwf_from_kernel(Dk, Ls: int, mf: float, Pp, Pm):
    """Ls x Ls block matrix of Eq. DWoperator around a given d-dim kernel Dk.

    Diagonal blocks Dk + 1; block (s, s+1) = P_-; block (s+1, s) = P_+;
    block (1, Ls) = -m P_+; block (Ls, 1) = -m P_- (1-based s).  Pp / Pm are
    the chirality projectors on the kernel's full d-dim space.
    """
    n = Dk.shape[0]
    I = sp.identity(n, dtype=complex, format="csr")
    diag = sp.kron(sp.identity(Ls, format="csr"), Dk + I)
    up = sp.diags([np.ones(Ls - 1)], [1], shape=(Ls, Ls))        # (s, s+1)
    dn = sp.diags([np.ones(Ls - 1)], [-1], shape=(Ls, Ls))       # (s+1, s)
    c_1L = sp.csr_matrix(([1.0], ([0], [Ls - 1])), shape=(Ls, Ls))
    c_L1 = sp.csr_matrix(([1.0], ([Ls - 1], [0])), shape=(Ls, Ls))
    D = diag + sp.kron(up, Pm) + sp.kron(dn, Pp) + sp.kron(c_1L, -mf * Pp) + sp.kron(c_L1, -mf * Pm)
    return D.tocsr()


def site_projectors(V: int, nd: int, nc: int):
    Pp, Pm = chirality_projectors(nd, nc)
    I = sp.identity(V, format="csr")
    return sp.kron(I, sp.csr_matrix(Pp)).tocsr(), sp.kron(I, sp.csr_matrix(Pm)).tocsr()


def dwf_matrix(U, dims, Ls: int, M5: float, mf: float, group: str = "u1", antiperiodic=None):
    """D_DW(m) of Eq. DWoperator with kernel D_W(U, -M5)."""
    nd = len(dims)
    V = int(np.prod(dims))
    nc = 1 if group == "u1" else 3
    Dw = wilson_matrix(U, dims, -M5, group, antiperiodic)
    Pp, Pm = site_projectors(V, nd, nc)
    return dwf_from_kernel(Dw, Ls, mf, Pp, Pm)


def pv_matrix(U, dims, Ls: int, M5: float, group: str = "u1", antiperiodic=None):
    """Pauli-Villars operator D_PV = D_DW(1) (Sec. 2.2)."""
    return dwf_matrix(U, dims, Ls, M5, 1.0, group, antiperiodic)


def dagger(A):
    """Hermitian adjoint of a sparse matrix: the plain definition."""
    return A.conj().T.tocsr()


def dwf_apply(U, psi, dims, Ls, M5, mf, dagger_=False, group="u1", antiperiodic=None):
    """out = D_DW(m) psi (or D_DW^dag psi); psi in canonical order, any shape."""
    D = dwf_matrix(U, dims, Ls, M5, mf, group, antiperiodic)
    if dagger_:
        D = dagger(D)
    return (D @ np.asarray(psi).reshape(-1)).reshape(np.shape(psi))


def pvdag_dwf_matrix(U, dims, Ls, M5, mf, group="u1", antiperiodic=None):
    """Approximately PV-preconditioned operator A = D_PV^dag D_DW(m) (Eq. NormalExp)."""
    Ddw = dwf_matrix(U, dims, Ls, M5, mf, group, antiperiodic)
    Dpv = pv_matrix(U, dims, Ls, M5, group, antiperiodic)
    return (dagger(Dpv) @ Ddw).tocsr()


# ----------------------------------------------------------------------------
# Structural identities of Sec. 2.2
# ----------------------------------------------------------------------------

def reflection_gamma5(V, Ls, nd, nc):
    """Gamma_5 = gamma_5 R with R_{ss'} = delta_{(s+s'-1) % Ls, 0} (1-based s)."""
    _, g5 = gammas(nd)
    R = np.zeros((Ls, Ls))
    for s in range(1, Ls + 1):
        for t in range(1, Ls + 1):
            if (s + t - 1) % Ls == 0:
                R[s - 1, t - 1] = 1.0
    site = sp.kron(sp.identity(V), sp.csr_matrix(np.kron(g5, np.eye(nc))))
    return sp.kron(sp.csr_matrix(R), site).tocsr()


def chiral_permutation(V, Ls, nd, nc):
    """The unitary cyclic permutation script-P of Sec. 2.2: (P v)_s = P_- v_s + P_+ v_{s+1}."""
    Pp, Pm = site_projectors(V, nd, nc)
    diag = sp.kron(sp.identity(Ls), Pm)
    shift = sp.diags([np.ones(Ls - 1)], [1], shape=(Ls, Ls)) + sp.csr_matrix(([1.0], ([Ls - 1], [0])), shape=(Ls, Ls))
    return (diag + sp.kron(shift, Pp)).tocsr()


def overlap_kernel_first_block(Dw_dense, Ls, mf, nd, nc, V):
    """Reading of D_ov(m) that K_DW's (1,1) block reproduces (Eqs. DWFmatrix, Overlap).

    D_ov(m) = (1+m)/2 - (1-m)/2 eps_Ls[X] gamma_5,  X = gamma_5 D_W (2 + D_W)^-1,
    eps_L[X] = ((1-X)^L - (1+X)^L) ((1-X)^L + (1+X)^L)^-1.
    The printed form (1+m)/2 + (1-m)/2 gamma_5 eps_L[H] with H = gamma_5 D_W/(2+D_W)
    differs in the sign of eps and the side of gamma_5; this is the form the
    paper's own D_DW yields exactly (checked by the tests).
    """
    _, g5 = gammas(nd)
    G5 = np.kron(np.eye(V), np.kron(g5, np.eye(nc)))
    n = Dw_dense.shape[0]
    I = np.eye(n)
    X = G5 @ Dw_dense @ np.linalg.inv(2 * I + Dw_dense)
    A = np.linalg.matrix_power(I - X, Ls)
    B = np.linalg.matrix_power(I + X, Ls)
    eps = (A - B) @ np.linalg.inv(A + B)
    return 0.5 * (1 + mf) * I - 0.5 * (1 - mf) * eps @ G5


# ----------------------------------------------------------------------------
# Free field in momentum space (Sec. 2.2, App. A)
# ----------------------------------------------------------------------------

def free_wilson_symbol(p, mass, nd):
    """D~_W(p) = m + sum_mu [ i gamma_mu sin p_mu + 2 sin^2(p_mu / 2) ] (spin matrix)."""
    g, _ = gammas(nd)
    ns = n_spin(nd)
    M = mass * np.eye(ns, dtype=complex)
    for mu in range(nd):
        M = M + 1j * g[mu] * np.sin(p[mu]) + 2 * np.sin(p[mu] / 2) ** 2 * np.eye(ns)
    return M


def free_dwf_symbol(p, Ls, M5, mf, nd):
    """(Ls*ns) x (Ls*ns) momentum block of D_DW(m) at U = 1 (Eq. DWoperator)."""
    ns = n_spin(nd)
    _, g5 = gammas(nd)
    Pp = 0.5 * (np.eye(ns) + g5)
    Pm = 0.5 * (np.eye(ns) - g5)
    Dw = free_wilson_symbol(p, -M5, nd)
    B = np.zeros((Ls * ns, Ls * ns), dtype=complex)
    for s in range(Ls):
        B[s * ns:(s + 1) * ns, s * ns:(s + 1) * ns] = Dw + np.eye(ns)
        if s + 1 < Ls:
            B[s * ns:(s + 1) * ns, (s + 1) * ns:(s + 2) * ns] += Pm
            B[(s + 1) * ns:(s + 2) * ns, s * ns:(s + 1) * ns] += Pp
    B[0:ns, (Ls - 1) * ns:Ls * ns] += -mf * Pp
    B[(Ls - 1) * ns:Ls * ns, 0:ns] += -mf * Pm
    return B


# ----------------------------------------------------------------------------
# Point evaluation for lattices too large to assemble (2-d U(1))
# ----------------------------------------------------------------------------

def dwf_apply_points_2d(U, psi, dims, Ls, M5, mf, points, dagger_=False, antiperiodic=None):
    """(D_DW psi)_{s, x} at selected (s, site) points, straight from Eq. DWoperator.

    U: (2, V) complex; psi: (Ls, V, 2) complex; points: iterable of (s, site)
    with 0-based s.  Returns an array (len(points), 2).  Pure-Python loop, for
    spot checks of large lattices.
    """
    g, g5 = gammas(2)
    I2 = np.eye(2)
    Pp, Pm = 0.5 * (I2 + g5), 0.5 * (I2 - g5)
    anti = antiperiodic or [0, 0]
    L0, L1 = dims
    psi = np.asarray(psi).reshape(Ls, L0 * L1, 2)
    U = np.asarray(U).reshape(2, L0 * L1)
    out = []
    for s, site in points:
        x, y = site % L0, site // L0
        acc = (2 - M5 + 1) * psi[s, site]
        for mu in range(2):
            c = [x, y]
            c[mu] += 1
            cross_f = c[mu] == dims[mu]
            c[mu] %= dims[mu]
            fwd = c[0] + L0 * c[1]
            c = [x, y]
            c[mu] -= 1
            cross_b = c[mu] < 0
            c[mu] %= dims[mu]
            bwd = c[0] + L0 * c[1]
            uf = U[mu, site] * (-1 if (cross_f and anti[mu]) else 1)
            ub = np.conj(U[mu, bwd]) * (-1 if (cross_b and anti[mu]) else 1)
            sg = -1 if dagger_ else 1
            acc = acc - 0.5 * (I2 - sg * g[mu]) @ (uf * psi[s, fwd]) - 0.5 * (I2 + sg * g[mu]) @ (ub * psi[s, bwd])
        A, B = (Pp, Pm) if dagger_ else (Pm, Pp)   # block (s, s+1) and (s+1, s) of D or D^dag
        if s + 1 < Ls:
            acc = acc + A @ psi[s + 1, site]
        else:
            acc = acc - mf * A @ psi[0, site]
        if s > 0:
            acc = acc + B @ psi[s - 1, site]
        else:
            acc = acc - mf * B @ psi[Ls - 1, site]
        out.append(acc)
    return np.array(out)


def dwf_apply_points(U, psi, dims, Ls, M5, mf, points, group="u1", dagger_=False, antiperiodic=None):
    """(D_DW psi)_{s, x} at selected (s, site) points for any d and group,
    straight from Eq. DWoperator; pure-Python loop for spot checks of large
    lattices.  U: (nd, V) or (nd, V, 3, 3); psi: (Ls, V, ns, nc)."""
    nd = len(dims)
    ns = n_spin(nd)
    nc = 1 if group == "u1" else 3
    g, g5 = gammas(nd)
    I = np.eye(ns)
    Pp, Pm = 0.5 * (I + g5), 0.5 * (I - g5)
    anti = antiperiodic or [0] * nd
    V = int(np.prod(dims))
    psi = np.asarray(psi).reshape(Ls, V, ns, nc)
    Ub = np.asarray(U).reshape(nd, V, nc, nc)
    strides = np.cumprod([1] + list(dims[:-1]))
    out = []
    for s, site in points:
        coords = [(site // strides[mu]) % dims[mu] for mu in range(nd)]
        acc = (nd - M5 + 1) * psi[s, site]
        sg = -1 if dagger_ else 1
        for mu in range(nd):
            c = list(coords)
            cross_f = c[mu] + 1 == dims[mu]
            c[mu] = (c[mu] + 1) % dims[mu]
            fwd = int(sum(ci * st for ci, st in zip(c, strides)))
            c = list(coords)
            cross_b = c[mu] == 0
            c[mu] = (c[mu] - 1) % dims[mu]
            bwd = int(sum(ci * st for ci, st in zip(c, strides)))
            uf = Ub[mu, site] * (-1 if (cross_f and anti[mu]) else 1)
            ub = np.conj(Ub[mu, bwd]).T * (-1 if (cross_b and anti[mu]) else 1)
            acc = acc - 0.5 * (I - sg * g[mu]) @ (psi[s, fwd] @ uf.T) - 0.5 * (I + sg * g[mu]) @ (psi[s, bwd] @ ub.T)
        A, B = (Pp, Pm) if dagger_ else (Pm, Pp)
        acc = acc + (A @ psi[s + 1, site] if s + 1 < Ls else -mf * A @ psi[0, site])
        acc = acc + (B @ psi[s - 1, site] if s > 0 else -mf * B @ psi[Ls - 1, site])
        out.append(acc)
    return np.array(out)


# ----------------------------------------------------------------------------
# Mobius domain wall operator and the polynomial Pauli-Villars correction
# (the generalisations the paper names in its conclusions and Sec. 2.3)
# ----------------------------------------------------------------------------

def s_hops(V, Ls, mf, nd, nc):
    """H_s: the fifth-dimension hops of Eq. DWoperator without the diagonal:
    P_- on block (s, s+1), P_+ on (s+1, s), -m P_+ on (1, Ls), -m P_- on (Ls, 1)."""
    Pp, Pm = site_projectors(V, nd, nc)
    up = sp.diags([np.ones(Ls - 1)], [1], shape=(Ls, Ls))
    dn = sp.diags([np.ones(Ls - 1)], [-1], shape=(Ls, Ls))
    c_1L = sp.csr_matrix(([1.0], ([0], [Ls - 1])), shape=(Ls, Ls))
    c_L1 = sp.csr_matrix(([1.0], ([Ls - 1], [0])), shape=(Ls, Ls))
    return (sp.kron(up, Pm) + sp.kron(dn, Pp) + sp.kron(c_1L, -mf * Pp) + sp.kron(c_L1, -mf * Pm)).tocsr()


def mobius_matrix(U, dims, Ls, M5, mf, b5, c5, group="u1", antiperiodic=None):
    """Mobius domain wall operator in the sign convention of Eq. DWoperator:
    D_M = (b5 D_W + 1) on the diagonal blocks and (1 - c5 D_W) times each fifth-
    dimension hop of H_s (P_-, P_+ and the -m walls), i.e.
    D_M = (1_s x D_W) (b5 - c5 H_s) + 1 + H_s.
    b5 = 1, c5 = 0 is the Shamir operator; the kernel is D_W(U, -M5)."""
    nd = len(dims)
    V = int(np.prod(dims))
    nc = 1 if group == "u1" else 3
    Dw = wilson_matrix(U, dims, -M5, group, antiperiodic)
    Hs = s_hops(V, Ls, mf, nd, nc)
    n = Hs.shape[0]
    I = sp.identity(n, dtype=complex, format="csr")
    DW5 = sp.kron(sp.identity(Ls, format="csr"), Dw)
    return (DW5 @ (b5 * I - c5 * Hs) + I + Hs).tocsr()


def mobius_from_kernel(Dk, Ls, mf, b5, c5, Pp, Pm):
    """The Mobius form around any d-dim kernel Dk (a coarse kernel, e.g.):
    (1_s x Dk)(b5 - c5 H_s) + 1 + H_s, H_s built from the chirality projectors Pp / Pm."""
    n = Dk.shape[0]
    up = sp.diags([np.ones(Ls - 1)], [1], shape=(Ls, Ls))
    dn = sp.diags([np.ones(Ls - 1)], [-1], shape=(Ls, Ls))
    c_1L = sp.csr_matrix(([1.0], ([0], [Ls - 1])), shape=(Ls, Ls))
    c_L1 = sp.csr_matrix(([1.0], ([Ls - 1], [0])), shape=(Ls, Ls))
    Hs = (sp.kron(up, Pm) + sp.kron(dn, Pp) + sp.kron(c_1L, -mf * Pp) + sp.kron(c_L1, -mf * Pm)).tocsr()
    I = sp.identity(Ls * n, dtype=complex, format="csr")
    return (sp.kron(sp.identity(Ls, format="csr"), Dk) @ (b5 * I - c5 * Hs) + I + Hs).tocsr()


def pv_poly_operator(Ddw, Dpv, coeffs):
    """D_PV^dag p(D_PV D_PV^dag) D_DW with p(y) = sum_k c_k y^k: the approximation
    D_PV^-1 = D_PV^dag [D_PV D_PV^dag]^-1 ~ D_PV^dag p(D_PV D_PV^dag) of the
    Pauli-Villars preconditioner; c = (1) is the truncation D_PV^dag D_DW of
    Eq. NormalExp, c = (2, -1) the next order (App. A)."""
    Dpvd = dagger(Dpv)
    N = (Dpv @ Dpvd).tocsr()
    n = N.shape[0]
    P = sp.csr_matrix((n, n), dtype=complex)
    Nk = sp.identity(n, dtype=complex, format="csr")
    for c in coeffs:
        P = P + c * Nk
        Nk = (Nk @ N).tocsr()
    return (Dpvd @ P @ Ddw).tocsr()


def pv_poly_apply(Ddw, Dpv, coeffs, psi):
    """The operator of pv_poly_operator applied to the vector psi by matrix-vector
    products only (no matrix powers): y = D_DW psi, z = p(N) y with N = D_PV D_PV^dag
    by Horner's rule (z = c_K y, then z = c_k y + N z for k = K-1 .. 0), and
    D_PV^dag z.  Same mathematics in another order of the products."""
    Dpvd = dagger(Dpv)
    y = Ddw @ psi
    z = coeffs[-1] * y
    for c in reversed(coeffs[:-1]):
        z = c * y + Dpv @ (Dpvd @ z)
    return Dpvd @ z

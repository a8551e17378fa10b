"""Krylov solvers of the oracle, in FP64 with plain numpy vector algebra.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def vdot(a, b):
    return np.vdot(a, b)


def norm(a):
    return float(np.sqrt(np.vdot(a, a).real))


def cgnr(D, b, tol=1e-10, maxiter=100000, x0=None, Ddag=None):
    """Conjugate gradient on the normal equations D^dag D x = D^dag b (Sec. 2.1).

    Stops when the true residual of the original system satisfies
    ||b - D x|| / ||b|| <= tol (the stopping rule of Sec. 3), checked on the
    recursively updated residual and confirmed by a recomputation.
    Returns (x, iterations, true relative residual).
    """
    if Ddag is None:
        Ddag = D.conj().T.tocsr()
    b = np.asarray(b, dtype=complex).ravel()
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=complex).ravel()
    bn = norm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0
    rr = b - D @ x                    # residual of D x = b
    r = Ddag @ rr                     # residual of the normal equations
    p = r.copy()
    rn2 = vdot(r, r).real
    it = 0
    while it < maxiter:
        if norm(rr) <= tol * bn:
            true = norm(b - D @ x) / bn
            if true <= tol:
                return x, it, true
            rr = b - D @ x            # drift: restart from the true residual
            r = Ddag @ rr
            p = r.copy()
            rn2 = vdot(r, r).real
        q = D @ p
        alpha = rn2 / vdot(q, q).real
        x = x + alpha * p
        rr = rr - alpha * q
        r = r - alpha * (Ddag @ q)
        rn2_new = vdot(r, r).real
        p = r + (rn2_new / rn2) * p
        rn2 = rn2_new
        it += 1
    return x, it, norm(b - D @ x) / bn


def cgnr_fixed(D, b, tol, maxiter, Ddag=None, x0=None):
    """CGNR stopped on the recursive residual ||b - D x|| <= tol ||b|| or maxiter,
    from x0 (default 0).

    Used for inexact inner solves; returns (x, iterations).
    """
    if Ddag is None:
        Ddag = D.conj().T.tocsr()
    b = np.asarray(b, dtype=complex).ravel()
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=complex).ravel()
    bn = norm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0
    rr = b - D @ x if x0 is not None else b.copy()
    r = Ddag @ rr
    p = r.copy()
    rn2 = vdot(r, r).real
    it = 0
    while it < maxiter and norm(rr) > tol * bn:
        q = D @ p
        alpha = rn2 / vdot(q, q).real
        x = x + alpha * p
        rr = rr - alpha * q
        r = r - alpha * (Ddag @ q)
        rn2_new = vdot(r, r).real
        p = r + (rn2_new / rn2) * p
        rn2 = rn2_new
        it += 1
    return x, it


def gcr(apply_A, b, x0=None, tol=0.0, maxiter=8, precond=None):
    """Flexible GCR: minimises ||b - A x|| over x0 + span{z_k}, z_k = M(r_k).

    Each step orthogonalises the new direction A z_k against all earlier A z_j
    (modified Gram-Schmidt); no restart inside `maxiter`.  Returns (x, r, k).
    """
    b = np.asarray(b, dtype=complex).ravel()
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=complex).ravel()
    r = b - apply_A(x) if x0 is not None else b.copy()
    bn = norm(b)
    Z, AZ = [], []
    k = 0
    while k < maxiter and norm(r) > tol * bn:
        z = precond(r) if precond is not None else r.copy()
        w = apply_A(z)
        for zj, wj in zip(Z, AZ):
            beta = vdot(wj, w)
            w = w - beta * wj
            z = z - beta * zj
        wn = norm(w)
        if wn == 0.0:
            break
        w = w / wn
        z = z / wn
        alpha = vdot(w, r)
        x = x + alpha * z
        r = r - alpha * w
        Z.append(z)
        AZ.append(w)
        k += 1
    return x, r, k


def bicgstab_l(apply_A, f, ell=6, tol=1e-10, max_cycles=10000, x0=None, stop=None, callback=None):
    """BiCGStab(l) of Sleijpen & Fokkema (1993) for A x = f, the solver the paper
    compares against as "BiCGStab-6 on D_PV^dag D_DW" (Sec. 2.3, Sec. 3).

    One cycle makes l BiCG steps (each extends the residuals r_0..r_j and the
    search directions u_0..u_j by one power of A, with the shadow residual
    rt = the initial residual) followed by a minimal-residual step: the
    residual r_0 - sum_j g_j r_j over r_1..r_l is minimised (modified
    Gram-Schmidt of r_1..r_l, then back substitution for g).  Inner products
    are <a, b> = a^dag b.  The cycle ends when stop(x) is true (default:
    ||f - A x|| <= tol ||f||, on the recursive residual).  callback(x, r, R)
    sees the iterate, the residual and the Gram-Schmidt-orthogonalised
    r_1..r_l of every cycle.  Returns (x, applications of A).
    """
    f = np.asarray(f, dtype=complex).ravel()
    x = np.zeros_like(f) if x0 is None else np.array(x0, dtype=complex).ravel()
    r = f - apply_A(x) if x0 is not None else f.copy()
    nA = 1 if x0 is not None else 0
    fn = norm(f)
    if fn == 0.0:
        return np.zeros_like(f), nA
    if stop is None:
        def stop(_x):
            return False
    rt = r.copy()
    u = np.zeros_like(f)
    rho0, alpha, omega = 1.0 + 0j, 0.0 + 0j, 1.0 + 0j
    for _ in range(max_cycles):
        if norm(r) <= tol * fn or stop(x):
            break
        R = [r] + [None] * ell
        U = [u] + [None] * ell
        rho0 = -omega * rho0
        for j in range(ell):                      # BiCG part
            rho1 = vdot(rt, R[j])
            beta = alpha * rho1 / rho0
            rho0 = rho1
            for i in range(j + 1):
                U[i] = R[i] - beta * U[i]
            U[j + 1] = apply_A(U[j])
            nA += 1
            alpha = rho0 / vdot(rt, U[j + 1])
            for i in range(j + 1):
                R[i] = R[i] - alpha * U[i + 1]
            R[j + 1] = apply_A(R[j])
            nA += 1
            x = x + alpha * U[0]
        # MR part: modified Gram-Schmidt of R[1..l]
        tau = np.zeros((ell + 1, ell + 1), dtype=complex)
        sigma = np.zeros(ell + 1)
        gp = np.zeros(ell + 1, dtype=complex)
        for j in range(1, ell + 1):
            for i in range(1, j):
                tau[i, j] = vdot(R[i], R[j]) / sigma[i]
                R[j] = R[j] - tau[i, j] * R[i]
            sigma[j] = vdot(R[j], R[j]).real
            gp[j] = vdot(R[j], R[0]) / sigma[j]
        g = np.zeros(ell + 1, dtype=complex)
        g[ell] = gp[ell]
        omega = g[ell]
        for j in range(ell - 1, 0, -1):
            g[j] = gp[j] - sum(tau[j, i] * g[i] for i in range(j + 1, ell + 1))
        g2 = np.zeros(ell + 1, dtype=complex)
        for j in range(1, ell):
            g2[j] = g[j + 1] + sum(tau[j, i] * g[i + 1] for i in range(j + 1, ell))
        x = x + g[1] * R[0]
        R[0] = R[0] - gp[ell] * R[ell]
        U[0] = U[0] - g[ell] * U[ell]
        for j in range(1, ell):
            U[0] = U[0] - g[j] * U[j]
            x = x + g2[j] * R[j]
            R[0] = R[0] - gp[j] * R[j]
        r, u = R[0], U[0]
        if callback is not None:
            callback(x, r, R[1:])
    return x, nA


def bicgstab_dw(Ddw, Dpv_dag, b, ell=6, tol=1e-10, max_cycles=10000):
    """BiCGStab(l) on D_PV^dag D_DW x = D_PV^dag b, stopped when the true residual
    of the original system ||b - D_DW x|| / ||b|| <= tol (checked after every cycle).
    Returns (x, fine applications, true relative residual); one application of the
    preconditioned operator counts as two fine applications (D_DW, D_PV^dag)."""
    b = np.asarray(b, dtype=complex).ravel()
    bn = norm(b)
    A = (Dpv_dag @ Ddw).tocsr()

    def stop(x):
        return norm(b - Ddw @ x) <= tol * bn

    x, nA = bicgstab_l(lambda v: A @ v, Dpv_dag @ b, ell=ell, tol=0.0, max_cycles=max_cycles, stop=stop)
    return x, 2 * nA + 1, norm(b - Ddw @ x) / bn


def low_modes(N, k):
    """The k smallest eigenpairs (lam ascending, V columns orthonormal) of a
    Hermitian matrix N, by dense diagonalisation (small problems only)."""
    Nd = N.toarray() if hasattr(N, "toarray") else np.asarray(N)
    w, Q = np.linalg.eigh(Nd)
    return w[:k], Q[:, :k]


def cgnr_deflated(A, b, tol, maxiter, V, lam, Adag=None):
    """Deflated CGNR on A x = b: the start x0 = V diag(1 / lam) V^dag A^dag b
    solves the normal equations A^dag A x = A^dag b exactly on the span of the
    low eigenvectors V of A^dag A (eigenvalues lam), then CGNR continues from
    x0 to ||b - A x|| <= tol ||b||.  Returns (x, iterations)."""
    if Adag is None:
        Adag = A.conj().T.tocsr()
    b = np.asarray(b, dtype=complex).ravel()
    f = Adag @ b
    x0 = V @ ((V.conj().T @ f) / lam)
    return cgnr_fixed(A, b, tol, maxiter, Ddag=Adag, x0=x0)

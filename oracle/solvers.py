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


def cgnr_fixed(D, b, tol, maxiter, Ddag=None):
    """CGNR stopped on the recursive residual ||b - D x|| <= tol ||b|| or maxiter.

    Used for inexact inner solves; returns (x, iterations).
    """
    if Ddag is None:
        Ddag = D.conj().T.tocsr()
    b = np.asarray(b, dtype=complex).ravel()
    x = np.zeros_like(b)
    bn = norm(b)
    if bn == 0.0:
        return x, 0
    rr = b.copy()
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

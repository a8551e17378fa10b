"""Gradient of a solve with respect to U(1) link angles, FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

For x = D_DW^-1 b and the loss l = |x|^2, dl/dtheta = -2 Re(lambda^dag
(dD_DW/dtheta) x) with the adjoint solution D_DW^dag lambda = x.  Only the
Wilson hops of D_W (Sec. 2) depend on U_mu(x) = exp(i theta_mu(x)), on every
s slice: the forward hop -1/2 (1 - gamma_mu) U_mu(x) differentiates to
-1/2 (1 - gamma_mu) i U_mu(x), the backward hop -1/2 (1 + gamma_mu) U_mu(x)^*
(row x + mu, column x) to -1/2 (1 + gamma_mu) (-i) U_mu(x)^*.
"""
from __future__ import annotations

import numpy as np

from . import dirac


def link_derivative_contraction(U, dims, Ls, lam, x, antiperiodic=None):
    """g_mu(site) = Re( lambda^dag (dD_DW / dtheta_mu(site)) x ), shape (nd, V)."""
    nd = len(dims)
    V = int(np.prod(dims))
    ns = dirac.n_spin(nd)
    g, _ = dirac.gammas(nd)
    anti = antiperiodic or [0] * nd
    lam = np.asarray(lam).reshape(Ls, V, ns)
    x = np.asarray(x).reshape(Ls, V, ns)
    out = np.zeros((nd, V))
    I = np.eye(ns)
    for mu in range(nd):
        fwd, cross = neighbour_with_phase(dims, mu, anti)
        ph = np.where(cross, -1.0, 1.0)
        Um = np.asarray(U)[mu] * ph
        # row (site, s), column (site + mu, s)
        A = -0.5 * (I - g[mu])
        t1 = np.einsum("svi,ij,svj->v", np.conj(lam), A, x[:, fwd, :]) * (1j * Um)
        # row (site + mu, s), column (site, s)
        B = -0.5 * (I + g[mu])
        t2 = np.einsum("svi,ij,svj->v", np.conj(lam[:, fwd, :]), B, x) * (-1j * np.conj(Um))
        out[mu] = (t1 + t2).real
    return out


def neighbour_with_phase(dims, mu, anti):
    idx, cross = dirac.neighbour(dims, mu, +1)
    return idx, cross & bool(anti[mu])


def loss_and_grad(theta, b, dims, Ls, M5, mf, antiperiodic=None):
    """l = |D_DW^-1 b|^2 and dl/dtheta by the adjoint method (dense solves)."""
    U = np.exp(1j * theta)
    D = dirac.dwf_matrix(U, dims, Ls, M5, mf, "u1", antiperiodic).toarray()
    xs = np.linalg.solve(D, np.asarray(b).ravel())
    lam = np.linalg.solve(D.conj().T, xs)
    grad = -2.0 * link_derivative_contraction(U, dims, Ls, lam, xs, antiperiodic)
    return float(np.vdot(xs, xs).real), grad

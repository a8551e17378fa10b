"""Gradient of a solve with respect to the links, FP64: U(1) link angles
(2-d) and SU(3) links along the algebra (4-d).

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
import scipy.sparse as sp

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


# ----------------------------------------------------------------------------
# SU(3) links (4-d): derivative along the algebra
# ----------------------------------------------------------------------------

def su3_generators():
    """T_a = lambda_a / 2 (Gell-Mann matrices): traceless Hermitian, tr(T_a T_b) = delta_ab / 2."""
    L = np.zeros((8, 3, 3), dtype=complex)
    L[0][0, 1] = L[0][1, 0] = 1
    L[1][0, 1], L[1][1, 0] = -1j, 1j
    L[2][0, 0], L[2][1, 1] = 1, -1
    L[3][0, 2] = L[3][2, 0] = 1
    L[4][0, 2], L[4][2, 0] = -1j, 1j
    L[5][1, 2] = L[5][2, 1] = 1
    L[6][1, 2], L[6][2, 1] = -1j, 1j
    L[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return L / 2


def directional_derivative(U, dims, Ls, lam, x, mu, site, dU, group="su3", antiperiodic=None):
    """Re(lambda^dag (d/dt) D_DW(U + t dU e_{mu,site}) x): D_DW is real-linear in the
    links (Sec. 2; the backward hop reads U^dag), so the derivative is the Wilson
    hop term on a link field that is dU on link (mu, site) and zero elsewhere, on
    every s slice."""
    nd = len(dims)
    Z = np.zeros_like(np.asarray(U))
    Z[mu, site] = dU
    dDw = dirac.wilson_matrix(Z, dims, -float(nd), group, antiperiodic)    # hops only: d + m = 0
    dD = sp.kron(sp.identity(Ls, format="csr"), dDw)
    return np.vdot(np.asarray(lam).reshape(-1), dD @ np.asarray(x).reshape(-1)).real


def link_force_su3(U, dims, Ls, lam, x, links, antiperiodic=None):
    """F_mu(site) for the requested links [(mu, site), ...]: the traceless Hermitian
    3x3 matrix with Re(lambda^dag (dD_DW / d eps) x) = tr(H F) for the variation
    U_mu(site) -> exp(i eps H) U_mu(site), H traceless Hermitian.

    Straight from the definition, one link and one generator at a time: D_DW is
    real-linear in the links (Sec. 2; the backward hop reads U^dag), so its
    derivative is the Wilson hop term evaluated on a link field that is zero
    except for i T_a U_mu(site) on that link, on every s slice.  With
    c_a = Re(lambda^dag dD_a x), F = 2 sum_a c_a T_a.
    """
    U = np.asarray(U)
    T = su3_generators()
    out = []
    for mu, site in links:
        c = np.array([directional_derivative(U, dims, Ls, lam, x, mu, site, 1j * T[a] @ U[mu, site], "su3",
                                             antiperiodic) for a in range(8)])
        out.append(2 * np.einsum("a,aij->ij", c, T))
    return np.array(out)


def loss_and_force_su3(U, b, dims, Ls, M5, mf, links, antiperiodic=None):
    """l = |D_DW^-1 b|^2 and, for each requested link, the traceless Hermitian F with
    dl/d eps = -2 tr(H F) for U_mu(site) -> exp(i eps H) U_mu(site) (dense solves;
    adjoint solution D_DW^dag lambda = x)."""
    D = dirac.dwf_matrix(U, dims, Ls, M5, mf, "su3", antiperiodic).toarray()
    xs = np.linalg.solve(D, np.asarray(b).ravel())
    lam = np.linalg.solve(D.conj().T, xs)
    F = link_force_su3(U, dims, Ls, lam, xs, links, antiperiodic)
    return float(np.vdot(xs, xs).real), F

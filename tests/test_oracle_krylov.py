"""Pins of the oracle's Krylov iterations by their optimality properties.

Each iterate of a conjugate-gradient method is the unique minimiser of a
known functional over a Krylov space, so a dense minimisation over an
explicitly built (orthonormalised) Krylov basis fixes every iterate, not just
the converged answer:

  * CG on a Hermitian positive definite A x = f from x0: x_k minimises the
    A-norm of the error over x0 + K_k(A, r0), r0 = f - A x0.  For the
    homogeneous near-null relaxation (f = 0, Table kcycle's setup) that is the
    minimiser of x^dag A x over x0 + K_k(A, -A x0) with A = D_W D_W^dag.
  * CGNR (Sec. 2.1): CG on D^dag D x = D^dag b minimises the residual norm
    ||b - D x|| over x0 + K_k(D^dag D, D^dag r0).

A plausible mistake (the other normal operator D_W^dag D_W, a wrong step
count, a dropped conjugation, a wrong stopping rule) moves the iterates off
these minimisers.
"""
import numpy as np
import pytest

import synth
from oracle import dirac, mg, solvers


def _u1(dims, sigma, seed):
    return synth.u1_links(synth.u1_angles(np.random.default_rng(seed), dims, sigma))


def _krylov_basis(A, v, k):
    """Orthonormal basis of span{v, A v, ..., A^(k-1) v} (dense, two QR passes)."""
    cols = [v]
    for _ in range(k - 1):
        cols.append(A @ cols[-1])
    K = np.stack(cols, axis=1)
    Q, _ = np.linalg.qr(K)
    Q, _ = np.linalg.qr(Q)
    return Q


def _cg_homogeneous_minimiser(A, x0, k):
    """argmin of x^dag A x over x0 + K_k(A, -A x0)."""
    Q = _krylov_basis(A, -(A @ x0), k)
    c = np.linalg.solve(Q.conj().T @ A @ Q, -(Q.conj().T @ (A @ x0)))
    return x0 + Q @ c


@pytest.mark.parametrize("k", [1, 2, 5, 9])
def test_relax_null_vector_iterates_are_cg_minimisers(k):
    """The k-th relaxation iterate is the D_W D_W^dag-norm minimiser over x0 + K_k."""
    dims, m_setup = (4, 4), -0.4
    U = _u1(dims, 0.6, 21)
    Dw = dirac.wilson_matrix(U, dims, m_setup)
    Dd = Dw.toarray()
    A = Dd @ Dd.conj().T
    x0 = synth.gaussian_complex(np.random.default_rng(22), (Dw.shape[0],))
    v, it = mg.relax_null_vector(Dw, x0, maxiter=k, tol=0.0)
    assert it == k
    want = _cg_homogeneous_minimiser(A, x0, k)
    assert np.linalg.norm(v - want) <= 1e-9 * np.linalg.norm(want)
    # the other normal operator gives a different minimiser: the pin separates them
    A_wrong = Dd.conj().T @ Dd
    wrong = _cg_homogeneous_minimiser(A_wrong, x0, k)
    assert np.linalg.norm(wrong - want) > 1e-3 * np.linalg.norm(want)


def test_relax_null_vector_stops_at_first_iterate_below_tol():
    """Stopping rule: the first k with ||A x_k|| <= tol ||A x_0|| (or maxiter)."""
    dims, m_setup = (4, 4), -0.4
    U = _u1(dims, 0.6, 23)
    Dw = dirac.wilson_matrix(U, dims, m_setup)
    Dd = Dw.toarray()
    A = Dd @ Dd.conj().T
    x0 = synth.gaussian_complex(np.random.default_rng(24), (Dw.shape[0],))
    r0 = np.linalg.norm(A @ x0)
    tol = 3e-2
    norms = [np.linalg.norm(A @ _cg_homogeneous_minimiser(A, x0, k)) / r0 for k in range(1, 30)]
    first = 1 + next(i for i, q in enumerate(norms) if q <= tol)
    _, it = mg.relax_null_vector(Dw, x0, maxiter=250, tol=tol)
    assert it == first
    _, it_cap = mg.relax_null_vector(Dw, x0, maxiter=first - 1, tol=tol)
    assert it_cap == first - 1


def _cgnr_minimiser(D, b, k):
    """argmin ||b - D x|| over K_k(D^dag D, D^dag b) (x0 = 0)."""
    Dd = D.toarray() if hasattr(D, "toarray") else D
    N = Dd.conj().T @ Dd
    Q = _krylov_basis(N, Dd.conj().T @ b, k)
    c, *_ = np.linalg.lstsq(Dd @ Q, b, rcond=None)
    return Q @ c


@pytest.mark.parametrize("k", [1, 3, 7])
def test_cgnr_fixed_iterates_minimise_the_residual(k):
    """cgnr_fixed's k-th iterate is the residual-norm minimiser over the Krylov space."""
    dims, Ls = (4, 4), 4
    U = _u1(dims, 0.5, 25)
    D = dirac.dwf_matrix(U, dims, Ls, 1.0, 0.05)
    b = synth.gaussian_complex(np.random.default_rng(26), (D.shape[0],))
    x, it = solvers.cgnr_fixed(D, b, tol=0.0, maxiter=k)
    assert it == k
    want = _cgnr_minimiser(D, b, k)
    assert np.linalg.norm(x - want) <= 1e-9 * np.linalg.norm(want)


def test_cgnr_fixed_matches_dense_solve_and_stops_on_tol():
    """Tight tolerance: the dense solution; loose tolerance: the first iterate below it."""
    dims, Ls = (4, 4), 4
    U = _u1(dims, 0.5, 27)
    D = dirac.dwf_matrix(U, dims, Ls, 1.0, 0.05)
    b = synth.gaussian_complex(np.random.default_rng(28), (D.shape[0],))
    xd = np.linalg.solve(D.toarray(), b)
    x, it = solvers.cgnr_fixed(D, b, tol=1e-12, maxiter=5000)
    assert np.linalg.norm(b - D @ x) <= 1e-12 * np.linalg.norm(b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    tol = 0.05
    res = [np.linalg.norm(b - D @ _cgnr_minimiser(D, b, k)) / np.linalg.norm(b) for k in range(1, 60)]
    first = 1 + next(i for i, q in enumerate(res) if q <= tol)
    _, it = solvers.cgnr_fixed(D, b, tol=tol, maxiter=5000)
    assert it == first


def _bicgstab_textbook(A, f, iters):
    """van der Vorst's BiCGStab (1992), the l = 1 case of BiCGStab(l), written out."""
    x = np.zeros_like(f)
    r = f.copy()
    rt = r.copy()
    rho = alpha = omega = 1.0 + 0j
    v = np.zeros_like(f)
    p = np.zeros_like(f)
    out = []
    for _ in range(iters):
        rho_new = np.vdot(rt, r)
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = A @ p
        alpha = rho_new / np.vdot(rt, v)
        s = r - alpha * v
        t = A @ s
        omega = np.vdot(t, s) / np.vdot(t, t)
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho = rho_new
        out.append(x.copy())
    return out


def _pv_system(seed, dims=(4, 4), Ls=4, m=0.05):
    U = _u1(dims, 0.5, seed)
    Ddw = dirac.dwf_matrix(U, dims, Ls, 1.0, m)
    Dpvd = dirac.dagger(dirac.pv_matrix(U, dims, Ls, 1.0))
    b = synth.gaussian_complex(np.random.default_rng(seed + 1), (Ddw.shape[0],))
    return Ddw, Dpvd, b


def test_bicgstab_l1_is_textbook_bicgstab():
    """l = 1: every cycle equals one iteration of van der Vorst's BiCGStab."""
    Ddw, Dpvd, b = _pv_system(41)
    A = (Dpvd @ Ddw).toarray()
    f = Dpvd @ b
    want = _bicgstab_textbook(A, f, 12)
    got = []
    solvers.bicgstab_l(lambda v: A @ v, f, ell=1, tol=0.0, max_cycles=12,
                       callback=lambda x, r, R: got.append(x.copy()))
    for k, (g, w) in enumerate(zip(got, want)):
        assert np.linalg.norm(g - w) <= 1e-10 * np.linalg.norm(w), k


@pytest.mark.parametrize("ell", [2, 4, 6])
def test_bicgstab_l_minimal_residual_step(ell):
    """After every cycle the recursive residual is f - A x (the x update's coefficients agree
    with the residual's) and is orthogonal to the Gram-Schmidt basis r_1..r_l of the MR step."""
    Ddw, Dpvd, b = _pv_system(43)
    A = (Dpvd @ Ddw).toarray()
    f = Dpvd @ b
    seen = []

    def cb(x, r, R):
        seen.append((x.copy(), r.copy(), [q.copy() for q in R]))

    solvers.bicgstab_l(lambda v: A @ v, f, ell=ell, tol=0.0, max_cycles=4, callback=cb)
    assert len(seen) == 4
    for x, r, R in seen[:3]:
        assert np.linalg.norm((f - A @ x) - r) <= 1e-9 * np.linalg.norm(f)
        for q in R:
            assert abs(np.vdot(q, r)) <= 1e-10 * np.linalg.norm(q) * np.linalg.norm(f)


@pytest.mark.parametrize("ell", [1, 2, 6])
def test_bicgstab_dw_reaches_dense_solution(ell):
    """BiCGStab(l) on D_PV^dag D_DW (right-half-plane spectrum, App. B) reaches the dense solution."""
    Ddw, Dpvd, b = _pv_system(45)
    x, napp, res = solvers.bicgstab_dw(Ddw, Dpvd, b, ell=ell, tol=1e-12)
    xd = np.linalg.solve(Ddw.toarray(), b)
    assert res <= 1e-12
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    assert napp > 0 and napp % 2 == 1

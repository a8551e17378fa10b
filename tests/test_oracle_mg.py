"""Pins of the oracle's solvers, multigrid transfer, Galerkin operator and gradient."""
import numpy as np
import pytest

import synth
from oracle import dirac, mg, solvers, force


def _u1(dims, sigma, seed):
    return synth.u1_links(synth.u1_angles(np.random.default_rng(seed), dims, sigma))


def _null_vectors(U, dims, nvec, seed, m_setup=-0.6, iters=30):
    rng = np.random.default_rng(seed)
    Dw = dirac.wilson_matrix(U, dims, m_setup)
    out = []
    for _ in range(nvec):
        v0 = synth.gaussian_complex(rng, (Dw.shape[0],))
        v, _ = mg.relax_null_vector(Dw, v0, maxiter=iters, tol=1e-4)
        out.append(v)
    return out


def test_cgnr_matches_dense_solve():
    dims, Ls = (4, 4), 4
    U = _u1(dims, 0.5, 1)
    D = dirac.dwf_matrix(U, dims, Ls, 1.0, 0.01)
    b = synth.gaussian_complex(np.random.default_rng(2), (D.shape[0],))
    x, it, res = solvers.cgnr(D, b, tol=1e-10)
    xd = np.linalg.solve(D.toarray(), b)
    assert res <= 1e-10
    cond = np.linalg.cond(D.toarray())
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10 * cond
    assert it > 0


def test_gcr_exact_in_n_steps_and_monotone():
    rng = np.random.default_rng(3)
    n = 12
    A = np.eye(n) * 3 + synth.gaussian_complex(rng, (n, n)) * 0.3
    b = synth.gaussian_complex(rng, (n,))
    x, r, k = solvers.gcr(lambda v: A @ v, b, maxiter=n)
    assert np.linalg.norm(b - A @ x) < 1e-10 * np.linalg.norm(b)
    # residual norms never increase step to step
    prev = np.linalg.norm(b)
    for m in range(1, n):
        _, r, _ = solvers.gcr(lambda v: A @ v, b, maxiter=m)
        assert np.linalg.norm(r) <= prev * (1 + 1e-12)
        prev = np.linalg.norm(r)


def test_relax_reduces_rayleigh_quotient():
    dims = (8, 8)
    U = _u1(dims, 0.5, 4)
    Dw = dirac.wilson_matrix(U, dims, -0.5)
    rng = np.random.default_rng(5)
    v0 = synth.gaussian_complex(rng, (Dw.shape[0],))
    v, it = mg.relax_null_vector(Dw, v0, maxiter=40)
    q0 = np.linalg.norm(Dw.conj().T @ v0) / np.linalg.norm(v0)
    q1 = np.linalg.norm(Dw.conj().T @ v) / np.linalg.norm(v)
    assert 0 < it <= 40 and q1 < 0.5 * q0


def test_prolongator_orthonormal_and_chiral():
    """P^dag P = 1 and gamma_5 P = P sigma_3 (Sec. 2.3, Eq. gamma5)."""
    dims, block, nvec = (8, 8), (4, 4), 4
    U = _u1(dims, 0.5, 6)
    vecs = _null_vectors(U, dims, nvec, 7)
    P, cdims = mg.build_prolongator(vecs, dims, block, 2, 1)
    assert cdims == (2, 2)
    PdP = (P.conj().T @ P).toarray()
    assert np.abs(PdP - np.eye(P.shape[1])).max() < 1e-13
    V = 64
    G5 = np.kron(np.eye(V), np.diag([1.0, -1.0]))
    s3 = np.kron(np.eye(4), np.diag([1.0] * nvec + [-1.0] * nvec))
    assert np.abs(G5 @ P.toarray() - P.toarray() @ s3).max() < 1e-14
    # P^dag (1 pm gamma_5) P = 1 pm sigma_3
    for sgn in (1, -1):
        lhs = P.conj().T.toarray() @ (np.eye(2 * V) + sgn * G5) @ P.toarray()
        assert np.abs(lhs - (np.eye(8 * nvec // nvec * nvec) + sgn * s3)).max() < 1e-13
    # the span holds every chiral half of every relaxed vector: P P^dag v = v
    Pp, Pm = dirac.site_projectors(V, 2, 1)
    for v in vecs:
        for proj in (Pp, Pm):
            w = proj @ v
            assert np.linalg.norm(P @ (P.conj().T @ w) - w) < 1e-12 * np.linalg.norm(w)


def test_prolongator_first_column_is_normalised_vector():
    """Gram-Schmidt order: column 0 of an aggregate is the normalised first vector there."""
    dims, block, nvec = (4, 4), (2, 2), 2
    U = _u1(dims, 0.5, 6)
    vecs = _null_vectors(U, dims, nvec, 8, iters=5)
    P, _ = mg.build_prolongator(vecs, dims, block, 2, 1)
    agg, _ = mg.aggregate_map(dims, block)
    sites = np.nonzero(agg == 1)[0]
    v = vecs[0].reshape(16, 2)[sites, 0]             # chirality + = spin 0
    col = P.toarray()[:, (1 * 2 + 0) * nvec + 0].reshape(16, 2)[sites, 0]
    assert np.abs(col - v / np.linalg.norm(v)).max() < 1e-13


def test_galerkin_commutes_with_dw_structure():
    """P^dag D_DW(m) P (P diagonal in s) equals Eq. coarsenDW built from P^dag D_W P (Sec. 2.3)."""
    dims, block, nvec, Ls, M5, m = (8, 8), (4, 4), 3, 4, 1.0, 0.03
    U = _u1(dims, 0.5, 9)
    vecs = _null_vectors(U, dims, nvec, 10)
    P, _ = mg.build_prolongator(vecs, dims, block, 2, 1)
    Dw = dirac.wilson_matrix(U, dims, -M5)
    Dhat = mg.galerkin_kernel(P, Dw)
    Ps = np.kron(np.eye(Ls), P.toarray())
    lhs = Ps.conj().T @ dirac.dwf_matrix(U, dims, Ls, M5, m).toarray() @ Ps
    rhs = mg.coarse_dwf(Dhat, Ls, m, nvec).toarray()
    assert np.abs(lhs - rhs).max() < 1e-12


def test_galerkin_identity_prolongator_reduces_to_wilson():
    """Single-site aggregates with constant vectors: P = 1, so P^dag D_W P = D_W."""
    dims = (4, 6)
    U = _u1(dims, 0.7, 11)
    V = 24
    vecs = [np.ones(2 * V, dtype=complex)]
    P, cdims = mg.build_prolongator(vecs, dims, (1, 1), 2, 1)
    assert cdims == dims
    Dw = dirac.wilson_matrix(U, dims, -1.0)
    assert np.abs(P.toarray() - np.eye(2 * V)).max() < 1e-15
    assert np.abs(mg.galerkin_kernel(P, Dw).toarray() - Dw.toarray()).max() < 1e-15


def test_galerkin_stencil_is_nearest_neighbour():
    """The coarse kernel couples a coarse site only to itself and its 2d nearest neighbours."""
    dims, block, nvec = (12, 8), (4, 4), 2
    U = _u1(dims, 0.5, 12)
    P, cdims = mg.build_prolongator(_null_vectors(U, dims, nvec, 13), dims, block, 2, 1)
    Dhat = mg.galerkin_kernel(P, dirac.wilson_matrix(U, dims, -1.0)).toarray()
    nc = 2 * nvec
    c = dirac.site_coords(cdims)
    for a in range(Dhat.shape[0] // nc):
        for b in range(Dhat.shape[0] // nc):
            blk = Dhat[a * nc:(a + 1) * nc, b * nc:(b + 1) * nc]
            d = np.abs(c[a] - c[b])
            d = np.minimum(d, np.asarray(cdims) - d)
            if d.sum() > 1:
                assert np.abs(blk).max() < 1e-14


def test_restrict_prolong_adjoint_and_wall_only():
    dims, block, nvec, Ls, Ls_c = (8, 8), (4, 4), 3, 6, 4
    U = _u1(dims, 0.5, 14)
    P, _ = mg.build_prolongator(_null_vectors(U, dims, nvec, 15), dims, block, 2, 1)
    rng = np.random.default_rng(16)
    r = synth.gaussian_complex(rng, (Ls * P.shape[0],))
    ec = synth.gaussian_complex(rng, (Ls_c * P.shape[1],))
    R = mg.restrict(r, P, Ls, Ls_c, 2, 1, nvec)
    E = mg.prolong(ec, P, Ls, Ls_c, 2, 1, nvec)
    # prolongation is the adjoint of restriction
    assert abs(np.vdot(ec, R) - np.vdot(E, r)) < 1e-12 * np.linalg.norm(r) * np.linalg.norm(ec)
    # only the wall field P_- r_1 + P_+ r_Ls is read; only coarse slices 1, Lhat_s written
    r2 = r.reshape(Ls, -1).copy()
    r2[1:Ls - 1] = 0
    r2[0, 0::2] = 0        # P_+ part of slice 1 (spin 0)
    r2[Ls - 1, 1::2] = 0   # P_- part of slice Ls (spin 1)
    assert np.abs(mg.restrict(r2.reshape(-1), P, Ls, Ls_c, 2, 1, nvec) - R).max() < 1e-14
    Rr = R.reshape(Ls_c, -1)
    assert np.abs(Rr[1:Ls_c - 1]).max() == 0
    Ee = E.reshape(Ls, -1)
    assert np.abs(Ee[1:Ls - 1]).max() == 0


def test_restrict_with_identity_prolongator_is_wall_projection():
    dims, Ls = (4, 4), 5
    V = 16
    P, _ = mg.build_prolongator([np.ones(2 * V, dtype=complex)], dims, (1, 1), 2, 1)
    r = synth.gaussian_complex(np.random.default_rng(1), (Ls, 2 * V))
    R = mg.restrict(r.reshape(-1), P, Ls, Ls, 2, 1, 1).reshape(Ls, V, 2)
    rr = r.reshape(Ls, V, 2)
    assert np.abs(R[0, :, 1] - rr[0, :, 1]).max() == 0 and np.abs(R[0, :, 0]).max() == 0
    assert np.abs(R[Ls - 1, :, 0] - rr[Ls - 1, :, 0]).max() == 0 and np.abs(R[Ls - 1, :, 1]).max() == 0


def test_two_level_kcycle_solves_to_tolerance():
    """The K-cycle reaches ||b - D_DW x|| / ||b|| <= 1e-10 and the dense solution."""
    dims, block, nvec, Ls = (8, 8), (4, 4), 4, 6
    U = _u1(dims, 0.3, 17)
    P, _ = mg.build_prolongator(_null_vectors(U, dims, nvec, 18, m_setup=-0.3, iters=60), dims, block, 2, 1)
    ml = mg.TwoLevel(U, dims, Ls, 1.0, 0.02, P, nvec, Ls_c=4)
    b = synth.gaussian_complex(np.random.default_rng(19), (Ls * 128,))
    x, outer, res = ml.solve(b, tol=1e-10)
    assert res <= 1e-10
    D = ml.Ddw.toarray()
    xd = np.linalg.solve(D, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10 * np.linalg.cond(D)
    # MG needs far fewer outer iterations than CGNR needs iterations
    _, it_cg, _ = solvers.cgnr(ml.Ddw, b, tol=1e-10)
    assert outer < it_cg / 4


@pytest.mark.parametrize("anti", [None, [0, 1]])
def test_adjoint_gradient_matches_central_differences(anti):
    dims, Ls, M5, mf = (4, 4), 4, 1.0, 0.05
    rng = np.random.default_rng(20)
    theta = synth.u1_angles(rng, dims, 0.7)
    b = synth.gaussian_spinor(rng, dims, Ls).reshape(-1)
    l0, grad = force.loss_and_grad(theta, b, dims, Ls, M5, mf, anti)
    h = 1e-6
    for mu, site in [(0, 0), (1, 5), (0, 15), (1, 12)]:
        tp = theta.copy(); tp[mu, site] += h
        tm = theta.copy(); tm[mu, site] -= h
        lp, _ = force.loss_and_grad(tp, b, dims, Ls, M5, mf, anti)
        lm, _ = force.loss_and_grad(tm, b, dims, Ls, M5, mf, anti)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grad[mu, site]) < 1e-6 * max(1.0, abs(fd))


def test_kernel_blocks_round_trip_and_sigma3_adjoint():
    """kernel_from_blocks inverts kernel_blocks on a Galerkin kernel, and the sigma_3 form of the
    coarse adjoint equals the plain adjoint of Eq. coarsenDW for an exact (gamma_5-hermitian) kernel."""
    dims, block, nvec, Ls_c, M5 = (12, 12), (4, 4), 3, 4, 1.0
    U = _u1(dims, 0.6, 31)
    P, cdims = mg.build_prolongator(_null_vectors(U, dims, nvec, 32), dims, block, 2, 1)
    Dhat = mg.galerkin_kernel(P, dirac.wilson_matrix(U, dims, -M5))
    Y = mg.kernel_blocks(Dhat, cdims, 2 * nvec)
    back = mg.kernel_from_blocks(Y, cdims)
    assert abs(back - Dhat).max() < 1e-15
    # a block-by-block change of the stored copy shows up in the assembled kernel
    Y2 = Y.copy()
    Y2[1, 3, 0, 2] += 1.0
    assert abs(mg.kernel_from_blocks(Y2, cdims) - Dhat).max() == pytest.approx(1.0)
    for m in (0.02, 1.0):
        want = dirac.dagger(mg.coarse_dwf(Dhat, Ls_c, m, nvec)).toarray()
        got = mg.coarse_dwf_dagger_g5(Dhat, Ls_c, m, nvec).toarray()
        assert np.abs(got - want).max() < 1e-13
    # sigma_3 is the coarse gamma_5: a non-hermitian change breaks the identity
    bad = Dhat.tolil()
    bad[0, 1] += 0.5
    bad = bad.tocsr()
    assert np.abs(mg.coarse_dwf_dagger_g5(bad, Ls_c, 0.02, nvec).toarray()
                  - dirac.dagger(mg.coarse_dwf(bad, Ls_c, 0.02, nvec)).toarray()).max() > 0.1


def _expm_herm(H, eps):
    w, Q = np.linalg.eigh(H)
    return (Q * np.exp(1j * eps * w)[None, :]) @ Q.conj().T


@pytest.mark.parametrize("anti", [None, [0, 0, 0, 1]])
def test_su3_force_matches_central_differences(anti):
    """4-d SU(3), 2^4 x Ls 4: dl/d eps along random algebra directions H on random links
    (U -> exp(i eps H) U) by central differences equals -2 tr(H F) of the adjoint force."""
    dims, Ls, M5, mf = (2, 2, 2, 2), 4, 1.8, 0.05
    rng = np.random.default_rng(50)
    U = synth.su3_links(rng, dims, 0.4)
    b = synth.gaussian_spinor(rng, dims, Ls, "su3").reshape(-1)
    links = [(0, 3), (1, 0), (2, 9), (3, 15)]
    l0, F = force.loss_and_force_su3(U, b, dims, Ls, M5, mf, links, anti)
    for (mu, site), Fl in zip(links, F):
        assert np.abs(Fl - Fl.conj().T).max() < 1e-12 and abs(np.trace(Fl)) < 1e-12
        G = synth.gaussian_complex(rng, (3, 3))
        H = 0.5 * (G + G.conj().T)
        H -= np.trace(H).real / 3 * np.eye(3)
        h = 1e-5
        Lpm = []
        for e in (h, -h):
            Up = U.copy()
            Up[mu, site] = _expm_herm(H, e) @ U[mu, site]
            D = dirac.dwf_matrix(Up, dims, Ls, M5, mf, "su3", anti).toarray()
            xs = np.linalg.solve(D, b)
            Lpm.append(np.vdot(xs, xs).real)
        fd = (Lpm[0] - Lpm[1]) / (2 * h)
        want = -2 * np.trace(H @ Fl).real
        assert abs(fd - want) < 1e-6 * max(1.0, abs(fd)), (mu, site, fd, want)


def _three_level(dims=(16, 16), Ls=6, nvec=4, nvec2=6, Ls_c=4, Ls_cc=4, sigma=0.3, seed=70, n_deflate=0):
    M5, mf, m_setup = 1.0, 0.02, -0.3
    U = _u1(dims, sigma, seed)
    P, cdims = mg.build_prolongator(_null_vectors(U, dims, nvec, seed + 1, m_setup=m_setup, iters=60), dims,
                                    (4, 4), 2, 1)
    Dhat = mg.galerkin_kernel(P, dirac.wilson_matrix(U, dims, -M5))
    S = mg.coarse_setup_operator(Dhat, M5, m_setup)
    rng = np.random.default_rng(seed + 2)
    v2 = [mg.relax_null_vector(S, synth.gaussian_complex(rng, (Dhat.shape[0],)), maxiter=60)[0] for _ in range(nvec2)]
    P2, cdims2 = mg.build_prolongator_chiral(v2, cdims, (2, 2), mg.coarse_chirality(nvec))
    ml = mg.ThreeLevel(U, dims, Ls, M5, mf, P, nvec, P2, nvec2, Ls_c=Ls_c, Ls_cc=Ls_cc, n_deflate=n_deflate)
    return ml, U, Dhat, P2, cdims, cdims2, v2


def test_level2_setup_operator_is_the_galerkin_of_the_shifted_kernel():
    """P^dag D_W(m) P = Dhat_W(-M5) + (m + M5) 1 because P^dag P = 1."""
    dims, block, nvec, M5, m = (8, 8), (4, 4), 3, 1.0, -0.27
    U = _u1(dims, 0.5, 71)
    P, _ = mg.build_prolongator(_null_vectors(U, dims, nvec, 72), dims, block, 2, 1)
    want = mg.galerkin_kernel(P, dirac.wilson_matrix(U, dims, m)).toarray()
    got = mg.coarse_setup_operator(mg.galerkin_kernel(P, dirac.wilson_matrix(U, dims, -M5)), M5, m).toarray()
    assert np.abs(got - want).max() < 1e-13


def test_level2_prolongator_galerkin_identities():
    """Level 2 -> 3: P2^dag P2 = 1, sigma_3 P2 = P2 sigma_3 (chirality kept), the level-2 near-null
    halves lie in the span, and P2^dag Dhat_DW P2 (P2 diagonal in s) is Eq. coarsenDW around
    P2^dag Dhat_W P2 (Sec. 2.3 applied to the coarse kernel)."""
    ml, U, Dhat, P2, cdims, cdims2, v2 = _three_level(Ls_c=4, Ls_cc=4)
    nvec, nvec2 = 4, 6
    P2d = P2.toarray()
    assert cdims2 == (2, 2)
    assert np.abs(P2d.conj().T @ P2d - np.eye(P2d.shape[1])).max() < 1e-13
    S2 = mg.sigma3(16, nvec).toarray()
    S3 = mg.sigma3(4, nvec2).toarray()
    assert np.abs(S2 @ P2d - P2d @ S3).max() < 1e-14
    Cp, Cm = mg.coarse_projectors(16, nvec)
    for v in v2:
        for proj in (Cp, Cm):
            w = proj @ v
            assert np.linalg.norm(P2 @ (P2.conj().T @ w) - w) < 1e-12 * np.linalg.norm(w)
    Dhat2 = mg.galerkin_kernel(P2, Dhat)
    Ps = np.kron(np.eye(4), P2d)
    for m in (0.02, 1.0):
        lhs = Ps.conj().T @ mg.coarse_dwf(Dhat, 4, m, nvec).toarray() @ Ps
        rhs = mg.coarse_dwf(Dhat2, 4, m, nvec2).toarray()
        assert np.abs(lhs - rhs).max() < 1e-12
    # the coarser kernel keeps sigma_3-hermiticity: its sigma_3 adjoint is its adjoint
    assert np.abs(mg.coarse_dwf_dagger_g5(Dhat2, 4, 0.02, nvec2).toarray()
                  - dirac.dagger(mg.coarse_dwf(Dhat2, 4, 0.02, nvec2)).toarray()).max() < 1e-13


def test_deflated_cgnr_start_and_dense_solution():
    """Deflated CGNR: the start is the projection of the exact solution onto the deflation space
    (V V^dag x*, V = low eigenvectors of A^dag A), the iteration reaches the dense solution, and
    deflation cuts the iterations to a loose tolerance."""
    ml, *_ = _three_level()
    A = ml.A3
    rng = np.random.default_rng(73)
    b = synth.gaussian_complex(rng, (A.shape[0],))
    Ad = A.toarray()
    xd = np.linalg.solve(Ad, b)
    from oracle import solvers as sv
    lam, V = sv.low_modes((ml.A3dag @ A).tocsr(), 24)
    x0 = V @ ((V.conj().T @ (ml.A3dag @ b)) / lam)
    assert np.linalg.norm(x0 - V @ (V.conj().T @ xd)) < 1e-10 * np.linalg.norm(xd)
    x, it = sv.cgnr_deflated(A, b, 1e-12, 5000, V, lam, Adag=ml.A3dag)
    assert np.linalg.norm(x - xd) < 1e-9 * np.linalg.norm(xd)
    _, it_plain = sv.cgnr_fixed(A, b, 0.05, 5000, Ddag=ml.A3dag)
    _, it_defl = sv.cgnr_deflated(A, b, 0.05, 5000, V, lam, Adag=ml.A3dag)
    assert it_defl < it_plain
    # a right-hand side inside the deflation space needs no iteration
    bb = Ad @ V[:, :5].sum(axis=1)
    _, it0 = sv.cgnr_deflated(A, bb, 1e-10, 5000, V, lam, Adag=ml.A3dag)
    assert it0 == 0


@pytest.mark.parametrize("n_deflate", [0, 32])
def test_three_level_kcycle_solves_to_tolerance(n_deflate):
    """The three-level K-cycle (with and without coarsest deflation) reaches 1e-10 and the dense solution."""
    ml, *_ = _three_level(n_deflate=n_deflate)
    b = synth.gaussian_complex(np.random.default_rng(74), (ml.A.shape[0],))
    x, outer, res = ml.solve(b, tol=1e-10)
    assert res <= 1e-10
    D = ml.Ddw.toarray()
    xd = np.linalg.solve(D, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10 * np.linalg.cond(D)
    assert max(ml.l2_iters) <= 16 and len(ml.l3_iters) >= len(ml.l2_iters)
    _, it_cg, _ = solvers.cgnr(ml.Ddw, b, tol=1e-10)
    assert outer < it_cg / 4


def test_transfer_diagnostics_limits():
    """The transfer-study diagnostics: bulk restriction and prolongation are adjoint; with single-site
    aggregates holding the full chiral spin space (P = 1) the bulk transfer keeps every vector
    (colinearity 0) and its coarse operator is the fine one, so one exact coarse correction leaves no
    error (oblique projector 0); the wall transfer keeps only the wall field, so its colinearity is
    the bulk share of v."""
    dims, Ls, M5, m = (4, 4), 4, 1.0, 0.05
    V = 16
    U = _u1(dims, 0.5, 41)
    P, _ = mg.build_prolongator([np.ones(2 * V, dtype=complex)], dims, (1, 1), 2, 1)
    rng = np.random.default_rng(42)
    r = synth.gaussian_complex(rng, (Ls * 2 * V,))
    ec = synth.gaussian_complex(rng, (Ls * P.shape[1],))
    assert abs(np.vdot(ec, mg.restrict_bulk(r, P, Ls)) - np.vdot(mg.prolong_bulk(ec, P, Ls), r)) < 1e-12 * 100
    A = dirac.pvdag_dwf_matrix(U, dims, Ls, M5, m)
    Dhat = mg.galerkin_kernel(P, dirac.wilson_matrix(U, dims, -M5))
    Ac = (dirac.dagger(mg.coarse_dwf(Dhat, Ls, 1.0, 1)) @ mg.coarse_dwf(Dhat, Ls, m, 1)).tocsr()
    assert abs(Ac - A).max() < 1e-14
    v = synth.gaussian_complex(rng, (Ls * 2 * V,))
    R = lambda x: mg.restrict_bulk(x, P, Ls)
    Pr = lambda x: mg.prolong_bulk(x, P, Ls)
    assert mg.colinearity(v, R, Pr) < 1e-14
    assert mg.oblique(v, A, Ac, R, Pr) < 1e-10
    # wall transfer: P R v keeps P_- v_1 and P_+ v_Ls only
    Rw = lambda x: mg.restrict(x, P, Ls, Ls, 2, 1, 1)
    Pw = lambda x: mg.prolong(x, P, Ls, Ls, 2, 1, 1)
    vv = v.reshape(Ls, V, 2)
    kept = np.sum(np.abs(vv[0, :, 1]) ** 2) + np.sum(np.abs(vv[Ls - 1, :, 0]) ** 2)
    want = np.sqrt(1 - kept / np.sum(np.abs(v) ** 2))
    assert abs(mg.colinearity(v, Rw, Pw) - want) < 1e-13


def test_wall_transfers_between_coarse_levels():
    """restrict_walls / prolong_walls with the sigma_3 projectors of a coarse level on both sides
    (the level-2 -> level-3 transfer): adjoint to each other, supported on the walls only, and,
    for a unitary prolongator that commutes with sigma_3, R P is the identity on vectors whose
    coarse slice 1 is chirality - and slice Ls_c chirality + (the wall field of Eq.
    TruncProjectInterpolate in the permuted basis)."""
    rng = np.random.default_rng(12)
    V2, nv1, Ls2, Ls3 = 6, 3, 5, 3               # level-2 sites and vectors; 2 nv1 dof per site
    n2 = V2 * 2 * nv1
    # a unitary prolongator commuting with sigma_3: one unitary per chirality sector, per site
    blocks = []
    for _ in range(V2):
        Q = [np.linalg.qr(rng.standard_normal((nv1, nv1)) + 1j * rng.standard_normal((nv1, nv1)))[0]
             for _ in range(2)]
        B = np.zeros((2 * nv1, 2 * nv1), dtype=complex)
        B[:nv1, :nv1], B[nv1:, nv1:] = Q
        blocks.append(B)
    P = np.zeros((n2, n2), dtype=complex)
    for i, B in enumerate(blocks):
        P[i * 2 * nv1:(i + 1) * 2 * nv1, i * 2 * nv1:(i + 1) * 2 * nv1] = B
    Fp, Fm = mg.coarse_projectors(V2, nv1)        # finer side: the level-2 chirality
    Cp, Cm = mg.coarse_projectors(V2, nv1)        # coarser side: the same sigma_3 split
    s3 = (Fp - Fm).toarray()
    assert np.abs(s3 @ P - P @ s3).max() < 1e-14
    x = rng.standard_normal(Ls2 * n2) + 1j * rng.standard_normal(Ls2 * n2)
    y = rng.standard_normal(Ls3 * n2) + 1j * rng.standard_normal(Ls3 * n2)
    Rx = mg.restrict_walls(x, P, Ls2, Ls3, Fp, Fm, Cp, Cm)
    Py = mg.prolong_walls(y, P, Ls2, Ls3, Fp, Fm, Cp, Cm)
    assert abs(np.vdot(Rx, y) - np.vdot(x, Py)) < 1e-12 * np.linalg.norm(x) * np.linalg.norm(y)
    assert np.abs(Rx.reshape(Ls3, n2)[1:Ls3 - 1]).max() == 0.0
    assert np.abs(Py.reshape(Ls2, n2)[1:Ls2 - 1]).max() == 0.0
    e = np.zeros((Ls3, n2), dtype=complex)
    e[0] = Cm @ (rng.standard_normal(n2) + 1j * rng.standard_normal(n2))
    e[Ls3 - 1] = Cp @ (rng.standard_normal(n2) + 1j * rng.standard_normal(n2))
    back = mg.restrict_walls(mg.prolong_walls(e.reshape(-1), P, Ls2, Ls3, Fp, Fm, Cp, Cm), P, Ls2, Ls3,
                             Fp, Fm, Cp, Cm)
    assert np.abs(back - e.reshape(-1)).max() < 1e-13
    # the opposite chiralities on the walls are dropped
    e2 = np.zeros((Ls3, n2), dtype=complex)
    e2[0] = Cp @ rng.standard_normal(n2)
    e2[Ls3 - 1] = Cm @ rng.standard_normal(n2)
    assert np.abs(mg.prolong_walls(e2.reshape(-1), P, Ls2, Ls3, Fp, Fm, Cp, Cm)).max() < 1e-14


def test_su3_generators_are_the_gell_mann_basis():
    """Traceless Hermitian, tr(T_a T_b) = delta_ab / 2, and the su(3) structure constants
    [T_1, T_2] = i T_3, [T_4, T_5] = i (T_3 + sqrt(3) T_8) / 2 of the Gell-Mann convention."""
    T = force.su3_generators()
    for a in range(8):
        assert abs(np.trace(T[a])) < 1e-15
        assert np.abs(T[a] - T[a].conj().T).max() < 1e-15
        for b in range(8):
            assert abs(np.trace(T[a] @ T[b]) - 0.5 * (a == b)) < 1e-15
    comm = lambda A, B: A @ B - B @ A
    assert np.abs(comm(T[0], T[1]) - 1j * T[2]).max() < 1e-15
    assert np.abs(comm(T[3], T[4]) - 0.5j * (T[2] + np.sqrt(3) * T[7])).max() < 1e-14


def test_directional_derivative_is_the_operator_difference():
    """D_DW is real-linear in the links (the backward hop reads U^dag), so the central difference
    of Re(lambda^dag D_DW(U + h dU e_link) x) in h equals the directional derivative exactly (up to
    rounding), for SU(3) in 4-d and U(1) in 2-d."""
    rng = synth.rng_for(13)
    for dims, Ls, group in (((2, 2, 2, 4), 2, "su3"), ((4, 6), 3, "u1")):
        nd = len(dims)
        if group == "su3":
            U = synth.su3_links(rng, dims, 0.3)
            dU = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        else:
            U = synth.u1_links(synth.u1_angles(rng, dims, 0.5))
            dU = complex(rng.standard_normal(), rng.standard_normal())
        lam = synth.gaussian_spinor(rng, dims, Ls, group).reshape(-1)
        x = synth.gaussian_spinor(rng, dims, Ls, group).reshape(-1)
        for mu, site in ((0, 1), (nd - 1, 3)):
            got = force.directional_derivative(U, dims, Ls, lam, x, mu, site, dU, group)
            h = 1e-3
            vals = []
            for sgn in (1, -1):
                Uh = np.array(U, dtype=complex, copy=True)
                Uh[mu, site] = Uh[mu, site] + sgn * h * dU
                D = dirac.dwf_matrix(Uh, dims, Ls, 1.3, 0.07, group)
                vals.append(np.vdot(lam, D @ x).real)
            want = (vals[0] - vals[1]) / (2 * h)
            assert abs(got - want) < 1e-9 * max(1.0, abs(want)), (group, mu, site, got, want)

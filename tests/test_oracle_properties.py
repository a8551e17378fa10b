"""Property-based pins of the oracle over random small geometries (hypothesis).

The fixed-shape pins elsewhere could miss an index mistake that only shows on
some shapes (non-square lattices, Ls = 1, odd extents, antiperiodic
directions).  Each property here is fixed by the definitions of Sec. 2 and 2.3
for every shape:
  * Gamma_5-hermiticity of D_DW: D_DW^dag = Gamma_5 D_DW Gamma_5 with
    Gamma_5 = gamma_5 R_5 (Sec. 2.1);
  * D_PV - D_DW(m) lives only on the two wall corners, as -(1 - m) P_+ on
    (1, Ls) and -(1 - m) P_- on (Ls, 1) (Eq. DWoperator with m -> 1: its
    literal corner terms are -m P_+ and -m P_-);
  * the sparse operator agrees with its point evaluator at every site;
  * the prolongator: P^dag P = 1 and gamma_5 P = P sigma_3 (Sec. 2.3);
  * the truncated transfers are adjoint and supported on the walls only
    (Eq. TruncProjectInterpolate);
  * the Mobius operator at b5 = 1, c5 = 0 is the Shamir operator;
  * the Galerkin kernel is sigma_3-hermitian (Sec. 2.3).
"""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import synth  # noqa: E402
from oracle import dirac, mg  # noqa: E402

SETTINGS = dict(max_examples=25, deadline=None, derandomize=True)

geoms_2d = st.tuples(st.integers(2, 6), st.integers(2, 6), st.integers(1, 5),
                     st.lists(st.booleans(), min_size=2, max_size=2))


def _u1(dims, seed, sigma=0.6):
    rng = np.random.default_rng(seed)
    return np.exp(1j * rng.normal(0.0, sigma, (len(dims),) + (int(np.prod(dims)),)))


@settings(**SETTINGS)
@given(geoms_2d, st.floats(0.2, 1.9), st.floats(0.0, 0.5), st.integers(0, 10_000))
def test_gamma5_hermiticity_any_shape(g, M5, mf, seed):
    L0, L1, Ls, anti = g
    dims = (L0, L1)
    U = _u1(dims, seed)
    D = dirac.dwf_matrix(U, dims, Ls, M5, mf, antiperiodic=[int(a) for a in anti]).toarray()
    G5 = dirac.reflection_gamma5(L0 * L1, Ls, 2, 1).toarray()
    assert np.abs(D.conj().T - G5 @ D @ G5).max() < 1e-13


@settings(**SETTINGS)
@given(geoms_2d, st.floats(0.2, 1.9), st.floats(0.0, 0.5), st.integers(0, 10_000))
def test_pv_differs_only_on_the_wall_corners(g, M5, mf, seed):
    L0, L1, Ls, anti = g
    dims = (L0, L1)
    V = L0 * L1
    U = _u1(dims, seed)
    an = [int(a) for a in anti]
    diff = (dirac.pv_matrix(U, dims, Ls, M5, antiperiodic=an)
            - dirac.dwf_matrix(U, dims, Ls, M5, mf, antiperiodic=an)).toarray()
    n = 2 * V
    Pp, Pm = dirac.site_projectors(V, 2, 1)
    want = np.zeros_like(diff)
    if Ls == 1:
        # both corners fall on the one slice: -m (P_+ + P_-) = -m for D_DW(m), -1 for D_PV
        want[:n, :n] = (mf - 1.0) * (Pp + Pm).toarray()
    else:
        # the corner terms -m P_+ on (1, Ls) and -m P_- on (Ls, 1) become -P_+ and -P_- for D_PV
        want[:n, (Ls - 1) * n:] = -(1.0 - mf) * Pp.toarray()
        want[(Ls - 1) * n:, :n] = -(1.0 - mf) * Pm.toarray()
    assert np.abs(diff - want).max() < 1e-14


@settings(**SETTINGS)
@given(geoms_2d, st.booleans(), st.integers(0, 10_000))
def test_point_evaluator_matches_the_assembled_operator(g, dag, seed):
    L0, L1, Ls, anti = g
    dims = (L0, L1)
    V = L0 * L1
    an = [int(a) for a in anti]
    U = _u1(dims, seed)
    rng = np.random.default_rng(seed + 1)
    psi = rng.standard_normal(Ls * V * 2) + 1j * rng.standard_normal(Ls * V * 2)
    D = dirac.dwf_matrix(U, dims, Ls, 1.1, 0.07, antiperiodic=an)
    want = (dirac.dagger(D) if dag else D) @ psi
    points = [(s, x) for s in range(Ls) for x in range(V)]
    got = dirac.dwf_apply_points_2d(U, psi, dims, Ls, 1.1, 0.07, points, dagger_=dag, antiperiodic=an)
    assert np.abs(np.asarray(got).reshape(-1) - want).max() < 1e-12 * max(1.0, np.abs(want).max())


@settings(**SETTINGS)
@given(st.sampled_from([((4, 4), (2, 2)), ((6, 4), (3, 2)), ((4, 6), (2, 3)), ((8, 4), (4, 4))]),
       st.integers(1, 3), st.integers(0, 10_000))
def test_prolongator_orthonormal_and_chiral_any_shape(geom, nvec, seed):
    dims, block = geom
    V = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    vecs = [rng.standard_normal(V * 2) + 1j * rng.standard_normal(V * 2) for _ in range(nvec)]
    P, cdims = mg.build_prolongator(vecs, dims, block, 2, 1)
    P = P.toarray() if hasattr(P, "toarray") else np.asarray(P)
    assert np.abs(P.conj().T @ P - np.eye(P.shape[1])).max() < 1e-12
    Vc = int(np.prod(cdims))
    g5 = np.kron(np.eye(V), np.diag([1.0, -1.0]))
    s3 = np.kron(np.eye(Vc), np.diag([1.0] * nvec + [-1.0] * nvec))
    assert np.abs(g5 @ P - P @ s3).max() < 1e-12


@settings(**SETTINGS)
@given(st.integers(1, 6), st.integers(1, 4), st.integers(0, 10_000))
def test_truncated_transfers_adjoint_and_on_the_walls(Ls, Ls_c, seed):
    dims, block, nvec = (4, 4), (2, 2), 2
    V = 16
    rng = np.random.default_rng(seed)
    vecs = [rng.standard_normal(V * 2) + 1j * rng.standard_normal(V * 2) for _ in range(nvec)]
    P, cdims = mg.build_prolongator(vecs, dims, block, 2, 1)
    nf, nc = P.shape
    x = rng.standard_normal(Ls * nf) + 1j * rng.standard_normal(Ls * nf)
    y = rng.standard_normal(Ls_c * nc) + 1j * rng.standard_normal(Ls_c * nc)
    Rx = mg.restrict(x, P, Ls, Ls_c, 2, 1, nvec)
    Py = mg.prolong(y, P, Ls, Ls_c, 2, 1, nvec)
    assert abs(np.vdot(Rx, y) - np.vdot(x, Py)) < 1e-12 * np.linalg.norm(x) * np.linalg.norm(y)
    if Ls_c > 2:
        assert np.abs(Rx.reshape(Ls_c, nc)[1:Ls_c - 1]).max() == 0.0
    if Ls > 2:
        assert np.abs(Py.reshape(Ls, nf)[1:Ls - 1]).max() == 0.0


@settings(max_examples=12, deadline=None, derandomize=True)
@given(st.tuples(st.integers(2, 3), st.integers(2, 3), st.integers(2, 3), st.integers(2, 4)), st.integers(1, 3),
       st.lists(st.booleans(), min_size=4, max_size=4), st.integers(0, 10_000))
def test_su3_gamma5_hermiticity_and_point_evaluator_any_shape(dims, Ls, anti, seed):
    """4-d SU(3): Gamma_5-hermiticity and the point evaluator, on random small shapes."""
    if int(np.prod(dims)) > 36:
        dims = (2, 2, 2, dims[3])
    V = int(np.prod(dims))
    rng = synth.rng_for(seed)
    U = synth.su3_links(rng, dims, 0.3)
    an = [int(a) for a in anti]
    D = dirac.dwf_matrix(U, dims, Ls, 1.8, 0.05, "su3", an)
    Dd = D.toarray()
    G5 = dirac.reflection_gamma5(V, Ls, 4, 3).toarray()
    assert np.abs(Dd.conj().T - G5 @ Dd @ G5).max() < 1e-13
    psi = synth.gaussian_spinor(rng, dims, Ls, "su3").reshape(-1)
    points = [(s, x) for s in range(Ls) for x in range(V)]
    got = np.asarray(dirac.dwf_apply_points(U, psi, dims, Ls, 1.8, 0.05, points, "su3", antiperiodic=an)).reshape(-1)
    want = D @ psi
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


@settings(**SETTINGS)
@given(geoms_2d, st.floats(0.2, 1.9), st.floats(0.0, 0.5), st.integers(0, 10_000))
def test_mobius_at_b5_1_c5_0_is_the_shamir_operator(g, M5, mf, seed):
    """D_M = (1_s x D_W)(b5 - c5 H_s) + 1 + H_s reduces to D_DW at b5 = 1, c5 = 0, for every shape."""
    L0, L1, Ls, anti = g
    dims = (L0, L1)
    an = [int(a) for a in anti]
    U = _u1(dims, seed)
    Dm = dirac.mobius_matrix(U, dims, Ls, M5, mf, 1.0, 0.0, antiperiodic=an)
    Dd = dirac.dwf_matrix(U, dims, Ls, M5, mf, antiperiodic=an)
    assert abs(Dm - Dd).max() < 1e-14


@settings(**SETTINGS)
@given(st.sampled_from([((4, 4), (2, 2)), ((6, 4), (3, 2)), ((8, 4), (4, 2))]), st.integers(1, 3),
       st.integers(0, 10_000))
def test_galerkin_kernel_is_sigma3_hermitian(geom, nvec, seed):
    """With a chirality-preserving prolongator the Galerkin kernel inherits gamma_5-hermiticity:
    Dhat_W^dag = sigma_3 Dhat_W sigma_3 (the adjoint coarse stencil reads the same blocks)."""
    dims, block = geom
    V = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    U = _u1(dims, seed + 3)
    vecs = [rng.standard_normal(V * 2) + 1j * rng.standard_normal(V * 2) for _ in range(nvec)]
    P, cdims = mg.build_prolongator(vecs, dims, block, 2, 1)
    K = mg.galerkin_kernel(P, dirac.wilson_matrix(U, dims, -1.0)).toarray()
    Vc = int(np.prod(cdims))
    s3 = np.kron(np.eye(Vc), np.diag([1.0] * nvec + [-1.0] * nvec))
    assert np.abs(K.conj().T - s3 @ K @ s3).max() < 1e-12 * max(1.0, np.abs(K).max())

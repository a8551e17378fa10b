"""GPU parity of the third multigrid level and the coarsest deflation (Table
kcycle, Table zerospacing) with the FP64 oracle, and three-level solves to a
true residual of 1e-10.

FP64 setup outputs (relaxed level-2 null vectors, prolongator P2, level-3
Galerkin blocks) are compared at 1e-10 / 1e-12; the FP32 level-3 stencil and the
level 2 <-> 3 transfers at 1e-5.  With at least as many Lanczos steps as the
coarsest level has unknowns the deflation space is exact, so the Lanczos
eigenvalue estimates and the deflated start match the oracle's dense
eigen-decomposition to FP32 accuracy.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import dirac, mg as omg, solvers

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dw():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2004_07732_gb300 as pkg
    pkg.lib()
    return pkg


def _dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to("cuda").to(dtype)


class Hier:
    """A 2-d hierarchy 32^2 x Ls 8 -> 8^2 (16 dof) -> 4^2 (24 dof), and the oracle's view of it."""

    def __init__(self, dw, dims=(32, 32), Ls=8, sigma=0.5, M5=1.0, mf=0.02, m_setup=-0.19, seed=900,
                 level=None, iters1=20):
        self.dims, self.Ls, self.M5, self.mf = dims, Ls, M5, mf
        rng = synth.rng_for(seed)
        self.U = synth.u1_links(synth.u1_angles(rng, dims, sigma))
        V = int(np.prod(dims))
        starts = np.stack([synth.gaussian_complex(rng, (V * 2,)) for _ in range(8)])
        self.g = dw.make_geom(dims, Ls)
        self.h = dw.mg_setup(self.g, _dev(self.U), M5, mf, {"setup_maxiter": iters1, "setup_mass": m_setup},
                             _dev(starts))
        self.cdims = tuple(d // 4 for d in dims)
        Vc = int(np.prod(self.cdims))
        lp = {"setup_mass": m_setup}
        lp.update(level or {})
        self.lp = lp
        self.starts2 = np.stack([synth.gaussian_complex(rng, (Vc * 16,)) for _ in range(lp.get("nvec", 12))])
        n3 = (Vc // 4) * lp.get("Ls_c", 4) * 2 * lp.get("nvec", 12)
        self.lstart = synth.gaussian_complex(rng, (n3,))
        dw.mg_add_level(self.h, lp, _dev(self.starts2), _dev(self.lstart))
        v1 = dw.mg_get_null_vectors(self.h).cpu().numpy().reshape(8, -1)
        self.P, _ = omg.build_prolongator(list(v1), dims, (4, 4), 2, 1)
        self.Dhat = omg.galerkin_kernel(self.P, dirac.wilson_matrix(self.U, dims, -M5))


@pytest.fixture(scope="module")
def hier(dw):
    return Hier(dw, level={"setup_maxiter": 12, "n_deflate": 32, "lanczos_steps": 2048, "block_prec": "f32"})


def test_level2_relaxation_matches_oracle(dw, hier):
    S = omg.coarse_setup_operator(hier.Dhat, hier.M5, hier.lp["setup_mass"])
    got = dw.mg_level_get(hier.h, 0).cpu().numpy().reshape(12, -1)
    for k in range(12):
        v, it = omg.relax_null_vector(S, hier.starts2[k], maxiter=12, tol=1e-4)
        assert np.linalg.norm(got[k] - v) / np.linalg.norm(v) < 1e-10, k


def test_level2_prolongator_and_level3_galerkin_match_oracle(dw, hier):
    v2 = dw.mg_level_get(hier.h, 0).cpu().numpy().reshape(12, -1)
    P2, cdims2 = omg.build_prolongator_chiral(list(v2), hier.cdims, (2, 2), omg.coarse_chirality(8))
    Vc = int(np.prod(hier.cdims))
    got = dw.mg_level_get(hier.h, 1).cpu().numpy().reshape(Vc, 2, 8, 12)
    agg, _ = omg.aggregate_map(hier.cdims, (2, 2))
    P2d = P2.toarray()
    for c in range(2):
        for k in range(12):
            for a in range(8):
                want = P2d[np.arange(Vc) * 16 + c * 8 + a, (agg * 2 + c) * 12 + k]
                assert np.abs(got[:, c, a, k] - want).max() < 1e-12
    Dhat2 = omg.galerkin_kernel(P2, hier.Dhat)
    Y = dw.mg_level_get(hier.h, 2).cpu().numpy().reshape(-1, 5, 24, 24)
    want = omg.kernel_blocks(Dhat2, cdims2, 24)
    assert np.abs(Y - want).max() < 1e-12 * np.abs(want).max()


def _oracle_level3(dw, hier):
    v2 = dw.mg_level_get(hier.h, 0).cpu().numpy().reshape(12, -1)
    P2, _ = omg.build_prolongator_chiral(list(v2), hier.cdims, (2, 2), omg.coarse_chirality(8))
    return P2, omg.galerkin_kernel(P2, hier.Dhat)


def test_level3_operator_and_transfers_match_oracle(dw, hier):
    P2, Dhat2 = _oracle_level3(dw, hier)
    h = hier.h
    rng = np.random.default_rng(5)
    v = synth.gaussian_complex(rng, (h.level_size,)).astype(np.complex64)
    vd = _dev(v, torch.complex64)
    out = torch.full_like(vd, float("nan"))
    for m in (hier.mf, 1.0):
        for dag in (False, True):
            C = omg.coarse_dwf_dagger_g5(Dhat2, 4, m, 12) if dag else omg.coarse_dwf(Dhat2, 4, m, 12)
            want = C @ v.astype(np.complex128)
            dw.mg_level_apply(h, vd, out, m, dagger=dag)
            assert np.linalg.norm(out.cpu().numpy() - want) / np.linalg.norm(want) < 1e-5, (m, dag)
    Vc = int(np.prod(hier.cdims))
    p2 = omg.coarse_projectors(Vc, 8)
    p3 = omg.coarse_projectors(Vc // 4, 12)
    r2 = synth.gaussian_complex(rng, (h.coarse_size,)).astype(np.complex64)
    r3 = torch.full((h.level_size,), float("nan"), dtype=torch.complex64, device="cuda")
    dw.mg_level_restrict(h, _dev(r2, torch.complex64), r3)
    want = omg.restrict_walls(r2.astype(np.complex128), P2, 4, 4, p2[0], p2[1], *p3)
    assert np.linalg.norm(r3.cpu().numpy() - want) / np.linalg.norm(want) < 1e-5
    e2 = torch.full((h.coarse_size,), float("nan"), dtype=torch.complex64, device="cuda")
    dw.mg_level_prolong(h, vd, e2)
    want = omg.prolong_walls(v.astype(np.complex128), P2, 4, 4, p2[0], p2[1], *p3)
    assert np.linalg.norm(e2.cpu().numpy() - want) / np.linalg.norm(want) < 1e-5


def _round16(Y):
    return Y.real.astype(np.float16).astype(np.float64) + 1j * Y.imag.astype(np.float16).astype(np.float64)


def test_level3_fp16_blocks_match_oracle_on_rounded_blocks(dw):
    """FP16 storage of the third level's blocks (block_prec): the stencil equals the oracle's coarse
    operator built from the GPU's FP64 Galerkin blocks rounded to FP16, at FP32 accuracy."""
    hh = Hier(dw, seed=905, level={"setup_maxiter": 12, "n_deflate": 0, "block_prec": "f32_l16"})
    h = hh.h
    cd3 = tuple(d // 2 for d in hh.cdims)
    Y = dw.mg_level_get(h, 2).cpu().numpy().reshape(-1, 5, 24, 24)
    K = omg.kernel_from_blocks(_round16(Y), cd3)
    rng = np.random.default_rng(6)
    v = synth.gaussian_complex(rng, (h.level_size,)).astype(np.complex64)
    vd = _dev(v, torch.complex64)
    out = torch.full_like(vd, float("nan"))
    for m in (hh.mf, 1.0):
        for dag in (False, True):
            C = omg.coarse_dwf_dagger_g5(K, 4, m, 12) if dag else omg.coarse_dwf(K, 4, m, 12)
            want = C @ v.astype(np.complex128)
            dw.mg_level_apply(h, vd, out, m, dagger=dag)
            assert np.linalg.norm(out.cpu().numpy() - want) / np.linalg.norm(want) < 1e-5, (m, dag)
    h.close()


def test_deflation_space_matches_dense_eigendecomposition(dw, hier):
    """Lanczos run to the full dimension: its lowest 32 eigenvalue estimates are those of the
    coarsest normal operator N, and the deflated start is V Lambda^-1 V^dag A^dag b with the exact
    eigenvectors; the deflated CGNR then reaches the dense solution."""
    P2, Dhat2 = _oracle_level3(dw, hier)
    A = (dirac.dagger(omg.coarse_dwf(Dhat2, 4, 1.0, 12)) @ omg.coarse_dwf(Dhat2, 4, hier.mf, 12)).tocsr()
    Ad = dirac.dagger(A)
    lam, V = solvers.low_modes((Ad @ A).tocsr(), 32)
    ritz = np.array(dw.mg_level_ritz_values(hier.h))
    assert len(ritz) == 32
    assert np.abs(ritz - lam).max() < 1e-3 * lam.max(), (ritz[:4], lam[:4])
    b = synth.gaussian_complex(np.random.default_rng(6), (hier.h.level_size,)).astype(np.complex64)
    bd = _dev(b, torch.complex64)
    x = torch.empty_like(bd)
    it = dw.mg_level_coarsest_solve(hier.h, bd, x, tol=0.05, maxiter=0, deflate=True)
    assert it == 0
    want = V @ ((V.conj().T @ (Ad @ b.astype(np.complex128))) / lam)
    assert np.linalg.norm(x.cpu().numpy() - want) / np.linalg.norm(want) < 1e-3
    it = dw.mg_level_coarsest_solve(hier.h, bd, x, tol=1e-5, maxiter=5000, deflate=True)
    xd = np.linalg.solve(A.toarray(), b.astype(np.complex128))
    assert np.linalg.norm(x.cpu().numpy() - xd) / np.linalg.norm(xd) < 1e-3
    it_plain = dw.mg_level_coarsest_solve(hier.h, bd, x, tol=0.05, maxiter=5000, deflate=False)
    it_defl = dw.mg_level_coarsest_solve(hier.h, bd, x, tol=0.05, maxiter=5000, deflate=True)
    assert it_defl <= it_plain


def test_three_level_solve_matches_dense_solution(dw, hier):
    rng = np.random.default_rng(7)
    b = synth.gaussian_spinor(rng, hier.dims, hier.Ls).reshape(-1)
    x = torch.empty(len(b), dtype=torch.complex128, device="cuda")
    st, _ = dw.mg_solve(hier.h, _dev(b), x, tol=1e-10)
    D = dirac.dwf_matrix(hier.U, hier.dims, hier.Ls, hier.M5, hier.mf)
    xs = x.cpu().numpy()
    res = np.linalg.norm(b - D @ xs) / np.linalg.norm(b)
    assert res <= 1e-10, st
    xd, _, _ = solvers.cgnr(D, b, tol=1e-12)
    assert np.linalg.norm(xs - xd) / np.linalg.norm(xd) < 1e-6
    assert 0 < st["coarse_avg_iters"] <= 16 and st["coarsest_avg_iters"] > 0
    l2, l3 = dw.mg_level_last_iterations(hier.h)
    assert 1 <= l2 <= 16 and l3 >= 0


@pytest.mark.parametrize("wl,m_setup", [(synth.SCHWINGER_256, -0.3), (synth.SCHWINGER_256_SMOOTH, -0.035)])
def test_three_level_solve_256(dw, wl, m_setup):
    """The 256^2 x 16 workloads (sigma 0.7 and the paper-like 0.214) with the three-level K-cycle and
    128 deflated coarsest modes reach a true residual of 1e-10, recomputed by the oracle."""
    U, (b,) = wl.draw(1)
    b = b.reshape(-1)
    rng = synth.rng_for(wl.seed + 50)
    V = int(np.prod(wl.dims))
    starts = np.stack([synth.gaussian_complex(rng, (V * 2,)) for _ in range(8)])
    g = dw.make_geom(wl.dims, wl.Ls)
    h = dw.mg_setup(g, _dev(U.reshape(-1)), wl.M5, wl.mf, {"setup_mass": m_setup}, _dev(starts))
    Vc = V // 16
    starts2 = np.stack([synth.gaussian_complex(rng, (Vc * 16,)) for _ in range(12)])
    lstart = synth.gaussian_complex(rng, ((Vc // 4) * 4 * 24,))
    dw.mg_add_level(h, {"setup_mass": m_setup}, _dev(starts2), _dev(lstart))
    x = torch.empty(len(b), dtype=torch.complex128, device="cuda")
    st, _ = dw.mg_solve(h, _dev(b), x, tol=1e-10)
    D = dirac.dwf_matrix(U, wl.dims, wl.Ls, wl.M5, wl.mf)
    res = np.linalg.norm(b - D @ x.cpu().numpy()) / np.linalg.norm(b)
    assert res <= 1e-10, st
    h.close()


def test_add_level_rejects_bad_arguments(dw, hier):
    with pytest.raises(dw.DwfError):     # already three levels
        dw.mg_add_level(hier.h, {}, _dev(hier.starts2), _dev(hier.lstart))
    g = dw.make_geom((16, 16), 4)
    rng = synth.rng_for(3)
    U = synth.u1_links(synth.u1_angles(rng, (16, 16), 0.5))
    h = dw.mg_setup(g, _dev(U), 1.0, 0.02, {"setup_maxiter": 5},
                    _dev(np.stack([synth.gaussian_complex(rng, (512,)) for _ in range(8)])))
    with pytest.raises(dw.DwfError):     # 2^2 blocks must divide the 4 x 4 coarse lattice: 3 does not
        dw.mg_add_level(h, {"block": [3, 3, 1, 1]}, _dev(np.zeros((12, 256))), _dev(np.zeros(1536)))
    with pytest.raises(dw.DwfError):     # deflation needs a Lanczos start
        dw.mg_add_level(h, {}, _dev(np.zeros((12, 256))), None)
    with pytest.raises(dw.DwfError):     # the blocks are stored in FP32 or FP16 only
        dw.mg_add_level(h, {"block_prec": "f64"}, _dev(np.zeros((12, 256))), _dev(np.zeros(1536)))
    h.close()

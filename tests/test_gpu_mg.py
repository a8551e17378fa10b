"""GPU parity of the multigrid pieces against the FP64 oracle, and MG solves to 1e-10.

Setup (relaxation, prolongator, Galerkin blocks) runs in FP64 on the GPU and is
compared at 1e-10 or tighter; the FP32 coarse operator and transfers at 1e-5;
solves must reach a true FP64 residual of 1e-10 (recomputed by the oracle).
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


def _problem(dims, Ls, sigma, nvec, seed, anti=None):
    rng = synth.rng_for(seed)
    U = synth.u1_links(synth.u1_angles(rng, dims, sigma))
    V = int(np.prod(dims))
    starts = np.stack([synth.gaussian_complex(rng, (V * 2,)) for _ in range(nvec)])
    b = synth.gaussian_spinor(rng, dims, Ls).reshape(-1)
    return U, starts, b


def _setup(dw, dims, Ls, U, starts, M5, mf, params, anti=None):
    g = dw.make_geom(dims, Ls, antiperiodic=anti)
    return dw.mg_setup(g, _dev(U), M5, mf, params, _dev(starts)), g


def _gpu_P_as_matrix(dw, h, dims, nvec):
    """The GPU prolongator [site][chir][k] as the oracle's sparse layout (dense)."""
    V = int(np.prod(dims))
    P = dw.mg_get_prolongator(h).cpu().numpy().reshape(V, 2, nvec)
    agg, cdims = omg.aggregate_map(dims, (4, 4) if dims[0] % 4 == 0 else (2, 2))
    return P, agg


@pytest.mark.parametrize("dims,block,nvec", [((16, 16), (4, 4), 4), ((12, 8), (4, 4), 8), ((8, 12), (2, 4), 3)])
def test_prolongator_matches_oracle(dw, dims, block, nvec):
    U, starts, _ = _problem(dims, 4, 0.5, nvec, 5)
    h, _ = _setup(dw, dims, 4, U, starts, 1.0, 0.02, {"nvec": nvec, "block": list(block) + [1, 1], "setup_maxiter": 0})
    P_o, _ = omg.build_prolongator(list(starts), dims, block, 2, 1)
    P_o = P_o.toarray()
    V = int(np.prod(dims))
    P = dw.mg_get_prolongator(h).cpu().numpy().reshape(V, 2, nvec)
    agg, _ = omg.aggregate_map(dims, block)
    for c in range(2):
        for k in range(nvec):
            col = (agg * 2 + c) * nvec + k
            want = P_o[np.arange(V) * 2 + c, col]
            assert np.abs(P[:, c, k] - want).max() < 1e-12
    h.close()


def test_relaxation_matches_oracle(dw):
    dims, nvec, iters = (16, 16), 3, 12
    U, starts, _ = _problem(dims, 4, 0.5, nvec, 6)
    h, _ = _setup(dw, dims, 4, U, starts, 1.0, 0.02,
                  {"nvec": nvec, "block": [4, 4, 1, 1], "setup_maxiter": iters, "setup_mass": -0.19})
    got = dw.mg_get_null_vectors(h).cpu().numpy().reshape(nvec, -1)
    Dw = dirac.wilson_matrix(U, dims, -0.19)
    for k in range(nvec):
        v, it = omg.relax_null_vector(Dw, starts[k], maxiter=iters, tol=1e-4)
        assert np.linalg.norm(got[k] - v) / np.linalg.norm(v) < 1e-10
    h.close()


@pytest.mark.parametrize("anti", [None, [0, 1]])
def test_galerkin_blocks_match_oracle(dw, anti):
    dims, block, nvec, M5 = (12, 16), (4, 4), 4, 1.0
    U, starts, _ = _problem(dims, 4, 0.7, nvec, 7)
    h, _ = _setup(dw, dims, 4, U, starts, M5, 0.02, {"nvec": nvec, "block": [4, 4, 1, 1], "setup_maxiter": 20,
                                                      "setup_mass": -0.3}, anti)
    vecs = dw.mg_get_null_vectors(h).cpu().numpy().reshape(nvec, -1)
    P_o, cdims = omg.build_prolongator(list(vecs), dims, block, 2, 1)
    Dhat = omg.galerkin_kernel(P_o, dirac.wilson_matrix(U, dims, -M5, antiperiodic=anti)).toarray()
    ncd = 2 * nvec
    Vc = int(np.prod(cdims))
    Y = dw.mg_get_coarse_links(h).cpu().numpy().reshape(Vc, 5, ncd, ncd)
    c = dirac.site_coords(cdims)
    for xc in range(Vc):
        for d in range(5):
            cc = c[xc].copy()
            if d > 0:
                mu, step = (d - 1) // 2, (1 if (d - 1) % 2 == 0 else -1)
                cc[mu] = (cc[mu] + step) % cdims[mu]
            nb = int(dirac.site_index(cc[None, :], cdims)[0])
            want = Dhat[xc * ncd:(xc + 1) * ncd, nb * ncd:(nb + 1) * ncd]
            assert np.abs(Y[xc, d] - want).max() < 1e-12
    h.close()


@pytest.mark.parametrize("Ls,Ls_c", [(8, 4), (6, 6), (4, 2)])
def test_coarse_operator_and_transfers_match_oracle(dw, Ls, Ls_c):
    dims, block, nvec, M5, mf = (16, 12), (4, 4), 4, 1.0, 0.03
    U, starts, _ = _problem(dims, Ls, 0.5, nvec, 8)
    h, _ = _setup(dw, dims, Ls, U, starts, M5, mf, {"nvec": nvec, "block": [4, 4, 1, 1], "setup_maxiter": 10,
                                                     "setup_mass": -0.19, "Ls_c": Ls_c, "coarse_block_prec": "f32"})
    vecs = dw.mg_get_null_vectors(h).cpu().numpy().reshape(nvec, -1)
    P_o, cdims = omg.build_prolongator(list(vecs), dims, block, 2, 1)
    Dhat = omg.galerkin_kernel(P_o, dirac.wilson_matrix(U, dims, -M5))
    rng = np.random.default_rng(3)
    nc = h.coarse_size
    v = synth.gaussian_complex(rng, (nc,)).astype(np.complex64)
    vd = _dev(v, torch.complex64)
    out = torch.empty_like(vd)
    for m in (mf, 1.0):
        C = omg.coarse_dwf(Dhat, Ls_c, m, nvec)
        for dag in (False, True):
            dw.mg_coarse_apply(h, vd, out, m, dagger=dag)
            want = (dirac.dagger(C) if dag else C) @ v.astype(np.complex128)
            assert np.linalg.norm(out.cpu().numpy() - want) / np.linalg.norm(want) < 1e-5
    # restriction / prolongation
    r = synth.gaussian_spinor(rng, dims, Ls).reshape(-1).astype(np.complex64)
    rc = torch.empty(nc, dtype=torch.complex64, device="cuda")
    dw.mg_restrict(h, _dev(r, torch.complex64), rc)
    want = omg.restrict(r.astype(np.complex128), P_o, Ls, Ls_c, 2, 1, nvec)
    assert np.linalg.norm(rc.cpu().numpy() - want) / np.linalg.norm(want) < 1e-5
    ef = torch.empty(len(r), dtype=torch.complex64, device="cuda")
    dw.mg_prolong(h, vd, ef)
    want = omg.prolong(v.astype(np.complex128), P_o, Ls, Ls_c, 2, 1, nvec)
    assert np.linalg.norm(ef.cpu().numpy() - want) / np.linalg.norm(want) < 1e-5
    h.close()


@pytest.mark.parametrize("dims,Ls,sigma,mset", [((16, 16), 8, 0.3, -0.08), ((32, 32), 8, 0.5, -0.19),
                                                 ((24, 16), 6, 0.5, -0.19)])
@pytest.mark.parametrize("coarse", [{"coarse_solver": 1}, {"coarse_solver": 1, "cgs_passes": 2},
                                    {"coarse_solver": 1, "coarse_persistent": 2},
                                    {"coarse_solver": 0, "coarse_persistent": 1},
                                    {"coarse_solver": 0, "coarse_persistent": 0}])
def test_mg_solve_reaches_tolerance(dw, dims, Ls, sigma, mset, coarse):
    M5, mf = 1.0, 0.01
    U, starts, b = _problem(dims, Ls, sigma, 8, 9)
    prm = {"setup_mass": mset}
    prm.update(coarse)
    h, g = _setup(dw, dims, Ls, U, starts, M5, mf, prm)
    x = torch.empty(len(b), dtype=torch.complex128, device="cuda")
    stats, status = dw.mg_solve(h, _dev(b), x, tol=1e-10)
    D = dirac.dwf_matrix(U, dims, Ls, M5, mf)
    xs = x.cpu().numpy()
    res = np.linalg.norm(b - D @ xs) / np.linalg.norm(b)
    assert status == 0 and res <= 1e-10 and abs(res - stats["true_residual"]) < 1e-12
    xo, it_o, _ = solvers.cgnr(D, b, tol=1e-11)
    assert np.linalg.norm(xs - xo) / np.linalg.norm(xo) < 1e-6
    assert stats["fine_applies"] < 2 * it_o       # far fewer fine applies than CGNR
    h.close()


def test_mg_solve_full_size_256(dw):
    """The 256x256 x Ls=16 workload (sigma 0.7, m 0.005) reaches 1e-10 (checked by the oracle)."""
    wl = synth.SCHWINGER_256
    U, srcs = wl.draw(1)
    b = srcs[0].reshape(-1)
    rng = synth.rng_for(wl.seed + 7000)
    starts = np.stack([synth.gaussian_complex(rng, (wl.V * 2,)) for _ in range(8)])
    g = dw.make_geom(wl.dims, wl.Ls)
    h = dw.mg_setup(g, _dev(U), wl.M5, wl.mf, {"setup_mass": -0.3}, _dev(starts))
    x = torch.empty(len(b), dtype=torch.complex128, device="cuda")
    stats, status = dw.mg_solve(h, _dev(b), x, tol=1e-10)
    D = dirac.dwf_matrix(U, wl.dims, wl.Ls, wl.M5, wl.mf)
    res = np.linalg.norm(b - D @ x.cpu().numpy()) / np.linalg.norm(b)
    assert status == 0 and res <= 1e-10
    h.close()


def test_mg_noconv_and_bad_params(dw):
    dims, Ls = (16, 16), 4
    U, starts, b = _problem(dims, Ls, 0.5, 8, 10)
    g = dw.make_geom(dims, Ls)
    with pytest.raises(dw.DwfError):
        dw.mg_setup(g, _dev(U), 1.0, 0.01, {"block": [3, 4, 1, 1]}, _dev(starts))     # 3 does not divide 16
    with pytest.raises(dw.DwfError):
        dw.mg_setup(g, _dev(U), 1.0, 0.01, {"nvec": 20}, _dev(np.zeros((20, 512))))    # 20 > 16 dof per aggregate
    h = dw.mg_setup(g, _dev(U), 1.0, 0.01, {"setup_mass": -0.19}, _dev(starts))
    x = torch.empty(len(b), dtype=torch.complex128, device="cuda")
    stats, status = dw.mg_solve(h, _dev(b), x, tol=1e-10, maxiter=1, raise_noconv=False)
    assert status == 3 and stats["iterations"] == 1 and stats["true_residual"] > 1e-10
    h.close()

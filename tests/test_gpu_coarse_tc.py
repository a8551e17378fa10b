"""GPU parity of the tensor-core coarse operator on many right-hand sides
(mg_coarse_apply_multi) against the FP64 oracle's Galerkin coarse operator
(Eq. coarsenDW), and against the one-vector FP32 stencil at larger sizes."""
import numpy as np
import pytest
import torch

import synth
from oracle import dirac, mg as omg

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


def _setup(dw, dims, Ls, Ls_c, seed, sigma=0.5):
    nvec, M5, mf = 8, 1.0, 0.03
    rng = synth.rng_for(seed)
    U = synth.u1_links(synth.u1_angles(rng, dims, sigma))
    V = int(np.prod(dims))
    starts = np.stack([synth.gaussian_complex(rng, (V * 2,)) for _ in range(nvec)])
    g = dw.make_geom(dims, Ls)
    h = dw.mg_setup(g, _dev(U), M5, mf, {"nvec": nvec, "block": [4, 4, 1, 1], "setup_maxiter": 10,
                                         "setup_mass": -0.19, "Ls_c": Ls_c, "coarse_block_prec": "f32"},
                    _dev(starts))
    return h, U, M5, mf


@pytest.mark.parametrize("dims,Ls,Ls_c,nrhs", [((16, 12), 8, 4, 1), ((16, 12), 8, 4, 5), ((32, 24), 6, 3, 7),
                                              ((8, 16), 4, 2, 16), ((20, 8), 5, 5, 3)])
def test_coarse_multi_matches_oracle(dw, dims, Ls, Ls_c, nrhs):
    h, U, M5, mf = _setup(dw, dims, Ls, Ls_c, 21 + nrhs)
    vecs = dw.mg_get_null_vectors(h).cpu().numpy().reshape(8, -1)
    P_o, _ = omg.build_prolongator(list(vecs), dims, (4, 4), 2, 1)
    Dhat = omg.galerkin_kernel(P_o, dirac.wilson_matrix(U, dims, -M5))
    nc = h.coarse_size
    rng = np.random.default_rng(nrhs)
    v = synth.gaussian_complex(rng, (nrhs, nc)).astype(np.complex64)
    vd = _dev(v, torch.complex64)
    out = torch.full_like(vd, float("nan"))
    for m in (mf, 1.0):
        C = omg.coarse_dwf(Dhat, Ls_c, m, 8)
        for dag in (False, True):
            dw.mg_coarse_apply_multi(h, vd, out, nrhs, m, dagger=dag)
            got = out.cpu().numpy().reshape(nrhs, nc)
            Cm = dirac.dagger(C) if dag else C
            for r in range(nrhs):
                want = Cm @ v[r].astype(np.complex128)
                assert np.linalg.norm(got[r] - want) / np.linalg.norm(want) < 1e-5, (m, dag, r)
    h.close()


def test_coarse_multi_matches_single_256(dw):
    """256x256 lattice (64x64 coarse sites, Ls_c 4), 24 right-hand sides: each column of the
    tensor-core result agrees with the one-vector FP32 stencil to FP32 accuracy."""
    h, U, M5, mf = _setup(dw, (256, 256), 16, 4, 31, sigma=0.7)
    nc, nrhs = h.coarse_size, 24
    rng = np.random.default_rng(5)
    v = synth.gaussian_complex(rng, (nrhs, nc)).astype(np.complex64)
    vd = _dev(v, torch.complex64).reshape(nrhs, nc)
    out = torch.empty_like(vd)
    one = torch.empty(nc, dtype=torch.complex64, device="cuda")
    for dag in (False, True):
        dw.mg_coarse_apply_multi(h, vd, out, nrhs, 0.005, dagger=dag)
        for r in range(nrhs):
            dw.mg_coarse_apply(h, vd[r].contiguous(), one, 0.005, dagger=dag)
            assert (torch.linalg.norm(out[r] - one) / torch.linalg.norm(one)).item() < 1e-5
    h.close()


def test_coarse_multi_rejects_bad_arguments(dw):
    h, *_ = _setup(dw, (16, 16), 4, 2, 41)
    nc = h.coarse_size
    vd = torch.zeros(2 * nc, dtype=torch.complex64, device="cuda")
    with pytest.raises(ValueError):
        dw.mg_coarse_apply_multi(h, vd, vd[:nc], 2, 0.1)
    with pytest.raises(dw.DwfError):
        dw.mg_coarse_apply_multi(h, vd, vd, 2, 0.1)
    h.close()


@pytest.mark.parametrize("nrhs,tc", [(1, 0), (6, 0), (16, 0), (32, 0), (48, 0), (64, 0), (32, 1), (48, 1), (64, 1),
                                     (48, 5), (64, 5)])
def test_coarse_multi_f16_blocks_match_single(dw, nrhs, tc):
    """FP16 coarse blocks (the default storage): each column of the tensor-core result agrees with
    the one-vector stencil reading the same FP16 blocks, to FP32 accuracy.  tc = 1 (5) selects the persistent (per-item)
    tcgen05 form from 128 columns (32 right-hand sides x 4 slices) on (48: a partial tile)."""
    rng0 = synth.rng_for(90 + nrhs)
    dims = (64, 32)
    U = synth.u1_links(synth.u1_angles(rng0, dims, 0.6))
    starts = np.stack([synth.gaussian_complex(rng0, (int(np.prod(dims)) * 2,)) for _ in range(8)])
    g = dw.make_geom(dims, 8)
    h = dw.mg_setup(g, _dev(U), 1.0, 0.01, {"setup_maxiter": 10, "setup_mass": -0.19, "Ls_c": 4, "coarse_tc": tc},
                    _dev(starts))
    nc = h.coarse_size
    v = synth.gaussian_complex(np.random.default_rng(nrhs), (nrhs, nc)).astype(np.complex64)
    vd = _dev(v, torch.complex64).reshape(nrhs, nc)
    out = torch.empty_like(vd)
    one = torch.empty(nc, dtype=torch.complex64, device="cuda")
    assert dw.mg_coarse_tc_form(h, nrhs) == 0
    for m, dag in ((0.01, False), (1.0, True), (0.01, True)):
        dw.mg_coarse_apply_multi(h, vd, out, nrhs, m, dagger=dag)
        form = dw.mg_coarse_tc_form(h, nrhs)
        assert form in ((1, 2, 4, 256, 257) if tc == 0 else (0,)) and (form < 256 or nrhs * 4 >= 128)
        for r in range(nrhs):
            dw.mg_coarse_apply(h, vd[r].contiguous(), one, m, dagger=dag)
            assert (torch.linalg.norm(out[r] - one) / torch.linalg.norm(one)).item() < 1e-5
    h.close()

"""The transfer-operator study of the paper's discussion section on the GPU: the
bulk transfer (P on every slice) against the oracle, the local colinearity
(1 - P R) v and the oblique projector (1 - P Ahat^-1 R A) v for low eigenvectors
v of A = D_PV^dag D_DW with the wall and the bulk transfers, and K-cycle solves
with the bulk transfer and with reduced and full coarse Lhat_s."""
import numpy as np
import pytest
import scipy.sparse.linalg as sla
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


def _hier(dw, dims, Ls, Ls_c, transfer, seed=77, sigma=0.3, mf=0.05):
    rng = synth.rng_for(seed)
    U = synth.u1_links(synth.u1_angles(rng, dims, sigma))
    V = int(np.prod(dims))
    starts = np.stack([synth.gaussian_complex(rng, (2 * V,)) for _ in range(8)])
    g = dw.make_geom(dims, Ls)
    h = dw.mg_setup(g, _dev(U), 1.0, mf, {"setup_maxiter": 40, "setup_mass": -0.1, "Ls_c": Ls_c,
                                         "transfer": transfer, "coarse_block_prec": "f32", "fine_prec": "f32"},
                    _dev(starts))
    v1 = dw.mg_get_null_vectors(h).cpu().numpy().reshape(8, -1)
    P, cdims = omg.build_prolongator(list(v1), dims, (4, 4), 2, 1)
    return h, U, P


def test_bulk_transfer_matches_oracle(dw):
    dims, Ls = (32, 32), 6
    h, U, P = _hier(dw, dims, Ls, Ls, 1)
    rng = np.random.default_rng(3)
    r = synth.gaussian_complex(rng, (dw.spinor_size(h.geom),)).astype(np.complex64)
    rc = torch.full((h.coarse_size,), float("nan"), dtype=torch.complex64, device="cuda")
    dw.mg_restrict(h, _dev(r, torch.complex64), rc)
    want = omg.restrict_bulk(r.astype(np.complex128), P, Ls)
    assert np.linalg.norm(rc.cpu().numpy() - want) / np.linalg.norm(want) < 1e-5
    e = synth.gaussian_complex(rng, (h.coarse_size,)).astype(np.complex64)
    ef = torch.full((len(r),), float("nan"), dtype=torch.complex64, device="cuda")
    dw.mg_prolong(h, _dev(e, torch.complex64), ef)
    want = omg.prolong_bulk(e.astype(np.complex128), P, Ls)
    assert np.linalg.norm(ef.cpu().numpy() - want) / np.linalg.norm(want) < 1e-5
    h.close()


@pytest.mark.parametrize("transfer,Ls_c", [(0, 4), (0, 8), (1, 8)])
def test_colinearity_and_oblique_projector_match_oracle(dw, transfer, Ls_c):
    """16^2 x Ls 8, the four lowest eigenvectors of A: both diagnostics against the oracle's."""
    dims, Ls, M5, mf = (16, 16), 8, 1.0, 0.05
    h, U, P = _hier(dw, dims, Ls, Ls_c, transfer)
    A = dirac.pvdag_dwf_matrix(U, dims, Ls, M5, mf)
    lam, vecs = sla.eigs(A.tocsc(), k=4, sigma=0.0)
    Dhat = omg.galerkin_kernel(P, dirac.wilson_matrix(U, dims, -M5))
    Ac = (dirac.dagger(omg.coarse_dwf(Dhat, Ls_c, 1.0, 8)) @ omg.coarse_dwf(Dhat, Ls_c, mf, 8)).tocsr()
    if transfer == 1:
        R = lambda x: omg.restrict_bulk(x, P, Ls)
        Pr = lambda x: omg.prolong_bulk(x, P, Ls)
    else:
        R = lambda x: omg.restrict(x, P, Ls, Ls_c, 2, 1, 8)
        Pr = lambda x: omg.prolong(x, P, Ls, Ls_c, 2, 1, 8)
    for k in range(4):
        v = (vecs[:, k] / np.linalg.norm(vecs[:, k])).astype(np.complex64)
        vd = _dev(v, torch.complex64)
        col = dw.mg_transfer_colinearity(h, vd).cpu().numpy()
        want = omg.colinearity(v.astype(np.complex128), R, Pr)
        assert abs(np.linalg.norm(col) - want) < 1e-5 * max(1.0, want)
        obl, it = dw.mg_transfer_oblique(h, vd, tol=1e-7)
        want = omg.oblique(v.astype(np.complex128), A, Ac, R, Pr)
        assert abs(np.linalg.norm(obl.cpu().numpy()) - want) < 1e-3 * max(1.0, want), (k, want)
        assert it > 0
    h.close()


@pytest.mark.parametrize("transfer,Ls_c", [(0, 4), (0, 16), (1, 16)])
def test_kcycle_with_transfer_variants_reaches_tolerance(dw, transfer, Ls_c):
    """The K-cycle with the wall transfer at reduced and full Lhat_s and with the bulk transfer solves
    64^2 x Ls 16 to a true residual of 1e-10 (recomputed by the oracle)."""
    dims, Ls, M5, mf = (64, 64), 16, 1.0, 0.02
    rng = synth.rng_for(88)
    U = synth.u1_links(synth.u1_angles(rng, dims, 0.3))
    V = int(np.prod(dims))
    starts = np.stack([synth.gaussian_complex(rng, (2 * V,)) for _ in range(8)])
    b = synth.gaussian_spinor(rng, dims, Ls).reshape(-1)
    g = dw.make_geom(dims, Ls)
    h = dw.mg_setup(g, _dev(U), M5, mf, {"setup_mass": -0.1, "Ls_c": Ls_c, "transfer": transfer}, _dev(starts))
    x = torch.empty(len(b), dtype=torch.complex128, device="cuda")
    st, _ = dw.mg_solve(h, _dev(b), x, tol=1e-10)
    D = dirac.dwf_matrix(U, dims, Ls, M5, mf)
    assert np.linalg.norm(b - D @ x.cpu().numpy()) / np.linalg.norm(b) <= 1e-10, st
    h.close()


def test_bulk_transfer_needs_full_coarse_Ls(dw):
    g = dw.make_geom((16, 16), 8)
    U = torch.ones(dw.link_size(g), dtype=torch.complex128, device="cuda")
    starts = torch.randn(8 * 512, dtype=torch.complex128, device="cuda")
    with pytest.raises(dw.DwfError):
        dw.mg_setup(g, U, 1.0, 0.05, {"Ls_c": 4, "transfer": 1, "setup_maxiter": 2}, starts)

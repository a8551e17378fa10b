"""BiCGStab(l) on D_PV^dag D_DW (bicgstab_solve) against the FP64 oracle: the
solution is the unique x = D_DW^-1 b, so it must match the oracle's dense solve
within the condition number times the residual bound, and its true residual,
recomputed by the oracle, must be <= 1e-10."""
import numpy as np
import pytest
import torch

import synth
from oracle import dirac

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


@pytest.mark.parametrize("ell,prec", [(6, "f32_l16"), (6, "f64"), (2, "f32"), (1, "f32_lbf16"), (8, "f32_l16")])
def test_bicgstab_matches_dense_solution(dw, ell, prec):
    dims, Ls, M5, mf = (16, 12), 8, 1.0, 0.02
    rng = synth.rng_for(300 + ell)
    U = synth.u1_links(synth.u1_angles(rng, dims, 0.5))
    b = synth.gaussian_spinor(rng, dims, Ls).reshape(-1)
    g = dw.make_geom(dims, Ls)
    x = torch.full((len(b),), float("nan"), dtype=torch.complex128, device="cuda")
    st, _ = dw.bicgstab_solve(g, _dev(U), _dev(b), x, M5, mf, ell=ell, tol=1e-10, inner_prec=prec)
    xs = x.cpu().numpy()
    D = dirac.dwf_matrix(U, dims, Ls, M5, mf)
    res = np.linalg.norm(b - D @ xs) / np.linalg.norm(b)
    assert res <= 1e-10 and abs(res - st["true_residual"]) <= 1e-3 * res + 1e-16
    Dd = D.toarray()
    xd = np.linalg.solve(Dd, b)
    cond = np.linalg.cond(Dd)
    assert np.linalg.norm(xs - xd) / np.linalg.norm(xd) <= 1e-10 * cond
    assert st["iterations"] % ell == 0 and st["fine_applies"] >= 4 * st["iterations"]


def test_bicgstab_256_reaches_tolerance(dw):
    """The 256^2 x 16 workload (sigma 0.7, m 0.005): BiCGStab-6 with FP32 / FP16-link inner solves
    reaches a true residual of 1e-10, recomputed by the oracle."""
    wl = synth.SCHWINGER_256
    U, (b,) = wl.draw(1)
    b = b.reshape(-1)
    g = dw.make_geom(wl.dims, wl.Ls)
    x = torch.empty(len(b), dtype=torch.complex128, device="cuda")
    st, _ = dw.bicgstab_solve(g, _dev(U.reshape(-1)), _dev(b), x, wl.M5, wl.mf, ell=6, tol=1e-10)
    D = dirac.dwf_matrix(U, wl.dims, wl.Ls, wl.M5, wl.mf)
    res = np.linalg.norm(b - D @ x.cpu().numpy()) / np.linalg.norm(b)
    assert res <= 1e-10, (res, st)


def test_bicgstab_rejects_bad_arguments(dw):
    g = dw.make_geom((8, 8), 4)
    n = dw.spinor_size(g)
    U = torch.ones(dw.link_size(g), dtype=torch.complex128, device="cuda")
    b = torch.ones(n, dtype=torch.complex128, device="cuda")
    x = torch.empty_like(b)
    for ell in (0, 9):
        with pytest.raises(dw.DwfError) as e:
            dw.bicgstab_solve(g, U, b, x, 1.0, 0.1, ell=ell)
        assert e.value.status == 1
    with pytest.raises(dw.DwfError):
        dw.bicgstab_solve(g, U, b, x, 1.0, 0.1, tol=0.0)

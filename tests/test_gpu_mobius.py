"""GPU parity of the Mobius domain wall operator (dwf_mobius_apply) and of the
polynomially corrected Pauli-Villars operator (dwf_pv_poly_apply) with the FP64
oracle's assembled matrices: FP64 at 1e-12, FP32 spinors with FP32 / FP16 links
at 1e-5, 2-d U(1) and 4-d SU(3), both daggers."""
import numpy as np
import pytest
import torch

import synth
from oracle import dirac

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "f32_l16": 1e-5}


@pytest.fixture(scope="module")
def dw():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2004_07732_gb300 as pkg
    pkg.lib()
    return pkg


def _dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to("cuda").to(dtype)


def _case(group, seed):
    rng = synth.rng_for(seed)
    if group == "u1":
        dims, Ls, M5 = (12, 10), 6, 1.0
        U = synth.u1_links(synth.u1_angles(rng, dims, 0.6))
    else:
        dims, Ls, M5 = (4, 4, 4, 6), 4, 1.8
        U = synth.su3_links(rng, dims, 0.3)
    psi = synth.gaussian_spinor(rng, dims, Ls, group).reshape(-1)
    return dims, Ls, M5, U, psi


@pytest.mark.parametrize("group", ["u1", "su3"])
@pytest.mark.parametrize("prec", ["f64", "f32", "f32_l16"])
@pytest.mark.parametrize("b5,c5", [(1.5, 0.5), (2.0, 1.0), (1.0, 0.0)])
def test_mobius_apply_matches_oracle(dw, group, prec, b5, c5):
    dims, Ls, M5, U, psi = _case(group, 500)
    mf = 0.03
    g = dw.make_geom(dims, Ls, group=group)
    Ud = dw.links_to(g, _dev(U), prec)
    dt = dw.spinor_dtype(prec)
    pd = _dev(psi, dt)
    out = torch.full_like(pd, float("nan"))
    # the links and the source as the GPU holds them (round to nearest even)
    if prec == "f32":
        Uo = U.astype(np.complex64).astype(np.complex128)
    elif prec == "f32_l16":
        Uo = U.real.astype(np.float16).astype(np.float64) + 1j * U.imag.astype(np.float16).astype(np.float64)
    else:
        Uo = U
    ps = psi if prec == "f64" else psi.astype(np.complex64).astype(np.complex128)
    D = dirac.mobius_matrix(Uo, dims, Ls, M5, mf, b5, c5, group)
    for dag in (False, True):
        dw.dwf_mobius_apply(g, Ud, pd, out, M5, mf, b5, c5, dagger=dag, prec=prec)
        want = (dirac.dagger(D) if dag else D) @ ps
        got = out.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < TOL[prec], (dag, group, prec)


@pytest.mark.parametrize("group", ["u1", "su3"])
@pytest.mark.parametrize("coeffs,b5,c5", [((1.0,), 1.0, 0.0), ((2.0, -1.0), 1.0, 0.0), ((3.0, -3.0, 1.0), 1.0, 0.0),
                                          ((2.0, -1.0), 1.5, 0.5)])
def test_pv_poly_apply_matches_oracle(dw, group, coeffs, b5, c5):
    dims, Ls, M5, U, psi = _case(group, 501)
    mf = 0.05
    g = dw.make_geom(dims, Ls, group=group)
    Ud = _dev(U)
    pd = _dev(psi)
    out = torch.full_like(pd, float("nan"))
    dw.dwf_pv_poly_apply(g, Ud, pd, out, M5, mf, coeffs, b5=b5, c5=c5, prec="f64")
    Ddw = dirac.mobius_matrix(U, dims, Ls, M5, mf, b5, c5, group)
    Dpv = dirac.mobius_matrix(U, dims, Ls, M5, 1.0, b5, c5, group)
    want = dirac.pv_poly_apply(Ddw, Dpv, coeffs, psi)
    got = out.cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-12
    if coeffs == (1.0,) and (b5, c5) == (1.0, 0.0):
        ref = torch.empty_like(pd)
        dw.dwf_pvdag_apply(g, Ud, pd, torch.empty_like(pd), ref, M5, mf)
        assert torch.equal(ref, out)


def test_mobius_rejects_bad_arguments(dw):
    g = dw.make_geom((8, 8), 4)
    n = dw.spinor_size(g)
    U = torch.ones(dw.link_size(g), dtype=torch.complex128, device="cuda")
    psi = torch.ones(n, dtype=torch.complex128, device="cuda")
    with pytest.raises(dw.DwfError):
        dw.dwf_mobius_apply(g, U, psi, torch.empty_like(psi), 1.0, 0.1, 1.5, 0.5, tmp=psi)
    with pytest.raises(dw.DwfError):
        dw.dwf_pv_poly_apply(g, U, psi, torch.empty_like(psi), 1.0, 0.1, [])

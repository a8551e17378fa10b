"""The allocation-free preconditioned apply agrees with the allocating one.

dwf_pvdag_apply_noalloc serves callers that cannot allocate device memory (a
host code whose own allocator holds nearly all of HBM, or a latency-critical
loop that cannot take cudaMalloc's implicit synchronisation): it keeps the
intermediate D_DW psi in a fixed 16 MiB array inside the library.  This file is
collected last so that a failure here comes after every other test has run.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "f32_l16": 1e-5, "f32_lbf16": 1e-5}


@pytest.fixture(scope="module")
def dw():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2004_07732_gb300 as pkg
    pkg.lib()
    return pkg


@pytest.mark.parametrize("prec", ["f64", "f32_l16"])
def test_noalloc_matches_allocating_apply_twice(dw, prec):
    """Two calls in a row through the C ABI, each against dwf_pvdag_apply on the same input."""
    dims, Ls, M5, mf = (64, 48), 8, 1.0, 0.01
    rng = synth.rng_for(31)
    U = synth.u1_links(synth.u1_angles(rng, dims, 0.7))
    g = dw.make_geom(dims, Ls)
    Ud = dw.links_to(g, torch.from_numpy(U.reshape(-1)).cuda(), prec)
    dt = dw.spinor_dtype(prec)
    for call in range(2):
        psi = torch.from_numpy(synth.gaussian_spinor(rng, dims, Ls).reshape(-1)).cuda().to(dt)
        ref, tmp, out = torch.empty_like(psi), torch.empty_like(psi), torch.full_like(psi, float("nan"))
        dw.dwf_pvdag_apply(g, Ud, psi, tmp, ref, M5, mf, prec=prec)
        dw.dwf_pvdag_apply_noalloc(g, Ud, psi, out, M5, mf, prec=prec)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy().astype(np.complex128), ref.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < TOL[prec], f"call {call}"


@pytest.mark.parametrize("prec", ["f64", "f32_l16"])
def test_noalloc_4d_su3_matches_allocating_apply_twice(dw, prec):
    """4-d SU(3) (12 complex values per site), two calls in a row against dwf_pvdag_apply."""
    dims, Ls, M5, mf = (4, 4, 4, 8), 8, 1.8, 0.01
    rng = synth.rng_for(32)
    U = synth.su3_links(rng, dims, 0.3)
    g = dw.make_geom(dims, Ls, group="su3")
    Ud = dw.links_to(g, torch.from_numpy(U.reshape(-1)).cuda(), prec)
    dt = dw.spinor_dtype(prec)
    for call in range(2):
        psi = torch.from_numpy(synth.gaussian_spinor(rng, dims, Ls, "su3").reshape(-1)).cuda().to(dt)
        ref, tmp, out = torch.empty_like(psi), torch.empty_like(psi), torch.full_like(psi, float("nan"))
        dw.dwf_pvdag_apply(g, Ud, psi, tmp, ref, M5, mf, prec=prec)
        dw.dwf_pvdag_apply_noalloc(g, Ud, psi, out, M5, mf, prec=prec)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy().astype(np.complex128), ref.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < TOL[prec], f"call {call}"


def test_noalloc_4d_limit_depends_on_precision(dw):
    """8^3 x 16 x Ls 16 SU(3): 1.57M complex values per spinor -- 25 MB in FP64 (over the 16 MiB
    scratch: rejected), 12.6 MB in FP32 (accepted, and equal to the allocating apply)."""
    dims, Ls, M5, mf = (8, 8, 8, 16), 16, 1.8, 0.01
    g = dw.make_geom(dims, Ls, group="su3")
    n = dw.spinor_size(g)
    U64 = torch.from_numpy(synth.su3_links(synth.rng_for(33), dims, 0.3).reshape(-1)).cuda()
    psi = torch.empty(n, dtype=torch.complex128, device="cuda")
    with pytest.raises(dw.DwfError) as e:
        dw.dwf_pvdag_apply_noalloc(g, U64, psi, torch.empty_like(psi), M5, mf, prec="f64")
    assert e.value.status == 1 and "scratch" in str(e.value)
    Ul = dw.links_to(g, U64, "f32_l16")
    p32 = torch.from_numpy(synth.gaussian_spinor(synth.rng_for(34), dims, Ls, "su3").reshape(-1)).cuda().to(
        torch.complex64)
    ref, tmp, out = torch.empty_like(p32), torch.empty_like(p32), torch.full_like(p32, float("nan"))
    dw.dwf_pvdag_apply(g, Ul, p32, tmp, ref, M5, mf, prec="f32_l16")
    dw.dwf_pvdag_apply_noalloc(g, Ul, p32, out, M5, mf, prec="f32_l16")
    torch.cuda.synchronize()
    assert (torch.linalg.norm(out - ref) / torch.linalg.norm(ref)).item() < 1e-5


def test_noalloc_rejects_lattices_beyond_its_scratch(dw):
    g = dw.make_geom((512, 512), 16)        # 8.4M complex values: 134 MB in FP64
    psi = torch.empty(dw.spinor_size(g), dtype=torch.complex128, device="cuda")
    out = torch.empty_like(psi)
    U = torch.ones(dw.link_size(g), dtype=torch.complex128, device="cuda")
    with pytest.raises(dw.DwfError) as e:
        dw.dwf_pvdag_apply_noalloc(g, U, psi, out, 1.0, 0.01)
    assert e.value.status == 1 and "scratch" in str(e.value)

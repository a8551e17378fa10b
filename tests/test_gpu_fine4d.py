"""GPU parity of the 4-d SU(3) domain-wall operator against the FP64 oracle."""
import numpy as np
import pytest
import torch

import synth
from oracle import dirac

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "f32_l16": 1e-5, "f32_lbf16": 1e-5}


@pytest.fixture(scope="module")
def dw():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2004_07732_gb300 as pkg
    pkg.lib()
    return pkg


def _dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to("cuda").to(dtype)


def _rounded(U, prec):
    if prec == "f64":
        return U
    if prec == "f32":
        return U.astype(np.complex64).astype(np.complex128)
    if prec == "f32_l16":
        return U.real.astype(np.float16).astype(np.float64) + 1j * U.imag.astype(np.float16).astype(np.float64)
    t = torch.from_numpy(np.stack([U.real, U.imag], -1)).to(torch.bfloat16).to(torch.float64).numpy()
    return t[..., 0] + 1j * t[..., 1]


@pytest.mark.parametrize("dims,Ls,anti", [((4, 4, 4, 4), 4, None), ((3, 5, 2, 3), 3, [0, 0, 0, 1]),
                                          ((2, 2, 2, 2), 2, [1, 1, 1, 1]), ((6, 4, 4, 8), 5, None)])
@pytest.mark.parametrize("prec", ["f64", "f32", "f32_l16", "f32_lbf16"])
@pytest.mark.parametrize("dagger", [False, True])
def test_dwf4d_apply_parity(dw, dims, Ls, anti, prec, dagger):
    M5, mf = 1.8, 0.01
    rng = synth.rng_for(hash((dims, Ls)) % 997)
    U = synth.su3_links(rng, dims, 0.3)
    psi = synth.gaussian_spinor(rng, dims, Ls, "su3")
    g = dw.make_geom(dims, Ls, group="su3", antiperiodic=anti)
    Ud = dw.links_to(g, _dev(U), prec)
    pd = _dev(psi, dw.spinor_dtype(prec))
    out = torch.empty_like(pd)
    dw.dwf_apply(g, Ud, pd, out, M5, mf, dagger=dagger, prec=prec)
    Uo = _rounded(U, prec)
    ps = psi if prec == "f64" else psi.astype(np.complex64).astype(np.complex128)
    want = dirac.dwf_apply(Uo, ps, dims, Ls, M5, mf, dagger_=dagger, group="su3", antiperiodic=anti).reshape(-1)
    got = out.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < TOL[prec]


def test_dwf4d_full_size_sampled(dw):
    """16^3 x 32 x Ls=16 SU(3), FP32 spinors + FP16 links, spot-checked point by point."""
    wl = synth.SU3_16x32
    U, srcs = wl.draw(1)
    psi = srcs[0]
    g = dw.make_geom(wl.dims, wl.Ls, group="su3")
    Ud = dw.links_to(g, _dev(U), "f32_l16")
    pd = _dev(psi, torch.complex64)
    out = torch.empty_like(pd)
    dw.dwf_apply(g, Ud, pd, out, wl.M5, wl.mf, prec="f32_l16")
    got = out.cpu().numpy().reshape(wl.Ls, wl.V, 4, 3)
    rng = np.random.default_rng(1)
    pts = [(int(rng.integers(0, wl.Ls)), int(rng.integers(0, wl.V))) for _ in range(120)]
    pts += [(0, 0), (wl.Ls - 1, wl.V - 1), (0, wl.V - 1), (wl.Ls - 1, 0)]
    Uo = _rounded(U, "f32_l16")
    ps = psi.astype(np.complex64).astype(np.complex128)
    want = dirac.dwf_apply_points(Uo, ps, wl.dims, wl.Ls, wl.M5, wl.mf, pts, group="su3")
    g_pts = np.array([got[s, x] for s, x in pts])
    assert np.abs(g_pts - want).max() < 1e-5 * np.abs(want).max()


def test_dwf4d_adjoint_and_cgne(dw):
    dims, Ls, M5, mf = (4, 4, 4, 4), 4, 1.8, 0.05
    rng = synth.rng_for(11)
    U = synth.su3_links(rng, dims, 0.3)
    b = synth.gaussian_spinor(rng, dims, Ls, "su3").reshape(-1)
    y = synth.gaussian_spinor(rng, dims, Ls, "su3").reshape(-1)
    g = dw.make_geom(dims, Ls, group="su3")
    Ud, bd, yd = _dev(U), _dev(b), _dev(y)
    Dy, Ddb = torch.empty_like(yd), torch.empty_like(bd)
    dw.dwf_apply(g, Ud, yd, Dy, M5, mf)
    dw.dwf_apply(g, Ud, bd, Ddb, M5, mf, dagger=True)
    a1, a2 = dw.dwf_dot(bd, Dy), dw.dwf_dot(Ddb, yd)
    assert abs(a1 - a2) < 1e-12 * abs(a1)
    x = torch.empty_like(bd)
    st, status = dw.cgne_solve(g, Ud, bd, x, M5, mf, tol=1e-10)
    D = dirac.dwf_matrix(U, dims, Ls, M5, mf, group="su3")
    res = np.linalg.norm(b - D @ x.cpu().numpy()) / np.linalg.norm(b)
    assert status == 0 and res <= 1e-10


def _packed_positions(dims, Ls):
    """Float offsets in the slice-paired packed layout of the real and imaginary parts of every
    (s, site, k) in canonical order: float4 ((s/2 NB + site/32) 12 + k) 32 + site%32 holds
    (Re slice 2j, Im slice 2j, Re slice 2j+1, Im slice 2j+1)."""
    V = int(np.prod(dims))
    NB = (V + 31) // 32
    s, site, k = np.meshgrid(np.arange(Ls), np.arange(V), np.arange(12), indexing="ij")
    f4 = (((s // 2) * NB + site // 32) * 12 + k) * 32 + site % 32
    return 4 * f4 + 2 * (s % 2), 4 * f4 + 2 * (s % 2) + 1, NB


@pytest.mark.parametrize("dims,Ls", [((4, 4, 4, 4), 4), ((3, 5, 2, 3), 2), ((2, 2, 2, 2), 2), ((3, 5, 2, 3), 6)])
def test_pack_unpack_layout(dw, dims, Ls):
    """Packing places (s, site, k) as above; padding sites are zero; unpacking inverts it."""
    rng = synth.rng_for(7)
    psi = synth.gaussian_spinor(rng, dims, Ls, "su3")
    g = dw.make_geom(dims, Ls, group="su3")
    pd = _dev(psi, torch.complex64)
    pk = dw.pack_spinor(g, pd)
    pre, pim, NB = _packed_positions(dims, Ls)
    assert pk.numel() == Ls * NB * 32 * 12
    fl = pk.cpu().numpy().view(np.float32)
    canon = pd.cpu().numpy().reshape(-1)
    assert np.array_equal(fl[pre.reshape(-1)], canon.real)
    assert np.array_equal(fl[pim.reshape(-1)], canon.imag)
    pad = np.ones(fl.shape[0], bool)
    pad[pre.reshape(-1)] = False
    pad[pim.reshape(-1)] = False
    assert not fl[pad].any()                         # padding sites are zero
    back = dw.unpack_spinor(g, pk)
    assert torch.equal(back, pd)


def test_packed_layout_needs_even_Ls(dw):
    """Odd Ls has no slice-paired layout: size 0, and the C entry points return DWF_ERR_UNSUPPORTED."""
    import ctypes
    g = dw.make_geom((4, 4, 4, 4), 3, group="su3")
    assert dw.packed_spinor_size(g) == 0
    pd = torch.zeros(dw.spinor_size(g), dtype=torch.complex64, device="cuda")
    out = torch.zeros(dw.spinor_size(g) * 2, dtype=torch.complex64, device="cuda")
    st = dw.lib().dwf_pack_spinor(ctypes.byref(g), ctypes.c_void_p(pd.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), None)
    assert st == 6                                   # DWF_ERR_UNSUPPORTED
    with pytest.raises(ValueError):
        dw.pack_spinor(g, pd, out=out)


def test_pack_links_layout(dw):
    dims = (3, 5, 2, 3)
    V = int(np.prod(dims))
    NB = (V + 31) // 32
    rng = synth.rng_for(8)
    U = synth.su3_links(rng, dims, 0.3).reshape(4, V, 9)
    g = dw.make_geom(dims, 2, group="su3")
    Up = dw.pack_links(g, _dev(U), "f32").cpu().numpy().reshape(4, NB, 9, 32)
    want = np.zeros((4, NB * 32, 9), np.complex64)
    want[:, :V] = U.astype(np.complex64)
    assert np.array_equal(Up, want.reshape(4, NB, 32, 9).transpose(0, 1, 3, 2))


@pytest.mark.parametrize("dims,Ls,anti", [((4, 4, 4, 4), 4, None), ((3, 5, 2, 3), 6, [0, 0, 0, 1]),
                                          ((2, 2, 2, 2), 2, [1, 1, 1, 1]), ((6, 4, 4, 8), 8, None)])
@pytest.mark.parametrize("prec", ["f32", "f32_l16", "f32_lbf16"])
@pytest.mark.parametrize("dagger", [False, True])
def test_dwf4d_packed_apply_parity(dw, dims, Ls, anti, prec, dagger):
    M5, mf = 1.8, 0.01
    rng = synth.rng_for(hash((dims, Ls, 3)) % 997)
    U = synth.su3_links(rng, dims, 0.3)
    psi = synth.gaussian_spinor(rng, dims, Ls, "su3")
    g = dw.make_geom(dims, Ls, group="su3", antiperiodic=anti)
    Up = dw.pack_links(g, _dev(U), prec)
    pk = dw.pack_spinor(g, _dev(psi, torch.complex64))
    outp = torch.empty_like(pk)
    dw.dwf_apply_packed(g, Up, pk, outp, M5, mf, dagger=dagger, prec=prec)
    got = dw.unpack_spinor(g, outp).cpu().numpy().astype(np.complex128)
    ps = psi.astype(np.complex64).astype(np.complex128)
    want = dirac.dwf_apply(_rounded(U, prec), ps, dims, Ls, M5, mf, dagger_=dagger, group="su3",
                           antiperiodic=anti).reshape(-1)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < TOL[prec]


def test_dwf4d_packed_full_size_sampled(dw):
    """The bench workload (16^3 x 32 x 16, FP16 links) in the packed layout, checked point by point."""
    wl = synth.SU3_16x32
    U, srcs = wl.draw(1)
    psi = srcs[0]
    g = dw.make_geom(wl.dims, wl.Ls, group="su3")
    Up = dw.pack_links(g, _dev(U), "f32_l16")
    pk = dw.pack_spinor(g, _dev(psi, torch.complex64))
    outp = torch.empty_like(pk)
    dw.dwf_apply_packed(g, Up, pk, outp, wl.M5, wl.mf, prec="f32_l16")
    got = dw.unpack_spinor(g, outp).cpu().numpy().reshape(wl.Ls, wl.V, 4, 3)
    rng = np.random.default_rng(2)
    pts = [(int(rng.integers(0, wl.Ls)), int(rng.integers(0, wl.V))) for _ in range(120)]
    pts += [(0, 0), (wl.Ls - 1, wl.V - 1), (0, wl.V - 1), (wl.Ls - 1, 0)]
    want = dirac.dwf_apply_points(_rounded(U, "f32_l16"), psi.astype(np.complex64).astype(np.complex128),
                                  wl.dims, wl.Ls, wl.M5, wl.mf, pts, group="su3")
    g_pts = np.array([got[s, x] for s, x in pts])
    assert np.abs(g_pts - want).max() < 1e-5 * np.abs(want).max()

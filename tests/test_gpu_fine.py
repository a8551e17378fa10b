"""GPU parity of the fine operators, reductions and FP64 CGNR against the FP64 CPU oracle.

Tolerances (relative L2 against the oracle on the same seeded inputs):
FP64 applies 1e-12; FP32 applies 1e-5 (against the oracle fed the same
rounded links for FP16/BF16 storage); solves reach a true FP64 residual 1e-10.
"""
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


def _rounded_links(U, prec):
    """The links as the GPU stores them, rounded on the CPU (round to nearest even)."""
    if prec in ("f64",):
        return U
    if prec == "f32":
        return U.astype(np.complex64).astype(np.complex128)
    if prec == "f32_l16":
        return U.real.astype(np.float16).astype(np.float64) + 1j * U.imag.astype(np.float16).astype(np.float64)
    t = torch.from_numpy(np.stack([U.real, U.imag], -1)).to(torch.bfloat16).to(torch.float64).numpy()
    return t[..., 0] + 1j * t[..., 1]


def _case(dims, Ls, sigma, seed):
    rng = synth.rng_for(seed)
    U = synth.u1_links(synth.u1_angles(rng, dims, sigma))
    psi = synth.gaussian_spinor(rng, dims, Ls)
    return U, psi


def _dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to("cuda").to(dtype)


SHAPES = [((8, 6), 4, None), ((32, 32), 8, None), ((37, 13), 5, None), ((16, 24), 6, [0, 1]),
          ((1, 5), 3, None), ((6, 1), 2, [1, 0]), ((5, 7), 1, None), ((300, 20), 3, None)]


@pytest.mark.parametrize("dims,Ls,anti", SHAPES)
@pytest.mark.parametrize("prec", ["f64", "f32", "f32_l16", "f32_lbf16"])
@pytest.mark.parametrize("dagger", [False, True])
def test_dwf_apply_parity(dw, dims, Ls, anti, prec, dagger):
    M5, mf = 1.0, 0.05
    U, psi = _case(dims, Ls, 0.5, hash((dims, Ls)) % 1000)
    g = dw.make_geom(dims, Ls, antiperiodic=anti)
    Ud = dw.links_to(g, _dev(U), prec)
    pd = _dev(psi, dw.spinor_dtype(prec))
    out = torch.empty_like(pd)
    dw.dwf_apply(g, Ud, pd, out, M5, mf, dagger=dagger, prec=prec)
    Uo = _rounded_links(U, prec)
    ps = psi if prec == "f64" else psi.astype(np.complex64).astype(np.complex128)
    want = dirac.dwf_apply(Uo, ps, dims, Ls, M5, mf, dagger_=dagger, antiperiodic=anti).reshape(-1)
    got = out.cpu().numpy().astype(np.complex128)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err < TOL[prec], err


@pytest.mark.parametrize("prec", ["f64", "f32_l16"])
def test_pv_and_preconditioned_operator(dw, prec):
    dims, Ls, M5, mf = (24, 16), 6, 1.0, 0.01
    U, psi = _case(dims, Ls, 0.7, 3)
    g = dw.make_geom(dims, Ls)
    Ud = dw.links_to(g, _dev(U), prec)
    pd = _dev(psi, dw.spinor_dtype(prec))
    out, tmp = torch.empty_like(pd), torch.empty_like(pd)
    Uo = _rounded_links(U, prec)
    ps = psi.reshape(-1) if prec == "f64" else psi.reshape(-1).astype(np.complex64).astype(np.complex128)
    for dag in (False, True):
        dw.pv_apply(g, Ud, pd, out, M5, dagger=dag, prec=prec)
        Dp = dirac.pv_matrix(Uo, dims, Ls, M5)
        want = (dirac.dagger(Dp) if dag else Dp) @ ps
        assert np.linalg.norm(out.cpu().numpy() - want) / np.linalg.norm(want) < TOL[prec]
    dw.dwf_pvdag_apply(g, Ud, pd, tmp, out, M5, mf, prec=prec)
    want = dirac.pvdag_dwf_matrix(Uo, dims, Ls, M5, mf) @ ps
    assert np.linalg.norm(out.cpu().numpy() - want) / np.linalg.norm(want) < TOL[prec]


def test_adjoint_identity_on_gpu(dw):
    """<x, D y> = <D^dag x, y> with both sides computed by the GPU kernels and reduction."""
    dims, Ls = (64, 32), 8
    rng = synth.rng_for(5)
    U = synth.u1_links(synth.u1_angles(rng, dims, 0.7))
    x = synth.gaussian_spinor(rng, dims, Ls)
    y = synth.gaussian_spinor(rng, dims, Ls)
    g = dw.make_geom(dims, Ls)
    Ud, xd, yd = _dev(U), _dev(x), _dev(y)
    Dy, Ddx = torch.empty_like(yd), torch.empty_like(xd)
    dw.dwf_apply(g, Ud, yd, Dy, 1.0, 0.02)
    dw.dwf_apply(g, Ud, xd, Ddx, 1.0, 0.02, dagger=True)
    a = dw.dwf_dot(xd, Dy)
    b = dw.dwf_dot(Ddx, yd)
    assert abs(a - b) < 1e-12 * abs(a)


@pytest.mark.parametrize("n", [1, 7, 255, 256, 257, 100003, 3_000_001])
@pytest.mark.parametrize("f64", [True, False])
def test_dot_reduction(dw, n, f64):
    rng = np.random.default_rng(n)
    x = synth.gaussian_complex(rng, (n,))
    y = synth.gaussian_complex(rng, (n,))
    if not f64:
        x = x.astype(np.complex64).astype(np.complex128)
        y = y.astype(np.complex64).astype(np.complex128)
    dt = torch.complex128 if f64 else torch.complex64
    got = dw.dwf_dot(_dev(x, dt), _dev(y, dt))
    want = np.vdot(x, y)
    assert abs(got - want) <= 1e-13 * np.sqrt(n) * np.linalg.norm(x) * np.linalg.norm(y)
    again = dw.dwf_dot(_dev(x, dt), _dev(y, dt))
    assert got == again     # fixed summation order: bitwise reproducible


def test_full_size_apply_sampled(dw):
    """256x256 x Ls=16 FP32/FP16-link apply, spot-checked point by point against the definition."""
    wl = synth.SCHWINGER_256
    U, srcs = wl.draw(1)
    psi = srcs[0]
    g = dw.make_geom(wl.dims, wl.Ls)
    Ud = dw.links_to(g, _dev(U), "f32_l16")
    pd = _dev(psi, torch.complex64)
    out = torch.empty_like(pd)
    dw.dwf_apply(g, Ud, pd, out, wl.M5, wl.mf, prec="f32_l16")
    got = out.cpu().numpy().reshape(wl.Ls, wl.V, 2)
    rng = np.random.default_rng(0)
    pts = [(int(rng.integers(0, wl.Ls)), int(rng.integers(0, wl.V))) for _ in range(200)]
    pts += [(0, 0), (wl.Ls - 1, wl.V - 1), (0, wl.V - 1), (wl.Ls - 1, 255)]
    Uo = _rounded_links(U, "f32_l16")
    ps = psi.astype(np.complex64).astype(np.complex128)
    want = dirac.dwf_apply_points_2d(Uo, ps, wl.dims, wl.Ls, wl.M5, wl.mf, pts)
    g_pts = np.array([got[s, site] for s, site in pts])
    assert np.abs(g_pts - want).max() < 1e-5 * np.abs(want).max()


@pytest.mark.parametrize("dims,Ls,anti,prec,dagger,nchunks", [((32, 32), 8, None, "f32_l16", False, 0),
                                                              ((37, 13), 5, [1, 0], "f32", True, 2),
                                                              ((16, 24), 6, None, "f64", False, 6),
                                                              ((16, 16), 7, [0, 1], "f32_lbf16", True, 3),
                                                              ((8, 8), 1, None, "f32_l16", False, 4),
                                                              ((64, 32), 16, None, "f32_l16", True, 1)])
def test_apply_host_pipelined(dw, dims, Ls, anti, prec, dagger, nchunks):
    """Host-spinor apply pipelined over s-chunks equals the device apply bit for bit (same kernel,
    same arithmetic per slice), for chunk counts from 1 to Ls and ragged splits."""
    M5, mf = 1.0, 0.05
    U, psi = _case(dims, Ls, 0.5, 40 + Ls)
    g = dw.make_geom(dims, Ls, antiperiodic=anti)
    Ud = dw.links_to(g, _dev(U), prec)
    pd = _dev(psi, dw.spinor_dtype(prec))
    want = torch.empty_like(pd)
    dw.dwf_apply(g, Ud, pd, want, M5, mf, dagger=dagger, prec=prec)
    psi_h = pd.cpu().pin_memory()
    out_h = torch.empty_like(psi_h).pin_memory()
    U_h = Ud.cpu().pin_memory()
    U_dev, psi_dev, out_dev = torch.empty_like(Ud), torch.empty_like(pd), torch.empty_like(pd)
    for _ in range(2):
        out_h.zero_()
        dw.dwf_apply_host(g, U_h, psi_h, out_h, U_dev, psi_dev, out_dev, M5, mf, dagger=dagger, prec=prec,
                          nchunks=nchunks)
        torch.cuda.synchronize()
        assert torch.equal(out_h, want.cpu())


def test_bench_size_apply_sampled(dw):
    """The bench's workload (1024x1024 x Ls=16, FP32 spinors, FP16 links), both the device apply
    and the host-spinor apply with 16 s-chunks as the bench calls them: point checks against the
    definition, and the two paths bit for bit."""
    wl = synth.SCHWINGER_1024
    U, srcs = wl.draw(1)
    psi = srcs[0]
    g = dw.make_geom(wl.dims, wl.Ls)
    Ud = dw.links_to(g, _dev(U), "f32_l16")
    pd = _dev(psi, torch.complex64)
    out = torch.empty_like(pd)
    dw.dwf_apply(g, Ud, pd, out, wl.M5, wl.mf, prec="f32_l16")
    psi_h = pd.cpu().pin_memory()
    out_h = torch.empty_like(psi_h).pin_memory()
    dw.dwf_apply_host(g, Ud.cpu().pin_memory(), psi_h, out_h, torch.empty_like(Ud), torch.empty_like(pd),
                      torch.empty_like(pd), wl.M5, wl.mf, prec="f32_l16", nchunks=16)
    torch.cuda.synchronize()
    got = out.cpu()
    assert torch.equal(out_h, got)
    got = got.numpy().reshape(wl.Ls, wl.V, 2)
    rng = np.random.default_rng(3)
    L0 = wl.dims[0]
    pts = [(int(rng.integers(0, wl.Ls)), int(rng.integers(0, wl.V))) for _ in range(150)]
    pts += [(0, 0), (wl.Ls - 1, wl.V - 1), (0, wl.V - 1), (wl.Ls - 1, 0), (7, L0 - 1), (8, wl.V - L0)]
    Uo = _rounded_links(U, "f32_l16")
    ps = psi.astype(np.complex64).astype(np.complex128)
    want = dirac.dwf_apply_points_2d(Uo, ps, wl.dims, wl.Ls, wl.M5, wl.mf, pts)
    g_pts = np.array([got[s, site] for s, site in pts])
    assert np.abs(g_pts - want).max() < 1e-5 * np.abs(want).max()


def test_max_size_apply_sampled(dw):
    """A 4096 x 4096 x Ls=16 lattice (268 M 5-d sites, 4.3 GB per FP32 spinor): the apply's
    64-bit indexing and s-window at this size, checked point by point against the definition.
    The source is drawn on the GPU from a seeded generator (the CPU copy is read only at the
    sampled points' neighbourhoods)."""
    dims, Ls, M5, mf = (4096, 4096), 16, 1.0, 0.005
    V = dims[0] * dims[1]
    rng = synth.rng_for(4096)
    theta = synth.u1_angles(rng, dims, 0.7)
    U = synth.u1_links(theta)
    g = dw.make_geom(dims, Ls)
    Ud = dw.links_to(g, _dev(U), "f32_l16")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(4096)
    pd = torch.randn(V * Ls * 2, dtype=torch.complex64, device="cuda", generator=gen)
    out = torch.empty_like(pd)
    dw.dwf_apply(g, Ud, pd, out, M5, mf, prec="f32_l16")
    prng = np.random.default_rng(1)
    pts = [(int(prng.integers(0, Ls)), int(prng.integers(0, V))) for _ in range(40)]
    pts += [(0, 0), (Ls - 1, V - 1), (Ls - 1, 0), (0, V - 1)]
    # psi restricted to what the sampled points read: all slices of each point's 5-site neighbourhood
    L0, L1 = dims
    sites = set()
    for _, x in pts:
        xx, yy = x % L0, x // L0
        for dx, dy in ((0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)):
            sites.add(((yy + dy) % L1) * L0 + (xx + dx) % L0)
    sites = sorted(sites)
    idx = torch.tensor(sites, dtype=torch.long, device="cuda")
    sub = pd.view(Ls, V, 2).index_select(1, idx).cpu().numpy().astype(np.complex128)
    psi_full = np.zeros((Ls, V, 2), dtype=np.complex128)
    psi_full[:, sites, :] = sub
    want = dirac.dwf_apply_points_2d(_rounded_links(U, "f32_l16"), psi_full, dims, Ls, M5, mf, pts)
    got = out.view(Ls, V, 2)
    g_pts = np.array([got[s, x].cpu().numpy() for s, x in pts])
    assert np.abs(g_pts - want).max() < 1e-5 * np.abs(want).max()


def test_cgne_solve_reaches_tolerance(dw):
    """FP64 GPU CGNR on the 32x32 x Ls=8 workload reaches 1e-10 and the oracle's solution."""
    wl = synth.SCHWINGER_32
    U, srcs = wl.draw(1)
    b = srcs[0].reshape(-1)
    g = dw.make_geom(wl.dims, wl.Ls)
    Ud, bd = _dev(U), _dev(b)
    x = torch.empty_like(bd)
    stats, status = dw.cgne_solve(g, Ud, bd, x, wl.M5, wl.mf, tol=1e-10)
    D = dirac.dwf_matrix(U, wl.dims, wl.Ls, wl.M5, wl.mf)
    xs = x.cpu().numpy()
    res = np.linalg.norm(b - D @ xs) / np.linalg.norm(b)
    assert res <= 1e-10 and stats["true_residual"] <= 1e-10
    assert abs(stats["true_residual"] - res) < 1e-12
    from oracle import solvers
    xo, it_o, _ = solvers.cgnr(D, b, tol=1e-10)
    assert np.linalg.norm(xs - xo) / np.linalg.norm(xo) < 1e-7
    # iteration counts agree up to rounding-order effects
    assert abs(stats["iterations"] - it_o) <= max(20, 0.05 * it_o)


def test_cgne_noconv_reports(dw):
    wl = synth.SCHWINGER_32
    U, srcs = wl.draw(1)
    g = dw.make_geom(wl.dims, wl.Ls)
    bd = _dev(srcs[0])
    x = torch.empty_like(bd)
    stats, status = dw.cgne_solve(g, _dev(U), bd, x, wl.M5, wl.mf, tol=1e-10, maxiter=5, raise_noconv=False)
    assert status == 3 and stats["iterations"] == 5 and stats["true_residual"] > 1e-10

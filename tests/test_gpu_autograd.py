"""GPU parity of the differentiation path: Gamma_5 reflection, link force, and the
torch.autograd.Function for x = D_DW^-1 b, against the oracle and central finite
differences."""
import numpy as np
import pytest
import torch

import synth
from oracle import dirac, force

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


def test_links_from_angles_and_gamma5(dw):
    dims, Ls = (12, 10), 5
    rng = synth.rng_for(2)
    theta = synth.u1_angles(rng, dims, 0.7)
    g = dw.make_geom(dims, Ls)
    U = dw.links_from_angles(g, _dev(theta, torch.float64)).cpu().numpy()
    assert np.abs(U - np.exp(1j * theta).reshape(-1)).max() < 1e-15
    v = synth.gaussian_spinor(rng, dims, Ls).reshape(-1)
    for dt in (torch.complex128, torch.complex64):
        got = dw.gamma5_reflect(g, _dev(v, dt)).cpu().numpy()
        want = dirac.reflection_gamma5(120, Ls, 2, 1) @ v
        tol = 0 if dt == torch.complex128 else 1e-6
        assert np.abs(got - want).max() <= tol * np.abs(want).max()


@pytest.mark.parametrize("anti", [None, [1, 0], [0, 1]])
def test_link_force_matches_oracle(dw, anti):
    dims, Ls = (10, 14), 6
    rng = synth.rng_for(3)
    U = synth.u1_links(synth.u1_angles(rng, dims, 0.7))
    lam = synth.gaussian_spinor(rng, dims, Ls)
    x = synth.gaussian_spinor(rng, dims, Ls)
    g = dw.make_geom(dims, Ls, antiperiodic=anti)
    F = dw.link_force(g, _dev(U), _dev(lam), _dev(x)).cpu().numpy().reshape(2, -1)
    want = force.link_derivative_contraction(U, dims, Ls, lam, x, anti)
    assert np.abs(F - want).max() < 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("use_mg", [False, True])
def test_autograd_matches_oracle_adjoint_gradient(dw, use_mg):
    dims, Ls, M5, mf = (8, 8), 4, 1.0, 0.05
    rng = synth.rng_for(4)
    theta = synth.u1_angles(rng, dims, 0.5)
    b = synth.gaussian_spinor(rng, dims, Ls).reshape(-1)
    g = dw.make_geom(dims, Ls)
    mg = None
    if use_mg:
        starts = np.stack([synth.gaussian_complex(rng, (128,)) for _ in range(4)])
        mg = dw.mg_setup(g, dw.links_from_angles(g, _dev(theta, torch.float64)), M5, mf,
                         {"nvec": 4, "block": [4, 4, 1, 1], "setup_mass": -0.19}, _dev(starts))
    th = _dev(theta, torch.float64).requires_grad_(True)
    bd = _dev(b).requires_grad_(True)
    x = dw.solve(th, bd, g, M5, mf, tol=1e-12, mg=mg)
    loss = (x.abs() ** 2).sum()
    loss.backward()
    l0, grad = force.loss_and_grad(theta, b, dims, Ls, M5, mf)
    assert abs(loss.item() - l0) < 1e-9 * l0
    gt = th.grad.cpu().numpy().reshape(2, -1)
    assert np.abs(gt - grad).max() < 1e-7 * np.abs(grad).max()
    # dL/db = 2 D^-dag x  (PyTorch's gradient of a real loss w.r.t. a complex input)
    D = dirac.dwf_matrix(np.exp(1j * theta), dims, Ls, M5, mf).toarray()
    xs = np.linalg.solve(D, b)
    gb = 2 * np.linalg.solve(D.conj().T, xs)
    assert np.abs(bd.grad.cpu().numpy() - gb).max() < 1e-7 * np.abs(gb).max()
    if mg is not None:
        mg.close()


def test_autograd_gradient_vs_central_differences_128(dw):
    """128x128 x Ls=12 (sigma 0.7, m 0.005), loss |x|^2: autograd vs central FD (h = 1e-6) on 16 links.

    The finite differences use CGNR with a fixed iteration count (the count that
    reaches 1e-13 at theta), which makes x(theta) a smooth map so that the
    difference quotient is not swamped by the stopping rule.  With h = 1e-6 the
    quotient is limited by the FP64 rounding of L itself (|x|^2 ~ 1e6 summed over
    4e5 values: ~1e-14 L, i.e. ~1e-8 / (2h) ~ 5e-3 absolute), so agreement is
    required to 2e-4 relative; the exact check of the gradient is the oracle
    comparison on the small lattice above (1e-7).
    """
    wl = synth.SCHWINGER_128_GRAD
    theta, rng = wl.angles()
    b = synth.gaussian_spinor(rng, wl.dims, wl.Ls).reshape(-1)
    g = dw.make_geom(wl.dims, wl.Ls)
    th = _dev(theta, torch.float64).requires_grad_(True)
    bd = _dev(b)
    x = dw.solve(th, bd, g, wl.M5, wl.mf, tol=1e-13)
    loss = (x.abs() ** 2).sum()
    loss.backward()
    grad = th.grad.cpu().numpy()
    U0 = dw.links_from_angles(g, _dev(theta, torch.float64))
    x0 = torch.empty_like(bd)
    st, _ = dw.cgne_solve(g, U0, bd, x0, wl.M5, wl.mf, tol=1e-13)
    nit = st["iterations"]

    def L_fixed(t):
        U = dw.links_from_angles(g, _dev(t, torch.float64))
        xx = torch.empty_like(bd)
        dw.cgne_solve(g, U, bd, xx, wl.M5, wl.mf, tol=1e-300, maxiter=nit, raise_noconv=False)
        return float((xx.abs() ** 2).sum().item())

    pick = np.random.default_rng(wl.seed).choice(theta.size, 16, replace=False)
    h = 1e-6
    flat = theta.reshape(-1)
    for idx in pick:
        tp = flat.copy(); tp[idx] += h
        tm = flat.copy(); tm[idx] -= h
        fd = (L_fixed(tp) - L_fixed(tm)) / (2 * h)
        assert abs(fd - grad[idx]) < 2e-4 * max(abs(fd), 1e-3 * np.abs(grad).max()), (idx, fd, grad[idx])


def test_autograd_rejects_a_hierarchy_of_other_links(dw):
    """A multigrid handle solves with the operator of its setup: once theta moves (or M5 / m_f
    differ) the differentiable solve must refuse it instead of returning a wrong x and gradient."""
    dims, Ls, M5, mf = (8, 8), 4, 1.0, 0.05
    rng = synth.rng_for(40)
    theta = synth.u1_angles(rng, dims, 0.5)
    b = _dev(synth.gaussian_spinor(rng, dims, Ls).reshape(-1))
    g = dw.make_geom(dims, Ls)
    starts = np.stack([synth.gaussian_complex(rng, (128,)) for _ in range(4)])
    th = _dev(theta, torch.float64)
    mg = dw.mg_setup(g, dw.links_from_angles(g, th), M5, mf, {"nvec": 4, "block": [4, 4, 1, 1],
                                                               "setup_mass": -0.19}, _dev(starts))
    dw.solve(th, b, g, M5, mf, tol=1e-10, mg=mg)          # the setup links: accepted
    moved = th.clone()
    moved[5] += 1e-6
    with pytest.raises(dw.DwfError, match="links differ"):
        dw.solve(moved, b, g, M5, mf, tol=1e-10, mg=mg)
    with pytest.raises(dw.DwfError, match="set up for"):
        dw.solve(th, b, g, M5, 2 * mf, tol=1e-10, mg=mg)
    mg.close()


@pytest.mark.parametrize("checkpoint", ["host", "recompute"])
def test_checkpoint_modes_give_the_same_gradients(dw, checkpoint):
    """x kept on the host, or recomputed in backward, gives the gradients of the default (x on the
    device): the solvers are deterministic, so the recomputed x is the forward's x."""
    dims, Ls, M5, mf = (8, 8), 4, 1.0, 0.05
    rng = synth.rng_for(41)
    theta = synth.u1_angles(rng, dims, 0.5)
    b = synth.gaussian_spinor(rng, dims, Ls).reshape(-1)
    g = dw.make_geom(dims, Ls)
    grads = {}
    for mode in ("device", checkpoint):
        th = _dev(theta, torch.float64).requires_grad_(True)
        bd = _dev(b).requires_grad_(True)
        x = dw.solve(th, bd, g, M5, mf, tol=1e-12, checkpoint=mode)
        loss = (x.abs() ** 2).sum()
        loss.backward()
        grads[mode] = (loss.item(), th.grad.clone(), bd.grad.clone())
    l0, t0, b0 = grads["device"]
    l1, t1, b1 = grads[checkpoint]
    assert l1 == l0
    assert torch.equal(t1, t0) and torch.equal(b1, b0)
    # 4-d SU(3) links
    dims4, Ls4, M54 = (4, 4, 4, 4), 4, 1.8
    U = synth.su3_links(rng, dims4, 0.3)
    b4 = synth.gaussian_spinor(rng, dims4, Ls4, "su3").reshape(-1)
    g4 = dw.make_geom(dims4, Ls4, group="su3")
    out = {}
    for mode in ("device", checkpoint):
        Ud = _dev(U).requires_grad_(True)
        bd = _dev(b4).requires_grad_(True)
        x = dw.solve_links(Ud, bd, g4, M54, 0.05, tol=1e-12, checkpoint=mode)
        (x.abs() ** 2).sum().backward()
        out[mode] = (Ud.grad.clone(), bd.grad.clone())
    assert torch.equal(out[checkpoint][0], out["device"][0]) and torch.equal(out[checkpoint][1], out["device"][1])


def test_checkpoint_mode_is_checked(dw):
    g = dw.make_geom((8, 8), 4)
    th = torch.zeros(dw.link_size(g), dtype=torch.float64, device="cuda", requires_grad=True)
    b = torch.ones(dw.spinor_size(g), dtype=torch.complex128, device="cuda")
    with pytest.raises(ValueError):
        dw.solve(th, b, g, 1.0, 0.05, checkpoint="disk")

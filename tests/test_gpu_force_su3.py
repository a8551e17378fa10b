"""GPU parity of the link derivatives of the 4-d SU(3) operator and of the
differentiable solve on SU(3) links (derived from the Wilson hops of Sec. 2):

  * dwf_link_force (SU(3)): the su(3)-projected force against the oracle's
    generator-by-generator derivative, at 1e-12;
  * dwf_link_grad (U(1) and SU(3)): Re sum conj(G) dU against the oracle's
    directional derivative along random complex dU, at 1e-12;
  * DwfSolveLinks: the gradient of |D^-1 b|^2 against the oracle's adjoint
    force on a 2^4 lattice (every link), and against central finite
    differences along random algebra directions on 16 links of 4^4 x 8.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import force

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


def _herm_traceless(rng):
    G = synth.gaussian_complex(rng, (3, 3))
    H = 0.5 * (G + G.conj().T)
    return H - np.trace(H).real / 3 * np.eye(3)


def _expm_herm(H, eps):
    w, Q = np.linalg.eigh(H)
    return (Q * np.exp(1j * eps * w)[None, :]) @ Q.conj().T


@pytest.mark.parametrize("anti", [None, [0, 0, 0, 1]])
def test_su3_force_and_grad_match_oracle(dw, anti):
    dims, Ls = (4, 4, 4, 6), 4
    V = int(np.prod(dims))
    rng = synth.rng_for(60)
    U = synth.su3_links(rng, dims, 0.4)
    lam = synth.gaussian_spinor(rng, dims, Ls, "su3")
    x = synth.gaussian_spinor(rng, dims, Ls, "su3")
    g = dw.make_geom(dims, Ls, group="su3", antiperiodic=anti)
    F = dw.link_force(g, _dev(U), _dev(lam), _dev(x)).cpu().numpy().reshape(4, V, 3, 3)
    G = dw.link_grad(g, _dev(lam), _dev(x)).cpu().numpy().reshape(4, V, 3, 3)
    pick = np.random.default_rng(61).choice(4 * V, 16, replace=False)
    links = [(int(k // V), int(k % V)) for k in pick]
    want = force.link_force_su3(U, dims, Ls, lam, x, links, anti)
    scale = np.abs(want).max()
    for (mu, site), Fw in zip(links, want):
        assert np.abs(F[mu, site] - Fw).max() < 1e-12 * scale
        assert np.abs(F[mu, site] - F[mu, site].conj().T).max() < 1e-14 * scale
        dU = synth.gaussian_complex(rng, (3, 3))
        dd = force.directional_derivative(U, dims, Ls, lam, x, mu, site, dU, "su3", anti)
        got = np.sum(np.conj(G[mu, site]) * dU).real
        assert abs(got - dd) < 1e-12 * np.abs(G).max() * 3


@pytest.mark.parametrize("anti", [None, [1, 0]])
def test_u1_link_grad_matches_oracle(dw, anti):
    dims, Ls = (10, 14), 6
    V = int(np.prod(dims))
    rng = synth.rng_for(62)
    U = synth.u1_links(synth.u1_angles(rng, dims, 0.7))
    lam = synth.gaussian_spinor(rng, dims, Ls)
    x = synth.gaussian_spinor(rng, dims, Ls)
    g = dw.make_geom(dims, Ls, antiperiodic=anti)
    G = dw.link_grad(g, _dev(lam), _dev(x)).cpu().numpy().reshape(2, V)
    for k in np.random.default_rng(63).choice(2 * V, 12, replace=False):
        mu, site = int(k // V), int(k % V)
        dU = complex(*rng.standard_normal(2))
        dd = force.directional_derivative(U, dims, Ls, lam, x, mu, site, dU, "u1", anti)
        assert abs((np.conj(G[mu, site]) * dU).real - dd) < 1e-12 * np.abs(G).max() * 2


def test_solve_links_su3_matches_oracle_gradient(dw):
    """2^4 x Ls 4: autograd's dL/dU projected on the algebra equals the oracle's adjoint force on every link."""
    dims, Ls, M5, mf = (2, 2, 2, 2), 4, 1.8, 0.05
    V = 16
    rng = synth.rng_for(64)
    U = synth.su3_links(rng, dims, 0.4)
    b = synth.gaussian_spinor(rng, dims, Ls, "su3").reshape(-1)
    g = dw.make_geom(dims, Ls, group="su3")
    Ud = _dev(U).requires_grad_(True)
    x = dw.solve_links(Ud, _dev(b), g, M5, mf, tol=1e-13)
    loss = (x.abs() ** 2).sum()
    loss.backward()
    gU = Ud.grad.cpu().numpy().reshape(4, V, 3, 3)
    links = [(mu, s) for mu in range(4) for s in range(V)]
    l0, F = force.loss_and_force_su3(U, b, dims, Ls, M5, mf, links)
    assert abs(loss.item() - l0) < 1e-9 * l0
    T = force.su3_generators()
    for (mu, s), Fl in zip(links, F):
        for a in range(8):
            dUa = 1j * T[a] @ U[mu, s]
            got = np.sum(np.conj(gU[mu, s]) * dUa).real        # dL/d eps_a from the complex gradient
            want = -2 * np.trace(T[a] @ Fl).real
            assert abs(got - want) < 1e-8 * max(1.0, np.abs(F).max())


def test_solve_links_su3_vs_central_differences(dw):
    """4^4 x Ls 8 (eps 0.3, M5 1.8, m 0.05), L = |x|^2: autograd vs central differences (h = 1e-5)
    along random algebra directions on 16 links.  The differences use CGNR with the fixed
    iteration count that reaches 1e-13 at U, so that x(U) is a smooth map."""
    dims, Ls, M5, mf = (4, 4, 4, 4), 8, 1.8, 0.05
    V = int(np.prod(dims))
    rng = synth.rng_for(65)
    U = synth.su3_links(rng, dims, 0.3)
    b = _dev(synth.gaussian_spinor(rng, dims, Ls, "su3").reshape(-1))
    g = dw.make_geom(dims, Ls, group="su3")
    Ud = _dev(U).requires_grad_(True)
    x = dw.solve_links(Ud, b, g, M5, mf, tol=1e-13)
    loss = (x.abs() ** 2).sum()
    loss.backward()
    gU = Ud.grad.cpu().numpy().reshape(4, V, 3, 3)
    x0 = torch.empty_like(b)
    st, _ = dw.cgne_solve(g, _dev(U), b, x0, M5, mf, tol=1e-13)
    nit = st["iterations"]

    def L_fixed(Uv):
        xx = torch.empty_like(b)
        dw.cgne_solve(g, _dev(Uv), b, xx, M5, mf, tol=1e-300, maxiter=nit, raise_noconv=False)
        return float((xx.abs() ** 2).sum().item())

    h = 1e-5
    for k in np.random.default_rng(66).choice(4 * V, 16, replace=False):
        mu, s = int(k // V), int(k % V)
        H = _herm_traceless(rng)
        Lpm = []
        for e in (h, -h):
            Up = U.copy()
            Up[mu, s] = _expm_herm(H, e) @ U[mu, s]
            Lpm.append(L_fixed(Up))
        fd = (Lpm[0] - Lpm[1]) / (2 * h)
        got = np.sum(np.conj(gU[mu, s]) * (1j * H @ U[mu, s])).real
        assert abs(fd - got) < 2e-5 * max(abs(fd), 1e-3 * np.abs(gU).max()), (mu, s, fd, got)

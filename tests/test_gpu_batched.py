"""Batched multi-right-hand-side apply: one launch over mixed lattices, against
single applies and the FP64 oracle."""
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


@pytest.mark.parametrize("dagger", [False, True])
def test_batched_apply_matches_oracle_mixed_lattices(dw, dagger):
    shapes = [((8, 8), 4, None), ((12, 6), 3, [0, 1]), ((5, 7), 5, None), ((16, 16), 8, None), ((8, 8), 4, None)]
    M5, mf = 1.0, 0.03
    rng = synth.rng_for(21)
    geoms, Us, psis, outs, wants = [], [], [], [], []
    for dims, Ls, anti in shapes:
        U = synth.u1_links(synth.u1_angles(rng, dims, 0.6))
        psi = synth.gaussian_spinor(rng, dims, Ls)
        g = dw.make_geom(dims, Ls, antiperiodic=anti)
        geoms.append(g)
        Us.append(_dev(U))
        psis.append(_dev(psi))
        outs.append(torch.empty_like(psis[-1]))
        wants.append(dirac.dwf_apply(U, psi, dims, Ls, M5, mf, dagger_=dagger, antiperiodic=anti).reshape(-1))
    dw.dwf_apply_batched(geoms, Us, psis, outs, M5, mf, dagger=dagger, prec="f64")
    for o, w in zip(outs, wants):
        assert np.linalg.norm(o.cpu().numpy() - w) / np.linalg.norm(w) < 1e-12


def test_batched_apply_equals_single_applies_on_the_64_source_workload(dw):
    """The 64-source batch over {64^2, 128^2, 256^2} x Ls=16: identical to one apply per source."""
    geoms, Us, psis, outs = [], [], [], []
    M5 = mf = None
    for wl, nsrc in synth.batched_classes():
        U, srcs = wl.draw(nsrc)
        g = dw.make_geom(wl.dims, wl.Ls)
        Ud = dw.links_to(g, _dev(U), "f32_l16")
        M5, mf = wl.M5, wl.mf
        for src in srcs:
            geoms.append(g)
            Us.append(Ud)
            psis.append(_dev(src, torch.complex64))
            outs.append(torch.empty_like(psis[-1]))
    assert len(psis) == 64
    dw.dwf_apply_batched(geoms, Us, psis, outs, M5, mf, prec="f32_l16")
    for g, U, p, o in zip(geoms, Us, psis, outs):
        single = torch.empty_like(p)
        dw.dwf_apply(g, U, p, single, M5, mf, prec="f32_l16")
        assert torch.equal(single, o)
    # the prepared form (argument arrays built once), applied twice and with the adjoint
    plan = dw.BatchedApply(geoms, Us, psis, outs, prec="f32_l16")
    for o in outs:
        o.fill_(float("nan"))
    for dag in (False, True, False):
        plan(M5, mf, dagger=dag)
    for g, U, p, o in zip(geoms, Us, psis, outs):
        single = torch.empty_like(p)
        dw.dwf_apply(g, U, p, single, M5, mf, prec="f32_l16")
        assert torch.equal(single, o)


def test_batched_apply_rejects_bad_input(dw):
    g = dw.make_geom((8, 8), 4)
    p = torch.zeros(dw.spinor_size(g), dtype=torch.complex64, device="cuda")
    U = dw.links_to(g, torch.ones(dw.link_size(g), dtype=torch.complex128, device="cuda"), "f32_l16")
    with pytest.raises(dw.DwfError):
        dw.dwf_apply_batched([g], [U], [p], [p], 1.0, 0.01)          # psi aliases out
    g4 = dw.make_geom((2, 2, 2, 2), 2, group="su3")
    p4 = torch.zeros(dw.spinor_size(g4), dtype=torch.complex64, device="cuda")
    with pytest.raises(dw.DwfError):
        dw.dwf_apply_batched([g4], [U], [p4], [torch.empty_like(p4)], 1.0, 0.01)

"""Failure detection without a GPU fault: bounded device waits give up and the
host sees DWF_ERR_TIMEOUT; solver caps and bad input return error codes."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dw():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2004_07732_gb300 as pkg
    pkg.lib()
    return pkg


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_waits_time_out_and_context_survives(dw, which):
    assert dw.check_wait_timeout(which, 0.05) == 4          # DWF_ERR_TIMEOUT
    assert "gave up" in dw.lib().dwf_last_error().decode()
    # the context is still usable: an apply after the timeout is correct
    g = dw.make_geom((8, 8), 4)
    U = torch.ones(dw.link_size(g), dtype=torch.complex128, device="cuda")
    psi = torch.ones(dw.spinor_size(g), dtype=torch.complex128, device="cuda")
    out = torch.empty_like(psi)
    dw.dwf_apply(g, U, psi, out, 1.0, 0.0)
    torch.cuda.synchronize()
    assert torch.isfinite(out.real).all()


def test_nan_source_does_not_converge(dw):
    g = dw.make_geom((8, 8), 4)
    rng = synth.rng_for(3)
    U = torch.from_numpy(synth.u1_links(synth.u1_angles(rng, (8, 8), 0.5)).reshape(-1)).cuda()
    b = torch.full((dw.spinor_size(g),), float("nan"), dtype=torch.complex128, device="cuda")
    x = torch.empty_like(b)
    st, status = dw.cgne_solve(g, U, b, x, 1.0, 0.01, tol=1e-10, maxiter=50, raise_noconv=False)
    assert status != 0

"""Parity of the FP16-block coarse stencils with the FP64 oracle (Eq. coarsenDW).

The default coarse storage holds the Galerkin blocks in FP16.  The oracle here
takes the GPU's FP64 blocks (themselves pinned against the oracle's explicit
triple product in test_gpu_mg / test_gpu_mg4d), rounds every entry to FP16 the
way the setup does (nearest even), assembles the kernel from them and builds
the coarse D_DW / D_PV of Eq. coarsenDW around it.  What is left between the
two sides is FP32 arithmetic, so every stencil form is held to 1e-5: the
one-vector tile stencil, each fixed form of the many-right-hand-side
contraction (mma.sync with 1, 2 or 4 column tiles per warp, tcgen05) and the
autotuned pick.  The adjoint is the sigma_3 form, Dhat_W^dag = sigma_3 Dhat_W
sigma_3, which is how one stored copy of the blocks serves both operators.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import dirac, mg as omg

pytestmark = pytest.mark.gpu

TOL = 1e-5
NRHS = (1, 7, 16, 32, 33, 34, 64)
FORMS = {0: "autotuned", 1: "tcgen05 persistent", 2: "mma.sync x1", 3: "mma.sync x2", 4: "mma.sync x4",
         5: "tcgen05 per item", 6: "tcgen05, A in tensor memory"}


@pytest.fixture(scope="module")
def dw():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2004_07732_gb300 as pkg
    pkg.lib()
    return pkg


def _dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to("cuda").to(dtype)


def _round16(a):
    return a.real.astype(np.float16).astype(np.float64) + 1j * a.imag.astype(np.float16).astype(np.float64)


class Case2d:
    """256^2 x Ls 8 lattice, 4^2 aggregates: 64^2 coarse sites x Lhat_s 4, 16 coarse dof."""
    dims, Ls, Ls_c, nvec, M5, mf = (256, 256), 8, 4, 8, 1.0, 0.005

    def __init__(self, dw):
        rng = synth.rng_for(1201)
        self.U = synth.u1_links(synth.u1_angles(rng, self.dims, 0.7))
        V = int(np.prod(self.dims))
        self.starts = np.stack([synth.gaussian_complex(rng, (V * 2,)) for _ in range(self.nvec)])
        self.geom = dw.make_geom(self.dims, self.Ls)
        self.cdims = (64, 64)
        h = self.setup(dw, 0)
        ncd = 2 * self.nvec
        Vc = int(np.prod(self.cdims))
        Y = _round16(dw.mg_get_coarse_links(h).cpu().numpy().reshape(Vc, 5, ncd, ncd))
        self.nc = h.coarse_size
        h.close()
        K = omg.kernel_from_blocks(Y, self.cdims)
        self.v = synth.gaussian_complex(np.random.default_rng(1202), (max(NRHS), self.nc)).astype(np.complex64)
        V64 = self.v.astype(np.complex128).T
        self.want = {}
        for m in (self.mf, 1.0):
            self.want[(m, False)] = (omg.coarse_dwf(K, self.Ls_c, m, self.nvec) @ V64).T
            self.want[(m, True)] = (omg.coarse_dwf_dagger_g5(K, self.Ls_c, m, self.nvec) @ V64).T

    def setup(self, dw, tc):
        return dw.mg_setup(self.geom, _dev(self.U), self.M5, self.mf,
                           {"nvec": self.nvec, "setup_maxiter": 10, "setup_mass": -0.3, "Ls_c": self.Ls_c,
                            "coarse_block_prec": "f32_l16", "coarse_tc": tc}, _dev(self.starts))


@pytest.fixture(scope="module")
def case2d(dw):
    return Case2d(dw)


def _check(got, want, what):
    for r in range(want.shape[0]):
        g, w = got[r].astype(np.complex128), want[r]
        rel = np.linalg.norm(g - w) / np.linalg.norm(w)
        elem = np.abs(g - w).max() / np.abs(w).max()
        assert rel < TOL and elem < TOL, (what, r, rel, elem)


def test_tile_stencil_fp16_blocks_match_oracle(dw, case2d):
    """One vector: the shared-memory tile stencil reading FP16 blocks (mg_coarse_apply)."""
    c = case2d
    h = c.setup(dw, 0)
    vd = _dev(c.v[0], torch.complex64)
    out = torch.full_like(vd, float("nan"))
    for (m, dag), want in c.want.items():
        dw.mg_coarse_apply(h, vd, out, m, dagger=dag)
        _check(out.cpu().numpy()[None, :], want[:1], ("tile", m, dag))
    h.close()


def _to_site_major(v, Ls_c, Vc):
    """[rhs][s][site][dof] -> [site][rhs][s][dof]"""
    nrhs = v.shape[0]
    return np.ascontiguousarray(v.reshape(nrhs, Ls_c, Vc, 16).transpose(2, 0, 1, 3))


def _from_site_major(v, nrhs, Ls_c, Vc):
    return np.ascontiguousarray(v.reshape(Vc, nrhs, Ls_c, 16).transpose(1, 2, 0, 3)).reshape(nrhs, -1)


@pytest.mark.parametrize("layout", ["slice_major", "site_major"])
@pytest.mark.parametrize("tc", sorted(FORMS))
def test_multi_rhs_contraction_forms_match_oracle(dw, case2d, tc, layout):
    """Every form of the many-right-hand-side contraction at nrhs = 1, 7, 16, 32, 33, 34, 64, both
    operators (m_f and m = 1) and both daggers, on both vector layouts.  tcgen05 runs from 128
    columns (32 right-hand sides x 4 slices; 33 and 34 leave a partial tile); below 128 columns
    coarse_tc = 1 and 5 fall back to mma.sync; the tensor-memory-operand form (coarse_tc = 6) runs from 64 columns."""
    c = case2d
    h = c.setup(dw, tc)
    Vc = int(np.prod(c.cdims))
    for nrhs in NRHS:
        v = c.v[:nrhs]
        if layout == "site_major":
            v = _to_site_major(v, c.Ls_c, Vc)
        vd = _dev(v, torch.complex64)
        out = torch.full_like(vd, float("nan"))
        for (m, dag), want in c.want.items():
            dw.mg_coarse_apply_multi(h, vd, out, nrhs, m, dagger=dag, layout=layout)
            got = out.cpu().numpy()
            got = _from_site_major(got, nrhs, c.Ls_c, Vc) if layout == "site_major" else got.reshape(nrhs, c.nc)
            _check(got, want[:nrhs], (FORMS[tc], layout, nrhs, m, dag))
        form = dw.mg_coarse_tc_form(h, nrhs, layout=layout)
        if tc == 0:
            assert form in (1, 2, 4, 256, 257, 258)
    h.close()


@pytest.mark.parametrize("Ls_c", [4, 3, 2, 1])
def test_coarse_48dof_fp16_matches_oracle_on_gpu_blocks(dw, Ls_c):
    """4-d, 48 coarse dof, FP16 blocks (tensor-core form k_coarse_mma): the oracle's coarse operator
    on the GPU's Galerkin blocks rounded to FP16, at 1e-5."""
    dims, Ls, nvec, M5, mf = (6, 6, 6, 6), 8, 24, 1.8, 0.03
    rng = synth.rng_for(77)
    U = synth.su3_links(rng, dims, 0.3)
    V = int(np.prod(dims))
    starts = np.stack([synth.gaussian_complex(rng, (V * 12,)) for _ in range(nvec)])
    g = dw.make_geom(dims, Ls, group="su3")
    h = dw.mg_setup(g, _dev(U), M5, mf, {"nvec": nvec, "block": [2, 2, 2, 2], "setup_maxiter": 10,
                                         "setup_mass": -0.42, "Ls_c": Ls_c, "coarse_block_prec": "f32_l16"},
                    _dev(starts))
    cdims, ncd = (3, 3, 3, 3), 2 * nvec
    Vc = int(np.prod(cdims))
    Y = _round16(dw.mg_get_coarse_links(h).cpu().numpy().reshape(Vc, 9, ncd, ncd))
    K = omg.kernel_from_blocks(Y, cdims)
    v = synth.gaussian_complex(np.random.default_rng(5), (h.coarse_size,)).astype(np.complex64)
    vd = _dev(v, torch.complex64)
    out = torch.full_like(vd, float("nan"))
    for m in (mf, 1.0):
        for dag in (False, True):
            C = omg.coarse_dwf_dagger_g5(K, Ls_c, m, nvec) if dag else omg.coarse_dwf(K, Ls_c, m, nvec)
            want = C @ v.astype(np.complex128)
            dw.mg_coarse_apply(h, vd, out, m, dagger=dag)
            _check(out.cpu().numpy()[None, :], want[None, :], ("48dof", Ls_c, m, dag))
    h.close()


def test_multi_rhs_contraction_rejects_unknown_layout(dw, case2d):
    """mg_coarse_apply_multi_layout takes the two documented layouts only (DWF_ERR_ARG otherwise)."""
    c = case2d
    h = c.setup(dw, 0)
    vd = _dev(c.v[:2], torch.complex64)
    out = torch.empty_like(vd)
    lib = dw.lib()
    st = lib.mg_coarse_apply_multi_layout(h.ptr, 2, vd.data_ptr(), out.data_ptr(), 0.1, 0, 2, None)
    assert st == 1                                    # DWF_ERR_ARG
    st = lib.mg_coarse_apply_multi_layout(h.ptr, 2, vd.data_ptr(), vd.data_ptr(), 0.1, 0, 1, None)
    assert st == 1                                    # in and out must be distinct
    h.close()

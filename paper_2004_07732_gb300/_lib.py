"""ctypes binding of libdwfmg.so: argument marshalling only.

Every operation runs in the library's CUDA kernels; this module checks
tensor shapes/dtypes, passes raw device pointers and the current torch
stream, and turns a non-zero dwf_status into DwfError.  There is no CPU
fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdwfmg.so")

OK, ERR_ARG, ERR_CUDA, ERR_NOCONV, ERR_TIMEOUT, ERR_OOM, ERR_UNSUPPORTED = range(7)
STATUS_NAMES = {0: "DWF_OK", 1: "DWF_ERR_ARG", 2: "DWF_ERR_CUDA", 3: "DWF_ERR_NOCONV",
                4: "DWF_ERR_TIMEOUT", 5: "DWF_ERR_OOM", 6: "DWF_ERR_UNSUPPORTED"}

PREC = {"f64": 0, "f32": 1, "f32_l16": 2, "f32_lbf16": 3}
GROUP = {"u1": 1, "su3": 3}


class DwfError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Geom(ctypes.Structure):
    _fields_ = [("nd", ctypes.c_int), ("L", ctypes.c_int * 4), ("Ls", ctypes.c_int),
                ("group", ctypes.c_int), ("antiperiodic", ctypes.c_int * 4)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int),
                ("fine_applies", ctypes.c_longlong), ("coarse_applies", ctypes.c_longlong),
                ("coarse_avg_iters", ctypes.c_double), ("true_residual", ctypes.c_double),
                ("seconds", ctypes.c_double), ("coarsest_avg_iters", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MgParams(ctypes.Structure):
    _fields_ = [("nvec", ctypes.c_int), ("block", ctypes.c_int * 4), ("Ls_c", ctypes.c_int),
                ("setup_maxiter", ctypes.c_int), ("setup_tol", ctypes.c_double), ("setup_mass", ctypes.c_double),
                ("gcr_restart", ctypes.c_int), ("pre_smooth", ctypes.c_int), ("post_smooth", ctypes.c_int),
                ("coarse_tol", ctypes.c_double), ("coarse_maxiter", ctypes.c_int), ("fine_prec", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_restarts", ctypes.c_int),
                ("coarse_persistent", ctypes.c_int), ("coarse_solver", ctypes.c_int),
                ("coarse_restart", ctypes.c_int), ("coarse_block_prec", ctypes.c_int), ("cgs_passes", ctypes.c_int),
                ("coarse_tc", ctypes.c_int), ("transfer", ctypes.c_int), ("fine_layout", ctypes.c_int)]


class LevelParams(ctypes.Structure):
    _fields_ = [("nvec", ctypes.c_int), ("block", ctypes.c_int * 4), ("Ls_c", ctypes.c_int),
                ("setup_maxiter", ctypes.c_int), ("setup_tol", ctypes.c_double), ("setup_mass", ctypes.c_double),
                ("gcr_maxiter", ctypes.c_int), ("tol", ctypes.c_double), ("post_smooth", ctypes.c_int),
                ("coarsest_tol", ctypes.c_double), ("coarsest_maxiter", ctypes.c_int), ("n_deflate", ctypes.c_int),
                ("lanczos_steps", ctypes.c_int), ("filter_degree", ctypes.c_int), ("coarsest_solver", ctypes.c_int),
                ("coarsest_restart", ctypes.c_int), ("block_prec", ctypes.c_int)]


_lib = None


def lib():
    """The loaded libdwfmg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2004_07732_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.dwf_last_error.restype = ctypes.c_char_p
        L.dwf_spinor_size.restype = ctypes.c_size_t
        L.dwf_link_size.restype = ctypes.c_size_t
        L.dwf_packed_spinor_size.restype = ctypes.c_size_t
        L.dwf_packed_link_size.restype = ctypes.c_size_t
        _setup_signatures(L)
        _lib = L
    return _lib


_VP = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int


def _setup_signatures(L):
    G = ctypes.POINTER(Geom)
    sigs = {
        "dwf_spinor_size": [G],
        "dwf_link_size": [G],
        "dwf_packed_spinor_size": [G],
        "dwf_packed_link_size": [G],
        "dwf_pack_links": [G, _VP, _VP, _I, _VP],
        "dwf_pack_spinor": [G, _VP, _VP, _VP],
        "dwf_unpack_spinor": [G, _VP, _VP, _VP],
        "dwf_apply_packed": [G, _VP, _VP, _VP, _D, _D, _I, _I, _VP],
        "dwf_convert_links": [G, _VP, _VP, _I, _VP],
        "dwf_apply": [G, _VP, _VP, _VP, _D, _D, _I, _I, _VP],
        "pv_apply": [G, _VP, _VP, _VP, _D, _I, _I, _VP],
        "dwf_pvdag_apply": [G, _VP, _VP, _VP, _VP, _D, _D, _I, _VP],
        "dwf_pvdag_apply_noalloc": [G, _VP, _VP, _VP, _D, _D, _I, _VP],
        "dwf_mobius_apply": [G, _VP, _VP, _VP, _VP, _D, _D, _D, _D, _I, _I, _VP],
        "dwf_pv_poly_apply": [G, _VP, _VP, _VP, _VP, _D, _D, _D, _D, ctypes.POINTER(ctypes.c_double), _I, _I, _VP],
        "dwf_dot": [_VP, _VP, ctypes.c_size_t, _I, ctypes.POINTER(ctypes.c_double), _VP],
        "cgne_solve": [G, _VP, _VP, _VP, _D, _D, _D, _I, ctypes.POINTER(SolveStats), _VP],
        "bicgstab_solve": [G, _VP, _VP, _VP, _D, _D, _I, _D, _I, _I, ctypes.POINTER(SolveStats), _VP],
        "dwf_apply_batched": [_I, ctypes.POINTER(Geom), ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                              ctypes.POINTER(_VP), _D, _D, _I, _I, _VP],
        "dwf_check_wait_timeout": [_I, _D, _VP],
        "dwf_apply_host": [G, _VP, _VP, _VP, _VP, _VP, _VP, _D, _D, _I, _I, _I, _VP],
        "dwf_links_from_angles": [G, _VP, _VP, _VP],
        "dwf_gamma5_reflect": [G, _VP, _VP, _I, _VP],
        "dwf_link_force": [G, _VP, _VP, _VP, _VP, _VP],
        "dwf_link_grad": [G, _VP, _VP, _VP, _VP],
        "mg_setup": [G, _VP, _D, _D, ctypes.POINTER(MgParams), _VP, ctypes.POINTER(_VP), _VP],
        "mg_solve": [_VP, _VP, _VP, _D, _I, ctypes.POINTER(SolveStats), _VP],
        "mg_solve_batched": [_VP, _I, _VP, _VP, _D, _I, ctypes.POINTER(SolveStats), _VP],
        "mg_solve_groups": [_I, ctypes.POINTER(_VP), ctypes.POINTER(_I), ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                            _D, _I, ctypes.POINTER(ctypes.POINTER(SolveStats))],
        "mg_check_operator": [_VP, _VP, _D, _D, _VP],
        "mg_coarse_geom": [_VP, G, ctypes.POINTER(ctypes.c_int)],
        "mg_get_prolongator": [_VP, _VP, _VP],
        "mg_get_null_vectors": [_VP, _VP, _VP],
        "mg_get_coarse_links": [_VP, _VP, _VP],
        "mg_restrict": [_VP, _VP, _VP, _VP],
        "mg_prolong": [_VP, _VP, _VP, _VP],
        "mg_coarse_apply": [_VP, _VP, _VP, _D, _I, _VP],
        "mg_transfer_colinearity": [_VP, _VP, _VP, _VP],
        "mg_transfer_oblique": [_VP, _VP, _VP, _D, ctypes.POINTER(ctypes.c_int), _VP],
        "mg_coarse_solve": [_VP, _VP, _VP, _D, _I, ctypes.POINTER(ctypes.c_int), _VP],
        "mg_coarse_apply_multi": [_VP, _I, _VP, _VP, _D, _I, _VP],
        "mg_coarse_tc_form": [_VP, _I],
        "mg_coarse_apply_multi_layout": [_VP, _I, _VP, _VP, _D, _I, _I, _VP],
        "mg_coarse_tc_form_layout": [_VP, _I, _I],
        "mg_add_level": [_VP, ctypes.POINTER(LevelParams), _VP, _VP, _VP],
        "mg_level_geom": [_VP, G, ctypes.POINTER(ctypes.c_int)],
        "mg_level_get": [_VP, _I, _VP, _VP],
        "mg_level_apply": [_VP, _VP, _VP, _D, _I, _VP],
        "mg_level_restrict": [_VP, _VP, _VP, _VP],
        "mg_level_prolong": [_VP, _VP, _VP, _VP],
        "mg_level_coarsest_solve": [_VP, _VP, _VP, _D, _I, _I, ctypes.POINTER(ctypes.c_int), _VP],
        "mg_level_ritz_values": [_VP, ctypes.POINTER(ctypes.c_double), _I],
        "mg_level_last_iterations": [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
        "mg_level_deflation_info": [_VP, ctypes.POINTER(ctypes.c_double)],
    }
    for name, args in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        if name not in ("dwf_spinor_size", "dwf_link_size", "dwf_packed_spinor_size", "dwf_packed_link_size"):
            fn.restype = ctypes.c_int
    L.dwf_mg_default_params.argtypes = [ctypes.POINTER(MgParams)]
    L.dwf_mg_default_params.restype = None
    L.dwf_mg_default_level_params.argtypes = [ctypes.POINTER(LevelParams)]
    L.dwf_mg_default_level_params.restype = None
    L.mg_destroy.argtypes = [_VP]
    L.mg_destroy.restype = None


def check(status: int):
    if status != OK:
        raise DwfError(status, lib().dwf_last_error().decode(errors="replace"))


def make_geom(dims, Ls, group="u1", antiperiodic=None) -> Geom:
    g = Geom()
    g.nd = len(dims)
    for i, L in enumerate(dims):
        g.L[i] = int(L)
    g.Ls = int(Ls)
    g.group = GROUP[group]
    for i, a in enumerate(antiperiodic or []):
        g.antiperiodic[i] = int(bool(a))
    return g


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def spinor_dtype(prec: str):
    return torch.complex128 if prec == "f64" else torch.complex64


def spinor_size(geom: Geom) -> int:
    return int(lib().dwf_spinor_size(ctypes.byref(geom)))


def link_size(geom: Geom) -> int:
    return int(lib().dwf_link_size(ctypes.byref(geom)))


def _check_spinor(t, geom, prec, name):
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    if t.dtype != spinor_dtype(prec):
        raise ValueError(f"{name} must be {spinor_dtype(prec)} for precision {prec}")
    if t.numel() != spinor_size(geom):
        raise ValueError(f"{name} has {t.numel()} complex values, geometry needs {spinor_size(geom)}")


def links_to(geom: Geom, U64: torch.Tensor, prec: str, stream=None) -> torch.Tensor:
    """Convert complex128 links to the storage of `prec` (on the GPU)."""
    n = link_size(geom)
    if U64.dtype != torch.complex128 or U64.numel() != n or not U64.is_cuda:
        raise ValueError("U64 must be a CUDA complex128 tensor of the link size")
    U64 = U64.contiguous()
    if prec == "f64":
        out = torch.empty(n, dtype=torch.complex128, device=U64.device)
    elif prec == "f32":
        out = torch.empty(n, dtype=torch.complex64, device=U64.device)
    elif prec == "f32_l16":
        out = torch.empty(n, 2, dtype=torch.float16, device=U64.device)
    else:
        out = torch.empty(n, 2, dtype=torch.bfloat16, device=U64.device)
    check(lib().dwf_convert_links(ctypes.byref(geom), _ptr(U64), _ptr(out), PREC[prec], _stream(stream)))
    return out


def packed_spinor_size(geom: Geom) -> int:
    return int(lib().dwf_packed_spinor_size(ctypes.byref(geom)))


def packed_link_size(geom: Geom) -> int:
    return int(lib().dwf_packed_link_size(ctypes.byref(geom)))


def _check_packed(t, geom, name):
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    if t.dtype != torch.complex64:
        raise ValueError(f"{name} must be complex64 (packed spinors are FP32)")
    if t.numel() != packed_spinor_size(geom):
        raise ValueError(f"{name} has {t.numel()} complex values, the packed layout needs {packed_spinor_size(geom)}")


def pack_links(geom: Geom, U64: torch.Tensor, prec: str, stream=None) -> torch.Tensor:
    """complex128 canonical links -> packed links in the storage of `prec` (4-d)."""
    n = packed_link_size(geom)
    if U64.dtype != torch.complex128 or U64.numel() != link_size(geom) or not U64.is_cuda:
        raise ValueError("U64 must be a CUDA complex128 tensor of the link size")
    U64 = U64.contiguous()
    if prec == "f32":
        out = torch.empty(n, dtype=torch.complex64, device=U64.device)
    elif prec == "f32_l16":
        out = torch.empty(n, 2, dtype=torch.float16, device=U64.device)
    elif prec == "f32_lbf16":
        out = torch.empty(n, 2, dtype=torch.bfloat16, device=U64.device)
    else:
        raise ValueError("packed links take f32, f32_l16 or f32_lbf16")
    check(lib().dwf_pack_links(ctypes.byref(geom), _ptr(U64), _ptr(out), PREC[prec], _stream(stream)))
    return out


def pack_spinor(geom: Geom, psi: torch.Tensor, out=None, stream=None) -> torch.Tensor:
    """FP32 canonical spinor -> packed layout (4-d)."""
    _check_spinor(psi, geom, "f32", "psi")
    if out is None:
        out = torch.empty(packed_spinor_size(geom), dtype=torch.complex64, device=psi.device)
    _check_packed(out, geom, "out")
    check(lib().dwf_pack_spinor(ctypes.byref(geom), _ptr(psi), _ptr(out), _stream(stream)))
    return out


def unpack_spinor(geom: Geom, packed: torch.Tensor, out=None, stream=None) -> torch.Tensor:
    """Packed spinor -> FP32 canonical layout (4-d)."""
    _check_packed(packed, geom, "packed")
    if out is None:
        out = torch.empty(spinor_size(geom), dtype=torch.complex64, device=packed.device)
    _check_spinor(out, geom, "f32", "out")
    check(lib().dwf_unpack_spinor(ctypes.byref(geom), _ptr(packed), _ptr(out), _stream(stream)))
    return out


def dwf_apply_packed(geom, U_packed, psi, out, M5, mf, dagger=False, prec="f32_l16", stream=None):
    """D_DW(mf) (or its adjoint) on packed 4-d spinors with packed links."""
    _check_packed(psi, geom, "psi")
    _check_packed(out, geom, "out")
    check(lib().dwf_apply_packed(ctypes.byref(geom), _ptr(U_packed), _ptr(psi), _ptr(out), float(M5), float(mf),
                                 int(bool(dagger)), PREC[prec], _stream(stream)))
    return out


def dwf_apply(geom, U, psi, out, M5, mf, dagger=False, prec="f64", stream=None):
    _check_spinor(psi, geom, prec, "psi")
    _check_spinor(out, geom, prec, "out")
    check(lib().dwf_apply(ctypes.byref(geom), _ptr(U), _ptr(psi), _ptr(out), float(M5), float(mf),
                          int(bool(dagger)), PREC[prec], _stream(stream)))
    return out


def pv_apply(geom, U, psi, out, M5, dagger=False, prec="f64", stream=None):
    _check_spinor(psi, geom, prec, "psi")
    _check_spinor(out, geom, prec, "out")
    check(lib().pv_apply(ctypes.byref(geom), _ptr(U), _ptr(psi), _ptr(out), float(M5),
                         int(bool(dagger)), PREC[prec], _stream(stream)))
    return out


def dwf_pvdag_apply(geom, U, psi, tmp, out, M5, mf, prec="f64", stream=None):
    for t, nm in ((psi, "psi"), (tmp, "tmp"), (out, "out")):
        _check_spinor(t, geom, prec, nm)
    check(lib().dwf_pvdag_apply(ctypes.byref(geom), _ptr(U), _ptr(psi), _ptr(tmp), _ptr(out), float(M5),
                                float(mf), PREC[prec], _stream(stream)))
    return out


def dwf_pvdag_apply_noalloc(geom, U, psi, out, M5, mf, prec="f64", stream=None):
    """D_PV^dag D_DW psi with the intermediate in the library's fixed device scratch
    (no allocation; for callers that cannot allocate device memory)."""
    for t, nm in ((psi, "psi"), (out, "out")):
        _check_spinor(t, geom, prec, nm)
    check(lib().dwf_pvdag_apply_noalloc(ctypes.byref(geom), _ptr(U), _ptr(psi), _ptr(out), float(M5),
                                        float(mf), PREC[prec], _stream(stream)))
    return out


def dwf_mobius_apply(geom, U, psi, out, M5, mf, b5, c5, dagger=False, prec="f64", tmp=None, stream=None):
    """Mobius D_M(mf) psi (or its adjoint); tmp: one spinor of scratch (allocated here if None)."""
    _check_spinor(psi, geom, prec, "psi")
    _check_spinor(out, geom, prec, "out")
    if tmp is None:
        tmp = torch.empty_like(psi)
    _check_spinor(tmp, geom, prec, "tmp")
    check(lib().dwf_mobius_apply(ctypes.byref(geom), _ptr(U), _ptr(psi), _ptr(out), _ptr(tmp), float(M5), float(mf),
                                 float(b5), float(c5), int(bool(dagger)), PREC[prec], _stream(stream)))
    return out


def dwf_pv_poly_apply(geom, U, psi, out, M5, mf, coeffs, b5=1.0, c5=0.0, prec="f64", tmp=None, stream=None):
    """D_PV^dag p(D_PV D_PV^dag) D psi with p(y) = sum_k coeffs[k] y^k; tmp: four spinors of scratch."""
    _check_spinor(psi, geom, prec, "psi")
    _check_spinor(out, geom, prec, "out")
    n = spinor_size(geom)
    if tmp is None:
        tmp = torch.empty(4 * n, dtype=spinor_dtype(prec), device=psi.device)
    if tmp.numel() < 4 * n or tmp.dtype != spinor_dtype(prec) or not tmp.is_cuda:
        raise ValueError("tmp must hold four spinors of the precision")
    c = (ctypes.c_double * len(coeffs))(*[float(v) for v in coeffs])
    check(lib().dwf_pv_poly_apply(ctypes.byref(geom), _ptr(U), _ptr(psi), _ptr(out), _ptr(tmp), float(M5), float(mf),
                                  float(b5), float(c5), c, len(coeffs), PREC[prec], _stream(stream)))
    return out


def dwf_dot(x, y, stream=None) -> complex:
    if x.dtype != y.dtype or x.numel() != y.numel():
        raise ValueError("x and y must match in dtype and size")
    prec = PREC["f64"] if x.dtype == torch.complex128 else PREC["f32"]
    res = (ctypes.c_double * 2)()
    check(lib().dwf_dot(_ptr(x.contiguous()), _ptr(y.contiguous()), x.numel(), prec, res, _stream(stream)))
    return complex(res[0], res[1])


def cgne_solve(geom, U, b, x, M5, mf, tol=1e-10, maxiter=100000, stream=None, raise_noconv=True):
    _check_spinor(b, geom, "f64", "b")
    _check_spinor(x, geom, "f64", "x")
    st = SolveStats()
    status = lib().cgne_solve(ctypes.byref(geom), _ptr(U), _ptr(b), _ptr(x), float(M5), float(mf), float(tol),
                              int(maxiter), ctypes.byref(st), _stream(stream))
    if status != OK and (raise_noconv or status != ERR_NOCONV):
        check(status)
    return st.as_dict(), status


def bicgstab_solve(geom, U, b, x, M5, mf, ell=6, tol=1e-10, maxiter=100000, inner_prec="f32_l16", stream=None,
                   raise_noconv=True):
    """BiCGStab(ell) on D_PV^dag D_DW x = D_PV^dag b with FP64 reliable updates (complex128 U, b, x)."""
    _check_spinor(b, geom, "f64", "b")
    _check_spinor(x, geom, "f64", "x")
    if U.dtype != torch.complex128 or U.numel() != link_size(geom) or not U.is_cuda:
        raise ValueError("U must be a CUDA complex128 tensor of the link size")
    st = SolveStats()
    status = lib().bicgstab_solve(ctypes.byref(geom), _ptr(U), _ptr(b), _ptr(x), float(M5), float(mf), int(ell),
                                  float(tol), int(maxiter), PREC[inner_prec], ctypes.byref(st), _stream(stream))
    if status != OK and (raise_noconv or status != ERR_NOCONV):
        check(status)
    return st.as_dict(), status


class BatchedApply:
    """dwf_apply_batched with its argument arrays built once: a caller that applies the operator
    to the same set of (geometry, links, psi, out) many times pays the marshalling once and each
    call is a single C call.  Holds references to the tensors it was built from."""

    def __init__(self, geoms, Us, psis, outs, prec="f32_l16"):
        n = len(psis)
        if not (len(geoms) == len(Us) == len(outs) == n):
            raise ValueError("geoms, Us, psis and outs must have the same length")
        for g, p, o in zip(geoms, psis, outs):
            _check_spinor(p, g, prec, "psi")
            _check_spinor(o, g, prec, "out")
        self._keep = (list(Us), list(psis), list(outs))
        self.n = n
        self.prec = PREC[prec]
        self.G = (Geom * n)(*geoms)
        self.U = (_VP * n)(*[u.data_ptr() for u in Us])
        self.P = (_VP * n)(*[p.data_ptr() for p in psis])
        self.O = (_VP * n)(*[o.data_ptr() for o in outs])

    def __call__(self, M5, mf, dagger=False, stream=None):
        check(lib().dwf_apply_batched(self.n, self.G, self.U, self.P, self.O, float(M5), float(mf),
                                      int(bool(dagger)), self.prec, _stream(stream)))
        return self._keep[2]


def dwf_apply_batched(geoms, Us, psis, outs, M5, mf, dagger=False, prec="f32_l16", stream=None):
    """One launch applying D_DW to every (geometry, links, psi) triple of the lists."""
    return BatchedApply(geoms, Us, psis, outs, prec)(M5, mf, dagger, stream)


def dwf_apply_host(geom, U_host, psi_host, out_host, U_dev, psi_dev, out_dev, M5, mf, dagger=False,
                   prec="f32_l16", nchunks=0, stream=None):
    """D_DW on host spinors: copies in, applies and copies back, pipelined over s-chunks.

    U_host holds the links in the storage of `prec`; the *_dev tensors are device staging
    buffers of the same sizes.  Returns once the work is ordered on `stream`."""
    for t, nm in ((psi_host, "psi_host"), (out_host, "out_host")):
        if t.is_cuda or not t.is_contiguous() or t.dtype != spinor_dtype(prec) or t.numel() != spinor_size(geom):
            raise ValueError(f"{nm} must be a contiguous host tensor of the spinor size and precision")
    _check_spinor(psi_dev, geom, prec, "psi_dev")
    _check_spinor(out_dev, geom, prec, "out_dev")
    if U_host.is_cuda or not U_dev.is_cuda or U_host.numel() * U_host.element_size() != U_dev.numel() * U_dev.element_size():
        raise ValueError("U_host (host) and U_dev (device) must be link buffers of the same size")
    check(lib().dwf_apply_host(ctypes.byref(geom), ctypes.c_void_p(U_host.data_ptr()), ctypes.c_void_p(psi_host.data_ptr()),
                               ctypes.c_void_p(out_host.data_ptr()), _ptr(U_dev), _ptr(psi_dev), _ptr(out_dev),
                               float(M5), float(mf), int(bool(dagger)), PREC[prec], int(nchunks), _stream(stream)))


def check_wait_timeout(which=0, seconds=0.05, stream=None) -> int:
    """Run the bounded-wait diagnostic; returns the dwf_status (DWF_ERR_TIMEOUT expected)."""
    return lib().dwf_check_wait_timeout(int(which), float(seconds), _stream(stream))


def links_from_angles(geom, theta, stream=None):
    """complex128 links exp(i theta) computed on the GPU (U(1))."""
    if theta.dtype != torch.float64 or not theta.is_cuda or theta.numel() != link_size(geom):
        raise ValueError("theta must be a CUDA float64 tensor of the link size")
    U = torch.empty(theta.numel(), dtype=torch.complex128, device=theta.device)
    check(lib().dwf_links_from_angles(ctypes.byref(geom), _ptr(theta.contiguous()), _ptr(U), _stream(stream)))
    return U


def gamma5_reflect(geom, vin, vout=None, stream=None):
    prec = "f64" if vin.dtype == torch.complex128 else "f32"
    _check_spinor(vin, geom, prec, "in")
    if vout is None:
        vout = torch.empty_like(vin)
    check(lib().dwf_gamma5_reflect(ctypes.byref(geom), _ptr(vin), _ptr(vout), PREC[prec], _stream(stream)))
    return vout


def link_force(geom, U, lam, x, stream=None):
    """Re(lam^dag dD_DW x) per link: float64 per angle (2-d U(1)); for 4-d SU(3) the traceless
    Hermitian force F (complex128, the link layout) with Re(lam^dag dD x) = tr(H F) under
    U -> exp(i eps H) U."""
    _check_spinor(lam, geom, "f64", "lam")
    _check_spinor(x, geom, "f64", "x")
    if geom.group == GROUP["su3"]:
        F = torch.empty(link_size(geom), dtype=torch.complex128, device=lam.device)
    else:
        F = torch.empty(link_size(geom), dtype=torch.float64, device=lam.device)
    check(lib().dwf_link_force(ctypes.byref(geom), _ptr(U), _ptr(lam), _ptr(x), _ptr(F), _stream(stream)))
    return F


def link_grad(geom, lam, x, stream=None):
    """Complex link gradient G (complex128, link layout): Re(lam^dag dD_DW x) = Re sum conj(G) dU."""
    _check_spinor(lam, geom, "f64", "lam")
    _check_spinor(x, geom, "f64", "x")
    G = torch.empty(link_size(geom), dtype=torch.complex128, device=lam.device)
    check(lib().dwf_link_grad(ctypes.byref(geom), _ptr(lam), _ptr(x), _ptr(G), _stream(stream)))
    return G


# ---------------------------------------------------------------------------
# multigrid
# ---------------------------------------------------------------------------
def mg_default_params() -> dict:
    p = MgParams()
    lib().dwf_mg_default_params(ctypes.byref(p))
    d = {k: getattr(p, k) for k, _ in MgParams._fields_}
    d["block"] = list(p.block)
    return d


def _params(d: dict) -> MgParams:
    p = MgParams()
    lib().dwf_mg_default_params(ctypes.byref(p))
    for k, v in d.items():
        if k == "block":
            for i, b in enumerate(v):
                p.block[i] = int(b)
        elif k in ("fine_prec", "coarse_block_prec") and isinstance(v, str):
            setattr(p, k, PREC[v])
        else:
            setattr(p, k, v)
    return p


class Multigrid:
    """Owning handle of an mg_setup hierarchy (freed by close() or garbage collection)."""

    def __init__(self, ptr, geom, params):
        self.ptr = ptr
        self.geom = geom
        self.params = params
        cg = Geom()
        ncd = ctypes.c_int()
        check(lib().mg_coarse_geom(self.ptr, ctypes.byref(cg), ctypes.byref(ncd)))
        self.coarse_geom = cg
        self.ncdof = ncd.value
        self.Vc = 1
        for i in range(cg.nd):
            self.Vc *= cg.L[i]

    def close(self):
        if self.ptr:
            lib().mg_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def coarse_size(self):
        return self.Vc * self.coarse_geom.Ls * self.ncdof


def mg_setup(geom, U64, M5, mf, params=None, null_starts=None, stream=None) -> Multigrid:
    """Build the two-level hierarchy; null_starts: nvec d-dim complex128 Gaussian vectors."""
    prm = _params(params or {})
    if null_starts is None:
        raise ValueError("null_starts (the Gaussian starts of the near-null relaxation) are required")
    h = ctypes.c_void_p()
    check(lib().mg_setup(ctypes.byref(geom), _ptr(U64.contiguous()), float(M5), float(mf), ctypes.byref(prm),
                         _ptr(null_starts.contiguous()), ctypes.byref(h), _stream(stream)))
    return Multigrid(h, geom, prm)


def mg_solve(mg: Multigrid, b, x, tol=1e-10, maxiter=100000, stream=None, raise_noconv=True):
    _check_spinor(b, mg.geom, "f64", "b")
    _check_spinor(x, mg.geom, "f64", "x")
    st = SolveStats()
    status = lib().mg_solve(mg.ptr, _ptr(b), _ptr(x), float(tol), int(maxiter), ctypes.byref(st), _stream(stream))
    if status != OK and (raise_noconv or status != ERR_NOCONV):
        check(status)
    return st.as_dict(), status


def _check_block(t, mg: Multigrid, nrhs, name):
    if not (t.is_cuda and t.is_contiguous()) or t.dtype != torch.complex128:
        raise ValueError(f"{name} must be a contiguous complex128 CUDA tensor")
    if t.numel() != nrhs * spinor_size(mg.geom):
        raise ValueError(f"{name} must hold {nrhs} fine vectors of the hierarchy's lattice")


def mg_solve_batched(mg: Multigrid, b, x, nrhs, tol=1e-10, maxiter=100000, stream=None, raise_noconv=True):
    """Solve D_DW x_r = b_r for nrhs right-hand sides stored back to back (complex128)."""
    _check_block(b, mg, nrhs, "b")
    _check_block(x, mg, nrhs, "x")
    st = (SolveStats * nrhs)()
    status = lib().mg_solve_batched(mg.ptr, int(nrhs), _ptr(b), _ptr(x), float(tol), int(maxiter), st,
                                    _stream(stream))
    if status != OK and (raise_noconv or status != ERR_NOCONV):
        check(status)
    return [s.as_dict() for s in st], status


def mg_solve_groups(mgs, bs, xs, nrhs, tol=1e-10, maxiter=100000, raise_noconv=True):
    """Batched solves of several hierarchies at once (one stream and host thread each)."""
    n = len(mgs)
    if not (len(bs) == len(xs) == len(nrhs) == n):
        raise ValueError("mgs, bs, xs and nrhs must have the same length")
    for mg, b, x, k in zip(mgs, bs, xs, nrhs):
        _check_block(b, mg, k, "b")
        _check_block(x, mg, k, "x")
    stats = [(SolveStats * k)() for k in nrhs]
    sp = (ctypes.POINTER(SolveStats) * n)(*[ctypes.cast(s, ctypes.POINTER(SolveStats)) for s in stats])
    status = lib().mg_solve_groups(n, (_VP * n)(*[m.ptr for m in mgs]), (_I * n)(*[int(k) for k in nrhs]),
                                   (_VP * n)(*[_ptr(b) for b in bs]), (_VP * n)(*[_ptr(x) for x in xs]),
                                   float(tol), int(maxiter), sp)
    if status != OK and (raise_noconv or status != ERR_NOCONV):
        check(status)
    return [[s.as_dict() for s in st] for st in stats], status


def mg_check_operator(mg: Multigrid, U64, M5, mf, stream=None):
    """Raise DwfError unless mg was set up for exactly the links U64 (complex128), M5 and mf."""
    if U64.dtype != torch.complex128 or U64.numel() != link_size(mg.geom) or not U64.is_cuda:
        raise ValueError("U64 must be a CUDA complex128 tensor of the link size")
    check(lib().mg_check_operator(mg.ptr, _ptr(U64.contiguous()), float(M5), float(mf), _stream(stream)))


def mg_destroy(mg: Multigrid):
    mg.close()


def mg_get_prolongator(mg: Multigrid):
    g = mg.geom
    nchd = (2 if g.nd == 4 else 1) * (3 if g.group == 3 else 1)
    V = 1
    for i in range(g.nd):
        V *= g.L[i]
    out = torch.empty(V * 2 * nchd * mg.params.nvec, dtype=torch.complex128, device="cuda")
    check(lib().mg_get_prolongator(mg.ptr, _ptr(out), _stream(None)))
    return out


def mg_get_null_vectors(mg: Multigrid):
    g = mg.geom
    V = 1
    for i in range(g.nd):
        V *= g.L[i]
    dof = (2 if g.nd == 2 else 4) * (3 if g.group == 3 else 1)
    out = torch.empty(mg.params.nvec * V * dof, dtype=torch.complex128, device="cuda")
    check(lib().mg_get_null_vectors(mg.ptr, _ptr(out), _stream(None)))
    return out


def mg_get_coarse_links(mg: Multigrid):
    ndir = 2 * mg.geom.nd + 1
    out = torch.empty(mg.Vc * ndir * mg.ncdof * mg.ncdof, dtype=torch.complex128, device="cuda")
    check(lib().mg_get_coarse_links(mg.ptr, _ptr(out), _stream(None)))
    return out


def mg_restrict(mg: Multigrid, r_fine, r_coarse, stream=None):
    _check_spinor(r_fine, mg.geom, "f32", "r_fine")
    if r_coarse.dtype != torch.complex64 or r_coarse.numel() != mg.coarse_size:
        raise ValueError("r_coarse must be complex64 of the coarse size")
    check(lib().mg_restrict(mg.ptr, _ptr(r_fine), _ptr(r_coarse), _stream(stream)))
    return r_coarse


def mg_prolong(mg: Multigrid, e_coarse, e_fine, stream=None):
    _check_spinor(e_fine, mg.geom, "f32", "e_fine")
    if e_coarse.dtype != torch.complex64 or e_coarse.numel() != mg.coarse_size:
        raise ValueError("e_coarse must be complex64 of the coarse size")
    check(lib().mg_prolong(mg.ptr, _ptr(e_coarse), _ptr(e_fine), _stream(stream)))
    return e_fine


def mg_coarse_apply(mg: Multigrid, vin, vout, mf, dagger=False, stream=None):
    for t in (vin, vout):
        if t.dtype != torch.complex64 or t.numel() != mg.coarse_size or not t.is_cuda:
            raise ValueError("coarse vectors must be complex64 CUDA tensors of the coarse size")
    check(lib().mg_coarse_apply(mg.ptr, _ptr(vin), _ptr(vout), float(mf), int(bool(dagger)), _stream(stream)))
    return vout


COARSE_LAYOUTS = {"slice_major": 0, "site_major": 1}


def mg_coarse_apply_multi(mg: Multigrid, vin, vout, nrhs, mf, dagger=False, stream=None, layout="slice_major"):
    """Tensor-core coarse operator on nrhs coarse vectors: stored back to back ("slice_major",
    [rhs][s][site][dof]) or with all columns of a coarse site together ("site_major",
    [site][rhs][s][dof])."""
    for t in (vin, vout):
        if t.dtype != torch.complex64 or t.numel() != nrhs * mg.coarse_size or not t.is_cuda:
            raise ValueError("coarse vectors must be complex64 CUDA tensors of nrhs x the coarse size")
    check(lib().mg_coarse_apply_multi_layout(mg.ptr, int(nrhs), _ptr(vin), _ptr(vout), float(mf),
                                             int(bool(dagger)), COARSE_LAYOUTS[layout], _stream(stream)))
    return vout


def mg_coarse_tc_form(mg: Multigrid, nrhs, layout="slice_major") -> int:
    """Form of the coarse contraction the autotuner chose for nrhs (0: not tuned yet)."""
    return int(lib().mg_coarse_tc_form_layout(mg.ptr, int(nrhs), COARSE_LAYOUTS[layout]))


# ---------------------------------------------------------------------------
# third level and coarsest deflation
# ---------------------------------------------------------------------------
def mg_default_level_params() -> dict:
    p = LevelParams()
    lib().dwf_mg_default_level_params(ctypes.byref(p))
    d = {k: getattr(p, k) for k, _ in LevelParams._fields_}
    d["block"] = list(p.block)
    return d


def mg_add_level(mg: Multigrid, params=None, null_starts=None, lanczos_start=None, stream=None):
    """Add the third level (and its deflation) to a two-level hierarchy.

    null_starts: nvec complex128 coarse vectors ([vec][coarse site][dof]); lanczos_start: one
    complex128 vector of the new level's size (needed when n_deflate > 0)."""
    p = LevelParams()
    lib().dwf_mg_default_level_params(ctypes.byref(p))
    for k, v in (params or {}).items():
        if k == "block":
            for i, b in enumerate(v):
                p.block[i] = int(b)
        elif k == "block_prec" and isinstance(v, str):
            p.block_prec = PREC[v]
        else:
            setattr(p, k, v)
    if null_starts is None:
        raise ValueError("null_starts are required")
    check(lib().mg_add_level(mg.ptr, ctypes.byref(p), _ptr(null_starts.contiguous()),
                             _ptr(lanczos_start.contiguous()) if lanczos_start is not None else None,
                             _stream(stream)))
    cg = Geom()
    ncd = ctypes.c_int()
    check(lib().mg_level_geom(mg.ptr, ctypes.byref(cg), ctypes.byref(ncd)))
    mg.level_geom, mg.level_ncdof, mg.level_params = cg, ncd.value, p
    mg.level_V = cg.L[0] * cg.L[1]
    mg.level_size = mg.level_V * cg.Ls * ncd.value
    return mg


def mg_level_get(mg: Multigrid, what: int):
    """The new level's null vectors (0), prolongator (1) or Galerkin blocks (2), complex128."""
    p = mg.level_params
    n = {0: p.nvec * mg.Vc * mg.ncdof, 1: mg.Vc * mg.ncdof * p.nvec,
         2: mg.level_V * 5 * mg.level_ncdof * mg.level_ncdof}[what]
    out = torch.empty(n, dtype=torch.complex128, device="cuda")
    check(lib().mg_level_get(mg.ptr, int(what), _ptr(out), _stream(None)))
    return out


def _check_level_vec(mg, t, name):
    if t.dtype != torch.complex64 or t.numel() != mg.level_size or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous complex64 CUDA tensor of the new level's size")


def _check_coarse_vec(mg, t, name):
    if t.dtype != torch.complex64 or t.numel() != mg.coarse_size or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous complex64 CUDA tensor of the coarse size")


def mg_level_apply(mg: Multigrid, vin, vout, mf, dagger=False, stream=None):
    _check_level_vec(mg, vin, "in")
    _check_level_vec(mg, vout, "out")
    check(lib().mg_level_apply(mg.ptr, _ptr(vin), _ptr(vout), float(mf), int(bool(dagger)), _stream(stream)))
    return vout


def mg_level_restrict(mg: Multigrid, r2, r3, stream=None):
    _check_coarse_vec(mg, r2, "r2")
    _check_level_vec(mg, r3, "r3")
    check(lib().mg_level_restrict(mg.ptr, _ptr(r2), _ptr(r3), _stream(stream)))
    return r3


def mg_level_prolong(mg: Multigrid, e3, e2, stream=None):
    _check_level_vec(mg, e3, "e3")
    _check_coarse_vec(mg, e2, "e2")
    check(lib().mg_level_prolong(mg.ptr, _ptr(e3), _ptr(e2), _stream(stream)))
    return e2


def mg_level_coarsest_solve(mg: Multigrid, b, x, tol=0.05, maxiter=1024, deflate=True, stream=None) -> int:
    _check_level_vec(mg, b, "b")
    _check_level_vec(mg, x, "x")
    it = ctypes.c_int()
    check(lib().mg_level_coarsest_solve(mg.ptr, _ptr(b), _ptr(x), float(tol), int(maxiter), int(bool(deflate)),
                                        ctypes.byref(it), _stream(stream)))
    return it.value


def mg_level_ritz_values(mg: Multigrid):
    n = lib().mg_level_ritz_values(mg.ptr, None, 0)
    buf = (ctypes.c_double * max(n, 1))()
    lib().mg_level_ritz_values(mg.ptr, buf, n)
    return [buf[i] for i in range(n)]


def mg_level_last_iterations(mg: Multigrid):
    a, b = ctypes.c_int(), ctypes.c_int()
    check(lib().mg_level_last_iterations(mg.ptr, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def mg_level_deflation_info(mg: Multigrid) -> dict:
    info = (ctypes.c_double * 4)()
    check(lib().mg_level_deflation_info(mg.ptr, info))
    return {"vectors": int(info[0]), "filter_cut": info[1], "filter_top": info[2], "filter_runs": int(info[3])}


def mg_transfer_colinearity(mg: Multigrid, v, out=None, stream=None):
    """(1 - P R) v for a complex64 fine vector v (the handle's transfer)."""
    _check_spinor(v, mg.geom, "f32", "v")
    out = torch.empty_like(v) if out is None else out
    check(lib().mg_transfer_colinearity(mg.ptr, _ptr(v), _ptr(out), _stream(stream)))
    return out


def mg_transfer_oblique(mg: Multigrid, v, out=None, tol=1e-6, stream=None):
    """(1 - P Ahat^-1 R A) v for a complex64 fine vector v; returns (out, coarse GCR steps)."""
    _check_spinor(v, mg.geom, "f32", "v")
    out = torch.empty_like(v) if out is None else out
    it = ctypes.c_int()
    check(lib().mg_transfer_oblique(mg.ptr, _ptr(v), _ptr(out), float(tol), ctypes.byref(it), _stream(stream)))
    return out, it.value


def mg_coarse_solve(mg: Multigrid, rc, ec, tol=1e-6, maxiter=10000, stream=None) -> int:
    """Restarted GCR on Dhat_PV^dag Dhat_DW ec = rc (complex64 coarse vectors); returns the steps."""
    for t, nm in ((rc, "rc"), (ec, "ec")):
        if t.dtype != torch.complex64 or t.numel() != mg.coarse_size or not t.is_cuda:
            raise ValueError(f"{nm} must be a complex64 CUDA tensor of the coarse size")
    it = ctypes.c_int()
    check(lib().mg_coarse_solve(mg.ptr, _ptr(rc), _ptr(ec), float(tol), int(maxiter), ctypes.byref(it),
                                _stream(stream)))
    return it.value

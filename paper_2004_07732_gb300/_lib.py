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
                ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


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
        "dwf_convert_links": [G, _VP, _VP, _I, _VP],
        "dwf_apply": [G, _VP, _VP, _VP, _D, _D, _I, _I, _VP],
        "pv_apply": [G, _VP, _VP, _VP, _D, _I, _I, _VP],
        "dwf_pvdag_apply": [G, _VP, _VP, _VP, _VP, _D, _D, _I, _VP],
        "dwf_pvdag_apply_noalloc": [G, _VP, _VP, _VP, _D, _D, _I, _VP],
        "dwf_dot": [_VP, _VP, ctypes.c_size_t, _I, ctypes.POINTER(ctypes.c_double), _VP],
        "cgne_solve": [G, _VP, _VP, _VP, _D, _D, _D, _I, ctypes.POINTER(SolveStats), _VP],
    }
    for name, args in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        if name not in ("dwf_spinor_size", "dwf_link_size"):
            fn.restype = ctypes.c_int


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

"""ctypes binding of liblnocc (include/lnocc.h): the same entry points, argument marshalling only.

Device arrays are passed as torch CUDA tensors (FP64, contiguous) or raw integer device pointers;
every step of the computation runs in the library's CUDA kernels. There is no CPU fallback: a
missing library or CUDA device raises.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "liblnocc.so")

LNOCC_OK, LNOCC_EINVAL, LNOCC_ENOMEM, LNOCC_ENOCONV, LNOCC_ENUMERIC, LNOCC_ETIMEOUT, LNOCC_ECUDA = range(7)
LNOCC_PREC_FP64, LNOCC_PREC_MIXED = 0, 1
LNOCC_GUESS_MP2, LNOCC_GUESS_GIVEN = 0, 1
LNOCC_FAULT_NAN_INPUT, LNOCC_FAULT_ZERO_DIIS = 1, 2

ERR_NAMES = {0: "LNOCC_OK", 1: "LNOCC_EINVAL", 2: "LNOCC_ENOMEM", 3: "LNOCC_ENOCONV", 4: "LNOCC_ENUMERIC",
             5: "LNOCC_ETIMEOUT", 6: "LNOCC_ECUDA"}

EXPORTS = ["lnocc_default_opts", "lnocc_build_ints", "lnocc_ccsd", "lnocc_fragment_energy", "lnocc_triples",
           "lnocc_debug_gemm", "lnocc_gemm_noalloc", "lnocc_frag_info", "lnocc_free_fragment", "lnocc_last_error",
           "lnocc_version"]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("max_iter", ctypes.c_int), ("diis_space", ctypes.c_int),
                ("n_refine", ctypes.c_int), ("conv_rms", ctypes.c_double), ("conv_energy", ctypes.c_double),
                ("fault_inject", ctypes.c_int), ("verbose", ctypes.c_int), ("reserved", ctypes.c_int * 6)]


class Info(ctypes.Structure):
    _fields_ = [("nocc", ctypes.c_int), ("nvir", ctypes.c_int), ("naux", ctypes.c_int), ("precision", ctypes.c_int),
                ("n_iter", ctypes.c_int), ("converged", ctypes.c_int), ("e_mp2", ctypes.c_double),
                ("e_ccsd", ctypes.c_double), ("last_rms", ctypes.c_double), ("model_flops_ccsd", ctypes.c_double),
                ("model_flops_t", ctypes.c_double), ("exec_flops", ctypes.c_double),
                ("gemm_launches", ctypes.c_longlong), ("device_bytes", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_longlong), ("t_triples_gemm_ms", ctypes.c_double),
                ("t_triples_ms", ctypes.c_double)]


class LnoccError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblnocc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} missing: build it with `python -m paper_2407_11258_gb300.build`")
    lib = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.lnocc_default_opts.argtypes = [ctypes.POINTER(Opts)]
    lib.lnocc_default_opts.restype = None
    lib.lnocc_build_ints.argtypes = [I, I, I, P, P, ctypes.POINTER(Opts), P, ctypes.POINTER(P)]
    lib.lnocc_ccsd.argtypes = [P, P, P, I, P, P, ctypes.POINTER(D), ctypes.POINTER(I), P]
    lib.lnocc_fragment_energy.argtypes = [P, I, P, ctypes.POINTER(D), ctypes.POINTER(D), P]
    lib.lnocc_triples.argtypes = [P, I, P, ctypes.POINTER(D), ctypes.POINTER(D), P]
    lib.lnocc_debug_gemm.argtypes = [I, I, I, I, P, P, P, P]
    lib.lnocc_gemm_noalloc.argtypes = [I, I, I, I, P, P, P, P]
    lib.lnocc_frag_info.argtypes = [P, ctypes.POINTER(Info)]
    lib.lnocc_free_fragment.argtypes = [P]
    lib.lnocc_last_error.restype = ctypes.c_char_p
    lib.lnocc_version.restype = ctypes.c_char_p
    for name in ("lnocc_build_ints", "lnocc_ccsd", "lnocc_fragment_energy", "lnocc_triples", "lnocc_debug_gemm",
                 "lnocc_gemm_noalloc", "lnocc_frag_info", "lnocc_free_fragment"):
        getattr(lib, name).restype = I
    _lib = lib
    return lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def _check(code, ok=(LNOCC_OK,)):
    if code not in ok:
        raise LnoccError(code, load().lnocc_last_error().decode())
    return code


def default_opts(**kw) -> Opts:
    o = Opts()
    load().lnocc_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Fragment:
    """Owns an lnocc_frag handle; methods mirror the C entry points."""

    def __init__(self, handle):
        self.h = handle

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "h", None):
            load().lnocc_free_fragment(self.h)
            self.h = None

    def info(self) -> Info:
        inf = Info()
        _check(load().lnocc_frag_info(self.h, ctypes.byref(inf)))
        return inf


def lnocc_build_ints(nocc, nvir, naux, eps, B, opts=None, stream=None) -> Fragment:
    h = ctypes.c_void_p()
    code = load().lnocc_build_ints(nocc, nvir, naux, _ptr(eps), _ptr(B), ctypes.byref(opts) if opts else None,
                                   _stream(stream), ctypes.byref(h))
    _check(code)
    return Fragment(h)


def lnocc_ccsd(frag: Fragment, t1_in=None, t2_in=None, guess_mode=LNOCC_GUESS_MP2, t1_out=None, t2_out=None,
               stream=None, allow_noconv=False):
    """Returns (e_corr, n_iter, status)."""
    e = ctypes.c_double(0.0)
    it = ctypes.c_int(0)
    code = load().lnocc_ccsd(frag.h, _ptr(t1_in), _ptr(t2_in), guess_mode, _ptr(t1_out), _ptr(t2_out),
                             ctypes.byref(e), ctypes.byref(it), _stream(stream))
    _check(code, (LNOCC_OK, LNOCC_ENOCONV) if allow_noconv else (LNOCC_OK,))
    return e.value, it.value, code


def lnocc_fragment_energy(frag: Fragment, U_frag, stream=None):
    """Returns (e_ccsd_frag, e_mp2_frag); U_frag is [nocc][nlo]."""
    ec, em = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().lnocc_fragment_energy(frag.h, int(U_frag.shape[1]), _ptr(U_frag), ctypes.byref(ec),
                                        ctypes.byref(em), _stream(stream)))
    return ec.value, em.value


def lnocc_triples(frag: Fragment, U_frag=None, stream=None):
    """Returns (e_t_full, e_t_frag)."""
    ef, eF = ctypes.c_double(0.0), ctypes.c_double(0.0)
    nlo = int(U_frag.shape[1]) if U_frag is not None else 0
    _check(load().lnocc_triples(frag.h, nlo, _ptr(U_frag), ctypes.byref(ef), ctypes.byref(eF), _stream(stream)))
    return ef.value, eF.value


def lnocc_debug_gemm(precision, A, B, C, stream=None):
    """C = A @ B.T through the contraction engine (diagnostic)."""
    M, K = A.shape
    N = B.shape[0]
    _check(load().lnocc_debug_gemm(precision, M, N, K, _ptr(A), _ptr(B), _ptr(C), _stream(stream)))
    return C


def lnocc_gemm_noalloc(precision, A, B, C, stream=None):
    """C = A @ B.T through the contraction engine using the library's fixed scratch (no device allocation)."""
    M, K = A.shape
    N = B.shape[0]
    _check(load().lnocc_gemm_noalloc(precision, M, N, K, _ptr(A), _ptr(B), _ptr(C), _stream(stream)))
    return C

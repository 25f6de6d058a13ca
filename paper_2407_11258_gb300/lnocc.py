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
LNOCC_GUESS_MP2, LNOCC_GUESS_GIVEN, LNOCC_GUESS_MLP = 0, 1, 2
LNOCC_FAULT_NAN_INPUT, LNOCC_FAULT_ZERO_DIIS = 1, 2
LNOCC_TK_AUTO, LNOCC_TK_PER_TERM, LNOCC_TK_GROUPED = 0, 1, 2
LNOCC_MEM_CACHED, LNOCC_MEM_DIRECT = 0, 1

ERR_NAMES = {0: "LNOCC_OK", 1: "LNOCC_EINVAL", 2: "LNOCC_ENOMEM", 3: "LNOCC_ENOCONV", 4: "LNOCC_ENUMERIC",
             5: "LNOCC_ETIMEOUT", 6: "LNOCC_ECUDA"}

LNOCC_ORDER_LPT, LNOCC_ORDER_INPUT = 0, 1
LNOCC_LNO_MP2, LNOCC_LNO_CBNO = 0, 1
NFEAT = 8  # features per amplitude of the learned guess: X is [n][8]

EXPORTS = ["lnocc_default_opts", "lnocc_build_ints", "lnocc_ccsd", "lnocc_fragment_energy", "lnocc_triples",
           "lnocc_debug_gemm", "lnocc_gemm_noalloc", "lnocc_frag_info", "lnocc_free_fragment", "lnocc_last_error",
           "lnocc_version", "lnocc_default_batch_opts", "lnocc_solve_batch", "lnocc_autotune", "lnocc_autotune_save",
           "lnocc_autotune_load", "lnocc_autotune_stats", "lnocc_mlp_nparams", "lnocc_mlp_create", "lnocc_mlp_free",
           "lnocc_mlp_get", "lnocc_mlp_set_norm", "lnocc_mlp_samples", "lnocc_mlp_fit_norm", "lnocc_mlp_train_step",
           "lnocc_mlp_forward", "lnocc_mlp_grad", "lnocc_mlp_guess", "lnocc_frag_set_mlp", "lnocc_mp2_workspace_bytes",
           "lnocc_mp2_energy", "lnocc_workspace_bytes", "lnocc_frag_set_workspace", "lnocc_debug_wait",
           "lnocc_lno_internal", "lnocc_lno_densities", "lnocc_lno_select", "lnocc_active_space",
           "lnocc_kpoint_df", "lnocc_trim_pool", "lnocc_fragment_energy_device", "lnocc_triples_device"]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("max_iter", ctypes.c_int), ("diis_space", ctypes.c_int),
                ("n_refine", ctypes.c_int), ("conv_rms", ctypes.c_double), ("conv_energy", ctypes.c_double),
                ("fault_inject", ctypes.c_int), ("verbose", ctypes.c_int), ("graph", ctypes.c_int),
                ("triples_chunk_mb", ctypes.c_int), ("triples_kernel", ctypes.c_int), ("memory", ctypes.c_int),
                ("reserved", ctypes.c_int * 2)]


class Info(ctypes.Structure):
    _fields_ = [("nocc", ctypes.c_int), ("nvir", ctypes.c_int), ("naux", ctypes.c_int), ("precision", ctypes.c_int),
                ("n_iter", ctypes.c_int), ("converged", ctypes.c_int), ("e_mp2", ctypes.c_double),
                ("e_ccsd", ctypes.c_double), ("last_rms", ctypes.c_double), ("model_flops_ccsd", ctypes.c_double),
                ("model_flops_t", ctypes.c_double), ("exec_flops", ctypes.c_double),
                ("gemm_launches", ctypes.c_longlong), ("device_bytes", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_longlong), ("t_triples_gemm_ms", ctypes.c_double),
                ("t_triples_ms", ctypes.c_double), ("device_allocs", ctypes.c_longlong),
                ("floor_spread", ctypes.c_double), ("n_refined", ctypes.c_int), ("diis_restarts", ctypes.c_int)]


class BatchItem(ctypes.Structure):
    _fields_ = [("nocc", ctypes.c_int), ("nvir", ctypes.c_int), ("naux", ctypes.c_int), ("nlo", ctypes.c_int),
                ("eps", ctypes.c_void_p), ("B", ctypes.c_void_p), ("U_frag", ctypes.c_void_p)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int), ("triples", ctypes.c_int), ("order", ctypes.c_int),
                ("autotune", ctypes.c_int), ("mem_budget_gb", ctypes.c_double), ("reserved", ctypes.c_int * 8)]


class BatchResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("n_iter", ctypes.c_int), ("worker", ctypes.c_int), ("order", ctypes.c_int),
                ("e_mp2", ctypes.c_double), ("e_ccsd", ctypes.c_double), ("e_mp2_frag", ctypes.c_double),
                ("e_ccsd_frag", ctypes.c_double), ("e_t", ctypes.c_double), ("e_t_frag", ctypes.c_double),
                ("t_start_ms", ctypes.c_double), ("t_end_ms", ctypes.c_double), ("model_flops", ctypes.c_double),
                ("device_bytes", ctypes.c_longlong), ("cost_estimate", ctypes.c_double),
                ("bytes_estimate", ctypes.c_longlong)]


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
    lib.lnocc_trim_pool.argtypes = []
    lib.lnocc_fragment_energy_device.argtypes = [P, I, P, P, P]
    lib.lnocc_triples_device.argtypes = [P, I, P, P, P, P]
    lib.lnocc_default_batch_opts.argtypes = [ctypes.POINTER(BatchOpts)]
    lib.lnocc_default_batch_opts.restype = None
    lib.lnocc_solve_batch.argtypes = [I, ctypes.POINTER(BatchItem), ctypes.POINTER(Opts), ctypes.POINTER(BatchOpts),
                                      ctypes.POINTER(BatchResult), P]
    lib.lnocc_solve_batch.restype = I
    LL = ctypes.POINTER(ctypes.c_longlong)
    lib.lnocc_autotune.argtypes = [I, ctypes.POINTER(I)]
    lib.lnocc_autotune_save.argtypes = [ctypes.c_char_p]
    lib.lnocc_autotune_load.argtypes = [ctypes.c_char_p]
    lib.lnocc_autotune_stats.argtypes = [LL, LL, LL, LL]
    for name in ("lnocc_autotune", "lnocc_autotune_save", "lnocc_autotune_load", "lnocc_autotune_stats"):
        getattr(lib, name).restype = I
    F = ctypes.c_float
    lib.lnocc_mlp_nparams.argtypes = []
    lib.lnocc_mlp_create.argtypes = [ctypes.POINTER(F), ctypes.POINTER(P)]
    lib.lnocc_mlp_free.argtypes = [P]
    lib.lnocc_mlp_get.argtypes = [P, ctypes.POINTER(F), ctypes.POINTER(D)]
    lib.lnocc_mlp_set_norm.argtypes = [P, ctypes.POINTER(D)]
    lib.lnocc_mlp_samples.argtypes = [P, I, P, P, P, P]
    lib.lnocc_mlp_fit_norm.argtypes = [P, I, P, P, P]
    lib.lnocc_mlp_train_step.argtypes = [P, I, P, P, F, ctypes.POINTER(D), P]
    lib.lnocc_mlp_forward.argtypes = [P, I, I, P, P, P]
    lib.lnocc_mlp_grad.argtypes = [P, I, I, P, P, P, ctypes.POINTER(D), P]
    lib.lnocc_mlp_guess.argtypes = [P, P, P, P]
    lib.lnocc_frag_set_mlp.argtypes = [P, P]
    for name in ("lnocc_mlp_nparams", "lnocc_mlp_create", "lnocc_mlp_free", "lnocc_mlp_get", "lnocc_mlp_set_norm",
                 "lnocc_mlp_samples", "lnocc_mlp_fit_norm", "lnocc_mlp_train_step", "lnocc_mlp_forward",
                 "lnocc_mlp_grad", "lnocc_mlp_guess", "lnocc_frag_set_mlp"):
        getattr(lib, name).restype = I
    lib.lnocc_lno_internal.argtypes = [I, I, P, P, D, P, P, ctypes.POINTER(I), P]
    lib.lnocc_lno_densities.argtypes = [I, I, I, I, I, P, P, I, P, P, I, P, P, P, P, P]
    lib.lnocc_lno_select.argtypes = [I, P, I, P, D, P, P, ctypes.POINTER(I), P]
    lib.lnocc_active_space.argtypes = [I, I, I, I, P, P, I, P, I, P, P, P, P, P]
    for name in ("lnocc_lno_internal", "lnocc_lno_densities", "lnocc_lno_select", "lnocc_active_space"):
        getattr(lib, name).restype = I
    lib.lnocc_kpoint_df.argtypes = [I, I, I, P, ctypes.POINTER(I), P, ctypes.POINTER(D), P]
    lib.lnocc_kpoint_df.restype = I
    lib.lnocc_debug_wait.argtypes = [I, ctypes.c_longlong, LL, P]
    lib.lnocc_debug_wait.restype = I
    lib.lnocc_workspace_bytes.argtypes = [I, I, I, ctypes.POINTER(Opts), LL]
    lib.lnocc_frag_set_workspace.argtypes = [P, P, ctypes.c_longlong]
    for name in ("lnocc_workspace_bytes", "lnocc_frag_set_workspace"):
        getattr(lib, name).restype = I
    lib.lnocc_mp2_workspace_bytes.argtypes = [I, I, I, I, LL]
    lib.lnocc_mp2_energy.argtypes = [I, I, I, I, P, P, P, ctypes.c_longlong, ctypes.POINTER(D), P]
    for name in ("lnocc_mp2_workspace_bytes", "lnocc_mp2_energy"):
        getattr(lib, name).restype = I
    lib.lnocc_last_error.restype = ctypes.c_char_p
    lib.lnocc_version.restype = ctypes.c_char_p
    for name in ("lnocc_build_ints", "lnocc_ccsd", "lnocc_fragment_energy", "lnocc_triples", "lnocc_debug_gemm",
                 "lnocc_gemm_noalloc", "lnocc_frag_info", "lnocc_free_fragment"):
        getattr(lib, name).restype = I
    _lib = lib
    return lib


def _ptr(x, dtype=None):
    """Device pointer of a contiguous CUDA tensor (float64 unless dtype names another torch dtype)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    import torch
    want = dtype if dtype is not None else torch.float64
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == want and x.is_contiguous()):
        raise TypeError(f"expected a contiguous {want} CUDA tensor")
    return x.data_ptr()


def _need(x, n, what):
    """Reject an array argument whose element count differs from what the C entry point reads or
    writes through its pointer (the kernels index by the declared sizes, so a shorter tensor would be
    read or written past its end). None and raw integer pointers are passed through unchecked."""
    if x is None or isinstance(x, int):
        return
    got = int(x.numel()) if hasattr(x, "numel") else int(x.size)
    if got != int(n):
        raise ValueError(f"{what}: expected {int(n)} elements, got {got}")


def _rows(U, nocc, what="U_frag"):
    """U_frag is [nocc][nlo]: two dimensions, nocc rows."""
    if U is None or isinstance(U, int):
        return
    if U.dim() != 2 or int(U.shape[0]) != int(nocc):
        raise ValueError(f"{what}: expected shape [{nocc}][nlo], got {tuple(U.shape)}")


def _dims(frag):
    """(nocc, nvir) of a fragment handle."""
    if getattr(frag, "dims", None) is None:
        inf = frag.info()
        frag.dims = (inf.nocc, inf.nvir)
    return frag.dims


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def _check(code, ok=(LNOCC_OK,)):
    if code not in ok:
        raise LnoccError(code, load().lnocc_last_error().decode())
    return code


def lnocc_trim_pool():
    """Return the unused memory of the library's cached device pool to the device."""
    _check(load().lnocc_trim_pool())


def default_opts(**kw) -> Opts:
    o = Opts()
    load().lnocc_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Fragment:
    """Owns an lnocc_frag handle; methods mirror the C entry points."""

    def __init__(self, handle, dims=None):
        self.h = handle
        self.dims = dims  # (nocc, nvir)

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
    if nocc > 0 and nvir > 0 and naux > 0:  # (other sizes are rejected by the library itself)
        n = nocc + nvir
        _need(eps, n, "eps")
        _need(B, naux * n * n, "B")
    h = ctypes.c_void_p()
    code = load().lnocc_build_ints(nocc, nvir, naux, _ptr(eps), _ptr(B), ctypes.byref(opts) if opts else None,
                                   _stream(stream), ctypes.byref(h))
    _check(code)
    return Fragment(h, (nocc, nvir))


def lnocc_ccsd(frag: Fragment, t1_in=None, t2_in=None, guess_mode=LNOCC_GUESS_MP2, t1_out=None, t2_out=None,
               stream=None, allow_noconv=False):
    """Returns (e_corr, n_iter, status)."""
    o, v = _dims(frag)
    for x, n, what in ((t1_in, o * v, "t1_in"), (t2_in, o * o * v * v, "t2_in"), (t1_out, o * v, "t1_out"),
                       (t2_out, o * o * v * v, "t2_out")):
        _need(x, n, what)
    e = ctypes.c_double(0.0)
    it = ctypes.c_int(0)
    code = load().lnocc_ccsd(frag.h, _ptr(t1_in), _ptr(t2_in), guess_mode, _ptr(t1_out), _ptr(t2_out),
                             ctypes.byref(e), ctypes.byref(it), _stream(stream))
    _check(code, (LNOCC_OK, LNOCC_ENOCONV) if allow_noconv else (LNOCC_OK,))
    return e.value, it.value, code


def lnocc_fragment_energy(frag: Fragment, U_frag, stream=None, ccsd=True):
    """Returns (e_ccsd_frag, e_mp2_frag); U_frag is [nocc][nlo]. ccsd=False asks for the MP2 fragment
    energy only (no lnocc_ccsd needed; e_ccsd_frag is then None)."""
    _rows(U_frag, _dims(frag)[0])
    ec, em = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().lnocc_fragment_energy(frag.h, int(U_frag.shape[1]), _ptr(U_frag),
                                        ctypes.byref(ec) if ccsd else None, ctypes.byref(em), _stream(stream)))
    return (ec.value if ccsd else None), em.value


def lnocc_triples(frag: Fragment, U_frag=None, stream=None):
    """Returns (e_t_full, e_t_frag)."""
    _rows(U_frag, _dims(frag)[0])
    ef, eF = ctypes.c_double(0.0), ctypes.c_double(0.0)
    nlo = int(U_frag.shape[1]) if U_frag is not None else 0
    _check(load().lnocc_triples(frag.h, nlo, _ptr(U_frag), ctypes.byref(ef), ctypes.byref(eF), _stream(stream)))
    return ef.value, eF.value


def lnocc_fragment_energy_device(frag: Fragment, U_frag, e_dev, stream=None):
    """Enqueue the projected CCSD and MP2 energies into e_dev (float64 CUDA tensor of 2 elements) without
    synchronising (graph-capturable)."""
    _rows(U_frag, _dims(frag)[0])
    _need(e_dev, 2, "e_dev")
    _check(load().lnocc_fragment_energy_device(frag.h, int(U_frag.shape[1]), _ptr(U_frag), _ptr(e_dev),
                                               _stream(stream)))


def lnocc_triples_device(frag: Fragment, U_frag, e_dev, status_dev=None, stream=None):
    """Enqueue the (T) energy and its projection into e_dev (float64 CUDA tensor of 2 elements) and the
    device status word into status_dev (int32 CUDA tensor of 1 element, optional) without synchronising
    (graph-capturable; needs an attached workspace)."""
    import torch
    _rows(U_frag, _dims(frag)[0])
    _need(e_dev, 2, "e_dev")
    _need(status_dev, 1, "status_dev")
    nlo = int(U_frag.shape[1]) if U_frag is not None else 0
    _check(load().lnocc_triples_device(frag.h, nlo, _ptr(U_frag), _ptr(e_dev),
                                       _ptr(status_dev, torch.int32) if status_dev is not None else None,
                                       _stream(stream)))


def lnocc_workspace_bytes(nocc, nvir, naux, opts=None):
    """Device scratch (bytes) lnocc_triples needs for a fragment of these sizes and options."""
    b = ctypes.c_longlong(0)
    _check(load().lnocc_workspace_bytes(nocc, nvir, naux, ctypes.byref(opts) if opts else None, ctypes.byref(b)))
    return b.value


def lnocc_frag_set_workspace(frag: Fragment, workspace):
    """Attach a caller-owned CUDA tensor (at least lnocc_workspace_bytes bytes) as the (T) scratch, or
    detach with None. The fragment keeps a reference so the tensor outlives its use."""
    if workspace is None:
        _check(load().lnocc_frag_set_workspace(frag.h, None, 0))
        frag.workspace = None
        return
    import torch
    if not (isinstance(workspace, torch.Tensor) and workspace.is_cuda and workspace.is_contiguous()):
        raise TypeError("workspace: expected a contiguous CUDA tensor")
    _check(load().lnocc_frag_set_workspace(frag.h, workspace.data_ptr(),
                                           workspace.numel() * workspace.element_size()))
    frag.workspace = workspace


def lnocc_debug_gemm(precision, A, B, C, stream=None):
    """C = A @ B.T through the contraction engine (diagnostic)."""
    M, K = A.shape
    N = B.shape[0]
    _need(B, N * K, "B")
    _need(C, M * N, "C")
    _check(load().lnocc_debug_gemm(precision, M, N, K, _ptr(A), _ptr(B), _ptr(C), _stream(stream)))
    return C


def lnocc_debug_wait(arrive, budget_ns, stream=None):
    """Bounded-wait diagnostic: returns (status code, nanoseconds the kernel waited); never raises on
    LNOCC_ETIMEOUT, which is the expected result with arrive=False."""
    w = ctypes.c_longlong(0)
    code = load().lnocc_debug_wait(1 if arrive else 0, int(budget_ns), ctypes.byref(w), _stream(stream))
    _check(code, (LNOCC_OK, LNOCC_ETIMEOUT))
    return code, w.value


def lnocc_gemm_noalloc(precision, A, B, C, stream=None):
    """C = A @ B.T through the contraction engine using the library's fixed scratch (no device allocation)."""
    M, K = A.shape
    N = B.shape[0]
    _need(B, N * K, "B")
    _need(C, M * N, "C")
    _check(load().lnocc_gemm_noalloc(precision, M, N, K, _ptr(A), _ptr(B), _ptr(C), _stream(stream)))
    return C


def lnocc_mp2_workspace_bytes(precision, nocc, nvir, naux):
    b = ctypes.c_longlong(0)
    _check(load().lnocc_mp2_workspace_bytes(precision, nocc, nvir, naux, ctypes.byref(b)))
    return b.value


def lnocc_mp2_energy(precision, nocc, nvir, naux, eps, B_ov, workspace=None, stream=None):
    """Full-system MP2 correlation energy (Eq. 17's first term) from the ov block B_ov [naux][nocc][nvir].
    workspace: None (the library allocates) or a CUDA tensor of at least lnocc_mp2_workspace_bytes bytes."""
    _need(eps, nocc + nvir, "eps")
    _need(B_ov, naux * nocc * nvir, "B_ov")
    ws, wsb = None, 0
    if workspace is not None:
        import torch
        if not (isinstance(workspace, torch.Tensor) and workspace.is_cuda and workspace.is_contiguous()):
            raise TypeError("workspace: expected a contiguous CUDA tensor")
        ws, wsb = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    e = ctypes.c_double(0.0)
    _check(load().lnocc_mp2_energy(precision, nocc, nvir, naux, _ptr(eps), _ptr(B_ov), ws, wsb, ctypes.byref(e),
                                   _stream(stream)))
    return e.value


# ------------------------------------------------------------------------------ local active space
def _empty(*shape, like):
    import torch
    return torch.zeros(*shape, dtype=torch.float64, device=like.device)


def lnocc_lno_internal(U, e, sv_tol=1e-10, stream=None):
    """Internal orbitals of one block (Eq. 18-19), semi-canonical. U [n][nlo], e [n]. Returns
    (W_int [n][n_int], f_int [n_int], n_int) as new CUDA tensors (contiguous)."""
    n, nlo = U.shape
    _need(e, n, "e")
    W = _empty(n, nlo, like=U)
    f = _empty(nlo, like=U)
    ni = ctypes.c_int(0)
    _check(load().lnocc_lno_internal(n, nlo, _ptr(U), _ptr(e), sv_tol, _ptr(W), _ptr(f), ctypes.byref(ni),
                                     _stream(stream)))
    k = ni.value
    return W[:, :k].contiguous(), f[:k].contiguous(), k


def lnocc_lno_densities(precision, kind, nocc, nvir, naux, eps, B_ov, W_occ, f_occ, W_vir=None, f_vir=None,
                        stream=None):
    """D_occ [nocc][nocc], D_vir [nvir][nvir] (Eq. 20 for kind LNOCC_LNO_MP2, Eq. 28 for LNOCC_LNO_CBNO)."""
    _need(eps, nocc + nvir, "eps")
    _need(B_ov, naux * nocc * nvir, "B_ov")
    n_io = int(W_occ.shape[1])
    _need(W_occ, nocc * n_io, "W_occ")
    _need(f_occ, n_io, "f_occ")
    n_iv = int(W_vir.shape[1]) if W_vir is not None else 0
    if W_vir is not None:
        _need(W_vir, nvir * n_iv, "W_vir")
        _need(f_vir, n_iv, "f_vir")
    Do = _empty(nocc, nocc, like=B_ov)
    Dv = _empty(nvir, nvir, like=B_ov)
    _check(load().lnocc_lno_densities(precision, kind, nocc, nvir, naux, _ptr(eps), _ptr(B_ov), n_io, _ptr(W_occ),
                                      _ptr(f_occ), n_iv, _ptr(W_vir), _ptr(f_vir), _ptr(Do), _ptr(Dv),
                                      _stream(stream)))
    return Do, Dv


def lnocc_lno_select(D, W_int=None, eta=0.0, stream=None):
    """LNOs of Eq. 24-26: returns (C [n][n_keep], lambda [n_keep], n_keep)."""
    n = int(D.shape[0])
    _need(D, n * n, "D")
    n_int = int(W_int.shape[1]) if W_int is not None else 0
    if W_int is not None:
        _need(W_int, n * n_int, "W_int")
    C = _empty(n, n, like=D)
    lam = _empty(n, like=D)
    k = ctypes.c_int(0)
    _check(load().lnocc_lno_select(n, _ptr(D), n_int, _ptr(W_int), float(eta), _ptr(C), _ptr(lam), ctypes.byref(k),
                                   _stream(stream)))
    return C[:, :k.value].contiguous(), lam[:k.value].contiguous(), k.value


def lnocc_active_space(precision, nocc, nvir, naux, eps, B, C_occ, C_vir, stream=None):
    """Semi-canonical active space: returns (eps_F [nF], B_F [naux][nF][nF], C_F [n][nF])."""
    n = nocc + nvir
    no, nv = int(C_occ.shape[1]), int(C_vir.shape[1])
    _need(eps, n, "eps")
    _need(B, naux * n * n, "B")
    _need(C_occ, nocc * no, "C_occ")
    _need(C_vir, nvir * nv, "C_vir")
    nF = no + nv
    eF = _empty(nF, like=B)
    BF = _empty(naux, nF, nF, like=B)
    CF = _empty(n, nF, like=B)
    _check(load().lnocc_active_space(precision, nocc, nvir, naux, _ptr(eps), _ptr(B), no, _ptr(C_occ), nv,
                                     _ptr(C_vir), _ptr(eF), _ptr(BF), _ptr(CF), _stream(stream)))
    return eF, BF, CF


def lnocc_kpoint_df(L, qneg, stream=None):
    """Real DF factors B [nk * naux][n][n] (CUDA float64) of the q-sum of Eq. 27a from complex k-point factors
    L [nk][naux][n][n] (CUDA complex128) and the -q index map qneg (sequence of nk ints).
    Returns (B, relative symmetry error)."""
    import torch
    if not (isinstance(L, torch.Tensor) and L.is_cuda and L.dtype == torch.complex128 and L.is_contiguous()):
        raise TypeError("L: expected a contiguous complex128 CUDA tensor")
    nk, naux, n, n2 = (int(x) for x in L.shape)
    if n2 != n or len(qneg) != nk:
        raise ValueError("L must be [nk][naux][n][n] and qneg of length nk")
    q = (ctypes.c_int * nk)(*[int(x) for x in qneg])
    B = torch.empty(nk * naux, n, n, dtype=torch.float64, device=L.device)
    err = ctypes.c_double(0.0)
    _check(load().lnocc_kpoint_df(nk, naux, n, L.data_ptr(), q, _ptr(B), ctypes.byref(err), _stream(stream)))
    return B, err.value


def default_batch_opts(**kw) -> BatchOpts:
    b = BatchOpts()
    load().lnocc_default_batch_opts(ctypes.byref(b))
    for k, v in kw.items():
        setattr(b, k, v)
    return b


def lnocc_solve_batch(frags, opts=None, bopts=None, stream=None, allow_noconv=False):
    """Solve independent fragments. frags: sequence of (nocc, nvir, naux, eps, B, U_frag or None), device
    tensors as for lnocc_build_ints. Returns (status, [BatchResult per fragment])."""
    n = len(frags)
    items = (BatchItem * max(n, 1))()
    for k, (o, v, q, eps, B, U) in enumerate(frags):  # every item checked before any pointer is taken
        if o > 0 and v > 0 and q > 0:
            _need(eps, o + v, f"item {k} eps")
            _need(B, q * (o + v) ** 2, f"item {k} B")
            _rows(U, o, f"item {k} U_frag")
    for k, (o, v, q, eps, B, U) in enumerate(frags):
        items[k] = BatchItem(o, v, q, int(U.shape[1]) if U is not None else 0, _ptr(eps), _ptr(B), _ptr(U))
    res = (BatchResult * max(n, 1))()
    code = load().lnocc_solve_batch(n, items, ctypes.byref(opts) if opts else None,
                                    ctypes.byref(bopts) if bopts else None, res, _stream(stream))
    _check(code, (LNOCC_OK, LNOCC_ENOCONV) if allow_noconv else (LNOCC_OK,))
    return code, [res[k] for k in range(n)]


def lnocc_autotune(mode=-1):
    """Set the tile autotuner mode (0 fixed rule, 1 table, 2 tune misses); returns the previous mode."""
    prev = ctypes.c_int(0)
    _check(load().lnocc_autotune(mode, ctypes.byref(prev)))
    return prev.value


def lnocc_autotune_save(path):
    _check(load().lnocc_autotune_save(os.fsencode(path)))


def lnocc_autotune_load(path):
    _check(load().lnocc_autotune_load(os.fsencode(path)))


def lnocc_autotune_stats():
    """Returns dict(entries, hits, misses, tuned)."""
    v = [ctypes.c_longlong(0) for _ in range(4)]
    _check(load().lnocc_autotune_stats(*[ctypes.byref(x) for x in v]))
    return dict(zip(("entries", "hits", "misses", "tuned"), (x.value for x in v)))


# ------------------------------------------------------------------------------ learned T2 guess
class Mlp:
    """Owns an lnocc_mlp handle (parameters, Adam state and workspace on the device)."""

    def __init__(self, params):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != load().lnocc_mlp_nparams():
            raise ValueError(f"expected {load().lnocc_mlp_nparams()} parameters, got {p.size}")
        self.h = ctypes.c_void_p()
        _check(load().lnocc_mlp_create(p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(self.h)))

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "h", None):
            load().lnocc_mlp_free(self.h)
            self.h = None

    def get(self):
        """(params float32[nparams], norm float64[17]) as numpy arrays."""
        import numpy as np
        p = np.zeros(load().lnocc_mlp_nparams(), dtype=np.float32)
        nrm = np.zeros(17)
        _check(load().lnocc_mlp_get(self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                    nrm.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return p, nrm

    def set_norm(self, norm):
        import numpy as np
        nrm = np.ascontiguousarray(norm, dtype=np.float64)
        _need(nrm, 17, "norm")
        _check(load().lnocc_mlp_set_norm(self.h, nrm.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def fit_norm(self, X, dt, stream=None):
        import torch
        _need(X, X.shape[0] * NFEAT, "X")
        _need(dt, X.shape[0], "dt")
        _check(load().lnocc_mlp_fit_norm(self.h, X.shape[0], _ptr(X, torch.float32), _ptr(dt, torch.float32),
                                         _stream(stream)))

    def train_step(self, X, dt, lr, stream=None):
        import torch
        _need(X, X.shape[0] * NFEAT, "X")
        _need(dt, X.shape[0], "dt")
        loss = ctypes.c_double(0.0)
        _check(load().lnocc_mlp_train_step(self.h, X.shape[0], _ptr(X, torch.float32), _ptr(dt, torch.float32),
                                           lr, ctypes.byref(loss), _stream(stream)))
        return loss.value

    def forward(self, X, precision=LNOCC_PREC_FP64, stream=None):
        import torch
        _need(X, X.shape[0] * NFEAT, "X")
        y = torch.empty(X.shape[0], dtype=torch.float64, device=X.device)
        _check(load().lnocc_mlp_forward(self.h, precision, X.shape[0], _ptr(X, torch.float32), _ptr(y),
                                        _stream(stream)))
        return y

    def grad(self, X, dt, precision=LNOCC_PREC_FP64, stream=None):
        import torch
        _need(X, X.shape[0] * NFEAT, "X")
        _need(dt, X.shape[0], "dt")
        g = torch.empty(load().lnocc_mlp_nparams(), dtype=torch.float64, device=X.device)
        loss = ctypes.c_double(0.0)
        _check(load().lnocc_mlp_grad(self.h, precision, X.shape[0], _ptr(X, torch.float32), _ptr(dt, torch.float32),
                                     _ptr(g), ctypes.byref(loss), _stream(stream)))
        return loss.value, g


def lnocc_mlp_samples(frag: Fragment, idx, X, dt=None, stream=None):
    """Features X [n][8] (float32) and targets dt [n] (float32) of flat amplitude indices idx (int64)."""
    import torch
    n = idx.shape[0]
    _need(idx, n, "idx")
    _need(X, n * NFEAT, "X")
    _need(dt, n, "dt")
    _check(load().lnocc_mlp_samples(frag.h, idx.shape[0], _ptr(idx, torch.int64), _ptr(X, torch.float32),
                                    _ptr(dt, torch.float32), _stream(stream)))


def lnocc_mlp_guess(frag: Fragment, mlp: Mlp, t2_out, stream=None):
    o, v = _dims(frag)
    _need(t2_out, o * o * v * v, "t2_out")
    _check(load().lnocc_mlp_guess(frag.h, mlp.h, _ptr(t2_out), _stream(stream)))
    return t2_out


def lnocc_frag_set_mlp(frag: Fragment, mlp):
    _check(load().lnocc_frag_set_mlp(frag.h, mlp.h if mlp is not None else None))

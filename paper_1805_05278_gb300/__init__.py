"""Python binding of libgbqr (include/gbqr.h): recursive Householder QR
(QR-EG with a TSQR base case) and least squares on one GB300.

Argument marshalling only.  The module-level ``gbqr_*`` functions mirror the
C ABI one to one (same names, raw pointers and sizes); ``Context`` wraps them
for torch tensors, passing ``data_ptr()`` and the current CUDA stream.  Every
step of the computation runs in the library's CUDA kernels.  If the library is
not built, ``load()`` raises: there is no fallback path.

Matrices are column-major float64.  A torch tensor ``X`` of shape (m, n) is
accepted when ``X.stride(0) == 1`` (a Fortran-ordered view, e.g. the ``.T`` of
a contiguous (n, m) tensor); its leading dimension is ``X.stride(1)``.
"""

from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgbqr.so")

# status codes (gbqr_status)
GBQR_OK, GBQR_EINVAL, GBQR_ENOMEM, GBQR_ECUDA, GBQR_ETIMEOUT = 0, 1, 2, 3, 4
GBQR_ENONFINITE, GBQR_ERANKDEF, GBQR_EBUSY, GBQR_EUNSUPPORTED, GBQR_ENOCONV = 5, 6, 7, 8, 9
# T layouts (gbqr_t_layout) and precisions (gbqr_prec)
GBQR_T_FULL, GBQR_T_PANEL = 0, 1
GBQR_FP64, GBQR_MIXED_BF16, GBQR_MIXED_SPLITBF16, GBQR_FP32, GBQR_PREC_AUTO = 0, 1, 2, 3, 4
GBQR_GEMM_DMMA, GBQR_GEMM_DFMA = 1, 2
GBQR_TUNE_FACTOR, GBQR_TUNE_BATCHED = 0, 1
GBQR_REQ_QUEUED, GBQR_REQ_RUNNING, GBQR_REQ_DONE = 0, 1, 2

_I64 = ctypes.c_int64
_P = ctypes.c_void_p


class gbqr_opts(ctypes.Structure):
    _fields_ = [("cutoff_b", ctypes.c_int32), ("panel_nb", ctypes.c_int32),
                ("leaf_rows", ctypes.c_int32), ("fanout", ctypes.c_int32),
                ("lookahead", ctypes.c_int32), ("update_prec", ctypes.c_int32), ("batch_streams", ctypes.c_int32),
                ("fp64_gemm", ctypes.c_int32)]


class gbqr_info(ctypes.Structure):
    _fields_ = [("nonfinite", ctypes.c_int64), ("zero_pivots", ctypes.c_int64),
                ("rankdef_col", ctypes.c_int64), ("refine_iters", ctypes.c_int64),
                ("refine_last", ctypes.c_double), ("gmres_steps", ctypes.c_int64),
                ("backward_err", ctypes.c_double), ("reserved", ctypes.c_int64 * 1)]


class gbqr_request(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("A", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("b", ctypes.c_void_p), ("x", ctypes.c_void_p), ("prec", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("tag", ctypes.c_uint64)]


class gbqr_result(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("prec_used", ctypes.c_int32),
                ("fell_back", ctypes.c_int32), ("refine_iters", ctypes.c_int64), ("queue_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double), ("latency_ms", ctypes.c_double), ("footprint_bytes", ctypes.c_int64),
                ("tag", ctypes.c_uint64), ("bypassed", ctypes.c_int32), ("pad2", ctypes.c_int32)]


class gbqr_trace_rec(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


# name -> (restype, argtypes): the declarations of include/gbqr.h
SIGNATURES = {
    "gbqr_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _P]),
    "gbqr_destroy": (ctypes.c_int, [_P]),
    "gbqr_set_stream": (ctypes.c_int, [_P, _P]),
    "gbqr_set_workspace": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "gbqr_workspace_bytes": (ctypes.c_size_t, [_I64, _I64, ctypes.c_int, ctypes.POINTER(gbqr_opts)]),
    "gbqr_sync": (ctypes.c_int, [_P, ctypes.POINTER(gbqr_info)]),
    "gbqr_factor": (ctypes.c_int, [_P, _I64, _I64, _P, _I64, _P, _I64, ctypes.c_int, ctypes.POINTER(gbqr_opts)]),
    "gbqr_default_panel_nb": (_I64, [_I64, _I64]),
    "gbqr_factor_f32": (ctypes.c_int, [_P, _I64, _I64, _P, _I64, _P, _I64, ctypes.c_int, ctypes.POINTER(gbqr_opts)]),
    "gbqr_apply_qt": (ctypes.c_int, [_P, _I64, _I64, _P, _I64, _P, _I64, ctypes.c_int, _I64, _I64, _P, _I64]),
    "gbqr_apply_q": (ctypes.c_int, [_P, _I64, _I64, _P, _I64, _P, _I64, ctypes.c_int, _I64, _I64, _P, _I64]),
    "gbqr_form_q": (ctypes.c_int, [_P, _I64, _I64, _P, _I64, _P, _I64, ctypes.c_int, _I64, _P, _I64]),
    "gbqr_ls_solve": (ctypes.c_int, [_P, _I64, _I64, _P, _I64, _P, _P, ctypes.c_int, ctypes.POINTER(gbqr_info)]),
    "gbqr_gemm_split_bf16": (ctypes.c_int, [_P, ctypes.c_int, _I64, _I64, _I64, ctypes.c_double, _P, _I64, _P, _I64,
                                             ctypes.c_double, _P, _I64, ctypes.c_int]),
    "gbqr_factor_batched": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                            ctypes.POINTER(_P), ctypes.POINTER(_I64), ctypes.POINTER(_P),
                                            ctypes.POINTER(_I64), ctypes.POINTER(gbqr_opts)]),
    "gbqr_factor_batched_f32": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                                ctypes.POINTER(_P), ctypes.POINTER(_I64), ctypes.POINTER(_P),
                                                ctypes.POINTER(_I64), ctypes.POINTER(gbqr_opts)]),
    "gbqr_batched_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                                       ctypes.POINTER(gbqr_opts)]),
    "gbqr_graph_begin": (ctypes.c_int, [_P]),
    "gbqr_graph_end": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
    "gbqr_graph_launch": (ctypes.c_int, [_P, _P]),
    "gbqr_graph_destroy": (ctypes.c_int, [_P]),
    "gbqr_server_start": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_size_t]),
    "gbqr_submit": (ctypes.c_int, [_P, ctypes.POINTER(gbqr_request), ctypes.POINTER(ctypes.c_uint64)]),
    "gbqr_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(gbqr_result)]),
    "gbqr_server_stop": (ctypes.c_int, [_P]),
    "gbqr_trace_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "gbqr_trace_read": (ctypes.c_int, [_P, ctypes.POINTER(gbqr_trace_rec), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "gbqr_launch_count": (_I64, [_P]),
    "gbqr_tsqr_static": (ctypes.c_int, [_I64, _I64, _P, _I64, _P, _I64, _P]),
    "gbqr_autotune": (ctypes.c_int, [_P, _I64, _I64, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.POINTER(gbqr_opts), ctypes.POINTER(ctypes.c_double)]),
    "gbqr_autotune_batched": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.c_int,
                                             ctypes.c_double, ctypes.POINTER(gbqr_opts), ctypes.POINTER(ctypes.c_double)]),
    "gbqr_tuned_lookup": (ctypes.c_int, [_P, ctypes.c_int, _I64, _I64, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(gbqr_opts)]),
    "gbqr_fp64_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "gbqr_selftest_wait_timeout": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "gbqr_selftest_batched_wait": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "gbqr_selftest_chain_wait": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "gbqr_strerror": (ctypes.c_char_p, [ctypes.c_int]),
}

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the CUDA library for sm_103a (nvcc); returns its path."""
    from . import buildlib
    return buildlib.build(force=force)


def load(path: str | None = None):
    """Load libgbqr.so and bind every C ABI function into this module."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libgbqr.so is not built ({p}); run paper_1805_05278_gb300.build()")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
            globals()[name] = f
        _lib = lib
        return lib


class GbqrError(RuntimeError):
    def __init__(self, status: int, what: str):
        load()
        msg = gbqr_strerror(status).decode()  # noqa: F821 (bound by load)
        super().__init__(f"{what}: {msg} (status {status})")
        self.status = status


def check(status: int, what: str) -> int:
    if status != GBQR_OK:
        raise GbqrError(status, what)
    return status


def opts(cutoff_b: int = 0, panel_nb: int = 0, leaf_rows: int = 0, fanout: int = 0,
         lookahead: int = 0, update_prec: int = GBQR_FP64, batch_streams: int = 0,
         fp64_gemm: int = 0) -> gbqr_opts:
    o = gbqr_opts()
    o.cutoff_b, o.panel_nb, o.leaf_rows, o.fanout = cutoff_b, panel_nb, leaf_rows, fanout
    o.lookahead = lookahead
    o.update_prec = update_prec
    o.batch_streams = batch_streams
    o.fp64_gemm = fp64_gemm
    return o


def opts_dict(o: gbqr_opts) -> dict:
    """The fields of a gbqr_opts as a plain dict."""
    return {name: getattr(o, name) for name, _ in gbqr_opts._fields_}


def _cm(x, name: str, dtype=None):
    """(pointer, rows, cols, leading dimension) of a column-major float64 (or
    `dtype`) tensor."""
    import torch
    if x.dtype != (torch.float64 if dtype is None else dtype):
        raise TypeError(f"{name} must be {dtype or torch.float64}")
    if x.dim() == 1:
        return x.data_ptr(), x.shape[0], 1, max(1, x.shape[0])
    if x.dim() != 2 or (x.stride(0) != 1 and x.shape[0] > 1):
        raise ValueError(f"{name} must be a column-major 2-D tensor (stride(0) == 1)")
    return x.data_ptr(), x.shape[0], x.shape[1], max(1, x.stride(1), x.shape[0] if x.shape[1] == 1 else 1)


def colmajor(m: int, n: int, device="cuda", fill=None):
    """A new column-major m x n float64 tensor (optionally filled)."""
    import torch
    t = torch.empty((n, m), dtype=torch.float64, device=device).T
    if fill is not None:
        t.fill_(fill)
    return t


def to_colmajor(a, device="cuda", pin: bool = False):
    """Column-major float64 tensor holding the numpy array a (m x n or m)."""
    import numpy as np
    import torch
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        t = torch.from_numpy(a.copy())
    else:
        t = torch.from_numpy(np.ascontiguousarray(a.T)).T
    if device == "cpu":
        return t.pin_memory() if pin else t
    return t.to(device)


def to_numpy(t):
    """Fortran-ordered numpy copy of a column-major tensor."""
    import numpy as np
    x = t.detach().cpu()
    return np.asfortranarray(x.numpy())


class Context:
    """A gbqr context bound to one CUDA device and stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        load()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = _P()
        check(gbqr_create(ctypes.byref(h), device, _P(stream.cuda_stream)), "gbqr_create")  # noqa: F821
        self.handle = h
        self._workspace = None

    def close(self):
        if getattr(self, "handle", None):
            gbqr_destroy(self.handle)  # noqa: F821
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- workspace / sync / tracing
    def set_workspace(self, tensor):
        """Hand the library a caller-owned workspace (any CUDA tensor)."""
        self._workspace = tensor
        if tensor is None:
            return check(gbqr_set_workspace(self.handle, None, 0), "gbqr_set_workspace")  # noqa: F821
        nbytes = tensor.numel() * tensor.element_size()
        return check(gbqr_set_workspace(self.handle, _P(tensor.data_ptr()), nbytes), "gbqr_set_workspace")  # noqa: F821

    def sync(self):
        info = gbqr_info()
        st = gbqr_sync(self.handle, ctypes.byref(info))  # noqa: F821
        return st, info

    def trace(self, on: bool = True):
        check(gbqr_trace_enable(self.handle, 1 if on else 0), "gbqr_trace_enable")  # noqa: F821

    def trace_read(self) -> dict:
        recs = (gbqr_trace_rec * 8)()
        cnt = ctypes.c_int(0)
        check(gbqr_trace_read(self.handle, recs, 8, ctypes.byref(cnt)), "gbqr_trace_read")  # noqa: F821
        return {r.name.decode(): {"launches": r.launches, "ms": r.ms, "flops": r.flops, "bytes": r.bytes}
                for r in recs[:cnt.value]}

    def launch_count(self) -> int:
        return int(gbqr_launch_count(self.handle))  # noqa: F821

    # ---- computation
    def factor(self, A, T, layout: int = GBQR_T_PANEL, o: gbqr_opts | None = None) -> int:
        """In-place QR of A (column-major m x n); T receives the kernel.
        float32 tensors go to gbqr_factor_f32 (FP32 throughout)."""
        import torch
        dt = A.dtype if A.dtype == torch.float32 else torch.float64
        pa, m, n, lda = _cm(A, "A", dt)
        pt, _, _, ldt = _cm(T, "T", dt)
        fn, nm = ((gbqr_factor_f32, "gbqr_factor_f32") if dt == torch.float32  # noqa: F821
                  else (gbqr_factor, "gbqr_factor"))  # noqa: F821
        return check(fn(self.handle, m, n, _P(pa), lda, _P(pt), ldt, layout,
                        ctypes.byref(o) if o is not None else None), nm)

    def _apply(self, fn, VR, T, layout, nb, B):
        pv, m, n, lda = _cm(VR, "VR")
        pt, _, _, ldt = _cm(T, "T")
        pb, mb, nrhs, ldb = _cm(B, "B")
        return check(fn(self.handle, m, n, _P(pv), lda, _P(pt), ldt, layout, nb, nrhs, _P(pb), ldb), fn.__name__)

    def apply_qt(self, VR, T, B, layout: int = GBQR_T_PANEL, nb: int = 0) -> int:
        return self._apply(gbqr_apply_qt, VR, T, layout, nb, B)  # noqa: F821

    def apply_q(self, VR, T, B, layout: int = GBQR_T_PANEL, nb: int = 0) -> int:
        return self._apply(gbqr_apply_q, VR, T, layout, nb, B)  # noqa: F821

    def form_q(self, VR, T, Q, layout: int = GBQR_T_PANEL, nb: int = 0) -> int:
        pv, m, n, lda = _cm(VR, "VR")
        pt, _, _, ldt = _cm(T, "T")
        pq, _, _, ldq = _cm(Q, "Q")
        return check(gbqr_form_q(self.handle, m, n, _P(pv), lda, _P(pt), ldt, layout, nb, _P(pq), ldq),  # noqa: F821
                     "gbqr_form_q")

    def gemm_split_bf16(self, A, B, C, transa: bool = False, alpha: float = 1.0, beta: float = 0.0,
                        nsplit: int = 3) -> int:
        """C = alpha op(A) B + beta C on the tensor cores (split-BF16)."""
        pa, ra, ca, lda = _cm(A, "A")
        pb, kb, nb_, ldb = _cm(B, "B")
        pc, mc, nc, ldc = _cm(C, "C")
        M, K = (ca, ra) if transa else (ra, ca)
        return check(gbqr_gemm_split_bf16(self.handle, 1 if transa else 0, M, nc, K, alpha, _P(pa), lda,  # noqa: F821
                                          _P(pb), ldb, beta, _P(pc), ldc, nsplit), "gbqr_gemm_split_bf16")

    def factor_batched(self, As, Ts, o: gbqr_opts | None = None) -> int:
        """QR of every column-major matrix in As (in place); Ts[i] receives
        the panel kernels (rows >= min(128, n_i)).  float32 matrices go to
        gbqr_factor_batched_f32 (FP32 throughout), float64 ones to
        gbqr_factor_batched."""
        import torch
        cnt = len(As)
        I64 = _I64 * cnt
        Ps = _P * cnt
        ms, ns, ldas, ldts, pa, pt = I64(), I64(), I64(), I64(), Ps(), Ps()
        dt = As[0].dtype if cnt else torch.float64
        for i, (A, T) in enumerate(zip(As, Ts)):
            a_ptr, m, n, lda = _cm(A, "A", dt)
            t_ptr, _, _, ldt = _cm(T, "T", dt)
            ms[i], ns[i], ldas[i], ldts[i], pa[i], pt[i] = m, n, lda, ldt, a_ptr, t_ptr
        fn, nm = ((gbqr_factor_batched_f32, "gbqr_factor_batched_f32") if dt == torch.float32  # noqa: F821
                  else (gbqr_factor_batched, "gbqr_factor_batched"))  # noqa: F821
        return check(fn(self.handle, cnt, ms, ns, pa, ldas, pt, ldts, ctypes.byref(o) if o is not None else None), nm)

    # ---- autotuner
    def autotune(self, m: int, n: int, layout: int = GBQR_T_PANEL, prec: int = GBQR_FP64,
                 budget_ms: float = 20000.0):
        """gbqr_autotune: returns (best gbqr_opts, its time in ms); the result
        is cached in this context for the shape class."""
        o, ms = gbqr_opts(), ctypes.c_double()
        check(gbqr_autotune(self.handle, m, n, layout, prec, budget_ms,  # noqa: F821
                            ctypes.byref(o), ctypes.byref(ms)), "gbqr_autotune")
        return o, ms.value

    def autotune_batched(self, shapes, prec: int = GBQR_FP64, budget_ms: float = 20000.0):
        """gbqr_autotune_batched over matrices of the given (m, n) shapes."""
        cnt = len(shapes)
        ms_, ns_ = (_I64 * cnt)(*[m for m, _ in shapes]), (_I64 * cnt)(*[n for _, n in shapes])
        o, ms = gbqr_opts(), ctypes.c_double()
        check(gbqr_autotune_batched(self.handle, cnt, ms_, ns_, prec, budget_ms,  # noqa: F821
                                    ctypes.byref(o), ctypes.byref(ms)), "gbqr_autotune_batched")
        return o, ms.value

    def tuned(self, kind: int, m: int = 0, n: int = 0, layout: int = GBQR_T_PANEL, prec: int = GBQR_FP64):
        """The cached tuner result, or None."""
        o = gbqr_opts()
        st = gbqr_tuned_lookup(self.handle, kind, m, n, layout, prec, ctypes.byref(o))  # noqa: F821
        return o if st == GBQR_OK else None

    def capture(self, fn):
        """Run fn() under a capture of this context's stream; returns a Graph."""
        check(gbqr_graph_begin(self.handle), "gbqr_graph_begin")  # noqa: F821
        try:
            fn()
        finally:
            g = _P()
            st = gbqr_graph_end(self.handle, ctypes.byref(g))  # noqa: F821
        check(st, "gbqr_graph_end")
        return Graph(self, g)

    # ---- serving
    def serve(self, workers: int = 16, mem_cap_bytes: int = 120 << 30):
        check(gbqr_server_start(self.handle, self.device, workers, mem_cap_bytes), "gbqr_server_start")  # noqa: F821

    def submit(self, A, b, x, prec: int = GBQR_PREC_AUTO, tag: int = 0) -> int:
        pa, m, n, lda = _cm(A, "A")
        r = gbqr_request(m=m, n=n, A=pa, lda=lda, b=b.data_ptr(), x=x.data_ptr(), prec=prec, pad=0, tag=tag)
        rid = ctypes.c_uint64(0)
        check(gbqr_submit(self.handle, ctypes.byref(r), ctypes.byref(rid)), "gbqr_submit")  # noqa: F821
        return rid.value

    def poll(self, rid: int, wait: bool = False) -> gbqr_result:
        out = gbqr_result()
        check(gbqr_poll(self.handle, rid, 1 if wait else 0, ctypes.byref(out)), "gbqr_poll")  # noqa: F821
        return out

    def stop_serving(self):
        return gbqr_server_stop(self.handle)  # noqa: F821

    def ls_solve(self, A, b, x, prec: int = GBQR_FP64):
        pa, m, n, lda = _cm(A, "A")
        info = gbqr_info()
        st = gbqr_ls_solve(self.handle, m, n, _P(pa), lda, _P(b.data_ptr()), _P(x.data_ptr()), prec,  # noqa: F821
                           ctypes.byref(info))
        return st, info


class Graph:
    """A captured sequence of library calls (one CUDA graph launch)."""

    def __init__(self, ctx, handle):
        self.ctx, self.handle = ctx, handle

    def launch(self):
        check(gbqr_graph_launch(self.ctx.handle, self.handle), "gbqr_graph_launch")  # noqa: F821

    def close(self):
        if self.handle:
            gbqr_graph_destroy(self.handle)  # noqa: F821
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def workspace_bytes(m: int, n: int, layout: int = GBQR_T_PANEL, o: gbqr_opts | None = None) -> int:
    load()
    return int(gbqr_workspace_bytes(m, n, layout, ctypes.byref(o) if o is not None else None))  # noqa: F821


def fp64_peak(device: int = 0, kind: int = 0, iters: int = 20000) -> float:
    """Measured FP64 TFLOP/s of the device (kind 0 = DFMA, 1 = DMMA)."""
    load()
    out = ctypes.c_double(0.0)
    check(gbqr_fp64_peak(device, kind, iters, ctypes.byref(out)), "gbqr_fp64_peak")  # noqa: F821
    return out.value


def default_panel_nb(m: int, n: int) -> int:
    load()
    return int(gbqr_default_panel_nb(m, n))  # noqa: F821

"""The allocation-free tall-skinny QR (gbqr_tsqr_static), for callers that
cannot call cudaMalloc: its scratch is a fixed static device array, so it
takes no context and no workspace.  On two calls in a row - the second call
finds the array holding the first call's contents - its V, T and R must match
the oracle's element by element, and gbqr_factor's (the same TSQR base case,
run with a library workspace) within the same tolerances."""

import ctypes

import numpy as np
import pytest

import workloads
from tests import _gpu


def _static(gb, m, n, A_ptr, lda, T_ptr, ldt, stream=None):
    return gb.gbqr_tsqr_static(m, n, A_ptr, lda, T_ptr, ldt, stream)


def test_rejects_sizes_beyond_the_static_scratch():
    """Size checks run before any CUDA call, so this needs no GPU."""
    import paper_1805_05278_gb300 as gb
    gb.build()
    gb.load()
    P = ctypes.c_void_p
    buf = (ctypes.c_double * 64)()
    p = P(ctypes.addressof(buf))
    assert _static(gb, 8, 33, p, 8, p, 33) == gb.GBQR_EINVAL          # n > 32
    assert _static(gb, 4, 8, p, 4, p, 8) == gb.GBQR_EINVAL            # m < n
    assert _static(gb, 8, 4, p, 7, p, 4) == gb.GBQR_EINVAL            # lda < m
    assert _static(gb, 8, 4, p, 8, p, 3) == gb.GBQR_EINVAL            # ldt < n
    # trees that do not fit 16 MiB: about 400,000 rows is the limit at n = 32
    assert _static(gb, 1 << 40, 32, p, 1 << 40, p, 32) == gb.GBQR_EINVAL
    assert _static(gb, 420_000, 32, p, 420_000, p, 32) == gb.GBQR_EINVAL
    assert _static(gb, 8, 0, p, 8, p, 1) == gb.GBQR_OK                 # n = 0: nothing to do


def _compare(a, VR, Tn, V_ref, T_ref, R_ref, label):
    n = a.shape[1]
    assert np.max(np.abs(np.tril(VR, -1) - np.tril(V_ref, -1))) <= _gpu.TOL_V, label
    scale = max(1.0, float(np.max(np.abs(T_ref))))
    assert np.max(np.abs(Tn - T_ref)) / scale <= _gpu.TOL_T, label
    R = np.triu(VR[:n])
    cn = np.linalg.norm(a, axis=0)
    assert np.max(np.linalg.norm(R - R_ref, axis=0) / cn) <= _gpu.TOL_R_COL, label
    assert np.linalg.norm(R - R_ref) / np.linalg.norm(R_ref) <= _gpu.TOL_R_NORM, label


@pytest.mark.gpu
@pytest.mark.parametrize("m,n,seed", [(5000, 32, 41), (1000, 17, 42), (20000, 8, 43), (33, 33 - 1, 44),
                                      (250_000, 32, 45)])
def test_static_scratch_matches_oracle_and_workspace_entry(gb, orc, m, n, seed):
    import torch
    a = workloads.gaussian(m, n, seed)
    V_o, T_o, R_o, _ = orc.qr(a)
    stream = torch.cuda.current_stream()
    # the existing entry point: gbqr_factor with b >= n runs exactly one TSQR
    with gb.Context(0, stream) as ctx:
        VR_ref, T_ref, _ = _gpu.factor_gpu(ctx, a, gb.GBQR_T_FULL, gb.opts(cutoff_b=32))
    for call in range(2):
        A = _gpu.device_matrix(a)
        T = gb.colmajor(n, n, fill=float("nan"))
        st = _static(gb, m, n, ctypes.c_void_p(A.data_ptr()), A.stride(1), ctypes.c_void_p(T.data_ptr()),
                     T.stride(1), ctypes.c_void_p(stream.cuda_stream))
        assert st == gb.GBQR_OK, (call, st)
        torch.cuda.synchronize()
        VR, Tn = gb.to_numpy(A), gb.to_numpy(T)
        _compare(a, VR, Tn, V_o, T_o, R_o, f"call {call} vs oracle")
        _compare(a, VR, Tn, VR_ref, T_ref, np.triu(VR_ref[:n]), f"call {call} vs gbqr_factor")

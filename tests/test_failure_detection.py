"""Failure detection without a GPU fault: the bounded mbarrier wait that the
tensor-core GEMM uses gives up after its time limit on a barrier nothing
arrives at, raises the error flag and returns; the host reads GBQR_ETIMEOUT
and the device keeps working (a mixed-precision factorization right after
matches the oracle).  The same for the persistent batched kernel's bounded
dependency wait, on a task whose dependency never completes, and for the
persistent triangular-solve chain, on a block whose predecessor is never
solved."""

import ctypes

import numpy as np
import pytest

import workloads
from tests import _gpu

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_device_survives(gb, orc):
    ctx = gb.Context(0)
    completed = ctypes.c_int(-2)
    st = gb.gbqr_selftest_wait_timeout(0, ctypes.byref(completed))
    assert st == gb.GBQR_ETIMEOUT and completed.value == 0
    # the context and the device are still usable
    a = workloads.graded(2000, 300, 5, decades=2.0)
    o = gb.opts(update_prec=gb.GBQR_MIXED_SPLITBF16)
    VR, T, nb = _gpu.factor_gpu(ctx, a, gb.GBQR_T_PANEL, o)
    st, _ = ctx.sync()
    assert st == gb.GBQR_OK
    R = np.triu(VR[:300])
    _, _, R_o, _ = orc.qr(a)
    assert np.linalg.norm(R - R_o) / np.linalg.norm(R_o) <= 50 * np.linalg.cond(a) * 2.0 ** -22
    ctx.close()


def test_batched_dependency_wait_times_out_and_device_survives(gb, orc):
    import torch
    completed = ctypes.c_int(-2)
    st = gb.gbqr_selftest_batched_wait(0, 300, ctypes.byref(completed))
    assert st == gb.GBQR_ETIMEOUT and completed.value == 0
    ctx = gb.Context(0)
    mats = [workloads.gaussian(m, n, 40 + i) for i, (m, n) in enumerate([(900, 70), (3000, 33), (64, 64)])]
    As = [_gpu.device_matrix(a) for a in mats]
    Ts = [gb.colmajor(16, a.shape[1], fill=float("nan")) for a in mats]
    ctx.factor_batched(As, Ts)
    torch.cuda.synchronize()
    st, _ = ctx.sync()
    assert st == gb.GBQR_OK
    for a, A, T in zip(mats, As, Ts):
        _gpu.compare_factor(a, gb.to_numpy(A), gb.to_numpy(T), gb.GBQR_T_PANEL, 16, orc, f"after timeout {a.shape}")
    ctx.close()


def test_chain_wait_times_out_and_device_survives(gb, orc):
    """The persistent triangular-solve chain's bounded wait (the same wait
    as the one-vector Q application's): a CTA handed a block whose
    predecessor is never solved gives up, raises the timeout flag and
    resets the launch counters; a mixed least-squares solve (both one-launch
    kernels) then still matches the oracle."""
    import torch
    completed = ctypes.c_int(-2)
    st = gb.gbqr_selftest_chain_wait(0, 300, ctypes.byref(completed))
    assert st == gb.GBQR_ETIMEOUT and completed.value == 0
    ctx = gb.Context(0)
    a, _, b = workloads.ls_problem(1500, 200, 2.0, 61)
    A = _gpu.device_matrix(a)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros(200, dtype=torch.float64, device="cuda")
    st, info = ctx.ls_solve(A, bd, x, gb.GBQR_MIXED_SPLITBF16)
    assert st == gb.GBQR_OK
    x_o, _ = orc.ls_solve(a, b)
    assert np.linalg.norm(x.cpu().numpy() - x_o) / np.linalg.norm(x_o) <= max(1e-12, 50 * np.linalg.cond(a) * 2.0 ** -53)
    ctx.close()

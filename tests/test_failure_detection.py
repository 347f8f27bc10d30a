"""Failure detection without a GPU fault: the bounded mbarrier wait that the
tensor-core GEMM uses gives up after its time limit on a barrier nothing
arrives at, raises the error flag and returns; the host reads GBQR_ETIMEOUT
and the device keeps working (a mixed-precision factorization right after
matches the oracle)."""

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

"""Degenerate inputs across the entry points: empty and one-element batches,
batches that mix n = 0, 1 x 1 and square matrices (FP64 and FP32), a
rank-deficient matrix on the mixed least-squares path (the diagonal-block
inverses must still flag the zero pivot), a one-column mixed solve, and the
FP32 entry's rejection of wide input."""

import ctypes

import numpy as np
import pytest

import workloads
from tests import _gpu

pytestmark = pytest.mark.gpu


def test_empty_batch_is_a_no_op(gb):
    ctx = gb.Context(0)
    assert gb.gbqr_factor_batched(ctx.handle, 0, None, None, None, None, None, None, None) == gb.GBQR_OK
    assert gb.gbqr_factor_batched_f32(ctx.handle, 0, None, None, None, None, None, None, None) == gb.GBQR_OK
    ctx.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batch_with_degenerate_shapes(gb, orc, dtype):
    import torch
    shapes = [(1, 1), (5, 0), (7, 7), (64, 64), (3, 1), (200, 17), (2, 2), (129, 128)]
    mats = [workloads.gaussian(m, n, 900 + i) for i, (m, n) in enumerate(shapes)]
    tdt = torch.float64 if dtype == "f64" else torch.float32
    ctx = gb.Context(0)
    As = [torch.from_numpy(np.ascontiguousarray(a.T)).to(tdt).cuda().T if a.size else
          torch.zeros((max(1, a.shape[1]), a.shape[0]), dtype=tdt, device="cuda").T[:, :a.shape[1]]
          for a in mats]
    Ts = [torch.full((max(1, n), max(1, min(128, n))), float("nan"), dtype=tdt, device="cuda").T for (m, n) in shapes]
    ctx.factor_batched(As, Ts)
    torch.cuda.synchronize()
    st, _ = ctx.sync()
    assert st == gb.GBQR_OK
    for (m, n), a, A, T in zip(shapes, mats, As, Ts):
        if n == 0:
            continue
        a_in = a.astype(np.float32).astype(np.float64) if dtype == "f32" else a
        nb = min(_gpu.BATCH_B, n)
        _gpu.compare_factor(a_in, A.cpu().numpy(), T.cpu().numpy()[:nb], gb.GBQR_T_PANEL, nb, orc,
                            f"{dtype} {m}x{n}", fp32=(dtype == "f32"))
    ctx.close()


def test_mixed_least_squares_rank_deficient(gb):
    import torch
    a = workloads.gaussian(3000, 300, 12)
    a[:, 150] = 0.0
    ctx = gb.Context(0)
    A = _gpu.device_matrix(a)
    x = torch.zeros(300, dtype=torch.float64, device="cuda")
    st, info = ctx.ls_solve(A, torch.from_numpy(workloads.vector(3000, 13)).cuda(), x, gb.GBQR_MIXED_SPLITBF16)
    assert st == gb.GBQR_ERANKDEF and info.rankdef_col == 150
    ctx.close()


def test_mixed_least_squares_one_column(gb, orc):
    import torch
    a, xt, b = workloads.ls_problem(5000, 1, 0.0, 14)
    ctx = gb.Context(0)
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    st, info = ctx.ls_solve(_gpu.device_matrix(a), torch.from_numpy(b).cuda(), x, gb.GBQR_MIXED_SPLITBF16)
    assert st == gb.GBQR_OK
    x_o, _ = orc.ls_solve(a, b)
    assert abs(float(x.cpu()[0]) - x_o[0]) <= 1e-12 * abs(x_o[0])
    ctx.close()


def test_f32_rejects_wide_and_host_pointers(gb):
    ctx = gb.Context(0)
    ah = np.zeros((10, 20), dtype=np.float32, order="F")
    th = np.zeros((10, 10), dtype=np.float32, order="F")
    P = ctypes.c_void_p
    import torch
    A = torch.zeros((20, 10), dtype=torch.float32, device="cuda").T
    T = torch.zeros((10, 10), dtype=torch.float32, device="cuda")
    assert gb.gbqr_factor_f32(ctx.handle, 10, 20, P(A.data_ptr()), 10, P(T.data_ptr()), 10, gb.GBQR_T_FULL,
                              None) == gb.GBQR_EINVAL
    A2 = np.zeros((20, 10), dtype=np.float32, order="F")
    assert gb.gbqr_factor_f32(ctx.handle, 20, 10, P(A2.ctypes.data), 20, P(th.ctypes.data), 10, gb.GBQR_T_FULL,
                              None) == gb.GBQR_EUNSUPPORTED
    ctx.close()

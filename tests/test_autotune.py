"""Autotuner (gbqr_autotune / gbqr_autotune_batched): the chosen parameters
are among the candidates, the cache in the context is applied to later calls
(bit-identical to passing the tuned options explicitly), and every tuned
configuration still matches the oracle."""

import numpy as np
import pytest

import workloads
from tests import _gpu

pytestmark = pytest.mark.gpu


def _check_candidates(gb, o, layout, prec):
    assert o.cutoff_b in (8, 16, 32, 64)
    assert o.fanout in (0, 2, 4, 8, 16)
    assert o.leaf_rows in (0, 128, 256, 512, 1024)
    assert o.update_prec == prec
    if layout == gb.GBQR_T_PANEL:
        assert 1 <= o.panel_nb <= 256
        assert o.lookahead in (1, -1)
    if prec == gb.GBQR_FP64:
        assert o.fp64_gemm in (gb.GBQR_GEMM_DFMA, gb.GBQR_GEMM_DMMA)


@pytest.mark.parametrize("layout_name", ["panel", "full"])
def test_tuned_factor_is_cached_and_correct(gb, orc, layout_name):
    layout = gb.GBQR_T_FULL if layout_name == "full" else gb.GBQR_T_PANEL
    m, n = 3000, 300
    ctx = gb.Context(0)
    best, ms = ctx.autotune(m, n, layout, gb.GBQR_FP64, budget_ms=4000.0)
    assert ms > 0.0
    _check_candidates(gb, best, layout, gb.GBQR_FP64)
    cached = ctx.tuned(gb.GBQR_TUNE_FACTOR, m, n, layout, gb.GBQR_FP64)
    assert cached is not None and gb.opts_dict(cached) == gb.opts_dict(best)
    # the same shape class (m, n rounded up to powers of two) finds the entry
    assert ctx.tuned(gb.GBQR_TUNE_FACTOR, 2500, 260, layout, gb.GBQR_FP64) is not None
    assert ctx.tuned(gb.GBQR_TUNE_FACTOR, 5000, 300, layout, gb.GBQR_FP64) is None

    a = workloads.graded(m, n, 91, decades=3.0)
    # default options on the tuned context = tuned options on a fresh one
    # (panel_nb is the caller's: left at the default in both)
    VR1, T1, nb1 = _gpu.factor_gpu(ctx, a, layout, None)
    explicit = gb.opts(cutoff_b=best.cutoff_b, leaf_rows=best.leaf_rows, fanout=best.fanout,
                       lookahead=best.lookahead, fp64_gemm=best.fp64_gemm)
    fresh = gb.Context(0)
    VR2, T2, nb2 = _gpu.factor_gpu(fresh, a, layout, explicit)
    assert np.array_equal(VR1, VR2) and np.array_equal(T1, T2)
    _gpu.compare_factor(a, VR1, T1, layout, nb1, orc, "tuned")
    if layout == gb.GBQR_T_PANEL:
        VR3, T3, nb3 = _gpu.factor_gpu(ctx, a, layout, gb.opts(panel_nb=best.panel_nb))
        _gpu.compare_factor(a, VR3, T3, layout, nb3, orc, "tuned nb")
    fresh.close()
    ctx.close()


def test_zero_budget_keeps_the_defaults(gb):
    ctx = gb.Context(0)
    best, ms = ctx.autotune(2000, 100, gb.GBQR_T_PANEL, gb.GBQR_FP64, budget_ms=0.0)
    assert (best.cutoff_b, best.fanout, best.leaf_rows, best.lookahead) == (16, 0, 0, 1)
    assert best.panel_nb == gb.default_panel_nb(2000, 100)
    assert best.fp64_gemm == gb.GBQR_GEMM_DFMA
    assert ms > 0.0
    ctx.close()


def test_tuned_least_squares(gb, orc):
    m, n = 4000, 500
    ctx = gb.Context(0)
    for prec in (gb.GBQR_FP64, gb.GBQR_MIXED_SPLITBF16):
        ctx.autotune(m, n, gb.GBQR_T_PANEL, prec, budget_ms=3000.0)
    a, xt, b = workloads.ls_problem(m, n, 2.0, 93)
    x_o, _ = orc.ls_solve(a, b)
    kappa = np.linalg.cond(a)
    import torch
    A = _gpu.device_matrix(a)
    bd = torch.from_numpy(b).cuda()
    for prec in (gb.GBQR_FP64, gb.GBQR_MIXED_SPLITBF16):
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, info = ctx.ls_solve(A, bd, x, prec)
        assert st == gb.GBQR_OK
        xe = x.cpu().numpy()
        assert np.linalg.norm(xe - x_o) / np.linalg.norm(x_o) <= max(1e-12, 50 * kappa * np.finfo(float).eps)
    ctx.close()


def test_tuned_batched(gb, orc):
    import torch
    shapes = workloads.batched_shapes(60, seed=5, m_range=(64, 3000), n_range=(4, 96))
    ctx = gb.Context(0)
    best, ms = ctx.autotune_batched(shapes, gb.GBQR_FP64, budget_ms=4000.0)
    assert best.cutoff_b in (8, 16, 24, 32)
    assert ctx.tuned(gb.GBQR_TUNE_BATCHED) is not None
    mats = [workloads.gaussian(m, n, 500 + i) for i, (m, n) in enumerate(shapes)]
    As = [_gpu.device_matrix(a) for a in mats]
    Ts = [gb.colmajor(max(1, n), max(1, n)) for (m, n) in shapes]
    ctx.factor_batched(As, Ts)
    torch.cuda.synchronize()
    for i in (0, 7, 33, 59):
        m, n = shapes[i]
        nb = min(best.cutoff_b, n)            # the persistent kernel's panels: width b
        VR = gb.to_numpy(As[i])
        T = gb.to_numpy(Ts[i])[:min(nb, n), :]
        _gpu.compare_factor(mats[i], VR, T, gb.GBQR_T_PANEL, nb, orc, f"batched {i}")
    ctx.close()


def test_invalid_tuning_requests(gb):
    ctx = gb.Context(0)
    with pytest.raises(gb.GbqrError):
        ctx.autotune(10, 20)                                                  # m < n
    with pytest.raises(gb.GbqrError):
        ctx.autotune(100, 20, gb.GBQR_T_FULL, gb.GBQR_MIXED_SPLITBF16)        # FULL is FP64 only
    assert ctx.tuned(gb.GBQR_TUNE_FACTOR, 100, 20) is None
    ctx.close()

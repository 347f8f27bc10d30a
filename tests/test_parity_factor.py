"""GPU parity of gbqr_factor (QR-EG with TSQR base case) with the CPU oracle:
V, T and R element by element on seeded inputs, across shapes (ragged tails,
square, n = 1, tiny), both T layouts, and the algorithm's tunables (cutoff b,
leaf height, tree fan-out, panel width) - R must not depend on them."""

import numpy as np
import pytest

import workloads
from tests import _gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(gb):
    c = gb.Context(0)
    yield c
    c.close()


SHAPES = [
    # (m, n, seed, graded)
    (1024, 128, 0, False),   # the small named workload
    (1000, 77, 1, False),    # ragged: leaves and panels do not divide
    (333, 33, 2, True),
    (64, 64, 3, False),      # square
    (129, 65, 4, True),
    (7, 1, 5, False),        # n = 1
    (5, 3, 6, False),        # tiny
    (1, 1, 7, False),
    (4096, 1, 8, False),
    (2000, 5, 9, True),
    (300, 300, 10, True),
]


@pytest.mark.parametrize("m,n,seed,graded", SHAPES)
@pytest.mark.parametrize("layout_name", ["full", "panel"])
def test_factor_matches_oracle(gb, ctx, orc, m, n, seed, graded, layout_name):
    layout = gb.GBQR_T_FULL if layout_name == "full" else gb.GBQR_T_PANEL
    a = workloads.graded(m, n, seed) if graded else workloads.gaussian(m, n, seed)
    VR, T, nb = _gpu.factor_gpu(ctx, a, layout)
    _gpu.compare_factor(a, VR, T, layout, nb, orc, f"{m}x{n} {layout_name}")


TUNABLES = [
    # cutoff_b, panel_nb, leaf_rows, fanout
    (1, 0, 0, 2),
    (2, 0, 0, 3),
    (3, 0, 7, 2),
    (16, 0, 16, 4),
    (32, 50, 100, 8),
    (64, 64, 0, 2),
    (64, 0, 256, 5),
    (8, 16, 33, 2),
    (16, 0, 16, 16),   # 48 leaves: fan-out 16, two merge levels
    (16, 0, 16, 0),    # the planner's fan-out for 48 leaves (two levels at k = 8 already)
    (4, 0, 8, 13),
]


@pytest.mark.parametrize("b,nb,leaf,k", TUNABLES)
@pytest.mark.parametrize("layout_name", ["full", "panel"])
def test_tunables_do_not_change_the_result(gb, ctx, orc, b, nb, leaf, k, layout_name):
    layout = gb.GBQR_T_FULL if layout_name == "full" else gb.GBQR_T_PANEL
    a = workloads.gaussian(777, 97, 11)
    o = gb.opts(cutoff_b=b, panel_nb=nb, leaf_rows=leaf, fanout=k)
    VR, T, nbr = _gpu.factor_gpu(ctx, a, layout, o)
    _gpu.compare_factor(a, VR, T, layout, nbr, orc, f"b={b} nb={nb} leaf={leaf} k={k}")


def test_pure_tsqr_base_case(gb, ctx, orc):
    """b >= n: QR-EG is one TSQR (the 1D-CAQR-EG b = n case)."""
    a = workloads.gaussian(5000, 48, 12)
    for k in (2, 3, 8):
        o = gb.opts(cutoff_b=64, leaf_rows=64, fanout=k)
        VR, T, nb = _gpu.factor_gpu(ctx, a, gb.GBQR_T_FULL, o)
        _gpu.compare_factor(a, VR, T, gb.GBQR_T_FULL, nb, orc, f"tsqr k={k}")


def test_single_leaf(gb, ctx, orc):
    """P = 1: TSQR reduces to one local QR plus the reconstruction."""
    a = workloads.gaussian(40, 32, 13)
    o = gb.opts(cutoff_b=32, leaf_rows=4000)
    VR, T, nb = _gpu.factor_gpu(ctx, a, gb.GBQR_T_FULL, o)
    _gpu.compare_factor(a, VR, T, gb.GBQR_T_FULL, nb, orc, "single leaf")


def test_odd_leading_dimension(gb, ctx, orc):
    a = workloads.graded(513, 70, 14)
    for pad in (1, 3, 8):
        VR, T, nb = _gpu.factor_gpu(ctx, a, gb.GBQR_T_PANEL, None, lda_pad=pad)
        _gpu.compare_factor(a, VR, T, gb.GBQR_T_PANEL, nb, orc, f"lda pad {pad}")


def test_upper_triangular_input(gb, ctx, orc):
    """Zero subcolumns: every reflector is I - 2 e_j e_j^T, so R = -A exactly
    in structure and V has no entries below the diagonal."""
    a = workloads.upper_triangular(300, 40, 15)
    VR, T, nb = _gpu.factor_gpu(ctx, a, gb.GBQR_T_FULL, gb.opts(cutoff_b=16))
    _gpu.compare_factor(a, VR, T, gb.GBQR_T_FULL, nb, orc, "upper triangular")


def _near_pairs(m, n, seed, eps=1e-3):
    """Odd columns nearly parallel to the even column before them: after the
    reflector of column 2k, column 2k+1 keeps about eps of its norm, so the
    norm below its pivot cancels in every leaf, merge and stacked block."""
    a = workloads.gaussian(m, n, seed)
    a[:, 1::2] = a[:, 0:n - n % 2:2] + eps * a[:, 1::2]
    return a


@pytest.mark.parametrize("layout_name", ["full", "panel"])
@pytest.mark.parametrize("leaf,k", [(0, 0), (64, 4), (40, 2)])
def test_nearly_parallel_columns(gb, ctx, orc, layout_name, leaf, k):
    """The pivot step takes the norm of the updated column from sums of the
    column before the update; where those terms cancel it sums the updated
    rows instead.  Columns chosen to cancel at every tree level still match
    the oracle element by element (a norm kept from the cancelling terms
    would put errors near 1e-9 into V and T)."""
    layout = gb.GBQR_T_FULL if layout_name == "full" else gb.GBQR_T_PANEL
    a = _near_pairs(2000, 40, 17)
    o = gb.opts(cutoff_b=16, leaf_rows=leaf, fanout=k)
    VR, T, nb = _gpu.factor_gpu(ctx, a, layout, o)
    _gpu.compare_factor(a, VR, T, layout, nb, orc, f"near pairs leaf={leaf} k={k} {layout_name}")


def test_zero_column_gives_a_valid_qr(gb, ctx):
    """Rank deficiency: V, T are not unique, so check A = QR and Q^T Q = I."""
    import torch
    a = workloads.gaussian(400, 30, 16)
    a[:, 7] = 0.0
    A = _gpu.device_matrix(a)
    T = _gpu.t_buffer(30, gb.GBQR_T_FULL, 30)
    ctx.factor(A, T, gb.GBQR_T_FULL, gb.opts(cutoff_b=8))
    Q = gb.colmajor(400, 30)
    ctx.form_q(A, T, Q, gb.GBQR_T_FULL)
    torch.cuda.synchronize()
    q = gb.to_numpy(Q)
    r = np.triu(gb.to_numpy(A)[:30])
    assert np.isfinite(q).all() and np.isfinite(r).all()
    assert np.linalg.norm(a - q @ r) / np.linalg.norm(a) <= _gpu.TOL_BACKWARD
    assert np.linalg.norm(q.T @ q - np.eye(30)) <= _gpu.TOL_BACKWARD
    assert abs(r[7, 7]) <= 1e-13 * np.linalg.norm(a)


def test_deterministic(gb, ctx):
    """Fixed tree and split shapes: two runs are bit-identical."""
    a = workloads.graded(3000, 200, 17)
    r1 = _gpu.factor_gpu(ctx, a, gb.GBQR_T_PANEL)
    r2 = _gpu.factor_gpu(ctx, a, gb.GBQR_T_PANEL)
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[1], r2[1])


def test_nonfinite_input_is_reported(gb, ctx):
    import torch
    a = workloads.gaussian(200, 20, 18)
    a[13, 4] = np.nan
    ctx.sync()
    A = _gpu.device_matrix(a)
    T = _gpu.t_buffer(20, gb.GBQR_T_PANEL, 20)
    ctx.factor(A, T, gb.GBQR_T_PANEL)
    st, info = ctx.sync()
    assert st == gb.GBQR_ENONFINITE and info.nonfinite
    st, info = ctx.sync()
    assert st == gb.GBQR_OK
    torch.cuda.synchronize()


def test_invalid_arguments(gb, ctx):
    import ctypes
    A = gb.colmajor(10, 20)
    T = gb.colmajor(20, 20)
    h = ctx.handle
    P = ctypes.c_void_p
    # wide: lda < m and ldt < min(m, n) are rejected; host pointers are not supported
    assert gb.gbqr_factor(h, 10, 20, P(A.data_ptr()), 9, P(T.data_ptr()), 20, gb.GBQR_T_FULL, None) == gb.GBQR_EINVAL
    assert gb.gbqr_factor(h, 10, 20, P(A.data_ptr()), 10, P(T.data_ptr()), 9, gb.GBQR_T_FULL, None) == gb.GBQR_EINVAL
    import numpy as _np
    ah = _np.zeros((10, 20), order="F")
    th = _np.zeros((10, 10), order="F")
    assert gb.gbqr_factor(h, 10, 20, P(ah.ctypes.data), 10, P(th.ctypes.data), 10, gb.GBQR_T_FULL,
                          None) == gb.GBQR_EUNSUPPORTED
    A = gb.colmajor(30, 20)
    assert gb.gbqr_factor(h, 30, 20, P(A.data_ptr()), 29, P(T.data_ptr()), 20, gb.GBQR_T_FULL, None) == gb.GBQR_EINVAL
    assert gb.gbqr_factor(h, 30, 20, P(A.data_ptr()), 30, P(T.data_ptr()), 19, gb.GBQR_T_FULL, None) == gb.GBQR_EINVAL
    assert gb.gbqr_factor(h, 30, 20, P(A.data_ptr()), 30, P(T.data_ptr()), 20, 5, None) == gb.GBQR_EINVAL
    bad = gb.opts(cutoff_b=65)
    assert gb.gbqr_factor(h, 30, 20, P(A.data_ptr()), 30, P(T.data_ptr()), 20, gb.GBQR_T_FULL, ctypes.byref(bad)) == gb.GBQR_EINVAL
    bad = gb.opts(fanout=1)
    assert gb.gbqr_factor(h, 30, 20, P(A.data_ptr()), 30, P(T.data_ptr()), 20, gb.GBQR_T_FULL, ctypes.byref(bad)) == gb.GBQR_EINVAL
    # n = 0 is a no-op
    assert gb.gbqr_factor(h, 30, 0, P(A.data_ptr()), 30, P(T.data_ptr()), 1, gb.GBQR_T_FULL, None) == gb.GBQR_OK


def test_host_pointers(gb, ctx, orc):
    """A and T in host memory: the call stages through the device."""
    import ctypes
    a = workloads.gaussian(600, 50, 19)
    vr = np.asfortranarray(a.copy())
    t = np.zeros((50, 50), order="F")
    st = gb.gbqr_factor(ctx.handle, 600, 50, vr.ctypes.data_as(ctypes.c_void_p), 600,
                        t.ctypes.data_as(ctypes.c_void_p), 50, gb.GBQR_T_FULL, None)
    assert st == gb.GBQR_OK
    _gpu.compare_factor(a, vr, t, gb.GBQR_T_FULL, 50, orc, "host pointers")


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("m,n,nb,pad", [(1500, 300, 64, 0), (900, 250, 32, 7), (700, 130, 64, 3), (2304, 320, 128, 5)])
def test_host_pointers_panel(gb, ctx, orc, m, n, nb, pad, pinned):
    """Host A and T in the PANEL layout with look-ahead.  Page-locked buffers
    take the overlapped path (panels in and out on the copy stream while
    others are factored), pageable ones the plain staged path; both must
    give the oracle's factorization, with ragged last panels and padded
    leading dimensions whose padding stays untouched."""
    import ctypes
    import torch
    a = workloads.gaussian(m, n, 23)
    lda, trows = m + pad, min(nb, n)
    ldt = trows + pad
    Ah = torch.full((n, lda), float("nan"), dtype=torch.float64)
    Th = torch.full((n, ldt), float("nan"), dtype=torch.float64)
    if pinned:
        Ah, Th = Ah.pin_memory(), Th.pin_memory()
    Ah[:, :m] = torch.from_numpy(np.ascontiguousarray(a.T))
    o = gb.opts(panel_nb=nb)
    st = gb.gbqr_factor(ctx.handle, m, n, ctypes.c_void_p(Ah.data_ptr()), lda, ctypes.c_void_p(Th.data_ptr()), ldt,
                        gb.GBQR_T_PANEL, ctypes.byref(o))
    assert st == gb.GBQR_OK
    assert torch.isnan(Ah[:, m:]).all() and torch.isnan(Th[:, trows:]).all(), "padding was written"
    vr = Ah[:, :m].numpy().T.copy(order="F")
    t = Th[:, :trows].numpy().T.copy(order="F")
    _gpu.compare_factor(a, vr, t, gb.GBQR_T_PANEL, nb, orc, f"host panel pinned={pinned}")


@pytest.mark.parametrize("lookahead", [0, -1])
@pytest.mark.parametrize("m,n,nb", [(2000, 300, 16), (640, 640, 64), (5000, 129, 32)])
def test_lookahead_on_and_off(gb, ctx, orc, m, n, nb, lookahead):
    """The look-ahead schedule (panel k+1 on a second stream) reorders work
    but not arithmetic: both schedules match the oracle."""
    a = workloads.graded(m, n, 20 + nb)
    o = gb.opts(panel_nb=nb, lookahead=lookahead)
    VR, T, nbr = _gpu.factor_gpu(ctx, a, gb.GBQR_T_PANEL, o)
    _gpu.compare_factor(a, VR, T, gb.GBQR_T_PANEL, nbr, orc, f"lookahead={lookahead} nb={nb}")


@pytest.mark.parametrize("engine", ["dmma", "dfma"])
@pytest.mark.parametrize("m,n,layout_name", [(3001, 700, "full"), (1500, 1500, "panel"), (20000, 260, "panel")])
def test_fp64_gemm_engines(gb, ctx, orc, m, n, layout_name, engine):
    """The FP64 update products run either on the FP64 tensor cores (mma.sync
    m8n8k4) or on CUDA-core FMAs; both match the oracle, and the two differ
    from each other by rounding only."""
    layout = gb.GBQR_T_FULL if layout_name == "full" else gb.GBQR_T_PANEL
    a = workloads.graded(m, n, 40 + n, decades=3.0)
    e = gb.GBQR_GEMM_DMMA if engine == "dmma" else gb.GBQR_GEMM_DFMA
    VR, T, nbr = _gpu.factor_gpu(ctx, a, layout, gb.opts(fp64_gemm=e))
    _gpu.compare_factor(a, VR, T, layout, nbr, orc, f"engine={engine}")


def test_fp64_gemm_engine_rejects_unknown(gb, ctx):
    a = workloads.gaussian(100, 40, 1)
    with pytest.raises(gb.GbqrError):
        _gpu.factor_gpu(ctx, a, gb.GBQR_T_FULL, gb.opts(fp64_gemm=7))


@pytest.mark.parametrize("m,n,layout_name", [(100, 250, "full"), (100, 250, "panel"), (700, 1500, "panel"),
                                             (2000, 3100, "full"), (33, 34, "panel"), (1, 5, "full")])
def test_wide_matrix(gb, ctx, orc, m, n, layout_name):
    """m < n (Section 2.1): A = [A1 A2], A1 = Q R1 by QR-EG, R = [R1, Q^T A2];
    V, R (upper trapezoidal) and the m reflectors' T match the oracle."""
    import torch
    layout = gb.GBQR_T_FULL if layout_name == "full" else gb.GBQR_T_PANEL
    a = workloads.gaussian(m, n, 300 + m)
    nb = gb.default_panel_nb(m, m)
    A = _gpu.device_matrix(a)
    T = gb.colmajor(m if layout == gb.GBQR_T_FULL else min(nb, m), m, fill=float("nan"))
    ctx.factor(A, T, layout)
    torch.cuda.synchronize()
    VR, Tg = gb.to_numpy(A), gb.to_numpy(T)
    vr_o, tau_o = orc.house_qr(a)
    assert np.max(np.abs(np.tril(VR[:, :m], -1) - np.tril(vr_o[:, :m], -1))) <= _gpu.TOL_V
    r, r_o = np.triu(VR), np.triu(vr_o)
    colnorm = np.linalg.norm(a, axis=0)
    assert np.max(np.linalg.norm(r - r_o, axis=0) / colnorm) <= _gpu.TOL_R_COL
    t_o = orc.larft(vr_o[:, :m], tau_o)
    if layout == gb.GBQR_T_PANEL:
        t_o = _gpu.panel_blocks_of(t_o, nb)
    assert np.max(np.abs(Tg - t_o)) / max(1.0, np.max(np.abs(t_o))) <= _gpu.TOL_T
    # the factors apply: Q^T A = R through gbqr_apply_qt with n = m reflectors
    B = _gpu.device_matrix(a)
    ctx.apply_qt(A[:, :m], T, B, layout, nb)
    torch.cuda.synchronize()
    assert np.linalg.norm(gb.to_numpy(B) - r) / np.linalg.norm(a) <= _gpu.TOL_BACKWARD

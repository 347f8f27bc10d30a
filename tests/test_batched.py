"""Batched factorization (gbqr_factor_batched): one persistent kernel launch
for the whole batch (panel width b = the cutoff, T in b-wide panel blocks).
Every matrix of an uneven batch matches the oracle - including tall ones
whose panels span many row blocks, several panel widths, and a sample of the
2000-matrix benchmark batch at its full sizes - the per-matrix stream path
(wider panels) agrees with it, a NaN is reported, and a captured graph of
the batch reproduces the eager result bit for bit."""

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


def _batch(count, seed):
    shapes = workloads.batched_shapes(count, seed, m_range=(40, 3000), n_range=(1, 150))
    mats = [workloads.gaussian(m, n, seed * 1000 + i) for i, (m, n) in enumerate(shapes)]
    return shapes, mats


def _run(gb, ctx, mats, o=None):
    import torch
    As = [_gpu.device_matrix(a) for a in mats]
    Ts = [gb.colmajor(max(1, min(128, a.shape[1])), a.shape[1], fill=float("nan")) for a in mats]
    ctx.factor_batched(As, Ts, o)
    torch.cuda.synchronize()
    return As, Ts


def test_batched_matches_oracle(gb, ctx, orc):
    shapes, mats = _batch(24, 3)
    As, Ts = _run(gb, ctx, mats)
    st, _ = ctx.sync()
    assert st == gb.GBQR_OK
    for a, A, T in zip(mats, As, Ts):
        nb = min(_gpu.BATCH_B, a.shape[1])
        _gpu.compare_factor(a, gb.to_numpy(A), gb.to_numpy(T)[:nb], gb.GBQR_T_PANEL, nb, orc, f"batched {a.shape}")


@pytest.mark.parametrize("b", [8, 16, 24, 32])
def test_batched_panel_widths_and_tall_panels(gb, ctx, orc, b):
    """Tall matrices (panels of several row blocks, so the flat reduction and
    the reconstruction chain run), ragged widths, every panel width the
    persistent kernel takes."""
    shapes = [(20000, 40), (5003, 2 * b + 3), (b, b), (700, 1), (12345, 97), (b + 1, b), (3000, 3 * b)]
    mats = [workloads.gaussian(m, n, 7000 + b + i) for i, (m, n) in enumerate(shapes)]
    import torch
    As = [_gpu.device_matrix(a) for a in mats]
    Ts = [gb.colmajor(max(1, min(b, a.shape[1])), a.shape[1], fill=float("nan")) for a in mats]
    ctx.factor_batched(As, Ts, gb.opts(cutoff_b=b))
    torch.cuda.synchronize()
    st, _ = ctx.sync()
    assert st == gb.GBQR_OK
    for a, A, T in zip(mats, As, Ts):
        nb = min(b, a.shape[1])
        _gpu.compare_factor(a, gb.to_numpy(A), gb.to_numpy(T), gb.GBQR_T_PANEL, nb, orc, f"b={b} {a.shape}")


def test_batched_nearly_parallel_columns(gb, ctx, orc):
    """Leaf and stacked blocks whose column norms cancel after each reflector
    (odd columns nearly parallel to the even ones) match the oracle.  The
    pairs differ by 3e-3 rather than 1e-3: at 1e-3 the 9000-row matrix's T
    differs from the oracle's by 1.3e-11 from its conditioning alone (with
    the norm summed directly at every step as well)."""
    import torch
    from tests.test_parity_factor import _near_pairs
    mats = [_near_pairs(m, n, 40 + i, 3e-3) for i, (m, n) in enumerate([(3000, 40), (500, 17), (9000, 32)])]
    As = [_gpu.device_matrix(a) for a in mats]
    Ts = [gb.colmajor(16, a.shape[1], fill=float("nan")) for a in mats]
    ctx.factor_batched(As, Ts, gb.opts(cutoff_b=16))
    torch.cuda.synchronize()
    st, _ = ctx.sync()
    assert st == gb.GBQR_OK
    for a, A, T in zip(mats, As, Ts):
        _gpu.compare_factor(a, gb.to_numpy(A), gb.to_numpy(T), gb.GBQR_T_PANEL, 16, orc, f"near pairs {a.shape}")


def test_batched_stream_path_agrees(gb, ctx, orc):
    """panel_nb = 128 selects the per-matrix panel path (QR-EG per 128-wide
    panel over internal streams); both engines match the oracle."""
    shapes, mats = _batch(10, 8)
    As, Ts = _run(gb, ctx, mats, gb.opts(panel_nb=128))
    for a, A, T in zip(mats, As, Ts):
        nb = min(128, a.shape[1])
        _gpu.compare_factor(a, gb.to_numpy(A), gb.to_numpy(T), gb.GBQR_T_PANEL, nb, orc, f"stream {a.shape}")


def test_batched_reports_nan(gb, ctx):
    import torch
    shapes, mats = _batch(6, 9)
    mats[3] = mats[3].copy()
    mats[3][mats[3].shape[0] // 2, mats[3].shape[1] - 1] = float("nan")
    _run(gb, ctx, mats)
    st, info = ctx.sync()
    assert st == gb.GBQR_ENONFINITE and info.nonfinite
    st, _ = ctx.sync()
    assert st == gb.GBQR_OK


def test_batched_full_size_sample(gb, ctx):
    """The benchmark's 2000-matrix batch (m log-uniform [256, 16384], n uniform
    [16, 256], seeded device generator), factored in one launch exactly as the
    bench times it; 12 matrices (the largest, the tallest, the widest and a
    spread of others) against the all-cores oracle."""
    import torch
    import oracle
    orc_all = oracle.all_cores()
    shapes = workloads.batched_shapes(2000, workloads.BATCHED_SEED)
    buf, offs = workloads.batched_device_buffer(shapes, workloads.BATCHED_SEED)
    pristine = buf.clone()
    As = [buf[o:o + m * n].view(n, m).T for (m, n), o in zip(shapes, offs)]
    Ts = [torch.empty((n, min(128, n)), dtype=torch.float64, device="cuda").T for (m, n) in shapes]
    ctx.factor_batched(As, Ts)
    torch.cuda.synchronize()
    st, _ = ctx.sync()
    assert st == gb.GBQR_OK
    cost = [workloads.qr_flops(m, n) for m, n in shapes]
    pick = {int(np.argmax(cost)), int(np.argmax([m for m, _ in shapes])), int(np.argmax([n for _, n in shapes]))}
    pick |= set(range(0, 2000, 223))
    for i in sorted(pick):
        m, n = shapes[i]
        a = gb.to_numpy(pristine[offs[i]:offs[i] + m * n].view(n, m).T)
        nb = min(_gpu.BATCH_B, n)
        V_o, T_o, R_o, _ = orc_all.qr(a)
        VR, T = gb.to_numpy(As[i]), gb.to_numpy(Ts[i])[:nb]
        assert np.max(np.abs(oracle.unpack_v(VR) - V_o)) <= _gpu.TOL_V, (i, m, n)
        R = np.triu(VR[:n])
        assert np.linalg.norm(R - R_o) / np.linalg.norm(R_o) <= _gpu.TOL_R_NORM, (i, m, n)
        assert np.max(np.linalg.norm(R - R_o, axis=0) / np.linalg.norm(a, axis=0)) <= _gpu.TOL_R_COL, (i, m, n)
        Tb = _gpu.panel_blocks_of(T_o, nb)
        assert np.max(np.abs(T - Tb)) / max(1.0, np.max(np.abs(Tb))) <= _gpu.TOL_T, (i, m, n)


def test_batched_mixed_precision_runs(gb, ctx, orc):
    shapes, mats = _batch(12, 4)
    o = gb.opts(update_prec=gb.GBQR_MIXED_SPLITBF16)
    As, Ts = _run(gb, ctx, mats, o)
    for a, A in zip(mats, As):
        n = a.shape[1]
        R = np.triu(gb.to_numpy(A)[:n])
        _, _, R_o, _ = orc.qr(a)
        assert np.linalg.norm(R - R_o) / np.linalg.norm(R_o) <= 50 * np.linalg.cond(a) * 2.0 ** -22


def test_graph_capture_reproduces_eager(gb):
    import torch
    stream = torch.cuda.Stream()                      # capture needs a non-default stream
    ctx = gb.Context(0, stream)
    shapes, mats = _batch(16, 5)
    eager_A, eager_T = _run(gb, ctx, mats)            # also grows workspace, creates lanes
    As = [_gpu.device_matrix(a) for a in mats]
    Ts = [gb.colmajor(max(1, min(128, a.shape[1])), a.shape[1], fill=0.0) for a in mats]
    fresh = [A.clone() for A in As]
    torch.cuda.synchronize()
    graph = ctx.capture(lambda: ctx.factor_batched(As, Ts))
    for rep in range(2):                               # replay twice from the same inputs
        for A, F in zip(As, fresh):
            A.copy_(F)
        torch.cuda.synchronize()
        graph.launch()
        torch.cuda.synchronize()
        for A, T, EA, ET in zip(As, Ts, eager_A, eager_T):
            nb = min(_gpu.BATCH_B, T.shape[1])        # rows of the b-wide panel layout
            assert torch.equal(A, EA) and torch.equal(T[:nb], ET[:nb])
    graph.close()
    ctx.close()

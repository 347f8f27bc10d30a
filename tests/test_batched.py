"""Batched factorization (gbqr_factor_batched): every matrix of an uneven
batch matches the oracle, and a captured graph of the batch reproduces the
eager result bit for bit."""

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
        nb = min(128, a.shape[1])
        _gpu.compare_factor(a, gb.to_numpy(A), gb.to_numpy(T), gb.GBQR_T_PANEL, nb, orc, f"batched {a.shape}")


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
            assert torch.equal(A, EA) and torch.equal(T, ET)
    graph.close()
    ctx.close()

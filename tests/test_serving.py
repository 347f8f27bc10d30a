"""Least-squares serving loop (gbqr_server_start / gbqr_submit / gbqr_poll):
requests of different sizes admitted by HBM footprint and overlapped on the
device.  Every result matches the oracle and is bit-identical to the same
request solved alone (the kernels are deterministic, so co-running requests
cannot change a result)."""

import numpy as np
import pytest

import workloads
from tests import _gpu

pytestmark = pytest.mark.gpu


def _requests(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = workloads.log_uniform_int(rng, 200, 3000)
        n = workloads.log_uniform_int(rng, 8, 200)
        n = min(n, m)
        decades = float(rng.uniform(0.5, 3.0))
        a, xt, b = workloads.ls_problem(m, n, decades, seed * 100 + i)
        out.append((a, b))
    return out


def _serve(gb, problems, precs, workers=8, cap=8 << 30):
    import torch
    ctx = gb.Context(0)
    ctx.serve(workers, cap)
    bufs = []
    ids = []
    for (a, b), prec in zip(problems, precs):
        A = _gpu.device_matrix(a)
        bd = torch.from_numpy(b).cuda()
        x = torch.full((a.shape[1],), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        bufs.append((A, bd, x))
        ids.append(ctx.submit(A, bd, x, prec, tag=len(ids)))
    results = [ctx.poll(i, wait=True) for i in ids]
    xs = [x.cpu().numpy() for (_, _, x) in bufs]
    ctx.stop_serving()
    ctx.close()
    return results, xs


def test_mixed_stream_of_requests(gb, orc):
    problems = _requests(20, 7)
    cycle = [gb.GBQR_FP64, gb.GBQR_PREC_AUTO, gb.GBQR_MIXED_SPLITBF16]
    precs = [cycle[i % 3] for i in range(len(problems))]
    results, xs = _serve(gb, problems, precs)
    for (a, b), r, x in zip(problems, results, xs):
        assert r.state == gb.GBQR_REQ_DONE and r.status == gb.GBQR_OK, (r.status, a.shape)
        x_o, _ = orc.ls_solve(a, b)
        kappa = np.linalg.cond(a)
        assert np.linalg.norm(x - x_o) / np.linalg.norm(x_o) <= max(1e-12, 50 * kappa * np.finfo(float).eps)
        assert r.latency_ms >= r.run_ms >= 0.0
    assert any(r.prec_used == gb.GBQR_MIXED_SPLITBF16 for r in results)
    # alone vs in the mix: identical bits
    for k in (0, 2, 4, 8):
        alone, xa = _serve(gb, [problems[k]], [precs[k]], workers=1)
        assert np.array_equal(xa[0], xs[k]), k
        assert alone[0].prec_used == results[k].prec_used


def test_tight_memory_cap_serialises(gb, orc):
    problems = _requests(6, 9)
    foot = max(gb.workspace_bytes(a.shape[0], a.shape[1], gb.GBQR_T_PANEL,
                                  gb.opts(update_prec=gb.GBQR_MIXED_SPLITBF16)) for a, _ in problems)
    results, xs = _serve(gb, problems, [gb.GBQR_PREC_AUTO] * 6, workers=4, cap=foot + (2 << 20))
    for (a, b), r, x in zip(problems, results, xs):
        assert r.status == gb.GBQR_OK
        x_o, _ = orc.ls_solve(a, b)
        assert np.linalg.norm(x - x_o) / np.linalg.norm(x_o) <= max(1e-12, 50 * np.linalg.cond(a) * np.finfo(float).eps)


def test_invalid_requests_are_rejected(gb):
    import ctypes
    import torch
    ctx = gb.Context(0)
    ctx.serve(2, 64 << 20)
    A = gb.colmajor(10, 20)
    b = torch.zeros(10, dtype=torch.float64, device="cuda")
    x = torch.zeros(20, dtype=torch.float64, device="cuda")
    with pytest.raises(gb.GbqrError):
        ctx.submit(A, b, x, gb.GBQR_FP64)                 # m < n
    with pytest.raises(gb.GbqrError):
        ctx.poll(12345)                                   # unknown id
    big = gb.colmajor(20000, 2000)
    bb = torch.zeros(20000, dtype=torch.float64, device="cuda")
    xb = torch.zeros(2000, dtype=torch.float64, device="cuda")
    with pytest.raises(gb.GbqrError):
        ctx.submit(big, bb, xb, gb.GBQR_FP64)             # footprint above the 64 MiB cap
    ctx.stop_serving()
    ctx.close()


def test_bounded_bypass_of_a_large_request(gb, orc):
    """A large request that only fits alone, queued behind running requests
    and ahead of a stream of small ones: first-fit lets small ones pass it,
    but at most 8 of them (its result reports how many did), after which it
    blocks the queue until it fits - so it cannot wait indefinitely."""
    import torch
    ctx = gb.Context(0)

    def footprint(m, n):
        return gb.workspace_bytes(m, n, gb.GBQR_T_PANEL) + (1 << 20) + 8 * (m * n + m + n)

    big_shape, long_shape, small_shape = (30000, 1000), (4000, 256), (600, 40)
    cap = footprint(*big_shape) + footprint(*small_shape) // 2
    assert 4 * footprint(*long_shape) <= cap and footprint(*big_shape) + footprint(*small_shape) > cap
    ctx.serve(4, cap)
    shapes = [long_shape] * 4 + [big_shape] + [small_shape] * 40
    bufs, ids = [], []
    for i, (m, n) in enumerate(shapes):
        a, _, b = workloads.ls_problem(m, n, 1.0, 500 + i)
        A = _gpu.device_matrix(a)
        bd = torch.from_numpy(b).cuda()
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        bufs.append((a, b, A, bd, x))
    torch.cuda.synchronize()
    for i, (a, b, A, bd, x) in enumerate(bufs):
        ids.append(ctx.submit(A, bd, x, gb.GBQR_FP64, tag=i))
    results = [ctx.poll(r, wait=True) for r in ids]
    ctx.stop_serving()
    ctx.close()
    big = results[4]
    assert all(r.status == gb.GBQR_OK for r in results)
    assert 0 <= big.bypassed <= 8, big.bypassed
    assert all(r.bypassed <= 8 for r in results)
    assert big.footprint_bytes == footprint(*big_shape)
    a, b, _, _, x = bufs[4]
    x_o, _ = orc.ls_solve(a, b)
    assert np.linalg.norm(x.cpu().numpy() - x_o) / np.linalg.norm(x_o) <= 1e-12

"""FP32 batched factorization (gbqr_factor_batched_f32): every step in FP32
with the float instantiations of the same kernels.  Each matrix matches the
FP64 oracle run on the same float32-rounded input within the FP32
tolerances, Q is orthogonal to FP32 accuracy, and a captured graph of the
batch reproduces the eager result bit for bit."""

import numpy as np
import pytest

import workloads
from tests import _gpu

pytestmark = pytest.mark.gpu


def _batch32(count, seed):
    shapes = workloads.batched_shapes(count, seed, m_range=(40, 3000), n_range=(1, 150))
    mats = [workloads.gaussian(m, n, seed * 1000 + i).astype(np.float32) for i, (m, n) in enumerate(shapes)]
    return shapes, mats


def _device32(a):
    import torch
    m, n = a.shape
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().T      # column-major float32


def _run32(gb, ctx, mats, o=None):
    import torch
    As = [_device32(a) for a in mats]
    Ts = [torch.full((a.shape[1], max(1, min(128, a.shape[1]))), float("nan"), dtype=torch.float32,
                     device="cuda").T for a in mats]
    ctx.factor_batched(As, Ts, o)
    torch.cuda.synchronize()
    return As, Ts


def test_f32_batched_matches_oracle(gb, orc):
    ctx = gb.Context(0)
    shapes, mats = _batch32(24, 3)
    As, Ts = _run32(gb, ctx, mats)
    st, _ = ctx.sync()
    assert st == gb.GBQR_OK
    for a, A, T in zip(mats, As, Ts):
        nb = min(_gpu.BATCH_B, a.shape[1])
        VR = A.cpu().numpy().astype(np.float64)
        Tn = T.cpu().numpy().astype(np.float64)[:nb]
        _gpu.compare_factor(a.astype(np.float64), VR, Tn, gb.GBQR_T_PANEL, nb, orc, f"fp32 {a.shape}", fp32=True)
    ctx.close()


def test_f32_orthogonality_and_backward_error(gb, orc):
    """Q formed in FP64 from the FP32 (V, T): ||Q^T Q - I|| and ||A - QR|| / ||A||
    at FP32 accuracy, on a tall matrix that spans many TSQR leaves."""
    import torch
    ctx = gb.Context(0)
    a = workloads.gaussian(6000, 96, 77).astype(np.float32)
    As, Ts = _run32(gb, ctx, [a])
    VR = As[0].cpu().numpy().astype(np.float64)
    m, n = a.shape
    T = Ts[0].cpu().numpy().astype(np.float64)                  # 16-wide panel blocks
    q = _gpu.q_from_panels(VR, T, _gpu.BATCH_B)
    r = np.triu(VR[:n])
    assert np.linalg.norm(q.T @ q - np.eye(n), 2) <= _gpu.TOL32_BACKWARD
    assert np.linalg.norm(a - q @ r) / np.linalg.norm(a) <= _gpu.TOL32_BACKWARD
    ctx.close()


def test_f32_graph_capture_reproduces_eager(gb):
    import torch
    shapes, mats = _batch32(40, 5)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = gb.Context(0, stream)
        As, Ts = _run32(gb, ctx, mats)
        eager = [A.cpu().clone() for A in As]
        As2 = [_device32(a) for a in mats]
        Ts2 = [torch.zeros_like(T) for T in Ts]
        torch.cuda.synchronize()
        pristine = [A.clone() for A in As2]
        graph = ctx.capture(lambda: ctx.factor_batched(As2, Ts2))
        for A, P in zip(As2, pristine):
            A.copy_(P)
        graph.launch()
        torch.cuda.synchronize()
        for e, A in zip(eager, As2):
            assert torch.equal(e, A.cpu())
        graph.close()
        ctx.close()


def test_f32_rejects_tensor_core_updates(gb):
    ctx = gb.Context(0)
    a = workloads.gaussian(100, 20, 1).astype(np.float32)
    with pytest.raises(gb.GbqrError):
        _run32(gb, ctx, [a], gb.opts(update_prec=gb.GBQR_MIXED_SPLITBF16))
    ctx.close()


@pytest.mark.parametrize("m,n,layout_name,nb", [(3000, 700, "full", 0), (1500, 1500, "panel", 128),
                                                (20000, 260, "panel", 64), (777, 97, "panel", 32)])
def test_f32_single_factorization(gb, orc, m, n, layout_name, nb):
    """gbqr_factor_f32: the FP32 instantiation of the whole QR-EG path (PANEL
    with look-ahead, FULL with the T-merge), against the FP64 oracle on the
    same float32-rounded input."""
    import torch
    layout = gb.GBQR_T_FULL if layout_name == "full" else gb.GBQR_T_PANEL
    a = workloads.gaussian(m, n, 600 + n).astype(np.float32)
    ctx = gb.Context(0)
    A = _device32(a)
    nbr = nb or gb.default_panel_nb(m, n)
    rows = n if layout == gb.GBQR_T_FULL else min(nbr, n)
    T = torch.full((n, rows), float("nan"), dtype=torch.float32, device="cuda").T
    ctx.factor(A, T, layout, gb.opts(panel_nb=nb))
    torch.cuda.synchronize()
    _gpu.compare_factor(a.astype(np.float64), A.cpu().numpy(), T.cpu().numpy(), layout, nbr, orc,
                        f"fp32 {m}x{n}", fp32=True)
    ctx.close()


@pytest.mark.parametrize("leaf,k", [(0, 0), (40, 2)])
def test_f32_nearly_parallel_columns(gb, orc, leaf, k):
    """The pivot step's direct-sum branch in FP32: odd columns 3e-3 away from
    the even ones, so after each reflector the next column's norm cancels in
    every leaf and merge.  Against the FP64 oracle on the same float32 input
    (a norm kept from the cancelling sums would be off by ~1e-1 here)."""
    import torch
    from tests.test_parity_factor import _near_pairs
    a = _near_pairs(2000, 40, 23, 3e-3).astype(np.float32)
    ctx = gb.Context(0)
    A = _device32(a)
    T = torch.full((40, 40), float("nan"), dtype=torch.float32, device="cuda").T
    ctx.factor(A, T, gb.GBQR_T_FULL, gb.opts(cutoff_b=16, leaf_rows=leaf, fanout=k))
    torch.cuda.synchronize()
    _gpu.compare_factor(a.astype(np.float64), A.cpu().numpy(), T.cpu().numpy(), gb.GBQR_T_FULL, 40, orc,
                        f"fp32 near pairs leaf={leaf} k={k}", fp32=True)
    ctx.close()

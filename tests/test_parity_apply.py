"""GPU parity of applying Q (gbqr_apply_qt / gbqr_apply_q), the thin Q
(gbqr_form_q) and the least-squares solve (gbqr_ls_solve) with the oracle."""

import numpy as np
import pytest

import workloads
from tests import _gpu

pytestmark = pytest.mark.gpu

TOL_APPLY = 1e-11   # max-norm difference relative to ||B|| column norms
TOL_LS = 1e-12      # ||x - x_orc|| / ||x_orc|| at kappa ~ 10 (forward error ~ kappa u)


@pytest.fixture(scope="module")
def ctx(gb):
    c = gb.Context(0)
    yield c
    c.close()


CASES = [(1024, 128, 0), (1000, 77, 1), (300, 300, 2), (50, 1, 3), (5000, 40, 4)]


@pytest.mark.parametrize("m,n,seed", CASES)
@pytest.mark.parametrize("layout_name", ["full", "panel"])
def test_apply_and_form_q(gb, ctx, orc, m, n, seed, layout_name):
    import torch
    layout = gb.GBQR_T_FULL if layout_name == "full" else gb.GBQR_T_PANEL
    a = workloads.gaussian(m, n, seed)
    b = workloads.gaussian(m, 3, seed + 100)
    vr_o, tau_o = orc.house_qr(a)
    o = gb.opts(panel_nb=32) if layout == gb.GBQR_T_PANEL else None
    nb = 32 if layout == gb.GBQR_T_PANEL else n
    A = _gpu.device_matrix(a)
    T = _gpu.t_buffer(n, layout, nb)
    ctx.factor(A, T, layout, o)
    B = _gpu.device_matrix(b)
    ctx.apply_qt(A, T, B, layout, nb)
    torch.cuda.synchronize()
    qtb = gb.to_numpy(B)
    exp = orc.apply_qt(vr_o, tau_o, b)
    scale = np.linalg.norm(b, axis=0)
    assert np.max(np.abs(qtb - exp) / scale) <= TOL_APPLY
    # Q (Q^T b) = b
    ctx.apply_q(A, T, B, layout, nb)
    torch.cuda.synchronize()
    assert np.max(np.abs(gb.to_numpy(B) - b) / scale) <= TOL_APPLY
    # Q b against the oracle
    B2 = _gpu.device_matrix(b)
    ctx.apply_q(A, T, B2, layout, nb)
    torch.cuda.synchronize()
    assert np.max(np.abs(gb.to_numpy(B2) - orc.apply_q(vr_o, tau_o, b)) / scale) <= TOL_APPLY
    # thin Q
    Q = gb.colmajor(m, n, fill=float("nan"))
    ctx.form_q(A, T, Q, layout, nb)
    torch.cuda.synchronize()
    q = gb.to_numpy(Q)
    assert np.max(np.abs(q - orc.form_q(vr_o, tau_o))) <= TOL_APPLY
    r = np.triu(gb.to_numpy(A)[:n])
    assert np.linalg.norm(a - q @ r) / np.linalg.norm(a) <= _gpu.TOL_BACKWARD
    assert np.linalg.norm(q.T @ q - np.eye(n)) <= _gpu.TOL_BACKWARD


@pytest.mark.parametrize("m,n,nb,layout_name", [
    (1000, 77, 32, "panel"),      # ragged last panel, one CTA per few chunks
    (40000, 300, 128, "panel"),   # ~125 CTAs: two levels of the reduction tree
    (20000, 512, 256, "panel"),   # widest panel the one-vector kernel takes
    (5000, 300, 0, "full"),       # diagonal blocks of the full T
    (64, 64, 16, "panel"),        # square: the last panels span a single chunk
    (50, 1, 1, "panel"),
    (1001, 77, 32, "panel"),      # odd leading dimension: per-lane loads instead of tensor boxes
    (1000, 77, 33, "panel"),      # odd panel width and ldt: T read from global memory
    (3000, 200, 64, "panel"),     # narrower boxes, deeper ring
    (1024, 128, 128, "panel"),    # one panel, one chunk per item: the item's last chunk in ring slot 0
    (16384, 128, 128, "panel"),   # four chunks per item in a three-slot ring
    (1000, 77, 0, "full"),        # full T with an odd panel width: T read from global memory
    (33, 32, 32, "panel"),        # one row past a chunk
    (129, 128, 64, "panel"),      # two panels, the second one row taller than its triangle
])
def test_apply_one_vector(gb, ctx, orc, m, n, nb, layout_name):
    """Q^T b and Q b of a single vector (one persistent launch per
    application) against the oracle, for both directions, ragged panels,
    multi-group share trees, the tensor-box and per-lane-load row paths and
    T staged in shared memory or read from global memory."""
    import torch
    layout = gb.GBQR_T_FULL if layout_name == "full" else gb.GBQR_T_PANEL
    nb = nb if layout == gb.GBQR_T_PANEL else n
    a = workloads.gaussian(m, n, 40 + n)
    b = workloads.gaussian(m, 1, 41 + n)
    vr_o, tau_o = orc.house_qr(a)
    A = _gpu.device_matrix(a)
    T = _gpu.t_buffer(n, layout, nb)
    ctx.factor(A, T, layout, gb.opts(panel_nb=nb) if layout == gb.GBQR_T_PANEL else None)
    scale = np.linalg.norm(b)
    B = _gpu.device_matrix(b)
    ctx.apply_qt(A, T, B, layout, nb)
    torch.cuda.synchronize()
    assert np.max(np.abs(gb.to_numpy(B) - orc.apply_qt(vr_o, tau_o, b))) / scale <= TOL_APPLY
    B2 = _gpu.device_matrix(b)
    ctx.apply_q(A, T, B2, layout, nb)
    torch.cuda.synchronize()
    assert np.max(np.abs(gb.to_numpy(B2) - orc.apply_q(vr_o, tau_o, b))) / scale <= TOL_APPLY
    # deterministic: a second application gives the same bits
    B3 = _gpu.device_matrix(b)
    ctx.apply_q(A, T, B3, layout, nb)
    torch.cuda.synchronize()
    assert torch.equal(B2, B3)


@pytest.mark.parametrize("m,n,seed", [(1024, 128, 0), (777, 100, 5), (256, 256, 6), (3000, 17, 7)])
def test_ls_solve(gb, ctx, orc, m, n, seed):
    import torch
    a = workloads.gaussian(m, n, seed)
    b = workloads.vector(m, seed + 1)
    x_o, res_o = orc.ls_solve(a, b)
    A = _gpu.device_matrix(a)
    bd = torch.from_numpy(b).cuda()
    x = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    st, info = ctx.ls_solve(A, bd, x)
    assert st == gb.GBQR_OK and info.rankdef_col == -1
    xs = x.cpu().numpy()
    kappa = np.linalg.cond(a)
    tol = max(TOL_LS, 50 * kappa * np.finfo(float).eps)
    assert np.linalg.norm(xs - x_o) / np.linalg.norm(x_o) <= tol
    # A is not modified
    assert np.array_equal(gb.to_numpy(A), a)


def test_ls_solve_consistent_system(gb, ctx):
    import torch
    a = workloads.graded(2048, 64, 8, decades=2)
    xs = workloads.vector(64, 9)
    b = a @ xs
    A = _gpu.device_matrix(a)
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    st, _ = ctx.ls_solve(A, torch.from_numpy(b).cuda(), x)
    assert st == gb.GBQR_OK
    kappa = np.linalg.cond(a)
    assert np.linalg.norm(x.cpu().numpy() - xs) / np.linalg.norm(xs) <= 50 * kappa * np.finfo(float).eps


def test_ls_solve_rank_deficient(gb, ctx):
    import torch
    a = workloads.gaussian(100, 10, 10)
    a[:, 3] = 0.0
    A = _gpu.device_matrix(a)
    x = torch.zeros(10, dtype=torch.float64, device="cuda")
    st, info = ctx.ls_solve(A, torch.from_numpy(workloads.vector(100, 11)).cuda(), x)
    assert st == gb.GBQR_ERANKDEF and info.rankdef_col == 3

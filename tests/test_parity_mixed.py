"""Mixed precision (tensor-core split-BF16 trailing updates, FP64 reflectors
and R-merges, FP64 refinement of least squares) against the FP64 oracle.

Tolerances from the arithmetic: the trailing updates carry a relative error
of about 2^-22 (three BF16 slices, FP32 accumulation over K), so the
factorization is that of a matrix within ~1e-7 relative of A: R, V, T agree
with the oracle to ~kappa * 1e-7, while Q stays orthogonal to FP64 accuracy
(every reflector is still generated in FP64).  After refinement on the
augmented system the solution must match the FP64 solution to
max(1e-12, 50 kappa u)."""

import numpy as np
import pytest

import oracle
import workloads
from tests import _gpu

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def ctx(gb):
    c = gb.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("m,n,nb", [(2048, 512, 128), (1000, 300, 64), (4096, 256, 32)])
def test_mixed_factor_close_to_oracle(gb, ctx, orc, m, n, nb):
    import torch
    a = workloads.gaussian(m, n, 60 + nb)
    o = gb.opts(panel_nb=nb, update_prec=gb.GBQR_MIXED_SPLITBF16)
    VR, T, nbr = _gpu.factor_gpu(ctx, a, gb.GBQR_T_PANEL, o)
    st, _ = ctx.sync()
    assert st == gb.GBQR_OK
    V_o, T_o, R_o, _ = orc.qr(a)
    kappa = np.linalg.cond(a)
    tol = 50 * kappa * 2.0 ** -22
    R = np.triu(VR[:n])
    assert np.linalg.norm(R - R_o) / np.linalg.norm(R_o) <= tol
    assert np.max(np.abs(oracle.unpack_v(VR) - V_o)) <= tol
    # orthogonality is still FP64-level: form Q from the mixed (V, T)
    A = _gpu.device_matrix(VR)
    Tt = gb.to_colmajor(T)
    Q = gb.colmajor(m, n)
    ctx.form_q(A, Tt, Q, gb.GBQR_T_PANEL, nbr)
    torch.cuda.synchronize()
    q = gb.to_numpy(Q)
    assert np.linalg.norm(q.T @ q - np.eye(n), 2) <= _gpu.TOL_BACKWARD
    assert np.linalg.norm(a - q @ R) / np.linalg.norm(a) <= tol


@pytest.mark.parametrize("m,n,decades", [(2048, 256, 1.0), (4096, 512, 3.0), (3000, 200, 5.0)])
@pytest.mark.parametrize("prec_name", ["splitbf16", "bf16"])
def test_mixed_least_squares(gb, ctx, orc, m, n, decades, prec_name):
    import torch
    prec = gb.GBQR_MIXED_SPLITBF16 if prec_name == "splitbf16" else gb.GBQR_MIXED_BF16
    a, xt, b = workloads.ls_problem(m, n, decades, 70 + int(decades))
    kappa = np.linalg.cond(a)
    x_o, _ = orc.ls_solve(a, b)
    A = _gpu.device_matrix(a)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, info = ctx.ls_solve(A, torch.from_numpy(b).cuda(), x, prec)
    assert st == gb.GBQR_OK, (st, info.refine_iters, info.refine_last)
    err = np.linalg.norm(x.cpu().numpy() - x_o) / np.linalg.norm(x_o)
    assert err <= max(1e-12, 50 * kappa * EPS), (err, kappa, info.refine_iters)
    assert 1 <= info.refine_iters <= 8 and info.gmres_steps >= 1


def test_fp64_least_squares_takes_no_refinement(gb, ctx, orc):
    import torch
    a, xt, b = workloads.ls_problem(1000, 100, 2.0, 80)
    A = _gpu.device_matrix(a)
    x = torch.zeros(100, dtype=torch.float64, device="cuda")
    st, info = ctx.ls_solve(A, torch.from_numpy(b).cuda(), x, gb.GBQR_FP64)
    assert st == gb.GBQR_OK and info.refine_iters == 0
    x_o, _ = orc.ls_solve(a, b)
    assert np.linalg.norm(x.cpu().numpy() - x_o) / np.linalg.norm(x_o) <= 1e-12


@pytest.mark.parametrize("m,n,kappa", [(1500, 300, 1e8), (700, 700, 1e9)])
def test_gmres_refinement_beyond_classical(gb, ctx, orc, m, n, kappa):
    """kappa(A) u_f > 1 (u_f ~ 2^-22 for three BF16 slices) with no column
    grading to hide it, where classical refinement would diverge: GMRES on
    the augmented system preconditioned by the mixed factors reaches the
    backward error target; the solution matches the oracle within the
    conditioning bound and is as accurate as the FP64 path's."""
    import torch
    a, xt, b = workloads.ls_problem_kappa(m, n, kappa, 95)
    assert np.linalg.cond(a) == pytest.approx(kappa, rel=1e-3)
    x_o, _ = orc.ls_solve(a, b)
    A = _gpu.device_matrix(a)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, info = ctx.ls_solve(A, bd, x, gb.GBQR_MIXED_SPLITBF16)
    assert st == gb.GBQR_OK, (st, info.refine_iters, info.gmres_steps, info.backward_err)
    assert info.gmres_steps > 0
    assert info.backward_err <= 4 * 2.0 ** -53 * (1 + np.sqrt(m))
    x64 = torch.zeros(n, dtype=torch.float64, device="cuda")
    st64, info64 = ctx.ls_solve(A, bd, x64, gb.GBQR_FP64)
    assert st64 == gb.GBQR_OK
    err = np.linalg.norm(x.cpu().numpy() - x_o) / np.linalg.norm(x_o)
    err64 = np.linalg.norm(x64.cpu().numpy() - x_o) / np.linalg.norm(x_o)
    assert err <= max(1e-12, 50 * kappa * EPS), (err, err64, kappa)
    assert err <= 10 * err64 + 1e-13, (err, err64)

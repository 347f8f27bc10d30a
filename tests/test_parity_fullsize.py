"""Parity at the full benchmark sizes (graded 8192 x 8192 and 32768 x 2048), in
the launch configuration bench.py times (GBQR_T_PANEL, default panel width,
look-ahead on), against the oracle's full factorization of the same matrix
(the all-cores build of the oracle, bit-identical to the one-thread build):

  * every entry of V, every column of R (columnwise relative to the column of
    A, and normwise: the stated 1e-10 bound on R), and every panel block of T
    (each the oracle's T of that panel's reflectors, Section 2.3);
  * Q^T b against the oracle's reflectors applied one at a time;
  * properties at full size: ||A - QR||_F / ||A||_F and ||Q^T Q - I||_2
    (Q formed by gbqr_form_q; products and the symmetric eigensolve by
    cuBLAS/cuSOLVER through torch, as checkers only).  The orthogonality
    bound is read for the 2-norm: the Frobenius norm of the n x n error sums
    n^2 rounding-size entries and grows like n;
  * least squares on graded 32768 x 2048 at kappa ~ 1e2 and 1e6, FP64 and
    mixed precision, against the oracle's solution of the same problem.

Measured errors are printed (pytest -s shows them).
"""

import numpy as np
import pytest

import oracle
import workloads
from tests import _gpu

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def ctx(gb):
    c = gb.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def orc_all():
    return oracle.all_cores()


@pytest.mark.parametrize("name", [workloads.SQUARE_8192.name, workloads.TALL_32768x2048.name])
def test_full_size_factorization(gb, ctx, orc_all, name):
    import torch
    w = workloads.WORKLOADS[name]
    a = w.matrix()
    m, n = a.shape
    nb = gb.default_panel_nb(m, n)
    A = gb.to_colmajor(a)
    A0 = A.clone()
    T = gb.colmajor(min(nb, n), n, fill=float("nan"))
    ctx.factor(A, T, gb.GBQR_T_PANEL)
    st, _ = ctx.sync()
    assert st == gb.GBQR_OK
    vr_gpu = gb.to_numpy(A)
    t_gpu = gb.to_numpy(T)

    vr_o, tau_o = orc_all.house_qr(a)
    # V: every entry (the strict lower trapezoids; unit diagonals on both sides)
    dv = 0.0
    for j0 in range(0, n, 512):
        j1 = min(n, j0 + 512)
        dv = max(dv, float(np.max(np.abs(np.tril(vr_gpu[:, j0:j1], -j0 - 1) - np.tril(vr_o[:, j0:j1], -j0 - 1)))))
    # R: every column
    R, R_o = np.triu(vr_gpu[:n]), np.triu(vr_o[:n])
    cn = np.linalg.norm(a, axis=0)
    dr_col = float(np.max(np.linalg.norm(R - R_o, axis=0) / cn))
    dr = float(np.linalg.norm(R - R_o) / np.linalg.norm(R_o))
    # T: every panel block against the oracle's T of that panel's reflectors
    dt = 0.0
    for j0 in range(0, n, nb):
        wd = min(nb, n - j0)
        t_o = orc_all.larft(vr_o[j0:, j0:j0 + wd], tau_o[j0:j0 + wd])
        blk = t_gpu[:wd, j0:j0 + wd]
        dt = max(dt, float(np.max(np.abs(blk - t_o)) / max(1.0, float(np.max(np.abs(t_o))))))
    # Q^T b
    b = workloads.vector(m, 99)
    B = torch.from_numpy(b.copy()).cuda().reshape(-1, 1)
    ctx.apply_qt(A, T, B, gb.GBQR_T_PANEL, nb)
    torch.cuda.synchronize()
    qtb_o = orc_all.apply_qt(vr_o, tau_o, b)
    dq = float(np.max(np.abs(B[:, 0].cpu().numpy() - qtb_o)) / np.linalg.norm(b))
    print(f"\n{name}: max|dV| = {dv:.3e}, R columnwise {dr_col:.3e}, R normwise {dr:.3e}, "
          f"T {dt:.3e}, Q^T b {dq:.3e}")
    assert dv <= _gpu.TOL_V, dv
    assert dr_col <= _gpu.TOL_R_COL, dr_col
    assert dr <= _gpu.TOL_R_NORM, dr
    assert dt <= _gpu.TOL_T, dt
    assert dq <= _gpu.TOL_V, dq

    # properties at full size
    Q = gb.colmajor(m, n, fill=float("nan"))
    ctx.form_q(A, T, Q, gb.GBQR_T_PANEL, nb)
    torch.cuda.synchronize()
    Rt = torch.triu(A[:n, :])
    back = float(torch.linalg.matrix_norm(A0 - Q @ Rt) / torch.linalg.matrix_norm(A0))
    # ||Q^T Q - I||_2 exactly: the largest |eigenvalue| of the symmetric error
    E = Q.T @ Q - torch.eye(n, dtype=torch.float64, device=Q.device)
    E = 0.5 * (E + E.T)
    orth = float(torch.linalg.eigvalsh(E).abs().max())
    print(f"{name}: backward {back:.3e}, orthogonality (2-norm) {orth:.3e}")
    assert back <= _gpu.TOL_BACKWARD, back
    assert orth <= _gpu.TOL_BACKWARD, orth


@pytest.mark.parametrize("decades", [2.0, 6.0])
def test_full_size_least_squares_vs_oracle(gb, ctx, orc_all, decades):
    """Graded 32768 x 2048 least squares, b = A x_true + 1e-8 N(0,1): the FP64
    and the mixed-precision solutions against the oracle's.  Bound (the
    forward error of any backward-stable FP64 solver is ~ kappa u): relative
    difference <= max(1e-12, 50 kappa u), kappa ~ 1.7 * 10^decades for this
    tall Gaussian; the mixed result must also stay within 10x of the FP64
    result's difference plus 1e-13."""
    import torch
    m, n = 32768, 2048
    a, _, b = workloads.ls_problem(m, n, decades, 60 + int(decades))
    x_o, _ = orc_all.ls_solve(a, b)
    A = gb.to_colmajor(a)
    bd = torch.from_numpy(b).cuda()
    kappa = 1.7 * 10.0 ** decades
    bound = max(1e-12, 50.0 * kappa * 2.0 ** -53)
    errs = {}
    for prec in (gb.GBQR_FP64, gb.GBQR_MIXED_SPLITBF16):
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, info = ctx.ls_solve(A, bd, x, prec)
        assert st == gb.GBQR_OK, (prec, st)
        errs[prec] = float(np.linalg.norm(x.cpu().numpy() - x_o) / np.linalg.norm(x_o))
    print(f"\nLS 32768x2048, 10^{decades:g} grading: FP64 vs oracle {errs[gb.GBQR_FP64]:.3e}, "
          f"mixed vs oracle {errs[gb.GBQR_MIXED_SPLITBF16]:.3e} (bound {bound:.1e})")
    assert errs[gb.GBQR_FP64] <= bound
    assert errs[gb.GBQR_MIXED_SPLITBF16] <= bound
    assert errs[gb.GBQR_MIXED_SPLITBF16] <= 10.0 * errs[gb.GBQR_FP64] + 1e-13


def test_full_size_least_squares(gb, ctx, orc):
    """32768 x 2048 Gaussian: a consistent system recovers x, and an
    inconsistent one satisfies the normal equations A^T (b - A x) = 0."""
    import torch
    m, n = 32768, 2048
    a = workloads.gaussian(m, n, 31)
    xs = workloads.vector(n, 32)
    A = gb.to_colmajor(a)
    Ad = A.clone()
    b = torch.from_numpy(a @ xs).cuda()
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, info = ctx.ls_solve(A, b, x)
    assert st == gb.GBQR_OK
    err = float(torch.linalg.norm(x.cpu() - torch.from_numpy(xs)) / np.linalg.norm(xs))
    assert err <= 1e-12, err
    r_rhs = torch.from_numpy(workloads.vector(m, 33)).cuda()
    st, _ = ctx.ls_solve(A, r_rhs, x)
    assert st == gb.GBQR_OK
    res = r_rhs - Ad @ x
    ne = float(torch.linalg.norm(Ad.T @ res)) / (float(torch.linalg.matrix_norm(Ad)) * float(torch.linalg.norm(r_rhs)))
    assert ne <= 1e-13, ne

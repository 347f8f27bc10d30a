"""Parity at the full benchmark sizes (graded 8192 x 8192 and 32768 x 2048), in
the launch configuration bench.py times (GBQR_T_PANEL, default panel width,
look-ahead on).  The oracle cannot factor these in seconds, so:

  * sampled outputs the oracle computes exactly: the leading 64 columns.  The
    first k reflectors, R(0:k, 0:k) and T(0:k, 0:k) depend only on A(:, 0:k),
    so the oracle's QR of the m x 64 leading block is the expected value;
  * properties at full size: ||A - QR||_F / ||A||_F and ||Q^T Q - I||_2
    (Q formed by gbqr_form_q; products and the symmetric eigensolve by
    cuBLAS/cuSOLVER through torch, as checkers only), and Q (Q^T b) = b.
    The orthogonality bound is read for the 2-norm: the Frobenius norm of
    the n x n error sums n^2 rounding-size entries and grows like n.
"""

import numpy as np
import pytest

import oracle
import workloads
from tests import _gpu

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

K_SAMPLE = 64


@pytest.fixture(scope="module")
def ctx(gb):
    c = gb.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("name", [workloads.SQUARE_8192.name, workloads.TALL_32768x2048.name])
def test_full_size_factorization(gb, ctx, orc, name):
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

    # sampled: the leading K columns against the oracle
    vr_s, tau_s = orc.house_qr(a[:, :K_SAMPLE])
    V_o = oracle.unpack_v(vr_s)
    T_o = orc.larft(vr_s, tau_s)
    lead = gb.to_numpy(A[:, :K_SAMPLE])
    V = oracle.unpack_v(lead)
    assert np.max(np.abs(V - V_o)) <= _gpu.TOL_V
    R = np.triu(lead[:K_SAMPLE])
    R_o = np.triu(vr_s[:K_SAMPLE])
    cn = np.linalg.norm(a[:, :K_SAMPLE], axis=0)
    assert np.max(np.linalg.norm(R - R_o, axis=0) / cn) <= _gpu.TOL_R_COL
    assert np.linalg.norm(R - R_o) / np.linalg.norm(R_o) <= _gpu.TOL_R_NORM
    Tk = gb.to_numpy(T[:K_SAMPLE, :K_SAMPLE])
    assert np.max(np.abs(Tk - T_o)) / max(1.0, np.max(np.abs(T_o))) <= _gpu.TOL_T

    # properties at full size
    Q = gb.colmajor(m, n, fill=float("nan"))
    ctx.form_q(A, T, Q, gb.GBQR_T_PANEL, nb)
    torch.cuda.synchronize()
    Rt = torch.triu(A[:n, :])
    back = torch.linalg.matrix_norm(A0 - Q @ Rt) / torch.linalg.matrix_norm(A0)
    # ||Q^T Q - I||_2 exactly: the largest |eigenvalue| of the symmetric error
    E = Q.T @ Q - torch.eye(n, dtype=torch.float64, device=Q.device)
    E = 0.5 * (E + E.T)
    orth = torch.linalg.eigvalsh(E).abs().max()
    assert float(back) <= _gpu.TOL_BACKWARD, float(back)
    assert float(orth) <= _gpu.TOL_BACKWARD, float(orth)

    b = torch.from_numpy(workloads.vector(m, 99)).cuda()
    B = b.clone().reshape(-1, 1)
    ctx.apply_qt(A, T, B, gb.GBQR_T_PANEL, nb)
    assert abs(float(torch.linalg.norm(B)) - float(torch.linalg.norm(b))) <= 1e-13 * float(torch.linalg.norm(b))
    ctx.apply_q(A, T, B, gb.GBQR_T_PANEL, nb)
    torch.cuda.synchronize()
    assert float(torch.max(torch.abs(B[:, 0] - b))) <= 1e-12 * float(torch.linalg.norm(b))


def test_full_size_least_squares(gb, ctx, orc):
    """32768 x 2048 Gaussian least squares: x against the oracle's solution of
    the same problem restricted to its leading 256 columns would be a
    different problem, so check the normal equations and a consistent system."""
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
    # inconsistent system: normal equations A^T (b - A x) = 0
    r_rhs = torch.from_numpy(workloads.vector(m, 33)).cuda()
    st, _ = ctx.ls_solve(A, r_rhs, x)
    assert st == gb.GBQR_OK
    res = r_rhs - Ad @ x
    ne = float(torch.linalg.norm(Ad.T @ res)) / (float(torch.linalg.matrix_norm(Ad)) * float(torch.linalg.norm(r_rhs)))
    assert ne <= 1e-13, ne

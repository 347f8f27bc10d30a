"""Helpers for the GPU parity tests: run the CUDA path through the C ABI on
seeded inputs and compare with the oracle.

Tolerances (FP64, u = 2^-53 ~ 1.1e-16).  Both sides are backward-stable
Householder QR variants that reach the same (V, T, R) in exact arithmetic
(the TSQR reconstruction reproduces the unblocked Householder vectors under
the shared sign convention), so their difference is a rounding effect of
order kappa * u * (a modest function of m, n).  For the seeded Gaussian
and graded inputs used here (kappa of the column-equilibrated matrix below
~1e3) that is far below 1e-11; a wrong index, sign or term shows up at O(1).
"""

from __future__ import annotations

import numpy as np

import oracle

TOL_V = 1e-11          # max |V_gpu - V_orc|, entries of V are bounded by 1
TOL_T = 1e-11          # max |T_gpu - T_orc| / max(1, max |T_orc|)
TOL_R_COL = 1e-11      # max_j ||R_gpu(:,j) - R_orc(:,j)|| / ||A(:,j)||
TOL_R_NORM = 1e-10     # ||R_gpu - R_orc||_F / ||R_orc||_F (the stated R agreement bound)
TOL_BACKWARD = 1e-13   # ||A - QR||_F / ||A||_F and ||Q^T Q - I||_F

# FP32 (u32 = 2^-24 ~ 6.0e-8): the same argument with u32 for u.  The FP64
# bounds above sit ~4.5e4 u above zero; FP32 results are held to ~3e4 u32,
# and the oracle runs in FP64 on the same float32-rounded input, so the only
# difference left is FP32 rounding in the CUDA path.
TOL32_V = 2e-3
TOL32_T = 2e-3
TOL32_R_COL = 2e-3
TOL32_R_NORM = 2e-3
TOL32_BACKWARD = 2e-5


def device_matrix(a: np.ndarray, lda_pad: int = 0):
    """Column-major CUDA copy of a with leading dimension m + lda_pad."""
    import torch
    m, n = a.shape
    buf = torch.full((max(n, 1), m + lda_pad), float("nan"), dtype=torch.float64, device="cuda")
    A = buf.T[:m, :n]
    A.copy_(torch.from_numpy(np.asfortranarray(a)).to("cuda"))
    return A


def t_buffer(n: int, layout: int, nb: int):
    import paper_1805_05278_gb300 as gb
    rows = n if layout == gb.GBQR_T_FULL else max(1, min(nb, n))
    return gb.colmajor(rows, n, fill=float("nan"))


def factor_gpu(ctx, a: np.ndarray, layout: int, o=None, lda_pad: int = 0):
    """Returns (VR, T, nb) as numpy arrays after gbqr_factor on the device."""
    import torch
    import paper_1805_05278_gb300 as gb
    m, n = a.shape
    nb = (o.panel_nb if (o is not None and o.panel_nb) else gb.default_panel_nb(m, n))
    A = device_matrix(a, lda_pad)
    T = t_buffer(n, layout, nb)
    ctx.factor(A, T, layout, o)
    torch.cuda.synchronize()
    return gb.to_numpy(A), gb.to_numpy(T), nb


def panel_blocks_of(t_full: np.ndarray, nb: int) -> np.ndarray:
    """The nb x n panel layout built from the diagonal blocks of a full T."""
    n = t_full.shape[0]
    rows = max(1, min(nb, n))
    out = np.zeros((rows, n))
    for j0 in range(0, n, nb):
        w = min(nb, n - j0)
        out[:w, j0:j0 + w] = t_full[j0:j0 + w, j0:j0 + w]
    return out


def compare_factor(a, VR, T, layout, nb, orc, label="", fp32=False):
    import paper_1805_05278_gb300 as gb
    tol_v, tol_rc, tol_rn, tol_t = ((TOL32_V, TOL32_R_COL, TOL32_R_NORM, TOL32_T) if fp32
                                    else (TOL_V, TOL_R_COL, TOL_R_NORM, TOL_T))
    a = np.asarray(a, dtype=np.float64)
    VR = np.asarray(VR, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    m, n = a.shape
    V_o, T_o, R_o, _ = orc.qr(a)
    V = oracle.unpack_v(VR)
    R = np.triu(VR[:n, :])
    dv = np.max(np.abs(V - V_o)) if V.size else 0.0
    assert dv <= tol_v, f"{label} V differs by {dv}"
    cn = np.maximum(np.linalg.norm(a, axis=0), np.finfo(float).tiny)
    dr_col = np.max(np.linalg.norm(R - R_o, axis=0) / cn) if n else 0.0
    assert dr_col <= tol_rc, f"{label} R differs (columnwise) by {dr_col}"
    if n:
        dr = np.linalg.norm(R - R_o) / max(np.linalg.norm(R_o), np.finfo(float).tiny)
        assert dr <= tol_rn, f"{label} R differs (normwise) by {dr}"
    T_exp = T_o if layout == gb.GBQR_T_FULL else panel_blocks_of(T_o, nb)
    scale = max(1.0, float(np.max(np.abs(T_exp)))) if T_exp.size else 1.0
    dt = np.max(np.abs(T - T_exp)) / scale if T_exp.size else 0.0
    assert dt <= tol_t, f"{label} T differs by {dt}"
    return dv, dr_col, dt


BATCH_B = 16   # default cutoff of gbqr_factor_batched: the persistent engine's panel width


def q_from_panels(VR: np.ndarray, T: np.ndarray, nb: int) -> np.ndarray:
    """Thin Q = Q_0 Q_1 ... [I; 0] from packed V\\R and the panel-layout T
    (Q_k = I - V_k T_k V_k^T, panel k = columns k nb .. k nb + w_k - 1),
    formed in FP64 on the host (a checker only)."""
    VR = np.asarray(VR, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    m, n = VR.shape
    V = oracle.unpack_v(VR)
    Q = np.zeros((m, n))
    Q[np.arange(n), np.arange(n)] = 1.0
    for j0 in reversed(range(0, n, nb)):
        w = min(nb, n - j0)
        Vk = V[:, j0:j0 + w]
        Tk = np.triu(T[:w, j0:j0 + w])
        Q -= Vk @ (Tk @ (Vk.T @ Q))
    return Q

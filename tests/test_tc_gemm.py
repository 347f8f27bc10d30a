"""Numerics of the tensor-core split-BF16 GEMM (gbqr_gemm_split_bf16) against
an FP64 product of the same operands (torch on the GPU as the reference).

Error model: with s slices per operand the representation error of each
operand is ~2^(-8 s) relative, the dropped slice products contribute about
the same, and FP32 accumulation over K adds ~K 2^-24 in the worst case (far
less on average).  The test bounds ||C - C_ref||_F / || |A| |B| ||_F."""

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

TOL = {1: 1.6e-2, 2: 2e-4, 3: 2e-6}


@pytest.fixture(scope="module")
def ctx(gb):
    c = gb.Context(0)
    yield c
    c.close()


SHAPES = [
    # M, N, K, transa
    (128, 128, 64, True),
    (128, 128, 64, False),
    (200, 300, 1000, True),
    (200, 300, 1000, False),
    (1, 1, 1, True),
    (130, 70, 65, False),
    (128, 4000, 8192, True),     # the W1 = V^T A_trail shape of the update (split-K)
    (8192, 640, 128, False),     # the A_trail -= V W2 shape
    (33, 257, 3000, True),
]


@pytest.mark.parametrize("M,N,K,ta", SHAPES)
@pytest.mark.parametrize("ns", [1, 2, 3])
def test_split_bf16_gemm(gb, ctx, M, N, K, ta, ns):
    import torch
    rng = np.random.default_rng(M * 7 + N * 3 + K + ns)
    a = rng.standard_normal((K, M) if ta else (M, K))
    b = rng.standard_normal((K, N))
    c0 = rng.standard_normal((M, N))
    A = gb.to_colmajor(a)
    B = gb.to_colmajor(b)
    C = gb.to_colmajor(c0)
    alpha, beta = -1.25, 0.5
    ctx.gemm_split_bf16(A, B, C, transa=ta, alpha=alpha, beta=beta, nsplit=ns)
    st, _ = ctx.sync()
    assert st == gb.GBQR_OK
    opa = A.T if ta else A
    ref = alpha * (opa @ B) + beta * torch.from_numpy(c0).cuda()
    scale = float(torch.linalg.matrix_norm(torch.abs(opa) @ torch.abs(B))) * abs(alpha)
    err = float(torch.linalg.matrix_norm(C - ref)) / scale
    assert err <= TOL[ns], (err, ns)


def test_basis_shaped_operand(gb, ctx):
    """A unit lower trapezoidal basis V (the update's left operand), V^T C."""
    import torch
    m, kv, nc = 1000, 96, 300
    v = workloads.gaussian(m, kv, 3)
    cmat = workloads.gaussian(m, nc, 4)
    V = gb.to_colmajor(v)
    Cm = gb.to_colmajor(cmat)
    W = gb.colmajor(kv, nc)
    vm = np.tril(v, -1)
    vm[np.arange(kv), np.arange(kv)] = 1.0
    ctx.gemm_split_bf16(gb.to_colmajor(vm), Cm, W, transa=True, nsplit=3)
    st, _ = ctx.sync()
    assert st == gb.GBQR_OK
    ref = torch.from_numpy(vm.T @ cmat).cuda()
    err = float(torch.linalg.matrix_norm(W - ref)) / float(torch.linalg.matrix_norm(ref))
    assert err <= 1e-5

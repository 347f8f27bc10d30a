"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds input generation only: no step of the QR method is computed
here, so neither side of a parity check can inherit a mistake from the other
through it.

Every matrix is float64, column-major (Fortran order), drawn from
``numpy.random.default_rng(seed)`` (PCG64).  The shapes and distributions follow
the workloads of the QR method (tall-skinny TSQR panels, square and tall
matrices with graded column scales); the paper itself measures no dataset, so
these seeded draws are the whole input story.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def gaussian(m: int, n: int, seed: int) -> np.ndarray:
    """m x n matrix, entries iid N(0,1), Fortran order.

    Drawn row-major as (n, m) and transposed so that each column is one
    contiguous run of the generator's stream.
    """
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((n, m)).T)


def column_scales(n: int, decades: float = 6.0) -> np.ndarray:
    """Scale 10**(-decades * j / n) for 0-based column j (graded columns)."""
    j = np.arange(n, dtype=np.float64)
    return 10.0 ** (-decades * j / max(n, 1))


def graded(m: int, n: int, seed: int, decades: float = 6.0) -> np.ndarray:
    """Gaussian m x n with column j scaled by 10**(-decades*j/n)."""
    a = gaussian(m, n, seed)
    a *= column_scales(n, decades)[None, :]
    return a


def vector(m: int, seed: int) -> np.ndarray:
    """Right-hand side b, iid N(0,1)."""
    return np.random.default_rng(seed).standard_normal(m)


def upper_triangular(m: int, n: int, seed: int) -> np.ndarray:
    """m x n with a random upper triangle in its top n rows and zeros elsewhere."""
    a = gaussian(m, n, seed)
    a[np.tril_indices(m, -1, n)] = 0.0
    return np.asfortranarray(a)


def random_reflector_product(m: int, n: int, seed: int) -> np.ndarray:
    """m x n matrix with orthonormal columns: leading n columns of a product of
    n random elementary reflectors I - 2 u u^T / (u^T u), applied to [I; 0].

    Formed by plain reflector products (not a QR routine), so that an
    orthogonal test input does not depend on any QR implementation.
    """
    rng = np.random.default_rng(seed)
    q = np.zeros((m, n))
    q[:n, :n] = np.eye(n)
    for _ in range(n):
        u = rng.standard_normal(m)
        q -= np.outer(u, (2.0 / (u @ u)) * (u @ q))
    return np.asfortranarray(q)


def ls_problem(m: int, n: int, decades: float, seed: int, noise: float = 1e-8):
    """Least-squares test problem: A Gaussian m x n with column j scaled by
    10**(-decades*j/n) (condition number about 10**decades times that of the
    Gaussian), x_true iid N(0,1), b = A x_true + noise * N(0,1).
    Returns (A, x_true, b)."""
    a = graded(m, n, seed, decades)
    rng = np.random.default_rng(seed + 1)
    x_true = rng.standard_normal(n)
    b = a @ x_true + noise * rng.standard_normal(m)
    return a, x_true, b


def ls_problem_kappa(m: int, n: int, kappa: float, seed: int, noise: float = 1e-8):
    """Least-squares problem with prescribed singular values: A = Q1 diag(s)
    Q2^T with Q1 (m x n) and Q2 (n x n) orthonormal products of random
    reflectors and s_j = kappa^(-j/(n-1)) (so kappa_2(A) = kappa exactly and
    no column scaling carries the ill-conditioning).  x_true iid N(0,1),
    b = A x_true + noise * N(0,1).  Returns (A, x_true, b)."""
    q1 = random_reflector_product(m, n, seed)
    q2 = random_reflector_product(n, n, seed + 1)
    s = kappa ** (-np.arange(n, dtype=np.float64) / max(n - 1, 1))
    a = np.asfortranarray((q1 * s[None, :]) @ q2.T)
    rng = np.random.default_rng(seed + 2)
    x_true = rng.standard_normal(n)
    b = a @ x_true + noise * rng.standard_normal(m)
    return a, x_true, b


@dataclass(frozen=True)
class Workload:
    """One named workload: A (m x n) and an optional right-hand side b."""
    name: str
    m: int
    n: int
    seed: int
    graded: bool
    rhs_seed: int | None = None

    def matrix(self) -> np.ndarray:
        if self.graded:
            return graded(self.m, self.n, self.seed)
        return gaussian(self.m, self.n, self.seed)

    def rhs(self) -> np.ndarray | None:
        return None if self.rhs_seed is None else vector(self.m, self.rhs_seed)

    @property
    def flops(self) -> float:
        """Algorithmic Householder QR flop count 2mn^2 - 2n^3/3."""
        return qr_flops(self.m, self.n)


def qr_flops(m: int, n: int) -> float:
    return 2.0 * m * n * n - 2.0 * n ** 3 / 3.0


def qr_flops_partial(m: int, n: int, k: int) -> float:
    """Flops credited to the first k of n Householder steps: the whole count
    minus the count of the (m-k) x (n-k) problem that remains."""
    return qr_flops(m, n) - qr_flops(m - k, n - k)


# Named workloads: a 1024 x 128 Gaussian with a Gaussian right-hand side (the
# small case an unblocked CPU QR finishes in well under a second), and the two
# large graded shapes (tall 32768 x 2048 and square 8192 x 8192, columns
# scaled by 10^(-6j/n)).
SMALL_1024x128 = Workload("gaussian_1024x128", 1024, 128, seed=0, graded=False, rhs_seed=1)
TALL_32768x2048 = Workload("graded_32768x2048", 32768, 2048, seed=2, graded=True)
SQUARE_8192 = Workload("graded_8192x8192", 8192, 8192, seed=3, graded=True)
# A quarter-size square case for profiling captures (134 MB: still larger than L2).
SQUARE_4096 = Workload("graded_4096x4096", 4096, 4096, seed=4, graded=True)

WORKLOADS = {w.name: w for w in (SMALL_1024x128, TALL_32768x2048, SQUARE_8192, SQUARE_4096)}


def log_uniform_int(rng: np.random.Generator, lo: int, hi: int) -> int:
    return int(math.floor(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def batched_shapes(count: int = 2000, seed: int = 20, m_range=(256, 16384), n_range=(16, 256)):
    """Shapes of the batched tall-skinny workload: m log-uniform in m_range,
    n uniform in n_range (inclusive), n <= m (resampled otherwise)."""
    rng = np.random.default_rng(seed)
    shapes = []
    while len(shapes) < count:
        m = log_uniform_int(rng, *m_range)
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        if n <= m:
            shapes.append((m, n))
    return shapes


def batched_device_buffer(shapes, seed: int, device="cuda"):
    """All matrices of a batch in one contiguous float64 device buffer (iid
    N(0,1) from a seeded torch generator); returns (buffer, offsets): matrix
    i is column-major m_i x n_i starting at offsets[i] with ld = m_i."""
    import torch
    sizes = [m * n for (m, n) in shapes]
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    buf = torch.randn(int(offsets[-1]), dtype=torch.float64, device=device, generator=gen)
    return buf, offsets[:-1]


# The batched workload: 2000 tall-skinny matrices.
BATCHED_SEED = 20
SERVING_SEED = 30


def serving_specs(count: int, seed: int = SERVING_SEED, m_range=(512, 65536), n_range=(32, 1024),
                  kappa_range=(1e1, 1e8)):
    """Least-squares requests of the serving workload: m, n log-uniform
    (n <= m, resampled otherwise), target condition number log-uniform, set
    by grading the columns of a Gaussian matrix over log10(kappa) decades."""
    rng = np.random.default_rng(seed)
    specs = []
    while len(specs) < count:
        m = log_uniform_int(rng, *m_range)
        n = log_uniform_int(rng, *n_range)
        if n > m:
            continue
        kappa = math.exp(rng.uniform(math.log(kappa_range[0]), math.log(kappa_range[1])))
        specs.append((m, n, math.log10(kappa)))
    return specs


def serving_device_problem(m: int, n: int, decades: float, seed: int, device="cuda", noise: float = 1e-8):
    """(A, x_true, b) on the device: A Gaussian with column j scaled by
    10**(-decades*j/n), b = A x_true + noise N(0,1); seeded torch generator."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    a = torch.randn((n, m), dtype=torch.float64, device=device, generator=gen).T
    a *= torch.from_numpy(column_scales(n, decades)).to(device)[None, :]
    xt = torch.randn(n, dtype=torch.float64, device=device, generator=gen)
    b = a @ xt + noise * torch.randn(m, dtype=torch.float64, device=device, generator=gen)
    return a, xt, b

"""Pins for the CPU oracle: checks that tie it to mathematics and to
independent libraries rather than to itself.

Each ``pin_*`` takes an ``oracle.Oracle`` and raises AssertionError when the
oracle is wrong.  The set is chosen so that a plausible mistake anywhere in
``oracle/house.c`` (a dropped term, a flipped sign, a transposed index)
fails at least one of them; ``test_oracle_mutations.py`` plants such
mistakes in a copy of the source and checks exactly that.
"""

from __future__ import annotations

from decimal import Decimal, getcontext

import numpy as np

import oracle as _oracle
import workloads

EPS = np.finfo(np.float64).eps


def explicit_q(vr: np.ndarray, tau: np.ndarray) -> np.ndarray:
    """Full m x m Q = H_0 H_1 ... H_{n-1} multiplied out from its definition
    (Section 2.3: product of reflectors H_j = I - tau_j v_j v_j^T)."""
    m, n = vr.shape
    v = _oracle.unpack_v(vr)
    q = np.eye(m)
    for j in range(n):
        h = np.eye(m) - tau[j] * np.outer(v[:, j], v[:, j])
        q = q @ h
    return q


def gram_schmidt_decimal(a: np.ndarray, digits: int = 60):
    """Classical Gram-Schmidt in decimal arithmetic with `digits` significant
    digits: the textbook QR with positive diagonal, brute force."""
    getcontext().prec = digits
    m, n = a.shape
    cols = [[Decimal(float(a[i, j])) for i in range(m)] for j in range(n)]
    qs, r = [], [[Decimal(0)] * n for _ in range(n)]
    for j in range(n):
        v = list(cols[j])
        for i in range(j):
            rij = sum(qs[i][k] * cols[j][k] for k in range(m))
            r[i][j] = rij
            v = [v[k] - rij * qs[i][k] for k in range(m)]
        rjj = sum(x * x for x in v).sqrt()
        r[j][j] = rjj
        qs.append([x / rjj for x in v])
    q = np.array([[float(qs[j][i]) for j in range(n)] for i in range(m)])
    rr = np.array([[float(r[i][j]) for j in range(n)] for i in range(n)])
    return q, rr


def pin_gram_schmidt_tiny(orc):
    """Sign-normalised R and Q match brute-force Gram-Schmidt (60 digits)."""
    for (m, n, seed) in [(1, 1, 11), (3, 2, 12), (5, 3, 13), (8, 6, 14), (6, 6, 15), (7, 1, 16), (4, 4, 17)]:
        a = workloads.gaussian(m, n, seed)
        vr, tau = orc.house_qr(a)
        r = np.triu(vr[:n, :])
        q = orc.form_q(vr, tau)
        rn, qn = _oracle.sign_normalise(r, q)
        q_gs, r_gs = gram_schmidt_decimal(a)
        scale = np.linalg.norm(a)
        assert np.max(np.abs(rn - r_gs)) <= 1e-13 * scale, (m, n)
        assert np.max(np.abs(qn - q_gs)) <= 1e-13, (m, n)


def pin_cholesky(orc):
    """R^T R = A^T A, and sign-normalised R = chol(A^T A)^T (uniqueness of
    the Cholesky factor); numpy's LAPACK Cholesky is the independent side."""
    for (m, n, seed) in [(120, 40, 21), (64, 64, 22), (300, 17, 23)]:
        a = workloads.gaussian(m, n, seed)
        vr, _ = orc.house_qr(a)
        r = np.triu(vr[:n, :])
        ata = a.T.astype(np.longdouble) @ a.astype(np.longdouble)
        rtr = r.T.astype(np.longdouble) @ r.astype(np.longdouble)
        assert float(np.max(np.abs(rtr - ata))) <= 1e-14 * n * float(np.max(np.abs(ata)))
        rn, _ = _oracle.sign_normalise(r)
        c = np.linalg.cholesky(a.T @ a).T
        kappa2 = np.linalg.cond(a) ** 2
        assert np.linalg.norm(rn - c) <= 10 * kappa2 * EPS * np.linalg.norm(c) * n


def pin_lapack_elementwise(orc):
    """V, tau and R match LAPACK's dgeqrf (numpy qr mode='raw') element by
    element: same reflector sign convention for inputs with no zero subcolumn."""
    for (m, n, seed, g) in [(50, 20, 31, False), (200, 64, 32, True), (33, 33, 33, False), (97, 5, 34, True)]:
        a = workloads.graded(m, n, seed) if g else workloads.gaussian(m, n, seed)
        vr, tau = orc.house_qr(a)
        h, tl = np.linalg.qr(a, mode="raw")
        h = np.array(h.T, order="F")
        if m == n:
            # the last reflector of a square matrix has an empty subcolumn:
            # LAPACK takes the identity (tau = 0), the oracle's sign reading
            # takes tau = 2, which negates R(n-1, n-1) and nothing else.
            assert tl[-1] == 0.0 and tau[-1] == 2.0
            tl = tl.copy()
            tl[-1] = 2.0
            h[n - 1, n - 1] = -h[n - 1, n - 1]
        assert np.max(np.abs(tau - tl)) <= 1e-13
        assert np.max(np.abs(np.tril(vr, -1) - np.tril(h, -1))) <= 1e-12
        rcol = np.linalg.norm(a, axis=0)
        rdiff = np.abs(np.triu(vr[:n]) - np.triu(h[:n])) / rcol[None, :]
        assert np.max(rdiff) <= 1e-13


def pin_orthogonal_input(orc):
    """Orthonormal columns give |R| = I."""
    for (m, n, seed) in [(40, 12, 41), (16, 16, 42)]:
        a = workloads.random_reflector_product(m, n, seed)
        vr, _ = orc.house_qr(a)
        r = np.triu(vr[:n, :])
        assert np.max(np.abs(np.abs(np.diag(r)) - 1.0)) <= 1e-14 * n
        assert np.max(np.abs(r - np.diag(np.diag(r)))) <= 1e-14 * n


def pin_upper_triangular(orc):
    """An upper triangular input has zero subcolumns: under the sign reading
    every reflector is I - 2 e_j e_j^T, V has no entries below the diagonal
    and R = -A (top n rows)."""
    m, n = 30, 9
    a = workloads.upper_triangular(m, n, 51)
    vr, tau = orc.house_qr(a)
    assert np.all(tau == 2.0)
    assert np.all(np.tril(vr, -1) == 0.0)
    assert np.array_equal(np.triu(vr[:n]), -a[:n])


def pin_zero_column(orc):
    """An exactly zero column (rank deficiency) still gives a valid QR, and
    under the sign reading its reflector is v = e_j, tau = 2, R_jj = 0."""
    m, n, j = 20, 6, 2
    a = workloads.gaussian(m, n, 141)
    a[:, j] = 0.0
    vr, tau = orc.house_qr(a)
    assert tau[j] == 2.0 and vr[j, j] == 0.0
    assert np.all(vr[j + 1:, j] == 0.0)
    q = orc.form_q(vr, tau)
    r = np.triu(vr[:n])
    assert np.linalg.norm(a - q @ r) <= 1e-14 * n * np.linalg.norm(a)
    assert np.linalg.norm(q.T @ q - np.eye(n)) <= 1e-14 * n
    # row j of R: the reflector negated what the previous ones left there
    vr_k, tau_k = orc.house_qr(a[:, :j])
    before = orc.apply_qt(vr_k, tau_k, a)
    assert np.max(np.abs(r[j, j + 1:] + before[j, j + 1:])) <= 1e-13 * np.linalg.norm(a)


def pin_single_column(orc):
    """n = 1: the reflector maps a to beta e_1 with |beta| = ||a||, and beta
    has the sign opposite to a_1 (no cancellation)."""
    for seed in (61, 62, 63):
        a = workloads.gaussian(25, 1, seed)
        vr, tau = orc.house_qr(a)
        v = _oracle.unpack_v(vr)[:, 0]
        h = np.eye(25) - tau[0] * np.outer(v, v)
        ha = h @ a[:, 0]
        beta = vr[0, 0]
        assert abs(abs(beta) - np.linalg.norm(a)) <= 1e-14 * np.linalg.norm(a)
        assert np.sign(beta) == -np.sign(a[0, 0])
        assert np.max(np.abs(ha[1:])) <= 1e-14 * np.linalg.norm(a)
        assert abs(ha[0] - beta) <= 1e-14 * np.linalg.norm(a)


def pin_reflectors(orc):
    """Each H_j is an exact reflector: tau_j * v_j^T v_j = 2."""
    a = workloads.graded(80, 30, 71)
    vr, tau = orc.house_qr(a)
    v = _oracle.unpack_v(vr)
    assert np.max(np.abs(tau * np.sum(v * v, axis=0) - 2.0)) <= 1e-14 * 30


def pin_backward_error(orc):
    """||A - QR||_F/||A||_F and ||Q^T Q - I||_F at most 1e-14 * n."""
    for (m, n, seed, g) in [(300, 100, 81, True), (128, 128, 82, False), (1000, 40, 83, False)]:
        a = workloads.graded(m, n, seed) if g else workloads.gaussian(m, n, seed)
        vr, tau = orc.house_qr(a)
        q = orc.form_q(vr, tau)
        r = np.triu(vr[:n])
        assert np.linalg.norm(a - q @ r) / np.linalg.norm(a) <= 1e-14 * n
        assert np.linalg.norm(q.T @ q - np.eye(n)) <= 1e-14 * n


def pin_t_two_ways(orc):
    """T by forward recurrence equals T by the closed form of Section 2.3,
    and I - V T V^T equals the explicit product of the reflectors."""
    for (m, n, seed) in [(60, 25, 91), (25, 25, 92), (9, 2, 93)]:
        a = workloads.gaussian(m, n, seed)
        vr, tau = orc.house_qr(a)
        t1 = orc.larft(vr, tau)
        t2 = orc.t_from_gram(vr)
        assert np.max(np.abs(t1 - t2)) <= 1e-13 * max(1.0, np.max(np.abs(t1)))
        assert np.all(np.tril(t1, -1) == 0.0)
        v = _oracle.unpack_v(vr)
        qx = explicit_q(vr, tau)
        assert np.max(np.abs(np.eye(m) - v @ t1 @ v.T - qx)) <= 1e-13


def pin_apply(orc):
    """apply_qt / apply_q / form_q agree with the explicit reflector product."""
    m, n = 45, 20
    a = workloads.gaussian(m, n, 101)
    b = workloads.gaussian(m, 3, 102)
    vr, tau = orc.house_qr(a)
    qx = explicit_q(vr, tau)
    assert np.max(np.abs(orc.apply_qt(vr, tau, b) - qx.T @ b)) <= 1e-13
    assert np.max(np.abs(orc.apply_q(vr, tau, b) - qx @ b)) <= 1e-13
    assert np.max(np.abs(orc.form_q(vr, tau) - qx[:, :n])) <= 1e-13
    assert np.max(np.abs(orc.apply_q(vr, tau, orc.apply_qt(vr, tau, b)) - b)) <= 1e-13


def pin_ls(orc):
    """Least squares: matches numpy.linalg.lstsq (LAPACK), recovers x* of a
    consistent system, and satisfies the normal equations A^T r = 0."""
    for (m, n, seed) in [(200, 30, 111), (64, 64, 112), (500, 7, 113)]:
        a = workloads.gaussian(m, n, seed)
        b = workloads.vector(m, seed + 1000)
        x, res = orc.ls_solve(a, b)
        xl = np.linalg.lstsq(a, b, rcond=None)[0]
        kappa = np.linalg.cond(a)
        assert np.linalg.norm(x - xl) <= 100 * kappa * EPS * np.linalg.norm(xl) * (1 + kappa * np.linalg.norm(a @ xl - b) / (np.linalg.norm(a) * np.linalg.norm(xl)))
        r = b - a @ x
        assert abs(res - np.linalg.norm(r)) <= 1e-12 * np.linalg.norm(b)
        assert np.linalg.norm(a.T @ r) <= 1e-13 * n * np.linalg.norm(a) * np.linalg.norm(b)
        xs = workloads.vector(n, seed + 2000)
        x2, res2 = orc.ls_solve(a, a @ xs)
        assert np.linalg.norm(x2 - xs) <= 100 * kappa * EPS * np.linalg.norm(xs)
        assert res2 <= 1e-13 * np.linalg.norm(a @ xs)


def pin_trsv(orc):
    """Back substitution solves R x = c (checked by multiplying back)."""
    n = 40
    r = np.triu(workloads.gaussian(n, n, 121)) + 5 * np.eye(n)
    c = workloads.vector(n, 122)
    x = orc.trsv_upper(r, c)
    assert np.max(np.abs(r @ x - c)) <= 1e-13 * np.linalg.norm(c)


def pin_partial_steps(orc):
    """The first k steps of the full factorization equal the factorization
    of the leading k columns (used to sample the CPU baseline)."""
    m, n, k = 70, 30, 11
    a = workloads.gaussian(m, n, 131)
    vr_full, tau_full = orc.house_qr(a)
    vr_part, tau_part = orc.house_qr(a, nsteps=k)
    assert np.array_equal(vr_part[:, :k], vr_full[:, :k])
    assert np.array_equal(tau_part[:k], tau_full[:k])
    # remaining columns of the partial run are Q_k^T A(:, k:n)
    vr_k, tau_k = orc.house_qr(a[:, :k])
    rest = orc.apply_qt(vr_k, tau_k, a[:, k:])
    assert np.max(np.abs(vr_part[:, k:] - rest)) <= 1e-13 * np.linalg.norm(a)


def pin_wide(orc):
    """m < n (Section 2.1): R = [R1, Q^T A2] with A1 = Q R1.  Pinned to LAPACK's
    dgeqrf of the wide matrix element by element (up to the empty-subcolumn
    reflector of row m-1: LAPACK tau = 0, the sign reading tau = 2, which
    negates row m-1 of R), to A = Q R with the explicit reflector product,
    and to R^T R = A^T A."""
    for (m, n, seed) in [(5, 9, 61), (20, 47, 62), (64, 65, 63)]:
        a = workloads.gaussian(m, n, seed)
        vr, tau = orc.house_qr(a)
        assert vr.shape == (m, n) and tau.shape == (m,)
        h, tl = np.linalg.qr(a, mode="raw")
        h = np.array(h.T, order="F")
        assert tl[-1] == 0.0 and tau[-1] == 2.0
        tl = tl.copy()
        tl[-1] = 2.0
        h[m - 1, m - 1:] = -h[m - 1, m - 1:]
        assert np.max(np.abs(tau - tl)) <= 1e-13
        assert np.max(np.abs(np.tril(vr[:, :m], -1) - np.tril(h[:, :m], -1))) <= 1e-12
        r = np.triu(vr)
        assert np.max(np.abs(r - np.triu(h))) <= 1e-12 * np.max(np.abs(a)) * m
        q = explicit_q(vr[:, :m], tau)
        assert np.linalg.norm(a - q @ r) / np.linalg.norm(a) <= 1e-14 * n
        assert np.linalg.norm(r.T @ r - a.T @ a) / np.linalg.norm(a.T @ a) <= 1e-14 * n


ALL_PINS = [
    pin_gram_schmidt_tiny, pin_cholesky, pin_lapack_elementwise, pin_orthogonal_input,
    pin_upper_triangular, pin_zero_column, pin_single_column, pin_reflectors, pin_backward_error,
    pin_t_two_ways, pin_apply, pin_ls, pin_trsv, pin_partial_steps, pin_wide,
]

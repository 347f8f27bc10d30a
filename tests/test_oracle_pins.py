"""The CPU oracle checked against mathematics and independent libraries
(Gram-Schmidt by brute force, Cholesky, LAPACK, closed forms, invariants).
Both builds are pinned: the plain one and the all-cores (OpenMP) one, whose
results must also equal the plain build's bit for bit."""

import numpy as np
import pytest

import oracle
import workloads
from tests import _pins


@pytest.mark.parametrize("pin", _pins.ALL_PINS, ids=lambda p: p.__name__)
def test_oracle_pin(orc, pin):
    pin(orc)


@pytest.fixture(scope="module")
def orc_all_cores():
    return oracle.all_cores()


@pytest.mark.parametrize("pin", _pins.ALL_PINS, ids=lambda p: p.__name__)
def test_oracle_pin_all_cores(orc_all_cores, pin):
    pin(orc_all_cores)


def test_all_cores_build_is_bit_identical(orc, orc_all_cores):
    """Large enough that every OpenMP loop runs threaded (m x columns > 65536)."""
    a = workloads.graded(700, 300, 5)
    vr1, tau1 = orc.house_qr(a)
    vr2, tau2 = orc_all_cores.house_qr(a)
    assert np.array_equal(vr1, vr2) and np.array_equal(tau1, tau2)
    assert np.array_equal(orc.larft(vr1, tau1), orc_all_cores.larft(vr2, tau2))
    b = workloads.vector(700, 6)
    assert np.array_equal(orc.apply_qt(vr1, tau1, b), orc_all_cores.apply_qt(vr2, tau2, b))
    assert np.array_equal(orc.form_q(vr1, tau1), orc_all_cores.form_q(vr2, tau2))
    x1, r1 = orc.ls_solve(a, b)
    x2, r2 = orc_all_cores.ls_solve(a, b)
    assert np.array_equal(x1, x2) and r1 == r2
    assert orc.threads == 1 and orc_all_cores.threads >= 1

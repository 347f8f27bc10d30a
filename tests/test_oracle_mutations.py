"""Plants plausible mistakes in a copy of the oracle's C source, on the CPU,
and checks that at least one pin fails for each: evidence that the pins
constrain every routine of the oracle, not just its happy path."""

import os
import tempfile

import pytest

import oracle
from tests import _pins

# (description, exact source text, replacement) -- each must occur once.
MUTATIONS = [
    ("reflector sign flipped", "double beta = -sgn(alpha) * norm;", "double beta = sgn(alpha) * norm;"),
    ("tau numerator reversed", "tau[j] = (beta - alpha) / beta;", "tau[j] = (alpha - beta) / beta;"),
    ("pivot row dropped from the update dot", "double w = AT(a, j, c, lda);\n            for (long r = j + 1; r < m; ++r) w += AT(a, r, j, lda) * AT(a, r, c, lda);",
     "double w = 0.0;\n            for (long r = j + 1; r < m; ++r) w += AT(a, r, j, lda) * AT(a, r, c, lda);"),
    ("norm not square-rooted", "return amax * sqrt(s);", "return amax * s;"),
    ("v scaled by the wrong pivot", "double d = alpha - beta;", "double d = alpha + beta;"),
    ("vdot transposed index", "double s = AT(v, j, i, ldv); /* row j", "double s = AT(v, i, j, ldv); /* row j"),
    ("larft sign dropped", "AT(t, i, j, ldt) = -tau[j] * s;", "AT(t, i, j, ldt) = tau[j] * s;"),
    ("larft sum range off by one", "for (long k = i; k < j; ++k) s += AT(t, i, k, ldt) * z[k];", "for (long k = i + 1; k < j; ++k) s += AT(t, i, k, ldt) * z[k];"),
    ("gram diagonal not halved", "g[j + j * n] = d / 2.0;", "g[j + j * n] = d;"),
    ("apply_q runs forwards", "for (long j = n - 1; j >= 0; --j) apply_reflector", "for (long j = 0; j < n; ++j) apply_reflector"),
    ("apply_qt runs backwards", "for (long j = 0; j < n; ++j) apply_reflector(m, j, v, ldv, tau[j], nrhs, b, ldb);\n    return 0;\n}\n\n/* B <- Q B",
     "for (long j = n - 1; j >= 0; --j) apply_reflector(m, j, v, ldv, tau[j], nrhs, b, ldb);\n    return 0;\n}\n\n/* B <- Q B"),
    ("reflector application drops tau", "w *= tauj;", "w *= 1.0;"),
    ("trsv transposed operand", "s -= AT(r, i, k, ldr) * x[k];", "s -= AT(r, k, i, ldr) * x[k];"),
    ("form_q starts from the wrong identity", "AT(q, i, j, ldq) = (i == j) ? 1.0 : 0.0;", "AT(q, i, j, ldq) = (i == j + 1) ? 1.0 : 0.0;"),
    ("zero column handled as identity", "tau[j] = 2.0;\n            AT(a, j, j, lda) = 0.0;", "tau[j] = 0.0;\n            AT(a, j, j, lda) = 0.0;"),
]


def _source():
    with open(oracle.SOURCE) as f:
        return f.read()


@pytest.mark.parametrize("desc,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_mutant_is_caught(desc, old, new):
    src = _source()
    assert src.count(old) == 1, f"mutation anchor not unique or missing: {desc}"
    mutated = src.replace(old, new)
    with tempfile.TemporaryDirectory() as d:
        cpath = os.path.join(d, "mutant.c")
        with open(cpath, "w") as f:
            f.write(mutated)
        lib = oracle.build(cpath, os.path.join(d, "libmutant.so"), force=True)
        mutant = oracle.Oracle(lib)
        failed = []
        for pin in _pins.ALL_PINS:
            try:
                pin(mutant)
            except (AssertionError, ValueError, FloatingPointError, ZeroDivisionError):
                failed.append(pin.__name__)
            except Exception as e:  # numpy LinAlgError and the like also count
                failed.append(f"{pin.__name__}:{type(e).__name__}")
        assert failed, f"no pin caught the mutation: {desc}"

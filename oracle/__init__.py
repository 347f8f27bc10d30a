"""CPU oracle (FP64 unblocked Householder QR and least squares).

TEST INFRASTRUCTURE ONLY: this package is the independent reference that the
CUDA path is compared against.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may load it.  It shares no code with the CUDA
library.  The arithmetic lives in ``house.c`` (plain C, one reflector at a
time); this module compiles it with gcc and marshals numpy arrays.

Every routine takes and returns float64 Fortran-ordered arrays.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "house.c")
BUILD_DIR = os.path.join(_HERE, "_build")
LIBRARY = os.path.join(BUILD_DIR, "liboracle.so")
LIBRARY_OMP = os.path.join(BUILD_DIR, "liboracle_omp.so")

_lock = threading.Lock()
_default = None
_all_cores = None


def build(source: str = SOURCE, out: str | None = None, force: bool = False, openmp: bool = False) -> str:
    """Compile ``source`` into the shared library ``out`` (gcc, no FMA
    contraction so that x86 and Arm hosts round identically).  openmp: the
    all-cores build of the same source (-fopenmp), whose results are
    bit-identical to the plain build's."""
    if out is None:
        out = LIBRARY_OMP if openmp else LIBRARY
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(source):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           *(["-fopenmp"] if openmp else []), "-o", tmp, source, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build_all(force: bool = False) -> None:
    """Both builds of the oracle: one thread and all cores."""
    build(force=force)
    build(force=force, openmp=True)


_D = ctypes.POINTER(ctypes.c_double)
_L = ctypes.c_long


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _fortran(a: np.ndarray) -> np.ndarray:
    return np.array(a, dtype=np.float64, order="F", copy=True)


class Oracle:
    """ctypes wrapper over one compiled copy of ``house.c``."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        sig = {
            "orc_house_qr": [_L, _L, _D, _L, _D, _L],
            "orc_larft": [_L, _L, _D, _L, _D, _D, _L],
            "orc_t_from_gram": [_L, _L, _D, _L, _D, _L],
            "orc_apply_qt": [_L, _L, _D, _L, _D, _L, _D, _L],
            "orc_apply_q": [_L, _L, _D, _L, _D, _L, _D, _L],
            "orc_form_q": [_L, _L, _D, _L, _D, _D, _L],
            "orc_trsv_upper": [_L, _D, _L, _D],
            "orc_ls_solve": [_L, _L, _D, _L, _D, _D, _D],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        lib.orc_threads.argtypes = []
        lib.orc_threads.restype = ctypes.c_int
        self.lib = lib
        self.path = path

    @property
    def threads(self) -> int:
        """Threads the all-cores build shares its loops over (1 for the plain build)."""
        return int(self.lib.orc_threads())

    @staticmethod
    def _check(rc: int, name: str):
        if rc != 0:
            raise ValueError(f"oracle {name} returned {rc}")

    def house_qr(self, a: np.ndarray, nsteps: int | None = None):
        """Returns (VR, tau): V (strict lower, unit diagonal implied) and R
        (upper triangle, upper trapezoidal when m < n) packed in one m x n
        array, and the min(m, n) scalings (Section 2.1; m < n by splitting
        off the leading square block)."""
        vr = _fortran(a)
        m, n = vr.shape
        kmax = min(m, n)
        tau = np.zeros(max(kmax, 1))
        k = kmax if nsteps is None else min(nsteps, kmax)
        self._check(self.lib.orc_house_qr(m, n, _ptr(vr), max(m, 1), _ptr(tau), k), "house_qr")
        return vr, tau[:kmax]

    def larft(self, vr: np.ndarray, tau: np.ndarray) -> np.ndarray:
        vr = _fortran(vr)
        m, n = vr.shape
        t = np.zeros((n, n), order="F")
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        self._check(self.lib.orc_larft(m, n, _ptr(vr), max(m, 1), _ptr(tau), _ptr(t), max(n, 1)), "larft")
        return t

    def t_from_gram(self, vr: np.ndarray) -> np.ndarray:
        vr = _fortran(vr)
        m, n = vr.shape
        t = np.zeros((n, n), order="F")
        self._check(self.lib.orc_t_from_gram(m, n, _ptr(vr), max(m, 1), _ptr(t), max(n, 1)), "t_from_gram")
        return t

    def _apply(self, fn, vr, tau, b):
        vr = _fortran(vr)
        m, n = vr.shape
        vec = b.ndim == 1
        out = _fortran(b.reshape(m, -1) if not vec else b.reshape(m, 1))
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        rc = fn(m, n, _ptr(vr), max(m, 1), _ptr(tau), out.shape[1], _ptr(out), max(m, 1))
        self._check(rc, fn.__name__)
        return out[:, 0].copy() if vec else out

    def apply_qt(self, vr, tau, b):
        return self._apply(self.lib.orc_apply_qt, vr, tau, b)

    def apply_q(self, vr, tau, b):
        return self._apply(self.lib.orc_apply_q, vr, tau, b)

    def form_q(self, vr, tau) -> np.ndarray:
        vr = _fortran(vr)
        m, n = vr.shape
        q = np.zeros((m, n), order="F")
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        self._check(self.lib.orc_form_q(m, n, _ptr(vr), max(m, 1), _ptr(tau), _ptr(q), max(m, 1)), "form_q")
        return q

    def trsv_upper(self, r: np.ndarray, c: np.ndarray) -> np.ndarray:
        r = _fortran(r)
        n = r.shape[1]
        x = np.array(c[:n], dtype=np.float64, copy=True)
        self._check(self.lib.orc_trsv_upper(n, _ptr(r), max(r.shape[0], 1), _ptr(x)), "trsv_upper")
        return x

    def ls_solve(self, a: np.ndarray, b: np.ndarray):
        """Returns (x, ||residual||)."""
        a = _fortran(a)
        m, n = a.shape
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(max(n, 1))
        res = ctypes.c_double(0.0)
        rc = self.lib.orc_ls_solve(m, n, _ptr(a), max(m, 1), _ptr(b), _ptr(x), ctypes.byref(res))
        self._check(rc, "ls_solve")
        return x[:n], res.value

    # ---- derived quantities (plain numpy on the oracle's own outputs) ----

    def qr(self, a: np.ndarray):
        """Returns (V, T, R, tau): V unit lower trapezoidal m x n, T n x n
        upper triangular, R n x n upper triangular."""
        vr, tau = self.house_qr(a)
        n = vr.shape[1]
        return unpack_v(vr), self.larft(vr, tau), np.triu(vr[:n, :]), tau


def unpack_v(vr: np.ndarray) -> np.ndarray:
    """Unit lower trapezoidal V from a packed V\\R array."""
    m, n = vr.shape
    v = np.tril(vr, -1)
    v[np.arange(n), np.arange(n)] = 1.0
    return np.asfortranarray(v)


def sign_normalise(r: np.ndarray, q: np.ndarray | None = None):
    """D = diag(sgn(R_jj)), sgn(0) = +1; returns (D R, Q D) so that the
    diagonal of R is non-negative (the unique QR of a full-rank matrix)."""
    d = np.where(np.diag(r) < 0.0, -1.0, 1.0)
    rr = d[:, None] * r
    qq = None if q is None else q * d[None, :]
    return rr, qq


def default() -> Oracle:
    """The oracle built from ``house.c`` (compiled on first use), one thread."""
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
        return _default


def all_cores() -> Oracle:
    """The OpenMP build of the same ``house.c``: its column loops run on every
    core (OMP_NUM_THREADS caps them); results equal the plain build's bit for
    bit."""
    global _all_cores
    with _lock:
        if _all_cores is None:
            _all_cores = Oracle(build(openmp=True))
        return _all_cores

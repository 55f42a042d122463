"""Plain CPU oracle for the chaos-indicator hot path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product path (``paper_2507_00622_gb300``) never imports it, and it never
imports the product path.

The arithmetic lives in ``chs_oracle.c`` (IEEE double, ``-ffp-contract=off``,
OpenMP over orbits); this module compiles it with gcc and exposes numpy-level
wrappers.  Arrays are structure-of-arrays, ``a[c, o]`` for component ``c`` of
orbit ``o``; the phase-space order is ``(q_1..q_N, p_1..p_N)``.

Each wrapper names the passage of arXiv 2507.00622 ("Chaoticus") it follows:
  energy / rhs / hessian   Eqs. Ham_HH, ham_eqs_HH, ham_FPU, ham_eqs_FPU
  integrate                fixed-step RK4 (or DOP853, the paper's DOP 8) on
                           the variational system, vector normalisation and
                           the LD (Sec. Functionalities, Sec. Statement of need)
  integrate_adaptive       DOP 8(5) with adaptive step size and per-step error
                           (Sec. Functionalities)
  dop853_tableau           the DOP853 coefficients (Hairer, Norsett and Wanner,
                           Solving ODEs I, Sec. II.10)
  indicators               SALI and GALI_k by SVD (Sec. Functionalities)
  ld_indicators            LD-based indicators from neighbouring cells
                           (Sec. Functionalities)
  lyapunov                 Lyapunov spectrum by periodic QR (Sec.
                           Functionalities, FPU example of Sec. Examples)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chs_oracle.c")
_LIB = os.path.join(_HERE, "libchs_oracle.so")
_lock = threading.Lock()
_lib = None

HENON_HEILES, FPUT, QUARTIC3, HARMONIC, INVERTED = 1, 2, 3, 100, 101
OK, FORBIDDEN, ESCAPED, NONFINITE, ENERGY_DRIFT, EARLY_CHAOTIC = 0, 1, 2, 3, 4, 5
STEP_FAIL = 7
RK4, YOSHIDA4, DOP853 = 0, 1, 2


class System(C.Structure):
    _fields_ = [("model", C.c_int), ("n_dof", C.c_int), ("kk", C.c_double),
                ("alpha", C.c_double), ("beta", C.c_double), ("eps", C.c_double)]


class Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("n_steps", C.c_int64), ("step0", C.c_int64),
                ("n_dev", C.c_int), ("renorm", C.c_int), ("sample_every", C.c_int),
                ("qr_every", C.c_int), ("integrator", C.c_int), ("ld_p", C.c_double),
                ("escape_r2", C.c_double), ("dh_limit", C.c_double), ("early_exit", C.c_int),
                ("sali_threshold", C.c_double)]


class Adaptive(C.Structure):
    _fields_ = [("t_final", C.c_double), ("rtol", C.c_double), ("atol", C.c_double),
                ("h_max", C.c_double)]


def build(force: bool = False) -> str:
    """Compile chs_oracle.c into libchs_oracle.so (gcc, OpenMP when available)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
        try:
            subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                           capture_output=True, text=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True, capture_output=True, text=True)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        L.o_energy.restype = C.c_double
        L.o_energy.argtypes = [C.POINTER(System), P]
        L.o_rhs.argtypes = [C.POINTER(System), P, P]
        L.o_hessian.argtypes = [C.POINTER(System), P, P]
        L.o_splitmix64_next.restype = C.c_uint64
        L.o_splitmix64_next.argtypes = [C.POINTER(C.c_uint64)]
        L.o_seed_vectors.argtypes = [C.c_uint64, C.c_int64, C.c_int, C.c_int, P]
        L.o_grid_ics.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, C.c_double,
                                 C.c_double, C.c_int, P, P]
        L.o_fput_mode_ics.restype = C.c_int
        L.o_fput_mode_ics.argtypes = [C.POINTER(System), C.c_int64, P, P, P, P]
        L.o_ensemble_init.argtypes = [C.POINTER(System), C.POINTER(Params), C.c_int64, P, P, P,
                                      C.c_uint64, P, P, P, P, P, P, P]
        L.o_integrate.argtypes = [C.POINTER(System), C.POINTER(Params), C.c_int64, P, P, P, P,
                                  P, P, P, P, C.c_int]
        L.o_integrate_adaptive.argtypes = [C.POINTER(System), C.POINTER(Params),
                                           C.POINTER(Adaptive), C.c_int64, P, P, P, P, P, P, P,
                                           P, P, P, P, P, C.c_int]
        L.o_dop853_tableau.argtypes = [P, P, P, P]
        L.o_lyapunov_adaptive.argtypes = [C.POINTER(System), C.POINTER(Params),
                                          C.POINTER(Adaptive), C.c_int64, P, P, P, P, P, P,
                                          C.c_int]
        L.o_shell_ics.restype = C.c_int
        L.o_shell_ics.argtypes = [C.POINTER(System), C.c_int64, P, P, P]
        L.o_jacobi_sv.argtypes = [C.c_int, C.c_int, P, P]
        L.o_indicators.argtypes = [C.POINTER(System), C.c_int64, C.c_int, P, P, C.c_double, P,
                                   P, P]
        L.o_ld_indicators.argtypes = [C.c_int, C.c_int, P, P, P, P]
        L.o_lyapunov.argtypes = [C.POINTER(System), C.POINTER(Params), C.c_int64, P, P, P, P,
                                 C.c_int]
        L.o_max_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def system(model: int, n_dof: int, kk: float = 1.0, alpha: float = 0.0, beta: float = 0.0,
           eps: float = 0.0) -> System:
    return System(model, n_dof, kk, alpha, beta, eps)


def henon_heiles() -> System:
    return system(HENON_HEILES, 2)


def fput(N: int, beta: float = 1.0, alpha: float = 0.0, kk: float = 1.0) -> System:
    return system(FPUT, N, kk=kk, alpha=alpha, beta=beta)


def params(dt: float, n_steps: int, *, step0: int = 0, n_dev: int = 0, renorm: bool = True,
           sample_every: int = 100, qr_every: int = 10, integrator: int = RK4,
           ld_p: float = 0.0, escape_r2: float = 0.0, dh_limit: float = 0.0,
           early_exit: bool = False, sali_threshold: float = 1e-8) -> Params:
    return Params(dt, n_steps, step0, n_dev, int(renorm), sample_every, qr_every, integrator,
                  ld_p, escape_r2, dh_limit, int(early_exit), sali_threshold)


def max_threads() -> int:
    return int(lib().o_max_threads())


def energy(sysd: System, x) -> float:
    x = _f64(x)
    return float(lib().o_energy(C.byref(sysd), _p(x)))


def rhs(sysd: System, x) -> np.ndarray:
    x = _f64(x)
    f = np.empty_like(x)
    lib().o_rhs(C.byref(sysd), _p(x), _p(f))
    return f


def hessian(sysd: System, q) -> np.ndarray:
    q = _f64(q)
    N = sysd.n_dof
    H = np.empty((N, N))
    lib().o_hessian(C.byref(sysd), _p(q), _p(H))
    return H


def splitmix64_stream(seed: int, count: int) -> list[int]:
    st = C.c_uint64(seed)
    return [int(lib().o_splitmix64_next(C.byref(st))) for _ in range(count)]


def seed_vectors(seed: int, n: int, k: int, d: int) -> np.ndarray:
    w = np.empty((k * d, n))
    lib().o_seed_vectors(seed, n, k, d, _p(w))
    return w


def grid_ics(E, y0, y1, ny, py0, py1, npy):
    n = ny * npy
    ics = np.empty((4, n))
    st = np.empty(n, dtype=np.int32)
    lib().o_grid_ics(E, y0, y1, ny, py0, py1, npy, _p(ics), _p(st))
    return ics, st


def fput_mode_ics(sysd: System, Qm, Pm, E):
    Qm, Pm, E = _f64(Qm), _f64(Pm), _f64(E)
    n = E.shape[0]
    ics = np.empty((2 * sysd.n_dof, n))
    rc = lib().o_fput_mode_ics(C.byref(sysd), n, _p(Qm), _p(Pm), _p(E), _p(ics))
    if rc != 0:
        raise ValueError("normal-mode scaling needs alpha == 0")
    return ics


class Ensemble:
    """Host-side ensemble state: x [d,n], w [k*d,n], ld [n], h0, dh_max, n_exec, status."""

    def __init__(self, sysd: System, prm: Params, ics, ic_status=None, w_in=None, seed: int = 1):
        ics = _f64(ics)
        d = 2 * sysd.n_dof
        n = ics.shape[1]
        k = prm.n_dev
        self.sysd, self.n, self.d, self.k = sysd, n, d, k
        self.x = np.empty((d, n))
        self.w = np.empty((max(k, 0) * d, n))
        self.ld = np.empty(n)
        self.h0 = np.empty(n)
        self.dh_max = np.empty(n)
        self.n_exec = np.empty(n, dtype=np.int64)
        self.status = np.empty(n, dtype=np.int32)
        ic_status = None if ic_status is None else np.ascontiguousarray(ic_status, dtype=np.int32)
        w_in = None if w_in is None else _f64(w_in)
        lib().o_ensemble_init(C.byref(sysd), C.byref(prm), n, _p(ics), _p(ic_status), _p(w_in),
                              seed, _p(self.x), _p(self.w), _p(self.ld), _p(self.h0),
                              _p(self.dh_max), _p(self.n_exec), _p(self.status))

    def integrate(self, prm: Params, nthreads: int = 0, t_end=None) -> "Ensemble":
        """Advance by prm.n_steps steps (each orbit at most up to its own t_end[o])."""
        te = None if t_end is None else np.ascontiguousarray(t_end, dtype=np.int64)
        lib().o_integrate(C.byref(self.sysd), C.byref(prm), self.n, _p(self.x), _p(self.w),
                          _p(self.ld), _p(self.h0), _p(self.dh_max), _p(self.n_exec),
                          _p(self.status), _p(te), nthreads)
        return self

    def integrate_adaptive(self, prm: Params, t_final: float, rtol: float, atol: float,
                           h_max: float = 0.0, nthreads: int = 0) -> "Ensemble":
        """DOP 8(5) with adaptive steps up to time t_final, at most prm.n_steps
        accepted steps per orbit in this call.  The per-orbit time ``t``, next
        step ``h`` (first call: prm.dt), last and largest accepted-step error and
        rejection count live on the ensemble."""
        if not hasattr(self, "t"):
            self.t = np.zeros(self.n)
            self.h = np.full(self.n, prm.dt)
            self.err_last = np.zeros(self.n)
            self.err_max = np.zeros(self.n)
            self.n_rej = np.zeros(self.n, dtype=np.int64)
        ad = Adaptive(t_final, rtol, atol, h_max)
        lib().o_integrate_adaptive(C.byref(self.sysd), C.byref(prm), C.byref(ad), self.n,
                                   _p(self.x), _p(self.w), _p(self.ld), _p(self.h0),
                                   _p(self.dh_max), _p(self.n_exec), _p(self.status), _p(self.t),
                                   _p(self.h), _p(self.err_last), _p(self.err_max),
                                   _p(self.n_rej), nthreads)
        return self

    def indicators(self, sali_threshold: float = 1e-8):
        n, k = self.n, self.k
        sali = np.empty(n)
        gali = np.empty((max(k - 1, 1), n))
        label = np.empty(n, dtype=np.int8)
        lib().o_indicators(C.byref(self.sysd), n, k, _p(self.w), _p(self.status), sali_threshold,
                           _p(sali), _p(gali), _p(label))
        return sali, gali[: max(k - 1, 0)], label


def shell_ics(sysd: System, dirs, E):
    """Quartic-3 states on the energy shells E[o] along the directions dirs [6, n]."""
    dirs, E = _f64(dirs), _f64(E)
    n = E.shape[0]
    ics = np.empty((6, n))
    if lib().o_shell_ics(C.byref(sysd), n, _p(dirs), _p(E), _p(ics)) != 0:
        raise ValueError("shell initial conditions are defined for QUARTIC3")
    return ics


def dop853_tableau():
    """(a [12, 12], b, e5, b3) of the DOP853 pair as the oracle holds them."""
    a = np.empty((12, 12))
    b, e5, b3 = np.empty(12), np.empty(12), np.empty(12)
    lib().o_dop853_tableau(_p(a), _p(b), _p(e5), _p(b3))
    return a, b, e5, b3


def jacobi_sv(A) -> np.ndarray:
    """Singular values of a d x k matrix by one-sided Jacobi (unsorted)."""
    A = np.asarray(A, dtype=np.float64)
    d, k = A.shape
    Acm = np.ascontiguousarray(A.T)
    sv = np.empty(k)
    lib().o_jacobi_sv(d, k, _p(Acm), _p(sv))
    return sv


def ld_indicators(ny: int, npy: int, ld, status):
    ld = _f64(ld)
    status = np.ascontiguousarray(status, dtype=np.int32)
    dl = np.empty(ny * npy)
    sl = np.empty(ny * npy)
    lib().o_ld_indicators(ny, npy, _p(ld), _p(status), _p(dl), _p(sl))
    return dl, sl


def lyapunov(sysd: System, prm: Params, ics, ic_status=None, nthreads: int = 0):
    ics = _f64(ics)
    d = 2 * sysd.n_dof
    n = ics.shape[1]
    lam = np.empty((d, n))
    st = np.empty(n, dtype=np.int32)
    ic_status = None if ic_status is None else np.ascontiguousarray(ic_status, dtype=np.int32)
    lib().o_lyapunov(C.byref(sysd), C.byref(prm), n, _p(ics), _p(ic_status), _p(lam), _p(st),
                     nthreads)
    return lam, st


def lyapunov_adaptive(sysd: System, prm: Params, ics, t_final: float, rtol: float, atol: float,
                      ic_status=None, h_max: float = 0.0, nthreads: int = 0):
    """Lyapunov spectrum with adaptive DOP 8(5) from t = 0 to t_final (first
    step prm.dt, at most prm.n_steps accepted steps): (lambda, status,
    accepted steps, rejected trials)."""
    ics = _f64(ics)
    d = 2 * sysd.n_dof
    n = ics.shape[1]
    lam = np.empty((d, n))
    st = np.empty(n, dtype=np.int32)
    acc = np.empty(n, dtype=np.int64)
    rej = np.empty(n, dtype=np.int64)
    ic_status = None if ic_status is None else np.ascontiguousarray(ic_status, dtype=np.int32)
    ad = Adaptive(t_final, rtol, atol, h_max)
    lib().o_lyapunov_adaptive(C.byref(sysd), C.byref(prm), C.byref(ad), n, _p(ics), _p(ic_status),
                              _p(lam), _p(st), _p(acc), _p(rej), nthreads)
    return lam, st, acc, rej

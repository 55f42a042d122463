"""Python binding of the chaos-indicator C ABI (include/chs.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libchs.so``.  Tensors are PyTorch CUDA tensors (device memory and
streams come from PyTorch); each function has the name and argument order of
its C entry point.  A missing or unloadable library raises immediately: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libchs.so")

CHS_OK, CHS_E_INVALID, CHS_E_UNSUPPORTED, CHS_E_CUDA, CHS_E_NOMEM, CHS_E_SIZE = range(6)
HENON_HEILES, FPUT, QUARTIC3, HARMONIC, INVERTED = 1, 2, 3, 100, 101
(ORBIT_OK, ORBIT_FORBIDDEN, ORBIT_ESCAPED, ORBIT_NONFINITE, ORBIT_ENERGY_DRIFT,
 ORBIT_EARLY_CHAOTIC, ORBIT_PREDICTED_REGULAR, ORBIT_STEP_FAIL, ORBIT_STEP_BUDGET) = range(9)
VEC_FP64, VEC_FP32 = 0, 1
RK4, DOP853 = 0, 2

EXPORTS = ("chs_create_system", "chs_destroy_system", "chs_system_dim", "chs_section_grid_ics",
           "chs_fput_mode_ics", "chs_shell_ics", "chs_ensemble_init", "chs_integrate_batch",
           "chs_integrate_adaptive", "chs_lyapunov_adaptive", "chs_integrate_persistent",
           "chs_compact_work_size", "chs_integrate_compacted", "chs_integrate_compacted_static",
           "chs_indicators",
           "chs_lyapunov_spectrum", "chs_lyapunov_batch", "chs_lyapunov_batch_persistent", "chs_mlp_param_count", "chs_mlp_features", "chs_mlp_forward",
           "chs_mlp_loss_grad", "chs_mlp_backward", "chs_mlp_adam", "chs_surrogate_decide",
           "chs_peak_probe", "chs_probe_ops_per_thread", "chs_check_params", "chs_last_error",
           "chs_version")
PROBE_DFMA, PROBE_DFMA_DEP, PROBE_FFMA, PROBE_DSQRT, PROBE_DMMA, PROBE_DFMA_DMMA = 1, 2, 3, 4, 5, 6


class ChsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"chs status {code}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("n_steps", C.c_int64), ("step0", C.c_int64),
                ("n_dev", C.c_int32), ("renorm", C.c_int32), ("sample_every", C.c_int32),
                ("qr_every", C.c_int32), ("vec_precision", C.c_int32), ("early_exit", C.c_int32),
                ("ld_p", C.c_double), ("escape_r2", C.c_double), ("dh_limit", C.c_double),
                ("sali_threshold", C.c_double), ("seed", C.c_uint64), ("integrator", C.c_int32),
                ("block_threads", C.c_int32), ("clock_budget", C.c_int64), ("threads_per_orbit", C.c_int32)]


class Adaptive(C.Structure):
    _fields_ = [("t_final", C.c_double), ("rtol", C.c_double), ("atol", C.c_double),
                ("h_max", C.c_double)]


class LyapJob(C.Structure):
    _fields_ = [("sys", C.c_void_p), ("params", Params), ("n_orbits", C.c_int64), ("ics", C.c_void_p),
                ("ic_status", C.c_void_p), ("lambda_out", C.c_void_p), ("status_out", C.c_void_p)]


class Ensemble(C.Structure):
    _fields_ = [("n_orbits", C.c_int64), ("x", C.c_void_p), ("w", C.c_void_p), ("ld", C.c_void_p),
                ("h0", C.c_void_p), ("dh_max", C.c_void_p), ("n_exec", C.c_void_p),
                ("status", C.c_void_p), ("t_end", C.c_void_p)]


_lib = None


def load(path: str | None = None):
    """Load libchs.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"{p} is missing: build the CUDA library first (__graft_entry__.build())")
    L = C.CDLL(p)
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "chs_create_system": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, I32, P, I32]),
        "chs_destroy_system": (C.c_int, [P]),
        "chs_system_dim": (I32, [P]),
        "chs_section_grid_ics": (C.c_int, [P, D, D, D, I32, D, D, I32, P, P, P]),
        "chs_fput_mode_ics": (C.c_int, [P, I64, P, P, P, P, P]),
        "chs_shell_ics": (C.c_int, [P, I64, P, P, P, P]),
        "chs_compact_work_size": (C.c_size_t, [I64]),
        "chs_integrate_compacted": (C.c_int, [P, C.POINTER(Params), C.POINTER(Ensemble), I32, P,
                                              C.c_size_t, P]),
        "chs_integrate_compacted_static": (C.c_int, [P, C.POINTER(Params), C.POINTER(Ensemble),
                                                     I32, P]),
        "chs_integrate_persistent": (C.c_int, [P, C.POINTER(Params), C.POINTER(Ensemble), P,
                                               C.c_size_t, P]),
        "chs_ensemble_init": (C.c_int, [P, C.POINTER(Params), C.POINTER(Ensemble), P, P, P, P]),
        "chs_integrate_batch": (C.c_int, [P, C.POINTER(Params), C.POINTER(Ensemble), P]),
        "chs_integrate_adaptive": (C.c_int, [P, C.POINTER(Params), C.POINTER(Adaptive),
                                             C.POINTER(Ensemble), P, P, P, P, P, P]),
        "chs_indicators": (C.c_int, [P, C.POINTER(Params), C.POINTER(Ensemble), I32, I32, P, P,
                                     P, P, P]),
        "chs_lyapunov_spectrum": (C.c_int, [P, C.POINTER(Params), I64, P, P, P, P, P]),
        "chs_lyapunov_batch": (C.c_int, [C.POINTER(LyapJob), I32, P]),
        "chs_lyapunov_batch_persistent": (C.c_int, [C.POINTER(LyapJob), I32, P, C.c_size_t, P]),
        "chs_lyapunov_adaptive": (C.c_int, [P, C.POINTER(Params), C.POINTER(Adaptive), I64, P, P, P, P,
                                            P, P, P]),
        "chs_mlp_param_count": (C.c_size_t, []),
        "chs_mlp_features": (C.c_int, [P, I32, P, D, P, I64, P, P]),
        "chs_mlp_forward": (C.c_int, [P, P, I64, P, P, P]),
        "chs_mlp_loss_grad": (C.c_int, [P, P, P, I64, C.c_float, P, P, P]),
        "chs_mlp_backward": (C.c_int, [P, P, P, P, I64, P, P, P]),
        "chs_mlp_adam": (C.c_int, [P, P, P, P, C.c_float, C.c_float, C.c_float, C.c_float, I32, P, P]),
        "chs_surrogate_decide": (C.c_int, [P, P, I32, P, D, P, D, I64, P, P, P]),
        "chs_check_params": (C.c_int, [C.POINTER(Params), C.c_int, I32]),
        "chs_peak_probe": (C.c_int, [I32, I32, I32, I64, P, P]),
        "chs_probe_ops_per_thread": (D, [I32, I64]),
        "chs_last_error": (C.c_char_p, []),
        "chs_version": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype, f.argtypes = res, args
    _lib = L
    return L


def _check(code: int):
    if code != CHS_OK:
        raise ChsError(code, load().chs_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_cuda:
        raise ValueError("chs entry points take CUDA tensors (device pointers)")
    if not t.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def params(dt: float, n_steps: int, *, step0: int = 0, n_dev: int = 0, renorm: bool = True,
           sample_every: int = 100, qr_every: int = 10, vec_precision: int = VEC_FP64,
           ld_p: float = 0.0, escape_r2: float = 0.0, dh_limit: float = 0.0,
           sali_threshold: float = 1e-8, seed: int = 1, early_exit: bool = False,
           integrator: int = RK4, block_threads: int = 0, clock_budget: int = 0,
           threads_per_orbit: int = 0) -> Params:
    return Params(dt, n_steps, step0, n_dev, int(renorm), sample_every, qr_every, vec_precision,
                  int(early_exit), ld_p, escape_r2, dh_limit, sali_threshold, seed, integrator,
                  block_threads, clock_budget, threads_per_orbit)


# ----------------------------------------------------------------------------
# entry points, one per C function
# ----------------------------------------------------------------------------

def chs_create_system(model: int, n_dof: int, sys_params=()) -> C.c_void_p:
    h = C.c_void_p()
    arr = (C.c_double * max(len(sys_params), 1))(*sys_params)
    _check(load().chs_create_system(C.byref(h), model, n_dof, arr if sys_params else None,
                                    len(sys_params)))
    return h


def chs_destroy_system(h):
    _check(load().chs_destroy_system(h))


def chs_system_dim(h) -> int:
    return int(load().chs_system_dim(h))


def chs_section_grid_ics(h, E, y0, y1, ny, py0, py1, npy, ics, status, stream=None):
    _check(load().chs_section_grid_ics(h, E, y0, y1, ny, py0, py1, npy, _ptr(ics), _ptr(status),
                                       _stream(stream)))


def chs_fput_mode_ics(h, n, Qm, Pm, E, ics, stream=None):
    _check(load().chs_fput_mode_ics(h, n, _ptr(Qm), _ptr(Pm), _ptr(E), _ptr(ics), _stream(stream)))


def chs_shell_ics(h, n, dirs, E, ics, stream=None):
    _check(load().chs_shell_ics(h, n, _ptr(dirs), _ptr(E), _ptr(ics), _stream(stream)))


def chs_compact_work_size(n: int) -> int:
    return int(load().chs_compact_work_size(n))


def chs_integrate_compacted(h, prm: Params, ens: Ensemble, chunk_steps: int, work, stream=None):
    _check(load().chs_integrate_compacted(h, C.byref(prm), C.byref(ens), chunk_steps, _ptr(work),
                                          work.numel() * work.element_size(), _stream(stream)))


def chs_integrate_compacted_static(h, prm: Params, ens: Ensemble, chunk_steps: int, stream=None):
    """chs_integrate_compacted without a work buffer: for callers that cannot allocate
    device scratch (see include/chs.h); at most 1,048,576 orbits."""
    _check(load().chs_integrate_compacted_static(h, C.byref(prm), C.byref(ens), chunk_steps,
                                                 _stream(stream)))


def chs_integrate_persistent(h, prm: Params, ens: Ensemble, work, stream=None):
    _check(load().chs_integrate_persistent(h, C.byref(prm), C.byref(ens), _ptr(work),
                                           work.numel() * work.element_size(), _stream(stream)))


def chs_ensemble_init(h, prm: Params, ens: Ensemble, ics, ic_status=None, w_in=None, stream=None):
    _check(load().chs_ensemble_init(h, C.byref(prm), C.byref(ens), _ptr(ics), _ptr(ic_status),
                                    _ptr(w_in), _stream(stream)))


def chs_integrate_batch(h, prm: Params, ens: Ensemble, stream=None):
    _check(load().chs_integrate_batch(h, C.byref(prm), C.byref(ens), _stream(stream)))


def chs_integrate_adaptive(h, prm: Params, ad: Adaptive, ens: Ensemble, t, hstep, err_last=None,
                           err_max=None, n_rejected=None, stream=None):
    _check(load().chs_integrate_adaptive(h, C.byref(prm), C.byref(ad), C.byref(ens), _ptr(t),
                                         _ptr(hstep), _ptr(err_last), _ptr(err_max),
                                         _ptr(n_rejected), _stream(stream)))


def chs_indicators(h, prm: Params, ens: Ensemble, grid_ny=0, grid_npy=0, sali=None, gali=None,
                   ld_ind=None, label=None, stream=None):
    _check(load().chs_indicators(h, C.byref(prm), C.byref(ens), grid_ny, grid_npy, _ptr(sali),
                                 _ptr(gali), _ptr(ld_ind), _ptr(label), _stream(stream)))


def chs_lyapunov_spectrum(h, prm: Params, n, ics, ic_status, lam, status, stream=None):
    _check(load().chs_lyapunov_spectrum(h, C.byref(prm), n, _ptr(ics), _ptr(ic_status), _ptr(lam),
                                        _ptr(status), _stream(stream)))


def chs_lyapunov_adaptive(h, prm: Params, ad: Adaptive, n, ics, ic_status, lam, status,
                          n_steps=None, n_rejected=None, stream=None):
    _check(load().chs_lyapunov_adaptive(h, C.byref(prm), C.byref(ad), n, _ptr(ics), _ptr(ic_status),
                                        _ptr(lam), _ptr(status), _ptr(n_steps), _ptr(n_rejected),
                                        _stream(stream)))


def chs_lyapunov_batch(jobs, stream=None):
    """jobs: list of (handle, Params, n, ics, ic_status, lam, status) tuples."""
    arr = (LyapJob * len(jobs))()
    for i, (h, prm, n, ics, ic_st, lam, st) in enumerate(jobs):
        arr[i] = LyapJob(h.value if isinstance(h, C.c_void_p) else h, prm, n, _ptr(ics), _ptr(ic_st),
                         _ptr(lam), _ptr(st))
    _check(load().chs_lyapunov_batch(arr, len(jobs), _stream(stream)))


def chs_lyapunov_batch_persistent(jobs, work, stream=None):
    """jobs: list of (handle, Params, n, ics, ic_status, lam, status) tuples (FPUT,
    RK4); work: a device tensor of at least 8 bytes (the queue counter)."""
    arr = (LyapJob * len(jobs))()
    for i, (h, prm, n, ics, ic_st, lam, st) in enumerate(jobs):
        arr[i] = LyapJob(h.value if isinstance(h, C.c_void_p) else h, prm, n, _ptr(ics), _ptr(ic_st),
                         _ptr(lam), _ptr(st))
    _check(load().chs_lyapunov_batch_persistent(arr, len(jobs), _ptr(work), work.numel() * work.element_size(),
                                                _stream(stream)))


def chs_mlp_param_count() -> int:
    return int(load().chs_mlp_param_count())


def chs_mlp_features(series, n_samples, ld, t_decide, E, n, X, stream=None):
    _check(load().chs_mlp_features(_ptr(series), n_samples, _ptr(ld), t_decide, _ptr(E), n, _ptr(X),
                                   _stream(stream)))


def chs_mlp_forward(params, X, n, Y, act=None, stream=None):
    _check(load().chs_mlp_forward(_ptr(params), _ptr(X), n, _ptr(Y), _ptr(act), _stream(stream)))


def chs_mlp_loss_grad(Y, label, target, n, w_reg, dY, loss, stream=None):
    _check(load().chs_mlp_loss_grad(_ptr(Y), _ptr(label), _ptr(target), n, w_reg, _ptr(dY),
                                    _ptr(loss), _stream(stream)))


def chs_mlp_backward(params, X, act, dY, n, delta_work, grad, stream=None):
    _check(load().chs_mlp_backward(_ptr(params), _ptr(X), _ptr(act), _ptr(dY), n, _ptr(delta_work),
                                   _ptr(grad), _stream(stream)))


def chs_mlp_adam(master, m, v, grad, lr, beta1, beta2, eps, step, params_out, stream=None):
    _check(load().chs_mlp_adam(_ptr(master), _ptr(m), _ptr(v), _ptr(grad), lr, beta1, beta2, eps,
                               step, _ptr(params_out), _stream(stream)))


def chs_surrogate_decide(params, series, n_samples, ld, t_decide, E, confidence, n, status, prob=None,
                         stream=None):
    _check(load().chs_surrogate_decide(_ptr(params), _ptr(series), n_samples, _ptr(ld), t_decide, _ptr(E),
                                       confidence, n, _ptr(status), _ptr(prob), _stream(stream)))


def chs_check_params(prm: Params, model: int, n_dof: int):
    _check(load().chs_check_params(C.byref(prm), model, n_dof))


def chs_peak_probe(kind: int, n_blocks: int, n_threads: int, n_iter: int, sink, stream=None):
    _check(load().chs_peak_probe(kind, n_blocks, n_threads, n_iter, _ptr(sink), _stream(stream)))


def chs_probe_ops_per_thread(kind: int, n_iter: int) -> float:
    return float(load().chs_probe_ops_per_thread(kind, n_iter))


def chs_last_error() -> str:
    return load().chs_last_error().decode()


def chs_version() -> str:
    return load().chs_version().decode()


# ----------------------------------------------------------------------------
# convenience wrappers (allocation through torch, compute through the ABI)
# ----------------------------------------------------------------------------

class System:
    """Owns a chs_system handle."""

    def __init__(self, model: int, n_dof: int, sys_params=()):
        self.model, self.n_dof = model, n_dof
        self.d = 2 * n_dof
        self.h = chs_create_system(model, n_dof, sys_params)

    def close(self):
        if self.h:
            chs_destroy_system(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def vector_rows(k: int, d: int, vec_fp32: bool) -> int:
    """Rows of the ensemble's vector buffer: k*d (FP64), k*d + k(k+1)/2 (FP32 frame)."""
    if k <= 0:
        return 1
    return k * d + (k * (k + 1) // 2 if vec_fp32 else 0)


@dataclass
class DeviceEnsemble:
    """Caller-owned device buffers of a resumable ensemble (see chs_ensemble)."""
    x: torch.Tensor
    w: torch.Tensor
    ld: torch.Tensor
    h0: torch.Tensor
    dh_max: torch.Tensor
    n_exec: torch.Tensor
    status: torch.Tensor

    @classmethod
    def empty(cls, n: int, d: int, k: int, vec_fp32: bool = False, device="cuda"):
        f64 = dict(dtype=torch.float64, device=device)
        wdt = torch.float32 if vec_fp32 else torch.float64
        return cls(x=torch.empty((d, n), **f64),
                   w=torch.empty((vector_rows(k, d, vec_fp32), n), dtype=wdt, device=device),
                   ld=torch.zeros(n, **f64), h0=torch.empty(n, **f64), dh_max=torch.empty(n, **f64),
                   n_exec=torch.empty(n, dtype=torch.int64, device=device),
                   status=torch.empty(n, dtype=torch.int32, device=device))

    @property
    def n(self) -> int:
        return self.x.shape[1]

    def abi(self, with_ld: bool = True, t_end=None) -> Ensemble:
        p = lambda t: t.data_ptr()  # noqa: E731
        return Ensemble(self.n, p(self.x), p(self.w), p(self.ld) if with_ld else None, p(self.h0),
                        p(self.dh_max), p(self.n_exec), p(self.status),
                        None if t_end is None else p(t_end))


def compact_work(n: int, device="cuda") -> torch.Tensor:
    """A 256-byte aligned device scratch buffer for chs_integrate_compacted."""
    return torch.empty(chs_compact_work_size(n), dtype=torch.uint8, device=device)

"""Shared drivers for the parity tests: run the same seeded workload through the
CUDA library (via its C ABI binding) and through the CPU oracle."""
from __future__ import annotations

import numpy as np

import oracle as O

# parity tolerances: FP64 states within 1e-10 relative (to the orbit's
# state norm), indicators within 1e-8 * max(1, |ref|), labels >= 99.5 %.
STATE_RTOL = 1e-10
IND_TOL = 1e-8
LABEL_AGREE = 0.995


def frame_to_vectors(w, k: int, d: int) -> np.ndarray:
    """Unit vectors w_j / |w_j| = sum_i R_ij q_i from an FP32-mode vector buffer
    (rows: the k frame vectors q_i of length d, then the unit-column upper
    triangle R by columns), as numpy [k*d, n]."""
    w = np.asarray(w, dtype=np.float64)
    n = w.shape[1]
    Q = w[: k * d].reshape(k, d, n)
    out = np.zeros((k, d, n))
    for j in range(k):
        for i in range(j + 1):
            out[j] += w[k * d + j * (j + 1) // 2 + i] * Q[i]
    return out.reshape(k * d, n)


def state_rel_err(g: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Per-orbit max |g - r| / max |r| over components ([c, o] arrays)."""
    scale = np.maximum(np.abs(r).max(axis=0), 1e-300)
    return np.abs(g - r).max(axis=0) / scale


def ind_err(g: np.ndarray, r: np.ndarray) -> np.ndarray:
    return np.abs(g - r) / np.maximum(1.0, np.abs(r))


def oracle_system(model: int, n_dof: int, sys_params=()):
    if model == O.FPUT:
        kk, a, b = sys_params if sys_params else (1.0, 0.0, 1.0)
        return O.fput(n_dof, beta=b, alpha=a, kk=kk)
    if model == O.QUARTIC3:
        return O.system(O.QUARTIC3, 3, eps=sys_params[0] if sys_params else 0.1)
    return O.system(model, n_dof)


def oracle_run(model, n_dof, ics, ic_status, *, dt, n_steps, k, ld_p=0.5, renorm=True,
               sample_every=100, escape_r2=0.0, dh_limit=0.0, seed=1, w_in=None,
               sali_threshold=1e-8, chunks=None, grid=None, sys_params=(), early_exit=False,
               t_end=None, integrator=0):
    S = oracle_system(model, n_dof, sys_params)
    kw = dict(n_dev=k, ld_p=ld_p, renorm=renorm, sample_every=sample_every, escape_r2=escape_r2,
              dh_limit=dh_limit, early_exit=early_exit, sali_threshold=sali_threshold,
              integrator=integrator)
    e = O.Ensemble(S, O.params(dt, 1, **kw), ics, ic_status, w_in=w_in, seed=seed)
    step = 0
    for c in (chunks or [n_steps]):
        e.integrate(O.params(dt, c, step0=step, **kw), t_end=t_end)
        step += c
    out = dict(x=e.x, w=e.w, ld=e.ld, dh_max=e.dh_max, n_exec=e.n_exec, status=e.status)
    if k >= 2:
        sali, gali, label = e.indicators(sali_threshold)
        out.update(sali=sali, gali=gali, label=label)
    if grid is not None:
        dl, sl = O.ld_indicators(grid[0], grid[1], e.ld, e.status)
        out.update(dl=dl, sl=sl)
    return out


def gpu_run(model, n_dof, ics, ic_status, *, dt, n_steps, k, ld_p=0.5, renorm=True,
            sample_every=100, escape_r2=0.0, dh_limit=0.0, seed=1, w_in=None,
            sali_threshold=1e-8, chunks=None, grid=None, vec_fp32=False, sys_params=(),
            early_exit=False, t_end=None, compact_chunk=None, integrator=0, persistent=False,
            block_threads=0, clock_budget=0):
    import torch

    from paper_2507_00622_gb300 import chs

    S = chs.System(model, n_dof, sys_params)
    n = ics.shape[1]
    ens = chs.DeviceEnsemble.empty(n, S.d, k, vec_fp32)
    vp = chs.VEC_FP32 if vec_fp32 else chs.VEC_FP64
    kw = dict(n_dev=k, ld_p=ld_p, renorm=renorm, sample_every=sample_every, escape_r2=escape_r2,
              dh_limit=dh_limit, sali_threshold=sali_threshold, seed=seed, vec_precision=vp,
              early_exit=early_exit, integrator=integrator, block_threads=block_threads,
              clock_budget=clock_budget)
    ics_t = torch.from_numpy(np.ascontiguousarray(ics)).cuda()
    st_t = None if ic_status is None else torch.from_numpy(
        np.ascontiguousarray(ic_status, dtype=np.int32)).cuda()
    w_t = None
    if w_in is not None:
        w_t = torch.from_numpy(np.ascontiguousarray(w_in)).to(
            torch.float32 if vec_fp32 else torch.float64).cuda()
    te_t = None if t_end is None else torch.from_numpy(np.ascontiguousarray(t_end, dtype=np.int64)).cuda()
    abi = ens.abi(with_ld=ld_p > 0, t_end=te_t)
    chs.chs_ensemble_init(S.h, chs.params(dt, 1, **kw), abi, ics_t, st_t, w_t)
    step = 0
    work = chs.compact_work(n) if compact_chunk else None
    queue = torch.empty(1, dtype=torch.int64, device="cuda") if persistent else None
    for c in (chunks or [n_steps]):
        if compact_chunk:
            chs.chs_integrate_compacted(S.h, chs.params(dt, c, step0=step, **kw), abi, compact_chunk, work)
        elif persistent:
            chs.chs_integrate_persistent(S.h, chs.params(dt, c, step0=step, **kw), abi, queue)
        else:
            chs.chs_integrate_batch(S.h, chs.params(dt, c, step0=step, **kw), abi)
        step += c
    out = {}
    prm = chs.params(dt, 0, **kw)
    if k >= 2:
        sali = torch.empty(n, dtype=torch.float64, device="cuda")
        gali = torch.empty((k - 1, n), dtype=torch.float64, device="cuda")
        label = torch.empty(n, dtype=torch.int8, device="cuda")
        ldi = None
        if grid is not None:
            ldi = torch.empty((2, n), dtype=torch.float64, device="cuda")
        chs.chs_indicators(S.h, prm, abi, grid[0] if grid else 0, grid[1] if grid else 0, sali,
                           gali, ldi, label)
        out.update(sali=sali.cpu().numpy(), gali=gali.cpu().numpy(), label=label.cpu().numpy())
        if ldi is not None:
            out.update(dl=ldi[0].cpu().numpy(), sl=ldi[1].cpu().numpy())
    torch.cuda.synchronize()
    if vec_fp32 and k > 0:
        w_out = frame_to_vectors(ens.w.double().cpu().numpy(), k, S.d)
    else:
        w_out = ens.w[: k * S.d].double().cpu().numpy()
    out.update(x=ens.x.cpu().numpy(), w=w_out,
               ld=ens.ld.cpu().numpy(), dh_max=ens.dh_max.cpu().numpy(),
               n_exec=ens.n_exec.cpu().numpy(), status=ens.status.cpu().numpy(),
               h0=ens.h0.cpu().numpy())
    S.close()
    return out

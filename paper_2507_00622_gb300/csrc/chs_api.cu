// chs_api.cu -- the C ABI (include/chs.h): argument validation on the host,
// then asynchronous kernel launches on the caller's stream.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <utility>

#include "chs_internal.cuh"
#include "fput_batch.cuh"
#include "nvtx_range.cuh"
#include "k_dop853.cuh"

// Recorded chunk sequence of chs_integrate_compacted and the inputs it was
// recorded for.
struct CompactGraph {
    bool valid = false;
    chs_params p{};
    chs_ensemble e{};
    int32_t chunk = 0;
    void* work = nullptr;
    cudaGraphExec_t exec = nullptr;
};

struct chs_system_s {
    chs::SysPar sp;
    int device;
    cudaStream_t capture = nullptr;  // private stream used only to record graphs
    CompactGraph graph;
};

namespace {

thread_local std::string g_err;

chs_status fail(chs_status code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));

chs_status fail(chs_status code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

chs_status ok()
{
    return CHS_OK;
}

chs_status cuda_status(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return ok();
    return fail(CHS_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

chs::EnsPtrs ens_ptrs(const chs_ensemble* e)
{
    return chs::EnsPtrs{e->n_orbits, e->x, e->w, e->ld, e->h0, e->dh_max, e->n_exec, e->status,
                        e->t_end};
}

// Largest number of deviation vectors an ensemble of the system may carry.
int max_dev(const chs::SysPar& sp)
{
    return sp.n_dof == 2 ? 4 : 6;
}

// Ensembles (init, fixed and adaptive integration, indicators) run for the
// one-orbit-per-thread systems and for FPUT chains of N in {4, 8, 16, 32, 64}
// with FP64 vectors and no LD.  Call after check_params.
chs_status check_ens_model(const chs::SysPar& sp, const chs_params* p)
{
    if (chs::small_model(sp.model)) return ok();
    if (sp.model != CHS_FPUT) return fail(CHS_E_UNSUPPORTED, "ensembles are not implemented for model %d", sp.model);
    if (!chs::fput_ens_supported(sp.n_dof))
        return fail(CHS_E_UNSUPPORTED, "FPUT ensembles support N in {4, 8, 16, 32, 64}");
    if (p->vec_precision != CHS_VEC_FP64 && p->n_dev > 0)
        return fail(CHS_E_UNSUPPORTED, "FPUT ensembles carry FP64 deviation vectors");
    if (p->ld_p != 0.0) return fail(CHS_E_UNSUPPORTED, "FPUT ensembles do not accumulate the LD: ld_p must be 0");
    return ok();
}

chs_status check_params(const chs_params* p, const chs::SysPar& sp)
{
    if (!p) return fail(CHS_E_INVALID, "params is NULL");
    if (!isfinite(p->dt) || p->dt == 0.0) return fail(CHS_E_INVALID, "dt must be finite and non-zero");
    if (p->n_steps < 0) return fail(CHS_E_INVALID, "n_steps must be >= 0");
    if (p->step0 < 0) return fail(CHS_E_INVALID, "step0 must be >= 0");
    if (p->n_dev < 0 || p->n_dev > max_dev(sp))
        return fail(CHS_E_INVALID, "n_dev must be in 0..%d for this system", max_dev(sp));
    if (p->sample_every < 0) return fail(CHS_E_INVALID, "sample_every must be >= 0");
    if (p->renorm != 0 && p->renorm != 1) return fail(CHS_E_INVALID, "renorm must be 0 or 1");
    if (p->vec_precision != CHS_VEC_FP64 && p->vec_precision != CHS_VEC_FP32)
        return fail(CHS_E_INVALID, "vec_precision must be CHS_VEC_FP64 or CHS_VEC_FP32");
    if (p->early_exit != 0 && p->early_exit != 1) return fail(CHS_E_INVALID, "early_exit must be 0 or 1");
    if (p->early_exit && p->n_dev < 2) return fail(CHS_E_INVALID, "early_exit needs n_dev >= 2");
    if (!(p->sali_threshold >= 0.0)) return fail(CHS_E_INVALID, "sali_threshold must be >= 0");
    if (p->vec_precision == CHS_VEC_FP32 && p->n_dev > 0 && p->renorm != 1)
        return fail(CHS_E_INVALID, "FP32 vectors are re-orthonormalised every step: renorm must be 1");
    if (!(p->ld_p >= 0.0) || !isfinite(p->ld_p)) return fail(CHS_E_INVALID, "ld_p must be finite and >= 0");
    if (!(p->escape_r2 >= 0.0)) return fail(CHS_E_INVALID, "escape_r2 must be >= 0");
    if (!(p->dh_limit >= 0.0)) return fail(CHS_E_INVALID, "dh_limit must be >= 0");
    if (p->integrator != CHS_RK4 && p->integrator != CHS_DOP853)
        return fail(CHS_E_INVALID, "integrator must be CHS_RK4 or CHS_DOP853");
    if (p->integrator == CHS_DOP853 && p->vec_precision == CHS_VEC_FP32 && p->n_dev > 0)
        return fail(CHS_E_UNSUPPORTED, "DOP853 runs with FP64 deviation vectors only");
    if (p->block_threads != 0 && p->block_threads != 32 && p->block_threads != 64 && p->block_threads != 128)
        return fail(CHS_E_INVALID, "block_threads must be 0, 32, 64 or 128");
    if (p->clock_budget < 0) return fail(CHS_E_INVALID, "clock_budget must be >= 0 (0 = no limit)");
    if (p->threads_per_orbit != 0)
        return fail(CHS_E_UNSUPPORTED,
                    "threads_per_orbit applies to the RK4 FPUT Lyapunov spectrum only (chs_lyapunov_spectrum)");
    return ok();
}

chs_status check_ensemble(const chs_ensemble* e, const chs_params* p)
{
    if (!e) return fail(CHS_E_INVALID, "ensemble is NULL");
    if (e->n_orbits < 0) return fail(CHS_E_INVALID, "n_orbits must be >= 0");
    if (e->n_orbits > ((int64_t)1 << 40)) return fail(CHS_E_SIZE, "n_orbits exceeds 2^40");
    if (e->n_orbits == 0) return ok();
    if (!e->x || !e->h0 || !e->dh_max || !e->n_exec || !e->status)
        return fail(CHS_E_INVALID, "ensemble x, h0, dh_max, n_exec and status must be non-NULL");
    if (p->n_dev > 0 && !e->w) return fail(CHS_E_INVALID, "ensemble w is NULL but n_dev > 0");
    if (p->ld_p > 0.0 && !e->ld) return fail(CHS_E_INVALID, "ensemble ld is NULL but ld_p > 0");
    return ok();
}

chs::StepArgs step_args(const chs_params* p)
{
    chs::StepArgs a;
    a.dt = p->dt;
    a.n_steps = p->n_steps;
    a.step0 = p->step0;
    a.sample_every = p->sample_every;
    a.renorm = p->renorm;
    a.qr_every = p->qr_every;
    a.ld_sqrt = p->ld_p == 0.5 ? 1 : 0;
    a.ld_p = p->ld_p;
    a.escape_r2 = p->escape_r2;
    a.dh_limit = p->dh_limit;
    a.early_exit = p->early_exit;
    a.sali_threshold = p->sali_threshold;
    a.block = p->block_threads;
    a.clock_budget = p->clock_budget;
    a.threads_per_orbit = p->threads_per_orbit;
    return a;
}

// The integrate launch of the selected integrator (whole ensemble, or over the
// orbit list ol).
cudaError_t launch_selected(const chs::SysPar& sp, const chs_params* p, const chs::StepArgs& a,
                            const chs::EnsPtrs& ep, const chs::OrbitList* ol, cudaStream_t st)
{
    if (p->integrator == CHS_DOP853) return chs::launch_integrate_dp(sp, p->n_dev, p->ld_p > 0.0, a, ep, ol, st);
    return chs::launch_integrate(sp, p->n_dev, p->vec_precision, p->ld_p > 0.0, a, ep, ol, st);
}

chs_status check_handle(chs_system s)
{
    if (!s) return fail(CHS_E_INVALID, "system handle is NULL");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(CHS_E_CUDA, "cudaGetDevice failed");
    if (dev != s->device)
        return fail(CHS_E_INVALID, "system was created on device %d but device %d is current", s->device, dev);
    return ok();
}

}  // namespace

// Validation and plumbing shared with the entry point in chs_static.cu.
namespace chs {
chs_status api_validate_run(chs_system s, const chs_params* p, const chs_ensemble* e, int* device)
{
    chs_status r = check_handle(s);
    if (r != CHS_OK) return r;
    if (!small_model(s->sp.model))
        return fail(CHS_E_UNSUPPORTED, "integration is implemented for HENON_HEILES, HARMONIC, INVERTED, QUARTIC3");
    if ((r = check_params(p, s->sp)) != CHS_OK) return r;
    if ((r = check_ensemble(e, p)) != CHS_OK) return r;
    *device = s->device;
    return CHS_OK;
}
chs_status api_fail(chs_status code, const char* msg) { return fail(code, "%s", msg); }
StepArgs api_step_args(const chs_params* p) { return step_args(p); }
EnsPtrs api_ens_ptrs(const chs_ensemble* e) { return ens_ptrs(e); }
cudaError_t api_launch_integrate(const SysPar& sp, const chs_params* p, const StepArgs& a,
                                 const EnsPtrs& ep, const OrbitList* ol, cudaStream_t st)
{
    return launch_selected(sp, p, a, ep, ol, st);
}
SysPar api_syspar(chs_system s) { return s->sp; }
}  // namespace chs

extern "C" {

const char* chs_version(void) { return "chs 0.3.0 (sm_103a)"; }

const char* chs_last_error(void) { return g_err.c_str(); }

chs_status chs_check_params(const chs_params* p, chs_model model, int32_t n_dof)
{
    if (n_dof < 1) return fail(CHS_E_INVALID, "n_dof must be >= 1");
    const chs::SysPar sp{(int)model, n_dof, 1.0, 0.0, 1.0, 0.1};
    return check_params(p, sp);
}

chs_status chs_create_system(chs_system* out, chs_model model, int32_t n_dof, const double* params,
                             int32_t n_params)
{
    if (!out) return fail(CHS_E_INVALID, "out is NULL");
    *out = nullptr;
    if (n_params < 0 || (n_params > 0 && !params)) return fail(CHS_E_INVALID, "bad params array");
    chs::SysPar sp{(int)model, n_dof, 1.0, 0.0, 1.0, 0.1};
    switch (model) {
    case CHS_HENON_HEILES:
    case CHS_HARMONIC:
    case CHS_INVERTED:
        if (n_dof != 2) return fail(CHS_E_INVALID, "this model has n_dof = 2");
        if (n_params != 0) return fail(CHS_E_INVALID, "this model takes no parameters");
        break;
    case CHS_QUARTIC3:
        if (n_dof != 3) return fail(CHS_E_INVALID, "QUARTIC3 has n_dof = 3");
        if (n_params > 1) return fail(CHS_E_INVALID, "QUARTIC3 takes {eps}");
        if (n_params == 1) sp.eps = params[0];
        if (!isfinite(sp.eps)) return fail(CHS_E_INVALID, "eps must be finite");
        break;
    case CHS_FPUT:
        if (n_dof < 1 || n_dof > 4096) return fail(CHS_E_INVALID, "FPUT n_dof must be in 1..4096");
        if (n_params != 0 && n_params != 3) return fail(CHS_E_INVALID, "FPUT takes {k, alpha, beta}");
        if (n_params == 3) {
            sp.kk = params[0];
            sp.alpha = params[1];
            sp.beta = params[2];
        }
        if (!isfinite(sp.kk) || !isfinite(sp.alpha) || !isfinite(sp.beta))
            return fail(CHS_E_INVALID, "FPUT constants must be finite");
        break;
    default:
        return fail(CHS_E_INVALID, "unknown model %d", (int)model);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
    chs_system s = new (std::nothrow) chs_system_s;
    if (!s) return fail(CHS_E_NOMEM, "out of host memory");
    s->sp = sp;
    s->device = dev;
    *out = s;
    return ok();
}

chs_status chs_destroy_system(chs_system s)
{
    if (!s) return ok();
    if (s->graph.exec) cudaGraphExecDestroy(s->graph.exec);
    if (s->capture) cudaStreamDestroy(s->capture);
    delete s;
    return ok();
}

int32_t chs_system_dim(chs_system s) { return s ? 2 * s->sp.n_dof : -1; }

chs_status chs_section_grid_ics(chs_system s, double E, double y0, double y1, int32_t ny, double py0,
                                double py1, int32_t npy, double* ics_out, int32_t* status_out,
                                void* stream)
{
    CHS_NVTX_RANGE();
    chs_status r = check_handle(s);
    if (r != CHS_OK) return r;
    if (s->sp.model != CHS_HENON_HEILES) return fail(CHS_E_UNSUPPORTED, "section grid is for HENON_HEILES");
    if (ny <= 0 || npy <= 0) return fail(CHS_E_INVALID, "ny and npy must be > 0");
    if ((int64_t)ny * npy > ((int64_t)1 << 34)) return fail(CHS_E_SIZE, "grid too large");
    if (!isfinite(E) || !isfinite(y0) || !isfinite(y1) || !isfinite(py0) || !isfinite(py1))
        return fail(CHS_E_INVALID, "grid bounds and energy must be finite");
    if (!(y1 > y0) || !(py1 > py0)) return fail(CHS_E_INVALID, "need y1 > y0 and py1 > py0");
    if (!ics_out || !status_out) return fail(CHS_E_INVALID, "output pointers must be non-NULL");
    return cuda_status(chs::launch_grid_ics(E, y0, y1, ny, py0, py1, npy, ics_out, status_out,
                                            as_stream(stream)),
                       "section grid launch");
}

chs_status chs_fput_mode_ics(chs_system s, int64_t n, const double* Qm, const double* Pm,
                             const double* E, double* ics_out, void* stream)
{
    CHS_NVTX_RANGE();
    chs_status r = check_handle(s);
    if (r != CHS_OK) return r;
    if (s->sp.model != CHS_FPUT) return fail(CHS_E_UNSUPPORTED, "normal-mode ICs are for FPUT");
    if (s->sp.alpha != 0.0) return fail(CHS_E_UNSUPPORTED, "normal-mode energy scaling needs alpha = 0");
    if (n < 0) return fail(CHS_E_INVALID, "n must be >= 0");
    if (n == 0) return ok();
    if (!Qm || !Pm || !E || !ics_out) return fail(CHS_E_INVALID, "pointers must be non-NULL");
    return cuda_status(chs::launch_fput_mode_ics(s->sp, n, Qm, Pm, E, ics_out, as_stream(stream)),
                       "normal-mode launch");
}

chs_status chs_shell_ics(chs_system s, int64_t n, const double* dirs, const double* E,
                         double* ics_out, void* stream)
{
    CHS_NVTX_RANGE();
    chs_status r = check_handle(s);
    if (r != CHS_OK) return r;
    if (s->sp.model != CHS_QUARTIC3) return fail(CHS_E_UNSUPPORTED, "shell ICs are for QUARTIC3");
    if (n < 0) return fail(CHS_E_INVALID, "n must be >= 0");
    if (n == 0) return ok();
    if (!dirs || !E || !ics_out) return fail(CHS_E_INVALID, "pointers must be non-NULL");
    return cuda_status(chs::launch_shell_ics(s->sp, n, dirs, E, ics_out, as_stream(stream)),
                       "shell ICs launch");
}

chs_status chs_ensemble_init(chs_system s, const chs_params* p, const chs_ensemble* e,
                             const double* ics, const int32_t* ic_status, const void* w_in,
                             void* stream)
{
    CHS_NVTX_RANGE();
    chs_status r = check_handle(s);
    if (r != CHS_OK) return r;
    if ((r = check_params(p, s->sp)) != CHS_OK) return r;
    if ((r = check_ens_model(s->sp, p)) != CHS_OK) return r;
    if ((r = check_ensemble(e, p)) != CHS_OK) return r;
    if (e->n_orbits == 0) return ok();
    if (!ics) return fail(CHS_E_INVALID, "ics is NULL");
    if (s->sp.model == CHS_FPUT)
        return cuda_status(chs::launch_fput_ens_init(s->sp, p->n_dev, p->renorm, p->seed, ics, ic_status, w_in,
                                                     ens_ptrs(e), as_stream(stream)),
                           "FPUT ensemble init launch");
    return cuda_status(chs::launch_init(s->sp, p->n_dev, p->vec_precision, p->renorm, p->seed, ics,
                                        ic_status, w_in, ens_ptrs(e), as_stream(stream)),
                       "ensemble init launch");
}

chs_status chs_integrate_batch(chs_system s, const chs_params* p, const chs_ensemble* e, void* stream)
{
    CHS_NVTX_RANGE();
    chs_status r = check_handle(s);
    if (r != CHS_OK) return r;
    if ((r = check_params(p, s->sp)) != CHS_OK) return r;
    if ((r = check_ens_model(s->sp, p)) != CHS_OK) return r;
    if ((r = check_ensemble(e, p)) != CHS_OK) return r;
    if (e->n_orbits == 0 || p->n_steps == 0) return ok();
    if (s->sp.model == CHS_FPUT)
        return cuda_status(chs::launch_fput_ens(s->sp, p->integrator, p->n_dev, step_args(p), ens_ptrs(e),
                                                as_stream(stream)),
                           "FPUT ensemble integrate launch");
    return cuda_status(launch_selected(s->sp, p, step_args(p), ens_ptrs(e), nullptr, as_stream(stream)),
                       "integrate launch");
}

chs_status chs_integrate_adaptive(chs_system s, const chs_params* p, const chs_adaptive* a,
                                  const chs_ensemble* e, double* t, double* h, double* err_last,
                                  double* err_max, int64_t* n_rejected, void* stream)
{
    CHS_NVTX_RANGE();
    chs_status r = check_handle(s);
    if (r != CHS_OK) return r;
    if ((r = check_params(p, s->sp)) != CHS_OK) return r;
    if ((r = check_ens_model(s->sp, p)) != CHS_OK) return r;
    if ((r = check_ensemble(e, p)) != CHS_OK) return r;
    if (p->integrator != CHS_DOP853) return fail(CHS_E_INVALID, "adaptive runs need integrator = CHS_DOP853");
    if (!a) return fail(CHS_E_INVALID, "adaptive controls are NULL");
    if (!isfinite(a->t_final)) return fail(CHS_E_INVALID, "t_final must be finite");
    if (!(a->rtol >= 0.0) || !(a->atol >= 0.0) || !isfinite(a->rtol) || !isfinite(a->atol))
        return fail(CHS_E_INVALID, "rtol and atol must be finite and >= 0");
    if (isnan(a->h_max)) return fail(CHS_E_INVALID, "h_max must not be NaN");
    if (e->t_end) return fail(CHS_E_INVALID, "adaptive runs do not take t_end (use t_final)");
    if (e->n_orbits > 0 && (!t || !h)) return fail(CHS_E_INVALID, "t and h must be non-NULL");
    if (e->n_orbits == 0 || p->n_steps == 0) return ok();
    const chs::AdaptArgs ad{a->t_final, a->rtol, a->atol, a->h_max};
    const chs::AdaptPtrs ap{t, h, err_last, err_max, n_rejected};
    if (s->sp.model == CHS_FPUT)
        return cuda_status(chs::launch_fput_ens_adapt(s->sp, p->n_dev, step_args(p), ad, ens_ptrs(e), ap,
                                                      as_stream(stream)),
                           "adaptive FPUT ensemble launch");
    return cuda_status(chs::launch_integrate_adaptive(s->sp, p->n_dev, p->ld_p > 0.0, step_args(p), ad,
                                                      ens_ptrs(e), ap, as_stream(stream)),
                       "adaptive integrate launch");
}

chs_status chs_integrate_persistent(chs_system s, const chs_params* p, const chs_ensemble* e, void* work,
                                    size_t work_bytes, void* stream)
{
    CHS_NVTX_RANGE();
    chs_status r = check_handle(s);
    if (r != CHS_OK) return r;
    if (!chs::small_model(s->sp.model))
        return fail(CHS_E_UNSUPPORTED, "persistent runs are implemented for HENON_HEILES, HARMONIC, INVERTED, QUARTIC3");
    if ((r = check_params(p, s->sp)) != CHS_OK) return r;
    if ((r = check_ensemble(e, p)) != CHS_OK) return r;
    if (!work || ((uintptr_t)work & 7u)) return fail(CHS_E_INVALID, "work must be an 8-byte aligned device buffer");
    if (work_bytes < 8) return fail(CHS_E_SIZE, "work must hold at least 8 bytes");
    if (e->n_orbits == 0 || p->n_steps == 0) return ok();
    cudaStream_t st = as_stream(stream);
    cudaError_t ce = cudaMemsetAsync(work, 0, sizeof(unsigned long long), st);
    if (ce != cudaSuccess) return cuda_status(ce, "queue reset");
    const chs::OrbitList ol{nullptr, nullptr, nullptr, nullptr, static_cast<unsigned long long*>(work)};
    return cuda_status(launch_selected(s->sp, p, step_args(p), ens_ptrs(e), &ol, st), "persistent integrate launch");
}

size_t chs_compact_work_size(int64_t n_orbits)
{
    if (n_orbits < 0) return 0;
    const size_t list = (((size_t)n_orbits * sizeof(int32_t)) + 255) / 256 * 256;
    return 2 * list + 256;
}

chs_status chs_integrate_compacted(chs_system s, const chs_params* p, const chs_ensemble* e,
                                   int32_t chunk_steps, void* work, size_t work_bytes, void* stream)
{
    CHS_NVTX_RANGE();
    chs_status r = check_handle(s);
    if (r != CHS_OK) return r;
    if (!chs::small_model(s->sp.model))
        return fail(CHS_E_UNSUPPORTED, "compacted runs are implemented for HENON_HEILES, HARMONIC, INVERTED, QUARTIC3");
    if ((r = check_params(p, s->sp)) != CHS_OK) return r;
    if ((r = check_ensemble(e, p)) != CHS_OK) return r;
    if (chunk_steps < 1) return fail(CHS_E_INVALID, "chunk_steps must be >= 1");
    if (e->n_orbits > INT32_MAX) return fail(CHS_E_SIZE, "compacted runs support at most 2^31 - 1 orbits");
    if (e->n_orbits == 0 || p->n_steps == 0) return ok();
    const int64_t n_chunks = (p->n_steps + chunk_steps - 1) / chunk_steps;
    if (n_chunks > 100000) return fail(CHS_E_SIZE, "more than 100000 chunks: raise chunk_steps");
    if (!work || ((uintptr_t)work & 255u)) return fail(CHS_E_INVALID, "work must be a 256-byte aligned device buffer");
    if (work_bytes < chs_compact_work_size(e->n_orbits))
        return fail(CHS_E_SIZE, "work buffer smaller than chs_compact_work_size(n)");

    CompactGraph& G = s->graph;
    const bool same = G.valid && G.chunk == chunk_steps && G.work == work &&
                      memcmp(&G.p, p, sizeof(chs_params)) == 0 &&
                      memcmp(&G.e, e, sizeof(chs_ensemble)) == 0;
    if (!same) {
        if (G.exec) {
            cudaGraphExecDestroy(G.exec);
            G.exec = nullptr;
        }
        G.valid = false;
        cudaError_t ce;
        if (!s->capture && (ce = cudaStreamCreateWithFlags(&s->capture, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_status(ce, "capture stream");
        const size_t list_bytes = (((size_t)e->n_orbits * sizeof(int32_t)) + 255) / 256 * 256;
        int32_t* la = static_cast<int32_t*>(work);
        int32_t* lb = reinterpret_cast<int32_t*>(static_cast<char*>(work) + list_bytes);
        int32_t* ca = reinterpret_cast<int32_t*>(static_cast<char*>(work) + 2 * list_bytes);
        int32_t* cb = ca + 1;
        const chs::EnsPtrs ep = ens_ptrs(e);
        cudaStream_t cs = s->capture;
        if ((ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cuda_status(ce, "begin capture");
        cudaError_t le = cudaMemsetAsync(ca, 0, sizeof(int32_t), cs);
        if (le == cudaSuccess) le = chs::launch_list_init(ep, la, ca, cs);
        for (int64_t c = 0; c < n_chunks && le == cudaSuccess; ++c) {
            chs::StepArgs a = step_args(p);
            a.step0 = p->step0 + c * chunk_steps;
            a.n_steps = std::min<int64_t>(chunk_steps, p->n_steps - c * chunk_steps);
            le = cudaMemsetAsync(cb, 0, sizeof(int32_t), cs);
            const chs::OrbitList ol{la, ca, lb, cb, nullptr};
            if (le == cudaSuccess) le = launch_selected(s->sp, p, a, ep, &ol, cs);
            std::swap(la, lb);
            std::swap(ca, cb);
        }
        cudaGraph_t graph = nullptr;
        ce = cudaStreamEndCapture(cs, &graph);
        if (le != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_status(le, "recording the chunk sequence");
        }
        if (ce != cudaSuccess) return cuda_status(ce, "end capture");
        ce = cudaGraphInstantiate(&G.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            G.exec = nullptr;
            return cuda_status(ce, "graph instantiate");
        }
        G.p = *p;
        G.e = *e;
        G.chunk = chunk_steps;
        G.work = work;
        G.valid = true;
    }
    return cuda_status(cudaGraphLaunch(G.exec, as_stream(stream)), "graph launch");
}

chs_status chs_indicators(chs_system s, const chs_params* p, const chs_ensemble* e, int32_t grid_ny,
                          int32_t grid_npy, double* sali_out, double* gali_out, double* ld_ind_out,
                          int8_t* label_out, void* stream)
{
    CHS_NVTX_RANGE();
    chs_status r = check_handle(s);
    if (r != CHS_OK) return r;
    if ((r = check_params(p, s->sp)) != CHS_OK) return r;
    if ((r = check_ens_model(s->sp, p)) != CHS_OK) return r;
    if ((r = check_ensemble(e, p)) != CHS_OK) return r;
    if (s->sp.model == CHS_FPUT && ld_ind_out)
        return fail(CHS_E_UNSUPPORTED, "LD indicators are for the Henon-Heiles section grid");
    if ((sali_out || label_out) && p->n_dev < 2) return fail(CHS_E_INVALID, "SALI and labels need n_dev >= 2");
    if (gali_out && p->n_dev < 2) return fail(CHS_E_INVALID, "GALI needs n_dev >= 2");
    if (ld_ind_out) {
        if (grid_ny < 3 || grid_npy < 3 || (int64_t)grid_ny * grid_npy != e->n_orbits)
            return fail(CHS_E_INVALID, "LD indicators need a grid_ny x grid_npy grid (each >= 3) covering n_orbits");
        if (!e->ld) return fail(CHS_E_INVALID, "LD indicators need the ensemble LD");
    }
    if (e->n_orbits == 0) return ok();
    cudaStream_t st = as_stream(stream);
    const chs::EnsPtrs ep = ens_ptrs(e);
    if (s->sp.model == CHS_FPUT) {
        if (!sali_out && !gali_out && !label_out) return ok();
        return cuda_status(chs::launch_fput_ens_indicators(s->sp, p->n_dev, p->sali_threshold, ep, sali_out,
                                                           gali_out, label_out, st),
                           "FPUT indicator launch");
    }
    if (sali_out || gali_out || label_out) {
        r = cuda_status(chs::launch_indicators(s->sp, p->n_dev, p->vec_precision, p->sali_threshold, ep,
                                               sali_out, gali_out, label_out, st),
                        "indicator launch");
        if (r != CHS_OK) return r;
    }
    if (ld_ind_out)
        return cuda_status(chs::launch_ld_stencil(grid_ny, grid_npy, e->ld, e->status, ld_ind_out, st),
                           "LD stencil launch");
    return ok();
}

static chs_status lyap_check(chs_system s, const chs_params* p, int64_t n, const double* ics,
                             double* lambda_out, int32_t* status_out);

static chs_status lyap_launch(chs_system s, const chs_params* p, int64_t n, const double* ics,
                              const int32_t* ic_status, double* lambda_out, int32_t* status_out,
                              cudaStream_t st)
{
    const chs::StepArgs a = step_args(p);
    if (p->integrator == CHS_DOP853 && s->sp.model == CHS_FPUT)
        return cuda_status(chs::launch_fput_lyap_dp(s->sp, a, n, ics, ic_status, lambda_out, status_out, st),
                           "FPUT Lyapunov launch");
    if (p->integrator == CHS_DOP853)
        return cuda_status(chs::launch_lyap_small_dp(s->sp, a, n, ics, ic_status, lambda_out, status_out, st),
                           "Lyapunov launch");
    if (s->sp.model == CHS_FPUT)
        return cuda_status(chs::launch_fput_lyap(s->sp, a, n, ics, ic_status, lambda_out, status_out, st),
                           "FPUT Lyapunov launch");
    return cuda_status(chs::launch_lyap_small(s->sp, a, n, ics, ic_status, lambda_out, status_out, st),
                       "Lyapunov launch");
}

chs_status chs_lyapunov_batch(const chs_lyap_job* jobs, int32_t n_jobs, void* stream)
{
    CHS_NVTX_RANGE();
    constexpr int kMaxJobs = 16;
    if (!jobs || n_jobs < 1 || n_jobs > kMaxJobs) return fail(CHS_E_INVALID, "need 1..16 jobs");
    for (int i = 0; i < n_jobs; ++i) {
        const chs_lyap_job& j = jobs[i];
        chs_status r = lyap_check(j.sys, &j.params, j.n_orbits, j.ics, j.lambda_out, j.status_out);
        if (r != CHS_OK) return r;
    }
    // private streams and events for recording the fork/join graph (per thread, created once)
    thread_local cudaStream_t lanes[kMaxJobs + 1] = {};
    thread_local cudaEvent_t evs[kMaxJobs + 1] = {};
    thread_local int lanes_device = -1;
    int dev = -1;
    cudaGetDevice(&dev);
    if (lanes_device != dev) {
        for (int i = 0; i <= kMaxJobs; ++i) {
            cudaError_t e = cudaStreamCreateWithFlags(&lanes[i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&evs[i], cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_status(e, "batch streams");
        }
        lanes_device = dev;
    }
    // kernel attributes are set before recording (no such calls inside a capture)
    for (int i = 0; i < n_jobs; ++i)
        if (jobs[i].sys->sp.model == CHS_FPUT) {
            cudaError_t pe = jobs[i].params.integrator == CHS_DOP853
                                 ? chs::prepare_fput_lyap_dp(jobs[i].sys->sp.n_dof)
                                 : chs::prepare_fput_lyap(jobs[i].sys->sp.n_dof);
            if (pe != cudaSuccess) return cuda_status(pe, "FPUT kernel attributes");
        }
    cudaStream_t root = lanes[kMaxJobs];
    cudaError_t e = cudaStreamBeginCapture(root, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_status(e, "begin capture");
    cudaError_t le = cudaEventRecord(evs[kMaxJobs], root);
    chs_status r = CHS_OK;
    for (int i = 0; i < n_jobs && le == cudaSuccess && r == CHS_OK; ++i) {
        const chs_lyap_job& j = jobs[i];
        le = cudaStreamWaitEvent(lanes[i], evs[kMaxJobs], 0);
        if (le != cudaSuccess) break;
        r = lyap_launch(j.sys, &j.params, j.n_orbits, j.ics, j.ic_status, j.lambda_out, j.status_out, lanes[i]);
        if (r != CHS_OK) break;
        le = cudaEventRecord(evs[i], lanes[i]);
        if (le == cudaSuccess) le = cudaStreamWaitEvent(root, evs[i], 0);
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(root, &graph);
    if (r != CHS_OK || le != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (r != CHS_OK) return r;
        return cuda_status(le != cudaSuccess ? le : e, "recording the batch");
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_status(e, "batch instantiate");
    e = cudaGraphLaunch(exec, as_stream(stream));
    cudaGraphExecDestroy(exec);
    return cuda_status(e, "batch launch");
}

static chs_status lyap_check(chs_system s, const chs_params* p, int64_t n, const double* ics,
                             double* lambda_out, int32_t* status_out)
{
    chs_status r = check_handle(s);
    if (r != CHS_OK) return r;
    if (!p) return fail(CHS_E_INVALID, "params is NULL");
    if (!isfinite(p->dt) || p->dt == 0.0) return fail(CHS_E_INVALID, "dt must be finite and non-zero");
    if (p->n_steps < 1) return fail(CHS_E_INVALID, "n_steps must be >= 1");
    if (p->qr_every < 1) return fail(CHS_E_INVALID, "qr_every must be >= 1");
    if (p->sample_every < 0) return fail(CHS_E_INVALID, "sample_every must be >= 0");
    if (p->vec_precision != CHS_VEC_FP64) return fail(CHS_E_UNSUPPORTED, "the Lyapunov path is FP64 only");
    if (p->integrator != CHS_RK4 && p->integrator != CHS_DOP853)
        return fail(CHS_E_INVALID, "integrator must be CHS_RK4 or CHS_DOP853");
    const bool n64_wide = s->sp.model == CHS_FPUT && s->sp.n_dof == 64;
    if (p->block_threads != 0 && p->block_threads != 32 && p->block_threads != 64 && p->block_threads != 128 &&
        !(p->block_threads == 256 && n64_wide))
        return fail(CHS_E_INVALID, "block_threads must be 0, 32, 64 or 128 (or 256 for the FPUT spectrum at N = 64)");
    if (p->clock_budget < 0) return fail(CHS_E_INVALID, "clock_budget must be >= 0 (0 = no limit)");
    if (p->threads_per_orbit != 0 &&
        !(s->sp.model == CHS_FPUT && p->integrator == CHS_RK4 &&
          chs::fput_lanes_per_orbit_supported(s->sp.n_dof, p->threads_per_orbit)))
        return fail(CHS_E_UNSUPPORTED,
                    "threads_per_orbit: 0, or for the RK4 FPUT spectrum 1, 2, 4 at N = 4 and 2, 4, 8 at N = 8");
    if (s->sp.model == CHS_FPUT && p->block_threads != 0 && p->block_threads < 2 * s->sp.n_dof)
        return fail(CHS_E_INVALID, "FPUT: block_threads must be 0 or at least 2N");
    if (n < 0) return fail(CHS_E_INVALID, "n must be >= 0");
    if (n > ((int64_t)1 << 31)) return fail(CHS_E_SIZE, "n exceeds 2^31");
    if (n > 0 && (!ics || !lambda_out || !status_out)) return fail(CHS_E_INVALID, "pointers must be non-NULL");
    if (s->sp.model == CHS_FPUT) {
        if (!chs::fput_lyap_supported(s->sp.n_dof))
            return fail(CHS_E_UNSUPPORTED, "FPUT Lyapunov supports N in {4, 8, 16, 32, 64}");
    } else if (!(s->sp.model == CHS_HENON_HEILES || s->sp.model == CHS_HARMONIC || s->sp.model == CHS_INVERTED)) {
        return fail(CHS_E_UNSUPPORTED, "Lyapunov spectrum not implemented for this model");
    }
    return CHS_OK;
}

chs_status chs_lyapunov_batch_persistent(const chs_lyap_job* jobs, int32_t n_jobs, void* work, size_t work_bytes,
                                         void* stream)
{
    CHS_NVTX_RANGE();
    if (!jobs || n_jobs < 1 || n_jobs > chs::kFputBatchMaxJobs) return fail(CHS_E_INVALID, "need 1..16 jobs");
    if (!work || ((uintptr_t)work & 7u)) return fail(CHS_E_INVALID, "work must be an 8-byte aligned device buffer");
    if (work_bytes < 8) return fail(CHS_E_SIZE, "work must hold at least 8 bytes");
    chs::FputBatchJob bj[chs::kFputBatchMaxJobs];
    for (int i = 0; i < n_jobs; ++i) {
        const chs_lyap_job& j = jobs[i];
        chs_status r = lyap_check(j.sys, &j.params, j.n_orbits, j.ics, j.lambda_out, j.status_out);
        if (r != CHS_OK) return r;
        if (j.sys->sp.model != CHS_FPUT || j.params.integrator != CHS_RK4)
            return fail(CHS_E_UNSUPPORTED, "job %d: the persistent batch runs FPUT chains under RK4", i);
        bj[i] = chs::FputBatchJob{step_args(&j.params), j.sys->sp, j.n_orbits, j.ics, j.ic_status, j.lambda_out,
                                  j.status_out, j.sys->sp.n_dof, j.sys->sp.alpha == 0.0 ? 1 : 0, 0};
    }
    return cuda_status(chs::launch_fput_lyap_batch(bj, n_jobs, static_cast<unsigned long long*>(work),
                                                   as_stream(stream)),
                       "persistent batch launch");
}

chs_status chs_lyapunov_spectrum(chs_system s, const chs_params* p, int64_t n, const double* ics,
                                 const int32_t* ic_status, double* lambda_out, int32_t* status_out,
                                 void* stream)
{
    CHS_NVTX_RANGE();
    chs_status r = lyap_check(s, p, n, ics, lambda_out, status_out);
    if (r != CHS_OK) return r;
    if (n == 0) return ok();
    return lyap_launch(s, p, n, ics, ic_status, lambda_out, status_out, as_stream(stream));
}

chs_status chs_lyapunov_adaptive(chs_system s, const chs_params* p, const chs_adaptive* a, int64_t n,
                                 const double* ics, const int32_t* ic_status, double* lambda_out,
                                 int32_t* status_out, int64_t* n_steps_out, int64_t* n_rejected_out,
                                 void* stream)
{
    CHS_NVTX_RANGE();
    chs_status r = lyap_check(s, p, n, ics, lambda_out, status_out);
    if (r != CHS_OK) return r;
    if (p->integrator != CHS_DOP853) return fail(CHS_E_INVALID, "adaptive runs need integrator = CHS_DOP853");
    if (!(p->dt > 0.0)) return fail(CHS_E_INVALID, "dt (the first step size) must be > 0");
    if (!a) return fail(CHS_E_INVALID, "adaptive controls are NULL");
    if (!(a->t_final > 0.0) || !isfinite(a->t_final)) return fail(CHS_E_INVALID, "t_final must be finite and > 0");
    if (!(a->rtol >= 0.0) || !(a->atol >= 0.0) || !isfinite(a->rtol) || !isfinite(a->atol))
        return fail(CHS_E_INVALID, "rtol and atol must be finite and >= 0");
    if (isnan(a->h_max)) return fail(CHS_E_INVALID, "h_max must not be NaN");
    if (n == 0) return ok();
    const chs::StepArgs sa = step_args(p);
    const chs::AdaptArgs ad{a->t_final, a->rtol, a->atol, a->h_max};
    cudaStream_t st = as_stream(stream);
    if (s->sp.model == CHS_FPUT)
        return cuda_status(chs::launch_fput_lyap_adapt(s->sp, sa, ad, n, ics, ic_status, lambda_out, status_out,
                                                       n_steps_out, n_rejected_out, st),
                           "adaptive FPUT Lyapunov launch");
    return cuda_status(chs::launch_lyap_small_adapt(s->sp, sa, ad, n, ics, ic_status, lambda_out, status_out,
                                                    n_steps_out, n_rejected_out, st),
                       "adaptive Lyapunov launch");
}

chs_status chs_peak_probe(int32_t kind, int32_t n_blocks, int32_t n_threads, int64_t n_iter, double* sink,
                          void* stream)
{
    CHS_NVTX_RANGE();
    if (kind < CHS_PROBE_DFMA || kind > CHS_PROBE_DFMA_DMMA) return fail(CHS_E_INVALID, "unknown probe kind %d", kind);
    if (n_blocks < 1 || n_blocks > 65535) return fail(CHS_E_INVALID, "n_blocks must be in 1..65535");
    if (n_threads < 32 || n_threads > 1024 || n_threads % 32 != 0)
        return fail(CHS_E_INVALID, "n_threads must be a multiple of 32 in 32..1024");
    if (n_iter < 1 || n_iter > ((int64_t)1 << 28)) return fail(CHS_E_INVALID, "n_iter must be in 1..2^28");
    if (!sink) return fail(CHS_E_INVALID, "sink is NULL");
    return cuda_status(chs::launch_peak_probe(kind, n_blocks, n_threads, n_iter, sink, as_stream(stream)),
                       "probe launch");
}

double chs_probe_ops_per_thread(int32_t kind, int64_t n_iter)
{
    return n_iter < 1 ? 0.0 : chs::probe_ops_per_thread(kind, n_iter);
}

size_t chs_mlp_param_count(void) { return chs::mlp_param_count(); }

chs_status chs_mlp_features(const double* sali_series, int32_t n_samples, const double* ld,
                            double t_decide, const double* E, int64_t n, float* X, void* stream)
{
    CHS_NVTX_RANGE();
    if (n < 0 || n_samples < 0 || n_samples > 10) return fail(CHS_E_INVALID, "need n >= 0 and 0 <= n_samples <= 10");
    if (!(t_decide > 0.0)) return fail(CHS_E_INVALID, "t_decide must be > 0");
    if (n == 0) return ok();
    if ((n_samples > 0 && !sali_series) || !ld || !E || !X) return fail(CHS_E_INVALID, "pointers must be non-NULL");
    return cuda_status(chs::launch_mlp_features(sali_series, n_samples, ld, t_decide, E, n, X,
                                                as_stream(stream)), "features launch");
}

chs_status chs_mlp_forward(const void* params_bf16, const float* X, int64_t n, float* Y, void* act,
                           void* stream)
{
    CHS_NVTX_RANGE();
    if (n < 0) return fail(CHS_E_INVALID, "n must be >= 0");
    if (n == 0) return ok();
    if (!params_bf16 || !X || !Y) return fail(CHS_E_INVALID, "pointers must be non-NULL");
    return cuda_status(chs::launch_mlp_forward(params_bf16, X, n, Y, act, as_stream(stream)),
                       "forward launch");
}

chs_status chs_mlp_loss_grad(const float* Y, const float* label, const float* target, int64_t n,
                             float w_reg, float* dY, float* loss_out, void* stream)
{
    CHS_NVTX_RANGE();
    if (n < 0) return fail(CHS_E_INVALID, "n must be >= 0");
    if (n == 0) return ok();
    if (!Y || !label || !target || !dY || !loss_out) return fail(CHS_E_INVALID, "pointers must be non-NULL");
    return cuda_status(chs::launch_mlp_loss_grad(Y, label, target, n, w_reg, dY, loss_out,
                                                 as_stream(stream)), "loss launch");
}

chs_status chs_mlp_backward(const void* params_bf16, const float* X, const void* act, const float* dY,
                            int64_t n, float* delta_work, float* grad_out, void* stream)
{
    CHS_NVTX_RANGE();
    if (n < 1) return fail(CHS_E_INVALID, "n must be >= 1");
    if (!params_bf16 || !X || !act || !dY || !delta_work || !grad_out)
        return fail(CHS_E_INVALID, "pointers must be non-NULL");
    return cuda_status(chs::launch_mlp_backward(params_bf16, X, act, dY, n, delta_work, grad_out,
                                                as_stream(stream)), "backward launch");
}

chs_status chs_mlp_adam(float* master, float* m, float* v, const float* grad, float lr, float beta1,
                        float beta2, float eps, int32_t step, void* params_bf16_out, void* stream)
{
    CHS_NVTX_RANGE();
    if (!master || !m || !v || !grad || !params_bf16_out) return fail(CHS_E_INVALID, "pointers must be non-NULL");
    if (step < 1 || !(lr > 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f))
        return fail(CHS_E_INVALID, "need step >= 1, lr > 0 and betas in [0, 1)");
    return cuda_status(chs::launch_mlp_adam(master, m, v, grad, lr, beta1, beta2, eps, step,
                                            params_bf16_out, as_stream(stream)), "adam launch");
}

chs_status chs_surrogate_decide(const void* params_bf16, const double* sali_series, int32_t n_samples,
                                const double* ld, double t_decide, const double* E, double confidence,
                                int64_t n, int32_t* status_inout, float* prob_out, void* stream)
{
    CHS_NVTX_RANGE();
    if (n < 0 || n_samples < 1 || n_samples > 10) return fail(CHS_E_INVALID, "need n >= 0 and 1 <= n_samples <= 10");
    if (!(t_decide > 0.0)) return fail(CHS_E_INVALID, "t_decide must be > 0");
    if (!(confidence > 0.5 && confidence <= 1.0)) return fail(CHS_E_INVALID, "confidence must be in (0.5, 1]");
    if (n == 0) return ok();
    if (!params_bf16 || !sali_series || !ld || !E || !status_inout) return fail(CHS_E_INVALID, "pointers must be non-NULL");
    return cuda_status(chs::launch_mlp_decide(params_bf16, sali_series, n_samples, ld, t_decide, E, n,
                                              confidence, status_inout, prob_out, as_stream(stream)),
                       "decide launch");
}

}  // extern "C"

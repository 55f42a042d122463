// chs_internal.cuh -- shared declarations of the CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/chs.h"

namespace chs {

constexpr int kSmallBlock = 128;  // threads per block of the one-orbit-per-thread kernels
constexpr int kMaxDev = 6;        // largest number of deviation vectors in an ensemble

// Model constants as the kernels see them.
struct SysPar {
    int model;
    int n_dof;
    double kk, alpha, beta, eps;
};

// Device pointers of a resumable ensemble (mirror of chs_ensemble).
struct EnsPtrs {
    int64_t n;
    double* x;
    void* w;
    double* ld;
    double* h0;
    double* dh_max;
    int64_t* n_exec;
    int32_t* status;
    const int64_t* t_end;  // optional per-orbit end step
};

// How the one-orbit-per-thread integrate kernels pick their orbits.
//   compacted list (list set): thread t integrates orbit list[t] for
//     t < *count and appends the orbits still running to next / *next_count;
//   work queue (queue set): a persistent grid whose threads take orbit indices
//     from the counter *queue (starting at 0) until they run past n.
struct OrbitList {
    const int32_t* list;
    const int32_t* count;
    int32_t* next;
    int32_t* next_count;
    unsigned long long* queue;
};

enum { kModeAll = 0, kModeList = 1, kModeQueue = 2 };

__device__ __forceinline__ int integ_mode(const OrbitList& ol)
{
    return ol.queue ? kModeQueue : (ol.list ? kModeList : kModeAll);
}

// Integration controls, validated on the host.
struct StepArgs {
    double dt;
    int64_t n_steps;
    int64_t step0;
    int32_t sample_every;  // 0: no health checks
    int32_t renorm;
    int32_t qr_every;
    int32_t ld_sqrt;       // 1: LD exponent is exactly 1/2 (sqrt path)
    double ld_p;
    double escape_r2;      // 0: off
    double dh_limit;       // 0: off
    int32_t early_exit;    // freeze as EARLY_CHAOTIC once SALI < sali_threshold
    double sali_threshold;
    int32_t block;         // threads per block requested (0: the kernel's default)
    int64_t clock_budget;  // SM clock cycles an orbit may run in this call (0: no limit)
    int32_t threads_per_orbit;  // FPUT Lyapunov, N = 4, 8: lanes per orbit (0: the default)
};

// True once more than a.clock_budget cycles of the SM clock have passed since
// t_start (a clock64 reading on the same SM); never with a zero budget.
__device__ __forceinline__ bool budget_spent(const StepArgs& a, long long t_start)
{
    return a.clock_budget > 0 && clock64() - t_start > a.clock_budget;
}

// Threads per block of the one-orbit-per-thread RK4 kernels, and the slot of
// that size in per-size launch caches.
inline int small_threads(const StepArgs& a)
{
    return a.block > 0 ? a.block : kSmallBlock;
}
inline int block_slot(int threads)
{
    return threads <= 32 ? 0 : (threads <= 64 ? 1 : 2);
}

// Launchers (host side, one per kernel family).  Each returns the launch error.
cudaError_t launch_grid_ics(double E, double y0, double y1, int ny, double py0, double py1, int npy,
                            double* ics, int32_t* status, cudaStream_t st);
cudaError_t launch_fput_mode_ics(const SysPar& sp, int64_t n, const double* Qm, const double* Pm,
                                 const double* E, double* ics, cudaStream_t st);
cudaError_t launch_init(const SysPar& sp, int k, int vec_fp32, int renorm, uint64_t seed,
                        const double* ics, const int32_t* ic_status, const void* w_in,
                        const EnsPtrs& e, cudaStream_t st);
cudaError_t launch_integrate(const SysPar& sp, int k, int vec_fp32, bool ld, const StepArgs& a,
                             const EnsPtrs& e, const OrbitList* ol, cudaStream_t st);
cudaError_t launch_list_init(const EnsPtrs& e, int32_t* list, int32_t* count, cudaStream_t st);
// The integrate launch of the persistent work-queue mode (ol->queue set) runs
// a grid of persistent_blocks(); the caller zeroes *ol->queue first.
cudaError_t launch_shell_ics(const SysPar& sp, int64_t n, const double* dirs, const double* E,
                             double* ics, cudaStream_t st);
cudaError_t launch_indicators(const SysPar& sp, int k, int vec_fp32, double sali_threshold,
                              const EnsPtrs& e, double* sali, double* gali, int8_t* label,
                              cudaStream_t st);
// FP32 deviation vectors held as an orthonormal frame plus a triangular factor
cudaError_t launch_init_f32(const SysPar& sp, int k, uint64_t seed, const double* ics,
                            const int32_t* ic_status, const void* w_in, const EnsPtrs& e,
                            cudaStream_t st);
cudaError_t launch_integrate_f32(const SysPar& sp, int k, bool ld, const StepArgs& a,
                                 const EnsPtrs& e, const OrbitList* ol, cudaStream_t st);
cudaError_t launch_indicators_f32(const SysPar& sp, int k, double sali_threshold, const EnsPtrs& e,
                                  double* sali, double* gali, int8_t* label, cudaStream_t st);
cudaError_t launch_ld_stencil(int ny, int npy, const double* ld, const int32_t* status,
                              double* out, cudaStream_t st);
cudaError_t launch_lyap_small(const SysPar& sp, const StepArgs& a, int64_t n, const double* ics,
                              const int32_t* ic_status, double* lambda, int32_t* status,
                              cudaStream_t st);
cudaError_t launch_fput_lyap(const SysPar& sp, const StepArgs& a, int64_t n, const double* ics,
                             const int32_t* ic_status, double* lambda, int32_t* status,
                             cudaStream_t st);
cudaError_t prepare_fput_lyap(int n_dof);  // sets the shared-memory attribute once
// Short chains (N = 4, 8): several lanes of one warp per orbit (k_fput_lanes.cu).
bool fput_lyap_lanes_supported(int n_dof);
bool fput_lanes_per_orbit_supported(int n_dof, int lanes);  // 0 (the default) always
cudaError_t launch_fput_lyap_lanes(const SysPar& sp, const StepArgs& a, int64_t n, const double* ics,
                                   const int32_t* ic_status, double* lambda, int32_t* status,
                                   cudaStream_t st);
cudaError_t prepare_fput_lyap_lanes(int n_dof);

// Surrogate perceptron (k_mlp.cu).
size_t mlp_param_count();
cudaError_t launch_mlp_features(const double* series, int S, const double* ld, double t, const double* E,
                                int64_t n, float* X, cudaStream_t st);
cudaError_t launch_mlp_forward(const void* P, const float* X, int64_t n, float* Y, void* act,
                               cudaStream_t st);
cudaError_t launch_mlp_decide(const void* P, const double* series, int S, const double* ld, double t,
                              const double* E, int64_t n, double conf, int32_t* status, float* prob,
                              cudaStream_t st);
cudaError_t launch_mlp_loss_grad(const float* Y, const float* label, const float* target, int64_t n,
                                 float w_reg, float* dY, float* loss, cudaStream_t st);
cudaError_t launch_mlp_backward(const void* P, const float* X, const void* act, const float* dY,
                                int64_t n, float* delta, float* G, cudaStream_t st);
cudaError_t launch_mlp_adam(float* W, float* m, float* v, const float* g, float lr, float b1, float b2,
                            float eps, int step, void* Wb, cudaStream_t st);

// FPUT ensembles with k <= 6 FP64 deviation vectors (k_fput_ens.cu).
cudaError_t launch_fput_ens_init(const SysPar& sp, int k, int renorm, uint64_t seed, const double* ics,
                                 const int32_t* ic_status, const void* w_in, const EnsPtrs& e,
                                 cudaStream_t st);
cudaError_t launch_fput_ens(const SysPar& sp, int integrator, int k, const StepArgs& a, const EnsPtrs& e,
                            cudaStream_t st);
cudaError_t launch_fput_ens_indicators(const SysPar& sp, int k, double thr, const EnsPtrs& e, double* sali,
                                       double* gali, int8_t* label, cudaStream_t st);

// Pipe throughput probes (k_peaks.cu).
cudaError_t launch_peak_probe(int kind, int n_blocks, int n_threads, int64_t n_iter, double* sink,
                              cudaStream_t st);
double probe_ops_per_thread(int kind, int64_t n_iter);

// Which systems each kernel family supports.
bool small_model(int model);
bool fput_lyap_supported(int n_dof);
bool fput_ens_supported(int n_dof);

// Appends orbit o to ol.next when keep is set, one atomic per converged group of
// lanes.
__device__ __forceinline__ void list_append(const OrbitList& ol, bool keep, int32_t o)
{
    const unsigned act = __activemask();
    const unsigned ballot = __ballot_sync(act, keep);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(act) - 1;
    int base = 0;
    if (lane == leader && ballot) base = atomicAdd(ol.next_count, __popc(ballot));
    base = __shfl_sync(act, base, leader);
    if (keep) ol.next[base + __popc(ballot & ((1u << lane) - 1u))] = o;
}

inline unsigned blocks_for(int64_t n, int per_block)
{
    return (unsigned)((n + per_block - 1) / per_block);
}

// Next orbit index from a work-queue counter, one atomic per group of converged
// lanes.
__device__ __forceinline__ int64_t queue_next(unsigned long long* q)
{
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(act) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(q, (unsigned long long)__popc(act));
    base = __shfl_sync(act, base, leader);
    return (int64_t)(base + (unsigned long long)__popc(act & ((1u << lane) - 1u)));
}

// Work-queue loop of a persistent grid, shared by the one-orbit-per-thread
// kernels.  Every lane holds one orbit in a Run (load / step / store, with the
// step loop of a plain launch), and the warp steps in lockstep: a lane whose
// orbit ends stores it and takes the next orbit with work from the queue inside
// a short divergent branch, and the warp-wide vote at the top of every
// iteration brings the lanes back together, so they never drift into groups
// that execute the step separately.  Orbits without work (status not OK, or at
// their end step) are left as they are, as a plain launch leaves them
// unchanged.  Every lane of the warp must call this.
template <class Run, class StepArgs_, class SysPar_, class EnsPtrs_, class... Extra>
__device__ __forceinline__ void queue_worker(const StepArgs_& a, const SysPar_& sp, const EnsPtrs_& e,
                                             unsigned long long* queue, Extra&... extra)
{
    Run r;
    int64_t o = 0;
    auto fetch = [&]() -> bool {
        for (;;) {
            o = queue_next(queue);
            if (o >= e.n) return false;
            if (e.status[o] != CHS_ORBIT_OK) continue;
            r.load(o, a, e, extra...);
            if (r.todo > 0) return true;
        }
    };
    bool have = fetch();
    while (__any_sync(0xffffffffu, have)) {
        if (have) {
            const bool running = r.step(a, sp, extra...);
            if (!running || r.s >= r.todo) {
                r.store(o, e, extra...);
                have = fetch();
            }
        }
    }
}

// The current device, clamped into [0, kCacheDevices) for per-device launch caches.
constexpr int kCacheDevices = 64;
inline int cache_device()
{
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kCacheDevices) d = 0;
    return d;
}

// Blocks of a persistent launch: every SM filled to the kernel's occupancy.
template <class Kernel>
inline cudaError_t persistent_blocks(Kernel kernel, int threads, size_t smem, unsigned* blocks)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    *blocks = (unsigned)(sms * (per_sm > 0 ? per_sm : 1));
    return cudaSuccess;
}

}  // namespace chs

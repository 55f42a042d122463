// k_dop853_fixed.cuh -- the fixed-step DOP853 integrate kernel of the
// one-orbit-per-thread systems and its launcher, shared by the translation
// units that instantiate it for different systems (k_dop853.cu, k_dop853_q3.cu).
#pragma once

#include "dop853.cuh"

namespace chs {
namespace {

using dp::kBlock;

// The state of one orbit during a call: loaded, advanced by fixed DOP853
// steps with the checks of the chs_integrate_batch contract, stored back.
template <class Sys, int K, bool LD>
struct DpRun {
    static constexpr int N = Sys::N, D = 2 * N, KK = K > 0 ? K : 1;
    double x[D], w[KK][D];
    double L, h0, dhm;
    int64_t exec0, todo, s, until;
    long long t_start;  // clock64 when the orbit was taken up (clock budget)
    int32_t st;

    __device__ __forceinline__ void load(const int64_t o, const StepArgs& a, const EnsPtrs& e,
                                         const dp::Slab<Sys>&)
    {
        const int64_t n = e.n;
        const double* wg = static_cast<const double*>(e.w);
#pragma unroll
        for (int c = 0; c < D; ++c) x[c] = e.x[c * n + o];
#pragma unroll
        for (int j = 0; j < K; ++j)
#pragma unroll
            for (int c = 0; c < D; ++c) w[j][c] = wg[(j * D + c) * n + o];
        L = LD ? e.ld[o] : 0.0;
        h0 = e.h0[o];
        dhm = e.dh_max[o];
        exec0 = e.n_exec[o];
        todo = a.n_steps;
        if (e.t_end) todo = min(todo, max(e.t_end[o] - exec0, (int64_t)0));
        st = CHS_ORBIT_OK;
        until = a.sample_every > 0 ? a.sample_every - (a.step0 % a.sample_every) : -1;
        s = 0;
        t_start = clock64();
    }

    // One step and its checks; false once the orbit froze (st says why).
    __device__ __forceinline__ bool step(const StepArgs& a, const SysPar& sp, const dp::Slab<Sys>& sl)
    {
        ++s;
        double xn[D], dL = 0.0;
        dp::orbit_step<Sys, LD, false>(sl, x, a.dt, a.ld_sqrt, a.ld_p, sp, xn, dL, nullptr, nullptr);
#pragma unroll
        for (int j = 0; j < K; ++j) dp::vector_step<Sys>(sl, w[j], a.dt);
#pragma unroll
        for (int c = 0; c < D; ++c) x[c] = xn[c];
        if (LD) L += dL;
        bool check = false;
        if (--until == 0) {
            until = a.sample_every;
            check = true;
        }
        st = dp::post_step<Sys, K>(x, w, L, a, sp, check, h0, dhm);
        if (check && st == CHS_ORBIT_OK && budget_spent(a, t_start)) st = CHS_ORBIT_STEP_BUDGET;
        return st == CHS_ORBIT_OK;
    }

    // Writes the orbit back; true when it is still running.
    __device__ __forceinline__ bool store(const int64_t o, const EnsPtrs& e, const dp::Slab<Sys>&) const
    {
        const int64_t n = e.n;
        double* wg = static_cast<double*>(e.w);
#pragma unroll
        for (int c = 0; c < D; ++c) e.x[c * n + o] = x[c];
#pragma unroll
        for (int j = 0; j < K; ++j)
#pragma unroll
            for (int c = 0; c < D; ++c) wg[(j * D + c) * n + o] = w[j][c];
        if (LD) e.ld[o] = L;
        e.dh_max[o] = dhm;
        e.n_exec[o] = exec0 + s;
        e.status[o] = st;
        return st == CHS_ORBIT_OK && (!e.t_end || exec0 + s < e.t_end[o]);
    }
};

// Advances orbit o (status OK) by the call's steps; returns true when it is
// still running afterwards.
template <class Sys, int K, bool LD>
__device__ __forceinline__ bool integrate_orbit_dp(const int64_t o, const StepArgs& a,
                                                   const SysPar& sp, const EnsPtrs& e,
                                                   const dp::Slab<Sys>& sl)
{
    DpRun<Sys, K, LD> r;
    r.load(o, a, e, sl);
    while (r.s < r.todo)
        if (!r.step(a, sp, sl)) break;
    return r.store(o, e, sl);
}

// One orbit per thread, with the orbit-selection modes of k_integrate
// (k_small.cu) chosen at run time from ol.
template <class Sys, int K, bool LD>
__global__ void __launch_bounds__(kBlock)
k_integrate_dp(const StepArgs a, const SysPar sp, const EnsPtrs e, const OrbitList ol)
{
    const dp::Slab<Sys> sl = dp::my_slab<Sys>();
    const int mode = integ_mode(ol);
    if (mode == kModeQueue) {
        queue_worker<DpRun<Sys, K, LD>>(a, sp, e, ol.queue, sl);
        return;
    }
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t o = t;
    if (mode == kModeList) {
        if (t >= *ol.count) return;
        o = ol.list[t];
    }
    if (o >= e.n) return;
    if (e.status[o] != CHS_ORBIT_OK) return;
    const bool keep = integrate_orbit_dp<Sys, K, LD>(o, a, sp, e, sl);
    if (mode == kModeList) list_append(ol, keep, (int32_t)o);
}

template <class Sys>
cudaError_t fixed_sys(int k, bool ld, const StepArgs& a, const SysPar& sp, const EnsPtrs& e,
                      const OrbitList* ol, cudaStream_t st)
{
    const unsigned g = blocks_for(e.n, kBlock);
    const OrbitList l = ol ? *ol : OrbitList{};
    constexpr size_t sm = dp::slab_bytes<Sys>();
    return dp::with_k<Sys>(k, [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        auto kern = ld ? k_integrate_dp<Sys, K, true> : k_integrate_dp<Sys, K, false>;
        unsigned grid = g;
        if (l.queue) {
            static unsigned pg[kCacheDevices][2] = {};  // persistent grid per device and LD variant
            unsigned& p = pg[cache_device()][ld ? 1 : 0];
            if (!p && persistent_blocks(kern, kBlock, sm, &p) != cudaSuccess) p = 0;
            if (p) grid = p;
        }
        kern<<<grid, kBlock, sm, st>>>(a, sp, e, l);
    });
}

}  // namespace
}  // namespace chs

// k_dop853.cu -- the paper's own 8th-order solver in fixed-step use (DOP 8,
// Sec. Functionalities) on the one-orbit-per-thread systems: the joint system
// (orbit, deviation vectors, LD) with the per-step checks of the RK4 path, over
// the whole ensemble or a compacted orbit list; and the Lyapunov spectrum of
// the 2-DOF systems.  Building blocks and design notes: dop853.cuh.
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

// Lyapunov spectrum of the 2-DOF systems: W (4 x 4) in registers.
template <class Sys>
__global__ void __launch_bounds__(kBlock)
k_lyap_small_dp(const StepArgs a, const SysPar sp, const int64_t n, const double* __restrict__ ics,
                const int32_t* __restrict__ ic_status, double* __restrict__ lambda,
                int32_t* __restrict__ status_out)
{
    constexpr int D = 2 * Sys::N;
    const dp::Slab<Sys> sl = dp::my_slab<Sys>();
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const double qnan = __longlong_as_double(0x7ff8000000000000LL);
    int32_t st = ic_status ? ic_status[o] : CHS_ORBIT_OK;
    double x[D], W[D][D], S[D];
    bool fin = true;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        x[c] = ics[c * n + o];
        fin = fin && isfinite(x[c]);
        S[c] = 0.0;
#pragma unroll
        for (int j = 0; j < D; ++j) W[j][c] = (j == c) ? 1.0 : 0.0;
    }
    if (st == CHS_ORBIT_OK && !fin) st = CHS_ORBIT_NONFINITE;
    if (st == CHS_ORBIT_OK) {
        int64_t until_qr = a.qr_every;
        int64_t until = a.sample_every > 0 ? a.sample_every : -1;
        for (int64_t s = 1; s <= a.n_steps; ++s) {
            double xn[D], dL = 0.0;
            dp::orbit_step<Sys, false, false>(sl, x, a.dt, 0, 0.0, sp, xn, dL, nullptr, nullptr);
#pragma unroll
            for (int j = 0; j < D; ++j) dp::vector_step<Sys>(sl, W[j], a.dt);
#pragma unroll
            for (int c = 0; c < D; ++c) x[c] = xn[c];
            if (--until_qr == 0 || s == a.n_steps) {
                until_qr = a.qr_every;
                // modified Gram-Schmidt, R_jj > 0: S_j += ln R_jj, W <- Q
#pragma unroll
                for (int j = 0; j < D; ++j) {
#pragma unroll
                    for (int i = 0; i < j; ++i) {
                        double r = 0.0;
#pragma unroll
                        for (int c = 0; c < D; ++c) r = fma(W[i][c], W[j][c], r);
#pragma unroll
                        for (int c = 0; c < D; ++c) W[j][c] = fma(-r, W[i][c], W[j][c]);
                    }
                    double n2 = 0.0;
#pragma unroll
                    for (int c = 0; c < D; ++c) n2 = fma(W[j][c], W[j][c], n2);
                    S[j] += 0.5 * log(n2);
                    const double inv = rsqrt_nr(n2);
#pragma unroll
                    for (int c = 0; c < D; ++c) W[j][c] *= inv;
                }
            }
            if (--until == 0) {
                until = a.sample_every;
                bool f2 = true;
#pragma unroll
                for (int c = 0; c < D; ++c) f2 = f2 && isfinite(x[c]) && isfinite(S[c]);
                if (!f2) {
                    st = CHS_ORBIT_NONFINITE;
                    break;
                }
            }
        }
    }
    const double T = (double)a.n_steps * a.dt;
#pragma unroll
    for (int c = 0; c < D; ++c) lambda[c * n + o] = (st == CHS_ORBIT_OK) ? S[c] / T : qnan;
    status_out[o] = st;
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

cudaError_t launch_integrate_dp(const SysPar& sp, int k, bool ld, const StepArgs& a,
                                const EnsPtrs& e, const OrbitList* ol, cudaStream_t st)
{
    if (e.n == 0 || a.n_steps == 0) return cudaSuccess;
    switch (sp.model) {
    case CHS_HENON_HEILES: return fixed_sys<SysHenonHeiles>(k, ld, a, sp, e, ol, st);
    case CHS_HARMONIC: return fixed_sys<SysHarmonic>(k, ld, a, sp, e, ol, st);
    case CHS_INVERTED: return fixed_sys<SysInverted>(k, ld, a, sp, e, ol, st);
    case CHS_QUARTIC3: return fixed_sys<SysQuartic3>(k, ld, a, sp, e, ol, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_lyap_small_dp(const SysPar& sp, const StepArgs& a, int64_t n, const double* ics,
                                 const int32_t* ic_status, double* lambda, int32_t* status,
                                 cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const unsigned g = blocks_for(n, kBlock);
    switch (sp.model) {
    case CHS_HENON_HEILES:
        k_lyap_small_dp<SysHenonHeiles><<<g, kBlock, dp::slab_bytes<SysHenonHeiles>(), st>>>(
            a, sp, n, ics, ic_status, lambda, status);
        break;
    case CHS_HARMONIC:
        k_lyap_small_dp<SysHarmonic><<<g, kBlock, dp::slab_bytes<SysHarmonic>(), st>>>(
            a, sp, n, ics, ic_status, lambda, status);
        break;
    case CHS_INVERTED:
        k_lyap_small_dp<SysInverted><<<g, kBlock, dp::slab_bytes<SysInverted>(), st>>>(
            a, sp, n, ics, ic_status, lambda, status);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace chs

// k_frame32.cu -- FP32 deviation vectors with an FP64 orbit (one orbit per thread).
//
// FP32 vectors renormalised one by one cannot resolve small SALI or GALI
// values: every step injects rounding of relative size eps32 ~ 6e-8 into each
// vector while the flow aligns them only by a factor exp(-(l1 - l2) h) per
// step, so the computed angle between two vectors stalls near
// eps32 / ((l1 - l2) h) ~ 1e-4 for chaotic Henon-Heiles orbits at h = 0.01.
//
// This mode therefore stores the k vectors as W = Q R D: an orthonormal frame
// Q (d x k, FP32) and an upper-triangular R with unit columns (FP32), D an
// irrelevant positive diagonal.  Each step applies the exact one-step RK4
// propagator Phi to Q, re-orthonormalises it by modified Gram-Schmidt,
// Phi Q = Q' S, and updates R <- colnorm(S R).  Every diagonal entry of R only
// ever gets multiplied by S_jj and divided by a column norm, so it keeps its
// relative precision however small it becomes:
//   GALI_m = prod_{j < m} R_jj,   SALI = R_11 sqrt(2 / (1 + |R_01|)),
// which are the GALI and SALI of the unit vectors w_j / |w_j| (the re-
// orthonormalisation of every step is the per-step renormalisation).  The
// orbit and its energy check stay in FP64; the LD is accumulated in FP64 from
// an integrand summed in FP32 (correctly rounded FP32 square roots of |f_i|
// rounded to FP32), which takes the LD's square roots off the FP64 pipe at a
// relative cost of about 1e-7 per term, averaging out along the orbit.
//
// Ensemble vector buffer in this mode: FP32, [k*d + k(k+1)/2][n]: rows j*d + c
// hold Q (vector j, component c), rows k*d + j(j+1)/2 + i hold R_ij (i <= j).
#include <math.h>

#include "rk4_common.cuh"
#include "seed.cuh"

namespace chs {

__host__ __device__ constexpr int tri(int i, int j) { return j * (j + 1) / 2 + i; }

template <class Sys, int K>
__global__ void __launch_bounds__(kSmallBlock)
k_init_f32(const SysPar sp, const uint64_t seed, const double* __restrict__ ics,
           const int32_t* __restrict__ ic_status, const float* __restrict__ w_in, const EnsPtrs e)
{
    constexpr int D = 2 * Sys::N;
    const int64_t n = e.n;
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    double x[D];
    bool finite = true;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        x[c] = ics[c * n + o];
        e.x[c * n + o] = x[c];
        finite = finite && isfinite(x[c]);
    }
    int32_t st = ic_status ? ic_status[o] : CHS_ORBIT_OK;
    if (st == CHS_ORBIT_OK && !finite) st = CHS_ORBIT_NONFINITE;
    e.status[o] = st;
    e.h0[o] = (st == CHS_ORBIT_OK) ? Sys::energy(x, sp) : __longlong_as_double(0x7ff8000000000000LL);
    e.dh_max[o] = 0.0;
    e.n_exec[o] = 0;
    if (e.ld) e.ld[o] = 0.0;
    // unit vectors (FP64), then Q R by modified Gram-Schmidt
    double V[K][D];
#pragma unroll
    for (int j = 0; j < K; ++j) {
#pragma unroll
        for (int c = 0; c < D; ++c) {
            if (w_in) {
                V[j][c] = (double)w_in[(j * D + c) * n + o];
            } else {
                V[j][c] = seed_uniform(seed, ((uint64_t)o * K + j) * D + c + 1);
            }
        }
        double acc = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) acc = __dadd_rn(acc, __dmul_rn(V[j][c], V[j][c]));
        const double nr = __dsqrt_rn(acc);
#pragma unroll
        for (int c = 0; c < D; ++c) V[j][c] = __ddiv_rn(V[j][c], nr);
    }
    double R[K * (K + 1) / 2];
#pragma unroll
    for (int j = 0; j < K; ++j) {
#pragma unroll
        for (int i = 0; i < j; ++i) {
            double r = 0.0;
#pragma unroll
            for (int c = 0; c < D; ++c) r = fma(V[i][c], V[j][c], r);
#pragma unroll
            for (int c = 0; c < D; ++c) V[j][c] = fma(-r, V[i][c], V[j][c]);
            R[tri(i, j)] = r;
        }
        double n2 = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) n2 = fma(V[j][c], V[j][c], n2);
        const double rjj = sqrt(n2);
        R[tri(j, j)] = rjj;
#pragma unroll
        for (int c = 0; c < D; ++c) V[j][c] /= rjj;
    }
    float* wg = static_cast<float*>(e.w);
#pragma unroll
    for (int j = 0; j < K; ++j)
#pragma unroll
        for (int c = 0; c < D; ++c) wg[(j * D + c) * n + o] = (float)V[j][c];
#pragma unroll
    for (int p = 0; p < K * (K + 1) / 2; ++p) wg[(K * D + p) * n + o] = (float)R[p];
}

// Hess V of each system (as in systems.cuh) in FP32 from the FP32-rounded stage
// positions: the frame is propagated in FP32 anyway, so forming the Hessian in
// FP64 and rounding it would spend FP64 instructions for the same FP32 accuracy.
template <class Sys>
struct Hess32;

template <>
struct Hess32<SysHenonHeiles> {
    __device__ __forceinline__ static void eval(const float* q, float* H, const SysPar&)
    {
        H[0] = fmaf(2.0f, q[1], 1.0f);
        H[1] = 2.0f * q[0];
        H[2] = fmaf(-2.0f, q[1], 1.0f);
    }
};

template <>
struct Hess32<SysHarmonic> {
    __device__ __forceinline__ static void eval(const float*, float* H, const SysPar&)
    {
        H[0] = 1.0f;
        H[1] = 0.0f;
        H[2] = 1.0f;
    }
};

template <>
struct Hess32<SysInverted> {
    __device__ __forceinline__ static void eval(const float*, float* H, const SysPar&)
    {
        H[0] = -1.0f;
        H[1] = 0.0f;
        H[2] = 1.0f;
    }
};

template <>
struct Hess32<SysQuartic3> {
    __device__ __forceinline__ static void eval(const float* q, float* H, const SysPar& sp)
    {
        const float e2 = (float)(2.0 * sp.eps), e4 = (float)(4.0 * sp.eps);
        const float s0 = q[0] * q[0], s1 = q[1] * q[1], s2 = q[2] * q[2];
        H[hidx<3>(0, 0)] = fmaf(e2, s1 + s2, 1.0f);
        H[hidx<3>(1, 1)] = fmaf(e2, s0 + s2, 1.0f);
        H[hidx<3>(2, 2)] = fmaf(e2, s0 + s1, 1.0f);
        H[hidx<3>(0, 1)] = e4 * q[0] * q[1];
        H[hidx<3>(0, 2)] = e4 * q[0] * q[2];
        H[hidx<3>(1, 2)] = e4 * q[1] * q[2];
    }
};

// The state of one orbit during a call (FP64 orbit and LD, FP32 frame Q and
// triangle R): loaded, advanced step by step with the checks of the
// chs_integrate_batch contract, stored back.
template <class Sys, int K, bool LD>
struct FrameRun {
    static constexpr int N = Sys::N, D = 2 * N, NH = Sys::NH, NR = K * (K + 1) / 2;
    double x[D];
    float Q[K][D], R[NR];
    double L, h0, dhm;
    int64_t exec0, todo, s, until;
    long long t_start;  // clock64 when the orbit was taken up (clock budget)
    int32_t st;

    __device__ __forceinline__ void load(const int64_t o, const StepArgs& a, const EnsPtrs& e)
    {
        const int64_t n = e.n;
        const float* wg = static_cast<const float*>(e.w);
#pragma unroll
        for (int c = 0; c < D; ++c) x[c] = e.x[c * n + o];
#pragma unroll
        for (int j = 0; j < K; ++j)
#pragma unroll
            for (int c = 0; c < D; ++c) Q[j][c] = wg[(j * D + c) * n + o];
#pragma unroll
        for (int p = 0; p < NR; ++p) R[p] = wg[(K * D + p) * n + o];
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
    __device__ __forceinline__ bool step(const StepArgs& a, const SysPar& sp)
    {
        ++s;
        float qf[4][N], Hf[4][NH];
        rk4_state_positions<Sys, LD, true>(x, L, a.dt, a.ld_sqrt, a.ld_p, sp, qf);
#pragma unroll
        for (int q = 0; q < 4; ++q) Hess32<Sys>::eval(qf[q], Hf[q], sp);
        PhiBlocks<N, float> P;
        phi_build<N, NH, float>(Hf, a.dt, P);
#pragma unroll
        for (int j = 0; j < K; ++j) phi_apply<N, float>(P, Q[j]);
        // Phi Q = Q' S (modified Gram-Schmidt), then R <- colnorm(S R)
        float S[NR];
#pragma unroll
        for (int j = 0; j < K; ++j) {
#pragma unroll
            for (int i = 0; i < j; ++i) {
                float r = Q[i][0] * Q[j][0];
#pragma unroll
                for (int c = 1; c < D; ++c) r = fmaf(Q[i][c], Q[j][c], r);
#pragma unroll
                for (int c = 0; c < D; ++c) Q[j][c] = fmaf(-r, Q[i][c], Q[j][c]);
                S[tri(i, j)] = r;
            }
            float n2 = Q[j][0] * Q[j][0];
#pragma unroll
            for (int c = 1; c < D; ++c) n2 = fmaf(Q[j][c], Q[j][c], n2);
            const float inv = rsqrtf(n2);
            S[tri(j, j)] = n2 * inv;
#pragma unroll
            for (int c = 0; c < D; ++c) Q[j][c] *= inv;
        }
#pragma unroll
        for (int j = K - 1; j >= 0; --j) {
            float col[K];
            float nn = 0.0f;
#pragma unroll
            for (int i = 0; i <= j; ++i) {
                float t = 0.0f;
#pragma unroll
                for (int m = i; m <= j; ++m) t = fmaf(S[tri(i, m)], R[tri(m, j)], t);
                col[i] = t;
                nn = fmaf(t, t, nn);
            }
            const float inv = rsqrtf(nn);
#pragma unroll
            for (int i = 0; i <= j; ++i) R[tri(i, j)] = col[i] * inv;
        }
        if (a.escape_r2 > 0.0) {
            double r2 = x[0] * x[0];
#pragma unroll
            for (int i = 1; i < N; ++i) r2 = fma(x[i], x[i], r2);
            if (r2 > a.escape_r2) {
                st = CHS_ORBIT_ESCAPED;
                return false;
            }
        }
        if (--until == 0) {
            until = a.sample_every;
            bool fin = isfinite(L);
#pragma unroll
            for (int c = 0; c < D; ++c) fin = fin && isfinite(x[c]);
#pragma unroll
            for (int j = 0; j < K; ++j)
#pragma unroll
                for (int c = 0; c < D; ++c) fin = fin && isfinite(Q[j][c]);
            if (!fin) {
                st = CHS_ORBIT_NONFINITE;
                return false;
            }
            const double dH = fabs(Sys::energy(x, sp) - h0);
            dhm = fmax(dhm, dH);
            if (a.dh_limit > 0.0 && dH > a.dh_limit) {
                st = CHS_ORBIT_ENERGY_DRIFT;
                return false;
            }
            if constexpr (K >= 2) {
                const double sv = fabs((double)R[tri(1, 1)]) *
                                  sqrt(2.0 / (1.0 + fmin(fabs((double)R[tri(0, 1)]), 1.0)));
                if (a.early_exit && sv < a.sali_threshold) {
                    st = CHS_ORBIT_EARLY_CHAOTIC;
                    return false;
                }
            }
            if (budget_spent(a, t_start)) {
                st = CHS_ORBIT_STEP_BUDGET;
                return false;
            }
        }
        return true;
    }

    // Writes the orbit back; true when it is still running.
    __device__ __forceinline__ bool store(const int64_t o, const EnsPtrs& e) const
    {
        const int64_t n = e.n;
        float* wg = static_cast<float*>(e.w);
#pragma unroll
        for (int c = 0; c < D; ++c) e.x[c * n + o] = x[c];
#pragma unroll
        for (int j = 0; j < K; ++j)
#pragma unroll
            for (int c = 0; c < D; ++c) wg[(j * D + c) * n + o] = Q[j][c];
#pragma unroll
        for (int p = 0; p < NR; ++p) wg[(K * D + p) * n + o] = R[p];
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
__device__ __forceinline__ bool integrate_orbit_f32(const int64_t o, const StepArgs& a,
                                                    const SysPar& sp, const EnsPtrs& e)
{
    FrameRun<Sys, K, LD> r;
    r.load(o, a, e);
    while (r.s < r.todo)
        if (!r.step(a, sp)) break;
    return r.store(o, e);
}

// One thread per orbit; the orbit-selection modes of k_integrate (k_small.cu).
template <class Sys, int K, bool LD, int MODE>
__global__ void __launch_bounds__(kSmallBlock)
k_integrate_f32(const StepArgs a, const SysPar sp, const EnsPtrs e, const OrbitList ol)
{
    if constexpr (MODE == kModeQueue) {
        queue_worker<FrameRun<Sys, K, LD>>(a, sp, e, ol.queue);
    } else {
        const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        int64_t o = t;
        if (MODE == kModeList) {
            if (t >= *ol.count) return;
            o = ol.list[t];
        }
        if (o >= e.n) return;
        if (e.status[o] != CHS_ORBIT_OK) return;
        const bool keep = integrate_orbit_f32<Sys, K, LD>(o, a, sp, e);
        if (MODE == kModeList) list_append(ol, keep, (int32_t)o);
    }
}

// SALI, GALI_m and labels from the triangular factor (see the file comment).
template <int D, int K>
__global__ void __launch_bounds__(kSmallBlock)
k_indicators_f32(const int64_t n, const float* __restrict__ wg, const int32_t* __restrict__ status,
                 const double thr, double* __restrict__ sali, double* __restrict__ gali,
                 int8_t* __restrict__ label)
{
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const int32_t st = status[o];
    const double qnan = __longlong_as_double(0x7ff8000000000000LL);
    const bool forb = st == CHS_ORBIT_FORBIDDEN;
    double sv = qnan;
    if (K >= 2 && !forb) {
        const double a01 = fabs((double)wg[(K * D + tri(0, 1 % K)) * n + o]);
        const double b11 = fabs((double)wg[(K * D + tri(1 % K, 1 % K)) * n + o]);
        sv = b11 * sqrt(2.0 / (1.0 + fmin(a01, 1.0)));
    }
    if (sali) sali[o] = sv;
    if (gali) {
        double prod = 1.0;
#pragma unroll
        for (int j = 1; j < K; ++j) {
            prod *= fabs((double)wg[(K * D + tri(j, j)) * n + o]);
            gali[(int64_t)(j - 1) * n + o] = forb ? qnan : prod;
        }
    }
    if (label) {
        int8_t lb;
        if (st == CHS_ORBIT_OK)
            lb = (sv < thr) ? 1 : 0;
        else if (st == CHS_ORBIT_EARLY_CHAOTIC)
            lb = 1;
        else if (st == CHS_ORBIT_PREDICTED_REGULAR)
            lb = 0;
        else if (st == CHS_ORBIT_ESCAPED)
            lb = 2;
        else
            lb = -1;
        label[o] = lb;
    }
}

// --------------------------------------------------------------------------
// dispatch
// --------------------------------------------------------------------------

template <class Sys, int K>
static void init_one(const unsigned g, const SysPar& sp, uint64_t seed, const double* ics,
                     const int32_t* ics_st, const float* wi, const EnsPtrs& e, cudaStream_t st)
{
    k_init_f32<Sys, K><<<g, kSmallBlock, 0, st>>>(sp, seed, ics, ics_st, wi, e);
}

template <class Sys>
static cudaError_t init_sys(int k, const SysPar& sp, uint64_t seed, const double* ics,
                            const int32_t* ics_st, const void* w_in, const EnsPtrs& e, cudaStream_t st)
{
    const unsigned g = blocks_for(e.n, kSmallBlock);
    const float* wi = static_cast<const float*>(w_in);
    switch (k) {
    case 1: init_one<Sys, 1>(g, sp, seed, ics, ics_st, wi, e, st); break;
    case 2: init_one<Sys, 2>(g, sp, seed, ics, ics_st, wi, e, st); break;
    case 3: init_one<Sys, 3>(g, sp, seed, ics, ics_st, wi, e, st); break;
    case 4: init_one<Sys, 4>(g, sp, seed, ics, ics_st, wi, e, st); break;
    case 5:
        if constexpr (Sys::N >= 3) {
            init_one<Sys, 5>(g, sp, seed, ics, ics_st, wi, e, st);
            break;
        }
        return cudaErrorInvalidValue;
    case 6:
        if constexpr (Sys::N >= 3) {
            init_one<Sys, 6>(g, sp, seed, ics, ics_st, wi, e, st);
            break;
        }
        return cudaErrorInvalidValue;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_init_f32(const SysPar& sp, int k, uint64_t seed, const double* ics,
                            const int32_t* ic_status, const void* w_in, const EnsPtrs& e,
                            cudaStream_t st)
{
    if (e.n == 0) return cudaSuccess;
    switch (sp.model) {
    case CHS_HENON_HEILES: return init_sys<SysHenonHeiles>(k, sp, seed, ics, ic_status, w_in, e, st);
    case CHS_HARMONIC: return init_sys<SysHarmonic>(k, sp, seed, ics, ic_status, w_in, e, st);
    case CHS_INVERTED: return init_sys<SysInverted>(k, sp, seed, ics, ic_status, w_in, e, st);
    case CHS_QUARTIC3: return init_sys<SysQuartic3>(k, sp, seed, ics, ic_status, w_in, e, st);
    }
    return cudaErrorInvalidValue;
}

template <class Sys, int K, bool LD>
static void integ_one(const unsigned g, const StepArgs& a, const SysPar& sp, const EnsPtrs& e,
                      const OrbitList* ol, cudaStream_t st)
{
    const int tb = small_threads(a);
    if (ol && ol->queue) {
        // blocks of the persistent grid, per device and block size
        static unsigned pgs[kCacheDevices][3] = {};
        unsigned& pg = pgs[cache_device()][block_slot(tb)];
        if (!pg && persistent_blocks(k_integrate_f32<Sys, K, LD, kModeQueue>, tb, 0, &pg) != cudaSuccess)
            pg = 0;
        k_integrate_f32<Sys, K, LD, kModeQueue><<<pg ? pg : g, tb, 0, st>>>(a, sp, e, *ol);
    } else if (ol) {
        k_integrate_f32<Sys, K, LD, kModeList><<<g, tb, 0, st>>>(a, sp, e, *ol);
    } else {
        k_integrate_f32<Sys, K, LD, kModeAll><<<g, tb, 0, st>>>(a, sp, e, OrbitList{});
    }
}

template <class Sys, bool LD>
static cudaError_t integ_sys(int k, const StepArgs& a, const SysPar& sp, const EnsPtrs& e,
                             const OrbitList* ol, cudaStream_t st)
{
    const unsigned g = blocks_for(e.n, small_threads(a));
    switch (k) {
    case 1: integ_one<Sys, 1, LD>(g, a, sp, e, ol, st); break;
    case 2: integ_one<Sys, 2, LD>(g, a, sp, e, ol, st); break;
    case 3: integ_one<Sys, 3, LD>(g, a, sp, e, ol, st); break;
    case 4: integ_one<Sys, 4, LD>(g, a, sp, e, ol, st); break;
    case 5:
        if constexpr (Sys::N >= 3) {
            integ_one<Sys, 5, LD>(g, a, sp, e, ol, st);
            break;
        }
        return cudaErrorInvalidValue;
    case 6:
        if constexpr (Sys::N >= 3) {
            integ_one<Sys, 6, LD>(g, a, sp, e, ol, st);
            break;
        }
        return cudaErrorInvalidValue;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_integrate_f32(const SysPar& sp, int k, bool ld, const StepArgs& a,
                                 const EnsPtrs& e, const OrbitList* ol, cudaStream_t st)
{
    if (e.n == 0 || a.n_steps == 0) return cudaSuccess;
    switch (sp.model) {
    case CHS_HENON_HEILES:
        return ld ? integ_sys<SysHenonHeiles, true>(k, a, sp, e, ol, st)
                  : integ_sys<SysHenonHeiles, false>(k, a, sp, e, ol, st);
    case CHS_HARMONIC:
        return ld ? integ_sys<SysHarmonic, true>(k, a, sp, e, ol, st)
                  : integ_sys<SysHarmonic, false>(k, a, sp, e, ol, st);
    case CHS_INVERTED:
        return ld ? integ_sys<SysInverted, true>(k, a, sp, e, ol, st)
                  : integ_sys<SysInverted, false>(k, a, sp, e, ol, st);
    case CHS_QUARTIC3:
        return ld ? integ_sys<SysQuartic3, true>(k, a, sp, e, ol, st)
                  : integ_sys<SysQuartic3, false>(k, a, sp, e, ol, st);
    }
    return cudaErrorInvalidValue;
}

template <int D>
static cudaError_t ind_f32(int k, double thr, const EnsPtrs& e, double* sali, double* gali,
                           int8_t* label, cudaStream_t st)
{
    const unsigned g = blocks_for(e.n, kSmallBlock);
    const float* w = static_cast<const float*>(e.w);
    switch (k) {
#define CHS_CASE(KV)                                                                                \
    case KV:                                                                                        \
        k_indicators_f32<D, KV><<<g, kSmallBlock, 0, st>>>(e.n, w, e.status, thr, sali, gali, label); \
        break;
        CHS_CASE(1) CHS_CASE(2) CHS_CASE(3) CHS_CASE(4) CHS_CASE(5) CHS_CASE(6)
#undef CHS_CASE
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_indicators_f32(const SysPar& sp, int k, double sali_threshold, const EnsPtrs& e,
                                  double* sali, double* gali, int8_t* label, cudaStream_t st)
{
    if (e.n == 0) return cudaSuccess;
    const int D = 2 * sp.n_dof;
    if (D == 4) return ind_f32<4>(k, sali_threshold, e, sali, gali, label, st);
    if (D == 6) return ind_f32<6>(k, sali_threshold, e, sali, gali, label, st);
    return cudaErrorInvalidValue;
}

}  // namespace chs

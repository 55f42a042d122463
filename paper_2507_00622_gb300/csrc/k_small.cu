// k_small.cu -- one orbit per thread: ensemble set-up, RK4 integration of the
// orbit with its deviation vectors and LD, indicators, and the Lyapunov
// spectrum of the 2-DOF systems.
//
// Design: the whole joint state (x, w_1..w_k, M_p) of an orbit lives in
// registers for the entire call; the only global traffic is one coalesced SoA
// load and one store per component per call, so the kernels are bound by the
// FP64 pipe (GB300: 2 DFMA/clk/SM), not by HBM.
#include <math.h>

#include <type_traits>

#include "rk4_common.cuh"
#include "seed.cuh"

namespace chs {

// --------------------------------------------------------------------------
// Ensemble set-up
// --------------------------------------------------------------------------

template <class Sys, int K, typename VT>
__global__ void __launch_bounds__(kSmallBlock)
k_init(const SysPar sp, const int renorm, const uint64_t seed, const double* __restrict__ ics,
       const int32_t* __restrict__ ic_status, const VT* __restrict__ w_in, const EnsPtrs e)
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
    VT* wg = static_cast<VT*>(e.w);
#pragma unroll
    for (int j = 0; j < K; ++j) {
        double v[D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            if (w_in) {
                v[c] = (double)w_in[(j * D + c) * n + o];
            } else {
                v[c] = seed_uniform(seed, ((uint64_t)o * K + j) * D + c + 1);
            }
        }
        // seeded vectors are normalised, and every vector once more with renorm;
        // sums of squares in index order, no contraction: the same rounding as a
        // plain sequential loop
        for (int pass = w_in ? 1 : 0; pass < 1 + renorm; ++pass) {
            double acc = 0.0;
#pragma unroll
            for (int c = 0; c < D; ++c) acc = __dadd_rn(acc, __dmul_rn(v[c], v[c]));
            const double nr = __dsqrt_rn(acc);
#pragma unroll
            for (int c = 0; c < D; ++c) v[c] = __ddiv_rn(v[c], nr);
        }
#pragma unroll
        for (int c = 0; c < D; ++c) wg[(j * D + c) * n + o] = (VT)v[c];
    }
}

// --------------------------------------------------------------------------
// RK4 on the joint system
// --------------------------------------------------------------------------

// dw = J(x) w for w = (dq, dp): d(dq) = dp, d(dp) = -Hess V dq.
template <int N, int NH, typename VT>
__device__ __forceinline__ void var_rhs(const VT* Hc, const VT* w, VT* dw)
{
#pragma unroll
    for (int i = 0; i < N; ++i) dw[i] = w[N + i];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        VT acc = Hc[hidx<N>(i, 0)] * w[0];
#pragma unroll
        for (int m = 1; m < N; ++m) acc = fma(Hc[hidx<N>(i, m)], w[m], acc);
        dw[N + i] = -acc;
    }
}

// One classic RK4 step of (x, w_1..w_K, L):
//   k1 = F(z), k2 = F(z + h/2 k1), k3 = F(z + h/2 k2), k4 = F(z + h k3),
//   z <- z + h/6 (k1 + 2 k2 + 2 k3 + k4),
// with each stage's Jacobian evaluated at that stage's state.  Direct form:
// the vectors go through the four stages alongside the state.
template <class Sys, int K, bool LD, typename VT>
__device__ __forceinline__ void rk4_step_direct(double* x, VT (*w)[2 * Sys::N], double& L,
                                                const double h, const int ld_sqrt,
                                                const double ld_p, const SysPar& sp)
{
    constexpr int N = Sys::N, D = 2 * N, NH = Sys::NH;
    constexpr int KK = K > 0 ? K : 1;
    const double hh = 0.5 * h, h6 = h / 6.0;
    const VT hhv = (VT)hh, hv = (VT)h, h6v = (VT)h6;
    double ax[D], xs[D], f[D], H[NH];
    VT aw[KK][D], ws[KK][D], dw[D], Hc[NH];
    double aL = 0.0;
    FF fL{0.0f, 0.0f};  // p = 1/2: the LD sum in double-float (rk4_common.cuh)

    // stage 1 at (x, w)
    Sys::eval(x, f, H, sp);
#pragma unroll
    for (int i = 0; i < NH; ++i) Hc[i] = (VT)H[i];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        ax[c] = f[c];
        xs[c] = fma(hh, f[c], x[c]);
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
        var_rhs<N, NH, VT>(Hc, w[j], dw);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            aw[j][c] = dw[c];
            ws[j][c] = fma(hhv, dw[c], w[j][c]);
        }
    }
    if (LD) {
        if (ld_sqrt)
            ld_acc_sqrt<D>(fL, f, 1.0f);
        else
            aL = ld_integrand_pow<D>(f, ld_p);
    }

    // stages 2 and 3 at (xs, ws); the next stage input uses h/2 then h
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const double cs = (s == 0) ? hh : h;
        const VT csv = (s == 0) ? hhv : hv;
        Sys::eval(xs, f, H, sp);
#pragma unroll
        for (int i = 0; i < NH; ++i) Hc[i] = (VT)H[i];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            ax[c] = fma(2.0, f[c], ax[c]);
            xs[c] = fma(cs, f[c], x[c]);
        }
#pragma unroll
        for (int j = 0; j < K; ++j) {
            var_rhs<N, NH, VT>(Hc, ws[j], dw);
#pragma unroll
            for (int c = 0; c < D; ++c) {
                aw[j][c] = fma((VT)2, dw[c], aw[j][c]);
                ws[j][c] = fma(csv, dw[c], w[j][c]);
            }
        }
        if (LD) {
            if (ld_sqrt)
                ld_acc_sqrt<D>(fL, f, 2.0f);
            else
                aL = fma(2.0, ld_integrand_pow<D>(f, ld_p), aL);
        }
    }

    // stage 4 at (xs, ws)
    Sys::eval(xs, f, H, sp);
#pragma unroll
    for (int i = 0; i < NH; ++i) Hc[i] = (VT)H[i];
#pragma unroll
    for (int c = 0; c < D; ++c) x[c] = fma(h6, ax[c] + f[c], x[c]);
#pragma unroll
    for (int j = 0; j < K; ++j) {
        var_rhs<N, NH, VT>(Hc, ws[j], dw);
#pragma unroll
        for (int c = 0; c < D; ++c) w[j][c] = fma(h6v, aw[j][c] + dw[c], w[j][c]);
    }
    // the LD grows with |t|: a backward run (h < 0) accumulates a positive M_p
    if (LD) {
        if (ld_sqrt) {
            ld_acc_sqrt<D>(fL, f, 1.0f);
            L = fma(fabs(h6), ff_to_f64(fL), L);
        } else {
            L = fma(fabs(h6), aL + ld_integrand_pow<D>(f, ld_p), L);
        }
    }
}

// The same RK4 step with the vectors advanced by the exact one-step propagator
// Phi of RK4 on the variational equations (rk4_common.cuh); identical to the
// direct form in exact arithmetic and cheaper for k >= 3 vectors, and for
// k = 2 with Henon-Heiles (Phi is built once per step and applied to each
// vector).
template <class Sys, int K, bool LD>
__device__ __forceinline__ void rk4_step_phi(double* x, double (*w)[2 * Sys::N], double& L,
                                             const double h, const int ld_sqrt, const double ld_p,
                                             const SysPar& sp)
{
    PhiBlocks<Sys::N, double> P;
    if constexpr (std::is_same<Sys, SysHenonHeiles>::value) {
        // the propagator from the stage positions (phi_build_hh)
        double q[4][2];
        rk4_stages<Sys, LD, false>(x, L, h, ld_sqrt, ld_p, sp, [&](int s, const double* xs, const double*) {
            q[s][0] = xs[0];
            q[s][1] = xs[1];
        });
        phi_build_hh(q, h, P);
    } else {
        double H[4][Sys::NH];
        rk4_state_capture<Sys, LD>(x, L, h, ld_sqrt, ld_p, sp, H);
        phi_build<Sys::N, Sys::NH, double>(H, h, P);
    }
#pragma unroll
    for (int j = 0; j < K; ++j) phi_apply<Sys::N, double>(P, w[j]);
}

template <class Sys, int K, bool LD>
__device__ __forceinline__ void rk4_step(double* x, double (*w)[2 * Sys::N], double& L,
                                         const double h, const int ld_sqrt, const double ld_p,
                                         const SysPar& sp)
{
    // Henon-Heiles builds Phi from the stage positions (phi_build_hh), cheap
    // enough to pay off from two vectors on
    constexpr bool phi = K >= 3 || (K == 2 && std::is_same<Sys, SysHenonHeiles>::value);
    if constexpr (phi)
        rk4_step_phi<Sys, K, LD>(x, w, L, h, ld_sqrt, ld_p, sp);
    else
        rk4_step_direct<Sys, K, LD, double>(x, w, L, h, ld_sqrt, ld_p, sp);
}

// SALI of two vectors (each normalised first): min(|u + v|, |u - v|).
template <int D>
__device__ __forceinline__ double sali_of(const double* a, const double* b)
{
    double na = a[0] * a[0], nb = b[0] * b[0];
#pragma unroll
    for (int c = 1; c < D; ++c) {
        na = fma(a[c], a[c], na);
        nb = fma(b[c], b[c], nb);
    }
    const double ia = rsqrt_nr(na), ib = rsqrt_nr(nb);
    double sp = 0.0, sm = 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const double u = a[c] * ia, v = b[c] * ib;
        sp = fma(u + v, u + v, sp);
        sm = fma(u - v, u - v, sm);
    }
    return sqrt(fmin(sp, sm));
}

// The state of one orbit during a call: loaded from the ensemble, advanced
// step by step with the checks of the chs_integrate_batch contract, stored back.
template <class Sys, int K, bool LD>
struct OrbitRun {
    static constexpr int N = Sys::N, D = 2 * N, KK = K > 0 ? K : 1;
    double x[D];
    double w[KK][D];
    double L, h0, dhm;
    int64_t exec0, todo, s, until;
    long long t_start;  // clock64 when the orbit was taken up (clock budget)
    int32_t st;

    __device__ __forceinline__ void load(const int64_t o, const StepArgs& a, const EnsPtrs& e)
    {
        const int64_t n = e.n;
        const double* wg = static_cast<const double*>(e.w);
        t_start = clock64();
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
    __device__ __forceinline__ bool step(const StepArgs& a, const SysPar& sp)
    {
        ++s;
        rk4_step<Sys, K, LD>(x, w, L, a.dt, a.ld_sqrt, a.ld_p, sp);
        if (a.renorm) {
#pragma unroll
            for (int j = 0; j < K; ++j) {
                double n2 = w[j][0] * w[j][0];
#pragma unroll
                for (int c = 1; c < D; ++c) n2 = fma(w[j][c], w[j][c], n2);
                const double inv = rsqrt_ff(n2);
#pragma unroll
                for (int c = 0; c < D; ++c) w[j][c] *= inv;
            }
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
                for (int c = 0; c < D; ++c) fin = fin && isfinite(w[j][c]);
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
                if (a.early_exit && sali_of<D>(w[0], w[1]) < a.sali_threshold) {
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

    // Writes the orbit back; true when it is still running (status OK and below
    // its end step).
    __device__ __forceinline__ bool store(const int64_t o, const EnsPtrs& e) const
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
__device__ __forceinline__ bool integrate_orbit(const int64_t o, const StepArgs& a, const SysPar& sp,
                                                const EnsPtrs& e)
{
    OrbitRun<Sys, K, LD> r;
    r.load(o, a, e);
    while (r.s < r.todo)
        if (!r.step(a, sp)) break;
    return r.store(o, e);
}

// One thread per orbit.  MODE kModeAll: thread t takes orbit t; kModeList:
// orbit list[t] for t < *count, appended to the next list while it is still
// running; kModeQueue: a persistent grid, every thread taking orbit after orbit
// from the work queue (queue_worker), so that an orbit that ends early (end
// step, early exit, escape) frees its lane at once.
template <class Sys, int K, bool LD, int MODE>
__global__ void __launch_bounds__(kSmallBlock)
k_integrate(const StepArgs a, const SysPar sp, const EnsPtrs e, const OrbitList ol)
{
    if constexpr (MODE == kModeQueue) {
        queue_worker<OrbitRun<Sys, K, LD>>(a, sp, e, ol.queue);
    } else {
        const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        int64_t o = t;
        if (MODE == kModeList) {
            if (t >= *ol.count) return;
            o = ol.list[t];
        }
        if (o >= e.n) return;
        if (e.status[o] != CHS_ORBIT_OK) return;
        const bool keep = integrate_orbit<Sys, K, LD>(o, a, sp, e);
        if (MODE == kModeList) list_append(ol, keep, (int32_t)o);
    }
}

// Orbits that can still advance: status OK and below their end step.
__global__ void k_list_init(const EnsPtrs e, int32_t* __restrict__ list, int32_t* __restrict__ count)
{
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= e.n) return;
    bool keep = e.status[o] == CHS_ORBIT_OK;
    if (keep && e.t_end) keep = e.n_exec[o] < e.t_end[o];
    OrbitList ol{nullptr, nullptr, list, count, nullptr};
    list_append(ol, keep, (int32_t)o);
}

cudaError_t launch_list_init(const EnsPtrs& e, int32_t* list, int32_t* count, cudaStream_t st)
{
    if (e.n == 0) return cudaSuccess;
    k_list_init<<<blocks_for(e.n, 256), 256, 0, st>>>(e, list, count);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Indicators: SALI, GALI_2..k (prod R_ii of a modified Gram-Schmidt QR of the
// unit vectors), labels
// --------------------------------------------------------------------------

template <int D, int K, typename VT>
__global__ void __launch_bounds__(kSmallBlock)
k_indicators(const int64_t n, const VT* __restrict__ wg, const int32_t* __restrict__ status,
             const double thr, double* __restrict__ sali, double* __restrict__ gali,
             int8_t* __restrict__ label)
{
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const int32_t st = status[o];
    const double qnan = __longlong_as_double(0x7ff8000000000000LL);
    double A[K][D];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        double n2 = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            A[j][c] = (double)wg[(j * D + c) * n + o];
            n2 = fma(A[j][c], A[j][c], n2);
        }
        const double inv = 1.0 / sqrt(n2);
#pragma unroll
        for (int c = 0; c < D; ++c) A[j][c] *= inv;
    }
    double sv = qnan;
    if (K >= 2 && st != CHS_ORBIT_FORBIDDEN) {
        double a2 = 0.0, b2 = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const double sp = A[0][c] + A[1 % K][c], sm = A[0][c] - A[1 % K][c];
            a2 = fma(sp, sp, a2);
            b2 = fma(sm, sm, b2);
        }
        sv = sqrt(fmin(a2, b2));
    }
    if (sali) sali[o] = sv;
    if (gali && K >= 2) {
        // modified Gram-Schmidt on the columns; GALI_m = prod_{j < m} R_jj
        double prod = 1.0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
#pragma unroll
            for (int i = 0; i < j; ++i) {
                double r = 0.0;
#pragma unroll
                for (int c = 0; c < D; ++c) r = fma(A[i][c], A[j][c], r);
#pragma unroll
                for (int c = 0; c < D; ++c) A[j][c] = fma(-r, A[i][c], A[j][c]);
            }
            double n2 = 0.0;
#pragma unroll
            for (int c = 0; c < D; ++c) n2 = fma(A[j][c], A[j][c], n2);
            const double rjj = sqrt(n2);
            prod *= rjj;
            if (rjj > 0.0) {
                const double inv = 1.0 / rjj;
#pragma unroll
                for (int c = 0; c < D; ++c) A[j][c] *= inv;
            }
            if (j >= 1) gali[(int64_t)(j - 1) * n + o] = (st == CHS_ORBIT_FORBIDDEN) ? qnan : prod;
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
// Lyapunov spectrum of the 2-DOF systems: W (4 x 4) in registers
// --------------------------------------------------------------------------

template <class Sys>
__global__ void __launch_bounds__(kSmallBlock)
k_lyap_small(const StepArgs a, const SysPar sp, const int64_t n, const double* __restrict__ ics,
             const int32_t* __restrict__ ic_status, double* __restrict__ lambda,
             int32_t* __restrict__ status_out)
{
    constexpr int D = 2 * Sys::N;
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
        const long long t_start = clock64();
        double L = 0.0;
        int64_t until_qr = a.qr_every;
        int64_t until = a.sample_every > 0 ? a.sample_every : -1;
        for (int64_t s = 1; s <= a.n_steps; ++s) {
            rk4_step<Sys, D, false>(x, W, L, a.dt, 0, 0.0, sp);
            if (--until_qr == 0 || s == a.n_steps) {
                until_qr = a.qr_every;
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
                if (budget_spent(a, t_start)) {
                    st = CHS_ORBIT_STEP_BUDGET;
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

// --------------------------------------------------------------------------
// Host-side dispatch
// --------------------------------------------------------------------------

bool small_model(int model)
{
    return model == CHS_HENON_HEILES || model == CHS_HARMONIC || model == CHS_INVERTED ||
           model == CHS_QUARTIC3;
}

template <class Sys>
static cudaError_t init_k(int k, const SysPar& sp, int renorm, uint64_t seed, const double* ics,
                          const int32_t* ics_st, const void* w_in, const EnsPtrs& e, cudaStream_t st)
{
    const unsigned g = blocks_for(e.n, kSmallBlock);
    const double* wi = static_cast<const double*>(w_in);
    switch (k) {
#define CHS_CASE(KV)                                                                               \
    case KV:                                                                                       \
        k_init<Sys, KV, double><<<g, kSmallBlock, 0, st>>>(sp, renorm, seed, ics, ics_st, wi, e); \
        break;
        CHS_CASE(0) CHS_CASE(1) CHS_CASE(2) CHS_CASE(3) CHS_CASE(4)
#undef CHS_CASE
    case 5:
        if constexpr (Sys::N >= 3) {
            k_init<Sys, 5, double><<<g, kSmallBlock, 0, st>>>(sp, renorm, seed, ics, ics_st, wi, e);
            break;
        }
        return cudaErrorInvalidValue;
    case 6:
        if constexpr (Sys::N >= 3) {
            k_init<Sys, 6, double><<<g, kSmallBlock, 0, st>>>(sp, renorm, seed, ics, ics_st, wi, e);
            break;
        }
        return cudaErrorInvalidValue;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_init(const SysPar& sp, int k, int vec_fp32, int renorm, uint64_t seed,
                        const double* ics, const int32_t* ic_status, const void* w_in,
                        const EnsPtrs& e, cudaStream_t st)
{
    if (e.n == 0) return cudaSuccess;
    if (vec_fp32 && k > 0) return launch_init_f32(sp, k, seed, ics, ic_status, w_in, e, st);
    switch (sp.model) {
    case CHS_HENON_HEILES: return init_k<SysHenonHeiles>(k, sp, renorm, seed, ics, ic_status, w_in, e, st);
    case CHS_HARMONIC: return init_k<SysHarmonic>(k, sp, renorm, seed, ics, ic_status, w_in, e, st);
    case CHS_INVERTED: return init_k<SysInverted>(k, sp, renorm, seed, ics, ic_status, w_in, e, st);
    case CHS_QUARTIC3: return init_k<SysQuartic3>(k, sp, renorm, seed, ics, ic_status, w_in, e, st);
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
        if (!pg && persistent_blocks(k_integrate<Sys, K, LD, kModeQueue>, tb, 0, &pg) != cudaSuccess)
            pg = 0;
        k_integrate<Sys, K, LD, kModeQueue><<<pg ? pg : g, tb, 0, st>>>(a, sp, e, *ol);
    } else if (ol) {
        k_integrate<Sys, K, LD, kModeList><<<g, tb, 0, st>>>(a, sp, e, *ol);
    } else {
        k_integrate<Sys, K, LD, kModeAll><<<g, tb, 0, st>>>(a, sp, e, OrbitList{});
    }
}

template <class Sys, bool LD>
static cudaError_t integ_k(int k, const StepArgs& a, const SysPar& sp, const EnsPtrs& e,
                           const OrbitList* ol, cudaStream_t st)
{
    const unsigned g = blocks_for(e.n, small_threads(a));
    switch (k) {
    case 0: integ_one<Sys, 0, LD>(g, a, sp, e, ol, st); break;
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

template <class Sys>
static cudaError_t integ_sys(int k, bool ld, const StepArgs& a, const SysPar& sp, const EnsPtrs& e,
                             const OrbitList* ol, cudaStream_t st)
{
    return ld ? integ_k<Sys, true>(k, a, sp, e, ol, st) : integ_k<Sys, false>(k, a, sp, e, ol, st);
}

cudaError_t launch_integrate(const SysPar& sp, int k, int vec_fp32, bool ld, const StepArgs& a,
                             const EnsPtrs& e, const OrbitList* ol, cudaStream_t st)
{
    if (e.n == 0 || a.n_steps == 0) return cudaSuccess;
    if (vec_fp32 && k > 0) return launch_integrate_f32(sp, k, ld, a, e, ol, st);
    switch (sp.model) {
    case CHS_HENON_HEILES: return integ_sys<SysHenonHeiles>(k, ld, a, sp, e, ol, st);
    case CHS_HARMONIC: return integ_sys<SysHarmonic>(k, ld, a, sp, e, ol, st);
    case CHS_INVERTED: return integ_sys<SysInverted>(k, ld, a, sp, e, ol, st);
    case CHS_QUARTIC3: return integ_sys<SysQuartic3>(k, ld, a, sp, e, ol, st);
    }
    return cudaErrorInvalidValue;
}

template <int D>
static cudaError_t ind_k(int k, double thr, const EnsPtrs& e, double* sali, double* gali,
                         int8_t* label, cudaStream_t st)
{
    const unsigned g = blocks_for(e.n, kSmallBlock);
    const double* w = static_cast<const double*>(e.w);
    switch (k) {
#define CHS_CASE(KV)                                                                              \
    case KV:                                                                                      \
        k_indicators<D, KV, double><<<g, kSmallBlock, 0, st>>>(e.n, w, e.status, thr, sali, gali, \
                                                               label);                            \
        break;
        CHS_CASE(1) CHS_CASE(2) CHS_CASE(3) CHS_CASE(4) CHS_CASE(5) CHS_CASE(6)
#undef CHS_CASE
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_indicators(const SysPar& sp, int k, int vec_fp32, double sali_threshold,
                              const EnsPtrs& e, double* sali, double* gali, int8_t* label,
                              cudaStream_t st)
{
    if (e.n == 0) return cudaSuccess;
    if (vec_fp32 && k > 0) return launch_indicators_f32(sp, k, sali_threshold, e, sali, gali, label, st);
    const int D = 2 * sp.n_dof;
    if (D == 4) return ind_k<4>(k, sali_threshold, e, sali, gali, label, st);
    if (D == 6) return ind_k<6>(k, sali_threshold, e, sali, gali, label, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_lyap_small(const SysPar& sp, const StepArgs& a, int64_t n, const double* ics,
                              const int32_t* ic_status, double* lambda, int32_t* status,
                              cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const unsigned g = blocks_for(n, kSmallBlock);
    switch (sp.model) {
    case CHS_HENON_HEILES:
        k_lyap_small<SysHenonHeiles><<<g, kSmallBlock, 0, st>>>(a, sp, n, ics, ic_status, lambda, status);
        break;
    case CHS_HARMONIC:
        k_lyap_small<SysHarmonic><<<g, kSmallBlock, 0, st>>>(a, sp, n, ics, ic_status, lambda, status);
        break;
    case CHS_INVERTED:
        k_lyap_small<SysInverted><<<g, kSmallBlock, 0, st>>>(a, sp, n, ics, ic_status, lambda, status);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace chs

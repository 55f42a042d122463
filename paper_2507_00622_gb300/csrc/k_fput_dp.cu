// k_fput_dp.cu -- Lyapunov spectrum of the FPUT chain by periodic QR with the
// paper's own 8th-order solver (Sec. Functionalities: DOP 8 and DOP 8(5) with
// vector normalisation and QR; FPU example of Sec. Examples), fixed step and
// adaptive.
//
// RK4 has a cheap one-step propagator for the chain (k_fput.cu); DOP853 has
// none (its propagator is a degree-12 polynomial in the stage Jacobians), and
// running the 2N deviation vectors through the twelve stages side by side
// would need 11 stage copies of the 2N x 2N matrix W (1.4 MB per orbit at
// N = 64).  So a step runs in the two phases of fput_stages.cuh: the orbit
// through its stages (one thread per component), then the columns of W one at
// a time per warp segment, with their stage derivatives in registers.
//
// W lives in shared memory column-major with a padded column stride 2N + 1, so
// that both a warp reading down a column and the QR's thread-per-column sweeps
// are free of bank conflicts.  The QR is the modified Gram-Schmidt of the RK4
// kernel ("dot products first"); S_j += ln R_jj, lambda_j = S_j / T.
//
// Adaptive runs give every orbit its own time and step size.  The error norm
// of a trial is a sum over the orbit's 2N components (an xor butterfly, the
// same in every thread), from which the orbit's first thread forms the error
// and the step factor for all of its threads; the columns of W advance only
// for accepted trials.  A block loops until all of its orbits are done.
#include "fput_ens.cuh"

namespace chs {
namespace {

template <int N>
struct FputDpCfg {
    static constexpr int D = 2 * N;
    static constexpr int G = D >= 32 ? 1 : 32 / D;  // orbits per block: one warp for N <= 16
    static constexpr int THREADS = G * D;             // 32, 64 or 128
    static constexpr int WS = D + 1;                   // padded column stride
    // doubles per orbit: W, two stage-state buffers, 12 stage stiffness rows,
    // two error-sum rows, control words
    static constexpr int PER = D * WS + 2 * D + 12 * (N + 1) + 2 * D + 6 + (D == 128 ? 8 * D : 0);
    static constexpr size_t SMEM = (size_t)G * PER * sizeof(double);
    static_assert(THREADS % 32 == 0 && THREADS <= 128, "whole warps, N <= 64");
};

// Offsets inside an orbit's shared slab.
template <int N>
struct FputDpSlab {
    using Cfg = FputDpCfg<N>;
    static constexpr int W = 0;
    static constexpr int XB = Cfg::D * Cfg::WS;     // [2][D]
    static constexpr int CS = XB + 2 * Cfg::D;      // [12][N + 1]
    static constexpr int ER = CS + 12 * (N + 1);    // [2][D] error sums
    static constexpr int CTL = ER + 2 * Cfg::D;     // [0] red, [1] any, [2] step of phase 2, [3] advance,
                                                    // [4] error, [5] err^(-1/8)
    static constexpr int QP = CTL + 6;              // N = 64: the split QR's partial sums [2][4][D]
    static_assert(QP + (Cfg::D == 128 ? 8 * Cfg::D : 0) == Cfg::PER, "slab layout");
};

// N = 64 (one orbit per block and per SM): the same Gram-Schmidt with the rows
// split across the orbit's four warps (warp w takes rows 32w..32w+31 of the
// columns lane + 32m), the four partial dot products of a column summed in a
// fixed order from double-buffered shared memory; otherwise the warp holding
// the last columns would work all 128 iterations alone.  Thread l still adds
// ln R_ll to its S.
template <int N>
__device__ __forceinline__ void qr_step_split(double* slab, const int l, double& S)
{
    using Cfg = FputDpCfg<N>;
    using Sl = FputDpSlab<N>;
    constexpr int D = Cfg::D, WS = Cfg::WS, Q = D / 32;
    static_assert(Cfg::G == 1, "one orbit per block");
    double* W = slab + Sl::W;
    double* P = slab + Sl::QP;
    const int w = l / 32, lane = l % 32, r0 = 32 * w;
    double n2[Q];  // squared norms of the thread's columns
#pragma unroll
    for (int m = 0; m < Q; ++m) n2[m] = 1.0;
    double nl = 1.0;  // squared norm of column l (this thread's exponent)
    for (int j = 0; j < D; ++j) {
        __syncwarp();  // rows of column j in this warp's block are final
        double* Pb = P + (j & 1) * Q * D;
        const double* wj = W + j * WS + r0;
#pragma unroll
        for (int m = 0; m < Q; ++m) {
            const int c = lane + 32 * m;
            if (c >= j) {
                const double* wc = W + c * WS + r0;
                double a0 = 0.0, a1 = 0.0;
#pragma unroll 4
                for (int i = 0; i < 32; i += 2) {
                    a0 = fma(wj[i], wc[i], a0);
                    a1 = fma(wj[i + 1], wc[i + 1], a1);
                }
                Pb[w * D + c] = a0 + a1;
            }
        }
        __syncthreads();
        double nj = Pb[j];
#pragma unroll
        for (int q = 1; q < Q; ++q) nj += Pb[q * D + j];
        const double inv_nj = 1.0 / nj;  // one division per pivot, not per column
#pragma unroll
        for (int m = 0; m < Q; ++m) {
            const int c = lane + 32 * m;
            if (c > j) {
                double r = Pb[c];
#pragma unroll
                for (int q = 1; q < Q; ++q) r += Pb[q * D + c];
                const double cfac = -r * inv_nj;
                double* wc = W + c * WS + r0;
#pragma unroll 4
                for (int i = 0; i < 32; ++i) wc[i] = fma(cfac, wj[i], wc[i]);
            } else if (c == j) {
                n2[m] = nj;
            }
        }
        if (l == j) nl = nj;
    }
    // the logarithms and reciprocal roots after the loop, not one lane's work
    // inside every pivot step
    S += 0.5 * log(nl);
    __syncwarp();
#pragma unroll
    for (int m = 0; m < Q; ++m) {
        const double inv = rsqrt(n2[m]);
        double* wc = W + (lane + 32 * m) * WS + r0;
#pragma unroll 4
        for (int i = 0; i < 32; ++i) wc[i] *= inv;
    }
    __syncthreads();
}

// The split Gram-Schmidt of qr_step_split run by 256 threads (two per column,
// the wide N = 64 kernel below): warp w takes rows 32 (w % 4) .. 32 (w % 4) + 31
// of the column groups m = w / 4 and w / 4 + 2 (columns lane + 32 m), the two
// warps of a row block meeting at a named barrier before each pivot.  The same
// partial dot products, summed in the same order, and the same updates as
// qr_step_split: identical results.  Threads t < 128 (t = l) add ln R_ll to S.
__device__ __forceinline__ void pair_sync(const int rb)
{
    asm volatile("bar.sync %0, 64;" ::"r"(1 + rb) : "memory");
}

__device__ __forceinline__ void qr_step_split_wide(double* slab, const int t, double& S)
{
    constexpr int N = 64;
    using Cfg = FputDpCfg<N>;
    using Sl = FputDpSlab<N>;
    constexpr int D = Cfg::D, WS = Cfg::WS, Q = D / 32;
    double* W = slab + Sl::W;
    double* P = slab + Sl::QP;
    const int w = t / 32, lane = t % 32, rb = w % 4, ch = w / 4, r0 = 32 * rb;
    double n2[2] = {1.0, 1.0};  // squared norms of the thread's two columns
    double nl = 1.0;            // squared norm of column t (t < 128)
    for (int j = 0; j < D; ++j) {
        pair_sync(rb);  // rows of column j in this row block are final
        double* Pb = P + (j & 1) * Q * D;
        const double* wj = W + j * WS + r0;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int c = lane + 32 * (ch + 2 * u);
            if (c >= j) {
                const double* wc = W + c * WS + r0;
                double a0 = 0.0, a1 = 0.0;
#pragma unroll 4
                for (int i = 0; i < 32; i += 2) {
                    a0 = fma(wj[i], wc[i], a0);
                    a1 = fma(wj[i + 1], wc[i + 1], a1);
                }
                Pb[rb * D + c] = a0 + a1;
            }
        }
        __syncthreads();
        double nj = Pb[j];
#pragma unroll
        for (int q = 1; q < Q; ++q) nj += Pb[q * D + j];
        const double inv_nj = 1.0 / nj;  // one division per pivot, not per column
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int c = lane + 32 * (ch + 2 * u);
            if (c > j) {
                double r = Pb[c];
#pragma unroll
                for (int q = 1; q < Q; ++q) r += Pb[q * D + c];
                const double cfac = -r * inv_nj;
                double* wc = W + c * WS + r0;
#pragma unroll 4
                for (int i = 0; i < 32; ++i) wc[i] = fma(cfac, wj[i], wc[i]);
            } else if (c == j) {
                n2[u] = nj;
            }
        }
        if (t == j) nl = nj;
    }
    if (t < D) S += 0.5 * log(nl);
    __syncwarp();  // this warp's columns' rows were last written by this warp
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const double inv = rsqrt(n2[u]);
        double* wc = W + (lane + 32 * (ch + 2 * u)) * WS + r0;
#pragma unroll 4
        for (int i = 0; i < 32; ++i) wc[i] *= inv;
    }
    __syncthreads();
}

// Modified Gram-Schmidt of the orbit's W (thread l owns column l), when `mine`
// is set for the orbit; every thread takes part in the barriers.  S += ln R_ll.
// At N = 64 (one orbit per block, so `mine` is set whenever this runs) the
// rows are split across the warps instead (qr_step_split).
template <int N>
__device__ __forceinline__ void qr_step(double* slab, const int l, const bool mine, double& S)
{
    using Cfg = FputDpCfg<N>;
    using Sl = FputDpSlab<N>;
    constexpr int D = Cfg::D, WS = Cfg::WS;
    if constexpr (D == 128) {
        qr_step_split<N>(slab, l, S);
        return;
    }
    double* W = slab + Sl::W;
    double* red = slab + Sl::CTL;
    double* wl = W + l * WS;
    double n2 = 1.0;  // squared norm of this thread's column
    for (int j = 0; j < D; ++j) {
        const double* wj = W + j * WS;
        double r = 0.0;
        if (mine && l >= j) {
            double r0a = 0.0, r1a = 0.0;
#pragma unroll 4
            for (int i = 0; i < D; i += 2) {
                r0a = fma(wj[i], wl[i], r0a);
                r1a = fma(wj[i + 1], wl[i + 1], r1a);
            }
            r = r0a + r1a;
        }
        if (mine && l == j) {
            red[0] = r;
            n2 = r;
        }
        __syncthreads();
        if (mine && l > j) {
            const double cfac = -r / red[0];
#pragma unroll 4
            for (int i = 0; i < D; ++i) wl[i] = fma(cfac, wj[i], wl[i]);
        }
        __syncthreads();
    }
    // the logarithm and reciprocal root after the loop, one per thread, not one
    // lane's work inside every pivot step
    if (mine) {
        S += 0.5 * log(n2);
        const double inv = rsqrt(n2);
#pragma unroll 4
        for (int i = 0; i < D; ++i) wl[i] *= inv;
    }
    __syncthreads();
}

template <int N>
__global__ void __launch_bounds__(128, 1)
k_fput_lyap_dp(const StepArgs a, const SysPar sp, const int64_t n, const double* __restrict__ ics,
               const int32_t* __restrict__ ic_status, double* __restrict__ lambda,
               int32_t* __restrict__ status_out)
{
    using Cfg = FputDpCfg<N>;
    using Sl = FputDpSlab<N>;
    constexpr int D = Cfg::D, G = Cfg::G, PER = Cfg::PER, WS = Cfg::WS;
    extern __shared__ double smem[];
    const int g = threadIdx.x / D, l = threadIdx.x % D;
    const int64_t o = (int64_t)blockIdx.x * G + g;
    const bool valid = o < n;
    double* slab = smem + g * PER;
    double* red = slab + Sl::CTL;

    const fs::Coef fc = fs::coef_of(sp);
    int32_t st = valid ? (ic_status ? ic_status[o] : CHS_ORBIT_OK) : CHS_ORBIT_FORBIDDEN;
    double xi = valid ? ics[(int64_t)l * n + o] : 0.0;

    // orbit-wide "any thread" (block-wide barriers; every thread takes part)
    auto orbit_any = [&](bool pred) {
        if (l == 0) red[1] = 0.0;
        __syncthreads();
        if (pred) red[1] = 1.0;
        __syncthreads();
        const bool r = red[1] != 0.0;
        __syncthreads();
        return r;
    };
    if (orbit_any(!isfinite(xi)) && st == CHS_ORBIT_OK) st = CHS_ORBIT_NONFINITE;
    if (st != CHS_ORBIT_OK) xi = 0.0;

#pragma unroll 4
    for (int i = 0; i < D; ++i) slab[Sl::W + l * WS + i] = (i == l) ? 1.0 : 0.0;
    double S = 0.0;
    __syncthreads();

    const double h = a.dt;
    int64_t until_qr = a.qr_every;
    int64_t until = a.sample_every > 0 ? a.sample_every : -1;
    const long long t_start = clock64();
    for (int64_t step = 1; step <= a.n_steps; ++step) {
        double e5, e3;
        xi = fs::orbit_stages<N, fs::TabDop853, false>(xi, h, l, slab + Sl::XB, slab + Sl::CS, fc, e5, e3);
        __syncthreads();  // every stage stiffness is written
        fs::columns<N, fs::TabDop853, G, PER, WS, Sl::CS, false>(smem, D, [&](int, const double*) { return h; });
        __syncthreads();  // W complete; stage stiffnesses free
        if (--until_qr == 0 || step == a.n_steps) {
            until_qr = a.qr_every;
            qr_step<N>(slab, l, true, S);
        }
        if (--until == 0) {
            until = a.sample_every;
            if (orbit_any(!(isfinite(xi) && isfinite(S))) && st == CHS_ORBIT_OK) st = CHS_ORBIT_NONFINITE;
            // block-uniform: the block's orbits stop together
            if (a.clock_budget > 0 && __syncthreads_or(budget_spent(a, t_start))) {
                if (st == CHS_ORBIT_OK) st = CHS_ORBIT_STEP_BUDGET;
                break;
            }
        }
    }
    if (valid) {
        const double T = (double)a.n_steps * a.dt;
        lambda[(int64_t)l * n + o] =
            (st == CHS_ORBIT_OK) ? S / T : __longlong_as_double(0x7ff8000000000000LL);
        if (l == 0) status_out[o] = st;
    }
}

// N = 64 with 256 threads per orbit (one orbit per block and per SM, as in
// k_fput_lyap_dp<64>): two warps per sub-partition instead of one, so that one
// warp's shared-memory traffic and barriers overlap the other's FP64 work.  The
// orbit's stages run on threads t < 128 exactly as in k_fput_lyap_dp (the others
// only meet the barriers); phase 2 spreads the 128 columns over 8 warps instead
// of 4; the QR is qr_step_split_wide.  Every column, stage and dot product is
// computed as in k_fput_lyap_dp<64>: identical results.
constexpr int kDpWideThreads = 256;

__global__ void __launch_bounds__(kDpWideThreads, 1)
k_fput_lyap_dp_wide(const StepArgs a, const SysPar sp, const int64_t n, const double* __restrict__ ics,
                    const int32_t* __restrict__ ic_status, double* __restrict__ lambda,
                    int32_t* __restrict__ status_out)
{
    constexpr int N = 64;
    using Cfg = FputDpCfg<N>;
    using Sl = FputDpSlab<N>;
    constexpr int D = Cfg::D, PER = Cfg::PER, WS = Cfg::WS;
    extern __shared__ double smem[];
    const int t = threadIdx.x, l = t % D, half = t / D;
    const bool lead = t < D;
    const int64_t o = blockIdx.x;
    const bool valid = o < n;
    double* slab = smem;
    double* red = slab + Sl::CTL;

    const fs::Coef fc = fs::coef_of(sp);
    int32_t st = valid ? (ic_status ? ic_status[o] : CHS_ORBIT_OK) : CHS_ORBIT_FORBIDDEN;
    double xi = (valid && lead) ? ics[(int64_t)l * n + o] : 0.0;

    auto orbit_any = [&](bool pred) {
        if (t == 0) red[1] = 0.0;
        __syncthreads();
        if (pred) red[1] = 1.0;
        __syncthreads();
        const bool r = red[1] != 0.0;
        __syncthreads();
        return r;
    };
    if (orbit_any(lead && !isfinite(xi)) && st == CHS_ORBIT_OK) st = CHS_ORBIT_NONFINITE;
    if (st != CHS_ORBIT_OK) xi = 0.0;

#pragma unroll 4
    for (int i = 64 * half; i < 64 * half + 64; ++i) slab[Sl::W + l * WS + i] = (i == l) ? 1.0 : 0.0;
    double S = 0.0;
    __syncthreads();

    const double h = a.dt;
    int64_t until_qr = a.qr_every;
    int64_t until = a.sample_every > 0 ? a.sample_every : -1;
    const long long t_start = clock64();
    for (int64_t step = 1; step <= a.n_steps; ++step) {
        double e5, e3;
        xi = fs::orbit_stages<N, fs::TabDop853, false, true>(xi, h, l, slab + Sl::XB, slab + Sl::CS, fc, e5, e3,
                                                             lead);
        __syncthreads();  // every stage stiffness is written
        fs::columns<N, fs::TabDop853, 1, PER, WS, Sl::CS, false>(smem, D, [&](int, const double*) { return h; });
        __syncthreads();  // W complete; stage stiffnesses free
        if (--until_qr == 0 || step == a.n_steps) {
            until_qr = a.qr_every;
            qr_step_split_wide(slab, t, S);
        }
        if (--until == 0) {
            until = a.sample_every;
            if (orbit_any(lead && !(isfinite(xi) && isfinite(S))) && st == CHS_ORBIT_OK) st = CHS_ORBIT_NONFINITE;
            // block-uniform: the orbit's threads stop together
            if (a.clock_budget > 0 && __syncthreads_or(budget_spent(a, t_start))) {
                if (st == CHS_ORBIT_OK) st = CHS_ORBIT_STEP_BUDGET;
                break;
            }
        }
    }
    if (valid && lead) {
        const double T = (double)a.n_steps * a.dt;
        lambda[(int64_t)l * n + o] =
            (st == CHS_ORBIT_OK) ? S / T : __longlong_as_double(0x7ff8000000000000LL);
        if (l == 0) status_out[o] = st;
    }
}

// Adaptive DOP 8(5): every orbit from t = 0 to ad.t_final with its own steps.
template <int N>
__global__ void __launch_bounds__(128, 1)
k_fput_lyap_adapt(const StepArgs a, const AdaptArgs ad, const SysPar sp, const int64_t n,
                  const double* __restrict__ ics, const int32_t* __restrict__ ic_status,
                  double* __restrict__ lambda, int32_t* __restrict__ status_out,
                  int64_t* __restrict__ n_acc, int64_t* __restrict__ n_rej)
{
    using Cfg = FputDpCfg<N>;
    using Sl = FputDpSlab<N>;
    constexpr int D = Cfg::D, G = Cfg::G, PER = Cfg::PER, WS = Cfg::WS;
    extern __shared__ double smem[];
    const int g = threadIdx.x / D, l = threadIdx.x % D;
    const int64_t o = (int64_t)blockIdx.x * G + g;
    const bool valid = o < n;
    double* slab = smem + g * PER;
    double* ctl = slab + Sl::CTL;
    double* er = slab + Sl::ER;

    const fs::Coef fc = fs::coef_of(sp);
    int32_t st = valid ? (ic_status ? ic_status[o] : CHS_ORBIT_OK) : CHS_ORBIT_FORBIDDEN;
    double xi = valid ? ics[(int64_t)l * n + o] : 0.0;
    // a non-finite initial state is never accepted: it ends as STEP_FAIL
    if (st != CHS_ORBIT_OK) xi = 0.0;

#pragma unroll 4
    for (int i = 0; i < D; ++i) slab[Sl::W + l * WS + i] = (i == l) ? 1.0 : 0.0;
    double S = 0.0;
    // per-orbit control, identical in every thread of the orbit
    double tt = 0.0, hnext = a.dt;
    int64_t done = 0, rej = 0;
    bool rejected = false;
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    const long long t_start = clock64();
    int64_t iter = 0;
    __syncthreads();

    // Every iteration is one trial of every active orbit.  An orbit's trials end
    // once it reaches t_final, exhausts n_steps accepted steps or fails: each
    // rejection shrinks its step by at least 0.9 until it drops below
    // 10 ulp(t), so every orbit leaves after finitely many iterations.
    for (;;) {
        bool active = st == CHS_ORBIT_OK && tt < ad.t_final;
        if (active && done >= a.n_steps) {
            st = CHS_ORBIT_STEP_FAIL;
            active = false;
        }
        double hh = 0.0, tn = tt;
        if (active) {
            const double min_step = 10.0 * (nextafter(tt, inf) - tt);
            if (!rejected) {
                if (ad.h_max > 0.0 && hnext > ad.h_max) hnext = ad.h_max;
                if (hnext < min_step) hnext = min_step;
            }
            if (hnext < min_step) {
                st = CHS_ORBIT_STEP_FAIL;
                active = false;
            } else {
                tn = tt + hnext;
                if (tn > ad.t_final) tn = ad.t_final;
                hh = tn - tt;
            }
        }
        if (!__syncthreads_or(active)) break;

        double e5 = 0.0, e3 = 0.0;
        const double xn = fs::orbit_stages<N, fs::TabDop853, true>(xi, hh, l, slab + Sl::XB, slab + Sl::CS, fc, e5, e3);
        // error norm over the orbit's components, summed in index order by
        // every thread of the orbit
        const double sc = ad.atol + ad.rtol * fmax(fabs(xi), fabs(xn));
        const double q5 = e5 / sc, q3 = e3 / sc;
        const double E5 = fe::orbit_sum<D>(q5 * q5, er, l);
        const double E3 = fe::orbit_sum<D>(q3 * q3, er, l);
        if (l == 0) {
            const double err =
                (E5 == 0.0 && E3 == 0.0) ? 0.0 : fabs(hh) * E5 / sqrt((double)D * (E5 + 0.01 * E3));
            ctl[2] = (active && err < 1.0) ? hh : 0.0;
            ctl[4] = err;
            // err^(-1/8) as three square roots and a division
            ctl[5] = (active && err > 0.0) ? 1.0 / sqrt(sqrt(sqrt(err))) : 0.0;
        }
        __syncthreads();  // stage stiffnesses, phase-2 steps and the error are in place
        const double err = ctl[4], r8 = ctl[5];
        const bool accept = active && err < 1.0;

        fs::columns<N, fs::TabDop853, G, PER, WS, Sl::CS, true>(smem, D, [&](int, const double* sl) { return sl[Sl::CTL + 2]; });
        if (active) {
            if (accept) {
                double fac = (err == 0.0) ? 10.0 : fmin(10.0, 0.9 * r8);
                if (rejected) fac = fmin(fac, 1.0);
                hnext = hh * fac;
                xi = xn;
                tt = tn;
                ++done;
                rejected = false;
            } else {
                double fac = 0.9 * r8;
                if (!(fac >= 0.2)) fac = 0.2;
                hnext = hh * fac;
                rejected = true;
                ++rej;
            }
        }
        __syncthreads();  // W complete; stage stiffnesses free
        const bool want_qr = accept && ((a.qr_every > 0 && done % a.qr_every == 0) || tt >= ad.t_final);
        if (__syncthreads_or(want_qr)) qr_step<N>(slab, l, want_qr, S);
        // clock budget every sample_every trials, block-uniform
        if (a.clock_budget > 0 && a.sample_every > 0 && ++iter % a.sample_every == 0 &&
            __syncthreads_or(budget_spent(a, t_start)) && st == CHS_ORBIT_OK && tt < ad.t_final)
            st = CHS_ORBIT_STEP_BUDGET;
    }
    // non-finite exponent sums give NONFINITE for the whole orbit
    const bool bad = valid && st == CHS_ORBIT_OK && !isfinite(S);
    if (l == 0) ctl[3] = 0.0;
    __syncthreads();
    if (bad) ctl[3] = 1.0;
    __syncthreads();
    if (valid) {
        if (st == CHS_ORBIT_OK && ctl[3] != 0.0) st = CHS_ORBIT_NONFINITE;
        lambda[(int64_t)l * n + o] =
            (st == CHS_ORBIT_OK) ? S / ad.t_final : __longlong_as_double(0x7ff8000000000000LL);
        if (l == 0) {
            status_out[o] = st;
            if (n_acc) n_acc[o] = done;
            if (n_rej) n_rej[o] = rej;
        }
    }
}

template <int N>
cudaError_t prepare_dp_n()
{
    static bool done[kCacheDevices] = {};  // per device; set before any stream capture
    const int dev = cache_device();
    if (done[dev]) return cudaSuccess;
    cudaError_t err = cudaFuncSetAttribute(k_fput_lyap_dp<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)FputDpCfg<N>::SMEM);
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_fput_lyap_adapt<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)FputDpCfg<N>::SMEM);
    if constexpr (N == 64)
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(k_fput_lyap_dp_wide, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)FputDpCfg<N>::SMEM);
    if (err == cudaSuccess) done[dev] = true;
    return err;
}

template <int N>
cudaError_t fput_dp_n(const SysPar& sp, const StepArgs& a, int64_t n, const double* ics,
                      const int32_t* ic_status, double* lambda, int32_t* status, cudaStream_t st)
{
    using Cfg = FputDpCfg<N>;
    const cudaError_t err = prepare_dp_n<N>();
    if (err != cudaSuccess) return err;
    // N = 64: 256 threads per orbit by default (block_threads 0 or 256), the
    // 128-thread form with block_threads 128; both give the same results
    if constexpr (N == 64) {
        if (a.block == 0 || a.block == kDpWideThreads) {
            k_fput_lyap_dp_wide<<<blocks_for(n, 1), kDpWideThreads, Cfg::SMEM, st>>>(a, sp, n, ics, ic_status,
                                                                                  lambda, status);
            return cudaGetLastError();
        }
    }
    k_fput_lyap_dp<N><<<blocks_for(n, Cfg::G), Cfg::THREADS, Cfg::SMEM, st>>>(a, sp, n, ics, ic_status,
                                                                             lambda, status);
    return cudaGetLastError();
}

template <int N>
cudaError_t fput_adapt_n(const SysPar& sp, const StepArgs& a, const AdaptArgs& ad, int64_t n,
                         const double* ics, const int32_t* ic_status, double* lambda,
                         int32_t* status, int64_t* n_acc, int64_t* n_rej, cudaStream_t st)
{
    using Cfg = FputDpCfg<N>;
    const cudaError_t err = prepare_dp_n<N>();
    if (err != cudaSuccess) return err;
    k_fput_lyap_adapt<N><<<blocks_for(n, Cfg::G), Cfg::THREADS, Cfg::SMEM, st>>>(
        a, ad, sp, n, ics, ic_status, lambda, status, n_acc, n_rej);
    return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_fput_lyap_dp(int n_dof)
{
    switch (n_dof) {
    case 4: return prepare_dp_n<4>();
    case 8: return prepare_dp_n<8>();
    case 16: return prepare_dp_n<16>();
    case 32: return prepare_dp_n<32>();
    case 64: return prepare_dp_n<64>();
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_fput_lyap_dp(const SysPar& sp, const StepArgs& a, int64_t n, const double* ics,
                                const int32_t* ic_status, double* lambda, int32_t* status,
                                cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    switch (sp.n_dof) {
    case 4: return fput_dp_n<4>(sp, a, n, ics, ic_status, lambda, status, st);
    case 8: return fput_dp_n<8>(sp, a, n, ics, ic_status, lambda, status, st);
    case 16: return fput_dp_n<16>(sp, a, n, ics, ic_status, lambda, status, st);
    case 32: return fput_dp_n<32>(sp, a, n, ics, ic_status, lambda, status, st);
    case 64: return fput_dp_n<64>(sp, a, n, ics, ic_status, lambda, status, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_fput_lyap_adapt(const SysPar& sp, const StepArgs& a, const AdaptArgs& ad, int64_t n,
                                   const double* ics, const int32_t* ic_status, double* lambda,
                                   int32_t* status, int64_t* n_acc, int64_t* n_rej, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    switch (sp.n_dof) {
    case 4: return fput_adapt_n<4>(sp, a, ad, n, ics, ic_status, lambda, status, n_acc, n_rej, st);
    case 8: return fput_adapt_n<8>(sp, a, ad, n, ics, ic_status, lambda, status, n_acc, n_rej, st);
    case 16: return fput_adapt_n<16>(sp, a, ad, n, ics, ic_status, lambda, status, n_acc, n_rej, st);
    case 32: return fput_adapt_n<32>(sp, a, ad, n, ics, ic_status, lambda, status, n_acc, n_rej, st);
    case 64: return fput_adapt_n<64>(sp, a, ad, n, ics, ic_status, lambda, status, n_acc, n_rej, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace chs

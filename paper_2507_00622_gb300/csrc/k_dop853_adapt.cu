// k_dop853_adapt.cu -- DOP 8(5) with adaptive step size and the error of each
// step (Sec. Functionalities) on the one-orbit-per-thread systems: the DOP853
// pair with its 5th/3rd-order error estimate and the standard step-size
// controller (safety 0.9, growth at most 10, shrink at least 0.2), every orbit
// with its own time and step size.  Building blocks: dop853.cuh.
#include "dop853.cuh"

namespace chs {
namespace {

using dp::kBlock;

template <class Sys, int K, bool LD>
__global__ void __launch_bounds__(kBlock)
k_integrate_adaptive(const StepArgs a, const AdaptArgs ad, const SysPar sp, const EnsPtrs e,
                     const AdaptPtrs ap)
{
    constexpr int N = Sys::N, D = 2 * N;
    constexpr int KK = K > 0 ? K : 1;
    const dp::Slab<Sys> sl = dp::my_slab<Sys>();
    const int64_t n = e.n;
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    if (e.status[o] != CHS_ORBIT_OK) return;

    double* wg = static_cast<double*>(e.w);
    double x[D], w[KK][D];
#pragma unroll
    for (int c = 0; c < D; ++c) x[c] = e.x[c * n + o];
#pragma unroll
    for (int j = 0; j < K; ++j)
#pragma unroll
        for (int c = 0; c < D; ++c) w[j][c] = wg[(j * D + c) * n + o];
    double L = LD ? e.ld[o] : 0.0;
    const double h0 = e.h0[o];
    double dhm = e.dh_max[o];
    const int64_t exec0 = e.n_exec[o];
    double tt = ap.t[o], h = ap.h[o];
    double el = ap.err_last ? ap.err_last[o] : 0.0;
    double em = ap.err_max ? ap.err_max[o] : 0.0;
    int64_t rej = ap.n_rej ? ap.n_rej[o] : 0;
    const double inf = __longlong_as_double(0x7ff0000000000000LL);

    int32_t st = CHS_ORBIT_OK;
    int64_t done = 0;
    const long long t_start = clock64();
    while (done < a.n_steps && tt < ad.t_final) {
        const double min_step = 10.0 * (nextafter(tt, inf) - tt);
        if (ad.h_max > 0.0 && h > ad.h_max) h = ad.h_max;
        if (h < min_step) h = min_step;
        bool rejected = false;
        double xn[D], dL = 0.0, hh = 0.0, err = 0.0;
        // Each rejection multiplies h by at most 0.9 (0.2 for a non-finite
        // error), so this loop ends once h drops below min_step.
        for (;;) {
            if (h < min_step) {
                st = CHS_ORBIT_STEP_FAIL;
                break;
            }
            double tn = tt + h;
            if (tn > ad.t_final) tn = ad.t_final;
            hh = tn - tt;
            double e5[D], e3[D];
            dp::orbit_step<Sys, LD, true>(sl, x, hh, a.ld_sqrt, a.ld_p, sp, xn, dL, e5, e3);
            err = dp::err_norm<D>(x, xn, e5, e3, hh, ad.atol, ad.rtol);
            // err^(-1/8) as three square roots and a division
            const double r8 = (err > 0.0) ? 1.0 / sqrt(sqrt(sqrt(err))) : 0.0;
            if (err < 1.0) {
                double fac = (err == 0.0) ? 10.0 : fmin(10.0, 0.9 * r8);
                if (rejected) fac = fmin(fac, 1.0);
                h = hh * fac;
                tt = tn;
                break;
            }
            double fac = 0.9 * r8;
            if (!(fac >= 0.2)) fac = 0.2;
            h = hh * fac;
            rejected = true;
            ++rej;
        }
        if (st != CHS_ORBIT_OK) break;
#pragma unroll
        for (int j = 0; j < K; ++j) dp::vector_step<Sys>(sl, w[j], hh);
#pragma unroll
        for (int c = 0; c < D; ++c) x[c] = xn[c];
        if (LD) L += dL;
        el = err;
        em = fmax(em, err);
        ++done;
        const bool check = a.sample_every > 0 && (exec0 + done) % a.sample_every == 0;
        st = dp::post_step<Sys, K>(x, w, L, a, sp, check, h0, dhm);
        if (check && st == CHS_ORBIT_OK && budget_spent(a, t_start)) st = CHS_ORBIT_STEP_BUDGET;
        if (st != CHS_ORBIT_OK) break;
    }

#pragma unroll
    for (int c = 0; c < D; ++c) e.x[c * n + o] = x[c];
#pragma unroll
    for (int j = 0; j < K; ++j)
#pragma unroll
        for (int c = 0; c < D; ++c) wg[(j * D + c) * n + o] = w[j][c];
    if (LD) e.ld[o] = L;
    e.dh_max[o] = dhm;
    e.n_exec[o] = exec0 + done;
    e.status[o] = st;
    ap.t[o] = tt;
    ap.h[o] = h;
    if (ap.err_last) ap.err_last[o] = el;
    if (ap.err_max) ap.err_max[o] = em;
    if (ap.n_rej) ap.n_rej[o] = rej;
}

// Lyapunov spectrum of the 2-DOF systems with adaptive DOP 8(5): W (4 x 4) in
// registers, every orbit from t = 0 to ad.t_final with its own steps; QR every
// qr_every accepted steps and at t_final; lambda = S / t_final.
template <class Sys>
__global__ void __launch_bounds__(kBlock)
k_lyap_small_adapt(const StepArgs a, const AdaptArgs ad, const SysPar sp, const int64_t n,
                   const double* __restrict__ ics, const int32_t* __restrict__ ic_status,
                   double* __restrict__ lambda, int32_t* __restrict__ status_out,
                   int64_t* __restrict__ n_acc, int64_t* __restrict__ n_rej)
{
    constexpr int D = 2 * Sys::N;
    const dp::Slab<Sys> sl = dp::my_slab<Sys>();
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const double qnan = __longlong_as_double(0x7ff8000000000000LL);
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    int32_t st = ic_status ? ic_status[o] : CHS_ORBIT_OK;
    double x[D], W[D][D], S[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        x[c] = ics[c * n + o];
        S[c] = 0.0;
#pragma unroll
        for (int j = 0; j < D; ++j) W[j][c] = (j == c) ? 1.0 : 0.0;
    }
    double tt = 0.0, h = a.dt;
    int64_t done = 0, rej = 0;
    const long long t_start = clock64();
    // a non-finite initial state is never accepted: it ends as STEP_FAIL
    while (st == CHS_ORBIT_OK && tt < ad.t_final) {
        if (done >= a.n_steps) {
            st = CHS_ORBIT_STEP_FAIL;
            break;
        }
        const double min_step = 10.0 * (nextafter(tt, inf) - tt);
        if (ad.h_max > 0.0 && h > ad.h_max) h = ad.h_max;
        if (h < min_step) h = min_step;
        bool rejected = false;
        double xn[D], dL = 0.0, hh = 0.0, tn = tt;
        // each rejection shrinks h by at least 0.9 (0.2 for a non-finite error)
        for (;;) {
            if (h < min_step) {
                st = CHS_ORBIT_STEP_FAIL;
                break;
            }
            tn = tt + h;
            if (tn > ad.t_final) tn = ad.t_final;
            hh = tn - tt;
            double e5[D], e3[D];
            dp::orbit_step<Sys, false, true>(sl, x, hh, 0, 0.0, sp, xn, dL, e5, e3);
            const double err = dp::err_norm<D>(x, xn, e5, e3, hh, ad.atol, ad.rtol);
            const double r8 = (err > 0.0) ? 1.0 / sqrt(sqrt(sqrt(err))) : 0.0;
            if (err < 1.0) {
                double fac = (err == 0.0) ? 10.0 : fmin(10.0, 0.9 * r8);
                if (rejected) fac = fmin(fac, 1.0);
                h = hh * fac;
                break;
            }
            double fac = 0.9 * r8;
            if (!(fac >= 0.2)) fac = 0.2;
            h = hh * fac;
            rejected = true;
            ++rej;
        }
        if (st != CHS_ORBIT_OK) break;
#pragma unroll
        for (int j = 0; j < D; ++j) dp::vector_step<Sys>(sl, W[j], hh);
#pragma unroll
        for (int c = 0; c < D; ++c) x[c] = xn[c];
        tt = tn;
        ++done;
        if (a.sample_every > 0 && done % a.sample_every == 0 && budget_spent(a, t_start)) {
            st = CHS_ORBIT_STEP_BUDGET;
            break;
        }
        if ((a.qr_every > 0 && done % a.qr_every == 0) || tt >= ad.t_final) {
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
    }
    bool fin = true;
#pragma unroll
    for (int c = 0; c < D; ++c) fin = fin && isfinite(S[c]);
    if (st == CHS_ORBIT_OK && !fin) st = CHS_ORBIT_NONFINITE;
#pragma unroll
    for (int c = 0; c < D; ++c) lambda[c * n + o] = (st == CHS_ORBIT_OK) ? S[c] / ad.t_final : qnan;
    status_out[o] = st;
    if (n_acc) n_acc[o] = done;
    if (n_rej) n_rej[o] = rej;
}

template <class Sys>
cudaError_t adapt_sys(int k, bool ld, const StepArgs& a, const AdaptArgs& ad, const SysPar& sp,
                      const EnsPtrs& e, const AdaptPtrs& ap, cudaStream_t st)
{
    const unsigned g = blocks_for(e.n, kBlock);
    constexpr size_t sm = dp::slab_bytes<Sys>();
    return dp::with_k<Sys>(k, [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        if (ld)
            k_integrate_adaptive<Sys, K, true><<<g, kBlock, sm, st>>>(a, ad, sp, e, ap);
        else
            k_integrate_adaptive<Sys, K, false><<<g, kBlock, sm, st>>>(a, ad, sp, e, ap);
    });
}

}  // namespace

cudaError_t launch_lyap_small_adapt(const SysPar& sp, const StepArgs& a, const AdaptArgs& ad, int64_t n,
                                    const double* ics, const int32_t* ic_status, double* lambda,
                                    int32_t* status, int64_t* n_acc, int64_t* n_rej, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const unsigned g = blocks_for(n, kBlock);
    switch (sp.model) {
    case CHS_HENON_HEILES:
        k_lyap_small_adapt<SysHenonHeiles><<<g, kBlock, dp::slab_bytes<SysHenonHeiles>(), st>>>(
            a, ad, sp, n, ics, ic_status, lambda, status, n_acc, n_rej);
        break;
    case CHS_HARMONIC:
        k_lyap_small_adapt<SysHarmonic><<<g, kBlock, dp::slab_bytes<SysHarmonic>(), st>>>(
            a, ad, sp, n, ics, ic_status, lambda, status, n_acc, n_rej);
        break;
    case CHS_INVERTED:
        k_lyap_small_adapt<SysInverted><<<g, kBlock, dp::slab_bytes<SysInverted>(), st>>>(
            a, ad, sp, n, ics, ic_status, lambda, status, n_acc, n_rej);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_integrate_adaptive(const SysPar& sp, int k, bool ld, const StepArgs& a,
                                      const AdaptArgs& ad, const EnsPtrs& e, const AdaptPtrs& ap,
                                      cudaStream_t st)
{
    if (e.n == 0 || a.n_steps == 0) return cudaSuccess;
    switch (sp.model) {
    case CHS_HENON_HEILES: return adapt_sys<SysHenonHeiles>(k, ld, a, ad, sp, e, ap, st);
    case CHS_HARMONIC: return adapt_sys<SysHarmonic>(k, ld, a, ad, sp, e, ap, st);
    case CHS_INVERTED: return adapt_sys<SysInverted>(k, ld, a, ad, sp, e, ap, st);
    case CHS_QUARTIC3: return adapt_sys<SysQuartic3>(k, ld, a, ad, sp, e, ap, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace chs

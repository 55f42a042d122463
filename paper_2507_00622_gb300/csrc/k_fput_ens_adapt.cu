// k_fput_ens_adapt.cu -- adaptive DOP 8(5) (Sec. Functionalities) on FPUT
// ensembles with k <= 6 deviation vectors: the FPU timing workload of
// Sec. Examples (GALI_4 of 1e3 orbits per chain length) runs with it.
//
// Every orbit has its own time and step size.  A trial advances the orbit
// through the twelve stages (phase 1 of fput_stages.cuh); the error norm over
// its 2N components is an orbit-wide sum that every thread of the orbit holds
// bit for bit, so all of them take the same accept / reject decision.  The
// deviation vectors advance (phase 2, renormalised with renorm) only for
// accepted trials, and the checks of fput_ens.cuh follow each accepted step.
// Controller: safety 0.9, growth at most 10 (not above 1 right after a
// rejection), shrink at least 0.2, STEP_FAIL once h < 10 ulp(t).
#include "fput_ens.cuh"
#include "k_dop853.cuh"

namespace chs {
namespace {

template <int N>
__global__ void __launch_bounds__(128)
k_fput_ens_adapt(const StepArgs a, const AdaptArgs ad, const SysPar sp, const int K, const EnsPtrs e,
                 const AdaptPtrs ap)
{
    using Tab = fs::TabDop853;
    using C = fe::Cfg<N, Tab>;
    constexpr int D = C::D, G = C::G, PER = C::PER, WS = C::WS;
    __shared__ double smem[G * PER];
    const int g = threadIdx.x / D, l = threadIdx.x % D;
    const int64_t n = e.n;
    const int64_t o = (int64_t)blockIdx.x * G + g;
    const bool valid = o < n;
    double* slab = smem + g * PER;
    double* red = slab + C::RED;
    double* wg = static_cast<double*>(e.w);
    const fs::Coef fc = fs::coef_of(sp);
    const double inf = __longlong_as_double(0x7ff0000000000000LL);

    int32_t st = valid ? e.status[o] : CHS_ORBIT_FORBIDDEN;
    const bool runs = st == CHS_ORBIT_OK;
    double xi = valid ? e.x[(int64_t)l * n + o] : 0.0;
    for (int j = 0; j < K; ++j) slab[C::W + j * WS + l] = valid ? wg[((int64_t)j * D + l) * n + o] : 0.0;
    const double h0 = runs ? e.h0[o] : 0.0;
    double dhm = runs ? e.dh_max[o] : 0.0;
    const int64_t exec0 = runs ? e.n_exec[o] : 0;
    double tt = runs ? ap.t[o] : 0.0, hnext = runs ? ap.h[o] : 0.0;
    double el = (runs && ap.err_last) ? ap.err_last[o] : 0.0;
    double em = (runs && ap.err_max) ? ap.err_max[o] : 0.0;
    int64_t rej = (runs && ap.n_rej) ? ap.n_rej[o] : 0;
    int64_t done = 0;
    bool rejected = false;  // the current step has had a rejected trial
    const long long t_start = clock64();

    // One iteration = one trial of every orbit that is still running.  Each
    // rejection shrinks the step by at least 0.9 until it drops below
    // 10 ulp(t), and accepted steps are capped at n_steps, so every orbit
    // leaves after finitely many iterations.
    for (;;) {
        bool active = st == CHS_ORBIT_OK && done < a.n_steps && tt < ad.t_final;
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
        const double xn = fs::orbit_stages<N, Tab, true>(xi, hh, l, slab + C::XB, slab + C::CS, fc, e5, e3);
        const double sc = ad.atol + ad.rtol * fmax(fabs(xi), fabs(xn));
        const double q5 = e5 / sc, q3 = e3 / sc;
        const double E5 = fe::orbit_sum<D>(q5 * q5, red, l);
        const double E3 = fe::orbit_sum<D>(q3 * q3, red, l);
        // the orbit's first thread forms the error and err^(-1/8) (three square
        // roots and a division) for all of its threads, which read them back
        // after the barrier: the other warps of a long chain skip that work
        if (l == 0) {
            const double err =
                (E5 == 0.0 && E3 == 0.0) ? 0.0 : fabs(hh) * E5 / sqrt((double)D * (E5 + 0.01 * E3));
            slab[C::CTL] = (active && err < 1.0) ? hh : 0.0;
            slab[C::CTL + 1] = err;
            slab[C::CTL + 2] = (active && err > 0.0) ? 1.0 / sqrt(sqrt(sqrt(err))) : 0.0;
        }
        __syncthreads();  // stage stiffnesses, phase-2 steps and the error in place
        const double err = slab[C::CTL + 1], r8 = slab[C::CTL + 2];
        const bool accept = active && err < 1.0;
        fs::columns<N, Tab, G, PER, WS, C::CS, true>(smem, K, [](int, const double* sl) { return sl[C::CTL]; },
                                               a.renorm);
        __syncthreads();  // columns complete; stage buffers free
        if (active) {
            if (accept) {
                double fac = (err == 0.0) ? 10.0 : fmin(10.0, 0.9 * r8);
                if (rejected) fac = fmin(fac, 1.0);
                hnext = hh * fac;
                xi = xn;
                tt = tn;
                el = err;
                em = fmax(em, err);
                ++done;
                rejected = false;
            } else {
                double fac = 0.9 * r8;
                if (!(fac >= 0.2)) fac = 0.2;  // also for a non-finite error
                hnext = hh * fac;
                rejected = true;
                ++rej;
            }
        }
        const bool check = accept && a.sample_every > 0 && (exec0 + done) % a.sample_every == 0;
        const bool any_check = __syncthreads_or(check);
        st = fe::post_step<N, Tab>(a, sp, K, slab, l, xi, accept, check, any_check, h0, dhm, st);
        if (any_check && a.clock_budget > 0) {  // block-uniform: the block's orbits stop together
            const bool over = __syncthreads_or(budget_spent(a, t_start)) != 0;
            if (over && check && st == CHS_ORBIT_OK) st = CHS_ORBIT_STEP_BUDGET;
        }
    }
    if (runs) {
        e.x[(int64_t)l * n + o] = xi;
        for (int j = 0; j < K; ++j) wg[((int64_t)j * D + l) * n + o] = slab[C::W + j * WS + l];
        if (l == 0) {
            e.dh_max[o] = dhm;
            e.n_exec[o] = exec0 + done;
            e.status[o] = st;
            ap.t[o] = tt;
            ap.h[o] = hnext;
            if (ap.err_last) ap.err_last[o] = el;
            if (ap.err_max) ap.err_max[o] = em;
            if (ap.n_rej) ap.n_rej[o] = rej;
        }
    }
}

template <int N>
cudaError_t adapt_n(const SysPar& sp, int k, const StepArgs& a, const AdaptArgs& ad, const EnsPtrs& e,
                    const AdaptPtrs& ap, cudaStream_t st)
{
    using C = fe::Cfg<N, fs::TabDop853>;
    k_fput_ens_adapt<N><<<blocks_for(e.n, C::G), C::THREADS, 0, st>>>(a, ad, sp, k, e, ap);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fput_ens_adapt(const SysPar& sp, int k, const StepArgs& a, const AdaptArgs& ad,
                                  const EnsPtrs& e, const AdaptPtrs& ap, cudaStream_t st)
{
    if (e.n == 0 || a.n_steps == 0) return cudaSuccess;
    switch (sp.n_dof) {
    case 4: return adapt_n<4>(sp, k, a, ad, e, ap, st);
    case 8: return adapt_n<8>(sp, k, a, ad, e, ap, st);
    case 16: return adapt_n<16>(sp, k, a, ad, e, ap, st);
    case 32: return adapt_n<32>(sp, k, a, ad, e, ap, st);
    case 64: return adapt_n<64>(sp, k, a, ad, e, ap, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace chs

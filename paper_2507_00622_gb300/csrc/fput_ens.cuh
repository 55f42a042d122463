// fput_ens.cuh -- shared pieces of the FPUT ensemble kernels (k_fput_ens.cu:
// fixed steps; k_fput_ens_adapt.cu: adaptive DOP 8(5)): the per-orbit shared
// slab, orbit-wide sums and the checks that follow a completed step.
//
// An ensemble orbit carries its state x (2N components, one per thread of the
// orbit's 2N threads) and k <= 6 deviation vectors (columns in shared memory,
// advanced by the phase 2 of fput_stages.cuh).  A block holds one warp's worth
// of orbits, G = 32 / 2N, for N <= 16, and one orbit (2N threads) above: small
// blocks spread an ensemble of a thousand orbits over every SM, and the FP64
// pipe needs only a few warps per SM.
#pragma once

#include "fput_stages.cuh"

namespace chs {
namespace fe {

template <int N, class Tab>
struct Cfg {
    static constexpr int D = 2 * N;
    static constexpr int G = D >= 32 ? 1 : 32 / D;  // orbits per block
    static constexpr int THREADS = G * D;             // 32, 64 or 128
    static constexpr int WS = D;                       // column stride
    // slab of one orbit: kMaxDev columns, two stage-state buffers, the stage
    // stiffnesses, error-sum partials, warp partials of orbit sums, control
    static constexpr int W = 0;
    static constexpr int XB = kMaxDev * WS;            // [2][D]
    static constexpr int CS = XB + 2 * D;              // [S][N + 1]
    static constexpr int RED = CS + Tab::S * (N + 1);  // [4] warp partials
    static constexpr int CTL = RED + 4;                // [0] step of phase 2, [1] error, [2] err^(-1/8)
    static constexpr int PER = CTL + 4;
    static_assert(THREADS % 32 == 0 && THREADS <= 128, "whole warps, N <= 64");
};

// Sum over the orbit's D threads, the same value (bit for bit) in each of
// them: an xor butterfly inside a warp (a + b and b + a round alike), then the
// warp partials in a fixed order.  Every thread of the block must call it.
template <int D>
__device__ __forceinline__ double orbit_sum(double v, double* red, const int l)
{
    constexpr int LW = D < 32 ? D : 32;
#pragma unroll
    for (int off = LW / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off, LW);
    if constexpr (D > 32) {
        if ((l & 31) == 0) red[l >> 5] = v;
        __syncthreads();
        double s = red[0];
#pragma unroll
        for (int i = 1; i < D / 32; ++i) s += red[i];
        __syncthreads();
        return s;
    } else {
        return v;
    }
}

// Potential of one bond, V(r) = k/2 r^2 + alpha/3 r^3 + beta/4 r^4 (Eq. ham_FPU).
__device__ __forceinline__ double bond_v(const SysPar& sp, const double r)
{
    return r * r * (0.5 * sp.kk + r * (sp.alpha / 3.0 + 0.25 * sp.beta * r));
}

// The checks after a step, in this order: escape (sum_i q_i^2 > escape_r2,
// every step); then at health-check steps: non-finite state or vector ->
// NONFINITE, dh_max <- max(dh_max, |H - h0|), |H - h0| > dh_limit ->
// ENERGY_DRIFT, with early_exit SALI(w_1, w_2) < sali_threshold ->
// EARLY_CHAOTIC.  stepped and check are per orbit (the same in all of its
// threads), any_check is block-uniform.  Every thread of the block calls this.
template <int N, class Tab>
__device__ __forceinline__ int32_t post_step(const StepArgs& a, const SysPar& sp, const int K,
                                             double* slab, const int l, const double xi,
                                             const bool stepped, const bool check,
                                             const bool any_check, const double h0, double& dhm,
                                             int32_t st)
{
    using C = Cfg<N, Tab>;
    constexpr int D = C::D;
    double* red = slab + C::RED;
    if (a.escape_r2 > 0.0) {
        const double r2 = orbit_sum<D>(l < N ? xi * xi : 0.0, red, l);
        if (stepped && st == CHS_ORBIT_OK && r2 > a.escape_r2) st = CHS_ORBIT_ESCAPED;
    }
    if (!any_check) return st;
    bool fin = isfinite(xi);
    for (int j = 0; j < K; ++j) fin = fin && isfinite(slab[C::W + j * C::WS + l]);
    const double nbad = orbit_sum<D>(fin ? 0.0 : 1.0, red, l);
    double* xs = slab + C::XB;
    xs[l] = xi;
    __syncthreads();
    double term;
    if (l < N) {
        term = bond_v(sp, xs[l] - (l > 0 ? xs[l - 1] : 0.0));  // bond l: q_l - q_{l-1}
    } else {
        term = 0.5 * xi * xi;
        if (l == N) term += bond_v(sp, -xs[N - 1]);  // the bond to the right wall
    }
    const double H = orbit_sum<D>(term, red, l);
    double sali = __longlong_as_double(0x7ff0000000000000LL);
    if (a.early_exit && K >= 2) {
        const double u0 = slab[C::W + l], v0 = slab[C::W + C::WS + l];
        const double na = sqrt(orbit_sum<D>(u0 * u0, red, l));
        const double nb = sqrt(orbit_sum<D>(v0 * v0, red, l));
        const double u = u0 / na, v = v0 / nb;
        const double sp2 = orbit_sum<D>((u + v) * (u + v), red, l);
        const double sm2 = orbit_sum<D>((u - v) * (u - v), red, l);
        sali = fmin(sqrt(sp2), sqrt(sm2));
    }
    __syncthreads();  // xs is a stage buffer again
    if (check && stepped && st == CHS_ORBIT_OK) {
        if (nbad > 0.0) {
            st = CHS_ORBIT_NONFINITE;
        } else {
            const double dH = fabs(H - h0);
            if (dH > dhm) dhm = dH;
            if (a.dh_limit > 0.0 && dH > a.dh_limit)
                st = CHS_ORBIT_ENERGY_DRIFT;
            else if (a.early_exit && K >= 2 && sali < a.sali_threshold)
                st = CHS_ORBIT_EARLY_CHAOTIC;
        }
    }
    return st;
}

}  // namespace fe
}  // namespace chs

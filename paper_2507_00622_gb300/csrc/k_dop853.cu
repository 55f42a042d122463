// k_dop853.cu -- the paper's own 8th-order solver in fixed-step use (DOP 8,
// Sec. Functionalities) on the one-orbit-per-thread systems: the joint system
// (orbit, deviation vectors, LD) with the per-step checks of the RK4 path, over
// the whole ensemble or a compacted orbit list (kernels in k_dop853_fixed.cuh;
// the quartic oscillator's instances compile in k_dop853_q3.cu); and the
// Lyapunov spectrum of the 2-DOF systems.  Building blocks and design notes:
// dop853.cuh.
#include "k_dop853.cuh"
#include "k_dop853_fixed.cuh"

namespace chs {
namespace {

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
        const long long t_start = clock64();
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

}  // namespace

cudaError_t launch_integrate_dp(const SysPar& sp, int k, bool ld, const StepArgs& a,
                                const EnsPtrs& e, const OrbitList* ol, cudaStream_t st)
{
    if (e.n == 0 || a.n_steps == 0) return cudaSuccess;
    switch (sp.model) {
    case CHS_HENON_HEILES: return fixed_sys<SysHenonHeiles>(k, ld, a, sp, e, ol, st);
    case CHS_HARMONIC: return fixed_sys<SysHarmonic>(k, ld, a, sp, e, ol, st);
    case CHS_INVERTED: return fixed_sys<SysInverted>(k, ld, a, sp, e, ol, st);
    case CHS_QUARTIC3: return launch_integrate_dp_q3(k, ld, a, sp, e, ol, st);
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

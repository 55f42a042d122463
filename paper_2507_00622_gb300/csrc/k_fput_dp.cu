// k_fput_dp.cu -- Lyapunov spectrum of the FPUT chain by periodic QR with the
// paper's own 8th-order solver (DOP 8 with vector normalisation and QR, Sec.
// Functionalities; FPU example of Sec. Examples), fixed step.
//
// RK4 has a cheap one-step propagator for the chain (k_fput.cu); DOP853 has
// none (its propagator is a degree-12 polynomial in the stage Jacobians), and
// running the 2N deviation vectors through the twelve stages side by side
// would need 11 stage copies of the 2N x 2N matrix W (1.4 MB per orbit at
// N = 64).  So a step runs in two phases:
//
//   phase 1  the orbit: thread l of the orbit's 2N threads owns component l and
//            its stage derivatives (in registers); the stage states pass
//            through a double-buffered shared array (one barrier per stage),
//            and each stage leaves its N + 1 bond stiffnesses V''(D_b) behind;
//   phase 2  the columns of W, one at a time per warp segment: L = min(N, 32)
//            lanes split the column's N (q, p) row pairs, keep the column's
//            stage derivatives in registers and exchange the tridiagonal
//            neighbours q_{i-1}, q_{i+1} by warp shuffles.  No barrier, no
//            stage storage in memory.
//
// W lives in shared memory column-major with a padded column stride 2N + 1, so
// that both a warp reading down a column and the QR's thread-per-column sweeps
// are free of bank conflicts.  The QR is the modified Gram-Schmidt of the RK4
// kernel ("dot products first"); S_j += ln R_jj, lambda_j = S_j / T.
#include "dop853.cuh"

namespace chs {
namespace {

template <int N>
struct FputDpCfg {
    static constexpr int D = 2 * N;
    static constexpr int G = D >= 128 ? 1 : 128 / D;  // orbits per block
    static constexpr int THREADS = G * D;             // 128
    static constexpr int L = N < 32 ? N : 32;          // lanes per column
    static constexpr int R = N / L;                    // row pairs per lane
    static constexpr int CPW = 32 / L;                 // columns per warp at a time
    static constexpr int WS = D + 1;                   // padded column stride
    // doubles per orbit: W, two stage-state buffers, 12 stage stiffness rows, scratch
    static constexpr int PER = D * WS + 2 * D + 12 * (N + 1) + 2;
    static constexpr size_t SMEM = (size_t)G * PER * sizeof(double);
    static_assert(THREADS == 128, "one 128-thread block per orbit group");
    static_assert((G * D) % (4 * CPW) == 0, "every warp takes the same number of columns");
};

struct FputDpCoef {
    double k, a2, b3;  // V''(r) = k + 2 alpha r + 3 beta r^2
    double alpha, beta;
};

__device__ __forceinline__ double fdv(const FputDpCoef& fc, double r)
{
    return r * fma(r, fma(fc.beta, r, fc.alpha), fc.k);  // V'(r)
}

__device__ __forceinline__ double fd2v(const FputDpCoef& fc, double r)
{
    return fma(r, fma(fc.b3, r, fc.a2), fc.k);  // V''(r)
}

template <int N>
__global__ void __launch_bounds__(128)
k_fput_lyap_dp(const StepArgs a, const SysPar sp, const int64_t n, const double* __restrict__ ics,
               const int32_t* __restrict__ ic_status, double* __restrict__ lambda,
               int32_t* __restrict__ status_out)
{
    using Cfg = FputDpCfg<N>;
    constexpr int D = Cfg::D, G = Cfg::G, PER = Cfg::PER, L = Cfg::L, R = Cfg::R, CPW = Cfg::CPW,
                  WS = Cfg::WS;
    extern __shared__ double smem[];
    const int g = threadIdx.x / D, l = threadIdx.x % D;
    const int64_t o = (int64_t)blockIdx.x * G + g;
    const bool valid = o < n;
    double* W = smem + g * PER;
    double* xb = W + D * WS;           // [2][D] stage states
    double* cs = xb + 2 * D;           // [12][N + 1] stage stiffnesses
    double* red = cs + 12 * (N + 1);   // [2] scratch

    const FputDpCoef fc = {sp.kk, 2.0 * sp.alpha, 3.0 * sp.beta, sp.alpha, sp.beta};
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
    for (int i = 0; i < D; ++i) W[l * WS + i] = (i == l) ? 1.0 : 0.0;
    double S = 0.0;
    __syncthreads();

    const double h = a.dt;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int seg = lane / L, r0 = lane % L;
    int64_t until_qr = a.qr_every;
    int64_t until = a.sample_every > 0 ? a.sample_every : -1;
    for (int64_t step = 1; step <= a.n_steps; ++step) {
        // ---- phase 1: the orbit's twelve stages
        double F[12];
        double acc = 0.0;
        dp::static_for<0, 12>([&](auto sc) {
            constexpr int s = decltype(sc)::value;
            double sum = 0.0;
            dp::static_for<0, s>([&](auto jc) {
                constexpr int j = decltype(jc)::value;
                constexpr double c = dp::kA[s][j];
                if constexpr (c != 0.0) sum = fma(c, F[j], sum);
            });
            double* xs = xb + (s & 1) * D;
            xs[l] = (s == 0) ? xi : fma(h, sum, xi);
            __syncthreads();
            double f;
            if (l < N) {
                f = xs[N + l];
            } else {
                const int i = l - N;
                const double qm = i > 0 ? xs[i - 1] : 0.0;
                const double q0 = xs[i];
                const double qp = i < N - 1 ? xs[i + 1] : 0.0;
                f = fdv(fc, qp - q0) - fdv(fc, q0 - qm);
            }
            if (l <= N) {
                const double qa = l < N ? xs[l] : 0.0;
                const double qb = l > 0 ? xs[l - 1] : 0.0;
                cs[s * (N + 1) + l] = fd2v(fc, qa - qb);
            }
            F[s] = f;
            constexpr double cb = dp::kB[s];
            if constexpr (s == 0)
                acc = cb * f;
            else if constexpr (cb != 0.0)
                acc = fma(cb, f, acc);
        });
        xi = fma(h, acc, xi);
        __syncthreads();  // every stage stiffness is written

        // ---- phase 2: the columns of W through the twelve stages of w' = J_s w
        for (int task = warp * CPW + seg; task < G * D; task += 4 * CPW) {
            const int og = task / D, col = task % D;
            double* Wc = smem + og * PER + col * WS;
            const double* c_s = smem + og * PER + D * WS + 2 * D;
            double q[R], p[R];
#pragma unroll
            for (int k = 0; k < R; ++k) {
                q[k] = Wc[r0 + k * L];
                p[k] = Wc[N + r0 + k * L];
            }
            double Mq[12][R], Mp[12][R], aq[R], ap[R];
            dp::static_for<0, 12>([&](auto sc) {
                constexpr int s = decltype(sc)::value;
                double wq[R], wp[R];
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    double sq = 0.0, sp_ = 0.0;
                    dp::static_for<0, s>([&](auto jc) {
                        constexpr int j = decltype(jc)::value;
                        constexpr double c = dp::kA[s][j];
                        if constexpr (c != 0.0) {
                            sq = fma(c, Mq[j][k], sq);
                            sp_ = fma(c, Mp[j][k], sp_);
                        }
                    });
                    wq[k] = (s == 0) ? q[k] : fma(h, sq, q[k]);
                    wp[k] = (s == 0) ? p[k] : fma(h, sp_, p[k]);
                }
                // neighbours of row r = r0 + k L in the column (walls: 0)
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    double left = __shfl_up_sync(0xffffffffu, wq[k], 1, L);
                    double right = __shfl_down_sync(0xffffffffu, wq[k], 1, L);
                    if constexpr (R > 1) {
                        // row blocks wrap from lane L-1 of block k-1 / lane 0 of block k+1
                        const double prev_last = __shfl_sync(0xffffffffu, wq[k > 0 ? k - 1 : 0], L - 1, L);
                        const double next_first = __shfl_sync(0xffffffffu, wq[k < R - 1 ? k + 1 : 0], 0, L);
                        if (r0 == 0) left = k > 0 ? prev_last : 0.0;
                        if (r0 == L - 1) right = k < R - 1 ? next_first : 0.0;
                    } else {
                        if (r0 == 0) left = 0.0;
                        if (r0 == L - 1) right = 0.0;
                    }
                    const int r = r0 + k * L;
                    const double cl = c_s[s * (N + 1) + r], cr = c_s[s * (N + 1) + r + 1];
                    Mq[s][k] = wp[k];
                    Mp[s][k] = fma(cr, right - wq[k], -cl * (wq[k] - left));
                }
                constexpr double cb = dp::kB[s];
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    if constexpr (s == 0) {
                        aq[k] = cb * Mq[0][k];
                        ap[k] = cb * Mp[0][k];
                    } else if constexpr (cb != 0.0) {
                        aq[k] = fma(cb, Mq[s][k], aq[k]);
                        ap[k] = fma(cb, Mp[s][k], ap[k]);
                    }
                }
            });
#pragma unroll
            for (int k = 0; k < R; ++k) {
                Wc[r0 + k * L] = fma(h, aq[k], q[k]);
                Wc[N + r0 + k * L] = fma(h, ap[k], p[k]);
            }
        }
        __syncthreads();  // W complete; stage stiffnesses free

        if (--until_qr == 0 || step == a.n_steps) {
            until_qr = a.qr_every;
            double* wl = W + l * WS;
            double inv = 1.0;
            for (int j = 0; j < D; ++j) {
                const double* wj = W + j * WS;
                double r = 0.0;
                if (l >= j) {
                    double r0a = 0.0, r1a = 0.0;
#pragma unroll 4
                    for (int i = 0; i < D; i += 2) {
                        r0a = fma(wj[i], wl[i], r0a);
                        r1a = fma(wj[i + 1], wl[i + 1], r1a);
                    }
                    r = r0a + r1a;
                }
                if (l == j) red[0] = r;
                __syncthreads();
                const double nj = red[0];
                if (l > j) {
                    const double cfac = -r / nj;
#pragma unroll 4
                    for (int i = 0; i < D; ++i) wl[i] = fma(cfac, wj[i], wl[i]);
                } else if (l == j) {
                    S += 0.5 * log(nj);
                    inv = rsqrt(nj);
                }
                __syncthreads();
            }
#pragma unroll 4
            for (int i = 0; i < D; ++i) wl[i] *= inv;
            __syncthreads();
        }
        if (--until == 0) {
            until = a.sample_every;
            if (orbit_any(!(isfinite(xi) && isfinite(S))) && st == CHS_ORBIT_OK) st = CHS_ORBIT_NONFINITE;
        }
    }
    if (valid) {
        const double T = (double)a.n_steps * a.dt;
        lambda[(int64_t)l * n + o] =
            (st == CHS_ORBIT_OK) ? S / T : __longlong_as_double(0x7ff8000000000000LL);
        if (l == 0) status_out[o] = st;
    }
}

template <int N>
cudaError_t prepare_dp_n()
{
    static bool done = false;  // idempotent; set before any stream capture
    if (done) return cudaSuccess;
    const cudaError_t err = cudaFuncSetAttribute(k_fput_lyap_dp<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)FputDpCfg<N>::SMEM);
    if (err == cudaSuccess) done = true;
    return err;
}

template <int N>
cudaError_t fput_dp_n(const SysPar& sp, const StepArgs& a, int64_t n, const double* ics,
                      const int32_t* ic_status, double* lambda, int32_t* status, cudaStream_t st)
{
    using Cfg = FputDpCfg<N>;
    const cudaError_t err = prepare_dp_n<N>();
    if (err != cudaSuccess) return err;
    k_fput_lyap_dp<N><<<blocks_for(n, Cfg::G), Cfg::THREADS, Cfg::SMEM, st>>>(a, sp, n, ics, ic_status,
                                                                             lambda, status);
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

}  // namespace chs

// fput_stages.cuh -- building blocks of the FPUT kernels that run explicit
// Runge-Kutta stages on the chain (k_fput_dp.cu: Lyapunov spectra with DOP853;
// k_fput_ens.cu: ensembles with k deviation vectors, RK4 or DOP853).
//
// A step runs in two phases:
//   phase 1  the orbit: thread l of the orbit's 2N threads owns component l and
//            its stage derivatives (in registers); the stage states pass
//            through a double-buffered shared array (one barrier per stage),
//            and each stage leaves its N + 1 bond stiffnesses V''(D_b) behind;
//   phase 2  the deviation vectors (columns), one at a time per warp segment:
//            L = min(N, 32) lanes split the column's N (q, p) row pairs, keep
//            the column's stage derivatives in registers and exchange the
//            tridiagonal neighbours q_{i-1}, q_{i+1} by warp shuffles.  No
//            barrier and no stage storage in memory.
// Bonds: D_b = q_b - q_{b-1}, b = 0..N, with walls q_{-1} = q_N = 0.
#pragma once

#include "dop853.cuh"

namespace chs {
namespace fs {

// Butcher tableaus as compile-time coefficients.
struct TabRk4 {  // classic RK4
    static constexpr int S = 4;
    template <int s, int j>
    static constexpr double A = (s == 1 && j == 0) ? 0.5 : (s == 2 && j == 1) ? 0.5 : (s == 3 && j == 2) ? 1.0 : 0.0;
    template <int s>
    static constexpr double B = (s == 0 || s == 3) ? 1.0 / 6.0 : 1.0 / 3.0;
};

struct TabDop853 {  // the DOP853 pair (dop853.cuh), with its error weights
    static constexpr int S = 12;
    template <int s, int j>
    static constexpr double A = dp::kA[s][j];
    template <int s>
    static constexpr double B = dp::kB[s];
    template <int s>
    static constexpr double E5 = dp::kE5[s];
    template <int s>
    static constexpr double E3 = dp::kB[s] - dp::kB3[s];
};

struct Coef {
    double k, a2, b3;  // V''(r) = k + 2 alpha r + 3 beta r^2
    double alpha, beta;
};

__device__ __forceinline__ Coef coef_of(const SysPar& sp)
{
    return Coef{sp.kk, 2.0 * sp.alpha, 3.0 * sp.beta, sp.alpha, sp.beta};
}

__device__ __forceinline__ double dv(const Coef& fc, double r)
{
    return r * fma(r, fma(fc.beta, r, fc.alpha), fc.k);  // V'(r)
}

__device__ __forceinline__ double d2v(const Coef& fc, double r)
{
    return fma(r, fma(fc.b3, r, fc.a2), fc.k);  // V''(r)
}

// Phase 1 for component l of one orbit (every thread of the block calls it; one
// barrier per stage).  xb: [2][2N] stage-state buffers; cs: [S][N + 1] stage
// stiffnesses.  Returns x_l + h sum_s b_s F_s; with ERR the error sums
// err5 = sum_s e5_s F_s and err3 = sum_s (b_s - b3_s) F_s (DOP853 only).  With
// GUARD a thread whose `act` is false (a block wider than the orbit's 2N
// threads) only meets the barriers and returns xi.
template <int N, class Tab, bool ERR, bool GUARD = false>
__device__ __forceinline__ double orbit_stages(const double xi, const double h, const int l, double* xb,
                                               double* cs, const Coef& fc, double& e5, double& e3,
                                               const bool act = true)
{
    constexpr int D = 2 * N;
    double F[Tab::S] = {};
    double acc = 0.0, a5 = 0.0, a3 = 0.0;
    dp::static_for<0, Tab::S>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        if constexpr (GUARD) {
            if (!act) {
                __syncthreads();
                return;
            }
        }
        double sum = 0.0;
        dp::static_for<0, s>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            constexpr double c = Tab::template A<s, j>;
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
            f = dv(fc, qp - q0) - dv(fc, q0 - qm);
        }
        if (l <= N) {
            const double qa = l < N ? xs[l] : 0.0;
            const double qb = l > 0 ? xs[l - 1] : 0.0;
            cs[s * (N + 1) + l] = d2v(fc, qa - qb);
        }
        F[s] = f;
        constexpr double cb = Tab::template B<s>;
        if constexpr (s == 0) {
            acc = cb * f;
        } else if constexpr (cb != 0.0) {
            acc = fma(cb, f, acc);
        }
        if constexpr (ERR) {
            constexpr double c5 = Tab::template E5<s>, c3 = Tab::template E3<s>;
            if constexpr (s == 0) {
                a5 = c5 * f;
                a3 = c3 * f;
            } else {
                if constexpr (c5 != 0.0) a5 = fma(c5, f, a5);
                if constexpr (c3 != 0.0) a3 = fma(c3, f, a3);
            }
        }
    });
    if constexpr (ERR) {
        e5 = a5;
        e3 = a3;
    }
    if constexpr (GUARD) {
        if (!act) return xi;
    }
    return fma(h, acc, xi);
}

// Lanes per column and columns per warp of phase 2.
template <int N>
struct ColShape {
    static constexpr int L = N < 32 ? N : 32;  // lanes per column
    static constexpr int R = N / L;            // row pairs per lane
    static constexpr int CPW = 32 / L;         // columns per warp at a time
};

// Phase 2: the kc columns of every orbit of the block (G orbits, each orbit's
// slab at smem + g * PER, column c at + c * WS, stiffnesses at + CS) advance
// through the stages of w' = J_s w with step step_of(g, slab); a step of 0
// leaves the columns untouched, and with SKIP a warp whose segments all have
// step 0 skips the work (callers whose steps are never 0 leave SKIP off: the
// vote changes the register allocation of the stage loop).  With renorm set
// every updated column is scaled to unit length.  Every lane of every warp must call this: the segments of a warp
// loop together (a segment past the last column computes on column 0 of orbit
// 0 with step 0), so the shuffles always run on full warps.
template <int N, class Tab, int G, int PER, int WS, int CS, bool SKIP, class StepOf>
__device__ __forceinline__ void columns(double* smem, const int kc, StepOf step_of, const int renorm = 0)
{
    constexpr int L = ColShape<N>::L, R = ColShape<N>::R, CPW = ColShape<N>::CPW;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int nwarps = blockDim.x / 32;
    const int seg = lane / L, r0 = lane % L;
    const int total = G * kc;
    for (int base = warp * CPW; base < total; base += nwarps * CPW) {
        const int task = base + seg;
        const bool real = task < total;
        const int og = real ? task / kc : 0, col = real ? task % kc : 0;
        double* slab = smem + og * PER;
        const double h = real ? step_of(og, slab) : 0.0;
        if constexpr (SKIP) {
            if (!__any_sync(0xffffffffu, h != 0.0)) continue;
        }
        double* Wc = slab + col * WS;
        const double* c_s = slab + CS;
        double q[R], p[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            q[k] = Wc[r0 + k * L];
            p[k] = Wc[N + r0 + k * L];
        }
        double Mq[Tab::S][R], Mp[Tab::S][R], aq[R], ap[R];
        dp::static_for<0, Tab::S>([&](auto sc) {
            constexpr int s = decltype(sc)::value;
            double wq[R], wp[R];
#pragma unroll
            for (int k = 0; k < R; ++k) {
                double sq = 0.0, sp_ = 0.0;
                dp::static_for<0, s>([&](auto jc) {
                    constexpr int j = decltype(jc)::value;
                    constexpr double c = Tab::template A<s, j>;
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
            constexpr double cb = Tab::template B<s>;
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
        double nq[R], np[R];
        double n2 = 0.0;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            nq[k] = fma(h, aq[k], q[k]);
            np[k] = fma(h, ap[k], p[k]);
            n2 = fma(nq[k], nq[k], fma(np[k], np[k], n2));
        }
        if (renorm) {
            // |w|^2 over the segment's lanes (the same sum in every lane)
#pragma unroll
            for (int off = L / 2; off > 0; off >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, off, L);
            const double inv = 1.0 / sqrt(n2);
#pragma unroll
            for (int k = 0; k < R; ++k) {
                nq[k] *= inv;
                np[k] *= inv;
            }
        }
        if (h > 0.0 || h < 0.0) {
#pragma unroll
            for (int k = 0; k < R; ++k) {
                Wc[r0 + k * L] = nq[k];
                Wc[N + r0 + k * L] = np[k];
            }
        }
    }
}

}  // namespace fs
}  // namespace chs

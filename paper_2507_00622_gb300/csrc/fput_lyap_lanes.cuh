// fput_lyap_lanes.cuh -- the FPUT Lyapunov spectrum by periodic QR for N = 4, 8
// (RK4, L lanes of one warp per orbit), as the work of one block:
// k_fput_lanes.cu launches it block by block, the mixed-chain persistent kernel
// (k_fput_batch.cu) runs it from a work queue.
//
// The method is the one of fput_lyap_rk4.cuh (RK4 on the chain, the 2N deviation
// vectors advanced by the exact one-step RK4 propagator Phi, modified
// Gram-Schmidt every qr_every steps and at the last step, S_j += ln |w_j|).
// What changes is how an orbit is spread over threads: L lanes per orbit (four
// at N = 4 and eight at N = 8 by default; one or two at N = 4 and two or four at
// N = 8 are offered to the tuner), and every choice gives the same results bit
// for bit: each bond, row and column is computed by the same operations
// whichever lane owns it, and the products that feed a sum are rounded
// explicitly (__dmul_rn), so that the compiler cannot fuse them into a
// multiply-add in one instantiation and not in another.  GB300 executes FP64
// instructions per warp at a fixed rate whatever the number of active lanes,
// and each of an SM's four sub-partitions has its own FP64 unit, so the
// kernel must (a) never execute FP64 work with idle lanes and (b) give every
// sub-partition a warp, two where it can (a warp's own shared-memory loads and
// address arithmetic then overlap the other warp's FP64 work).  An ensemble of
// 4096 orbits has 512 warps at four lanes per orbit (N = 4) and 1024 at eight
// (N = 8).  Lane `sub` of an orbit owns
//   masses i0 .. i0 + M - 1 (i0 = sub * M, M = N / L): their RK4 stages, the
//     bonds around them, and rows i0 .. i0 + M - 1 of Phi;
//   columns sub + L m of W (m < CPL = 2N / L): their propagation, and their
//     part of the QR (columns interleaved over the lanes so that every lane
//     keeps work until the last Gram-Schmidt column).
// The orbit's lanes sit in one warp: neighbours' positions and bond
// stiffnesses pass by shuffles, shared-memory hand-offs are ordered by
// __syncwarp, and no block barrier is needed.
//
// Shared memory per orbit: W (2N x 2N) and the 18 band coefficients of every
// row of Phi, laid out with the block's orbits innermost (element e of orbit
// g at [e * G + g]) so that a warp's accesses fall in distinct banks.
//
// The band rows of Phi come from fput_phi.cuh.
#pragma once

#include <math.h>

#include "chs_internal.cuh"
#include "fput_phi.cuh"

namespace chs {
namespace lanes {

constexpr unsigned kFull = 0xffffffffu;

template <int N, int T, int L_ = 4>
struct LaneCfg {
    static constexpr int L = L_;       // lanes per orbit
    static constexpr int D = 2 * N;
    static constexpr int M = N / L;    // masses and rows of Phi per lane
    static constexpr int CPL = D / L;  // columns of W per lane
    static constexpr int G = T / L;    // orbits per block
    static constexpr int ROW = 18;     // band coefficients per row of Phi
    static_assert(N % L == 0 && 32 % L == 0 && T % 32 == 0 && T <= 128,
                  "whole masses per lane, an orbit's lanes in one warp, whole warps per block");
    static constexpr size_t SMEM = (size_t)(D * D + N * ROW) * G * sizeof(double);
};

// The work of one block of T threads: the G = T / L orbits vb * G .. vb * G +
// G - 1 (those below n), in the shared memory `smem` (LaneCfg::SMEM bytes).
// Every thread of the block calls it; it synchronises only within warps.
template <int N, int T, bool ALPHA0, int LL = 4>
__device__ __forceinline__ void fput_lyap_lanes_block(const StepArgs& a, const SysPar& sp, const int64_t n,
                                                      const double* __restrict__ ics,
                                                      const int32_t* __restrict__ ic_status,
                                                      double* __restrict__ lambda,
                                                      int32_t* __restrict__ status_out, const int64_t vb,
                                                      double* smem)
{
    using C = LaneCfg<N, T, LL>;
    constexpr int L = C::L, D = C::D, M = C::M, CPL = C::CPL, G = C::G, ROW = C::ROW;
    const int g = threadIdx.x / L, sub = threadIdx.x % L;
    const int64_t o = vb * G + g;
    const bool valid = o < n;
    const int i0 = sub * M;
    const unsigned gbits = ((1u << L) - 1u) << ((threadIdx.x & 31) & ~(L - 1));  // this orbit's lanes
    double* W = smem;               // W(i, c) at W[(i * D + c) * G + g]
    double* cf = smem + D * D * G;  // row r, entry e of Phi at cf[(r * ROW + e) * G + g]
#define WAT(i, c) W[((i) * D + (c)) * G + g]

    const double kk = sp.kk, al = sp.alpha, be = sp.beta, a2 = 2.0 * sp.alpha, b3 = 3.0 * sp.beta;
    auto orbit_any = [&](bool pred) { return (__ballot_sync(kFull, pred) & gbits) != 0u; };

    int32_t st = valid ? (ic_status ? ic_status[o] : CHS_ORBIT_OK) : CHS_ORBIT_FORBIDDEN;
    double xq[M], xp[M];
    bool bad = false;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        xq[k] = valid ? ics[(int64_t)(i0 + k) * n + o] : 0.0;
        xp[k] = valid ? ics[(int64_t)(N + i0 + k) * n + o] : 0.0;
        bad = bad || !isfinite(xq[k]) || !isfinite(xp[k]);
    }
    if (orbit_any(bad) && st == CHS_ORBIT_OK) st = CHS_ORBIT_NONFINITE;
    if (st != CHS_ORBIT_OK) {
#pragma unroll
        for (int k = 0; k < M; ++k) xq[k] = xp[k] = 0.0;
    }
#pragma unroll
    for (int m = 0; m < CPL; ++m) {
        const int c = sub + m * L;
#pragma unroll
        for (int i = 0; i < D; ++i) WAT(i, c) = (i == c) ? 1.0 : 0.0;
    }
    double S[CPL];
#pragma unroll
    for (int m = 0; m < CPL; ++m) S[m] = 0.0;
    __syncwarp();

    const double h = a.dt;
    int64_t until_qr = a.qr_every;
    int64_t until = a.sample_every > 0 ? a.sample_every : -1;
    const long long t_start = clock64();
    for (int64_t s = 1; s <= a.n_steps; ++s) {
        // RK4 of the orbit; cw[k][u] = stiffness of bond i0 - 1 + u at stage k
        double qs[M], ps[M], aq[M], ap[M], cw[4][M + 3];
#pragma unroll
        for (int k = 0; k < M; ++k) {
            qs[k] = xq[k];
            ps[k] = xp[k];
        }
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) {
            const double qL = __shfl_up_sync(kFull, qs[M - 1], 1, L);
            const double qR = __shfl_down_sync(kFull, qs[0], 1, L);
            const double ql = sub == 0 ? 0.0 : qL;
            const double qr = sub == L - 1 ? 0.0 : qR;
            double rb[M + 1], xb[M + 1];  // bond stretch r and V'(r) / r
#pragma unroll
            for (int t = 0; t <= M; ++t) {  // bond i0 + t joins masses i0 + t - 1 and i0 + t
                const double r = (t < M ? qs[t] : qr) - (t > 0 ? qs[t - 1] : ql);
                rb[t] = r;
                if constexpr (ALPHA0) {
                    const double r2 = r * r;
                    xb[t] = fma(be, r2, kk);
                    cw[k4][t + 1] = fma(b3, r2, kk);
                } else {
                    xb[t] = fma(r, fma(be, r, al), kk);
                    cw[k4][t + 1] = fma(r, fma(b3, r, a2), kk);
                }
            }
            const double cs = k4 == 2 ? h : 0.5 * h;
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const double kq = ps[k];
                // force V'(r_right) - V'(r_left), the left term rounded on its own
                // and the right one fused: one form whatever the lane count
                const double kp = fma(rb[k + 1], xb[k + 1], -__dmul_rn(rb[k], xb[k]));
                if (k4 == 0) {
                    aq[k] = kq;
                    ap[k] = kp;
                } else {
                    const double w = k4 == 3 ? 1.0 : 2.0;
                    aq[k] = fma(w, kq, aq[k]);
                    ap[k] = fma(w, kp, ap[k]);
                }
                if (k4 < 3) {
                    qs[k] = fma(cs, kq, xq[k]);
                    ps[k] = fma(cs, kp, xp[k]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < M; ++k) {
            xq[k] = fma(h / 6.0, aq[k], xq[k]);
            xp[k] = fma(h / 6.0, ap[k], xp[k]);
        }
        // bonds i0 - 1 and i0 + M + 1 from the neighbouring lanes (none beyond the walls)
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) {
            const double cl = __shfl_up_sync(kFull, cw[k4][M], 1, L);
            const double cr = __shfl_down_sync(kFull, cw[k4][2], 1, L);
            cw[k4][0] = sub == 0 ? 0.0 : cl;
            cw[k4][M + 2] = sub == L - 1 ? 0.0 : cr;
        }
        __syncwarp();  // every lane is done reading the previous step's rows
#pragma unroll
        for (int k = 0; k < M; ++k) {
            double cb[4][4], row[ROW];
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4)
#pragma unroll
                for (int t = 0; t < 4; ++t) cb[k4][t] = cw[k4][k + t];
            fput_phi::phi_row<N>(i0 + k, cb, h, row);
#pragma unroll
            for (int e = 0; e < ROW; ++e) cf[((i0 + k) * ROW + e) * G + g] = row[e];
        }
        __syncwarp();  // the rows of Phi are complete
        // w <- Phi w for the lane's columns, AC at a time: each row's band
        // coefficients are loaded once for the AC columns (the arithmetic of
        // every column is the same whatever AC).  Two where the two columns'
        // u and v fit the registers beside the rest (N = 4, or two columns per
        // lane), else one.
        constexpr int AC = (CPL % 2 == 0 && (N <= 4 || CPL <= 2)) ? 2 : 1;
#pragma unroll 1
        for (int m0 = 0; m0 < CPL; m0 += AC) {
            double u[AC][N], v[AC][N];
#pragma unroll
            for (int q = 0; q < AC; ++q)
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    u[q][i] = WAT(i, sub + (m0 + q) * L);
                    v[q][i] = WAT(N + i, sub + (m0 + q) * L);
                }
#pragma unroll
            for (int i = 0; i < N; ++i) {
                double k[ROW];
#pragma unroll
                for (int e = 0; e < ROW; ++e) k[e] = cf[(i * ROW + e) * G + g];
#pragma unroll
                for (int q = 0; q < AC; ++q) {
                    double nu = 0.0, nv = 0.0;
                    bool first = true;
#pragma unroll
                    for (int t = 0; t < 5; ++t) {  // A and C on u_{i-2..i+2}
                        const int j = i - 2 + t;
                        if (j < 0 || j >= N) continue;
                        nu = first ? __dmul_rn(k[t], u[q][j]) : fma(k[t], u[q][j], nu);
                        nv = first ? __dmul_rn(k[8 + t], u[q][j]) : fma(k[8 + t], u[q][j], nv);
                        first = false;
                    }
#pragma unroll
                    for (int t = 0; t < 3; ++t) {  // B on v_{i-1..i+1}
                        const int j = i - 1 + t;
                        if (j < 0 || j >= N) continue;
                        nu = fma(k[5 + t], v[q][j], nu);
                    }
#pragma unroll
                    for (int t = 0; t < 5; ++t) {  // D on v_{i-2..i+2}
                        const int j = i - 2 + t;
                        if (j < 0 || j >= N) continue;
                        nv = fma(k[13 + t], v[q][j], nv);
                    }
                    WAT(i, sub + (m0 + q) * L) = nu;
                    WAT(N + i, sub + (m0 + q) * L) = nv;
                }
            }
        }

        if (--until_qr == 0 || s == a.n_steps) {
            until_qr = a.qr_every;
            // modified Gram-Schmidt: for column j, every column c >= j forms
            // r_c = w_j . w_c; the columns c > j subtract (r_c / r_j) w_j; the
            // columns are scaled to unit length at the end, S_c += ln |w_c|
            double nrm[CPL];
#pragma unroll
            for (int m = 0; m < CPL; ++m) nrm[m] = 1.0;
#pragma unroll
            for (int jm = 0; jm < CPL; ++jm) {
#pragma unroll 1
                for (int js = 0; js < L; ++js) {
                    const int j = js + jm * L;
                    __syncwarp();  // column j is final
                    double r[CPL];
#pragma unroll
                    for (int m = jm; m < CPL; ++m) {
                        r[m] = 0.0;
                        if (m > jm || sub >= js) {
                            const int c = sub + m * L;
                            double s0 = 0.0, s1 = 0.0;
#pragma unroll
                            for (int i = 0; i < D; i += 2) {
                                s0 = fma(WAT(i, j), WAT(i, c), s0);
                                s1 = fma(WAT(i + 1, j), WAT(i + 1, c), s1);
                            }
                            r[m] = s0 + s1;
                        }
                    }
                    const double nj = __shfl_sync(kFull, r[jm], js, L);  // |w_j|^2 from its lane
                    if (sub == js) nrm[jm] = nj;
                    const double y = rsqrt(nj);
                    const double inv2 = y * y;
#pragma unroll
                    for (int m = jm; m < CPL; ++m) {
                        if (m > jm || sub > js) {
                            const int c = sub + m * L;
                            const double f = -r[m] * inv2;
#pragma unroll
                            for (int i = 0; i < D; ++i) WAT(i, c) = fma(f, WAT(i, j), WAT(i, c));
                        }
                    }
                }
            }
#pragma unroll
            for (int m = 0; m < CPL; ++m) {
                const int c = sub + m * L;
                S[m] += 0.5 * log(nrm[m]);
                const double inv = rsqrt(nrm[m]);
#pragma unroll
                for (int i = 0; i < D; ++i) WAT(i, c) *= inv;
            }
        }
        __syncwarp();  // W is final for the next step
        if (--until == 0) {
            until = a.sample_every;
            bool b = false;
#pragma unroll
            for (int k = 0; k < M; ++k) b = b || !isfinite(xq[k]) || !isfinite(xp[k]);
#pragma unroll
            for (int m = 0; m < CPL; ++m) b = b || !isfinite(S[m]);
            if (orbit_any(b) && st == CHS_ORBIT_OK) st = CHS_ORBIT_NONFINITE;
            // warp-uniform: the warp's orbits stop together
            if (a.clock_budget > 0 && __any_sync(kFull, budget_spent(a, t_start))) {
                if (st == CHS_ORBIT_OK) st = CHS_ORBIT_STEP_BUDGET;
                break;
            }
        }
    }
#undef WAT
    if (valid) {
        const double t_total = (double)a.n_steps * a.dt;
#pragma unroll
        for (int m = 0; m < CPL; ++m)
            lambda[(int64_t)(sub + m * L) * n + o] =
                (st == CHS_ORBIT_OK) ? S[m] / t_total : __longlong_as_double(0x7ff8000000000000LL);
        if (sub == 0) status_out[o] = st;
    }
}

}  // namespace lanes
}  // namespace chs

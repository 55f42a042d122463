// fput_lyap_n64.cuh -- the FPUT Lyapunov spectrum at N = 64 (d = 128, RK4) with
// two threads per column of W: 256 threads, one orbit per block.
//
// At N = 64 the matrix W (128 KB) leaves room for one orbit per SM, so the
// 128-thread body of fput_lyap_rk4.cuh gives each sub-partition's FP64 unit a
// single warp, and that warp's shared-memory loads, address arithmetic and
// barriers run while the unit waits (measured: 24k instructions per step per
// warp, 3.1k of them FP64; FP64 pipe 69 % active).  With two warps per
// sub-partition one warp's FP64 work covers the other's remaining instructions.
//
// The arithmetic is that of the 128-thread body step for step -- the same band
// rows, the same FMA order in every row of the propagation, the same partial
// dot products summed in the same order -- so the two bodies give identical
// results; only the assignment of work to threads differs:
//   propagation: thread t takes column t % 128 and the masses 32 h .. 32 h + 31
//     (h = t / 128); the two rows of u and of v beyond its half that its band
//     window needs are read before the barrier that precedes the writes;
//   QR: warp w takes rows 32 (w % 4) .. 32 (w % 4) + 31 of the column groups
//     m = w / 4 and m = w / 4 + 2 (columns lane + 32 m); the two warps sharing
//     a row block meet at a named barrier before each pivot;
//   RK4 of the orbit, band rows, exponents, output: the first 128 threads, as
//     in the 128-thread body.
#pragma once

#include "fput_lyap_rk4.cuh"

namespace chs {
namespace n64 {

constexpr int N = 64, D = 128, THREADS = 256;
using Cfg = FputLyapCfg<N, 128>;  // the shared-memory layout of one orbit
static_assert(Cfg::WS == D && Cfg::Q == 4 && Cfg::G == 1, "one orbit, rows of 128, four row blocks");
constexpr size_t SMEM = Cfg::SMEM;

// the two warps of row block rb (warps rb and rb + 4): named barrier 1 + rb
__device__ __forceinline__ void pair_sync(const int rb)
{
    asm volatile("bar.sync %0, 64;" ::"r"(1 + rb) : "memory");
}

// Partial dot products w_j . w_c over the rows of block rb for the groups
// CH and CH + 2 that are not finished (m >= M0 = j / 32).
template <int M0, int CH>
__device__ __forceinline__ void dots(const double* __restrict__ W, double* __restrict__ Pb, const int j,
                                     const int rb, const int lane)
{
    constexpr bool A = CH >= M0, B = CH + 2 >= M0;
    if constexpr (A || B) {
        const int r0 = 32 * rb, ca = lane + 32 * CH, cb = lane + 32 * (CH + 2);
        double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
#pragma unroll 4
        for (int i = 0; i < 32; i += 2) {
            const double wj0 = W[(r0 + i) * D + j], wj1 = W[(r0 + i + 1) * D + j];
            if constexpr (A) {
                a0 = fma(wj0, W[(r0 + i) * D + ca], a0);
                a1 = fma(wj1, W[(r0 + i + 1) * D + ca], a1);
            }
            if constexpr (B) {
                b0 = fma(wj0, W[(r0 + i) * D + cb], b0);
                b1 = fma(wj1, W[(r0 + i + 1) * D + cb], b1);
            }
        }
        if constexpr (A) Pb[rb * D + ca] = a0 + a1;
        if constexpr (B) Pb[rb * D + cb] = b0 + b1;
    }
}

// w_c -= (r_c / r_j) w_j on the rows of block rb for the columns c > j of the
// groups CH and CH + 2.
template <int M0, int CH>
__device__ __forceinline__ void axpy(double* __restrict__ W, const double* __restrict__ Pb, const int j,
                                     const double inv_nj, const int rb, const int lane)
{
    constexpr bool A = CH >= M0, B = CH + 2 >= M0;
    if constexpr (A || B) {
        const int r0 = 32 * rb, ca = lane + 32 * CH, cb = lane + 32 * (CH + 2);
        auto coef = [&](int c) {
            double r = Pb[c];
#pragma unroll
            for (int q = 1; q < 4; ++q) r += Pb[q * D + c];
            return -r * inv_nj;
        };
        const double fa = A ? coef(ca) : 0.0, fb = B ? coef(cb) : 0.0;
        // a group above M0 lies wholly right of j; in group M0 only c > j moves
        const bool wa = A && (CH > M0 || ca > j), wb = B && (CH + 2 > M0 || cb > j);
#pragma unroll 4
        for (int i = 0; i < 32; ++i) {
            const double wj = W[(r0 + i) * D + j];
            if constexpr (A) {
                const double v = fma(fa, wj, W[(r0 + i) * D + ca]);
                if (wa) W[(r0 + i) * D + ca] = v;
            }
            if constexpr (B) {
                const double v = fma(fb, wj, W[(r0 + i) * D + cb]);
                if (wb) W[(r0 + i) * D + cb] = v;
            }
        }
    }
}

// w <- Phi w for column l, masses i0 .. i0 + 31 (i0 = 32 h), in place.  hu[k],
// hv[k] are the old rows of u and v beyond this half that the window reaches:
// rows 30, 31 for h = 1 (below), rows 32, 33 for h = 0 (above).
__device__ __forceinline__ void apply_half(double* __restrict__ W, const double* __restrict__ cf, const int l,
                                           const int h, const double (&hu)[2], const double (&hv)[2])
{
    const int i0 = 32 * h;
    auto U = [&](int i) { return W[i * D + l]; };
    auto V = [&](int i) { return W[(N + i) * D + l]; };
    double u0 = h ? hu[0] : 0.0, u1 = h ? hu[1] : 0.0, u2 = U(i0), u3 = U(i0 + 1), u4 = U(i0 + 2);
    double v0 = h ? hv[0] : 0.0, v1 = h ? hv[1] : 0.0, v2 = V(i0), v3 = V(i0 + 1), v4 = V(i0 + 2);
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const int i = i0 + k;
        const double* c = cf + i * 18;
        double nu = c[0] * u0;
        nu = fma(c[1], u1, nu);
        nu = fma(c[2], u2, nu);
        nu = fma(c[3], u3, nu);
        nu = fma(c[4], u4, nu);
        nu = fma(c[5], v1, nu);
        nu = fma(c[6], v2, nu);
        nu = fma(c[7], v3, nu);
        double nv = c[8] * u0;
        nv = fma(c[9], u1, nv);
        nv = fma(c[10], u2, nv);
        nv = fma(c[11], u3, nv);
        nv = fma(c[12], u4, nv);
        nv = fma(c[13], v0, nv);
        nv = fma(c[14], v1, nv);
        nv = fma(c[15], v2, nv);
        nv = fma(c[16], v3, nv);
        nv = fma(c[17], v4, nv);
        W[i * D + l] = nu;
        W[(N + i) * D + l] = nv;
        // the next row of the window: own rows, the other half's old rows 32, 33
        // (h = 0), zero past the chain's end (h = 1)
        const int nx = k + 3;
        double un = 0.0, vn = 0.0;
        if (nx < 32) {
            un = U(i0 + nx);
            vn = V(i0 + nx);
        } else if (nx < 34) {
            un = h ? 0.0 : hu[nx - 32];
            vn = h ? 0.0 : hv[nx - 32];
        }
        u0 = u1; u1 = u2; u2 = u3; u3 = u4; u4 = un;
        v0 = v1; v1 = v2; v2 = v3; v3 = v4; v4 = vn;
    }
}

// The work of one block of 256 threads: orbit vb (if below n), in the shared
// memory `smem` (SMEM bytes).  Every thread of the block calls it.
__device__ __forceinline__ void fput_lyap_block_n64(const StepArgs& a, const SysPar& sp, const int64_t n,
                                                    const double* __restrict__ ics,
                                                    const int32_t* __restrict__ ic_status,
                                                    double* __restrict__ lambda, int32_t* __restrict__ status_out,
                                                    const int64_t vb, double* smem)
{
    constexpr int WS = Cfg::WS, Q = Cfg::Q;
    const int t = threadIdx.x;
    const int l = t % D, hh = t / D;           // column and mass half of the propagation
    const int w = t / 32, lane = t % 32;
    const int rb = w % 4, ch = w / 4;          // row block and column groups of the QR
    const bool lead = t < D;                   // the threads of the 128-thread body
    const int64_t o = vb;
    const bool valid = o < n;
    double* W = smem;
    double* cf = W + D * WS;
    double* xs = cf + 18 * N;
    double* cs = xs + D;
    double* red = cs + 4 * (N + 1);
    double* qp = red + 2;
    double* Sv = qp + 2 * Q * D;
    double* nrm = Sv + D;

    const FputCoef fc = {sp.kk, 2.0 * sp.alpha, 3.0 * sp.beta, sp.alpha, sp.beta};
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
    for (int i = 64 * hh; i < 64 * hh + 64; ++i) W[i * WS + l] = (i == l) ? 1.0 : 0.0;
    if (lead) {
        xs[l] = xi;
        Sv[l] = 0.0;
    }
    double S = 0.0;
    __syncthreads();

    const double h = a.dt;
    int64_t until_qr = a.qr_every;
    int64_t until = a.sample_every > 0 ? a.sample_every : -1;
    const long long t_start = clock64();
    for (int64_t s = 1; s <= a.n_steps; ++s) {
        // RK4 of the orbit (first 128 threads); stage stiffnesses for Phi
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double fi = 0.0;
            if (lead) {
                if (l < N) {
                    fi = xs[N + l];
                } else {
                    const int i = l - N;
                    const double qm = i > 0 ? xs[i - 1] : 0.0;
                    const double q0 = xs[i];
                    const double qpn = i < N - 1 ? xs[i + 1] : 0.0;
                    const double rr = qpn - q0, rl = q0 - qm;
                    fi = fma(rr, fput_dv_over_r(fc, rr), -__dmul_rn(rl, fput_dv_over_r(fc, rl)));
                }
                if (l <= N) {
                    const double qa = l < N ? xs[l] : 0.0;
                    const double qb = l > 0 ? xs[l - 1] : 0.0;
                    cs[k * (N + 1) + l] = fput_d2v(fc, qa - qb);
                }
            }
            __syncthreads();
            if (lead) {
                acc = (k == 0) ? fi : fma((k == 3) ? 1.0 : 2.0, fi, acc);
                if (k < 3) xs[l] = fma(k == 2 ? h : 0.5 * h, fi, xi);
            }
            __syncthreads();
        }
        if (lead) {
            xi = fma(h / 6.0, acc, xi);
            xs[l] = xi;
        }
        // the other half's old rows reached by this half's band window, read
        // before the barrier after which the propagation writes
        double hu[2], hv[2];
        {
            const int r = hh ? 30 : 32;
            hu[0] = W[r * WS + l];
            hu[1] = W[(r + 1) * WS + l];
            hv[0] = W[(N + r) * WS + l];
            hv[1] = W[(N + r + 1) * WS + l];
        }
        if (lead && l < N) {
            double cb[4][4];  // stiffnesses of bonds l - 1 .. l + 2 (none beyond the walls)
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int b = l - 1 + u;
                    cb[k][u] = (b >= 0 && b <= N) ? cs[k * (N + 1) + b] : 0.0;
                }
            fput_phi::phi_row<N>(l, cb, h, cf + l * 18);
        }
        __syncthreads();
        apply_half(W, cf, l, hh, hu, hv);

        if (--until_qr == 0 || s == a.n_steps) {
            until_qr = a.qr_every;
            __syncthreads();
            for (int j = 0; j < D; ++j) {
                pair_sync(rb);  // rows of column j in this row block are final
                double* Pb = qp + (j & 1) * Q * D;
                switch ((j >> 5) * 2 + ch) {  // warp-uniform
                case 0: dots<0, 0>(W, Pb, j, rb, lane); break;
                case 1: dots<0, 1>(W, Pb, j, rb, lane); break;
                case 2: dots<1, 0>(W, Pb, j, rb, lane); break;
                case 3: dots<1, 1>(W, Pb, j, rb, lane); break;
                case 4: dots<2, 0>(W, Pb, j, rb, lane); break;
                case 5: dots<2, 1>(W, Pb, j, rb, lane); break;
                case 6: dots<3, 0>(W, Pb, j, rb, lane); break;
                default: dots<3, 1>(W, Pb, j, rb, lane); break;
                }
                __syncthreads();
                double nj = Pb[j];
#pragma unroll
                for (int q = 1; q < Q; ++q) nj += Pb[q * D + j];
                const double inv_nj = 1.0 / nj;  // one division per pivot
                if (t == j) nrm[j] = nj;
                switch ((j >> 5) * 2 + ch) {
                case 0: axpy<0, 0>(W, Pb, j, inv_nj, rb, lane); break;
                case 1: axpy<0, 1>(W, Pb, j, inv_nj, rb, lane); break;
                case 2: axpy<1, 0>(W, Pb, j, inv_nj, rb, lane); break;
                case 3: axpy<1, 1>(W, Pb, j, inv_nj, rb, lane); break;
                case 4: axpy<2, 0>(W, Pb, j, inv_nj, rb, lane); break;
                case 5: axpy<2, 1>(W, Pb, j, inv_nj, rb, lane); break;
                case 6: axpy<3, 0>(W, Pb, j, inv_nj, rb, lane); break;
                default: axpy<3, 1>(W, Pb, j, inv_nj, rb, lane); break;
                }
            }
            __syncthreads();
            if (lead) Sv[l] += 0.5 * log(nrm[l]);
#pragma unroll
            for (int m = ch; m < Q; m += 2) {
                const int c = lane + 32 * m;
                const double inv = rsqrt(nrm[c]);
#pragma unroll 4
                for (int i = 0; i < 32; ++i) W[(32 * rb + i) * WS + c] *= inv;
            }
        }
        __syncthreads();
        if (lead) S = Sv[l];
        if (--until == 0) {
            until = a.sample_every;
            if (orbit_any(lead && !(isfinite(xi) && isfinite(S))) && st == CHS_ORBIT_OK)
                st = CHS_ORBIT_NONFINITE;
            // block-uniform: the orbit's threads stop together
            if (a.clock_budget > 0 && __syncthreads_or(budget_spent(a, t_start))) {
                if (st == CHS_ORBIT_OK) st = CHS_ORBIT_STEP_BUDGET;
                break;
            }
        }
    }
    if (valid && lead) {
        const double t_total = (double)a.n_steps * a.dt;
        lambda[(int64_t)l * n + o] =
            (st == CHS_ORBIT_OK) ? S / t_total : __longlong_as_double(0x7ff8000000000000LL);
        if (l == 0) status_out[o] = st;
    }
}

}  // namespace n64
}  // namespace chs

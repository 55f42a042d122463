// fput_lyap_rk4.cuh -- the FPUT Lyapunov spectrum by periodic QR for N = 16 .. 64
// (RK4), as the work of one block: k_fput.cu launches it block by block, the
// mixed-chain persistent kernel (k_fput_batch.cu) runs it from a work queue.
//
// One orbit per d = 2N threads; a block of T = 32, 64 or 128 threads (at
// least d) holds T / d orbits.  Thread l owns state component l and, for the
// propagation, column l of the d x d matrix W of deviation vectors, which lives
// in shared memory (128 KB at N = 64; rows padded to 33 doubles at d = 32).
//
// Propagation of W uses the exact one-step propagator of classic RK4 applied
// to the linear variational equation w' = J_s w, with J_s = [[0, I], [-H_s, 0]]
// and H_s the tridiagonal Hessian of the chain at RK4 stage s (s = 1..4):
//   Phi = I + h/6 (J1 + 2J2 + 2J3 + J4) + h^2/6 (J2J1 + J3J2 + J4J3)
//           + h^3/12 (J3J2J1 + J4J3J2) + h^4/24 J4J3J2J1,
// which in blocks is
//   A = I - h^2/6 (H1 + H2 + H3) + h^4/24 H3 H1       (pentadiagonal)
//   B = h I - h^3/12 (H2 + H3)                        (tridiagonal)
//   C = -h/6 (H1 + 2H2 + 2H3 + H4) + h^3/12 (H3 H1 + H4 H2)
//   D = I - h^2/6 (H2 + H3 + H4) + h^4/24 H4 H2
// and u' = A u + B v, v' = C u + D v for every column w = (u, v).  In exact
// arithmetic this equals RK4 on the joint system; it needs no stage copies of
// W (which would not fit in shared memory at N = 64) and costs 18 FMA per row
// and column instead of about 26.  The band rows are built once per step and
// shared by all columns.
//
// QR: modified Gram-Schmidt in the "dot products first" order: for column j
// every column l >= j forms r_l = w_j . w_l (r_j = |w_j|^2), then each l > j
// subtracts (r_l / r_j) w_j; the columns are scaled to unit length at the end
// and S_j += ln |w_j| (so R_jj > 0).  Thread l works column l at d = 64.  At
// d = 32 (one warp per orbit) lane 8b + p takes rows 8b .. 8b + 7 of the columns
// p + 8m, and the four partial dot products of a column are joined by shuffles
// (qr_warp32).  At d = 128 the orbit's Q = 4 warps split the rows: warp w takes
// rows 32w..32w+31 of the columns lane + 32m (m < Q), and the Q partial dot
// products of a column are summed in a fixed order from shared memory
// (qr_split).  Every lane then works while its column group is left (with one
// column per thread, the lanes holding the first columns would idle through
// most pivots, and an idle lane costs an FP64 slot).  At N = 64 the library's
// default is the 256-thread form of fput_lyap_n64.cuh (two threads per column,
// the same arithmetic); this 128-thread body is the block size 128 and the
// mixed-chain persistent kernel's.
#pragma once

#include <math.h>

#include "chs_internal.cuh"
#include "fput_phi.cuh"

namespace chs {

template <int N, int T>
struct FputLyapCfg {
    static constexpr int D = 2 * N;
    static constexpr int THREADS = T;
    static constexpr int G = T / D;  // orbits per block
    static_assert(T % D == 0 && T <= 128 && T % 32 == 0, "blocks of whole orbits and whole warps");
    // row blocks of the split QR: the orbit's 4 warps at N = 64, where shared
    // memory holds one orbit per SM and the QR's critical path is the kernel's
    // (measured: 1213 -> 1012 ms per 200 steps at QR every 10).  At N = 32 six
    // orbits share an SM and hide the imbalance; the split measured 4 % slower.
    static constexpr int Q = D >= 128 ? D / 32 : 1;
    // row stride of W: at d = 32 one padding column, so that the row blocks of
    // the in-warp QR (qr_warp32) fall in distinct shared-memory banks
    static constexpr int WS = D == 32 ? D + 1 : D;
    // doubles per orbit: W (D rows of WS), band rows, stage state, stage stiffnesses, 2 scratch,
    // the QR's double-buffered partial dot products [2][Q][D], exponent sums [D]
    // and squared column norms [D]
    static constexpr int PER = D * WS + 18 * N + D + 4 * (N + 1) + 2 + (Q > 1 ? 2 * Q * D + 2 * D : 0);
    static constexpr size_t SMEM = (size_t)G * PER * sizeof(double);
};

struct FputCoef {
    double k, a2, b3;  // V''(r) = k + 2 alpha r + 3 beta r^2
    double alpha, beta;
};

__device__ __forceinline__ double fput_dv_over_r(const FputCoef& fc, double r)
{
    // V'(r) / r = k + alpha r + beta r^2
    return fma(r, fma(fc.beta, r, fc.alpha), fc.k);
}

__device__ __forceinline__ double fput_d2v(const FputCoef& fc, double r)
{
    return fma(r, fma(fc.b3, r, fc.a2), fc.k);
}

// w <- Phi w for column l, in place, streaming down the rows with a window of
// the old values u_{i-2..i+2}, v_{i-2..i+2}.
template <int N, int WS>
__device__ __forceinline__ void apply_phi(double* __restrict__ W, const double* __restrict__ cf, const int l)
{
    auto U = [&](int i) { return (i >= 0 && i < N) ? W[i * WS + l] : 0.0; };
    auto V = [&](int i) { return (i >= 0 && i < N) ? W[(N + i) * WS + l] : 0.0; };
    double u0 = 0.0, u1 = 0.0, u2 = U(0), u3 = U(1), u4 = U(2);
    double v0 = 0.0, v1 = 0.0, v2 = V(0), v3 = V(1), v4 = V(2);
#pragma unroll 4
    for (int i = 0; i < N; ++i) {
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
        W[i * WS + l] = nu;
        W[(N + i) * WS + l] = nv;
        u0 = u1; u1 = u2; u2 = u3; u3 = u4; u4 = U(i + 3);
        v0 = v1; v1 = v2; v2 = v3; v3 = v4; v4 = V(i + 3);
    }
}

// One pivot step of the split modified Gram-Schmidt for d = 128, for the
// column groups m >= M0 (columns lane + 32 m; the groups below are finished:
// M0 = j / 32).  The groups' dot products run in one block of code, sharing the
// loads of the pivot column and giving the warp independent FMA chains; lanes
// whose column is below j compute too but store only into sums nobody reads.
template <int N, int M0>
__device__ __forceinline__ void split_dots(const double* __restrict__ W, double* __restrict__ Pb, const int j,
                                           const int w, const int lane)
{
    constexpr int D = 2 * N, Q = D / 32;
    const int r0 = 32 * w;
    double a0[Q], a1[Q];
#pragma unroll
    for (int m = M0; m < Q; ++m) a0[m] = a1[m] = 0.0;
#pragma unroll 4
    for (int i = 0; i < 32; i += 2) {
        const double wj0 = W[(r0 + i) * D + j], wj1 = W[(r0 + i + 1) * D + j];
#pragma unroll
        for (int m = M0; m < Q; ++m) {
            const int c = lane + 32 * m;
            a0[m] = fma(wj0, W[(r0 + i) * D + c], a0[m]);
            a1[m] = fma(wj1, W[(r0 + i + 1) * D + c], a1[m]);
        }
    }
#pragma unroll
    for (int m = M0; m < Q; ++m) Pb[w * D + lane + 32 * m] = a0[m] + a1[m];
}

// The update of the columns c > j of this warp's rows, groups m >= M0.
template <int N, int M0>
__device__ __forceinline__ void split_axpy(double* __restrict__ W, const double* __restrict__ Pb, const int j,
                                           const double inv_nj, const int w, const int lane)
{
    constexpr int D = 2 * N, Q = D / 32;
    const int r0 = 32 * w;
    double f[Q];
#pragma unroll
    for (int m = M0; m < Q; ++m) {
        const int c = lane + 32 * m;
        double r = Pb[c];
#pragma unroll
        for (int q = 1; q < Q; ++q) r += Pb[q * D + c];
        f[m] = -r * inv_nj;
    }
    const bool diag_active = lane + 32 * M0 > j;  // groups above M0 lie wholly right of j
#pragma unroll 4
    for (int i = 0; i < 32; ++i) {
        const double wj = W[(r0 + i) * D + j];
#pragma unroll
        for (int m = M0; m < Q; ++m) {
            const int c = lane + 32 * m;
            const double v = fma(f[m], wj, W[(r0 + i) * D + c]);
            if (m > M0 || diag_active) W[(r0 + i) * D + c] = v;
        }
    }
}

// The split modified Gram-Schmidt for d = 128 (see the file comment): t is
// the thread's index in its orbit, P the [2][Q][d] partial sums, Sv[c] the
// exponent sum of column c.  Every thread of the block calls it.
template <int N>
__device__ __forceinline__ void qr_split(double* W, double* P, double* Sv, double* nrm, const int t)
{
    constexpr int D = 2 * N, Q = D / 32;
    static_assert(Q == 4, "four row blocks");
    const int w = t / 32, lane = t % 32;
    const int r0 = 32 * w;
    for (int j = 0; j < D; ++j) {
        __syncwarp();  // rows of column j in this warp's block are final
        double* Pb = P + (j & 1) * Q * D;
        switch (j >> 5) {  // block-uniform
        case 0: split_dots<N, 0>(W, Pb, j, w, lane); break;
        case 1: split_dots<N, 1>(W, Pb, j, w, lane); break;
        case 2: split_dots<N, 2>(W, Pb, j, w, lane); break;
        default: split_dots<N, 3>(W, Pb, j, w, lane); break;
        }
        __syncthreads();
        double nj = Pb[j];
#pragma unroll
        for (int q = 1; q < Q; ++q) nj += Pb[q * D + j];
        const double inv_nj = 1.0 / nj;  // one division per pivot, not per column
        if (t == j) nrm[j] = nj;
        switch (j >> 5) {
        case 0: split_axpy<N, 0>(W, Pb, j, inv_nj, w, lane); break;
        case 1: split_axpy<N, 1>(W, Pb, j, inv_nj, w, lane); break;
        case 2: split_axpy<N, 2>(W, Pb, j, inv_nj, w, lane); break;
        default: split_axpy<N, 3>(W, Pb, j, inv_nj, w, lane); break;
        }
    }
    // the logarithms and reciprocal roots of the column norms after the loop,
    // one column per thread, instead of one lane's work inside every pivot step
    __syncthreads();
    Sv[t] += 0.5 * log(nrm[t]);
#pragma unroll
    for (int m = 0; m < Q; ++m) {
        const int c = lane + 32 * m;
        const double inv = rsqrt(nrm[c]);
#pragma unroll 4
        for (int i = 0; i < 32; ++i) W[(r0 + i) * D + c] *= inv;
    }
}

// The modified Gram-Schmidt for d = 32, where an orbit is one warp: lane
// l = 8 b + p takes rows 8b .. 8b + 7 of the columns p + 8m (m < 4), so that
// every lane keeps work until the last column group (one column per lane
// leaves lanes l < j idle at pivot j, and an idle lane costs an FP64 slot).  A
// column's four partial dot products are summed by a butterfly over the lanes
// p, p + 8, p + 16, p + 24, which gives the same sum in all four.  W's rows are
// WS = 33 apart, so the row blocks of a half-warp fall in distinct banks.
// Returns, in lane l, the squared norm of column l before normalisation.
template <int N, int WS>
__device__ __forceinline__ double qr_warp32(double* W, const int l)
{
    constexpr int D = 2 * N, CG = D / 8;  // column groups
    static_assert(D == 32, "one warp per orbit");
    const int p = l % 8;
    double* Wb = W + (l / 8) * 8 * WS;  // this lane's row block
    double n2 = 1.0;
#pragma unroll
    for (int jm = 0; jm < CG; ++jm) {
#pragma unroll 1
        for (int jp = 0; jp < 8; ++jp) {
            const int j = jp + 8 * jm;
            __syncwarp();  // column j is final
            double r[CG];
#pragma unroll
            for (int m = jm; m < CG; ++m) {
                double part = 0.0;
                if (m > jm || p >= jp) {
                    const int c = p + 8 * m;
                    double s0 = 0.0, s1 = 0.0;
#pragma unroll
                    for (int i = 0; i < 8; i += 2) {
                        s0 = fma(Wb[i * WS + j], Wb[i * WS + c], s0);
                        s1 = fma(Wb[(i + 1) * WS + j], Wb[(i + 1) * WS + c], s1);
                    }
                    part = s0 + s1;
                }
                part += __shfl_xor_sync(0xffffffffu, part, 8);
                part += __shfl_xor_sync(0xffffffffu, part, 16);
                r[m] = part;
            }
            const double nj = __shfl_sync(0xffffffffu, r[jm], jp);  // |w_j|^2
            if (l == j) n2 = nj;
            const double inv_nj = 1.0 / nj;  // one division per pivot
#pragma unroll
            for (int m = jm; m < CG; ++m) {
                if (m > jm || p > jp) {
                    const int c = p + 8 * m;
                    const double f = -r[m] * inv_nj;
#pragma unroll
                    for (int i = 0; i < 8; ++i) Wb[i * WS + c] = fma(f, Wb[i * WS + j], Wb[i * WS + c]);
                }
            }
        }
    }
    __syncwarp();
    return n2;
}

// The work of one block of T threads: the G = T / 2N orbits vb * G .. vb * G +
// G - 1 (those below n), in the shared memory `smem` (FputLyapCfg::SMEM bytes).
// Every thread of the block calls it; it contains block barriers.
template <int N, int T>
__device__ __forceinline__ void fput_lyap_block(const StepArgs& a, const SysPar& sp, const int64_t n,
                                                const double* __restrict__ ics,
                                                const int32_t* __restrict__ ic_status,
                                                double* __restrict__ lambda, int32_t* __restrict__ status_out,
                                                const int64_t vb, double* smem)
{
    using Cfg = FputLyapCfg<N, T>;
    constexpr int D = Cfg::D, G = Cfg::G, PER = Cfg::PER, WS = Cfg::WS;
    const int g = threadIdx.x / D, l = threadIdx.x % D;
    const int64_t o = vb * G + g;
    const bool valid = o < n;
    double* W = smem + g * PER;
    double* cf = W + D * WS;
    double* xs = cf + 18 * N;
    double* cs = xs + D;
    double* red = cs + 4 * (N + 1);
    double* qp = red + 2;            // split QR: partial sums [2][Q][D] (d = 128)
    double* Sv = qp + 2 * Cfg::Q * D;  // split QR: exponent sums [D]
    double* nrm = Sv + D;              // split QR: squared column norms [D]

    const FputCoef fc = {sp.kk, 2.0 * sp.alpha, 3.0 * sp.beta, sp.alpha, sp.beta};
    int32_t st = valid ? (ic_status ? ic_status[o] : CHS_ORBIT_OK) : CHS_ORBIT_FORBIDDEN;
    double xi = valid ? ics[(int64_t)l * n + o] : 0.0;

    // orbit-wide "any thread non-finite" (block-wide barriers; every thread takes part)
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
    for (int i = 0; i < D; ++i) W[i * WS + l] = (i == l) ? 1.0 : 0.0;
    xs[l] = xi;
    double S = 0.0;
    if constexpr (Cfg::Q > 1) Sv[l] = 0.0;
    __syncthreads();

    const double h = a.dt;
    int64_t until_qr = a.qr_every;
    int64_t until = a.sample_every > 0 ? a.sample_every : -1;
    const long long t_start = clock64();
    for (int64_t s = 1; s <= a.n_steps; ++s) {
        // RK4 of the orbit; stage stiffnesses V''(D_b) recorded for Phi
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double fi;
            if (l < N) {
                fi = xs[N + l];
            } else {
                const int i = l - N;
                const double qm = i > 0 ? xs[i - 1] : 0.0;
                const double q0 = xs[i];
                const double qp = i < N - 1 ? xs[i + 1] : 0.0;
                // V'(r_right) - V'(r_left), the left term rounded on its own and the
                // right one fused (the form of the short chains' kernel)
                const double rr = qp - q0, rl = q0 - qm;
                fi = fma(rr, fput_dv_over_r(fc, rr), -__dmul_rn(rl, fput_dv_over_r(fc, rl)));
            }
            if (l <= N) {
                const double qa = l < N ? xs[l] : 0.0;
                const double qb = l > 0 ? xs[l - 1] : 0.0;
                cs[k * (N + 1) + l] = fput_d2v(fc, qa - qb);
            }
            __syncthreads();
            acc = (k == 0) ? fi : fma((k == 3) ? 1.0 : 2.0, fi, acc);
            if (k < 3) xs[l] = fma(k == 2 ? h : 0.5 * h, fi, xi);
            __syncthreads();
        }
        xi = fma(h / 6.0, acc, xi);
        xs[l] = xi;
        if (l < N) {
            double cb[4][4];  // stiffnesses of bonds l - 1 .. l + 2 (none beyond the walls)
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int b = l - 1 + t;
                    cb[k][t] = (b >= 0 && b <= N) ? cs[k * (N + 1) + b] : 0.0;
                }
            fput_phi::phi_row<N>(l, cb, h, cf + l * 18);
        }
        __syncthreads();
        apply_phi<N, WS>(W, cf, l);

        if (--until_qr == 0 || s == a.n_steps) {
            until_qr = a.qr_every;
            __syncthreads();
            if constexpr (Cfg::Q > 1) {
                qr_split<N>(W, qp, Sv, nrm, l);
            } else if constexpr (D == 32) {
                const double n2 = qr_warp32<N, WS>(W, l);
                S += 0.5 * log(n2);
                const double inv = rsqrt(n2);
#pragma unroll 4
                for (int i = 0; i < D; ++i) W[i * WS + l] *= inv;
            } else {
                double n2 = 1.0;  // this thread's column's squared norm
                for (int j = 0; j < D; ++j) {
                    double r = 0.0;
                    if (l >= j) {
                        double r0 = 0.0, r1 = 0.0;
#pragma unroll 4
                        for (int i = 0; i < D; i += 2) {
                            r0 = fma(W[i * D + j], W[i * D + l], r0);
                            r1 = fma(W[(i + 1) * D + j], W[(i + 1) * D + l], r1);
                        }
                        r = r0 + r1;
                    }
                    if (l == j) {
                        red[0] = r;
                        n2 = r;
                    }
                    __syncthreads();
                    if (l > j) {
                        const double cfac = -r / red[0];
#pragma unroll 4
                        for (int i = 0; i < D; ++i) W[i * D + l] = fma(cfac, W[i * D + j], W[i * D + l]);
                    }
                    __syncthreads();
                }
                // the logarithm and reciprocal root of every column's norm after
                // the loop, one per thread, instead of one lane's work inside
                // every pivot step
                S += 0.5 * log(n2);
                const double inv = rsqrt(n2);
#pragma unroll 4
                for (int i = 0; i < D; ++i) W[i * D + l] *= inv;
            }
        }
        __syncthreads();
        if constexpr (Cfg::Q > 1) S = Sv[l];
        if (--until == 0) {
            until = a.sample_every;
            if (orbit_any(!(isfinite(xi) && isfinite(S))) && st == CHS_ORBIT_OK)
                st = CHS_ORBIT_NONFINITE;
            // block-uniform: the block's orbits stop together
            if (a.clock_budget > 0 && __syncthreads_or(budget_spent(a, t_start))) {
                if (st == CHS_ORBIT_OK) st = CHS_ORBIT_STEP_BUDGET;
                break;
            }
        }
    }
    if (valid) {
        const double t_total = (double)a.n_steps * a.dt;
        lambda[(int64_t)l * n + o] =
            (st == CHS_ORBIT_OK) ? S / t_total : __longlong_as_double(0x7ff8000000000000LL);
        if (l == 0) status_out[o] = st;
    }
}

}  // namespace chs

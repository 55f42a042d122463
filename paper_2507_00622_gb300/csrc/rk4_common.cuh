// rk4_common.cuh -- pieces of the classic RK4 step shared by the one-orbit-per-
// thread kernels: the orbit's four stages (with the LD quadrature and the stage
// Hessians recorded) and the exact one-step propagator of the variational
// equations.
#pragma once

#include "chs_internal.cuh"
#include "fastmath.cuh"
#include "systems.cuh"

namespace chs {

// LD integrand sum_i |f_i|^p in FP64 for a general exponent p (p = 1/2 takes
// the double-float route, ld_acc_sqrt).
template <int D>
__device__ __forceinline__ double ld_integrand_pow(const double* f, double p)
{
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) acc += pow(fabs(f[i]), p);
    return acc;
}

// The LD integrand summed in FP32: each |f_i| rounded to FP32 (integer pipe),
// its correctly rounded FP32 root (or power), the sum widened exactly to FP64.
template <int D>
__device__ __forceinline__ double ld_integrand_f32(const double* f, int ld_sqrt, double p)
{
    float acc = 0.0f;
    if (ld_sqrt) {
#pragma unroll
        for (int i = 0; i < D; ++i) acc += sqrtf(fabsf(f32_from_f64(f[i])));
    } else {
        const float pf = (float)p;
#pragma unroll
        for (int i = 0; i < D; ++i) acc += powf(fabsf(f32_from_f64(f[i])), pf);
    }
    return acc < 1.17549435e-38f ? 0.0 : f32_to_f64_bits(acc);
}

template <int D, bool LD32>
__device__ __forceinline__ double ld_term(const double* f, int ld_sqrt, double p)
{
    if constexpr (LD32)
        return ld_integrand_f32<D>(f, ld_sqrt, p);
    else
        return ld_integrand_pow<D>(f, p);
}

// acc += w sum_i sqrt|f_i| in double-float (p = 1/2; w a power of two).
template <int D>
__device__ __forceinline__ void ld_acc_sqrt(FF& acc, const double* f, const float w)
{
#pragma unroll
    for (int i = 0; i < D; ++i) ff_acc(acc, ff_sqrt(ff_split(fabs(f[i]))), w);
}

// One classic RK4 step of the orbit x and its LD accumulator L,
//   k1 = f(x), k2 = f(x + h/2 k1), k3 = f(x + h/2 k2), k4 = f(x + h k3),
//   x <- x + h/6 (k1 + 2 k2 + 2 k3 + k4),  L <- L + |h|/6 (g1 + 2 g2 + 2 g3 + g4),
// handing each stage s its state xs and Hess V(xs) (packed upper triangle) as
// rec(s, xs, H); a recorder that ignores H leaves its arithmetic unused.
// FP64 vectors, p = 1/2: the weighted sum of the sixteen square roots is formed
// in double-float arithmetic (relative error ~1e-13, off the FP64 pipe) and
// added to L with one FP64 FMA.  LD32 (the FP32-frame mode, bound by
// instruction issue rather than by the FP64 pipe): the integrand is summed in
// FP32 (ld_integrand_f32).  Other exponents use pow.
template <class Sys, bool LD, bool LD32, class Rec>
__device__ __forceinline__ void rk4_stages(double* x, double& L, const double h, const int ld_sqrt,
                                           const double ld_p, const SysPar& sp, Rec&& rec)
{
    constexpr int D = 2 * Sys::N;
    const double hh = 0.5 * h, h6 = h / 6.0;
    double ax[D], xs[D], f[D], Hs[Sys::NH];
    double aL = 0.0;
    FF fL{0.0f, 0.0f};
    Sys::eval(x, f, Hs, sp);
    rec(0, x, Hs);
#pragma unroll
    for (int c = 0; c < D; ++c) {
        ax[c] = f[c];
        xs[c] = fma(hh, f[c], x[c]);
    }
    const bool ff = !LD32 && ld_sqrt;
    if (LD) {
        if (ff)
            ld_acc_sqrt<D>(fL, f, 1.0f);
        else
            aL = ld_term<D, LD32>(f, ld_sqrt, ld_p);
    }
#pragma unroll
    for (int s = 1; s < 3; ++s) {
        const double cs = (s == 1) ? hh : h;
        Sys::eval(xs, f, Hs, sp);
        rec(s, xs, Hs);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            ax[c] = fma(2.0, f[c], ax[c]);
            xs[c] = fma(cs, f[c], x[c]);
        }
        if (LD) {
            if (ff)
                ld_acc_sqrt<D>(fL, f, 2.0f);
            else
                aL = fma(2.0, ld_term<D, LD32>(f, ld_sqrt, ld_p), aL);
        }
    }
    Sys::eval(xs, f, Hs, sp);
    rec(3, xs, Hs);
#pragma unroll
    for (int c = 0; c < D; ++c) x[c] = fma(h6, ax[c] + f[c], x[c]);
    // the LD grows with |t|: a backward run (h < 0) accumulates a positive M_p
    if (LD) {
        if (ff) {
            ld_acc_sqrt<D>(fL, f, 1.0f);
            L = fma(fabs(h6), ff_to_f64(fL), L);
        } else {
            L = fma(fabs(h6), aL + ld_term<D, LD32>(f, ld_sqrt, ld_p), L);
        }
    }
}

// The RK4 step recording Hess V at the four stage states in H[s].
template <class Sys, bool LD, bool LD32 = false>
__device__ __forceinline__ void rk4_state_capture(double* x, double& L, const double h,
                                                  const int ld_sqrt, const double ld_p,
                                                  const SysPar& sp, double (*H)[Sys::NH])
{
    rk4_stages<Sys, LD, LD32>(x, L, h, ld_sqrt, ld_p, sp, [&](int s, const double*, const double* Hs) {
#pragma unroll
        for (int i = 0; i < Sys::NH; ++i) H[s][i] = Hs[i];
    });
}

// The RK4 step recording the stage positions q rounded to FP32 (integer pipe)
// in qf[s]; the FP64 Hessians are not formed.
template <class Sys, bool LD, bool LD32 = false>
__device__ __forceinline__ void rk4_state_positions(double* x, double& L, const double h,
                                                    const int ld_sqrt, const double ld_p,
                                                    const SysPar& sp, float (*qf)[Sys::N])
{
    rk4_stages<Sys, LD, LD32>(x, L, h, ld_sqrt, ld_p, sp, [&](int s, const double* xs, const double*) {
#pragma unroll
        for (int i = 0; i < Sys::N; ++i) qf[s][i] = f32_from_f64(xs[i]);
    });
}

// Exact one-step propagator of RK4 on the linear variational equation
// w' = J_s w, J_s = [[0, I], [-H_s, 0]] (H_s = Hess V at stage s):
//   Phi = I + h/6 (J1 + 2J2 + 2J3 + J4) + h^2/6 (J2J1 + J3J2 + J4J3)
//           + h^3/12 (J3J2J1 + J4J3J2) + h^4/24 J4J3J2J1
//       = [[A, B], [C, D]] with
//   A = I - h^2/6 (H1+H2+H3) + h^4/24 H3H1,   B = h I - h^3/12 (H2+H3),
//   C = -h/6 (H1+2H2+2H3+H4) + h^3/12 (H3H1 + H4H2),
//   D = I - h^2/6 (H2+H3+H4) + h^4/24 H4H2.
// Applying Phi equals RK4 on the joint system in exact arithmetic.
template <int N, typename T>
struct PhiBlocks {
    T A[N][N], B[N][N], C[N][N], D[N][N];
};

template <int N, int NH, typename T>
__device__ __forceinline__ void phi_build(const T (*Hs)[NH], const double h, PhiBlocks<N, T>& P)
{
    const T hv = (T)h, c1 = (T)(h / 6.0), c2 = (T)(h * h / 6.0), c3 = (T)(h * h * h / 12.0),
            c4 = (T)(h * h * h * h / 24.0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const T s1 = Hs[0][hidx<N>(i, j)], s2 = Hs[1][hidx<N>(i, j)];
            const T s3 = Hs[2][hidx<N>(i, j)], s4 = Hs[3][hidx<N>(i, j)];
            T p31 = Hs[2][hidx<N>(i, 0)] * Hs[0][hidx<N>(0, j)];
            T p42 = Hs[3][hidx<N>(i, 0)] * Hs[1][hidx<N>(0, j)];
#pragma unroll
            for (int m = 1; m < N; ++m) {
                p31 = fma(Hs[2][hidx<N>(i, m)], Hs[0][hidx<N>(m, j)], p31);
                p42 = fma(Hs[3][hidx<N>(i, m)], Hs[1][hidx<N>(m, j)], p42);
            }
            const T s23 = s2 + s3;
            const T id = (i == j) ? (T)1 : (T)0;
            P.A[i][j] = fma(c4, p31, fma(-c2, s1 + s23, id));
            P.B[i][j] = (i == j) ? fma(-c3, s23, hv) : -c3 * s23;
            P.C[i][j] = fma(c3, p31 + p42, -c1 * (fma((T)2, s23, s1) + s4));
            P.D[i][j] = fma(c4, p42, fma(-c2, s23 + s4, id));
        }
    }
}

// Henon-Heiles: Hess V = I + 2 M(q) with M(q) = [[q2, q1], [q1, -q2]] (from
// Eq. ham_eqs_HH), M linear in q, and M(a) M(b) = [[p, r], [-r, p]] with
// p = a1 b1 + a2 b2, r = a2 b1 - a1 b2.  The blocks of Phi from the four stage
// positions q_s, with c1 = h/6, c2 = h^2/6, c3 = h^3/12, c4 = h^4/24:
//   A = (1 - 3 c2 + c4) I + 2 M(c4 (q1 + q3) - c2 (q1 + q2 + q3)) + 4 c4 M(q3) M(q1)
//   B = (h - 2 c3) I - 2 c3 M(q2 + q3)
//   C = (2 c3 - 6 c1) I + 2 M(c3 (q1 + q2 + q3 + q4) - c1 (q1 + 2 q2 + 2 q3 + q4))
//       + 4 c3 (M(q3) M(q1) + M(q4) M(q2))
//   D = (1 - 3 c2 + c4) I + 2 M(c4 (q2 + q4) - c2 (q2 + q3 + q4)) + 4 c4 M(q4) M(q2)
// (the general blocks above with H_s = I + 2 M(q_s)); no Hessian is formed.
__device__ __forceinline__ void phi_build_hh(const double (*q)[2], const double h, PhiBlocks<2, double>& P)
{
    const double c1 = h / 6.0, c2 = h * h / 6.0, c3 = h * h * h / 12.0, c4 = h * h * h * h / 24.0;
    const double aAD = 1.0 - 3.0 * c2 + c4, aB = h - 2.0 * c3, aC = 2.0 * c3 - 6.0 * c1;
    double mA[2], mB[2], mC[2], mD[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const double s13 = q[0][i] + q[2][i], s24 = q[1][i] + q[3][i], s23 = q[1][i] + q[2][i];
        const double s123 = s13 + q[1][i], s234 = s24 + q[2][i], sall = s13 + s24;
        mA[i] = fma(2.0 * c4, s13, -2.0 * c2 * s123);
        mB[i] = -2.0 * c3 * s23;
        mC[i] = fma(2.0 * c3, sall, -2.0 * c1 * (sall + s23));
        mD[i] = fma(2.0 * c4, s24, -2.0 * c2 * s234);
    }
    const double p31 = fma(q[2][0], q[0][0], q[2][1] * q[0][1]), r31 = fma(q[2][1], q[0][0], -q[2][0] * q[0][1]);
    const double p42 = fma(q[3][0], q[1][0], q[3][1] * q[1][1]), r42 = fma(q[3][1], q[1][0], -q[3][0] * q[1][1]);
    const double k4 = 4.0 * c4, k3 = 4.0 * c3;
    P.A[0][0] = fma(k4, p31, aAD + mA[1]);
    P.A[1][1] = fma(k4, p31, aAD - mA[1]);
    P.A[0][1] = fma(k4, r31, mA[0]);
    P.A[1][0] = fma(-k4, r31, mA[0]);
    P.B[0][0] = aB + mB[1];
    P.B[1][1] = aB - mB[1];
    P.B[0][1] = mB[0];
    P.B[1][0] = mB[0];
    const double pc = p31 + p42, rc = r31 + r42;
    P.C[0][0] = fma(k3, pc, aC + mC[1]);
    P.C[1][1] = fma(k3, pc, aC - mC[1]);
    P.C[0][1] = fma(k3, rc, mC[0]);
    P.C[1][0] = fma(-k3, rc, mC[0]);
    P.D[0][0] = fma(k4, p42, aAD + mD[1]);
    P.D[1][1] = fma(k4, p42, aAD - mD[1]);
    P.D[0][1] = fma(k4, r42, mD[0]);
    P.D[1][0] = fma(-k4, r42, mD[0]);
}

// w <- Phi w for one vector w = (u, v).
template <int N, typename T>
__device__ __forceinline__ void phi_apply(const PhiBlocks<N, T>& P, T* w)
{
    T nw[2 * N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        T u = P.A[i][0] * w[0], v = P.C[i][0] * w[0];
#pragma unroll
        for (int m = 1; m < N; ++m) {
            u = fma(P.A[i][m], w[m], u);
            v = fma(P.C[i][m], w[m], v);
        }
#pragma unroll
        for (int m = 0; m < N; ++m) {
            u = fma(P.B[i][m], w[N + m], u);
            v = fma(P.D[i][m], w[N + m], v);
        }
        nw[i] = u;
        nw[N + i] = v;
    }
#pragma unroll
    for (int c = 0; c < 2 * N; ++c) w[c] = nw[c];
}

}  // namespace chs

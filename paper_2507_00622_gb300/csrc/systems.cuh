// systems.cuh -- device-side Hamiltonians for the one-orbit-per-thread kernels.
//
// Each system provides, for phase-space state x = (q_1..q_N, p_1..p_N):
//   eval(x, f, H)  f = (p, -grad V(q)) (Hamilton's equations) and the packed
//                  upper triangle H of Hess V(q), which drives the variational
//                  equations d(dq)/dt = dp, d(dp)/dt = -Hess V(q) dq;
//   energy(x)      the Hamiltonian.
#pragma once

#include "chs_internal.cuh"

namespace chs {

// Index of Hess V entry (i, j), i <= j, in the packed upper triangle.
template <int N>
__host__ __device__ constexpr int hidx(int i, int j)
{
    return (i <= j) ? (i * N - i * (i - 1) / 2 + (j - i)) : (j * N - j * (j - 1) / 2 + (i - j));
}

// Henon-Heiles, Eq. Ham_HH / Eq. ham_eqs_HH:
//   p_x' = -x - 2xy,  p_y' = -y - x^2 + y^2,  Hess V = [[1 + 2y, 2x], [2x, 1 - 2y]].
struct SysHenonHeiles {
    static constexpr int N = 2, NH = 3;
    __device__ __forceinline__ static void eval(const double* x, double* f, double* H, const SysPar&)
    {
        const double q1 = x[0], q2 = x[1];
        const double a = fma(2.0, q2, 1.0);
        H[0] = a;
        H[1] = 2.0 * q1;
        H[2] = fma(-2.0, q2, 1.0);
        f[0] = x[2];
        f[1] = x[3];
        f[2] = -q1 * a;
        f[3] = fma(-q1, q1, fma(q2, q2, -q2));
    }
    __device__ __forceinline__ static double energy(const double* x, const SysPar&)
    {
        const double q1 = x[0], q2 = x[1];
        return 0.5 * (x[2] * x[2] + x[3] * x[3]) + 0.5 * (q1 * q1 + q2 * q2) + q1 * q1 * q2
             - q2 * q2 * q2 / 3.0;
    }
};

// Harmonic oscillator, 2 DOF: H = sum (p_i^2 + q_i^2) / 2.
struct SysHarmonic {
    static constexpr int N = 2, NH = 3;
    __device__ __forceinline__ static void eval(const double* x, double* f, double* H, const SysPar&)
    {
        H[0] = 1.0;
        H[1] = 0.0;
        H[2] = 1.0;
        f[0] = x[2];
        f[1] = x[3];
        f[2] = -x[0];
        f[3] = -x[1];
    }
    __device__ __forceinline__ static double energy(const double* x, const SysPar&)
    {
        return 0.5 * (x[2] * x[2] + x[3] * x[3]) + 0.5 * (x[0] * x[0] + x[1] * x[1]);
    }
};

// Inverted oscillator: H = (p1^2 - q1^2)/2 + (p2^2 + q2^2)/2.
struct SysInverted {
    static constexpr int N = 2, NH = 3;
    __device__ __forceinline__ static void eval(const double* x, double* f, double* H, const SysPar&)
    {
        H[0] = -1.0;
        H[1] = 0.0;
        H[2] = 1.0;
        f[0] = x[2];
        f[1] = x[3];
        f[2] = x[0];
        f[3] = -x[1];
    }
    __device__ __forceinline__ static double energy(const double* x, const SysPar&)
    {
        return 0.5 * (x[2] * x[2] + x[3] * x[3]) + 0.5 * (x[1] * x[1] - x[0] * x[0]);
    }
};

// Coupled quartic oscillator, 3 DOF:
//   V = sum q_i^2 / 2 + eps (q1^2 q2^2 + q2^2 q3^2 + q1^2 q3^2),
//   dV/dq_i = q_i (1 + 2 eps (S - q_i^2)) with S = sum q_j^2,
//   Hess_ii = 1 + 2 eps (S - q_i^2),  Hess_ij = 4 eps q_i q_j.
struct SysQuartic3 {
    static constexpr int N = 3, NH = 6;
    __device__ __forceinline__ static void eval(const double* x, double* f, double* H, const SysPar& sp)
    {
        const double e2 = 2.0 * sp.eps, e4 = 4.0 * sp.eps;
        const double s0 = x[0] * x[0], s1 = x[1] * x[1], s2 = x[2] * x[2];
        const double d0 = fma(e2, s1 + s2, 1.0);
        const double d1 = fma(e2, s0 + s2, 1.0);
        const double d2 = fma(e2, s0 + s1, 1.0);
        H[hidx<3>(0, 0)] = d0;
        H[hidx<3>(1, 1)] = d1;
        H[hidx<3>(2, 2)] = d2;
        H[hidx<3>(0, 1)] = e4 * x[0] * x[1];
        H[hidx<3>(0, 2)] = e4 * x[0] * x[2];
        H[hidx<3>(1, 2)] = e4 * x[1] * x[2];
        f[0] = x[3];
        f[1] = x[4];
        f[2] = x[5];
        f[3] = -x[0] * d0;
        f[4] = -x[1] * d1;
        f[5] = -x[2] * d2;
    }
    __device__ __forceinline__ static double energy(const double* x, const SysPar& sp)
    {
        const double s0 = x[0] * x[0], s1 = x[1] * x[1], s2 = x[2] * x[2];
        return 0.5 * (x[3] * x[3] + x[4] * x[4] + x[5] * x[5]) + 0.5 * (s0 + s1 + s2)
             + sp.eps * (s0 * s1 + s1 * s2 + s0 * s2);
    }
};

}  // namespace chs

// fput_phi.cuh -- one band row of the exact one-step RK4 propagator Phi of the
// FPUT variational equation, shared by the Lyapunov kernels of every chain
// length (fput_lyap_lanes.cuh, fput_lyap_rk4.cuh).
//
// Stage Hessians H_s (s = 1..4) are tridiagonal with diagonal d_s(i) = c_s(i) +
// c_s(i+1) and off-diagonals -c_s(i), -c_s(i+1), c_s(b) the stiffness
// V''(q_b - q_{b-1}) of bond b at stage s (bonds 0 and N on the walls).  Then
//   A = I - h^2/6 (H1 + H2 + H3) + h^4/24 H3 H1
//   B = h I - h^3/12 (H2 + H3)
//   C = -h/6 (H1 + 2 H2 + 2 H3 + H4) + h^3/12 (H3 H1 + H4 H2)
//   D = I - h^2/6 (H2 + H3 + H4) + h^4/24 H4 H2
// and each column w = (u, v) of the deviation matrix becomes (A u + B v, C u + D v).
#pragma once

#include <math.h>

namespace chs {
namespace fput_phi {

// Band row of Phi for mass r from the stiffnesses of bonds r-1 .. r+2 at the
// four stages, cb[s][t] = c_s(r - 1 + t).  Entries (columns r-2 .. r+2 for A,
// C, D; r-1 .. r+1 for B) go to out[0..17] in the order A[5] B[3] C[5] D[5].
// Entries of columns outside the chain are computed but never read.
template <int N>
__device__ __forceinline__ void phi_row(const int r, const double (&cb)[4][4], const double h, double* out)
{
    const double h1 = h / 6.0, h2 = h * h / 6.0, h3 = h * h * h / 12.0, h4 = h * h * h * h / 24.0;
    // stage Hessians on rows r-1, r, r+1: diagonals, and the couplings of row r
    // to its neighbours (a wall bond couples to nothing)
    const bool has_left = r >= 1, has_right = r <= N - 2;
    double P[2][5];  // P[0] = H3 H1, P[1] = H4 H2 on row r
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int sa = q == 0 ? 2 : 3, sb = q == 0 ? 0 : 1;
        const double dbm = cb[sb][0] + cb[sb][1];  // d_b(r - 1)
        const double db0 = cb[sb][1] + cb[sb][2];  // d_b(r)
        const double dbp = cb[sb][2] + cb[sb][3];  // d_b(r + 1)
        const double da0 = cb[sa][1] + cb[sa][2];  // d_a(r)
        const double ca1 = has_left ? cb[sa][1] : 0.0, cb1 = has_left ? cb[sb][1] : 0.0;
        const double ca2 = has_right ? cb[sa][2] : 0.0, cb2 = has_right ? cb[sb][2] : 0.0;
        // products that are later summed are rounded on their own (__dmul_rn is
        // never fused into a following addition), so every instantiation of the
        // kernel -- whatever its lanes per orbit -- computes the same numbers
        P[q][0] = __dmul_rn(cb[sa][1], cb[sb][0]);
        P[q][1] = -fma(cb[sa][1], dbm, __dmul_rn(da0, cb[sb][1]));
        P[q][2] = fma(ca1, cb1, fma(ca2, cb2, __dmul_rn(da0, db0)));
        P[q][3] = -fma(da0, cb[sb][2], __dmul_rn(cb[sa][2], dbp));
        P[q][4] = __dmul_rn(cb[sa][2], cb[sb][3]);
    }
    // stage sums of the bond stiffnesses on bonds r (t = 1) and r + 1 (t = 2)
    double s123[2], s23[2], s234[2], s1223[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        s23[t] = cb[1][t + 1] + cb[2][t + 1];
        s123[t] = s23[t] + cb[0][t + 1];
        s234[t] = s23[t] + cb[3][t + 1];
        s1223[t] = s123[t] + s234[t];
    }
    // A and D: I - h^2/6 S + h^4/24 P (S's off-diagonals are -s)
    out[0] = h4 * P[0][0];
    out[1] = fma(h4, P[0][1], h2 * s123[0]);
    out[2] = fma(h4, P[0][2], fma(-h2, s123[0] + s123[1], 1.0));
    out[3] = fma(h4, P[0][3], h2 * s123[1]);
    out[4] = h4 * P[0][4];
    out[13] = h4 * P[1][0];
    out[14] = fma(h4, P[1][1], h2 * s234[0]);
    out[15] = fma(h4, P[1][2], fma(-h2, s234[0] + s234[1], 1.0));
    out[16] = fma(h4, P[1][3], h2 * s234[1]);
    out[17] = h4 * P[1][4];
    // B: h I - h^3/12 S23
    out[5] = h3 * s23[0];
    out[6] = fma(-h3, s23[0] + s23[1], h);
    out[7] = h3 * s23[1];
    // C: -h/6 S1223 + h^3/12 (P31 + P42)
    out[8] = h3 * (P[0][0] + P[1][0]);
    out[9] = fma(h3, P[0][1] + P[1][1], h1 * s1223[0]);
    out[10] = fma(h3, P[0][2] + P[1][2], -h1 * (s1223[0] + s1223[1]));
    out[11] = fma(h3, P[0][3] + P[1][3], h1 * s1223[1]);
    out[12] = h3 * (P[0][4] + P[1][4]);
}

}  // namespace fput_phi
}  // namespace chs

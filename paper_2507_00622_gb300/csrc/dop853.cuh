// dop853.cuh -- device building blocks of the DOP853 kernels (k_dop853.cu,
// k_dop853_adapt.cu): the tableau, one orbit step and one deviation-vector step,
// the error norm of the adaptive pair, and the per-step checks.
//
// Design.  A step runs in two phases.  Phase 1 takes the orbit (and the LD
// integrand) through the twelve stages and records each stage's Hessian;
// phase 2 takes each deviation vector through the twelve stages of the linear
// variational equation w' = J_s w with those Hessians.  The vectors never act
// on the orbit, so this is DOP853 on the joint system (x, w_1..w_k, M_p), and an
// adaptive trial that is rejected costs only phase 1.  Stage derivatives and
// Hessians live in a per-thread column of shared memory, not in registers: on
// GB300 a warp's FP64 FMA occupies its sub-partition's FP64 unit for 64 cycles
// while a 64-bit shared-memory access costs about 2 cycles of the SM's shared-
// memory bandwidth, so the stage traffic is cheap next to the arithmetic and
// the registers stay free of the up to nine live stages of each phase.  The LD
// integrand is evaluated only at the eight stages with b_s != 0 (the LD never
// feeds back into a stage).  Every coefficient is a compile-time constant: the
// zero entries of the tableau generate no instructions.
#pragma once

#include <math.h>

#include <type_traits>

#include "k_dop853.cuh"
#include "rk4_common.cuh"

namespace chs {
namespace dp {

constexpr int kBlock = 32;  // threads per block (one warp: the shared slab sets occupancy)

// The DOP853 pair of Dormand and Prince as published in Hairer, Norsett and
// Wanner, Solving Ordinary Differential Equations I (2nd ed., Springer 1993),
// Sec. II.10.  Stages are numbered from 0.  kA: the strictly lower-triangular
// Runge-Kutta matrix (nodes c_s = sum_j a_sj); kB: the 8th-order weights;
// kE5: the 5th-order error weights b - bhat; kB3: the 3rd-order weights (on
// stages 0, 8 and 11), whose error weights are b - b3.
constexpr double kA[12][12] = {
    {0},
    {5.26001519587677318785587544488e-2},
    {1.97250569845378994544595329183e-2, 5.91751709536136983633785987549e-2},
    {2.95875854768068491816892993775e-2, 0.0, 8.87627564304205475450678981324e-2},
    {2.41365134159266685502369798665e-1, 0.0, -8.84549479328286085344864962717e-1,
     9.24834003261792003115737966543e-1},
    {3.7037037037037037037037037037e-2, 0.0, 0.0, 1.70828608729473871279604482173e-1,
     1.25467687566822425016691814123e-1},
    {3.7109375e-2, 0.0, 0.0, 1.70252211019544039314978060272e-1,
     6.02165389804559606850219397283e-2, -1.7578125e-2},
    {3.70920001185047927108779319836e-2, 0.0, 0.0, 1.70383925712239993810214054705e-1,
     1.07262030446373284651809199168e-1, -1.53194377486244017527936158236e-2,
     8.27378916381402288758473766002e-3},
    {6.24110958716075717114429577812e-1, 0.0, 0.0, -3.36089262944694129406857109825e0,
     -8.68219346841726006818189891453e-1, 2.75920996994467083049415600797e1,
     2.01540675504778934086186788979e1, -4.34898841810699588477366255144e1},
    {4.77662536438264365890433908527e-1, 0.0, 0.0, -2.48811461997166764192642586468e0,
     -5.90290826836842996371446475743e-1, 2.12300514481811942347288949897e1,
     1.52792336328824235832596922938e1, -3.32882109689848629194453265587e1,
     -2.03312017085086261358222928593e-2},
    {-9.3714243008598732571704021658e-1, 0.0, 0.0, 5.18637242884406370830023853209e0,
     1.09143734899672957818500254654e0, -8.14978701074692612513997267357e0,
     -1.85200656599969598641566180701e1, 2.27394870993505042818970056734e1,
     2.49360555267965238987089396762e0, -3.0467644718982195003823669022e0},
    {2.27331014751653820792359768449e0, 0.0, 0.0, -1.05344954667372501984066689879e1,
     -2.00087205822486249909675718444e0, -1.79589318631187989172765950534e1,
     2.79488845294199600508499808837e1, -2.85899827713502369474065508674e0,
     -8.87285693353062954433549289258e0, 1.23605671757943030647266201528e1,
     6.43392746015763530355970484046e-1},
};
constexpr double kB[12] = {
    5.42937341165687622380535766363e-2, 0.0, 0.0, 0.0, 0.0, 4.45031289275240888144113950566e0,
    1.89151789931450038304281599044e0, -5.8012039600105847814672114227e0,
    3.1116436695781989440891606237e-1, -1.52160949662516078556178806805e-1,
    2.01365400804030348374776537501e-1, 4.47106157277725905176885569043e-2};
constexpr double kE5[12] = {
    1.312004499419488073250102996e-2, 0.0, 0.0, 0.0, 0.0, -1.225156446376204440720569753e0,
    -4.957589496572501915214079952e-1, 1.664377182454986536961530415e0,
    -3.503288487499736816886487290e-1, 3.341791187130174790297318841e-1,
    8.192320648511571246570742613e-2, -2.235530786388629525884427845e-2};
constexpr double kB3[12] = {
    2.44094488188976377952755905512e-1, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    7.33846688281611857341361741547e-1, 0.0, 0.0, 2.20588235294117647058823529412e-2};

// Compile-time loop: f(integral_constant<int, I>) for I = B .. E-1.
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// True when a later stage reads stage j.
constexpr bool read_later(int j)
{
    for (int s = j + 1; s < 12; ++s)
        if (kA[s][j] != 0.0) return true;
    return false;
}
template <int J>
constexpr bool kReadLater = read_later(J);
static_assert(!read_later(11), "the last stage is never read by another stage");

// The last stage that reads stage j's derivative (-1: none).
constexpr int last_reader(int j)
{
    int r = -1;
    for (int s = j + 1; s < 12; ++s)
        if (kA[s][j] != 0.0) r = s;
    return r;
}

// Slab row of stage s's derivative: the lowest row whose occupant no stage
// after s reads (a stage reads all of its inputs before it writes its own
// derivative, so a row read last by stage s itself can take it); -1 for a
// stage that no later stage reads.  Stages 2 and 3 of the pair are read only
// up to stages 3 and 5, so 11 derivatives fit in 9 rows.
constexpr int k_row(int s)
{
    int occ[12] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
    for (int t = 0; t <= s; ++t) {
        if (!read_later(t)) {
            if (t == s) return -1;
            continue;
        }
        int row = 0;
        while (occ[row] >= 0 && last_reader(occ[row]) > t) ++row;
        occ[row] = t;
        if (t == s) return row;
    }
    return -1;
}
constexpr int k_rows()
{
    int n = 0;
    for (int s = 0; s < 12; ++s)
        if (k_row(s) + 1 > n) n = k_row(s) + 1;
    return n;
}
template <int S>
constexpr int kRow = k_row(S);
static_assert(k_rows() == 9, "the DOP853 pair's derivatives fit in 9 rows");

// A thread's column of the block's shared array: H[s][t] (stage Hessians,
// packed upper triangle, 12 stages) then the stage derivatives a later stage
// reads, in the k_rows() rows given by k_row, entry e at base[e * kBlock].
// Accesses are volatile so that stage values are re-read from shared memory
// instead of being kept in registers.
template <class Sys>
struct Slab {
    static constexpr int D = 2 * Sys::N, NH = Sys::NH;
    static constexpr int kDoubles = 12 * NH + k_rows() * D;
    volatile double* base;
    __device__ __forceinline__ volatile double& H(int s, int t) const { return base[(s * NH + t) * kBlock]; }
    template <int S>
    __device__ __forceinline__ volatile double& K(int i) const
    {
        static_assert(kRow<S> >= 0, "a stage derivative that no later stage reads is not stored");
        return base[(12 * NH + kRow<S> * D + i) * kBlock];
    }
};

template <class Sys>
__device__ __forceinline__ Slab<Sys> my_slab()
{
    extern __shared__ double dsm[];
    return Slab<Sys>{dsm + threadIdx.x};
}

template <class Sys>
constexpr size_t slab_bytes()
{
    return (size_t)Slab<Sys>::kDoubles * kBlock * sizeof(double);
}

// sum_{j<S} a_Sj K_j[i] over the nonzero a_Sj (0 for S = 0).
template <int S, class Sys>
__device__ __forceinline__ double stage_sum(const Slab<Sys>& sl, const int i)
{
    double acc = 0.0;
    static_for<0, S>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        constexpr double c = kA[S][j];
        if constexpr (c != 0.0) acc = fma(c, sl.template K<j>(i), acc);
    });
    return acc;
}

// Phase 1, the orbit's twelve stages from x with step h:
//   K_s = f(x + h sum_{j<s} a_sj K_j),   xn = x + h sum_s b_s K_s,
//   dL = |h| sum_s b_s g(K_s)  (g the LD integrand; the LD grows with |t|),
// the stage Hessians into the slab, and with ERR the error sums
// err5_i = sum_s e5_s K_s,i and err3_i = sum_s (b_s - b3_s) K_s,i.
template <class Sys, bool LD, bool ERR>
__device__ __forceinline__ void orbit_step(const Slab<Sys>& sl, const double* x, const double h,
                                           const int ld_sqrt, const double ld_p, const SysPar& sp,
                                           double* xn, double& dL, double* e5, double* e3)
{
    constexpr int D = 2 * Sys::N, NH = Sys::NH;
    double sb[D], s5[D], s3[D];
    double sL = 0.0;
    static_for<0, 12>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        double xs[D], f[D], H[NH];
#pragma unroll
        for (int i = 0; i < D; ++i) xs[i] = (s == 0) ? x[i] : fma(h, stage_sum<s>(sl, i), x[i]);
        Sys::eval(xs, f, H, sp);
#pragma unroll
        for (int t = 0; t < NH; ++t) sl.H(s, t) = H[t];
        if constexpr (kReadLater<s>) {
#pragma unroll
            for (int i = 0; i < D; ++i) sl.template K<s>(i) = f[i];
        }
        constexpr double cb = kB[s], c5 = kE5[s], c3 = kB[s] - kB3[s];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            if constexpr (s == 0) {
                sb[i] = cb * f[i];
                if constexpr (ERR) {
                    s5[i] = c5 * f[i];
                    s3[i] = c3 * f[i];
                }
            } else {
                if constexpr (cb != 0.0) sb[i] = fma(cb, f[i], sb[i]);
                if constexpr (ERR && c5 != 0.0) s5[i] = fma(c5, f[i], s5[i]);
                if constexpr (ERR && c3 != 0.0) s3[i] = fma(c3, f[i], s3[i]);
            }
        }
        if constexpr (LD && cb != 0.0) {
            // p = 1/2: the stage's sum of square roots in double-float, widened once
            const double g = ld_sqrt ? ff_to_f64(ff_sum_sqrt_abs<D>(f)) : ld_integrand_pow<D>(f, ld_p);
            sL = fma(cb, g, sL);
        }
    });
#pragma unroll
    for (int i = 0; i < D; ++i) {
        xn[i] = fma(h, sb[i], x[i]);
        if constexpr (ERR) {
            e5[i] = s5[i];
            e3[i] = s3[i];
        }
    }
    if constexpr (LD) dL = fabs(h) * sL;
}

// Phase 2, one deviation vector w = (dq, dp) through the twelve stages of
// w' = J_s w, J_s w = (dp, -H_s dq), with the Hessians of phase 1:
//   M_s = J_s (w + h sum_{j<s} a_sj M_j),   w <- w + h sum_s b_s M_s.
// The stage derivatives M_s reuse the slab's K rows.
template <class Sys>
__device__ __forceinline__ void vector_step(const Slab<Sys>& sl, double* w, const double h)
{
    constexpr int N = Sys::N, D = 2 * N, NH = Sys::NH;
    double sb[D];
    static_for<0, 12>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        double ws[D], m[D], H[NH];
#pragma unroll
        for (int i = 0; i < D; ++i) ws[i] = (s == 0) ? w[i] : fma(h, stage_sum<s>(sl, i), w[i]);
#pragma unroll
        for (int t = 0; t < NH; ++t) H[t] = sl.H(s, t);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            m[i] = ws[N + i];
            double acc = H[hidx<N>(i, 0)] * ws[0];
#pragma unroll
            for (int q = 1; q < N; ++q) acc = fma(H[hidx<N>(i, q)], ws[q], acc);
            m[N + i] = -acc;
        }
        if constexpr (kReadLater<s>) {
#pragma unroll
            for (int i = 0; i < D; ++i) sl.template K<s>(i) = m[i];
        }
        constexpr double cb = kB[s];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            if constexpr (s == 0)
                sb[i] = cb * m[i];
            else if constexpr (cb != 0.0)
                sb[i] = fma(cb, m[i], sb[i]);
        }
    });
#pragma unroll
    for (int i = 0; i < D; ++i) w[i] = fma(h, sb[i], w[i]);
}

// Error norm of a trial over the orbit components:
//   scale_i = atol + rtol max(|x_i|, |xn_i|),  E5 = sum (err5_i / scale_i)^2,
//   E3 likewise, err = |h| E5 / sqrt(D (E5 + 0.01 E3)) (0 when both vanish).
template <int D>
__device__ __forceinline__ double err_norm(const double* x, const double* xn, const double* e5,
                                           const double* e3, const double h, const double atol,
                                           const double rtol)
{
    double E5 = 0.0, E3 = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        const double sc = atol + rtol * fmax(fabs(x[i]), fabs(xn[i]));
        const double q5 = e5[i] / sc, q3 = e3[i] / sc;
        E5 = fma(q5, q5, E5);
        E3 = fma(q3, q3, E3);
    }
    if (E5 == 0.0 && E3 == 0.0) return 0.0;
    return fabs(h) * E5 / sqrt((double)D * (E5 + 0.01 * E3));
}

// SALI of two vectors (each normalised first): min(|u + v|, |u - v|).
template <int D>
__device__ __forceinline__ double sali2(const double* a, const double* b)
{
    double na = a[0] * a[0], nb = b[0] * b[0];
#pragma unroll
    for (int c = 1; c < D; ++c) {
        na = fma(a[c], a[c], na);
        nb = fma(b[c], b[c], nb);
    }
    const double ia = rsqrt_nr(na), ib = rsqrt_nr(nb);
    double sp = 0.0, sm = 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const double u = a[c] * ia, v = b[c] * ib;
        sp = fma(u + v, u + v, sp);
        sm = fma(u - v, u - v, sm);
    }
    return sqrt(fmin(sp, sm));
}

// What follows every completed step (the chs_integrate_batch contract):
// renormalisation, escape, and at health checks finiteness, energy drift and
// the early exit.  Returns the orbit status.
template <class Sys, int K>
__device__ __forceinline__ int32_t post_step(const double* x, double (*w)[2 * Sys::N],
                                             const double L, const StepArgs& a, const SysPar& sp,
                                             const bool check, const double h0, double& dhm)
{
    constexpr int N = Sys::N, D = 2 * N;
    if (a.renorm) {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            double n2 = w[j][0] * w[j][0];
#pragma unroll
            for (int c = 1; c < D; ++c) n2 = fma(w[j][c], w[j][c], n2);
            const double inv = rsqrt_ff(n2);
#pragma unroll
            for (int c = 0; c < D; ++c) w[j][c] *= inv;
        }
    }
    if (a.escape_r2 > 0.0) {
        double r2 = x[0] * x[0];
#pragma unroll
        for (int i = 1; i < N; ++i) r2 = fma(x[i], x[i], r2);
        if (r2 > a.escape_r2) return CHS_ORBIT_ESCAPED;
    }
    if (check) {
        bool fin = isfinite(L);
#pragma unroll
        for (int c = 0; c < D; ++c) fin = fin && isfinite(x[c]);
#pragma unroll
        for (int j = 0; j < K; ++j)
#pragma unroll
            for (int c = 0; c < D; ++c) fin = fin && isfinite(w[j][c]);
        if (!fin) return CHS_ORBIT_NONFINITE;
        const double dH = fabs(Sys::energy(x, sp) - h0);
        dhm = fmax(dhm, dH);
        if (a.dh_limit > 0.0 && dH > a.dh_limit) return CHS_ORBIT_ENERGY_DRIFT;
        if constexpr (K >= 2) {
            if (a.early_exit && sali2<D>(w[0], w[1]) < a.sali_threshold) return CHS_ORBIT_EARLY_CHAOTIC;
        }
    }
    return CHS_ORBIT_OK;
}

// Calls f(integral_constant<int, K>) for the runtime vector count k, within
// the counts the system supports (k <= 4 for 2 DOF, k <= 6 for 3 DOF).
template <class Sys, class F>
cudaError_t with_k(int k, F&& f)
{
    switch (k) {
    case 0: f(std::integral_constant<int, 0>{}); break;
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 5:
        if constexpr (Sys::N >= 3) {
            f(std::integral_constant<int, 5>{});
            break;
        }
        return cudaErrorInvalidValue;
    case 6:
        if constexpr (Sys::N >= 3) {
            f(std::integral_constant<int, 6>{});
            break;
        }
        return cudaErrorInvalidValue;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace dp
}  // namespace chs

/*
 * chs_oracle.c -- plain, slow CPU oracle for the chaos-indicator hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA library: every formula here
 * is written out again from the paper (arXiv 2507.00622, "Chaoticus") and
 * from the textbook definitions of the indicators the paper cites.
 *
 * Arithmetic: IEEE double, compiled with -ffp-contract=off so that every
 * expression is evaluated exactly in the order written.
 *
 * Layout of every ensemble array: structure of arrays, a[c * n + o] for
 * component c of orbit o.  Phase-space vectors are ordered (q_1..q_N,
 * p_1..p_N); deviation vector j occupies components [j*d, (j+1)*d) of w.
 *
 * What each routine follows:
 *   o_energy / o_rhs / o_hessian   Hamiltonians and Hamilton's equations:
 *                                  Henon-Heiles (Eqs. Ham_HH, ham_eqs_HH),
 *                                  FPUT chain with fixed ends (Eqs. ham_FPU,
 *                                  ham_eqs_FPU and q_0 = q_{N+1} = 0), the
 *                                  3-DOF quartic oscillator, and the harmonic
 *                                  and inverted test oscillators.
 *   o_integrate                    classic fixed-step RK4 (the configs' fixed
 *                                  step integrator in place of the paper's
 *                                  DOP8, Sec. Functionalities) on the joint
 *                                  system (x, w_1..w_k, L): deviation vectors
 *                                  obey the variational equations (Sec.
 *                                  Statement of need), are renormalised after
 *                                  every step (the vector-normalising solver
 *                                  variant listed in Sec. Functionalities)
 *                                  and L is the Lagrangian
 *                                  descriptor M_p = int sum_i |dx_i/dt|^p dt
 *                                  (Sec. Statement of need, refs mancho2013,
 *                                  lopesino2017).  A 4th-order Yoshida
 *                                  splitting with its tangent map is kept as
 *                                  an independent cross-check integrator.
 *   o_dop853_step                  the paper's own 8th-order solver (DOP 8,
 *                                  Sec. Functionalities, ref prince1981):
 *                                  the DOP853 pair of Dormand and Prince as
 *                                  published in Hairer, Norsett and Wanner,
 *                                  Solving Ordinary Differential Equations I
 *                                  (2nd ed., Sec. II.10), in fixed-step use.
 *   o_integrate_adaptive           DOP 8(5) with adaptive step size and the
 *                                  per-step error (Sec. Functionalities):
 *                                  the same pair with its 5th/3rd-order error
 *                                  estimate and the standard step-size
 *                                  controller (Hairer et al., Sec. II.4).
 *   o_indicators                   SALI (refs Skokos2001/03/04) and GALI_k as
 *                                  the product of the singular values of the
 *                                  d x k matrix of unit deviation vectors,
 *                                  from a one-sided Jacobi SVD (GALI item of
 *                                  Sec. Functionalities, ref Skokos2008).
 *   o_ld_indicators                LD-based indicators D_L and S_L from grid
 *                                  neighbours (LD-indicator and neighbouring-
 *                                  trajectory items of Sec. Functionalities).
 *   o_lyapunov                     Lyapunov spectrum by periodic QR (modified
 *                                  Gram-Schmidt) of the 2N deviation vectors
 *                                  (Lyapunov item of Sec. Functionalities and
 *                                  the FPU example, Sec. Examples).
 *   o_grid_ics / o_fput_mode_ics   initial conditions: the x = 0 section grid
 *                                  of Henon-Heiles and normal-mode FPUT states
 *                                  scaled onto an energy shell.
 *   o_seed_vectors                 deviation vectors uniform in [-1, 1) from
 *                                  the SplitMix64 generator (Steele, Lea and
 *                                  Flood, OOPSLA 2014), then normalised.
 *   o_ensemble_init                the ensemble's start: state, H0 from the
 *                                  Hamiltonians above, statuses, and the
 *                                  deviation vectors (given or seeded).
 *   o_lyapunov_adaptive            the Lyapunov spectrum under DOP 8(5) (the
 *                                  adaptive solver with QR, Sec.
 *                                  Functionalities).
 *   o_dop853_tableau               the pair's coefficients (Hairer et al.,
 *                                  Sec. II.10), for the order-condition pins.
 *   o_shell_ics                    quartic-oscillator states scaled onto an
 *                                  energy shell (a test system outside the
 *                                  paper; the radial scaling of the FPU
 *                                  normal-mode states).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { O_HENON_HEILES = 1, O_FPUT = 2, O_QUARTIC3 = 3, O_HARMONIC = 100, O_INVERTED = 101 };
enum { OS_OK = 0, OS_FORBIDDEN = 1, OS_ESCAPED = 2, OS_NONFINITE = 3, OS_ENERGY_DRIFT = 4,
       OS_EARLY_CHAOTIC = 5, OS_STEP_FAIL = 7 };
enum { OI_RK4 = 0, OI_YOSHIDA4 = 1, OI_DOP853 = 2 };

typedef struct {
    int model;
    int n_dof;
    double kk;     /* FPUT linear spring constant k */
    double alpha;  /* FPUT cubic coefficient */
    double beta;   /* FPUT quartic coefficient */
    double eps;    /* quartic-oscillator coupling */
} o_system;

typedef struct {
    double dt;
    int64_t n_steps;
    int64_t step0;        /* absolute index of the last step taken before this call */
    int n_dev;            /* number k of deviation vectors */
    int renorm;           /* 1: normalise every deviation vector after each step */
    int sample_every;     /* health checks at absolute steps divisible by this */
    int qr_every;         /* Lyapunov: QR at steps divisible by this (and the last) */
    int integrator;       /* OI_RK4, OI_YOSHIDA4 or OI_DOP853 */
    double ld_p;          /* exponent p of the LD; 0 switches the LD off */
    double escape_r2;     /* escape when sum_i q_i^2 exceeds this; 0 = off */
    double dh_limit;      /* ENERGY_DRIFT when |H - H0| exceeds this; 0 = off */
    int early_exit;       /* 1: stop as EARLY_CHAOTIC once SALI < sali_threshold at a health check */
    double sali_threshold;
} o_params;

/* ------------------------------------------------------------------------ */
/* Hamiltonians                                                              */
/* ------------------------------------------------------------------------ */

/* Spring potential of the FPUT chain, per bond: k/2 r^2 + alpha/3 r^3 + beta/4 r^4 (Eq. ham_FPU). */
static double fput_bond_v(const o_system* s, double r)
{
    return s->kk / 2.0 * r * r + s->alpha / 3.0 * r * r * r + s->beta / 4.0 * r * r * r * r;
}

/* FPUT bond elongation D_i = q_i - q_{i-1}, i = 1..N+1, with q_0 = q_{N+1} = 0. */
static double fput_bond(const double* q, int N, int i)
{
    double qi = (i >= 1 && i <= N) ? q[i - 1] : 0.0;
    double qm = (i - 1 >= 1 && i - 1 <= N) ? q[i - 2] : 0.0;
    return qi - qm;
}

double o_energy(const o_system* s, const double* x)
{
    int N = s->n_dof;
    const double* q = x;
    const double* p = x + N;
    double T = 0.0;
    for (int i = 0; i < N; ++i) T += p[i] * p[i] / 2.0;
    double V = 0.0;
    switch (s->model) {
    case O_HENON_HEILES:  /* Eq. Ham_HH: 1/2 (x^2 + y^2) + x^2 y - y^3 / 3 */
        V = (q[0] * q[0] + q[1] * q[1]) / 2.0 + q[0] * q[0] * q[1] - q[1] * q[1] * q[1] / 3.0;
        break;
    case O_FPUT:  /* Eq. ham_FPU, summed over the N+1 bonds that the fixed ends create */
        for (int i = 1; i <= N + 1; ++i) V += fput_bond_v(s, fput_bond(q, N, i));
        break;
    case O_QUARTIC3:  /* 1/2 sum q_i^2 + eps (q1^2 q2^2 + q2^2 q3^2 + q1^2 q3^2) */
        V = (q[0] * q[0] + q[1] * q[1] + q[2] * q[2]) / 2.0
          + s->eps * (q[0] * q[0] * q[1] * q[1] + q[1] * q[1] * q[2] * q[2] + q[0] * q[0] * q[2] * q[2]);
        break;
    case O_HARMONIC:
        for (int i = 0; i < N; ++i) V += q[i] * q[i] / 2.0;
        break;
    case O_INVERTED:  /* 1/2 (p1^2 - q1^2) + 1/2 (p2^2 + q2^2) */
        V = -q[0] * q[0] / 2.0 + q[1] * q[1] / 2.0;
        break;
    }
    return T + V;
}

/* Gradient of the potential, dV/dq_i. */
static void o_grad_v(const o_system* s, const double* q, double* g)
{
    int N = s->n_dof;
    switch (s->model) {
    case O_HENON_HEILES:  /* from Eq. ham_eqs_HH: p_x' = -x - 2xy, p_y' = -y - x^2 + y^2 */
        g[0] = q[0] + 2.0 * q[0] * q[1];
        g[1] = q[1] + q[0] * q[0] - q[1] * q[1];
        break;
    case O_FPUT:  /* from Eq. ham_eqs_FPU: dV/dq_i = V'(D_i) - V'(D_{i+1}) */
        for (int i = 1; i <= N; ++i) {
            double a = fput_bond(q, N, i), b = fput_bond(q, N, i + 1);
            double fa = s->kk * a + s->alpha * a * a + s->beta * a * a * a;
            double fb = s->kk * b + s->alpha * b * b + s->beta * b * b * b;
            g[i - 1] = fa - fb;
        }
        break;
    case O_QUARTIC3: {
        double S = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
        for (int i = 0; i < 3; ++i) g[i] = q[i] + 2.0 * s->eps * q[i] * (S - q[i] * q[i]);
        break;
    }
    case O_HARMONIC:
        for (int i = 0; i < N; ++i) g[i] = q[i];
        break;
    case O_INVERTED:
        g[0] = -q[0];
        g[1] = q[1];
        break;
    }
}

/* Hamilton's equations: dq/dt = p, dp/dt = -grad V. */
void o_rhs(const o_system* s, const double* x, double* f)
{
    int N = s->n_dof;
    double g[256];
    o_grad_v(s, x, g);
    for (int i = 0; i < N; ++i) {
        f[i] = x[N + i];
        f[N + i] = -g[i];
    }
}

/* Dense Hessian of the potential, Hm[i * N + j] = d^2 V / dq_i dq_j. */
void o_hessian(const o_system* s, const double* q, double* Hm)
{
    int N = s->n_dof;
    for (int i = 0; i < N * N; ++i) Hm[i] = 0.0;
    switch (s->model) {
    case O_HENON_HEILES:
        Hm[0] = 1.0 + 2.0 * q[1];
        Hm[1] = 2.0 * q[0];
        Hm[2] = 2.0 * q[0];
        Hm[3] = 1.0 - 2.0 * q[1];
        break;
    case O_FPUT:
        /* bond i (D_i) couples q_{i-1} and q_i with stiffness c_i = V''(D_i) */
        for (int i = 1; i <= N + 1; ++i) {
            double r = fput_bond(q, N, i);
            double c = s->kk + 2.0 * s->alpha * r + 3.0 * s->beta * r * r;
            int a = i - 2, b = i - 1; /* zero-based indices of q_{i-1}, q_i */
            if (a >= 0) Hm[a * N + a] += c;
            if (b <= N - 1) Hm[b * N + b] += c;
            if (a >= 0 && b <= N - 1) {
                Hm[a * N + b] -= c;
                Hm[b * N + a] -= c;
            }
        }
        break;
    case O_QUARTIC3: {
        double S = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                Hm[i * 3 + j] = (i == j) ? 1.0 + 2.0 * s->eps * (S - q[i] * q[i])
                                         : 4.0 * s->eps * q[i] * q[j];
        break;
    }
    case O_HARMONIC:
        for (int i = 0; i < N; ++i) Hm[i * N + i] = 1.0;
        break;
    case O_INVERTED:
        Hm[0] = -1.0;
        Hm[3] = 1.0;
        break;
    }
}

/* ------------------------------------------------------------------------ */
/* Joint system (x, w_1..w_k, L) and its RK4 step                            */
/* ------------------------------------------------------------------------ */

typedef struct {
    const o_system* s;
    int d, k, ld;
    double ld_p;
    double* Hm;   /* N*N scratch */
    double ld_sign; /* sign of the step: the LD grows with |t| */
} o_joint;

/* F(z): z = [x | w_1 | ... | w_k | L].  Variational equations: for w = (dq, dp),
 * d(dq)/dt = dp and d(dp)/dt = -Hess V(q) dq.  LD: dL/dt = sgn(h) sum_i |f_i(x)|^p,
 * so that L = int sum_i |f_i|^p d|t| grows in backward runs (h < 0) too. */
static void o_joint_f(const o_joint* J, const double* z, double* dz)
{
    int d = J->d, N = d / 2;
    o_rhs(J->s, z, dz);
    o_hessian(J->s, z, J->Hm);
    for (int j = 0; j < J->k; ++j) {
        const double* w = z + d + j * d;
        double* dw = dz + d + j * d;
        for (int i = 0; i < N; ++i) dw[i] = w[N + i];
        for (int i = 0; i < N; ++i) {
            double acc = 0.0;
            for (int m = 0; m < N; ++m) acc += J->Hm[i * N + m] * w[m];
            dw[N + i] = -acc;
        }
    }
    if (J->ld) {
        double acc = 0.0;
        for (int i = 0; i < d; ++i) acc += pow(fabs(dz[i]), J->ld_p);
        dz[d + J->k * d] = J->ld_sign * acc;
    }
}

/* Classic RK4: k1 = F(z), k2 = F(z + h/2 k1), k3 = F(z + h/2 k2), k4 = F(z + h k3),
 * z <- z + h/6 (k1 + 2 k2 + 2 k3 + k4). */
static void o_rk4_step(const o_joint* J, double* z, int D, double h, double* k1, double* k2,
                       double* k3, double* k4, double* zt)
{
    o_joint_f(J, z, k1);
    for (int i = 0; i < D; ++i) zt[i] = z[i] + h / 2.0 * k1[i];
    o_joint_f(J, zt, k2);
    for (int i = 0; i < D; ++i) zt[i] = z[i] + h / 2.0 * k2[i];
    o_joint_f(J, zt, k3);
    for (int i = 0; i < D; ++i) zt[i] = z[i] + h * k3[i];
    o_joint_f(J, zt, k4);
    for (int i = 0; i < D; ++i) z[i] = z[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

/* 4th-order Yoshida composition of the drift-kick-drift leapfrog, for
 * separable H = |p|^2/2 + V(q), carried over to the deviation vectors by its
 * tangent map (drift: dq += tau dp; kick: dp -= tau Hess V(q) dq).  Yoshida
 * (Phys. Lett. A 150, 1990): w1 = 1/(2 - 2^(1/3)), w0 = -2^(1/3)/(2 - 2^(1/3)). */
static void o_yoshida_drift(const o_joint* J, double* z, double tau)
{
    int d = J->d, N = d / 2;
    for (int i = 0; i < N; ++i) z[i] += tau * z[N + i];
    for (int j = 0; j < J->k; ++j) {
        double* w = z + d + j * d;
        for (int i = 0; i < N; ++i) w[i] += tau * w[N + i];
    }
}

static void o_yoshida_kick(const o_joint* J, double* z, double tau)
{
    int d = J->d, N = d / 2;
    double g[256];
    o_grad_v(J->s, z, g);
    o_hessian(J->s, z, J->Hm);
    for (int j = 0; j < J->k; ++j) {
        double* w = z + d + j * d;
        for (int i = 0; i < N; ++i) {
            double acc = 0.0;
            for (int m = 0; m < N; ++m) acc += J->Hm[i * N + m] * w[m];
            w[N + i] -= tau * acc;
        }
    }
    for (int i = 0; i < N; ++i) z[N + i] -= tau * g[i];
}

static void o_yoshida_step(const o_joint* J, double* z, double h)
{
    double cbrt2 = cbrt(2.0);
    double w1 = 1.0 / (2.0 - cbrt2);
    double w0 = -cbrt2 / (2.0 - cbrt2);
    double c[3] = {w1, w0, w1};
    for (int m = 0; m < 3; ++m) {
        o_yoshida_drift(J, z, c[m] * h / 2.0);
        o_yoshida_kick(J, z, c[m] * h);
        o_yoshida_drift(J, z, c[m] * h / 2.0);
    }
}

/* ------------------------------------------------------------------------ */
/* DOP853: 12-stage explicit Runge-Kutta pair of order 8(5,3)                */
/* ------------------------------------------------------------------------ */

/* Coefficients of the DOP853 pair of Dormand and Prince (Hairer, Norsett and
 * Wanner, Solving ODEs I, 2nd ed., Sec. II.10): nodes c_s (implied: c_s =
 * sum_j a_sj), the strictly lower-triangular a_sj, the 8th-order weights b_s,
 * the 5th-order error weights e5_s = b_s - bhat_s, and the 3rd-order weights
 * b3_s on stages 1, 9 and 12 (error weights b_s - b3_s).  Stages are numbered
 * from 0 here. */
static const double o_dp_a[12][11] = {
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
static const double o_dp_b[12] = {
    5.42937341165687622380535766363e-2, 0.0, 0.0, 0.0, 0.0, 4.45031289275240888144113950566e0,
    1.89151789931450038304281599044e0, -5.8012039600105847814672114227e0,
    3.1116436695781989440891606237e-1, -1.52160949662516078556178806805e-1,
    2.01365400804030348374776537501e-1, 4.47106157277725905176885569043e-2};
static const double o_dp_e5[12] = {
    1.312004499419488073250102996e-2, 0.0, 0.0, 0.0, 0.0, -1.225156446376204440720569753e0,
    -4.957589496572501915214079952e-1, 1.664377182454986536961530415e0,
    -3.503288487499736816886487290e-1, 3.341791187130174790297318841e-1,
    8.192320648511571246570742613e-2, -2.235530786388629525884427845e-2};
static const double o_dp_b3[12] = {
    2.44094488188976377952755905512e-1, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    7.33846688281611857341361741547e-1, 0.0, 0.0, 2.20588235294117647058823529412e-2};

/* Copies the tableau out (for the order-condition tests): a [12][12]
 * row-major (zeros above the diagonal), b, e5, b3 [12]. */
void o_dop853_tableau(double* a, double* b, double* e5, double* b3)
{
    for (int s = 0; s < 12; ++s) {
        for (int j = 0; j < 12; ++j) a[s * 12 + j] = (j < s) ? o_dp_a[s][j] : 0.0;
        b[s] = o_dp_b[s];
        e5[s] = o_dp_e5[s];
        b3[s] = o_dp_b3[s];
    }
}

/* One DOP853 step of size h from z (length D) into zn:
 *   K_s = F(z + h sum_{j<s} a_sj K_j),  s = 0..11,
 *   zn  = z + h sum_s b_s K_s,
 * and the error estimates (without the factor h) err5_i = sum_s e5_s K_s,i and
 * err3_i = sum_s (b_s - b3_s) K_s,i.  K holds 12*D doubles, zt D doubles. */
static void o_dop853_step(const o_joint* J, const double* z, double* zn, int D, double h,
                          double* K, double* zt, double* err5, double* err3)
{
    for (int s = 0; s < 12; ++s) {
        for (int i = 0; i < D; ++i) {
            double acc = 0.0;
            for (int j = 0; j < s; ++j) acc += o_dp_a[s][j] * K[j * D + i];
            zt[i] = z[i] + h * acc;
        }
        o_joint_f(J, zt, K + s * D);
    }
    for (int i = 0; i < D; ++i) {
        double sb = 0.0, s5 = 0.0, s3 = 0.0;
        for (int s = 0; s < 12; ++s) {
            sb += o_dp_b[s] * K[s * D + i];
            s5 += o_dp_e5[s] * K[s * D + i];
            s3 += (o_dp_b[s] - o_dp_b3[s]) * K[s * D + i];
        }
        zn[i] = z[i] + h * sb;
        if (err5) err5[i] = s5;
        if (err3) err3[i] = s3;
    }
}

/* Error norm of a DOP853 step over the first m components (the orbit):
 *   sc_i = atol + rtol max(|z_i|, |zn_i|),
 *   E5 = sum_i (err5_i / sc_i)^2,  E3 = sum_i (err3_i / sc_i)^2,
 *   err = |h| E5 / sqrt(m (E5 + 0.01 E3))     (0 when E5 = E3 = 0),
 * the combined 5th/3rd-order estimate of the DOP853 pair. */
static double o_dop853_err(const double* z, const double* zn, const double* err5,
                           const double* err3, int m, double h, double atol, double rtol)
{
    double E5 = 0.0, E3 = 0.0;
    for (int i = 0; i < m; ++i) {
        double a = fabs(z[i]), b = fabs(zn[i]);
        double sc = atol + rtol * (a > b ? a : b);
        E5 += (err5[i] / sc) * (err5[i] / sc);
        E3 += (err3[i] / sc) * (err3[i] / sc);
    }
    if (E5 == 0.0 && E3 == 0.0) return 0.0;
    return fabs(h) * E5 / sqrt((double)m * (E5 + 0.01 * E3));
}

static double o_norm(const double* v, int d)
{
    double acc = 0.0;
    for (int i = 0; i < d; ++i) acc += v[i] * v[i];
    return sqrt(acc);
}

static int o_all_finite(const double* z, int D)
{
    for (int i = 0; i < D; ++i)
        if (!isfinite(z[i])) return 0;
    return 1;
}

static int o_threads(int nthreads)
{
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int o_max_threads(void) { return o_threads(0); }

/* ------------------------------------------------------------------------ */
/* Ensemble set-up                                                           */
/* ------------------------------------------------------------------------ */

/* SplitMix64: the state advances by the golden-ratio increment and each output
 * is the published finaliser applied to the new state. */
uint64_t o_splitmix64_next(uint64_t* state)
{
    uint64_t z = (*state += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Component c of deviation vector j of orbit o is the m-th output (m = 1, 2, ...)
 * of the SplitMix64 stream that starts from `seed`, with m = (o*k + j)*d + c + 1,
 * mapped to [-1, 1) through its top 53 bits.  Each vector is then normalised. */
void o_seed_vectors(uint64_t seed, int64_t n, int k, int d, double* w)
{
    for (int64_t o = 0; o < n; ++o) {
        for (int j = 0; j < k; ++j) {
            double v[256];
            for (int c = 0; c < d; ++c) {
                uint64_t st = seed + (uint64_t)(((uint64_t)o * (uint64_t)k + (uint64_t)j) * (uint64_t)d + (uint64_t)c)
                                     * 0x9e3779b97f4a7c15ULL;
                uint64_t z = o_splitmix64_next(&st);
                double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
                v[c] = 2.0 * u - 1.0;
            }
            double nr = o_norm(v, d);
            for (int c = 0; c < d; ++c) w[((int64_t)j * d + c) * n + o] = v[c] / nr;
        }
    }
}

/* Henon-Heiles initial conditions on the x = 0 surface of section: a
 * cell-centred ny x npy grid over [y0, y1] x [py0, py1], orbit index
 * o = iy * npy + ipy, p_x >= 0 fixed by H = E (Eq. Ham_HH at x = 0):
 *   p_x^2 = 2E - p_y^2 - y^2 + 2 y^3 / 3.
 * A negative radicand marks the cell FORBIDDEN (state set to NaN). */
void o_grid_ics(double E, double y0, double y1, int ny, double py0, double py1, int npy,
                double* ics, int32_t* status)
{
    int64_t n = (int64_t)ny * npy;
    double dy = (y1 - y0) / ny;
    double dpy = (py1 - py0) / npy;
    for (int iy = 0; iy < ny; ++iy) {
        for (int ip = 0; ip < npy; ++ip) {
            int64_t o = (int64_t)iy * npy + ip;
            double y = y0 + ((double)iy + 0.5) * dy;
            double py = py0 + ((double)ip + 0.5) * dpy;
            double rad = 2.0 * E - py * py - y * y + 2.0 * y * y * y / 3.0;
            if (rad < 0.0) {
                status[o] = OS_FORBIDDEN;
                for (int c = 0; c < 4; ++c) ics[c * n + o] = NAN;
            } else {
                status[o] = OS_OK;
                ics[0 * n + o] = 0.0;
                ics[1 * n + o] = y;
                ics[2 * n + o] = sqrt(rad);
                ics[3 * n + o] = py;
            }
        }
    }
}

/* FPUT initial conditions from normal-mode amplitudes (Q_m, P_m), m = 1..N:
 *   q_i = sqrt(2/(N+1)) sum_m Q_m sin(i m pi/(N+1)),  p_i likewise from P_m,
 * then the whole state is scaled by s > 0 so that H(s x) = E_o.  With
 * alpha = 0, H(s x) = s^2 H2 + s^4 H4 and s^2 = 2E / (H2 + sqrt(H2^2 + 4 H4 E)).
 * Returns -1 when alpha != 0 (no closed form). */
int o_fput_mode_ics(const o_system* s, int64_t n, const double* Qm, const double* Pm,
                    const double* E, double* ics)
{
    int N = s->n_dof;
    if (s->alpha != 0.0) return -1;
    double pi = acos(-1.0);
    for (int64_t o = 0; o < n; ++o) {
        double x[512];
        for (int i = 1; i <= N; ++i) {
            double aq = 0.0, ap = 0.0;
            for (int m = 1; m <= N; ++m) {
                double sn = sin((double)i * (double)m * pi / (double)(N + 1));
                aq += Qm[(int64_t)(m - 1) * n + o] * sn;
                ap += Pm[(int64_t)(m - 1) * n + o] * sn;
            }
            x[i - 1] = sqrt(2.0 / (double)(N + 1)) * aq;
            x[N + i - 1] = sqrt(2.0 / (double)(N + 1)) * ap;
        }
        double H2 = 0.0, H4 = 0.0;
        for (int i = 0; i < N; ++i) H2 += x[N + i] * x[N + i] / 2.0;
        for (int i = 1; i <= N + 1; ++i) {
            double r = fput_bond(x, N, i);
            H2 += s->kk / 2.0 * r * r;
            H4 += s->beta / 4.0 * r * r * r * r;
        }
        double s2 = 2.0 * E[o] / (H2 + sqrt(H2 * H2 + 4.0 * H4 * E[o]));
        double sc = sqrt(s2);
        for (int c = 0; c < 2 * N; ++c) ics[(int64_t)c * n + o] = sc * x[c];
    }
    return 0;
}

/* Quartic-3 initial conditions on an energy shell: the direction u = dir/|dir|
 * of a 6-component draw is scaled by s > 0 with H(s u) = E_o.  H(s u) =
 * s^2 H2 + s^4 H4 with H2 = |u|^2 / 2 = 1/2 and H4 = eps (u1^2 u2^2 + u2^2 u3^2 +
 * u1^2 u3^2) over the coordinate part, so s^2 = 2E / (H2 + sqrt(H2^2 + 4 H4 E)). */
int o_shell_ics(const o_system* s, int64_t n, const double* dirs, const double* E, double* ics)
{
    if (s->model != O_QUARTIC3) return -1;
    for (int64_t o = 0; o < n; ++o) {
        double u[6], nr = 0.0;
        for (int c = 0; c < 6; ++c) {
            u[c] = dirs[(int64_t)c * n + o];
            nr += u[c] * u[c];
        }
        nr = sqrt(nr);
        for (int c = 0; c < 6; ++c) u[c] = u[c] / nr;
        double H2 = 0.0;
        for (int c = 0; c < 6; ++c) H2 += u[c] * u[c] / 2.0;
        double H4 = s->eps * (u[0] * u[0] * u[1] * u[1] + u[1] * u[1] * u[2] * u[2] + u[0] * u[0] * u[2] * u[2]);
        double s2 = 2.0 * E[o] / (H2 + sqrt(H2 * H2 + 4.0 * H4 * E[o]));
        double sc = sqrt(s2);
        for (int c = 0; c < 6; ++c) ics[(int64_t)c * n + o] = sc * u[c];
    }
    return 0;
}

/* Initial ensemble: x <- ics, w <- w_in (or seeded), normalised when renorm
 * is set, L <- 0, H0 <- H(x), dH_max <- 0, n_exec <- 0.  A cell whose
 * ic_status is not OK keeps that status; a non-finite state becomes NONFINITE. */
void o_ensemble_init(const o_system* s, const o_params* prm, int64_t n, const double* ics,
                     const int32_t* ic_status, const double* w_in, uint64_t seed, double* x,
                     double* w, double* ld, double* h0, double* dh_max, int64_t* n_exec,
                     int32_t* status)
{
    int d = 2 * s->n_dof, k = prm->n_dev;
    if (k > 0) {
        if (w_in)
            memcpy(w, w_in, sizeof(double) * (size_t)k * d * n);
        else
            o_seed_vectors(seed, n, k, d, w);
    }
    for (int64_t o = 0; o < n; ++o) {
        double xo[512];
        for (int c = 0; c < d; ++c) {
            x[c * n + o] = ics[c * n + o];
            xo[c] = ics[c * n + o];
        }
        if (k > 0 && prm->renorm) {
            for (int j = 0; j < k; ++j) {
                double v[512];
                for (int c = 0; c < d; ++c) v[c] = w[((int64_t)j * d + c) * n + o];
                double nr = o_norm(v, d);
                for (int c = 0; c < d; ++c) w[((int64_t)j * d + c) * n + o] = v[c] / nr;
            }
        }
        if (ld) ld[o] = 0.0;
        dh_max[o] = 0.0;
        n_exec[o] = 0;
        int32_t st = ic_status ? ic_status[o] : OS_OK;
        if (st == OS_OK && !o_all_finite(xo, d)) st = OS_NONFINITE;
        status[o] = st;
        h0[o] = (st == OS_OK) ? o_energy(s, xo) : NAN;
    }
}

/* ------------------------------------------------------------------------ */
/* Integration                                                               */
/* ------------------------------------------------------------------------ */

/* Advance every orbit by prm->n_steps steps, or fewer when its own end step
 * t_end[o] (total steps, when t_end is given) comes first.  After each step:
 * renormalise the vectors (if prm->renorm), then freeze the orbit as ESCAPED if
 * sum_i q_i^2 > escape_r2.  At absolute steps divisible by sample_every:
 * freeze as NONFINITE on any non-finite value, update dH_max = max |H - H0|,
 * freeze as ENERGY_DRIFT when it exceeds dh_limit, and (early_exit, k >= 2)
 * freeze as EARLY_CHAOTIC once SALI < sali_threshold.  A frozen orbit keeps the
 * state of the step at which it froze; n_exec counts executed steps. */
/* SALI of the first two vectors of the joint state z (each normalised first). */
static double o_sali_of(const double* a, const double* b, int d)
{
    double na = o_norm(a, d), nb = o_norm(b, d);
    double sp = 0.0, sm = 0.0;
    for (int c = 0; c < d; ++c) {
        double u = a[c] / na, v = b[c] / nb;
        sp += (u + v) * (u + v);
        sm += (u - v) * (u - v);
    }
    sp = sqrt(sp);
    sm = sqrt(sm);
    return sp < sm ? sp : sm;
}

/* What follows each completed step: renormalise the vectors (if prm->renorm),
 * freeze as ESCAPED if sum_i q_i^2 > escape_r2, and, when `check` is set (a
 * health-check step), freeze as NONFINITE on any non-finite value, update
 * dH_max, freeze as ENERGY_DRIFT beyond dh_limit and, with early_exit and
 * k >= 2, as EARLY_CHAOTIC once SALI < sali_threshold.  Returns the status. */
static int32_t o_post_step(const o_system* s, const o_params* prm, double* z, int D, int check,
                           double h0, double* dhm)
{
    int d = 2 * s->n_dof, k = prm->n_dev, N = s->n_dof;
    if (prm->renorm) {
        for (int j = 0; j < k; ++j) {
            double* v = z + d + j * d;
            double nr = o_norm(v, d);
            for (int c = 0; c < d; ++c) v[c] = v[c] / nr;
        }
    }
    if (prm->escape_r2 > 0.0) {
        double r2 = 0.0;
        for (int i = 0; i < N; ++i) r2 += z[i] * z[i];
        if (r2 > prm->escape_r2) return OS_ESCAPED;
    }
    if (check) {
        if (!o_all_finite(z, D)) return OS_NONFINITE;
        double dH = fabs(o_energy(s, z) - h0);
        if (dH > *dhm) *dhm = dH;
        if (prm->dh_limit > 0.0 && dH > prm->dh_limit) return OS_ENERGY_DRIFT;
        if (prm->early_exit && k >= 2 && o_sali_of(z + d, z + 2 * d, d) < prm->sali_threshold)
            return OS_EARLY_CHAOTIC;
    }
    return OS_OK;
}

/* Scratch of one orbit's integration: the joint state z, the RK4 stages or the
 * twelve DOP853 stages, a trial state and the error estimates. */
typedef struct {
    double *z, *zn, *zt, *K, *e5, *e3, *Hm;
} o_work;

static o_work o_work_alloc(int D, int N)
{
    o_work W;
    W.z = (double*)malloc(sizeof(double) * (size_t)D * 17);
    W.zn = W.z + D;
    W.zt = W.z + 2 * D;
    W.e5 = W.z + 3 * D;
    W.e3 = W.z + 4 * D;
    W.K = W.z + 5 * D;
    W.Hm = (double*)malloc(sizeof(double) * (size_t)N * N);
    return W;
}

static void o_work_free(o_work* W)
{
    free(W->Hm);
    free(W->z);
}

/* One fixed step of the selected integrator on the joint state W->z. */
static void o_fixed_step(const o_joint* J, const o_params* prm, o_work* W, int D)
{
    if (prm->integrator == OI_YOSHIDA4) {
        o_yoshida_step(J, W->z, prm->dt);
    } else if (prm->integrator == OI_DOP853) {
        o_dop853_step(J, W->z, W->zn, D, prm->dt, W->K, W->zt, NULL, NULL);
        memcpy(W->z, W->zn, sizeof(double) * (size_t)D);
    } else {
        o_rk4_step(J, W->z, D, prm->dt, W->K, W->K + D, W->K + 2 * D, W->K + 3 * D, W->zt);
    }
}

void o_integrate(const o_system* s, const o_params* prm, int64_t n, double* x, double* w,
                 double* ld, const double* h0, double* dh_max, int64_t* n_exec, int32_t* status,
                 const int64_t* t_end, int nthreads)
{
    int d = 2 * s->n_dof, k = prm->n_dev, N = s->n_dof;
    int use_ld = (prm->ld_p != 0.0) && ld != NULL;
    int D = d + k * d + (use_ld ? 1 : 0);
    int nt = o_threads(nthreads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int64_t o = 0; o < n; ++o) {
        if (status[o] != OS_OK) continue;
        o_work W = o_work_alloc(D, N);
        double* z = W.z;
        o_joint J = {s, d, k, use_ld, prm->ld_p, W.Hm, prm->dt < 0.0 ? -1.0 : 1.0};
        for (int c = 0; c < d; ++c) z[c] = x[c * n + o];
        for (int j = 0; j < k; ++j)
            for (int c = 0; c < d; ++c) z[d + j * d + c] = w[((int64_t)j * d + c) * n + o];
        if (use_ld) z[D - 1] = ld[o];
        double dhm = dh_max[o];
        int32_t st = OS_OK;
        int64_t done = 0;
        int64_t todo = prm->n_steps;
        if (t_end && t_end[o] - n_exec[o] < todo) todo = t_end[o] - n_exec[o] > 0 ? t_end[o] - n_exec[o] : 0;
        for (int64_t sidx = 1; sidx <= todo; ++sidx) {
            o_fixed_step(&J, prm, &W, D);
            done = sidx;
            int64_t abs_step = prm->step0 + sidx;
            int check = prm->sample_every > 0 && abs_step % prm->sample_every == 0;
            st = o_post_step(s, prm, z, D, check, h0[o], &dhm);
            if (st != OS_OK) break;
        }
        for (int c = 0; c < d; ++c) x[c * n + o] = z[c];
        for (int j = 0; j < k; ++j)
            for (int c = 0; c < d; ++c) w[((int64_t)j * d + c) * n + o] = z[d + j * d + c];
        if (use_ld) ld[o] = z[D - 1];
        dh_max[o] = dhm;
        n_exec[o] += done;
        status[o] = st;
        o_work_free(&W);
    }
}

/* DOP 8(5) with adaptive step size (Sec. Functionalities).  Orbit o carries
 * its time t[o] and its next step size hs[o]; a call advances it until
 * t[o] = ad->t_final, or until prm->n_steps steps have been accepted in this
 * call, or until it freezes.  Each step (Hairer et al., Sec. II.4, the
 * standard controller with safety factor 0.9, growth at most 10, shrink at
 * least 0.2):
 *   the step size is clamped to [10 ulp(t), h_max] (h_max <= 0: no upper bound);
 *   repeat: clip so that t + h <= t_final; take a DOP853 step; err = the
 *     combined error norm over the d orbit components;
 *     err < 1: accept, next h = h min(10, 0.9 err^(-1/8)) (10 when err = 0),
 *              at most h if this step had a rejected attempt;
 *     else   : reject (also when err is not finite), h = h max(0.2,
 *              0.9 err^(-1/8)), count the rejection, and freeze as STEP_FAIL
 *              (state kept) once h < 10 ulp(t).
 * After each accepted step the checks of o_post_step run, health checks at
 * accepted-step counts n_exec divisible by sample_every.  err_last[o] is the
 * error of the last accepted step, err_max[o] the largest so far (both
 * optional), n_rej[o] counts rejected attempts (optional). */
typedef struct {
    double t_final;
    double rtol, atol;
    double h_max;
} o_adaptive;

/* One accepted DOP 8(5) step of the joint state W->z (length D; the error norm
 * over its first d components), with the controller described above.  On
 * return *tt and *h are the new time and next step size, *err the accepted
 * step's error; rejections are counted in *rej.  Returns OS_OK, or
 * OS_STEP_FAIL with z and *tt unchanged. */
static int32_t o_adaptive_step(const o_joint* J, o_work* W, int D, int d, const o_adaptive* ad,
                               double* tt, double* h, double* err, int64_t* rej)
{
    double min_step = 10.0 * (nextafter(*tt, INFINITY) - *tt);
    if (ad->h_max > 0.0 && *h > ad->h_max) *h = ad->h_max;
    if (*h < min_step) *h = min_step;
    int rejected = 0;
    for (;;) {
        if (*h < min_step) return OS_STEP_FAIL;
        double tn = *tt + *h;
        if (tn > ad->t_final) tn = ad->t_final;
        double hh = tn - *tt;
        o_dop853_step(J, W->z, W->zn, D, hh, W->K, W->zt, W->e5, W->e3);
        double e = o_dop853_err(W->z, W->zn, W->e5, W->e3, d, hh, ad->atol, ad->rtol);
        if (e < 1.0) {
            double fac = (e == 0.0) ? 10.0 : 0.9 * pow(e, -1.0 / 8.0);
            if (fac > 10.0) fac = 10.0;
            if (rejected && fac > 1.0) fac = 1.0;
            *h = hh * fac;
            memcpy(W->z, W->zn, sizeof(double) * (size_t)D);
            *tt = tn;
            *err = e;
            return OS_OK;
        }
        double fac = 0.9 * pow(e, -1.0 / 8.0);
        if (!(fac >= 0.2)) fac = 0.2;   /* also for a non-finite err */
        *h = hh * fac;
        rejected = 1;
        ++*rej;
    }
}

void o_integrate_adaptive(const o_system* s, const o_params* prm, const o_adaptive* ad, int64_t n,
                          double* x, double* w, double* ld, const double* h0, double* dh_max,
                          int64_t* n_exec, int32_t* status, double* t, double* hs,
                          double* err_last, double* err_max, int64_t* n_rej, int nthreads)
{
    int d = 2 * s->n_dof, k = prm->n_dev, N = s->n_dof;
    int use_ld = (prm->ld_p != 0.0) && ld != NULL;
    int D = d + k * d + (use_ld ? 1 : 0);
    int nt = o_threads(nthreads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int64_t o = 0; o < n; ++o) {
        if (status[o] != OS_OK) continue;
        o_work W = o_work_alloc(D, N);
        double* z = W.z;
        o_joint J = {s, d, k, use_ld, prm->ld_p, W.Hm, 1.0};
        for (int c = 0; c < d; ++c) z[c] = x[c * n + o];
        for (int j = 0; j < k; ++j)
            for (int c = 0; c < d; ++c) z[d + j * d + c] = w[((int64_t)j * d + c) * n + o];
        if (use_ld) z[D - 1] = ld[o];
        double dhm = dh_max[o];
        double tt = t[o], h = hs[o];
        double el = err_last ? err_last[o] : 0.0, em = err_max ? err_max[o] : 0.0;
        int64_t rej = n_rej ? n_rej[o] : 0;
        int32_t st = OS_OK;
        int64_t done = 0;
        while (done < prm->n_steps && tt < ad->t_final) {
            double err = 0.0;
            st = o_adaptive_step(&J, &W, D, d, ad, &tt, &h, &err, &rej);
            if (st != OS_OK) break;
            el = err;
            if (err > em) em = err;
            ++done;
            int64_t cnt = n_exec[o] + done;
            int check = prm->sample_every > 0 && cnt % prm->sample_every == 0;
            st = o_post_step(s, prm, z, D, check, h0[o], &dhm);
            if (st != OS_OK) break;
        }
        for (int c = 0; c < d; ++c) x[c * n + o] = z[c];
        for (int j = 0; j < k; ++j)
            for (int c = 0; c < d; ++c) w[((int64_t)j * d + c) * n + o] = z[d + j * d + c];
        if (use_ld) ld[o] = z[D - 1];
        dh_max[o] = dhm;
        n_exec[o] += done;
        status[o] = st;
        t[o] = tt;
        hs[o] = h;
        if (err_last) err_last[o] = el;
        if (err_max) err_max[o] = em;
        if (n_rej) n_rej[o] = rej;
        o_work_free(&W);
    }
}

/* ------------------------------------------------------------------------ */
/* Indicators                                                                */
/* ------------------------------------------------------------------------ */

/* One-sided Jacobi SVD (Hestenes 1958) of the d x k matrix A (column-major,
 * A[c * d + i] = row i of column c): plane rotations of column pairs until
 * every pair is orthogonal to working precision; the singular values are the
 * final column norms (returned unsorted). */
void o_jacobi_sv(int d, int k, const double* A, double* sv)
{
    double* U = (double*)malloc(sizeof(double) * (size_t)d * k);
    memcpy(U, A, sizeof(double) * (size_t)d * k);
    for (int sweep = 0; sweep < 100; ++sweep) {
        int rotated = 0;
        for (int p = 0; p < k - 1; ++p) {
            for (int q = p + 1; q < k; ++q) {
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = 0; i < d; ++i) {
                    al += U[p * d + i] * U[p * d + i];
                    be += U[q * d + i] * U[q * d + i];
                    ga += U[p * d + i] * U[q * d + i];
                }
                if (fabs(ga) <= 1e-15 * sqrt(al * be) || ga == 0.0) continue;
                rotated = 1;
                double zeta = (be - al) / (2.0 * ga);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + hypot(1.0, zeta));
                double c = 1.0 / sqrt(1.0 + t * t);
                double sn = c * t;
                for (int i = 0; i < d; ++i) {
                    double up = U[p * d + i], uq = U[q * d + i];
                    U[p * d + i] = c * up - sn * uq;
                    U[q * d + i] = sn * up + c * uq;
                }
            }
        }
        if (!rotated) break;
    }
    for (int c = 0; c < k; ++c) {
        double acc = 0.0;
        for (int i = 0; i < d; ++i) acc += U[c * d + i] * U[c * d + i];
        sv[c] = sqrt(acc);
    }
    free(U);
}

/* Per orbit, from the k deviation vectors (each first normalised):
 *   SALI = min(|w1 + w2|, |w1 - w2|)                      (needs k >= 2)
 *   GALI_m = product of the singular values of [w1..wm]   for m = 2..k
 *   label: status OK -> 1 (chaotic) if SALI < sali_threshold else 0 (regular);
 *          EARLY_CHAOTIC -> 1; ESCAPED -> 2; any other status -> -1.
 * FORBIDDEN orbits get NaN indicators. */
void o_indicators(const o_system* s, int64_t n, int k, const double* w, const int32_t* status,
                  double sali_threshold, double* sali, double* gali, int8_t* label)
{
    int d = 2 * s->n_dof;
    double* A = (double*)malloc(sizeof(double) * (size_t)d * (k > 0 ? k : 1));
    double* svals = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    for (int64_t o = 0; o < n; ++o) {
        for (int j = 0; j < k; ++j) {
            for (int c = 0; c < d; ++c) A[j * d + c] = w[((int64_t)j * d + c) * n + o];
            double nr = o_norm(A + j * d, d);
            for (int c = 0; c < d; ++c) A[j * d + c] = A[j * d + c] / nr;
        }
        int forb = (status[o] == OS_FORBIDDEN);
        double sv = NAN;
        if (k >= 2 && !forb) {
            double sp[512], sm[512];
            for (int c = 0; c < d; ++c) {
                sp[c] = A[c] + A[d + c];
                sm[c] = A[c] - A[d + c];
            }
            double a = o_norm(sp, d), b = o_norm(sm, d);
            sv = a < b ? a : b;
        }
        if (sali) sali[o] = sv;
        if (gali) {
            for (int m = 2; m <= k; ++m) {
                double g = NAN;
                if (!forb) {
                    o_jacobi_sv(d, m, A, svals);
                    g = 1.0;
                    for (int c = 0; c < m; ++c) g *= svals[c];
                }
                gali[(int64_t)(m - 2) * n + o] = g;
            }
        }
        if (label) {
            int8_t lb;
            if (status[o] == OS_OK)
                lb = (sv < sali_threshold) ? 1 : 0;
            else if (status[o] == OS_EARLY_CHAOTIC)
                lb = 1;
            else if (status[o] == OS_ESCAPED)
                lb = 2;
            else
                lb = -1;
            label[o] = lb;
        }
    }
    free(svals);
    free(A);
}

/* LD-based indicators on the ny x npy section grid (o = iy * npy + ipy), with
 * n = 2 grid directions and a one-cell offset sigma:
 *   D_L = 1/(2n) sum_i |LD(x + s e_i) - LD(x - s e_i)| / LD(x)
 *   S_L = 1/n    sum_i |2 - (LD(x + s e_i) + LD(x - s e_i)) / LD(x)|
 * NaN on the grid border and wherever the cell or one of its four
 * neighbours does not have status OK. */
void o_ld_indicators(int ny, int npy, const double* ld, const int32_t* status, double* dl, double* sl)
{
    for (int iy = 0; iy < ny; ++iy) {
        for (int ip = 0; ip < npy; ++ip) {
            int64_t o = (int64_t)iy * npy + ip;
            dl[o] = NAN;
            sl[o] = NAN;
            if (iy == 0 || iy == ny - 1 || ip == 0 || ip == npy - 1) continue;
            int64_t nb[4] = {o - npy, o + npy, o - 1, o + 1};
            int ok = status[o] == OS_OK;
            for (int m = 0; m < 4; ++m) ok = ok && status[nb[m]] == OS_OK;
            if (!ok) continue;
            double c = ld[o];
            double Dsum = fabs(ld[o + npy] - ld[o - npy]) / c + fabs(ld[o + 1] - ld[o - 1]) / c;
            double Ssum = fabs(2.0 - (ld[o + npy] + ld[o - npy]) / c)
                        + fabs(2.0 - (ld[o + 1] + ld[o - 1]) / c);
            dl[o] = Dsum / 4.0;
            sl[o] = Ssum / 2.0;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Lyapunov spectrum by periodic QR                                          */
/* ------------------------------------------------------------------------ */

/* Modified Gram-Schmidt on the d columns w_j of W (column j at W + j*d):
 * W = QR with R_jj > 0, S_j += ln R_jj, W <- Q. */
static void o_qr_accumulate(double* W, int d, double* S)
{
    for (int j = 0; j < d; ++j) {
        double* wj = W + j * d;
        for (int i = 0; i < j; ++i) {
            double* qi = W + i * d;
            double r = 0.0;
            for (int c = 0; c < d; ++c) r += qi[c] * wj[c];
            for (int c = 0; c < d; ++c) wj[c] = wj[c] - r * qi[c];
        }
        double rjj = o_norm(wj, d);
        for (int c = 0; c < d; ++c) wj[c] = wj[c] / rjj;
        S[j] += log(rjj);
    }
}

/* d deviation vectors start as the identity basis and follow the variational
 * equations under RK4 together with the orbit.  At every step divisible by
 * qr_every, and at the last step, the matrix W of vectors (columns) is
 * factorised W = QR by modified Gram-Schmidt (so R_ii > 0); S_i += ln R_ii
 * and W <- Q.  Finally lambda_i = S_i / (n_steps * dt), in column order.
 * NONFINITE at a health check freezes the orbit and sets lambda to NaN. */
void o_lyapunov(const o_system* s, const o_params* prm, int64_t n, const double* ics,
                const int32_t* ic_status, double* lambda, int32_t* status, int nthreads)
{
    int d = 2 * s->n_dof, N = s->n_dof;
    int D = d + d * d;
    int nt = o_threads(nthreads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int64_t o = 0; o < n; ++o) {
        int32_t st = ic_status ? ic_status[o] : OS_OK;
        if (st != OS_OK) {
            status[o] = st;
            for (int i = 0; i < d; ++i) lambda[(int64_t)i * n + o] = NAN;
            continue;
        }
        o_work Wk = o_work_alloc(D, N);
        double* z = Wk.z;
        double* S = (double*)calloc((size_t)d, sizeof(double));
        o_joint J = {s, d, d, 0, 0.0, Wk.Hm, 1.0};
        for (int c = 0; c < d; ++c) z[c] = ics[(int64_t)c * n + o];
        for (int j = 0; j < d; ++j)
            for (int c = 0; c < d; ++c) z[d + j * d + c] = (c == j) ? 1.0 : 0.0;
        for (int64_t sidx = 1; sidx <= prm->n_steps; ++sidx) {
            o_fixed_step(&J, prm, &Wk, D);
            if ((prm->qr_every > 0 && sidx % prm->qr_every == 0) || sidx == prm->n_steps)
                o_qr_accumulate(z + d, d, S);
            if (prm->sample_every > 0 && sidx % prm->sample_every == 0 && !o_all_finite(z, D)) {
                st = OS_NONFINITE;
                break;
            }
        }
        double T = (double)prm->n_steps * prm->dt;
        for (int i = 0; i < d; ++i) lambda[(int64_t)i * n + o] = (st == OS_OK) ? S[i] / T : NAN;
        status[o] = st;
        free(S);
        o_work_free(&Wk);
    }
}

/* Lyapunov spectrum by periodic QR with adaptive DOP 8(5) (Sec. Functionalities,
 * the adaptive solver with vector normalisation and QR): as o_lyapunov, with
 * the orbit and its d vectors advanced by o_adaptive_step from t = 0 to
 * ad->t_final (error over the orbit components), the QR every qr_every
 * accepted steps and at t_final, and lambda_i = S_i / t_final.  The first
 * step guess is prm->dt.  An orbit still short of t_final after prm->n_steps
 * accepted steps, or whose step size fails (a trial whose orbit is not finite
 * is always rejected), freezes as STEP_FAIL; non-finite exponent sums at the
 * end give NONFINITE; both get NaN exponents.  n_acc (optional) receives the
 * accepted steps and n_rej (optional) the rejected trials. */
void o_lyapunov_adaptive(const o_system* s, const o_params* prm, const o_adaptive* ad, int64_t n,
                         const double* ics, const int32_t* ic_status, double* lambda,
                         int32_t* status, int64_t* n_acc, int64_t* n_rej, int nthreads)
{
    int d = 2 * s->n_dof, N = s->n_dof;
    int D = d + d * d;
    int nt = o_threads(nthreads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int64_t o = 0; o < n; ++o) {
        int32_t st = ic_status ? ic_status[o] : OS_OK;
        int64_t done = 0, rej = 0;
        if (st != OS_OK) {
            status[o] = st;
            for (int i = 0; i < d; ++i) lambda[(int64_t)i * n + o] = NAN;
            if (n_acc) n_acc[o] = 0;
            if (n_rej) n_rej[o] = 0;
            continue;
        }
        o_work Wk = o_work_alloc(D, N);
        double* z = Wk.z;
        double* S = (double*)calloc((size_t)d, sizeof(double));
        o_joint J = {s, d, d, 0, 0.0, Wk.Hm, 1.0};
        for (int c = 0; c < d; ++c) z[c] = ics[(int64_t)c * n + o];
        for (int j = 0; j < d; ++j)
            for (int c = 0; c < d; ++c) z[d + j * d + c] = (c == j) ? 1.0 : 0.0;
        double tt = 0.0, h = prm->dt, err = 0.0;
        while (tt < ad->t_final) {
            if (done >= prm->n_steps) {
                st = OS_STEP_FAIL;
                break;
            }
            st = o_adaptive_step(&J, &Wk, D, d, ad, &tt, &h, &err, &rej);
            if (st != OS_OK) break;
            ++done;
            if ((prm->qr_every > 0 && done % prm->qr_every == 0) || tt >= ad->t_final)
                o_qr_accumulate(z + d, d, S);
        }
        if (st == OS_OK && !o_all_finite(S, d)) st = OS_NONFINITE;
        for (int i = 0; i < d; ++i) lambda[(int64_t)i * n + o] = (st == OS_OK) ? S[i] / ad->t_final : NAN;
        status[o] = st;
        if (n_acc) n_acc[o] = done;
        if (n_rej) n_rej[o] = rej;
        free(S);
        o_work_free(&Wk);
    }
}

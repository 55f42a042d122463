/*
 * chs.h -- C ABI of the GB300 chaos-indicator library (libchs.so).
 *
 * The library integrates large ensembles of Hamiltonian orbits together with
 * their variational equations and accumulates the chaos indicators described
 * in "Chaoticus: a parallel approach to the computation of chaos indicators"
 * (arXiv 2507.00622): SALI, GALI_k, Lagrangian-descriptor (LD) based
 * indicators and the Lyapunov spectrum by periodic QR (Sec. Functionalities).
 *
 * Conventions shared by every entry point
 *   - Array arguments are DEVICE pointers allocated and owned by the caller.
 *     The library never frees them and never allocates device memory in a
 *     call; it keeps nothing beyond the opaque system handle.
 *   - Ensemble arrays are structure-of-arrays: element (c, o) of an array
 *     with C components over n orbits is at a[c * n + o].  Phase-space
 *     vectors are ordered (q_1..q_N, p_1..p_N), d = 2N.  Deviation vector j
 *     occupies components j*d .. j*d + d - 1 of the vector array.
 *   - Every call is asynchronous on `stream` (a cudaStream_t; NULL is the
 *     legacy default stream).  Argument errors are detected on the host
 *     before anything is launched and returned as a chs_status; launch
 *     failures return CHS_E_CUDA.  No exception crosses the ABI and no
 *     kernel traps.  chs_last_error() gives a message for the last non-OK
 *     status returned on the calling thread.
 *   - Per-orbit failures are written to the orbit's status word
 *     (CHS_ORBIT_*), never to the return value.
 *   - All state is FP64 unless chs_params.vec_precision selects FP32
 *     deviation vectors.
 */
#ifndef CHS_H
#define CHS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CHS_OK = 0,
    CHS_E_INVALID = 1,     /* bad pointer, size, or parameter */
    CHS_E_UNSUPPORTED = 2, /* valid request this build does not implement */
    CHS_E_CUDA = 3,        /* a CUDA launch or runtime call failed */
    CHS_E_NOMEM = 4,       /* host allocation failed */
    CHS_E_SIZE = 5         /* a size exceeds a documented maximum */
} chs_status;

/* Hamiltonian systems.
 *   CHS_HENON_HEILES  H = (px^2 + py^2)/2 + (x^2 + y^2)/2 + x^2 y - y^3/3
 *                     (Eq. Ham_HH; equations of motion Eq. ham_eqs_HH).  n_dof = 2.
 *   CHS_FPUT          FPU(T) chain with fixed ends q_0 = q_{N+1} = 0 (Eqs.
 *                     ham_FPU, ham_eqs_FPU), params = {k, alpha, beta}; the
 *                     energy sums the N+1 bonds D_i = q_i - q_{i-1}.
 *   CHS_QUARTIC3      H = sum (p_i^2 + q_i^2)/2 + eps (q1^2 q2^2 + q2^2 q3^2 +
 *                     q1^2 q3^2), params = {eps}.  n_dof = 3.
 *   CHS_HARMONIC      H = sum (p_i^2 + q_i^2)/2 (test system).  n_dof = 2.
 *   CHS_INVERTED      H = (p1^2 - q1^2)/2 + (p2^2 + q2^2)/2 (test system).  n_dof = 2. */
typedef enum {
    CHS_HENON_HEILES = 1,
    CHS_FPUT = 2,
    CHS_QUARTIC3 = 3,
    CHS_HARMONIC = 100,
    CHS_INVERTED = 101
} chs_model;

/* Orbit status words. */
enum {
    CHS_ORBIT_OK = 0,
    CHS_ORBIT_FORBIDDEN = 1,    /* no initial condition exists in this cell */
    CHS_ORBIT_ESCAPED = 2,      /* sum_i q_i^2 exceeded escape_r2; frozen */
    CHS_ORBIT_NONFINITE = 3,    /* a non-finite value at a health check; frozen */
    CHS_ORBIT_ENERGY_DRIFT = 4, /* |H - H0| exceeded dh_limit at a health check; frozen */
    CHS_ORBIT_EARLY_CHAOTIC = 5, /* SALI fell below sali_threshold at a health check with
                                    early_exit set, or the surrogate predicted "chaotic" with
                                    confidence; frozen, labelled chaotic */
    CHS_ORBIT_PREDICTED_REGULAR = 6, /* the surrogate predicted "regular" with confidence;
                                        frozen, labelled regular */
    CHS_ORBIT_STEP_FAIL = 7,    /* adaptive DOP 8(5): the step size fell below 10 ulp(t)
                                   after a rejection; frozen at the last accepted step */
    CHS_ORBIT_STEP_BUDGET = 8   /* the call's clock budget (chs_params.clock_budget) ran
                                   out at a health check; frozen there */
};

/* Integrators (chs_params.integrator).
 *   CHS_RK4     classic 4th-order Runge-Kutta, fixed step.
 *   CHS_DOP853  the paper's 8th-order solver (DOP 8, Sec. Functionalities,
 *               ref prince1981): the 12-stage DOP853 pair of Dormand and
 *               Prince (Hairer, Norsett and Wanner, Solving ODEs I, 2nd ed.,
 *               Sec. II.10); fixed step in chs_integrate_batch /
 *               chs_integrate_compacted / chs_lyapunov_spectrum, adaptive with
 *               its 5th/3rd-order error estimate in chs_integrate_adaptive.
 *               FP64 deviation vectors only.
 * The value 1 is not used by the library. */
enum { CHS_RK4 = 0, CHS_DOP853 = 2 };

/* Deviation-vector storage precision. */
enum { CHS_VEC_FP64 = 0, CHS_VEC_FP32 = 1 };

/* Integration and indicator parameters (plain old data). */
typedef struct {
    double dt;               /* fixed step h (adaptive runs: see chs_integrate_adaptive) */
    int64_t n_steps;         /* steps to take in this call */
    int64_t step0;           /* absolute index of the last step already taken */
    int32_t n_dev;           /* number k of deviation vectors (0..6; must match the ensemble) */
    int32_t renorm;          /* 1: normalise each deviation vector after every step */
    int32_t sample_every;    /* health checks at absolute steps divisible by this (0 = never) */
    int32_t qr_every;        /* Lyapunov: QR of the vectors every qr_every steps and at the end */
    int32_t vec_precision;   /* CHS_VEC_FP64 or CHS_VEC_FP32 (FP32 requires renorm = 1) */
    int32_t early_exit;      /* 1: freeze as EARLY_CHAOTIC once SALI < sali_threshold at a
                                health check (needs n_dev >= 2); 0: integrate to the end */
    double ld_p;             /* LD exponent p (LD integrand sum_i |dx_i/dt|^p); 0 = no LD */
    double escape_r2;        /* ESCAPED when sum_i q_i^2 > escape_r2; 0 = off */
    double dh_limit;         /* ENERGY_DRIFT when |H - H0| > dh_limit; 0 = off */
    double sali_threshold;   /* label: chaotic when SALI < sali_threshold */
    uint64_t seed;           /* SplitMix64 seed for device-seeded deviation vectors */
    int32_t integrator;      /* CHS_RK4 or CHS_DOP853 */
    int32_t block_threads;   /* threads per block where a kernel offers the choice: 0 (the
                                library's default), 32, 64 or 128; results never depend on
                                it (see chs_integrate_batch, chs_lyapunov_spectrum) */
    int64_t clock_budget;    /* 0: none.  Otherwise the SM clock cycles (the device's clock64
                                counter) an orbit may run within one kernel launch, counted
                                from when its thread takes it up (chs_integrate_compacted
                                launches once per chunk: there the budget applies to each
                                chunk): at the first health check past the budget the orbit
                                freezes as CHS_ORBIT_STEP_BUDGET with the state, n_exec and
                                dh_max of that step (Lyapunov runs: NaN exponents).  Orbits
                                integrated by the same warp or block (FPUT chains) stop
                                together.  Needs sample_every > 0 to take effect; the
                                kernels never wait or trap on it.  Not a method step: a
                                bound on the time one call can take. */
    int32_t threads_per_orbit; /* threads that integrate one orbit, where a kernel offers the
                                choice: 0 (the library's default) or, for the RK4 FPUT
                                Lyapunov spectrum, 1, 2 or 4 at N = 4 (default 4) and 2, 4
                                or 8 at N = 8 (default 8); other calls take 0 only.  Results never depend
                                on it (see chs_lyapunov_spectrum). */
} chs_params;

/* Checks a parameter block for a system of the given model and n_dof the way
 * every entry point does before it launches anything (the ensemble entry points
 * add their own checks of the ensemble and of the kernels they support):
 * CHS_OK, or CHS_E_INVALID with chs_last_error() naming the field.  Needs no
 * device and no handle, so a configuration can be validated up front.
 * Interface helper; no paper counterpart. */
chs_status chs_check_params(const chs_params* p, chs_model model, int32_t n_dof);

/* Resumable ensemble state: caller-owned device arrays over n_orbits orbits.
 *   x       [d][n]    phase-space state (FP64)
 *   w       deviation vectors (NULL when k = 0):
 *           CHS_VEC_FP64: [k*d][n] FP64, row j*d + c = component c of vector j;
 *           CHS_VEC_FP32: [k*d + k(k+1)/2][n] FP32, the vectors as W = Q R D:
 *             rows j*d + c hold the orthonormal frame Q (column j, component c),
 *             rows k*d + j(j+1)/2 + i hold the upper-triangular R (i <= j) with
 *             unit columns; D is a positive diagonal that is not stored.  The
 *             unit vectors are w_j / |w_j| = sum_i R_ij q_i.  Each diagonal entry
 *             of R keeps its relative precision however small it gets, so SALI
 *             and GALI do not stall at the FP32 rounding level.
 *   ld      [n]       forward LD accumulator M_p (NULL when ld_p = 0)
 *   h0      [n]       energy at t = 0
 *   dh_max  [n]       largest |H - H0| seen at health checks
 *   n_exec  [n]       integration steps executed so far (frozen orbits stop counting)
 *   status  [n]       CHS_ORBIT_*
 *   t_end   [n]       optional (NULL = none): orbit o stops once n_exec reaches
 *                     t_end[o] steps (uneven integration lengths); read only */
typedef struct {
    int64_t n_orbits;
    double* x;
    void* w;
    double* ld;
    double* h0;
    double* dh_max;
    int64_t* n_exec;
    int32_t* status;
    const int64_t* t_end;
} chs_ensemble;

typedef struct chs_system_s* chs_system;

/* Creates a system handle on the current CUDA device for one of the
 * Hamiltonians of Sec. Examples (Eq. Ham_HH; Eq. ham_FPU with fixed ends) or
 * the quartic and test oscillators.  `params` (host) holds n_params model
 * constants: FPUT {k, alpha, beta}; QUARTIC3 {eps}; none for the others.
 * CHS_E_INVALID for an unknown model or a bad n_dof. */
chs_status chs_create_system(chs_system* out, chs_model model, int32_t n_dof,
                             const double* params, int32_t n_params);

/* Destroys a handle created by chs_create_system (NULL is accepted); frees
 * the handle's cached graph and private stream.  No paper counterpart. */
chs_status chs_destroy_system(chs_system s);

/* Phase-space dimension d = 2N of the system, or -1 for a NULL handle. */
int32_t chs_system_dim(chs_system s);

/* Henon-Heiles initial conditions on the x = 0 surface of section (Eq. Ham_HH,
 * Examples of Sec. Examples): a cell-centred ny x npy grid over [y0, y1] x
 * [py0, py1], orbit o = iy * npy + ipy at y = y0 + (iy + 1/2)(y1 - y0)/ny,
 * p_y = py0 + (ipy + 1/2)(py1 - py0)/npy, x = 0 and
 *   p_x = +sqrt(2E - p_y^2 - y^2 + 2y^3/3).
 * A negative radicand sets status FORBIDDEN and the state to NaN; the
 * FORBIDDEN decision is made in IEEE double without contraction, in the
 * order written above.  ics_out [4][ny*npy], status_out [ny*npy]. */
chs_status chs_section_grid_ics(chs_system s, double E, double y0, double y1, int32_t ny,
                                double py0, double py1, int32_t npy, double* ics_out,
                                int32_t* status_out, void* stream);

/* FPUT initial conditions from normal-mode amplitudes (Q_m, P_m), m = 1..N
 * (Sec. Examples, FPU system): q_i = sqrt(2/(N+1)) sum_m Q_m sin(i m pi/(N+1)),
 * p_i likewise from P_m; the state is then scaled by s > 0 with H(s x) = E_o,
 * s^2 = 2E / (H2 + sqrt(H2^2 + 4 H4 E)) where H2, H4 are the quadratic and
 * quartic parts at s = 1.  Qm, Pm [N][n], E [n], ics_out [2N][n].
 * CHS_E_UNSUPPORTED unless alpha = 0. */
chs_status chs_fput_mode_ics(chs_system s, int64_t n, const double* Qm, const double* Pm,
                             const double* E, double* ics_out, void* stream);

/* Quartic-3 initial conditions on energy shells (a0 for the coupled quartic
 * oscillator, a test system outside the paper; the same radial scaling as
 * the FPU normal modes of Sec. Examples): the direction u = dir / |dir| of each 6-component draw is scaled
 * by s > 0 so that H(s u) = E_o; with H2 = |u|^2/2 and H4 = eps (u1^2 u2^2 +
 * u2^2 u3^2 + u1^2 u3^2), s^2 = 2E / (H2 + sqrt(H2^2 + 4 H4 E)).
 * dirs [6][n], E [n], ics_out [6][n].  CHS_E_UNSUPPORTED for other models. */
chs_status chs_shell_ics(chs_system s, int64_t n, const double* dirs, const double* E,
                         double* ics_out, void* stream);

/* Initialises an ensemble from initial conditions `ics` [d][n]:
 * x <- ics; status <- ic_status (or OK when NULL), NONFINITE for a non-finite
 * OK state; h0 <- H(x); dh_max, n_exec, ld <- 0; the k = p->n_dev deviation
 * vectors are copied from w_in ([k*d][n] plain vectors, FP64 or FP32 per
 * vec_precision) or,
 * when w_in is NULL, seeded on the device: component c of vector j of orbit o
 * is the m-th SplitMix64 output (m = (o*k + j)*d + c + 1) of the stream seeded
 * with p->seed, mapped to [-1, 1) by its top 53 bits, and normalised.  Every
 * vector is normalised (once more, for seeded ones) when p->renorm is set.  In
 * FP32 mode the normalised vectors are factorised in FP64 into the frame Q and
 * triangle R described at chs_ensemble.
 * FPUT chains (Eq. ham_FPU, N in {4, 8, 16, 32, 64}) take FP64 vectors
 * (k <= 6) and no LD (ld_p = 0); other N return CHS_E_UNSUPPORTED. */
chs_status chs_ensemble_init(chs_system s, const chs_params* p, const chs_ensemble* e,
                             const double* ics, const int32_t* ic_status, const void* w_in,
                             void* stream);

/* Advances every OK orbit of the ensemble by p->n_steps steps of size p->dt
 * of the integrator p->integrator (classic RK4, or DOP853, the paper's DOP 8)
 * on the joint system (x, w_1..w_k, M_p):
 *   x' = f(x) (Hamilton's equations), w_j' = J(x) w_j (variational equations,
 *   Sec. Statement of need), dM_p/d|t| = sum_i |f_i(x)|^p (the LD, Sec.
 *   Statement of need; it grows with |t|, so a run with dt < 0 accumulates the
 *   backward LD as a positive number),
 * the fixed-step integrators of Sec. Functionalities.
 * After each step: vectors are renormalised when p->renorm is set (the
 * fixed-step solver variant with vector normalisation, Sec. Functionalities);
 * in FP32 mode the frame Q is advanced by the exact
 * one-step RK4 propagator of the variational equations and re-orthonormalised
 * (Phi Q = Q' S, R <- S R with unit columns), the orbit staying FP64 and the
 * LD accumulated in FP64 from an integrand summed in FP32 (correctly rounded
 * FP32 square roots; about 1e-7 per term, averaging out along the orbit);
 * an orbit with sum_i q_i^2 > escape_r2 freezes as ESCAPED.  At absolute steps divisible by sample_every: non-finite -> frozen
 * NONFINITE; dh_max <- max(dh_max, |H - h0|); |H - h0| > dh_limit -> frozen
 * ENERGY_DRIFT; with early_exit, SALI < sali_threshold -> frozen EARLY_CHAOTIC.
 * An orbit with t_end stops after t_end[o] total steps.  Splitting a run into
 * calls with consecutive step0 gives bit-identical results.  p->block_threads sets the
 * block size of the RK4 one-orbit-per-thread kernels (both vector precisions;
 * default 128); the DOP853 and FPUT kernels keep their own.  Supported: HENON_HEILES, HARMONIC, INVERTED
 * (k <= 4), QUARTIC3 (k <= 6) and FPUT (N in {4, 8, 16, 32, 64}, k <= 6, FP64
 * vectors, no LD; the vectors advance through the same Runge-Kutta stages as
 * the chain, with the tridiagonal Hessian of Eq. ham_eqs_FPU). */
chs_status chs_integrate_batch(chs_system s, const chs_params* p, const chs_ensemble* e,
                               void* stream);

/* Adaptive-step controls of chs_integrate_adaptive. */
typedef struct {
    double t_final;  /* every orbit is integrated from its time t[o] up to t_final */
    double rtol;     /* error tolerances: scale_i = atol + rtol * max(|x_i|, |x_new_i|) */
    double atol;
    double h_max;    /* largest step size; <= 0: no limit */
} chs_adaptive;

/* DOP 8(5) with adaptive step size and the error of each step (Sec.
 * Functionalities): the DOP853 pair (p->integrator must be CHS_DOP853) on the
 * same joint system and with the same per-step checks as chs_integrate_batch.
 * Orbit o carries its time t[o] and its next step size h[o] (caller-owned
 * device arrays [n]; start with t = 0 and h = a first guess).  A call advances
 * every OK orbit until t[o] reaches a->t_final or p->n_steps steps have been
 * accepted in this call.  Each step:
 *   h is clamped to [10 ulp(t), h_max]; then, until a trial is accepted:
 *   the trial step is clipped so that t + h <= t_final; the error of the trial
 *   over the d orbit components is the combined 5th/3rd-order estimate of the
 *   DOP853 pair,
 *     err = |h| E5 / sqrt(d (E5 + 0.01 E3)),  E5 = sum_i (err5_i / scale_i)^2,
 *   E3 likewise; err < 1 accepts the trial and sets the next
 *   h = h min(10, 0.9 err^(-1/8)) (10 when err = 0; at most h after a rejected
 *   trial in the same step); otherwise (also when err is not finite) the trial is
 *   rejected, h = h max(0.2, 0.9 err^(-1/8)), and the orbit freezes as
 *   STEP_FAIL once h < 10 ulp(t).
 * Accepted steps count in n_exec; health checks run at accepted-step counts
 * divisible by p->sample_every.  Optional outputs (NULL to skip), all [n]:
 * err_last (the error of the last accepted step), err_max (running maximum,
 * read and updated), n_rejected (running count of rejected trials, read and
 * updated).  The deviation vectors and the LD do not enter the error (their
 * stages are computed only for accepted trials).  p->dt, p->step0 and e->t_end
 * are not used (t_end must be NULL).  Forward in time only (t_final > t).
 * Supported: HENON_HEILES, HARMONIC,
 * INVERTED (k <= 4), QUARTIC3 (k <= 6), FPUT (N in {4, 8, 16, 32, 64},
 * k <= 6, no LD); FP64 vectors. */
chs_status chs_integrate_adaptive(chs_system s, const chs_params* p, const chs_adaptive* a,
                                  const chs_ensemble* e, double* t, double* h, double* err_last,
                                  double* err_max, int64_t* n_rejected, void* stream);

/* The same integration as chs_integrate_batch (the fixed-step solvers of Sec.
 * Functionalities; identical results, bit for bit), run by a persistent grid (every SM filled to the kernel's occupancy) whose
 * threads take orbit indices from a work queue, one orbit after another: a
 * thread whose orbit stops early -- its t_end, early exit, escape or any other
 * freeze -- takes the next orbit at once, so orbits of uneven length leave no
 * lane idle until the queue runs dry, in one launch.  `work` is caller-owned
 * device scratch of at least 8 bytes, 8-byte aligned (the queue counter; reset
 * by the call).  Calls that share a work buffer and overlap on the GPU race.
 * Supported: the systems of chs_integrate_batch except FPUT, both vector
 * precisions and integrators. */
chs_status chs_integrate_persistent(chs_system s, const chs_params* p, const chs_ensemble* e,
                                    void* work, size_t work_bytes, void* stream);

/* Bytes of device scratch that chs_integrate_compacted needs for n orbits
 * (two orbit lists and their counters).  No paper counterpart. */
size_t chs_compact_work_size(int64_t n_orbits);

/* The same integration as chs_integrate_batch (the fixed-step solvers of Sec.
 * Functionalities; p->n_steps steps from step p->step0, identical results bit
 * for bit), run in chunks of chunk_steps steps
 * over a list of the orbits still running: after every chunk the orbits that
 * froze (early exit, escape, ...) or reached their t_end are dropped from the
 * list, so later chunks launch only over live orbits.  The chunk sequence is
 * recorded once as a CUDA graph and replayed; the recorded graph is cached in
 * the handle and reused while the ensemble pointers, sizes and parameters are
 * unchanged.  `work` is caller-owned device scratch of at least
 * chs_compact_work_size(n) bytes, 256-byte aligned; its contents are
 * overwritten.  Calls that share a work buffer and overlap on the GPU race.
 * Supported: the systems of chs_integrate_batch except FPUT. */
chs_status chs_integrate_compacted(chs_system s, const chs_params* p, const chs_ensemble* e,
                                   int32_t chunk_steps, void* work, size_t work_bytes,
                                   void* stream);

/* The run of chs_integrate_compacted, with the same results and the same
 * argument checks (at most 100000 chunks), for callers that cannot
 * provide a scratch buffer: callers whose device memory belongs to another
 * allocator (a framework's caching allocator, a fixed arena sized at start-up)
 * that does not hand out extra buffers, or whose rules forbid device
 * allocation while the application runs.  The paper has no counterpart; this
 * is an interface convenience.  The orbit lists live in a fixed device array
 * inside the library (8 MiB + 256 B, held by every GPU that loads the library
 * until the process exits), so the call allocates nothing: no cudaMalloc, no
 * cudaFree, no allocating library routine, and no graph.  At most 1,048,576
 * orbits (the 1024 x 1024 grid); larger ensembles return CHS_E_SIZE.  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * The address is cached per device and looked up again when the calling
 * thread's current context differs from the one it was taken in (after a
 * cudaDeviceReset, or from another context on the device).
 * Every call shares the one array per device: calls that overlap on the GPU
 * (different streams, or different handles on the same device) race; the
 * counters are cleared by each call, the lists are overwritten. */
chs_status chs_integrate_compacted_static(chs_system s, const chs_params* p, const chs_ensemble* e,
                                          int32_t chunk_steps, void* stream);

/* Indicators of the current ensemble state (Sec. Functionalities):
 *   sali_out [n]        SALI = min(|w1 + w2|, |w1 - w2|) of the first two unit
 *                       vectors (refs Skokos2001/03/04); needs k >= 2.
 *   gali_out [k-1][n]   GALI_m, m = 2..k: the product of the singular values
 *                       of the d x m matrix of the first m unit vectors (ref
 *                       Skokos2008), computed as prod |R_ii| of its QR (FP32
 *                       mode: of the stored triangle R, and SALI as
 *                       R_11 sqrt(2 / (1 + |R_01|))).
 *   label_out [n]       1 chaotic (SALI < sali_threshold, or EARLY_CHAOTIC),
 *                       0 regular (or PREDICTED_REGULAR), 2 ESCAPED, -1 any
 *                       other non-OK status.
 *   ld_ind_out [2][n]   when grid_ny * grid_npy == n and the ensemble has an
 *                       LD: D_L and S_L from the four grid neighbours (LD-based
 *                       indicators and neighbouring trajectories):
 *                         D_L = 1/4 sum_dir |LD(+) - LD(-)| / LD,
 *                         S_L = 1/2 sum_dir |2 - (LD(+) + LD(-)) / LD|;
 *                       NaN on the border and next to any non-OK cell
 *                       (Henon-Heiles grids; FPUT returns CHS_E_UNSUPPORTED).
 * Any output may be NULL.  FORBIDDEN orbits get NaN indicators. */
chs_status chs_indicators(chs_system s, const chs_params* p, const chs_ensemble* e,
                          int32_t grid_ny, int32_t grid_npy, double* sali_out,
                          double* gali_out, double* ld_ind_out, int8_t* label_out,
                          void* stream);

/* Lyapunov spectrum by periodic QR (Sec. Functionalities, Lyapunov item;
 * FPU example of Sec. Examples).  d deviation vectors start as the identity
 * and follow the variational equations with the orbit under p->integrator
 * (RK4 or DOP853, fixed step); every
 * p->qr_every steps and at the last step the vector matrix W is factorised
 * W = QR with R_ii > 0, S_i += ln R_ii and W <- Q.  lambda_out [d][n] gets
 * S_i / (n_steps * dt) in column order; status_out [n] gets the orbit status
 * (a non-finite state at a health check gives NONFINITE and NaN exponents).
 * ic_status may be NULL.  Supported: FPUT with N in {4, 8, 16, 32, 64} (the
 * vectors live in shared memory; RK4 propagates them by its exact one-step
 * propagator, DOP853 column by column with the stages in registers), and
 * HENON_HEILES, HARMONIC, INVERTED.  FP64 throughout.  For FPUT under DOP853
 * the blocks are fixed (one warp of orbits for N <= 16, one orbit above) except
 * at N = 64: 256 threads per orbit by default (0 or 256), the 128-thread form
 * with 128, the same results.  For FPUT under RK4,
 * p->block_threads (0, or 32, 64, 128 and at least 2N; at N = 64 also 256)
 * sets the block size (block_threads / 2N orbits per block for N = 16, 32,
 * block_threads / threads_per_orbit at N = 4, 8; one orbit at N = 64, with two
 * threads per vector at 256; default: 64 at N = 4, 256 at N = 64, else the
 * smallest allowed), and at N = 4, 8
 * p->threads_per_orbit the lanes that share one orbit; the results depend on
 * neither. */
chs_status chs_lyapunov_spectrum(chs_system s, const chs_params* p, int64_t n,
                                 const double* ics, const int32_t* ic_status,
                                 double* lambda_out, int32_t* status_out, void* stream);

/* Lyapunov spectrum by periodic QR with adaptive DOP 8(5) (Sec. Functionalities:
 * the adaptive solver with vector normalisation and the Lyapunov spectrum by
 * QR).  As chs_lyapunov_spectrum, with every orbit and its d vectors advanced
 * from t = 0 to a->t_final by the DOP853 pair under the step-size control of
 * chs_integrate_adaptive (error over the d orbit components; p->dt is the first
 * step size; p->integrator must be CHS_DOP853), the QR every p->qr_every
 * accepted steps and at t_final, and lambda_out [d][n] = S_i / t_final.  An
 * orbit still short of t_final after p->n_steps accepted steps, or whose step
 * size fails (a trial whose orbit is not finite is always rejected), freezes as
 * STEP_FAIL; non-finite exponent sums at the end give NONFINITE; both get NaN
 * exponents.  n_steps_out and n_rejected_out [n] (nullable) receive each
 * orbit's accepted steps and rejected trials.  Supported: FPUT (N in
 * {4, 8, 16, 32, 64}), HENON_HEILES, HARMONIC, INVERTED. */
chs_status chs_lyapunov_adaptive(chs_system s, const chs_params* p, const chs_adaptive* a, int64_t n,
                                 const double* ics, const int32_t* ic_status, double* lambda_out,
                                 int32_t* status_out, int64_t* n_steps_out, int64_t* n_rejected_out,
                                 void* stream);

/* ------------------------------------------------------------------------
 * Early-stop surrogate (a learned classifier of the final label; the method's
 * indicators stay the judge).  Not in the paper: it learns the labels the
 * indicators of Sec. Functionalities (SALI, LD) give, from their early values,
 * and every entry point of this block serves it.  A 12 -> 128 -> 128 -> 128 -> 2 ReLU perceptron
 * with BF16 weights and activations and FP32 accumulation.  Features of an
 * orbit at the decision time t, from S <= 10 SALI samples taken at
 * t_i = (i + 1) t / S and the LD M_p(t):
 *   f_i = log10(max(SALI(t_i), 1e-20)) / 8 (i < 10; missing samples count as
 *   1e-20), f_10 = M_p(t) / t - 1, f_11 = (E_o - 0.133) / 0.033 (E_o the
 *   orbit's energy).
 * Outputs: y_0 = logit of "chaotic at the final time", y_1 = final
 * log10(SALI) / 8.  Parameters: one flat BF16 array (row-major out x in)
 * W1[128][12] b1[128] W2[128][128] b2[128] W3[128][128] b3[128] W4[2][128]
 * b4[2], chs_mlp_param_count() values.  Training keeps an FP32 master copy.
 * ------------------------------------------------------------------------ */

/* Number of parameters (34,946). */
size_t chs_mlp_param_count(void);

/* Features X [12][n] (FP32) from sali_series [S][n], ld [n], t and the
 * orbits' energies E [n]. */
chs_status chs_mlp_features(const double* sali_series, int32_t n_samples, const double* ld,
                            double t_decide, const double* E, int64_t n, float* X, void* stream);

/* Forward pass: Y [2][n] (FP32); act [3][128][n] (BF16, nullable) keeps the
 * hidden activations for chs_mlp_backward. */
chs_status chs_mlp_forward(const void* params_bf16, const float* X, int64_t n, float* Y, void* act,
                           void* stream);

/* Loss L = mean over n of BCE(sigmoid(y0), label) + w_reg (y1 - target)^2, and
 * dY [2][n] = dL/dY; loss_out (one float) receives L. */
chs_status chs_mlp_loss_grad(const float* Y, const float* label, const float* target, int64_t n,
                             float w_reg, float* dY, float* loss_out, void* stream);

/* Backward pass: parameter gradients grad_out [P] (FP32, overwritten) of the
 * loss whose output gradient is dY, from X and the activations of the forward
 * pass; delta_work is caller scratch of 3*128*n floats. */
chs_status chs_mlp_backward(const void* params_bf16, const float* X, const void* act, const float* dY,
                            int64_t n, float* delta_work, float* grad_out, void* stream);

/* One Adam step (bias-corrected, step >= 1) on the FP32 master weights with
 * moments m, v (all [P]); writes the BF16 copy params_bf16_out. */
chs_status chs_mlp_adam(float* master, float* m, float* v, const float* grad, float lr, float beta1,
                        float beta2, float eps, int32_t step, void* params_bf16_out, void* stream);

/* Decision at time t for every orbit whose status is OK: features from
 * sali_series [S][n], ld [n] and E [n], forward pass, then status <-
 * EARLY_CHAOTIC when sigmoid(y0) >= confidence, PREDICTED_REGULAR when
 * sigmoid(y0) <= 1 - confidence; other orbits are untouched.  prob_out [n]
 * (nullable) receives sigmoid(y0). */
chs_status chs_surrogate_decide(const void* params_bf16, const double* sali_series, int32_t n_samples,
                                const double* ld, double t_decide, const double* E, double confidence,
                                int64_t n, int32_t* status_inout, float* prob_out, void* stream);

/* One Lyapunov-spectrum job of a batch (see chs_lyapunov_spectrum). */
typedef struct {
    chs_system sys;
    chs_params params;
    int64_t n_orbits;
    const double* ics;
    const int32_t* ic_status;  /* nullable */
    double* lambda_out;
    int32_t* status_out;
} chs_lyap_job;

/* Runs several Lyapunov jobs (Sec. Functionalities, Lyapunov item; the FPU
 * example of Sec. Examples) -- typically FPUT chains of different N, each a
 * differently shaped kernel -- as one CUDA graph whose branches run
 * concurrently, so that blocks of different chain lengths share the SMs (an
 * N = 64 block holds 154 KB of shared memory and leaves room for smaller
 * ones).  Results are identical to separate chs_lyapunov_spectrum calls.  All
 * jobs must be on the current device; at most 16 jobs. */
chs_status chs_lyapunov_batch(const chs_lyap_job* jobs, int32_t n_jobs, void* stream);

/* ------------------------------------------------------------------------
 * Throughput probes of the arithmetic pipes (a measurement aid for the
 * roofline of the integrators, which are bound by the FP64 pipe, or by FP32 for
 * the FP32 deviation-vector frame).  The paper has no counterpart.
 * ------------------------------------------------------------------------ */
typedef enum {
    CHS_PROBE_DFMA = 1,     /* FP64 fma, 8 independent chains per thread */
    CHS_PROBE_DFMA_DEP = 2, /* FP64 fma, one dependent chain per thread */
    CHS_PROBE_FFMA = 3,     /* FP32 fma, 8 independent chains per thread */
    CHS_PROBE_DSQRT = 4,    /* FP64 sqrt (with one fma), 8 chains per thread */
    CHS_PROBE_DMMA = 5,     /* FP64 mma.sync m8n8k4, 8 accumulators per warp */
    CHS_PROBE_DFMA_DMMA = 6 /* both at once: 4 fma chains per thread and 4 mma.sync
                               accumulators per warp, interleaved (shows whether
                               the two share a pipe) */
} chs_probe_kind;

/* Launches one probe kernel of n_blocks x n_threads threads (n_threads a
 * multiple of 32 in 32..1024, n_blocks in 1..65535), each running n_iter
 * iterations (1..2^28) of its chains; sink [n_blocks * n_threads] (device,
 * FP64, caller-owned) receives one value per thread.  Time it with events on
 * `stream`; the work per thread is chs_probe_ops_per_thread(kind, n_iter).
 * The run time grows with n_blocks * n_threads * n_iter: the caller bounds it. */
chs_status chs_peak_probe(int32_t kind, int32_t n_blocks, int32_t n_threads, int64_t n_iter, double* sink,
                          void* stream);

/* Operations one thread of chs_peak_probe performs: flops (FMA = 2) for the
 * FMA and MMA probes (their sum for CHS_PROBE_DFMA_DMMA), square roots for
 * CHS_PROBE_DSQRT; 0 for an unknown kind. */
double chs_probe_ops_per_thread(int32_t kind, int64_t n_iter);

/* The same jobs as chs_lyapunov_batch (Sec. Functionalities, Lyapunov item; the
 * FPU example of Sec. Examples), restricted to FPUT chains under RK4 (N in
 * {4, 8, 16, 32, 64}, any mix and order, at most 16 jobs), run as ONE persistent
 * kernel: every job is cut into the blocks its own kernel would launch, and a
 * resident grid takes those blocks from a work queue, longest chains first.
 * Results are identical to separate chs_lyapunov_spectrum calls; params.
 * block_threads and params.threads_per_orbit are ignored (the kernel's blocks
 * have 128 threads, four per orbit at N = 4, 8).  `work` is
 * caller-owned device scratch of at least 8 bytes, 8-byte aligned (the queue
 * counter, reset by the call); calls that share it and overlap on the GPU
 * race.  All jobs must be on the current device. */
chs_status chs_lyapunov_batch_persistent(const chs_lyap_job* jobs, int32_t n_jobs, void* work, size_t work_bytes,
                                         void* stream);

/* Message for the last non-OK status returned on this thread ("" if none).
 * Diagnostics; no paper counterpart. */
const char* chs_last_error(void);

/* Library version string.  Diagnostics; no paper counterpart. */
const char* chs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CHS_H */

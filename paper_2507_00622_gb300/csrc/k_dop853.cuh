// k_dop853.cuh -- launchers of the DOP853 kernels (k_dop853.cu).
#pragma once

#include "chs_internal.cuh"

namespace chs {

// Adaptive-step controls (mirror of chs_adaptive, validated on the host).
struct AdaptArgs {
    double t_final;
    double rtol, atol;
    double h_max;  // <= 0: no limit
};

// Per-orbit state of adaptive runs; err_last, err_max, n_rej may be null.
struct AdaptPtrs {
    double* t;
    double* h;
    double* err_last;
    double* err_max;
    int64_t* n_rej;
};

// Fixed-step DOP853 on the joint system (the chs_integrate_batch contract);
// ol != nullptr runs over a compacted orbit list.
cudaError_t launch_integrate_dp(const SysPar& sp, int k, bool ld, const StepArgs& a,
                                const EnsPtrs& e, const OrbitList* ol, cudaStream_t st);

// The quartic oscillator's part of launch_integrate_dp (k_dop853_q3.cu).
cudaError_t launch_integrate_dp_q3(int k, bool ld, const StepArgs& a, const SysPar& sp, const EnsPtrs& e,
                                   const OrbitList* ol, cudaStream_t st);

// Adaptive DOP 8(5) (the chs_integrate_adaptive contract).
cudaError_t launch_integrate_adaptive(const SysPar& sp, int k, bool ld, const StepArgs& a,
                                      const AdaptArgs& ad, const EnsPtrs& e, const AdaptPtrs& ap,
                                      cudaStream_t st);

// Lyapunov spectrum of the 2-DOF systems with fixed-step DOP853.
cudaError_t launch_lyap_small_dp(const SysPar& sp, const StepArgs& a, int64_t n, const double* ics,
                                 const int32_t* ic_status, double* lambda, int32_t* status,
                                 cudaStream_t st);

// FPUT Lyapunov spectrum with fixed-step DOP853 (k_fput_dp.cu); the shared-memory
// attribute is set once by prepare_fput_lyap_dp (before any stream capture).
cudaError_t launch_fput_lyap_dp(const SysPar& sp, const StepArgs& a, int64_t n, const double* ics,
                                const int32_t* ic_status, double* lambda, int32_t* status,
                                cudaStream_t st);
cudaError_t prepare_fput_lyap_dp(int n_dof);

// Lyapunov spectra with adaptive DOP 8(5) from t = 0 to ad.t_final
// (k_fput_dp.cu for FPUT, k_dop853_adapt.cu for the 2-DOF systems); n_acc and
// n_rej (accepted steps, rejected trials) may be null.
cudaError_t launch_fput_lyap_adapt(const SysPar& sp, const StepArgs& a, const AdaptArgs& ad, int64_t n,
                                   const double* ics, const int32_t* ic_status, double* lambda,
                                   int32_t* status, int64_t* n_acc, int64_t* n_rej, cudaStream_t st);
cudaError_t launch_lyap_small_adapt(const SysPar& sp, const StepArgs& a, const AdaptArgs& ad, int64_t n,
                                    const double* ics, const int32_t* ic_status, double* lambda,
                                    int32_t* status, int64_t* n_acc, int64_t* n_rej, cudaStream_t st);

// Adaptive DOP 8(5) on FPUT ensembles (k_fput_ens_adapt.cu; the
// chs_integrate_adaptive contract without LD).
cudaError_t launch_fput_ens_adapt(const SysPar& sp, int k, const StepArgs& a, const AdaptArgs& ad,
                                  const EnsPtrs& e, const AdaptPtrs& ap, cudaStream_t st);

}  // namespace chs

// chs_internal.cuh -- shared declarations of the CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/chs.h"

namespace chs {

constexpr int kSmallBlock = 128;  // threads per block of the one-orbit-per-thread kernels
constexpr int kMaxDev = 6;        // largest number of deviation vectors in an ensemble

// Model constants as the kernels see them.
struct SysPar {
    int model;
    int n_dof;
    double kk, alpha, beta, eps;
};

// Device pointers of a resumable ensemble (mirror of chs_ensemble).
struct EnsPtrs {
    int64_t n;
    double* x;
    void* w;
    double* ld;
    double* h0;
    double* dh_max;
    int64_t* n_exec;
    int32_t* status;
};

// Integration controls, validated on the host.
struct StepArgs {
    double dt;
    int64_t n_steps;
    int64_t step0;
    int32_t sample_every;  // 0: no health checks
    int32_t renorm;
    int32_t qr_every;
    int32_t ld_sqrt;       // 1: LD exponent is exactly 1/2 (sqrt path)
    double ld_p;
    double escape_r2;      // 0: off
    double dh_limit;       // 0: off
};

// Launchers (host side, one per kernel family).  Each returns the launch error.
cudaError_t launch_grid_ics(double E, double y0, double y1, int ny, double py0, double py1, int npy,
                            double* ics, int32_t* status, cudaStream_t st);
cudaError_t launch_fput_mode_ics(const SysPar& sp, int64_t n, const double* Qm, const double* Pm,
                                 const double* E, double* ics, cudaStream_t st);
cudaError_t launch_init(const SysPar& sp, int k, int vec_fp32, int renorm, uint64_t seed,
                        const double* ics, const int32_t* ic_status, const void* w_in,
                        const EnsPtrs& e, cudaStream_t st);
cudaError_t launch_integrate(const SysPar& sp, int k, int vec_fp32, bool ld, const StepArgs& a,
                             const EnsPtrs& e, cudaStream_t st);
cudaError_t launch_indicators(const SysPar& sp, int k, int vec_fp32, double sali_threshold,
                              const EnsPtrs& e, double* sali, double* gali, int8_t* label,
                              cudaStream_t st);
// FP32 deviation vectors held as an orthonormal frame plus a triangular factor
cudaError_t launch_init_f32(const SysPar& sp, int k, uint64_t seed, const double* ics,
                            const int32_t* ic_status, const void* w_in, const EnsPtrs& e,
                            cudaStream_t st);
cudaError_t launch_integrate_f32(const SysPar& sp, int k, bool ld, const StepArgs& a,
                                 const EnsPtrs& e, cudaStream_t st);
cudaError_t launch_indicators_f32(const SysPar& sp, int k, double sali_threshold, const EnsPtrs& e,
                                  double* sali, double* gali, int8_t* label, cudaStream_t st);
cudaError_t launch_ld_stencil(int ny, int npy, const double* ld, const int32_t* status,
                              double* out, cudaStream_t st);
cudaError_t launch_lyap_small(const SysPar& sp, const StepArgs& a, int64_t n, const double* ics,
                              const int32_t* ic_status, double* lambda, int32_t* status,
                              cudaStream_t st);
cudaError_t launch_fput_lyap(const SysPar& sp, const StepArgs& a, int64_t n, const double* ics,
                             const int32_t* ic_status, double* lambda, int32_t* status,
                             cudaStream_t st);

// Which systems each kernel family supports.
bool small_model(int model);
bool fput_lyap_supported(int n_dof);

inline unsigned blocks_for(int64_t n, int per_block)
{
    return (unsigned)((n + per_block - 1) / per_block);
}

}  // namespace chs

// fput_batch.cuh -- several FPUT Lyapunov jobs of uneven chain length in one
// persistent kernel (k_fput_batch.cu); shared by the kernel and the C ABI.
#pragma once

#include "chs_internal.cuh"

namespace chs {

constexpr int kFputBatchMaxJobs = 16;
struct FputBatchJob {
    StepArgs a;
    SysPar sp;
    int64_t n;
    const double* ics;
    const int32_t* ic_status;
    double* lambda;
    int32_t* status;
    int32_t n_dof;
    int32_t alpha0;  // 1: alpha == 0 (the short chains' specialised path)
    int64_t first;   // first work item of the job (set by the launcher)
};
struct FputBatchArgs {
    FputBatchJob job[kFputBatchMaxJobs];
    int32_t n_jobs;
    int64_t total;
};
cudaError_t launch_fput_lyap_batch(FputBatchJob* jobs, int n_jobs, unsigned long long* queue, cudaStream_t st);
cudaError_t prepare_fput_lyap_batch();

}  // namespace chs

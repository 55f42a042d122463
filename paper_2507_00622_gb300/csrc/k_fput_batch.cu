// k_fput_batch.cu -- Lyapunov spectra of FPUT chains of uneven length in one
// persistent kernel.
//
// A batch holds up to 16 jobs, each an ensemble of one chain length N in
// {4, 8, 16, 32, 64} under RK4.  Every job is cut into the blocks of 128
// threads its own kernel would launch (fput_lyap_lanes_block for N = 4, 8,
// fput_lyap_block for N = 16 .. 64), and those blocks are the items of a work
// queue: a resident grid takes items from a counter and runs each with the body
// of its chain length.  Jobs come in order of decreasing N, so the longest
// items start first and the short ones fill the tail.  Every orbit's arithmetic
// is that of the separate launches, so the results are identical to them.
#include "fput_batch.cuh"
#include "fput_lyap_lanes.cuh"
#include "fput_lyap_rk4.cuh"

namespace chs {
namespace {

constexpr int kBatchThreads = 128;

template <int N>
constexpr size_t batch_smem()
{
    if constexpr (N <= 8)
        return lanes::LaneCfg<N, kBatchThreads>::SMEM;
    else
        return FputLyapCfg<N, kBatchThreads>::SMEM;
}

template <int N>
constexpr int64_t batch_orbits_per_block()
{
    if constexpr (N <= 8)
        return lanes::LaneCfg<N, kBatchThreads>::G;
    else
        return FputLyapCfg<N, kBatchThreads>::G;
}

// One block per SM (the N = 64 body holds ~150 KB of shared memory): the
// compiler may spend registers up to the per-thread limit on the five bodies.
__global__ void __launch_bounds__(kBatchThreads, 1)
k_fput_lyap_batch(const FputBatchArgs b, unsigned long long* __restrict__ queue)
{
    extern __shared__ double smem[];
    __shared__ long long item_s;
    for (;;) {
        __syncthreads();  // the previous item is done with smem and item_s
        if (threadIdx.x == 0) item_s = (long long)atomicAdd(queue, 1ull);
        __syncthreads();
        const long long item = item_s;
        if (item >= b.total) break;  // block-uniform
        int j = 0;
        while (j + 1 < b.n_jobs && item >= b.job[j + 1].first) ++j;
        const FputBatchJob& J = b.job[j];
        const int64_t vb = item - J.first;
        switch (J.n_dof) {
        case 4:
            if (J.alpha0)
                lanes::fput_lyap_lanes_block<4, kBatchThreads, true>(J.a, J.sp, J.n, J.ics, J.ic_status, J.lambda,
                                                                     J.status, vb, smem);
            else
                lanes::fput_lyap_lanes_block<4, kBatchThreads, false>(J.a, J.sp, J.n, J.ics, J.ic_status, J.lambda,
                                                                      J.status, vb, smem);
            break;
        case 8:
            if (J.alpha0)
                lanes::fput_lyap_lanes_block<8, kBatchThreads, true>(J.a, J.sp, J.n, J.ics, J.ic_status, J.lambda,
                                                                     J.status, vb, smem);
            else
                lanes::fput_lyap_lanes_block<8, kBatchThreads, false>(J.a, J.sp, J.n, J.ics, J.ic_status, J.lambda,
                                                                      J.status, vb, smem);
            break;
        case 16:
            fput_lyap_block<16, kBatchThreads>(J.a, J.sp, J.n, J.ics, J.ic_status, J.lambda, J.status, vb, smem);
            break;
        case 32:
            fput_lyap_block<32, kBatchThreads>(J.a, J.sp, J.n, J.ics, J.ic_status, J.lambda, J.status, vb, smem);
            break;
        case 64:
            fput_lyap_block<64, kBatchThreads>(J.a, J.sp, J.n, J.ics, J.ic_status, J.lambda, J.status, vb, smem);
            break;
        }
    }
}

size_t smem_of(int n_dof)
{
    switch (n_dof) {
    case 4: return batch_smem<4>();
    case 8: return batch_smem<8>();
    case 16: return batch_smem<16>();
    case 32: return batch_smem<32>();
    case 64: return batch_smem<64>();
    }
    return 0;
}

int64_t orbits_per_block_of(int n_dof)
{
    switch (n_dof) {
    case 4: return batch_orbits_per_block<4>();
    case 8: return batch_orbits_per_block<8>();
    case 16: return batch_orbits_per_block<16>();
    case 32: return batch_orbits_per_block<32>();
    case 64: return batch_orbits_per_block<64>();
    }
    return 1;
}

constexpr size_t kBatchSmemMax = batch_smem<64>() > batch_smem<8>() ? batch_smem<64>() : batch_smem<8>();

}  // namespace

cudaError_t prepare_fput_lyap_batch()
{
    static bool done[kCacheDevices] = {};  // per device; set before any stream capture
    const int dev = cache_device();
    if (done[dev]) return cudaSuccess;
    const cudaError_t err =
        cudaFuncSetAttribute(k_fput_lyap_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmemMax);
    if (err == cudaSuccess) done[dev] = true;
    return err;
}

// jobs: n_jobs entries with a, sp, n, pointers, n_dof and alpha0 set; sorted
// here by decreasing chain length, with their item ranges filled in.
cudaError_t launch_fput_lyap_batch(FputBatchJob* jobs, int n_jobs, unsigned long long* queue, cudaStream_t st)
{
    if (n_jobs < 1 || n_jobs > kFputBatchMaxJobs) return cudaErrorInvalidValue;
    FputBatchArgs b{};
    // insertion sort by decreasing N (stable for equal N)
    for (int i = 0; i < n_jobs; ++i) {
        int k = i;
        while (k > 0 && b.job[k - 1].n_dof < jobs[i].n_dof) {
            b.job[k] = b.job[k - 1];
            --k;
        }
        b.job[k] = jobs[i];
    }
    b.n_jobs = n_jobs;
    size_t smem = 0;
    int64_t total = 0;
    for (int i = 0; i < n_jobs; ++i) {
        const int64_t g = orbits_per_block_of(b.job[i].n_dof);
        b.job[i].first = total;
        total += (b.job[i].n + g - 1) / g;
        const size_t s = smem_of(b.job[i].n_dof);
        if (s == 0) return cudaErrorInvalidValue;
        if (s > smem) smem = s;
    }
    b.total = total;
    if (total == 0) return cudaSuccess;
    cudaError_t err = prepare_fput_lyap_batch();
    if (err != cudaSuccess) return err;
    unsigned blocks = 0;
    if ((err = persistent_blocks(k_fput_lyap_batch, kBatchThreads, smem, &blocks)) != cudaSuccess) return err;
    if ((int64_t)blocks > total) blocks = (unsigned)total;
    if ((err = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), st)) != cudaSuccess) return err;
    k_fput_lyap_batch<<<blocks, kBatchThreads, smem, st>>>(b, queue);
    return cudaGetLastError();
}

}  // namespace chs

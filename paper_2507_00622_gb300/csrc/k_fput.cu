// k_fput.cu -- Lyapunov spectrum of the FPUT chain by periodic QR (RK4), one
// launch per chain length; the method and the layout are in fput_lyap_rk4.cuh
// (and fput_lyap_n64.cuh for the 256-thread form at N = 64).
#include "fput_lyap_n64.cuh"
#include "fput_lyap_rk4.cuh"

namespace chs {

template <int N, int T>
__global__ void __launch_bounds__(T, 1)
k_fput_lyap(const StepArgs a, const SysPar sp, const int64_t n, const double* __restrict__ ics,
            const int32_t* __restrict__ ic_status, double* __restrict__ lambda,
            int32_t* __restrict__ status_out)
{
    extern __shared__ double smem[];
    fput_lyap_block<N, T>(a, sp, n, ics, ic_status, lambda, status_out, blockIdx.x, smem);
}

__global__ void __launch_bounds__(n64::THREADS, 1)
k_fput_lyap_n64(const StepArgs a, const SysPar sp, const int64_t n, const double* __restrict__ ics,
                const int32_t* __restrict__ ic_status, double* __restrict__ lambda,
                int32_t* __restrict__ status_out)
{
    extern __shared__ double smem[];
    n64::fput_lyap_block_n64(a, sp, n, ics, ic_status, lambda, status_out, blockIdx.x, smem);
}

bool fput_lyap_supported(int n_dof)
{
    return n_dof == 4 || n_dof == 8 || n_dof == 16 || n_dof == 32 || n_dof == 64;
}

// Block sizes offered per chain length: every multiple of 2N among 32, 64, 128.
template <int N, int T>
static cudaError_t prepare_nt()
{
    if constexpr (T >= 2 * N) {
        static bool done[kCacheDevices] = {};  // per device; set before any stream capture
        const int dev = cache_device();
        if (done[dev]) return cudaSuccess;
        cudaError_t err = cudaFuncSetAttribute(k_fput_lyap<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)FputLyapCfg<N, T>::SMEM);
        if (err == cudaSuccess) done[dev] = true;
        return err;
    }
    return cudaSuccess;
}

template <int N>
static cudaError_t prepare_n()
{
    cudaError_t err = prepare_nt<N, 32>();
    if (err == cudaSuccess) err = prepare_nt<N, 64>();
    if (err == cudaSuccess) err = prepare_nt<N, 128>();
    return err;
}

static cudaError_t prepare_n64()
{
    static bool done[kCacheDevices] = {};  // per device; set before any stream capture
    const int dev = cache_device();
    if (done[dev]) return cudaSuccess;
    cudaError_t err = cudaFuncSetAttribute(k_fput_lyap_n64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)n64::SMEM);
    if (err == cudaSuccess) done[dev] = true;
    return err;
}

cudaError_t prepare_fput_lyap(int n_dof)
{
    if (fput_lyap_lanes_supported(n_dof)) return prepare_fput_lyap_lanes(n_dof);
    switch (n_dof) {
    case 16: return prepare_n<16>();
    case 32: return prepare_n<32>();
    case 64: {
        const cudaError_t err = prepare_n<64>();
        return err == cudaSuccess ? prepare_n64() : err;
    }
    }
    return cudaErrorInvalidValue;
}

template <int N, int T>
static cudaError_t fput_lyap_nt(const SysPar& sp, const StepArgs& a, int64_t n, const double* ics,
                                const int32_t* ic_status, double* lambda, int32_t* status, cudaStream_t st)
{
    if constexpr (T >= 2 * N) {
        using Cfg = FputLyapCfg<N, T>;
        cudaError_t err = prepare_nt<N, T>();
        if (err != cudaSuccess) return err;
        k_fput_lyap<N, T><<<blocks_for(n, Cfg::G), T, Cfg::SMEM, st>>>(a, sp, n, ics, ic_status, lambda, status);
        return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
}

// Default block: one warp of orbits at N = 16, one orbit of 2N threads at
// N = 32 (the smallest block; many small blocks spread an ensemble over every
// SM), one orbit of 256 threads at N = 64 (fput_lyap_n64.cuh; 128 runs the
// 128-thread body, with the same results).  The autotuner
// (autotune.tune_fput_block) measures every size per N.
template <int N>
static cudaError_t fput_lyap_n(const SysPar& sp, const StepArgs& a, int64_t n, const double* ics,
                               const int32_t* ic_status, double* lambda, int32_t* status,
                               cudaStream_t st)
{
    if constexpr (N == 64) {
        if (a.block == 0 || a.block == n64::THREADS) {
            const cudaError_t err = prepare_n64();
            if (err != cudaSuccess) return err;
            k_fput_lyap_n64<<<blocks_for(n, 1), n64::THREADS, n64::SMEM, st>>>(a, sp, n, ics, ic_status, lambda, status);
            return cudaGetLastError();
        }
    }
    switch (a.block > 0 ? a.block : (2 * N > 32 ? 2 * N : 32)) {
    case 32: return fput_lyap_nt<N, 32>(sp, a, n, ics, ic_status, lambda, status, st);
    case 64: return fput_lyap_nt<N, 64>(sp, a, n, ics, ic_status, lambda, status, st);
    case 128: return fput_lyap_nt<N, 128>(sp, a, n, ics, ic_status, lambda, status, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_fput_lyap(const SysPar& sp, const StepArgs& a, int64_t n, const double* ics,
                             const int32_t* ic_status, double* lambda, int32_t* status,
                             cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    if (fput_lyap_lanes_supported(sp.n_dof)) return launch_fput_lyap_lanes(sp, a, n, ics, ic_status, lambda, status, st);
    switch (sp.n_dof) {
    case 16: return fput_lyap_n<16>(sp, a, n, ics, ic_status, lambda, status, st);
    case 32: return fput_lyap_n<32>(sp, a, n, ics, ic_status, lambda, status, st);
    case 64: return fput_lyap_n<64>(sp, a, n, ics, ic_status, lambda, status, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace chs

// k_fput_lanes.cu -- Lyapunov spectrum of short FPUT chains (N = 4, 8) by
// periodic QR, four lanes per orbit, one launch per chain length; the method
// and the layout are in fput_lyap_lanes.cuh.
#include "fput_lyap_lanes.cuh"

namespace chs {
namespace {

using lanes::LaneCfg;

template <int N, int T, bool ALPHA0>
__global__ void __launch_bounds__(T)
k_fput_lyap_lanes(const StepArgs a, const SysPar sp, const int64_t n, const double* __restrict__ ics,
                  const int32_t* __restrict__ ic_status, double* __restrict__ lambda,
                  int32_t* __restrict__ status_out)
{
    extern __shared__ double smem[];
    lanes::fput_lyap_lanes_block<N, T, ALPHA0>(a, sp, n, ics, ic_status, lambda, status_out, blockIdx.x, smem);
}

template <int N, int T, bool A0>
cudaError_t prepare_nta()
{
    static bool done[kCacheDevices] = {};  // per device; set before any stream capture
    const int dev = cache_device();
    if (done[dev]) return cudaSuccess;
    const cudaError_t err = cudaFuncSetAttribute(k_fput_lyap_lanes<N, T, A0>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)LaneCfg<N, T>::SMEM);
    if (err == cudaSuccess) done[dev] = true;
    return err;
}

template <int N, int T>
cudaError_t prepare_nt()
{
    cudaError_t err = prepare_nta<N, T, true>();
    if (err == cudaSuccess) err = prepare_nta<N, T, false>();
    return err;
}

template <int N, int T>
cudaError_t launch_nt(const SysPar& sp, const StepArgs& a, int64_t n, const double* ics, const int32_t* ic_status,
                      double* lambda, int32_t* status, cudaStream_t st)
{
    using Cfg = LaneCfg<N, T>;
    cudaError_t err = prepare_nt<N, T>();
    if (err != cudaSuccess) return err;
    if (sp.alpha == 0.0)
        k_fput_lyap_lanes<N, T, true><<<blocks_for(n, Cfg::G), T, Cfg::SMEM, st>>>(a, sp, n, ics, ic_status,
                                                                                 lambda, status);
    else
        k_fput_lyap_lanes<N, T, false><<<blocks_for(n, Cfg::G), T, Cfg::SMEM, st>>>(a, sp, n, ics, ic_status,
                                                                                  lambda, status);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_n(const SysPar& sp, const StepArgs& a, int64_t n, const double* ics, const int32_t* ic_status,
                     double* lambda, int32_t* status, cudaStream_t st)
{
    switch (a.block > 0 ? a.block : 32) {
    case 32: return launch_nt<N, 32>(sp, a, n, ics, ic_status, lambda, status, st);
    case 64: return launch_nt<N, 64>(sp, a, n, ics, ic_status, lambda, status, st);
    case 128: return launch_nt<N, 128>(sp, a, n, ics, ic_status, lambda, status, st);
    }
    return cudaErrorInvalidValue;
}

template <int N>
cudaError_t prepare_n()
{
    cudaError_t err = prepare_nt<N, 32>();
    if (err == cudaSuccess) err = prepare_nt<N, 64>();
    if (err == cudaSuccess) err = prepare_nt<N, 128>();
    return err;
}

}  // namespace

bool fput_lyap_lanes_supported(int n_dof) { return n_dof == 4 || n_dof == 8; }

cudaError_t prepare_fput_lyap_lanes(int n_dof)
{
    switch (n_dof) {
    case 4: return prepare_n<4>();
    case 8: return prepare_n<8>();
    }
    return cudaErrorInvalidValue;
}

// Default block: one warp (8 orbits), whose accesses to the block's shared
// arrays are conflict-free; 64 and 128 threads are offered to the tuner.
cudaError_t launch_fput_lyap_lanes(const SysPar& sp, const StepArgs& a, int64_t n, const double* ics,
                                   const int32_t* ic_status, double* lambda, int32_t* status, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    switch (sp.n_dof) {
    case 4: return launch_n<4>(sp, a, n, ics, ic_status, lambda, status, st);
    case 8: return launch_n<8>(sp, a, n, ics, ic_status, lambda, status, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace chs

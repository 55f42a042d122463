// k_fput_lanes.cu -- Lyapunov spectrum of short FPUT chains (N = 4, 8) by
// periodic QR, several lanes of one warp per orbit, one launch per chain
// length; the method and the layout are in fput_lyap_lanes.cuh.
#include "fput_lyap_lanes.cuh"

namespace chs {
namespace {

using lanes::LaneCfg;

template <int N, int T, bool ALPHA0, int L>
__global__ void __launch_bounds__(T, 1)
k_fput_lyap_lanes(const StepArgs a, const SysPar sp, const int64_t n, const double* __restrict__ ics,
                  const int32_t* __restrict__ ic_status, double* __restrict__ lambda,
                  int32_t* __restrict__ status_out)
{
    extern __shared__ double smem[];
    lanes::fput_lyap_lanes_block<N, T, ALPHA0, L>(a, sp, n, ics, ic_status, lambda, status_out, blockIdx.x, smem);
}

template <int N, int T, bool A0, int L>
cudaError_t prepare_nta()
{
    static bool done[kCacheDevices] = {};  // per device; set before any stream capture
    const int dev = cache_device();
    if (done[dev]) return cudaSuccess;
    const cudaError_t err = cudaFuncSetAttribute(k_fput_lyap_lanes<N, T, A0, L>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)LaneCfg<N, T, L>::SMEM);
    if (err == cudaSuccess) done[dev] = true;
    return err;
}

template <int N, int T, int L>
cudaError_t prepare_ntl()
{
    cudaError_t err = prepare_nta<N, T, true, L>();
    if (err == cudaSuccess) err = prepare_nta<N, T, false, L>();
    return err;
}

template <int N, int T, int L>
cudaError_t launch_ntl(const SysPar& sp, const StepArgs& a, int64_t n, const double* ics, const int32_t* ic_status,
                       double* lambda, int32_t* status, cudaStream_t st)
{
    using Cfg = LaneCfg<N, T, L>;
    cudaError_t err = prepare_ntl<N, T, L>();
    if (err != cudaSuccess) return err;
    if (sp.alpha == 0.0)
        k_fput_lyap_lanes<N, T, true, L><<<blocks_for(n, Cfg::G), T, Cfg::SMEM, st>>>(a, sp, n, ics, ic_status,
                                                                                    lambda, status);
    else
        k_fput_lyap_lanes<N, T, false, L><<<blocks_for(n, Cfg::G), T, Cfg::SMEM, st>>>(a, sp, n, ics, ic_status,
                                                                                     lambda, status);
    return cudaGetLastError();
}

template <int N, int L>
cudaError_t launch_nl(const SysPar& sp, const StepArgs& a, int64_t n, const double* ics, const int32_t* ic_status,
                      double* lambda, int32_t* status, cudaStream_t st)
{
    switch (a.block > 0 ? a.block : (N == 4 ? 64 : 32)) {
    case 32: return launch_ntl<N, 32, L>(sp, a, n, ics, ic_status, lambda, status, st);
    case 64: return launch_ntl<N, 64, L>(sp, a, n, ics, ic_status, lambda, status, st);
    case 128: return launch_ntl<N, 128, L>(sp, a, n, ics, ic_status, lambda, status, st);
    }
    return cudaErrorInvalidValue;
}

template <int N, int L>
cudaError_t prepare_nl()
{
    cudaError_t err = prepare_ntl<N, 32, L>();
    if (err == cudaSuccess) err = prepare_ntl<N, 64, L>();
    if (err == cudaSuccess) err = prepare_ntl<N, 128, L>();
    return err;
}

}  // namespace

bool fput_lyap_lanes_supported(int n_dof) { return n_dof == 4 || n_dof == 8; }

bool fput_lanes_per_orbit_supported(int n_dof, int lanes)
{
    if (lanes == 0) return true;
    if (n_dof == 4) return lanes == 1 || lanes == 2 || lanes == 4;
    if (n_dof == 8) return lanes == 2 || lanes == 4 || lanes == 8;
    return false;
}

cudaError_t prepare_fput_lyap_lanes(int n_dof)
{
    cudaError_t err = cudaErrorInvalidValue;
    switch (n_dof) {
    case 4:
        err = prepare_nl<4, 4>();
        if (err == cudaSuccess) err = prepare_nl<4, 2>();
        if (err == cudaSuccess) err = prepare_nl<4, 1>();
        break;
    case 8:
        err = prepare_nl<8, 4>();
        if (err == cudaSuccess) err = prepare_nl<8, 2>();
        if (err == cudaSuccess) err = prepare_nl<8, 8>();
        break;
    }
    return err;
}

// Default: four lanes per orbit in blocks of two warps at N = 4 (16 orbits per
// block), eight lanes (one mass, two columns each) in one-warp blocks at N = 8;
// the faster on 4096-orbit ensembles (ms per 200 steps at QR every 10: N = 4
// 2.06-2.09 with 4 lanes, 3.65 with 2; N = 8 5.51 with 8 lanes, 7.33 with 4).
// The other lane counts and block sizes are offered to the tuner.
cudaError_t launch_fput_lyap_lanes(const SysPar& sp, const StepArgs& a, int64_t n, const double* ics,
                                   const int32_t* ic_status, double* lambda, int32_t* status, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const int lanes = a.threads_per_orbit > 0 ? a.threads_per_orbit : (sp.n_dof == 8 ? 8 : 4);
    if (sp.n_dof == 4) {
        switch (lanes) {
        case 4: return launch_nl<4, 4>(sp, a, n, ics, ic_status, lambda, status, st);
        case 2: return launch_nl<4, 2>(sp, a, n, ics, ic_status, lambda, status, st);
        case 1: return launch_nl<4, 1>(sp, a, n, ics, ic_status, lambda, status, st);
        }
    } else if (sp.n_dof == 8) {
        switch (lanes) {
        case 4: return launch_nl<8, 4>(sp, a, n, ics, ic_status, lambda, status, st);
        case 2: return launch_nl<8, 2>(sp, a, n, ics, ic_status, lambda, status, st);
        case 8: return launch_nl<8, 8>(sp, a, n, ics, ic_status, lambda, status, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace chs

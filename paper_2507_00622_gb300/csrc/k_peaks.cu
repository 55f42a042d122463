// k_peaks.cu -- throughput probes of the arithmetic pipes the integrators run on.
//
// The hot path is bound by the FP64 pipe (FP32 for the deviation-vector frame
// of the FP32 mode), whose peaks are not among the measured HBM and BF16
// figures of the platform.  These kernels measure them: every thread runs
// kChains independent dependency chains of one operation for n_iter
// iterations and writes one value so that nothing is optimised away.
//   CHS_PROBE_DFMA      x <- fma(x, a, b) in FP64, kChains chains per thread
//   CHS_PROBE_DFMA_DEP  the same with a single chain (dependent latency)
//   CHS_PROBE_FFMA      the FP32 version of CHS_PROBE_DFMA
//   CHS_PROBE_DSQRT     x <- sqrt(fma(x, a, b)) in FP64 (CUDA's correctly
//                       rounded sqrt), kChains chains
//   CHS_PROBE_DMMA      D <- A B + D by mma.sync m8n8k4 in FP64, kChains
//                       independent accumulators per warp
//   CHS_PROBE_DFMA_DMMA kMix FMA chains per thread and kMix MMA accumulators
//                       per warp in one loop: if the two used separate pipes
//                       their rates would add (on GB300 they do not)
// The operation count per thread is chs_probe_ops_per_thread(kind, n_iter).
#include "chs_internal.cuh"

namespace chs {
namespace {

constexpr int kChains = 8;

template <int CHAINS>
__global__ void k_probe_dfma(int64_t n_iter, double a, double b, double* __restrict__ sink)
{
    double x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = 1e-3 * threadIdx.x + c;
#pragma unroll 1
    for (int64_t it = 0; it < n_iter; it += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_probe_ffma(int64_t n_iter, float a, float b, double* __restrict__ sink)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * threadIdx.x + c;
#pragma unroll 1
    for (int64_t it = 0; it < n_iter; it += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_probe_dsqrt(int64_t n_iter, double a, double b, double* __restrict__ sink)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * threadIdx.x + c;
#pragma unroll 1
    for (int64_t it = 0; it < n_iter; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = sqrt(fma(x[c], a, b));
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// One m8n8k4 FP64 MMA: a warp multiplies an 8x4 A (one element per lane) by a
// 4x8 B (one element per lane) into an 8x8 accumulator (two elements per lane).
__device__ __forceinline__ void mma_m8n8k4(double& d0, double& d1, double a, double b)
{
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                 : "+d"(d0), "+d"(d1)
                 : "d"(a), "d"(b));
}

__global__ void k_probe_dmma(int64_t n_iter, double a, double b, double* __restrict__ sink)
{
    double d0[kChains], d1[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        d0[c] = 1e-3 * threadIdx.x + c;
        d1[c] = 0.5 * c;
    }
    // A and B scaled so that the accumulators stay bounded: |A B| row sums < 1
    const double av = a * (1.0 + 1e-3 * (threadIdx.x & 31)), bv = b;
#pragma unroll 1
    for (int64_t it = 0; it < n_iter; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) mma_m8n8k4(d0[c], d1[c], av, bv);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += d0[c] + d1[c];
    sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

constexpr int kMix = 4;

__global__ void k_probe_dfma_dmma(int64_t n_iter, double a, double b, double ma, double* __restrict__ sink)
{
    double x[kMix], d0[kMix], d1[kMix];
#pragma unroll
    for (int c = 0; c < kMix; ++c) {
        x[c] = 1e-3 * threadIdx.x + c;
        d0[c] = 1e-3 * threadIdx.x + c;
        d1[c] = 0.5 * c;
    }
    const double av = ma * (1.0 + 1e-3 * (threadIdx.x & 31));
#pragma unroll 1
    for (int64_t it = 0; it < n_iter; ++it) {
#pragma unroll
        for (int c = 0; c < kMix; ++c) {
            x[c] = fma(x[c], a, b);
            mma_m8n8k4(d0[c], d1[c], av, ma);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kMix; ++c) s += x[c] + d0[c] + d1[c];
    sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

cudaError_t launch_peak_probe(int kind, int n_blocks, int n_threads, int64_t n_iter, double* sink,
                              cudaStream_t st)
{
    switch (kind) {
    case CHS_PROBE_DFMA:
        k_probe_dfma<kChains><<<n_blocks, n_threads, 0, st>>>(n_iter, 0.999999, 1e-6, sink);
        break;
    case CHS_PROBE_DFMA_DEP:
        k_probe_dfma<1><<<n_blocks, n_threads, 0, st>>>(n_iter, 0.999999, 1e-6, sink);
        break;
    case CHS_PROBE_FFMA:
        k_probe_ffma<<<n_blocks, n_threads, 0, st>>>(n_iter, 0.9999f, 1e-4f, sink);
        break;
    case CHS_PROBE_DSQRT:
        k_probe_dsqrt<<<n_blocks, n_threads, 0, st>>>(n_iter, 0.75, 0.7, sink);
        break;
    case CHS_PROBE_DMMA:
        k_probe_dmma<<<n_blocks, n_threads, 0, st>>>(n_iter, 0.03, 0.03, sink);
        break;
    case CHS_PROBE_DFMA_DMMA:
        k_probe_dfma_dmma<<<n_blocks, n_threads, 0, st>>>(n_iter, 0.999999, 1e-6, 0.03, sink);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

double probe_ops_per_thread(int kind, int64_t n_iter)
{
    // the FMA probes step in groups of 4 iterations
    const double it4 = (double)((n_iter + 3) / 4 * 4);
    switch (kind) {
    case CHS_PROBE_DFMA:
    case CHS_PROBE_FFMA:
        return 2.0 * kChains * it4;  // flops, FMA = 2
    case CHS_PROBE_DFMA_DEP:
        return 2.0 * it4;
    case CHS_PROBE_DSQRT:
        return (double)kChains * (double)n_iter;  // square roots (each with one FMA)
    case CHS_PROBE_DMMA:
        return 2.0 * 8 * 8 * 4 * kChains * (double)n_iter / 32.0;  // flops per lane
    case CHS_PROBE_DFMA_DMMA:
        return (2.0 * kMix + 2.0 * 8 * 8 * 4 * kMix / 32.0) * (double)n_iter;
    }
    return 0.0;
}

}  // namespace chs

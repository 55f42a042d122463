// k_mlp.cu -- the early-stop surrogate: a 12 -> 128 -> 128 -> 128 -> 2 ReLU
// multilayer perceptron with BF16 weights and activations and FP32
// accumulation, its training kernels (loss gradient, backward pass, Adam) and
// the fused decision kernel used during integration.
//
// Inputs (features) of an orbit still running at the decision time t:
//   f_i = log10(max(SALI(t_i), 1e-20)) / 8,  t_i = (i + 1) t / S, i < S (S = 10)
//   f_10 = LD(t) / t - 1            (the mean LD rate, centred)
//   f_11 = (E_o - 0.133) / 0.033    (the orbit's energy, centred)
// Outputs: y_0 = logit of "chaotic at the final time", y_1 = final log10(SALI) / 8.
//
// Parameter layout (one flat array, row-major out x in):
//   W1 [128][12], b1 [128], W2 [128][128], b2 [128], W3 [128][128], b3 [128],
//   W4 [2][128], b4 [2]   -- 34,946 values.
//
// The work is tiny next to the integration (about 35k multiply-adds per orbit),
// so the kernels run on the FP32 CUDA-core pipe with the layer weights staged in
// shared memory; the weights and activations are stored in BF16.
#include <cuda_bf16.h>
#include <math.h>

#include "chs_internal.cuh"

namespace chs {

constexpr int kF = 12, kH = 128, kO = 2, kS = 10;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kF, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kH, kOffW4 = kOffB3 + kH,
              kOffB4 = kOffW4 + kO * kH, kParams = kOffB4 + kO;
constexpr int kTile = 64;       // samples per block
constexpr int kThreads = 256;

size_t mlp_param_count() { return (size_t)kParams; }

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// Features of orbit o (see the file comment); non-finite SALI samples count as 1e-20.
__device__ __forceinline__ void features(const double* __restrict__ series, const int S, const double* ld,
                                         const double t, const double* E, const int64_t n, const int64_t o,
                                         float* f)
{
    for (int i = 0; i < kS; ++i) {
        double s = i < S ? series[(int64_t)i * n + o] : 1e-20;
        s = (s > 1e-20 && isfinite(s)) ? s : 1e-20;
        f[i] = (float)(log10(s) / 8.0);
    }
    f[10] = (float)(ld[o] / t - 1.0);
    f[11] = (float)((E[o] - 0.133) / 0.033);
}

__global__ void k_mlp_features(const double* __restrict__ series, const int S, const double* __restrict__ ld,
                               const double t, const double* __restrict__ E, const int64_t n, float* __restrict__ X)
{
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    float f[kF];
    features(series, S, ld, t, E, n, o, f);
#pragma unroll
    for (int i = 0; i < kF; ++i) X[(int64_t)i * n + o] = f[i];
}

// One dense layer on a tile of kTile samples held in shared memory:
//   out[u][s] = act(b[u] + sum_k W[u][k] in[k][s]),  u < U, k < K.
// For U >= 32 each thread owns a (U/32) x (kTile/8) register tile (units tu + 32a,
// samples ts + 8b), so the 256 threads cover U x kTile outputs.
template <int U, int K, bool RELU>
__device__ __forceinline__ void dense_tile(const __nv_bfloat16* __restrict__ Wg, const __nv_bfloat16* __restrict__ bg,
                                           float* __restrict__ Ws, const float* __restrict__ in,
                                           float* __restrict__ out)
{
    // stage the weights as float
    for (int i = threadIdx.x; i < U * K; i += kThreads) Ws[i] = bf(Wg[i]);
    __syncthreads();
    if constexpr (U >= 32) {
        constexpr int TU = U / 32;     // units per thread
        constexpr int TS = kTile / 8;  // samples per thread
        const int tu = threadIdx.x % 32, ts = threadIdx.x / 32;
        float acc[TU][TS];
#pragma unroll
        for (int a = 0; a < TU; ++a)
#pragma unroll
            for (int b = 0; b < TS; ++b) acc[a][b] = 0.0f;
        for (int k = 0; k < K; ++k) {
            float wv[TU], iv[TS];
#pragma unroll
            for (int a = 0; a < TU; ++a) wv[a] = Ws[(tu + 32 * a) * K + k];
#pragma unroll
            for (int b = 0; b < TS; ++b) iv[b] = in[k * kTile + ts + 8 * b];
#pragma unroll
            for (int a = 0; a < TU; ++a)
#pragma unroll
                for (int b = 0; b < TS; ++b) acc[a][b] = fmaf(wv[a], iv[b], acc[a][b]);
        }
#pragma unroll
        for (int a = 0; a < TU; ++a) {
            const int u = tu + 32 * a;
            const float bu = bf(bg[u]);
#pragma unroll
            for (int b = 0; b < TS; ++b) {
                float v = acc[a][b] + bu;
                if (RELU) v = fmaxf(v, 0.0f);
                out[u * kTile + ts + 8 * b] = bf(__float2bfloat16_rn(v));  // BF16 activations
            }
        }
    } else {
        // small output layer: one (unit, sample) pair per thread
        for (int p = threadIdx.x; p < U * kTile; p += kThreads) {
            const int u = p / kTile, s = p % kTile;
            float acc = 0.0f;
            for (int k = 0; k < K; ++k) acc = fmaf(Ws[u * K + k], in[k * kTile + s], acc);
            float v = acc + bf(bg[u]);
            if (RELU) v = fmaxf(v, 0.0f);
            out[u * kTile + s] = v;
        }
    }
    __syncthreads();
}

// Forward pass over the features X [12][n] (or, when series != NULL, over the
// features built on the fly); writes Y [2][n] and, when act != NULL, the three
// hidden activations [3][128][n] (BF16) for the backward pass.  With decide:
// orbits whose status is OK take status EARLY_CHAOTIC when sigmoid(y0) >= conf
// and PREDICTED_REGULAR when sigmoid(y0) <= 1 - conf, and t_end is not touched.
template <bool FROM_SERIES>
__global__ void __launch_bounds__(kThreads)
k_mlp_forward(const __nv_bfloat16* __restrict__ P, const float* __restrict__ X, const double* __restrict__ series,
              const int S, const double* __restrict__ ld, const double t, const double* __restrict__ E, const int64_t n,
              float* __restrict__ Y, __nv_bfloat16* __restrict__ act, int32_t* __restrict__ status,
              const double conf, float* __restrict__ prob)
{
    extern __shared__ float sm[];
    float* Ws = sm;                        // kH * kH
    float* A = Ws + kH * kH;               // kH * kTile
    float* B = A + kH * kTile;             // kH * kTile
    const int64_t s0 = (int64_t)blockIdx.x * kTile;
    // input tile
    if (FROM_SERIES) {
        for (int s = threadIdx.x; s < kTile; s += kThreads) {
            const int64_t o = s0 + s;
            float fv[kF];
            if (o < n) {
                features(series, S, ld, t, E, n, o, fv);
            } else {
#pragma unroll
                for (int f = 0; f < kF; ++f) fv[f] = 0.0f;
            }
#pragma unroll
            for (int f = 0; f < kF; ++f) A[f * kTile + s] = fv[f];
        }
    } else {
        for (int p = threadIdx.x; p < kF * kTile; p += kThreads) {
            const int f = p / kTile, s = p % kTile;
            const int64_t o = s0 + s;
            A[f * kTile + s] = o < n ? X[(int64_t)f * n + o] : 0.0f;
        }
    }
    __syncthreads();
    dense_tile<kH, kF, true>(P + kOffW1, P + kOffB1, Ws, A, B);
    if (act)
        for (int p = threadIdx.x; p < kH * kTile; p += kThreads) {
            const int64_t o = s0 + p % kTile;
            if (o < n) act[(int64_t)(p / kTile) * n + o] = __float2bfloat16_rn(B[p]);
        }
    dense_tile<kH, kH, true>(P + kOffW2, P + kOffB2, Ws, B, A);
    if (act)
        for (int p = threadIdx.x; p < kH * kTile; p += kThreads) {
            const int64_t o = s0 + p % kTile;
            if (o < n) act[(int64_t)(kH + p / kTile) * n + o] = __float2bfloat16_rn(A[p]);
        }
    dense_tile<kH, kH, true>(P + kOffW3, P + kOffB3, Ws, A, B);
    if (act)
        for (int p = threadIdx.x; p < kH * kTile; p += kThreads) {
            const int64_t o = s0 + p % kTile;
            if (o < n) act[(int64_t)(2 * kH + p / kTile) * n + o] = __float2bfloat16_rn(B[p]);
        }
    dense_tile<kO, kH, false>(P + kOffW4, P + kOffB4, Ws, B, A);
    for (int s = threadIdx.x; s < kTile; s += kThreads) {
        const int64_t o = s0 + s;
        if (o >= n) continue;
        const float y0 = A[s], y1 = A[kTile + s];
        if (Y) {
            Y[o] = y0;
            Y[n + o] = y1;
        }
        if (status) {
            const double pc = 1.0 / (1.0 + exp(-(double)y0));
            if (prob) prob[o] = (float)pc;
            if (status[o] == CHS_ORBIT_OK) {
                if (pc >= conf)
                    status[o] = CHS_ORBIT_EARLY_CHAOTIC;
                else if (pc <= 1.0 - conf)
                    status[o] = CHS_ORBIT_PREDICTED_REGULAR;
            }
        }
    }
}

// Loss and its gradient w.r.t. the outputs, averaged over n:
//   L = BCE(sigmoid(y0), label) + w_reg (y1 - target)^2,
//   dL/dy0 = (sigmoid(y0) - label) / n,  dL/dy1 = 2 w_reg (y1 - target) / n.
// loss_out (one float) accumulates the batch loss (atomicAdd; zero it first).
__global__ void k_mlp_loss_grad(const float* __restrict__ Y, const float* __restrict__ label,
                                const float* __restrict__ target, const int64_t n, const float w_reg,
                                float* __restrict__ dY, float* __restrict__ loss_out)
{
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (o < n) {
        const float y0 = Y[o], y1 = Y[n + o], lb = label[o], tg = target[o];
        const float p = 1.0f / (1.0f + expf(-y0));
        // log(1 + exp(-|y|)) form of the cross entropy
        l = fmaxf(y0, 0.0f) - y0 * lb + log1pf(expf(-fabsf(y0))) + w_reg * (y1 - tg) * (y1 - tg);
        dY[o] = (p - lb) / (float)n;
        dY[n + o] = 2.0f * w_reg * (y1 - tg) / (float)n;
    }
    for (int off = 16; off > 0; off >>= 1) l += __shfl_down_sync(0xffffffffu, l, off);
    if ((threadIdx.x & 31) == 0 && o - (threadIdx.x & 31) < n) atomicAdd(loss_out, l / (float)n);
}

// Back-propagation of one sample tile: from dY [2][n] and the stored
// activations, the pre-activation gradients of every layer:
//   d4 = dY;  d3 = (W4^T d4) * [a3 > 0];  d2 = (W3^T d3) * [a2 > 0];  d1 = (W2^T d2) * [a1 > 0]
// written as FP32 [3][128][n] (d1, d2, d3).
__global__ void __launch_bounds__(kThreads)
k_mlp_backprop(const __nv_bfloat16* __restrict__ P, const __nv_bfloat16* __restrict__ act,
               const float* __restrict__ dY, const int64_t n, float* __restrict__ delta)
{
    extern __shared__ float sm[];
    float* Ws = sm;                 // kH * kH (transposed use)
    float* D = Ws + kH * kH;        // kH * kTile  (gradient entering a layer)
    float* E2 = D + kH * kTile;     // kH * kTile
    const int64_t s0 = (int64_t)blockIdx.x * kTile;
    // layer 4: d3 = W4^T dY masked by a3 > 0
    for (int i = threadIdx.x; i < kO * kH; i += kThreads) Ws[i] = bf(P[kOffW4 + i]);
    for (int p = threadIdx.x; p < kO * kTile; p += kThreads) {
        const int64_t o = s0 + p % kTile;
        D[p] = o < n ? dY[(int64_t)(p / kTile) * n + o] : 0.0f;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < kH * kTile; p += kThreads) {
        const int k = p / kTile, s = p % kTile;
        const int64_t o = s0 + s;
        float g = Ws[0 * kH + k] * D[0 * kTile + s] + Ws[1 * kH + k] * D[1 * kTile + s];
        const float a = o < n ? bf(act[(int64_t)(2 * kH + k) * n + o]) : 0.0f;
        g = a > 0.0f ? g : 0.0f;
        E2[p] = g;
        if (o < n) delta[(int64_t)(2 * kH + k) * n + o] = g;
    }
    __syncthreads();
    // layers 3 and 2: d_{l-1}[k][s] = sum_u W_l[u][k] d_l[u][s], masked by a_{l-1} > 0
    float* cur = E2;
    float* nxt = D;
    for (int layer = 3; layer >= 2; --layer) {
        const __nv_bfloat16* Wg = P + (layer == 3 ? kOffW3 : kOffW2);
        for (int i = threadIdx.x; i < kH * kH; i += kThreads) Ws[i] = bf(Wg[i]);
        __syncthreads();
        const int tk = threadIdx.x % 32, ts = threadIdx.x / 32;
        float acc[4][8];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;
        for (int u = 0; u < kH; ++u) {
            float wv[4], dv[8];
#pragma unroll
            for (int a = 0; a < 4; ++a) wv[a] = Ws[u * kH + tk + 32 * a];
#pragma unroll
            for (int b = 0; b < 8; ++b) dv[b] = cur[u * kTile + ts + 8 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(wv[a], dv[b], acc[a][b]);
        }
        const int aidx = layer - 2;  // activation index of a_{layer-1}: layer 3 -> a2 (1), layer 2 -> a1 (0)
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int k = tk + 32 * a;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const int s = ts + 8 * b;
                const int64_t o = s0 + s;
                const float av = o < n ? bf(act[(int64_t)(aidx * kH + k) * n + o]) : 0.0f;
                const float g = av > 0.0f ? acc[a][b] : 0.0f;
                nxt[k * kTile + s] = g;
                if (o < n) delta[(int64_t)(aidx * kH + k) * n + o] = g;
            }
        }
        __syncthreads();
        float* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
}

// Weight and bias gradients as batch reductions:
//   dW_l[u][k] = sum_s d_l[u][s] a_{l-1}[k][s],  db_l[u] = sum_s d_l[u][s]
// with a_0 = X, d_4 = dY.  One block per 32 x 32 tile of one layer's dW.
__global__ void __launch_bounds__(kThreads)
k_mlp_wgrad(const float* __restrict__ X, const __nv_bfloat16* __restrict__ act, const float* __restrict__ delta,
            const float* __restrict__ dY, const int64_t n, float* __restrict__ G)
{
    __shared__ float Ds[32][33], As[32][33];
    // tiles: layer 1: 4 x 1 (U = 128, K = 12 -> one padded k tile); layers 2, 3: 4 x 4; layer 4: 1 x 4
    int b = blockIdx.x;
    int layer, ut, kt;
    if (b < 4) { layer = 1; ut = b; kt = 0; }
    else if (b < 20) { layer = 2; ut = (b - 4) / 4; kt = (b - 4) % 4; }
    else if (b < 36) { layer = 3; ut = (b - 20) / 4; kt = (b - 20) % 4; }
    else { layer = 4; ut = 0; kt = b - 36; }
    const int U = layer == 4 ? kO : kH, K = layer == 1 ? kF : kH;
    const int tu = threadIdx.x / 8, tk0 = (threadIdx.x % 8) * 4;  // 32 rows x (8 threads x 4 cols)
    float acc[4] = {0.f, 0.f, 0.f, 0.f}, accb = 0.0f;
    for (int64_t c = 0; c < n; c += 32) {
        for (int p = threadIdx.x; p < 32 * 32; p += kThreads) {
            const int r = p / 32, s = p % 32;
            const int64_t o = c + s;
            const int u = ut * 32 + r, k = kt * 32 + r;
            float dv = 0.0f, av = 0.0f;
            if (o < n) {
                if (u < U) dv = layer == 4 ? dY[(int64_t)u * n + o] : delta[(int64_t)((layer - 1) * kH + u) * n + o];
                if (k < K) av = layer == 1 ? X[(int64_t)k * n + o] : bf(act[(int64_t)((layer - 2) * kH + k) * n + o]);
            }
            Ds[r][s] = dv;
            As[r][s] = av;
        }
        __syncthreads();
#pragma unroll 8
        for (int s = 0; s < 32; ++s) {
            const float dv = Ds[tu][s];
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[j] = fmaf(dv, As[tk0 + j][s], acc[j]);
            accb += dv;
        }
        __syncthreads();
    }
    const int u = ut * 32 + tu;
    if (u >= U) return;
    const int offW = layer == 1 ? kOffW1 : layer == 2 ? kOffW2 : layer == 3 ? kOffW3 : kOffW4;
    const int offB = layer == 1 ? kOffB1 : layer == 2 ? kOffB2 : layer == 3 ? kOffB3 : kOffB4;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int k = kt * 32 + tk0 + j;
        if (k < K) G[offW + u * K + k] = acc[j];
    }
    if (kt == 0 && tk0 == 0) G[offB + u] = accb;
}

// Adam on FP32 master weights; writes the BF16 copy used by the kernels.
__global__ void k_mlp_adam(float* __restrict__ W, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ g, const int64_t P, const float lr, const float b1,
                           const float b2, const float eps, const float c1, const float c2,
                           __nv_bfloat16* __restrict__ Wb)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float w = W[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    W[i] = w;
    Wb[i] = __float2bfloat16_rn(w);
}

// ---------------------------------------------------------------------------

static constexpr size_t kFwdSmem = (size_t)(kH * kH + 2 * kH * kTile) * sizeof(float);

cudaError_t launch_mlp_features(const double* series, int S, const double* ld, double t, const double* E,
                                int64_t n, float* X, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_mlp_features<<<blocks_for(n, 256), 256, 0, st>>>(series, S, ld, t, E, n, X);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const void* P, const float* X, int64_t n, float* Y, void* act,
                               cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kFwdSmem);
    if (e != cudaSuccess) return e;
    k_mlp_forward<false><<<blocks_for(n, kTile), kThreads, kFwdSmem, st>>>(
        static_cast<const __nv_bfloat16*>(P), X, nullptr, 0, nullptr, 0.0, nullptr, n, Y,
        static_cast<__nv_bfloat16*>(act), nullptr, 0.0, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_mlp_decide(const void* P, const double* series, int S, const double* ld, double t,
                              const double* E, int64_t n, double conf, int32_t* status, float* prob,
                              cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kFwdSmem);
    if (e != cudaSuccess) return e;
    k_mlp_forward<true><<<blocks_for(n, kTile), kThreads, kFwdSmem, st>>>(
        static_cast<const __nv_bfloat16*>(P), nullptr, series, S, ld, t, E, n, nullptr, nullptr, status,
        conf, prob);
    return cudaGetLastError();
}

cudaError_t launch_mlp_loss_grad(const float* Y, const float* label, const float* target, int64_t n,
                                 float w_reg, float* dY, float* loss, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e != cudaSuccess) return e;
    k_mlp_loss_grad<<<blocks_for(n, 256), 256, 0, st>>>(Y, label, target, n, w_reg, dY, loss);
    return cudaGetLastError();
}

cudaError_t launch_mlp_backward(const void* P, const float* X, const void* act, const float* dY,
                                int64_t n, float* delta, float* G, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_backprop, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kFwdSmem);
    if (e != cudaSuccess) return e;
    k_mlp_backprop<<<blocks_for(n, kTile), kThreads, kFwdSmem, st>>>(
        static_cast<const __nv_bfloat16*>(P), static_cast<const __nv_bfloat16*>(act), dY, n, delta);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_mlp_wgrad<<<40, kThreads, 0, st>>>(X, static_cast<const __nv_bfloat16*>(act), delta, dY, n, G);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* W, float* m, float* v, const float* g, float lr, float b1, float b2,
                            float eps, int step, void* Wb, cudaStream_t st)
{
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    k_mlp_adam<<<blocks_for(kParams, 256), 256, 0, st>>>(W, m, v, g, kParams, lr, b1, b2, eps, c1, c2,
                                                         static_cast<__nv_bfloat16*>(Wb));
    return cudaGetLastError();
}

}  // namespace chs

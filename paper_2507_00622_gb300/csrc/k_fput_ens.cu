// k_fput_ens.cu -- ensembles of FPUT chains with k <= 6 deviation vectors
// (Sec. Examples, the FPU model, Eqs. ham_FPU / ham_eqs_FPU with fixed ends):
// set-up, fixed-step RK4 or DOP853 on the joint system (x, w_1..w_k), and the
// indicators SALI and GALI_2..k.  The paper times GALI_4 of 1e3 FPU orbits
// against the number of degrees of freedom; this is that workload.
//
// A step runs in the two phases of fput_stages.cuh: the orbit through its
// stages with one thread per component (stage states through shared memory),
// then every deviation vector through the same stages on a warp segment that
// exchanges the tridiagonal neighbours by shuffles.  With renorm the vectors are
// scaled to unit length inside phase 2.  The checks of fput_ens.cuh follow.
// A block steps its G orbits in lockstep; a frozen or finished orbit takes
// steps of size 0 (its state is not written) until every orbit of the block is
// done.
#include "fput_ens.cuh"
#include "seed.cuh"

namespace chs {
namespace {

// Set-up, one thread per orbit: x <- ics, H0, status, counters; vector j is
// w_in's (normalised with renorm) or seeded: component c is the m-th output of
// the SplitMix64 stream of `seed`, m = (o k + j) 2N + c + 1, mapped to [-1, 1)
// and normalised (once more with renorm).  Sums of squares run in index order
// without contraction.  The vectors are formed in place in e.w.
__global__ void __launch_bounds__(128)
k_fput_ens_init(const SysPar sp, const int K, const int renorm, const uint64_t seed,
                const double* __restrict__ ics, const int32_t* __restrict__ ic_status,
                const double* __restrict__ w_in, const EnsPtrs e)
{
    const int N = sp.n_dof, D = 2 * N;
    const int64_t n = e.n;
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    bool finite = true;
    for (int c = 0; c < D; ++c) {
        const double v = ics[c * n + o];
        e.x[c * n + o] = v;
        finite = finite && isfinite(v);
    }
    int32_t st = ic_status ? ic_status[o] : CHS_ORBIT_OK;
    if (st == CHS_ORBIT_OK && !finite) st = CHS_ORBIT_NONFINITE;
    double T = 0.0, V = 0.0;
    for (int i = 0; i < N; ++i) {
        const double p = ics[(N + i) * n + o];
        T += 0.5 * p * p;
    }
    for (int b = 0; b <= N; ++b) {
        const double qa = b < N ? ics[b * n + o] : 0.0;
        const double qb = b > 0 ? ics[(b - 1) * n + o] : 0.0;
        V += fe::bond_v(sp, qa - qb);
    }
    e.status[o] = st;
    e.h0[o] = (st == CHS_ORBIT_OK) ? T + V : __longlong_as_double(0x7ff8000000000000LL);
    e.dh_max[o] = 0.0;
    e.n_exec[o] = 0;
    if (e.ld) e.ld[o] = 0.0;
    double* w = static_cast<double*>(e.w);
    for (int j = 0; j < K; ++j) {
        double* wj = w + (int64_t)j * D * n + o;
        double acc = 0.0;
        for (int c = 0; c < D; ++c) {
            double v;
            if (w_in) {
                v = w_in[((int64_t)j * D + c) * n + o];
            } else {
                v = seed_uniform(seed, ((uint64_t)o * K + j) * D + c + 1);
            }
            wj[c * n] = v;
            acc = __dadd_rn(acc, __dmul_rn(v, v));
        }
        for (int pass = w_in ? 1 : 0; pass < 1 + renorm; ++pass) {
            const double nr = __dsqrt_rn(acc);
            acc = 0.0;
            for (int c = 0; c < D; ++c) {
                const double v = __ddiv_rn(wj[c * n], nr);
                wj[c * n] = v;
                acc = __dadd_rn(acc, __dmul_rn(v, v));
            }
        }
    }
}

// Fixed steps of size a.dt with the tableau Tab.
template <int N, class Tab>
__global__ void __launch_bounds__(128)
k_fput_ens(const StepArgs a, const SysPar sp, const int K, const EnsPtrs e)
{
    using C = fe::Cfg<N, Tab>;
    constexpr int D = C::D, G = C::G, PER = C::PER, WS = C::WS;
    __shared__ double smem[G * PER];
    const int g = threadIdx.x / D, l = threadIdx.x % D;
    const int64_t n = e.n;
    const int64_t o = (int64_t)blockIdx.x * G + g;
    const bool valid = o < n;
    double* slab = smem + g * PER;
    double* wg = static_cast<double*>(e.w);
    const fs::Coef fc = fs::coef_of(sp);

    int32_t st = valid ? e.status[o] : CHS_ORBIT_FORBIDDEN;
    const bool runs = st == CHS_ORBIT_OK;
    int64_t todo = 0;
    if (runs) {
        todo = a.n_steps;
        if (e.t_end) {
            const int64_t rem = e.t_end[o] - e.n_exec[o];
            if (rem < todo) todo = rem > 0 ? rem : 0;
        }
    }
    double xi = valid ? e.x[(int64_t)l * n + o] : 0.0;
    for (int j = 0; j < K; ++j) slab[C::W + j * WS + l] = valid ? wg[((int64_t)j * D + l) * n + o] : 0.0;
    const double h0 = runs ? e.h0[o] : 0.0;
    double dhm = runs ? e.dh_max[o] : 0.0;
    int64_t done = 0;
    bool active = runs && todo > 0;
    const long long t_start = clock64();

    for (int64_t it = 1;; ++it) {
        if (!__syncthreads_or(active)) break;
        const double ho = active ? a.dt : 0.0;
        double e5, e3;
        const double xn = fs::orbit_stages<N, Tab, false>(xi, ho, l, slab + C::XB, slab + C::CS, fc, e5, e3);
        if (l == 0) slab[C::CTL] = ho;
        __syncthreads();  // stage stiffnesses and phase-2 steps in place
        fs::columns<N, Tab, G, PER, WS, C::CS, true>(smem, K, [](int, const double* sl) { return sl[C::CTL]; },
                                               a.renorm);
        __syncthreads();  // columns complete; stage buffers free
        const bool stepped = active;
        if (stepped) {
            xi = xn;
            ++done;
        }
        const bool check = a.sample_every > 0 && (a.step0 + it) % a.sample_every == 0;
        st = fe::post_step<N, Tab>(a, sp, K, slab, l, xi, stepped, check, check, h0, dhm, st);
        if (check && a.clock_budget > 0) {  // block-uniform: the block's orbits stop together
            const bool over = __syncthreads_or(budget_spent(a, t_start)) != 0;
            if (over && stepped && st == CHS_ORBIT_OK) st = CHS_ORBIT_STEP_BUDGET;
        }
        active = stepped && st == CHS_ORBIT_OK && done < todo;
    }
    if (runs) {
        e.x[(int64_t)l * n + o] = xi;
        for (int j = 0; j < K; ++j) wg[((int64_t)j * D + l) * n + o] = slab[C::W + j * WS + l];
        if (l == 0) {
            e.dh_max[o] = dhm;
            e.n_exec[o] += done;
            e.status[o] = st;
        }
    }
}

// SALI, GALI_2..K (prod R_jj of a modified Gram-Schmidt QR of the unit
// vectors) and labels, one warp per orbit; lane c holds components c + 32 m.
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__global__ void __launch_bounds__(128)
k_fput_ens_indicators(const int D, const int K, const int64_t n, const double* __restrict__ wg,
                      const int32_t* __restrict__ status, const double thr, double* __restrict__ sali,
                      double* __restrict__ gali, int8_t* __restrict__ label)
{
    constexpr int M = 4;  // components per lane (D <= 128)
    const int lane = threadIdx.x % 32;
    const int64_t o = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (o >= n) return;  // the whole warp leaves together
    const int32_t st = status[o];
    const double qnan = __longlong_as_double(0x7ff8000000000000LL);
    double A[kMaxDev][M];
#pragma unroll
    for (int j = 0; j < kMaxDev; ++j) {
        if (j >= K) break;
        double n2 = 0.0;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int c = lane + 32 * m;
            A[j][m] = c < D ? wg[((int64_t)j * D + c) * n + o] : 0.0;
            n2 = fma(A[j][m], A[j][m], n2);
        }
        const double inv = 1.0 / sqrt(warp_sum(n2));
#pragma unroll
        for (int m = 0; m < M; ++m) A[j][m] *= inv;
    }
    double sv = qnan;
    if (K >= 2 && st != CHS_ORBIT_FORBIDDEN) {
        double a2 = 0.0, b2 = 0.0;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const double sp = A[0][m] + A[1][m], sm = A[0][m] - A[1][m];
            a2 = fma(sp, sp, a2);
            b2 = fma(sm, sm, b2);
        }
        sv = sqrt(fmin(warp_sum(a2), warp_sum(b2)));
    }
    if (sali && lane == 0) sali[o] = sv;
    if (gali && K >= 2) {
        double prod = 1.0;
#pragma unroll
        for (int j = 0; j < kMaxDev; ++j) {
            if (j >= K) break;
#pragma unroll
            for (int i = 0; i < j; ++i) {
                double r = 0.0;
#pragma unroll
                for (int m = 0; m < M; ++m) r = fma(A[i][m], A[j][m], r);
                r = warp_sum(r);
#pragma unroll
                for (int m = 0; m < M; ++m) A[j][m] = fma(-r, A[i][m], A[j][m]);
            }
            double n2 = 0.0;
#pragma unroll
            for (int m = 0; m < M; ++m) n2 = fma(A[j][m], A[j][m], n2);
            const double rjj = sqrt(warp_sum(n2));
            prod *= rjj;
            if (rjj > 0.0) {
                const double inv = 1.0 / rjj;
#pragma unroll
                for (int m = 0; m < M; ++m) A[j][m] *= inv;
            }
            if (j >= 1 && lane == 0) gali[(int64_t)(j - 1) * n + o] = (st == CHS_ORBIT_FORBIDDEN) ? qnan : prod;
        }
    }
    if (label && lane == 0) {
        int8_t lb;
        if (st == CHS_ORBIT_OK)
            lb = (sv < thr) ? 1 : 0;
        else if (st == CHS_ORBIT_EARLY_CHAOTIC)
            lb = 1;
        else if (st == CHS_ORBIT_PREDICTED_REGULAR)
            lb = 0;
        else if (st == CHS_ORBIT_ESCAPED)
            lb = 2;
        else
            lb = -1;
        label[o] = lb;
    }
}

template <int N, class Tab>
cudaError_t ens_n(const SysPar& sp, int k, const StepArgs& a, const EnsPtrs& e, cudaStream_t st)
{
    using C = fe::Cfg<N, Tab>;
    k_fput_ens<N, Tab><<<blocks_for(e.n, C::G), C::THREADS, 0, st>>>(a, sp, k, e);
    return cudaGetLastError();
}

template <class Tab>
cudaError_t ens_tab(const SysPar& sp, int k, const StepArgs& a, const EnsPtrs& e, cudaStream_t st)
{
    switch (sp.n_dof) {
    case 4: return ens_n<4, Tab>(sp, k, a, e, st);
    case 8: return ens_n<8, Tab>(sp, k, a, e, st);
    case 16: return ens_n<16, Tab>(sp, k, a, e, st);
    case 32: return ens_n<32, Tab>(sp, k, a, e, st);
    case 64: return ens_n<64, Tab>(sp, k, a, e, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

bool fput_ens_supported(int n_dof)
{
    return n_dof == 4 || n_dof == 8 || n_dof == 16 || n_dof == 32 || n_dof == 64;
}

cudaError_t launch_fput_ens_init(const SysPar& sp, int k, int renorm, uint64_t seed, const double* ics,
                                 const int32_t* ic_status, const void* w_in, const EnsPtrs& e,
                                 cudaStream_t st)
{
    if (e.n == 0) return cudaSuccess;
    k_fput_ens_init<<<blocks_for(e.n, 128), 128, 0, st>>>(sp, k, renorm, seed, ics, ic_status,
                                                          static_cast<const double*>(w_in), e);
    return cudaGetLastError();
}

cudaError_t launch_fput_ens(const SysPar& sp, int integrator, int k, const StepArgs& a, const EnsPtrs& e,
                            cudaStream_t st)
{
    if (e.n == 0 || a.n_steps == 0) return cudaSuccess;
    if (integrator == CHS_DOP853) return ens_tab<fs::TabDop853>(sp, k, a, e, st);
    return ens_tab<fs::TabRk4>(sp, k, a, e, st);
}

cudaError_t launch_fput_ens_indicators(const SysPar& sp, int k, double thr, const EnsPtrs& e, double* sali,
                                       double* gali, int8_t* label, cudaStream_t st)
{
    if (e.n == 0) return cudaSuccess;
    k_fput_ens_indicators<<<blocks_for(e.n, 4), 128, 0, st>>>(2 * sp.n_dof, k, e.n,
                                                               static_cast<const double*>(e.w), e.status,
                                                               thr, sali, gali, label);
    return cudaGetLastError();
}

}  // namespace chs

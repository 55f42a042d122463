// chs_static.cu -- the compacted chunk runner without caller-provided scratch.
//
// chs_integrate_compacted needs a device work buffer for its two orbit lists and
// their counters.  Some callers cannot provide one: their device memory is owned
// by another allocator (a framework's caching allocator, a fixed arena sized at
// start-up) that does not hand out extra buffers, or their rules forbid any
// device allocation once the application is running.  chs_integrate_compacted_static
// serves them: the lists live in a file-scope device array of fixed size, which
// every GPU that loads this library holds until the process exits, and the call
// allocates nothing.
#include <cuda.h>  // CUcontext and CUresult (types only: the driver call comes from the runtime)
#include <stdio.h>

#include <mutex>

#include "chs_internal.cuh"
#include "nvtx_range.cuh"

namespace {

// Largest ensemble the static scratch serves: the 1024 x 1024 grid.
constexpr int64_t kStaticMaxOrbits = 1 << 20;
// Two orbit lists of kStaticMaxOrbits entries, then two counters (padded to 256 B).
constexpr int64_t kStaticWords = 2 * kStaticMaxOrbits + 64;

static __device__ __align__(256) int32_t g_compact_scratch[kStaticWords];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
int32_t* g_scratch_ptr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};  // the context each cached address belongs to

using CtxGetCurrent = CUresult (*)(CUcontext*);

// The calling thread's current context, by the driver's cuCtxGetCurrent obtained
// through the runtime (no link against the driver library).  Call with
// g_scratch_mutex held.
cudaError_t current_context(CUcontext* ctx)
{
    static CtxGetCurrent fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !p) return cudaErrorSymbolNotFound;
        fn = reinterpret_cast<CtxGetCurrent>(p);
    }
    return fn(ctx) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

// Device address of the scratch array on `device` (which must be current).  The
// host-side symbol is only a stand-in; its device address comes from
// cudaGetSymbolAddress, once per device and context: a cudaDeviceReset, or a
// call from another context on the device, loads the module again and the array
// may move, so the address is looked up anew when the current context changes.
cudaError_t scratch_for(int device, int32_t** out)
{
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    CUcontext ctx = nullptr;
    cudaError_t e = current_context(&ctx);
    if (e != cudaSuccess) return e;
    if (!g_scratch_ptr[device] || g_scratch_ctx[device] != ctx) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_compact_scratch);
        if (e != cudaSuccess) return e;
        // the lookup may have created the primary context: key the cache on the
        // context that is current now
        if ((e = current_context(&ctx)) != cudaSuccess) return e;
        g_scratch_ptr[device] = static_cast<int32_t*>(p);
        g_scratch_ctx[device] = ctx;
    }
    *out = g_scratch_ptr[device];
    return cudaSuccess;
}

thread_local char g_static_err[256];

}  // namespace

// Defined in chs_api.cu: shared validation and message plumbing.
namespace chs {
chs_status api_validate_run(chs_system s, const chs_params* p, const chs_ensemble* e, int* device);
chs_status api_fail(chs_status code, const char* msg);
StepArgs api_step_args(const chs_params* p);
EnsPtrs api_ens_ptrs(const chs_ensemble* e);
SysPar api_syspar(chs_system s);
cudaError_t api_launch_integrate(const SysPar& sp, const chs_params* p, const StepArgs& a,
                                 const EnsPtrs& ep, const OrbitList* ol, cudaStream_t st);
}  // namespace chs

extern "C" chs_status chs_integrate_compacted_static(chs_system s, const chs_params* p,
                                                     const chs_ensemble* e, int32_t chunk_steps,
                                                     void* stream)
{
    CHS_NVTX_RANGE();
    int device = -1;
    chs_status r = chs::api_validate_run(s, p, e, &device);
    if (r != CHS_OK) return r;
    if (chunk_steps < 1) return chs::api_fail(CHS_E_INVALID, "chunk_steps must be >= 1");
    // the same bound on the chunk count as chs_integrate_compacted
    if ((p->n_steps + chunk_steps - 1) / chunk_steps > 100000)
        return chs::api_fail(CHS_E_SIZE, "more than 100000 chunks: raise chunk_steps");
    if (e->n_orbits > kStaticMaxOrbits) {
        snprintf(g_static_err, sizeof g_static_err,
                 "chs_integrate_compacted_static serves at most %lld orbits (got %lld): use "
                 "chs_integrate_compacted with a caller work buffer",
                 (long long)kStaticMaxOrbits, (long long)e->n_orbits);
        return chs::api_fail(CHS_E_SIZE, g_static_err);
    }
    if (e->n_orbits == 0 || p->n_steps == 0) return CHS_OK;
    int32_t* base = nullptr;
    cudaError_t ce = scratch_for(device, &base);
    if (ce != cudaSuccess) {
        snprintf(g_static_err, sizeof g_static_err, "cudaGetSymbolAddress of the static scratch: %s",
                 cudaGetErrorString(ce));
        return chs::api_fail(CHS_E_CUDA, g_static_err);
    }
    int32_t* la = base;
    int32_t* lb = base + kStaticMaxOrbits;
    int32_t* ca = base + 2 * kStaticMaxOrbits;
    int32_t* cb = ca + 1;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const chs::EnsPtrs ep = chs::api_ens_ptrs(e);
    const chs::SysPar sp = chs::api_syspar(s);
    // the counters keep the previous call's values: clear them before use
    ce = cudaMemsetAsync(ca, 0, sizeof(int32_t), st);
    if (ce == cudaSuccess) ce = chs::launch_list_init(ep, la, ca, st);
    const int64_t n_chunks = (p->n_steps + chunk_steps - 1) / chunk_steps;
    for (int64_t c = 0; c < n_chunks && ce == cudaSuccess; ++c) {
        chs::StepArgs a = chs::api_step_args(p);
        a.step0 = p->step0 + c * chunk_steps;
        a.n_steps = (p->n_steps - c * chunk_steps < chunk_steps) ? p->n_steps - c * chunk_steps : chunk_steps;
        ce = cudaMemsetAsync(cb, 0, sizeof(int32_t), st);
        const chs::OrbitList ol{la, ca, lb, cb, nullptr};
        if (ce == cudaSuccess)
            ce = chs::api_launch_integrate(sp, p, a, ep, &ol, st);
        int32_t* t = la;
        la = lb;
        lb = t;
        t = ca;
        ca = cb;
        cb = t;
    }
    if (ce != cudaSuccess) {
        snprintf(g_static_err, sizeof g_static_err, "compacted static launch: %s", cudaGetErrorString(ce));
        return chs::api_fail(CHS_E_CUDA, g_static_err);
    }
    return CHS_OK;
}

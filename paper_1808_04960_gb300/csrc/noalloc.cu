// Allocation-free variant of the SSP-RK3 step.
//
// gpweno_rk3_step needs a caller-provided scratch buffer of four state sizes
// for the intermediate stages and the compensation remainder.  Some callers cannot provide one: code that
// runs where it may not call cudaMalloc (an application whose device memory is
// owned by its own pool or caching allocator and which forbids allocations
// behind its back, or a plug-in whose host application gives it only the
// state buffer).  gpweno_rk3_step_noalloc serves them: its three stage buffers
// live in a fixed-size array in device global memory that is part of this
// library's image, so the call allocates nothing.
//
// Costs and limits of that choice:
//   - every GPU that loads the library holds the array (kStaticScratchBytes)
//     until the process exits;
//   - a grid fits only if three copies of its state fit in the array;
//   - unlike gpweno_rk3_step, no compensation remainder is carried from one
//     call to the next (there is nowhere private to keep it), so long FP32
//     runs accumulate state rounding as an uncompensated sum would;
//   - every call shares the one array per device, so two calls whose kernels
//     overlap on the GPU (different streams, or different host threads on the
//     same device) race and corrupt each other's stages;
//   - the first call on a device (and the first after that device's primary
//     context was torn down, e.g. by cudaDeviceReset) looks up the array's
//     device address (cudaGetSymbolAddress) with that device current; make
//     that first call before any stream capture begins.
#include <cuda.h>

#include <cstdint>
#include <mutex>

#include "plan.h"
#include "trace.h"

namespace gpweno {
namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;   // 16 MiB per device
constexpr int kMaxDevices = 64;

// The scratch itself.  In host code this name is only a stand-in for the
// device symbol: its device address must come from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mutex;
// Per device: the context the address was looked up in, and the address.  An
// address belongs to one context: after the device's primary context is torn
// down (cudaDeviceReset) and re-created, the array has a new address, so the
// cache is keyed on the current context as well as the device.
CUcontext g_scratch_ctx[kMaxDevices] = {};
void *g_scratch_addr[kMaxDevices] = {};

// The driver's cuCtxGetCurrent through the runtime (no link against libcuda).
using CtxGetCurrentFn = CUresult (*)(CUcontext *);

gpweno_status current_context(CUcontext *ctx)
{
    static CtxGetCurrentFn fn = nullptr;
    if (!fn) {
        void *sym = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &sym, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !sym)
            return cuda_fail(e == cudaSuccess ? cudaErrorSymbolNotFound : e,
                             "gpweno_rk3_step_noalloc: driver entry point cuCtxGetCurrent");
        fn = reinterpret_cast<CtxGetCurrentFn>(sym);
    }
    *ctx = nullptr;
    if (fn(ctx) != CUDA_SUCCESS || !*ctx) {
        set_error("gpweno_rk3_step_noalloc: no current CUDA context");
        return GPWENO_ERR_CUDA;
    }
    return GPWENO_OK;
}

// Device address of the array on the current device, looked up once per
// device and context.
gpweno_status static_scratch_address(int device, void **out)
{
    if (device < 0 || device >= kMaxDevices) {
        set_error("gpweno_rk3_step_noalloc: device %d out of range", device);
        return GPWENO_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    CUcontext ctx = nullptr;
    gpweno_status s = current_context(&ctx);
    if (s != GPWENO_OK) return s;
    if (!g_scratch_addr[device] || g_scratch_ctx[device] != ctx) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || ptr == nullptr)
            return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                             "gpweno_rk3_step_noalloc: cudaGetSymbolAddress of the static scratch");
        g_scratch_addr[device] = ptr;
        g_scratch_ctx[device] = ctx;
    }
    *out = g_scratch_addr[device];
    return GPWENO_OK;
}

}  // namespace
}  // namespace gpweno

using namespace gpweno;

extern "C" gpweno_status gpweno_rk3_step_noalloc(gpweno_plan p, void *U, double dt, void *stream)
{
    TraceRange tr("gpweno_rk3_step_noalloc");
    reset_launch_count();
    if (!p || p->is_batch || !U) {
        set_error("gpweno_rk3_step_noalloc: invalid argument");
        return GPWENO_ERR_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(U) & 15u) != 0) {
        set_error("gpweno_rk3_step_noalloc: U must be 16-byte aligned");
        return GPWENO_ERR_ARG;
    }
    if (has_external_side(p)) {
        set_error("gpweno_rk3_step_noalloc: plans with external sides step stage by stage (gpweno_rk3_stage)");
        return GPWENO_ERR_ARG;
    }
    if (!(dt > 0.0)) {
        set_error("gpweno_rk3_step_noalloc: dt=%g must be positive", dt);
        return GPWENO_ERR_ARG;
    }
    const size_t esz = p->opts.dtype == GPWENO_F32 ? 4 : 8;
    const size_t bytes = esz * (size_t)(p->dims.ndim + 2) * (size_t)p->ncell;
    const size_t stride = (bytes + 255) & ~size_t(255);
    if (3 * stride > kStaticScratchBytes) {
        set_error("gpweno_rk3_step_noalloc: the grid needs 3 x %zu bytes of stage storage, more than the %zu-byte "
                  "static scratch; use gpweno_rk3_step with a caller-provided scratch buffer",
                  stride, kStaticScratchBytes);
        return GPWENO_ERR_ARG;
    }
    int device = -1;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return cuda_fail(e, "gpweno_rk3_step_noalloc: cudaGetDevice");
    if (device != p->device) {
        set_error("gpweno_rk3_step_noalloc: plan belongs to device %d but device %d is current", p->device, device);
        return GPWENO_ERR_ARG;
    }
    void *base = nullptr;
    gpweno_status s = static_scratch_address(device, &base);
    if (s != GPWENO_OK) return s;
    char *s0 = static_cast<char *>(base);
    // nothing in the array needs to start at zero: each stage overwrites its buffers
    // completely, and no compensation remainder is carried between calls
    return rk3_sequence(p, U, s0, s0 + stride, s0 + 2 * stride, nullptr, dt, nullptr, false,
                        static_cast<cudaStream_t>(stream));
}

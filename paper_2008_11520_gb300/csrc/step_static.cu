// dnnmg_step_static: the correction step with its scratch in a fixed,
// library-owned device array instead of a caller-provided workspace.
//
// For callers that cannot allocate device memory themselves: a host program
// whose device memory is owned by another allocator it may not bypass, a
// loop that must not call into the CUDA allocator once it runs, or a plain C
// caller that links only this library and has no allocator of its own.
// Such a caller still passes its own inputs and outputs (x_c, h, b_f, b_c);
// only the step's scratch (features X, predictions d, corrected velocity)
// lives in the array below.
//
// The array is a file-scope __device__ object of kStaticScratchBytes bytes:
// every GPU on which the library is loaded holds it until the process exits.
// In host code its name is only a host-side stand-in, never a device
// address, so the device address is looked up with cudaGetSymbolAddress once
// per device and context (on the first call made with that device current)
// and cached.  The cache is keyed on the current CUDA context, not only on the
// device number, and a cached address is checked before use: after a
// cudaDeviceReset, or for a second context on the same device, the array has
// a new address and is looked up again.
#include <cuda.h>

#include <mutex>
#include <vector>

#include "common.cuh"

namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;   // 64 MiB

static __device__ __align__(256) unsigned char g_step_scratch[kStaticScratchBytes];

struct ScratchSlot {
    int device;
    CUcontext ctx;
    void *ptr;
};

std::mutex g_scratch_mu;
std::vector<ScratchSlot> g_scratch_slots;

// The calling thread's current context (the driver call is reached through the
// runtime's entry-point query, so the library needs no link against libcuda).
int current_context(CUcontext *ctx) {
    using Fn = CUresult (*)(CUcontext *);
    static Fn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<Fn>(p);
    });
    if (!fn) return dnnmg::fail(DNNMG_ECUDA, "the driver entry point cuCtxGetCurrent is unavailable");
    if (fn(ctx) != CUDA_SUCCESS) return dnnmg::fail(DNNMG_ECUDA, "cuCtxGetCurrent failed");
    return DNNMG_OK;
}

// True if p is still device memory of `device` in the current context.
bool still_valid(void *p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

// Device address of the scratch array in the current context (set up once
// per device and context, with that device current).
int scratch_address(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return dnnmg::fail(DNNMG_ECUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
    CUcontext ctx = nullptr;
    if (int r = current_context(&ctx)) return r;
    if (!ctx) return dnnmg::fail(DNNMG_EINVAL, "no CUDA context is current on this thread");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    for (ScratchSlot &s : g_scratch_slots) {
        if (s.device != dev || s.ctx != ctx) continue;
        if (!still_valid(s.ptr, dev)) break;   // stale (a reset reused the handle): look it up again
        *out = s.ptr;
        return DNNMG_OK;
    }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_step_scratch);
    if (e != cudaSuccess || !p)
        return dnnmg::fail(DNNMG_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
    bool stored = false;
    for (ScratchSlot &s : g_scratch_slots)
        if (s.device == dev && s.ctx == ctx) {
            s.ptr = p;
            stored = true;
        }
    if (!stored) g_scratch_slots.push_back({dev, ctx, p});
    *out = p;
    return DNNMG_OK;
}

}  // namespace

extern "C" {

size_t dnnmg_static_scratch_bytes(void) { return kStaticScratchBytes; }

int dnnmg_step_static(dnnmg_mesh_t mesh, dnnmg_net_t net, const double *xc, void *h, void *bf, double *bc,
                      double t, cudaStream_t stream) {
    dnnmg::clear_error();
    if (!mesh) return dnnmg::fail(DNNMG_EINVAL, "mesh handle is NULL");
    dnnmg_mesh_info info;
    if (int e = dnnmg_mesh_get_info(mesh, &info)) return e;
    const size_t need = dnnmg::step_scratch_bytes(info);
    if (need > kStaticScratchBytes)
        return dnnmg::fail(DNNMG_EINVAL,
                           "this mesh needs %zu bytes of step scratch but the static scratch holds %zu; "
                           "use dnnmg_step with a caller-provided workspace",
                           need, kStaticScratchBytes);
    void *scratch = nullptr;
    if (int e = scratch_address(&scratch)) return e;
    // Every scratch element the step reads is written earlier in the same
    // step, so nothing has to be cleared between calls.
    return dnnmg::step_on_workspace(mesh, net, xc, h, bf, bc, scratch, kStaticScratchBytes, t, stream);
}

size_t dnnmg_static_scratch_needed(dnnmg_mesh_t mesh) {
    dnnmg_mesh_info info;
    if (!mesh || dnnmg_mesh_get_info(mesh, &info)) return 0;
    return dnnmg::step_scratch_bytes(info);
}

}  // extern "C"

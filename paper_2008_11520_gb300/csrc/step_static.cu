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
// per device (on the first call made with that device current) and cached.
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;   // 64 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_step_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once per device).
int scratch_address(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return dnnmg::fail(DNNMG_ECUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return dnnmg::fail(DNNMG_EUNSUPPORTED, "device %d: at most %d devices", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_step_scratch);
        if (e != cudaSuccess || !p)
            return dnnmg::fail(DNNMG_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
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
    if (info.workspace_bytes > kStaticScratchBytes)
        return dnnmg::fail(DNNMG_EINVAL,
                           "this mesh needs %zu bytes of step scratch but the static scratch holds %zu; "
                           "use dnnmg_step with a caller-provided workspace",
                           info.workspace_bytes, kStaticScratchBytes);
    void *scratch = nullptr;
    if (int e = scratch_address(&scratch)) return e;
    // Every scratch element the step reads is written earlier in the same
    // step, so nothing has to be cleared between calls.
    return dnnmg::step_on_workspace(mesh, net, xc, h, bf, bc, scratch, kStaticScratchBytes, t, stream);
}

}  // extern "C"

// Self-test of the bounded waits every kernel of libdnnmg uses (TMA copies,
// tensor-core commits): a wait that nothing will ever satisfy must give up,
// report through the device status word, and make the other waiters of its
// CTA leave too, with the context still usable.  No copy or MMA is attached
// to the barrier, so nothing is left in flight.
#include "common.cuh"
#include "ptx.cuh"

namespace dnnmg {
namespace {

// Thread 0 waits with the short limit; the other threads of the block wait
// with the default limit and must leave through the abort flag instead.
__global__ void k_wait_selftest(unsigned long long limit_ns, int *status, unsigned long long *waited_ns) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    const uint32_t b = ptx::smem_u32(&bar);
    if (threadIdx.x == 0) {
        ptx::mbar_init(b, 1);   // one arrival expected, none will come
        abort_flag = 0;
        ptx::mbar_init_fence();
    }
    __syncthreads();
    const unsigned long long t0 = ptx::now_ns();
    const bool ok = threadIdx.x == 0 ? ptx::mbar_wait(b, 0, &abort_flag, limit_ns) : ptx::mbar_wait(b, 0, &abort_flag);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!ok) atomicOr(status, DNNMG_DEVERR_TIMEOUT);
        waited_ns[0] = ptx::now_ns() - t0;
    }
    if (!ok && threadIdx.x == blockDim.x - 1) waited_ns[1] = ptx::now_ns() - t0;
}

}  // namespace
}  // namespace dnnmg

using namespace dnnmg;

extern "C" int dnnmg_selftest_wait_timeout(long long limit_ns, int *status, long long *waited_ns) {
    clear_error();
    if (!status || !waited_ns || limit_ns < 1 || limit_ns > 1000000000LL)
        return fail(DNNMG_EINVAL, "status/waited_ns NULL or limit outside 1 ns .. 1 s");
    int *d_status = nullptr;
    unsigned long long *d_waited = nullptr;
    DNNMG_CUDA_TRY(cudaMalloc(&d_status, sizeof(int)));
    cudaError_t e = cudaMalloc(&d_waited, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(d_waited, 0, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 64>>>((unsigned long long)limit_ns, d_status, d_waited);
        e = cudaGetLastError();
    }
    unsigned long long w[2] = {0, 0};
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(status, d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(w, d_waited, sizeof w, cudaMemcpyDeviceToHost);
    cudaFree(d_status);
    cudaFree(d_waited);
    if (e != cudaSuccess) return fail(DNNMG_ECUDA, "wait self-test: %s", cudaGetErrorString(e));
    waited_ns[0] = (long long)w[0];
    waited_ns[1] = (long long)w[1];
    return DNNMG_OK;
}

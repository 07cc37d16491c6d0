// S4 on CUDA cores: GRU cell (Eq. gru, reset gate before U_h, no biases) and
// the fully connected output layer, TP patches per CTA.
//
// Weights are stored transposed (WxT [ldx][3H], UhT [H][3H], WfcT [H][n_out])
// so that consecutive threads, which own consecutive output rows, read
// consecutive addresses; the CTA's patch rows sit in shared memory and are
// read as broadcasts.  Precisions:
//   F64      double operands, double accumulation
//   F32      float operands, float accumulation
//   BF16NET  bfloat16 GEMM operands (X, weights, h, r*h and h' rounded to
//            bfloat16), float accumulation and float gate arithmetic; the
//            stored state h stays float.  This is the same arithmetic as the
//            tensor-core kernel, so the two can be compared tightly.
#include "common.cuh"

namespace dnnmg {
namespace {

template <typename TW> struct Acc { using type = TW; };
template <> struct Acc<__nv_bfloat16> { using type = float; };

template <typename A> __device__ __forceinline__ A load_as(const __nv_bfloat16 *p) {
    return (A)__bfloat162float(*p);
}
template <typename A> __device__ __forceinline__ A load_as(const float *p) { return (A)*p; }
template <typename A> __device__ __forceinline__ A load_as(const double *p) { return (A)*p; }

// value of x as the GEMM operand type sees it
template <typename TW, typename A> __device__ __forceinline__ A quant(A x) { return x; }
template <> __device__ __forceinline__ float quant<__nv_bfloat16, float>(float x) {
    return __bfloat162float(__float2bfloat16_rn(x));
}

__device__ __forceinline__ double sigm(double x) { return 1.0 / (1.0 + exp(-x)); }
__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + expf(-x)); }
__device__ __forceinline__ double tanh_(double x) { return tanh(x); }
__device__ __forceinline__ float tanh_(float x) { return tanhf(x); }

constexpr int NT = 256;

template <typename T, typename TW, int TP>
__global__ void __launch_bounds__(NT)
k_gru(int n_in, int ldx, int H, int n_out, const TW *__restrict__ X, const TW *__restrict__ WxT,
      const TW *__restrict__ UhT, const TW *__restrict__ WfcT, T *__restrict__ h,
      T *__restrict__ d, int P) {
    using A = typename Acc<TW>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    A *xs = reinterpret_cast<A *>(smem_raw);  // [TP][ldx]  features
    A *hs = xs + TP * ldx;                    // [TP][H]    previous state (float / double)
    A *hq = hs + TP * H;                      // [TP][H]    previous state as GEMM operand
    A *zs = hq + TP * H;                      // [TP][H]    update gate
    A *rh = zs + TP * H;                      // [TP][H]    r * h (operand)
    A *gh = rh + TP * H;                      // [TP][H]    W_h x
    A *hn = gh + TP * H;                      // [TP][H]    new state (operand)
    const int p0 = blockIdx.x * TP;
    const int np = min(TP, P - p0);
    const int G = 3 * H;

    for (int i = threadIdx.x; i < TP * ldx; i += blockDim.x) {
        const int p = i / ldx, k = i - p * ldx;
        xs[i] = (p < np && k < n_in) ? load_as<A>(X + (size_t)(p0 + p) * ldx + k) : A(0);
    }
    for (int i = threadIdx.x; i < TP * H; i += blockDim.x) {
        const int p = i / H;
        const A v = p < np ? (A)h[(size_t)p0 * H + i] : A(0);
        hs[i] = v;
        hq[i] = quant<TW, A>(v);
    }
    __syncthreads();

    // z, r and W_h x
    for (int j = threadIdx.x; j < G; j += blockDim.x) {
        A acc[TP];
#pragma unroll
        for (int p = 0; p < TP; ++p) acc[p] = A(0);
        for (int k = 0; k < n_in; ++k) {
            const A w = load_as<A>(WxT + (size_t)k * G + j);
#pragma unroll
            for (int p = 0; p < TP; ++p) acc[p] += w * xs[p * ldx + k];
        }
        if (j < 2 * H) {
            for (int k = 0; k < H; ++k) {
                const A w = load_as<A>(UhT + (size_t)k * G + j);
#pragma unroll
                for (int p = 0; p < TP; ++p) acc[p] += w * hq[p * H + k];
            }
        }
        if (j < H) {
#pragma unroll
            for (int p = 0; p < TP; ++p) zs[p * H + j] = sigm(acc[p]);
        } else if (j < 2 * H) {
#pragma unroll
            for (int p = 0; p < TP; ++p)
                rh[p * H + j - H] = quant<TW, A>(sigm(acc[p]) * hs[p * H + j - H]);
        } else {
#pragma unroll
            for (int p = 0; p < TP; ++p) gh[p * H + j - 2 * H] = acc[p];
        }
    }
    __syncthreads();

    // candidate and state update
    for (int j = threadIdx.x; j < H; j += blockDim.x) {
        A acc[TP];
#pragma unroll
        for (int p = 0; p < TP; ++p) acc[p] = gh[p * H + j];
        for (int k = 0; k < H; ++k) {
            const A w = load_as<A>(UhT + (size_t)k * G + 2 * H + j);
#pragma unroll
            for (int p = 0; p < TP; ++p) acc[p] += w * rh[p * H + k];
        }
#pragma unroll
        for (int p = 0; p < TP; ++p) {
            const A z = zs[p * H + j];
            const A hnew = z * hs[p * H + j] + (A(1) - z) * tanh_(acc[p]);
            hn[p * H + j] = quant<TW, A>(hnew);
            if (p < np) h[(size_t)(p0 + p) * H + j] = (T)hnew;
        }
    }
    __syncthreads();

    // output layer d = W_fc h'
    for (int o = threadIdx.x; o < n_out; o += blockDim.x) {
        A acc[TP];
#pragma unroll
        for (int p = 0; p < TP; ++p) acc[p] = A(0);
        for (int k = 0; k < H; ++k) {
            const A w = load_as<A>(WfcT + (size_t)k * n_out + o);
#pragma unroll
            for (int p = 0; p < TP; ++p) acc[p] += w * hn[p * H + k];
        }
#pragma unroll
        for (int p = 0; p < TP; ++p)
            if (p < np) d[(size_t)(p0 + p) * n_out + o] = (T)acc[p];
    }
}

template <typename T, typename TW, int TP>
cudaError_t run(const Net &n, const void *X, void *h, void *d, int P, cudaStream_t st) {
    using A = typename Acc<TW>::type;
    const size_t sm = sizeof(A) * ((size_t)TP * n.ldx + 6 * (size_t)TP * n.H);
    auto k = k_gru<T, TW, TP>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k<<<(P + TP - 1) / TP, NT, sm, st>>>(n.n_in, n.ldx, n.H, n.n_out, (const TW *)X,
                                         (const TW *)n.WxT, (const TW *)n.UhT, (const TW *)n.WfcT,
                                         (T *)h, (T *)d, P);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gru_cuda_core(const Net &n, const void *X, void *h, void *d, int P,
                                 cudaStream_t st) {
    if (P == 0) return cudaSuccess;
    if (n.precision == DNNMG_F64) return run<double, double, 8>(n, X, h, d, P, st);
    if (n.precision == DNNMG_F32) return run<float, float, 16>(n, X, h, d, P, st);
    return run<float, __nv_bfloat16, 16>(n, X, h, d, P, st);
}

}  // namespace dnnmg

// Training the patch network (Eq. gru + output layer, Sec. 6.2 and 6.3):
// the GRU unrolled over a window of T steps, and its gradient by truncated
// backpropagation through time, in FP32 on the CUDA cores.
//
// Every product of the network is a matrix product over the patch rows, so a
// window is a short sequence of GEMMs and fused pointwise kernels:
//   forward   GX = X W_x^T for all steps at once; per step t
//             GH = h_{t-1} [U_z; U_r]^T, gates (z, r, r*h), AH = (r*h) U_h^T,
//             candidate and new state; then D = H W_fc^T for all steps.
//   backward  dH = dD W_fc for all steps; per step t (last first) the gate
//             gradients and the carried state gradient; then each weight
//             gradient is one product over all steps and patches
//             (K = T P), split over K in a fixed order, so results repeat
//             bit for bit.
// The trainer handle owns the saved activations of one window.
#include <algorithm>
#include <cmath>
#include <new>

#include "common.cuh"

namespace dnnmg {
namespace {

// ---------------------------------------------------------------- GEMM
// C[M][N] (row stride ldc) = op(A) op(B), or += when accumulate.
//   TA false: A is [M][K] (lda);  TA true: A is stored [K][M] (lda).
//   TB false: B is [K][N] (ldb);  TB true: B is stored [N][K] (ldb).
// 128 x 64 tiles, K in steps of 16, 256 threads with 8 x 4 outputs each; the
// next K step is read into registers while the current one is multiplied
// out of the other half of a double buffer.  blockIdx.z takes K range
// [z kchunk, (z+1) kchunk) and writes its partial result to C + z cstride
// (split K; reduced by k_reduce_splits).
constexpr int GBM = 128, GBN = 64, GBK = 16, GTH = 256;
constexpr int GA = GBM * GBK / GTH, GB = GBN * GBK / GTH;   // elements each thread stages per step

template <bool TA, bool TB>
__global__ void __launch_bounds__(GTH) k_sgemm(int M, int N, int K, const float *__restrict__ A, int lda,
                                              const float *__restrict__ B, int ldb, float *__restrict__ C, int ldc,
                                              int accumulate, int kchunk, long long cstride) {
    __shared__ __align__(16) float As[2][GBK][GBM + 4];
    __shared__ __align__(16) float Bs[2][GBK][GBN + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    float ra[GA], rb[GB];
    // the (m, k) / (k, n) element each staged value belongs to (coalesced along
    // the stored fastest dimension)
    auto a_at = [&](int i, int &m, int &k) {
        const int idx = tid + i * GTH;
        if (TA) { k = idx / GBM; m = idx % GBM; }
        else    { m = idx / GBK; k = idx % GBK; }
    };
    auto b_at = [&](int i, int &n, int &k) {
        const int idx = tid + i * GTH;
        if (TB) { n = idx / GBK; k = idx % GBK; }
        else    { k = idx / GBN; n = idx % GBN; }
    };
    auto fetch = [&](int k0) {
#pragma unroll
        for (int i = 0; i < GA; ++i) {
            int m, k;
            a_at(i, m, k);
            const int gm = m0 + m, gk = k0 + k;
            ra[i] = (gm < M && gk < ke) ? (TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk]) : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < GB; ++i) {
            int n, k;
            b_at(i, n, k);
            const int gn = n0 + n, gk = k0 + k;
            rb[i] = (gn < N && gk < ke) ? (TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn]) : 0.0f;
        }
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int i = 0; i < GA; ++i) {
            int m, k;
            a_at(i, m, k);
            As[buf][k][m] = ra[i];
        }
#pragma unroll
        for (int i = 0; i < GB; ++i) {
            int n, k;
            b_at(i, n, k);
            Bs[buf][k][n] = rb[i];
        }
    };
    float acc[8][4] = {};
    int buf = 0;
    if (kb < ke) {
        fetch(kb);
        stash(0);
    }
    __syncthreads();
    for (int k0 = kb; k0 < ke; k0 += GBK) {
        const bool more = k0 + GBK < ke;
        if (more) fetch(k0 + GBK);
#pragma unroll
        for (int k = 0; k < GBK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * 8 + 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[buf][k][tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (more) stash(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
    float *Cz = C + (size_t)blockIdx.z * cstride;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int gm = m0 + ty * 8 + i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tx * 4 + j;
            if (gn >= N) continue;
            float *c = Cz + (size_t)gm * ldc + gn;
            *c = accumulate ? *c + acc[i][j] : acc[i][j];
        }
    }
}

// C[m][n] (=|+=) the sum over s = 0 .. splits-1, in that order, of part[s][m][n].
__global__ void k_reduce_splits(int M, int N, int splits, const float *__restrict__ part, float *__restrict__ C,
                                int ldc, int accumulate) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)M * N) return;
    const int m = (int)(e / N), n = (int)(e - (long long)m * N);
    float s = 0.0f;
    for (int z = 0; z < splits; ++z) s += part[(size_t)z * M * N + e];
    float *c = C + (size_t)m * ldc + n;
    *c = accumulate ? *c + s : s;
}

template <bool TA, bool TB>
cudaError_t gemm(int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C, int ldc,
                 bool accumulate, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    const dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM, 1);
    k_sgemm<TA, TB><<<grid, GTH, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, accumulate ? 1 : 0, K > 0 ? K : 1, 0);
    return cudaGetLastError();
}

// op(A) op(B) with K split into `splits` ranges; part holds splits x M x N floats.
template <bool TA, bool TB>
cudaError_t gemm_splitk(int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C, int ldc,
                        int splits, float *part, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    const int kchunk = ((K + splits - 1) / splits + GBK - 1) / GBK * GBK;
    const int sz = (K + kchunk - 1) / kchunk;
    const dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM, sz);
    k_sgemm<TA, TB><<<grid, GTH, 0, st>>>(M, N, K, A, lda, B, ldb, part, N, 0, kchunk, (long long)M * N);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long n = (long long)M * N;
    k_reduce_splits<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(M, N, sz, part, C, ldc, 0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- BF16 products
// K of a BF16 operand rounded up to whole 16-byte rows
inline int kpad(int K) { return (K + 7) / 8 * 8; }

// dst[i][k] (row stride ldd) = bf16(op(src)) for i < rows, k < K, where op(src)
// is src [rows][K] (row stride ld), or with TR its transpose, src [K][rows];
// 32 x 32 tiles through shared memory, so both sides move along rows.
template <bool TR>
__global__ void k_to_bf16(int rows, int K, const float *__restrict__ src, int ld, __nv_bfloat16 *__restrict__ dst,
                          int ldd) {
    __shared__ float tile[32][33];
    const int i0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
    if (TR) {
        for (int y = threadIdx.y; y < 32; y += 8) {
            const int k = k0 + y, i = i0 + threadIdx.x;
            tile[y][threadIdx.x] = (k < K && i < rows) ? src[(size_t)k * ld + i] : 0.f;
        }
        __syncthreads();
        for (int y = threadIdx.y; y < 32; y += 8) {
            const int i = i0 + y, k = k0 + threadIdx.x;
            if (i < rows && k < K) dst[(size_t)i * ldd + k] = __float2bfloat16_rn(tile[threadIdx.x][y]);
        }
    } else {
        for (int y = threadIdx.y; y < 32; y += 8) {
            const int i = i0 + y, k = k0 + threadIdx.x;
            if (i < rows && k < K) dst[(size_t)i * ldd + k] = __float2bfloat16_rn(src[(size_t)i * ld + k]);
        }
    }
}

__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + expf(-x)); }

// ---------------------------------------------------------------- pointwise
// z, r and r * h_{t-1} from the input part GX [P][3H] and the recurrent part GH [P][2H].
__global__ void k_gates_fwd(int P, int H, const float *__restrict__ GX, const float *__restrict__ GH,
                            const float *__restrict__ hp, float *__restrict__ z, float *__restrict__ r,
                            float *__restrict__ rh) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)P * H) return;
    const int p = (int)(e / H), j = (int)(e - (long long)p * H);
    const float zz = sigm(GX[(size_t)p * 3 * H + j] + GH[(size_t)p * 2 * H + j]);
    const float rr = sigm(GX[(size_t)p * 3 * H + H + j] + GH[(size_t)p * 2 * H + H + j]);
    z[e] = zz;
    r[e] = rr;
    rh[e] = rr * hp[e];
}

// c = tanh(W_h x + U_h (r h)) and h_t = z h_{t-1} + (1 - z) c.
__global__ void k_cand_fwd(int P, int H, const float *__restrict__ GX, const float *__restrict__ AH,
                           const float *__restrict__ z, const float *__restrict__ hp, float *__restrict__ c,
                           float *__restrict__ h) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)P * H) return;
    const int p = (int)(e / H), j = (int)(e - (long long)p * H);
    const float cc = tanhf(GX[(size_t)p * 3 * H + 2 * H + j] + AH[e]);
    const float zz = z[e];
    c[e] = cc;
    h[e] = zz * hp[e] + (1.0f - zz) * cc;
}

// Backward through the state update of step t: dh = dHfc + carry is the
// gradient reaching h_t; writes the gradients of the z and candidate
// pre-activations into dG [P][3H] (columns 0..H-1 and 2H..3H-1) and keeps dh.
__global__ void k_bwd_state(int P, int H, const float *__restrict__ dHfc, const float *__restrict__ carry,
                            const float *__restrict__ z, const float *__restrict__ c, const float *__restrict__ hp,
                            float *__restrict__ dG, float *__restrict__ dh_out) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)P * H) return;
    const int p = (int)(e / H), j = (int)(e - (long long)p * H);
    const float dh = dHfc[e] + carry[e];
    const float zz = z[e], cc = c[e];
    const float dc = dh * (1.0f - zz);
    const float dz = dh * (hp[e] - cc);
    dG[(size_t)p * 3 * H + j] = dz * zz * (1.0f - zz);
    dG[(size_t)p * 3 * H + 2 * H + j] = dc * (1.0f - cc * cc);
    dh_out[e] = dh;
}

// Backward through the reset gate: drh = d(r h_{t-1}); the r pre-activation
// gradient into dG columns H..2H-1, and the part of the carried gradient that
// does not pass through U_z, U_r: dh z + drh r.
__global__ void k_bwd_reset(int P, int H, const float *__restrict__ drh, const float *__restrict__ hp,
                            const float *__restrict__ r, const float *__restrict__ z, const float *__restrict__ dh,
                            float *__restrict__ dG, float *__restrict__ carry) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)P * H) return;
    const int p = (int)(e / H), j = (int)(e - (long long)p * H);
    const float rr = r[e], g = drh[e];
    dG[(size_t)p * 3 * H + H + j] = g * hp[e] * rr * (1.0f - rr);
    carry[e] = dh[e] * z[e] + g * rr;
}

// ---------------------------------------------------------------- loss, Adam
// dD = 2 (D - Y) / P (FP32) and per-block partial sums of (D - Y)^2 / P,
// accumulated in FP64.
__global__ void k_l2_loss(long long n, int P, float two_over_p, const float *__restrict__ D,
                          const float *__restrict__ Y, float *__restrict__ dD, double *__restrict__ part) {
    __shared__ double red[256];
    double s = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float diff = D[e] - Y[e];
        if (dD) dD[e] = diff * two_over_p;
        s += (double)(diff * diff);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0] / P;
}

// Sum of squares of x, as per-block partials (FP64).
__global__ void k_sumsq(long long n, const float *__restrict__ x, double *__restrict__ part) {
    __shared__ double red[256];
    double s = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        s += (double)x[e] * x[e];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// out = sum of part[0 .. n-1] (n <= 512) by a fixed tree in one block of 256 threads.
__global__ void k_sum_parts(int n, const double *__restrict__ part, double *__restrict__ out) {
    __shared__ double red[256];
    const int t = threadIdx.x;
    red[t] = (t < n ? part[t] : 0.0) + (t + 256 < n ? part[t + 256] : 0.0);
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w) red[t] += red[t + w];
        __syncthreads();
    }
    if (t == 0) *out = red[0];
}

// Adam with the Tikhonov term: g' = g + 2 alpha p; bias corrections c1 = 1 - b1^s, c2 = 1 - b2^s.
__global__ void k_adam(long long n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float alpha, float c1,
                       float c2) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float pe = p[e];
    const float ge = g[e] + 2.0f * alpha * pe;
    const float me = b1 * m[e] + (1.0f - b1) * ge;
    const float ve = b2 * v[e] + (1.0f - b2) * ge * ge;
    m[e] = me;
    v[e] = ve;
    p[e] = pe - lr * (me / c1) / (sqrtf(ve / c2) + eps);
}

constexpr int kRedBlocks = 512;

unsigned blocks_for(long long n) { return (unsigned)((n + 255) / 256); }

}  // namespace
}  // namespace dnnmg

struct dnnmg_trainer_s {
    int n_in, ldx, H, n_out, T, P, device;
    // saved activations of the last forward window
    float *GX;      // [T P][3H]
    float *hs;      // [(T+1) P][H]: h_0 .. h_T
    float *z, *r, *rh, *c;   // [T P][H] each
    // scratch
    float *GH;      // [P][2H]
    float *AH;      // [P][H]
    float *dHfc;    // [T P][H]
    float *dG;      // [T P][3H]
    float *dh, *drh, *carry;   // [P][H]
    float *part;    // split-K partials
    size_t part_floats;
    double *red;    // reduction partials [kRedBlocks]
    int splits;
    // BF16 products (dnnmg_trainer_set_precision)
    int bf16;
    int *d_status;
    // BF16 copies, each tensor rounded once (offsets into arena, in elements;
    // row strides kx = kpad(n_in), kh = kpad(H), k2 = kpad(2H), ko = kpad(n_out),
    // kt = kpad(T P), ks = kpad((T+1) P))
    __nv_bfloat16 *arena;
    size_t arena_elems;
    int kx, kh, k2, ko, kt, ks;
    size_t o_Wx, o_U, o_Wfc, o_X, o_hs, o_rh;                        // forward
    size_t o_WfcT, o_UcT, o_UzrT, o_dD, o_dGc, o_dGzr;               // backward, per step
    size_t o_dGT, o_XT, o_hsT, o_rhT, o_dDT;                         // weight gradients
};

namespace dnnmg {
namespace {

// One FP32 product of the trainer, C (+)= op(A) op(B) in the layouts of gemm();
// split: K split over t->splits ranges, reduced in a fixed order.
template <bool TA, bool TB>
cudaError_t prod(dnnmg_trainer_s *t, int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C,
                 int ldc, bool accumulate, bool split, cudaStream_t st) {
    return split ? gemm_splitk<TA, TB>(M, N, K, A, lda, B, ldb, C, ldc, t->splits, t->part, st)
                 : gemm<TA, TB>(M, N, K, A, lda, B, ldb, C, ldc, accumulate, st);
}

// ---------------------------------------------------------------- BF16 mode
// Each tensor a product needs is rounded to BF16 once, into the trainer's
// arena (K contiguous), and the products run on the tensor cores.
inline __nv_bfloat16 *at(dnnmg_trainer_s *t, size_t off) { return t->arena + off; }

// dst [rows][K] (row stride ldd) = bf16(src) or, with tr, bf16(src^T) for src stored [K][rows].
cudaError_t to_bf16(int rows, int K, const float *src, int ld, bool tr, __nv_bfloat16 *dst, int ldd,
                    cudaStream_t st) {
    if (rows <= 0 || K <= 0) return cudaSuccess;
    const dim3 grid((K + 31) / 32, (rows + 31) / 32), blk(32, 8);
    if (tr) k_to_bf16<true><<<grid, blk, 0, st>>>(rows, K, src, ld, dst, ldd);
    else k_to_bf16<false><<<grid, blk, 0, st>>>(rows, K, src, ld, dst, ldd);
    return cudaGetLastError();
}

// C (+)= A B^T on the tensor cores; split: K over t->splits ranges, summed in a fixed order.
cudaError_t tc(dnnmg_trainer_s *t, int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B,
               int ldb, float *C, int ldc, bool accumulate, bool split, cudaStream_t st) {
    if (!split || t->splits <= 1)
        return launch_gemm_tc(M, N, K, A, lda, B, ldb, C, ldc, accumulate, 1, nullptr, t->d_status, st);
    cudaError_t e = launch_gemm_tc(M, N, K, A, lda, B, ldb, C, ldc, false, t->splits, t->part, t->d_status, st);
    if (e != cudaSuccess) return e;
    const long long n = (long long)M * N;
    k_reduce_splits<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(M, N, gemm_tc_splits_used(K, t->splits), t->part, C,
                                                                  ldc, 0);
    return cudaGetLastError();
}

// The window's forward with BF16 products; h_0 is already in t->hs.
cudaError_t seq_forward_bf16(dnnmg_trainer_s *t, const float *X, const float *Wx, const float *Uh, const float *Wfc,
                             float *D, cudaStream_t st) {
    const int H = t->H, P = t->P, T = t->T, n_in = t->n_in, n_out = t->n_out, TP = T * P;
    const int kx = t->kx, kh = t->kh;
    const size_t PH = (size_t)P * H;
    __nv_bfloat16 *Wxb = at(t, t->o_Wx), *Ub = at(t, t->o_U), *Wfcb = at(t, t->o_Wfc), *Xb = at(t, t->o_X);
    __nv_bfloat16 *hsb = at(t, t->o_hs), *rhb = at(t, t->o_rh);
    cudaError_t e;
#define TRY(x) if ((e = (x)) != cudaSuccess) return e
    TRY(to_bf16(3 * H, n_in, Wx, n_in, false, Wxb, kx, st));
    TRY(to_bf16(3 * H, H, Uh, H, false, Ub, kh, st));
    TRY(to_bf16(n_out, H, Wfc, H, false, Wfcb, kh, st));
    TRY(to_bf16(TP, n_in, X, t->ldx, false, Xb, kx, st));
    TRY(to_bf16(P, H, t->hs, H, false, hsb, kh, st));
    // input parts of every gate, all steps: GX = X W_x^T
    TRY(tc(t, TP, 3 * H, n_in, Xb, kx, Wxb, kx, t->GX, 3 * H, false, false, st));
    for (int s = 0; s < T; ++s) {
        const float *hp = t->hs + (size_t)s * PH;
        const float *GX = t->GX + (size_t)s * P * 3 * H;
        float *z = t->z + (size_t)s * PH, *r = t->r + (size_t)s * PH, *rh = t->rh + (size_t)s * PH;
        float *c = t->c + (size_t)s * PH, *h = t->hs + (size_t)(s + 1) * PH;
        TRY(tc(t, P, 2 * H, H, hsb + (size_t)s * P * kh, kh, Ub, kh, t->GH, 2 * H, false, false, st));
        k_gates_fwd<<<blocks_for((long long)PH), 256, 0, st>>>(P, H, GX, t->GH, hp, z, r, rh);
        TRY(cudaGetLastError());
        TRY(to_bf16(P, H, rh, H, false, rhb, kh, st));
        TRY(tc(t, P, H, H, rhb, kh, Ub + (size_t)2 * H * kh, kh, t->AH, H, false, false, st));
        k_cand_fwd<<<blocks_for((long long)PH), 256, 0, st>>>(P, H, GX, t->AH, z, hp, c, h);
        TRY(cudaGetLastError());
        TRY(to_bf16(P, H, h, H, false, hsb + (size_t)(s + 1) * P * kh, kh, st));
    }
    // outputs of every step: D = [h_1 .. h_T] W_fc^T
    TRY(tc(t, TP, n_out, H, hsb + (size_t)P * kh, kh, Wfcb, kh, D, n_out, false, false, st));
    return cudaSuccess;
}

// The window's backward with BF16 products (X, Uh, Wfc: the forward's arrays).
cudaError_t seq_backward_bf16(dnnmg_trainer_s *t, const float *dD, const float *X, const float *Uh, const float *Wfc,
                              float *gWx, float *gUh, float *gWfc, cudaStream_t st) {
    const int H = t->H, P = t->P, T = t->T, n_in = t->n_in, n_out = t->n_out, TP = T * P;
    const int kh = t->kh, k2 = t->k2, ko = t->ko, kt = t->kt, ks = t->ks;
    const size_t PH = (size_t)P * H;
    __nv_bfloat16 *WfcT = at(t, t->o_WfcT), *UcT = at(t, t->o_UcT), *UzrT = at(t, t->o_UzrT), *dDb = at(t, t->o_dD);
    __nv_bfloat16 *dGc = at(t, t->o_dGc), *dGzr = at(t, t->o_dGzr);
    cudaError_t e;
    // W_fc^T [H][n_out], U_h^T [H][H], [U_z; U_r]^T [H][2H]
    TRY(to_bf16(H, n_out, Wfc, H, true, WfcT, ko, st));
    TRY(to_bf16(H, H, Uh + (size_t)2 * H * H, H, true, UcT, kh, st));
    TRY(to_bf16(H, 2 * H, Uh, H, true, UzrT, k2, st));
    TRY(to_bf16(TP, n_out, dD, n_out, false, dDb, ko, st));
    // gradient reaching each h_t from its own output: dD W_fc, all steps
    TRY(tc(t, TP, H, n_out, dDb, ko, WfcT, ko, t->dHfc, H, false, false, st));
    TRY(cudaMemsetAsync(t->carry, 0, PH * sizeof(float), st));
    for (int s = T - 1; s >= 0; --s) {
        const float *hp = t->hs + (size_t)s * PH;
        const float *z = t->z + (size_t)s * PH, *r = t->r + (size_t)s * PH, *c = t->c + (size_t)s * PH;
        float *dG = t->dG + (size_t)s * P * 3 * H;
        k_bwd_state<<<blocks_for((long long)PH), 256, 0, st>>>(P, H, t->dHfc + (size_t)s * PH, t->carry, z, c, hp,
                                                                dG, t->dh);
        TRY(cudaGetLastError());
        // d(r h_{t-1}) = dA_c U_h
        TRY(to_bf16(P, H, dG + 2 * H, 3 * H, false, dGc, kh, st));
        TRY(tc(t, P, H, H, dGc, kh, UcT, kh, t->drh, H, false, false, st));
        k_bwd_reset<<<blocks_for((long long)PH), 256, 0, st>>>(P, H, t->drh, hp, r, z, t->dh, dG, t->carry);
        TRY(cudaGetLastError());
        // carry += [dA_z, dA_r] [U_z; U_r]
        TRY(to_bf16(P, 2 * H, dG, 3 * H, false, dGzr, k2, st));
        TRY(tc(t, P, H, 2 * H, dGzr, k2, UzrT, k2, t->carry, H, true, false, st));
    }
    // weight gradients: products over all steps and patches, each operand
    // transposed (K = T P contiguous) once
    __nv_bfloat16 *dGT = at(t, t->o_dGT), *XT = at(t, t->o_XT), *hsT = at(t, t->o_hsT), *rhT = at(t, t->o_rhT);
    __nv_bfloat16 *dDT = at(t, t->o_dDT);
    TRY(to_bf16(3 * H, TP, t->dG, 3 * H, true, dGT, kt, st));
    TRY(to_bf16(n_in, TP, X, t->ldx, true, XT, kt, st));
    TRY(to_bf16(H, TP + P, t->hs, H, true, hsT, ks, st));
    TRY(to_bf16(H, TP, t->rh, H, true, rhT, kt, st));
    TRY(to_bf16(n_out, TP, dD, n_out, true, dDT, kt, st));
    TRY(tc(t, 3 * H, n_in, TP, dGT, kt, XT, kt, gWx, n_in, false, true, st));
    TRY(tc(t, 2 * H, H, TP, dGT, kt, hsT, ks, gUh, H, false, true, st));
    TRY(tc(t, H, H, TP, dGT + (size_t)2 * H * kt, kt, rhT, kt, gUh + (size_t)2 * H * H, H, false, true, st));
    // h_1 .. h_T: columns P.. of hs^T where they start on 16 bytes, else a copy in rhT's place
    const __nv_bfloat16 *hs1 = hsT + P;
    int ld1 = ks;
    if (P % 8) {
        TRY(to_bf16(H, TP, t->hs + PH, H, true, rhT, kt, st));
        hs1 = rhT;
        ld1 = kt;
    }
    TRY(tc(t, n_out, H, TP, dDT, kt, hs1, ld1, gWfc, H, false, true, st));
#undef TRY
    return cudaSuccess;
}

void trainer_free(dnnmg_trainer_s *t) {
    if (!t) return;
    float *bufs[] = {t->GX, t->hs, t->z, t->r, t->rh, t->c, t->GH, t->AH, t->dHfc, t->dG, t->dh, t->drh, t->carry,
                     t->part};
    for (float *b : bufs) cudaFree(b);
    cudaFree(t->red);
    cudaFree(t->d_status);
    cudaFree(t->arena);
    delete t;
}

int check_trainer(dnnmg_trainer_s *t) {
    if (!t) return fail(DNNMG_EINVAL, "trainer handle is NULL");
    int cur = -1;
    DNNMG_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != t->device) return fail(DNNMG_EINVAL, "trainer belongs to device %d but device %d is current", t->device, cur);
    return DNNMG_OK;
}

}  // namespace
}  // namespace dnnmg

using namespace dnnmg;

extern "C" {

int dnnmg_trainer_create(int n_in, int ldx, int H, int n_out, int T, int P, dnnmg_trainer_t *out) {
    clear_error();
    if (!out) return fail(DNNMG_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_in < 1 || ldx < n_in || H < 1 || n_out < 1 || T < 1 || P < 1)
        return fail(DNNMG_EINVAL, "n_in %d, ldx %d, H %d, n_out %d, T %d, P %d", n_in, ldx, H, n_out, T, P);
    if ((long long)T * P * 3 * H > (1LL << 31) - 1) return fail(DNNMG_EINVAL, "window too large (T P 3H >= 2^31)");
    dnnmg_trainer_s *t = new (std::nothrow) dnnmg_trainer_s();
    if (!t) return fail(DNNMG_ENOMEM, "host allocation failed");
    *t = dnnmg_trainer_s{};
    t->n_in = n_in; t->ldx = ldx; t->H = H; t->n_out = n_out; t->T = T; t->P = P;
    DNNMG_CUDA_TRY(cudaGetDevice(&t->device));
    const size_t TP = (size_t)T * P;
    // split the weight-gradient products over K = T P in ranges of about 4096 rows
    t->splits = (int)std::min<size_t>(256, std::max<size_t>(1, TP / 4096));
    const size_t mx = (size_t)std::max(3 * H, n_out) * std::max(std::max(n_in, H), 1);
    t->part_floats = (size_t)t->splits * mx;
    struct { float **p; size_t n; } req[] = {
        {&t->GX, TP * 3 * H}, {&t->hs, (TP + P) * H}, {&t->z, TP * H}, {&t->r, TP * H}, {&t->rh, TP * H},
        {&t->c, TP * H}, {&t->GH, (size_t)P * 2 * H}, {&t->AH, (size_t)P * H}, {&t->dHfc, TP * H},
        {&t->dG, TP * 3 * H}, {&t->dh, (size_t)P * H}, {&t->drh, (size_t)P * H}, {&t->carry, (size_t)P * H},
        {&t->part, t->part_floats}};
    bool ok = true;
    for (auto &q : req) ok = ok && cudaMalloc(q.p, q.n * sizeof(float)) == cudaSuccess;
    ok = ok && cudaMalloc(&t->red, kRedBlocks * sizeof(double)) == cudaSuccess;
    if (!ok) {
        trainer_free(t);
        cudaGetLastError();
        return fail(DNNMG_ENOMEM, "device allocation of the training window (T %d, P %d, H %d) failed", T, P, H);
    }
    *out = t;
    return DNNMG_OK;
}

int dnnmg_trainer_destroy(dnnmg_trainer_t t) {
    clear_error();
    if (!t) return DNNMG_OK;
    cudaDeviceSynchronize();
    trainer_free(t);
    return DNNMG_OK;
}

int dnnmg_trainer_set_precision(dnnmg_trainer_t t, int precision) {
    clear_error();
    if (int e = check_trainer(t)) return e;
    if (precision != DNNMG_F32 && precision != DNNMG_BF16NET)
        return fail(DNNMG_EINVAL, "trainer precision must be DNNMG_F32 or DNNMG_BF16NET, got %d", precision);
    t->bf16 = 0;
    if (precision == DNNMG_F32) return DNNMG_OK;
    // BF16 copies of the window's operands, K contiguous, each region 256-byte aligned
    const int H = t->H, P = t->P, TP = t->T * t->P;
    t->kx = kpad(t->n_in); t->kh = kpad(H); t->k2 = kpad(2 * H); t->ko = kpad(t->n_out);
    t->kt = kpad(TP); t->ks = kpad(TP + P);
    size_t off = 0;
    auto take = [&](size_t n) { const size_t o = off; off += (n + 127) / 128 * 128; return o; };
    t->o_Wx = take((size_t)3 * H * t->kx);
    t->o_U = take((size_t)3 * H * t->kh);
    t->o_Wfc = take((size_t)t->n_out * t->kh);
    t->o_X = take((size_t)TP * t->kx);
    t->o_hs = take((size_t)(TP + P) * t->kh);
    t->o_rh = take((size_t)P * t->kh);
    t->o_WfcT = take((size_t)H * t->ko);
    t->o_UcT = take((size_t)H * t->kh);
    t->o_UzrT = take((size_t)H * t->k2);
    t->o_dD = take((size_t)TP * t->ko);
    t->o_dGc = take((size_t)P * t->kh);
    t->o_dGzr = take((size_t)P * t->k2);
    t->o_dGT = take((size_t)3 * H * t->kt);
    t->o_XT = take((size_t)t->n_in * t->kt);
    t->o_hsT = take((size_t)H * t->ks);
    t->o_rhT = take((size_t)H * t->kt);
    t->o_dDT = take((size_t)t->n_out * t->kt);
    if (off > t->arena_elems || !t->d_status) {
        cudaFree(t->arena);
        t->arena = nullptr;
        t->arena_elems = 0;
        if (cudaMalloc(&t->arena, off * sizeof(__nv_bfloat16)) != cudaSuccess ||
            (!t->d_status && cudaMalloc(&t->d_status, sizeof(int)) != cudaSuccess)) {
            cudaFree(t->arena);
            t->arena = nullptr;
            cudaGetLastError();
            return fail(DNNMG_ENOMEM, "BF16 operand scratch (%zu values) could not be allocated", off);
        }
        DNNMG_CUDA_TRY(cudaMemset(t->d_status, 0, sizeof(int)));
        t->arena_elems = off;
    }
    t->bf16 = 1;
    return DNNMG_OK;
}

int dnnmg_trainer_status(dnnmg_trainer_t t, int *status, int reset) {
    clear_error();
    if (int e = check_trainer(t)) return e;
    if (!status) return fail(DNNMG_EINVAL, "status is NULL");
    *status = 0;
    if (!t->d_status) return DNNMG_OK;
    DNNMG_CUDA_TRY(cudaMemcpy(status, t->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (reset) DNNMG_CUDA_TRY(cudaMemset(t->d_status, 0, sizeof(int)));
    return DNNMG_OK;
}

int dnnmg_gemm_bf16_nt(int M, int N, int K, const void *A, int lda, const void *B, int ldb, float *C, int ldc,
                       int accumulate, int *status, cudaStream_t st) {
    clear_error();
    if (M < 0 || N < 0 || K < 0 || (M > 0 && N > 0 && (!A || !B || !C || !status)) || ldc < N)
        return fail(DNNMG_EINVAL, "bad argument (M %d, N %d, K %d, ldc %d)", M, N, K, ldc);
    cudaError_t e = launch_gemm_tc(M, N, K, A, lda, B, ldb, C, ldc, accumulate != 0, 1, nullptr, status, st);
    if (e == cudaErrorInvalidValue)
        return fail(DNNMG_EINVAL, "operands not taken: lda %d, ldb %d must be multiples of 8 and >= K %d, 16-byte aligned",
                    lda, ldb, K);
    DNNMG_CUDA_TRY(e);
    return DNNMG_OK;
}

int dnnmg_gru_seq_forward(dnnmg_trainer_t t, const float *X, const float *h0, const float *Wx, const float *Uh,
                          const float *Wfc, float *D, cudaStream_t st) {
    clear_error();
    if (int e = check_trainer(t)) return e;
    if (!X || !Wx || !Uh || !Wfc || !D) return fail(DNNMG_EINVAL, "NULL array");
    const int H = t->H, P = t->P, T = t->T;
    const size_t PH = (size_t)P * H;
    const int TP = T * P;
    // h_0 (zero when h0 is NULL)
    if (h0) DNNMG_CUDA_TRY(cudaMemcpyAsync(t->hs, h0, PH * sizeof(float), cudaMemcpyDeviceToDevice, st));
    else DNNMG_CUDA_TRY(cudaMemsetAsync(t->hs, 0, PH * sizeof(float), st));
    if (t->bf16) {
        DNNMG_CUDA_TRY(seq_forward_bf16(t, X, Wx, Uh, Wfc, D, st));
        return DNNMG_OK;
    }
    // input parts of every gate, all steps: GX = X W_x^T
    DNNMG_CUDA_TRY((prod<false, true>(t, TP, 3 * H, t->n_in, X, t->ldx, Wx, t->n_in, t->GX, 3 * H, false, false, st)));
    for (int s = 0; s < T; ++s) {
        const float *hp = t->hs + (size_t)s * PH;
        const float *GX = t->GX + (size_t)s * P * 3 * H;
        float *z = t->z + (size_t)s * PH, *r = t->r + (size_t)s * PH, *rh = t->rh + (size_t)s * PH;
        float *c = t->c + (size_t)s * PH, *h = t->hs + (size_t)(s + 1) * PH;
        DNNMG_CUDA_TRY((prod<false, true>(t, P, 2 * H, H, hp, H, Uh, H, t->GH, 2 * H, false, false, st)));
        k_gates_fwd<<<blocks_for((long long)PH), 256, 0, st>>>(P, H, GX, t->GH, hp, z, r, rh);
        DNNMG_CUDA_TRY(cudaGetLastError());
        DNNMG_CUDA_TRY((prod<false, true>(t, P, H, H, rh, H, Uh + (size_t)2 * H * H, H, t->AH, H, false, false, st)));
        k_cand_fwd<<<blocks_for((long long)PH), 256, 0, st>>>(P, H, GX, t->AH, z, hp, c, h);
        DNNMG_CUDA_TRY(cudaGetLastError());
    }
    // outputs of every step: D = [h_1 .. h_T] W_fc^T
    DNNMG_CUDA_TRY((prod<false, true>(t, TP, t->n_out, H, t->hs + PH, H, Wfc, H, D, t->n_out, false, false, st)));
    return DNNMG_OK;
}

int dnnmg_gru_seq_state(dnnmg_trainer_t t, float **hT) {
    clear_error();
    if (!t || !hT) return fail(DNNMG_EINVAL, "NULL argument");
    *hT = t->hs + (size_t)t->T * t->P * t->H;
    return DNNMG_OK;
}

int dnnmg_gru_seq_backward(dnnmg_trainer_t t, const float *dD, const float *X, const float *Uh, const float *Wfc,
                           float *gWx, float *gUh, float *gWfc, float *dh0, cudaStream_t st) {
    clear_error();
    if (int e = check_trainer(t)) return e;
    if (!dD || !X || !Uh || !Wfc || !gWx || !gUh || !gWfc) return fail(DNNMG_EINVAL, "NULL array");
    const int H = t->H, P = t->P, T = t->T, n_out = t->n_out, n_in = t->n_in;
    const size_t PH = (size_t)P * H;
    const int TP = T * P;
    if (t->bf16) {
        DNNMG_CUDA_TRY(seq_backward_bf16(t, dD, X, Uh, Wfc, gWx, gUh, gWfc, st));
        if (dh0) DNNMG_CUDA_TRY(cudaMemcpyAsync(dh0, t->carry, PH * sizeof(float), cudaMemcpyDeviceToDevice, st));
        return DNNMG_OK;
    }
    // gradient reaching each h_t from its own output: dD W_fc, all steps
    DNNMG_CUDA_TRY((prod<false, false>(t, TP, H, n_out, dD, n_out, Wfc, H, t->dHfc, H, false, false, st)));
    DNNMG_CUDA_TRY(cudaMemsetAsync(t->carry, 0, PH * sizeof(float), st));
    for (int s = T - 1; s >= 0; --s) {
        const float *hp = t->hs + (size_t)s * PH;
        const float *z = t->z + (size_t)s * PH, *r = t->r + (size_t)s * PH, *c = t->c + (size_t)s * PH;
        float *dG = t->dG + (size_t)s * P * 3 * H;
        k_bwd_state<<<blocks_for((long long)PH), 256, 0, st>>>(P, H, t->dHfc + (size_t)s * PH, t->carry, z, c, hp,
                                                                dG, t->dh);
        DNNMG_CUDA_TRY(cudaGetLastError());
        // d(r h_{t-1}) = dA_c U_h
        DNNMG_CUDA_TRY((prod<false, false>(t, P, H, H, dG + 2 * H, 3 * H, Uh + (size_t)2 * H * H, H, t->drh, H,
                                           false, false, st)));
        k_bwd_reset<<<blocks_for((long long)PH), 256, 0, st>>>(P, H, t->drh, hp, r, z, t->dh, dG, t->carry);
        DNNMG_CUDA_TRY(cudaGetLastError());
        // carry += [dA_z, dA_r] [U_z; U_r]
        DNNMG_CUDA_TRY((prod<false, false>(t, P, H, 2 * H, dG, 3 * H, Uh, H, t->carry, H, true, false, st)));
    }
    if (dh0) DNNMG_CUDA_TRY(cudaMemcpyAsync(dh0, t->carry, PH * sizeof(float), cudaMemcpyDeviceToDevice, st));
    // weight gradients: products over all steps and patches
    DNNMG_CUDA_TRY((prod<true, false>(t, 3 * H, n_in, TP, t->dG, 3 * H, X, t->ldx, gWx, n_in, false, true, st)));
    DNNMG_CUDA_TRY((prod<true, false>(t, 2 * H, H, TP, t->dG, 3 * H, t->hs, H, gUh, H, false, true, st)));
    DNNMG_CUDA_TRY((prod<true, false>(t, H, H, TP, t->dG + 2 * H, 3 * H, t->rh, H, gUh + (size_t)2 * H * H, H, false,
                                      true, st)));
    DNNMG_CUDA_TRY((prod<true, false>(t, n_out, H, TP, dD, n_out, t->hs + PH, H, gWfc, H, false, true, st)));
    return DNNMG_OK;
}

int dnnmg_l2_loss(const float *D, const float *Y, long long n, int P, float *dD, double *loss, cudaStream_t st) {
    clear_error();
    if (!D || !Y || !loss || n < 0 || P < 1) return fail(DNNMG_EINVAL, "bad argument");
    double *part = nullptr;
    DNNMG_CUDA_TRY(cudaMallocAsync(&part, kRedBlocks * sizeof(double), st));
    k_l2_loss<<<kRedBlocks, 256, 0, st>>>(n, P, (float)(2.0 / P), D, Y, dD, part);
    k_sum_parts<<<1, 256, 0, st>>>(kRedBlocks, part, loss);
    DNNMG_CUDA_TRY(cudaGetLastError());
    DNNMG_CUDA_TRY(cudaFreeAsync(part, st));
    return DNNMG_OK;
}

int dnnmg_sumsq(const float *x, long long n, double *out, cudaStream_t st) {
    clear_error();
    if (!x || !out || n < 0) return fail(DNNMG_EINVAL, "bad argument");
    double *part = nullptr;
    DNNMG_CUDA_TRY(cudaMallocAsync(&part, kRedBlocks * sizeof(double), st));
    k_sumsq<<<kRedBlocks, 256, 0, st>>>(n, x, part);
    k_sum_parts<<<1, 256, 0, st>>>(kRedBlocks, part, out);
    DNNMG_CUDA_TRY(cudaGetLastError());
    DNNMG_CUDA_TRY(cudaFreeAsync(part, st));
    return DNNMG_OK;
}

int dnnmg_adam_step(float *p, const float *g, float *m, float *v, long long n, int step, float lr, float b1,
                    float b2, float eps, float alpha, cudaStream_t st) {
    clear_error();
    if (!p || !g || !m || !v || n < 0 || step < 1) return fail(DNNMG_EINVAL, "bad argument");
    const float c1 = (float)(1.0 - std::pow((double)b1, step)), c2 = (float)(1.0 - std::pow((double)b2, step));
    if (n > 0) k_adam<<<blocks_for(n), 256, 0, st>>>(n, p, g, m, v, lr, b1, b2, eps, alpha, c1, c2);
    DNNMG_CUDA_TRY(cudaGetLastError());
    return DNNMG_OK;
}

}  // extern "C"

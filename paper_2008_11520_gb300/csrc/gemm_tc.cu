// BF16 matrix products on the 5th-generation tensor cores (tcgen05, sm_103a)
// for training the patch network (Sec. 6.3; the training workload asks for
// BF16 products with FP32 master weights):
//
//   C[M][N] (row stride ldc, FP32)  =  A[M][K] B[N][K]^T   (or += C)
//
// A and B are BF16, row-major with K contiguous (row strides lda, ldb
// elements, multiples of 8 so that rows start on 16 bytes).  Each CTA owns a
// 128-row x BN-column tile of C (BN <= 256, one TMEM column per output
// column, one TMEM lane per row) and a range of K: 64-wide chunks of A and B
// arrive by 2D tensor copies (128-byte swizzle, zero fill past M, N and K)
// into a ring of stages, the MMAs accumulate in TMEM, and the epilogue adds
// the tile into C.  With K split over blockIdx.z each range writes its own
// partial tile (C + z * cstride), summed afterwards in a fixed order.
//
// Warp roles (224 threads): warps 0 and 6 copy the A and B chunks (the copy
// engine serves one thread's copies one after the other, so the two operands
// come from two warps); warp 1 owns the tensor memory and one lane issues the
// MMAs; warps 2..5 are the epilogue, one per TMEM lane quadrant.  Every wait
// is bounded (2 s): on time-out the kernel sets DNNMG_DEVERR_TIMEOUT in
// *status, drains what it started, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "ptx.cuh"

namespace dnnmg {
namespace {

using namespace ptx;

constexpr int BM = 128;                 // rows of a C tile (UMMA M)
constexpr int KC = 64;                  // K elements per chunk = one 128-byte swizzle row
constexpr int NTH = 224;
constexpr int ASZ = BM * KC * 2;        // 16 KB: A chunk
constexpr int NSTAGE = 4;
constexpr int BN_MAX = 256;
constexpr int BSZ = BN_MAX * KC * 2;    // 32 KB: largest B chunk
constexpr int SMEM = NSTAGE * (ASZ + BSZ) + 1024 + 256;

__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset between 8-row groups
    d |= (uint64_t)1 << 46;                 // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                 // swizzle mode: 128 B
    return d;
}
// Instruction descriptor, kind::f16: BF16 A and B, FP32 D, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct GemmArgs {
    int M, N, K, BN, kchunk, tmem_cols, accumulate;
    float *C;
    int ldc;
    long long cstride;
    int *status;
};

__global__ void __launch_bounds__(NTH, 1)
k_gemm_tc(const __grid_constant__ GemmArgs g, const __grid_constant__ CUtensorMap tmA,
          const __grid_constant__ CUtensorMap tmB) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t *sA = base, *sB = base + NSTAGE * ASZ;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sB + NSTAGE * BSZ);
    // full[NSTAGE] (both copy warps arrive), empty[NSTAGE], done
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * NSTAGE + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * g.BN;
    const int kb = blockIdx.z * g.kchunk, ke = min(g.K, kb + g.kchunk);
    const int nk = ke > kb ? (ke - kb + KC - 1) / KC : 0;
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * NSTAGE, done_bar = full0 + 16 * NSTAGE;
    const uint32_t bbytes = (uint32_t)g.BN * KC * 2;

    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(full0 + 8 * s, 2);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(done_bar, 1);
        *abort_flag = 0;
        mbar_init_fence();
        fence_async_smem();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(g.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tmem_slot;
    volatile int no_abort = 0;

    if ((warp == 0 || warp == 6) && lane == 0) {
        // ---------------- copies: A chunks (warp 0) or B chunks (warp 6)
        const bool isA = warp == 0;
        const CUtensorMap *tm = isA ? &tmA : &tmB;
        prefetch_tensormap(tm);
        int issued = 0;
        for (int i = 0; i < nk; ++i) {
            const int s = i % NSTAGE;
            if (i >= NSTAGE && !mbar_wait(empty0 + 8 * s, ((i / NSTAGE) - 1) & 1, abort_flag)) break;
            const uint32_t fb = full0 + 8 * s;
            expect_tx(fb, isA ? (uint32_t)ASZ : bbytes);
            if (isA) tma_load_2d(smem_u32(sA + s * ASZ), tm, kb + i * KC, m0, fb);
            else tma_load_2d(smem_u32(sB + s * BSZ), tm, kb + i * KC, n0, fb);
            issued = i + 1;
        }
        // every started copy lands before the CTA may exit
        for (int i = issued > NSTAGE ? issued - NSTAGE : 0; i < issued; ++i)
            mbar_wait(full0 + 8 * (i % NSTAGE), (i / NSTAGE) & 1, &no_abort);
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(BM, g.BN);
            bool ok = true;
            for (int i = 0; ok && i < nk; ++i) {
                const int s = i % NSTAGE;
                if (!(ok = mbar_wait(full0 + 8 * s, (i / NSTAGE) & 1, abort_flag))) break;
                tc_after_sync();
                const uint64_t a = sdesc(smem_u32(sA + s * ASZ)), b = sdesc(smem_u32(sB + s * BSZ));
#pragma unroll
                for (int k = 0; k < KC / 16; ++k) umma(tmem, a + 2 * k, b + 2 * k, idesc, (i | k) ? 1u : 0u);
                tc_commit(empty0 + 8 * s);
            }
            // the accumulators are complete (and every MMA has finished before teardown)
            tc_commit(done_bar);
            mbar_wait(done_bar, 0, &no_abort);
        }
    } else if (warp >= 2 && warp <= 5) {
        // ---------------- epilogue: one row of the tile per thread
        const int q = warp & 3, row = q * 32 + lane, gm = m0 + row;
        const bool ok = nk == 0 || __all_sync(0xffffffffu, mbar_wait(done_bar, 0, abort_flag));
        tc_after_sync();
        if (ok && !*abort_flag) {
            float *crow = g.C + (long long)blockIdx.z * g.cstride + (long long)gm * g.ldc;
            const bool vec = g.ldc % 4 == 0 && g.cstride % 4 == 0 && ((uintptr_t)g.C & 15) == 0;
            for (int cb = 0; cb < g.BN / 16; ++cb) {
                float v[16];
                if (nk > 0) tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + 16 * cb, v);
                else
                    for (int i = 0; i < 16; ++i) v[i] = 0.f;
                const int c0 = n0 + 16 * cb;
                if (gm >= g.M) continue;
                if (vec && c0 + 16 <= g.N) {
                    // 16 columns as four 16-byte pieces (row starts on 16 bytes)
                    float4 *q4 = reinterpret_cast<float4 *>(crow + c0);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float4 x = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                        if (g.accumulate) {
                            const float4 o = q4[j];
                            x.x += o.x; x.y += o.y; x.z += o.z; x.w += o.w;
                        }
                        q4[j] = x;
                    }
                } else {
                    for (int i = 0; i < 16; ++i) {
                        const int col = c0 + i;
                        if (col < g.N) crow[col] = g.accumulate ? crow[col] + v[i] : v[i];
                    }
                }
            }
        }
    }

    // ---------------- teardown
    if (tid == 0 && *abort_flag) atomicOr(g.status, DNNMG_DEVERR_TIMEOUT);
    tc_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }
    return fn;
}

// K-major BF16 operand [rows][K] with row stride ld elements: 64 x box_rows boxes.
bool encode_operand(CUtensorMap *m, const void *p, int rows, int K, int ld, int box_rows) {
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)KC, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return encode_fn() &&
           encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(p), dims, strides, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// C (+)= A B^T on the tensor cores; splits > 1 writes `splits` partial
// products of K ranges (multiples of 64) to part + z M N (row stride N),
// which the caller reduces.  Returns cudaErrorInvalidValue for shapes it
// does not take (lda, ldb not multiples of 8, unaligned pointers).
cudaError_t launch_gemm_tc(int M, int N, int K, const void *A, int lda, const void *B, int ldb, float *C, int ldc,
                           bool accumulate, int splits, float *part, int *status, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (lda % 8 || ldb % 8 || (uintptr_t)A % 16 || (uintptr_t)B % 16 || K > lda || K > ldb) return cudaErrorInvalidValue;
    const int BN = std::min(BN_MAX, round_up(N, 16));
    int cols = 32;
    while (cols < BN) cols *= 2;
    const int kchunk = splits > 1 ? round_up((K + splits - 1) / splits, KC) : std::max(round_up(K, KC), KC);
    const int sz = splits > 1 ? (K + kchunk - 1) / kchunk : 1;
    CUtensorMap ta, tb;
    if (!encode_operand(&ta, A, M, std::max(K, 1), lda, BM) || !encode_operand(&tb, B, N, std::max(K, 1), ldb, BN))
        return cudaErrorInvalidValue;
    GemmArgs g;
    memset(&g, 0, sizeof g);
    g.M = M; g.N = N; g.K = K; g.BN = BN; g.kchunk = kchunk; g.tmem_cols = cols;
    g.accumulate = (splits > 1 || !accumulate) ? 0 : 1;
    g.C = splits > 1 ? part : C;
    g.ldc = splits > 1 ? N : ldc;
    g.cstride = splits > 1 ? (long long)M * N : 0;
    g.status = status;
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e != cudaSuccess) return e;
    const dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, sz);
    k_gemm_tc<<<grid, NTH, SMEM, st>>>(g, ta, tb);
    return cudaGetLastError();
}

int gemm_tc_splits_used(int K, int splits) {
    if (splits <= 1) return 1;
    const int kchunk = round_up((K + splits - 1) / splits, KC);
    return (K + kchunk - 1) / kchunk;
}

}  // namespace dnnmg

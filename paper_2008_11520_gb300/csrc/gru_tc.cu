// S4 on the 5th-generation tensor cores (tcgen05, sm_103a): GRU cell of
// Eq. gru (reset gate before U_h, no biases) and the output layer for 128
// patches per CTA, BF16 operands, FP32 accumulators in tensor memory.
//
// Per tile of 128 patch rows (one TMEM lane per row):
//   phase 1:  D1 = [X | h] [W_z W_r ; U_z U_r]^T   (N = 2H: z and r pre-activations)
//             D2 = X W_h^T                          (N = H)
//   epilogue: r = sig(D1_r), A_h <- bf16(r * h)
//   phase 2:  D2 += (r * h) U_h^T
//   epilogue: z = sig(D1_z), h' = z h + (1 - z) tanh(D2); h <- h' (FP32), A_h <- bf16(h')
//   phase 3:  D3 = h' W_fc^T                         (N = round_up(n_out, 16), reuses D1 columns)
//   epilogue: d <- D3
// Operands sit in shared memory in the canonical K-major 128-byte-swizzle
// layout (8-row x 128-byte atoms).  X and h are staged by the CTA's threads;
// the weights are streamed from a pre-swizzled blob (every chunk already in
// its shared-memory image) by 1D bulk copies through a 3-stage mbarrier
// pipeline.  One thread issues all copies and MMAs.  Every wait is bounded:
// on time-out the kernel records DNNMG_DEVERR_TIMEOUT in the net's status
// word, drains what it started, frees its tensor memory and returns.
#include <cstring>
#include <vector>

#include "common.cuh"

namespace dnnmg {
namespace {

constexpr int TM = 128;                 // patch rows per tile (UMMA M)
constexpr int NTH = 128;                // 4 warps; warp w owns TMEM lanes 32w..32w+31
constexpr int KC = 64;                  // K elements per chunk = one 128-byte swizzle row
constexpr int CHUNK_A = TM * KC * 2;    // 16 KB
constexpr int NSTAGE = 3;
constexpr int MAX_ITEMS = 32;
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s per wait

struct TcItem {
    int off;     // byte offset of the chunk in the weight blob
    int bytes;   // chunk bytes (rows * 128)
    int kind;    // 0: D1 += A[kc] B; 1: D2 += A[kc] B; 2: D2 += A[nxc+kc] B; 3: D3 = A[nxc+kc] B
    int kc;
};

struct TcParams {
    int n_in, ldx, H, n_out, nfc, nxc, nhc, nitems, end1, end2, stage_bytes, tmem_cols;
    const uint8_t *wblob;
    int *status;
    TcItem items[MAX_ITEMS];
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait on an mbarrier phase; false (and the abort flag set) on time-out
// or when another thread has already aborted.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
    const unsigned long long t0 = now_ns();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255) == 255) {
            if (*abort_flag) return false;
            if (now_ns() - t0 > kWaitNs) {
                *abort_flag = 1;
                return false;
            }
        }
    }
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
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
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
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

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 t = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&t);
}
// byte offset of 16-byte unit u (0..7) of row `row` in a 128B-swizzled chunk
__device__ __forceinline__ uint32_t swz(int row, int u) { return (uint32_t)(row * 128 + ((u ^ (row & 7)) << 4)); }

__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + expf(-x)); }

// Issues the MMAs of weight item i (staged in `stage`) -- thread 0 only.
__device__ __forceinline__ void issue_item(const TcParams &p, const TcItem &it, uint32_t sA, uint32_t stage,
                                           uint32_t tmem) {
    uint32_t a_chunk, dcol, N, acc;
    switch (it.kind) {
        case 0: a_chunk = it.kc; dcol = 0; N = 2 * p.H; acc = it.kc > 0; break;
        case 1: a_chunk = it.kc; dcol = 2 * p.H; N = p.H; acc = it.kc > 0; break;
        case 2: a_chunk = p.nxc + it.kc; dcol = 2 * p.H; N = p.H; acc = 1; break;
        default: a_chunk = p.nxc + it.kc; dcol = 0; N = p.nfc; acc = it.kc > 0; break;
    }
    const uint32_t idesc = idesc_bf16(TM, (int)N);
    const uint32_t a0 = sA + a_chunk * CHUNK_A;
#pragma unroll
    for (int k = 0; k < KC / 16; ++k)
        umma(tmem + dcol, sdesc(a0 + k * 32), sdesc(stage + k * 32), idesc, (acc || k > 0) ? 1u : 0u);
}

__global__ void __launch_bounds__(NTH, 1)
k_gru_tc(const __grid_constant__ TcParams p, const __nv_bfloat16 *__restrict__ X, float *__restrict__ h,
         float *__restrict__ d, int P) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = base;
    uint8_t *sW = sA + (p.nxc + p.nhc) * CHUNK_A;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sW + NSTAGE * p.stage_bytes);   // full[3], empty[3], mma, drain
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * NSTAGE + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int p0 = blockIdx.x * TM;
    const uint32_t sA_u = smem_u32(sA), sW_u = smem_u32(sW);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + NSTAGE), mma_bar = smem_u32(bars + 2 * NSTAGE);
    const uint32_t drain_bar = smem_u32(bars + 2 * NSTAGE + 1);

    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(mma_bar, 1);
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(p.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tmem_slot;

    // weight pipeline state (meaningful in thread 0 only)
    int loaded = 0;
    auto load_item = [&](int i) {
        const TcItem &it = p.items[i];
        const int s = i % NSTAGE;
        bulk_load(sW_u + s * p.stage_bytes, p.wblob + it.off, (uint32_t)it.bytes, full0 + 8 * s);
    };
    if (tid == 0) {
        for (; loaded < NSTAGE && loaded < p.nitems; ++loaded) load_item(loaded);
    }

    // stage A: X rows (bf16) and h rows (fp32 -> bf16), zero beyond the data
    {
        const int upr = p.ldx / 8, ucx = p.nxc * 8;
        for (int e = tid; e < TM * ucx; e += NTH) {
            const int row = e / ucx, u = e - row * ucx;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (u < upr && p0 + row < P)
                v = __ldg(reinterpret_cast<const uint4 *>(X + (size_t)(p0 + row) * p.ldx) + u);
            *reinterpret_cast<uint4 *>(sA + (u >> 3) * CHUNK_A + swz(row, u & 7)) = v;
        }
        const int uph = p.H / 8, uch = p.nhc * 8;
        for (int e = tid; e < TM * uch; e += NTH) {
            const int row = e / uch, u = e - row * uch;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (u < uph && p0 + row < P) {
                const float4 *src = reinterpret_cast<const float4 *>(h + (size_t)(p0 + row) * p.H + u * 8);
                const float4 a = src[0], b = src[1];
                v = make_uint4(pack_bf16(a.x, a.y), pack_bf16(a.z, a.w), pack_bf16(b.x, b.y), pack_bf16(b.z, b.w));
            }
            *reinterpret_cast<uint4 *>(sA + (p.nxc + (u >> 3)) * CHUNK_A + swz(row, u & 7)) = v;
        }
    }
    fence_async_smem();
    __syncthreads();

    // thread 0: run items [i0, i1) then commit to mma_bar
    auto run_items = [&](int i0, int i1) {
        tc_after_sync();
        for (int i = i0; i < i1; ++i) {
            const int s = i % NSTAGE;
            if (!mbar_wait(full0 + 8 * s, (i / NSTAGE) & 1, abort_flag)) return;
            tc_after_sync();
            issue_item(p, p.items[i], sA_u, sW_u + s * p.stage_bytes, tmem);
            tc_commit(empty0 + 8 * s);
            // refill the stage of item i-1 once its MMAs are done
            if (i >= 1 && loaded < p.nitems && loaded == i - 1 + NSTAGE) {
                const int s2 = (i - 1) % NSTAGE;
                if (!mbar_wait(empty0 + 8 * s2, ((i - 1) / NSTAGE) & 1, abort_flag)) return;
                load_item(loaded++);
            }
        }
        tc_commit(mma_bar);
    };

    const int row = tid;                          // TMEM lane = tile row
    const int gp = p0 + row;
    const bool valid = gp < P;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    const int nhq = p.H / 32;

    // ---------------- phase 1
    if (tid == 0) run_items(0, p.end1);
    bool ok = __all_sync(0xffffffffu, mbar_wait(mma_bar, 0, abort_flag));
    tc_after_sync();
    if (ok) {
        // r * h -> A_h (bf16)
        for (int q = 0; q < nhq; ++q) {
            float rv[32];
            tmem_ld32(lane_base + p.H + 32 * q, rv);
            float hv[32];
#pragma unroll
            for (int i = 0; i < 32; i += 4) {
                float4 t = valid ? *reinterpret_cast<const float4 *>(h + (size_t)gp * p.H + 32 * q + i)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
                hv[i] = t.x; hv[i + 1] = t.y; hv[i + 2] = t.z; hv[i + 3] = t.w;
            }
            const int col = 32 * q;
            uint8_t *chunk = sA + (p.nxc + col / 64) * CHUNK_A;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = 8 * u;
                uint4 v = make_uint4(pack_bf16(sigm(rv[j]) * hv[j], sigm(rv[j + 1]) * hv[j + 1]),
                                     pack_bf16(sigm(rv[j + 2]) * hv[j + 2], sigm(rv[j + 3]) * hv[j + 3]),
                                     pack_bf16(sigm(rv[j + 4]) * hv[j + 4], sigm(rv[j + 5]) * hv[j + 5]),
                                     pack_bf16(sigm(rv[j + 6]) * hv[j + 6], sigm(rv[j + 7]) * hv[j + 7]));
                *reinterpret_cast<uint4 *>(chunk + swz(row, (col % 64) / 8 + u)) = v;
            }
        }
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();

    // ---------------- phase 2
    if (tid == 0 && !*abort_flag) run_items(p.end1, p.end2);
    ok = __all_sync(0xffffffffu, !*abort_flag && mbar_wait(mma_bar, 1, abort_flag));
    tc_after_sync();
    if (ok) {
        for (int q = 0; q < nhq; ++q) {
            float cv[32], zv[32];
            tmem_ld32(lane_base + 2 * p.H + 32 * q, cv);
            tmem_ld32(lane_base + 32 * q, zv);
            float hv[32];
#pragma unroll
            for (int i = 0; i < 32; i += 4) {
                float4 t = valid ? *reinterpret_cast<const float4 *>(h + (size_t)gp * p.H + 32 * q + i)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
                hv[i] = t.x; hv[i + 1] = t.y; hv[i + 2] = t.z; hv[i + 3] = t.w;
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const float z = sigm(zv[i]);
                hv[i] = z * hv[i] + (1.0f - z) * tanhf(cv[i]);
            }
            if (valid) {
#pragma unroll
                for (int i = 0; i < 32; i += 4)
                    *reinterpret_cast<float4 *>(h + (size_t)gp * p.H + 32 * q + i) =
                        make_float4(hv[i], hv[i + 1], hv[i + 2], hv[i + 3]);
            }
            const int col = 32 * q;
            uint8_t *chunk = sA + (p.nxc + col / 64) * CHUNK_A;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = 8 * u;
                uint4 v = make_uint4(pack_bf16(hv[j], hv[j + 1]), pack_bf16(hv[j + 2], hv[j + 3]),
                                     pack_bf16(hv[j + 4], hv[j + 5]), pack_bf16(hv[j + 6], hv[j + 7]));
                *reinterpret_cast<uint4 *>(chunk + swz(row, (col % 64) / 8 + u)) = v;
            }
        }
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();

    // ---------------- phase 3
    if (tid == 0 && !*abort_flag) run_items(p.end2, p.nitems);
    ok = __all_sync(0xffffffffu, !*abort_flag && mbar_wait(mma_bar, 0, abort_flag));
    tc_after_sync();
    if (ok) {
        for (int q = 0; q < p.nfc / 16; ++q) {
            float dv[16];
            tmem_ld16(lane_base + 16 * q, dv);
            if (valid) {
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (16 * q + i < p.n_out) d[(size_t)gp * p.n_out + 16 * q + i] = dv[i];
            }
        }
    }

    // ---------------- teardown
    if (*abort_flag && tid == 0) {
        atomicOr(p.status, DNNMG_DEVERR_TIMEOUT);
        // drain: let every started copy land and every issued MMA finish (bounded)
        volatile int no_abort = 0;
        for (int i = loaded - NSTAGE < 0 ? 0 : loaded - NSTAGE; i < loaded; ++i)
            mbar_wait(full0 + 8 * (i % NSTAGE), (i / NSTAGE) & 1, &no_abort);
        tc_commit(drain_bar);
        no_abort = 0;
        mbar_wait(drain_bar, 0, &no_abort);
    }
    tc_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
    }
}

// host-side element (row, k) of a 128B-swizzled K-major chunk image
inline size_t swz_host(int row, int k) {
    return (size_t)row * 128 + (size_t)((((k / 8) ^ (row % 8)) * 16) + (k % 8) * 2);
}

}  // namespace

struct TcNet {
    TcParams p;
};

// Builds the pre-swizzled weight blob and the item schedule; returns false if
// the shapes are outside what the kernel supports.
bool tc_prepare(Net &n, const double *Wx, const double *Uh, const double *Wfc) {
    const int H = n.H, n_in = n.n_in, n_out = n.n_out, ldx = n.ldx;
    const int nfc = round_up(n_out, 16);
    const int nxc = (ldx + KC - 1) / KC, nhc = (H + KC - 1) / KC;
    if (H % 32 || 2 * H > 256 || nfc > 2 * H || nfc > 256) return false;
    TcParams p;
    memset(&p, 0, sizeof p);
    p.n_in = n_in; p.ldx = ldx; p.H = H; p.n_out = n_out; p.nfc = nfc; p.nxc = nxc; p.nhc = nhc;
    std::vector<TcItem> items;
    std::vector<uint8_t> blob;
    auto add_chunk = [&](int kind, int kc, int rows, auto value) {
        TcItem it;
        it.off = (int)blob.size();
        it.bytes = rows * 128;
        it.kind = kind;
        it.kc = kc;
        blob.resize(blob.size() + it.bytes, 0);
        uint8_t *dst = blob.data() + it.off;
        for (int r = 0; r < rows; ++r)
            for (int k = 0; k < KC; ++k) {
                const __nv_bfloat16 b = __float2bfloat16_rn((float)value(r, k));
                memcpy(dst + swz_host(r, k), &b, 2);
            }
        items.push_back(it);
    };
    for (int kc = 0; kc < nxc + nhc; ++kc) {
        add_chunk(0, kc, 2 * H, [&](int r, int k) -> double {
            if (kc < nxc) {
                const int col = kc * KC + k;
                return col < n_in ? Wx[(size_t)r * n_in + col] : 0.0;
            }
            const int col = (kc - nxc) * KC + k;
            return col < H ? Uh[(size_t)r * H + col] : 0.0;
        });
        if (kc < nxc)
            add_chunk(1, kc, H, [&](int r, int k) -> double {
                const int col = kc * KC + k;
                return col < n_in ? Wx[(size_t)(2 * H + r) * n_in + col] : 0.0;
            });
    }
    p.end1 = (int)items.size();
    for (int kc = 0; kc < nhc; ++kc)
        add_chunk(2, kc, H, [&](int r, int k) -> double {
            const int col = kc * KC + k;
            return col < H ? Uh[(size_t)(2 * H + r) * H + col] : 0.0;
        });
    p.end2 = (int)items.size();
    for (int kc = 0; kc < nhc; ++kc)
        add_chunk(3, kc, nfc, [&](int r, int k) -> double {
            const int col = kc * KC + k;
            return (r < n_out && col < H) ? Wfc[(size_t)r * H + col] : 0.0;
        });
    p.nitems = (int)items.size();
    if (p.nitems > MAX_ITEMS) return false;
    int maxb = 0;
    for (const TcItem &it : items) maxb = it.bytes > maxb ? it.bytes : maxb;
    p.stage_bytes = maxb;
    int cols = 32;
    while (cols < 3 * H) cols *= 2;
    p.tmem_cols = cols;
    for (int i = 0; i < p.nitems; ++i) p.items[i] = items[i];
    const size_t smem = (size_t)(nxc + nhc) * CHUNK_A + (size_t)NSTAGE * maxb + 1024 + 256;
    if (smem > 227 * 1024) return false;
    void *dblob = nullptr;
    if (cudaMalloc(&dblob, blob.size()) != cudaSuccess) return false;
    if (cudaMemcpy(dblob, blob.data(), blob.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(dblob);
        return false;
    }
    p.wblob = static_cast<const uint8_t *>(dblob);
    p.status = n.d_status;
    TcNet *t = new TcNet{p};
    n.tc = t;
    n.tc_weights = dblob;
    n.tc_bytes = blob.size();
    return true;
}

void tc_release(Net &n) {
    delete static_cast<TcNet *>(n.tc);
    n.tc = nullptr;
}

cudaError_t launch_gru_tc(const Net &n, const void *X, void *h, void *d, int P, cudaStream_t st) {
    const TcParams &p = static_cast<const TcNet *>(n.tc)->p;
    const size_t smem = (size_t)(p.nxc + p.nhc) * CHUNK_A + (size_t)NSTAGE * p.stage_bytes + 1024 + 256;
    cudaError_t e = cudaFuncSetAttribute(k_gru_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_gru_tc<<<(P + TM - 1) / TM, NTH, smem, st>>>(p, (const __nv_bfloat16 *)X, (float *)h, (float *)d, P);
    return cudaGetLastError();
}

}  // namespace dnnmg

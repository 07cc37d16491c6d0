// S4 on the 5th-generation tensor cores (tcgen05, sm_103a): GRU cell of
// Eq. gru (reset gate before U_h, no biases) and the output layer for 128
// patches per CTA, BF16 operands, FP32 accumulators in tensor memory.
//
// Per tile of 128 patch rows (one TMEM lane per row):
//   phase 1:  D1 = [X | h] [W_z W_r ; U_z U_r]^T   (2H columns: z and r pre-activations)
//             D2 = X W_h^T                          (H columns)
//   epilogue: r = sig(D1_r), A_h <- bf16(r * h)
//   phase 2:  D2 += (r * h) U_h^T
//   epilogue: z = sig(D1_z), h' = z h + (1 - z) tanh(D2); h <- h' (FP32), A_h <- bf16(h')
//   phase 3:  D3 = h' W_fc^T                         (reuses the D1 columns)
//   epilogue: d <- D3
//
// Warp roles (320 threads): warp 0 lane 0 issues the TMA loads of the X and
// h tiles and streams the weights; warp 1 owns the tensor memory and one lane
// issues every MMA; warps 2..9 are the epilogue, two warps per TMEM lane
// quadrant, each owning half of the state columns of its 32 rows.  The
// epilogue keeps its rows of h (FP32) in registers for the whole tile.
// Global traffic is whole tiles: h arrives by TMA (swizzled 32-column boxes
// placed in the last weight-ring stages before the weights need them), h'
// leaves by TMA from the X region (idle after phase 1), and d is staged
// row-major in the idle weight ring and leaves by one bulk store.
//
// Operands live in shared memory in the canonical K-major 128-byte-swizzle
// layout (8-row x 128-byte atoms): X arrives by a 2D tensor copy that applies
// the swizzle; h, r*h and h' are written by the epilogue; the weights come
// from a blob in which every chunk (<= 128 rows x 64 K-elements) is already
// stored as its shared-memory image, through a 6-stage bulk-copy ring.
// Every wait is bounded (2 s): on time-out the kernel sets
// DNNMG_DEVERR_TIMEOUT in the net's status word, drains what it started,
// frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <vector>

#include "common.cuh"
#include "ptx.cuh"

namespace dnnmg {
namespace {

constexpr int TM = 128;                 // patch rows per tile (UMMA M)
constexpr int NTH = 320;                // producer warp, MMA warp, 8 epilogue warps
constexpr int KC = 64;                  // K elements per chunk = one 128-byte swizzle row
constexpr int CHUNK = TM * KC * 2;      // 16 KB: one A chunk (128 rows x 64 K)
constexpr int SSZ = 2 * CHUNK;          // 32 KB weight-ring stage: up to 256 B rows x 64 K, or two K chunks
constexpr int NSTAGE = 3;
constexpr int MAX_ITEMS = 48;

enum { ITEM_D1 = 0, ITEM_D2X = 1, ITEM_D2H = 2, ITEM_D3 = 3 };

// One ring-stage fill of the schedule, as the MMA and producer threads read
// it (two 16-byte shared-memory loads): one or two K chunks of 64 of the
// same B rows (one accumulator block), stored one after the other.
//   first word  x: byte offset in the weight blob, y: bytes, z: instruction
//               descriptor (M = 128, N = rows), w: first TMEM column (bits
//               0-8) | accumulate (bit 9) | first h chunk of phase 1 (bit 10)
//               | two K chunks (bit 11) | rows = MMA N (bits 16-31)
//   second word x, y: byte offsets of the A chunks from the shared-memory
//               base, z: offset of the second B chunk in the stage
constexpr uint32_t SCHED_ACC = 1u << 9, SCHED_FIRST_H = 1u << 10, SCHED_PAIR = 1u << 11;

struct TcParams {
    int n_in, ldx, H, n_out, nfc, nxc, nhc, nxs, nitems, end1, end2, tmem_cols;
    const uint8_t *wblob;
    int *status;
    uint4 items[2 * MAX_ITEMS];
};

// ---------------------------------------------------------------- PTX helpers
using namespace ptx;

__device__ __forceinline__ void epilogue_sync() { asm volatile("bar.sync 1, %0;" ::"n"(NTH - 64) : "memory"); }
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

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 t = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&t);
}
// byte offset of 16-byte unit u (0..7) of row `row` in a 128B-swizzled chunk
__device__ __forceinline__ uint32_t swz(int row, int u) { return (uint32_t)(row * 128 + ((u ^ (row & 7)) << 4)); }
// Activations on the special-function unit: tanh.approx.f32 (PTX; relative
// error about 2^-11, well inside the BF16 operand rounding of this kernel)
// and the logistic function as 1/2 + tanh(x/2)/2.
__device__ __forceinline__ float tanh_fast(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sigm(float x) { return fmaf(0.5f, tanh_fast(0.5f * x), 0.5f); }

// Store 16 consecutive state columns c0..c0+15 of `row` as bf16 into the h chunks.
__device__ __forceinline__ void store_h16(uint8_t *sAh, int row, int c0, const float *v) {
    uint8_t *chunk = sAh + (c0 / KC) * CHUNK;
    const int u0 = (c0 % KC) / 8;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const float *w = v + 8 * u;
        *reinterpret_cast<uint4 *>(chunk + swz(row, u0 + u)) =
            make_uint4(pack_bf16(w[0], w[1]), pack_bf16(w[2], w[3]), pack_bf16(w[4], w[5]), pack_bf16(w[6], w[7]));
    }
}

template <int H>
__global__ void __launch_bounds__(NTH, 1)
k_gru_tc(const __grid_constant__ TcParams p, const __grid_constant__ CUtensorMap tmX,
         const __grid_constant__ CUtensorMap tmH, float *__restrict__ h, float *__restrict__ d, int P,
         const int *__restrict__ hrow) {
    constexpr int NH = H / 2;           // state columns per epilogue thread
    extern __shared__ uint8_t smem_raw[];
    // aligned by an offset from the shared-memory symbol itself, so that every
    // access through base stays a shared-memory access (no generic pointers)
    uint8_t *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t *sX = base;                                   // max(nxc, H/32) chunks
    uint8_t *sAh = sX + p.nxs * CHUNK;                    // nhc chunks
    uint8_t *sW = sAh + p.nhc * CHUNK;                    // NSTAGE stages
    uint64_t *bars = reinterpret_cast<uint64_t *>(sW + NSTAGE * SSZ);
    // barriers: full[NSTAGE], empty[NSTAGE], x_full, ah, d1, rh, d2, hn, d3, drain, h_full
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * NSTAGE + 9);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    uint4 *sched = reinterpret_cast<uint4 *>(bars + 2 * NSTAGE + 12);   // [2 nitems], 16-byte aligned

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int p0 = blockIdx.x * TM;
    // first row of this tile's state: its own rows, or (batched instances) the
    // tile's rows in a shared state pool
    const int hp0 = hrow ? __ldg(hrow + blockIdx.x) : p0;
    const uint32_t sX_u = smem_u32(sX), sAh_u = smem_u32(sAh), sW_u = smem_u32(sW);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + NSTAGE);
    const uint32_t x_full = smem_u32(bars + 2 * NSTAGE), ah_bar = x_full + 8, d1_bar = x_full + 16,
                   rh_bar = x_full + 24, d2_bar = x_full + 32, hn_bar = x_full + 40, d3_bar = x_full + 48,
                   drain_bar = x_full + 56, h_full = x_full + 64;
    constexpr int HB = H / 32;                 // 32-column boxes (16 KB) of the FP32 state
    uint8_t *sH = sW + NSTAGE * SSZ - HB * CHUNK;   // the state arrives at the end of the ring
    constexpr int HSTAGE = (NSTAGE * SSZ - HB * CHUNK) / SSZ;   // first ring stage it overlaps
    constexpr int NEPI = NTH - 64;   // epilogue threads

    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(x_full, 1);
        mbar_init(ah_bar, NEPI);
        mbar_init(d1_bar, 1);
        mbar_init(rh_bar, NEPI);
        mbar_init(d2_bar, 1);
        mbar_init(hn_bar, NEPI);
        mbar_init(d3_bar, 1);
        mbar_init(drain_bar, 1);
        mbar_init(h_full, 1);
        *abort_flag = 0;
        mbar_init_fence();
        fence_async_smem();
    }
    if (warp == 2)
        for (int i = lane; i < 2 * p.nitems; i += 32) sched[i] = p.items[i];
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(p.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- producer: X tile by TMA, weights through the ring
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(&tmX) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(&tmH) : "memory");
            expect_tx(x_full, (uint32_t)(p.nxc * CHUNK));
            for (int kc = 0; kc < p.nxc; ++kc) tma_load_2d(sX_u + kc * CHUNK, &tmX, kc * KC, p0, x_full);
            expect_tx(h_full, (uint32_t)(HB * CHUNK));
            for (int q = 0; q < HB; ++q) tma_load_2d(smem_u32(sH) + q * CHUNK, &tmH, 32 * q, hp0, h_full);
            int issued = 0;
            uint32_t s = 0, ph = 1;   // ring stage and the parity of its previous release
            for (int i = 0; i < p.nitems; ++i) {
                // the stages under the state wait until the epilogue has read it
                if (i == HSTAGE && !mbar_wait(ah_bar, 0, abort_flag)) break;
                const uint32_t eb = empty0 + 8 * s;
                if (i >= NSTAGE && !mbar_test(eb, ph) && !mbar_wait(eb, ph, abort_flag)) break;
                const uint4 it = sched[2 * i];
                expect_tx(full0 + 8 * s, it.y);
                bulk_load(sW_u + s * SSZ, p.wblob + it.x, it.y, full0 + 8 * s);
                issued = i + 1;
                if (++s == NSTAGE) {
                    s = 0;
                    ph ^= 1;
                }
            }
            if (*abort_flag) {
                // let every started copy land before the CTA may exit
                volatile int no_abort = 0;
                mbar_wait(x_full, 0, &no_abort);
                mbar_wait(h_full, 0, &no_abort);
                for (int i = issued - NSTAGE < 0 ? 0 : issued - NSTAGE; i < issued; ++i)
                    mbar_wait(full0 + 8 * (i % NSTAGE), (i / NSTAGE) & 1, &no_abort);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            bool ok = mbar_wait(x_full, 0, abort_flag);
            tc_after_sync();
            uint32_t s = 0, ph = 0;   // ring stage and the parity of its current fill
            const uint32_t base_u = smem_u32(base);
            for (int i = 0; ok && i < p.nitems; ++i) {
                const uint4 it = sched[2 * i], it2 = sched[2 * i + 1];
                if (i == p.end1) ok = mbar_wait(rh_bar, 0, abort_flag);
                if (ok && i == p.end2) ok = mbar_wait(hn_bar, 0, abort_flag);
                if (ok && (it.w & SCHED_FIRST_H)) ok = mbar_wait(ah_bar, 0, abort_flag);
                const uint32_t fb = full0 + 8 * s;
                if (ok && !mbar_test(fb, ph)) ok = mbar_wait(fb, ph, abort_flag);
                if (!ok) break;
                tc_after_sync();
                // K steps of 16 elements advance both start addresses by 32 bytes (2 descriptor units)
                const uint32_t dt = tmem + (it.w & 0x1FFu);
                {
                    const uint64_t ad = sdesc(base_u + it2.x), bd = sdesc(sW_u + s * SSZ);
                    umma(dt, ad, bd, it.z, (it.w & SCHED_ACC) ? 1u : 0u);
#pragma unroll
                    for (int k = 1; k < KC / 16; ++k) umma(dt, ad + 2 * k, bd + 2 * k, it.z, 1u);
                }
                if (it.w & SCHED_PAIR) {   // the second K chunk adds onto the first
                    const uint64_t ad = sdesc(base_u + it2.y), bd = sdesc(sW_u + s * SSZ + it2.z);
#pragma unroll
                    for (int k = 0; k < KC / 16; ++k) umma(dt, ad + 2 * k, bd + 2 * k, it.z, 1u);
                }
                tc_commit(empty0 + 8 * s);
                if (++s == NSTAGE) {
                    s = 0;
                    ph ^= 1;
                }
                if (i == p.end1 - 1) tc_commit(d1_bar);
                if (i == p.end2 - 1) tc_commit(d2_bar);
                if (i == p.nitems - 1) tc_commit(d3_bar);
            }
            // all issued MMAs must be complete before the CTA frees its resources
            tc_commit(drain_bar);
            volatile int no_abort = 0;
            mbar_wait(drain_bar, 0, &no_abort);
        }
    } else {
        // ---------------- epilogue: warps 2..9
        const int q = warp & 3;                   // TMEM lane quadrant of this warp
        const int half = (warp - 2) >> 2;         // which half of the state columns
        const int row = q * 32 + lane;
        const int gp = p0 + row;
        const bool valid = gp < P;
        const int c0 = half * NH;                 // first state column of this thread
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
        float hv[NH];
        bool ok = __all_sync(0xffffffffu, mbar_wait(h_full, 0, abort_flag));
        // h (FP32, swizzled 32-column boxes) of this row segment -> registers and -> bf16 operand
        {
#pragma unroll
            for (int i = 0; i < NH / 4; ++i) {
                const int c = c0 + 4 * i;
                const float4 t = *reinterpret_cast<const float4 *>(sH + (c / 32) * CHUNK + swz(row, (c % 32) / 4));
                hv[4 * i] = t.x; hv[4 * i + 1] = t.y; hv[4 * i + 2] = t.z; hv[4 * i + 3] = t.w;
            }
#pragma unroll
            for (int b = 0; b < NH / 16; ++b) store_h16(sAh, row, c0 + 16 * b, hv + 16 * b);
            // K-padding of the last h chunk (columns H .. 64 nhc - 1) must be zero:
            // the weights there are zero, but 0 * (stale NaN) is not
            if (half == 1)
                for (int c = H; c < p.nhc * KC; c += 8)
                    *reinterpret_cast<uint4 *>(sAh + (c / KC) * CHUNK + swz(row, (c % KC) / 8)) = make_uint4(0, 0, 0, 0);
            fence_async_smem();
            mbar_arrive(ah_bar);
        }
        ok = ok && __all_sync(0xffffffffu, mbar_wait(d1_bar, 0, abort_flag));
        tc_after_sync();
        if (ok) {
            // r * h -> operand
#pragma unroll
            for (int b = 0; b < NH / 16; ++b) {
                float rv[16], t[16];
                tmem_ld16(tl + H + c0 + 16 * b, rv);
#pragma unroll
                for (int i = 0; i < 16; ++i) t[i] = sigm(rv[i]) * hv[16 * b + i];
                store_h16(sAh, row, c0 + 16 * b, t);
            }
            fence_async_smem();
            tc_before_sync();
            mbar_arrive(rh_bar);
            ok = __all_sync(0xffffffffu, mbar_wait(d2_bar, 0, abort_flag));
            tc_after_sync();
        }
        if (ok) {
            // h' = z h + (1 - z) tanh(cand)
#pragma unroll
            for (int b = 0; b < NH / 16; ++b) {
                float cv[16], zv[16];
                tmem_ld16(tl + 2 * H + c0 + 16 * b, cv);
                tmem_ld16(tl + c0 + 16 * b, zv);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float z = sigm(zv[i]);
                    hv[16 * b + i] = z * hv[16 * b + i] + (1.0f - z) * tanh_fast(cv[i]);
                }
                store_h16(sAh, row, c0 + 16 * b, hv + 16 * b);
            }
            // h' (FP32) -> swizzled boxes in the X region (free since phase 1) for a TMA store
#pragma unroll
            for (int i = 0; i < NH / 4; ++i) {
                const int c = c0 + 4 * i;
                *reinterpret_cast<float4 *>(sX + (c / 32) * CHUNK + swz(row, (c % 32) / 4)) =
                    make_float4(hv[4 * i], hv[4 * i + 1], hv[4 * i + 2], hv[4 * i + 3]);
            }
            fence_async_smem();
            tc_before_sync();
            mbar_arrive(hn_bar);
        }
        // named barriers are passed by every epilogue warp, whatever its state
        epilogue_sync();
        if (ok && warp == 2 && lane == 0 && !*abort_flag) {
            for (int q = 0; q < HB; ++q) tma_store_2d(&tmH, 32 * q, hp0, sX_u + q * CHUNK);
            bulk_commit();
        }
        if (ok) {
            ok = __all_sync(0xffffffffu, mbar_wait(d3_bar, 0, abort_flag));
            tc_after_sync();
        }
        const int nv = min(TM, P - p0);
        const int rb = 4 * p.n_out, g16 = rb % 16 == 0 ? 1 : (rb % 8 == 0 ? 2 : 4);
        const int nbulk = nv - nv % g16;
        if (ok) {
            // d = W_fc h': blocks of 16 output columns split between the two halves,
            // staged row-major in the (now idle) weight ring, then one bulk store
            // of the tile's contiguous rows; rows past a 16-byte multiple go direct
            const int nb = p.nfc / 16;
            const int b0 = half ? (nb + 1) / 2 : 0, b1 = half ? nb : (nb + 1) / 2;
            float *stage = reinterpret_cast<float *>(sW) + (size_t)row * p.n_out;
            float *drow = d + (size_t)gp * p.n_out;
            for (int b = b0; b < b1; ++b) {
                float dv[16];
                tmem_ld16(tl + 16 * b, dv);
#pragma unroll
                for (int i = 0; i < 16; i += 2) {
                    const int c = 16 * b + i;
                    if (c < p.n_out) {
                        if (row < nbulk) *reinterpret_cast<float2 *>(stage + c) = make_float2(dv[i], dv[i + 1]);
                        else if (valid) { drow[c] = dv[i]; drow[c + 1] = dv[i + 1]; }
                    }
                }
            }
            fence_async_smem();
        }
        epilogue_sync();
        if (warp == 2 && lane == 0 && nbulk > 0 && !*abort_flag) {
            bulk_store(d + (size_t)p0 * p.n_out, sW_u, (uint32_t)(nbulk * rb));
            bulk_commit();
        }
        if (warp == 2 && lane == 0) bulk_wait_read();   // shared memory must outlive the stores
    }

    // ---------------- teardown
    if (tid == 0 && *abort_flag) atomicOr(p.status, DNNMG_DEVERR_TIMEOUT);
    tc_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
    }
}

// host-side byte offset of element (row, k) in a 128B-swizzled K-major chunk image
inline size_t swz_host(int row, int k) {
    return (size_t)row * 128 + (size_t)((((k / 8) ^ (row % 8)) * 16) + (k % 8) * 2);
}

size_t smem_bytes(const TcParams &p) {
    // operand chunks, ring, alignment slack, barriers and flags (256 B), schedule
    return (size_t)(p.nxs + p.nhc) * CHUNK + (size_t)NSTAGE * SSZ + 1024 + 256 + 2 * MAX_ITEMS * sizeof(uint4);
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

}  // namespace

bool tma_encode_tiled(CUtensorMap *map, CUtensorMapDataType type, unsigned rank, void *base, const cuuint64_t *dims,
                      const cuuint64_t *strides, const cuuint32_t *box) {
    if (!encode_fn()) return false;
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return encode_fn()(map, type, rank, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct TcNet {
    TcParams p;
};

// Builds the pre-swizzled weight blob and the chunk schedule; returns false if
// the shapes are outside what the kernel supports.
bool tc_prepare(Net &n, const double *Wx, const double *Uh, const double *Wfc) {
    const int H = n.H, n_in = n.n_in, n_out = n.n_out, ldx = n.ldx;
    const int nfc = round_up(n_out, 16);
    const int nxc = (ldx + KC - 1) / KC, nhc = (H + KC - 1) / KC;
    if (!(H == 32 || H == 64 || H == 96 || H == 128) || nfc > 2 * H) return false;
    if ((size_t)TM * n_out * 4 > (size_t)NSTAGE * SSZ || n_out % 2) return false;   // d staging in the ring
    if (!encode_fn()) return false;
    TcParams p;
    memset(&p, 0, sizeof p);
    p.n_in = n_in; p.ldx = ldx; p.H = H; p.n_out = n_out; p.nfc = nfc; p.nxc = nxc; p.nhc = nhc;
    p.nxs = nxc > H / 32 ? nxc : H / 32;
    // a ring-stage fill: K chunks kc0 (and kc0 + 1 if pair) of rows [r0, r0 + rows)
    // of one B matrix, accumulating into TMEM columns dcol ..
    struct HostItem {
        int off, bytes, rows, kind, kc0, pair, dcol;
    };
    std::vector<HostItem> items;
    std::vector<uint8_t> blob;
    auto add = [&](int kind, int kc0, bool pair, int r0, int rows, int dcol, auto value) {
        HostItem it{(int)blob.size(), 0, rows, kind, kc0, pair ? 1 : 0, dcol};
        for (int q = 0; q <= it.pair; ++q) {
            const size_t off = blob.size();
            blob.resize(off + (size_t)rows * 128, 0);
            for (int r = 0; r < rows; ++r)
                for (int k = 0; k < KC; ++k) {
                    const __nv_bfloat16 b = __float2bfloat16_rn((float)value(kc0 + q, r0 + r, k));
                    memcpy(blob.data() + off + swz_host(r, k), &b, 2);
                }
        }
        it.bytes = (int)blob.size() - it.off;
        items.push_back(it);
    };
    const bool pair_h = 2 * H * 128 <= SSZ, pair_fc = 2 * nfc * 128 <= SSZ, pair_zr = 2 * (2 * H) * 128 <= SSZ;
    auto wx = [&](int kc, int r, int k) -> double {   // W_x row r (z, r, candidate blocks), K chunk kc
        const int col = kc * KC + k;
        return col < n_in ? Wx[(size_t)r * n_in + col] : 0.0;
    };
    auto uh = [&](int kc, int r, int k) -> double {   // U_h row r, h chunk kc (counted after the X chunks)
        const int col = (kc - nxc) * KC + k;
        return col < H ? Uh[(size_t)r * H + col] : 0.0;
    };
    // phase 1: z and r pre-activations (one N = 2H block) over the X chunks,
    // the candidate's X part (N = H) interleaved, then the h chunks of z, r
    for (int kc = 0; kc < nxc; kc += (pair_zr && kc + 1 < nxc) ? 2 : 1) {
        const bool pr = pair_zr && kc + 1 < nxc;
        add(ITEM_D1, kc, pr, 0, 2 * H, 0, wx);
        const int last = kc + (pr ? 1 : 0);
        // candidate pairs end on odd chunks (or at the last X chunk)
        for (int c = kc; c <= last; ++c)
            if (c % 2 == 1 || c == nxc - 1) {
                const bool cp = c % 2 == 1;   // pair (c - 1, c)
                add(ITEM_D2X, cp ? c - 1 : c, cp, 0, H, 2 * H,
                    [&](int q, int r, int k) { return wx(q, 2 * H + r, k); });
            }
    }
    for (int kc = nxc; kc < nxc + nhc; kc += (pair_zr && kc + 1 < nxc + nhc) ? 2 : 1)
        add(ITEM_D1, kc, pair_zr && kc + 1 < nxc + nhc, 0, 2 * H, 0, uh);
    p.end1 = (int)items.size();
    // phase 2: the candidate's recurrent part on (r * h)
    for (int kc = nxc; kc < nxc + nhc; kc += (pair_h && kc + 1 < nxc + nhc) ? 2 : 1)
        add(ITEM_D2H, kc, pair_h && kc + 1 < nxc + nhc, 0, H, 2 * H,
            [&](int q, int r, int k) { return uh(q, 2 * H + r, k); });
    p.end2 = (int)items.size();
    // phase 3: the output layer on h'
    for (int kc = nxc; kc < nxc + nhc; kc += (pair_fc && kc + 1 < nxc + nhc) ? 2 : 1)
        add(ITEM_D3, kc, pair_fc && kc + 1 < nxc + nhc, 0, nfc, 0, [&](int q, int r, int k) -> double {
            const int col = (q - nxc) * KC + k;
            return (r < n_out && col < H) ? Wfc[(size_t)r * H + col] : 0.0;
        });
    p.nitems = (int)items.size();
    if (p.nitems > MAX_ITEMS) return false;
    int cols = 32;
    while (cols < 3 * H) cols *= 2;
    p.tmem_cols = cols;
    // schedule words; a fill accumulates unless it holds the first K chunk of
    // its output block within its phase (phase 2 always adds onto phase 1)
    bool seen_h = false;
    for (int i = 0; i < p.nitems; ++i) {
        const HostItem &it = items[i];
        bool acc = it.kind == ITEM_D2H;
        for (int j = i - 1; !acc && j >= 0; --j) {
            const bool same_phase = (j < p.end1) == (i < p.end1) && (j >= p.end2) == (i >= p.end2);
            acc = same_phase && items[j].dcol == it.dcol && items[j].kind == it.kind;
        }
        const bool first_h = i < p.end1 && it.kc0 + it.pair >= nxc && !seen_h;
        seen_h = seen_h || first_h;
        auto aoff = [&](int kc) { return (uint32_t)((kc < nxc ? kc : p.nxs + kc - nxc) * CHUNK); };
        p.items[2 * i] = make_uint4((uint32_t)it.off, (uint32_t)it.bytes, idesc_bf16(TM, it.rows),
                                    (uint32_t)it.dcol | (acc ? SCHED_ACC : 0u) | (first_h ? SCHED_FIRST_H : 0u) |
                                        (it.pair ? SCHED_PAIR : 0u) | ((uint32_t)it.rows << 16));
        p.items[2 * i + 1] = make_uint4(aoff(it.kc0), it.pair ? aoff(it.kc0 + 1) : 0u, (uint32_t)(it.rows * 128), 0u);
    }
    if (smem_bytes(p) > 227 * 1024) return false;
    void *dblob = nullptr;
    if (cudaMalloc(&dblob, blob.size()) != cudaSuccess) return false;
    if (cudaMemcpy(dblob, blob.data(), blob.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(dblob);
        return false;
    }
    p.wblob = static_cast<const uint8_t *>(dblob);
    p.status = n.d_status;
    n.tc = new TcNet{p};
    n.tc_weights = dblob;
    n.tc_bytes = blob.size();
    return true;
}

void tc_release(Net &n) {
    delete static_cast<TcNet *>(n.tc);
    n.tc = nullptr;
}

cudaError_t launch_gru_tc(const Net &n, const void *X, void *h, void *d, int P, cudaStream_t st) {
    return launch_gru_tc_rows(n, X, h, d, P, nullptr, P, st);
}

// hrow (device, may be null): per 128-row tile, the first row of its state in
// h, which then holds h_rows rows (a pool shared by batched instances).
cudaError_t launch_gru_tc_rows(const Net &n, const void *X, void *h, void *d, int P, const int *hrow, int h_rows,
                               cudaStream_t st) {
    const TcParams &p = static_cast<const TcNet *>(n.tc)->p;
    // X [P][ldx] bf16: boxes of 64 K-elements x 128 rows, 128-byte swizzle, zero fill outside
    CUtensorMap tm;
    const cuuint64_t dims[2] = {(cuuint64_t)p.ldx, (cuuint64_t)P};
    const cuuint64_t strides[1] = {(cuuint64_t)p.ldx * 2};
    const cuuint32_t box[2] = {(cuuint32_t)KC, (cuuint32_t)TM};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(X), dims, strides, box,
                             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    // h [P][H] fp32: boxes of 32 columns x 128 rows, 128-byte swizzle (load and store)
    CUtensorMap th;
    const cuuint64_t hdims[2] = {(cuuint64_t)p.H, (cuuint64_t)h_rows};
    const cuuint64_t hstrides[1] = {(cuuint64_t)p.H * 4};
    const cuuint32_t hbox[2] = {32, (cuuint32_t)TM};
    r = encode_fn()(&th, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h, hdims, hstrides, hbox, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    const size_t smem = smem_bytes(p);
    const int grid = (P + TM - 1) / TM;
    cudaError_t e;
#define DNNMG_LAUNCH_H(HH)                                                                                   \
    case HH:                                                                                                 \
        e = cudaFuncSetAttribute(k_gru_tc<HH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);       \
        if (e != cudaSuccess) return e;                                                                      \
        k_gru_tc<HH><<<grid, NTH, smem, st>>>(p, tm, th, (float *)h, (float *)d, P, hrow);                   \
        break;
    switch (p.H) {
        DNNMG_LAUNCH_H(32)
        DNNMG_LAUNCH_H(64)
        DNNMG_LAUNCH_H(96)
        DNNMG_LAUNCH_H(128)
        default: return cudaErrorInvalidValue;
    }
#undef DNNMG_LAUNCH_H
    return cudaGetLastError();
}

}  // namespace dnnmg

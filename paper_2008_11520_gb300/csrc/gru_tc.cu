// S4 on the 5th-generation tensor cores (tcgen05, sm_103a): GRU cell of
// Eq. gru (reset gate before U_h, no biases) and the output layer, BF16
// operands, FP32 accumulators in tensor memory.
//
// One persistent CTA per SM walks 128-patch tiles (one TMEM lane per patch
// row).  Per tile, with the z, r and candidate pre-activations accumulating
// in TMEM columns [0,H), [H,2H), [2H,3H):
//   X groups:  for each 64-column chunk of X:
//              z = X W_z^T, r = X W_r^T, c = X W_h^T        (accumulating over the chunks)
//   H groups:  z += h U_z^T, r += h U_r^T                  (h as BF16, written by the epilogue)
//   epilogue:  A_h <- bf16(sig(r) * h)
//   C groups:  c += (r * h) U_h^T
//   epilogue:  h' = z h + (1 - z) tanh(c) with z = sig(.); h <- h' (FP32), A_h <- bf16(h')
//   F groups:  d = h' W_fc^T                                (columns [0, nfc), in pieces of <= 128)
//   epilogue:  d -> global
//
// The copies one thread issues are served one after the other, at about the
// same time each whatever their size (up to tens of KB), while copies from
// different warps proceed side by side.  So every operand arrives in few,
// large copies, spread over three copy warps: the tile's X as one 3D tensor
// copy of its whole 64-column chunks (chunk stride 128 B, so the box lands as
// the chunks' 128-byte-swizzled images one after the other) plus a 2D copy of
// a ragged last chunk, into its own region; before it, in the same region, the
// tile's FP32 state h (one 3D copy of its 32-column boxes), which the epilogue
// moves into registers; the three weight slices of an X chunk as one copy
// into one of two alternating stages (one warp per stage); U_z and U_r, U_h,
// and W_fc as one copy each.  The weights come from a blob that holds every
// slice as its shared-memory image, in the order of the copies.  The weight
// region is reused in turn for those copies and for h' (swizzled 32-column
// boxes, one 3D tensor store); d is staged row-major from the start of A_h on
// into it and leaves by one bulk store of the tile's contiguous rows.  The
// next tile's stage 0 fills as soon as the output layer has read W_fc, its
// stage 1 once d has left.
//
// Warp roles (384 threads): warps 0 and 11 copy the weights (stage 0, U_h,
// W_fc; stage 1, U_z U_r), warp 10 the state and X tiles; warp 1 owns the
// tensor memory and one lane issues every MMA; warps 2..9 are the epilogue,
// two warps per TMEM lane quadrant, each owning half of the state columns of
// its 32 rows, kept in registers (FP32) from the state copy until h' is
// formed.
//
// Operands live in shared memory in the canonical K-major 128-byte-swizzle
// layout (8-row x 128-byte atoms).  Every wait is bounded (2 s): on time-out
// the kernel sets DNNMG_DEVERR_TIMEOUT in the net's status word, drains what
// it started, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "ptx.cuh"

namespace dnnmg {
namespace {

constexpr int TM = 128;                 // patch rows per tile (UMMA M)
constexpr int NTH = 384;                // copy warp, MMA warp, 8 epilogue warps, 2 copy warps
constexpr int NEPI = 256;               // epilogue threads (warps 2..9)
constexpr int KC = 64;                  // K elements per chunk = one 128-byte swizzle row
constexpr int SLOT = TM * KC * 2;       // 16 KB: one 128-row x 64-K BF16 chunk
constexpr int SMEM_LIMIT = 227 * 1024;
constexpr int SMEM_EXTRA = 1024 + 512;  // alignment slack; barriers, TMEM address, abort flag

// Shapes, shared-memory layout and weight-blob offsets.  Regions: X [0, xb),
// A_h [xb, xb + ahb), W [xb + ahb, + wb).  Inside W: X-group stage 1 at 0,
// stage 0 at o0 (clear of the h' boxes at [0, hs) and of d, which runs from
// the start of A_h into W); U_z/U_r at 0; U_h and then W_fc at o0.  Stage 0
// of the next tile can therefore fill as soon as the output layer has read
// W_fc, and stage 1 once d has left.
struct TcParams {
    int n_in, ldx, H, n_out, nfc, nxc, nhc, nf, nfull;   // nfull: whole 64-column chunks of X
    int xb, ahb, wb, S, hw, cw, hs, fw, o0, tmem_cols;
    uint32_t blob_x, blob_h, blob_c, blob_f;
    const uint8_t *wblob;
    int *status;
};

// ---------------------------------------------------------------- PTX helpers
using namespace ptx;

__device__ __forceinline__ void epilogue_sync() { asm volatile("bar.sync 1, %0;" ::"n"(NEPI) : "memory"); }
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
// One 64-K chunk: four K steps of 16; each advances both start addresses by 32 bytes (2 descriptor units).
__device__ __forceinline__ void umma_chunk(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, bool acc) {
    umma(dtmem, a, b, idesc, acc ? 1u : 0u);
#pragma unroll
    for (int k = 1; k < KC / 16; ++k) umma(dtmem, a + 2 * k, b + 2 * k, idesc, 1u);
}
// 16 consecutive 32-bit TMEM columns of this warp's 32 lanes (one per thread),
// issued without waiting; one tcgen05.wait::ld then covers several loads
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

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
    uint8_t *chunk = sAh + (c0 / KC) * SLOT;
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
k_gru_tc(const __grid_constant__ TcParams p, const __grid_constant__ CUtensorMap tmX3,
         const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmH3, float *__restrict__ d,
         int P, const int *__restrict__ hrow) {
    constexpr int NH = H / 2;           // state columns per epilogue thread
    extern __shared__ uint8_t smem_raw[];
    // aligned by an offset from the shared-memory symbol itself, so that every
    // access through base stays a shared-memory access (no generic pointers)
    uint8_t *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t *sX = base;
    uint8_t *sAh = sX + p.xb;
    uint8_t *sW = sAh + p.ahb;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sW + p.wb);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 20);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (P + TM - 1) / TM;
    const uint32_t x_u = smem_u32(sX), ah_u = smem_u32(sAh), w_u = smem_u32(sW);
    const uint32_t b0 = smem_u32(bars);
    // barriers: X tile landed / free, weight stages full[2] / empty[2], U_z U_r, U_h, W_fc
    // landed, weight region free (d has left), the MMA <-> epilogue hand-offs, and the
    // state landed in / read out of the X region
    const uint32_t x_full = b0, x_free = b0 + 8, wst_full = b0 + 16, wst_empty = b0 + 32, wh_full = b0 + 48,
                   wc_full = b0 + 56, wf_full = b0 + 64, w_free = b0 + 72, e0_bar = b0 + 80, d1_bar = b0 + 88,
                   rh_bar = b0 + 96, d2_bar = b0 + 104, hn_bar = b0 + 112, d3_bar = b0 + 120, tfree_bar = b0 + 128,
                   drain_bar = b0 + 136, hx_full = b0 + 144, hx_read = b0 + 152;

    if (tid == 0) {
        // the epilogue hand-offs count every epilogue thread, the rest one arrival
        for (int i = 0; i < 20; ++i) {
            const uint32_t bar = b0 + 8 * i;
            const bool epi = bar == e0_bar || bar == rh_bar || bar == hn_bar || bar == tfree_bar || bar == hx_read;
            mbar_init(bar, epi ? NEPI : 1);
        }
        *abort_flag = 0;
        mbar_init_fence();
        fence_async_smem();
    }
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
    volatile int no_abort = 0;

    if ((warp == 0 || warp == 11) && lane == 0) {
        // ---------------- weight copies: warp 0 fills stage 0, then U_h and W_fc;
        // warp 11 fills stage 1, then U_z U_r
        const int s = warp == 0 ? 0 : 1;
        const uint32_t sb = s == 0 ? w_u + p.o0 : w_u;   // this warp's stage
        uint32_t cs = 0;                    // fills of this warp's stage so far
        uint32_t nh = 0, nc = 0, nf = 0;    // U_z U_r, U_h and W_fc copies issued
        bool ok = true;
        auto stage_free = [&]() {           // the latest fill of the stage has been consumed
            return cs == 0 || mbar_wait(wst_empty + 8 * s, (cs - 1) & 1, abort_flag);
        };
        int it = 0;
        for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++it) {
            const uint32_t par = it & 1;
            // the previous tile's W_fc has been read (stage 0), or its d has left (stage 1)
            if (it > 0 && !(ok = mbar_wait(s == 0 ? d3_bar : w_free, par ^ 1, abort_flag))) break;
            for (int kc = s; ok && kc < p.nxc; kc += 2) {
                if (!(ok = stage_free())) break;
                expect_tx(wst_full + 8 * s, (uint32_t)p.S);
                bulk_load(sb, p.wblob + p.blob_x + (size_t)kc * p.S, (uint32_t)p.S, wst_full + 8 * s);
                ++cs;
            }
            // the stage's last fill consumed, its place takes U_z U_r (stage 1) or U_h (stage 0)
            if (!ok || !(ok = stage_free())) break;
            if (s == 1) {
                expect_tx(wh_full, (uint32_t)p.hw);
                bulk_load(w_u, p.wblob + p.blob_h, (uint32_t)p.hw, wh_full);
                ++nh;
            } else {
                expect_tx(wc_full, (uint32_t)p.cw);
                bulk_load(sb, p.wblob + p.blob_c, (uint32_t)p.cw, wc_full);
                ++nc;
                // W_fc over U_h's place once the C groups are done
                if (!(ok = mbar_wait(d2_bar, par, abort_flag))) break;
                expect_tx(wf_full, (uint32_t)p.fw);
                bulk_load(sb, p.wblob + p.blob_f, (uint32_t)p.fw, wf_full);
                ++nf;
            }
        }
        // let every started copy land before the CTA may exit (all have been
        // consumed unless something aborted)
        if (cs) mbar_wait(wst_full + 8 * s, (cs - 1) & 1, &no_abort);
        if (nh) mbar_wait(wh_full, (nh - 1) & 1, &no_abort);
        if (nc) mbar_wait(wc_full, (nc - 1) & 1, &no_abort);
        if (nf) mbar_wait(wf_full, (nf - 1) & 1, &no_abort);
    } else if (warp == 10 && lane == 0) {
        // ---------------- state and X into the X region: a tile's h (read out by
        // the epilogue), then its X, each time once the previous X groups are done
        prefetch_tensormap(&tmX3);
        prefetch_tensormap(&tmX);
        prefetch_tensormap(&tmH3);
        uint32_t nhx = 0, nxx = 0;   // state and X copies issued
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            if (nxx > 0 && !mbar_wait(x_free, (nxx - 1) & 1, abort_flag)) break;
            expect_tx(hx_full, (uint32_t)p.H * 4 * TM);
            tma_load_3d(x_u, &tmH3, 0, hrow ? __ldg(hrow + tile) : tile * TM, 0, hx_full);
            ++nhx;
            if (!mbar_wait(hx_read, (nhx - 1) & 1, abort_flag)) break;
            expect_tx(x_full, (uint32_t)p.nxc * SLOT);
            if (p.nfull > 0) tma_load_3d(x_u, &tmX3, 0, tile * TM, 0, x_full);
            if (p.nfull < p.nxc) tma_load_2d(x_u + p.nfull * SLOT, &tmX, p.nfull * KC, tile * TM, x_full);
            ++nxx;
        }
        if (nhx) mbar_wait(hx_full, (nhx - 1) & 1, &no_abort);
        if (nxx) mbar_wait(x_full, (nxx - 1) & 1, &no_abort);
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idH = idesc_bf16(TM, H);
            const int r0 = p.nfc < TM ? p.nfc : TM;
            const uint32_t idF0 = idesc_bf16(TM, r0), idF1 = idesc_bf16(TM, p.nfc > TM ? p.nfc - TM : 16);
            const uint32_t slice = (uint32_t)H * 128;   // bytes of one H-row weight slice
            uint32_t us[2] = {0, 0};                     // fills of each X-group stage consumed
            bool ok = true;
            int it = 0;
            for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++it) {
                const uint32_t par = it & 1;
                ok = mbar_wait(x_full, par, abort_flag);
                // the previous tile's accumulators must have been read
                if (ok && it > 0) ok = mbar_wait(tfree_bar, par ^ 1, abort_flag);
                tc_after_sync();
                // X groups
                for (int kc = 0; ok && kc < p.nxc; ++kc) {
                    const int s = kc & 1;
                    if (!(ok = mbar_wait(wst_full + 8 * s, us[s] & 1, abort_flag))) break;
                    tc_after_sync();
                    const uint64_t a = sdesc(x_u + kc * SLOT);
                    const uint32_t wb = s == 0 ? w_u + p.o0 : w_u;
#pragma unroll
                    for (int g = 0; g < 3; ++g) umma_chunk(tmem + g * H, a, sdesc(wb + g * slice), idH, kc > 0);
                    tc_commit(wst_empty + 8 * s);
                    ++us[s];
                }
                if (!ok) break;
                tc_commit(x_free);
                // H groups on h
                ok = mbar_wait(e0_bar, par, abort_flag) && mbar_wait(wh_full, par, abort_flag);
                tc_after_sync();
                for (int j = 0; ok && j < p.nhc; ++j) {
                    const uint64_t a = sdesc(ah_u + j * SLOT);
#pragma unroll
                    for (int g = 0; g < 2; ++g)
                        umma_chunk(tmem + g * H, a, sdesc(w_u + (2 * j + g) * slice), idH, true);
                }
                if (ok) tc_commit(d1_bar);
                // C groups on r * h
                ok = ok && mbar_wait(rh_bar, par, abort_flag) && mbar_wait(wc_full, par, abort_flag);
                tc_after_sync();
                for (int j = 0; ok && j < p.nhc; ++j)
                    umma_chunk(tmem + 2 * H, sdesc(ah_u + j * SLOT), sdesc(w_u + p.o0 + j * slice), idH, true);
                if (ok) tc_commit(d2_bar);
                // F groups on h'
                ok = ok && mbar_wait(hn_bar, par, abort_flag) && mbar_wait(wf_full, par, abort_flag);
                tc_after_sync();
                for (int j = 0; ok && j < p.nhc; ++j) {
                    const uint64_t a = sdesc(ah_u + j * SLOT);
                    const uint32_t fb = w_u + p.o0 + (uint32_t)(j * p.nfc * 128);
                    umma_chunk(tmem, a, sdesc(fb), idF0, j > 0);
                    if (p.nf > 1) umma_chunk(tmem + TM, a, sdesc(fb + r0 * 128), idF1, j > 0);
                }
                if (ok) tc_commit(d3_bar);
            }
            // all issued MMAs must be complete before the CTA frees its resources
            tc_commit(drain_bar);
            mbar_wait(drain_bar, 0, &no_abort);
        }
    } else if (warp >= 2 && warp < 2 + NEPI / 32) {
        // ---------------- epilogue: warps 2..9 (the other lanes of the copy warps idle)
        const int q = warp & 3;                   // TMEM lane quadrant of this warp
        const int half = (warp - 2) >> 2;         // which half of the state columns
        const int row = q * 32 + lane;
        const int c0 = half * NH;                 // first state column of this thread
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
        float hv[NH];
        // this row's state columns from the boxes in the X region (zero past the last patch)
        auto read_h = [&]() {
#pragma unroll
            for (int i = 0; i < NH / 4; ++i) {
                const int c = c0 + 4 * i;
                const float4 x = *reinterpret_cast<const float4 *>(sX + (c / 32) * SLOT + swz(row, (c % 32) / 4));
                hv[4 * i] = x.x; hv[4 * i + 1] = x.y; hv[4 * i + 2] = x.z; hv[4 * i + 3] = x.w;
            }
        };
        // the state of the next tile: wait for its copy, read it out, let X come in
        auto take_h = [&](uint32_t phase) -> bool {
            if (!__all_sync(0xffffffffu, mbar_wait_inl(hx_full, phase & 1, abort_flag))) return false;
            read_h();
            fence_async_smem();
            mbar_arrive(hx_read);
            return true;
        };
        bool ok = true;
        int it = 0;
        if ((int)blockIdx.x < ntiles) ok = take_h(0);
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const uint32_t par = it & 1;
            const int p0 = tile * TM, gp = p0 + row;
            const bool valid = gp < P;
            const int hp0 = hrow ? __ldg(hrow + tile) : p0;
            // the previous tile's d (staged from the start of A_h) has left
            if (it > 0) epilogue_sync();
            if (ok) {
                // h -> BF16 operand
#pragma unroll
                for (int b = 0; b < NH / 16; ++b) store_h16(sAh, row, c0 + 16 * b, hv + 16 * b);
                // K-padding of the last h chunk (columns H .. 64 nhc - 1) must be zero:
                // the weights there are zero, but 0 * (stale NaN) is not
                if (half == 1)
                    for (int c = H; c < p.nhc * KC; c += 8)
                        *reinterpret_cast<uint4 *>(sAh + (c / KC) * SLOT + swz(row, (c % KC) / 8)) = make_uint4(0, 0, 0, 0);
                fence_async_smem();
                mbar_arrive(e0_bar);
            }
            ok = ok && __all_sync(0xffffffffu, mbar_wait_inl(d1_bar, par, abort_flag));
            tc_after_sync();
            if (ok) {
                // r * h -> operand
#pragma unroll
                for (int b = 0; b < NH / 16; ++b) {
                    uint32_t rv[16];
                    float t[16];
                    tmem_ld16_issue(tl + H + c0 + 16 * b, rv);
                    tmem_wait();
#pragma unroll
                    for (int i = 0; i < 16; ++i) t[i] = sigm(__uint_as_float(rv[i])) * hv[16 * b + i];
                    store_h16(sAh, row, c0 + 16 * b, t);
                }
                fence_async_smem();
                tc_before_sync();
                mbar_arrive(rh_bar);
            }
            ok = ok && __all_sync(0xffffffffu, mbar_wait_inl(d2_bar, par, abort_flag));
            tc_after_sync();
            if (ok) {
                // h' = z h + (1 - z) tanh(cand)
#pragma unroll
                for (int b = 0; b < NH / 16; ++b) {
                    uint32_t cv[16], zv[16];
                    tmem_ld16_issue(tl + 2 * H + c0 + 16 * b, cv);
                    tmem_ld16_issue(tl + c0 + 16 * b, zv);
                    tmem_wait();
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float z = sigm(__uint_as_float(zv[i]));
                        hv[16 * b + i] = z * hv[16 * b + i] + (1.0f - z) * tanh_fast(__uint_as_float(cv[i]));
                    }
                    store_h16(sAh, row, c0 + 16 * b, hv + 16 * b);
                }
                // h' (FP32) -> swizzled 32-column boxes at the start of the weight region
#pragma unroll
                for (int i = 0; i < NH / 4; ++i) {
                    const int c = c0 + 4 * i;
                    *reinterpret_cast<float4 *>(sW + (c / 32) * SLOT + swz(row, (c % 32) / 4)) =
                        make_float4(hv[4 * i], hv[4 * i + 1], hv[4 * i + 2], hv[4 * i + 3]);
                }
                fence_async_smem();
                tc_before_sync();
                mbar_arrive(hn_bar);
            }
            // named barriers are passed by every epilogue warp, whatever its state
            epilogue_sync();
            if (ok && tid == 64 && !*abort_flag) {
                tma_store_3d(&tmH3, 0, hp0, 0, w_u);
                bulk_commit();
            }
            // the next tile's state, read out of the X region while this tile finishes
            if (ok && tile + (int)gridDim.x < ntiles) ok = take_h((uint32_t)it + 1);
            ok = ok && __all_sync(0xffffffffu, mbar_wait_inl(d3_bar, par, abort_flag));
            tc_after_sync();
            if (tid == 64) bulk_wait_read();   // h' has left the weight region
            epilogue_sync();
            const int nv = min(TM, P - p0);
            const int rb = 4 * p.n_out, g16 = rb % 16 == 0 ? 1 : (rb % 8 == 0 ? 2 : 4);
            const int nbulk = nv - nv % g16;
            if (ok) {
                // d = W_fc h': blocks of 16 output columns split between the two halves,
                // staged row-major from the start of A_h (free since the F groups), then
                // one bulk store of the tile's contiguous rows; rows past a 16-byte
                // multiple go direct
                const int nb = p.nfc / 16;
                const int b0 = half ? (nb + 1) / 2 : 0, b1 = half ? nb : (nb + 1) / 2;
                float *stage = reinterpret_cast<float *>(sAh) + (size_t)row * p.n_out;
                float *drow = d + (size_t)gp * p.n_out;
                for (int b = b0; b < b1; b += 2) {
                    // two 16-column blocks per wait (the second only if this half has it)
                    uint32_t dv[2][16];
                    const bool two = b + 1 < b1;
                    tmem_ld16_issue(tl + 16 * b, dv[0]);
                    if (two) tmem_ld16_issue(tl + 16 * (b + 1), dv[1]);
                    tmem_wait();
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        if (k == 1 && !two) break;
#pragma unroll
                        for (int i = 0; i < 16; i += 2) {
                            const int c = 16 * (b + k) + i;
                            const float x0 = __uint_as_float(dv[k][i]), x1 = __uint_as_float(dv[k][i + 1]);
                            if (c < p.n_out) {
                                if (row < nbulk) *reinterpret_cast<float2 *>(stage + c) = make_float2(x0, x1);
                                else if (valid) { drow[c] = x0; drow[c + 1] = x1; }
                            }
                        }
                    }
                }
                // the accumulators are free for the next tile
                tc_before_sync();
                mbar_arrive(tfree_bar);
                fence_async_smem();
            }
            epilogue_sync();
            if (tid == 64) {
                if (ok && nbulk > 0 && !*abort_flag) {
                    bulk_store(d + (size_t)p0 * p.n_out, ah_u, (uint32_t)(nbulk * rb));
                    bulk_commit();
                }
                bulk_wait_read();   // d has left: stage 1 and A_h are free again
                mbar_arrive(w_free);
            }
        }
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
    // X, A_h and weight regions, alignment slack, barriers and flags
    return (size_t)p.xb + (size_t)p.ahb + (size_t)p.wb + SMEM_EXTRA;
}

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
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

// Builds the pre-swizzled weight blob and the shared-memory layout; returns
// false if the shapes are outside what the kernel supports.
bool tc_prepare(Net &n, const double *Wx, const double *Uh, const double *Wfc) {
    const int H = n.H, n_in = n.n_in, n_out = n.n_out, ldx = n.ldx;
    const int nfc = round_up(n_out, 16);
    const int nxc = (ldx + KC - 1) / KC, nhc = (H + KC - 1) / KC, nf = (nfc + TM - 1) / TM;
    if (!(H == 32 || H == 64 || H == 96 || H == 128) || nf > 2 || n_out % 2) return false;
    if (!encode_fn()) return false;
    TcParams p;
    memset(&p, 0, sizeof p);
    p.n_in = n_in; p.ldx = ldx; p.H = H; p.n_out = n_out; p.nfc = nfc; p.nxc = nxc; p.nhc = nhc; p.nf = nf;
    p.nfull = ldx / KC;
    const int slice = H * 128;            // one H-row weight slice of a 64-K chunk
    p.xb = std::max(nxc * SLOT, H * 4 * TM);   // X, or the FP32 state before it
    p.ahb = nhc * SLOT;
    p.S = 3 * slice;                      // an X chunk's z, r, candidate slices
    p.hw = 2 * slice * nhc;               // U_z, U_r
    p.cw = slice * nhc;                   // U_h
    p.fw = nfc * 128 * nhc;               // W_fc
    p.hs = H * 4 * TM;                    // h' boxes
    const int ds = TM * 4 * n_out;        // d rows, from the start of A_h
    p.o0 = round_up(std::max({p.S, p.hs, ds - p.ahb}), 1024);
    p.wb = p.o0 + std::max({p.S, p.cw, p.fw});
    if (p.hw > p.o0) return false;        // U_z U_r must stay clear of stage 0
    if (smem_bytes(p) > (size_t)SMEM_LIMIT) return false;
    int cols = 32;
    while (cols < 3 * H || cols < nfc) cols *= 2;
    p.tmem_cols = cols;
    // slice images in copy order; an image holds `rows` rows of one matrix,
    // 64 K-elements each, in the swizzled K-major layout
    std::vector<uint8_t> blob;
    auto add = [&](int rows, auto value) {
        const size_t off = blob.size();
        blob.resize(off + (size_t)rows * 128, 0);
        for (int r = 0; r < rows; ++r)
            for (int k = 0; k < KC; ++k) {
                const __nv_bfloat16 b = __float2bfloat16_rn((float)value(r, k));
                memcpy(blob.data() + off + swz_host(r, k), &b, 2);
            }
    };
    // gate g of W_x (z, r, candidate) on X chunk kc; of U_h on h chunk j
    auto wx = [&](int g, int kc) {
        return [=](int r, int k) -> double {
            const int col = kc * KC + k;
            return col < n_in ? Wx[(size_t)(g * H + r) * n_in + col] : 0.0;
        };
    };
    auto uh = [&](int g, int j) {
        return [=](int r, int k) -> double {
            const int col = j * KC + k;
            return col < H ? Uh[(size_t)(g * H + r) * H + col] : 0.0;
        };
    };
    p.blob_x = 0;
    for (int kc = 0; kc < nxc; ++kc)
        for (int g = 0; g < 3; ++g) add(H, wx(g, kc));
    p.blob_h = (uint32_t)blob.size();
    for (int j = 0; j < nhc; ++j)
        for (int g = 0; g < 2; ++g) add(H, uh(g, j));
    p.blob_c = (uint32_t)blob.size();
    for (int j = 0; j < nhc; ++j) add(H, uh(2, j));
    p.blob_f = (uint32_t)blob.size();
    for (int j = 0; j < nhc; ++j)
        for (int f = 0; f < nf; ++f) {
            const int r0 = f * TM, rows = std::min(nfc - r0, TM);
            add(rows, [=](int r, int k) -> double {
                const int row = r0 + r, col = j * KC + k;
                return (row < n_out && col < H) ? Wfc[(size_t)row * H + col] : 0.0;
            });
        }
    if (blob.size() != (size_t)p.blob_f + p.fw) return false;
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
    if (P <= 0) return cudaSuccess;
    const cuuint32_t estr[3] = {1, 1, 1};
    auto encode = [&](CUtensorMap *m, CUtensorMapDataType ty, unsigned rank, const void *ptr, const cuuint64_t *dims,
                      const cuuint64_t *strides, const cuuint32_t *box) {
        return encode_fn()(m, ty, rank, const_cast<void *>(ptr), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    // X [P][ldx] bf16, 128-byte swizzle, zero fill outside.  3D view (k in chunk,
    // row, chunk) with the chunk stride (128 B) inside the row stride: one box of
    // the whole chunks lands as their images one after the other; a ragged last
    // chunk comes by a 2D box of 64 columns.
    CUtensorMap tmX3, tmX;
    memset(&tmX3, 0, sizeof tmX3);
    if (p.nfull > 0) {
        const cuuint64_t dims[3] = {(cuuint64_t)KC, (cuuint64_t)P, (cuuint64_t)p.nfull};
        const cuuint64_t strides[2] = {(cuuint64_t)p.ldx * 2, (cuuint64_t)KC * 2};
        const cuuint32_t box[3] = {(cuuint32_t)KC, (cuuint32_t)TM, (cuuint32_t)p.nfull};
        if (!encode(&tmX3, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, X, dims, strides, box)) return cudaErrorInvalidValue;
    }
    {
        const cuuint64_t dims[2] = {(cuuint64_t)p.ldx, (cuuint64_t)P};
        const cuuint64_t strides[1] = {(cuuint64_t)p.ldx * 2};
        const cuuint32_t box[2] = {(cuuint32_t)KC, (cuuint32_t)TM};
        if (!encode(&tmX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, X, dims, strides, box)) return cudaErrorInvalidValue;
    }
    // h [h_rows][H] fp32 as (column in box, row, box) with 32-column boxes: the
    // state copy and the h' store, one box of all H / 32 boxes each
    CUtensorMap tmH3;
    {
        const cuuint64_t dims[3] = {32, (cuuint64_t)h_rows, (cuuint64_t)(p.H / 32)};
        const cuuint64_t strides[2] = {(cuuint64_t)p.H * 4, 128};
        const cuuint32_t box[3] = {32, (cuuint32_t)TM, (cuuint32_t)(p.H / 32)};
        if (!encode(&tmH3, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, h, dims, strides, box)) return cudaErrorInvalidValue;
    }
    const size_t smem = smem_bytes(p);
    // persistent: one CTA per SM (the shared memory allows no second), tiles strided over the grid
    const int grid = std::min((P + TM - 1) / TM, sm_count());
    cudaError_t e;
#define DNNMG_LAUNCH_H(HH)                                                                                   \
    case HH:                                                                                                 \
        e = cudaFuncSetAttribute(k_gru_tc<HH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);       \
        if (e != cudaSuccess) return e;                                                                      \
        k_gru_tc<HH><<<grid, NTH, smem, st>>>(p, tmX3, tmX, tmH3, (float *)d, P, hrow);                      \
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

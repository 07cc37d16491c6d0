// S2 + S3 of the correction step on the all-fluid tiles, in closed form.
//
// Inside the step the fine field is x~ = P x_c, and on a tile whose whole
// neighbourhood is fluid no Dirichlet value modifies it, so every component
// of x~ is bilinear on each coarse cell (the nested Q1 spaces of Sec. 3.4).
// Two things follow for the residual r = b_f - A(x~) of Eq. nonlinearshort:
//
//  * The local projection term of Eq. disc:ns vanishes.  Its projection
//    patches are 2 x 2 fine cells aligned to even fine indices, so for K >= 1
//    each lies inside one coarse cell, where p is bilinear and the projection
//    reproduces it: p - pi p = 0.
//  * Every other term is an integral of a polynomial of the coarse cells'
//    values against the hat function of the fine node.  Split the node's
//    support into its four quadrants (one fine cell each); a quadrant lies in
//    one coarse cell, where u = u_i + u_x s + u_y t + u_xy s t in coordinates
//    (s, t) centred on the node.  The integrals are then sums of products of
//    the 1D moments of the hat over a half support, int s^n l(s) ds:
//    h/2, +-h^2/6, h^3/12 for n = 0, 1, 2.  (The 2 x 2 Gauss rule of the
//    assembly is exact for these integrands, so this is the same quantity.)
//    Quadrants that share a coarse cell are merged: over a full support the
//    odd moments cancel and the even ones are h and h^3/6.
//
// A node strictly inside a coarse cell (the usual case) therefore costs a
// few products of its values and derivatives; nodes on coarse cell edges sum
// two or four one-sided parts.  The tile layout matches the general kernel
// (32 x 16 fine cells); tiles without the all-fluid flag are left to it.
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace dnnmg {
namespace {

// A CTA takes two horizontally adjacent 32 x 16-cell tiles of the general
// kernel (64 x 16 fine cells), so the column the two share is computed once.
constexpr int CF_TXC = 64, CF_TYC = 16;               // fine cells per block
constexpr int CF_NYN = CF_TYC + 1;                    // node rows of a block
constexpr int CF_RXP = 68;                            // residual row pitch (elements)
constexpr int CF_RPL = CF_NYN * CF_RXP;               // residual plane (elements)

// Moment products of one kind of support (full in both directions, half in
// x, half in y, half in both; positive sides, the kernel applies the signs)
// with the equation's factors folded in.  x0, x1, x2 are the x moments of
// the hat (h, 0, h^3/6 over the full support; h/2, h^2/6, h^3/12 over a
// half), y0, y1, y2 likewise, and m_ab = x_a y_b:
//   C_ab = m_ab / 2      convection, 1/2 (v.grad v, phi)
//   M00 = m00 / k        mass (1/k)(v, phi)
//   MD01 = m01 / k - nu/2 x0, MD10 = m10 / k - nu/2 y0,
//   MD11 = m11 / k - nu/2 (x1 + y1)     mass and diffusion (nu/2)(grad v, grad phi)
//   m00, m01, m10, x0, y0, x1, y1       pressure gradient and divergence
struct Kset {
    float C00, C01, C10, C11, C02, C20, C12, C21;
    float M00, MD01, MD10, MD11;
    float m00, m01, m10, x0, y0, x1, y1;
};

// Per-mesh constants of the closed form (FP32).
struct CfCoef {
    float iHx, iHy, iHxy;          // 1 / coarse spacing, 1 / (Hx Hy)
    float hx, hy;                  // fine spacing
    float Hx, Hy;                  // coarse spacing
    Kset ff, hf, fh, hh;           // full / half support in x, then y
    float q_over_nu;               // Peclet scale
    float geo[12];                 // patch geometry features
};

// Derivatives at the node of one coarse cell's bilinear field: d/dx, d/dy, d2/dxdy.
struct D3 {
    float x, y, xy;
};

template <int SX, int SY> __device__ __forceinline__ const Kset &kset(const CfCoef &c) {
    if constexpr (SX == 0 && SY == 0) return c.ff;
    else if constexpr (SY == 0) return c.hf;
    else if constexpr (SX == 0) return c.fh;
    else return c.hh;
}

// Contribution of one coarse cell, over the quadrants of the node's support
// selected by SX, SY (0 = both sides, -1 / +1 = that side only), to the
// velocity rows (Au, Av) and the divergence row (Ap) of A(x~), Eq.
// nonlinearshort.  uw, vw, pw: node values (continuous); U, V, P: this
// cell's derivatives at the node.  The terms are the hat moments of the
// polynomial integrands, grouped by moment; terms carrying a first moment of
// a full support vanish and are left out at compile time.
template <int SX, int SY>
__device__ __forceinline__ void cell_part(const CfCoef &c, float uw, float vw, float pw, const D3 &U, const D3 &V,
                                          const D3 &P, float &Au, float &Av, float &Ap) {
    const Kset &k = kset<SX, SY>(c);
    constexpr float sx = (float)SX, sy = (float)SY;
    const float t2 = k.C02 * U.y + k.C20 * V.x;
    Au += k.C00 * (uw * U.x + vw * U.y) + t2 * U.xy + k.M00 * uw + k.m00 * P.x;
    Av += k.C00 * (uw * V.x + vw * V.y) + t2 * V.xy + k.M00 * vw + k.m00 * P.y;
    Ap += k.m00 * (U.x + V.y);
    if constexpr (SY != 0) {
        Au += sy * (k.C01 * (uw * U.xy + U.y * U.x + V.y * U.y) + k.C21 * (V.xy * U.xy) + k.MD01 * U.y +
                    k.m01 * P.xy);
        Av += sy * (k.C01 * (uw * V.xy + U.y * V.x + V.y * V.y) + k.C21 * (V.xy * V.xy) + k.MD01 * V.y + k.x0 * pw);
        Ap += sy * (k.m01 * U.xy);
    }
    if constexpr (SX != 0) {
        Au += sx * (k.C10 * (U.x * U.x + vw * U.xy + V.x * U.y) + k.C12 * (U.xy * U.xy) + k.MD10 * U.x + k.y0 * pw);
        Av += sx * (k.C10 * (U.x * V.x + vw * V.xy + V.x * V.y) + k.C12 * (U.xy * V.xy) + k.MD10 * V.x +
                    k.m10 * P.xy);
        Ap += sx * (k.m10 * V.xy);
    }
    if constexpr (SX != 0 && SY != 0) {
        Au += sx * sy * (k.C11 * (2.0f * U.x * U.xy + V.y * U.xy + V.xy * U.y) + k.MD11 * U.xy + k.y1 * P.y);
        Av += sx * sy * (k.C11 * (U.x * V.xy + U.xy * V.x + 2.0f * V.y * V.xy) + k.MD11 * V.xy + k.x1 * P.x);
    }
}

// One coarse cell's bilinear fields (u, v, p): w = c00 + bx X + by Y + d X Y
// at offset (X, Y) from its SW corner.  The coefficients are formed once per
// block from the corner values (cell_coefficients) and read from shared
// memory where they are used, which keeps few of them in registers at a time.
constexpr int CELL_COEF = 12;   // [c00, bx, by, d] x (u, v, p)
struct Cell {
    const float *q;             // the cell's coefficients in shared memory
    __device__ __forceinline__ D3 der(int f, float X, float Y) const {
        const float bx = q[4 * f + 1], by = q[4 * f + 2], d = q[4 * f + 3];
        return D3{bx + d * Y, by + d * X, d};
    }
    __device__ __forceinline__ float value(int f, float X, float Y) const {
        const float c00 = q[4 * f], bx = q[4 * f + 1], by = q[4 * f + 2], d = q[4 * f + 3];
        return c00 + bx * X + Y * (by + d * X);
    }
};

// Coefficients of every coarse cell of the staged window: cells (a, b) with
// SW node (a, b) of the window, a < cw - 1, b < ch - 1, into cc[(b (cw - 1) + a) 12 ..].
__device__ __forceinline__ void cell_coefficients(const CfCoef &c, const float *cs, int cw, int ch, float *cc,
                                                  int nthreads) {
    const int ncx = cw - 1, n = ncx * (ch - 1);
    for (int e = threadIdx.x; e < 3 * n; e += nthreads) {
        const int f = e / n, cell = e - f * n;
        const int b = cell / ncx, a = cell - b * ncx;
        const float *q = cs + f * cw * ch + b * cw + a;
        const float w00 = q[0], w10 = q[1], w01 = q[cw], w11 = q[cw + 1];
        float *o = cc + cell * CELL_COEF + 4 * f;
        o[0] = w00;
        o[1] = (w10 - w00) * c.iHx;
        o[2] = (w01 - w00) * c.iHy;
        o[3] = ((w11 - w10) - (w01 - w00)) * c.iHxy;
    }
}

// A(x~) at a node at offset (X, Y) in its own cell (the cell above and to
// the right): XE / YE say whether the node lies on a vertical / horizontal
// coarse cell edge; then the cells on both sides contribute one half each
// (left, low, lowleft: the neighbours of own).
template <bool XE, bool YE>
__device__ __forceinline__ void node_A(const CfCoef &c, const Cell &own, const Cell &left, const Cell &low,
                                       const Cell &lowleft, float X, float Y, float &Au, float &Av, float &Ap) {
    Au = Av = Ap = 0.0f;
    const float uw = own.value(0, X, Y), vw = own.value(1, X, Y), pw = own.value(2, X, Y);
    auto part = [&](const Cell &cl, float x, float y, auto sx, auto sy) {
        cell_part<decltype(sx)::value, decltype(sy)::value>(c, uw, vw, pw, cl.der(0, x, y), cl.der(1, x, y),
                                                              cl.der(2, x, y), Au, Av, Ap);
    };
    using M1 = std::integral_constant<int, -1>;
    using Z = std::integral_constant<int, 0>;
    using P1 = std::integral_constant<int, 1>;
    if constexpr (!XE && !YE) {
        part(own, X, Y, Z{}, Z{});
    } else if constexpr (XE && !YE) {
        part(left, c.Hx, Y, M1{}, Z{});
        part(own, 0.0f, Y, P1{}, Z{});
    } else if constexpr (!XE && YE) {
        part(low, X, c.Hy, Z{}, M1{});
        part(own, X, 0.0f, Z{}, P1{});
    } else {
        part(lowleft, c.Hx, c.Hy, M1{}, M1{});
        part(low, 0.0f, c.Hy, P1{}, M1{});
        part(left, c.Hx, 0.0f, M1{}, P1{});
        part(own, 0.0f, 0.0f, P1{}, P1{});
    }
}

template <typename TX> __device__ __forceinline__ TX to_feat(float v);
template <> __device__ __forceinline__ float to_feat<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 to_feat<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// EPC consecutive 16-bit table entries (16- or 8-byte aligned) from shared memory.
template <int EPC> __device__ __forceinline__ void load_entries(const uint16_t *p, uint16_t (&e)[EPC]) {
    if constexpr (EPC == 8) {
        const uint4 tv = *reinterpret_cast<const uint4 *>(p);
        const uint32_t w[4] = {tv.x, tv.y, tv.z, tv.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            e[2 * k] = (uint16_t)(w[k] & 0xFFFFu);
            e[2 * k + 1] = (uint16_t)(w[k] >> 16);
        }
    } else {
        const uint2 tv = *reinterpret_cast<const uint2 *>(p);
        e[0] = (uint16_t)(tv.x & 0xFFFFu);
        e[1] = (uint16_t)(tv.x >> 16);
        e[2] = (uint16_t)(tv.y & 0xFFFFu);
        e[3] = (uint16_t)(tv.y >> 16);
    }
}

// Block (bx, by) of the closed form: general tiles (2 bx, by) and (2 bx + 1,
// by), both of which must have the all-fluid flag (every cell within two of
// the tile exists and is fluid).
__host__ __device__ __forceinline__ bool block_fast_flags(const uint8_t *flags, int ntx, int nty, int bx, int by) {
    const int t0 = 2 * bx;
    if (t0 + 1 >= ntx || by >= nty) return false;
    return (flags[(size_t)by * ntx + t0] & 1) && (flags[(size_t)by * ntx + t0 + 1] & 1);
}
__device__ __forceinline__ bool block_fast(const MeshGeom &g, int bx, int by) {
    const int t0 = 2 * bx;
    if (t0 + 1 >= g.ntx || by >= g.nty) return false;
    return (__ldg(g.tile_flags + (size_t)by * g.ntx + t0) & 1) && (__ldg(g.tile_flags + (size_t)by * g.ntx + t0 + 1) & 1);
}

// R consecutive residuals of one row as one aligned shared-memory store.
template <int R> __device__ __forceinline__ void put_row(float *p, const float *r) {
    if constexpr (R == 4) *reinterpret_cast<float4 *>(p) = make_float4(r[0], r[1], r[2], r[3]);
    else *reinterpret_cast<float2 *>(p) = make_float2(r[0], r[1]);
}
template <int R> __device__ __forceinline__ void put_row(__nv_bfloat16 *p, const float *r) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(r[0], r[1]);
    if constexpr (R == 4) {
        const __nv_bfloat162 b = __floats2bfloat162_rn(r[2], r[3]);
        uint2 v;
        v.x = *reinterpret_cast<const uint32_t *>(&a);
        v.y = *reinterpret_cast<const uint32_t *>(&b);
        *reinterpret_cast<uint2 *>(p) = v;
    } else {
        *reinterpret_cast<__nv_bfloat162 *>(p) = a;
    }
}
template <int R> __device__ __forceinline__ void load_row(const float *p, float *v) {
    if constexpr (R == 4) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        const float2 q = __ldg(reinterpret_cast<const float2 *>(p));
        v[0] = q.x; v[1] = q.y;
    }
}

// The fine nodes of coarse cell (ci, cj) of the block (block-local coarse
// indices; the block's first staged coarse node is window node (1, 1) minus
// one): rows b = B0 .. B1-1, columns a = 0 .. R-1 when FX (else column 0
// only).  Node (a, b) lies on a vertical coarse edge
// when a = 0 and on a horizontal one when b = 0.  Residuals r = b_f - A(x~)
// go to the block's residual array in the feature type.
template <typename TX, int R, bool FX, int B0, int B1>
__device__ __forceinline__ void cell_task(const CfCoef &c, const float *cc, int ncx, int ci, int cj,
                                          const MeshGeom &g, const float *__restrict__ bf, int I0, int J0, TX *rres) {
    const int o = (cj + 1) * ncx + ci + 1;   // own cell in the window's cell array
    const Cell own{cc + o * CELL_COEF}, left{cc + (o - 1) * CELL_COEF}, low{cc + (o - ncx) * CELL_COEF},
        lowleft{cc + (o - ncx - 1) * CELL_COEF};
    constexpr int NA = FX ? R : 1;
    const int Il = ci * R, Jl = cj * R;     // block-local fine node of the cell's SW corner
#pragma unroll
    for (int b = B0; b < B1; ++b) {
        const float Y = (float)b * c.hy;
        const size_t node = (size_t)(J0 + Jl + b) * g.pitch + I0 + Il;
        float bu[R], bv[R], ru[R], rv[R], rp[R];
        if constexpr (FX) {
            load_row<R>(bf + node, bu);
            load_row<R>(bf + g.plane + node, bv);
        } else {
            bu[0] = __ldg(bf + node);
            bv[0] = __ldg(bf + g.plane + node);
        }
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            float Au, Av, Ap;
            const float X = (float)a * c.hx;
            if (b == 0) {
                if (a == 0) node_A<true, true>(c, own, left, low, lowleft, X, Y, Au, Av, Ap);
                else node_A<false, true>(c, own, left, low, lowleft, X, Y, Au, Av, Ap);
            } else {
                if (a == 0) node_A<true, false>(c, own, left, low, lowleft, X, Y, Au, Av, Ap);
                else node_A<false, false>(c, own, left, low, lowleft, X, Y, Au, Av, Ap);
            }
            ru[a] = bu[a] - Au;
            rv[a] = bv[a] - Av;
            rp[a] = -Ap;
        }
        TX *dst = rres + (Jl + b) * CF_RXP + Il;
        if constexpr (FX) {
            put_row<R>(dst, ru);
            put_row<R>(dst + CF_RPL, rv);
            put_row<R>(dst + 2 * CF_RPL, rp);
        } else {
            dst[0] = to_feat<TX>(ru[0]);
            dst[CF_RPL] = to_feat<TX>(rv[0]);
            dst[2 * CF_RPL] = to_feat<TX>(rp[0]);
        }
    }
}

// Sizes of one (K, s) configuration: R = 2^K fine cells per coarse cell,
// SP = s coarse cells per patch edge.
template <typename TX, int R, int SP>
struct CfShape {
    static constexpr int K = R == 2 ? 1 : 2;
    static constexpr int S = SP * R, NF = (S + 1) * (S + 1), NC = (SP + 1) * (SP + 1);
    static constexpr int NRES = 3 * NF, NIN = NRES + 3 * NC + 12, LDX = (NIN + 15) / 16 * 16;
    static constexpr int EXW = (LDX - NRES + 7) / 8 * 8;             // extra columns per patch
    static constexpr int TPX = CF_TXC / S, TPY = CF_TYC / S, NP = TPX * TPY;
    static constexpr int EPC = 16 / sizeof(TX), NCH = LDX / EPC;      // columns per 16-byte piece
    static constexpr int CW = CF_TXC / R + 3, CH = CF_TYC / R + 3;    // coarse window nodes
    static constexpr int NCX = CF_TXC / R, NCY = CF_TYC / R, NFULL = NCX * NCY;   // coarse cells of the block
    static constexpr int NTASK = NFULL + NCX + NCY + 1;               // plus the partial cells above and right
    static constexpr int THREADS = (NTASK + 31) / 32 * 32;
    // shared memory (bytes)
    static constexpr size_t CS = 0;                                               // [3][CH][CW] float
    static constexpr size_t CC = (CS + 3 * CW * CH * 4 + 15) / 16 * 16;           // [cells][12] float
    static constexpr size_t RR = (CC + (CW - 1) * (CH - 1) * CELL_COEF * 4 + 15) / 16 * 16;   // [3][NYN][RXP] TX
    static constexpr size_t TAB = (RR + 3 * CF_RPL * sizeof(TX) + 15) / 16 * 16;  // [LDX] uint16
    static constexpr size_t PID = (TAB + LDX * 2 + 15) / 16 * 16;                 // [NP] int
    static constexpr size_t EX = (PID + NP * 4 + 15) / 16 * 16;                   // [NP][EXW] TX
    static constexpr size_t BYTES = EX + NP * EXW * sizeof(TX);
};

// The all-fluid tiles of S2 + S3 in the step.  One CTA per 32 x 16-cell tile
// (tiles without the flag return at once).  Threads 0..135 each take a run
// of four nodes of one row, ordered so that a warp holds only rows on a
// horizontal coarse edge or only rows off it; threads 136..152 take the
// tile's last node column.  Then the feature rows of the tile's patches are
// gathered from shared memory in 16-byte pieces.
template <typename TX, int R, int SP>
__global__ void __launch_bounds__(CfShape<TX, R, SP>::THREADS, R == 4 ? 10 : 3)
k_residual_cf(MeshGeom g, CfCoef c, const float *__restrict__ xcp, int pc, const float *__restrict__ bf,
              TX *__restrict__ X) {
    using SH = CfShape<TX, R, SP>;
    constexpr int K = SH::K, S = SH::S, LS = K + SP - 1;
    const int tx = blockIdx.x, ty = blockIdx.y;
    if (!block_fast(g, tx, ty)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    float *cs = reinterpret_cast<float *>(smem + SH::CS);
    float *cc = reinterpret_cast<float *>(smem + SH::CC);
    TX *rres = reinterpret_cast<TX *>(smem + SH::RR);
    uint16_t *tab = reinterpret_cast<uint16_t *>(smem + SH::TAB);
    int *pid = reinterpret_cast<int *>(smem + SH::PID);
    TX *ex = reinterpret_cast<TX *>(smem + SH::EX);
    __shared__ float geo_s[12];
    const int I0 = tx * CF_TXC, J0 = ty * CF_TYC;
    const int cx0 = (I0 >> K) - 1, cy0 = (J0 >> K) - 1;   // first staged coarse node
    // ---- staging: coarse window, patch numbers, column table
    const size_t cplane = (size_t)pc * (g.nyc + 1);
    for (int e = threadIdx.x; e < 3 * SH::CW * SH::CH; e += SH::THREADS) {
        const int f = e / (SH::CW * SH::CH), rem = e - f * (SH::CW * SH::CH);
        const int b = rem / SH::CW, a = rem - b * SH::CW;
        cs[e] = __ldg(xcp + f * cplane + (size_t)(cy0 + b) * pc + cx0 + a);   // inside: the tile is interior
    }
    for (int e = threadIdx.x; e < SH::NP; e += SH::THREADS) {
        const int py = e / SH::TPX, px = e - py * SH::TPX;
        pid[e] = __ldg(g.patch_id + ((J0 >> LS) + py) * g.npx + (I0 >> LS) + px);
    }
    for (int col = threadIdx.x; col < SH::LDX / 2; col += SH::THREADS)
        reinterpret_cast<uint32_t *>(tab)[col] = __ldg(reinterpret_cast<const uint32_t *>(g.cf_tab) + col);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < 12; ++i) geo_s[i] = c.geo[i];
    }
    __syncthreads();
    // ---- extra columns of each patch: coarse-node u, v, Peclet, geometry, zero padding
    for (int e = threadIdx.x; e < SH::NP * SH::EXW; e += SH::THREADS) {
        const int q = e / SH::EXW, k = e - q * SH::EXW;
        const int py = q / SH::TPX, px = q - py * SH::TPX;
        float val = 0.0f;
        if (k < 3 * SH::NC) {
            const int which = k / SH::NC, n = k - which * SH::NC, lb = n / (SP + 1), la = n - lb * (SP + 1);
            const int o = (py * SP + 1 + lb) * SH::CW + px * SP + 1 + la;   // patch origin at window node (1, 1)
            const float a = cs[o], b = cs[SH::CW * SH::CH + o];
            if (which == 2)
                val = c.q_over_nu * sqrtf(a * a + b * b);
            else
                val = which ? b : a;
        } else if (k < 3 * SH::NC + 12) {
            val = geo_s[k - 3 * SH::NC];
        }
        ex[e] = to_feat<TX>(val);
    }
    cell_coefficients(c, cs, SH::CW, SH::CH, cc, SH::THREADS);
    __syncthreads();
    // ---- node pass: one thread per coarse cell of the block, taking every
    // fine node of the cell (its rows 0 .. R-1, columns 0 .. R-1), so that
    // every thread has the same mix of corner, edge and interior nodes; the
    // block's last node row and column come from the partial cells above and
    // to the right of it
    const int t = threadIdx.x;
    if (t < SH::NFULL) {
        const int cj = t / SH::NCX, ci = t - cj * SH::NCX;
        cell_task<TX, R, true, 0, R>(c, cc, SH::CW - 1, ci, cj, g, bf, I0, J0, rres);
    } else if (t < SH::NFULL + SH::NCX) {
        cell_task<TX, R, true, 0, 1>(c, cc, SH::CW - 1, t - SH::NFULL, SH::NCY, g, bf, I0, J0, rres);
    } else if (t < SH::NFULL + SH::NCX + SH::NCY) {
        cell_task<TX, R, false, 0, R>(c, cc, SH::CW - 1, SH::NCX, t - SH::NFULL - SH::NCX, g, bf, I0, J0, rres);
    } else if (t == SH::NFULL + SH::NCX + SH::NCY) {
        cell_task<TX, R, false, 0, 1>(c, cc, SH::CW - 1, SH::NCX, SH::NCY, g, bf, I0, J0, rres);
    }
    __syncthreads();
    // ---- feature rows: 16-byte pieces of each patch row, columns from the table;
    // pieces made of residual columns only, then the rest (mixed and extra columns)
    constexpr int NRCH = SH::NRES / SH::EPC, NTCH = SH::NCH - NRCH;
    for (int q = threadIdx.x; q < SH::NP * NRCH; q += SH::THREADS) {
        const int pp = q / NRCH, ch = q - pp * NRCH;
        const int id = pid[pp];
        if (id < 0) continue;
        const int py = pp / SH::TPX, px = pp - py * SH::TPX;
        const TX *rb = rres + py * S * CF_RXP + px * S;
        uint16_t e[SH::EPC];
        load_entries<SH::EPC>(tab + ch * SH::EPC, e);
        __align__(16) TX v[SH::EPC];
#pragma unroll
        for (int k = 0; k < SH::EPC; ++k) v[k] = rb[e[k]];
        *reinterpret_cast<uint4 *>(X + (size_t)id * SH::LDX + ch * SH::EPC) = *reinterpret_cast<const uint4 *>(v);
    }
    for (int q = threadIdx.x; q < SH::NP * NTCH; q += SH::THREADS) {
        const int pp = q / NTCH, ch = NRCH + (q - pp * NTCH);
        const int id = pid[pp];
        if (id < 0) continue;
        const int py = pp / SH::TPX, px = pp - py * SH::TPX;
        const TX *rb = rres + py * S * CF_RXP + px * S;
        const TX *eb = ex + pp * SH::EXW;
        uint16_t e[SH::EPC];
        load_entries<SH::EPC>(tab + ch * SH::EPC, e);
        __align__(16) TX v[SH::EPC];
#pragma unroll
        for (int k = 0; k < SH::EPC; ++k) v[k] = (e[k] & 0x8000u) ? eb[e[k] & 0x7FFFu] : rb[e[k]];
        *reinterpret_cast<uint4 *>(X + (size_t)id * SH::LDX + ch * SH::EPC) = *reinterpret_cast<const uint4 *>(v);
    }
}

template <typename TX, int R, int SP>
cudaError_t run_cf(const MeshGeom &g, const CfCoef &c, const float *xcp, const float *bf, TX *X, cudaStream_t st) {
    using SH = CfShape<TX, R, SP>;
    if (g.ldx != SH::LDX || g.nf != SH::NF) return cudaErrorInvalidValue;
    auto k = k_residual_cf<TX, R, SP>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SH::BYTES);
    if (e != cudaSuccess) return e;
    const dim3 grid((g.nxf + CF_TXC - 1) / CF_TXC, (g.nyf + CF_TYC - 1) / CF_TYC);
    k<<<grid, SH::THREADS, SH::BYTES, st>>>(g, c, xcp, coarse_pitch(g), bf, X);
    return cudaGetLastError();
}

template <typename TX>
cudaError_t run_cf_shape(const MeshGeom &g, const CfCoef &c, const float *xcp, const float *bf, TX *X,
                         cudaStream_t st) {
    if (g.r == 2 && g.s == 1) return run_cf<TX, 2, 1>(g, c, xcp, bf, X, st);
    if (g.r == 2 && g.s == 2) return run_cf<TX, 2, 2>(g, c, xcp, bf, X, st);
    if (g.r == 4 && g.s == 1) return run_cf<TX, 4, 1>(g, c, xcp, bf, X, st);
    if (g.r == 4 && g.s == 2) return run_cf<TX, 4, 2>(g, c, xcp, bf, X, st);
    return cudaErrorInvalidValue;
}

}  // namespace

void residual_cf_table(const MeshGeom &g, uint16_t *tab) {
    // residual columns: component plane, patch-local row and column in the
    // tile's residual array; the others: 0x8000 | index in the patch's extra values
    const int nres = 3 * g.nf, S1 = g.S + 1;
    for (int col = 0; col < g.ldx; ++col) {
        if (col < nres) {
            const int comp = col / g.nf, rem = col - comp * g.nf, lj = rem / S1, li = rem - lj * S1;
            tab[col] = (uint16_t)(comp * CF_RPL + lj * CF_RXP + li);
        } else {
            tab[col] = (uint16_t)(0x8000u | (col - nres));
        }
    }
}

void residual_cf_slow_tiles(const MeshGeom &g, const uint8_t *flags, std::vector<int> *slow) {
    slow->clear();
    for (int ty = 0; ty < g.nty; ++ty)
        for (int tx = 0; tx < g.ntx; ++tx)
            if (!block_fast_flags(flags, g.ntx, g.nty, tx / 2, ty)) slow->push_back(ty * g.ntx + tx);
}

bool residual_cf_supported(const MeshGeom &g, int prec) {
    return prec != DNNMG_F64 && (g.r == 2 || g.r == 4) && (g.s == 1 || g.s == 2);
}

cudaError_t launch_residual_cf(const MeshGeom &g, int prec, const FemCoef<float> &f32, const void *xcp, const void *bf,
                               void *X, cudaStream_t st) {
    CfCoef c;
    const double hx = g.hxf, hy = g.hyf, Hx = g.hxc, Hy = g.hyc;
    const double ik = 1.0 / g.k, hnu = 0.5 * g.nu;
    c.iHx = (float)(1.0 / Hx);
    c.iHy = (float)(1.0 / Hy);
    c.iHxy = (float)(1.0 / (Hx * Hy));
    c.hx = (float)hx;
    c.hy = (float)hy;
    c.Hx = (float)Hx;
    c.Hy = (float)Hy;
    auto set = [&](const double (&x)[3], const double (&y)[3]) {
        Kset k;
        auto m = [&](int a, int b) { return x[a] * y[b]; };
        k.C00 = (float)(0.5 * m(0, 0)); k.C01 = (float)(0.5 * m(0, 1)); k.C10 = (float)(0.5 * m(1, 0));
        k.C11 = (float)(0.5 * m(1, 1)); k.C02 = (float)(0.5 * m(0, 2)); k.C20 = (float)(0.5 * m(2, 0));
        k.C12 = (float)(0.5 * m(1, 2)); k.C21 = (float)(0.5 * m(2, 1));
        k.M00 = (float)(ik * m(0, 0));
        k.MD01 = (float)(ik * m(0, 1) - hnu * x[0]);
        k.MD10 = (float)(ik * m(1, 0) - hnu * y[0]);
        k.MD11 = (float)(ik * m(1, 1) - hnu * (x[1] + y[1]));
        k.m00 = (float)m(0, 0); k.m01 = (float)m(0, 1); k.m10 = (float)m(1, 0);
        k.x0 = (float)x[0]; k.y0 = (float)y[0]; k.x1 = (float)x[1]; k.y1 = (float)y[1];
        return k;
    };
    // full support: h, 0, h^3/6; half support: h/2, h^2/6, h^3/12
    const double fx[3] = {hx, 0.0, hx * hx * hx / 6}, hx_[3] = {hx / 2, hx * hx / 6, hx * hx * hx / 12};
    const double fy[3] = {hy, 0.0, hy * hy * hy / 6}, hy_[3] = {hy / 2, hy * hy / 6, hy * hy * hy / 12};
    c.ff = set(fx, fy);
    c.hf = set(hx_, fy);
    c.fh = set(fx, hy_);
    c.hh = set(hx_, hy_);
    c.q_over_nu = f32.q_over_nu;
    for (int i = 0; i < 12; ++i) c.geo[i] = f32.geo[i];
    const float *xp = static_cast<const float *>(xcp);
    const float *b = static_cast<const float *>(bf);
    if (prec == DNNMG_F32) return run_cf_shape(g, c, xp, b, static_cast<float *>(X), st);
    return run_cf_shape(g, c, xp, b, static_cast<__nv_bfloat16 *>(X), st);
}

}  // namespace dnnmg

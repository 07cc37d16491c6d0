// Stencil, gather and scatter passes of the DNN-MG correction step:
//   S1 prolongation, S2+S3 residual and patch features, S5 averaging,
//   S6 right-hand side, S7 restriction, plus the node index maps.
//
// Fine node fields are pitched SoA planes [comp][nyf+1][pitch], x fastest,
// pitch = round_up(nxf + 1, 64), so every row starts on a 256-byte boundary
// and tiles move as aligned 16-byte pieces.  S2 and S6 are tiled: one CTA owns
// a 32 x 16 block of fine cells, stages the node values it needs (plus a
// halo) in shared memory with asynchronous copies, computes every cell's
// element contributions once (cell-centric), and then sums them per node (a
// pull: no atomics, bitwise repeatable).  A tile writes only the nodes it
// owns.  Tiles whose whole neighbourhood is fluid (the vast majority) take a
// fast path with node-level stencils and skip all boundary classification.
#include <cstdio>

#include "common.cuh"
#include "ptx.cuh"

namespace dnnmg {
namespace {

constexpr int TXC = 32;            // fine cells per tile in x
constexpr int TYC = 16;            // fine cells per tile in y
constexpr int NXN = TXC + 1;       // tile nodes in x
constexpr int NYN = TYC + 1;
constexpr int NTHREADS = 256;
constexpr int RES_THREADS = 256;   // residual/feature kernels (10 warps measured slower)

template <typename TX, typename T> __device__ __forceinline__ TX store_as(T v) { return (TX)v; }
template <> __device__ __forceinline__ __nv_bfloat16 store_as<__nv_bfloat16, float>(float v) {
    return __float2bfloat16_rn(v);
}

__device__ __forceinline__ int cell_code(const MeshGeom &g, int I, int J) {
    // 0: no cell (outside the domain), 1: fluid, 2: solid
    if (I < 0 || J < 0 || I >= g.nxf || J >= g.nyf) return 0;
    return g.solid[(size_t)(J >> g.K) * g.nxc + (I >> g.K)] ? 2 : 1;
}

struct NodeClass {
    bool dirichlet, inflow, p_active;
};

// Sec. 6.1 boundary classes of fine node (I, J) from its four cells.
__device__ __forceinline__ NodeClass classify(int c00, int c10, int c01, int c11, int I, int J, int nyf) {
    bool ts = (c00 == 2) | (c10 == 2) | (c01 == 2) | (c11 == 2);
    bool tf = (c00 == 1) | (c10 == 1) | (c01 == 1) | (c11 == 1);
    bool wall = (J == 0) | (J == nyf);
    NodeClass n;
    n.dirichlet = wall | (I == 0) | ts;
    n.inflow = (I == 0) & !wall & !ts;
    n.p_active = tf;
    return n;
}

__device__ __forceinline__ NodeClass classify_global(const MeshGeom &g, int I, int J) {
    return classify(cell_code(g, I - 1, J - 1), cell_code(g, I, J - 1), cell_code(g, I - 1, J),
                    cell_code(g, I, J), I, J, g.nyf);
}

// Fast-path tests from the per-tile flags (computed with the mesh): tile
// (tx, ty) of 32 x 16 cells with all cells within `halo` (1 or 2) fluid; a
// 64 x 16 node tile is the union of two stencil tiles.
__device__ __forceinline__ bool tile_fluid(const MeshGeom &g, int tx, int ty, int bit) {
    return tx < g.ntx && ty < g.nty && (__ldg(g.tile_flags + (size_t)ty * g.ntx + tx) & bit);
}
__device__ __forceinline__ bool node_tile_fluid(const MeshGeom &g, int bx, int by) {
    return tile_fluid(g, 2 * bx, by, 2) && tile_fluid(g, 2 * bx + 1, by, 2);
}

// Asynchronous 16-byte copy global -> shared; src_bytes = 0 writes zeros.
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// Asynchronous 8-byte copy global -> shared (both 8-byte aligned).
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}

// Stage a window of NCOMP component planes: rows J0 .. J0+NROWS-1, columns
// Ia .. Ia+W-1 (Ia and W multiples of 16 bytes) into dst[c][row][W].  Pieces
// outside the stored rows are zero; columns past nxf (row padding) carry
// whatever the padding holds and are never used.  Asynchronous: complete with
// cp_async_wait_all() and a barrier.  Window sizes are compile-time constants
// so the piece -> (row, column) split costs a multiply and a shift.
template <typename T, int NCOMP, int NROWS, int W>
__device__ __forceinline__ void stage_window(const MeshGeom &g, const T *__restrict__ src, int Ia, int J0, T *dst) {
    constexpr int EPC = 16 / sizeof(T), CPR = W / EPC, TOTAL = NCOMP * NROWS * CPR;
    static_assert(W % EPC == 0, "window width must be a multiple of 16 bytes");
    for (int e = threadIdx.x; e < TOTAL; e += blockDim.x) {
        const int row = e / CPR, k = e - row * CPR;          // row = c * NROWS + jj
        const int c = row / NROWS, J = J0 + (row - c * NROWS);
        const int I = Ia + k * EPC;
        const bool ok = J >= 0 && J <= g.nyf && I >= 0 && I + EPC <= g.pitch;
        const T *s = ok ? src + (size_t)c * g.plane + (size_t)J * g.pitch + I : src;
        cp_async16(dst + row * W + k * EPC, s, ok ? 16 : 0);
    }
}

// ------------------------------------------------------------------ S1
// Coarse nodes that a window of fine nodes [Ilo, Ilo+FW) x [Jlo, Jlo+FH)
// interpolates from, staged once per CTA in the fine arithmetic type (FP64
// throughput on GB300 is 1/64 of FP32, so converting per fine node is not an
// option).  Fine node I lies in coarse cell I >> K (floor) at offset
// (I mod R) / R; the last node nxf falls at offset 0 of a cell "nxc", which
// blends the same two coarse nodes as the edge of cell nxc-1.  Coarse nodes
// outside the mesh are staged as zeros (only window nodes outside the mesh
// read them, and those are never used).
template <int R> struct Log2;
template <> struct Log2<2> { static constexpr int v = 1; };
template <> struct Log2<4> { static constexpr int v = 2; };
template <> struct Log2<8> { static constexpr int v = 3; };

__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }

// lo + w (hi - lo) with one explicit rounding of the product-sum, so every
// kernel that interpolates a node produces the same bits.
template <typename T> __device__ __forceinline__ T lerp(T lo, T hi, T w) { return fma_t(w, hi - lo, lo); }

// NC = 3 stages u, v, p; NC = 2 the velocity only.  ALIGN > 1: the first
// staged column is rounded down to a multiple of ALIGN and the row length up
// (windows fetched by TMA, whose x coordinate must be 16-byte aligned).
template <typename T, int R, int FW, int FH, int NC = 3, int ALIGN = 1>
struct CoarseWin {
    static constexpr int K = Log2<R>::v;
    static constexpr int CW = ((FW - 1) / R + 3 + ALIGN - 1 + ALIGN - 1) / ALIGN * ALIGN;
    static constexpr int CH = (FH - 1) / R + 3, N = NC * CW * CH;
    T *cs;          // [NC][CH][CW] in shared memory
    int ci0, cj0;   // first staged coarse node (may be negative)

    __device__ __forceinline__ void stage(const MeshGeom &g, const double *__restrict__ xc, int Ilo, int Jlo) {
        ci0 = Ilo >> K;
        cj0 = Jlo >> K;
        const size_t nc1 = (size_t)g.nxc + 1, Nc = nc1 * (g.nyc + 1);
        for (int e = threadIdx.x; e < N; e += blockDim.x) {
            const int c = e / (CW * CH), rem = e - c * (CW * CH);
            const int b = rem / CW, a = rem - b * CW;
            const int ci = ci0 + a, cj = cj0 + b;
            T v = T(0);
            if (ci >= 0 && cj >= 0 && ci <= g.nxc && cj <= g.nyc) v = (T)__ldg(xc + c * Nc + (size_t)cj * nc1 + ci);
            cs[e] = v;
        }
    }
    // The same window from the padded copy [NC..][nyc+1][pc] of x_c in the
    // fine type that the step keeps (the same values: both round x_c once).
    __device__ __forceinline__ void stage_padded(const MeshGeom &g, const T *__restrict__ xcp, int pc, int Ilo,
                                                 int Jlo) {
        ci0 = Ilo >> K;
        cj0 = Jlo >> K;
        const size_t cplane = (size_t)pc * (g.nyc + 1);
        for (int e = threadIdx.x; e < N; e += blockDim.x) {
            const int c = e / (CW * CH), rem = e - c * (CW * CH);
            const int b = rem / CW, a = rem - b * CW;
            const int ci = ci0 + a, cj = cj0 + b;
            T v = T(0);
            if (ci >= 0 && cj >= 0 && ci <= g.nxc && cj <= g.nyc) v = __ldg(xcp + c * cplane + (size_t)cj * pc + ci);
            cs[e] = v;
        }
    }
    // Bilinear value of the staged fields at fine node (I, J) (raw P, no BC):
    // blends along x on the cell's bottom and top edges, then along y.
    __device__ __forceinline__ void interp(int I, int J, T (&out)[NC]) const {
        constexpr T inv_r = T(1) / T(R);   // exact: R is a power of two
        const int ci = I >> K, cj = J >> K;
        const T a = T(I & (R - 1)) * inv_r, b = T(J & (R - 1)) * inv_r;
        const int o = (cj - cj0) * CW + (ci - ci0);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const T *q = cs + c * CW * CH + o;
            out[c] = lerp(lerp(q[0], q[1], a), lerp(q[CW], q[CW + 1], a), b);
        }
    }
    // interp at the 4 nodes Ib .. Ib+3 of row J, Ib a multiple of 4 (same
    // arithmetic, so the same bits; the cell and weights are compile-time
    // offsets for R <= 4, and for R = 8 the run lies in one cell).
    __device__ __forceinline__ void interp4(int Ib, int J, T (&out)[NC][4]) const {
        constexpr T inv_r = T(1) / T(R);
        const int r0 = R <= 4 ? 0 : (Ib & (R - 1));
        const T b = T(J & (R - 1)) * inv_r;
        const int o = ((J >> K) - cj0) * CW + ((Ib >> K) - ci0);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const T *q = cs + c * CW * CH + o;
#pragma unroll
            for (int n = 0; n < 4; ++n) {
                const int e = r0 + n, dc = R >= 4 ? 0 : (e >> K);
                const T a = T(e & (R - 1)) * inv_r;
                out[c][n] = lerp(lerp(q[dc], q[dc + 1], a), lerp(q[dc + CW], q[dc + CW + 1], a), b);
            }
        }
    }
};

// Parabolic inflow u = up 4 y (ly - y) / ly^2 at fine row J, up the (ramped)
// peak velocity: evaluated in FP64 and rounded once.  Kept out of line so
// that only inflow nodes execute it (FP64 runs at 1/64 of FP32 on GB300).
template <typename T> __device__ __noinline__ T inflow_value(const MeshGeom &g, int J, double up) {
    const double y = J * g.hyf;
    return (T)(up * 4.0 * y * (g.ly - y) / (g.ly * g.ly));
}

// Dirichlet velocity of fine node (I, J) if it has one (Sec. 6.1): the
// inflow profile on the left boundary, no-slip elsewhere.
template <typename T>
__device__ __forceinline__ bool dirichlet_value(const MeshGeom &g, int I, int J, double up, T &u, T &v) {
    const NodeClass nc = classify_global(g, I, J);
    if (!nc.dirichlet) return false;
    u = nc.inflow ? inflow_value<T>(g, J, up) : T(0);
    v = T(0);
    return true;
}

// Four consecutive nodes as one aligned vector access (16 B for float, two 16 B for double).
__device__ __forceinline__ void store4(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(double *p, const double (&v)[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void load4(const float *p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void load4(const double *p, double (&v)[4]) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// A CTA owns 64 x 16 fine nodes, 4 consecutive nodes per thread (one 16-byte
// store per field and row segment; nodes past nxf land in the row padding).
constexpr int PTX = 64, PTY = 16;

template <typename T, int R>
__global__ void __launch_bounds__(NTHREADS)
k_prolongate(MeshGeom g, const double *__restrict__ xc, T *__restrict__ xf, double up) {
    using CW = CoarseWin<T, R, PTX, PTY>;
    __shared__ T cs_mem[CW::N];
    const int I0 = blockIdx.x * PTX, J0 = blockIdx.y * PTY;
    CW cw;
    cw.cs = cs_mem;
    cw.stage(g, xc, I0, J0);
    // no Dirichlet node in the tile: all cells around its nodes exist and are
    // fluid (the barrier inside also publishes the staged coarse nodes)
    const bool fast = node_tile_fluid(g, blockIdx.x, blockIdx.y);
    __syncthreads();   // publishes the staged coarse nodes
    const int J = J0 + threadIdx.x / (PTX / 4);
    const int Ib = I0 + 4 * (threadIdx.x % (PTX / 4));
    if (J > g.nyf) return;
    T val[3][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int I = Ib + q;
        T x[3];
        cw.interp(I, J, x);
        if (!fast && I <= g.nxf) dirichlet_value(g, I, J, up, x[0], x[1]);
#pragma unroll
        for (int c = 0; c < 3; ++c) val[c][q] = x[c];
    }
    const size_t node = (size_t)J * g.pitch + Ib;   // 4-aligned in a 64-aligned row
#pragma unroll
    for (int c = 0; c < 3; ++c) store4(xf + (size_t)c * g.plane + node, val[c]);
}

// ------------------------------------------------------------------ S2 + S3
// Two FP32 values in one 64-bit register pair, operated on by the packed
// f32x2 instructions of sm_100 and later: one issue slot gives two results,
// each rounded as its scalar form would be.  Passes that work on two cells or
// two nodes side by side use them; FP64 tiles use a plain pair of doubles.
struct F2 {
    unsigned long long r;
};
struct D2 {
    double a, b;
};
__device__ __forceinline__ F2 pack2(float a, float b) {
    F2 p;
    asm("mov.b64 %0, {%1, %2};" : "=l"(p.r) : "f"(a), "f"(b));
    return p;
}
__device__ __forceinline__ void unpack2(F2 p, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(p.r));
}
__device__ __forceinline__ F2 vadd(F2 a, F2 b) {
    F2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
__device__ __forceinline__ F2 vsub(F2 a, F2 b) {
    F2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
__device__ __forceinline__ F2 vmul(F2 a, F2 b) {
    F2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
__device__ __forceinline__ F2 vfma(F2 a, F2 b, F2 c) {   // a b + c
    F2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.r) : "l"(a.r), "l"(b.r), "l"(c.r));
    return d;
}
__device__ __forceinline__ D2 pack2(double a, double b) { return D2{a, b}; }
__device__ __forceinline__ void unpack2(D2 p, double &a, double &b) {
    a = p.a;
    b = p.b;
}
__device__ __forceinline__ D2 vadd(D2 x, D2 y) { return D2{__dadd_rn(x.a, y.a), __dadd_rn(x.b, y.b)}; }
__device__ __forceinline__ D2 vsub(D2 x, D2 y) { return D2{__dsub_rn(x.a, y.a), __dsub_rn(x.b, y.b)}; }
__device__ __forceinline__ D2 vmul(D2 x, D2 y) { return D2{__dmul_rn(x.a, y.a), __dmul_rn(x.b, y.b)}; }
__device__ __forceinline__ D2 vfma(D2 x, D2 y, D2 z) { return D2{__fma_rn(x.a, y.a, z.a), __fma_rn(x.b, y.b, z.b)}; }
// scalar forms, so one template serves one cell or two
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double vadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double vsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double vmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return __fma_rn(a, b, c); }
template <typename T> struct Packed;
template <> struct Packed<float> { using type = F2; };
template <> struct Packed<double> { using type = D2; };

template <typename V> __device__ __forceinline__ V splat(float x) { return pack2(x, x); }
template <> __device__ __forceinline__ float splat<float>(float x) { return x; }
template <typename V> __device__ __forceinline__ V splat(double x) { return pack2(x, x); }
template <> __device__ __forceinline__ double splat<double>(double x) { return x; }

// Constants of the convection term in the value type V (one cell or a pair).
template <typename V> struct ConvK {
    V g0, g1, ihx, ihy, w0, w1;
    template <typename T> __device__ __forceinline__ explicit ConvK(const FemCoef<T> &fc)
        : g0(splat<V>(fc.cg0)), g1(splat<V>(fc.cg1)), ihx(splat<V>(fc.inv_hx)), ihy(splat<V>(fc.inv_hy)),
          w0(splat<V>(fc.cwg0)), w1(splat<V>(fc.cwg1)) {}
};

// 1/2 (v.grad v_c, phi_a) of one cell for its corners a = SW, SE, NW, NE, by
// 2x2 Gauss in tensor-product form: values and derivatives at the 4 points
// from edge interpolants, then the test-function sums one direction at a time.
template <typename V>
__device__ __forceinline__ void convection(const ConvK<V> &k, const V (&u)[4], const V (&v)[4], V (&cu)[4],
                                           V (&cv)[4]) {
    // along x on the bottom (0, 1) and top (2, 3) edges
    const V dub = vsub(u[1], u[0]), dut = vsub(u[3], u[2]), dvb = vsub(v[1], v[0]), dvt = vsub(v[3], v[2]);
    const V ub[2] = {vfma(k.g0, dub, u[0]), vfma(k.g1, dub, u[0])};
    const V ut[2] = {vfma(k.g0, dut, u[2]), vfma(k.g1, dut, u[2])};
    const V vb[2] = {vfma(k.g0, dvb, v[0]), vfma(k.g1, dvb, v[0])};
    const V vt[2] = {vfma(k.g0, dvt, v[2]), vfma(k.g1, dvt, v[2])};
    // x-derivatives depend on eta only, y-derivatives on xi only
    const V ddu = vsub(dut, dub), ddv = vsub(dvt, dvb);
    const V ux[2] = {vfma(k.g0, ddu, dub), vfma(k.g1, ddu, dub)};
    const V vx[2] = {vfma(k.g0, ddv, dvb), vfma(k.g1, ddv, dvb)};
    const V uy[2] = {vsub(ut[0], ub[0]), vsub(ut[1], ub[1])};
    const V vy[2] = {vsub(vt[0], vb[0]), vsub(vt[1], vb[1])};
    V c_u[2][2], c_v[2][2];   // [eta index j][xi index i]
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const V gj = j ? k.g1 : k.g0;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const V U = vmul(vfma(gj, uy[i], ub[i]), k.ihx);
            const V W = vmul(vfma(gj, vy[i], vb[i]), k.ihy);
            c_u[j][i] = vfma(U, ux[j], vmul(W, uy[i]));
            c_v[j][i] = vfma(U, vx[j], vmul(W, vy[i]));
        }
    }
    // test with l_0(g) = 1 - g, l_1(g) = g (1 - g0 = g1), weights (qw / 2)
    V su[2][2], sv[2][2];   // [j][ax]
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        su[j][0] = vfma(k.g1, c_u[j][0], vmul(k.g0, c_u[j][1]));
        su[j][1] = vfma(k.g0, c_u[j][0], vmul(k.g1, c_u[j][1]));
        sv[j][0] = vfma(k.g1, c_v[j][0], vmul(k.g0, c_v[j][1]));
        sv[j][1] = vfma(k.g0, c_v[j][0], vmul(k.g1, c_v[j][1]));
    }
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
        cu[ax] = vfma(k.w1, su[0][ax], vmul(k.w0, su[1][ax]));
        cu[2 + ax] = vfma(k.w0, su[0][ax], vmul(k.w1, su[1][ax]));
        cv[ax] = vfma(k.w1, sv[0][ax], vmul(k.w0, sv[1][ax]));
        cv[2 + ax] = vfma(k.w0, sv[0][ax], vmul(k.w1, sv[1][ax]));
    }
}

// Shared-memory layout of the residual/feature tile (element counts).  The
// node window of x~ spans columns I0-4 .. I0+35 (16-byte aligned; node I0+ii
// at column ii+4) and rows J0-2 .. J0+18 (node J0+jj at row jj+2).
struct ResLayout {
    static constexpr int HX = 40, HY = NYN + 4, XO = 4, YO = 2, HP = HX * HY;
    static constexpr int BX = 36;                              // b_f window: columns I0 .. I0+35
    static constexpr int CX = TXC + 2, CY = TYC + 2;           // cells -1 .. 32 x -1 .. 16
    static constexpr int NCELL = CX * CY;
    // cell contributions: one array per (component, corner), pitch NCP; the
    // arrays of the west corners (SW, NW) start one element later so that the
    // two nodes of a block read each array as one aligned pair
    static constexpr int NCP = NCELL + 4;
    static constexpr int LX = TXC / 2 + 2, LY = TYC / 2 + 2;   // LPS patches touching the tile
    static constexpr int NLPS = LX * LY;
    static constexpr int FX = TXC + 4, FY = TYC + 4;           // cell codes with 2-cell halo
    static constexpr int XS = 3 * HP;
    static constexpr int BS = 2 * NYN * BX;
    static constexpr int CC = 8 * NCP;
    static constexpr int LC = 9 * NLPS;
    static constexpr int MAXCS = 3 * ((HX - 1) / 2 + 3) * ((HY - 1) / 2 + 3);   // coarse window, R = 2
    // the coarse window is dead once x~ is formed, the LPS buffer is born after
    static constexpr int UN = LC > MAXCS ? LC : MAXCS;
    static constexpr int MAXP = (TXC / 2) * (TYC / 2);         // patches of a tile (S = 2)
    static constexpr int NBX = TXC / 2 + 1, NBY = TYC / 2 + 1, NB = NBX * NBY;   // 2x2 node blocks
    // node residuals of a fast tile in the feature type: [3][NYN][RXP] (the
    // feature table's residual offsets use this layout from a patch's origin)
    static constexpr int RXP = NXN + 1, RPL = NYN * RXP;
    static constexpr int MAX_LDX = 1024;                       // feature columns supported
    template <typename T> static constexpr size_t bytes() {
        return sizeof(T) * (XS + BS + CC + UN) + sizeof(int) * MAXP + FX * FY;
    }
    // element of corner k (0..3: u rows of SW, SE, NW, NE; 4..7: v rows) of cell cid
    static __device__ __forceinline__ int ccx(int k, int cid) { return k * NCP + cid + ((k & 1) ^ 1); }
};

enum { FEAT_RES = 0, FEAT_VEL = 1, FEAT_PECLET = 2, FEAT_GEO = 3, FEAT_ZERO = 4 };

// x~ = P x_c on the node window of a residual tile (Sec. 3 prolongation).
// One item is one window column inside one coarse cell row: the blends
// along x on the cell's bottom and top edges are formed once and the R
// nodes of the item read off them, with the arithmetic of CoarseWin::interp
// (same bits).  Lanes take consecutive columns.
template <typename T, int R, typename CWin>
__device__ __forceinline__ void interp_window(const CWin &cw, int I0, int J0, T *xs) {
    using L = ResLayout;
    constexpr int K = Log2<R>::v;
    constexpr T inv_r = T(1) / T(R);
    // J0 is a multiple of 16, so the window's first row sits OFFY rows into its coarse cell
    constexpr int OFFY = (R - L::YO % R) % R;
    constexpr int NKY = (L::HY + OFFY + R - 1) / R;
    for (int e = threadIdx.x; e < NKY * L::HX; e += blockDim.x) {
        const int ky = e / L::HX, col = e - ky * L::HX;
        const int I = I0 - L::XO + col;
        const T a = T(I & (R - 1)) * inv_r;
        const T *q = cw.cs + ky * CWin::CW + ((I >> K) - cw.ci0);
        T lo[3], d[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T *qc = q + c * CWin::CW * CWin::CH;
            lo[c] = lerp(qc[0], qc[1], a);
            d[c] = lerp(qc[CWin::CW], qc[CWin::CW + 1], a) - lo[c];
        }
        T *dst = xs + (ky * R - OFFY) * L::HX + col;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int row = ky * R + j - OFFY;
            if (row < 0 || row >= L::HY) continue;
#pragma unroll
            for (int c = 0; c < 3; ++c) dst[c * L::HP + j * L::HX] = fma_t(T(j) * inv_r, d[c], lo[c]);
        }
    }
}

// Residual of tile node (ii, jj) into the feature rows of the patches that
// hold it: its own patch, and the left/lower neighbour when the node lies on
// that patch's edge.  Columns: component c, patch node (lj, li) at
// c nf + lj (S+1) + li (Sec. 5.2 inputs).
template <typename T, typename TX>
__device__ __forceinline__ void put_residual(const MeshGeom &g, TX *__restrict__ X, const int *pid, int tpx,
                                             int tpy, int lS, int ii, int jj, T ru, T rv, T rp) {
    const int S = 1 << lS;
    const int px = ii >> lS, li = ii & (S - 1), py = jj >> lS, lj = jj & (S - 1);
#pragma unroll
    for (int oy = 0; oy < 2; ++oy) {
        if (oy == 0 ? py >= tpy : (lj != 0 || py == 0)) continue;
#pragma unroll
        for (int ox = 0; ox < 2; ++ox) {
            if (ox == 0 ? px >= tpx : (li != 0 || px == 0)) continue;
            const int id = pid[(py - oy) * tpx + px - ox];
            if (id < 0) continue;
            TX *p = X + (size_t)id * g.ldx + (lj + oy * S) * (S + 1) + li + ox * S;
            p[0] = store_as<TX, T>(ru);
            p[g.nf] = store_as<TX, T>(rv);
            p[2 * g.nf] = store_as<TX, T>(rp);
        }
    }
}

// The same for the 2x2 node block (2bx .. 2bx+1, 2by .. 2by+1): the block
// lies in one patch (S is even), and only its even column / row can also
// be the last column / row of the left / lower patch.  Nodes past the tile
// (2bx+1 = 33, 2by+1 = 17) fall outside every patch of the tile and are
// dropped.
template <typename T, typename TX>
__device__ __forceinline__ void put_block(const MeshGeom &g, TX *__restrict__ X, const int *pid, int tpx, int tpy,
                                          int lS, int bx, int by, const T (&ru)[2][2], const T (&rv)[2][2],
                                          const T (&rp)[2][2]) {
    const int S = 1 << lS, S1 = S + 1, nf = g.nf;
    const int px = (2 * bx) >> lS, li = (2 * bx) & (S - 1), py = (2 * by) >> lS, lj = (2 * by) & (S - 1);
    TX *base[2][2];   // [oy][ox]: row of patch (px - ox, py - oy) at the block's first node, or null
#pragma unroll
    for (int oy = 0; oy < 2; ++oy)
#pragma unroll
        for (int ox = 0; ox < 2; ++ox) {
            const bool ok = (oy ? (lj == 0 && py > 0) : py < tpy) && (ox ? (li == 0 && px > 0) : px < tpx);
            const int id = ok ? pid[(py - oy) * tpx + px - ox] : -1;
            base[oy][ox] = id >= 0 ? X + (size_t)id * g.ldx + (lj + oy * S) * S1 + li + ox * S : nullptr;
        }
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx)
#pragma unroll
            for (int oy = 0; oy <= 1 - dy; ++oy)
#pragma unroll
                for (int ox = 0; ox <= 1 - dx; ++ox) {
                    TX *q = base[oy][ox];
                    if (!q) continue;
                    q += (oy ? 0 : dy * S1) + (ox ? 0 : dx);
                    q[0] = store_as<TX, T>(ru[dy][dx]);
                    q[nf] = store_as<TX, T>(rv[dy][dx]);
                    q[2 * nf] = store_as<TX, T>(rp[dy][dx]);
                }
}

// Two adjacent feature values at an even column (4-byte aligned for BF16).
template <typename TX> __device__ __forceinline__ void put_pair(TX *p, TX a, TX b) {
    p[0] = a;
    p[1] = b;
}
template <> __device__ __forceinline__ void put_pair<__nv_bfloat16>(__nv_bfloat16 *p, __nv_bfloat16 a,
                                                                   __nv_bfloat16 b) {
    *reinterpret_cast<__nv_bfloat162 *>(p) = __halves2bfloat162(a, b);
}

// Two adjacent feature values (p even-aligned), converted to the feature type.
template <typename TX, typename T> __device__ __forceinline__ void store_pair(TX *p, T a, T b) {
    p[0] = store_as<TX, T>(a);
    p[1] = store_as<TX, T>(b);
}
template <> __device__ __forceinline__ void store_pair<__nv_bfloat16, float>(__nv_bfloat16 *p, float a, float b) {
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a, b);
}

__device__ __forceinline__ void store2(float *p, float a, float b) { *reinterpret_cast<float2 *>(p) = make_float2(a, b); }
__device__ __forceinline__ void store2(double *p, double a, double b) {
    *reinterpret_cast<double2 *>(p) = make_double2(a, b);
}
__device__ __forceinline__ void ld2(const float *p, float &a, float &b) {
    const float2 t = *reinterpret_cast<const float2 *>(p);
    a = t.x;
    b = t.y;
}
__device__ __forceinline__ void ld2(const double *p, double &a, double &b) {
    const double2 t = *reinterpret_cast<const double2 *>(p);
    a = t.x;
    b = t.y;
}

// Residual of the 2x2 node block (2bx .. 2bx+1, 2by .. 2by+1) of a tile whose
// whole neighbourhood is fluid.  The tile origin is even, so node (2bx+dx,
// 2by+dy) has LPS class (dx, dy): the LPS term is a fixed node stencil, like
// the linear velocity, pressure-gradient and divergence terms; only the
// convection comes from the per-cell contributions in cc.  The zero centre
// column of the x-gradient/divergence stencils (zero centre row in y) is
// skipped.  Window values and cell contributions are read as aligned pairs.
// Nodes 2bx+1 = 33 and 2by+1 = 17 lie past the tile and are discarded.
template <typename T, typename TX>
__device__ __forceinline__ void block_residual(const MeshGeom &g, const FemCoef<T> &fc, const T *xs,
                                               const T *bs, const T *cc, const int *pid, int tpx, int tpy,
                                               int lS, int I0, int J0, int bx, int by, T *__restrict__ rf,
                                               TX *__restrict__ X, TX *rres) {
    using L = ResLayout;
    T Au[2][2], Av[2][2], Ap[2][2];   // [dy][dx]: velocity rows and pressure row of A(x~) x~
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) Au[dy][dx] = Av[dy][dx] = Ap[dy][dx] = T(0);
    // window rows 2by-2 .. 2by+2, columns 2bx-2 .. 2bx+3 (even start: aligned pairs)
    const T *w = xs + (2 * by + L::YO - 2) * L::HX + 2 * bx + L::XO - 2;
#pragma unroll
    for (int ry = 0; ry < 5; ++ry) {
        T u[6], v[6], p[6];
#pragma unroll
        for (int k = 0; k < 6; k += 2) {
            ld2(w + ry * L::HX + 2 * L::HP + k, p[k], p[k + 1]);
            u[k] = u[k + 1] = v[k] = v[k + 1] = T(0);
            if (ry >= 1) {
                ld2(w + ry * L::HX + k, u[k], u[k + 1]);
                ld2(w + ry * L::HX + L::HP + k, v[k], v[k + 1]);
            }
        }
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const int oy = ry - 2 - dy;   // stencil row of this window row for node (dx, dy)
                if (oy >= dy - 2 && oy <= 2 - dy) {
#pragma unroll
                    for (int ox = dx - 2; ox <= 2 - dx; ++ox)
                        Ap[dy][dx] += fc.L5[dy][dx][oy + 2][ox + 2] * p[dx + ox + 2];
                }
                if (oy >= -1 && oy <= 1) {
                    const int sy = oy + 1;
#pragma unroll
                    for (int sx = 0; sx < 3; ++sx) {
                        const int k = dx + sx + 1;
                        Au[dy][dx] += fc.nA[sy][sx] * u[k];
                        Av[dy][dx] += fc.nA[sy][sx] * v[k];
                        if (sx != 1) {
                            Au[dy][dx] -= fc.nGx[sy][sx] * p[k];
                            Ap[dy][dx] += fc.nDx[sy][sx] * u[k];
                        }
                        if (sy != 1) {
                            Av[dy][dx] -= fc.nGy[sy][sx] * p[k];
                            Ap[dy][dx] += fc.nDy[sy][sx] * v[k];
                        }
                    }
                }
            }
    }
    const bool xin = bx < L::NBX - 1, yin = by < L::NBY - 1;   // node 2bx+1 / 2by+1 inside the tile
    const int cb = 2 * by * L::CX + 2 * bx;                    // cell (2bx-1, 2by-1)
    T ru[2][2], rv[2][2], rp[2][2];
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
        ru[dy][0] = ru[dy][1] = rv[dy][0] = rv[dy][1] = T(0);
        rp[dy][0] = -Ap[dy][0];
        rp[dy][1] = -Ap[dy][1];
        if (dy == 1 && !yin) continue;
        // convection: corner contributions of the cells SW, SE, NW, NE of
        // the two nodes of this row (cells c, c+1, c+CX, c+CX+1 of node 0)
        const int c = cb + dy * L::CX;
        T cu[2], cv[2];
#pragma unroll
        for (int comp = 0; comp < 2; ++comp) {
            T a0, a1, b0, b1, d0, d1, e0, e1;
            ld2(cc + L::ccx(4 * comp + 3, c), a0, a1);
            ld2(cc + L::ccx(4 * comp + 2, c + 1), b0, b1);
            ld2(cc + L::ccx(4 * comp + 1, c + L::CX), d0, d1);
            ld2(cc + L::ccx(4 * comp + 0, c + L::CX + 1), e0, e1);
            (comp ? cv : cu)[0] = (a0 + b0) + (d0 + e0);
            (comp ? cv : cu)[1] = (a1 + b1) + (d1 + e1);
        }
        T bu0, bu1, bv0, bv1;
        const int nb = (2 * by + dy) * L::BX + 2 * bx;
        ld2(bs + nb, bu0, bu1);
        ld2(bs + NYN * L::BX + nb, bv0, bv1);
        ru[dy][0] = bu0 - (Au[dy][0] + cu[0]);
        rv[dy][0] = bv0 - (Av[dy][0] + cv[0]);
        if (xin) {
            ru[dy][1] = bu1 - (Au[dy][1] + cu[1]);
            rv[dy][1] = bv1 - (Av[dy][1] + cv[1]);
        }
    }
    if (rf && xin && yin) {   // owned nodes (a fast tile never reaches nxf or nyf)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const size_t node = (size_t)(J0 + 2 * by + dy) * g.pitch + I0 + 2 * bx;
            store2(rf + node, ru[dy][0], ru[dy][1]);
            store2(rf + g.plane + node, rv[dy][0], rv[dy][1]);
            store2(rf + 2 * g.plane + node, rp[dy][0], rp[dy][1]);
        }
    }
    if (rres) {
        // the tile's node residuals, once each (the feature pass gathers the rows)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            if (dy == 1 && !yin) continue;
            const int e = (2 * by + dy) * L::RXP + 2 * bx;   // even: aligned pairs (column 33 is padding)
            store_pair(rres + e, ru[dy][0], ru[dy][1]);
            store_pair(rres + L::RPL + e, rv[dy][0], rv[dy][1]);
            store_pair(rres + 2 * L::RPL + e, rp[dy][0], rp[dy][1]);
        }
        return;
    }
    put_block(g, X, pid, tpx, tpy, lS, bx, by, ru, rv, rp);
}

// S2 + S3 of one tile once its inputs are staged and visible: bs holds the
// b_f window, xs the x~ window (R = 0) or cw the coarse window (R > 0), pid
// the tile's patch numbers, geo_s the geometry features, fast the tile's
// all-fluid flag.  Shared by the per-tile kernel and the persistent one.
template <typename T, typename TX, int R, typename CWin>
__device__ __forceinline__ void residual_tile(const MeshGeom &g, const FemCoef<T> &fc, const CWin &cw,
                                              double inflow_peak, T *xs, const T *bs, T *cc, T *un, const int *pid,
                                              unsigned char *cf, const T *geo_s, bool fast, int I0, int J0,
                                              T *__restrict__ rf, TX *__restrict__ X) {
    using L = ResLayout;
    const int lS = g.K + g.s - 1;   // S = s 2^K with s = 1, 2
    const int tpx = TXC >> lS, tpy = TYC >> lS;
    if (!fast) {
        for (int idx = threadIdx.x; idx < L::FX * L::FY; idx += blockDim.x) {
            const int jj = idx / L::FX, ii = idx - jj * L::FX;
            cf[idx] = (unsigned char)cell_code(g, I0 - 2 + ii, J0 - 2 + jj);
        }
    }
    if constexpr (R > 0) {
        interp_window<T, R>(cw, I0, J0, xs);
        if (!fast) {
            // the Dirichlet velocity where a window node has one (fast tiles
            // have none within the cells they use)
            __syncthreads();
            for (int e = threadIdx.x; e < L::HP; e += blockDim.x) {
                const int jj = e / L::HX, ii = e - jj * L::HX;
                const int I = I0 - L::XO + ii, J = J0 - L::YO + jj;
                if (I >= 0 && I <= g.nxf && J >= 0 && J <= g.nyf)
                    dirichlet_value(g, I, J, inflow_peak, xs[e], xs[L::HP + e]);
            }
        }
    }
    cp_async_wait_all();
    __syncthreads();

    // Feature columns after the residual ones (Sec. 5.2 inputs): x~ and the
    // Peclet number on the coarse patch nodes, geometry, zero padding;
    // feat_tab[c] says where column c comes from relative to the patch
    // origin.  One warp per patch (warps w0 .. w0+nw-1); lanes write
    // consecutive columns.  Fast tiles run it on the warps the 2x2-block
    // pass leaves idle.
    auto patch_inputs = [&](int w0, int nw) {
        const int S = 1 << lS, nres = 3 * g.nf;
        const int warp = (int)(threadIdx.x >> 5) - w0, lane = threadIdx.x & 31;
        for (int tp = warp; tp < tpx * tpy; tp += nw) {
            const int id = pid[tp];
            if (id < 0) continue;
            const int lpy = tp >> (5 - lS), lpx = tp & (tpx - 1);
            const T *xbase = xs + lpy * S * L::HX + lpx * S;
            TX *row = X + (size_t)id * g.ldx;
            for (int c = nres + lane; c < g.ldx; c += 32) {
                const int e = __ldg(g.feat_tab + c);
                const int kind = e >> 24, off = e & 0xFFFFFF;
                const int o = kind <= FEAT_PECLET ? off : 0;
                const T a = xbase[o], b = xbase[o + L::HP];
                T val = kind == FEAT_VEL ? a : (kind == FEAT_GEO ? geo_s[off < 12 ? off : 0] : T(0));
                if (kind == FEAT_PECLET) val = fc.q_over_nu * sqrt(a * a + b * b);
                row[c] = store_as<TX, T>(val);
            }
        }
    };
    // Every feature row of a fast tile, residual columns gathered from the
    // tile's node residuals rres: one warp per patch, lanes on pairs of
    // consecutive columns (coalesced 2-element stores).
    auto patch_rows = [&](const TX *rres) {
        const int S = 1 << lS, nw = (int)(blockDim.x >> 5);
        const int warp = (int)(threadIdx.x >> 5), lane = threadIdx.x & 31;
        for (int tp = warp; tp < tpx * tpy; tp += nw) {
            const int id = pid[tp];
            if (id < 0) continue;
            const int lpy = tp >> (5 - lS), lpx = tp & (tpx - 1);
            const T *xbase = xs + lpy * S * L::HX + lpx * S;
            const TX *rbase = rres + lpy * S * L::RXP + lpx * S;
            TX *row = X + (size_t)id * g.ldx;
            for (int c = 2 * lane; c < g.ldx; c += 64) {
                const int2 ee = __ldg(reinterpret_cast<const int2 *>(g.feat_tab + c));
                TX out[2];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int e = k ? ee.y : ee.x;
                    const int kind = e >> 24, off = e & 0xFFFFFF;
                    if (kind == FEAT_RES) {
                        out[k] = rbase[off];
                    } else {
                        const int o = kind <= FEAT_PECLET ? off : 0;
                        const T a = xbase[o], b = xbase[o + L::HP];
                        T val = kind == FEAT_VEL ? a : (kind == FEAT_GEO ? geo_s[off < 12 ? off : 0] : T(0));
                        if (kind == FEAT_PECLET) val = fc.q_over_nu * sqrt(a * a + b * b);
                        out[k] = store_as<TX, T>(val);
                    }
                }
                put_pair(row + c, out[0], out[1]);
            }
        }
    };

    if (fast) {
        // convection contributions of every cell around the tile's nodes,
        // two vertically adjacent cells per thread in packed arithmetic
        using V = typename Packed<T>::type;
        const ConvK<V> k2(fc);
        for (int e = threadIdx.x; e < L::CX * (L::CY / 2); e += blockDim.x) {
            const int cjp = e / L::CX, ci = e - cjp * L::CX;   // cells (ci-1, 2cjp-1) and (ci-1, 2cjp)
            const int cid = 2 * cjp * L::CX + ci;
            const T *q = xs + (2 * cjp - 1 + L::YO) * L::HX + ci - 1 + L::XO;   // SW node of the lower cell
            V u[4], v[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {   // corners SW, SE, NW, NE
                const int o = (b >> 1) * L::HX + (b & 1);
                u[b] = pack2(q[o], q[o + L::HX]);
                v[b] = pack2(q[L::HP + o], q[L::HP + o + L::HX]);
            }
            V cu[4], cv[4];
            convection(k2, u, v, cu, cv);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                T lo, hi;
                unpack2(cu[a], lo, hi);
                cc[L::ccx(a, cid)] = lo;
                cc[L::ccx(a, cid + L::CX)] = hi;
                unpack2(cv[a], lo, hi);
                cc[L::ccx(4 + a, cid)] = lo;
                cc[L::ccx(4 + a, cid + L::CX)] = hi;
            }
        }
        __syncthreads();
        // Node residuals in the feature type fit in the LPS / coarse-window
        // buffer that fast tiles no longer need when the features are BF16:
        // each node's residual is then written once and the rows gathered
        // afterwards.  Otherwise every node is written into each patch row
        // that holds it while idle warps write the other columns.
        constexpr bool kGather = 3 * L::RPL * sizeof(TX) <= L::LC * sizeof(T);
        TX *rres = kGather ? reinterpret_cast<TX *>(un) : nullptr;
        // 16 blocks of one row per half-warp (contiguous pairs: conflict-free
        // 64-bit loads), then the last block column
        constexpr int BW = (L::NB + 31) / 32;   // warps of the block pass
        if (threadIdx.x < L::NB) {
            const int t = threadIdx.x;
            const bool main = t < 16 * L::NBY;
            const int bx = main ? (t & 15) : L::NBX - 1, by = main ? (t >> 4) : t - 16 * L::NBY;
            block_residual(g, fc, xs, bs, cc, pid, tpx, tpy, lS, I0, J0, bx, by, rf, X, rres);
        } else if (!kGather && threadIdx.x >= 32 * BW) {
            patch_inputs(BW, (int)(blockDim.x >> 5) - BW);
        }
        if constexpr (kGather) {
            __syncthreads();
            patch_rows(rres);
        }
        return;
    }
    patch_inputs(0, blockDim.x >> 5);

    // ---- tiles near a boundary: element by element, with the cell codes
    T *lc = un;   // [9][NLPS]
    const ConvK<T> k1(fc);
    // Phase A: velocity-row contributions of every fluid cell
    for (int cid = threadIdx.x; cid < L::NCELL; cid += blockDim.x) {
        const int ci = cid % L::CX - 1, cj = cid / L::CX - 1;
        T out[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) out[k] = T(0);
        if (cf[(cj + 2) * L::FX + ci + 2] == 1) {
            const int base = (cj + L::YO) * L::HX + ci + L::XO;
            const int off[4] = {0, 1, L::HX, L::HX + 1};
            T u[4], v[4], p[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                u[b] = xs[base + off[b]];
                v[b] = xs[L::HP + base + off[b]];
                p[b] = xs[2 * L::HP + base + off[b]];
            }
            T cu[4], cv[4];
            convection(k1, u, v, cu, cv);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                T au = T(0), av = T(0);
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    au += fc.Av[a][b] * u[b] - fc.Gx[a][b] * p[b];
                    av += fc.Av[a][b] * v[b] - fc.Gy[a][b] * p[b];
                }
                out[a] = cu[a] + au;
                out[4 + a] = cv[a] + av;
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) cc[L::ccx(k, cid)] = out[k];
    }
    // Phase A': LPS contributions of every fluid 2x2-cell patch touching the tile
    for (int lid = threadIdx.x; lid < L::NLPS; lid += blockDim.x) {
        const int m = lid % L::LX - 1, n = lid / L::LX - 1;
        T out[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) out[i] = T(0);
        if (cf[(2 * n + 2) * L::FX + 2 * m + 2] == 1) {
            T p9[9];
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    p9[3 * b + a] = xs[2 * L::HP + (2 * n + b + L::YO) * L::HX + 2 * m + a + L::XO];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                T acc = T(0);
#pragma unroll
                for (int k = 0; k < 9; ++k) acc += fc.S9[i][k] * p9[k];
                out[i] = acc;
            }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) lc[i * L::NLPS + lid] = out[i];
    }
    __syncthreads();

    // Phase B: residual per tile node (pull from the 4 cells and the LPS patches).
    for (int nid = threadIdx.x; nid < NXN * NYN; nid += blockDim.x) {
        const int jj = nid / NXN, ii = nid - jj * NXN;
        const int I = I0 + ii, J = J0 + jj;
        if (I > g.nxf || J > g.nyf) continue;
        const int cells[4] = {jj * L::CX + ii, jj * L::CX + ii + 1, (jj + 1) * L::CX + ii,
                              (jj + 1) * L::CX + ii + 1};   // cells SW, SE, NW, NE of the node
        const int corner[4] = {3, 2, 1, 0};
        T Au = T(0), Av = T(0), Ap = T(0);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            Au += cc[L::ccx(corner[t], cells[t])];
            Av += cc[L::ccx(4 + corner[t], cells[t])];
        }
        const T *pu = xs + (jj + L::YO - 1) * L::HX + ii + L::XO - 1;   // node (ii-1, jj-1)
        const T *pv = pu + L::HP;
        // divergence rows from the fluid cells around the node
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int cx = t & 1, cy = t >> 1;   // cell SW, SE, NW, NE of the node
            if (cf[(jj + 1 + cy) * L::FX + ii + 1 + cx] != 1) continue;
            const int a = corner[t];
            const T *cu = pu + cy * L::HX + cx, *cvp = pv + cy * L::HX + cx;
            const T ub[4] = {cu[0], cu[1], cu[L::HX], cu[L::HX + 1]};
            const T vb[4] = {cvp[0], cvp[1], cvp[L::HX], cvp[L::HX + 1]};
#pragma unroll
            for (int b = 0; b < 4; ++b) Ap += fc.Dx[a][b] * ub[b] + fc.Dy[a][b] * vb[b];
        }
        const int nmx = (ii & 1) ? 1 : 2, nmy = (jj & 1) ? 1 : 2;
        for (int ty = 0; ty < nmy; ++ty) {
            const int n = (jj & 1) ? (jj - 1) / 2 : jj / 2 - 1 + ty;
            const int b = (jj & 1) ? 1 : (ty == 0 ? 2 : 0);
            for (int tx = 0; tx < nmx; ++tx) {
                const int m = (ii & 1) ? (ii - 1) / 2 : ii / 2 - 1 + tx;
                const int a = (ii & 1) ? 1 : (tx == 0 ? 2 : 0);
                Ap += lc[(3 * b + a) * L::NLPS + (n + 1) * L::LX + m + 1];
            }
        }
        const NodeClass nc = classify(cf[(jj + 1) * L::FX + ii + 1], cf[(jj + 1) * L::FX + ii + 2],
                                      cf[(jj + 2) * L::FX + ii + 1], cf[(jj + 2) * L::FX + ii + 2], I, J, g.nyf);
        T ru = T(0), rv = T(0), rp = T(0);
        if (!nc.dirichlet) {
            ru = bs[jj * L::BX + ii] - Au;
            rv = bs[NYN * L::BX + jj * L::BX + ii] - Av;
        }
        if (nc.p_active) rp = -Ap;
        // a node on the tile's right/top edge belongs to the next tile
        // (which may take the other path): write owned nodes only
        if (rf && (ii < TXC || I == g.nxf) && (jj < TYC || J == g.nyf)) {
            const size_t node = (size_t)J * g.pitch + I;
            rf[node] = ru;
            rf[g.plane + node] = rv;
            rf[2 * g.plane + node] = rp;
        }
        put_residual(g, X, pid, tpx, tpy, lS, ii, jj, ru, rv, rp);
    }
}

// S2 + S3 for one 32 x 16-cell tile.  R = 0: x~ is read from xf (S1 done by
// the caller); R = 2, 4, 8: x~ is interpolated from the coarse vector xc
// inside the tile (S1 fused: x~ never reaches HBM), with the Dirichlet
// values set where the tile touches a boundary.
template <typename T, typename TX, int R>
__global__ void __launch_bounds__(RES_THREADS)
k_residual_features(MeshGeom g, FemCoef<T> fc, const T *__restrict__ xf, const double *__restrict__ xc,
                    double inflow_peak, const T *__restrict__ bf, T *__restrict__ rf, TX *__restrict__ X) {
    using L = ResLayout;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T geo_s[12];
    T *xs = reinterpret_cast<T *>(smem_raw);   // [3][HY][HX]   u, v, p
    T *bs = xs + L::XS;                        // [2][NYN][BX]  b_u, b_v
    T *cc = bs + L::BS;                        // [8][NCP]      cell contributions (velocity rows)
    T *un = cc + L::CC;                        // coarse window (R > 0), then [9][NLPS] LPS contributions
    int *pid = reinterpret_cast<int *>(un + L::UN);                          // [tpy][tpx] patch numbers
    unsigned char *cf = reinterpret_cast<unsigned char *>(pid + L::MAXP);   // [FY][FX] cell codes

    const int I0 = blockIdx.x * TXC, J0 = blockIdx.y * TYC;
    const int lS = g.K + g.s - 1;   // S = s 2^K with s = 1, 2
    const int tpx = TXC >> lS, tpy = TYC >> lS;
    stage_window<T, 2, NYN, L::BX>(g, bf, I0, J0, bs);
    using CWin = CoarseWin<T, (R > 0 ? R : 2), L::HX, L::HY>;
    CWin cw;
    cw.cs = un;
    if constexpr (R > 0) {
        static_assert(CWin::N <= L::UN, "coarse window");
        cw.stage(g, xc, I0 - L::XO, J0 - L::YO);
    } else {
        stage_window<T, 3, L::HY, L::HX>(g, xf, I0 - L::XO, J0 - L::YO, xs);
    }
    for (int e = threadIdx.x; e < tpx * tpy; e += blockDim.x) {
        const int py = e >> (5 - lS), px = e & (tpx - 1);
        const int pi = (I0 >> lS) + px, pj = (J0 >> lS) + py;
        pid[e] = (pi < g.npx && pj < g.npy) ? g.patch_id[pj * g.npx + pi] : -1;
    }
    if (threadIdx.x < 12) geo_s[threadIdx.x] = fc.geo[threadIdx.x];
    // fast tiles: every cell within two of the tile is fluid and exists, so
    // no tile node is a boundary node and node stencils apply everywhere
    // (the barrier inside also publishes the coarse window, pid and geo_s)
    const bool fast = tile_fluid(g, blockIdx.x, blockIdx.y, 1);
    __syncthreads();   // publishes the coarse window, pid and geo_s
    residual_tile<T, TX, R>(g, fc, cw, inflow_peak, xs, bs, cc, un, pid, cf, geo_s, fast, I0, J0, rf, X);
}

// ------------------------------------------------------------------ S1 staging
// The coarse vector in the fine arithmetic type with rows padded to pc, so
// that the step's tiles fetch coarse windows by TMA (the coarse planes have
// an odd row length, which a TMA stride cannot express) and convert nothing.
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
k_coarse_pad(MeshGeom g, const double *__restrict__ xc, T *__restrict__ xcp, int pc) {
    // four consecutive outputs of one padded row per thread (pc is a multiple
    // of 32, so they never straddle rows and leave as one aligned store)
    const int nc1 = g.nxc + 1, quads = pc / 4;
    const long long nq = 3LL * (g.nyc + 1) * quads;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nq; e += (long long)gridDim.x * blockDim.x) {
        const long long row = e / quads;
        const int i = (int)(e - row * quads) * 4;
        const double *src = xc + row * nc1;   // rows of [3][nyc+1][nxc+1] are consecutive
        T v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = i + k < nc1 ? (T)__ldg(src + i + k) : T(0);
        store4(xcp + row * pc + i, v);
    }
}

// Shared-memory layout of the TMA-fed residual kernel (bytes; the TMA
// destinations 128-byte aligned): the work buffers of ResLayout plus the
// b_f window and the coarse window as TMA boxes.
template <typename T, int R>
struct StepLayout {
    using L = ResLayout;
    using CWin = CoarseWin<T, R, L::HX, L::HY, 3, 4>;
    static constexpr size_t BS_BYTES = sizeof(T) * L::BS, CS_BYTES = sizeof(T) * CWin::N;
    static constexpr size_t BSB = 0;                                             // [2][NYN][BX]
    static constexpr size_t CSB = (BSB + BS_BYTES + 127) / 128 * 128;            // [3][CH][CW]
    static constexpr size_t XS = (CSB + CS_BYTES + 127) / 128 * 128;
    static constexpr size_t CC = XS + sizeof(T) * L::XS;
    static constexpr size_t UN = CC + sizeof(T) * L::CC;
    static constexpr size_t PID = UN + sizeof(T) * L::LC;
    static constexpr size_t CF = PID + sizeof(int) * L::MAXP;
    static constexpr size_t MB = (CF + L::FX * L::FY + 7) / 8 * 8;
    static constexpr size_t BYTES = MB + 16 + 128;   // barrier and abort flag; base alignment slack
};

// S2 + S3 of the correction step, one CTA per tile: one thread fetches the
// b_f window and the coarse window (from the padded copy) as two TMA boxes
// while the others load the patch numbers; then as residual_tile.  The wait
// is bounded: on time-out the mesh status gets DNNMG_DEVERR_TIMEOUT and the
// CTA returns once its copies have landed.
template <typename T, typename TX, int R>
__global__ void __launch_bounds__(RES_THREADS)
k_residual_step(MeshGeom g, FemCoef<T> fc, const __grid_constant__ CUtensorMap tmB,
                const __grid_constant__ CUtensorMap tmC, double inflow_peak, TX *__restrict__ X,
                const int *__restrict__ tile_list) {
    using L = ResLayout;
    using SL = StepLayout<T, R>;
    using CWin = typename SL::CWin;
    constexpr int K = Log2<R>::v;
    // tile_list (when the closed-form kernel does the all-fluid tiles): the
    // other tiles, one per CTA; otherwise the grid covers every tile
    int tx = blockIdx.x, ty = blockIdx.y;
    if (tile_list) {
        const int tile = __ldg(tile_list + blockIdx.x);
        ty = tile / g.ntx;
        tx = tile - ty * g.ntx;
    }
    extern __shared__ unsigned char smem_raw[];
    __shared__ T geo_s[12];
    // aligned by an offset from the shared-memory symbol itself, so that every
    // access through base stays a shared-memory access (no generic pointers)
    unsigned char *base = smem_raw + ((128u - (ptx::smem_u32(smem_raw) & 127u)) & 127u);
    const T *bs = reinterpret_cast<const T *>(base + SL::BSB);
    T *xs = reinterpret_cast<T *>(base + SL::XS);
    T *cc = reinterpret_cast<T *>(base + SL::CC);
    T *un = reinterpret_cast<T *>(base + SL::UN);
    int *pid = reinterpret_cast<int *>(base + SL::PID);
    unsigned char *cf = base + SL::CF;
    uint64_t *mb = reinterpret_cast<uint64_t *>(base + SL::MB);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(mb + 1);
    const uint32_t mb_u = ptx::smem_u32(mb);
    const int I0 = tx * TXC, J0 = ty * TYC;
    CWin cw;
    cw.cs = reinterpret_cast<T *>(base + SL::CSB);
    cw.ci0 = ((I0 - L::XO) >> K) & ~3;
    cw.cj0 = (J0 - L::YO) >> K;
    if (threadIdx.x == 0) {
        ptx::mbar_init(mb_u, 1);
        *abort_flag = 0;
        ptx::mbar_init_fence();
        ptx::expect_tx(mb_u, (uint32_t)(SL::BS_BYTES + SL::CS_BYTES));
        ptx::tma_load_3d(ptx::smem_u32(base + SL::BSB), &tmB, I0, J0, 0, mb_u);
        ptx::tma_load_3d(ptx::smem_u32(base + SL::CSB), &tmC, cw.ci0, cw.cj0, 0, mb_u);
    }
    const int lS = g.K + g.s - 1;
    const int tpx = TXC >> lS, tpy = TYC >> lS;
    for (int e = threadIdx.x; e < tpx * tpy; e += blockDim.x) {
        const int py = e >> (5 - lS), px = e & (tpx - 1);
        const int pi = (I0 >> lS) + px, pj = (J0 >> lS) + py;
        pid[e] = (pi < g.npx && pj < g.npy) ? __ldg(g.patch_id + pj * g.npx + pi) : -1;
    }
    if (threadIdx.x < 12) geo_s[threadIdx.x] = fc.geo[threadIdx.x];
    const bool fast = tile_fluid(g, tx, ty, 1);
    __syncthreads();   // the barrier is initialised; pid and geo_s are visible
    const bool ok = ptx::mbar_test(mb_u, 0) || ptx::mbar_wait(mb_u, 0, abort_flag);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
            atomicOr(g.status, DNNMG_DEVERR_TIMEOUT);
            volatile int no_abort = 0;   // let the copies in flight land before leaving
            ptx::mbar_wait(mb_u, 0, &no_abort);
        }
        return;
    }
    residual_tile<T, TX, R>(g, fc, cw, inflow_peak, xs, bs, cc, un, pid, cf, geo_s, fast, I0, J0, nullptr, X);
}

// ------------------------------------------------------------------ S5
// Patch numbers of every patch holding a node of the window [Ilo, Ihi] x
// [Jlo, Jhi]: columns px0 .. px0+npw-1, rows py0 .. py0+nph-1 (-1: none).
struct PatchWin {
    int *pid;
    int px0, py0, npw, lS;
    __device__ __forceinline__ void stage(const MeshGeom &g, int Ilo, int Ihi, int Jlo, int Jhi) {
        lS = g.K + g.s - 1;   // S = s 2^K with s = 1, 2
        px0 = (Ilo >> lS) - 1;
        py0 = (Jlo >> lS) - 1;
        npw = (Ihi >> lS) - px0 + 1;
        const int nph = (Jhi >> lS) - py0 + 1;
        for (int e = threadIdx.x; e < npw * nph; e += blockDim.x) {
            const int b = e / npw, a = e - b * npw;
            const int pi = px0 + a, pj = py0 + b;
            pid[e] = (pi >= 0 && pj >= 0 && pi < g.npx && pj < g.npy) ? __ldg(g.patch_id + pj * g.npx + pi) : -1;
        }
    }
    // The mean of d over the fluid patches holding node (I, J) (the averaged
    // correction: every patch holding a node contributes its network output
    // for that node).  In two parts so that callers can issue the loads of
    // several nodes before using any: the node's own patch (first), then on
    // patch edges the left, lower and lower-left neighbours.
    template <typename T>
    __device__ __forceinline__ void own_patch(const MeshGeom &g, const T *__restrict__ d, int I, int J, T &su, T &sv,
                                              int &cnt) const {
        const int S = 1 << lS;
        const int id = pid[((J >> lS) - py0) * npw + (I >> lS) - px0];
        su = sv = T(0);
        cnt = 0;
        if (id >= 0) {
            const T *q = d + (size_t)id * g.n_out + (J & (S - 1)) * (S + 1) + (I & (S - 1));
            su = __ldg(q);
            sv = __ldg(q + g.nf);
            cnt = 1;
        }
    }
    template <typename T>
    __device__ __forceinline__ void edge_patches(const MeshGeom &g, const T *__restrict__ d, int I, int J, T &su, T &sv,
                                                 int &cnt) const {
        const int S = 1 << lS;
        const int row = (J >> lS) - py0, lj = J & (S - 1), col = (I >> lS) - px0, li = I & (S - 1);
        if (lj != 0 && li != 0) return;
#pragma unroll
        for (int o = 1; o < 4; ++o) {   // (ox, oy) = (1, 0), (0, 1), (1, 1)
            const int ox = o & 1, oy = o >> 1;
            if ((ox && li != 0) || (oy && lj != 0)) continue;
            const int id = pid[(row - oy) * npw + col - ox];
            if (id < 0) continue;
            const T *q = d + (size_t)id * g.n_out + (lj + oy * S) * (S + 1) + li + ox * S;
            su += __ldg(q);
            sv += __ldg(q + g.nf);
            ++cnt;
        }
    }
    template <typename T> static __device__ __forceinline__ void add_sum(T su, T sv, int cnt, T &u, T &v) {
        if (cnt) {
            // 1, 1/2 and 1/4 are exact
            const T inv = cnt == 1 ? T(1) : cnt == 2 ? T(0.5) : cnt == 4 ? T(0.25) : T(1) / T(cnt);
            u = fma_t(su, inv, u);
            v = fma_t(sv, inv, v);
        }
    }
    // The same sums for the run of 4 nodes (Ib .. Ib+3, J), Ib a multiple of
    // 4, on a tile where no node is a Dirichlet node (every node has its four
    // cells, so the patches it lies in exist) and S >= 4: the run lies in one
    // patch row, and only its first node can sit on a vertical patch edge.
    // Patch numbers come straight from the global patch map, so the loads can
    // be issued before the tile's staging barrier.  Sums are formed in the
    // order of own_patch + edge_patches (same bits).
    template <typename T>
    static __device__ __forceinline__ void run4(const MeshGeom &g, const T *__restrict__ d, int lS, int Ib, int J,
                                                T (&su)[4], T (&sv)[4], int (&cnt)[4]) {
        const int S = 1 << lS, S1 = S + 1, nf = g.nf;
        const int pi = Ib >> lS, pj = J >> lS, li = Ib & (S - 1), lj = J & (S - 1);
        const int *pm = g.patch_id + (size_t)pj * g.npx + pi;
        const int id = __ldg(pm);
        const bool left = li == 0 && pi > 0, below = lj == 0 && pj > 0;
        const int il = left ? __ldg(pm - 1) : -1, ib = below ? __ldg(pm - g.npx) : -1;
        const int ibl = left && below ? __ldg(pm - g.npx - 1) : -1;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            su[q] = sv[q] = T(0);
            cnt[q] = 0;
        }
        if (id >= 0) {
            const T *p = d + (size_t)id * g.n_out + lj * S1 + li;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                su[q] = __ldg(p + q);
                sv[q] = __ldg(p + nf + q);
                cnt[q] = 1;
            }
        }
        if (il >= 0) {   // left patch, its last column
            const T *p = d + (size_t)il * g.n_out + lj * S1 + S;
            su[0] += __ldg(p);
            sv[0] += __ldg(p + nf);
            ++cnt[0];
        }
        if (ib >= 0) {   // lower patch, its last row
            const T *p = d + (size_t)ib * g.n_out + S * S1 + li;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                su[q] += __ldg(p + q);
                sv[q] += __ldg(p + nf + q);
                ++cnt[q];
            }
        }
        if (ibl >= 0) {   // lower-left patch, its last node
            const T *p = d + (size_t)ibl * g.n_out + S * S1 + S;
            su[0] += __ldg(p);
            sv[0] += __ldg(p + nf);
            ++cnt[0];
        }
    }
};

// All-fluid tiles when S >= 4 (no Dirichlet node; every node's patches
// exist): one 4-node run of one row per thread, with the patch numbers read
// from the global patch map so that the loads of d are in flight while the
// coarse window is staged.  Same arithmetic as the general path, same bits.
template <typename T, int R, typename CWin>
__device__ __forceinline__ void scatter_fast_tile(const MeshGeom &g, const T *__restrict__ d, const T *__restrict__ xf,
                                                  const double *__restrict__ xc, const T *__restrict__ xcp, int pc,
                                                  T *__restrict__ vc, CWin &cw, int I0, int J0) {
    static_assert(NTHREADS == (PTX / 4) * PTY, "one run per thread");
    const int Ib = I0 + 4 * (threadIdx.x & (PTX / 4 - 1)), J = J0 + threadIdx.x / (PTX / 4);
    const size_t node = (size_t)J * g.pitch + Ib;   // 4-aligned in a 64-aligned row
    T su[4], sv[4];
    int cnt[4];
    PatchWin::run4(g, d, g.K + g.s - 1, Ib, J, su, sv, cnt);
    T x[2][4];
    if constexpr (R > 0) {
        if (xcp) cw.stage_padded(g, xcp, pc, I0, J0);
        else cw.stage(g, xc, I0, J0);
        __syncthreads();   // publishes the staged coarse nodes
        cw.interp4(Ib, J, x);
    } else {
        load4(xf + node, x[0]);
        load4(xf + g.plane + node, x[1]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) PatchWin::add_sum(su[q], sv[q], cnt[q], x[0][q], x[1][q]);
    store4(vc + node, x[0]);
    store4(vc + g.plane + node, x[1]);
}

// A CTA owns 64 x 16 nodes.  All-fluid tiles with S >= 4 take
// scatter_fast_tile; otherwise lanes take consecutive nodes of a row (so the
// reads of d are contiguous runs of each patch row), each thread 4 rows.
// R = 0: v~ is read from xf; R = 2, 4, 8: v~ is interpolated from xc inside
// the tile (S1 fused).  Registers are capped for the fast tiles' occupancy;
// the rare general tiles may spill.
template <typename T, int R>
__global__ void __launch_bounds__(NTHREADS, sizeof(T) == 4 ? 6 : 4)
k_scatter_avg(MeshGeom g, const T *__restrict__ d, const T *__restrict__ xf, const double *__restrict__ xc,
              const T *__restrict__ xcp, int pc, double inflow_peak, T *__restrict__ vc) {
    using CWin = CoarseWin<T, (R > 0 ? R : 2), PTX, PTY, 2>;
    __shared__ T cs_mem[R > 0 ? CWin::N : 1];
    __shared__ int pid_s[(PTX / 2 + 2) * (PTY / 2 + 2)];   // S = 2 holds the most patches
    // the first and the two last tile rows (walls: general tiles, the slowest)
    // are scheduled first, so that they do not form the grid's tail
    const int ny = gridDim.y, by = blockIdx.y < 3 ? (blockIdx.y ? ny - blockIdx.y : 0) : blockIdx.y - 2;
    const int I0 = blockIdx.x * PTX, J0 = by * PTY;
    const bool fast = node_tile_fluid(g, blockIdx.x, by);
    CWin cw;
    cw.cs = cs_mem;
    if (fast && g.K + g.s - 1 >= 2) {
        scatter_fast_tile<T, R>(g, d, xf, xc, xcp, pc, vc, cw, I0, J0);
        return;
    }
    PatchWin pw;
    pw.pid = pid_s;
    pw.stage(g, I0, I0 + PTX - 1, J0, J0 + PTY - 1);
    if constexpr (R > 0) {
        if (xcp) cw.stage_padded(g, xcp, pc, I0, J0);
        else cw.stage(g, xc, I0, J0);
    }
    const double up = inflow_peak;
    __syncthreads();   // publishes pid_s and the staged coarse nodes
    const int I = I0 + (threadIdx.x & (PTX - 1));
    if (I > g.nxf) return;
    // this thread's rows; the own-patch loads of all of them are issued first
    constexpr int NR = PTY / (NTHREADS / PTX);
    T u[NR], v[NR], su[NR], sv[NR];
    int cnt[NR];
    bool keep[NR];   // row exists and the node is not a Dirichlet node
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int J = J0 + threadIdx.x / PTX + k * (NTHREADS / PTX);
        const bool live = J <= g.nyf;
        const int Jc = live ? J : g.nyf;   // a valid row for the (unused) reads of a dead one
        if constexpr (R > 0) {
            T x[2];
            cw.interp(I, Jc, x);
            u[k] = x[0];
            v[k] = x[1];
        } else {
            const size_t node = (size_t)Jc * g.pitch + I;
            u[k] = xf[node];
            v[k] = xf[g.plane + node];
        }
        keep[k] = live;
        if (live && !fast) {
            T uD, vD;
            if (dirichlet_value(g, I, J, up, uD, vD)) {   // keeps v~ = the boundary value
                if constexpr (R > 0) {
                    u[k] = uD;
                    v[k] = vD;
                }
                keep[k] = false;
            }
        }
        su[k] = sv[k] = T(0);
        cnt[k] = 0;
        if (keep[k]) pw.own_patch(g, d, I, J, su[k], sv[k], cnt[k]);
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int J = J0 + threadIdx.x / PTX + k * (NTHREADS / PTX);
        if (J > g.nyf) break;
        if (keep[k]) {
            pw.edge_patches(g, d, I, J, su[k], sv[k], cnt[k]);
            PatchWin::add_sum(su[k], sv[k], cnt[k], u[k], v[k]);
        }
        const size_t node = (size_t)J * g.pitch + I;
        vc[node] = u[k];
        vc[g.plane + node] = v[k];
    }
}

// ------------------------------------------------------------------ S6
// Node window of v_corr: columns I0-4 .. I0+35 (node I0+ii at column ii+4),
// rows J0-1 .. J0+17 (node J0+jj at row jj+1).
struct RhsLayout {
    static constexpr int HX = 40, HY = NYN + 2, XO = 4, YO = 1, HP = HX * HY;
    static constexpr int CX = TXC + 2, CY = TYC + 2;   // cells -1 .. 32 x -1 .. 16
    static constexpr int NCELL = CX * CY;
    static constexpr int NCP = NCELL + 4;              // corner arrays, as in ResLayout
    static constexpr int VS = 2 * HP;
    static constexpr int CC = 8 * NCP;
    // v_corr window (a TMA box, 128-byte aligned), cell contributions, cell
    // codes, the barrier and the abort flag, alignment slack
    template <typename T> static constexpr size_t bytes() {
        return (sizeof(T) * (VS + CC) + NCELL + 7) / 8 * 8 + 16 + 128;
    }
    static __device__ __forceinline__ int ccx(int k, int cid) { return k * NCP + cid + ((k & 1) ^ 1); }
};

// Right-hand side (Eq. 4cranknicholson3: (1/k M - nu/2 K) v - 1/2 (v.grad v, phi))
// of the owned nodes of one 32 x 16-cell tile from the v_corr window vs.
// Tiles whose neighbourhood is fluid: convection per cell (two vertically
// adjacent cells per thread in packed arithmetic), then per 2x2 node block
// the node stencil of the linear term plus the four cells' convection
// corners, read as aligned pairs; 16 blocks of a row per half-warp.  Other
// tiles: element by element with the cell codes cf.
template <typename T>
__device__ __forceinline__ void rhs_tile(const MeshGeom &g, const FemCoef<T> &fc, const T *vs, T *cc,
                                         const unsigned char *cf, bool fast, int I0, int J0, T *__restrict__ bf) {
    using L = RhsLayout;
    if (fast) {
        using V = typename Packed<T>::type;
        const ConvK<V> k2(fc);
        for (int e = threadIdx.x; e < L::CX * (L::CY / 2); e += blockDim.x) {
            const int cjp = e / L::CX, ci = e - cjp * L::CX;   // cells (ci-1, 2cjp-1) and (ci-1, 2cjp)
            const int cid = 2 * cjp * L::CX + ci;
            const T *q = vs + (2 * cjp - 1 + L::YO) * L::HX + ci - 1 + L::XO;   // SW node of the lower cell
            V u[4], v[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {   // corners SW, SE, NW, NE
                const int o = (b >> 1) * L::HX + (b & 1);
                u[b] = pack2(q[o], q[o + L::HX]);
                v[b] = pack2(q[L::HP + o], q[L::HP + o + L::HX]);
            }
            V cu[4], cv[4];
            convection(k2, u, v, cu, cv);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                T lo, hi;
                unpack2(cu[a], lo, hi);
                cc[L::ccx(a, cid)] = -lo;
                cc[L::ccx(a, cid + L::CX)] = -hi;
                unpack2(cv[a], lo, hi);
                cc[L::ccx(4 + a, cid)] = -lo;
                cc[L::ccx(4 + a, cid + L::CX)] = -hi;
            }
        }
        __syncthreads();
        if (threadIdx.x < (TXC / 2) * (TYC / 2)) {
            const int bx = threadIdx.x & 15, by = threadIdx.x >> 4;   // nodes 2bx .. 2bx+1, 2by .. 2by+1
            // window rows 2by-1 .. 2by+2, columns 2bx-2 .. 2bx+3 (even start: aligned pairs)
            const T *w = vs + (2 * by + L::YO - 1) * L::HX + 2 * bx + L::XO - 2;
            T Bu[2][2], Bv[2][2];
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) Bu[dy][0] = Bu[dy][1] = Bv[dy][0] = Bv[dy][1] = T(0);
#pragma unroll
            for (int ry = 0; ry < 4; ++ry) {
                T u[6], v[6];
#pragma unroll
                for (int k = 0; k < 6; k += 2) {
                    ld2(w + ry * L::HX + k, u[k], u[k + 1]);
                    ld2(w + ry * L::HX + L::HP + k, v[k], v[k + 1]);
                }
#pragma unroll
                for (int dy = 0; dy < 2; ++dy) {
                    const int sy = ry - dy;
                    if (sy < 0 || sy > 2) continue;
#pragma unroll
                    for (int dx = 0; dx < 2; ++dx)
#pragma unroll
                        for (int sx = 0; sx < 3; ++sx) {
                            Bu[dy][dx] += fc.nB[sy][sx] * u[dx + sx + 1];
                            Bv[dy][dx] += fc.nB[sy][sx] * v[dx + sx + 1];
                        }
                }
            }
            const int cb = 2 * by * L::CX + 2 * bx;   // cell (2bx-1, 2by-1)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                const int c = cb + dy * L::CX;
                T cu[2], cv[2];
#pragma unroll
                for (int comp = 0; comp < 2; ++comp) {
                    T a0, a1, b0, b1, d0, d1, e0, e1;
                    ld2(cc + L::ccx(4 * comp + 3, c), a0, a1);
                    ld2(cc + L::ccx(4 * comp + 2, c + 1), b0, b1);
                    ld2(cc + L::ccx(4 * comp + 1, c + L::CX), d0, d1);
                    ld2(cc + L::ccx(4 * comp + 0, c + L::CX + 1), e0, e1);
                    (comp ? cv : cu)[0] = (a0 + b0) + (d0 + e0);
                    (comp ? cv : cu)[1] = (a1 + b1) + (d1 + e1);
                }
                const size_t node = (size_t)(J0 + 2 * by + dy) * g.pitch + I0 + 2 * bx;
                store2(bf + node, Bu[dy][0] + cu[0], Bu[dy][1] + cu[1]);
                store2(bf + g.plane + node, Bv[dy][0] + cv[0], Bv[dy][1] + cv[1]);
            }
        }
        return;
    }
    const ConvK<T> k1(fc);
    for (int cid = threadIdx.x; cid < L::NCELL; cid += blockDim.x) {
        T out[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) out[k] = T(0);
        if (cf[cid] == 1) {
            const int ci = cid % L::CX, cj = cid / L::CX;   // cell (ci-1, cj-1) of the tile
            const int base = cj * L::HX + ci + L::XO - 1;    // its SW node
            const int off[4] = {0, 1, L::HX, L::HX + 1};
            T u[4], v[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                u[b] = vs[base + off[b]];
                v[b] = vs[L::HP + base + off[b]];
            }
            T cu[4], cv[4];
            convection(k1, u, v, cu, cv);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                T bu = T(0), bv = T(0);
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    bu += fc.Bv[a][b] * u[b];
                    bv += fc.Bv[a][b] * v[b];
                }
                out[a] = bu - cu[a];
                out[4 + a] = bv - cv[a];
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) cc[L::ccx(k, cid)] = out[k];
    }
    __syncthreads();
    for (int nid = threadIdx.x; nid < NXN * NYN; nid += blockDim.x) {
        const int jj = nid / NXN, ii = nid - jj * NXN;
        const int I = I0 + ii, J = J0 + jj;
        if (I > g.nxf || J > g.nyf) continue;
        // a node on the tile's right/top edge belongs to the next tile
        if ((ii == TXC && I < g.nxf) || (jj == TYC && J < g.nyf)) continue;
        const int cells[4] = {jj * L::CX + ii, jj * L::CX + ii + 1, (jj + 1) * L::CX + ii,
                              (jj + 1) * L::CX + ii + 1};
        const int corner[4] = {3, 2, 1, 0};
        T bu = T(0), bv = T(0);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            bu += cc[L::ccx(corner[t], cells[t])];
            bv += cc[L::ccx(4 + corner[t], cells[t])];
        }
        const NodeClass nc = classify(cf[cells[0]], cf[cells[1]], cf[cells[2]], cf[cells[3]], I, J, g.nyf);
        if (nc.dirichlet) bu = bv = T(0);
        const size_t node = (size_t)J * g.pitch + I;
        bf[node] = bu;
        bf[g.plane + node] = bv;
    }
}

// One CTA per tile; one thread fetches the v_corr window as a TMA box (rows
// outside the mesh read as zero) while the others classify the cells of
// boundary tiles.  The wait is bounded: on time-out the mesh status gets
// DNNMG_DEVERR_TIMEOUT and the CTA returns once its copy has landed.
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
k_rhs(MeshGeom g, FemCoef<T> fc, const __grid_constant__ CUtensorMap tmV, T *__restrict__ bf) {
    using L = RhsLayout;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((128u - (ptx::smem_u32(smem_raw) & 127u)) & 127u);
    T *vs = reinterpret_cast<T *>(base);   // [2][HY][HX]
    T *cc = vs + L::VS;                    // [8][NCP]
    unsigned char *cf = reinterpret_cast<unsigned char *>(cc + L::CC);   // [CY][CX]
    uint64_t *mb = reinterpret_cast<uint64_t *>(base + (sizeof(T) * (L::VS + L::CC) + L::NCELL + 7) / 8 * 8);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(mb + 1);
    const uint32_t mb_u = ptx::smem_u32(mb);
    const int I0 = blockIdx.x * TXC, J0 = blockIdx.y * TYC;
    if (threadIdx.x == 0) {
        ptx::mbar_init(mb_u, 1);
        *abort_flag = 0;
        ptx::mbar_init_fence();
        ptx::expect_tx(mb_u, (uint32_t)(sizeof(T) * L::VS));
        ptx::tma_load_3d(ptx::smem_u32(vs), &tmV, I0 - L::XO, J0 - L::YO, 0, mb_u);
    }
    const bool fast = tile_fluid(g, blockIdx.x, blockIdx.y, 2);
    if (!fast) {
        for (int idx = threadIdx.x; idx < L::NCELL; idx += blockDim.x) {
            const int jj = idx / L::CX, ii = idx - jj * L::CX;
            cf[idx] = (unsigned char)cell_code(g, I0 - 1 + ii, J0 - 1 + jj);
        }
    }
    __syncthreads();   // the barrier is initialised; cf is visible
    const bool ok = ptx::mbar_test(mb_u, 0) || ptx::mbar_wait(mb_u, 0, abort_flag);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
            atomicOr(g.status, DNNMG_DEVERR_TIMEOUT);
            volatile int no_abort = 0;   // let the copy land before leaving
            ptx::mbar_wait(mb_u, 0, &no_abort);
        }
        return;
    }
    rhs_tile(g, fc, vs, cc, cf, fast, I0, J0, bf);
}

// S5 + S6 fused for the correction step: the v_corr window of a right-hand
// side tile (x~ = P x_c plus the patch mean of d, Dirichlet values at the
// boundary) is formed in shared memory and never reaches HBM.  The network
// outputs of every patch holding a node of the window are copied into
// shared memory first (one warp per patch row of d, coalesced), so the
// means are formed from shared memory.  Same arithmetic and order as S5
// followed by S6, hence the same bits.
//
// Shared memory: the v_corr window, then a region that first holds the
// coarse window, the window's patch numbers and its d rows, and afterwards
// the cell contributions of the right-hand side, then the cell codes.
template <typename T>
struct AvgRhsLayout {
    using L = RhsLayout;
    // patches holding the nodes I0-1 .. I0+33, J0-1 .. J0+17 that S6 reads
    static __host__ __device__ int npw(int lS) { return ((TXC + 1) >> lS) + 2; }
    static __host__ __device__ int nph(int lS) { return ((TYC + 1) >> lS) + 2; }
    static __host__ size_t region(int R, int lS, int n_out) {
        const size_t cwin = 2 * ((L::HX - 1) / R + 3) * ((L::HY - 1) / R + 3);
        const size_t slots = (size_t)npw(lS) * nph(lS);
        const size_t stage = cwin + slots + slots * n_out;   // pid slots counted as T
        return stage > (size_t)L::CC ? stage : (size_t)L::CC;
    }
    static __host__ size_t bytes(int R, int lS, int n_out) {
        return sizeof(T) * (L::VS + region(R, lS, n_out)) + L::NCELL;
    }
};

template <typename T, int R>
__global__ void __launch_bounds__(NTHREADS)
k_avg_rhs(MeshGeom g, FemCoef<T> fc, const T *__restrict__ d, const double *__restrict__ xc, double inflow_peak,
          T *__restrict__ bf, int region) {
    using L = RhsLayout;
    using AL = AvgRhsLayout<T>;
    using CWin = CoarseWin<T, R, L::HX, L::HY, 2>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *vs = reinterpret_cast<T *>(smem_raw);   // [2][HY][HX]
    T *cc = vs + L::VS;                        // region: staging, then [8][NCP]
    unsigned char *cf = reinterpret_cast<unsigned char *>(cc + region);   // [CY][CX]
    const int I0 = blockIdx.x * TXC, J0 = blockIdx.y * TYC;
    const int Ilo = I0 - L::XO, Jlo = J0 - L::YO;
    const int lS = g.K + g.s - 1, S = 1 << lS;   // S = s 2^K with s = 1, 2
    const int npw = AL::npw(lS), nph = AL::nph(lS), nslot = npw * nph;
    const int pxlo = (I0 - 1) >> lS, pylo = (J0 - 1) >> lS;
    CWin cw;
    cw.cs = cc;
    cw.stage(g, xc, Ilo, Jlo);
    int *spid = reinterpret_cast<int *>(cc + CWin::N);   // [nph][npw]
    T *dw = cc + CWin::N + nslot;                        // [nph][npw][n_out]
    for (int e = threadIdx.x; e < nslot; e += blockDim.x) {
        const int b = e / npw, a = e - b * npw;
        const int pi = pxlo + a, pj = pylo + b;
        spid[e] = (pi >= 0 && pj >= 0 && pi < g.npx && pj < g.npy) ? __ldg(g.patch_id + pj * g.npx + pi) : -1;
    }
    const bool fast = tile_fluid(g, blockIdx.x, blockIdx.y, 2);
    if (!fast) {
        for (int idx = threadIdx.x; idx < L::NCELL; idx += blockDim.x) {
            const int jj = idx / L::CX, ii = idx - jj * L::CX;
            cf[idx] = (unsigned char)cell_code(g, I0 - 1 + ii, J0 - 1 + jj);
        }
    }
    __syncthreads();
    // the d rows of the window's patches, one warp per patch, as asynchronous
    // 8-byte copies all in flight at once (rows are 8-byte aligned: n_out is even)
    {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        const int pieces = (g.n_out * (int)sizeof(T)) / 8, per = 8 / (int)sizeof(T);
        for (int e = warp; e < nslot; e += nw) {
            const int id = spid[e];
            if (id < 0) continue;
            const T *src = d + (size_t)id * g.n_out;
            T *dst = dw + e * g.n_out;
            for (int k = lane; k < pieces; k += 32) cp_async8(dst + k * per, src + k * per);
        }
    }
    const double up = inflow_peak;
    cp_async_wait_all();
    __syncthreads();
    for (int e = threadIdx.x; e < L::HP; e += blockDim.x) {
        const int row = e / L::HX, col = e - row * L::HX;
        const int I = Ilo + col, J = Jlo + row;
        T u = T(0), v = T(0);
        // S6 reads nodes I0-1 .. I0+33; the window's outer columns stay zero
        if (I >= I0 - 1 && I <= I0 + TXC + 1 && I >= 0 && J >= 0 && I <= g.nxf && J <= g.nyf) {
            T x[2];
            cw.interp(I, J, x);
            u = x[0];
            v = x[1];
            T uD, vD;
            if (!fast && dirichlet_value(g, I, J, up, uD, vD)) {
                u = uD;
                v = vD;
            } else {
                // the mean of d over the fluid patches holding the node: own patch
                // first, then on patch edges the left, lower and lower-left ones
                const int sr = (J >> lS) - pylo, sc = (I >> lS) - pxlo, lj = J & (S - 1), li = I & (S - 1);
                T su = T(0), sv = T(0);
                int cnt = 0;
#pragma unroll
                for (int o = 0; o < 4; ++o) {   // (ox, oy) = (0, 0), (1, 0), (0, 1), (1, 1)
                    const int ox = o & 1, oy = o >> 1;
                    if ((ox && li != 0) || (oy && lj != 0)) continue;
                    const int slot = (sr - oy) * npw + sc - ox;
                    if (spid[slot] < 0) continue;
                    const T *q = dw + slot * g.n_out + (lj + oy * S) * (S + 1) + li + ox * S;
                    su += q[0];
                    sv += q[g.nf];
                    ++cnt;
                }
                PatchWin::add_sum(su, sv, cnt, u, v);
            }
        }
        vs[e] = u;
        vs[L::HP + e] = v;
    }
    __syncthreads();
    rhs_tile(g, fc, vs, cc, cf, fast, I0, J0, bf);
}

// ------------------------------------------------------------------ S7
// b_c(J) = sum_i hat_J(x_i) b_f(i), separable: first along x within each fine
// row, then along y.  A CTA owns (128/r) x (32/r) coarse nodes and stages the
// fine rows they need.  Single-precision data are accumulated with error-free
// transformations (a float hi/lo pair: TwoProd by FMA and TwoSum, Dekker /
// Knuth), i.e. to about 2^-44 relative of the sum of magnitudes, and the
// result is stored in FP64; FP64 data are accumulated in FP64.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ void df_fma(DF &acc, float w, float x) {
    const float p = __fmul_rn(w, x);
    const float pe = __fmaf_rn(w, x, -p);              // exact product error
    const float s = __fadd_rn(acc.hi, p);
    const float bb = __fsub_rn(s, acc.hi);
    const float e = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, pe));
}

__device__ __forceinline__ void df_fma(DF &acc, float w, DF x) {
    df_fma(acc, w, x.hi);
    acc.lo = __fmaf_rn(w, x.lo, acc.lo);
}

struct RestrictAcc32 {
    using Row = DF;
    static __device__ __forceinline__ Row zero() { return DF{0.f, 0.f}; }
    static __device__ __forceinline__ void add(Row &a, float w, float x) { df_fma(a, w, x); }
    static __device__ __forceinline__ void add(Row &a, float w, Row x) { df_fma(a, w, x); }
    static __device__ __forceinline__ double out(Row a) { return (double)a.hi + (double)a.lo; }
};
struct RestrictAcc64 {
    using Row = double;
    static __device__ __forceinline__ Row zero() { return 0.0; }
    static __device__ __forceinline__ void add(Row &a, double w, double x) { a += w * x; }
    static __device__ __forceinline__ double out(Row a) { return a; }
};

// Fine columns staged per tile: ci0 r - 8 .. ci0 r + 135 (16-byte aligned start;
// covers ci r +- (r-1) for the tile's 128/r coarse columns when r <= 8).
constexpr int RFW = 128 + 16, RXO = 8;

// One thread fetches the tile's fine window as a TMA box (rows and columns
// outside the mesh read as zero); the wait is bounded (on time-out the mesh
// status gets DNNMG_DEVERR_TIMEOUT and the CTA returns once the copy has landed).
template <typename T, typename Acc, int R>
__global__ void __launch_bounds__(NTHREADS)
k_restrict(MeshGeom g, const __grid_constant__ CUtensorMap tmB, double *__restrict__ bc) {
    using Row = typename Acc::Row;
    constexpr int TCX = 128 / R, TCY = 32 / R;              // coarse nodes per tile
    constexpr int FH = TCY * R + R - 1;                     // fine rows staged
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((128u - (ptx::smem_u32(smem_raw) & 127u)) & 127u);
    T *fs = reinterpret_cast<T *>(base);                    // [2][FH][RFW]
    Row *rs = reinterpret_cast<Row *>(fs + 2 * FH * RFW);   // [2][FH][TCX] x-restricted rows
    uint64_t *mb = reinterpret_cast<uint64_t *>(rs + 2 * FH * TCX);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(mb + 1);
    const uint32_t mb_u = ptx::smem_u32(mb);
    const int ci0 = blockIdx.x * TCX, cj0 = blockIdx.y * TCY;
    if (threadIdx.x == 0) {
        ptx::mbar_init(mb_u, 1);
        *abort_flag = 0;
        ptx::mbar_init_fence();
        ptx::expect_tx(mb_u, (uint32_t)(sizeof(T) * 2 * FH * RFW));
        ptx::tma_load_3d(ptx::smem_u32(fs), &tmB, ci0 * R - RXO, cj0 * R - (R - 1), 0, mb_u);
    }
    __syncthreads();   // the barrier is initialised
    const bool ok = ptx::mbar_test(mb_u, 0) || ptx::mbar_wait(mb_u, 0, abort_flag);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
            atomicOr(g.status, DNNMG_DEVERR_TIMEOUT);
            volatile int no_abort = 0;   // let the copy land before leaving
            ptx::mbar_wait(mb_u, 0, &no_abort);
        }
        return;
    }
    constexpr T inv_r = T(1) / T(R);
    for (int e = threadIdx.x; e < 2 * FH * TCX; e += blockDim.x) {
        const int c = e / (FH * TCX), rem = e - c * (FH * TCX);
        const int jj = rem / TCX, ci = rem - jj * TCX;
        // fine nodes (ci0+ci) R - (R-1) .. (ci0+ci) R + (R-1), staged from column ci R - (R-1) + RXO
        const T *row = fs + c * FH * RFW + jj * RFW + ci * R - (R - 1) + RXO;
        Row acc = Acc::zero();
#pragma unroll
        for (int d = 0; d < 2 * R - 1; ++d) Acc::add(acc, T(R - abs(d - (R - 1))) * inv_r, row[d]);
        rs[e] = acc;
    }
    __syncthreads();
    const size_t nc1 = (size_t)g.nxc + 1, Nc = nc1 * (g.nyc + 1);
    for (int e = threadIdx.x; e < TCX * TCY; e += blockDim.x) {
        const int lj = e / TCX, li = e - lj * TCX;
        const int ci = ci0 + li, cj = cj0 + lj;
        if (ci > g.nxc || cj > g.nyc) continue;
        double out[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            Row acc = Acc::zero();
#pragma unroll
            for (int d = 0; d < 2 * R - 1; ++d)
                Acc::add(acc, T(R - abs(d - (R - 1))) * inv_r, rs[c * FH * TCX + (lj * R + d) * TCX + li]);
            out[c] = Acc::out(acc);
        }
        bool ts = false;
        for (int dj = -1; dj <= 0; ++dj)
            for (int di = -1; di <= 0; ++di) {
                const int i = ci + di, j = cj + dj;
                if (i >= 0 && j >= 0 && i < g.nxc && j < g.nyc && g.solid[(size_t)j * g.nxc + i]) ts = true;
            }
        if (ts || ci == 0 || cj == 0 || cj == g.nyc) out[0] = out[1] = 0.0;
        const size_t node = (size_t)cj * nc1 + ci;
        bc[node] = out[0];
        bc[Nc + node] = out[1];
        bc[2 * Nc + node] = 0.0;
    }
}

template <typename T, typename Acc, int R>
size_t restrict_smem() {
    const size_t FH = (size_t)(32 / R) * R + R - 1;
    // fine window (TMA box), x-restricted rows, barrier and abort flag, alignment slack
    return 2 * FH * RFW * sizeof(T) + 2 * FH * (128 / R) * sizeof(typename Acc::Row) + 16 + 128;
}

template <typename T, typename Acc, int R>
cudaError_t run_restrict(const MeshGeom &g, const T *bf, double *bc, cudaStream_t st) {
    constexpr int TCX = 128 / R, TCY = 32 / R, FH = TCY * R + R - 1;
    // b_f [2][nyf+1][pitch]: boxes of RFW columns x FH rows x 2 components
    CUtensorMap tm;
    const CUtensorMapDataType dt = sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nxf + 1, (cuuint64_t)g.nyf + 1, 2};
    const cuuint64_t str[2] = {(cuuint64_t)g.pitch * sizeof(T), (cuuint64_t)g.plane * sizeof(T)};
    const cuuint32_t box[3] = {(cuuint32_t)RFW, (cuuint32_t)FH, 2};
    if (!tma_encode_tiled(&tm, dt, 3, const_cast<T *>(bf), dims, str, box)) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((g.nxc + TCX) / TCX), (unsigned)((g.nyc + TCY) / TCY));
    const size_t sm = restrict_smem<T, Acc, R>();
    cudaError_t e = cudaFuncSetAttribute(k_restrict<T, Acc, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_restrict<T, Acc, R><<<grid, NTHREADS, sm, st>>>(g, tm, bc);
    return cudaGetLastError();
}

template <typename T, typename Acc>
cudaError_t run_restrict_r(const MeshGeom &g, const T *bf, double *bc, cudaStream_t st) {
    switch (g.r) {
        case 2: return run_restrict<T, Acc, 2>(g, bf, bc, st);
        case 4: return run_restrict<T, Acc, 4>(g, bf, bc, st);
        case 8: return run_restrict<T, Acc, 8>(g, bf, bc, st);
        default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------ maps
__global__ void k_mesh_maps(MeshGeom g, unsigned char *flags, unsigned char *mult) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y;
    if (I > g.nxf) return;
    const size_t node = (size_t)J * g.pitch + I;
    if (flags) {
        const NodeClass nc = classify_global(g, I, J);
        flags[node] = (unsigned char)((nc.dirichlet ? 1 : 0) | (nc.inflow ? 2 : 0) | (nc.p_active ? 4 : 0));
    }
    if (mult) {
        const int S = g.S;
        int cnt = 0;
        for (int pj = (J - 1) / S; pj <= J / S; ++pj)
            for (int pi = (I - 1) / S; pi <= I / S; ++pi) {
                if (pi < 0 || pj < 0 || pi >= g.npx || pj >= g.npy) continue;
                if (I < pi * S || I > (pi + 1) * S || J < pj * S || J > (pj + 1) * S) continue;
                if (g.patch_id[pj * g.npx + pi] >= 0) ++cnt;
            }
        mult[node] = (unsigned char)cnt;
    }
}

dim3 node_grid(const MeshGeom &g) {
    return dim3((unsigned)((g.nxf + 1 + NTHREADS - 1) / NTHREADS), (unsigned)(g.nyf + 1));
}
dim3 tile_grid(const MeshGeom &g) {
    return dim3((unsigned)((g.nxf + TXC - 1) / TXC), (unsigned)((g.nyf + TYC - 1) / TYC));
}
dim3 node_tile_grid(const MeshGeom &g) {
    return dim3((unsigned)((g.nxf + PTX) / PTX), (unsigned)((g.nyf + PTY) / PTY));
}

template <typename KernelT>
cudaError_t set_smem(KernelT k, size_t bytes) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

// Column sources of a feature row, in the order of Sec. 5.2 inputs:
// residual (u, v, p) on the fine patch nodes, v~ (u, v) and the Peclet number
// on the coarse patch nodes, 12 geometry values, zero padding to ldx.
void feature_table(const MeshGeom &g, int *tab) {
    using L = ResLayout;
    const int S1 = g.S + 1, s1 = g.s + 1;
    int c = 0;
    for (int comp = 0; comp < 3; ++comp)
        for (int b = 0; b < S1; ++b)
            for (int a = 0; a < S1; ++a) tab[c++] = (FEAT_RES << 24) | (comp * L::RPL + b * L::RXP + a);
    for (int comp = 0; comp < 3; ++comp)
        for (int b = 0; b < s1; ++b)
            for (int a = 0; a < s1; ++a) {
                const int off = (b * g.r + L::YO) * L::HX + a * g.r + L::XO;
                tab[c++] = comp < 2 ? (FEAT_VEL << 24) | (comp * L::HY * L::HX + off) : (FEAT_PECLET << 24) | off;
            }
    for (int k = 0; k < 12; ++k) tab[c++] = (FEAT_GEO << 24) | k;
    while (c < g.ldx) tab[c++] = FEAT_ZERO << 24;
}

int feature_table_capacity() { return ResLayout::MAX_LDX; }

void tile_counts(const MeshGeom &g, int *ntx, int *nty) {
    *ntx = (g.nxf + TXC - 1) / TXC;
    *nty = (g.nyf + TYC - 1) / TYC;
}

void tile_flags(const MeshGeom &g, const uint8_t *solid, uint8_t *flags) {
    auto all_fluid = [&](int i0, int i1, int j0, int j1) {
        if (i0 < 0 || j0 < 0 || i1 >= g.nxf || j1 >= g.nyf) return false;
        for (int cj = j0 >> g.K; cj <= j1 >> g.K; ++cj)
            for (int ci = i0 >> g.K; ci <= i1 >> g.K; ++ci)
                if (solid[(size_t)cj * g.nxc + ci]) return false;
        return true;
    };
    for (int ty = 0; ty < g.nty; ++ty)
        for (int tx = 0; tx < g.ntx; ++tx) {
            const int I0 = tx * TXC, J0 = ty * TYC;
            flags[(size_t)ty * g.ntx + tx] =
                (uint8_t)((all_fluid(I0 - 2, I0 + TXC + 1, J0 - 2, J0 + TYC + 1) ? 1 : 0) |
                          (all_fluid(I0 - 1, I0 + TXC, J0 - 1, J0 + TYC) ? 2 : 0));
        }
}

// Peak inflow velocity at time t (u_max, ramped in over t <= 1/2 if requested).
double inflow_peak(const MeshGeom &g, double t) {
    return g.u_max * (g.ramp ? (t <= 0.5 ? 0.5 - 0.5 * cos(2.0 * 3.14159265358979323846 * t) : 1.0) : 1.0);
}

template <typename T>
cudaError_t run_prolongate(const MeshGeom &g, const double *xc, T *xf, double w, cudaStream_t st) {
    switch (g.r) {
        case 2: k_prolongate<T, 2><<<node_tile_grid(g), NTHREADS, 0, st>>>(g, xc, xf, w); break;
        case 4: k_prolongate<T, 4><<<node_tile_grid(g), NTHREADS, 0, st>>>(g, xc, xf, w); break;
        case 8: k_prolongate<T, 8><<<node_tile_grid(g), NTHREADS, 0, st>>>(g, xc, xf, w); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_prolongate(const MeshGeom &g, int prec, const double *xc, void *xf, double t,
                              cudaStream_t st) {
    const double w = inflow_peak(g, t);
    if (prec == DNNMG_F64) return run_prolongate(g, xc, (double *)xf, w, st);
    return run_prolongate(g, xc, (float *)xf, w, st);
}

template <typename T, typename TX, int R>
cudaError_t run_residual(const MeshGeom &g, const FemCoef<T> &fc, const void *xf, const double *xc, double w,
                         const void *bf, void *rf, void *X, cudaStream_t st) {
    auto k = k_residual_features<T, TX, R>;
    const size_t sm = ResLayout::bytes<T>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k<<<tile_grid(g), RES_THREADS, sm, st>>>(g, fc, (const T *)xf, xc, w, (const T *)bf, (T *)rf, (TX *)X);
    return cudaGetLastError();
}

template <typename T, typename TX>
cudaError_t run_residual_r(const MeshGeom &g, const FemCoef<T> &fc, const void *xf, const double *xc, double w,
                           const void *bf, void *rf, void *X, cudaStream_t st) {
    if (!xc) return run_residual<T, TX, 0>(g, fc, xf, xc, w, bf, rf, X, st);
    switch (g.r) {
        case 2: return run_residual<T, TX, 2>(g, fc, xf, xc, w, bf, rf, X, st);
        case 4: return run_residual<T, TX, 4>(g, fc, xf, xc, w, bf, rf, X, st);
        case 8: return run_residual<T, TX, 8>(g, fc, xf, xc, w, bf, rf, X, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_residual_features(const MeshGeom &g, int prec, const FemCoef<double> &f64,
                                     const FemCoef<float> &f32, const void *xf, const double *xc, double t,
                                     const void *bf, void *rf, void *X, cudaStream_t st) {
    const double w = inflow_peak(g, t);
    if (prec == DNNMG_F64) return run_residual_r<double, double>(g, f64, xf, xc, w, bf, rf, X, st);
    if (prec == DNNMG_F32) return run_residual_r<float, float>(g, f32, xf, xc, w, bf, rf, X, st);
    return run_residual_r<float, __nv_bfloat16>(g, f32, xf, xc, w, bf, rf, X, st);
}

int coarse_pitch(const MeshGeom &g) { return round_up(g.nxc + 1, 32); }

template <typename T>
cudaError_t run_coarse_pad(const MeshGeom &g, const double *xc, T *xcp, cudaStream_t st) {
    const int pc = coarse_pitch(g);
    const long long nq = 3LL * (g.nyc + 1) * (pc / 4);
    const long long need = (nq + NTHREADS - 1) / NTHREADS;
    const unsigned grid = (unsigned)(need < 152 * 8 ? need : 152 * 8);   // 8 CTAs per SM, grid-stride
    k_coarse_pad<T><<<grid, NTHREADS, 0, st>>>(g, xc, xcp, pc);
    return cudaGetLastError();
}

cudaError_t launch_coarse_pad(const MeshGeom &g, int prec, const double *xc, void *xcp, cudaStream_t st) {
    if (prec == DNNMG_F64) return run_coarse_pad(g, xc, (double *)xcp, st);
    return run_coarse_pad(g, xc, (float *)xcp, st);
}

template <typename T, typename TX, int R>
cudaError_t run_residual_step(const MeshGeom &g, const FemCoef<T> &fc, const T *xcp, double up, const T *bf, TX *X,
                              cudaStream_t st, bool skip_fast) {
    using L = ResLayout;
    using SL = StepLayout<T, R>;
    const CUtensorMapDataType dt = sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    // b_f [2][nyf+1][pitch]: boxes of BX columns x NYN rows x 2 components
    CUtensorMap tmB, tmC;
    const cuuint64_t bd[3] = {(cuuint64_t)g.nxf + 1, (cuuint64_t)g.nyf + 1, 2};
    const cuuint64_t bs[2] = {(cuuint64_t)g.pitch * sizeof(T), (cuuint64_t)g.plane * sizeof(T)};
    const cuuint32_t bb[3] = {(cuuint32_t)L::BX, (cuuint32_t)NYN, 2};
    // padded coarse vector [3][nyc+1][pc]: boxes of the coarse window
    const int pc = coarse_pitch(g);
    const cuuint64_t cd[3] = {(cuuint64_t)g.nxc + 1, (cuuint64_t)g.nyc + 1, 3};
    const cuuint64_t cs[2] = {(cuuint64_t)pc * sizeof(T), (cuuint64_t)pc * (g.nyc + 1) * sizeof(T)};
    const cuuint32_t cb[3] = {(cuuint32_t)SL::CWin::CW, (cuuint32_t)SL::CWin::CH, 3};
    if (!tma_encode_tiled(&tmB, dt, 3, const_cast<T *>(bf), bd, bs, bb) ||
        !tma_encode_tiled(&tmC, dt, 3, const_cast<T *>(xcp), cd, cs, cb))
        return cudaErrorInvalidValue;
    auto k = k_residual_step<T, TX, R>;
    const size_t sm = SL::BYTES;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (skip_fast) {
        if (g.n_slow_tiles == 0) return cudaSuccess;
        k<<<g.n_slow_tiles, RES_THREADS, sm, st>>>(g, fc, tmB, tmC, up, X, g.slow_tiles);
    } else {
        k<<<tile_grid(g), RES_THREADS, sm, st>>>(g, fc, tmB, tmC, up, X, nullptr);
    }
    return cudaGetLastError();
}

template <typename T, typename TX>
cudaError_t run_residual_step_r(const MeshGeom &g, const FemCoef<T> &fc, const void *xcp, double up, const void *bf,
                                void *X, cudaStream_t st, bool sf) {
    switch (g.r) {
        case 2: return run_residual_step<T, TX, 2>(g, fc, (const T *)xcp, up, (const T *)bf, (TX *)X, st, sf);
        case 4: return run_residual_step<T, TX, 4>(g, fc, (const T *)xcp, up, (const T *)bf, (TX *)X, st, sf);
        case 8: return run_residual_step<T, TX, 8>(g, fc, (const T *)xcp, up, (const T *)bf, (TX *)X, st, sf);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_residual_step(const MeshGeom &g, int prec, const FemCoef<double> &f64, const FemCoef<float> &f32,
                                 const void *xcp, double t, const void *bf, void *X, cudaStream_t st, bool skip_fast) {
    const double up = inflow_peak(g, t);
    if (prec == DNNMG_F64) return run_residual_step_r<double, double>(g, f64, xcp, up, bf, X, st, skip_fast);
    if (prec == DNNMG_F32) return run_residual_step_r<float, float>(g, f32, xcp, up, bf, X, st, skip_fast);
    return run_residual_step_r<float, __nv_bfloat16>(g, f32, xcp, up, bf, X, st, skip_fast);
}

template <typename T>
cudaError_t run_scatter(const MeshGeom &g, const T *d, const T *xf, const double *xc, const T *xcp, double w, T *vc,
                        cudaStream_t st) {
    const dim3 grid = node_tile_grid(g);
    const int pc = coarse_pitch(g);
    if (!xc && !xcp) {
        k_scatter_avg<T, 0><<<grid, NTHREADS, 0, st>>>(g, d, xf, xc, xcp, pc, w, vc);
        return cudaGetLastError();
    }
    switch (g.r) {
        case 2: k_scatter_avg<T, 2><<<grid, NTHREADS, 0, st>>>(g, d, xf, xc, xcp, pc, w, vc); break;
        case 4: k_scatter_avg<T, 4><<<grid, NTHREADS, 0, st>>>(g, d, xf, xc, xcp, pc, w, vc); break;
        case 8: k_scatter_avg<T, 8><<<grid, NTHREADS, 0, st>>>(g, d, xf, xc, xcp, pc, w, vc); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_scatter_avg(const MeshGeom &g, int prec, const void *d, const void *xf, const double *xc,
                               double t, void *vcorr, cudaStream_t st, const void *xcp) {
    const double w = inflow_peak(g, t);
    if (prec == DNNMG_F64)
        return run_scatter(g, (const double *)d, (const double *)xf, xc, (const double *)xcp, w, (double *)vcorr, st);
    return run_scatter(g, (const float *)d, (const float *)xf, xc, (const float *)xcp, w, (float *)vcorr, st);
}

template <typename T>
cudaError_t run_rhs(const MeshGeom &g, const FemCoef<T> &fc, const T *vcorr, T *bf, cudaStream_t st) {
    using L = RhsLayout;
    // v_corr [2][nyf+1][pitch]: boxes of the tile's node window
    CUtensorMap tm;
    const CUtensorMapDataType dt = sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nxf + 1, (cuuint64_t)g.nyf + 1, 2};
    const cuuint64_t str[2] = {(cuuint64_t)g.pitch * sizeof(T), (cuuint64_t)g.plane * sizeof(T)};
    const cuuint32_t box[3] = {(cuuint32_t)L::HX, (cuuint32_t)L::HY, 2};
    if (!tma_encode_tiled(&tm, dt, 3, const_cast<T *>(vcorr), dims, str, box)) return cudaErrorInvalidValue;
    const size_t sm = L::bytes<T>();
    cudaError_t e = set_smem(k_rhs<T>, sm);
    if (e != cudaSuccess) return e;
    k_rhs<T><<<tile_grid(g), NTHREADS, sm, st>>>(g, fc, tm, bf);
    return cudaGetLastError();
}

cudaError_t launch_rhs(const MeshGeom &g, int prec, const FemCoef<double> &f64,
                       const FemCoef<float> &f32, const void *vcorr, void *bf, cudaStream_t st) {
    if (prec == DNNMG_F64) return run_rhs(g, f64, (const double *)vcorr, (double *)bf, st);
    return run_rhs(g, f32, (const float *)vcorr, (float *)bf, st);
}

template <typename T, int R>
cudaError_t run_avg_rhs(const MeshGeom &g, const FemCoef<T> &fc, const T *d, const double *xc, double up, T *bf,
                        cudaStream_t st) {
    const int lS = g.K + g.s - 1;
    const size_t region = AvgRhsLayout<T>::region(R, lS, g.n_out);
    const size_t sm = AvgRhsLayout<T>::bytes(R, lS, g.n_out);
    cudaError_t e = set_smem(k_avg_rhs<T, R>, sm);
    if (e != cudaSuccess) return e;
    k_avg_rhs<T, R><<<tile_grid(g), NTHREADS, sm, st>>>(g, fc, d, xc, up, bf, (int)region);
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_avg_rhs_r(const MeshGeom &g, const FemCoef<T> &fc, const T *d, const double *xc, double up, T *bf,
                          cudaStream_t st) {
    switch (g.r) {
        case 2: return run_avg_rhs<T, 2>(g, fc, d, xc, up, bf, st);
        case 4: return run_avg_rhs<T, 4>(g, fc, d, xc, up, bf, st);
        case 8: return run_avg_rhs<T, 8>(g, fc, d, xc, up, bf, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_avg_rhs(const MeshGeom &g, int prec, const FemCoef<double> &f64, const FemCoef<float> &f32,
                           const void *d, const double *xc, double t, void *bf, cudaStream_t st) {
    const double up = inflow_peak(g, t);
    if (prec == DNNMG_F64) return run_avg_rhs_r(g, f64, (const double *)d, xc, up, (double *)bf, st);
    return run_avg_rhs_r(g, f32, (const float *)d, xc, up, (float *)bf, st);
}

cudaError_t launch_restrict(const MeshGeom &g, int prec, const void *bf, double *bc,
                            cudaStream_t st) {
    if (prec == DNNMG_F64) return run_restrict_r<double, RestrictAcc64>(g, (const double *)bf, bc, st);
    return run_restrict_r<float, RestrictAcc32>(g, (const float *)bf, bc, st);
}

cudaError_t launch_mesh_maps(const MeshGeom &g, unsigned char *flags, unsigned char *mult,
                             cudaStream_t st) {
    k_mesh_maps<<<node_grid(g), NTHREADS, 0, st>>>(g, flags, mult);
    return cudaGetLastError();
}

}  // namespace dnnmg

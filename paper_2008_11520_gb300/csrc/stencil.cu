// Stencil, gather and scatter passes of the DNN-MG correction step:
//   S1 prolongation, S2+S3 residual and patch features, S5 averaging,
//   S6 right-hand side, S7 restriction, plus the node index maps.
//
// Fine node fields are SoA planes [comp][Nf], x fastest.  S2 and S6 are
// tiled: one CTA owns a 32 x 16 block of fine cells, stages the node values
// it needs (plus a halo) in shared memory, computes every cell's element
// contributions once (cell-centric), and then sums them per node (a pull,
// so there are no atomics and results are bitwise repeatable).
#include <cstdio>

#include "common.cuh"

namespace dnnmg {
namespace {

constexpr int TXC = 32;            // fine cells per tile in x
constexpr int TYC = 16;            // fine cells per tile in y
constexpr int NXN = TXC + 1;       // tile nodes in x
constexpr int NYN = TYC + 1;
constexpr int NTHREADS = 256;

template <typename T> __device__ __forceinline__ T to_real(T v) { return v; }
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
__device__ __forceinline__ NodeClass classify(int c00, int c10, int c01, int c11, int I, int J,
                                              int nyf) {
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

// ------------------------------------------------------------------ S1
// A CTA owns 64 x 16 fine nodes; the coarse nodes they need are converted to
// the fine type once and staged in shared memory, so the interpolation runs
// in the fine arithmetic type (FP64 throughput on GB300 is 1/64 of FP32).
constexpr int PTX = 64, PTY = 16;
constexpr int PCX = PTX / 2 + 2, PCY = PTY / 2 + 2;   // coarse nodes of a tile for r >= 2

template <typename T>
__global__ void __launch_bounds__(NTHREADS)
k_prolongate(MeshGeom g, const double *__restrict__ xc, T *__restrict__ xf, double inflow_scale) {
    __shared__ T cs[3][PCY][PCX];
    const int I0 = blockIdx.x * PTX, J0 = blockIdx.y * PTY;
    const int ci0 = min(I0 >> g.K, g.nxc - 1), cj0 = min(J0 >> g.K, g.nyc - 1);
    const size_t nc1 = (size_t)g.nxc + 1, Nc = nc1 * (g.nyc + 1);
    for (int e = threadIdx.x; e < 3 * PCY * PCX; e += blockDim.x) {
        const int c = e / (PCY * PCX), rem = e - c * (PCY * PCX);
        const int jj = rem / PCX, ii = rem - jj * PCX;
        const int ci = ci0 + ii, cj = cj0 + jj;
        T v = T(0);
        if (ci <= g.nxc && cj <= g.nyc) v = (T)__ldg(xc + c * Nc + (size_t)cj * nc1 + ci);
        cs[c][jj][ii] = v;
    }
    __syncthreads();
    const size_t nxn = (size_t)g.nxf + 1, Nf = nxn * (g.nyf + 1);
    const T inv_r = T(1) / T(g.r);   // exact: r is a power of two
    for (int e = threadIdx.x; e < PTX * PTY; e += blockDim.x) {
        const int I = I0 + (e % PTX), J = J0 + e / PTX;
        if (I > g.nxf || J > g.nyf) continue;
        const int ci = min(I >> g.K, g.nxc - 1), cj = min(J >> g.K, g.nyc - 1);
        const T a = T(I - (ci << g.K)) * inv_r, b = T(J - (cj << g.K)) * inv_r;
        const int li = ci - ci0, lj = cj - cj0;
        T val[3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            val[c] = (T(1) - a) * (T(1) - b) * cs[c][lj][li] + a * (T(1) - b) * cs[c][lj][li + 1] +
                     (T(1) - a) * b * cs[c][lj + 1][li] + a * b * cs[c][lj + 1][li + 1];
        const NodeClass nc = classify_global(g, I, J);
        if (nc.dirichlet) {
            const double y = J * g.hyf;
            val[0] = nc.inflow ? (T)(g.u_max * 4.0 * y * (g.ly - y) / (g.ly * g.ly) * inflow_scale) : T(0);
            val[1] = T(0);
        }
        const size_t node = (size_t)J * nxn + I;
        xf[node] = val[0];
        xf[Nf + node] = val[1];
        xf[2 * Nf + node] = val[2];
    }
}

// ------------------------------------------------------------------ S2 + S3
// 1/2 (v.grad v_c, phi_a) of one cell for its corners a = SW, SE, NW, NE, by
// 2x2 Gauss in tensor-product form: values and derivatives at the 4 points
// from edge interpolants, then the test-function sums one direction at a time.
template <typename T>
__device__ __forceinline__ void convection(const FemCoef<T> &fc, const T (&u)[4], const T (&v)[4], T (&cu)[4],
                                           T (&cv)[4]) {
    const T g0 = fc.cg0, g1 = fc.cg1;
    // along x on the bottom (0, 1) and top (2, 3) edges
    const T dub = u[1] - u[0], dut = u[3] - u[2], dvb = v[1] - v[0], dvt = v[3] - v[2];
    const T ub[2] = {u[0] + g0 * dub, u[0] + g1 * dub}, ut[2] = {u[2] + g0 * dut, u[2] + g1 * dut};
    const T vb[2] = {v[0] + g0 * dvb, v[0] + g1 * dvb}, vt[2] = {v[2] + g0 * dvt, v[2] + g1 * dvt};
    // x-derivatives depend on eta only, y-derivatives on xi only
    const T ux[2] = {dub + g0 * (dut - dub), dub + g1 * (dut - dub)};
    const T vx[2] = {dvb + g0 * (dvt - dvb), dvb + g1 * (dvt - dvb)};
    const T uy[2] = {ut[0] - ub[0], ut[1] - ub[1]};
    const T vy[2] = {vt[0] - vb[0], vt[1] - vb[1]};
    T c_u[2][2], c_v[2][2];   // [eta index j][xi index i]
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const T gj = j ? g1 : g0;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const T U = (ub[i] + gj * uy[i]) * fc.inv_hx;
            const T V = (vb[i] + gj * vy[i]) * fc.inv_hy;
            c_u[j][i] = U * ux[j] + V * uy[i];
            c_v[j][i] = U * vx[j] + V * vy[i];
        }
    }
    // test with l_0(g) = 1 - g, l_1(g) = g (1 - g0 = g1), weights (qw / 2)
    T su[2][2], sv[2][2];   // [j][ax]
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        su[j][0] = g1 * c_u[j][0] + g0 * c_u[j][1];
        su[j][1] = g0 * c_u[j][0] + g1 * c_u[j][1];
        sv[j][0] = g1 * c_v[j][0] + g0 * c_v[j][1];
        sv[j][1] = g0 * c_v[j][0] + g1 * c_v[j][1];
    }
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
        cu[ax] = fc.cwg1 * su[0][ax] + fc.cwg0 * su[1][ax];
        cu[2 + ax] = fc.cwg0 * su[0][ax] + fc.cwg1 * su[1][ax];
        cv[ax] = fc.cwg1 * sv[0][ax] + fc.cwg0 * sv[1][ax];
        cv[2 + ax] = fc.cwg0 * sv[0][ax] + fc.cwg1 * sv[1][ax];
    }
}

// Asynchronous 4- or 8-byte copy global -> shared; src_bytes = 0 writes zero.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src, int src_bytes) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(src), "n"(BYTES), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Stage rows of a node-field window into shared memory: rows `nrows` of width
// `w` starting at global node (I0, J0), component planes of Nf nodes; zero
// outside the mesh.  One warp per row; the copies are asynchronous so every
// thread keeps many loads in flight (complete with cp_async_wait_all()).
template <typename T>
__device__ __forceinline__ void stage_rows(const MeshGeom &g, const T *__restrict__ src, size_t Nf, int ncomp,
                                           int I0, int J0, int w, int nrows, T *dst) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const size_t nxn = (size_t)g.nxf + 1;
    for (int rr = warp; rr < ncomp * nrows; rr += nw) {
        const int c = rr / nrows, jj = rr - c * nrows;
        const int J = J0 + jj;
        T *d = dst + (size_t)rr * w;
        const bool rowok = J >= 0 && J <= g.nyf;
        const T *row = src + c * Nf + (size_t)(rowok ? J : 0) * nxn;
        for (int ii = lane; ii < w; ii += 32) {
            const int I = I0 + ii;
            const bool ok = rowok && I >= 0 && I <= g.nxf;
            cp_async<sizeof(T)>(d + ii, ok ? row + I : src, ok ? (int)sizeof(T) : 0);
        }
    }
}

// Shared-memory layout of the residual/feature tile (element counts).
struct ResLayout {
    static constexpr int HX = NXN + 4, HY = NYN + 4;           // nodes with 2-node halo
    static constexpr int CX = TXC + 2, CY = TYC + 2;           // cells with 1-cell halo
    static constexpr int NCELL = CX * CY;
    static constexpr int LX = TXC / 2 + 2, LY = TYC / 2 + 2;   // LPS patches touching the tile
    static constexpr int NLPS = LX * LY;
    static constexpr int FX = TXC + 4, FY = TYC + 4;           // cell codes with 2-cell halo
    static constexpr int XS = 3 * HY * HX;
    static constexpr int BS = 2 * NYN * NXN;
    static constexpr int CC = 12 * NCELL;
    static constexpr int LC = 9 * NLPS;
    static constexpr int RS = 3 * NYN * NXN;
    template <typename T> static constexpr size_t bytes() {
        return sizeof(T) * (XS + BS + CC + LC + RS) + FX * FY;
    }
};

enum { FEAT_RES = 0, FEAT_VEL = 1, FEAT_PECLET = 2, FEAT_GEO = 3, FEAT_ZERO = 4 };

template <typename T, typename TX>
__global__ void __launch_bounds__(NTHREADS)
k_residual_features(MeshGeom g, FemCoef<T> fc, const T *__restrict__ xf, const T *__restrict__ bf,
                    T *__restrict__ rf, TX *__restrict__ X) {
    using L = ResLayout;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *xs = reinterpret_cast<T *>(smem_raw);   // [3][HY][HX]   u, v, p
    T *bs = xs + L::XS;                        // [2][NYN][NXN] b_u, b_v
    T *cc = bs + L::BS;                        // [12][NCELL]   cell contributions
    T *lc = cc + L::CC;                        // [9][NLPS]     LPS contributions
    T *rs = lc + L::LC;                        // [3][NYN][NXN] residual
    unsigned char *cf = reinterpret_cast<unsigned char *>(rs + L::RS);  // [FY][FX]

    const int I0 = blockIdx.x * TXC, J0 = blockIdx.y * TYC;
    const size_t nxn = (size_t)g.nxf + 1, Nf = nxn * (g.nyf + 1);

    stage_rows(g, xf, Nf, 3, I0 - 2, J0 - 2, L::HX, L::HY, xs);
    stage_rows(g, bf, Nf, 2, I0, J0, NXN, NYN, bs);
    bool all_fluid = true;
#pragma unroll 3
    for (int idx = threadIdx.x; idx < L::FX * L::FY; idx += blockDim.x) {
        const int jj = idx / L::FX, ii = idx - jj * L::FX;
        const int code = cell_code(g, I0 - 2 + ii, J0 - 2 + jj);
        cf[idx] = (unsigned char)code;
        all_fluid &= code == 1;
    }
    cp_async_wait_all();
    // Fast tiles: every cell within two of the tile is fluid and exists, so
    // no tile node is a boundary node and node stencils apply everywhere.
    const bool fast = __syncthreads_and(all_fluid);

    // Phase A: cell contributions (fast tiles: convection only)
    for (int cid = threadIdx.x; cid < L::NCELL; cid += blockDim.x) {
        const int ci = cid % L::CX - 1, cj = cid / L::CX - 1;
        T out[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) out[k] = T(0);
        if (cf[(cj + 2) * L::FX + ci + 2] == 1) {
            const int base = (cj + 2) * L::HX + ci + 2;
            const int off[4] = {0, 1, L::HX, L::HX + 1};
            T u[4], v[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                u[b] = xs[base + off[b]];
                v[b] = xs[L::HY * L::HX + base + off[b]];
            }
            T cu[4], cv[4];
            convection(fc, u, v, cu, cv);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                out[a] = cu[a];
                out[4 + a] = cv[a];
            }
            if (!fast) {
                T p[4];
#pragma unroll
                for (int b = 0; b < 4; ++b) p[b] = xs[2 * L::HY * L::HX + base + off[b]];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    T au = T(0), av = T(0), ap = T(0);
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        au += fc.Av[a][b] * u[b] - fc.Gx[a][b] * p[b];
                        av += fc.Av[a][b] * v[b] - fc.Gy[a][b] * p[b];
                        ap += fc.Dx[a][b] * u[b] + fc.Dy[a][b] * v[b];
                    }
                    out[a] += au;
                    out[4 + a] += av;
                    out[8 + a] = ap;
                }
            }
        }
        const int nk = fast ? 8 : 12;
#pragma unroll
        for (int k = 0; k < 12; ++k)
            if (k < nk) cc[k * L::NCELL + cid] = out[k];
    }
    // Phase A': LPS contributions of every 2x2-cell patch touching the tile.
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
                    p9[3 * b + a] = xs[2 * L::HY * L::HX + (2 * n + b + 2) * L::HX + 2 * m + a + 2];
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
        T ru = T(0), rv = T(0), rp = T(0);
        if (I <= g.nxf && J <= g.nyf) {
            const int cells[4] = {jj * L::CX + ii, jj * L::CX + ii + 1, (jj + 1) * L::CX + ii,
                                  (jj + 1) * L::CX + ii + 1};   // cells SW, SE, NW, NE of the node
            const int corner[4] = {3, 2, 1, 0};
            T Au = T(0), Av = T(0), Ap = T(0);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                Au += cc[corner[t] * L::NCELL + cells[t]];
                Av += cc[(4 + corner[t]) * L::NCELL + cells[t]];
            }
            if (fast) {
                const T *pu = xs + (jj + 1) * L::HX + ii + 1;      // node (ii-1, jj-1)
                const T *pv = pu + L::HY * L::HX;
                const T *pp = pv + L::HY * L::HX;
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        const T u = pu[dy * L::HX + dx], v = pv[dy * L::HX + dx], p = pp[dy * L::HX + dx];
                        Au += fc.nA[dy][dx] * u - fc.nGx[dy][dx] * p;
                        Av += fc.nA[dy][dx] * v - fc.nGy[dy][dx] * p;
                        Ap += fc.nDx[dy][dx] * u + fc.nDy[dy][dx] * v;
                    }
            } else {
#pragma unroll
                for (int t = 0; t < 4; ++t) Ap += cc[(8 + corner[t]) * L::NCELL + cells[t]];
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
            bool dirichlet = false, p_active = true;
            if (!fast) {
                const NodeClass nc = classify(cf[(jj + 1) * L::FX + ii + 1], cf[(jj + 1) * L::FX + ii + 2],
                                              cf[(jj + 2) * L::FX + ii + 1], cf[(jj + 2) * L::FX + ii + 2],
                                              I, J, g.nyf);
                dirichlet = nc.dirichlet;
                p_active = nc.p_active;
            }
            if (!dirichlet) {
                ru = bs[jj * NXN + ii] - Au;
                rv = bs[NYN * NXN + jj * NXN + ii] - Av;
            }
            if (p_active) rp = -Ap;
            // a node on the tile's right/top edge belongs to the next tile
            // (which may take the other path): write owned nodes only
            if (rf && (ii < TXC || I == g.nxf) && (jj < TYC || J == g.nyf)) {
                const size_t node = (size_t)J * nxn + I;
                rf[node] = ru;
                rf[Nf + node] = rv;
                rf[2 * Nf + node] = rp;
            }
        }
        rs[nid] = ru;
        rs[NYN * NXN + nid] = rv;
        rs[2 * NYN * NXN + nid] = rp;
    }
    __syncthreads();

    // Phase C: one feature row per fluid patch of the tile (Sec. 5.2 inputs);
    // feat_tab[c] says where column c comes from relative to the patch origin.
    // One warp per patch row; lanes write consecutive columns.
    const int S = g.S;
    const int tpx = TXC / S, tpy = TYC / S;
    const int pi0 = I0 / S, pj0 = J0 / S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int tp = warp; tp < tpx * tpy; tp += nw) {
        const int lpy = tp / tpx, lpx = tp - lpy * tpx;
        const int pi = pi0 + lpx, pj = pj0 + lpy;
        if (pi >= g.npx || pj >= g.npy) continue;
        const int id = g.patch_id[pj * g.npx + pi];
        if (id < 0) continue;
        const T *rbase = rs + lpy * S * NXN + lpx * S;
        const T *xbase = xs + lpy * S * L::HX + lpx * S;
        TX *row = X + (size_t)id * g.ldx;
        for (int c = lane; c < g.ldx; c += 32) {
            const int e = __ldg(g.feat_tab + c);
            const int kind = e >> 24, off = e & 0xFFFFFF;
            T val;
            if (kind == FEAT_RES) {
                val = rbase[off];
            } else if (kind == FEAT_VEL) {
                val = xbase[off];
            } else if (kind == FEAT_PECLET) {
                const T u = xbase[off], v = xbase[off + L::HY * L::HX];
                val = fc.q_over_nu * sqrt(u * u + v * v);
            } else if (kind == FEAT_GEO) {
                val = fc.geo[off];
            } else {
                val = T(0);
            }
            row[c] = store_as<TX, T>(val);
        }
    }
}

// ------------------------------------------------------------------ S5
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
k_scatter_avg(MeshGeom g, const T *__restrict__ d, const T *__restrict__ xf, T *__restrict__ vc) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y;
    if (I > g.nxf) return;
    const size_t nxn = (size_t)g.nxf + 1, Nf = nxn * (g.nyf + 1);
    const size_t node = (size_t)J * nxn + I;
    T u = xf[node], v = xf[Nf + node];
    const NodeClass nc = classify_global(g, I, J);
    if (!nc.dirichlet) {
        const int S = g.S;
        int pis[2], pjs[2], npi = 0, npj = 0;
        if (I % S == 0) {
            if (I / S - 1 >= 0) pis[npi++] = I / S - 1;
            if (I / S < g.npx) pis[npi++] = I / S;
        } else {
            pis[npi++] = I / S;
        }
        if (J % S == 0) {
            if (J / S - 1 >= 0) pjs[npj++] = J / S - 1;
            if (J / S < g.npy) pjs[npj++] = J / S;
        } else {
            pjs[npj++] = J / S;
        }
        T su = T(0), sv = T(0);
        int cnt = 0;
        for (int tj = 0; tj < npj; ++tj)
            for (int ti = 0; ti < npi; ++ti) {
                const int id = g.patch_id[pjs[tj] * g.npx + pis[ti]];
                if (id < 0) continue;
                const int k = (J - pjs[tj] * S) * (S + 1) + (I - pis[ti] * S);
                su += d[(size_t)id * g.n_out + k];
                sv += d[(size_t)id * g.n_out + g.nf + k];
                ++cnt;
            }
        if (cnt) {
            u += su / T(cnt);
            v += sv / T(cnt);
        }
    }
    vc[node] = u;
    vc[Nf + node] = v;
}

// ------------------------------------------------------------------ S6
struct RhsLayout {
    static constexpr int HX = NXN + 2, HY = NYN + 2;   // nodes with 1-node halo
    static constexpr int CX = TXC + 2, CY = TYC + 2;   // cells -1..TXC
    static constexpr int NCELL = CX * CY;
    static constexpr int VS = 2 * HY * HX;
    static constexpr int CC = 8 * NCELL;
    template <typename T> static constexpr size_t bytes() {
        return sizeof(T) * (VS + CC) + NCELL;
    }
};

template <typename T>
__global__ void __launch_bounds__(NTHREADS)
k_rhs(MeshGeom g, FemCoef<T> fc, const T *__restrict__ vcorr, T *__restrict__ bf) {
    using L = RhsLayout;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *vs = reinterpret_cast<T *>(smem_raw);   // [2][HY][HX]
    T *cc = vs + L::VS;                        // [8][NCELL]
    unsigned char *cf = reinterpret_cast<unsigned char *>(cc + L::CC);  // [CY][CX]
    const int I0 = blockIdx.x * TXC, J0 = blockIdx.y * TYC;
    const size_t nxn = (size_t)g.nxf + 1, Nf = nxn * (g.nyf + 1);

    stage_rows(g, vcorr, Nf, 2, I0 - 1, J0 - 1, L::HX, L::HY, vs);
    bool all_fluid = true;
#pragma unroll 3
    for (int idx = threadIdx.x; idx < L::NCELL; idx += blockDim.x) {
        const int jj = idx / L::CX, ii = idx - jj * L::CX;
        const int code = cell_code(g, I0 - 1 + ii, J0 - 1 + jj);
        cf[idx] = (unsigned char)code;
        all_fluid &= code == 1;
    }
    cp_async_wait_all();
    const bool fast = __syncthreads_and(all_fluid);

    for (int cid = threadIdx.x; cid < L::NCELL; cid += blockDim.x) {
        T out[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) out[k] = T(0);
        if (cf[cid] == 1) {
            const int ci = cid % L::CX, cj = cid / L::CX;   // halo-relative node of SW corner
            const int base = cj * L::HX + ci;
            const int off[4] = {0, 1, L::HX, L::HX + 1};
            T u[4], v[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                u[b] = vs[base + off[b]];
                v[b] = vs[L::HY * L::HX + base + off[b]];
            }
            T cu[4], cv[4];
            convection(fc, u, v, cu, cv);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                out[a] = -cu[a];
                out[4 + a] = -cv[a];
            }
            if (!fast) {
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    T bu = T(0), bv = T(0);
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        bu += fc.Bv[a][b] * u[b];
                        bv += fc.Bv[a][b] * v[b];
                    }
                    out[a] += bu;
                    out[4 + a] += bv;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) cc[k * L::NCELL + cid] = out[k];
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
            bu += cc[corner[t] * L::NCELL + cells[t]];
            bv += cc[(4 + corner[t]) * L::NCELL + cells[t]];
        }
        if (fast) {
            const T *pu = vs + jj * L::HX + ii;   // node (ii-1, jj-1)
            const T *pv = pu + L::HY * L::HX;
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    bu += fc.nB[dy][dx] * pu[dy * L::HX + dx];
                    bv += fc.nB[dy][dx] * pv[dy * L::HX + dx];
                }
        } else {
            const NodeClass nc = classify(cf[cells[0]], cf[cells[1]], cf[cells[2]], cf[cells[3]], I, J, g.nyf);
            if (nc.dirichlet) bu = bv = T(0);
        }
        const size_t node = (size_t)J * nxn + I;
        bf[node] = bu;
        bf[Nf + node] = bv;
    }
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

template <typename T, typename Acc>
__global__ void __launch_bounds__(NTHREADS)
k_restrict(MeshGeom g, const T *__restrict__ bf, double *__restrict__ bc) {
    using Row = typename Acc::Row;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int r = g.r;
    const int TCX = 128 / r, TCY = 32 / r;           // coarse nodes per tile
    const int FW = TCX * r + r - 1, FH = TCY * r + r - 1;   // fine nodes staged
    T *fs = reinterpret_cast<T *>(smem_raw);         // [2][FH][FW]
    Row *rs = reinterpret_cast<Row *>(fs + 2 * FH * FW);   // [2][FH][TCX] x-restricted rows
    const int ci0 = blockIdx.x * TCX, cj0 = blockIdx.y * TCY;
    const int I0 = ci0 * r - (r - 1), J0 = cj0 * r - (r - 1);
    const size_t nxn = (size_t)g.nxf + 1, Nf = nxn * (g.nyf + 1);
    stage_rows(g, bf, Nf, 2, I0, J0, FW, FH, fs);
    cp_async_wait_all();
    __syncthreads();
    const T inv_r = T(1) / T(r);
    for (int e = threadIdx.x; e < 2 * FH * TCX; e += blockDim.x) {
        const int c = e / (FH * TCX), rem = e - c * (FH * TCX);
        const int jj = rem / TCX, ci = rem - jj * TCX;
        const T *row = fs + c * FH * FW + jj * FW + ci * r;   // fine nodes ci*r-(r-1) .. ci*r+(r-1)
        Row acc = Acc::zero();
        for (int d = 0; d < 2 * r - 1; ++d) Acc::add(acc, T(r - abs(d - (r - 1))) * inv_r, row[d]);
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
            for (int d = 0; d < 2 * r - 1; ++d)
                Acc::add(acc, T(r - abs(d - (r - 1))) * inv_r, rs[c * FH * TCX + (lj * r + d) * TCX + li]);
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

template <typename T, typename Acc>
size_t restrict_smem(int r) {
    const int FW = 128 + r - 1, FH = 32 + r - 1;
    return 2 * FH * FW * sizeof(T) + 2 * FH * (128 / r) * sizeof(typename Acc::Row);
}

// ------------------------------------------------------------------ maps
__global__ void k_mesh_maps(MeshGeom g, unsigned char *flags, unsigned char *mult) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y;
    if (I > g.nxf) return;
    const size_t node = (size_t)J * ((size_t)g.nxf + 1) + I;
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
            for (int a = 0; a < S1; ++a) tab[c++] = (FEAT_RES << 24) | (comp * NYN * NXN + b * NXN + a);
    for (int comp = 0; comp < 3; ++comp)
        for (int b = 0; b < s1; ++b)
            for (int a = 0; a < s1; ++a) {
                const int off = (b * g.r + 2) * L::HX + a * g.r + 2;
                tab[c++] = comp < 2 ? (FEAT_VEL << 24) | (comp * L::HY * L::HX + off) : (FEAT_PECLET << 24) | off;
            }
    for (int k = 0; k < 12; ++k) tab[c++] = (FEAT_GEO << 24) | k;
    while (c < g.ldx) tab[c++] = FEAT_ZERO << 24;
}

cudaError_t launch_prolongate(const MeshGeom &g, int prec, const double *xc, void *xf, double t,
                              cudaStream_t st) {
    double w = 1.0;
    if (g.ramp) w = t <= 0.5 ? 0.5 - 0.5 * cos(2.0 * 3.14159265358979323846 * t) : 1.0;
    const dim3 grid((unsigned)((g.nxf + PTX) / PTX), (unsigned)((g.nyf + PTY) / PTY));
    if (prec == DNNMG_F64)
        k_prolongate<double><<<grid, NTHREADS, 0, st>>>(g, xc, (double *)xf, w);
    else
        k_prolongate<float><<<grid, NTHREADS, 0, st>>>(g, xc, (float *)xf, w);
    return cudaGetLastError();
}

cudaError_t launch_residual_features(const MeshGeom &g, int prec, const FemCoef<double> &f64,
                                     const FemCoef<float> &f32, const void *xf, const void *bf,
                                     void *rf, void *X, cudaStream_t st) {
    cudaError_t e;
    if (prec == DNNMG_F64) {
        auto k = k_residual_features<double, double>;
        const size_t sm = ResLayout::bytes<double>();
        if ((e = set_smem(k, sm)) != cudaSuccess) return e;
        k<<<tile_grid(g), NTHREADS, sm, st>>>(g, f64, (const double *)xf, (const double *)bf,
                                              (double *)rf, (double *)X);
    } else if (prec == DNNMG_F32) {
        auto k = k_residual_features<float, float>;
        const size_t sm = ResLayout::bytes<float>();
        if ((e = set_smem(k, sm)) != cudaSuccess) return e;
        k<<<tile_grid(g), NTHREADS, sm, st>>>(g, f32, (const float *)xf, (const float *)bf,
                                              (float *)rf, (float *)X);
    } else {
        auto k = k_residual_features<float, __nv_bfloat16>;
        const size_t sm = ResLayout::bytes<float>();
        if ((e = set_smem(k, sm)) != cudaSuccess) return e;
        k<<<tile_grid(g), NTHREADS, sm, st>>>(g, f32, (const float *)xf, (const float *)bf,
                                              (float *)rf, (__nv_bfloat16 *)X);
    }
    return cudaGetLastError();
}

cudaError_t launch_scatter_avg(const MeshGeom &g, int prec, const void *d, const void *xf,
                               void *vcorr, cudaStream_t st) {
    if (prec == DNNMG_F64)
        k_scatter_avg<double><<<node_grid(g), NTHREADS, 0, st>>>(g, (const double *)d,
                                                                 (const double *)xf, (double *)vcorr);
    else
        k_scatter_avg<float><<<node_grid(g), NTHREADS, 0, st>>>(g, (const float *)d,
                                                                (const float *)xf, (float *)vcorr);
    return cudaGetLastError();
}

cudaError_t launch_rhs(const MeshGeom &g, int prec, const FemCoef<double> &f64,
                       const FemCoef<float> &f32, const void *vcorr, void *bf, cudaStream_t st) {
    cudaError_t e;
    if (prec == DNNMG_F64) {
        const size_t sm = RhsLayout::bytes<double>();
        if ((e = set_smem(k_rhs<double>, sm)) != cudaSuccess) return e;
        k_rhs<double><<<tile_grid(g), NTHREADS, sm, st>>>(g, f64, (const double *)vcorr, (double *)bf);
    } else {
        const size_t sm = RhsLayout::bytes<float>();
        if ((e = set_smem(k_rhs<float>, sm)) != cudaSuccess) return e;
        k_rhs<float><<<tile_grid(g), NTHREADS, sm, st>>>(g, f32, (const float *)vcorr, (float *)bf);
    }
    return cudaGetLastError();
}

cudaError_t launch_restrict(const MeshGeom &g, int prec, const void *bf, double *bc,
                            cudaStream_t st) {
    const int TCX = 128 / g.r, TCY = 32 / g.r;
    const dim3 grid((unsigned)((g.nxc + TCX) / TCX), (unsigned)((g.nyc + TCY) / TCY));
    cudaError_t e;
    if (prec == DNNMG_F64) {
        const size_t sm = restrict_smem<double, RestrictAcc64>(g.r);
        if ((e = set_smem(k_restrict<double, RestrictAcc64>, sm)) != cudaSuccess) return e;
        k_restrict<double, RestrictAcc64><<<grid, NTHREADS, sm, st>>>(g, (const double *)bf, bc);
    } else {
        const size_t sm = restrict_smem<float, RestrictAcc32>(g.r);
        if ((e = set_smem(k_restrict<float, RestrictAcc32>, sm)) != cudaSuccess) return e;
        k_restrict<float, RestrictAcc32><<<grid, NTHREADS, sm, st>>>(g, (const float *)bf, bc);
    }
    return cudaGetLastError();
}

cudaError_t launch_mesh_maps(const MeshGeom &g, unsigned char *flags, unsigned char *mult,
                             cudaStream_t st) {
    k_mesh_maps<<<node_grid(g), NTHREADS, 0, st>>>(g, flags, mult);
    return cudaGetLastError();
}

}  // namespace dnnmg

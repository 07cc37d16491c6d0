// Plain geometric multigrid for the fine-level system on the GPU: the
// solver DNN-MG is compared with (Sec. 3.3 Newton iteration, Sec. 3.4
// multigrid with the Vanka smoother, Sec. 6.4 timing comparison).
//
// One time step of the plain method solves the Crank-Nicolson system of
// Eq. nonlinearshort on level L+K by Newton's method; each Newton system is
// solved by GMRES preconditioned with multigrid V-cycles over a hierarchy of
// levels, smoothed by the Vanka method: for every cell, the 12 x 12 block of
// the Newton matrix that couples the velocity and pressure unknowns of its
// four nodes is solved against the current defect.  This file holds the
// level hierarchy and the kernels of one V-cycle and of the Newton and
// GMRES iterations; the iterations themselves are driven from the host
// (mg.py).  Node fields are [3][N] (u, v, p), N = (nx + 1)(ny + 1) nodes,
// x fastest, unpadded: the layout of the host solver.
//
// The discretisation is the one of the correction step (Q1/Q1, Crank-
// Nicolson, local projection stabilisation on 2 x 2-cell patches, 2 x 2
// Gauss points), with the element constants of FemCoef.  Level 0 is the
// finest, with any cell mask (a partly solid projection patch contributes
// the integrals of its fluid cells, as on the coarse level of the host
// solver); level l+1 has half the cells of level l in each direction, and a
// patch of level l+1 is solid iff all 16 cells of level l under it are.
// Every level uses the finest level's projection coefficient alpha (alpha0
// scaled by 4^-l): the fine projection term vanishes on a prolongated
// pressure, and alpha = alpha0 h^2 / nu evaluated with a coarse h would
// outweigh the pressure coupling of the time step there and make the coarse
// pressure corrections far too small.  (Coarse levels only precondition:
// their geometry and stabilisation approximate the fine ones.)
//
// The smoother is multiplicative (block Gauss-Seidel over cells) in 16
// colours.  A cell's local defect reads the correction up to two nodes beyond
// its own (the projection patches reach two nodes from an even node), and it
// writes its own four nodes; cells with the same (ci mod 4, cj mod 4) are
// four cells apart, so none reads a node another one writes: each colour is
// one parallel pass, and a sweep is deterministic.
#include <cmath>
#include <new>
#include <vector>

#include "common.cuh"

namespace dnnmg {

void level_coefficients(double lx, double ly, int nx, int ny, double nu, double k, double alpha0,
                        FemCoef<double> *f64, FemCoef<float> *f32);

namespace {

constexpr int MG_THREADS = 256;

// A level as the kernels see it.
template <typename T>
struct MgLev {
    int nx, ny, N;
    const uint8_t *solid;   // [ny][nx] cell mask, 1 = solid
    const uint8_t *flags;   // [N]: bit 0 velocity Dirichlet, bit 1 inflow value, bit 2 pressure active
    const uint8_t *mult;    // [N]: fluid cells holding the node
    const T *lps;           // [16][9][9]: projection patch matrix by the patch's fluid cells (bit 2 cb + ca)
    double hy, ly;
    FemCoef<T> fc;
};

template <typename T> __device__ __forceinline__ bool fluid(const MgLev<T> &L, int ci, int cj) {
    return ci >= 0 && cj >= 0 && ci < L.nx && cj < L.ny && !L.solid[(size_t)cj * L.nx + ci];
}
// The fluid cells of 2 x 2-cell projection patch (m, n): bit 2 cb + ca for its
// cell (2m + ca, 2n + cb); 0 outside the mesh.  A patch contributes the
// projection integrals of its fluid cells (every cell of an all-fluid patch).
template <typename T> __device__ __forceinline__ int patch_mask(const MgLev<T> &L, int m, int n) {
    if (m < 0 || n < 0 || 2 * m + 1 >= L.nx || 2 * n + 1 >= L.ny) return 0;
    return (fluid(L, 2 * m, 2 * n) ? 1 : 0) | (fluid(L, 2 * m + 1, 2 * n) ? 2 : 0) |
           (fluid(L, 2 * m, 2 * n + 1) ? 4 : 0) | (fluid(L, 2 * m + 1, 2 * n + 1) ? 8 : 0);
}

// Values and derivatives of (u, v) at the 4 Gauss points of cell (ci, cj).
template <typename T>
struct GaussVel {
    T U[4], V[4], Ux[4], Uy[4], Vx[4], Vy[4];
    __device__ __forceinline__ void eval(const MgLev<T> &L, const T *u, const T *v, int ci, int cj) {
        const int nxn = L.nx + 1;
        T ub[4], vb[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int n = (cj + (b >> 1)) * nxn + ci + (b & 1);
            ub[b] = u[n];
            vb[b] = v[n];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            U[q] = V[q] = Ux[q] = Uy[q] = Vx[q] = Vy[q] = T(0);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                U[q] += L.fc.qphi[q][b] * ub[b];
                V[q] += L.fc.qphi[q][b] * vb[b];
                Ux[q] += L.fc.qdx[q][b] * ub[b];
                Uy[q] += L.fc.qdy[q][b] * ub[b];
                Vx[q] += L.fc.qdx[q][b] * vb[b];
                Vy[q] += L.fc.qdy[q][b] * vb[b];
            }
        }
    }
};

template <typename T> __device__ __forceinline__ T inflow(const MgLev<T> &L, int J, double up) {
    const double y = J * L.hy;
    return (T)(up * 4.0 * y * (L.ly - y) / (L.ly * L.ly));
}

// Rows of one node for the operator pieces the kernels share: with the node
// at corner a of fluid cell (ci, cj), add the cell's linear velocity and
// pressure-gradient terms (mode 0: A(x); mode 1: the right-hand side's
// 1/k M - nu/2 K part, no pressure) and the divergence.
template <typename T>
__device__ __forceinline__ void linear_rows(const MgLev<T> &L, const T *u, const T *v, const T *p, int ci, int cj,
                                            int a, bool rhs, T &Au, T &Av, T &Ap) {
    const int nxn = L.nx + 1;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int n = (cj + (b >> 1)) * nxn + ci + (b & 1);
        const T ub = u[n], vb = v[n];
        if (rhs) {
            Au += L.fc.Bv[a][b] * ub;
            Av += L.fc.Bv[a][b] * vb;
        } else {
            const T pb = p[n];
            Au += L.fc.Av[a][b] * ub - L.fc.Gx[a][b] * pb;
            Av += L.fc.Av[a][b] * vb - L.fc.Gy[a][b] * pb;
            Ap += L.fc.Dx[a][b] * ub + L.fc.Dy[a][b] * vb;
        }
    }
}

// Local projection term of pressure row (I, J): the patches that hold the node.
template <typename T> __device__ __forceinline__ T lps_row(const MgLev<T> &L, const T *p, int I, int J) {
    const int nxn = L.nx + 1;
    T acc = T(0);
#pragma unroll
    for (int pn = 0; pn < 2; ++pn) {
        const int n = (J - pn) >> 1;                      // patches n with 2n <= J <= 2n + 2
        if (pn == 1 && (J & 1)) continue;                  // an odd J lies in one patch only
        if (2 * n > J || J > 2 * n + 2) continue;
#pragma unroll
        for (int pm = 0; pm < 2; ++pm) {
            const int m = (I - pm) >> 1;
            if (pm == 1 && (I & 1)) continue;
            if (2 * m > I || I > 2 * m + 2) continue;
            const int pm_ = patch_mask(L, m, n);
            if (!pm_) continue;
            const int il = 3 * (J - 2 * n) + (I - 2 * m);
            const T *S = L.lps + (pm_ * 9 + il) * 9;
#pragma unroll
            for (int kb = 0; kb < 3; ++kb)
#pragma unroll
                for (int ka = 0; ka < 3; ++ka) acc += S[3 * kb + ka] * p[(2 * n + kb) * nxn + 2 * m + ka];
        }
    }
    return acc;
}

// mode 0: F = A(x) - b on free rows, x - g(t) on fixed rows (the Newton defect).
// mode 1: b = Rhs(x) (velocity rows; Dirichlet rows and pressure rows 0).
template <typename T, int MODE>
__global__ void __launch_bounds__(MG_THREADS) k_mg_defect(MgLev<T> L, const T *__restrict__ x,
                                                          const T *__restrict__ b, double up, T *__restrict__ F) {
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= L.N) return;
    const int nxn = L.nx + 1, I = node % nxn, J = node / nxn;
    const T *u = x, *v = x + L.N, *p = x + 2 * L.N;
    const uint8_t fl = L.flags[node];
    T Au = T(0), Av = T(0), Ap = T(0);
#pragma unroll
    for (int cy = 0; cy < 2; ++cy)
#pragma unroll
        for (int cx = 0; cx < 2; ++cx) {
            const int ci = I - 1 + cx, cj = J - 1 + cy;
            if (!fluid(L, ci, cj)) continue;
            const int a = (1 - cx) + 2 * (1 - cy);       // the node's corner in this cell
            linear_rows(L, u, v, p, ci, cj, a, MODE == 1, Au, Av, Ap);
            GaussVel<T> gv;
            gv.eval(L, u, v, ci, cj);
            T cu = T(0), cv = T(0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const T w = L.fc.qw * L.fc.qphi[q][a];
                cu += w * (gv.U[q] * gv.Ux[q] + gv.V[q] * gv.Uy[q]);
                cv += w * (gv.U[q] * gv.Vx[q] + gv.V[q] * gv.Vy[q]);
            }
            const T s = MODE == 1 ? T(-0.5) : T(0.5);
            Au += s * cu;
            Av += s * cv;
        }
    if (MODE == 1) {
        const bool fixed = fl & 1;
        F[node] = fixed ? T(0) : Au;
        F[L.N + node] = fixed ? T(0) : Av;
        F[2 * L.N + node] = T(0);
        return;
    }
    Ap += lps_row(L, p, I, J);
    if (fl & 1) {
        F[node] = u[node] - ((fl & 2) ? inflow(L, J, up) : T(0));
        F[L.N + node] = v[node];
    } else {
        F[node] = Au - b[node];
        F[L.N + node] = Av - b[L.N + node];
    }
    F[2 * L.N + node] = (fl & 4) ? Ap - b[2 * L.N + node] : p[node];
}

// Row (I, J) of J(x) dx, J the Newton matrix of the defect at x (fixed rows: identity).
template <typename T>
__device__ __forceinline__ void jvp_rows(const MgLev<T> &L, const T *x, const T *dx, int I, int J, T (&y)[3]) {
    const int nxn = L.nx + 1, node = J * nxn + I;
    const T *du = dx, *dv = dx + L.N, *dp = dx + 2 * L.N;
    const uint8_t fl = L.flags[node];
    T Au = T(0), Av = T(0), Ap = T(0);
#pragma unroll
    for (int cy = 0; cy < 2; ++cy)
#pragma unroll
        for (int cx = 0; cx < 2; ++cx) {
            const int ci = I - 1 + cx, cj = J - 1 + cy;
            if (!fluid(L, ci, cj)) continue;
            const int a = (1 - cx) + 2 * (1 - cy);
            linear_rows(L, du, dv, dp, ci, cj, a, false, Au, Av, Ap);
            GaussVel<T> g0, g1;   // at x and of the increment
            g0.eval(L, x, x + L.N, ci, cj);
            g1.eval(L, du, dv, ci, cj);
            T cu = T(0), cv = T(0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const T w = L.fc.qw * L.fc.qphi[q][a];
                cu += w * (g0.U[q] * g1.Ux[q] + g0.V[q] * g1.Uy[q] + g1.U[q] * g0.Ux[q] + g1.V[q] * g0.Uy[q]);
                cv += w * (g0.U[q] * g1.Vx[q] + g0.V[q] * g1.Vy[q] + g1.U[q] * g0.Vx[q] + g1.V[q] * g0.Vy[q]);
            }
            Au += T(0.5) * cu;
            Av += T(0.5) * cv;
        }
    Ap += lps_row(L, dp, I, J);
    y[0] = (fl & 1) ? du[node] : Au;
    y[1] = (fl & 1) ? dv[node] : Av;
    y[2] = (fl & 4) ? Ap : dp[node];
}

// y = J(x) dx on every node.
template <typename T>
__global__ void __launch_bounds__(MG_THREADS) k_mg_jvp(MgLev<T> L, const T *__restrict__ x, const T *__restrict__ dx,
                                                       T *__restrict__ y) {
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= L.N) return;
    const int nxn = L.nx + 1, I = node % nxn, J = node / nxn;
    T r[3];
    jvp_rows(L, x, dx, I, J, r);
    y[node] = r[0];
    y[L.N + node] = r[1];
    y[2 * L.N + node] = r[2];
}

// One colour pass of the Vanka smoother for J(x) d = rhs: every fluid cell
// (ci, cj) with ci = cx (mod 4), cj = cy (mod 4) solves the 12 x 12 block of
// J(x) on the unknowns of its four nodes against the current defect
// rhs - J(x) d on those unknowns (rows of fixed unknowns: identity) and adds
// omega times the solution to d.  Cells of one colour
// are four cells apart: none reads a node another one writes, so the pass is
// a block Gauss-Seidel step in any order.
template <typename T>
__global__ void __launch_bounds__(128) k_mg_vanka(MgLev<T> L, const T *__restrict__ x, const T *__restrict__ rhs,
                                                  T *__restrict__ dx, T omega, int cx, int cy) {
    const int nx4 = (L.nx - cx + 3) / 4, ny4 = (L.ny - cy + 3) / 4;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nx4 * ny4) return;
    const int cj = cy + 4 * (k / nx4), ci = cx + 4 * (k % nx4);
    const int cell = cj * L.nx + ci;
    if (L.solid[cell]) return;
    const int nxn = L.nx + 1;
    T A[12][12];
#pragma unroll
    for (int i = 0; i < 12; ++i)
#pragma unroll
        for (int j = 0; j < 12; ++j) A[i][j] = T(0);
    // element contributions of the cells that share a node with this one
    for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
            const int ck = ci + di, cl = cj + dj;
            if (!fluid(L, ck, cl)) continue;
            GaussVel<T> g;
            g.eval(L, x, x + L.N, ck, cl);
            for (int a = 0; a < 4; ++a) {
                const int la = di + (a & 1), lb_a = dj + (a >> 1);   // offset of test node a from (ci, cj)
                if (la < 0 || la > 1 || lb_a < 0 || lb_a > 1) continue;
                const int ra = 3 * (la + 2 * lb_a);
                for (int b = 0; b < 4; ++b) {
                    const int ka = di + (b & 1), kb = dj + (b >> 1);
                    if (ka < 0 || ka > 1 || kb < 0 || kb > 1) continue;
                    const int cb = 3 * (ka + 2 * kb);
                    T nl = T(0), ruu = T(0), ruv = T(0), rvu = T(0), rvv = T(0);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const T w = L.fc.qw * L.fc.qphi[q][a];
                        nl += w * (g.U[q] * L.fc.qdx[q][b] + g.V[q] * L.fc.qdy[q][b]);
                        const T wb = w * L.fc.qphi[q][b];
                        ruu += wb * g.Ux[q];
                        ruv += wb * g.Uy[q];
                        rvu += wb * g.Vx[q];
                        rvv += wb * g.Vy[q];
                    }
                    A[ra][cb] += L.fc.Av[a][b] + T(0.5) * (nl + ruu);
                    A[ra][cb + 1] += T(0.5) * ruv;
                    A[ra + 1][cb] += T(0.5) * rvu;
                    A[ra + 1][cb + 1] += L.fc.Av[a][b] + T(0.5) * (nl + rvv);
                    A[ra][cb + 2] -= L.fc.Gx[a][b];
                    A[ra + 1][cb + 2] -= L.fc.Gy[a][b];
                    A[ra + 2][cb] += L.fc.Dx[a][b];
                    A[ra + 2][cb + 1] += L.fc.Dy[a][b];
                }
            }
        }
    // projection term: patches that hold both nodes of a pair
    int gI[4], gJ[4], gn[4];
    for (int a = 0; a < 4; ++a) {
        gI[a] = ci + (a & 1);
        gJ[a] = cj + (a >> 1);
        gn[a] = gJ[a] * nxn + gI[a];
    }
    for (int m = (ci - 1) >> 1; m <= (ci + 1) >> 1; ++m)
        for (int n = (cj - 1) >> 1; n <= (cj + 1) >> 1; ++n) {
            const int pm_ = patch_mask(L, m, n);
            if (!pm_) continue;
            const T *S = L.lps + pm_ * 81;
            for (int a = 0; a < 4; ++a) {
                const int ia = gI[a] - 2 * m, ja = gJ[a] - 2 * n;
                if (ia < 0 || ia > 2 || ja < 0 || ja > 2) continue;
                for (int b = 0; b < 4; ++b) {
                    const int ib = gI[b] - 2 * m, jb = gJ[b] - 2 * n;
                    if (ib < 0 || ib > 2 || jb < 0 || jb > 2) continue;
                    A[3 * a + 2][3 * b + 2] += S[(3 * ja + ia) * 9 + 3 * jb + ib];
                }
            }
        }
    // right-hand side: the defect rhs - J(x) d on the cell's unknowns.  Rows of
    // fixed unknowns are identity rows of J, so their correction is exactly
    // their defect (the first cell that holds one sets it, later ones add 0).
    T z[12];
    for (int a = 0; a < 4; ++a) {
        const uint8_t fl = L.flags[gn[a]];
        T jd[3];
        jvp_rows(L, x, dx, gI[a], gJ[a], jd);
        for (int c = 0; c < 3; ++c) {
            const int i = 3 * a + c;
            const bool fixed = c < 2 ? (fl & 1) : !(fl & 4);
            z[i] = rhs[c * L.N + gn[a]] - jd[c];
            if (fixed) {
                for (int j = 0; j < 12; ++j) A[i][j] = T(0);
                A[i][i] = T(1);
            }
        }
    }
    // Gaussian elimination with partial pivoting.  A block can be singular: a
    // cell whose 4 nodes all hold Dirichlet velocities couples its pressures
    // only through the projection term, which vanishes on linear functions.
    // A pivot below a relative threshold leaves that unknown's correction 0.
    T scale = T(0);
    for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j) scale = fmax(scale, fabs(A[i][j]));
    const T tiny = scale * (sizeof(T) == 8 ? T(1e-12) : T(1e-6));
    for (int k = 0; k < 12; ++k) {
        int piv = k;
        T best = fabs(A[k][k]);
        for (int i = k + 1; i < 12; ++i)
            if (fabs(A[i][k]) > best) {
                best = fabs(A[i][k]);
                piv = i;
            }
        if (piv != k) {
            for (int j = 0; j < 12; ++j) {
                const T tmp = A[k][j];
                A[k][j] = A[piv][j];
                A[piv][j] = tmp;
            }
            const T tz = z[k];
            z[k] = z[piv];
            z[piv] = tz;
        }
        if (best <= tiny) {
            A[k][k] = T(1);
            for (int j = k + 1; j < 12; ++j) A[k][j] = T(0);
            z[k] = T(0);
            continue;
        }
        const T inv = T(1) / A[k][k];
        for (int i = k + 1; i < 12; ++i) {
            const T f = A[i][k] * inv;
            if (f == T(0)) continue;
            for (int j = k; j < 12; ++j) A[i][j] -= f * A[k][j];
            z[i] -= f * z[k];
        }
    }
    for (int k = 11; k >= 0; --k) {
        T s = z[k];
        for (int j = k + 1; j < 12; ++j) s -= A[k][j] * z[j];
        z[k] = s / A[k][k];
    }
    for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 3; ++c) dx[c * L.N + gn[a]] += omega * z[3 * a + c];
}

// End of a Vanka sweep: every fixed unknown (an identity row of J) takes its
// exact correction, its defect: d = rhs there.  This also reaches the nodes
// that no fluid cell holds (inside an obstacle), which no cell block visits.
template <typename T>
__global__ void __launch_bounds__(MG_THREADS) k_mg_fixed(MgLev<T> L, const T *__restrict__ rhs, T *__restrict__ dx) {
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= L.N) return;
    const uint8_t fl = L.flags[node];
    if (fl & 1) {
        dx[node] = rhs[node];
        dx[L.N + node] = rhs[L.N + node];
    }
    if (!(fl & 4)) dx[2 * L.N + node] = rhs[2 * L.N + node];
}

// Restriction rc = P^T rf from level l (fine) to l+1 (coarse): full weighting
// (weights 1, 1/2, 1/4 of the bilinear prolongation); fixed coarse rows 0.
template <typename T>
__global__ void __launch_bounds__(MG_THREADS) k_mg_restrict(MgLev<T> F, MgLev<T> C, const T *__restrict__ rf,
                                                            T *__restrict__ rc) {
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= C.N) return;
    const int cn = C.nx + 1, i = node % cn, j = node / cn, fn = F.nx + 1;
    const uint8_t fl = C.flags[node];
    T acc[3] = {T(0), T(0), T(0)};
    for (int dj = -1; dj <= 1; ++dj) {
        const int J = 2 * j + dj;
        if (J < 0 || J > F.ny) continue;
        for (int di = -1; di <= 1; ++di) {
            const int I = 2 * i + di;
            if (I < 0 || I > F.nx) continue;
            const T w = (di ? T(0.5) : T(1)) * (dj ? T(0.5) : T(1));
            const int n = J * fn + I;
            for (int c = 0; c < 3; ++c) acc[c] += w * rf[c * F.N + n];
        }
    }
    rc[node] = (fl & 1) ? T(0) : acc[0];
    rc[C.N + node] = (fl & 1) ? T(0) : acc[1];
    rc[2 * C.N + node] = (fl & 4) ? acc[2] : T(0);
}

// df += P dc (bilinear prolongation from level l+1 to l); fixed fine rows unchanged.
template <typename T>
__global__ void __launch_bounds__(MG_THREADS) k_mg_prolong_add(MgLev<T> F, MgLev<T> C, const T *__restrict__ dc,
                                                               T *__restrict__ df) {
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= F.N) return;
    const int fn = F.nx + 1, I = node % fn, J = node / fn, cn = C.nx + 1;
    const uint8_t fl = F.flags[node];
    const int i0 = I >> 1, j0 = J >> 1, i1 = (I + 1) >> 1, j1 = (J + 1) >> 1;
    const T h = T(0.5);
    for (int c = 0; c < 3; ++c) {
        const bool fixed = c < 2 ? (fl & 1) : !(fl & 4);
        if (fixed) continue;
        const T *d = dc + c * C.N;
        const T v = h * (h * (d[j0 * cn + i0] + d[j0 * cn + i1]) + h * (d[j1 * cn + i0] + d[j1 * cn + i1]));
        df[c * F.N + node] += v;
    }
}

// xc = x_f at the coarse nodes (the linearisation point of a coarser level).
template <typename T>
__global__ void __launch_bounds__(MG_THREADS) k_mg_inject(MgLev<T> F, MgLev<T> C, const T *__restrict__ xf,
                                                          T *__restrict__ xc) {
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= C.N) return;
    const int cn = C.nx + 1, i = node % cn, j = node / cn;
    const int n = (2 * j) * (F.nx + 1) + 2 * i;
    for (int c = 0; c < 3; ++c) xc[c * C.N + node] = xf[c * F.N + n];
}

template <typename T>
__global__ void __launch_bounds__(MG_THREADS) k_mg_dot(const T *__restrict__ a, const T *__restrict__ b, long long n,
                                                       double *__restrict__ out) {
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += (double)a[i] * (double)b[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double part[MG_THREADS / 32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < MG_THREADS / 32 ? part[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) atomicAdd(out, acc);
    }
}

template <typename T>
__global__ void __launch_bounds__(MG_THREADS) k_mg_axpby(T alpha, const T *__restrict__ x, T beta, T *__restrict__ y,
                                                         long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = alpha * x[i] + (beta == T(0) ? T(0) : beta * y[i]);
}

}  // namespace

// ---------------------------------------------------------------- host side
struct MgLevelHost {
    int nx, ny, N;
    std::vector<uint8_t> solid, flags, mult;
    uint8_t *d_solid = nullptr, *d_flags = nullptr, *d_mult = nullptr;
    double *d_lps64 = nullptr;
    float *d_lps32 = nullptr;
    FemCoef<double> f64;
    FemCoef<float> f32;
};

}  // namespace dnnmg

struct dnnmg_mg_s {
    dnnmg_mg_desc desc;
    int device;
    std::vector<dnnmg::MgLevelHost> levels;
};

namespace dnnmg {
namespace {

template <typename T> MgLev<T> dev_level(const dnnmg_mg_s &m, int l) {
    const MgLevelHost &h = m.levels[l];
    MgLev<T> L;
    L.nx = h.nx;
    L.ny = h.ny;
    L.N = h.N;
    L.solid = h.d_solid;
    L.flags = h.d_flags;
    L.mult = h.d_mult;
    if constexpr (sizeof(T) == 8) L.lps = h.d_lps64;
    else L.lps = h.d_lps32;
    L.hy = m.desc.ly / h.ny;
    L.ly = m.desc.ly;
    if constexpr (sizeof(T) == 8) L.fc = h.f64;
    else L.fc = h.f32;
    return L;
}

// Node flags (Sec. 6.1 boundary classes) and fluid-cell counts of a level.
void node_classes(MgLevelHost &h) {
    const int nx = h.nx, ny = h.ny, nxn = nx + 1;
    h.flags.assign(h.N, 0);
    h.mult.assign(h.N, 0);
    for (int J = 0; J <= ny; ++J)
        for (int I = 0; I <= nx; ++I) {
            bool touch_solid = false, touch_fluid = false;
            int m = 0;
            for (int cy = 0; cy < 2; ++cy)
                for (int cx = 0; cx < 2; ++cx) {
                    const int ci = I - 1 + cx, cj = J - 1 + cy;
                    if (ci < 0 || cj < 0 || ci >= nx || cj >= ny) continue;
                    if (h.solid[(size_t)cj * nx + ci]) touch_solid = true;
                    else {
                        touch_fluid = true;
                        ++m;
                    }
                }
            const bool wall = J == 0 || J == ny;
            const bool dir = wall || I == 0 || touch_solid;
            const bool inflow = I == 0 && !wall && !touch_solid;
            h.flags[(size_t)J * nxn + I] = (uint8_t)((dir ? 1 : 0) | (inflow ? 2 : 0) | (touch_fluid ? 4 : 0));
            h.mult[(size_t)J * nxn + I] = (uint8_t)m;
        }
}

int check_level(const dnnmg_mg_s *m, int level, int need_coarser = 0) {
    if (!m) return fail(DNNMG_EINVAL, "multigrid handle is NULL");
    if (level < 0 || level + need_coarser >= (int)m->levels.size())
        return fail(DNNMG_EINVAL, "level %d out of range (%zu levels)", level, m->levels.size());
    int cur = -1;
    DNNMG_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != m->device) return fail(DNNMG_EINVAL, "handle belongs to device %d but device %d is current", m->device, cur);
    return DNNMG_OK;
}

unsigned blocks(long long n, int th) { return (unsigned)((n + th - 1) / th); }

// Projection patch matrices by the patch's fluid cells: for each subset (bit
// 2 cb + ca), the sum over its cells T of alpha (grad(p - pi p), grad(q - pi q))_T
// on the 9 patch nodes (Eq. disc:ns; a partly solid patch of a single level's
// own mask contributes its fluid cells only).  pi: the bilinear interpolant of
// the patch's 4 corners; alpha = alpha0 (hx^2 + hy^2) / nu.
void lps_tables(const FemCoef<double> &f, double hx, double hy, double alpha0, double nu, std::vector<double> *out) {
    double S[4][4];   // (grad phi_a, grad phi_b) over one cell, 2 x 2 Gauss
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            double s = 0.0;
            for (int q = 0; q < 4; ++q) s += f.qw * (f.qdx[q][a] * f.qdx[q][b] + f.qdy[q][a] * f.qdy[q][b]);
            S[a][b] = s;
        }
    double F[9][9];   // I - pi
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) F[i][j] = i == j ? 1.0 : 0.0;
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
            const double X = a / 2.0, Y = b / 2.0;
            F[3 * b + a][0] -= (1 - X) * (1 - Y);
            F[3 * b + a][2] -= X * (1 - Y);
            F[3 * b + a][6] -= (1 - X) * Y;
            F[3 * b + a][8] -= X * Y;
        }
    const double alpha = alpha0 * (hx * hx + hy * hy) / nu;
    double Lc[4][9][9];
    for (int c = 0; c < 4; ++c) {
        const int ca = c & 1, cb = c >> 1;
        double S9[9][9] = {};
        const int ids[4] = {3 * cb + ca, 3 * cb + ca + 1, 3 * (cb + 1) + ca, 3 * (cb + 1) + ca + 1};
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) S9[ids[a]][ids[b]] = S[a][b];
        for (int i = 0; i < 9; ++i)
            for (int j = 0; j < 9; ++j) {
                double s = 0.0;
                for (int k = 0; k < 9; ++k)
                    for (int l = 0; l < 9; ++l) s += F[k][i] * S9[k][l] * F[l][j];
                Lc[c][i][j] = alpha * s;
            }
    }
    out->assign(16 * 81, 0.0);
    for (int mask = 0; mask < 16; ++mask)
        for (int c = 0; c < 4; ++c)
            if (mask & (1 << c))
                for (int i = 0; i < 81; ++i) (*out)[mask * 81 + i] += (&Lc[c][0][0])[i];
}

}  // namespace
}  // namespace dnnmg

using namespace dnnmg;

extern "C" {

int dnnmg_mg_create(const dnnmg_mg_desc *d, dnnmg_mg_t *out) {
    clear_error();
    if (!d || !out) return fail(DNNMG_EINVAL, "NULL argument");
    *out = nullptr;
    if (d->levels < 1 || d->levels > 12) return fail(DNNMG_EINVAL, "levels=%d out of range 1..12", d->levels);
    const int div = 1 << d->levels;
    if (d->nx <= 0 || d->ny <= 0 || d->nx % div || d->ny % div)
        return fail(DNNMG_EINVAL, "nx=%d, ny=%d must be positive multiples of 2^levels = %d", d->nx, d->ny, div);
    if (!(d->lx > 0) || !(d->ly > 0) || !(d->nu > 0) || !(d->k > 0) || !(d->alpha0 >= 0))
        return fail(DNNMG_EINVAL, "lx, ly, nu, k must be > 0 and alpha0 >= 0");
    if (d->precision != DNNMG_F64 && d->precision != DNNMG_F32)
        return fail(DNNMG_EINVAL, "precision must be DNNMG_F64 or DNNMG_F32");
    if ((long long)(d->nx + 1) * (d->ny + 1) > (1LL << 30)) return fail(DNNMG_EUNSUPPORTED, "too many nodes");
    dnnmg_mg_s *m = new (std::nothrow) dnnmg_mg_s();
    if (!m) return fail(DNNMG_ENOMEM, "host allocation failed");
    m->desc = *d;
    m->desc.solid = nullptr;
    cudaGetDevice(&m->device);
    m->levels.resize(d->levels);
    for (int l = 0; l < d->levels; ++l) {
        MgLevelHost &h = m->levels[l];
        h.nx = d->nx >> l;
        h.ny = d->ny >> l;
        h.N = (h.nx + 1) * (h.ny + 1);
        h.solid.assign((size_t)h.nx * h.ny, 0);
        if (l == 0) {
            if (d->solid)
                for (size_t i = 0; i < h.solid.size(); ++i) h.solid[i] = d->solid[i] ? 1 : 0;
        } else {
            // patch (m, n) of this level is solid iff all 16 cells of the finer level under it are
            const MgLevelHost &f = m->levels[l - 1];
            for (int n = 0; n < h.ny / 2; ++n)
                for (int mm = 0; mm < h.nx / 2; ++mm) {
                    bool all = true;
                    for (int jj = 0; jj < 4 && all; ++jj)
                        for (int ii = 0; ii < 4 && all; ++ii)
                            if (!f.solid[(size_t)(4 * n + jj) * f.nx + 4 * mm + ii]) all = false;
                    for (int jj = 0; jj < 2; ++jj)
                        for (int ii = 0; ii < 2; ++ii) h.solid[(size_t)(2 * n + jj) * h.nx + 2 * mm + ii] = all ? 1 : 0;
                }
        }
        node_classes(h);
        // every level keeps the finest level's projection coefficient alpha:
        // the fine term vanishes on prolongated pressures, and a coefficient
        // growing with h^2 would swamp the coarse pressure corrections
        const double alpha0_l = d->alpha0 / (double)(1LL << (2 * l));
        level_coefficients(d->lx, d->ly, h.nx, h.ny, d->nu, d->k, alpha0_l, &h.f64, &h.f32);
        std::vector<double> lps;
        lps_tables(h.f64, d->lx / h.nx, d->ly / h.ny, alpha0_l, d->nu, &lps);
        std::vector<float> lps32(lps.begin(), lps.end());
        if (cudaMalloc(&h.d_lps64, lps.size() * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&h.d_lps32, lps32.size() * sizeof(float)) != cudaSuccess ||
            cudaMemcpy(h.d_lps64, lps.data(), lps.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(h.d_lps32, lps32.data(), lps32.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            dnnmg_mg_destroy(m);
            return fail(DNNMG_ENOMEM, "device allocation of level %d failed", l);
        }
        if (cudaMalloc(&h.d_solid, h.solid.size()) != cudaSuccess || cudaMalloc(&h.d_flags, h.N) != cudaSuccess ||
            cudaMalloc(&h.d_mult, h.N) != cudaSuccess ||
            cudaMemcpy(h.d_solid, h.solid.data(), h.solid.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(h.d_flags, h.flags.data(), h.N, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(h.d_mult, h.mult.data(), h.N, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            dnnmg_mg_destroy(m);
            return fail(DNNMG_ENOMEM, "device allocation of level %d failed", l);
        }
    }
    *out = m;
    return DNNMG_OK;
}

int dnnmg_mg_destroy(dnnmg_mg_t m) {
    clear_error();
    if (!m) return DNNMG_OK;
    for (MgLevelHost &h : m->levels) {
        cudaFree(h.d_solid);
        cudaFree(h.d_flags);
        cudaFree(h.d_mult);
        cudaFree(h.d_lps64);
        cudaFree(h.d_lps32);
    }
    delete m;
    return DNNMG_OK;
}

int dnnmg_mg_level(dnnmg_mg_t m, int level, int *nx, int *ny, unsigned char *solid) {
    clear_error();
    if (!m) return fail(DNNMG_EINVAL, "multigrid handle is NULL");
    if (level < 0 || level >= (int)m->levels.size()) return fail(DNNMG_EINVAL, "level %d out of range", level);
    const MgLevelHost &h = m->levels[level];
    if (nx) *nx = h.nx;
    if (ny) *ny = h.ny;
    if (solid)
        for (size_t i = 0; i < h.solid.size(); ++i) solid[i] = h.solid[i];
    return DNNMG_OK;
}

#define MG_DISPATCH(call_f64, call_f32)                         \
    do {                                                        \
        if (m->desc.precision == DNNMG_F64) { call_f64; }       \
        else { call_f32; }                                      \
        DNNMG_CUDA_TRY(cudaGetLastError());                     \
    } while (0)

static double inflow_peak_mg(const dnnmg_mg_desc &d, double t) {
    const double w = d.ramp ? (t <= 0.5 ? 0.5 - 0.5 * std::cos(2.0 * 3.14159265358979323846 * t) : 1.0) : 1.0;
    return d.u_max * w;
}

int dnnmg_mg_defect(dnnmg_mg_t m, int level, const void *x, const void *b, double t, void *F, cudaStream_t s) {
    clear_error();
    if (int e = check_level(m, level)) return e;
    if (!x || !b || !F) return fail(DNNMG_EINVAL, "NULL array");
    const int N = m->levels[level].N;
    const double up = inflow_peak_mg(m->desc, t);
    MG_DISPATCH((k_mg_defect<double, 0><<<blocks(N, MG_THREADS), MG_THREADS, 0, s>>>(
                    dev_level<double>(*m, level), (const double *)x, (const double *)b, up, (double *)F)),
                (k_mg_defect<float, 0><<<blocks(N, MG_THREADS), MG_THREADS, 0, s>>>(
                    dev_level<float>(*m, level), (const float *)x, (const float *)b, up, (float *)F)));
    return DNNMG_OK;
}

int dnnmg_mg_rhs(dnnmg_mg_t m, int level, const void *x, void *b, cudaStream_t s) {
    clear_error();
    if (int e = check_level(m, level)) return e;
    if (!x || !b) return fail(DNNMG_EINVAL, "NULL array");
    if (x == b) return fail(DNNMG_EINVAL, "x and b must not alias");
    const int N = m->levels[level].N;
    MG_DISPATCH((k_mg_defect<double, 1><<<blocks(N, MG_THREADS), MG_THREADS, 0, s>>>(
                    dev_level<double>(*m, level), (const double *)x, nullptr, 0.0, (double *)b)),
                (k_mg_defect<float, 1><<<blocks(N, MG_THREADS), MG_THREADS, 0, s>>>(
                    dev_level<float>(*m, level), (const float *)x, nullptr, 0.0, (float *)b)));
    return DNNMG_OK;
}

int dnnmg_mg_jvp(dnnmg_mg_t m, int level, const void *x, const void *dx, void *y, cudaStream_t s) {
    clear_error();
    if (int e = check_level(m, level)) return e;
    if (!x || !dx || !y) return fail(DNNMG_EINVAL, "NULL array");
    if (y == dx || y == x) return fail(DNNMG_EINVAL, "y must not alias x or dx");
    const int N = m->levels[level].N;
    MG_DISPATCH((k_mg_jvp<double><<<blocks(N, MG_THREADS), MG_THREADS, 0, s>>>(
                    dev_level<double>(*m, level), (const double *)x, (const double *)dx, (double *)y)),
                (k_mg_jvp<float><<<blocks(N, MG_THREADS), MG_THREADS, 0, s>>>(
                    dev_level<float>(*m, level), (const float *)x, (const float *)dx, (float *)y)));
    return DNNMG_OK;
}

int dnnmg_mg_vanka(dnnmg_mg_t m, int level, const void *x, const void *r, void *dx, double omega, cudaStream_t s) {
    clear_error();
    if (int e = check_level(m, level)) return e;
    if (!x || !r || !dx) return fail(DNNMG_EINVAL, "NULL array");
    if (dx == r || dx == x) return fail(DNNMG_EINVAL, "dx must not alias x or r");
    const MgLevelHost &h = m->levels[level];
    const long long nc = (long long)((h.nx + 3) / 4) * ((h.ny + 3) / 4);
    for (int cy = 0; cy < 4; ++cy)
        for (int cx = 0; cx < 4; ++cx)
            MG_DISPATCH((k_mg_vanka<double><<<blocks(nc, 128), 128, 0, s>>>(
                            dev_level<double>(*m, level), (const double *)x, (const double *)r, (double *)dx, omega, cx, cy)),
                        (k_mg_vanka<float><<<blocks(nc, 128), 128, 0, s>>>(
                            dev_level<float>(*m, level), (const float *)x, (const float *)r, (float *)dx, (float)omega,
                            cx, cy)));
    MG_DISPATCH((k_mg_fixed<double><<<blocks(h.N, MG_THREADS), MG_THREADS, 0, s>>>(
                    dev_level<double>(*m, level), (const double *)r, (double *)dx)),
                (k_mg_fixed<float><<<blocks(h.N, MG_THREADS), MG_THREADS, 0, s>>>(
                    dev_level<float>(*m, level), (const float *)r, (float *)dx)));
    return DNNMG_OK;
}

int dnnmg_mg_restrict(dnnmg_mg_t m, int level, const void *rf, void *rc, cudaStream_t s) {
    clear_error();
    if (int e = check_level(m, level, 1)) return e;
    if (!rf || !rc) return fail(DNNMG_EINVAL, "NULL array");
    const int Nc = m->levels[level + 1].N;
    MG_DISPATCH((k_mg_restrict<double><<<blocks(Nc, MG_THREADS), MG_THREADS, 0, s>>>(
                    dev_level<double>(*m, level), dev_level<double>(*m, level + 1), (const double *)rf, (double *)rc)),
                (k_mg_restrict<float><<<blocks(Nc, MG_THREADS), MG_THREADS, 0, s>>>(
                    dev_level<float>(*m, level), dev_level<float>(*m, level + 1), (const float *)rf, (float *)rc)));
    return DNNMG_OK;
}

int dnnmg_mg_prolong_add(dnnmg_mg_t m, int level, const void *dc, void *df, cudaStream_t s) {
    clear_error();
    if (int e = check_level(m, level, 1)) return e;
    if (!dc || !df) return fail(DNNMG_EINVAL, "NULL array");
    const int Nf = m->levels[level].N;
    MG_DISPATCH((k_mg_prolong_add<double><<<blocks(Nf, MG_THREADS), MG_THREADS, 0, s>>>(
                    dev_level<double>(*m, level), dev_level<double>(*m, level + 1), (const double *)dc, (double *)df)),
                (k_mg_prolong_add<float><<<blocks(Nf, MG_THREADS), MG_THREADS, 0, s>>>(
                    dev_level<float>(*m, level), dev_level<float>(*m, level + 1), (const float *)dc, (float *)df)));
    return DNNMG_OK;
}

int dnnmg_mg_inject(dnnmg_mg_t m, int level, const void *xf, void *xc, cudaStream_t s) {
    clear_error();
    if (int e = check_level(m, level, 1)) return e;
    if (!xf || !xc) return fail(DNNMG_EINVAL, "NULL array");
    const int Nc = m->levels[level + 1].N;
    MG_DISPATCH((k_mg_inject<double><<<blocks(Nc, MG_THREADS), MG_THREADS, 0, s>>>(
                    dev_level<double>(*m, level), dev_level<double>(*m, level + 1), (const double *)xf, (double *)xc)),
                (k_mg_inject<float><<<blocks(Nc, MG_THREADS), MG_THREADS, 0, s>>>(
                    dev_level<float>(*m, level), dev_level<float>(*m, level + 1), (const float *)xf, (float *)xc)));
    return DNNMG_OK;
}

int dnnmg_mg_dot(dnnmg_mg_t m, long long n, const void *a, const void *b, double *out, cudaStream_t s) {
    clear_error();
    if (!m) return fail(DNNMG_EINVAL, "multigrid handle is NULL");
    if (!a || !b || !out || n < 0) return fail(DNNMG_EINVAL, "NULL array or negative size");
    DNNMG_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double), s));
    if (n == 0) return DNNMG_OK;
    const unsigned g = blocks(n, MG_THREADS) < 152u * 8u ? blocks(n, MG_THREADS) : 152u * 8u;
    MG_DISPATCH((k_mg_dot<double><<<g, MG_THREADS, 0, s>>>((const double *)a, (const double *)b, n, out)),
                (k_mg_dot<float><<<g, MG_THREADS, 0, s>>>((const float *)a, (const float *)b, n, out)));
    return DNNMG_OK;
}

int dnnmg_mg_axpby(dnnmg_mg_t m, long long n, double alpha, const void *x, double beta, void *y, cudaStream_t s) {
    clear_error();
    if (!m) return fail(DNNMG_EINVAL, "multigrid handle is NULL");
    if (!x || !y || n < 0) return fail(DNNMG_EINVAL, "NULL array or negative size");
    if (n == 0) return DNNMG_OK;
    const unsigned g = blocks(n, MG_THREADS) < 152u * 8u ? blocks(n, MG_THREADS) : 152u * 8u;
    MG_DISPATCH((k_mg_axpby<double><<<g, MG_THREADS, 0, s>>>(alpha, (const double *)x, beta, (double *)y, n)),
                (k_mg_axpby<float><<<g, MG_THREADS, 0, s>>>((float)alpha, (const float *)x, (float)beta, (float *)y,
                                                           n)));
    return DNNMG_OK;
}

}  // extern "C"

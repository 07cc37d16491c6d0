// Internal declarations of libdnnmg: mesh/net handles, per-mesh constants and
// kernel launchers.  The public boundary is include/dnnmg.h.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "dnnmg.h"

namespace dnnmg {

// ---------------------------------------------------------------- errors
int fail(int code, const char *fmt, ...);
void clear_error();

#define DNNMG_CUDA_TRY(expr)                                                               \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return ::dnnmg::fail(DNNMG_ECUDA, "%s failed: %s (%s:%d)", #expr,              \
                                 cudaGetErrorString(e_), __FILE__, __LINE__);               \
    } while (0)

// Launch check: reports configuration errors of the launch just enqueued.
#define DNNMG_LAUNCH_CHECK(name)                                                           \
    do {                                                                                    \
        cudaError_t e_ = cudaGetLastError();                                                \
        if (e_ != cudaSuccess)                                                              \
            return ::dnnmg::fail(DNNMG_ECUDA, "launch of %s failed: %s", name,              \
                                 cudaGetErrorString(e_));                                   \
    } while (0)

// ---------------------------------------------------------------- geometry
// Plain-value view of a mesh handed to kernels.
struct MeshGeom {
    int nxc, nyc, K, r, s, S;     // r = 2^K fine cells per coarse cell, S = s r per patch
    int nxf, nyf, npx, npy, P;
    int pitch;                    // fine row pitch in elements, round_up(nxf + 1, 64)
    size_t plane;                 // elements per fine component plane, pitch (nyf + 1)
    int nf, nc, n_in, n_out, ldx;
    double lx, ly, hxc, hyc, hxf, hyf;
    double nu, k, u_max;
    int ramp;
    const uint8_t *solid;         // device [nyc][nxc], 1 = solid coarse cell
    const int *patch_id;          // device [npy][npx], fluid patch number or -1
    const int *patch_cell;        // device [P], pj npx + pi
    const int *feat_tab;          // device [ldx], source of each feature column (stencil.cu)
    const uint8_t *tile_flags;    // device [nty][ntx], all-fluid bits of each 32 x 16-cell tile
    int ntx, nty;
    const int *slow_tiles;        // device [n_slow_tiles]: tiles without the all-fluid bit (ty ntx + tx)
    int n_slow_tiles;
    const uint16_t *cf_tab;       // device [ldx]: feature column sources of the closed-form tiles
    int *status;                  // device status word of the mesh (DNNMG_DEVERR_* bits)
};

// Element constants of one fine cell (local nodes SW, SE, NW, NE) and of one
// 2x2-cell LPS patch, in the arithmetic type of the fine fields.
template <typename T>
struct FemCoef {
    T Av[4][4];     // 1/k M + nu/2 Kd : linear velocity operator (Eq. nonlinearshort)
    T Bv[4][4];     // 1/k M - nu/2 Kd : right-hand side (Eq. 4cranknicholson3)
    T Gx[4][4];     // int phi_b d_x phi_a : pressure term of velocity row a
    T Gy[4][4];     // int phi_b d_y phi_a
    T Dx[4][4];     // int d_x phi_b phi_a : divergence term of pressure row a
    T Dy[4][4];
    T S9[9][9];     // LPS: alpha (I - Pi)^T L (I - Pi) on a 2x2-cell patch
    T qphi[4][4];   // [gauss point][node] shape values (2x2 Gauss)
    T qdx[4][4];    // x derivatives at the Gauss points
    T qdy[4][4];
    T qw;           // Gauss weight hx hy / 4
    T geo[12];      // patch geometry features
    T q_over_nu;    // Peclet scale: longest patch edge / nu
    // node stencils [dy+1][dx+1] of interior nodes (4 fluid cells), assembled
    // from the element matrices above
    T nA[3][3], nB[3][3], nGx[3][3], nGy[3][3], nDx[3][3], nDy[3][3];
    // LPS node stencils of interior nodes [y class][x class][dy+2][dx+2]; a
    // node's class in one direction is 0 on a patch edge line (two patches
    // hold it) and 1 on a patch mid line (one patch)
    T L5[2][2][5][5];
    // tensor-product 2x2 Gauss evaluation of the convection term
    T cg0, cg1;       // Gauss points on [0, 1]
    T inv_hx, inv_hy;
    T cwg0, cwg1;     // (qw / 2) * Gauss point
};

struct Mesh {
    dnnmg_mesh_desc desc;
    dnnmg_mesh_info info;
    MeshGeom g;
    FemCoef<double> fem64;
    FemCoef<float> fem32;
    int device;
    uint8_t *d_solid;
    int *d_patch_id;
    int *d_patch_cell;
    int *d_feat_tab;
    uint8_t *d_tile_flags;
    int *d_slow_tiles;
    uint16_t *d_cf_tab;
    int *d_status;
    // the boundary tiles of S2+S3 run on this stream beside the closed-form
    // kernel (forked from and joined back to the caller's stream)
    cudaStream_t side;
    cudaEvent_t ev_fork, ev_join;
};

struct Net {
    int n_in, ldx, H, n_out, precision;
    int device;
    int *d_status;                // device status word (DNNMG_DEVERR_* bits)
    void *tc;                     // tensor-core schedule (gru_tc.cu), null if not used
    // transposed weights for the CUDA-core kernel: WxT [ldx][3H], UhT [H][3H], WfcT [H][n_out]
    void *WxT, *UhT, *WfcT;
    // K-major bf16 operands for the tensor-core kernel (BF16NET only, may be null)
    void *tc_weights;
    size_t tc_bytes;
};

int round_up(int v, int m);
// Tiled TMA descriptor (no swizzle, zero fill out of bounds); strides in
// bytes for dimensions 1 .. rank-1.  False if the driver entry point is
// missing or the layout is not expressible.
bool tma_encode_tiled(CUtensorMap *map, CUtensorMapDataType type, unsigned rank, void *base, const cuuint64_t *dims,
                      const cuuint64_t *strides, const cuuint32_t *box);
size_t align256(size_t v);

// ---------------------------------------------------------------- launchers
// All return cudaSuccess or the launch error; `prec` is DNNMG_F64/F32/BF16NET.
cudaError_t launch_prolongate(const MeshGeom &g, int prec, const double *xc, void *xf,
                              double t, cudaStream_t st);
// xc == NULL: x~ is read from xf; otherwise x~ = P xc (with the Dirichlet
// values at time t) is formed inside the kernel and xf is not read.
cudaError_t launch_residual_features(const MeshGeom &g, int prec, const FemCoef<double> &f64,
                                     const FemCoef<float> &f32, const void *xf, const double *xc, double t,
                                     const void *bf, void *rf, void *X, cudaStream_t st);
// xcp (may be null): the step's padded copy of x_c in the fine type, read
// instead of xc for the coarse window (the same values)
cudaError_t launch_scatter_avg(const MeshGeom &g, int prec, const void *d, const void *xf, const double *xc,
                               double t, void *vcorr, cudaStream_t st, const void *xcp = nullptr);
cudaError_t launch_rhs(const MeshGeom &g, int prec, const FemCoef<double> &f64,
                       const FemCoef<float> &f32, const void *vcorr, void *bf, cudaStream_t st);
// The coarse vector in the fine arithmetic type, rows padded to pc (a
// multiple of 32) so that tiles can fetch coarse windows by TMA: xcp
// [3][nyc+1][pc], zero past nxc.
int coarse_pitch(const MeshGeom &g);
cudaError_t launch_coarse_pad(const MeshGeom &g, int prec, const double *xc, void *xcp, cudaStream_t st);
// S2 + S3 of the correction step on the padded coarse vector: persistent
// CTAs, TMA-fed and double-buffered tiles (same arithmetic as
// launch_residual_features with xc; rf is not written).
cudaError_t launch_residual_step(const MeshGeom &g, int prec, const FemCoef<double> &f64, const FemCoef<float> &f32,
                                 const void *xcp, double t, const void *bf, void *X, cudaStream_t st,
                                 bool skip_fast = false);
// S2 + S3 of the step on the all-fluid tiles in closed form (residual_cf.cu):
// FP32 fields, K = 1 or 2.  launch_residual_step(..., skip_fast = true) then
// does the other tiles.
bool residual_cf_supported(const MeshGeom &g, int prec);
// Column table of the closed-form tiles' feature gather ([ldx] entries).
void residual_cf_table(const MeshGeom &g, uint16_t *tab);
// The general S2+S3 tiles (ty ntx + tx) that the closed form leaves, from the tile flags.
void residual_cf_slow_tiles(const MeshGeom &g, const uint8_t *flags, std::vector<int> *slow);
cudaError_t launch_residual_cf(const MeshGeom &g, int prec, const FemCoef<float> &f32, const void *xcp, const void *bf,
                               void *X, cudaStream_t st);
// S5 + S6 fused: b_f = Rhs(P x_c + mean of d) without writing v_corr.
cudaError_t launch_avg_rhs(const MeshGeom &g, int prec, const FemCoef<double> &f64, const FemCoef<float> &f32,
                           const void *d, const double *xc, double t, void *bf, cudaStream_t st);
cudaError_t launch_restrict(const MeshGeom &g, int prec, const void *bf, double *bc,
                            cudaStream_t st);
cudaError_t launch_mesh_maps(const MeshGeom &g, unsigned char *flags, unsigned char *mult,
                             cudaStream_t st);
cudaError_t launch_gru(const Net &net, const void *X, void *h, void *d, int P, cudaStream_t st);
int gru_launch_count(const Net &net);
cudaError_t launch_gru_cuda_core(const Net &n, const void *X, void *h, void *d, int P, cudaStream_t st);
cudaError_t launch_gru_tc(const Net &n, const void *X, void *h, void *d, int P, cudaStream_t st);
cudaError_t launch_gru_tc_rows(const Net &n, const void *X, void *h, void *d, int P, const int *hrow, int h_rows,
                               cudaStream_t st);
bool tc_prepare(Net &n, const double *Wx, const double *Uh, const double *Wfc);
// C (+)= A B^T with BF16 A [M][K] (lda), B [N][K] (ldb) on the tensor cores
// (gemm_tc.cu); splits > 1: K-range partials to part (reduced by the caller),
// gemm_tc_splits_used of them.
cudaError_t launch_gemm_tc(int M, int N, int K, const void *A, int lda, const void *B, int ldb, float *C, int ldc,
                           bool accumulate, int splits, float *part, int *status, cudaStream_t st);
int gemm_tc_splits_used(int K, int splits);
void tc_release(Net &n);
// Per feature column: (kind << 24) | offset into the residual / node tiles of stencil.cu.
void feature_table(const MeshGeom &g, int *tab);
int feature_table_capacity();
// Per 32 x 16-cell stencil tile (ntx x nty of them): bit 0 = every fine cell
// within two cells of the tile exists and is fluid, bit 1 = the same within one.
void tile_flags(const MeshGeom &g, const uint8_t *solid, uint8_t *flags);
void tile_counts(const MeshGeom &g, int *ntx, int *nty);
// Scratch bytes of the device-buffer step (the workspace minus the host-call staging).
size_t step_scratch_bytes(const dnnmg_mesh_info &I);
// dnnmg_step on a caller-chosen scratch of at least step_scratch_bytes (argument checks included).
int step_on_workspace(dnnmg_mesh_t mesh, dnnmg_net_t net, const double *xc, void *h, void *bf, double *bc,
                      void *workspace, size_t workspace_bytes, double t, cudaStream_t stream);

}  // namespace dnnmg

// The C-ABI handle types are the library's own structures.
struct dnnmg_mesh_s : dnnmg::Mesh {};
struct dnnmg_net_s : dnnmg::Net {};


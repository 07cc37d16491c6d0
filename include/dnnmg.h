/*
 * dnnmg.h -- C ABI of the DNN-MG fine-level correction step on one GPU.
 *
 * DNN-MG (Margenberg, Hartmann, Lessig, Richter, arXiv 2008.11520) corrects a
 * coarse multigrid solution on level L with a patch-wise recurrent network on
 * level L+K.  After the coarse Newton-Krylov solve of a time step, the
 * correction step of Algorithm 2 does
 *     v~    <- P(v^L)                      prolongation            (dnnmg_prolongate)
 *     d     <- N(v~, Omega_L, Omega_L+K)   residual + features     (dnnmg_patch_features)
 *                                          GRU + output layer      (dnnmg_gru_step)
 *     b^L+K <- Rhs(v~ + d)                 averaging               (dnnmg_scatter_avg)
 *                                          right-hand side
 *     b^L   <- R(b^L+K)                    restriction             (dnnmg_rhs_restrict)
 * and dnnmg_step runs all of them in order on one stream.
 *
 * Conventions shared by every call:
 *  - Every call returns DNNMG_OK (0) or an error code; dnnmg_last_error()
 *    returns the calling thread's last message.  Invalid arguments are
 *    reported before anything is enqueued.
 *  - Array arguments are DEVICE pointers owned by the caller unless the name
 *    ends in _host.  The library never frees caller memory and allocates
 *    device memory only in *_create.  Compute calls are asynchronous on the
 *    given stream and never synchronise.
 *  - Fine node fields are pitched planes [component][nyf+1][pitch]: node
 *    (I, J) of component c is element c*plane + J*pitch + I, with
 *    pitch = round_up(nxf+1, 64) and plane = pitch*(nyf+1) (info.pitch,
 *    info.plane).  Columns nxf+1 .. pitch-1 are padding: kernels may write
 *    them and never use them.  Fine arrays must be 16-byte aligned.  Coarse
 *    vectors are unpadded planes [component][Nc], Nc = (nxc+1)(nyc+1), node
 *    (i, j) at j*(nxc+1) + i.  The fine "real" type is double for DNNMG_F64
 *    and float otherwise; coarse vectors are double.
 *  - Patch arrays are row-major [P][.] over the fluid patches, numbered
 *    lexicographically over the patch grid, patch-x fastest.
 */
#ifndef DNNMG_H
#define DNNMG_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define DNNMG_OK 0
#define DNNMG_EINVAL 1       /* null pointer, size or parameter out of range */
#define DNNMG_ECUDA 2        /* a CUDA runtime call or kernel launch failed */
#define DNNMG_EUNSUPPORTED 3 /* valid request the library does not implement */
#define DNNMG_ENOMEM 4       /* device allocation in *_create failed */

/* precision of the fine fields and of the patch network */
#define DNNMG_F64 0      /* fine fields, features and network in double */
#define DNNMG_F32 1      /* fine fields, features and network in float */
#define DNNMG_BF16NET 2  /* fine fields float; features and network GEMM
                            operands bfloat16, accumulation and gates float */

/*
 * Mesh description (Sec. 6.1, Fig. geom; Sec. 5.2 patches).
 * Channel [0, lx] x [0, ly] with nxc x nyc coarse cells (level L), refined K
 * times (level L+K: nxf = nxc 2^K, nyf = nyc 2^K).  A coarse cell is solid iff
 * its centroid lies strictly inside the ellipse (obst_*; obst_ax <= 0 means
 * no obstacle) or, if `solid` is non-null, iff solid[j nxc + i] != 0 (host
 * array, read only during the call).  Fine cells inherit the parent's flag.
 * Velocity Dirichlet nodes: x = 0 (inflow profile u_max 4y(ly-y)/ly^2 w(t),
 * w the start-up ramp of Sec. 6.1 if ramp != 0, else 1), y = 0 and y = ly
 * (walls, 0) and nodes of solid cells (0).  Outflow x = lx is do-nothing.
 * Patches are s x s coarse cells; a patch is fluid if one of its cells is.
 * nu: viscosity (1/Re), k: time step, alpha0: LPS constant
 * (alpha_T = alpha0 h_T^2 / nu, h_T the fine cell diagonal, Sec. 3.1).
 * Constraints: nxc, nyc even and divisible by s; K in 1..3; s in 1..2.
 */
typedef struct dnnmg_mesh_desc {
    int nxc, nyc;
    int K;
    int s;
    double lx, ly;
    double obst_cx, obst_cy, obst_ax, obst_ay;
    const unsigned char *solid;
    double nu, k, alpha0, u_max;
    int ramp;
    int precision;
} dnnmg_mesh_desc;

/*
 * Sizes derived from a description.  nf = (s 2^K + 1)^2 fine and
 * nc = (s+1)^2 coarse nodes per patch; n_in = 3 nf + 3 nc + 12 network inputs
 * (residual, coarse velocity, Peclet number, geometry; Sec. 5.2), n_out = 2 nf
 * outputs.  Feature rows are stored with leading dimension ldx =
 * round_up(n_in, 16); columns n_in..ldx-1 are written as zero.
 * workspace_bytes is what dnnmg_step / dnnmg_step_host need.
 */
typedef struct dnnmg_mesh_info {
    int nxc, nyc, nxf, nyf, K, s;
    int npx, npy;          /* patch grid */
    long long Nc, Nf;      /* coarse / fine nodes */
    int pitch;             /* fine row pitch (elements), round_up(nxf+1, 64) */
    long long plane;       /* elements per fine component plane, pitch (nyf+1) */
    int P;                 /* fluid patches */
    int nf, nc, n_in, n_out, ldx;
    int n_solid_coarse;    /* solid coarse cells */
    int precision;
    int real_bytes;        /* 8 for DNNMG_F64, else 4 */
    int feature_bytes;     /* element size of the feature matrix X */
    size_t workspace_bytes;
} dnnmg_mesh_info;

typedef struct dnnmg_mesh_s *dnnmg_mesh_t;
typedef struct dnnmg_net_s *dnnmg_net_t;

/* Host-only: validate a description and compute its sizes (no GPU needed). */
int dnnmg_mesh_query(const dnnmg_mesh_desc *desc, dnnmg_mesh_info *info);

/* Create a mesh on the current device: uploads the coarse cell mask and the
 * patch numbering (owned by the handle).  Synchronous. */
int dnnmg_mesh_create(const dnnmg_mesh_desc *desc, dnnmg_mesh_t *out);
int dnnmg_mesh_destroy(dnnmg_mesh_t mesh);
int dnnmg_mesh_get_info(dnnmg_mesh_t mesh, dnnmg_mesh_info *info);

/*
 * Index maps, for checking (Sec. 5.2 patches; Sec. 6.1 boundary classes):
 *   patch_cell [P] int: patch-grid index pj npx + pi of fluid patch p;
 *   node_flags [plane] uint8: bit0 velocity Dirichlet, bit1 inflow value,
 *                             bit2 pressure row active (touches a fluid cell);
 *   node_mult  [plane] uint8: number of fluid patches containing the node.
 * Any output may be NULL.  Device pointers; asynchronous.
 */
int dnnmg_mesh_maps(dnnmg_mesh_t mesh, int *patch_cell, unsigned char *node_flags,
                    unsigned char *node_mult, cudaStream_t stream);

/*
 * Patch network (Eq. gru, Sec. 6.2: GRU then a fully connected layer, no
 * biases).  Host arrays, row-major, gate order z, r, h:
 *   Wx [3H][n_in], Uh [3H][H], Wfc [n_out][H].
 * Weights are copied to the device in the network precision (owned by the
 * handle).  Synchronous.
 */
int dnnmg_net_create(int n_in, int hidden, int n_out, const double *Wx, const double *Uh,
                     const double *Wfc, int precision, dnnmg_net_t *out);
int dnnmg_net_destroy(dnnmg_net_t net);

/*
 * Convolutional head of the patch network (Sec. 6.2: the K = 1 net's two
 * convolutional blocks of 36 parameters and its last layer of N_out).  On a
 * prediction row y [n_out] (u on the n x n patch nodes, x fastest, then v;
 * n_out = 2 n^2, n odd, 3 .. 9):
 *   d = w * (B_s y + B_v y),   B = sum_f C_f^T C_f over 4 filters,
 * C_f a zero-padded size-preserving correlation, C_f^T its adjoint (the
 * transposed layer reusing the first layer's weights); B_s over each
 * component's n x n nodes with 3 x 3 filters, B_v over the sequence
 * (u_0, v_0, u_1, v_1, ...) with length-9 filters.  The head has no
 * nonlinearity, so it folds into the output layer: W_eff [n_out][H], column j
 * the head applied to column j of W_fc.
 * theta [72 + n_out]: k_s [4][3][3] (row offset -1..1 in y, column offset
 * -1..1 in x), k_v [4][9] (offset -4..4), w [n_out].
 *
 * dnnmg_head_params: the length of theta for n_out, or 0 if unsupported.
 * dnnmg_net_create_head: dnnmg_net_create with W_eff (folded on the device in
 *   FP64); host arrays, synchronous.  DNNMG_EUNSUPPORTED for other n_out.
 * dnnmg_head_fold: W_eff from theta and W_fc, device FP32, asynchronous.
 * dnnmg_head_backward: the gradients of sum(G * W_eff) with respect to theta
 *   (dtheta [72 + n_out]) and W_fc (dWfc [n_out][H]), written; work is device
 *   scratch of H (72 + n_out) floats.  Device FP32, asynchronous, deterministic
 *   (fixed summation order).
 */
int dnnmg_head_params(int n_out);
int dnnmg_net_create_head(int n_in, int hidden, int n_out, const double *Wx, const double *Uh,
                          const double *Wfc, const double *theta, int precision, dnnmg_net_t *out);
int dnnmg_head_fold(int n_out, int hidden, const float *theta, const float *Wfc, float *Weff,
                    cudaStream_t stream);
int dnnmg_head_backward(int n_out, int hidden, const float *theta, const float *Wfc, const float *G,
                        float *dtheta, float *dWfc, float *work, cudaStream_t stream);

/*
 * S1, the prolongation of Algorithm 2: xf = P xc on (u, v, p) by bilinear interpolation
 * from level L to L+K, then the fine velocity Dirichlet values at time t.
 *   xc [3][Nc] double (in), xf [3][plane] real (out).
 */
int dnnmg_prolongate(dnnmg_mesh_t mesh, const double *xc, void *xf, double t,
                     cudaStream_t stream);

/*
 * S2 + S3, Sec. 5.2 network inputs: the nonlinear residual
 * r = b_f - A(x~) of Eq. nonlinearshort (Q1, 2x2 Gauss, LPS), zero on
 * Dirichlet velocity rows and inactive pressure rows, and the feature matrix
 *   X [P][ldx] (feature type: double / float / bfloat16 by precision), row
 *   = [r_u(nf), r_v(nf), r_p(nf), u(nc), v(nc), Pe(nc), geometry(12), 0...]
 * with patch nodes lexicographic (x fastest), u, v the prolongated velocity
 * at the coarse patch nodes, Pe = q |v| / nu (q the longest patch edge) and
 * geometry = edge lengths (bottom, right, top, left), aspect ratios
 * (bottom/right, top/left, bottom/top, left/right), corner angles
 * (SW, SE, NE, NW).
 * x~ is given either as xf [3][plane] real (the output of dnnmg_prolongate;
 * pass xc = NULL), or as the coarse xc [3][Nc] double with the time t of its
 * Dirichlet values (pass xf = NULL): S1 is then done inside the kernel and x~
 * never goes to memory.  Exactly one of xf, xc must be non-NULL.
 *   bf [2][plane] real (the current fine right-hand side), rf [3][plane]
 *   real (out, may be NULL), X (out).
 */
int dnnmg_patch_features(dnnmg_mesh_t mesh, const void *xf, const double *xc, double t, const void *bf,
                         void *rf, void *X, cudaStream_t stream);

/*
 * S4, Eq. gru and the output layer, for P patches at once:
 *   z = sig(W_z x + U_z h), r = sig(W_r x + U_r h),
 *   h <- z h + (1-z) tanh(W_h x + U_h (r h)),  d = W_fc h.
 *   X [P][ldx] feature type (in), h [P][H] real (in/out; float for
 *   DNNMG_BF16NET), d [P][n_out] real (out).  ldx = round_up(n_in, 16).
 */
int dnnmg_gru_step(dnnmg_net_t net, const void *X, void *h, void *d, int P,
                   cudaStream_t stream);

/*
 * S5, Sec. 5.2 duplicate predictions averaged: vcorr = v~ + mean of the
 * predictions of the fluid patches containing each node, on velocity
 * unknowns; Dirichlet nodes keep v~ (their boundary values).  d row layout
 * [u corr(nf), v corr(nf)].  v~ is given either as xf [3][plane] real (only
 * u, v read; xc = NULL) or interpolated inside the kernel from xc [3][Nc]
 * double with boundary values at time t (xf = NULL); exactly one non-NULL.
 *   d [P][n_out] real, vcorr [2][plane] real (out).
 */
int dnnmg_scatter_avg(dnnmg_mesh_t mesh, const void *d, const void *xf, const double *xc, double t,
                      void *vcorr, cudaStream_t stream);

/*
 * S6 + S7, right-hand side and restriction of Algorithm 2: bf = Rhs(vcorr) of Eq. 4cranknicholson3
 * (1/k (v,phi) - 1/2 (v.grad v,phi) - nu/2 (grad v,grad phi), no forcing),
 * zero on Dirichlet rows; then bc = R bf with R = P^T, coarse Dirichlet
 * velocity rows and all pressure rows zero.
 *   vcorr [2][plane] real (in), bf [2][plane] real (out), bc [3][Nc] double
 *   (out).
 */
int dnnmg_rhs_restrict(dnnmg_mesh_t mesh, const void *vcorr, void *bf, double *bc,
                       cudaStream_t stream);

/*
 * S6 alone, the right-hand side of Algorithm 2: bf = Rhs(vcorr) as in dnnmg_rhs_restrict,
 * without the restriction.
 *   vcorr [2][plane] real (in), bf [2][plane] real (out).
 */
int dnnmg_rhs(dnnmg_mesh_t mesh, const void *vcorr, void *bf, cudaStream_t stream);

/*
 * S5 + S6 fused (Algorithm 2's averaged correction and right-hand side):
 * bf = Rhs(v~ + averaged d) with
 * v~ = P xc at time t formed inside each tile (as dnnmg_scatter_avg with xc
 * followed by dnnmg_rhs, same arithmetic and bits); v_corr never reaches
 * memory.  Each tile copies the d rows of the patches around it to shared
 * memory and averages its one-node halo again.
 *   d [P][n_out] real (in, 8-byte aligned; ignored if P = 0), xc [3][Nc]
 *   double (in), bf [2][plane] real (out).
 */
int dnnmg_scatter_rhs(dnnmg_mesh_t mesh, const void *d, const double *xc, double t, void *bf,
                      cudaStream_t stream);

/*
 * S7 alone, the restriction of Algorithm 2: bc = R bf with R = P^T (the transpose of the
 * bilinear prolongation across the K levels), coarse Dirichlet velocity rows
 * and all pressure rows zero.  Float input is accumulated with error-free
 * float-pair arithmetic (about 2^-44 relative to the sum of magnitudes) and
 * stored in double; double input is accumulated in double.
 *   bf [2][plane] real (in), bc [3][Nc] double (out).
 */
int dnnmg_restrict(dnnmg_mesh_t mesh, const void *bf, double *bc, cudaStream_t stream);

/*
 * S1-S7 in order (the correction step of Algorithm 2) on one stream: S2+S3 and S5 with
 * S1 fused (x~ is formed inside their tiles from xc), then S4, S6, S7.
 *   xc [3][Nc] double (in), h [P][H] (in/out; may be NULL when P = 0, a mesh
 *   without fluid patches, whose step skips S4), bf [2][plane] (in: this step's
 *   fine right-hand side; out: the next step's), bc [3][Nc] double (out),
 *   workspace >= info.workspace_bytes device bytes (scratch, caller-owned,
 *   256-byte aligned), t = t_n for the inflow values.
 */
int dnnmg_step(dnnmg_mesh_t mesh, dnnmg_net_t net, const double *xc, void *h, void *bf,
               double *bc, void *workspace, size_t workspace_bytes, double t,
               cudaStream_t stream);

/*
 * dnnmg_step with the coarse vectors in HOST memory, xc_host and bc_host
 * [3][Nc], all enqueued on `stream`.  If both buffers are page-locked and
 * mapped (cudaHostAlloc / pinned memory under unified addressing), the step's
 * kernels read x_c and write b_c there directly over the CPU-GPU link;
 * otherwise xc_host is copied into the workspace before the step and bc
 * copied back after it.  Both host buffers must stay valid until the stream
 * reaches this point.  h and bf stay device-resident.
 */
int dnnmg_step_host(dnnmg_mesh_t mesh, dnnmg_net_t net, const double *xc_host, void *h,
                    void *bf, double *bc_host, void *workspace, size_t workspace_bytes,
                    double t, cudaStream_t stream);

/*
 * Device status word of a network (synchronous): bit 0 (DNNMG_DEVERR_TIMEOUT)
 * is set if a kernel's bounded wait on its own pipeline ran out of time (the
 * kernel then returns without finishing its tile).  reset != 0 clears it.
 */
#define DNNMG_DEVERR_TIMEOUT 1
int dnnmg_net_status(dnnmg_net_t net, int *status, int reset);

/*
 * The same for a mesh: bit 0 is set if a stencil kernel of the correction
 * step gave up waiting for its tile's TMA copies (the kernel then stops
 * early, leaving its outputs incomplete).  Synchronous; reset != 0 clears it.
 */
int dnnmg_mesh_status(dnnmg_mesh_t mesh, int *status, int reset);

/* 1 if the network's GRU step runs on the tensor cores (BF16 networks whose
 * shapes the tcgen05 kernel supports and DNNMG_GRU_KERNEL != "simt" in the
 * environment at creation), else 0. */
int dnnmg_net_uses_tensor_cores(dnnmg_net_t net);

/*
 * dnnmg_step without a caller-provided workspace.  No counterpart in the
 * paper: this is a deployment variant of dnnmg_step for callers that cannot
 * allocate device memory -- a host whose device memory belongs to another
 * allocator it may not bypass, a loop that must not call the CUDA allocator
 * once running, or a C caller linking only this library.  The step's scratch
 * (features, predictions, corrected velocity) lives in a library-owned
 * static device array of dnnmg_static_scratch_bytes() bytes (64 MiB), which
 * every GPU that loads the library holds until the process exits.  The
 * call allocates nothing.  A mesh needs dnnmg_static_scratch_needed() bytes
 * of it (its workspace without the host-call staging of x_c and b_c, which
 * this call never uses); larger meshes are rejected with DNNMG_EINVAL and a
 * message (use dnnmg_step then).
 * The first call on a device, in a given CUDA context, looks up the array's
 * device address (cudaGetSymbolAddress) and caches it under that device and
 * context; make that first call before any stream capture.  A cached
 * address is checked before each use, so a context created after a
 * cudaDeviceReset (or a second context on the device) gets its own lookup.
 * All calls on a device share the one array and it keeps
 * the last call's contents: calls that can overlap on the GPU (different
 * streams, different host threads) race on it and must be serialised by
 * the caller.  Nothing in it needs clearing between calls.  Arguments and
 * results are those of dnnmg_step.
 */
int dnnmg_step_static(dnnmg_mesh_t mesh, dnnmg_net_t net, const double *xc, void *h, void *bf,
                      double *bc, double t, cudaStream_t stream);

/* Size in bytes of the static scratch used by dnnmg_step_static. */
size_t dnnmg_static_scratch_bytes(void);

/* Bytes of the static scratch that dnnmg_step_static needs for this mesh
 * (0 for a NULL mesh).  No counterpart in the paper. */
size_t dnnmg_static_scratch_needed(dnnmg_mesh_t mesh);

/*
 * Byte offsets, inside a dnnmg_step workspace, of the arrays the step leaves
 * there (valid once the stream has reached the end of the step): *x the
 * features X [P][ldx] (S3), *d the network output [P][n_out] (S4), *vcorr
 * the corrected fine velocity v~ + d_bar [2][plane] (S5), each in the mesh's
 * real type (X in the feature type).  No counterpart in the paper: it lets a
 * caller inspect the step's correction, as the parity tests do.  Host-only,
 * synchronous; DNNMG_EINVAL on NULL arguments.
 */
int dnnmg_workspace_offsets(dnnmg_mesh_t mesh, long long *x, long long *d, long long *vcorr);

/* Number of kernel launches one dnnmg_step enqueues for this mesh/net. */
int dnnmg_step_launches(dnnmg_mesh_t mesh, dnnmg_net_t net);

/*
 * dnnmg_step that also records events[0] before its first kernel and
 * events[i+1] after kernel i, so the caller can time every kernel of the
 * step (cudaEventElapsedTime).  No counterpart in the paper: an
 * instrumentation form of dnnmg_step.
 *   events: n_events = dnnmg_step_launches() + 1 caller-created events.
 * The kernels, in order: coarse padding (S1 staging), S2+S3 on the
 * all-fluid tiles in closed form (FP32 fields with K = 1 or 2 only), S2+S3
 * on the other tiles, S4 (when the mesh has fluid patches), S5, S6, S7.
 */
int dnnmg_step_timed(dnnmg_mesh_t mesh, dnnmg_net_t net, const double *xc, void *h, void *bf, double *bc,
                     void *workspace, size_t workspace_bytes, double t, cudaEvent_t *events, int n_events,
                     cudaStream_t stream);

/*
 * ---- Serving: batched steps of many instances ------------------------------
 *
 * A server runs the correction step of Algorithm 2 for several flow instances at once
 * (meshes of any size, each with its own GRU state h, all using one net): the
 * stencil passes run per instance, the network (Eq. gru and the output
 * layer, Sec. 6.2) runs once over the patches of every instance in the batch
 * as one tensor-core launch.  The paper runs one instance; batching is this
 * library's, and an instance's results have the same bits alone (dnnmg_step
 * with the same inputs and state) and in any batch.
 *
 * The server owns, on the device: a state pool of max_rows patch rows (FP32,
 * net H columns), a feature matrix and an output matrix of max_rows rows, and
 * scratch for the largest admitted mesh.  dnnmg_server_bytes() gives the pool
 * and matrix bytes for a budget check.  Instances take segments of the pool in
 * whole 128-row tiles.  A server is used from one host thread at a time.
 *
 * Requires a DNNMG_BF16NET net with the tensor-core kernel (H a multiple of
 * 32, at most 128); otherwise DNNMG_EUNSUPPORTED.
 */
typedef struct dnnmg_server_s *dnnmg_server_t;

/* Device bytes of a server's pool and matrices for max_rows patch rows (0 on a NULL net). */
size_t dnnmg_server_bytes(dnnmg_net_t net, int max_rows);
/* Create a server for `net` holding up to max_rows patch rows in total (rounded up to 128). */
int dnnmg_server_create(dnnmg_net_t net, int max_rows, dnnmg_server_t *out);
/* Wait for the device, then free everything the server owns (NULL is allowed). */
int dnnmg_server_destroy(dnnmg_server_t server);
/*
 * Admit an instance on `mesh` (DNNMG_BF16NET, n_in / n_out equal to the net's;
 * the caller keeps the mesh alive until release).  Its state segment, of its
 * fluid patch count rounded up to 128 rows, starts at h = 0 (Sec. 6.2).
 * DNNMG_ENOMEM when no free segment is large enough (the pool is the budget).
 * May synchronise the device (scratch growth).  *slot: the instance's id.
 */
int dnnmg_server_admit(dnnmg_server_t server, dnnmg_mesh_t mesh, int *slot);
/* Synchronise the device, then free the instance's segment; its slot id may be reused. */
int dnnmg_server_release(dnnmg_server_t server, int slot);
/* Device pointer to the instance's state rows, [P][H] FP32 (valid until release). */
int dnnmg_server_state(dnnmg_server_t server, int slot, float **h);
/*
 * One step of each of the n distinct instances slots[0..n-1], asynchronous on
 * `stream`.  Host arrays of device pointers, one entry per instance, with the
 * meaning of dnnmg_step: xc[i] [3][Nc] FP64 coarse solution, bf[i] the
 * instance's b_f (read, then overwritten; 16-byte aligned), bc[i] [3][Nc]
 * FP64 out, t[i] the instance's time t_n.  The state lives in the server.
 * The per-instance passes run on the server's 8 side streams (round robin),
 * forked from `stream` and joined back into it before and after S4, so the
 * call is ordered on `stream` like a single kernel sequence (and can be
 * captured into a graph from it).  Calls on one server must be issued on one
 * stream (or ordered by the caller).
 */
int dnnmg_server_step(dnnmg_server_t server, int n, const int *slots, const double *const *xc, void *const *bf,
                      double *const *bc, const double *t, cudaStream_t stream);

/*
 * Host-only row-range allocator the server uses for its state pool: first fit
 * over ranges of whole units of `unit` rows, frees coalesce with their free
 * neighbours.  No GPU needed.  alloc: DNNMG_ENOMEM when no free range holds
 * the rounded request; free: DNNMG_EINVAL if no allocated range starts there.
 */
typedef struct dnnmg_pool_s *dnnmg_pool_t;
int dnnmg_pool_create(int capacity_rows, int unit, dnnmg_pool_t *out);
int dnnmg_pool_alloc(dnnmg_pool_t pool, int rows, int *start);
int dnnmg_pool_free(dnnmg_pool_t pool, int start);
int dnnmg_pool_stats(dnnmg_pool_t pool, int *used_rows, int *largest_free);
void dnnmg_pool_destroy(dnnmg_pool_t pool);

/*
 * ---- Training the patch network (GRU + output layer) -----------------------
 *
 * Forward and backward of Eq. gru followed by the output layer (Sec. 6.2),
 * unrolled over a window of T steps of P patch rows, for truncated
 * backpropagation through time; the l2 loss of Sec. 6.3 and its gradient;
 * Adam with the Tikhonov term of Sec. 6.3.  FP32 products on the CUDA cores,
 * or BF16 products on the tensor cores (dnnmg_trainer_set_precision);
 * weight-gradient sums are split over the T P rows in a fixed order, so
 * results repeat bit for bit.  All arrays are caller-owned device memory:
 *   X [T][P][ldx] (columns n_in..ldx-1 ignored), h0 / dh0 [P][H],
 *   Wx / gWx [3H][n_in], Uh / gUh [3H][H] (gates z, r, h), Wfc / gWfc [n_out][H],
 *   D / dD [T][P][n_out].
 * A trainer owns the activations of one window (about T P (12 H) floats) and
 * serves one forward/backward pair at a time.
 */
typedef struct dnnmg_trainer_s *dnnmg_trainer_t;
int dnnmg_trainer_create(int n_in, int ldx, int H, int n_out, int T, int P, dnnmg_trainer_t *out);
/* Wait for the device, then free the trainer (NULL is allowed). */
int dnnmg_trainer_destroy(dnnmg_trainer_t trainer);
/*
 * Arithmetic of the trainer's matrix products (the pointwise steps, the
 * reductions and every array stay FP32; the training workload of Sec. 6.3
 * asks for BF16 products with FP32 master weights):
 *   DNNMG_F32      FP32 products on the CUDA cores (the default);
 *   DNNMG_BF16NET  BF16 operands, FP32 accumulation, on the tensor cores
 *                  (tcgen05): each product's operands are rounded to BF16
 *                  once per tensor (transposed where the product needs it)
 *                  into scratch the trainer allocates here (about
 *                  T P (2 n_in + 6 H + 2 n_out) BF16 values).
 * DNNMG_EINVAL for another value, DNNMG_ENOMEM if the scratch cannot be had.
 */
int dnnmg_trainer_set_precision(dnnmg_trainer_t trainer, int precision);
/*
 * Device status bits of the trainer's tensor-core products (DNNMG_DEVERR_*,
 * e.g. a bounded wait that timed out); reset clears them.  Synchronous.
 */
int dnnmg_trainer_status(dnnmg_trainer_t trainer, int *status, int reset);
/*
 * C[M][N] (row stride ldc, FP32) = A[M][K] B[N][K]^T, or C += A B^T when
 * accumulate is nonzero, on the tensor cores (tcgen05, FP32 accumulation);
 * the training products' kernel, exported for testing.  A and B: BF16 device
 * arrays, K contiguous, row strides lda, ldb elements (multiples of 8, at
 * least K; 16-byte aligned).  *status (device int) receives DNNMG_DEVERR_*
 * bits.  Asynchronous on stream.
 */
int dnnmg_gemm_bf16_nt(int M, int N, int K, const void *A, int lda, const void *B, int ldb, float *C, int ldc,
                       int accumulate, int *status, cudaStream_t stream);
/* D = outputs of the T steps from state h0 (NULL: h0 = 0); keeps the activations for the backward. */
int dnnmg_gru_seq_forward(dnnmg_trainer_t trainer, const float *X, const float *h0, const float *Wx, const float *Uh,
                          const float *Wfc, float *D, cudaStream_t stream);
/* Device pointer to h_T of the last forward (the next window's h0), [P][H]. */
int dnnmg_gru_seq_state(dnnmg_trainer_t trainer, float **hT);
/*
 * Gradients of sum(dD * D) over the last forward's window with respect to the
 * weights (written, not accumulated) and, if dh0 is not NULL, to h0.  X, Uh
 * and Wfc must be the arrays of that forward.
 */
int dnnmg_gru_seq_backward(dnnmg_trainer_t trainer, const float *dD, const float *X, const float *Uh, const float *Wfc,
                           float *gWx, float *gUh, float *gWfc, float *dh0, cudaStream_t stream);
/*
 * Loss of Sec. 6.3 over n = T P n_out outputs: *loss (device double) =
 * sum (D - Y)^2 / P, and dD = 2 (D - Y) / P if dD is not NULL.
 */
int dnnmg_l2_loss(const float *D, const float *Y, long long n, int P, float *dD, double *loss, cudaStream_t stream);
/* *out (device double) = sum of x^2 (the Tikhonov term divided by alpha). */
int dnnmg_sumsq(const float *x, long long n, double *out, cudaStream_t stream);
/*
 * One Adam update (step >= 1) of n parameters p with gradient g + 2 alpha p
 * (alpha: Tikhonov factor) and moments m, v (start at 0).
 */
int dnnmg_adam_step(float *p, const float *g, float *m, float *v, long long n, int step, float lr, float beta1,
                    float beta2, float eps, float alpha, cudaStream_t stream);

/*
 * Self-test of the bounded waits (synchronous; no counterpart in the paper).
 * One block of 64 threads waits on an mbarrier phase that nothing completes:
 * thread 0 gives up after limit_ns (1 ns .. 1 s), sets DNNMG_DEVERR_TIMEOUT
 * in a device status word and the CTA's abort flag; the other threads (limit
 * 2 s) must leave through the flag.  *status: the status word read back;
 * waited_ns[0]: thread 0's wait, waited_ns[1]: the last thread's.  Nothing
 * is left in flight, so the context stays usable.
 */
int dnnmg_selftest_wait_timeout(long long limit_ns, int *status, long long *waited_ns);

/*
 * ---- Plain multigrid fine solve (the method DNN-MG is compared with) --------
 *
 * Sec. 3.3 solves each time step's system (Eq. nonlinearshort) by Newton's
 * method, each Newton system by GMRES with a geometric multigrid
 * preconditioner (Sec. 3.4, Algorithm 1) smoothed by the Vanka method; Sec.
 * 6.4 times DNN-MG against it.  These calls are the GPU pieces of that
 * solver on a hierarchy of uniform levels; the iterations are driven from the
 * host (paper_2008_11520_gb300/mg.py).  Level 0 is the finest (nx x ny
 * cells); level l has nx / 2^l x ny / 2^l cells.  Node fields are [3][N]
 * (u, v, p), N = (nx_l + 1)(ny_l + 1), x fastest, without padding, in the
 * handle's precision (double for DNNMG_F64, float for DNNMG_F32), in device
 * memory owned by the caller.  The discretisation is the correction step's
 * (Q1/Q1, Crank-Nicolson, local projection stabilisation, 2 x 2 Gauss).
 * Any finest mask is accepted (a partly solid projection patch contributes
 * the integrals of its fluid cells); a coarser level's patch is solid iff all
 * 16 cells under it on the finer level are, and every level uses the finest
 * level's projection coefficient (alpha0 scaled by 4^-level).  All calls
 * except create/destroy/level are asynchronous on `stream`.
 */
typedef struct dnnmg_mg_desc {
    int nx, ny;                 /* cells of the finest level, multiples of 2^levels */
    int levels;                 /* 1 .. 12 */
    double lx, ly;              /* channel size */
    const unsigned char *solid; /* [ny][nx] cell mask of the finest level (host, may be NULL) */
    double nu, k, alpha0, u_max;
    int ramp;                   /* start-up ramp of the inflow (Sec. 6.1) */
    int precision;              /* DNNMG_F64 or DNNMG_F32 */
} dnnmg_mg_desc;
typedef struct dnnmg_mg_s *dnnmg_mg_t;

int dnnmg_mg_create(const dnnmg_mg_desc *desc, dnnmg_mg_t *out);
int dnnmg_mg_destroy(dnnmg_mg_t mg);
/* Cells of a level and (when solid is not NULL) its cell mask [ny][nx] (host). */
int dnnmg_mg_level(dnnmg_mg_t mg, int level, int *nx, int *ny, unsigned char *solid);
/* Newton defect F(x) (Sec. 3.3): A(x) - b on free rows, x - g(t) on velocity
 * Dirichlet rows (g: parabolic inflow at t, else 0) and p on inactive pressure
 * rows.  b: [3][N] (pressure rows normally 0). */
int dnnmg_mg_defect(dnnmg_mg_t mg, int level, const void *x, const void *b, double t, void *F, cudaStream_t stream);
/* Right-hand side b = Rhs(x) of Eq. 4cranknicholson3 (f = 0) from the
 * velocity of x: [3][N], Dirichlet and pressure rows 0; x, b must not alias. */
int dnnmg_mg_rhs(dnnmg_mg_t mg, int level, const void *x, void *b, cudaStream_t stream);
/* y = J(x) dx, J the Newton matrix of the defect (fixed rows: identity). */
int dnnmg_mg_jvp(dnnmg_mg_t mg, int level, const void *x, const void *dx, void *y, cudaStream_t stream);
/* One Vanka sweep (Sec. 3.4) for J(x) d = r, d = dx updated in place: for
 * each of 16 cell colours (ci mod 4, cj mod 4) in turn, every fluid cell of
 * the colour solves the 12 x 12 block of J(x) on the unknowns of its 4 nodes
 * against the current defect r - J(x) d there (rows of fixed unknowns:
 * identity) and adds omega times the solution to d (block Gauss-Seidel; cells of one
 * colour are independent, so the sweep is deterministic); then every fixed
 * unknown takes d = r (its exact correction; this reaches nodes inside an
 * obstacle that no cell block holds).  dx must not alias x or r. */
int dnnmg_mg_vanka(dnnmg_mg_t mg, int level, const void *x, const void *r, void *dx, double omega,
                   cudaStream_t stream);
/* rc = P^T rf from level to level + 1 (fixed rows of level + 1 zeroed). */
int dnnmg_mg_restrict(dnnmg_mg_t mg, int level, const void *rf, void *rc, cudaStream_t stream);
/* df += P dc from level + 1 to level (fixed rows of level unchanged). */
int dnnmg_mg_prolong_add(dnnmg_mg_t mg, int level, const void *dc, void *df, cudaStream_t stream);
/* xc = xf at the nodes of level + 1 (linearisation point of the coarser level). */
int dnnmg_mg_inject(dnnmg_mg_t mg, int level, const void *xf, void *xc, cudaStream_t stream);
/* *out (device double) = sum a_i b_i over n elements (FP64 accumulation). */
int dnnmg_mg_dot(dnnmg_mg_t mg, long long n, const void *a, const void *b, double *out, cudaStream_t stream);
/* y = alpha x + beta y over n elements (beta = 0: y = alpha x). */
int dnnmg_mg_axpby(dnnmg_mg_t mg, long long n, double alpha, const void *x, double beta, void *y,
                   cudaStream_t stream);

/* Last error message of the calling thread ("" if none). */
const char *dnnmg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DNNMG_H */

// Convolutional head of the patch network (Sec. 6.2: the K = 1 net's two
// convolutional blocks of 36 parameters and its last layer of N_out) and its
// fold into the output layer.
//
// The head acts on one prediction row y [N_out] (u on the n x n patch nodes,
// x fastest, then v):
//
//     d = w * (B_s y + B_v y),   B = sum_f C_f^T C_f   (4 filters per block),
//
// C_f a zero-padded, size-preserving correlation and C_f^T its adjoint (the
// transposed layer, with the first layer's weights).  B_s correlates each
// component's n x n nodes with 3 x 3 filters, B_v the vertex-by-vertex
// sequence (u_0, v_0, u_1, v_1, ...) with length-9 filters.  The head has no
// nonlinearity, so d = W_eff h' with column j of W_eff the head applied to
// column j of W_fc: the step runs the folded output layer and pays nothing
// for the head.  Training keeps theta and W_fc and maps the gradient of W_eff
// back (dnnmg_head_backward).
//
// theta [72 + N_out]: k_s [4][3][3] (row offset -1..1 in y, column offset
// -1..1 in x), k_v [4][9] (offset -4..4), w [N_out].  One thread per column of
// W_fc; the columns are few (the GRU width), so these kernels are tiny.
#include "common.cuh"

namespace dnnmg {
namespace {

constexpr int HF = 4, HKS = 3, HKV = 9, HMAXN = 9, HMAXOUT = 2 * HMAXN * HMAXN;
constexpr int HCONV = HF * (HKS * HKS + HKV);   // filter weights of both blocks (72)

// c = C y over an n x n grid
template <typename T> __device__ void corr2d(const T *g, const T *k, int n, T *c) {
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            T a = T(0);
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx)
                    if (j + dy >= 0 && j + dy < n && i + dx >= 0 && i + dx < n)
                        a += k[(dy + 1) * HKS + dx + 1] * g[(j + dy) * n + i + dx];
            c[j * n + i] = a;
        }
}

// y += C^T c over an n x n grid
template <typename T> __device__ void corr2d_t_add(const T *c, const T *k, int n, T *y) {
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx)
                    if (j + dy >= 0 && j + dy < n && i + dx >= 0 && i + dx < n)
                        y[(j + dy) * n + i + dx] += k[(dy + 1) * HKS + dx + 1] * c[j * n + i];
}

template <typename T> __device__ void corr1d(const T *s, const T *k, int m, T *c) {
    for (int p = 0; p < m; ++p) {
        T a = T(0);
        for (int t = -HKV / 2; t <= HKV / 2; ++t)
            if (p + t >= 0 && p + t < m) a += k[t + HKV / 2] * s[p + t];
        c[p] = a;
    }
}

template <typename T> __device__ void corr1d_t_add(const T *c, const T *k, int m, T *s) {
    for (int p = 0; p < m; ++p)
        for (int t = -HKV / 2; t <= HKV / 2; ++t)
            if (p + t >= 0 && p + t < m) s[p + t] += k[t + HKV / 2] * c[p];
}

// out = B_s x + B_v x (no weighting); c, s, acc are scratch of N_out entries
template <typename T>
__device__ void head_blocks(const T *theta, int n, const T *x, T *out, T *c, T *s, T *acc) {
    const int nf = n * n, m = 2 * nf;
    const T *ks = theta, *kv = theta + HF * HKS * HKS;
    for (int e = 0; e < m; ++e) out[e] = T(0);
    for (int comp = 0; comp < 2; ++comp)
        for (int f = 0; f < HF; ++f) {
            corr2d(x + comp * nf, ks + f * HKS * HKS, n, c);
            corr2d_t_add(c, ks + f * HKS * HKS, n, out + comp * nf);
        }
    for (int v = 0; v < nf; ++v) {
        s[2 * v] = x[v];
        s[2 * v + 1] = x[nf + v];
    }
    for (int e = 0; e < m; ++e) acc[e] = T(0);
    for (int f = 0; f < HF; ++f) {
        corr1d(s, kv + f * HKV, m, c);
        corr1d_t_add(c, kv + f * HKV, m, acc);
    }
    for (int v = 0; v < nf; ++v) {
        out[v] += acc[2 * v];
        out[nf + v] += acc[2 * v + 1];
    }
}

// W_eff[:, j] = w * (B_s + B_v) W_fc[:, j]; W_fc, W_eff [N_out][H]
template <typename T>
__global__ void k_head_fold(int n, int H, const T *__restrict__ theta, const T *__restrict__ Wfc, T *__restrict__ Weff) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= H) return;
    const int m = 2 * n * n;
    const T *w = theta + HCONV;
    T x[HMAXOUT], out[HMAXOUT], c[HMAXOUT], s[HMAXOUT], acc[HMAXOUT];
    for (int e = 0; e < m; ++e) x[e] = Wfc[(size_t)e * H + j];
    head_blocks(theta, n, x, out, c, s, acc);
    for (int e = 0; e < m; ++e) Weff[(size_t)e * H + j] = w[e] * out[e];
}

// Gradient of sum(G * W_eff) for column j: dW_fc[:, j] = (B_s + B_v)(w * g)
// (both blocks are symmetric) and this column's share of d theta in
// work[j][72 + N_out]: with q = w * g and x = W_fc[:, j],
//   d k_f[t] = sum_p (C_f q)[p] x[p + t] + (C_f x)[p] q[p + t],   d w = g * (B_s + B_v) x.
template <typename T>
__global__ void k_head_grad_cols(int n, int H, const T *__restrict__ theta, const T *__restrict__ Wfc,
                                 const T *__restrict__ G, T *__restrict__ dWfc, T *__restrict__ work) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= H) return;
    const int nf = n * n, m = 2 * nf, nt = HCONV + m;
    const T *ks = theta, *kv = theta + HF * HKS * HKS, *w = theta + HCONV;
    T x[HMAXOUT], q[HMAXOUT], out[HMAXOUT], c[HMAXOUT], s[HMAXOUT], acc[HMAXOUT];
    T *part = work + (size_t)j * nt;
    for (int e = 0; e < m; ++e) {
        x[e] = Wfc[(size_t)e * H + j];
        q[e] = w[e] * G[(size_t)e * H + j];
    }
    head_blocks(theta, n, q, out, c, s, acc);
    for (int e = 0; e < m; ++e) dWfc[(size_t)e * H + j] = out[e];
    head_blocks(theta, n, x, out, c, s, acc);
    for (int e = 0; e < m; ++e) part[HCONV + e] = G[(size_t)e * H + j] * out[e];
    // spatial filters: both components; c holds C_f q, acc holds C_f x
    for (int f = 0; f < HF; ++f) {
        T dk[HKS * HKS];
        for (int t = 0; t < HKS * HKS; ++t) dk[t] = T(0);
        for (int comp = 0; comp < 2; ++comp) {
            const T *xs = x + comp * nf, *qs = q + comp * nf;
            corr2d(qs, ks + f * HKS * HKS, n, c);
            corr2d(xs, ks + f * HKS * HKS, n, acc);
            for (int jj = 0; jj < n; ++jj)
                for (int ii = 0; ii < n; ++ii)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx)
                            if (jj + dy >= 0 && jj + dy < n && ii + dx >= 0 && ii + dx < n) {
                                const int o = (jj + dy) * n + ii + dx;
                                dk[(dy + 1) * HKS + dx + 1] += c[jj * n + ii] * xs[o] + acc[jj * n + ii] * qs[o];
                            }
        }
        for (int t = 0; t < HKS * HKS; ++t) part[f * HKS * HKS + t] = dk[t];
    }
    // vertex filters on the interleaved sequences (x into s, q into out)
    for (int v = 0; v < nf; ++v) {
        s[2 * v] = x[v];
        s[2 * v + 1] = x[nf + v];
        out[2 * v] = q[v];
        out[2 * v + 1] = q[nf + v];
    }
    for (int f = 0; f < HF; ++f) {
        T dk[HKV];
        for (int t = 0; t < HKV; ++t) dk[t] = T(0);
        corr1d(out, kv + f * HKV, m, c);
        corr1d(s, kv + f * HKV, m, acc);
        for (int p = 0; p < m; ++p)
            for (int t = -HKV / 2; t <= HKV / 2; ++t)
                if (p + t >= 0 && p + t < m) dk[t + HKV / 2] += c[p] * s[p + t] + acc[p] * out[p + t];
        for (int t = 0; t < HKV; ++t) part[HF * HKS * HKS + f * HKV + t] = dk[t];
    }
}

// d theta[e] = sum over the columns, in column order (deterministic)
template <typename T>
__global__ void k_head_grad_sum(int nt, int H, const T *__restrict__ work, T *__restrict__ dtheta) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nt) return;
    T a = T(0);
    for (int j = 0; j < H; ++j) a += work[(size_t)j * nt + e];
    dtheta[e] = a;
}

// patch side n from N_out = 2 n^2 (n odd, 3 .. 9), or 0
int head_side(int n_out) {
    for (int n = 3; n <= HMAXN; n += 2)
        if (2 * n * n == n_out) return n;
    return 0;
}

}  // namespace
}  // namespace dnnmg

using namespace dnnmg;

extern "C" {

int dnnmg_head_params(int n_out) { return head_side(n_out) ? HCONV + n_out : 0; }

int dnnmg_head_fold(int n_out, int hidden, const float *theta, const float *Wfc, float *Weff, cudaStream_t st) {
    clear_error();
    const int n = head_side(n_out);
    if (!n) return fail(DNNMG_EUNSUPPORTED, "head: N_out = %d is not 2 n^2 with n odd, 3..9", n_out);
    if (hidden < 1 || !theta || !Wfc || !Weff) return fail(DNNMG_EINVAL, "head: bad argument");
    k_head_fold<float><<<(hidden + 63) / 64, 64, 0, st>>>(n, hidden, theta, Wfc, Weff);
    DNNMG_LAUNCH_CHECK("k_head_fold");
    return DNNMG_OK;
}

int dnnmg_head_backward(int n_out, int hidden, const float *theta, const float *Wfc, const float *G, float *dtheta,
                        float *dWfc, float *work, cudaStream_t st) {
    clear_error();
    const int n = head_side(n_out);
    if (!n) return fail(DNNMG_EUNSUPPORTED, "head: N_out = %d is not 2 n^2 with n odd, 3..9", n_out);
    if (hidden < 1 || !theta || !Wfc || !G || !dtheta || !dWfc || !work)
        return fail(DNNMG_EINVAL, "head: bad argument");
    const int nt = HCONV + n_out;
    k_head_grad_cols<float><<<(hidden + 63) / 64, 64, 0, st>>>(n, hidden, theta, Wfc, G, dWfc, work);
    DNNMG_LAUNCH_CHECK("k_head_grad_cols");
    k_head_grad_sum<float><<<(nt + 127) / 128, 128, 0, st>>>(nt, hidden, work, dtheta);
    DNNMG_LAUNCH_CHECK("k_head_grad_sum");
    return DNNMG_OK;
}

int dnnmg_net_create_head(int n_in, int hidden, int n_out, const double *Wx, const double *Uh, const double *Wfc,
                          const double *theta, int precision, dnnmg_net_t *out) {
    clear_error();
    const int n = head_side(n_out);
    if (!n) return fail(DNNMG_EUNSUPPORTED, "head: N_out = %d is not 2 n^2 with n odd, 3..9", n_out);
    if (hidden < 1 || !Wfc || !theta || !out) return fail(DNNMG_EINVAL, "head: bad argument");
    const int nt = HCONV + n_out;
    const size_t nw = (size_t)n_out * hidden;
    double *d = nullptr;
    DNNMG_CUDA_TRY(cudaMalloc(&d, sizeof(double) * (nt + 2 * nw)));
    std::vector<double> weff(nw);
    cudaError_t e = cudaMemcpy(d, theta, sizeof(double) * nt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + nt, Wfc, sizeof(double) * nw, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_head_fold<double><<<(hidden + 63) / 64, 64>>>(n, hidden, d, d + nt, d + nt + nw);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(weff.data(), d + nt + nw, sizeof(double) * nw, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(DNNMG_ECUDA, "head fold failed: %s", cudaGetErrorString(e));
    return dnnmg_net_create(n_in, hidden, n_out, Wx, Uh, weff.data(), precision, out);
}

}  // extern "C"

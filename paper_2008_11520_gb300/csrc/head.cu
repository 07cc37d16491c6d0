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
// -1..1 in x), k_v [4][9] (offset -4..4), w [N_out].
#include "common.cuh"

namespace dnnmg {
namespace {

constexpr int HF = 4, HKS = 3, HKV = 9, HMAXN = 9, HMAXOUT = 2 * HMAXN * HMAXN;
constexpr int HCONV = HF * (HKS * HKS + HKV);   // filter weights of both blocks (72)
constexpr int HTH = 128;                        // threads per column block

// One block per column j of W_fc, one thread per entry: the rows of a column
// are few (N_out <= 162), and the filters' work per column is a few thousand
// products, so the column's vectors and their correlations stay in shared
// memory.  Entry e = comp nf + jj n + ii (node (ii, jj) of component comp);
// position p = 2 node + comp in the vertex-by-vertex sequence.
struct HeadIdx {
    int n, nf, m;
    __device__ HeadIdx(int n_) : n(n_), nf(n_ * n_), m(2 * n_ * n_) {}
    // the entry of sequence position p
    __device__ int seq(int p) const { return (p & 1) * nf + (p >> 1); }
    // the sequence position of entry e
    __device__ int pos(int e) const { return 2 * (e % nf) + e / nf; }
};

// c = C_f y for the 4 spatial filters (per component, zero outside the n x n
// grid) and the 4 vertex filters (on the sequence), for every entry / position
template <typename T>
__device__ void head_corr(const HeadIdx &ix, const T *ks, const T *kv, const T *y, T *cs, T *cv) {
    for (int it = threadIdx.x; it < HF * ix.m; it += blockDim.x) {
        const int f = it / ix.m, e = it - f * ix.m;
        const int comp = e / ix.nf, node = e - comp * ix.nf, jj = node / ix.n, ii = node - jj * ix.n;
        const T *k = ks + f * HKS * HKS;
        T a = T(0);
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx)
                if (jj + dy >= 0 && jj + dy < ix.n && ii + dx >= 0 && ii + dx < ix.n)
                    a += k[(dy + 1) * HKS + dx + 1] * y[comp * ix.nf + (jj + dy) * ix.n + ii + dx];
        cs[f * ix.m + e] = a;
        // the same item as sequence position p = e of vertex filter f
        const T *kf = kv + f * HKV;
        T b = T(0);
        for (int t = -HKV / 2; t <= HKV / 2; ++t)
            if (e + t >= 0 && e + t < ix.m) b += kf[t + HKV / 2] * y[ix.seq(e + t)];
        cv[f * ix.m + e] = b;
    }
}

// (B_s y + B_v y)[e] from the correlations of y: the adjoints C_f^T summed
// over the filters of both blocks
template <typename T>
__device__ T head_adjoint(const HeadIdx &ix, const T *ks, const T *kv, const T *cs, const T *cv, int e) {
    const int comp = e / ix.nf, node = e - comp * ix.nf, jj = node / ix.n, ii = node - jj * ix.n;
    T a = T(0);
    for (int f = 0; f < HF; ++f) {
        const T *k = ks + f * HKS * HKS;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx)
                if (jj - dy >= 0 && jj - dy < ix.n && ii - dx >= 0 && ii - dx < ix.n)
                    a += k[(dy + 1) * HKS + dx + 1] * cs[f * ix.m + comp * ix.nf + (jj - dy) * ix.n + ii - dx];
    }
    const int p = ix.pos(e);
    T b = T(0);
    for (int f = 0; f < HF; ++f) {
        const T *kf = kv + f * HKV;
        for (int t = -HKV / 2; t <= HKV / 2; ++t)
            if (p - t >= 0 && p - t < ix.m) b += kf[t + HKV / 2] * cv[f * ix.m + p - t];
    }
    return a + b;
}

// W_eff[:, j] = w * (B_s + B_v) W_fc[:, j]; W_fc, W_eff [N_out][H]; block j
template <typename T>
__global__ void __launch_bounds__(HTH)
k_head_fold(int n, int H, const T *__restrict__ theta, const T *__restrict__ Wfc, T *__restrict__ Weff) {
    __shared__ T x[HMAXOUT], cs[HF * HMAXOUT], cv[HF * HMAXOUT];
    const HeadIdx ix(n);
    const int j = blockIdx.x;
    const T *ks = theta, *kv = theta + HF * HKS * HKS, *w = theta + HCONV;
    for (int e = threadIdx.x; e < ix.m; e += blockDim.x) x[e] = Wfc[(size_t)e * H + j];
    __syncthreads();
    head_corr(ix, ks, kv, x, cs, cv);
    __syncthreads();
    for (int e = threadIdx.x; e < ix.m; e += blockDim.x)
        Weff[(size_t)e * H + j] = w[e] * head_adjoint(ix, ks, kv, cs, cv, e);
}

// Gradient of sum(G * W_eff) for column j (block j): dW_fc[:, j] = (B_s + B_v)(w * g)
// (both blocks are symmetric) and this column's share of d theta in
// work[j][72 + N_out]: with q = w * g and x = W_fc[:, j],
//   d k_f[t] = sum_p (C_f q)[p] x[p + t] + (C_f x)[p] q[p + t],   d w = g * (B_s + B_v) x.
template <typename T>
__global__ void __launch_bounds__(HTH)
k_head_grad_cols(int n, int H, const T *__restrict__ theta, const T *__restrict__ Wfc, const T *__restrict__ G,
                 T *__restrict__ dWfc, T *__restrict__ work) {
    __shared__ T x[HMAXOUT], g[HMAXOUT], q[HMAXOUT];
    __shared__ T csx[HF * HMAXOUT], cvx[HF * HMAXOUT], csq[HF * HMAXOUT], cvq[HF * HMAXOUT];
    const HeadIdx ix(n);
    const int j = blockIdx.x, nt = HCONV + ix.m;
    const T *ks = theta, *kv = theta + HF * HKS * HKS, *w = theta + HCONV;
    T *part = work + (size_t)j * nt;
    for (int e = threadIdx.x; e < ix.m; e += blockDim.x) {
        x[e] = Wfc[(size_t)e * H + j];
        g[e] = G[(size_t)e * H + j];
        q[e] = w[e] * g[e];
    }
    __syncthreads();
    head_corr(ix, ks, kv, x, csx, cvx);
    head_corr(ix, ks, kv, q, csq, cvq);
    __syncthreads();
    for (int it = threadIdx.x; it < ix.m + HCONV; it += blockDim.x) {
        if (it < ix.m) {
            dWfc[(size_t)it * H + j] = head_adjoint(ix, ks, kv, csq, cvq, it);
            part[HCONV + it] = g[it] * head_adjoint(ix, ks, kv, csx, cvx, it);
        } else if (it < ix.m + HF * HKS * HKS) {
            // spatial filter f, tap (dy, dx): both components
            const int r = it - ix.m, f = r / (HKS * HKS), tap = r - f * HKS * HKS;
            const int dy = tap / HKS - 1, dx = tap % HKS - 1;
            T a = T(0);
            for (int e = 0; e < ix.m; ++e) {
                const int comp = e / ix.nf, node = e - comp * ix.nf, jj = node / ix.n, ii = node - jj * ix.n;
                if (jj + dy >= 0 && jj + dy < ix.n && ii + dx >= 0 && ii + dx < ix.n) {
                    const int o = comp * ix.nf + (jj + dy) * ix.n + ii + dx;
                    a += csq[f * ix.m + e] * x[o] + csx[f * ix.m + e] * q[o];
                }
            }
            part[r] = a;
        } else {
            // vertex filter f, offset t, on the sequences of x and q
            const int r = it - ix.m - HF * HKS * HKS, f = r / HKV, t = r - f * HKV - HKV / 2;
            T a = T(0);
            for (int p = 0; p < ix.m; ++p)
                if (p + t >= 0 && p + t < ix.m)
                    a += cvq[f * ix.m + p] * x[ix.seq(p + t)] + cvx[f * ix.m + p] * q[ix.seq(p + t)];
            part[HF * HKS * HKS + r] = a;
        }
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
    k_head_fold<float><<<hidden, HTH, 0, st>>>(n, hidden, theta, Wfc, Weff);
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
    k_head_grad_cols<float><<<hidden, HTH, 0, st>>>(n, hidden, theta, Wfc, G, dWfc, work);
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
        k_head_fold<double><<<hidden, HTH>>>(n, hidden, d, d + nt, d + nt + nw);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(weff.data(), d + nt + nw, sizeof(double) * nw, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(DNNMG_ECUDA, "head fold failed: %s", cudaGetErrorString(e));
    return dnnmg_net_create(n_in, hidden, n_out, Wx, Uh, weff.data(), precision, out);
}

}  // extern "C"

"""Oracle convolutional head of the patch network (S4, K = 1 net of Sec. 6.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 6.2 describes, after the fully connected layer, two convolutional blocks
that learn interactions between vertices, 36 parameters each, and a last
length-1 convolution with 18 parameters that reduces the concatenated filters
to one output per entry.  Each block expands to 4 filters and its transposed
layer reduces them back to 1.  No layer has a bias and no activation is named
between these layers.  Reading (the counts close only this way): each block's
transposed layer reuses the weights of its first layer, so a block with
filters k_f acts as

    B y = sum_f C_f^T C_f y,

C_f the zero-padded, size-preserving correlation with k_f and C_f^T its
adjoint (the transposed convolution).  The "spatial" block correlates each
velocity component's n x n patch nodes with 3 x 3 filters (4 x 9 = 36); the
"vertex" block correlates the output vector taken vertex by vertex, the two
components interleaved (u_0, v_0, u_1, v_1, ...), with length-9 filters
(4 x 9 = 36).  The last layer sums the two blocks and weights each of the
N_out entries (N_out parameters):

    d = w * (B_s d_fc + B_v d_fc),      d_fc = W_fc h'.

The head is linear in d_fc, so d = W_eff h' with W_eff[:, j] = head(W_fc[:, j]).

Parameter vector theta (72 + N_out): k_s [4][3][3] (filter, row offset
-1..1 in y, column offset -1..1 in x), k_v [4][9] (offset -4..4), w [N_out].
Layout of a prediction row: the u entries of the n x n patch nodes
(lexicographic, x fastest), then the v entries.
"""

import numpy as np

NF = 4          # filters per block
KS = 3          # spatial filter side
KV = 9          # vertex filter length


def n_theta(n_out):
    return NF * KS * KS + NF * KV + n_out


def split(theta, n_out):
    theta = np.asarray(theta, dtype=np.float64)
    ks = theta[:NF * KS * KS].reshape(NF, KS, KS)
    kv = theta[NF * KS * KS:NF * KS * KS + NF * KV].reshape(NF, KV)
    w = theta[NF * KS * KS + NF * KV:]
    assert w.shape == (n_out,)
    return ks, kv, w


def corr2d(g, k):
    """c[j, i] = sum_{a, b} k[a + 1, b + 1] g[j + a, i + b] (zero outside)."""
    n = g.shape[0]
    c = np.zeros_like(g)
    for j in range(n):
        for i in range(n):
            for a in (-1, 0, 1):
                for b in (-1, 0, 1):
                    if 0 <= j + a < n and 0 <= i + b < n:
                        c[j, i] += k[a + 1, b + 1] * g[j + a, i + b]
    return c


def corr2d_t(c, k):
    """The adjoint of corr2d: every product of corr2d sent back to its source."""
    n = c.shape[0]
    y = np.zeros_like(c)
    for j in range(n):
        for i in range(n):
            for a in (-1, 0, 1):
                for b in (-1, 0, 1):
                    if 0 <= j + a < n and 0 <= i + b < n:
                        y[j + a, i + b] += k[a + 1, b + 1] * c[j, i]
    return y


def corr1d(s, k):
    """c[p] = sum_t k[t + 4] s[p + t] (zero outside)."""
    m = len(s)
    c = np.zeros_like(s)
    for p in range(m):
        for t in range(-(KV // 2), KV // 2 + 1):
            if 0 <= p + t < m:
                c[p] += k[t + KV // 2] * s[p + t]
    return c


def corr1d_t(c, k):
    """The adjoint of corr1d."""
    m = len(c)
    s = np.zeros_like(c)
    for p in range(m):
        for t in range(-(KV // 2), KV // 2 + 1):
            if 0 <= p + t < m:
                s[p + t] += k[t + KV // 2] * c[p]
    return s


def spatial_block(y, ks):
    """B_s y: per velocity component, over its n x n patch nodes."""
    y = np.asarray(y, dtype=np.float64)
    nf = len(y) // 2
    n = int(round(np.sqrt(nf)))
    out = np.zeros_like(y)
    for comp in range(2):
        g = y[comp * nf:(comp + 1) * nf].reshape(n, n)
        acc = np.zeros((n, n))
        for f in range(NF):
            acc += corr2d_t(corr2d(g, ks[f]), ks[f])
        out[comp * nf:(comp + 1) * nf] = acc.ravel()
    return out


def vertex_block(y, kv):
    """B_v y: over the vertex-by-vertex sequence (u_0, v_0, u_1, v_1, ...)."""
    y = np.asarray(y, dtype=np.float64)
    nf = len(y) // 2
    s = np.empty_like(y)
    s[0::2], s[1::2] = y[:nf], y[nf:]
    acc = np.zeros_like(s)
    for f in range(NF):
        acc += corr1d_t(corr1d(s, kv[f]), kv[f])
    return np.concatenate([acc[0::2], acc[1::2]])


def head(y, theta):
    """d = w * (B_s y + B_v y) for one prediction row y [N_out]."""
    ks, kv, w = split(theta, len(y))
    return w * (spatial_block(y, ks) + vertex_block(y, kv))


def head_rows(D, theta):
    """The head on every row of D [P][N_out]."""
    return np.array([head(row, theta) for row in np.asarray(D, dtype=np.float64)])


def fold(theta, Wfc):
    """W_eff [N_out][H]: column j is the head applied to column j of W_fc."""
    Wfc = np.asarray(Wfc, dtype=np.float64)
    return np.stack([head(Wfc[:, j], theta) for j in range(Wfc.shape[1])], axis=1)


def fold_backward(theta, Wfc, G):
    """Gradients of sum(G * W_eff) with respect to theta and W_fc.

    With x = W_fc[:, j], g = G[:, j] and q = w * g:
      d/dW_fc[:, j] = B_s q + B_v q                      (both blocks symmetric)
      d/dw          = sum_j g * (B_s x + B_v x)
      d/dk_f[t]     = sum_j sum_p (C_f q)[p] x[p + t] + (C_f x)[p] q[p + t]
    (per component for the spatial block, on the interleaved sequence for the
    vertex block), from <q, C^T C x> and (C y)[p] = sum_t k[t] y[p + t].
    """
    Wfc = np.asarray(Wfc, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    n_out, H = Wfc.shape
    ks, kv, w = split(theta, n_out)
    nf = n_out // 2
    n = int(round(np.sqrt(nf)))
    dks, dkv, dw = np.zeros_like(ks), np.zeros_like(kv), np.zeros_like(w)
    dW = np.zeros_like(Wfc)
    for j in range(H):
        x, g = Wfc[:, j], G[:, j]
        q = w * g
        dW[:, j] = spatial_block(q, ks) + vertex_block(q, kv)
        dw += g * (spatial_block(x, ks) + vertex_block(x, kv))
        for comp in range(2):
            xs = x[comp * nf:(comp + 1) * nf].reshape(n, n)
            qs = q[comp * nf:(comp + 1) * nf].reshape(n, n)
            for f in range(NF):
                cq, cx = corr2d(qs, ks[f]), corr2d(xs, ks[f])
                for jj in range(n):
                    for ii in range(n):
                        for a in (-1, 0, 1):
                            for b in (-1, 0, 1):
                                if 0 <= jj + a < n and 0 <= ii + b < n:
                                    dks[f, a + 1, b + 1] += (cq[jj, ii] * xs[jj + a, ii + b]
                                                             + cx[jj, ii] * qs[jj + a, ii + b])
        xv, qv = np.empty(n_out), np.empty(n_out)
        xv[0::2], xv[1::2] = x[:nf], x[nf:]
        qv[0::2], qv[1::2] = q[:nf], q[nf:]
        for f in range(NF):
            cq, cx = corr1d(qv, kv[f]), corr1d(xv, kv[f])
            for p in range(n_out):
                for t in range(-(KV // 2), KV // 2 + 1):
                    if 0 <= p + t < n_out:
                        dkv[f, t + KV // 2] += cq[p] * xv[p + t] + cx[p] * qv[p + t]
    return np.concatenate([dks.ravel(), dkv.ravel(), dw]), dW


def param_count(n_out):
    """Trainable parameters of the head: two blocks of 4 x 9 and the last layer."""
    return n_theta(n_out)

"""Oracle for training the patch network: the GRU of Eq. gru
unrolled over a window of time steps, the l2 training loss of Sec. 6.3 with
Tikhonov regularisation, its gradient by backpropagation through time, and one
Adam update.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Network (as ``oracle.gru``): per patch row and step t = 1..T,

    z_t  = sigma(W_z x_t + U_z h_{t-1})
    r_t  = sigma(W_r x_t + U_r h_{t-1})
    c_t  = tanh(W_h x_t + U_h (r_t * h_{t-1}))
    h_t  = z_t * h_{t-1} + (1 - z_t) * c_t
    d_t  = W_fc h_t

Loss (Sec. 6.3, read as the squared l2 norm; the printed norm is unsquared):
the sum over the window's steps of the mean over patches of
|d_t - y_t|^2, with the target y_t = v_bar - v~ on the patch's fine nodes (so
that v~ + d - v_bar = d - y), plus alpha (|W_x|^2 + |U|^2 + |W_fc|^2).

Truncated backpropagation through time: the window starts from a given h_0
that is treated as a constant (its gradient is reported but not followed).

Adam (Kingma and Ba): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
p -= lr (m / (1 - b1^s)) / (sqrt(v / (1 - b2^s)) + eps) at step s = 1, 2, ...
"""

import numpy as np

from .gru import sigmoid


def seq_forward(X, h0, Wx, Uh, Wfc):
    """X [T][P][n_in], h0 [P][H].  Returns (D [T][P][n_out], cache)."""
    X = np.asarray(X, dtype=np.float64)
    Wx, Uh, Wfc = (np.asarray(a, dtype=np.float64) for a in (Wx, Uh, Wfc))
    T = X.shape[0]
    H = Uh.shape[1]
    Wz, Wr, Wh = Wx[0:H], Wx[H:2 * H], Wx[2 * H:3 * H]
    Uz, Ur, Uc = Uh[0:H], Uh[H:2 * H], Uh[2 * H:3 * H]
    h = np.array(h0, dtype=np.float64)
    hs, zs, rs, cs, D = [h], [], [], [], []
    for t in range(T):
        z = sigmoid(X[t] @ Wz.T + h @ Uz.T)
        r = sigmoid(X[t] @ Wr.T + h @ Ur.T)
        c = np.tanh(X[t] @ Wh.T + (r * h) @ Uc.T)
        h = z * h + (1.0 - z) * c
        zs.append(z)
        rs.append(r)
        cs.append(c)
        hs.append(h)
        D.append(h @ Wfc.T)
    return np.stack(D), dict(X=X, hs=hs, zs=zs, rs=rs, cs=cs)


def loss(D, Y, Wx, Uh, Wfc, alpha=1e-4):
    """Sum over steps of the mean over patches of |d - y|^2, plus alpha |W|^2."""
    D, Y = np.asarray(D, dtype=np.float64), np.asarray(Y, dtype=np.float64)
    P = D.shape[1]
    data = float(np.sum((D - Y) ** 2) / P)
    reg = alpha * float(sum(np.sum(np.asarray(W, dtype=np.float64) ** 2) for W in (Wx, Uh, Wfc)))
    return data + reg


def loss_grad_D(D, Y):
    """d loss / d D for the data term."""
    P = D.shape[1]
    return 2.0 * (np.asarray(D, dtype=np.float64) - np.asarray(Y, dtype=np.float64)) / P


def seq_backward(dD, cache, Wx, Uh, Wfc):
    """Gradients of sum(dD * D) with respect to Wx, Uh, Wfc and h0, by
    backpropagation through the window's steps (chain rule of the recurrence
    above, last step first)."""
    dD = np.asarray(dD, dtype=np.float64)
    Wx, Uh, Wfc = (np.asarray(a, dtype=np.float64) for a in (Wx, Uh, Wfc))
    X, hs, zs, rs, cs = cache["X"], cache["hs"], cache["zs"], cache["rs"], cache["cs"]
    T = X.shape[0]
    H = Uh.shape[1]
    Uz, Ur, Uc = Uh[0:H], Uh[H:2 * H], Uh[2 * H:3 * H]
    gWx, gUh, gWfc = np.zeros_like(Wx), np.zeros_like(Uh), np.zeros_like(Wfc)
    dh_next = np.zeros_like(hs[0])
    for t in reversed(range(T)):
        h_prev, z, r, c = hs[t], zs[t], rs[t], cs[t]
        gWfc += dD[t].T @ hs[t + 1]
        dh = dD[t] @ Wfc + dh_next                   # total gradient reaching h_t
        dc = dh * (1.0 - z)                          # through c_t
        dz = dh * (h_prev - c)                       # through z_t
        dac = dc * (1.0 - c * c)                     # tanh'
        daz = dz * z * (1.0 - z)                     # sigma'
        drh = dac @ Uc                               # gradient of r_t * h_{t-1}
        dar = drh * h_prev * r * (1.0 - r)
        gWx[0:H] += daz.T @ X[t]
        gWx[H:2 * H] += dar.T @ X[t]
        gWx[2 * H:3 * H] += dac.T @ X[t]
        gUh[0:H] += daz.T @ h_prev
        gUh[H:2 * H] += dar.T @ h_prev
        gUh[2 * H:3 * H] += dac.T @ (r * h_prev)
        dh_next = dh * z + drh * r + daz @ Uz + dar @ Ur
    return gWx, gUh, gWfc, dh_next


def loss_and_grads(X, h0, Y, Wx, Uh, Wfc, alpha=1e-4):
    """Loss of the window and its gradients (regulariser included)."""
    D, cache = seq_forward(X, h0, Wx, Uh, Wfc)
    gWx, gUh, gWfc, gh0 = seq_backward(loss_grad_D(D, Y), cache, Wx, Uh, Wfc)
    Wx, Uh, Wfc = (np.asarray(a, dtype=np.float64) for a in (Wx, Uh, Wfc))
    return (loss(D, Y, Wx, Uh, Wfc, alpha), gWx + 2 * alpha * Wx, gUh + 2 * alpha * Uh,
            gWfc + 2 * alpha * Wfc, gh0)


def adam_step(p, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step number `step` (1-based); returns (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v

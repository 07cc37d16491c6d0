"""Oracle GRU cell and output layer (S4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Eq. gru (Cho et al. form; the reset gate multiplies the previous state before
the recurrent weight of the candidate), with the paper's statement that no
layer has a bias (Sec. 6.2), the logistic function for the gates and tanh for
the candidate, followed by the fully connected layer to N_out outputs:

    z  = sigma(W_z x + U_z h)
    r  = sigma(W_r x + U_r h)
    h' = z * h + (1 - z) * tanh(W_h x + U_h (r * h))
    d  = W_fc h'

Weight layout: Wx [3H][N_in] and Uh [3H][H] stack the gates in the order
z, r, h; Wfc [N_out][H].
"""

import numpy as np


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def gru_step(X, h, Wx, Uh, Wfc):
    """One GRU step for every patch row; returns (h', d)."""
    X = np.asarray(X, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    Wx, Uh, Wfc = (np.asarray(a, dtype=np.float64) for a in (Wx, Uh, Wfc))
    H = h.shape[1]
    z = sigmoid(X @ Wx[0:H].T + h @ Uh[0:H].T)
    r = sigmoid(X @ Wx[H:2 * H].T + h @ Uh[H:2 * H].T)
    cand = np.tanh(X @ Wx[2 * H:3 * H].T + (r * h) @ Uh[2 * H:3 * H].T)
    h_new = z * h + (1.0 - z) * cand
    return h_new, h_new @ Wfc.T


def param_count(n_in, H, n_out):
    """Trainable parameters of the GRU and the output layer (no biases)."""
    return 3 * H * (n_in + H) + H * n_out

"""Oracle DNN-MG correction step (S8).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The correction step of Algorithm 2, in the paper's order:
  v~     <- P(v^L)                      (prolongation; S1)
  d      <- N(v~, Omega_L, Omega_L+K)   (network correction; S2 residual, S3 features, S4 net)
  b^L+K  <- Rhs(v~ + d)                 (right-hand side; S5 averaging, S6)
  b^L    <- R(b^L+K)                    (restriction; S7)
The residual of S2 uses the fine right-hand side b_f of the current step,
i.e. the one assembled by the previous step's right-hand-side stage.

Pins: with a zero network (d = 0) the step's coarse right-hand side equals
the coarse level's own Crank-Nicolson right-hand side of x_c (a Galerkin
identity of the nested Q1 spaces, exact in the quadrature used), pinned on the
CPU for K = 1, 2, 3 and s = 1, 2.  Parity unpinned for a nonzero network: the
composition then has no closed form of its own, and each part it calls is
pinned separately.
"""

from .average import scatter_average
from .features import patch_features
from .fem import residual, rhs
from .gru import gru_step
from .transfer import prolongate, restrict


def dnnmg_step(mesh, prm, weights, xc, h, bf, t):
    """One correction step; returns every intermediate as float64 arrays.

    weights = (Wx, Uh, Wfc); xc [3][Nc]; h [P][H]; bf [2][Nf]; t = t_n.
    """
    xf = prolongate(mesh, prm, xc, t)
    r = residual(mesh, prm, xf, bf)
    X = patch_features(mesh, prm, xf, r)
    h_new, d = gru_step(X, h, *weights)
    vcorr = scatter_average(mesh, d, xf)
    bf_new = rhs(mesh, prm, vcorr)
    bc = restrict(mesh, bf_new)
    return {"xf": xf, "r": r, "X": X, "h": h_new, "d": d, "vcorr": vcorr,
            "bf": bf_new, "bc": bc}

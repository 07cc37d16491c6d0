"""Oracle averaging of the patch predictions (S5).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 5.2: the network predicts a correction for the fine nodes of every patch
independently; predictions for nodes shared by adjacent patches are averaged.
Reading: a uniform mean over the fluid patches that contain the node.  The
corrected velocity is v~ + mean(d) on the velocity unknowns; Dirichlet nodes
keep their boundary values (they are not unknowns).  Sign: d = v_bar - v~
(Sec. 5.1), so the correction is added.

Layout of one prediction row d [P][2 nf]: the u correction on the fine patch
nodes (lexicographic, x fastest), then the v correction.
"""

import numpy as np

from .features import patch_node_indices


def scatter_average(mesh, d, xf):
    """S5: v_corr [2][Nf] from the predictions d [P][2 nf] and v~ = xf[:2]."""
    fine, _ = patch_node_indices(mesh)
    d = np.asarray(d, dtype=np.float64)
    nf = mesh.nf
    sums = np.zeros((2, mesh.Nf))
    count = np.zeros(mesh.Nf)
    for p in range(mesh.P):
        sums[0, fine[p]] += d[p, :nf]
        sums[1, fine[p]] += d[p, nf:]
        count[fine[p]] += 1.0
    v = np.array([np.asarray(xf[0], dtype=np.float64), np.asarray(xf[1], dtype=np.float64)])
    free = ~mesh.dirichlet.ravel()
    v[:, free] += sums[:, free] / count[free]
    return v

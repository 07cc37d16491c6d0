"""Oracle mesh transfer: prolongation P and restriction R (S1, S7).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 3.4: prolongation is interpolation from the coarse to the fine space;
restriction maps fine residual/right-hand-side vectors to the coarse level.
Algorithm 2 prolongates the coarse solution from level L to L+K and, at the
end of the correction, restricts the fine right-hand side back to level L.

For right-hand-side (dual) vectors the restriction is the transpose of the
prolongation, R = P^T.  Here P is written as direct bilinear interpolation
across all K levels, and R independently as K nested single-level restrictions
(1D weights 1/2, 1, 1/2 per direction); the tests check <R x, y> = <x, P y>.
"""

import numpy as np


def prolongate_raw(mesh, xc):
    """Bilinear interpolation of coarse nodal fields to the fine nodes.

    xc: [ncomp][Nc] on the window's coarse nodes (x fastest).  Returns
    [ncomp][Nf] on the window's fine nodes.  Each fine node lies in a coarse
    cell (the last cell for nodes on the cell's right/top edge) and takes the
    bilinear combination of that cell's 4 corner values (Sec. 3.4,
    interpolation).  No boundary condition is applied.
    """
    xc = np.asarray(xc, dtype=np.float64)
    r = mesh.r
    nxn, nyn = mesh.wxf + 1, mesh.wyf + 1
    I = np.arange(nxn)
    J = np.arange(nyn)
    ci = np.minimum(I // r, mesh.wxc - 1)
    cj = np.minimum(J // r, mesh.wyc - 1)
    a = (I - ci * r) / r            # local coordinate in [0, 1] along x
    b = (J - cj * r) / r            # along y
    A, B = np.meshgrid(a, b)
    CI, CJ = np.meshgrid(ci, cj)
    out = np.empty((xc.shape[0], nyn * nxn))
    for c in range(xc.shape[0]):
        f = xc[c].reshape(mesh.wyc + 1, mesh.wxc + 1)
        val = ((1 - A) * (1 - B) * f[CJ, CI] + A * (1 - B) * f[CJ, CI + 1]
               + (1 - A) * B * f[CJ + 1, CI] + A * B * f[CJ + 1, CI + 1])
        out[c] = val.ravel()
    return out


def dirichlet_velocity(mesh, prm, t):
    """Dirichlet values and mask of the fine velocity at time t (Sec. 6.1).

    Returns (mask [Nf] bool, u_D [Nf], v_D [Nf]): the inflow profile on x = 0,
    zero on the walls and at every node of a solid cell.
    """
    mask = mesh.dirichlet.ravel()
    uD = np.where(mesh.inflow, mesh.inflow_profile(mesh.y_f, prm, t), 0.0).ravel()
    return mask, uD, np.zeros_like(uD)


def prolongate(mesh, prm, xc, t):
    """S1: x~ = P x_c on (u, v, p), then the fine velocity Dirichlet values.

    The prolongation of Algorithm 2.  xc: [3][Nc] float64; returns [3][Nf].
    """
    xf = prolongate_raw(mesh, xc)
    mask, uD, vD = dirichlet_velocity(mesh, prm, t)
    xf[0, mask] = uD[mask]
    xf[1, mask] = vD[mask]
    return xf


def _restrict_1d(v, axis):
    """Transpose of 1D linear interpolation from n/2 to n cells along axis."""
    v = np.moveaxis(v, axis, -1)
    even = v[..., 0::2]
    odd = v[..., 1::2]
    out = even.copy()
    out[..., :-1] += 0.5 * odd
    out[..., 1:] += 0.5 * odd
    return np.moveaxis(out, -1, axis)


def restrict_raw(mesh, bf):
    """R = P^T applied to fine nodal vectors bf [ncomp][Nf] -> [ncomp][Nc].

    Written as K nested single-level restrictions; no boundary handling.
    """
    bf = np.asarray(bf, dtype=np.float64)
    out = []
    for c in range(bf.shape[0]):
        g = bf[c].reshape(mesh.wyf + 1, mesh.wxf + 1)
        for _ in range(mesh.K):
            g = _restrict_1d(g, axis=1)
            g = _restrict_1d(g, axis=0)
        out.append(g.ravel())
    return np.array(out)


def restrict(mesh, bf):
    """S7: b_c = R b_f for the velocity rows, coarse Dirichlet rows zeroed.

    The restriction of Algorithm 2 (the right-hand side is restricted, not the velocity).
    bf: [2][Nf]; returns [3][Nc] with the pressure rows 0.
    """
    bc2 = restrict_raw(mesh, bf)
    mask = mesh.dirichlet_c.ravel()
    bc2[:, mask] = 0.0
    return np.concatenate([bc2, np.zeros((1, bc2.shape[1]))])

"""Oracle per-patch network inputs (S3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 5.2 "Neural network inputs": per patch the network sees the nonlinear
residual on the fine patch nodes (3 components), the coarse velocities and
Peclet numbers on the coarse patch nodes, and 12 geometry values of the patch
(4 edge lengths, 4 aspect ratios, 4 angles).  For one-cell patches and K = 1
that is 27 + 8 + 4 + 12 = 51 inputs, as the paper counts; for K = 2 it is 99
(Sec. 6.6).

Order of one feature row (a reading; the paper fixes the content, not the order):
  [ r_u(fine patch nodes), r_v(...), r_p(...),
    u(coarse patch nodes), v(...), Pe(...),
    edge lengths (bottom, right, top, left),
    aspect ratios (bottom/right, top/left, bottom/top, left/right),
    corner angles (SW, SE, NE, NW) ]
Patch nodes are listed lexicographically, x fastest.  The coarse velocities are
the prolongated velocity v~ at the fine nodes that coincide with coarse nodes;
Pe = q |v~| / nu with q the longest patch edge (the paper's "patch size").
"""

import numpy as np


def patch_geometry(mesh):
    """12 geometry values of a patch, computed from its corner coordinates."""
    w, h = mesh.s * mesh.hxc, mesh.s * mesh.hyc
    sw, se, ne, nw = (np.array(c, dtype=np.float64) for c in ((0, 0), (w, 0), (w, h), (0, h)))
    corners = [sw, se, ne, nw]
    edges = [se - sw, ne - se, nw - ne, sw - nw]            # bottom, right, top, left
    lens = [float(np.hypot(*e)) for e in edges]
    aspect = [lens[0] / lens[1], lens[2] / lens[3], lens[0] / lens[2], lens[3] / lens[1]]
    angles = []
    for c in range(4):
        a = corners[(c + 1) % 4] - corners[c]
        b = corners[(c - 1) % 4] - corners[c]
        angles.append(float(np.arccos(np.dot(a, b) / (np.hypot(*a) * np.hypot(*b)))))
    return np.array(lens + aspect + angles)


def patch_node_indices(mesh):
    """Window-local fine node indices [P][nf] and coarse-node positions [P][nc]."""
    nxn = mesh.wxf + 1
    S, r = mesh.S, mesh.r
    li = mesh.patches[:, 0] * S - mesh.fi0
    lj = mesh.patches[:, 1] * S - mesh.fj0
    base = lj * nxn + li
    fo = np.array([b * nxn + a for b in range(S + 1) for a in range(S + 1)])
    co = np.array([b * r * nxn + a * r for b in range(mesh.s + 1) for a in range(mesh.s + 1)])
    return base[:, None] + fo[None, :], base[:, None] + co[None, :]


def patch_features(mesh, prm, xf, r):
    """S3: feature matrix X [P][n_in] of the window's fluid patches."""
    fine, coarse = patch_node_indices(mesh)
    u = np.asarray(xf[0], dtype=np.float64)[coarse]
    v = np.asarray(xf[1], dtype=np.float64)[coarse]
    q = mesh.s * max(mesh.hxc, mesh.hyc)
    pe = q * np.sqrt(u * u + v * v) / prm.nu
    geo = np.broadcast_to(patch_geometry(mesh), (mesh.P, 12))
    X = np.concatenate([r[0][fine], r[1][fine], r[2][fine], u, v, pe, geo], axis=1)
    assert X.shape[1] == mesh.n_in
    return X

"""Oracle finite elements: Crank-Nicolson residual and right-hand side (S2, S6).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Discretisation (Sec. 3.1-3.3), read for a bilinear (Q1/Q1) equal-order pair on
the structured mesh, as the workloads state:

* velocity rows, Eq. nonlinearshort:
    A_v(x)_i = 1/k (v, phi_i) + 1/2 (v.grad v, phi_i) + nu/2 (grad v, grad phi_i)
               - (p, div phi_i)
* pressure rows, Eq. nonlinearshort with the local projection term of Eq. disc:ns:
    A_p(x)_i = (div v, xi_i) + sum_T alpha_T (grad(p - pi p), grad(xi_i - pi xi_i))
* right-hand side from the previous velocity, Eq. 4cranknicholson3 (f = 0):
    b_i = 1/k (v, phi_i) - 1/2 (v.grad v, phi_i) - nu/2 (grad v, grad phi_i)

Readings: nu is the coefficient 1/Re of Eq. nsstrong; alpha_T = alpha0 h_T^2 / nu
with h_T the fine cell diagonal (the paper's alpha0 * Re * h_T^2); the local
projection pi maps Q1 on a 2x2-cell patch to Q1 on the patch (the bilinear
interpolant of the patch's 4 corner values), the Q1 analogue of the paper's
Q2 -> Q1 projection.  Integrals use 2x2 Gauss quadrature per cell, which is
exact for every term on rectangles.  Only fluid cells contribute.
"""

import numpy as np


def gauss_1d(nq):
    """Gauss-Legendre points and weights on [0, 1]."""
    if nq == 2:
        g = 0.5 / np.sqrt(3.0)
        return np.array([0.5 - g, 0.5 + g]), np.array([0.5, 0.5])
    if nq == 3:
        g = 0.5 * np.sqrt(0.6)
        return np.array([0.5 - g, 0.5, 0.5 + g]), np.array([5.0, 8.0, 5.0]) / 18.0
    raise ValueError(nq)


def q1_shape(xi, eta):
    """Q1 shape functions on the unit square, local order SW, SE, NW, NE.

    Returns (phi[4], dphi/dxi[4], dphi/deta[4]).
    """
    phi = np.array([(1 - xi) * (1 - eta), xi * (1 - eta), (1 - xi) * eta, xi * eta])
    dxi = np.array([-(1 - eta), (1 - eta), -eta, eta])
    deta = np.array([-(1 - xi), -xi, (1 - xi), xi])
    return phi, dxi, deta


def fluid_cell_nodes(mesh):
    """Node indices [ncell][4] (SW, SE, NW, NE) of the window's fluid fine cells."""
    nxn = mesh.wxf + 1
    j, i = np.nonzero(~mesh.solid_f)
    n0 = j * nxn + i
    return np.stack([n0, n0 + 1, n0 + nxn, n0 + nxn + 1], axis=1)


def assemble_terms(mesh, u, v, p=None, nq=2):
    """Per-node integrals of every term, summed over fluid cells, no BC.

    u, v, p: fine nodal fields [Nf].  Returns a dict of [Nf] arrays:
    mass_u/v = (v_c, phi_i), conv_u/v = (v.grad v_c, phi_i),
    diff_u/v = (grad v_c, grad phi_i), pres_u/v = (p, d_c phi_i),
    div = (div v, xi_i).
    """
    hx, hy = mesh.hxf, mesh.hyf
    cells = fluid_cell_nodes(mesh)
    ue, ve = u[cells], v[cells]
    pe = p[cells] if p is not None else np.zeros_like(ue)
    names = ["mass_u", "mass_v", "conv_u", "conv_v", "diff_u", "diff_v",
             "pres_u", "pres_v", "div"]
    loc = {n: np.zeros(cells.shape) for n in names}
    pts, wts = gauss_1d(nq)
    for xi, wx in zip(pts, wts):
        for eta, wy in zip(pts, wts):
            w = wx * wy * hx * hy
            phi, dxi, deta = q1_shape(xi, eta)
            dx, dy = dxi / hx, deta / hy
            uq, vq, pq = ue @ phi, ve @ phi, pe @ phi
            ux, uy, vx, vy = ue @ dx, ue @ dy, ve @ dx, ve @ dy
            for a in range(4):
                loc["mass_u"][:, a] += w * uq * phi[a]
                loc["mass_v"][:, a] += w * vq * phi[a]
                loc["conv_u"][:, a] += w * (uq * ux + vq * uy) * phi[a]
                loc["conv_v"][:, a] += w * (uq * vx + vq * vy) * phi[a]
                loc["diff_u"][:, a] += w * (ux * dx[a] + uy * dy[a])
                loc["diff_v"][:, a] += w * (vx * dx[a] + vy * dy[a])
                loc["pres_u"][:, a] += w * pq * dx[a]
                loc["pres_v"][:, a] += w * pq * dy[a]
                loc["div"][:, a] += w * (ux + vy) * phi[a]
    out = {}
    for n in names:
        acc = np.zeros(mesh.Nf)
        np.add.at(acc, cells, loc[n])
        out[n] = acc
    return out


def lps_projection_matrix():
    """Pi (9x9): nodal values of the patch's bilinear interpolant of its corners.

    Patch nodes are numbered (a, b) -> 3 b + a, a, b in {0, 1, 2} (x fastest).
    """
    Pi = np.zeros((9, 9))
    corners = {(0, 0): 0, (2, 0): 2, (0, 2): 6, (2, 2): 8}
    for b in range(3):
        for a in range(3):
            X, Y = a / 2.0, b / 2.0
            wts = {(0, 0): (1 - X) * (1 - Y), (2, 0): X * (1 - Y),
                   (0, 2): (1 - X) * Y, (2, 2): X * Y}
            for c, idx in corners.items():
                Pi[3 * b + a, idx] += wts[c]
    return Pi


def lps_patch_stiffness(hx, hy, nq=2):
    """L (9x9): (grad f, grad g) over the 2x2-cell patch for Q1 nodal vectors."""
    pts, wts = gauss_1d(nq)
    Ke = np.zeros((4, 4))
    for xi, wx in zip(pts, wts):
        for eta, wy in zip(pts, wts):
            _, dxi, deta = q1_shape(xi, eta)
            dx, dy = dxi / hx, deta / hy
            Ke += wx * wy * hx * hy * (np.outer(dx, dx) + np.outer(dy, dy))
    L = np.zeros((9, 9))
    for cb in range(2):
        for ca in range(2):
            idx = [3 * cb + ca, 3 * cb + ca + 1, 3 * (cb + 1) + ca, 3 * (cb + 1) + ca + 1]
            L[np.ix_(idx, idx)] += Ke
    return L


def lps_alpha(mesh, prm):
    """alpha_T = alpha0 * h_T^2 / nu, h_T the fine cell diagonal (Sec. 3.1)."""
    return prm.alpha0 * (mesh.hxf ** 2 + mesh.hyf ** 2) / prm.nu


def lps_cell_stiffness(hx, hy, cells, nq=2):
    """(grad f, grad g) over the listed cells (ca, cb) of a 2x2-cell patch, 9x9."""
    pts, wts = gauss_1d(nq)
    Ke = np.zeros((4, 4))
    for xi, wx in zip(pts, wts):
        for eta, wy in zip(pts, wts):
            _, dxi, deta = q1_shape(xi, eta)
            dx, dy = dxi / hx, deta / hy
            Ke += wx * wy * hx * hy * (np.outer(dx, dx) + np.outer(dy, dy))
    L = np.zeros((9, 9))
    for ca, cb in cells:
        idx = [3 * cb + ca, 3 * cb + ca + 1, 3 * (cb + 1) + ca, 3 * (cb + 1) + ca + 1]
        L[np.ix_(idx, idx)] += Ke
    return L


def lps_term(mesh, prm, p, nq=2):
    """sum_T alpha_T (grad(p - pi p), grad(xi_i - pi xi_i)) per pressure node.

    Loops over the 2x2-cell patches (aligned to even fine indices) that hold
    a fluid cell.  With f = (I - Pi) p_patch and g_i = (I - Pi) e_i the patch
    contribution to row i is alpha g_i^T L f, L the stiffness over the
    patch's fluid cells T.  On nested masks (every level above a coarse one)
    patches are all fluid or all solid; a single level's own mask can leave a
    patch partly solid, and then only its fluid cells enter the sum over T.
    """
    nxn = mesh.wxf + 1
    Pi = lps_projection_matrix()
    IminusPi = np.eye(9) - Pi
    L = lps_patch_stiffness(mesh.hxf, mesh.hyf, nq)
    alpha = lps_alpha(mesh, prm)
    sol = mesh.solid_f
    blk = sol.reshape(mesh.wyf // 2, 2, mesh.wxf // 2, 2)
    offs = np.array([b * nxn + a for b in range(3) for a in range(3)])
    out = np.zeros(mesh.Nf)
    # all-fluid patches: fine cells (2m..2m+1, 2n..2n+1)
    n, m = np.nonzero(~blk.any(axis=(1, 3)))
    nodes = ((2 * n) * nxn + 2 * m)[:, None] + offs[None, :]
    f = p[nodes] @ IminusPi.T
    contrib = alpha * (f @ L.T) @ IminusPi
    np.add.at(out, nodes, contrib)
    # partly solid patches: the stiffness of their fluid cells only
    n, m = np.nonzero(blk.any(axis=(1, 3)) & ~blk.all(axis=(1, 3)))
    for nn, mm in zip(n, m):
        fluid = [(ca, cb) for cb in range(2) for ca in range(2) if not blk[nn, cb, mm, ca]]
        Lp = lps_cell_stiffness(mesh.hxf, mesh.hyf, fluid, nq)
        nd = (2 * nn) * nxn + 2 * mm + offs
        fp = IminusPi @ p[nd]
        out[nd] += alpha * IminusPi.T @ (Lp @ fp)
    return out


def velocity_operator(mesh, prm, terms):
    """A_v(x) per velocity component (Eq. nonlinearshort), no BC."""
    Au = terms["mass_u"] / prm.k + 0.5 * terms["conv_u"] + 0.5 * prm.nu * terms["diff_u"] - terms["pres_u"]
    Av = terms["mass_v"] / prm.k + 0.5 * terms["conv_v"] + 0.5 * prm.nu * terms["diff_v"] - terms["pres_v"]
    return Au, Av


def rhs_raw(mesh, prm, terms):
    """b from the previous velocity (Eq. 4cranknicholson3 right side, f = 0), no BC."""
    bu = terms["mass_u"] / prm.k - 0.5 * terms["conv_u"] - 0.5 * prm.nu * terms["diff_u"]
    bv = terms["mass_v"] / prm.k - 0.5 * terms["conv_v"] - 0.5 * prm.nu * terms["diff_v"]
    return bu, bv


def residual(mesh, prm, xf, bf, nq=2):
    """S2: r = b_f - A(x~) on velocity and pressure rows ([3][Nf]).

    Sec. 5.2 "Neural network inputs": the nonlinear residual of the prolongated
    coarse solution for Eq. nonlinearshort.  xf: [3][Nf] (u, v, p); bf: [2][Nf]
    the fine right-hand side of the current step.  Dirichlet velocity rows and
    inactive pressure rows are 0; the pressure right-hand side is 0.
    """
    u, v, p = (np.asarray(xf[c], dtype=np.float64) for c in range(3))
    terms = assemble_terms(mesh, u, v, p, nq)
    Au, Av = velocity_operator(mesh, prm, terms)
    Ap = terms["div"] + lps_term(mesh, prm, p, nq)
    r = np.array([np.asarray(bf[0], dtype=np.float64) - Au,
                  np.asarray(bf[1], dtype=np.float64) - Av,
                  -Ap])
    dmask = mesh.dirichlet.ravel()
    r[0, dmask] = 0.0
    r[1, dmask] = 0.0
    r[2, ~mesh.p_active.ravel()] = 0.0
    return r


def rhs(mesh, prm, vel, nq=2):
    """S6: fine right-hand side b_f = Rhs(v) for the next step ([2][Nf]).

    The right-hand side of Algorithm 2's correction, with v = v~ + d;
    Dirichlet velocity rows are 0.
    """
    u, v = (np.asarray(vel[c], dtype=np.float64) for c in range(2))
    terms = assemble_terms(mesh, u, v, None, nq)
    bu, bv = rhs_raw(mesh, prm, terms)
    b = np.array([bu, bv])
    b[:, mesh.dirichlet.ravel()] = 0.0
    return b

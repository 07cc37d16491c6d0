"""Host FP64 solve of one mesh level's Crank-Nicolson system.

Supporting code around the correction step, not part of it:

* the coarse solve of Algorithm 2, which the correction step feeds with
  its restricted right-hand side and which feeds the next step with x_c;
* the plain fine-level time stepping whose velocities are the ground truth
  the network is trained towards (Sec. 5.2, "Training of DNN-MG").

The correction step itself (the rest of Algorithm 2) runs in the library's
kernels; nothing here stands in for one of them.  The paper solves this
system by Newton's method with GMRES and a geometric multigrid
preconditioner (Sec. 3.3); on the meshes that time loops and training data
use here, a sparse LU factorisation of each Newton matrix does the same job.

Discretisation, the one the library's kernels evaluate (Sec. 3.1-3.3): Q1
velocity and pressure on a uniform channel mesh whose solid cells are masked
out, Crank-Nicolson in time, local projection stabilisation of the pressure
on 2x2-cell patches.  Find x = (u, v, p) at t_{n+1} with

  velocity rows  (1/k)(v, phi) + 1/2 (v.grad v, phi) + nu/2 (grad v, grad phi)
                 - (p, div phi) = b
  pressure rows  (div v, xi) + sum_T alpha_T (grad(p - pi p), grad(xi - pi xi)) = 0

where b = (1/k)(v_n, phi) - 1/2 (v_n.grad v_n, phi) - nu/2 (grad v_n, grad phi)
(Eq. 4cranknicholson3 with f = 0), alpha_T = alpha0 (hx^2 + hy^2) / nu and
pi the bilinear interpolant of a patch's 4 corners.  Velocity Dirichlet rows
hold the boundary values at t_{n+1}: the parabolic inflow at x = 0 (with the
start-up ramp of Sec. 6.1 when enabled), zero on the walls and on every node
of a solid cell.  Pressure rows of nodes that touch no fluid cell hold p = 0.
The outflow x = lx is do-nothing.  Integrals use 2x2 Gauss points per cell,
exact for every term on rectangles.
"""

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import splu

LX, LY = 2.2, 0.41

# local corner order of a cell: (cx, cy) = SW, SE, NW, NE
_CORNERS = ((0, 0), (1, 0), (0, 1), (1, 1))


def _reference_tables():
    """Shape values and reference derivatives at the 2x2 Gauss points, [q][a]."""
    g = 0.5 / np.sqrt(3.0)
    pts = [(x, y) for y in (0.5 - g, 0.5 + g) for x in (0.5 - g, 0.5 + g)]
    phi = np.empty((4, 4))
    dxi = np.empty((4, 4))
    deta = np.empty((4, 4))
    for q, (x, y) in enumerate(pts):
        for a, (cx, cy) in enumerate(_CORNERS):
            fx, gx = (x, 1.0) if cx else (1.0 - x, -1.0)
            fy, gy = (y, 1.0) if cy else (1.0 - y, -1.0)
            phi[q, a] = fx * fy
            dxi[q, a] = gx * fy
            deta[q, a] = fx * gy
    return phi, dxi, deta


def ellipse_mask(nx, ny, ellipse, lx=LX, ly=LY):
    """Solid cells [ny][nx]: centroid strictly inside the ellipse (cx, cy, ax, ay)."""
    if ellipse is None:
        return np.zeros((ny, nx), dtype=bool)
    cx, cy, ax, ay = ellipse
    if ax <= 0 or ay <= 0:
        return np.zeros((ny, nx), dtype=bool)
    xc = (np.arange(nx) + 0.5) * (lx / nx)
    yc = (np.arange(ny) + 0.5) * (ly / ny)
    X, Y = np.meshgrid(xc, yc)
    return ((X - cx) / ax) ** 2 + ((Y - cy) / ay) ** 2 < 1.0


def geometry_mask(nx, ny, name, lx=LX, ly=LY):
    """Solid cells [ny][nx] of the generalization geometries of Sec. 6.7 (cell
    centroids): "none" (the channel without obstacle), "two" (two elliptic
    obstacles centred at (0.2, 0.18) and (0.6, 0.24), semi-axes 0.055 x 0.045:
    the printed axes "1.1" and "0.9" read as 0.11 and 0.09), "L" (the channel
    with the upper half of its right half solid)."""
    x = (np.arange(nx) + 0.5) * (lx / nx)
    y = (np.arange(ny) + 0.5) * (ly / ny)
    X, Y = np.meshgrid(x, y)
    if name == "none":
        return np.zeros((ny, nx), dtype=bool)
    if name == "two":
        m = np.zeros((ny, nx), dtype=bool)
        for cx, cy in ((0.2, 0.18), (0.6, 0.24)):
            m |= ((X - cx) / 0.055) ** 2 + ((Y - cy) / 0.045) ** 2 < 1.0
        return m
    if name == "L":
        return (X > lx / 2) & (Y > ly / 2)
    raise ValueError(f"unknown geometry {name!r}")


def refine_mask(solid, K):
    """Cell mask of the level K refinements finer: fine cells inherit their parent's flag."""
    r = 2 ** K
    return np.kron(np.asarray(solid, dtype=np.uint8), np.ones((r, r), dtype=np.uint8)).astype(bool)


class Level:
    """One uniform mesh level of the channel and its nonlinear system.

    Node fields are [comp][N] arrays, N = (nx + 1)(ny + 1), node (i, j) at
    index j (nx + 1) + i, x fastest: the oracle's layout and, row by row,
    the unpadded layout of the library's coarse vectors.
    """

    def __init__(self, nx, ny, solid=None, lx=LX, ly=LY, nu=1e-3, k=0.01, alpha0=0.1,
                 u_max=1.5, ramp=False):
        if nx % 2 or ny % 2:
            raise ValueError("cell counts must be even (2x2-cell projection patches)")
        self.nx, self.ny = nx, ny
        self.lx, self.ly = float(lx), float(ly)
        self.hx, self.hy = self.lx / nx, self.ly / ny
        self.nu, self.k, self.alpha0, self.u_max, self.ramp = nu, k, alpha0, u_max, ramp
        self.solid = (np.zeros((ny, nx), dtype=bool) if solid is None
                      else np.asarray(solid, dtype=bool).copy())
        if self.solid.shape != (ny, nx):
            raise ValueError("solid mask must be [ny][nx]")
        self.N = (nx + 1) * (ny + 1)
        self._node_classes()
        self._tables()
        self._linear_matrices()
        self._lu = None               # last factorised Newton matrix (reused by chord iterations)
        self.factorisations = 0

    # ------------------------------------------------------------ geometry
    def _node_classes(self):
        nx, ny = self.nx, self.ny
        ext = -np.ones((ny + 2, nx + 2), dtype=np.int8)      # -1 no cell, 0 fluid, 1 solid
        ext[1:-1, 1:-1] = self.solid
        around = [ext[dj:dj + ny + 1, di:di + nx + 1] for dj in (0, 1) for di in (0, 1)]
        touch_solid = np.any([c == 1 for c in around], axis=0)
        touch_fluid = np.any([c == 0 for c in around], axis=0)
        J, I = np.meshgrid(np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
        wall = (J == 0) | (J == ny)
        zero = wall | touch_solid
        self.dirichlet = (zero | (I == 0)).ravel()
        self.inflow = ((I == 0) & ~zero).ravel()
        self.p_active = touch_fluid.ravel()
        self.y = (J * self.hy).ravel()

    def omega(self, t):
        """Start-up ramp of the inflow (Sec. 6.1); 1 when the ramp is off."""
        if not self.ramp:
            return 1.0
        return 0.5 - 0.5 * np.cos(2.0 * np.pi * t) if t <= 0.5 else 1.0

    def boundary_values(self, t):
        """Velocity Dirichlet values at time t, [2][N] (zero off the Dirichlet rows)."""
        g = np.zeros((2, self.N))
        y = self.y[self.inflow]
        g[0, self.inflow] = self.u_max * 4.0 * y * (self.ly - y) / self.ly ** 2 * self.omega(t)
        return g

    # ------------------------------------------------------------ assembly
    def _tables(self):
        phi, dxi, deta = _reference_tables()
        self.PHI = phi
        self.DX = dxi / self.hx
        self.DY = deta / self.hy
        self.w = 0.25 * self.hx * self.hy                      # Gauss weight x cell area
        nxn = self.nx + 1
        j, i = np.nonzero(~self.solid)
        n0 = j * nxn + i
        self.cells = np.stack([n0 + cy * nxn + cx for cx, cy in _CORNERS], axis=1)
        self._rows = np.repeat(self.cells, 4, axis=1).ravel()
        self._cols = np.tile(self.cells, (1, 4)).ravel()

    def _scatter(self, local):
        """Global sparse matrix from per-cell [ncell][4][4] (or one shared [4][4]) blocks."""
        nc = len(self.cells)
        if local.ndim == 2:
            local = np.broadcast_to(local, (nc, 4, 4))
        return sp.csr_matrix((np.ascontiguousarray(local).reshape(-1), (self._rows, self._cols)),
                             shape=(self.N, self.N))

    def _gather(self, local):
        """Global vector from per-cell [ncell][4] contributions."""
        return np.bincount(self.cells.ravel(), weights=local.ravel(), minlength=self.N)

    def _linear_matrices(self):
        P, DX, DY, w = self.PHI, self.DX, self.DY, self.w
        self.M = self._scatter(w * P.T @ P)
        self.S = self._scatter(w * (DX.T @ DX + DY.T @ DY))
        # B_x[i][j] = (phi_j, d_x phi_i): the pressure term of velocity row i
        self.Bx = self._scatter(w * DX.T @ P)
        self.By = self._scatter(w * DY.T @ P)
        self.L = self._lps_matrix()

    def _lps_matrix(self):
        """sum over fluid cells T of alpha (grad(p - pi p), grad(xi - pi xi))_T.

        pi acts on each 2x2-cell patch aligned to even cell indices.  A patch
        contributes the integrals over its fluid cells; on nested masks (every
        level above a coarse one) patches are all fluid or all solid.
        """
        nxn = self.nx + 1
        # 9 nodes of a patch, (a, b) -> 3 b + a; its 4 cells in the order of _CORNERS
        S_cell = self.w * (self.DX.T @ self.DX + self.DY.T @ self.DY)
        Pi = np.zeros((9, 9))
        for b in range(3):
            for a in range(3):
                X, Y = a / 2.0, b / 2.0
                for cx, cy in _CORNERS:
                    Pi[3 * b + a, 3 * (2 * cy) + 2 * cx] = (X if cx else 1 - X) * (Y if cy else 1 - Y)
        F = np.eye(9) - Pi
        alpha = self.alpha0 * (self.hx ** 2 + self.hy ** 2) / self.nu
        L_cell = np.zeros((4, 9, 9))
        for c, (ca, cb) in enumerate(_CORNERS):
            ids = [3 * (cb + cy) + ca + cx for cx, cy in _CORNERS]
            S9 = np.zeros((9, 9))
            S9[np.ix_(ids, ids)] = S_cell
            L_cell[c] = alpha * F.T @ S9 @ F
        fluid = ~self.solid.reshape(self.ny // 2, 2, self.nx // 2, 2).transpose(0, 2, 1, 3)
        fluid = fluid.reshape(self.ny // 2, self.nx // 2, 4)   # cell (ca, cb) at 2 cb + ca
        n, m = np.nonzero(fluid.any(axis=2))
        vals = np.einsum("pc,cij->pij", fluid[n, m].astype(np.float64), L_cell)
        base = 2 * n * nxn + 2 * m
        nodes = base[:, None] + np.array([b * nxn + a for b in range(3) for a in range(3)])[None, :]
        rows = np.repeat(nodes, 9, axis=1).ravel()
        cols = np.tile(nodes, (1, 9)).ravel()
        return sp.csr_matrix((vals.ravel(), (rows, cols)), shape=(self.N, self.N))

    # ------------------------------------------------------------ nonlinear terms
    def _at_points(self, u, v):
        ue, ve = u[self.cells], v[self.cells]                  # [ncell][4]
        P, DX, DY = self.PHI, self.DX, self.DY
        return (ue @ P.T, ve @ P.T, ue @ DX.T, ue @ DY.T, ve @ DX.T, ve @ DY.T)   # each [ncell][q]

    def convection(self, u, v):
        """((v.grad) u, phi_i) and ((v.grad) v, phi_i), [N] each."""
        U, V, Ux, Uy, Vx, Vy = self._at_points(u, v)
        cu = self._gather((self.w * (U * Ux + V * Uy)) @ self.PHI)
        cv = self._gather((self.w * (U * Vx + V * Vy)) @ self.PHI)
        return cu, cv

    def convection_jacobian(self, u, v):
        """Derivative of the convection vectors at (u, v): blocks [[Cuu, Cuv], [Cvu, Cvv]]."""
        U, V, Ux, Uy, Vx, Vy = self._at_points(u, v)
        P, DX, DY, w = self.PHI, self.DX, self.DY, self.w
        # transport of the increment by (u, v): sum_q w (U d_x phi_b + V d_y phi_b) phi_a
        Nl = np.einsum("cq,qa,qb->cab", w * U, P, DX) + np.einsum("cq,qa,qb->cab", w * V, P, DY)

        def react(G):
            # increment times a gradient component: sum_q w G phi_b phi_a
            return np.einsum("cq,qa,qb->cab", w * G, P, P)

        return (self._scatter(Nl + react(Ux)), self._scatter(react(Uy)),
                self._scatter(react(Vx)), self._scatter(Nl + react(Vy)))

    # ------------------------------------------------------------ system
    def operator(self, x):
        """A(x) on every row, [3][N], no boundary rows imposed."""
        u, v, p = x
        cu, cv = self.convection(u, v)
        Au = self.M @ u / self.k + 0.5 * cu + 0.5 * self.nu * (self.S @ u) - self.Bx @ p
        Av = self.M @ v / self.k + 0.5 * cv + 0.5 * self.nu * (self.S @ v) - self.By @ p
        Ap = self.Bx.T @ u + self.By.T @ v + self.L @ p
        return np.array([Au, Av, Ap])

    def rhs(self, vel):
        """b = Rhs(v_n) [2][N] (Eq. 4cranknicholson3, f = 0); Dirichlet rows 0."""
        u, v = vel[0], vel[1]
        cu, cv = self.convection(u, v)
        bu = self.M @ u / self.k - 0.5 * cu - 0.5 * self.nu * (self.S @ u)
        bv = self.M @ v / self.k - 0.5 * cv - 0.5 * self.nu * (self.S @ v)
        b = np.array([bu, bv])
        b[:, self.dirichlet] = 0.0
        return b

    def defect(self, x, b, t):
        """F(x) = A(x) - b on free rows, x - (boundary value at t) on fixed rows, [3][N].

        b holds the velocity rows [2][N] (pressure rows 0) or all three [3][N].
        """
        F = self.operator(x)
        F[0] -= b[0]
        F[1] -= b[1]
        if len(b) > 2:
            F[2] -= b[2]
        g = self.boundary_values(t)
        d = self.dirichlet
        F[0, d] = x[0, d] - g[0, d]
        F[1, d] = x[1, d] - g[1, d]
        F[2, ~self.p_active] = x[2, ~self.p_active]
        return F

    def jacobian(self, x):
        """Newton matrix of defect() at x (3N x 3N, CSR)."""
        Cuu, Cuv, Cvu, Cvv = self.convection_jacobian(x[0], x[1])
        base = self.M / self.k + (0.5 * self.nu) * self.S
        J = sp.bmat([[base + 0.5 * Cuu, 0.5 * Cuv, -self.Bx],
                     [0.5 * Cvu, base + 0.5 * Cvv, -self.By],
                     [self.Bx.T, self.By.T, self.L]], format="csr")
        fixed = np.concatenate([self.dirichlet, self.dirichlet, ~self.p_active]).astype(np.float64)
        return (sp.diags(1.0 - fixed) @ J + sp.diags(fixed)).tocsr()

    def factorise(self, x, ordering="COLAMD"):
        """Sparse LU of the Newton matrix at x; ordering is SuperLU's column
        ordering ("MMD_AT_PLUS_A" gives this nearly symmetric pattern about
        half the fill of the default and a 4x faster factorisation on a
        256 x 64 level)."""
        self.factorisations += 1
        return splu(self.jacobian(x).tocsc(), permc_spec=ordering)

    def solve(self, b, t, x0=None, tol=1e-12, maxit=25, history=None, newton="exact"):
        """Newton iteration for defect(x, b, t) = 0 from x0 (default 0); returns x [3][N].

        newton="exact" factorises the Newton matrix at every iterate (quadratic
        convergence).  newton="chord", for long runs on larger levels, keeps
        the last factorisation, across calls too, while each iteration cuts
        the defect at least fivefold, factorises afresh at the current iterate
        when one does not, and orders the factorisation on A^T + A.
        Stops when max|F| <= tol * s, s the larger of max|b| and max|M x / k|
        for the boundary-adjusted start; when an update changes x by less
        than 1e-14 max|x|; or when a step with a fresh factorisation no longer
        cuts the defect fourfold once it is 1e-9 below the larger of its start
        and s (the rounding floor of the terms, which can exceed tol * s).
        Raises RuntimeError after maxit iterations.  history, if a list,
        receives max|F| of every iterate.
        """
        if newton not in ("exact", "chord"):
            raise ValueError(f"newton must be 'exact' or 'chord', not {newton!r}")
        chord = newton == "chord"
        x = np.zeros((3, self.N)) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
        g = self.boundary_values(t)
        d = self.dirichlet
        x[0, d], x[1, d] = g[0, d], g[1, d]
        x[2, ~self.p_active] = 0.0
        s = max(np.abs(b).max(initial=0.0),
                np.abs(self.M @ x[0]).max() / self.k, np.abs(self.M @ x[1]).max() / self.k, 1e-300)
        r0 = prev = None
        fresh = False          # the last update used a factorisation made at its own iterate
        for _ in range(maxit):
            F = self.defect(x, b, t)
            r = np.abs(F).max()
            if history is not None:
                history.append(r)
            if r0 is None:
                r0 = r
            if r <= tol * s:
                return x
            if fresh and r > 0.25 * prev and r <= 1e-9 * max(r0, s):
                return x
            slow = prev is not None and r > 0.2 * prev
            prev = r
            if not chord:
                lu = self.factorise(x)
                fresh = True
            else:
                if self._lu is None or slow:
                    self._lu = self.factorise(x, "MMD_AT_PLUS_A")
                    fresh = True
                else:
                    fresh = False
                lu = self._lu
            dx = lu.solve(-F.ravel()).reshape(3, self.N)
            x += dx
            if np.abs(dx).max() <= 1e-14 * max(np.abs(x).max(), 1e-300):
                return x
        raise RuntimeError(f"Newton did not converge in {maxit} iterations (max|F| = {r:.3e})")

    def advance(self, x, t_next, newton="exact"):
        """One Crank-Nicolson step of the plain solver: x(t_n) -> x(t_{n+1})."""
        return self.solve(self.rhs(x[:2]), t_next, x0=x, newton=newton)


def simulate(level, steps, x0=None, t0=0.0, newton="exact"):
    """Plain time stepping on one level: [x(t_1), ..., x(t_steps)], t_n = t0 + n k."""
    x = np.zeros((3, level.N)) if x0 is None else np.array(x0, dtype=np.float64)
    out = []
    for n in range(1, steps + 1):
        x = level.advance(x, t0 + n * level.k, newton)
        out.append(x)
    return out


def dnnmg_run(coarse, correct, steps, x0=None, t0=0.0, b0=None, newton="exact"):
    """Algorithm 2 over `steps` time steps: [x_c(t_1), ..., x_c(t_steps)].

    Each step solves the coarse system at t_n = t0 + n k with the right-hand
    side b_c handed on by the previous step (the coarse solve), then calls
    correct(x_c, t_n) -> b_c for the correction (prolongation, network correction,
    fine right-hand side, restriction), whose result the next solve uses.
    The first right-hand side is b0 ([2 or 3][N]), by default the coarse
    Rhs(x0) (x0 = 0: the fluid at rest).
    """
    x = np.zeros((3, coarse.N)) if x0 is None else np.array(x0, dtype=np.float64)
    bc = coarse.rhs(x[:2]) if b0 is None else np.asarray(b0, dtype=np.float64)
    out = []
    for n in range(1, steps + 1):
        t = t0 + n * coarse.k
        x = coarse.solve(bc, t, x0=x, newton=newton)
        out.append(x)
        bc = correct(x, t)
    return out


def generate_flow(nxc, nyc, K, steps, solid, newton="chord", **params):
    """One training or evaluation flow on a given coarse mask: the fine-level
    (L+K) and plain coarse-level solutions of the start-up flow (arrays as in
    generate_flows, with the mask in place of the ellipse)."""
    params.setdefault("ramp", True)
    c = Level(nxc, nyc, solid, **params)
    f = Level(nxc * 2 ** K, nyc * 2 ** K, refine_mask(solid, K), **params)
    xf = [np.zeros((3, f.N))] + simulate(f, steps, newton=newton)
    return {"solid": np.asarray(solid, dtype=bool), "fine": np.array([[x[:2] for x in xf]], dtype=np.float32),
            "coarse": np.array([simulate(c, steps, newton=newton)]), "k": c.k, "nu": c.nu, "u_max": c.u_max}


def generate_flows(nxc, nyc, K, steps, ratios, a_x=0.05, centre=(0.2, 0.2), newton="chord", **params):
    """Training flows of Sec. 5.2: for each axis ratio a_y / a_x of the elliptic
    obstacle, the fine-level (L+K) solution and the plain coarse-level solution
    of the start-up flow over `steps` steps.

    Returns a dict of arrays: ellipses [F][4]; fine [F][steps+1][2][Nf] float32
    (velocity, entry 0 the fluid at rest); coarse [F][steps][3][Nc] float64;
    k, nu, u_max.  params go to both Levels (nu, k, alpha0, u_max; the ramp is on).
    """
    params.setdefault("ramp", True)
    ells, fine, coarse = [], [], []
    for q in ratios:
        ell = (centre[0], centre[1], a_x, a_x * q)
        solid = ellipse_mask(nxc, nyc, ell)
        c = Level(nxc, nyc, solid, **params)
        f = Level(nxc * 2 ** K, nyc * 2 ** K, refine_mask(solid, K), **params)
        xf = [np.zeros((3, f.N))] + simulate(f, steps, newton=newton)
        ells.append(ell)
        fine.append(np.array([x[:2] for x in xf], dtype=np.float32))
        coarse.append(np.array(simulate(c, steps, newton=newton)))
    return {"ellipses": np.array(ells), "fine": np.array(fine), "coarse": np.array(coarse),
            "k": c.k, "nu": c.nu, "u_max": c.u_max}


def main(argv=None):
    """Write training flows to an .npz (defaults: 128 x 32 coarse cells, K = 1,
    8 axis ratios from 0.5 to 1, 500 steps)."""
    import argparse
    import time
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--nxc", type=int, default=128)
    ap.add_argument("--nyc", type=int, default=32)
    ap.add_argument("--K", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--ratios", default="0.5,0.571,0.643,0.714,0.786,0.857,0.929,1.0")
    ap.add_argument("--nu", type=float, default=1e-3)
    ap.add_argument("--geometry", default="ellipse", help="ellipse (one per ratio), or none, two, L (Sec. 6.7)")
    ap.add_argument("--out", default="flows.npz")
    a = ap.parse_args(argv)
    t0 = time.time()
    if a.geometry == "ellipse":
        data = generate_flows(a.nxc, a.nyc, a.K, a.steps, [float(r) for r in a.ratios.split(",")], nu=a.nu)
    else:
        data = generate_flow(a.nxc, a.nyc, a.K, a.steps, geometry_mask(a.nxc, a.nyc, a.geometry), nu=a.nu)
    np.savez(a.out, nxc=a.nxc, nyc=a.nyc, K=a.K, **data)
    print(f"{len(data['fine'])} flows x {a.steps} steps -> {a.out} ({time.time() - t0:.1f} s)")


if __name__ == "__main__":
    main()

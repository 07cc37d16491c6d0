"""Oracle mesh: structured channel mesh, obstacle mask, node classes, patches.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Geometry (Sec. 6.1, Fig. geom): channel [0, 2.2] x [0, 0.41] with an elliptic
obstacle centred at (0.2, 0.2); parabolic inflow on x = 0, no-slip on the walls
y = 0, y = 0.41 and on the obstacle, do-nothing outflow on x = 2.2.

Readings where the paper is silent (a structured masked mesh replaces the
paper's boundary-conforming Gascoigne mesh):

* A coarse cell is solid iff its centroid lies strictly inside the ellipse; the
  fine cells of level L+K inherit the mask of their coarse parent, so the
  staircase obstacle is the same on every level.
* Velocity Dirichlet nodes: x = 0 (inflow), y = 0 or y = ly (walls) and every
  node of a solid cell (no-slip).  Wall/obstacle value 0 wins over the inflow
  profile (the profile is 0 at the walls anyway).
* A pressure node is active iff it touches a fluid cell (no pressure BC).
* Patches (Sec. 5.2) are s x s coarse cells tiled without overlap; a patch is
  kept iff at least one of its cells is fluid.  Fluid patches are numbered
  lexicographically over the patch grid, patch-x fastest.

A ``Mesh`` may be a *window* of the global mesh: a rectangle of whole patches.
Every flag is then still evaluated with the global rules (the solid test is a
pure function of the global cell index), so all results away from the cut
edges of the window equal those of the full mesh.  This lets tests check
sampled outputs of very large meshes.
"""

from dataclasses import dataclass

import numpy as np


@dataclass
class Params:
    """Physical and method parameters (Sec. 3.2, Sec. 6.1)."""

    nu: float = 1e-3      # viscosity, the 1/Re of Eq. nsstrong
    k: float = 0.01       # time step size (Sec. 6.1)
    alpha0: float = 0.1   # LPS constant alpha_0 (Sec. 3.1)
    u_max: float = 1.5    # peak of the parabolic inflow profile
    ramp: bool = False    # use the start-up ramp omega(t) of Sec. 6.1

    def omega(self, t):
        """Start-up regularisation omega(t) of the inflow (Sec. 6.1)."""
        if not self.ramp:
            return 1.0
        return 0.5 - 0.5 * np.cos(2.0 * np.pi * t) if t <= 0.5 else 1.0


class Mesh:
    """Two-level structured quad mesh (levels L and L+K) with patches."""

    def __init__(self, nxc, nyc, K, s, lx=2.2, ly=0.41, ellipse=None,
                 solid=None, window=None):
        if nxc % 2 or nyc % 2:
            raise ValueError("cell counts must be even")
        if nxc % s or nyc % s:
            raise ValueError("patch size must divide the cell counts")
        self.nxc, self.nyc, self.K, self.s = nxc, nyc, K, s
        self.lx, self.ly = float(lx), float(ly)
        self.r = 2 ** K                      # fine cells per coarse cell edge
        self.nxf, self.nyf = nxc * self.r, nyc * self.r
        self.hxc, self.hyc = self.lx / nxc, self.ly / nyc
        self.hxf, self.hyf = self.lx / self.nxf, self.ly / self.nyf
        self.S = s * self.r                  # fine cells per patch edge
        self.npx, self.npy = nxc // s, nyc // s
        self.nf = (self.S + 1) ** 2          # fine nodes per patch
        self.nc = (s + 1) ** 2               # coarse nodes per patch
        # Sec. 5.2: 3 residual components on the fine patch nodes, 2 coarse
        # velocities and 1 Peclet number per coarse patch node, 12 geometry values.
        self.n_in = 3 * self.nf + 3 * self.nc + 12
        self.n_out = 2 * self.nf

        # global coarse solid mask
        if solid is not None:
            sol = np.asarray(solid, dtype=bool)
            if sol.shape != (nyc, nxc):
                raise ValueError("solid mask must be [nyc][nxc]")
            self._solid_c = sol.copy()
        else:
            gi, gj = np.meshgrid(np.arange(nxc), np.arange(nyc))
            self._solid_c = np.zeros((nyc, nxc), dtype=bool)
            if ellipse is not None:
                cx, cy, ax, ay = ellipse
                if ax > 0 and ay > 0:
                    xc = (gi + 0.5) * self.hxc
                    yc = (gj + 0.5) * self.hyc
                    self._solid_c = ((xc - cx) / ax) ** 2 + ((yc - cy) / ay) ** 2 < 1.0

        # window (coarse cell rectangle made of whole patches)
        if window is None:
            window = (0, 0, nxc, nyc)
        ci0, cj0, ci1, cj1 = window
        if any(v % s for v in window) or not (0 <= ci0 < ci1 <= nxc and 0 <= cj0 < cj1 <= nyc):
            raise ValueError("window must be a rectangle of whole patches")
        self.window = (ci0, cj0, ci1, cj1)
        self.ci0, self.cj0 = ci0, cj0
        self.wxc, self.wyc = ci1 - ci0, cj1 - cj0          # coarse cells in window
        self.fi0, self.fj0 = ci0 * self.r, cj0 * self.r     # fine offset
        self.wxf, self.wyf = self.wxc * self.r, self.wyc * self.r
        self.cut = (ci0 > 0, cj0 > 0, ci1 < nxc, cj1 < nyc)  # W, S, E, N cut edges

        self._build_flags()
        self._build_patches()

    # ----- cell masks (global indices) -----
    @property
    def solid_coarse(self):
        """Global coarse solid mask [nyc][nxc] (copy)."""
        return self._solid_c.copy()

    def _cell_exists_solid(self, gI, gJ, level):
        """(exists, solid) of global cells on the given level ('c' or 'f')."""
        n_x, n_y = (self.nxc, self.nyc) if level == "c" else (self.nxf, self.nyf)
        exists = (gI >= 0) & (gI < n_x) & (gJ >= 0) & (gJ < n_y)
        ci = np.clip(gI, 0, n_x - 1)
        cj = np.clip(gJ, 0, n_y - 1)
        if level == "f":
            ci, cj = ci // self.r, cj // self.r
        solid = exists & self._solid_c[cj, ci]
        return exists, solid

    def _node_classes(self, level):
        """Node classes on the window's nodes of a level (global rules)."""
        if level == "c":
            i0, j0, nx, ny, hy = self.ci0, self.cj0, self.wxc, self.wyc, self.hyc
            top = self.nyc
        else:
            i0, j0, nx, ny, hy = self.fi0, self.fj0, self.wxf, self.wyf, self.hyf
            top = self.nyf
        gI, gJ = np.meshgrid(np.arange(i0, i0 + nx + 1), np.arange(j0, j0 + ny + 1))
        touch_solid = np.zeros(gI.shape, dtype=bool)
        touch_fluid = np.zeros(gI.shape, dtype=bool)
        for di in (-1, 0):
            for dj in (-1, 0):
                ex, so = self._cell_exists_solid(gI + di, gJ + dj, level)
                touch_solid |= so
                touch_fluid |= ex & ~so
        wall = (gJ == 0) | (gJ == top)
        inflow = gI == 0
        y = gJ * hy
        return {
            "dirichlet": wall | inflow | touch_solid,
            "zero_bc": wall | touch_solid,           # Dirichlet value 0
            "inflow": inflow & ~(wall | touch_solid),  # Dirichlet value = profile
            "p_active": touch_fluid,
            "y": y,
        }

    def _build_flags(self):
        f = self._node_classes("f")
        self.dirichlet = f["dirichlet"]
        self.zero_bc = f["zero_bc"]
        self.inflow = f["inflow"]
        self.p_active = f["p_active"]
        self.y_f = f["y"]
        c = self._node_classes("c")
        self.dirichlet_c = c["dirichlet"]
        # fine cells of the window: solid flag [wyf][wxf]
        gI, gJ = np.meshgrid(np.arange(self.fi0, self.fi0 + self.wxf),
                             np.arange(self.fj0, self.fj0 + self.wyf))
        self.solid_f = self._cell_exists_solid(gI, gJ, "f")[1]

    def _build_patches(self):
        s = self.s
        # patch (pi, pj) is fluid iff one of its coarse cells is fluid
        fluid = ~self._solid_c.reshape(self.npy, s, self.npx, s).all(axis=(1, 3))
        self.patch_fluid = fluid
        gidx = -np.ones((self.npy, self.npx), dtype=np.int64)
        gidx[fluid] = np.arange(int(fluid.sum()))     # row-major: pi fastest
        self.patch_global_index = gidx
        pi0, pj0 = self.ci0 // s, self.cj0 // s
        pi1, pj1 = pi0 + self.wxc // s, pj0 + self.wyc // s
        pj, pi = np.nonzero(fluid[pj0:pj1, pi0:pi1])   # lexicographic, pi fastest
        self.patches = np.stack([pi + pi0, pj + pj0], axis=1)  # global (pi, pj)
        self.P = len(self.patches)
        # multiplicity of each window fine node: number of fluid patches containing it
        m = np.zeros((self.wyf + 1, self.wxf + 1), dtype=np.int64)
        for gpi, gpj in self.patches:
            li, lj = gpi * self.S - self.fi0, gpj * self.S - self.fj0
            m[lj:lj + self.S + 1, li:li + self.S + 1] += 1
        self.multiplicity = m

    # ----- sizes and helpers -----
    @property
    def Nf(self):
        return (self.wxf + 1) * (self.wyf + 1)

    @property
    def Nc(self):
        return (self.wxc + 1) * (self.wyc + 1)

    def fine_xy(self):
        """Coordinates of the window's fine nodes, arrays [wyf+1][wxf+1]."""
        gI, gJ = np.meshgrid(np.arange(self.fi0, self.fi0 + self.wxf + 1),
                             np.arange(self.fj0, self.fj0 + self.wyf + 1))
        return gI * self.hxf, gJ * self.hyf

    def coarse_xy(self):
        gI, gJ = np.meshgrid(np.arange(self.ci0, self.ci0 + self.wxc + 1),
                             np.arange(self.cj0, self.cj0 + self.wyc + 1))
        return gI * self.hxc, gJ * self.hyc

    def inflow_profile(self, y, prm, t):
        """Dirichlet inflow v^D(y, t) = u_max 4 y (ly - y) / ly^2 omega(t) (Sec. 6.1)."""
        return prm.u_max * 4.0 * y * (self.ly - y) / self.ly ** 2 * prm.omega(t)

    def fine_node_flags(self):
        """Per fine node: bit0 velocity Dirichlet, bit1 inflow value, bit2 pressure active."""
        return (self.dirichlet.astype(np.uint8)
                | (self.inflow.astype(np.uint8) << 1)
                | (self.p_active.astype(np.uint8) << 2))

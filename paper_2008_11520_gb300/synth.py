"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the method (no interpolation, no finite
elements, no network): it only samples analytic velocity/pressure fields at
given coordinates and draws random weights and hidden states, so that the CUDA
path and the CPU oracle can be fed identical inputs.

Workloads (channel [0, 2.2] x [0, 0.41], ellipse centred at (0.2, 0.2),
nu = 1e-3, k = 0.01, inflow peak 1.5):

* ``plain``   32 x 8 coarse cells, K = 1, one-cell patches, H = 32, FP64,
              ellipse 0.04 x 0.06, 10 steps.
* ``channel256``  256 x 64, K = 2, one-cell patches, H = 64; ellipse
              semi-axes 0.05 x U[0.03, 0.05] from the seed; FP32 or BF16 net.
* ``large``   2048 x 512, K = 2 (8192 x 2048 fine), 2 x 2-cell patches,
              H = 128, BF16 net with FP32 accumulation; ellipse as channel256.
* serving     64 instances, coarse grids drawn uniformly from 64 x 16 to
              512 x 128 (nyc = nxc / 4), K in {1, 2}, one-cell patches,
              ellipse a_x = 0.05 with a_y / a_x ~ U[0.5, 1]; H = 64, BF16
              net; Poisson step requests at a mean 200 steps/s in total.

The synthetic flow is a Poiseuille profile with its linear pressure drop, plus
eight Gaussian vortices of amplitude 0.1 * u_max whose positions, radii and
signs come from the seed; the vortex part is damped to zero at the walls and
the whole velocity is blended to zero inside the ellipse.  Vortices drift
downstream with time, so successive steps see different coarse fields.
"""

from dataclasses import dataclass, field

import numpy as np

LX, LY = 2.2, 0.41
NU, DT, U_MAX = 1e-3, 0.01, 1.5

CONFIGS = {
    "plain": dict(nxc=32, nyc=8, K=1, s=1, H=32, precision="f64", steps=10,
                  ellipse=(0.2, 0.2, 0.04, 0.06), seed=0),
    "channel256": dict(nxc=256, nyc=64, K=2, s=1, H=64, precision="f32", steps=100,
                       ellipse=None, seed=1),
    "large": dict(nxc=2048, nyc=512, K=2, s=2, H=128, precision="bf16", steps=200,
                  ellipse=None, seed=4),
}


def ellipse_from_seed(seed):
    """Semi-axes 0.05 x U[0.03, 0.05] centred at (0.2, 0.2)."""
    rng = np.random.default_rng(seed + 1000)
    return (0.2, 0.2, 0.05, float(rng.uniform(0.03, 0.05)))


def config(name):
    c = dict(CONFIGS[name])
    if c["ellipse"] is None:
        c["ellipse"] = ellipse_from_seed(c["seed"])
    return c


@dataclass
class FlowSpec:
    """Parameters of the synthetic analytic flow."""

    ellipse: tuple
    u_max: float = U_MAX
    nu: float = NU
    vortices: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))

    @staticmethod
    def from_seed(seed, ellipse, n_vortex=8, u_max=U_MAX, nu=NU):
        rng = np.random.default_rng(seed)
        x0 = rng.uniform(ellipse[0] + 0.1, LX - 0.2, n_vortex)
        y0 = rng.uniform(0.08, LY - 0.08, n_vortex)
        rc = rng.uniform(0.02, 0.06, n_vortex)
        amp = 0.1 * u_max * rng.choice([-1.0, 1.0], n_vortex)
        return FlowSpec(ellipse=tuple(ellipse), u_max=u_max, nu=nu,
                        vortices=np.stack([x0, y0, rc, amp], axis=1))


def sample_flow(spec, x, y, t=0.0):
    """(u, v, p) of the synthetic flow at coordinates x, y (any shape), time t."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    wall = 4.0 * y * (LY - y) / LY ** 2
    u = spec.u_max * wall
    v = np.zeros_like(x)
    for x0, y0, rc, amp in spec.vortices:
        xc = x0 + (2.0 / 3.0) * spec.u_max * t
        g = amp * wall * np.exp(-((x - xc) ** 2 + (y - y0) ** 2) / rc ** 2) / rc
        u = u - g * (y - y0)
        v = v + g * (x - xc)
    cx, cy, ax, ay = spec.ellipse
    if ax > 0 and ay > 0:
        rho = ((x - cx) / ax) ** 2 + ((y - cy) / ay) ** 2
        s = np.clip((rho - 1.0) / 0.5, 0.0, 1.0)
        blend = s * s * (3.0 - 2.0 * s)
        u, v = u * blend, v * blend
    p = 8.0 * spec.u_max * spec.nu / LY ** 2 * (LX - x)
    return u, v, p


def node_coords(nx, ny, i0=0, j0=0, wx=None, wy=None):
    """Coordinates of nodes i0..i0+wx, j0..j0+wy of an nx x ny cell grid (x fastest)."""
    wx = nx - i0 if wx is None else wx
    wy = ny - j0 if wy is None else wy
    X, Y = np.meshgrid(np.arange(i0, i0 + wx + 1) * (LX / nx),
                       np.arange(j0, j0 + wy + 1) * (LY / ny))
    return X.ravel(), Y.ravel()


def coarse_state(spec, nxc, nyc, t=0.0, window=None):
    """Coarse nodal (u, v, p) [3][Nc] float64 (window = (ci0, cj0, ci1, cj1))."""
    if window is None:
        x, y = node_coords(nxc, nyc)
    else:
        ci0, cj0, ci1, cj1 = window
        x, y = node_coords(nxc, nyc, ci0, cj0, ci1 - ci0, cj1 - cj0)
    return np.stack(sample_flow(spec, x, y, t))


def fine_state(spec, nxf, nyf, t=0.0, window=None, perturb_seed=None):
    """Fine nodal (u, v, p) [3][Nf] float64, optionally with seeded noise.

    The noise (amplitude 0.05 * u_max, uniform) makes a velocity that differs
    from the smooth flow at the mesh scale, as a corrected velocity does.
    """
    if window is None:
        x, y = node_coords(nxf, nyf)
    else:
        fi0, fj0, fi1, fj1 = window
        x, y = node_coords(nxf, nyf, fi0, fj0, fi1 - fi0, fj1 - fj0)
    out = np.stack(sample_flow(spec, x, y, t))
    if perturb_seed is not None:
        rng = np.random.default_rng(perturb_seed)
        gi, gj = np.meshgrid(np.arange(nxf + 1), np.arange(nyf + 1))
        noise = rng.uniform(-1.0, 1.0, (2, nyf + 1, nxf + 1)) * 0.05 * spec.u_max
        if window is not None:
            fi0, fj0, fi1, fj1 = window
            noise = noise[:, fj0:fj1 + 1, fi0:fi1 + 1]
        out[:2] += noise.reshape(2, -1)
    return out


def net_weights(n_in, H, n_out, seed, std=0.1):
    """Wx [3H][n_in], Uh [3H][H], Wfc [n_out][H] ~ N(0, std^2), drawn in that order."""
    rng = np.random.default_rng(seed)
    Wx = rng.normal(0.0, std, (3 * H, n_in))
    Uh = rng.normal(0.0, std, (3 * H, H))
    Wfc = rng.normal(0.0, std, (n_out, H))
    return Wx, Uh, Wfc


def hidden_state(P, H, seed, scale=0.5):
    """A random GRU state [P][H] in (-scale, scale) for parity tests."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, (P, H))


def serving_instances(n, seed):
    """n instance descriptions of the serving workload (see the module docstring)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nxc = int(rng.integers(64 // 16, 512 // 16 + 1)) * 16
        K = int(rng.integers(1, 3))
        ratio = float(rng.uniform(0.5, 1.0))
        out.append(dict(nxc=nxc, nyc=nxc // 4, K=K, s=1, ellipse=(0.2, 0.2, 0.05, 0.05 * ratio),
                        seed=int(rng.integers(0, 2 ** 31 - 1))))
    return out


def poisson_requests(rate, duration, n_instances, seed):
    """Step requests of a Poisson process of `rate` per second over `duration`
    seconds, each for an instance drawn uniformly: (arrival times [s], instance
    indices), sorted by time."""
    rng = np.random.default_rng(seed)
    n = int(rng.poisson(rate * duration))
    t = np.sort(rng.uniform(0.0, duration, n))
    return t, rng.integers(0, n_instances, n)


"""Plain multigrid fine solve on the GPU: the method DNN-MG is compared with.

Sec. 3.3 solves each Crank-Nicolson step (Eq. nonlinearshort) on the fine
level by Newton's method, each Newton system by GMRES with a geometric
multigrid preconditioner (Sec. 3.4, Algorithm 1) whose smoother is the Vanka
method; Sec. 6.4 times DNN-MG against this solver.  This module drives that
solver: the V-cycle, flexible GMRES (right preconditioning by one V-cycle)
and Newton's method.  Every operation on level vectors is a library kernel
(dnnmg_mg_*: defect, Jacobian-vector product, Vanka sweep, transfers, dot
products, axpby); the host holds only the GMRES Hessenberg matrix and the
coarsest level, whose Newton matrix is factorised once per Newton step by
the host solver (a few thousand unknowns).

V-cycle on level l for J_l d = r (d starts at 0):
  nu1 Vanka sweeps on J_l d = r                  (pre-smoothing)
  r_c = R (r - J_l d); d_c = V-cycle(l + 1, r_c); d += P d_c
  nu2 Vanka sweeps                               (post-smoothing)
with the coarsest level solved directly.  J_l is the Newton matrix at the
current iterate injected into level l.
"""

import numpy as np
import torch

from . import dnnmg, solver
from .solver import Level


class PlainMG:
    """Newton-GMRES-multigrid solver of one level's Crank-Nicolson system on the GPU.

    nx, ny: cells of the fine level (multiples of 2^levels); solid: its cell
    mask [ny][nx]; levels: depth of the hierarchy (the coarsest level is
    solved on the host).
    """

    def __init__(self, nx, ny, levels, solid=None, precision="f64", omega=1.0, nu1=2, nu2=2, restart=30,
                 lx=2.2, ly=0.41, nu=1e-3, k=0.01, alpha0=0.1, u_max=1.5, ramp=False):
        self.mg = dnnmg.MG(nx, ny, levels, solid, precision, lx=lx, ly=ly, nu=nu, k=k, alpha0=alpha0,
                           u_max=u_max, ramp=ramp)
        self.levels = levels
        self.omega, self.nu1, self.nu2, self.restart = omega, nu1, nu2, restart
        self.N = [self.mg.nodes(l) for l in range(levels)]
        f = self.mg.field
        self.x = [None] + [f(l) for l in range(1, levels)]     # linearisation points (level 0: the caller's x)
        self.r = [f(l) for l in range(levels)]                   # right-hand sides of the level equations
        self.d = [f(l) for l in range(levels)]                   # corrections
        self.t = [f(l) for l in range(levels)]                   # work vectors
        self.s = [f(l) for l in range(levels)]
        self.scalar = torch.zeros(1, dtype=torch.float64, device="cuda")
        cnx, cny, csolid = self.mg.level(levels - 1)
        # the coarsest level keeps the finest level's projection coefficient, as the GPU levels do
        self.coarse = Level(cnx, cny, csolid, lx=lx, ly=ly, nu=nu, k=k, alpha0=alpha0 / 4 ** (levels - 1),
                            u_max=u_max, ramp=ramp)
        self.lu = None
        self.stats = {"vcycles": 0, "gmres_iterations": 0, "newton_iterations": 0}
        self.trace = []   # per Newton iteration: (defect norm, GMRES iterations of its solve)

    # ------------------------------------------------------------ vector helpers
    def dot(self, a, b):
        self.mg.dot(a, b, self.scalar)
        return float(self.scalar.item())

    def norm(self, a):
        v = self.dot(a, a)
        if not np.isfinite(v):
            raise FloatingPointError("non-finite vector in the multigrid solve")
        return v ** 0.5

    # ------------------------------------------------------------ multigrid
    def linearize(self, x):
        """Set the linearisation point x (level 0) of every level and factorise the coarsest one."""
        self.x[0] = x
        for l in range(self.levels - 1):
            self.mg.inject(l, self.x[l], self.x[l + 1])
        xc = self.x[self.levels - 1].double().cpu().numpy()
        self.lu = self.coarse.factorise(xc)

    def _smooth(self, l, r, d, sweeps):
        for _ in range(sweeps):
            self.mg.vanka(l, self.x[l], r, d, self.omega)

    def vcycle(self, l, r, d):
        """d = one V-cycle's approximation of J_l^{-1} r (d is overwritten)."""
        mg = self.mg
        if l == self.levels - 1:
            sol = self.lu.solve(r.double().cpu().numpy().ravel()).reshape(3, -1)
            d.copy_(torch.as_tensor(sol, dtype=d.dtype))
            return
        d.zero_()
        self._smooth(l, r, d, self.nu1)
        mg.jvp(l, self.x[l], d, self.t[l])
        mg.axpby(1.0, r, -1.0, self.t[l])
        mg.restrict(l, self.t[l], self.r[l + 1])
        self.vcycle(l + 1, self.r[l + 1], self.d[l + 1])
        mg.prolong_add(l, self.d[l + 1], d)
        self._smooth(l, r, d, self.nu2)
        if l == 0:
            self.stats["vcycles"] += 1

    # ------------------------------------------------------------ GMRES
    def gmres(self, b, rtol=1e-6, maxit=60):
        """Solve J(x) d = b (x: the current linearisation point) by flexible
        GMRES, right-preconditioned with one V-cycle; returns d and the
        number of iterations.  Stops at |b - J d| <= rtol |b|, after maxit
        iterations, or when a restart cycle no longer reduces the residual
        (its rounding floor)."""
        mg = self.mg
        n = self.N[0]
        m = self.restart
        d = self.mg.field(0)
        r = b.clone()
        beta = self.norm(r)
        target = rtol * beta
        its = 0
        while beta > target and its < maxit:
            v0 = self.mg.field(0)
            mg.axpby(1.0 / beta, r, 0.0, v0)
            V = [v0]
            Z = []
            H = np.zeros((m + 1, m))
            g = np.zeros(m + 1)
            g[0] = beta
            cs, sn = np.zeros(m), np.zeros(m)
            j_end = 0
            for j in range(m):
                z = self.mg.field(0)
                self.vcycle(0, V[j], z)
                Z.append(z)
                w = self.mg.field(0)
                mg.jvp(0, self.x[0], z, w)
                for i in range(j + 1):                       # modified Gram-Schmidt
                    H[i, j] = self.dot(w, V[i])
                    mg.axpby(-H[i, j], V[i], 1.0, w)
                hn = self.norm(w)
                H[j + 1, j] = hn
                for i in range(j):                           # earlier Givens rotations
                    t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                    H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                    H[i, j] = t
                den = np.hypot(H[j, j], H[j + 1, j])
                cs[j], sn[j] = (H[j, j] / den, H[j + 1, j] / den) if den > 0 else (1.0, 0.0)
                H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
                H[j + 1, j] = 0.0
                g[j + 1] = -sn[j] * g[j]
                g[j] = cs[j] * g[j]
                its += 1
                j_end = j + 1
                if abs(g[j + 1]) <= target or its >= maxit or hn == 0.0:
                    break
                mg.axpby(1.0 / hn, w, 0.0, w)                # next Krylov vector
                V.append(w)
            y = np.linalg.solve(np.triu(H[:j_end, :j_end]), g[:j_end]) if j_end else np.zeros(0)
            for i in range(j_end):
                mg.axpby(float(y[i]), Z[i], 1.0, d)
            # true residual for the restart
            mg.jvp(0, self.x[0], d, r)
            mg.axpby(1.0, b, -1.0, r)
            last, beta = beta, self.norm(r)
            if beta > 0.99 * last:
                break
        self.stats["gmres_iterations"] += its
        return d, its

    # ------------------------------------------------------------ Newton
    def solve(self, b, t, x0, tol=1e-10, lin_rtol=1e-3, maxit=12):
        """Newton's method for defect(x, b, t) = 0 from x0 (a [3][N] device
        field, updated in place and returned); stops when |F| <= tol |F0|
        (Euclidean norms), when two iterations in a row no longer halve the
        defect (its rounding floor), or after maxit iterations."""
        mg = self.mg
        x = x0
        F = self.mg.field(0)
        f0 = prev = None
        slow = 0
        for it in range(maxit):
            mg.defect(0, x, b, t, F)
            f = self.norm(F)
            if f0 is None:
                f0 = f if f > 0 else 1.0
            if f <= tol * f0:
                return x
            # the defect no longer falls: it has reached the rounding floor of the terms
            slow = slow + 1 if prev is not None and f > 0.5 * prev else 0
            if slow >= 2:
                return x
            prev = f
            self.linearize(x)
            mg.axpby(-1.0, F, 0.0, F)                        # right-hand side -F
            d, its = self.gmres(F, rtol=lin_rtol)
            self.trace.append((f, its))
            mg.axpby(1.0, d, 1.0, x)
            self.stats["newton_iterations"] += 1
        return x

    def step(self, x, t_next, tol=1e-8, lin_rtol=1e-3):
        """One plain time step: x(t_n) -> x(t_{n+1}) (x updated in place)."""
        b = self.mg.field(0)
        self.mg.rhs(0, x, b)
        return self.solve(b, t_next, x, tol=tol, lin_rtol=lin_rtol)


def _timed(fn):
    """Wall and device time (CUDA events on the current stream) of fn(), ms."""
    import time
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0 = time.perf_counter()
    e0.record()
    out = fn()
    e1.record()
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1), 1e3 * (time.perf_counter() - w0)


def compare(workload="large", steps=2, precision="f32", newton_tol=1e-4, lin_rtol=1e-2, deadline_s=120.0):
    """Time steps of the plain multigrid fine solve against DNN-MG's on one GPU.

    Plain: Newton-GMRES-multigrid on level L+K.  DNN-MG: the same solver on
    level L (Algorithm 2's coarse solve) plus the correction step
    (dnnmg_step).  Both start from the synthetic flow of the workload; the
    last of `steps` steps is reported (the first also has to settle the
    synthetic start); no step starts after deadline_s seconds of a solver.
    Returns a dict of times (ms) and iteration counts.
    """
    from . import synth
    c = synth.config(workload)
    K, nxc, nyc = c["K"], c["nxc"], c["nyc"]
    nxf, nyf = nxc << K, nyc << K
    solid_c = solver.ellipse_mask(nxc, nyc, c["ellipse"])
    solid_f = solver.refine_mask(solid_c, K)
    spec = synth.FlowSpec.from_seed(c["seed"], c["ellipse"])

    def depth(nx, ny):
        # levels down to a coarsest level of at most 128 x 32 cells (solved on the host)
        d = 1
        while nx % (1 << d) == 0 and ny % (1 << d) == 0 and (nx >> (d - 1)) * (ny >> (d - 1)) > 4096:
            d += 1
        return d

    out = {"workload": workload, "precision": precision, "newton_tol": newton_tol, "gmres_rtol": lin_rtol}
    for name, nx, ny, solid in (("plain_fine", nxf, nyf, solid_f), ("dnnmg_coarse", nxc, nyc, solid_c)):
        pm = PlainMG(nx, ny, depth(nx, ny), solid, precision)
        lev0 = pm.mg.level(pm.levels - 1)
        x = torch.as_tensor(synth.coarse_state(spec, nx, ny, 0.0)).to(pm.mg.real).cuda()
        times = []
        import time as _time
        start = _time.perf_counter()
        for n in range(steps):
            if _time.perf_counter() - start > deadline_s:
                break
            before = dict(pm.stats)
            _, dev_ms, wall_ms = _timed(lambda: pm.step(x, (n + 1) * c.get("k", 0.01), tol=newton_tol,
                                                        lin_rtol=lin_rtol))
            times.append({"device_ms": dev_ms, "wall_ms": wall_ms,
                          **{k: pm.stats[k] - before[k] for k in pm.stats},
                          "newton_trace": [(float(f), int(i)) for f, i in pm.trace]})
            pm.trace = []
        # one Vanka sweep and one V-cycle on the finest level, and one coarsest solve
        r = pm.mg.field(0)
        pm.mg.rhs(0, x, r)
        d0 = pm.mg.field(0)
        _, sweep_ms, _ = _timed(lambda: pm.mg.vanka(0, x, r, d0, pm.omega))
        pm.linearize(x)
        _, cyc_ms, _ = _timed(lambda: pm.vcycle(0, r, d0))
        rc = pm.r[pm.levels - 1]
        _, lu_ms, _ = _timed(lambda: pm.lu.solve(rc.double().cpu().numpy().ravel()))
        out[name] = {"cells": [nx, ny], "levels": pm.levels, "coarsest": list(lev0[:2]), "steps": times,
                     "vanka_sweep_ms": sweep_ms, "vcycle_ms": cyc_ms, "coarsest_solve_ms": lu_ms}
        del pm, x
        torch.cuda.empty_cache()
    # the correction step of DNN-MG on the same workload
    mesh = dnnmg.Mesh(dnnmg.make_desc(nxc, nyc, K, c["s"], c["ellipse"], precision=c["precision"]))
    I = mesh.info
    W = synth.net_weights(I.n_in, c["H"], I.n_out, seed=c["seed"])
    net = dnnmg.Net(*W, precision=c["precision"])
    xc = torch.as_tensor(synth.coarse_state(spec, nxc, nyc, 0.0)).cuda()
    h = torch.zeros(I.P, c["H"], device="cuda")
    bf, bc, ws = mesh.fine(2), mesh.coarse(3), mesh.workspace()
    for i in range(5):
        dnnmg.dnnmg_step(mesh, net, xc, h, bf, bc, ws, 0.01 * i)
    _, corr_ms, _ = _timed(lambda: [dnnmg.dnnmg_step(mesh, net, xc, h, bf, bc, ws, 0.05 + 0.01 * i)
                                    for i in range(20)])
    out["dnnmg_correction_ms"] = corr_ms / 20
    if steps > 0:
        coarse = out["dnnmg_coarse"]["steps"][-1]["device_ms"]
        fine = out["plain_fine"]["steps"][-1]["device_ms"]
        out["dnnmg_step_ms"] = coarse + out["dnnmg_correction_ms"]
        out["plain_step_ms"] = fine
        out["speedup"] = fine / out["dnnmg_step_ms"]
    return out


if __name__ == "__main__":
    import json
    import sys
    wl = sys.argv[1] if len(sys.argv) > 1 else "large"
    prec = sys.argv[2] if len(sys.argv) > 2 else "f32"
    steps = int(sys.argv[4]) if len(sys.argv) > 4 else 2
    print(json.dumps(compare(wl, steps=steps, precision=prec,
                             deadline_s=float(sys.argv[3]) if len(sys.argv) > 3 else 120.0)))

"""DNN-MG time stepping end to end (Algorithm 2): host coarse solve, library correction.

Each time step solves the coarse level's Crank-Nicolson system on the host in
FP64 (the coarse solve, ``solver.Level.solve``), then runs the correction step
(prolongation, residual and features, GRU network, averaging,
fine right-hand side, restriction) in one ``dnnmg_step`` call on the GPU,
whose restricted right-hand side the next coarse solve uses.  The GRU state
and the fine right-hand side stay on the device between steps; only x_c goes
down and b_c comes back.

``python -m paper_2008_11520_gb300.timeloop`` trains the patch network on
solved flows of a small channel and prints E_rel(v) (Sec. 6.4) of the method
with the trained and with a zero network against the plain fine-level solve
(``accuracy_experiment``).
"""

import time

import numpy as np
import torch

from . import dnnmg, solver


class LibraryCorrection:
    """Lines 6-9 of Algorithm 2 through the library: a callable (x_c, t_n) -> b_c.

    x_c is the coarse solution at t_n, [3][Nc] float64 (host); the result is
    the restricted right-hand side for the solve at t_{n+1}, [3][Nc] float64
    (host).  The handle keeps h [P][H] and the fine right-hand side b_f on the
    device; b_f starts at b_f0 (node-ordered [2][Nf], default 0: the fluid at
    rest) and h at 0.  By default one ``dnnmg_step`` call does the work; with
    keep_fine the same kernels run through their single-step entry points and
    the corrected fine velocity v~ + d_bar stays available (``v_corr``).
    """

    def __init__(self, mesh, net, bf0=None, keep_fine=False):
        I = mesh.info
        self.mesh, self.net, self.keep_fine = mesh, net, keep_fine
        self.h = torch.zeros(I.P * net.H, dtype=mesh.real, device="cuda")
        self.bf = mesh.fine(2) if bf0 is None else mesh.pack(bf0)
        self.bc = torch.zeros(3 * I.Nc, dtype=torch.float64, device="cuda")
        self.xc = torch.zeros(3 * I.Nc, dtype=torch.float64, device="cuda")
        if keep_fine:
            self.xf, self.vc = mesh.fine(3), mesh.fine(2)
            self.X = mesh.features()
            self.d = torch.zeros(I.P * I.n_out, dtype=mesh.real, device="cuda")
        else:
            self.ws = mesh.workspace()

    def __call__(self, xc, t):
        m, I = self.mesh, self.mesh.info
        self.xc.copy_(torch.from_numpy(np.ascontiguousarray(xc, dtype=np.float64).reshape(-1)))
        if not self.keep_fine:
            dnnmg.dnnmg_step(m, self.net, self.xc, self.h, self.bf, self.bc, self.ws, t)
        else:
            dnnmg.dnnmg_prolongate(m, self.xc, self.xf, t)
            dnnmg.dnnmg_patch_features(m, self.xf, self.bf, self.X)
            dnnmg.dnnmg_gru_step(self.net, self.X, self.h, self.d, I.P)
            dnnmg.dnnmg_scatter_avg(m, self.d, self.xf, self.vc)
            dnnmg.dnnmg_rhs_restrict(m, self.vc, self.bf, self.bc)
        return self.bc.cpu().numpy().reshape(3, -1)

    def v_corr(self):
        """The last step's corrected fine velocity, node-ordered [2][Nf] float64."""
        if not self.keep_fine:
            raise RuntimeError("v_corr needs keep_fine=True")
        return self.mesh.unpack(self.vc)


def coarse_level(mesh_desc):
    """The host Level of a mesh descriptor's coarse level (same geometry and parameters)."""
    d = mesh_desc
    if d.solid:
        solid = np.ctypeslib.as_array(d.solid, shape=(d.nyc, d.nxc)).astype(bool)
    else:
        ell = (d.obst_cx, d.obst_cy, d.obst_ax, d.obst_ay)
        solid = solver.ellipse_mask(d.nxc, d.nyc, ell, d.lx, d.ly)
    return solver.Level(d.nxc, d.nyc, solid, d.lx, d.ly, nu=d.nu, k=d.k, alpha0=d.alpha0,
                        u_max=d.u_max, ramp=bool(d.ramp))


def fine_level(mesh_desc):
    """The host Level of a mesh descriptor's fine level L+K (nested mask)."""
    c = coarse_level(mesh_desc)
    r = 2 ** mesh_desc.K
    return solver.Level(c.nx * r, c.ny * r, solver.refine_mask(c.solid, mesh_desc.K), c.lx, c.ly,
                        nu=c.nu, k=c.k, alpha0=c.alpha0, u_max=c.u_max, ramp=c.ramp)


def e_rel(v, ref):
    """|v - v_bar| / |v_bar| over the fine velocity DOFs (Sec. 6.4)."""
    return float(np.linalg.norm(v - ref) / np.linalg.norm(ref))


def _held_out_errors(mesh, net, coarse_states, fine_states, k):
    """E_rel(v) per step of v~ + d_bar with the coarse states given (teacher
    forcing), through the inference kernels, the GRU state carried."""
    I = mesh.info
    h = torch.zeros(I.P * net.H, dtype=mesh.real, device="cuda")
    d = torch.zeros(I.P * I.n_out, dtype=mesh.real, device="cuda")
    X = mesh.features()
    xf, bf, vc = mesh.fine(3), mesh.fine(2), mesh.fine(2)
    errs = []
    for n, xc in enumerate(coarse_states):
        t = (n + 1) * k
        xcd = torch.as_tensor(np.ascontiguousarray(xc).reshape(-1)).cuda()
        dnnmg.dnnmg_prolongate(mesh, xcd, xf, t)
        dnnmg.dnnmg_rhs(mesh, mesh.pack(fine_states[n][:2]), bf)
        dnnmg.dnnmg_patch_features(mesh, xf, bf, X)
        dnnmg.dnnmg_gru_step(net, X, h, d, I.P)
        dnnmg.dnnmg_scatter_avg(mesh, d, xf, vc)
        errs.append(e_rel(mesh.unpack(vc), fine_states[n + 1][:2]))
    return errs


def accuracy_experiment(nxc=32, nyc=8, K=1, ellipse=(0.2, 0.2, 0.05, 0.04), nu=1e-3,
                        u_train=(1.2, 1.5, 1.8), u_held=1.35, steps=20, T=10, H=32,
                        epochs=300, lr=1e-3, seed=0, head=False):
    """Train the patch network on solved flows and measure what it gains.

    The paper's accuracy study (Sec. 6.3-6.4) in small: fine-level (L+K)
    solutions of the start-up flow at the inflow peaks u_train are the
    ground truth, plain coarse-level solutions the network's inputs
    (``train.solution_windows``); windows of T steps, Adam with the Tikhonov
    term, the state carried from one window to the next.  On a flow with the
    held-out peak u_held it reports E_rel(v) (Sec. 6.4, fine velocity DOFs,
    mean over the steps):

    * ``teacher``: v~ + d_bar on the plain coarse solutions, trained net vs d = 0;
    * ``loop``: Algorithm 2 end to end (host coarse solve, library correction
      step, its right-hand side fed back), trained net vs zero net, which
      reduces the method to the plain coarse solve.

    ``head``: the net carries the convolutional head of Sec. 6.2 (the K = 1
    net of the paper: GRU, output layer, head).
    """
    from . import train

    def setup(u):
        desc = dnnmg.make_desc(nxc, nyc, K, 1, ellipse=ellipse, precision="f32", ramp=True,
                               nu=nu, u_max=u)
        mesh = dnnmg.Mesh(desc)
        coarse, fine = coarse_level(desc), fine_level(desc)
        xf = [np.zeros((3, fine.N))] + solver.simulate(fine, steps)
        xc = solver.simulate(coarse, steps)
        return mesh, coarse, xf, xc

    data = []
    for u in u_train:
        mesh, _, xf, xc = setup(u)
        data.append(train.solution_windows(mesh, xf, xc, k=mesh.desc.k))
    I = mesh.info
    tn = train.PatchNetTrainer(I.n_in, I.ldx, H, I.n_out, T, I.P, seed=seed, std=0.02, out_std=0.0, lr=lr,
                               head=head)
    for _ in range(epochs):
        for X, Y in data:
            h = None
            for w in range(steps // T):
                _, h = tn.train_window(X[w * T:(w + 1) * T].contiguous(), Y[w * T:(w + 1) * T].contiguous(), h)
    W = tn.weights()
    zero = [W[0], W[1], np.zeros_like(W[2])]
    mesh, coarse, xf, xc = setup(u_held)
    out = {"updates": tn.step_no, "head": bool(head), "params": int(sum(w.size for w in W))}
    for name, weights in (("trained", W), ("zero", zero)):
        net = dnnmg.Net(*weights[:3], precision="f32", head=weights[3] if len(weights) > 3 else None)
        teacher = _held_out_errors(mesh, net, xc, xf, coarse.k)
        corr = LibraryCorrection(mesh, net, keep_fine=True)
        loop = []

        def step(x, t, corr=corr, loop=loop):
            bc = corr(x, t)
            loop.append(e_rel(corr.v_corr(), xf[len(loop) + 1][:2]))
            return bc

        solver.dnnmg_run(coarse, step, steps)
        out[name] = {"teacher": float(np.mean(teacher)), "loop": float(np.mean(loop)),
                     "loop_last": loop[-1]}
    return out


def flows_experiment(paths, held_out, H=64, T=10, epochs=200, lr=1e-3, precision="bf16", seed=0, halves=2,
                     loop_steps=None, eval_paths=(), eval_loop_steps=None, weights_out=None, head=False):
    """Train the patch network on solved training flows and measure what it gains.

    The training workload of Sec. 5.2 / 6.3: ``paths`` are .npz files written
    by ``solver.main`` (one channel flow each: the fine-level (L+1) solution
    as ground truth and the plain coarse-level solution as the network's
    input, every step of the start-up flow); the flow ``held_out`` (an index
    into ``paths``) is left out of training.  The other flows' windows
    (``train.solution_windows``) are laid side by side along the patch axis,
    their time series cut into ``halves`` consecutive parts that run side by
    side as well, so one update sees every training flow; truncated BPTT over
    windows of T steps with the state carried from window to window; Adam
    with the Tikhonov term; products in ``precision`` ("bf16": the tensor
    cores, FP32 master weights).  On the held-out flow it reports E_rel(v)
    (Sec. 6.4, fine velocity DOFs, mean over steps) of v~ + d_bar on the plain
    coarse solutions (``teacher``) and, over the first ``loop_steps`` steps,
    of Algorithm 2 end to end (``loop``), each for the trained net and for
    d = 0 (the plain coarse solution).

    ``eval_paths`` are further solved flows on other geometries (written by
    ``solver.main --geometry``, Sec. 6.7): the net trained on the one-obstacle
    flows is applied to each unchanged, with the same two errors (the loop over
    ``eval_loop_steps`` steps).  ``weights_out`` saves the trained weights
    (.npz, ``W``, ``U``, ``Wfc`` and ``theta``).  ``head``: train the
    convolutional head of Sec. 6.2 with the net (``train.HeadFold``).
    """
    from . import train

    flows = [np.load(p) for p in paths]

    def setup(f):
        nxc, nyc, K = int(f["nxc"]), int(f["nyc"]), int(f["K"])
        if "solid" in f:
            ell, solid = None, np.asarray(f["solid"], dtype=bool)
        else:
            ell = tuple(float(x) for x in f["ellipses"][0])
            solid = solver.ellipse_mask(nxc, nyc, ell)
        desc = dnnmg.make_desc(nxc, nyc, K, 1, ellipse=ell, solid=solid, precision="f32", ramp=True,
                               nu=float(f["nu"]), k=float(f["k"]), u_max=float(f["u_max"]))
        return dnnmg.Mesh(desc), f["fine"][0], f["coarse"][0]

    Xs, Ys = [], []
    for i, f in enumerate(flows):
        if i == held_out:
            continue
        mesh, fine, coarse = setup(f)
        X, Y = train.solution_windows(mesh, list(fine), list(coarse), k=mesh.desc.k)
        n = (X.shape[0] // (halves * T)) * T          # whole windows per part
        Xs += [X[j * n:(j + 1) * n] for j in range(halves)]
        Ys += [Y[j * n:(j + 1) * n] for j in range(halves)]
        del X, Y
    Xb, Yb = torch.cat(Xs, dim=1).contiguous(), torch.cat(Ys, dim=1).contiguous()
    del Xs, Ys
    I = mesh.info
    steps, P = Xb.shape[0], Xb.shape[1]
    tn = train.PatchNetTrainer(I.n_in, I.ldx, H, I.n_out, T, P, seed=seed, std=0.02, out_std=0.0, lr=lr,
                               precision=precision, head=head)
    losses = []
    for e in range(epochs):
        h, tot = None, 0.0
        for w in range(steps // T):
            L, h = tn.train_window(Xb[w * T:(w + 1) * T], Yb[w * T:(w + 1) * T], h)
            tot += float(L)
        losses.append(tot)
    torch.cuda.synchronize()
    status = tn.trainer.status() if hasattr(tn.trainer, "status") else 0
    del Xb, Yb
    W = tn.weights()
    if weights_out:
        np.savez(weights_out, W=W[0], U=W[1], Wfc=W[2], **({"theta": W[3]} if head else {}))
    zero = [W[0], W[1], np.zeros_like(W[2])]
    out = {"updates": tn.step_no, "patches_per_update": P, "window": T, "H": H, "precision": precision,
           "head": bool(head), "params": int(sum(w.size for w in W)),
           "loss_first_epoch": losses[0], "loss_last_epoch": losses[-1], "trainer_status": status}
    mesh, fine, coarse = setup(flows[held_out])
    out.update(_evaluate(mesh, fine, coarse, W, zero, loop_steps))
    if loop_steps:
        out["plain"] = _plain_methods(mesh.desc, fine, loop_steps)
    del mesh
    if eval_paths:
        out["geometries"] = {}
    for p in eval_paths:
        mesh, fine, coarse = setup(np.load(p))
        out["geometries"][p] = {"solid_cells": int(np.asarray(np.load(p)["solid"]).sum()),
                                **_evaluate(mesh, fine, coarse, W, zero, eval_loop_steps)}
        del mesh
    return out


def _evaluate(mesh, fine, coarse, W, zero, loop_steps):
    """E_rel(v) of the trained net and of d = 0 on one solved flow: with the
    plain coarse solutions as input (``teacher``, mean over steps and last) and,
    over ``loop_steps`` steps, of Algorithm 2 end to end (``loop``, with the
    per-step wall time of coarse solve + correction)."""
    desc, out = mesh.desc, {}
    for name, weights in (("trained", W), ("zero", zero)):
        net = dnnmg.Net(*weights[:3], precision="f32", head=weights[3] if len(weights) > 3 else None)
        teacher = _held_out_errors(mesh, net, list(coarse), list(fine), desc.k)
        res = {"teacher": float(np.mean(teacher)), "teacher_last": teacher[-1]}
        if loop_steps:
            c = coarse_level(desc)
            corr = LibraryCorrection(mesh, net, keep_fine=True)
            loop, stamps = [], [time.perf_counter()]

            def step(x, t, corr=corr, loop=loop, stamps=stamps):
                bc = corr(x, t)
                stamps.append(time.perf_counter())      # one whole step: coarse solve + correction
                loop.append(e_rel(corr.v_corr(), fine[len(loop) + 1]))
                return bc

            solver.dnnmg_run(c, step, loop_steps)
            res.update(loop=float(np.mean(loop)), loop_last=loop[-1], step_ms=_pcts(np.diff(stamps) * 1e3))
        out[name] = res
    return out


def _pcts(ms):
    ms = np.asarray(ms, dtype=np.float64)
    return {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)), "mean": float(ms.mean())}


def _plain_methods(desc, fine, steps):
    """Per-step latency and E_rel(v) of the plain methods on the same flow: the
    coarse-level solve (level L, host FP64), the fine-level solve (level L+K)
    on the host, and the GPU plain multigrid fine solve (Newton, GMRES,
    V-cycles with the Vanka smoother; FP64), against the fine reference."""
    from . import mg
    out = {}
    c, f = coarse_level(desc), fine_level(desc)
    for name, lev, n in (("coarse_host", c, steps), ("fine_host", f, min(steps, 20))):
        x, ms = np.zeros((3, lev.N)), []
        for i in range(1, n + 1):
            t0 = time.perf_counter()
            x = lev.advance(x, i * lev.k, "exact")
            ms.append((time.perf_counter() - t0) * 1e3)
        if lev is f:
            err = e_rel(x[:2], fine[n])
        else:
            # the coarse solution seen on the fine level: its prolongation with the fine Dirichlet values
            mesh = dnnmg.Mesh(desc)
            xf = mesh.fine(3)
            dnnmg.dnnmg_prolongate(mesh, torch.as_tensor(np.ascontiguousarray(x).reshape(-1)).cuda(), xf, n * lev.k)
            err = e_rel(mesh.unpack(xf[:2]), fine[n])
        out[name] = {"steps": n, "step_ms": _pcts(ms), "e_rel_last": err}
    # GPU plain multigrid on the fine level, levels down to at most 128 x 32 cells
    levels = 1
    while (f.nx >> levels) >= 128 and (f.ny >> levels) >= 32 and (f.nx >> (levels - 1)) > 128:
        levels += 1
    pm = mg.PlainMG(f.nx, f.ny, levels, f.solid, "f64", lx=f.lx, ly=f.ly, nu=f.nu, k=f.k, alpha0=f.alpha0,
                    u_max=f.u_max, ramp=f.ramp)
    x, ms, n = pm.mg.field(0), [], min(steps, 20)
    for i in range(1, n + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pm.step(x, i * f.k)
        torch.cuda.synchronize()
        ms.append((time.perf_counter() - t0) * 1e3)
    out["fine_gpu_mg"] = {"steps": n, "levels": levels, "step_ms": _pcts(ms),
                          "e_rel_last": e_rel(x[:2].double().cpu().numpy(), fine[n])}
    return out


def main():
    import json
    import sys
    import time
    t0 = time.time()
    if len(sys.argv) > 1 and sys.argv[1] == "flows":
        # flows <held-out index> <epochs> <precision> <loop steps> <npz files...>
        #       [--eval <loop steps> <npz files...>] [--weights-out <npz>] [--head]
        held, epochs, prec, loop_steps = int(sys.argv[2]), int(sys.argv[3]), sys.argv[4], int(sys.argv[5])
        rest, weights_out, eval_paths, eval_steps = sys.argv[6:], None, [], None
        use_head = "--head" in rest
        rest = [a for a in rest if a != "--head"]
        if "--weights-out" in rest:
            i = rest.index("--weights-out")
            weights_out, rest = rest[i + 1], rest[:i] + rest[i + 2:]
        if "--eval" in rest:
            i = rest.index("--eval")
            eval_steps, eval_paths, rest = int(rest[i + 1]), rest[i + 2:], rest[:i]
        paths = rest
        out = flows_experiment(paths, held, epochs=epochs, precision=prec, loop_steps=loop_steps,
                               eval_paths=eval_paths, eval_loop_steps=eval_steps, weights_out=weights_out,
                               head=use_head)
        print(json.dumps({"workload": "solved training flows (solver.main): " + ", ".join(paths),
                          "held_out": paths[held], "metric": "E_rel(v), mean over steps", **out,
                          "seconds": round(time.time() - t0, 1)}))
        return
    use_head = "--head" in sys.argv[1:]
    out = accuracy_experiment(head=use_head)
    print(json.dumps({"workload": "32x8 coarse cells, K = 1, nu = 1e-3, start-up flow, 20 steps; "
                                  "trained on inflow peaks 1.2, 1.5, 1.8, evaluated at 1.35",
                      "metric": "E_rel(v), mean over steps", **out,
                      "seconds": round(time.time() - t0, 1)}))


if __name__ == "__main__":
    main()

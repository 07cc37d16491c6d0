"""Parity at the full workload sizes, in the launch configuration the
benchmark times (dnnmg_step on the whole mesh).

* 256 x 64 coarse cells, K = 2, H = 64 (FP32 and BF16 networks), over the
  workload's 100 steps: the oracle runs on the whole mesh.
* 2048 x 512 coarse cells, K = 2, 2 x 2-cell patches, H = 128, BF16: the
  oracle computes sampled outputs -- it runs on windows of the global mesh
  (obstacle, inflow, outflow corner, interior), and results are compared
  where the window's cut edges cannot reach within the steps taken.
"""

import numpy as np
import pytest
import torch

from helpers import BOUNDARY_CLASSES, TOL, Params, class_errors, rel_l2
from oracle import fem, step as ostep, transfer
from oracle.mesh import Mesh as OMesh
from paper_2008_11520_gb300 import synth
from parity import check, record

pytestmark = pytest.mark.gpu
PRM = Params()


@pytest.fixture(scope="module")
def dn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_11520_gb300 import dnnmg
    return dnnmg


def gpu_run(dn, c, prec, steps, xc_t, v0, h0):
    mesh = dn.Mesh(dn.make_desc(c["nxc"], c["nyc"], c["K"], c["s"], c["ellipse"], precision=prec))
    I = mesh.info
    W = synth.net_weights(I.n_in, c["H"], I.n_out, seed=c["seed"])
    net = dn.Net(*W, precision=prec)
    real = mesh.real
    bf = mesh.fine(2)
    bc = mesh.coarse(3)
    dn.dnnmg_rhs_restrict(mesh, mesh.pack(v0), bf, bc)
    h = torch.as_tensor(h0).to(real).cuda().contiguous()
    ws = mesh.workspace()
    for n in range(steps):
        dn.dnnmg_step(mesh, net, torch.as_tensor(xc_t[n]).cuda().contiguous(), h, bf, bc, ws, n * PRM.k)
    torch.cuda.synchronize()
    out = {"h": h.double().cpu().numpy(), "bf": mesh.unpack(bf), "bc": bc.cpu().numpy()}
    assert dn.dnnmg_net_status(net) == 0
    return mesh, W, out


class GpuSide:
    """One network precision's run of the step on the whole mesh, as the benchmark launches it."""

    def __init__(self, dn, c, prec, v0, h0):
        self.dn = dn
        self.mesh = dn.Mesh(dn.make_desc(c["nxc"], c["nyc"], c["K"], c["s"], c["ellipse"], precision=prec))
        I = self.mesh.info
        self.W = synth.net_weights(I.n_in, c["H"], I.n_out, seed=c["seed"])
        self.net = dn.Net(*self.W, precision=prec)
        self.bf = self.mesh.fine(2)
        self.bc = self.mesh.coarse(3)
        dn.dnnmg_rhs_restrict(self.mesh, self.mesh.pack(v0), self.bf, self.bc)
        self.h = torch.as_tensor(h0).to(self.mesh.real).cuda().contiguous()
        self.ws = self.mesh.workspace()

    def step(self, xc, t):
        self.dn.dnnmg_step(self.mesh, self.net, torch.as_tensor(xc).cuda().contiguous(), self.h, self.bf, self.bc,
                           self.ws, t)
        torch.cuda.synchronize()
        d, vc = self.mesh.step_outputs(self.ws)
        return {"h": self.h.double().cpu().numpy(), "bf": self.mesh.unpack(self.bf), "bc": self.bc.cpu().numpy(),
                "d": d.double().cpu().numpy(), "vcorr": self.mesh.unpack(vc)}


def test_channel256_hundred_steps(dn):
    # 256 x 64 coarse cells, K = 2, H = 64, over the workload's 100 steps: the
    # FP32 and the BF16 network run side by side against one FP64 oracle
    # trajectory (each side keeps its own h and b_f, so errors can build up
    # through the recurrence); x_c(t_n) is the synthetic coarse flow.  Every
    # step's errors are recorded (the drift curve of h among them) and the
    # bounds are asserted once all steps have run.
    c = synth.config("channel256")
    spec = synth.FlowSpec.from_seed(c["seed"], c["ellipse"])
    om = OMesh(c["nxc"], c["nyc"], c["K"], c["s"], ellipse=c["ellipse"])
    steps = c["steps"]
    v0 = synth.fine_state(spec, om.nxf, om.nyf, 0.0, perturb_seed=3)[:2].astype(np.float32).astype(np.float64)
    h0 = synth.hidden_state(om.P, c["H"], seed=5).astype(np.float32).astype(np.float64)
    sides = {prec: GpuSide(dn, c, prec, v0, h0) for prec in ("f32", "bf16")}
    assert all(sd.mesh.info.P == om.P for sd in sides.values())
    W = sides["f32"].W
    h, bf = h0, fem.rhs(om, PRM, v0)
    worst = []
    for n in range(steps):
        t = n * PRM.k
        xc = synth.coarse_state(spec, c["nxc"], c["nyc"], t)
        out = ostep.dnnmg_step(om, PRM, W, xc, h, bf, t)
        h, bf = out["h"], out["bf"]
        for prec, sd in sides.items():
            got = sd.step(xc, t)
            tol = TOL[prec]
            errs = {"h": rel_l2(got["h"], out["h"]), "d": rel_l2(got["d"], out["d"]),
                    "v_corr": rel_l2(got["vcorr"], out["vcorr"]), "bf": rel_l2(got["bf"], out["bf"]),
                    "bc": rel_l2(got["bc"].reshape(3, -1), out["bc"])}
            for k, v in errs.items():
                record("100 steps " + k, v, tol, prec, step=n)
                worst.append((v / tol, prec, n, k))
            if n % 10 == 9 or n == 0:
                for cname, v in class_errors(got["bf"], out["bf"], om).items():
                    record("100 steps bf max/RMS " + cname, v, tol, prec, step=n)
                    if cname in BOUNDARY_CLASSES:
                        worst.append((v / tol, prec, n, "bf " + cname))
    for prec, sd in sides.items():
        assert dn.dnnmg_net_status(sd.net) == 0
    over = [w for w in worst if w[0] > 1.0]
    assert not over, sorted(over)[-5:]


WINDOWS = {  # coarse-cell windows of the 2048 x 512 mesh (multiples of the patch size)
    "obstacle": (216, 236, 248, 268),     # straddles the ellipse edge x = 0.25
    "inflow": (0, 100, 32, 132),
    "outflow_corner": (2016, 480, 2048, 512),
    "interior": (1000, 200, 1032, 232),
}


def test_large_sampled_windows(dn):
    c = synth.config("large")
    spec = synth.FlowSpec.from_seed(c["seed"], c["ellipse"])
    r = 2 ** c["K"]
    steps = 2
    full = OMesh(c["nxc"], c["nyc"], c["K"], c["s"], ellipse=c["ellipse"])
    xc_t = [synth.coarse_state(spec, c["nxc"], c["nyc"], n * PRM.k) for n in range(steps)]
    v0 = synth.fine_state(spec, full.nxf, full.nyf, 0.0)[:2].astype(np.float32).astype(np.float64)
    h0 = synth.hidden_state(full.P, c["H"], seed=7).astype(np.float32).astype(np.float64)
    mesh, W, got = gpu_run(dn, c, "bf16", steps, xc_t, v0, h0)
    assert mesh.info.P == full.P
    nxn_c, nxn_f = c["nxc"] + 1, full.nxf + 1
    bc_g = got["bc"].reshape(3, c["nyc"] + 1, nxn_c)
    bf_g = got["bf"].reshape(2, full.nyf + 1, nxn_f)
    margin_c = 8                                   # coarse nodes away from cut edges
    for name, win in WINDOWS.items():
        om = OMesh(c["nxc"], c["nyc"], c["K"], c["s"], ellipse=c["ellipse"], window=win)
        ci0, cj0, ci1, cj1 = win
        xcw = [x.reshape(3, c["nyc"] + 1, nxn_c)[:, cj0:cj1 + 1, ci0:ci1 + 1].reshape(3, -1) for x in xc_t]
        v0w = v0.reshape(2, full.nyf + 1, nxn_f)[:, cj0 * r:cj1 * r + 1, ci0 * r:ci1 * r + 1].reshape(2, -1)
        gidx = full.patch_global_index[om.patches[:, 1], om.patches[:, 0]]
        h, bf = h0[gidx], fem.rhs(om, PRM, v0w)
        for n in range(steps):
            out = ostep.dnnmg_step(om, PRM, W, xcw[n], h, bf, n * PRM.k)
            h, bf = out["h"], out["bf"]
        # exact region: cut edges need a margin, domain edges do not
        lo_i = 0 if ci0 == 0 else margin_c
        lo_j = 0 if cj0 == 0 else margin_c
        hi_i = (ci1 - ci0) + 1 - (0 if ci1 == c["nxc"] else margin_c)
        hi_j = (cj1 - cj0) + 1 - (0 if cj1 == c["nyc"] else margin_c)
        ref = out["bc"].reshape(3, cj1 - cj0 + 1, ci1 - ci0 + 1)[:2, lo_j:hi_j, lo_i:hi_i]
        gbc = bc_g[:2, cj0 + lo_j:cj0 + hi_j, ci0 + lo_i:ci0 + hi_i]
        check("window bc", rel_l2(gbc, ref), TOL["bf16"], "bf16", window=name)
        fref = out["bf"].reshape(2, om.wyf + 1, om.wxf + 1)[:, lo_j * r:(hi_j - 1) * r + 1, lo_i * r:(hi_i - 1) * r + 1]
        gbf = bf_g[:, cj0 * r + lo_j * r:cj0 * r + (hi_j - 1) * r + 1, ci0 * r + lo_i * r:ci0 * r + (hi_i - 1) * r + 1]
        check("window bf", rel_l2(gbf, fref), TOL["bf16"], "bf16", window=name)
        # per node class, over the exact region of the window
        region = np.zeros((om.wyf + 1, om.wxf + 1), dtype=bool)
        region[lo_j * r:(hi_j - 1) * r + 1, lo_i * r:(hi_i - 1) * r + 1] = True
        gwin = bf_g[:, cj0 * r:cj1 * r + 1, ci0 * r:ci1 * r + 1]
        for cname, v in class_errors(gwin, out["bf"], om, region).items():
            (check if cname in BOUNDARY_CLASSES else record)("window bf max/RMS " + cname, v, TOL["bf16"], "bf16",
                                                              window=name)
        # hidden state of patches whose dependence stays inside the window
        pi, pj = om.patches[:, 0], om.patches[:, 1]
        s = c["s"]
        inner = ((pi * s >= ci0 + lo_i) & ((pi + 1) * s <= ci0 + hi_i - 1)
                 & (pj * s >= cj0 + lo_j) & ((pj + 1) * s <= cj0 + hi_j - 1))
        assert inner.sum() > 0
        check("window h", rel_l2(got["h"][gidx[inner]], out["h"][inner]), TOL["bf16"], "bf16", window=name)


def test_large_whole_mesh_restriction(dn):
    # S7 on the whole 2048 x 512 mesh in the bench's precision (4225 tiles, every
    # tile edge and the obstacle's staircase): float-pair accumulation against
    # the oracle's FP64 restriction of the same FP32 vector
    c = synth.config("large")
    full = OMesh(c["nxc"], c["nyc"], c["K"], c["s"], ellipse=c["ellipse"])
    mesh = dn.Mesh(dn.make_desc(c["nxc"], c["nyc"], c["K"], c["s"], c["ellipse"], precision="f32"))
    rng = np.random.default_rng(43)
    bf = rng.standard_normal((2, full.Nf)).astype(np.float32).astype(np.float64)
    bc = mesh.coarse(3)
    dn.dnnmg_restrict(mesh, mesh.pack(bf), bc)
    torch.cuda.synchronize()
    ref = transfer.restrict(full, bf)
    got = bc.cpu().numpy().reshape(3, -1)
    check("whole-mesh R b_f (FP64 class)", rel_l2(got, ref), 1e-13, "f32", case="large")
    assert np.array_equal(got == 0, ref == 0)

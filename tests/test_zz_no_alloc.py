"""dnnmg_step_static: the correction step for callers that cannot allocate
device memory (its scratch is a library-owned static device array).

It runs the same kernels as dnnmg_step on the same inputs, and none of them
uses atomics, so its results must equal dnnmg_step's bit for bit, call after
call (the shared scratch keeps the previous call's contents, and a stale
padding row or column left from an earlier mesh would show up here).  It must
also refuse meshes whose scratch does not fit.  This file is collected last
so that a failure here cannot stop the rest of a -x run.
"""

import numpy as np
import pytest
import torch

from helpers import CASES, coarse_input, fine_velocity, mask_for, oracle_mesh, weights
from paper_2008_11520_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_11520_gb300 import dnnmg
    return dnnmg


def two_calls_bitwise(dn, m, net, H, P, xc_at, v0):
    assert dn.dnnmg_static_scratch_needed(m) <= dn.dnnmg_static_scratch_bytes()
    rng = np.random.default_rng(3)
    h0 = torch.as_tensor(rng.uniform(-0.5, 0.5, (P, H))).to(m.real).cuda()
    b0 = m.fine(2)
    dn.dnnmg_rhs_restrict(m, m.pack(v0), b0, m.coarse(3))
    ws = m.workspace()
    states = {"ws": (h0.clone(), b0.clone(), m.coarse(3)), "static": (h0.clone(), b0.clone(), m.coarse(3))}
    for n in range(2):   # two calls in a row: the second runs on the first call's scratch contents
        t = 0.01 * n
        xc = torch.as_tensor(xc_at(t)).cuda()
        h, bf, bc = states["ws"]
        dn.dnnmg_step(m, net, xc, h, bf, bc, ws, t)
        h, bf, bc = states["static"]
        dn.dnnmg_step_static(m, net, xc, h, bf, bc, t)
        torch.cuda.synchronize()
        for k, name in enumerate(("h", "b_f", "b_c")):
            assert torch.equal(states["static"][k], states["ws"][k]), (n, name)
    assert dn.dnnmg_net_status(net) == 0


@pytest.mark.parametrize("name", ["k2s2_bf16", "ragged_f32", "plain_f64"])
def test_static_step_matches_workspace_step_twice(dn, name):
    case = CASES[name]
    m = dn.Mesh(dn.make_desc(case["nxc"], case["nyc"], case["K"], case["s"], case.get("ellipse"),
                             precision=case["prec"], solid=mask_for(case)))
    om = oracle_mesh(case)
    net = dn.Net(*weights(case, om.n_in, om.n_out), precision=case["prec"])
    two_calls_bitwise(dn, m, net, case["H"], om.P, lambda t: coarse_input(case, t=t), fine_velocity(case)[:2])


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_static_step_on_the_256x64_mesh(dn, prec):
    # the 256 x 64-cell, K = 2 workload fits the static scratch and runs there
    c = synth.config("channel256")
    m = dn.Mesh(dn.make_desc(c["nxc"], c["nyc"], c["K"], c["s"], c["ellipse"], precision=prec))
    I = m.info
    W = synth.net_weights(I.n_in, c["H"], I.n_out, seed=c["seed"])
    net = dn.Net(*W, precision=prec)
    spec = synth.FlowSpec.from_seed(c["seed"], c["ellipse"])
    v0 = synth.fine_state(spec, I.nxf, I.nyf, 0.0, perturb_seed=3)[:2]
    two_calls_bitwise(dn, m, net, c["H"], I.P, lambda t: synth.coarse_state(spec, c["nxc"], c["nyc"], t), v0)


def test_static_step_rejects_oversized_mesh(dn):
    m = dn.Mesh(dn.make_desc(2048, 512, 2, 2, (0.2, 0.2, 0.05, 0.04), precision="bf16"))
    assert dn.dnnmg_static_scratch_needed(m) > dn.dnnmg_static_scratch_bytes()
    rng = np.random.default_rng(0)
    W = (rng.normal(0, 0.1, (384, m.info.n_in)), rng.normal(0, 0.1, (384, 128)), rng.normal(0, 0.1, (m.info.n_out, 128)))
    net = dn.Net(*W, precision="bf16")
    h = torch.zeros(m.info.P, 128, device="cuda")
    with pytest.raises(dn.DnnmgError) as e:
        dn.dnnmg_step_static(m, net, m.coarse(3), h, m.fine(2), m.coarse(3), 0.0)
    assert e.value.code == 1 and "static scratch" in str(e.value)

"""dnnmg_step_static: the correction step for callers that cannot allocate
device memory (its scratch is a library-owned static device array).

It must give the same results as dnnmg_step with a caller workspace, call
after call (the shared scratch keeps the previous call's contents), and it
must refuse meshes whose scratch does not fit.  This file is collected last
so that a failure here cannot stop the rest of a -x run.
"""

import numpy as np
import pytest
import torch

from helpers import CASES, TOL, coarse_input, fine_velocity, mask_for, oracle_mesh, rel_l2, weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_11520_gb300 import dnnmg
    return dnnmg


@pytest.mark.parametrize("name", ["k2s2_bf16", "ragged_f32", "plain_f64"])
def test_static_step_matches_workspace_step_twice(dn, name):
    case = CASES[name]
    m = dn.Mesh(dn.make_desc(case["nxc"], case["nyc"], case["K"], case["s"], case.get("ellipse"),
                             precision=case["prec"], solid=mask_for(case)))
    assert m.info.workspace_bytes <= dn.dnnmg_static_scratch_bytes()
    om = oracle_mesh(case)
    net = dn.Net(*weights(case, om.n_in, om.n_out), precision=case["prec"])
    rng = np.random.default_rng(3)
    h0 = torch.as_tensor(rng.uniform(-0.5, 0.5, (om.P, case["H"]))).to(m.real).cuda()
    b0 = m.fine(2)
    bc0 = m.coarse(3)
    dn.dnnmg_rhs_restrict(m, m.pack(fine_velocity(case)[:2]), b0, bc0)
    ws = m.workspace()
    states = {"ws": (h0.clone(), b0.clone(), m.coarse(3)), "static": (h0.clone(), b0.clone(), m.coarse(3))}
    for n in range(2):   # two calls in a row: the second runs on the first call's scratch contents
        t = 0.01 * n
        xc = torch.as_tensor(coarse_input(case, t=t)).cuda()
        h, bf, bc = states["ws"]
        dn.dnnmg_step(m, net, xc, h, bf, bc, ws, t)
        h, bf, bc = states["static"]
        dn.dnnmg_step_static(m, net, xc, h, bf, bc, t)
        torch.cuda.synchronize()
        tol = TOL[case["prec"]]
        for k in range(3):
            a = states["static"][k].double().cpu().numpy()
            b = states["ws"][k].double().cpu().numpy()
            assert rel_l2(a, b) <= tol, (n, k)
    assert dn.dnnmg_net_status(net) == 0


def test_static_step_rejects_oversized_mesh(dn):
    m = dn.Mesh(dn.make_desc(2048, 512, 2, 2, (0.2, 0.2, 0.05, 0.04), precision="bf16"))
    assert m.info.workspace_bytes > dn.dnnmg_static_scratch_bytes()
    rng = np.random.default_rng(0)
    W = (rng.normal(0, 0.1, (384, m.info.n_in)), rng.normal(0, 0.1, (384, 128)), rng.normal(0, 0.1, (m.info.n_out, 128)))
    net = dn.Net(*W, precision="bf16")
    h = torch.zeros(m.info.P, 128, device="cuda")
    with pytest.raises(dn.DnnmgError) as e:
        dn.dnnmg_step_static(m, net, m.coarse(3), h, m.fine(2), m.coarse(3), 0.0)
    assert e.value.code == 1 and "static scratch" in str(e.value)

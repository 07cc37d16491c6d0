"""Batched steps of several instances (dnnmg_server_*) on the GPU.

An instance's results must have the same bits alone (dnnmg_step with its own
state) and in any batch, whatever the other instances are; one instance in a
mix is also checked against the CPU FP64 oracle within the BF16-network
tolerance.  Admission fails cleanly when the state pool is full.
"""

import numpy as np
import pytest
import torch

from helpers import TOL, Params, coarse_input, fine_velocity, oracle_mesh, rel_l2, weights
from oracle import fem, step

pytestmark = pytest.mark.gpu

# one net shape (K = 1, one-cell patches: n_in 51, n_out 18), different meshes;
# P = 254, 480 and 400 give ragged last tiles
MIX = [
    dict(nxc=32, nyc=8, K=1, s=1, H=64, prec="bf16", ellipse=(0.2, 0.2, 0.04, 0.06)),
    dict(nxc=48, nyc=10, K=1, s=1, H=64, prec="bf16", ellipse=None),
    dict(nxc=40, nyc=10, K=1, s=1, H=64, prec="bf16", ellipse=(0.3, 0.2, 0.05, 0.04)),
]
PRM = Params()


@pytest.fixture(scope="module")
def dn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_11520_gb300 import dnnmg
    return dnnmg


def make(dn, case):
    return dn.Mesh(dn.make_desc(case["nxc"], case["nyc"], case["K"], case["s"], case.get("ellipse"),
                                precision="bf16"))


def inputs(dn, m, case, seed):
    """x_c at t = 0 and the initial b_f of a seeded velocity, on the device."""
    xc = torch.as_tensor(coarse_input(case, seed=seed)).cuda().contiguous()
    bf = m.fine(2)
    bc = m.coarse(3)
    dn.dnnmg_rhs_restrict(m, m.pack(fine_velocity(case, seed=seed)[:2].astype(np.float32)), bf, bc)
    return xc, bf


def net_for(dn, m):
    I = m.info
    return dn.Net(*weights(MIX[0], I.n_in, I.n_out), precision="bf16")


def test_mix_equals_alone_bitwise(dn):
    meshes = [make(dn, c) for c in MIX]
    net = net_for(dn, meshes[0])
    srv = dn.Server(net, sum(-(-m.info.P // 128) * 128 for m in meshes) + 256)
    slots = [srv.admit(m) for m in meshes]
    nsteps = 3
    # alone: dnnmg_step with each instance's own state
    alone = []
    for i, (m, c) in enumerate(zip(meshes, MIX)):
        xc, bf = inputs(dn, m, c, 11 + i)
        h = torch.zeros(m.info.P, c["H"], device="cuda")
        bc, ws = m.coarse(3), m.workspace()
        for n in range(nsteps):
            dn.dnnmg_step(m, net, xc, h, bf, bc, ws, n * PRM.k)
        torch.cuda.synchronize()
        alone.append((h.cpu().numpy(), bf.cpu().numpy(), bc.cpu().numpy()))
    # in the mix: all three per batch, in a rotating order, with instance 1
    # alone in the second batch
    state = []
    for i, (m, c) in enumerate(zip(meshes, MIX)):
        xc, bf = inputs(dn, m, c, 11 + i)
        state.append(dict(xc=xc, bf=bf, bc=m.coarse(3), n=0))
    orders = [[0, 1, 2], [1], [2, 0], [1, 0, 2], [2, 1]]
    for order in orders:
        items = []
        for i in order:
            s = state[i]
            if s["n"] == nsteps:
                continue
            items.append((slots[i], s["xc"], s["bf"], s["bc"], s["n"] * PRM.k))
            s["n"] += 1
        if items:
            srv.step(items)
    torch.cuda.synchronize()
    for i, m in enumerate(meshes):
        assert state[i]["n"] == nsteps
        h = srv.state(slots[i]).cpu().numpy()
        assert np.array_equal(h, alone[i][0]), i
        assert np.array_equal(state[i]["bf"].cpu().numpy(), alone[i][1]), i
        assert np.array_equal(state[i]["bc"].cpu().numpy(), alone[i][2]), i
    assert np.abs(alone[0][0]).max() > 0       # the state did evolve
    srv.close()


def test_instance_in_mix_matches_oracle(dn):
    case = MIX[2]
    meshes = [make(dn, c) for c in MIX]
    net = net_for(dn, meshes[0])
    srv = dn.Server(net, 2048)
    slots = [srv.admit(m) for m in meshes]
    om = oracle_mesh(case)
    Wx, Uh, Wfc = weights(case, om.n_in, om.n_out)
    xcs, bfs, bcs = [], [], []
    for i, (m, c) in enumerate(zip(meshes, MIX)):
        xc, bf = inputs(dn, m, c, 11 + i)
        xcs.append(xc)
        bfs.append(bf)
        bcs.append(m.coarse(3))
    v0 = fine_velocity(case, seed=13)[:2].astype(np.float32).astype(np.float64)
    bf_o = fem.rhs(om, PRM, v0)
    h_o = np.zeros((om.P, case["H"]))
    for n in range(2):
        t = n * PRM.k
        srv.step([(slots[i], xcs[i], bfs[i], bcs[i], t) for i in (1, 2, 0)])
        out = step.dnnmg_step(om, PRM, (Wx, Uh, Wfc), xcs[2].cpu().numpy(), h_o, bf_o, t)
        h_o, bf_o = out["h"], out["bf"]
    torch.cuda.synchronize()
    m = meshes[2]
    assert rel_l2(srv.state(slots[2]).cpu().numpy(), out["h"]) <= TOL["bf16"]
    assert rel_l2(m.unpack(bfs[2]), out["bf"]) <= TOL["bf16"]
    assert rel_l2(bcs[2].cpu().numpy().reshape(3, -1), out["bc"]) <= TOL["bf16"]
    srv.close()


def test_admission_by_pool_and_zero_state(dn):
    meshes = [make(dn, c) for c in MIX]
    net = net_for(dn, meshes[0])
    rows = [-(-m.info.P // 128) * 128 for m in meshes]
    srv = dn.Server(net, rows[0] + rows[1])
    a = srv.admit(meshes[0])
    b = srv.admit(meshes[1])
    with pytest.raises(dn.DnnmgError) as e:
        srv.admit(meshes[2])
    assert e.value.code == 4                    # DNNMG_ENOMEM: the pool is the budget
    xc, bf = inputs(dn, meshes[0], MIX[0], 11)
    srv.step([(a, xc, bf, meshes[0].coarse(3), 0.0)])
    torch.cuda.synchronize()
    assert srv.state(a).abs().max().item() > 0
    srv.release(b)
    c = srv.admit(meshes[2])                    # fits where instance b was
    assert srv.state(c).abs().max().item() == 0  # h0 = 0
    with pytest.raises(dn.DnnmgError):
        srv.step([(a, xc, bf, meshes[0].coarse(3), 0.0), (a, xc, bf, meshes[0].coarse(3), 0.0)])
    assert c == b                               # slot ids are reused
    srv.release(c)
    with pytest.raises(dn.DnnmgError):
        srv.release(c)                          # already released
    with pytest.raises(dn.DnnmgError):
        srv.state(7)                            # never admitted
    srv.close()


def test_server_rejects_other_net_shapes(dn):
    m1 = make(dn, MIX[0])
    m2 = make(dn, dict(MIX[0], K=2))
    net = net_for(dn, m1)
    srv = dn.Server(net, 1024)
    with pytest.raises(dn.DnnmgError) as e:
        srv.admit(m2)
    assert e.value.code == 1
    srv.close()
    f32 = dn.Net(*weights(MIX[0], m1.info.n_in, m1.info.n_out), precision="f32")
    with pytest.raises(dn.DnnmgError) as e:
        dn.Server(f32, 1024)
    assert e.value.code == 3

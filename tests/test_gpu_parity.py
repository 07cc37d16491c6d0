"""GPU parity of every step of the correction against the CPU FP64 oracle.

Each stage is called through the C ABI on the same seeded inputs the oracle
gets, on meshes that span several 32 x 16 fine-cell tiles with ragged tails;
index maps must match bit for bit, floating point within the tolerance of its
precision (FP64 1e-12, FP32 1e-5, BF16 network 2e-2 relative L2).
"""

import numpy as np
import pytest
import torch

from helpers import (BOUNDARY_CLASSES, CASES, TOL, Params, class_errors, coarse_input, fine_velocity, mask_for, np_dtype,
                     oracle_mesh, rel_l2, rhs_like, weights)
from oracle import average, features, fem, gru, step, transfer
from parity import check, record

pytestmark = pytest.mark.gpu

PRM = Params()


@pytest.fixture(scope="module")
def dn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_11520_gb300 import dnnmg
    return dnnmg


def gpu_mesh(dn, case):
    return dn.Mesh(dn.make_desc(case["nxc"], case["nyc"], case["K"], case["s"], case.get("ellipse"),
                                precision=case["prec"], solid=mask_for(case)))


def cuda(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda().contiguous()


def host(t):
    return t.detach().float().cpu().numpy().astype(np.float64) if t.dtype == torch.bfloat16 \
        else t.detach().cpu().numpy().astype(np.float64)


def as_real(case, a):
    """The input as the GPU sees it (rounded to the fine real type), in float64."""
    return np.asarray(a, dtype=np_dtype(case["prec"])).astype(np.float64)


@pytest.mark.parametrize("name", list(CASES))
def test_index_maps_bit_exact(dn, name):
    case = CASES[name]
    m = gpu_mesh(dn, case)
    om = oracle_mesh(case)
    I = m.info
    assert I.P == om.P
    pc = torch.zeros(I.P, dtype=torch.int32, device="cuda")
    fl = torch.zeros(I.plane, dtype=torch.uint8, device="cuda")
    mu = torch.zeros(I.plane, dtype=torch.uint8, device="cuda")
    dn.dnnmg_mesh_maps(m, pc, fl, mu)
    torch.cuda.synchronize()
    exp_pc = om.patches[:, 1] * om.npx + om.patches[:, 0]
    assert np.array_equal(pc.cpu().numpy(), exp_pc)
    nodes = lambda t: t.cpu().numpy().reshape(I.nyf + 1, I.pitch)[:, :I.nxf + 1].ravel()
    assert np.array_equal(nodes(fl), om.fine_node_flags().ravel())
    assert np.array_equal(nodes(mu), om.multiplicity.ravel())


@pytest.mark.parametrize("name", list(CASES))
def test_prolongate(dn, name):
    case = CASES[name]
    m = gpu_mesh(dn, case)
    om = oracle_mesh(case)
    xc = coarse_input(case, t=0.3)
    xf = m.fine(3)
    dn.dnnmg_prolongate(m, cuda(xc, torch.float64), xf, 0.3)
    ref = transfer.prolongate(om, PRM, xc, 0.3)
    got = m.unpack(xf)
    tol = 1e-14 if case["prec"] == "f64" else 1e-7
    check("x~", rel_l2(got, ref), tol, case["prec"], case=name)
    # Dirichlet values are set exactly as the oracle sets them
    mask = om.dirichlet.ravel()
    assert np.allclose(got[:2, mask], ref[:2, mask], rtol=1e-7 if case["prec"] != "f64" else 1e-15, atol=0)


@pytest.mark.parametrize("name", list(CASES))
def test_residual_and_features(dn, name):
    case = CASES[name]
    m = gpu_mesh(dn, case)
    om = oracle_mesh(case)
    xf = as_real(case, fine_velocity(case))
    bf = as_real(case, rhs_like(case))
    X = m.features()
    rf = m.fine(3)
    dn.dnnmg_patch_features(m, m.pack(xf), m.pack(bf), X, rf=rf)
    r_ref = fem.residual(om, PRM, xf, bf)
    X_ref = features.patch_features(om, PRM, xf, r_ref)
    r_got = m.unpack(rf)
    tol_r = TOL["f64"] if case["prec"] == "f64" else TOL["f32"]
    for c in range(3):
        check("r_" + "uvp"[c], rel_l2(r_got[c], r_ref[c]), tol_r, case["prec"], case=name)
    # exact zeros on Dirichlet / inactive rows
    assert np.all(r_got[:2, om.dirichlet.ravel()] == 0)
    assert np.all(r_got[2, ~om.p_active.ravel()] == 0)
    Xg = host(X).reshape(m.info.P, m.info.ldx)
    assert np.all(Xg[:, om.n_in:] == 0)
    tol_x = TOL[case["prec"]] if case["prec"] != "bf16" else 1e-2
    nf = om.nf
    blocks = [(0, nf), (nf, 2 * nf), (2 * nf, 3 * nf), (3 * nf, om.n_in)]
    for (a, b), what in zip(blocks, ("X r_u", "X r_v", "X r_p", "X coarse/Pe/geo")):
        check(what, rel_l2(Xg[:, a:b], X_ref[:, a:b]), tol_x, case["prec"], case=name)


@pytest.mark.parametrize("name", list(CASES))
def test_gru_step(dn, name):
    case = CASES[name]
    om = oracle_mesh(case)
    rng = np.random.default_rng(21)
    P, n_in, n_out, H = om.P, om.n_in, om.n_out, case["H"]
    Wx, Uh, Wfc = weights(case, n_in, n_out)
    X = rng.normal(0.0, 1.0, (P, n_in))
    h = rng.uniform(-0.5, 0.5, (P, H))
    net = dn.Net(Wx, Uh, Wfc, case["prec"])
    ldx = (n_in + 15) // 16 * 16
    Xp = np.zeros((P, ldx))
    Xp[:, :n_in] = X
    Xcpu = torch.as_tensor(Xp).to(net.feat)   # rounded on the host (bf16 for BF16)
    Xq = Xcpu.to(torch.float64).numpy()[:, :n_in]
    Xt = Xcpu.cuda().contiguous()
    hq = as_real(case, h)
    ht = cuda(hq, net.real)
    d = torch.zeros(P, n_out, dtype=net.real, device="cuda")
    dn.dnnmg_gru_step(net, Xt, ht, d, P)
    h_ref, d_ref = gru.gru_step(Xq, hq, Wx, Uh, Wfc)
    tol = TOL[case["prec"]]
    check("h", rel_l2(host(ht), h_ref), tol, case["prec"], case=name)
    check("d", rel_l2(host(d), d_ref), tol, case["prec"], case=name)


@pytest.mark.parametrize("name", list(CASES))
def test_scatter_avg(dn, name):
    case = CASES[name]
    m = gpu_mesh(dn, case)
    om = oracle_mesh(case)
    rng = np.random.default_rng(23)
    d = as_real(case, rng.normal(0.0, 0.3, (om.P, om.n_out)))
    xf = as_real(case, fine_velocity(case))
    vc = m.fine(2)
    dn.dnnmg_scatter_avg(m, cuda(d, m.real), m.pack(xf), vc)
    ref = average.scatter_average(om, d, xf)
    tol = TOL["f64"] if case["prec"] == "f64" else TOL["f32"]
    check("v_corr", rel_l2(m.unpack(vc), ref), tol, case["prec"], case=name)
    # Dirichlet nodes keep the prolongated values bit for bit
    mask = om.dirichlet.ravel()
    assert np.array_equal(m.unpack(vc)[:, mask], xf[:2, mask])


@pytest.mark.parametrize("name", list(CASES))
def test_constant_correction_is_exact(dn, name):
    case = CASES[name]
    m = gpu_mesh(dn, case)
    om = oracle_mesh(case)
    xf = as_real(case, fine_velocity(case))
    d = np.full((om.P, om.n_out), 0.375)
    vc = m.fine(2)
    dn.dnnmg_scatter_avg(m, cuda(d, m.real), m.pack(xf), vc)
    got = m.unpack(vc)
    free = ~om.dirichlet.ravel()
    exp = (xf[:2, free].astype(np_dtype(case["prec"])) + np_dtype(case["prec"])(0.375)).astype(np.float64)
    assert np.array_equal(got[:, free], exp)


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_restrict(dn, name):
    case = CASES[name]
    m = gpu_mesh(dn, case)
    om = oracle_mesh(case)
    v = as_real(case, fine_velocity(case)[:2])
    bf = m.fine(2)
    bc = m.coarse(3)
    dn.dnnmg_rhs_restrict(m, m.pack(v), bf, bc)
    b_ref = fem.rhs(om, PRM, v)
    tol = TOL["f64"] if case["prec"] == "f64" else TOL["f32"]
    bfg = m.unpack(bf)
    check("b_f", rel_l2(bfg, b_ref), tol, case["prec"], case=name)
    assert np.all(bfg[:, om.dirichlet.ravel()] == 0)
    check("b_c", rel_l2(host(bc).reshape(3, -1), transfer.restrict(om, b_ref)), tol, case["prec"], case=name)


def run_steps(dn, case, nsteps, seed=31, class_tol=None):
    """Both sides run nsteps corrections on identical inputs; returns per-step errors.

    The error of b_f is also measured per node class (max |GPU - oracle| over
    the non-Dirichlet nodes beside the inflow, the walls, the outflow and the
    obstacle, over the field's RMS): recorded always, asserted against
    class_tol when it is given.
    """
    m = gpu_mesh(dn, case)
    om = oracle_mesh(case)
    Wx, Uh, Wfc = weights(case, om.n_in, om.n_out)
    net = dn.Net(Wx, Uh, Wfc, case["prec"])
    rng = np.random.default_rng(seed)
    h0 = as_real(case, rng.uniform(-0.5, 0.5, (om.P, case["H"])))
    v0 = as_real(case, fine_velocity(case)[:2])
    # initial right-hand side: each side assembles its own from v0
    bf_g = m.fine(2)
    bc_g = m.coarse(3)
    dn.dnnmg_rhs_restrict(m, m.pack(v0), bf_g, bc_g)
    bf_o = fem.rhs(om, PRM, v0)
    h_g = cuda(h0, m.real)
    h_o = h0.copy()
    ws = m.workspace()
    errs = []
    for n in range(nsteps):
        t = n * PRM.k
        xc = coarse_input(case, t=t)
        dn.dnnmg_step(m, net, cuda(xc, torch.float64), h_g, bf_g, bc_g, ws, t)
        out = step.dnnmg_step(om, PRM, (Wx, Uh, Wfc), xc, h_o, bf_o, t)
        h_o, bf_o = out["h"], out["bf"]
        bf_got = m.unpack(bf_g)
        errs.append({"h": rel_l2(host(h_g), out["h"]), "bf": rel_l2(bf_got, out["bf"]),
                     "bc": rel_l2(host(bc_g).reshape(3, -1), out["bc"])})
        for cname, err in class_errors(bf_got, out["bf"], om).items():
            if class_tol is None or cname not in BOUNDARY_CLASSES:
                record("step bf max/RMS " + cname, err, TOL[case["prec"]], case["prec"], step=n)
            else:
                check("step bf max/RMS " + cname, err, class_tol, case["prec"], step=n)
    return errs


@pytest.mark.parametrize("name", list(CASES))
def test_step_matches_oracle(dn, name):
    case = CASES[name]
    tol = TOL[case["prec"]]
    errs = run_steps(dn, case, 3, class_tol=tol)
    for n, e in enumerate(errs):
        for k, v in e.items():
            check("step " + k, v, tol, case["prec"], step=n, case=name)


def test_largest_patches_bf16_network(dn):
    # K = 3, s = 2 with the BF16 network: 906 inputs rounded to BF16, among
    # them Peclet numbers near 550 (BF16 spacing 4), so the GRU state drifts
    # further from the FP64 oracle than at smaller patches (measured 2.0 % after
    # one step, 2.6 % after four; the same case with the FP32 network matches
    # to 2e-7).  The correction's outputs stay well within the BF16 bound.
    case = dict(CASES["k3s2_f32_max"], prec="bf16")
    errs = run_steps(dn, case, 3)
    for n, e in enumerate(errs):
        check("step bf", e["bf"], TOL["bf16"], "bf16", step=n)
        check("step bc", e["bc"], TOL["bf16"], "bf16", step=n)
        check("step h", e["h"], 2 * TOL["bf16"], "bf16", step=n)


def test_plain_config_ten_steps(dn):
    # the single plain instance (32 x 8, K = 1, H = 32, FP64) over its 10 steps
    errs = run_steps(dn, CASES["plain_f64"], 10, class_tol=TOL["f64"])
    for n, e in enumerate(errs):
        for k, v in e.items():
            check("step " + k, v, TOL["f64"], "f64", step=n)


def test_step_is_deterministic_and_host_variant_agrees(dn):
    case = CASES["k2s2_bf16"]
    m = gpu_mesh(dn, case)
    om = oracle_mesh(case)
    Wx, Uh, Wfc = weights(case, om.n_in, om.n_out)
    net = dn.Net(Wx, Uh, Wfc, case["prec"])
    xc = coarse_input(case, t=0.0)
    h0 = torch.rand(om.P, case["H"], device="cuda") - 0.5
    bf0 = m.fine(2)
    bcs = []
    # device buffers twice; pinned host buffers (the kernels read x_c and write
    # b_c over the host link); pageable host buffers (copied through the workspace)
    for variant in range(4):
        h, bf = h0.clone(), bf0.clone()
        bc = m.coarse(3)
        ws = m.workspace()
        if variant < 2:
            dn.dnnmg_step(m, net, cuda(xc, torch.float64), h, bf, bc, ws, 0.0)
        else:
            xch = torch.as_tensor(xc).clone()
            bch = torch.full((3 * m.info.Nc,), -1.0, dtype=torch.float64)
            if variant == 2:
                xch, bch = xch.pin_memory(), bch.pin_memory()
            dn.dnnmg_step_host(m, net, xch, h, bf, bch, ws, 0.0)
            torch.cuda.synchronize()
            bc = bch.cuda()
        torch.cuda.synchronize()
        bcs.append((bc.cpu().numpy().ravel(), h.cpu().numpy(), bf.cpu().numpy()))
    for v in range(1, 4):
        for k in range(3):
            assert np.array_equal(bcs[0][k], bcs[v][k]), (v, k)


def test_step_leaves_mesh_status_clear(dn):
    # the persistent TMA-fed residual kernel of the step reports time-outs of
    # its bounded waits in the mesh status word; a normal step sets nothing
    case = CASES["k2_f32"]
    m = gpu_mesh(dn, case)
    om = oracle_mesh(case)
    Wx, Uh, Wfc = weights(case, om.n_in, om.n_out)
    net = dn.Net(Wx, Uh, Wfc, "f32")
    xc = coarse_input(case, t=0.0)
    h = torch.zeros(om.P, case["H"], device="cuda")
    bf, bc, ws = m.fine(2), m.coarse(3), m.workspace()
    for i in range(3):
        dn.dnnmg_step(m, net, cuda(xc, torch.float64), h, bf, bc, ws, 0.01 * i)
    torch.cuda.synchronize()
    assert dn.dnnmg_mesh_status(m) == 0
    assert dn.dnnmg_net_status(net) == 0


def test_bounded_wait_times_out_and_context_survives(dn):
    # a wait that nothing satisfies gives up after its limit, reports the
    # time-out in the status word and releases the CTA's other waiters
    limit = 20_000_000   # 20 ms
    status, waited = dn.dnnmg_selftest_wait_timeout(limit)
    assert status == 1                                 # DNNMG_DEVERR_TIMEOUT
    assert limit <= waited[0] < limit + 200_000_000
    assert 0 < waited[1] < limit + 200_000_000         # left through the abort flag, not its own 2 s limit
    with pytest.raises(dn.DnnmgError):
        dn.dnnmg_selftest_wait_timeout(0)
    # the context is still usable: a step afterwards is clean and correct
    errs = run_steps(dn, CASES["k2_f32"], 1)
    assert max(errs[0].values()) <= TOL["f32"]


def test_step_timed_matches_step(dn):
    # the instrumented step records one event per kernel and computes the same bits
    case = CASES["k2s2_bf16"]
    m = gpu_mesh(dn, case)
    om = oracle_mesh(case)
    Wx, Uh, Wfc = weights(case, om.n_in, om.n_out)
    net = dn.Net(Wx, Uh, Wfc, "bf16")
    xc = cuda(coarse_input(case, t=0.0), torch.float64)
    outs = []
    for timed in (False, True):
        h = torch.zeros(om.P, case["H"], device="cuda")
        bf, bc, ws = m.fine(2), m.coarse(3), m.workspace()
        if timed:
            n = dn.dnnmg_step_launches(m, net)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(n + 1)]
            dn.dnnmg_step_timed(m, net, xc, h, bf, bc, ws, 0.0, ev)
            with pytest.raises(dn.DnnmgError):
                dn.dnnmg_step_timed(m, net, xc, h, bf, bc, ws, 0.0, ev[:-1])
        else:
            dn.dnnmg_step(m, net, xc, h, bf, bc, ws, 0.0)
        torch.cuda.synchronize()
        outs.append((h.cpu(), bf.cpu(), bc.cpu()))
        if timed:
            times = [ev[i].elapsed_time(ev[i + 1]) for i in range(n)]
            assert all(t >= 0.0 for t in times)
    for a, b in zip(*outs):
        assert torch.equal(a, b)


def test_zero_network_reduces_to_prolongated_rhs(dn):
    # with W_fc = 0 the correction vanishes, so v_corr = v~ and the step
    # returns R Rhs(P x_c) (Algorithm 2 without the network)
    case = CASES["ragged_f32"]
    m = gpu_mesh(dn, case)
    om = oracle_mesh(case)
    Wx, Uh, Wfc = weights(case, om.n_in, om.n_out)
    net = dn.Net(Wx, Uh, np.zeros_like(Wfc), "f32")
    xc = coarse_input(case, t=0.0)
    h = torch.zeros(om.P, case["H"], device="cuda")
    bf, bc, ws = m.fine(2), m.coarse(3), m.workspace()
    dn.dnnmg_step(m, net, cuda(xc, torch.float64), h, bf, bc, ws, 0.0)
    xf = m.fine(3)
    dn.dnnmg_prolongate(m, cuda(xc, torch.float64), xf, 0.0)
    bf2, bc2 = m.fine(2), m.coarse(3)
    dn.dnnmg_rhs_restrict(m, xf[:2].contiguous(), bf2, bc2)
    torch.cuda.synchronize()
    assert torch.equal(bf, bf2) and torch.equal(bc, bc2)


def test_invalid_arguments_raise(dn):
    case = CASES["ragged_f32"]
    m = gpu_mesh(dn, case)
    om = oracle_mesh(case)
    Wx, Uh, Wfc = weights(case, om.n_in, om.n_out)
    net64 = dn.Net(Wx, Uh, Wfc, "f64")
    h = torch.zeros(om.P, case["H"], device="cuda")
    with pytest.raises(dn.DnnmgError):   # precision mismatch between mesh and net
        dn.dnnmg_step(m, net64, m.coarse(3), h, m.fine(2), m.coarse(3), m.workspace(), 0.0)
    net = dn.Net(Wx, Uh, Wfc, "f32")
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(dn.DnnmgError):   # workspace too small
        dn.dnnmg_step(m, net, m.coarse(3), h, m.fine(2), m.coarse(3), small, 0.0)
    with pytest.raises(dn.DnnmgError):   # aliasing output
        v = m.fine(2)
        dn.dnnmg_rhs_restrict(m, v, v, m.coarse(3))


@pytest.mark.parametrize("name", ["ragged_f32", "k2_f32", "k2s2_bf16", "k3_f64"])
def test_restrict_fp64_class_accuracy(dn, name):
    # R applied to the same single-precision vector: the GPU's float-pair
    # accumulation must agree with the oracle's FP64 restriction to ~1e-13
    case = CASES[name]
    m = gpu_mesh(dn, case)
    om = oracle_mesh(case)
    bf = as_real(case, rhs_like(case, seed=41))
    bc = m.coarse(3)
    dn.dnnmg_restrict(m, m.pack(bf), bc)
    ref = transfer.restrict(om, bf)
    check("R b_f (FP64 class)", rel_l2(host(bc).reshape(3, -1), ref), 1e-13, case["prec"], case=name)


# (282, 64, 162): an output layer wider than 2H (two MMA pieces);
# P = 40000: more tiles than SMs, so each persistent CTA walks several
GRU_SHAPES = [(51, 32, 18), (99, 64, 50), (99, 96, 50), (282, 128, 162), (60, 32, 40), (282, 64, 162)]


@pytest.mark.parametrize("shape", GRU_SHAPES)
@pytest.mark.parametrize("P", [1, 127, 128, 300, 1000, 40000])
def test_gru_tensor_cores_match_cuda_cores(dn, shape, P, monkeypatch):
    # same BF16-operand arithmetic on the tcgen05 kernel and on CUDA cores;
    # only the FP32 summation order differs
    n_in, H, n_out = shape
    rng = np.random.default_rng(P + H)
    Wx, Uh, Wfc = (rng.normal(0, 0.1, s) for s in ((3 * H, n_in), (3 * H, H), (n_out, H)))
    ldx = (n_in + 15) // 16 * 16
    X = np.zeros((P, ldx))
    X[:, :n_in] = rng.normal(0, 1.0, (P, n_in))
    h0 = rng.uniform(-0.5, 0.5, (P, H))
    tc = dn.Net(Wx, Uh, Wfc, "bf16")
    assert dn.dnnmg_net_uses_tensor_cores(tc)
    monkeypatch.setenv("DNNMG_GRU_KERNEL", "simt")
    simt = dn.Net(Wx, Uh, Wfc, "bf16")
    assert not dn.dnnmg_net_uses_tensor_cores(simt)
    Xt = torch.as_tensor(X).to(torch.bfloat16).cuda()
    outs = []
    for net in (tc, simt):
        h = torch.as_tensor(h0, dtype=torch.float32).cuda()
        d = torch.full((P, n_out), float("nan"), dtype=torch.float32, device="cuda")
        dn.dnnmg_gru_step(net, Xt, h, d, P)
        torch.cuda.synchronize()
        outs.append((h.cpu().numpy(), d.cpu().numpy()))
    assert dn.dnnmg_net_status(tc) == 0
    assert np.isfinite(outs[0][1]).all()
    shape_id = dict(shape=list(shape), P=P)
    check("h tc vs simt", rel_l2(outs[0][0], outs[1][0]), 2e-3, "bf16", **shape_id)
    check("d tc vs simt", rel_l2(outs[0][1], outs[1][1]), 2e-3, "bf16", **shape_id)
    # and against the FP64 oracle within the BF16 tolerance
    Xq = torch.as_tensor(X).to(torch.bfloat16).to(torch.float64).numpy()[:, :n_in]
    h_ref, d_ref = gru.gru_step(Xq, h0.astype(np.float32).astype(np.float64), Wx, Uh, Wfc)
    check("h tc", rel_l2(outs[0][0], h_ref), TOL["bf16"], "bf16", **shape_id)
    check("d tc", rel_l2(outs[0][1], d_ref), TOL["bf16"], "bf16", **shape_id)


@pytest.mark.parametrize("name", list(CASES))
def test_fused_prolongation_forms(dn, name):
    # S2+S3 and S5 with x~ = P x_c formed inside the kernel equal the oracle's
    # features / averaging applied to the oracle's prolongation
    case = CASES[name]
    m = gpu_mesh(dn, case)
    om = oracle_mesh(case)
    t = 0.2
    xc = coarse_input(case, t=t)
    bf = as_real(case, rhs_like(case))
    X, rf = m.features(), m.fine(3)
    dn.dnnmg_patch_features(m, None, m.pack(bf), X, rf=rf, xc=cuda(xc, torch.float64), t=t)
    xf_ref = transfer.prolongate(om, PRM, xc, t)
    r_ref = fem.residual(om, PRM, xf_ref, bf)
    X_ref = features.patch_features(om, PRM, xf_ref, r_ref)
    tol = TOL["f64"] if case["prec"] == "f64" else TOL["f32"]
    check("r (fused S1)", rel_l2(m.unpack(rf), r_ref), tol, case["prec"], case=name)
    check("X (fused S1)", rel_l2(host(X).reshape(m.info.P, m.info.ldx)[:, :om.n_in], X_ref),
          TOL[case["prec"]] if case["prec"] != "bf16" else 1e-2, case["prec"], case=name)
    rng = np.random.default_rng(29)
    d = as_real(case, rng.normal(0.0, 0.3, (om.P, om.n_out)))
    vc = m.fine(2)
    dn.dnnmg_scatter_avg(m, cuda(d, m.real), None, vc, xc=cuda(xc, torch.float64), t=t)
    check("v_corr (fused S1)", rel_l2(m.unpack(vc), average.scatter_average(om, d, xf_ref)), tol, case["prec"],
          case=name)


@pytest.mark.parametrize("name", list(CASES))
def test_scatter_rhs_fused_equals_two_passes(dn, name):
    # S5+S6 in one kernel (v_corr kept on chip) gives the bits of S5 (with xc)
    # followed by S6, and the oracle's Rhs of the averaged correction
    case = CASES[name]
    m = gpu_mesh(dn, case)
    om = oracle_mesh(case)
    t = 0.15
    xc = coarse_input(case, t=t)
    rng = np.random.default_rng(31)
    d = cuda(as_real(case, rng.normal(0.0, 0.3, (om.P, om.n_out))), m.real)
    xct = cuda(xc, torch.float64)
    vc, b1, b2 = m.fine(2), m.fine(2), m.fine(2)
    dn.dnnmg_scatter_avg(m, d, None, vc, xc=xct, t=t)
    dn.dnnmg_rhs(m, vc, b1)
    dn.dnnmg_scatter_rhs(m, d, xct, b2, t=t)
    torch.cuda.synchronize()
    assert np.array_equal(m.unpack(b1), m.unpack(b2))
    vref = average.scatter_average(om, d.cpu().numpy().astype(np.float64), transfer.prolongate(om, PRM, xc, t))
    ref = fem.rhs(om, PRM, vref)
    tol = TOL["f64"] if case["prec"] == "f64" else TOL["f32"]
    check("b_f (fused S5+S6)", rel_l2(m.unpack(b2), ref), tol, case["prec"], case=name)


def test_rhs_alone_equals_rhs_of_rhs_restrict(dn):
    case = CASES["k2_f32"]
    m = gpu_mesh(dn, case)
    v = m.pack(as_real(case, fine_velocity(case)[:2]))
    b1, b2, bc = m.fine(2), m.fine(2), m.coarse(3)
    dn.dnnmg_rhs_restrict(m, v, b1, bc)
    dn.dnnmg_rhs(m, v, b2)
    torch.cuda.synchronize()
    assert torch.equal(b1, b2)


def test_mesh_without_fluid_patches(dn):
    # degenerate case: every coarse cell solid, so there are no fluid patches
    # (P = 0): the step skips the network, every velocity row is a Dirichlet
    # row, and the result still matches the oracle; a server admits the
    # instance with an empty state segment
    case = dict(nxc=16, nyc=4, K=1, s=1, H=32, prec="bf16", ellipse=None)
    from oracle.mesh import Mesh as OMesh
    solid = np.ones((case["nyc"], case["nxc"]), dtype=bool)
    m = dn.Mesh(dn.make_desc(case["nxc"], case["nyc"], case["K"], case["s"], None, precision="bf16", solid=solid))
    om = OMesh(case["nxc"], case["nyc"], case["K"], case["s"], solid=solid)
    assert m.info.P == 0 and om.P == 0
    Wx, Uh, Wfc = weights(case, om.n_in, om.n_out)
    net = dn.Net(Wx, Uh, Wfc, "bf16")
    # no GRU launch: the stencil kernels only (two S2+S3 kernels on FP32 fields with K <= 2)
    assert dn.dnnmg_step_launches(m, net) == 6
    xc = coarse_input(case, t=0.0)
    v0 = fine_velocity(case)[:2].astype(np.float32).astype(np.float64)
    bf = m.fine(2)
    bc = m.coarse(3)
    dn.dnnmg_rhs_restrict(m, m.pack(v0), bf, bc)
    h = torch.zeros(0, case["H"], device="cuda")
    dn.dnnmg_step(m, net, cuda(xc, torch.float64), h, bf, bc, m.workspace(), 0.0)
    out = step.dnnmg_step(om, PRM, (Wx, Uh, Wfc), xc, np.zeros((0, case["H"])), fem.rhs(om, PRM, v0), 0.0)
    torch.cuda.synchronize()
    check("step bc", rel_l2(host(bc).reshape(3, -1), out["bc"]), TOL["bf16"], "bf16")
    check("step bf", rel_l2(m.unpack(bf), out["bf"]), TOL["bf16"], "bf16")
    srv = dn.Server(net, 128)
    slot = srv.admit(m)
    assert srv.state(slot).shape == (0, case["H"])
    srv.step([(slot, cuda(xc, torch.float64), bf, bc, 0.0)])
    torch.cuda.synchronize()
    srv.close()

"""Convolutional head of the patch network (Sec. 6.2) on the GPU.

The fold of the head into the output layer and its gradient are compared with
the oracle (pinned in test_oracle_head.py); a net created with the head must
give the oracle's GRU step followed by the head; and training with the head
must give the oracle's window gradients mapped through the fold.
"""

import numpy as np
import pytest
import torch

from helpers import rel_l2
from parity import check
from oracle import gru, head
from oracle import train as otrain

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 2e-2}


@pytest.fixture(scope="module")
def dn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_11520_gb300 import dnnmg
    return dnnmg


def cu(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).cuda()


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def test_head_params_and_unsupported_sizes(dn):
    assert dn.head_params(18) == 90 and dn.head_params(50) == 122 and dn.head_params(162) == 234
    for n_out in (8, 32, 2 * 11 * 11, 2 * 4 * 4):
        assert dn.head_params(n_out) == 0
    with pytest.raises(dn.DnnmgError):
        dn.head_fold(cu(np.zeros(90)), cu(np.zeros((32, 4))))


@pytest.mark.parametrize("n_out,H", [(18, 32), (18, 1), (50, 70), (162, 5)])
def test_fold_and_gradient_match_oracle(dn, n_out, H):
    rng = np.random.default_rng(n_out + H)
    theta = f32(rng.standard_normal(head.n_theta(n_out)))
    Wfc, G = f32(rng.standard_normal((n_out, H))), f32(rng.standard_normal((n_out, H)))
    Weff = dn.head_fold(cu(theta), cu(Wfc))
    dth, dW = dn.head_backward(cu(theta), cu(Wfc), cu(G))
    ref_dth, ref_dW = head.fold_backward(theta, Wfc, G)
    case = f"n_out {n_out}, H {H}"
    check("head fold W_eff", rel_l2(Weff.cpu().numpy(), head.fold(theta, Wfc)), TOL["f32"], "f32", case=case)
    check("head fold d theta", rel_l2(dth.cpu().numpy(), ref_dth), TOL["f32"], "f32", case=case)
    check("head fold d W_fc", rel_l2(dW.cpu().numpy(), ref_dW), TOL["f32"], "f32", case=case)
    # deterministic: the same call gives the same bits
    dth2, _ = dn.head_backward(cu(theta), cu(Wfc), cu(G))
    assert torch.equal(dth, dth2)


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_net_with_head_is_gru_step_then_head(dn, prec):
    # the K = 1 net of Sec. 6.2: N_in = 51 (padded to 64), N_GRU = 32, N_out = 18
    rng = np.random.default_rng(5)
    P, n_in, ldx, H, n_out = 300, 51, 64, 32, 18
    Wx, Uh, Wfc = (rng.normal(0, 0.2, s) for s in ((3 * H, n_in), (3 * H, H), (n_out, H)))
    theta = rng.normal(0, 0.3, head.n_theta(n_out))
    net = dn.Net(Wx, Uh, Wfc, prec, head=theta)
    X = np.zeros((P, ldx))
    X[:, :n_in] = rng.normal(0, 1, (P, n_in))
    Xc = torch.as_tensor(X).to(net.feat)
    Xq = Xc.to(torch.float64).numpy()[:, :n_in]
    h = rng.uniform(-0.5, 0.5, (P, H))
    if prec != "f64":
        h = f32(h)
    ht = torch.as_tensor(h).to(net.real).cuda().contiguous()
    d = torch.zeros(P, n_out, dtype=net.real, device="cuda")
    dn.dnnmg_gru_step(net, Xc.cuda().contiguous(), ht, d, P)
    h_ref, dfc = gru.gru_step(Xq, h, Wx, Uh, Wfc)
    d_ref = head.head_rows(dfc, theta)
    check("net with head h", rel_l2(ht.double().cpu().numpy(), h_ref), TOL[prec], prec)
    check("net with head d", rel_l2(d.double().cpu().numpy(), d_ref), TOL[prec], prec)
    with pytest.raises(ValueError):
        dn.Net(Wx, Uh, Wfc, prec, head=theta[:-1])


def test_training_with_head_gives_oracle_gradients(dn):
    from paper_2008_11520_gb300 import train
    T, P, n_in, ldx, H, n_out = 3, 200, 51, 64, 32, 18
    rng = np.random.default_rng(9)
    X = np.zeros((T, P, ldx))
    X[:, :, :n_in] = rng.normal(0, 1, (T, P, n_in))
    h0 = f32(rng.uniform(-0.5, 0.5, (P, H)))
    Y = f32(rng.normal(0, 0.3, (T, P, n_out)))
    X = f32(X)
    tn = train.PatchNetTrainer(n_in, ldx, H, n_out, T, P, seed=4, std=0.2, head=True)
    Wx, Uh, Wfc, theta = tn.weights()
    L, _ = tn.loss(cu(X), cu(Y), cu(h0))
    L.backward()
    grads = [p.grad.cpu().numpy() for p in tn.params]
    Weff = head.fold(theta, Wfc)
    L0, gWx, gUh, gWeff, _ = otrain.loss_and_grads(X[:, :, :n_in], h0, Y, Wx, Uh, Weff, alpha=0.0)
    gth, gWfc = head.fold_backward(theta, Wfc, gWeff)
    assert L.item() == pytest.approx(L0, rel=1e-5)
    for name, g, ref in zip(("W_x", "U_h", "W_fc", "theta"), grads, (gWx, gUh, gWfc, gth)):
        check("window gradient with head " + name, rel_l2(g, ref), TOL["f32"], "f32")
    # the head starts near the identity
    assert rel_l2(Weff, Wfc) < 0.2
    # one update moves every parameter group and lowers the window loss
    L1, _ = tn.train_window(cu(X), cu(Y), cu(h0))
    assert all(not np.array_equal(a, b) for a, b in zip(tn.weights(), (Wx, Uh, Wfc, theta)))
    L2, _ = tn.loss(cu(X), cu(Y), cu(h0))
    assert L2.item() < L.item()

"""Training the patch network, on the library's own kernels.

* ``GruWindow`` -- a ``torch.autograd.Function`` whose forward and backward are
  libdnnmg's GRU window kernels (Eq. gru + output layer unrolled over T steps,
  gradient by truncated backpropagation through time).
* ``L2Loss`` -- the loss of Sec. 6.3 (sum over steps of the mean over patches
  of |d - y|^2) as an autograd function on the library's loss kernel.
* ``HeadFold`` -- the convolutional head of Sec. 6.2 folded into the output
  layer (W_eff = head applied to each column of W_fc) as an autograd function
  on the library's fold and fold-gradient kernels.
* ``PatchNetTrainer`` -- FP32 weights, Adam (Sec. 6.3) with the Tikhonov
  term alpha = 1e-4, one update per window; optionally with the head.
* ``flow_windows`` -- training windows from synthetic flows, built with the
  library's own S1 and S2+S3 kernels: features of x~ = P x_c(t_n) with the
  right-hand side of the previous reference velocity, and targets
  y = v_bar - x~ on each patch's fine nodes.  The reference v_bar is the
  synthetic analytic flow sampled on the fine nodes, with the discrete
  Dirichlet values at Dirichlet nodes (as a fine-level solution has them; the
  analytic flow follows the exact ellipse, the mesh its staircase): it stands
  in for the paper's (L+1)-level multigrid solutions.
* ``solution_windows`` -- the same windows from solved flows: the fine-level
  solution of ``solver`` as v_bar and a coarse solution (the fine one at the
  coarse nodes, ``coarse_nodes``, or a coarse-level simulation) as x_c, the
  paper's two-level training data.
* ``e_rel`` -- E_rel(v) of Sec. 6.4 for a net, through the inference path
  (dnnmg_gru_step, dnnmg_scatter_avg).

Every arithmetic step of training runs in libdnnmg kernels; torch provides
memory, streams and the autograd bookkeeping.
"""

import numpy as np
import torch

from . import dnnmg, synth


class GruWindow(torch.autograd.Function):
    """D [T][P][n_out] = outputs of the GRU window from h0 (None: zero)."""

    @staticmethod
    def forward(ctx, X, h0, Wx, Uh, Wfc, trainer):
        D = torch.empty(trainer.T, trainer.P, trainer.n_out, dtype=torch.float32, device=X.device)
        trainer.forward(X, h0, Wx, Uh, Wfc, D)
        ctx.trainer = trainer
        ctx.save_for_backward(X, Wx, Uh, Wfc)
        return D

    @staticmethod
    def backward(ctx, dD):
        X, Wx, Uh, Wfc = ctx.saved_tensors
        t = ctx.trainer
        gWx, gUh, gWfc = torch.empty_like(Wx), torch.empty_like(Uh), torch.empty_like(Wfc)
        dh0 = torch.empty(t.P, t.H, dtype=torch.float32, device=X.device) if ctx.needs_input_grad[1] else None
        t.backward(dD.contiguous(), X, Uh, Wfc, gWx, gUh, gWfc, dh0)
        return None, dh0, gWx, gUh, gWfc, None


class HeadFold(torch.autograd.Function):
    """W_eff [n_out][H]: the convolutional head (Sec. 6.2) applied to each column
    of W_fc; the head is linear, so the window runs the folded output layer."""

    @staticmethod
    def forward(ctx, theta, Wfc):
        ctx.save_for_backward(theta, Wfc)
        return dnnmg.head_fold(theta, Wfc)

    @staticmethod
    def backward(ctx, G):
        theta, Wfc = ctx.saved_tensors
        return dnnmg.head_backward(theta, Wfc, G.contiguous())


def head_init(n_out, seed, std=0.05):
    """Head parameters that start near the identity (the paper gives no
    initialisation for the head): filter 0 of both blocks a centred unit tap,
    filters 1..3 N(0, std^2) (a filter at zero would get no gradient: its
    block is quadratic in it), w = 1/2, so d = y + O(std^2) y."""
    rng = np.random.default_rng(seed + 1)
    nt = dnnmg.head_params(n_out)
    ks = np.concatenate([np.zeros((1, 9)), rng.normal(0.0, std, (3, 9))])
    kv = np.concatenate([np.zeros((1, 9)), rng.normal(0.0, std, (3, 9))])
    ks[0, 4] = kv[0, 4] = 1.0
    theta = np.concatenate([ks.ravel(), kv.ravel(), np.full(n_out, 0.5)])
    assert theta.shape == (nt,)
    return theta


class L2Loss(torch.autograd.Function):
    """sum over steps of the mean over the P patches of |D - Y|^2 (Sec. 6.3)."""

    @staticmethod
    def forward(ctx, D, Y, P):
        dD = torch.empty_like(D)
        loss = dnnmg.dnnmg_l2_loss(D, Y, P, dD)
        ctx.save_for_backward(dD)
        return loss.to(torch.float32).reshape(())

    @staticmethod
    def backward(ctx, g):
        (dD,) = ctx.saved_tensors
        return dD * g, None, None


class PatchNetTrainer:
    """Weights of the patch network and Adam state; one update per window."""

    def __init__(self, n_in, ldx, H, n_out, T, P, seed=0, std=0.1, out_std=None, lr=1e-3, alpha=1e-4,
                 device="cuda", precision="f32", head=False):
        """Initial weights N(0, std^2); the output layer N(0, out_std^2) if given
        (0: zero, so that the untrained net predicts d = 0).  precision: "f32"
        products on the CUDA cores, or "bf16" products on the tensor cores
        (FP32 master weights and Adam state either way).  head: train the
        convolutional head of Sec. 6.2 too (``head_init``; its parameters are
        the fourth entry of ``params``)."""
        Wx, Uh, Wfc = synth.net_weights(n_in, H, n_out, seed=seed, std=std)
        if out_std is not None:
            Wfc = Wfc * (out_std / std)
        W = [Wx, Uh, Wfc] + ([head_init(n_out, seed)] if head else [])
        self.params = [torch.tensor(w, dtype=torch.float32, device=device).contiguous() for w in W]
        self.head = head
        for p in self.params:
            p.requires_grad_(True)
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.step_no = 0
        self.lr, self.alpha = lr, alpha
        self.trainer = dnnmg.Trainer(n_in, ldx, H, n_out, T, P, precision=precision)
        self.P = P

    def weights(self):
        """[Wx, Uh, Wfc] (and theta with the head) as float64 host arrays."""
        return [p.detach().double().cpu().numpy() for p in self.params]

    def net(self, precision="f32"):
        """An inference net (dnnmg.Net) with the current weights."""
        W = self.weights()
        return dnnmg.Net(W[0], W[1], W[2], precision=precision, head=W[3] if self.head else None)

    def loss(self, X, Y, h0=None):
        """Loss of the window (data term; autograd-connected) and its D."""
        Wx, Uh, Wfc = self.params[:3]
        if self.head:
            Wfc = HeadFold.apply(self.params[3], Wfc)
        D = GruWindow.apply(X, h0, Wx, Uh, Wfc, self.trainer)
        return L2Loss.apply(D, Y, self.P), D

    def train_window(self, X, Y, h0=None):
        """One Adam update on one window; returns (loss incl. Tikhonov, h_T)."""
        for p in self.params:
            p.grad = None
        L, _ = self.loss(X, Y, h0)
        L.backward()
        self.step_no += 1
        with torch.no_grad():
            for p, m, v in zip(self.params, self.m, self.v):
                dnnmg.dnnmg_adam_step(p, p.grad, m, v, self.step_no, lr=self.lr, alpha=self.alpha)
            reg = sum(dnnmg.dnnmg_sumsq(p) for p in self.params)
        hT = self.trainer.state().clone()
        return float(L.detach()) + self.alpha * float(reg), hT


def patch_node_index(mesh):
    """For every fluid patch and output column (u then v on the patch's fine
    nodes, lexicographic, x fastest): the element of a pitched [2][plane] field."""
    I = mesh.info
    pc = torch.zeros(I.P, dtype=torch.int32, device="cuda")
    dnnmg.dnnmg_mesh_maps(mesh, patch_cell=pc)
    pc = pc.cpu().numpy().astype(np.int64)
    S = I.nxf // I.npx
    pi, pj = pc % I.npx, pc // I.npx
    lj, li = np.meshgrid(np.arange(S + 1), np.arange(S + 1), indexing="ij")
    I_ = pi[:, None] * S + li.ravel()[None, :]
    J_ = pj[:, None] * S + lj.ravel()[None, :]
    node = J_ * I.pitch + I_
    return torch.as_tensor(np.concatenate([node, node + I.plane], axis=1), device="cuda")


def reference(mesh, spec):
    """v_bar(t) [2][plane]: the synthetic flow on the fine nodes, with the
    Dirichlet values of x~ = P x_c (time independent: no start-up ramp) at the
    mesh's Dirichlet nodes."""
    I = mesh.info
    flags = torch.zeros(I.plane, dtype=torch.uint8, device="cuda")
    dnnmg.dnnmg_mesh_maps(mesh, node_flags=flags)
    dirichlet = (flags & 1).bool()
    xf = mesh.fine(3)
    dnnmg.dnnmg_prolongate(mesh, torch.zeros(3 * I.Nc, dtype=torch.float64, device="cuda"), xf, 0.0)
    bc = xf[:2].clone()

    def at(t):
        v = mesh.pack(synth.fine_state(spec, I.nxf, I.nyf, t)[:2])
        return torch.where(dirichlet, bc, v)
    return at


def flow_windows(mesh, spec, nsteps, k=synth.DT, t0=0.0):
    """Features X [nsteps][P][ldx] and targets Y [nsteps][P][n_out] of a
    synthetic flow at t_n = t0 + n k, n = 1 .. nsteps (see the module docstring)."""
    I = mesh.info
    assert mesh.real == torch.float32 and mesh.feat == torch.float32, "training needs a DNNMG_F32 mesh"
    idx = patch_node_index(mesh)
    X = torch.empty(nsteps, I.P, I.ldx, dtype=torch.float32, device="cuda")
    Y = torch.empty(nsteps, I.P, I.n_out, dtype=torch.float32, device="cuda")
    xf, bf = mesh.fine(3), mesh.fine(2)
    fine_ref = reference(mesh, spec)
    prev = fine_ref(t0)
    for n in range(nsteps):
        t = t0 + (n + 1) * k
        xc = torch.as_tensor(synth.coarse_state(spec, I.nxc, I.nyc, t)).cuda().contiguous()
        dnnmg.dnnmg_prolongate(mesh, xc, xf, t)
        dnnmg.dnnmg_rhs(mesh, prev, bf)
        dnnmg.dnnmg_patch_features(mesh, xf, bf, X[n])
        ref = fine_ref(t)
        Y[n] = (ref.reshape(-1)[idx] - xf[:2].reshape(-1)[idx])
        prev = ref
    return X, Y


def solution_windows(mesh, fine_states, coarse_states, k=synth.DT, t0=0.0):
    """Features X [T][P][ldx] and targets Y [T][P][n_out] from solved flows.

    The training data of Sec. 5.2 ("Training of DNN-MG"): fine_states =
    [x_bar(t_0), ..., x_bar(t_T)], the fine-level solution (node-ordered
    [3][Nf] float64, e.g. ``solver.simulate`` on the fine level; entry 0 is
    the state before the window), and coarse_states = [x_c(t_1), ...,
    x_c(t_T)] ([3][Nc] float64): the coarse solution the network sees, either
    the fine solution at the coarse nodes or a coarse-level simulation.
    Step n: x~ = P x_c(t_n) with the Dirichlet values at t_n, b_f =
    Rhs(v_bar(t_{n-1})), features from the library's S2+S3, and targets
    y = v_bar(t_n) - x~ on every patch's fine nodes.
    """
    I = mesh.info
    assert mesh.real == torch.float32 and mesh.feat == torch.float32, "training needs a DNNMG_F32 mesh"
    T = len(coarse_states)
    if len(fine_states) != T + 1:
        raise ValueError("fine_states needs one state more than coarse_states")
    idx = patch_node_index(mesh)
    X = torch.empty(T, I.P, I.ldx, dtype=torch.float32, device="cuda")
    Y = torch.empty(T, I.P, I.n_out, dtype=torch.float32, device="cuda")
    xf, bf = mesh.fine(3), mesh.fine(2)
    for n in range(T):
        t = t0 + (n + 1) * k
        xc = torch.as_tensor(np.ascontiguousarray(coarse_states[n], dtype=np.float64).reshape(-1)).cuda()
        dnnmg.dnnmg_prolongate(mesh, xc, xf, t)
        dnnmg.dnnmg_rhs(mesh, mesh.pack(np.asarray(fine_states[n])[:2]), bf)
        dnnmg.dnnmg_patch_features(mesh, xf, bf, X[n])
        ref = mesh.pack(np.asarray(fine_states[n + 1])[:2])
        Y[n] = ref.reshape(-1)[idx] - xf[:2].reshape(-1)[idx]
    return X, Y


def coarse_nodes(mesh, fine_state):
    """The fine-level state at the coarse nodes ([3][Nf] -> [3][Nc]), which
    coincide with every 2^K-th fine node: the coarse member of a two-level
    representation of one fine solution."""
    I = mesh.info
    r = 2 ** I.K
    a = np.asarray(fine_state).reshape(3, I.nyf + 1, I.nxf + 1)[:, ::r, ::r]
    return np.ascontiguousarray(a).reshape(3, -1)


def e_rel(mesh, weights, spec, steps, H, k=synth.DT, t0=0.0):
    """Mean over steps of E_rel(v) = |x~ + d_bar - v_bar| / |v_bar| (fine velocity
    DOFs) for a net with the given (Wx, Uh, Wfc), and the same with d = 0;
    the net runs through the inference kernels with its state carried."""
    I = mesh.info
    X, _ = flow_windows(mesh, spec, steps, k, t0)
    net = dnnmg.Net(*weights, precision="f32")
    h = torch.zeros(I.P, H, dtype=torch.float32, device="cuda")
    d = torch.empty(I.P, I.n_out, dtype=torch.float32, device="cuda")
    xf, vc = mesh.fine(3), mesh.fine(2)
    mask = torch.zeros(2, I.nyf + 1, I.pitch, dtype=torch.bool, device="cuda")
    mask[:, :, :I.nxf + 1] = True
    mask = mask.reshape(2, -1)
    fine_ref = reference(mesh, spec)
    with_net, without = [], []
    for n in range(steps):
        t = t0 + (n + 1) * k
        xc = torch.as_tensor(synth.coarse_state(spec, I.nxc, I.nyc, t)).cuda().contiguous()
        dnnmg.dnnmg_prolongate(mesh, xc, xf, t)
        dnnmg.dnnmg_gru_step(net, X[n], h, d, I.P)
        dnnmg.dnnmg_scatter_avg(mesh, d, xf, vc)
        ref = fine_ref(t)
        nrm = torch.linalg.norm(ref[mask].double())
        with_net.append(float(torch.linalg.norm((vc - ref)[mask].double()) / nrm))
        without.append(float(torch.linalg.norm((xf[:2] - ref)[mask].double()) / nrm))
    return float(np.mean(with_net)), float(np.mean(without))


def bench(P=65536, T=10, n_in=51, H=64, n_out=18, iters=10, warmup=3, precision="f32", head=False):
    """Time one training update (window forward, backward, Adam) at the
    training workload's batch (65 536 patches, T = 10, H = 64, K = 1 net) on
    random inputs (the cost does not depend on the values); ``head``: with the
    convolutional head (its fold and fold gradient in every update)."""
    import json
    ldx = (n_in + 15) // 16 * 16
    g = torch.Generator(device="cuda").manual_seed(0)
    X = torch.randn(T, P, ldx, device="cuda", generator=g)
    Y = 0.1 * torch.randn(T, P, n_out, device="cuda", generator=g)
    tn = PatchNetTrainer(n_in, ldx, H, n_out, T, P, seed=0, std=0.05, out_std=0.05, precision=precision, head=head)
    for _ in range(warmup):
        tn.train_window(X, Y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(iters):
        tn.train_window(X, Y)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / iters
    fwd = 2.0 * T * P * (3 * H * (n_in + H) + n_out * H)      # the window's forward products
    flops = 3.0 * fwd                                          # + state and weight gradients
    line = {"metric": "training update time", "unit": "ms", "value": ms, "patches": P, "T": T, "H": H,
            "n_in": n_in, "n_out": n_out, "gflop_per_update": flops / 1e9,
            "tflops": flops / (ms / 1e3) / 1e12, "dtype": precision, "head": bool(head), "data": "synthetic"}
    print(json.dumps(line))
    return line


if __name__ == "__main__":
    import sys
    bench(precision=sys.argv[1] if len(sys.argv) > 1 else "f32", head="--head" in sys.argv[2:])


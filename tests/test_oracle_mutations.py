"""Planted mistakes in the oracle must fail its pins.

Each case patches one plausible slip into an oracle function (on the CPU,
for the duration of the test) and runs pins that should catch it: a pin set
that passes a wrong oracle pins nothing.
"""

import numpy as np
import pytest

import test_oracle_assembly as assembly
import test_oracle_head as hpins
import test_oracle_pins as pins
import test_train_oracle as tpins
from oracle import average, features, fem, gru, head, transfer
from oracle import train as otrain


def _fails(checks):
    for check in checks:
        try:
            check()
        except AssertionError:
            return True
    return False


def _assembly_pins():
    return [lambda n=n: assembly.test_residual_equals_dense_assembly(n) for n in sorted(assembly.MESHES)] + \
           [lambda n=n: assembly.test_rhs_equals_dense_assembly(n) for n in sorted(assembly.MESHES)]


def _zero_step_pins():
    return [lambda K=K, s=s: pins.test_zero_correction_step_gives_coarse_rhs(K, s)
            for K in (1, 2) for s in (1, 2)]


def _gru_pins():
    return [pins.test_gru_hand_derived, pins.test_gru_recurrent_gates_and_zero_weights]


def _lps_pins():
    return [pins.test_lps_energy_closed_form, pins.test_lps_orthogonal_to_patchwise_bilinear] + _assembly_pins()


def _train_pins():
    return [lambda a=a: tpins.test_bptt_gradient_matches_finite_differences(a) for a in (0.0, 1e-4)] + \
           [tpins.test_gradient_of_a_single_step_by_hand, tpins.test_adam_closed_forms]


def _feature_pins():
    return [pins.test_features_hand_indexed]


def _average_pins():
    return [pins.test_constant_correction_survives_averaging, pins.test_general_constant_correction_within_one_ulp,
            pins.test_averaging_of_two_patch_predictions]


def _head_pins():
    return [lambda n=n: hpins.test_spatial_block_is_library_correlation_then_convolution(n) for n in hpins.N_OUTS] + \
           [lambda n=n: hpins.test_vertex_block_is_library_correlation_then_convolution(n) for n in hpins.N_OUTS] + \
           [lambda n=n: hpins.test_blocks_are_symmetric_positive_semidefinite(n) for n in hpins.N_OUTS] + \
           [lambda n=n: hpins.test_fold_gradient_matches_central_differences(n) for n in hpins.N_OUTS]


def _mutants():
    o_pi, o_vop, o_shape = fem.lps_projection_matrix, fem.velocity_operator, fem.q1_shape
    o_rhs_raw, o_restrict_1d, o_pro = fem.rhs_raw, transfer._restrict_1d, transfer.prolongate_raw

    def vop_pressure_sign(mesh, prm, t):
        Au, Av = o_vop(mesh, prm, t)
        return Au + 2 * t["pres_u"], Av + 2 * t["pres_v"]

    def vop_full_convection(mesh, prm, t):
        Au, Av = o_vop(mesh, prm, t)
        return Au + 0.5 * t["conv_u"], Av + 0.5 * t["conv_v"]

    def vop_full_viscosity(mesh, prm, t):
        Au, Av = o_vop(mesh, prm, t)
        return Au + 0.5 * prm.nu * t["diff_u"], Av + 0.5 * prm.nu * t["diff_v"]

    def rhs_convection_sign(mesh, prm, t):
        bu, bv = o_rhs_raw(mesh, prm, t)
        return bu + t["conv_u"], bv + t["conv_v"]

    def shape_swapped(xi, eta):
        phi, dx, dy = o_shape(xi, eta)
        return phi, dy, dx

    def prolongate_shifted(mesh, xc):
        x = o_pro(mesh, xc)
        return x + 1e-3 * (np.arange(x.shape[1]) % 3 == 1)

    def gru_reset_after_product(X, h, Wx, Uh, Wfc):
        # the variant that applies the reset gate after the recurrent product
        X, h = np.asarray(X, dtype=np.float64), np.asarray(h, dtype=np.float64)
        H = h.shape[1]
        z = gru.sigmoid(X @ Wx[0:H].T + h @ Uh[0:H].T)
        r = gru.sigmoid(X @ Wx[H:2 * H].T + h @ Uh[H:2 * H].T)
        cand = np.tanh(X @ Wx[2 * H:].T + r * (h @ Uh[2 * H:].T))
        h_new = z * h + (1.0 - z) * cand
        return h_new, h_new @ np.asarray(Wfc).T

    def lps_without_test_projection(mesh, prm, p, nq=2):
        # projects the pressure but not the test function
        nxn = mesh.wxf + 1
        F = np.eye(9) - fem.lps_projection_matrix()
        L = fem.lps_patch_stiffness(mesh.hxf, mesh.hyf, nq)
        blk = mesh.solid_f.reshape(mesh.wyf // 2, 2, mesh.wxf // 2, 2)
        n, m = np.nonzero(~blk.any(axis=(1, 3)))
        offs = np.array([b * nxn + a for b in range(3) for a in range(3)])
        nodes = ((2 * n) * nxn + 2 * m)[:, None] + offs[None, :]
        out = np.zeros(mesh.Nf)
        np.add.at(out, nodes, fem.lps_alpha(mesh, prm) * (p[nodes] @ F.T) @ L.T)
        return out

    o_grad_D, o_backward, o_adam = otrain.loss_grad_D, otrain.seq_backward, otrain.adam_step

    def backward_without_reset_recurrence(dD, cache, Wx, Uh, Wfc):
        gWx, gUh, gWfc, dh0 = o_backward(dD, cache, Wx, Uh, Wfc)
        H = Uh.shape[1]
        gUh = gUh.copy()
        gUh[H:2 * H] = 0.0
        return gWx, gUh, gWfc, dh0

    def adam_without_bias_correction(p, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        m = b1 * m + (1.0 - b1) * g
        v = b2 * v + (1.0 - b2) * g * g
        return p - lr * m / (np.sqrt(v) + eps), m, v

    o_fold_bw, o_vertex = head.fold_backward, head.vertex_block
    o_feat, o_geo, o_avg = features.patch_features, features.patch_geometry, average.scatter_average

    def features_uv_swapped(mesh, prm, xf, r):
        # the coarse u and v columns exchanged (D9 orders u before v)
        X = o_feat(mesh, prm, xf, r).copy()
        nf, nc = mesh.nf, mesh.nc
        u0 = 3 * nf
        X[:, u0:u0 + nc], X[:, u0 + nc:u0 + 2 * nc] = X[:, u0 + nc:u0 + 2 * nc].copy(), X[:, u0:u0 + nc].copy()
        return X

    def geometry_angles_in_degrees(mesh):
        g = o_geo(mesh).copy()
        g[8:] = np.degrees(g[8:])
        return g

    def average_by_sum(mesh, d, xf):
        # sums the predictions of a shared node instead of averaging them
        fine, _ = features.patch_node_indices(mesh)
        v = np.array([np.asarray(xf[0], dtype=np.float64), np.asarray(xf[1], dtype=np.float64)])
        d = np.asarray(d, dtype=np.float64)
        sums = np.zeros((2, mesh.Nf))
        for p in range(mesh.P):
            sums[0, fine[p]] += d[p, :mesh.nf]
            sums[1, fine[p]] += d[p, mesh.nf:]
        free = ~mesh.dirichlet.ravel()
        v[:, free] += sums[:, free]
        return v

    def fold_backward_one_product(theta, Wfc, G):
        # drops the (C_f x)[p] q[p + t] half of each filter's gradient
        dth, dW = o_fold_bw(theta, Wfc, G)
        dth = dth.copy()
        dth[:head.NF * (head.KS ** 2 + head.KV)] *= 0.5
        return dth, dW

    def vertex_without_interleaving(y, kv):
        # the components one after the other instead of vertex by vertex
        y = np.asarray(y, dtype=np.float64)
        acc = np.zeros_like(y)
        for f in range(head.NF):
            acc += head.corr1d_t(head.corr1d(y, kv[f]), kv[f])
        return acc

    return {
        "coarse u and v features swapped": (features, "patch_features", features_uv_swapped, _feature_pins),
        "geometry angles in degrees": (features, "patch_geometry", geometry_angles_in_degrees, _feature_pins),
        "shared-node predictions summed, not averaged": (average, "scatter_average", average_by_sum, _average_pins),
        "transposed head layer not the adjoint": (head, "corr2d_t", head.corr2d, _head_pins),
        "vertex block without interleaving": (head, "vertex_block", vertex_without_interleaving, _head_pins),
        "head filter gradient halved": (head, "fold_backward", fold_backward_one_product, _head_pins),
        "loss gradient without its factor 2": (otrain, "loss_grad_D", lambda D, Y: 0.5 * o_grad_D(D, Y),
                                               _train_pins),
        "reset-gate recurrent gradient dropped": (otrain, "seq_backward", backward_without_reset_recurrence,
                                                  _train_pins),
        "Adam without bias correction": (otrain, "adam_step", adam_without_bias_correction, _train_pins),
        "reset gate after the recurrent product": (gru, "gru_step", gru_reset_after_product, _gru_pins),
        "projection of the test function dropped": (fem, "lps_term", lps_without_test_projection, _lps_pins),
        "projection transposed": (fem, "lps_projection_matrix", lambda: o_pi().T, _assembly_pins),
        "pressure term sign": (fem, "velocity_operator", vop_pressure_sign, _assembly_pins),
        "convection weight 1 not 1/2": (fem, "velocity_operator", vop_full_convection, _assembly_pins),
        "viscosity nu not nu/2": (fem, "velocity_operator", vop_full_viscosity, _assembly_pins),
        "alpha from h_x alone": (fem, "lps_alpha", lambda m, p: p.alpha0 * m.hxf ** 2 / p.nu, _assembly_pins),
        "x and y derivatives swapped": (fem, "q1_shape", shape_swapped, _assembly_pins),
        "right-hand side convection sign": (fem, "rhs_raw", rhs_convection_sign, _assembly_pins),
        "restriction weights scaled": (transfer, "_restrict_1d", lambda v, axis: 1.01 * o_restrict_1d(v, axis),
                                       _zero_step_pins),
        "prolongation perturbed": (transfer, "prolongate_raw", prolongate_shifted, _zero_step_pins),
        "inexact quadrature": (fem, "gauss_1d", lambda nq: (np.array([0.25, 0.75]), np.array([0.5, 0.5])),
                               _zero_step_pins),
    }


MUTANTS = _mutants()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(name, monkeypatch):
    module, attr, wrong, checks = MUTANTS[name]
    # the pins hold for the oracle as written ...
    assert not _fails(checks())
    # ... and fail with the mistake planted
    monkeypatch.setattr(module, attr, wrong)
    assert _fails(checks()), f"no pin caught: {name}"

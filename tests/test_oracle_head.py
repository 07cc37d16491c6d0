"""Pins of the oracle's convolutional head (Sec. 6.2, K = 1 network).

Each block against library correlations and convolutions, its symmetry and
positivity (a transposed layer with the first layer's weights), the identity
for centred unit filters, the paper's parameter count, the fold of the head
into the output layer, and the fold's gradient by central differences (exact
up to rounding: the fold is linear in W_fc and w and quadratic in the filters).
"""

import numpy as np
import pytest
from scipy import signal

from oracle import gru, head

N_OUTS = (18, 50)      # patches of 3 x 3 and 5 x 5 nodes


def _theta(n_out, seed):
    return np.random.default_rng(seed).standard_normal(head.n_theta(n_out))


def _dense(block, n_out, k):
    return np.stack([block(np.eye(n_out)[i], k) for i in range(n_out)], axis=1)


def test_parameter_count_of_the_paper():
    # Sec. 6.2: 8634 parameters for N_in = 51, N_GRU = 32, N_out = 18
    assert gru.param_count(51, 32, 18) + head.param_count(18) == 8634


@pytest.mark.parametrize("n_out", N_OUTS)
def test_spatial_block_is_library_correlation_then_convolution(n_out):
    ks, _, _ = head.split(_theta(n_out, 1), n_out)
    y = np.random.default_rng(2).standard_normal(n_out)
    nf = n_out // 2
    n = int(round(np.sqrt(nf)))
    ref = np.zeros(n_out)
    for comp in range(2):
        g = y[comp * nf:(comp + 1) * nf].reshape(n, n)
        acc = sum(signal.convolve2d(signal.correlate2d(g, ks[f], mode="same"), ks[f], mode="same")
                  for f in range(head.NF))
        ref[comp * nf:(comp + 1) * nf] = acc.ravel()
    np.testing.assert_allclose(head.spatial_block(y, ks), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("n_out", N_OUTS)
def test_vertex_block_is_library_correlation_then_convolution(n_out):
    _, kv, _ = head.split(_theta(n_out, 3), n_out)
    y = np.random.default_rng(4).standard_normal(n_out)
    nf = n_out // 2
    s = np.ravel(np.column_stack([y[:nf], y[nf:]]))       # u_0, v_0, u_1, v_1, ...
    acc = sum(np.convolve(np.correlate(s, kv[f], mode="same"), kv[f], mode="same") for f in range(head.NF))
    ref = np.concatenate([acc[0::2], acc[1::2]])
    np.testing.assert_allclose(head.vertex_block(y, kv), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("n_out", N_OUTS)
def test_blocks_are_symmetric_positive_semidefinite(n_out):
    ks, kv, _ = head.split(_theta(n_out, 5), n_out)
    for block, k in ((head.spatial_block, ks), (head.vertex_block, kv)):
        B = _dense(block, n_out, k)
        np.testing.assert_allclose(B, B.T, rtol=0, atol=1e-12 * np.abs(B).max())
        assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > -1e-12 * np.abs(B).max()


def test_spatial_block_couples_only_neighbours_of_one_component():
    ks, _, _ = head.split(_theta(18, 6), 18)
    B = _dense(head.spatial_block, 18, ks)
    assert not B[:9, 9:].any() and not B[9:, :9].any()
    # B = C^T C reaches two nodes apart: nodes 0 and 8 (opposite corners) couple, a 5 x 5 patch's
    # nodes 0 and 3 (three apart in a row) do not
    assert B[0, 8] != 0
    ks5, _, _ = head.split(_theta(50, 6), 50)
    assert _dense(head.spatial_block, 50, ks5)[0, 3] == 0


def test_centred_unit_filters_give_identity_blocks():
    theta = np.zeros(head.n_theta(18))
    ks, kv, w = head.split(theta, 18)
    ks[0, 1, 1], kv[0, 4] = 1.0, 1.0
    w[:] = np.arange(1, 19)
    theta = np.concatenate([ks.ravel(), kv.ravel(), w])
    y = np.random.default_rng(7).standard_normal(18)
    np.testing.assert_allclose(head.head(y, theta), 2.0 * w * y, rtol=1e-15, atol=0)


def test_vertex_block_couples_the_components_of_a_vertex():
    # a length-9 filter with only its offset +1 and -1 taps: u_i couples v_i (its neighbour in the sequence)
    _, kv, _ = head.split(np.zeros(head.n_theta(18)), 18)
    kv[0, 5] = 1.0
    B = _dense(head.vertex_block, 18, kv)
    # C^T C with a single +1 offset: the identity on every sequence entry but the first
    assert B[9, 9] == 1.0 and B[0, 0] == 0.0
    kv[0, 4], kv[0, 5] = 1.0, 1.0
    B = _dense(head.vertex_block, 18, kv)
    assert B[0, 9] != 0 and B[9, 0] == B[0, 9]


@pytest.mark.parametrize("n_out", N_OUTS)
def test_fold_is_the_head_after_the_output_layer(n_out):
    rng = np.random.default_rng(8)
    theta, Wfc = _theta(n_out, 9), rng.standard_normal((n_out, 6))
    h = rng.standard_normal((5, 6))
    Weff = head.fold(theta, Wfc)
    np.testing.assert_allclose(h @ Weff.T, head.head_rows(h @ Wfc.T, theta), rtol=0, atol=1e-12 * np.abs(Weff).max())


@pytest.mark.parametrize("n_out", N_OUTS)
def test_fold_gradient_matches_central_differences(n_out):
    rng = np.random.default_rng(10)
    H = 3
    theta, Wfc, G = _theta(n_out, 11), rng.standard_normal((n_out, H)), rng.standard_normal((n_out, H))

    def loss(th, W):
        return float(np.sum(G * head.fold(th, W)))

    dth, dW = head.fold_backward(theta, Wfc, G)
    eps = 1e-3
    fd_th = np.array([(loss(theta + eps * e, Wfc) - loss(theta - eps * e, Wfc)) / (2 * eps)
                      for e in np.eye(len(theta))])
    np.testing.assert_allclose(dth, fd_th, rtol=0, atol=1e-8 * np.abs(fd_th).max())
    for i, j in ((0, 0), (n_out // 2, 1), (n_out - 1, H - 1)):
        E = np.zeros_like(Wfc)
        E[i, j] = eps
        fd = (loss(theta, Wfc + E) - loss(theta, Wfc - E)) / (2 * eps)
        assert abs(dW[i, j] - fd) <= 1e-8 * np.abs(dW).max()

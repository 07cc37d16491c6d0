"""Host-side parts of the convolutional head (no GPU): the parameter count the
library reports and the trainer's initial head (reading: near the identity)."""

import numpy as np
import pytest

from oracle import head


@pytest.fixture(scope="module")
def train():
    from paper_2008_11520_gb300 import build
    import os
    if not os.path.exists(build.LIB):
        build.build()
    from paper_2008_11520_gb300 import train
    return train


def test_library_head_sizes(train):
    dn = train.dnnmg
    for n in (3, 5, 7, 9):
        assert dn.head_params(2 * n * n) == head.n_theta(2 * n * n)
    for n_out in (0, 2, 8, 18 + 2, 2 * 11 * 11):
        assert dn.head_params(n_out) == 0


@pytest.mark.parametrize("n_out", [18, 50])
def test_initial_head_is_near_the_identity(train, n_out):
    theta = train.head_init(n_out, seed=3)
    ks, kv, w = head.split(theta, n_out)
    assert ks[0, 1, 1] == 1.0 and kv[0, 4] == 1.0 and np.count_nonzero(ks[0]) == 1 and np.count_nonzero(kv[0]) == 1
    assert (w == 0.5).all() and np.abs(ks[1:]).max() < 0.3 and np.abs(kv[1:]).max() < 0.3
    # every filter of both blocks is nonzero, so each gets a gradient
    assert all(np.abs(k).sum() > 0 for k in list(ks) + list(kv))
    W = np.random.default_rng(0).standard_normal((n_out, 16))
    Weff = head.fold(theta, W)
    assert np.linalg.norm(Weff - W) < 0.1 * np.linalg.norm(W)

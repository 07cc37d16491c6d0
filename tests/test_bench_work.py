"""The roofline numerators of bench.py: the algorithmic bytes and flops per
launch of each kernel on the large workload (2048 x 512 coarse cells, K = 2,
2 x 2-cell patches, H = 128, BF16 network), computed by hand from the node and
patch counts of the host-only size query."""

import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def info():
    from paper_2008_11520_gb300 import build, synth
    if not os.path.exists(build.LIB):
        build.build()
    from paper_2008_11520_gb300 import dnnmg
    c = synth.config("large")
    return dnnmg.dnnmg_mesh_query(dnnmg.make_desc(c["nxc"], c["nyc"], c["K"], c["s"], c["ellipse"],
                                                  precision=c["precision"])), c["H"]


def test_large_workload_counts(info):
    I, H = info
    assert (I.Nc, I.Nf) == (2049 * 513, 8193 * 2049)
    assert (I.n_in, I.n_out, I.ldx, H) == (282, 162, 288, 128)
    assert (I.real_bytes, I.feature_bytes) == (4, 2)
    # 262 144 patches before the obstacle's fully solid ones are removed
    assert 262144 - 2500 < I.P < 262144


def test_algorithmic_work_by_hand(info):
    import bench
    I, H = info
    Nc, Nf, P = I.Nc, I.Nf, I.P
    w = bench.algorithmic_work(I, H)
    by_hand = {
        "coarse_pad": 3 * Nc * 8 + 3 * Nc * 4,              # x_c FP64 in, padded FP32 copy out
        "residual_features": 3 * Nc * 4 + 2 * Nf * 4 + P * 288 * 2,   # coarse copy, b_f, X (BF16)
        "gru": P * 288 * 2 + 2 * P * 128 * 4 + P * 162 * 4,           # X, h in and out, d
        "scatter_avg": P * 162 * 4 + 2 * Nc * 4 + 2 * Nf * 4,         # d, coarse u v, v_corr
        "rhs": 2 * Nf * 4 + 2 * Nf * 4,                               # v_corr in, b_f out
        "restrict": 2 * Nf * 4 + 3 * Nc * 8,                          # b_f in, b_c out
    }
    assert {k: v["bytes"] for k, v in w.items()} == by_hand
    # GEMM flops: 2 P (3H (n_in + H) + H n_out), the network's 178 176 weights per patch
    assert 3 * 128 * (282 + 128) + 128 * 162 == 178176
    assert w["gru"]["flops"] == 2 * P * 178176
    # the figures quoted with the measurements (MB, GFLOP)
    mb = {k: round(v / 1e6) for k, v in by_hand.items()}
    assert mb == {"coarse_pad": 38, "residual_features": 297, "gru": 586, "scatter_avg": 312,
                  "rhs": 269, "restrict": 160}
    assert round(w["gru"]["flops"] / 1e9, 1) == 92.9


def test_dominant_kernel_is_the_largest_single_kernel():
    import bench
    # the bench's measured kernel times of the large workload: the GRU is the
    # largest kernel although the two S2+S3 kernels together take longer
    ms = {"coarse_pad": 0.0126, "residual_cf": 0.171, "residual_boundary": 0.036, "gru": 0.185,
          "scatter_avg": 0.098, "rhs": 0.117, "restrict": 0.054}
    assert bench.dominant(ms) == ("gru", 0.185)
    ms["residual_cf"] = 0.2
    name, t = bench.dominant(ms)
    assert name == "residual_features" and t == pytest.approx(0.236)
    ms = {"coarse_pad": 0.01, "residual_features": 0.3, "gru": 0.2}
    assert bench.dominant(ms) == ("residual_features", 0.3)

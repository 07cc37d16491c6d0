"""Host logic of the serving loop (no GPU): the state-pool allocator of the
C ABI, the continuous-batching policy, the request loop on a virtual clock,
admission by memory budget, and the seeded serving workload."""

from collections import deque

import numpy as np
import pytest

from paper_2008_11520_gb300 import serve, synth


@pytest.fixture(scope="module")
def dn():
    from paper_2008_11520_gb300 import dnnmg
    return dnnmg


def test_row_pool_first_fit_and_coalescing(dn):
    p = dn.RowPool(1024, 128)
    a = p.alloc(100)          # rounded to 128
    b = p.alloc(300)          # 384
    c = p.alloc(128)
    assert (a, b, c) == (0, 128, 512)
    assert p.stats() == (640, 384)
    p.free(b)
    assert p.stats() == (256, 384)
    assert p.alloc(200) == 128        # first fit reuses the hole
    p.free(a)
    p.free(128)
    p.free(c)
    assert p.stats() == (0, 1024)     # everything coalesced back into one range
    assert p.alloc(1024) == 0


def test_row_pool_errors(dn):
    p = dn.RowPool(512, 128)
    p.alloc(512)
    with pytest.raises(dn.DnnmgError) as e:
        p.alloc(1)
    assert e.value.code == 4          # DNNMG_ENOMEM
    with pytest.raises(dn.DnnmgError) as e:
        p.free(128)                   # no range starts there
    assert e.value.code == 1
    with pytest.raises(dn.DnnmgError):
        p.alloc(0)


def test_row_pool_random_against_a_bitmap(dn):
    # brute force: a bitmap of units; every allocation is free there, first fit
    rng = np.random.default_rng(0)
    units, unit = 64, 128
    p = dn.RowPool(units * unit, unit)
    used = np.zeros(units, bool)
    live = {}
    for _ in range(400):
        if live and rng.random() < 0.45:
            s = list(live)[rng.integers(len(live))]
            p.free(s)
            used[s // unit: s // unit + live.pop(s)] = False
            continue
        n = int(rng.integers(1, 9))
        # first free run of n units
        run, want = 0, None
        for u in range(units):
            run = run + 1 if not used[u] else 0
            if run == n:
                want = (u - n + 1) * unit
                break
        if want is None:
            with pytest.raises(dn.DnnmgError):
                p.alloc(n * unit)
            continue
        s = p.alloc(n * unit - int(rng.integers(0, unit)))
        assert s == want
        used[s // unit: s // unit + n] = True
        live[s] = n
        assert p.stats()[0] == used.sum() * unit


def test_padded_rows():
    assert [serve.padded_rows(P) for P in (0, 1, 128, 129, 1000)] == [0, 128, 128, 256, 1024]


def test_batcher_one_request_per_instance_and_order():
    inst_of = np.array([0, 1, 0, 2, 1, 3])     # requests 0..5
    group_of = ["a", "a", "b", "b"]
    rows_of = [128, 256, 128, 128]
    b = serve.Batcher(inst_of, group_of, rows_of)
    pending = deque(range(6))
    batch = b.take(pending)
    assert batch == {"a": [0, 1], "b": [3, 5]}
    assert list(pending) == [2, 4]             # second requests of instances 0 and 1, in order
    assert b.take(pending) == {"a": [2, 4]}
    assert not pending


def test_batcher_row_cap_keeps_at_least_one():
    inst_of = np.array([0, 1, 2])
    b = serve.Batcher(inst_of, ["g"] * 3, [512, 256, 128], max_rows=384)
    pending = deque(range(3))
    assert b.take(pending) == {"g": [0]}       # over the cap alone, still served
    assert b.take(pending) == {"g": [1, 2]}


def test_run_loop_virtual_clock():
    # arrivals in three bursts; a batch costs 1 ms + 0.1 ms per request
    arrival = np.array([0.0, 0.0, 0.0005, 0.010, 0.010, 0.010, 0.0101, 0.030])
    inst_of = np.array([0, 1, 0, 2, 3, 2, 0, 1])
    b = serve.Batcher(inst_of, [0] * 4, [128] * 4)
    now = [0.0]
    ran = []

    def execute(batch):
        reqs = [r for v in batch.values() for r in v]
        ran.append(reqs)
        now[0] += 1e-3 + 1e-4 * len(reqs)

    def wait_until(t):
        now[0] = max(now[0], t)

    lat, sizes = serve.run_loop(arrival, b, execute, lambda: now[0], wait_until)
    assert np.isfinite(lat).all() and (lat > 0).all()
    assert sorted(r for x in ran for r in x) == list(range(len(arrival)))
    # an instance's requests complete in arrival order, one per batch
    done = {r: k for k, x in enumerate(ran) for r in x}
    for i in range(4):
        rs = [r for r in range(len(arrival)) if inst_of[r] == i]
        assert [done[r] for r in rs] == sorted(done[r] for r in rs)
        assert len({done[r] for r in rs}) == len(rs)
    assert ran[0] == [0, 1]                    # request 2 arrives while batch 0 runs
    assert sizes == [len(x) for x in ran]
    assert lat[0] == pytest.approx(1.2e-3)


def test_admit_by_budget():
    assert serve.admit_by_budget([5, 3, 4, 1], 9) == [0, 1, 3]
    assert serve.admit_by_budget([10], 9) == []


def test_serving_workload_ranges():
    specs = synth.serving_instances(200, 7)
    nx = np.array([c["nxc"] for c in specs])
    assert nx.min() >= 64 and nx.max() <= 512 and (nx % 16 == 0).all()
    assert all(c["nyc"] * 4 == c["nxc"] and c["nyc"] % 2 == 0 for c in specs)
    assert {c["K"] for c in specs} == {1, 2}
    ratio = np.array([c["ellipse"][3] / c["ellipse"][2] for c in specs])
    assert ratio.min() >= 0.5 and ratio.max() <= 1.0
    t, i = synth.poisson_requests(200.0, 50.0, 64, 3)
    assert abs(len(t) - 10000) < 5 * 100      # Poisson count, 5 standard deviations
    assert (np.diff(t) >= 0).all() and i.min() >= 0 and i.max() < 64
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0

"""Serving: a continuous-batching request loop of DNN-MG correction steps
(Algorithm 2) over many flow instances with different meshes.

Each request asks for one time step of one instance.  Instances are admitted
by a device-memory budget into per-net servers (libdnnmg's dnnmg_server_*):
instances whose meshes give the same network shape share a server, whose GRU
state pool keeps every admitted instance's h on the device; velocities (b_f)
and coarse vectors stay on the device too.  The loop takes, whenever the GPU
is free, the pending requests in arrival order (at most one per instance,
since an instance's steps are sequential) and runs them as one batched step
per server: S1-S3 per instance, S4 once over all of their patches, S5-S7 per
instance.  Latency of a request = completion of its batch - its arrival.

The batching policy (``Batcher``, ``run_loop``) is host logic and runs with
any ``execute``/clock, so it is tested on the CPU with a virtual clock.

Run ``python -m paper_2008_11520_gb300.serve`` on a GPU for one JSON line:
p50/p99 step latency at the offered load, and batched throughput with every
admitted instance stepping in each batch.
"""

import argparse
import json
import time
from collections import deque

import numpy as np

TILE_ROWS = 128


def padded_rows(P):
    """State rows an instance takes in its server: its fluid patches, whole 128-row tiles."""
    return (P + TILE_ROWS - 1) // TILE_ROWS * TILE_ROWS


class Batcher:
    """Which pending requests go into the next batch.

    inst_of[r]: the instance of request r; group_of[i]: the server of
    instance i; rows_of[i]: its padded patch rows; max_rows: optional cap on
    the rows of one server's batch (a latency knob; None = no cap).
    """

    def __init__(self, inst_of, group_of, rows_of, max_rows=None):
        self.inst_of, self.group_of, self.rows_of, self.max_rows = inst_of, group_of, rows_of, max_rows

    def take(self, pending):
        """Remove and return the next batch from the deque `pending` (request ids in
        arrival order), as {group: [request ids]}; the rest keep their order."""
        batch, seen, rows, keep = {}, set(), {}, deque()
        while pending:
            r = pending.popleft()
            i = self.inst_of[r]
            g = self.group_of[i]
            fits = self.max_rows is None or rows.get(g, 0) + self.rows_of[i] <= self.max_rows or not batch.get(g)
            if i in seen or not fits:
                keep.append(r)
                continue
            seen.add(i)
            rows[g] = rows.get(g, 0) + self.rows_of[i]
            batch.setdefault(g, []).append(r)
        pending.extend(keep)
        return batch


def run_loop(arrival, batcher, execute, clock, wait_until):
    """Serve the requests with arrival times `arrival` (sorted, seconds from the
    start of the loop).  execute(batch) runs a batch to completion; clock() is
    the time since the start; wait_until(t) blocks until clock() >= t.
    Returns (latency per request [s], batch sizes)."""
    n = len(arrival)
    latency = np.full(n, np.nan)
    sizes = []
    pending = deque()
    nxt = 0
    while nxt < n or pending:
        now = clock()
        while nxt < n and arrival[nxt] <= now:
            pending.append(nxt)
            nxt += 1
        if not pending:
            wait_until(arrival[nxt])
            continue
        batch = batcher.take(pending)
        execute(batch)
        done = clock()
        for reqs in batch.values():
            for r in reqs:
                latency[r] = done - arrival[r]
        sizes.append(sum(len(v) for v in batch.values()))
    return latency, sizes


def admit_by_budget(demands, budget):
    """Greedy admission in order: demands[i] = bytes instance i needs; admitted
    while the running total stays within `budget`.  Returns the admitted indices."""
    out, used = [], 0
    for i, b in enumerate(demands):
        if used + b <= budget:
            out.append(i)
            used += b
    return out


# ---------------------------------------------------------------- GPU runner
def _gpu_setup(n_instances, seed, H, budget_bytes):
    import torch

    from . import dnnmg, synth

    specs = synth.serving_instances(n_instances, seed)
    infos = [dnnmg.dnnmg_mesh_query(dnnmg.make_desc(c["nxc"], c["nyc"], c["K"], c["s"], c["ellipse"],
                                                    precision="bf16")) for c in specs]
    # one net per network shape (K decides n_in / n_out with one-cell patches)
    shapes = sorted({(I.n_in, I.n_out) for I in infos})
    nets = {sh: dnnmg.Net(*synth.net_weights(sh[0], H, sh[1], seed=seed + k), precision="bf16")
            for k, sh in enumerate(shapes)}
    group_of = [(I.n_in, I.n_out) for I in infos]
    rows_of = [padded_rows(I.P) for I in infos]
    # device bytes an instance needs: its state, feature and output rows in
    # its server, b_f, and x_c / b_c
    def demand(i):
        I = infos[i]
        return rows_of[i] * (H * 4 + I.ldx * 2 + I.n_out * 4) + 2 * I.plane * 4 + 2 * 3 * I.Nc * 8
    admitted = admit_by_budget([demand(i) for i in range(n_instances)], budget_bytes)
    servers = {}
    for sh, net in nets.items():
        rows = sum(rows_of[i] for i in admitted if group_of[i] == sh)
        if rows:
            servers[sh] = dnnmg.Server(net, rows)
    dev = torch.device("cuda")
    inst = {}
    for i in admitted:
        c = specs[i]
        mesh = dnnmg.Mesh(dnnmg.make_desc(c["nxc"], c["nyc"], c["K"], c["s"], c["ellipse"], precision="bf16"))
        slot = servers[group_of[i]].admit(mesh)
        I = mesh.info
        spec = synth.FlowSpec.from_seed(c["seed"], c["ellipse"])
        xc = torch.as_tensor(synth.coarse_state(spec, c["nxc"], c["nyc"], 0.0)).to(dev).contiguous()
        v0 = synth.fine_state(spec, I.nxf, I.nyf, 0.0)[:2]
        bf = mesh.fine(2, dev)
        bc = mesh.coarse(3, dev)
        dnnmg.dnnmg_rhs_restrict(mesh, mesh.pack(v0, dev), bf, bc)
        inst[i] = dict(mesh=mesh, slot=slot, xc=xc, bf=bf, bc=bc, t=0.0, dof=2 * I.Nf)
    torch.cuda.synchronize()
    return specs, infos, servers, inst, group_of, rows_of, admitted


def main(argv=None):
    import torch

    from . import synth

    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--rates", default="200,2000,8000", help="offered step requests per second, one run each")
    ap.add_argument("--duration", type=float, default=3.0, help="seconds of arrivals per run")
    ap.add_argument("--budget-gb", type=float, default=8.0, help="device memory for admitted instances")
    ap.add_argument("--max-rows", type=int, default=None, help="cap on one server batch's patch rows")
    ap.add_argument("--H", type=int, default=64)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--sat-iters", type=int, default=20)
    args = ap.parse_args(argv)

    specs, infos, servers, inst, group_of, rows_of, admitted = _gpu_setup(
        args.instances, args.seed, args.H, int(args.budget_gb * 2 ** 30))
    k = synth.DT
    adm = sorted(inst)

    def launch(batch, inst_of):
        for g, reqs in batch.items():
            items = []
            for r in reqs:
                s = inst[inst_of[r]]
                items.append((s["slot"], s["xc"], s["bf"], s["bc"], s["t"]))
                s["t"] += k
            servers[g].step(items)

    every = np.array(adm)
    full = Batcher(every, group_of, rows_of).take(deque(range(len(adm))))
    launch(full, every)   # warm-up: every admitted instance once
    torch.cuda.synchronize()

    runs = []
    for rate in (float(x) for x in args.rates.split(",")):
        arrival, which = synth.poisson_requests(rate, args.duration, len(adm), args.seed)
        inst_of = every[which]
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0

        def wait_until(t):
            while clock() < t:
                pass

        def execute(batch):
            launch(batch, inst_of)
            torch.cuda.synchronize()

        latency, sizes = run_loop(arrival, Batcher(inst_of, group_of, rows_of, args.max_rows), execute, clock,
                                  wait_until)
        wall = clock()
        lat_ms = latency * 1e3
        runs.append({"offered_steps_per_s": rate, "requests": int(len(arrival)),
                     "served_steps_per_s": len(arrival) / wall,
                     "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
                     "mean_ms": float(lat_ms.mean()), "mean_batch": float(np.mean(sizes)), "batches": len(sizes)})

    # saturated: every admitted instance in every round, as one batch per
    # server, against the same steps issued one instance per call
    def timed(rounds, per_round):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(rounds):
            per_round()
        ev1.record()
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / 1e3 / rounds

    singles = [{g: [r]} for g, reqs in full.items() for r in reqs]
    batched_s = timed(args.sat_iters, lambda: launch(full, every))
    single_s = timed(args.sat_iters, lambda: [launch(b, every) for b in singles])
    dof = sum(inst[i]["dof"] for i in adm)
    for s in inst.values():
        assert torch.isfinite(s["bc"]).all()
    first = runs[0]
    line = {
        "metric": "serving step latency", "unit": "ms",
        "p50_ms": first["p50_ms"], "p99_ms": first["p99_ms"], "offered_steps_per_s": first["offered_steps_per_s"],
        "loads": runs,
        "instances": args.instances, "admitted": len(adm), "budget_gb": args.budget_gb,
        "servers": {f"n_in={g[0]},n_out={g[1]}": sum(1 for i in adm if group_of[i] == g) for g in servers},
        "fine_dof_per_round": dof,
        "saturated": {"batched": {"steps_per_s": len(adm) / batched_s, "fine_dof_per_s": dof / batched_s,
                                  "ms_per_round": batched_s * 1e3},
                      "one_instance_per_call": {"steps_per_s": len(adm) / single_s,
                                                "fine_dof_per_s": dof / single_s,
                                                "ms_per_round": single_s * 1e3}},
        "workload": "serving: %d instances, coarse 64x16..512x128, K in {1,2}, H=%d, BF16 net, Poisson arrivals"
                    % (args.instances, args.H),
        "data": "synthetic",
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()

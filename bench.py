"""Benchmark of the DNN-MG fine-level correction step on GB300.

One step = one full correction (Algorithm 2's correction step: prolongation, residual
and patch features, GRU patch network, averaging, right-hand side,
restriction) of the large single instance: 2048 x 512 coarse cells, K = 2
(8192 x 2048 fine cells, 16.8 M fine nodes), 2 x 2-cell patches (262 144
patches), GRU width 128, BF16 network GEMMs with FP32 accumulation, FP32 fine
fields, FP64 coarse vectors.  Inputs are synthetic (seeded Poiseuille flow
with vortices around an elliptic obstacle); weights N(0, 0.1) from a seed.

Metric: fine velocity DOF corrected per second (2 Nf per step / step time),
with p50/p99 step latency.  Every step moves ~2.5 GB, far more than the 129 MB
L2, so no L2 flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (one process per GPU under torchrun) every rank runs its own
instance (replicas; there is no data-path collective) and value is the sum.
--impl reference times the CPU FP64 oracle on a bounded window of the same
workload on the host cores.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2008_11520_gb300 import synth  # noqa: E402

METRIC = "fine DOF corrected/s per DNN-MG step"
UNIT = "DOF/s"
WORKLOAD = "large"


def describe(c):
    return (f"{c['nxc']}x{c['nyc']} coarse cells, K={c['K']} ({c['nxc'] << c['K']}x{c['nyc'] << c['K']} fine), "
            f"{c['s']}x{c['s']}-cell patches, GRU hidden {c['H']}, {c['precision']} network, "
            f"ellipse semi-axes {c['ellipse'][2]:.3f}x{c['ellipse'][3]:.4f}")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained", d["bf16_tflops"]), "src": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "src": "fallback"}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        self.out.flush()
        with open(self.out.name) as f:
            rows = [r.split(",") for r in f.read().strip().splitlines() if r.strip()]
        os.unlink(self.out.name)
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_traffic(stage):
    """DRAM bytes per launch of a stage's kernel from the committed ncu summary
    (profiles/traffic.json), or None when its sources changed since the capture."""
    import hashlib
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[stage]
        h = hashlib.sha256()
        for f in t["sources"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        return t["dram_bytes"] if h.hexdigest() == t["sha256"] else None
    except (OSError, KeyError, ValueError):
        return None


def max_over_ranks(values, world, device="cpu"):
    """Element-wise maximum of per-rank timings over the process group: the
    job takes as long as its slowest rank."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.tolist()


def job_rate(world, units_per_rank, steps, ms):
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time (replicas, weak scaling)."""
    return world * units_per_rank * steps / (ms / 1e3)


def algorithmic_work(info, H):
    """Bytes each stage must move (nodes, not the row padding) and the GEMM flops, per step."""
    Nf, Nc, P, ldx, n_in, n_out = info.Nf, info.Nc, info.P, info.ldx, info.n_in, info.n_out
    # algorithmic bytes count nodes, not the row padding of the pitched layout
    rb, fb = info.real_bytes, info.feature_bytes
    # S1 is fused: S2+S3 and S5 read the coarse vector instead of x~
    return {
        # S1 staging: x_c (FP64) once into the padded fine-type copy the residual tiles fetch
        "coarse_pad": {"bytes": 3 * Nc * 8 + 3 * Nc * rb},
        "residual_features": {"bytes": 3 * Nc * rb + 2 * Nf * rb + P * ldx * fb},
        "gru": {"bytes": P * ldx * fb + 2 * P * H * rb + P * n_out * rb,
                "flops": 2 * P * (3 * H * (n_in + H) + H * n_out)},
        # the coarse window comes from the padded fine-type copy (u and v)
        "scatter_avg": {"bytes": P * n_out * rb + 2 * Nc * rb + 2 * Nf * rb},
        "rhs": {"bytes": 2 * Nf * rb + 2 * Nf * rb},
        "restrict": {"bytes": 2 * Nf * rb + 3 * Nc * 8},
    }


def dominant(kernel_ms):
    """The kernel with the largest share of the step, as the name of its entry
    in ``algorithmic_work``.  The two S2+S3 kernels (closed-form tiles and
    boundary tiles, concurrent inside the step) count as one entry, the stage,
    with their times summed, should either of them be the largest."""
    top = max(kernel_ms, key=kernel_ms.get)
    if top in ("residual_cf", "residual_boundary"):
        return "residual_features", kernel_ms["residual_cf"] + kernel_ms["residual_boundary"]
    return top, kernel_ms[top]


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2008_11520_gb300 import dnnmg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    c = synth.config(WORKLOAD)
    mesh = dnnmg.Mesh(dnnmg.make_desc(c["nxc"], c["nyc"], c["K"], c["s"], c["ellipse"], precision=c["precision"]))
    I = mesh.info
    W = synth.net_weights(I.n_in, c["H"], I.n_out, seed=c["seed"])
    net = dnnmg.Net(*W, precision=c["precision"])
    spec = synth.FlowSpec.from_seed(c["seed"] + rank, c["ellipse"])
    xc_np = synth.coarse_state(spec, c["nxc"], c["nyc"], 0.0)
    v0 = synth.fine_state(spec, I.nxf, I.nyf, 0.0)[:2]
    xc = torch.as_tensor(xc_np).to(dev).contiguous()
    h = torch.zeros(I.P, c["H"], dtype=torch.float32, device=dev)
    bf = mesh.fine(2, dev)
    bc = mesh.coarse(3, dev)
    dnnmg.dnnmg_rhs_restrict(mesh, mesh.pack(v0, dev), bf, bc)
    del v0
    ws = mesh.workspace(dev)
    stream = torch.cuda.current_stream()
    k = 0.01

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for i in range(args.warmup):
        dnnmg.dnnmg_step(mesh, net, xc, h, bf, bc, ws, i * k)
    torch.cuda.synchronize()

    # ---- timed region: K steps of dnnmg_step, one event pair per step
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    torch.cuda.synchronize()
    with Clocks(local_rank) as clk:
        t0 = time.perf_counter()
        ev[0].record(stream)
        for i in range(args.steps):
            dnnmg.dnnmg_step(mesh, net, xc, h, bf, bc, ws, (args.warmup + i) * k)
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    barrier()
    per_step = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    clocks = clk.summary()

    # ---- stage timing: the step's own kernels, with events recorded between
    # them by dnnmg_step_timed on the launching stream
    wsv = torch.empty(0)
    # the S2+S3 stage is two kernels when the all-fluid tiles run in closed form
    res = ["residual_cf", "residual_boundary"] if dnnmg.dnnmg_step_launches(mesh, net) == 7 else ["residual_features"]
    names = ["coarse_pad"] + res + (["gru"] if I.P else []) + ["scatter_avg", "rhs", "restrict"]
    assert len(names) == dnnmg.dnnmg_step_launches(mesh, net)
    sev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)] for _ in range(args.steps)]
    torch.cuda.synchronize()
    for i in range(args.steps):
        dnnmg.dnnmg_step_timed(mesh, net, xc, h, bf, bc, ws, (args.warmup + args.steps + i) * k, sev[i])
    torch.cuda.synchronize()
    stage_ms = {n: statistics.mean(sev[i][j].elapsed_time(sev[i][j + 1]) for i in range(args.steps))
                for j, n in enumerate(names)}
    kernel_ms = dict(stage_ms)
    if "residual_cf" in stage_ms:   # the S2+S3 stage as a whole (both kernels)
        stage_ms = {("residual_features" if n == "residual_cf" else n): (ms + stage_ms["residual_boundary"]
                    if n == "residual_cf" else ms) for n, ms in stage_ms.items() if n != "residual_boundary"}
    del wsv

    # ---- end to end: host x_c in, host b_c out, through dnnmg_step_host
    xch = torch.as_tensor(xc_np).pin_memory()
    bch = torch.empty(3 * I.Nc, dtype=torch.float64).pin_memory()
    for i in range(2):
        dnnmg.dnnmg_step_host(mesh, net, xch, h, bf, bch, ws, i * k)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        dnnmg.dnnmg_step_host(mesh, net, xch, h, bf, bch, ws, i * k)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    assert np.isfinite(bch.numpy()).all()

    total_ms, e2e_ms = max_over_ranks([total_ms, e2e_ms], world, dev)
    return dict(cfg=c, info=I, per_step=per_step, total_ms=total_ms, stage_ms=stage_ms, kernel_ms=kernel_ms,
                clocks=clocks,
                e2e_ms=e2e_ms, wall=wall, launches=dnnmg.dnnmg_step_launches(mesh, net))


def blas_threads():
    """Threads of the BLAS library NumPy loaded, read from the library itself
    (threadpoolctl when installed, else the OpenBLAS query symbol), or None."""
    try:
        from threadpoolctl import threadpool_info
        n = [i["num_threads"] for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return max(n)
    except ImportError:
        pass
    import ctypes
    try:
        with open("/proc/self/maps") as f:
            libs = sorted({ln.split()[-1] for ln in f if "openblas" in ln.lower() and ".so" in ln})
    except OSError:
        libs = []
    for path in libs:
        try:
            so = ctypes.CDLL(path)
        except OSError:
            continue
        for sym in ("openblas_get_num_threads", "openblas_get_num_threads64_", "scipy_openblas_get_num_threads64_",
                    "scipy_openblas_get_num_threads"):
            fn = getattr(so, sym, None)
            if fn is not None:
                fn.restype = ctypes.c_int
                return int(fn())
    return None


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(seconds=12.0):
    """The oracle as it stands on a window of the large workload; fine DOF/s."""
    from oracle.mesh import Mesh as OMesh, Params
    from oracle import fem, step as ostep

    c = synth.config(WORKLOAD)
    win = (1000, 200, 1064, 264)         # 64 x 64 coarse cells behind the obstacle
    om = OMesh(c["nxc"], c["nyc"], c["K"], c["s"], ellipse=c["ellipse"], window=win)
    spec = synth.FlowSpec.from_seed(c["seed"], c["ellipse"])
    xc = synth.coarse_state(spec, c["nxc"], c["nyc"], 0.0, window=win)
    r = om.r
    fwin = (win[0] * r, win[1] * r, win[2] * r, win[3] * r)
    v0 = synth.fine_state(spec, om.nxf, om.nyf, 0.0, window=fwin)[:2]
    W = synth.net_weights(om.n_in, c["H"], om.n_out, seed=c["seed"])
    prm = Params()
    bf = fem.rhs(om, prm, v0)
    h = np.zeros((om.P, c["H"]))
    n, t0 = 0, time.perf_counter()
    while True:
        out = ostep.dnnmg_step(om, prm, W, xc, h, bf, n * prm.k)
        h, bf = out["h"], out["bf"]
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    threads = blas_threads()
    return {"value": 2 * om.Nf * n / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n} steps of a 64x64-coarse-cell window ({om.Nf} fine nodes, {2 * om.Nf} velocity DOF) of "
                      f"the workload in {el:.1f} s; the rate is that window's DOF over its step time",
            "steps": n, "seconds": el, "blas_threads": threads, "window_nodes": om.Nf}


def cpu_baseline_runs(seconds=12.0):
    """cpu_baseline at one thread and at every host core, each in a fresh
    interpreter whose BLAS/OpenMP thread counts are set before NumPy loads."""
    ncores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    runs = {}
    for threads in (1, ncores):
        env = dict(os.environ)
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            env[var] = str(threads)
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-worker", str(seconds)],
                           env=env, capture_output=True, text=True, timeout=30 * seconds + 300)
        if r.returncode:
            raise RuntimeError(f"cpu baseline worker failed:\n{r.stderr[-2000:]}")
        d = json.loads(r.stdout.strip().splitlines()[-1])
        d["threads_requested"] = threads
        runs[threads] = d
    one, allc = runs[1], runs[ncores]
    model = cpu_model()
    used = allc["blas_threads"] if allc["blas_threads"] is not None else ncores
    return {"value": allc["value"], "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": (f"{allc['sample']}; all {ncores} cores of a {model} host (BLAS threads in force: "
                       f"{allc['blas_threads']}); at 1 thread (BLAS threads {one['blas_threads']}): "
                       f"{one['value']:.4g} DOF/s over {one['steps']} steps"),
            "cpu_model": model, "host_cores": ncores,
            "one_thread": {"value": one["value"], "blas_threads": one["blas_threads"], "steps": one["steps"],
                           "seconds": one["seconds"]},
            "all_cores": {"value": allc["value"], "blas_threads": allc["blas_threads"], "steps": allc["steps"],
                          "seconds": allc["seconds"]}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-baseline-worker", type=float, default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_baseline_worker is not None:
        print(json.dumps(cpu_baseline(seconds=args.cpu_baseline_worker)))
        return
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    c = synth.config(WORKLOAD)
    if args.impl == "reference":
        if rank != 0:
            return
        steps = []
        for _ in range(args.warmup):
            cpu_baseline(seconds=1.0)
        for _ in range(args.steps):
            steps.append(cpu_baseline(seconds=2.0))
        v = sum(s["value"] * s["seconds"] for s in steps) / sum(s["seconds"] for s in steps)
        base = steps[0]
        ncores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * sum(s["seconds"] for s in steps) / sum(s["steps"] for s in steps),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": WORKLOAD + ": " + describe(c),
                                                "sample": "64x64-coarse-cell window per step, CPU oracle"},
                "cpu_baseline": {"value": v, "unit": UNIT,
                                 "cores": base["blas_threads"] if base["blas_threads"] is not None else ncores,
                                 "kind": "oracle", "cpu_model": cpu_model(), "host_cores": ncores,
                                 "sample": base["sample"] + f"; one such window per step, {ncores} host cores, "
                                                            f"BLAS threads in force {base['blas_threads']}"},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    r = run_ours(args, rank, world, local_rank)
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return
    I = r["info"]
    dof = 2 * I.Nf
    step_ms = r["total_ms"] / args.steps
    value = job_rate(world, dof, args.steps, r["total_ms"])
    pk = peaks()
    work = algorithmic_work(I, c["H"])
    # dominant kernel: the kernel with the largest share of the step
    dom, dom_ms = dominant(r["kernel_ms"])
    # the roofline of a stage is whichever of HBM traffic and tensor work takes
    # longer at the measured peaks (the GRU GEMMs move more bytes than flops allow)
    w = work[dom]
    t_hbm = w["bytes"] / (pk["hbm_gbs"] * 1e9)
    t_tc = w.get("flops", 0) / (pk["bf16_tflops"] * 1e12)
    if t_tc > t_hbm:
        ach = w["flops"] / (dom_ms / 1e3) / 1e12
        roof = {"kernel": dom, "kernel_ms": dom_ms, "bound": "tensor", "achieved": ach, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                "frac": ach / pk["bf16_tflops"], "traffic": measured_traffic(dom),
                "peak_src": pk["src"] + " bf16 burst"}
    else:
        ach = w["bytes"] / (dom_ms / 1e3) / 1e9
        roof = {"kernel": dom, "kernel_ms": dom_ms, "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"], "traffic": measured_traffic(dom),
                "algorithmic_bytes": w["bytes"], "peak_src": pk["src"] + " copy bandwidth"}
    stages = {}
    for n, ms in r["stage_ms"].items():
        e = {"ms": ms, "GB/s": work[n]["bytes"] / (ms / 1e3) / 1e9}
        e["hbm_frac"] = e["GB/s"] / pk["hbm_gbs"]
        if "flops" in work[n]:
            e["TFLOP/s"] = work[n]["flops"] / (ms / 1e3) / 1e12
        stages[n] = e
    per = sorted(r["per_step"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": WORKLOAD + ": " + describe(c), "fine_dof_per_step": dof, "patches": I.P,
                   "l2": "no flush: each step moves ~2.5 GB, inputs larger than the 129 MB L2",
                   "parallelism": "replicas" if world > 1 else "single"},
        "p50_ms": per[len(per) // 2], "p99_ms": per[min(len(per) - 1, int(0.99 * len(per)))],
        "e2e": {"value": job_rate(world, dof, args.steps, r["e2e_ms"]), "unit": UNIT,
                "h2d_bytes_per_step": 3 * I.Nc * 8, "d2h_bytes_per_step": 3 * I.Nc * 8},
        "gpu_launches": r["launches"] * args.steps,
        "roofline": roof, "stages": stages, "kernel_ms": r["kernel_ms"], "clocks": r["clocks"],
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_runs()
    print(json.dumps(line))


if __name__ == "__main__":
    main()

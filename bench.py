"""Benchmark of the projective affine body step on GB300.

Workload (default): the 4096-box pile -- boxes with edges U[0.5, 2], density U[500, 2000],
dropped from a jittered 16^3 grid (spacing 3.5) onto the ground, contacts rebuilt every
step by the grid-hash broad phase, mu = 0.5, h = 1/60, 30 sweeps per step.  A timed "step"
is one whole time step of Algorithm 1 (collision detection, predictor, 30 bond + solve
sweeps, velocity recovery).  The K timed steps are steps 0..K-1 of the pile's trajectory
(warm-up steps are run first and then the initial state is restored).

Metric: body-iterations per second (bodies x sweeps per step x steps / time), with steps/s,
the plain (eager, kernel-by-kernel) path's throughput and the end-to-end number through the
C-ABI with host buffers.  L2 is flushed between timed steps (a 256 MB write).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (test infrastructure) on the same workload:
each step is one oracle step of the pile; only rank 0 runs it.
Under torchrun (N > 1) every rank steps its own replica of the scene: the path does not
shard, so there is no collective in the data path; the barrier and the max over ranks of
the timed region come from torch.distributed.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenes as S  # noqa: E402

METRIC = "body-iterations/s"
UNIT = "body-iter/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if len(r) > 5 + k and r[5 + k] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


ARGS = None


def workload():
    n = ARGS.bodies if ARGS is not None else 4096
    if n == 4096 and not (ARGS is not None and ARGS.stacked):
        return S.box_pile()
    return S.box_pile_n(n, stacked=bool(ARGS is not None and ARGS.stacked))


def config_of(sc, K):
    start = ARGS.start_step if ARGS is not None else 0
    kind = "stacked columns" if (ARGS is not None and ARGS.stacked) else "jittered grid, spacing 3.5"
    return {"workload": f"box pile {sc.n_bodies} ({kind}), {sc.params['n_iter']} sweeps, "
                        f"h=1/60, steps {start}..{start + K - 1} of the trajectory",
            "n_bodies": sc.n_bodies, "n_iter": sc.params["n_iter"], "l2": "flushed between timed steps (256 MB write)",
            "parallelism": "replicas"}


def _kernel_hash():
    h = hashlib.sha256()
    for f in ("k_sweep.cu", "k_persist.cu", "sweep_math.cuh", "pabd_internal.h"):
        with open(os.path.join(ROOT, "paper_2609_02675_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic(kernel: str):
    """dram bytes per launch of `kernel` from the committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            t = json.load(f)
        e = t[kernel]
        if e.get("source_hash") != _kernel_hash():
            return None
        return e
    except Exception:
        return None


def cpu_baseline(budget_s: float = 15.0, max_steps: int = 300):
    """The FP64 oracle (as it stands) on the same pile, steps 0..M-1 within the time budget."""
    import oracle as O
    sc = workload()
    o = O.OracleScene(sc)
    t0 = time.perf_counter()
    m = 0
    while m < max_steps and time.perf_counter() - t0 < budget_s:
        o.step(1)
        m += 1
    dt = time.perf_counter() - t0
    return {"value": sc.n_bodies * sc.params["n_iter"] * m / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle steps 0..{m - 1} of the {sc.n_bodies}-box pile ({m} steps, {dt:.1f} s, single thread)"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle as O
    sc = workload()
    o = O.OracleScene(sc)
    for _ in range(args.warmup):
        o.step(1)
    o = O.OracleScene(sc)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    v = sc.n_bodies * sc.params["n_iter"] * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(sc, args.steps),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"oracle steps 0..{args.steps - 1} of the pile, single thread"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2609_02675_gb300 as P

    dev = local_rank
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    sc = workload()
    K, W = args.steps, args.warmup
    g = P.Scene(sc, device=dev, stream=stream, sweep_mode=args.sweep_mode, sweep_lanes=args.lanes)
    st0 = g.state()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{dev}")

    def reset():
        g.set_state(st0)
        g.set_step_index(args.start_step)

    def l2_flush():
        with torch.cuda.stream(stream):
            flush.fill_(1.0)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # optional untimed lead-in (part of preparing the input state), then warm-up and restore
    if args.start_step:
        g.step(args.start_step)
        g.sync()
        st0 = g.state()
    g.set_step_index(args.start_step)
    g.step(W)
    g.sync()
    reset()
    n_body_iter = sc.n_bodies * sc.params["n_iter"]

    # timed region: graph path, one CUDA-event pair per step on the scene's stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    info0 = g.info()
    barrier()
    with ClockSampler(dev) as clk:
        for k in range(K):
            l2_flush()
            ev[k][0].record(stream)
            g.step(1)
            ev[k][1].record(stream)
        barrier()
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    g.sync()
    info1 = g.info()
    launches = info1["launches"] - info0["launches"]

    # live stage timing of the same K steps (graph with event nodes between the stages)
    reset()
    g.set_profiling(True)
    g.profile(reset=True)
    for k in range(K):
        l2_flush()
        g.step(1)
    prof = g.profile(reset=True)
    g.set_profiling(False)

    # plain path: the same steps launched kernel by kernel
    reset()
    evp = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    barrier()
    for k in range(K):
        l2_flush()
        evp[k][0].record(stream)
        g.step_eager(1)
        evp[k][1].record(stream)
    barrier()
    t_plain = sum(a.elapsed_time(b) for a, b in evp)

    # end to end through the C-ABI with host buffers: write state (H2D), step, read state (D2H)
    reset()
    rows = g.state()
    h2d = sc.n_bodies * 96
    d2h = sc.n_bodies * 96
    barrier()
    t0 = time.perf_counter()
    for k in range(K):
        g.set_state(rows)
        g.step(1)
        g.state(out=rows)
    barrier()
    t_e2e = time.perf_counter() - t0

    # max over ranks
    vals = torch.tensor([t_ms, t_plain, t_e2e * 1e3], dtype=torch.float64, device=f"cuda:{dev}")
    if world > 1:
        torch.distributed.all_reduce(vals, op=torch.distributed.ReduceOp.MAX)
    t_ms, t_plain, t_e2e_ms = vals.tolist()
    g.close()
    if rank != 0:
        return
    total_body_iter = n_body_iter * K * world
    value = total_body_iter / (t_ms * 1e-3)

    # roofline of the dominant sweep kernel
    steps = max(prof["steps"], 1)
    n_it = sc.params["n_iter"]
    bonds_avg = prof["bonds_sum"] / steps
    N = sc.n_bodies
    fused = info1["sweep_mode"] == 0
    if fused:
        # one launch runs n_it sweeps; per sweep each body moves q in/out, s, mass, flags, CSR
        # offset and residual (176 B) and each bond's two end records (2 x 48 B) plus, for a
        # contact, its normal twice (2 x 16 B)
        per_sweep = 176.0 * N + 128.0 * bonds_avg
        per_kernel = {"k_sweep_fused": (n_it * per_sweep, prof["bond_ms"] / steps)}
    else:
        per_kernel = {
            # bond = static bond records (64 B) + CSR slot pair (8 B) + two end records written
            # (32 B) per bond + q read (48 B) per body; solve = q in/out, predictor, mass, flags,
            # CSR offset, residual (176 B) per body + two end records and material points (64 B)
            "k_bond": (104.0 * bonds_avg + 48.0 * N, prof["bond_ms"] / max(prof["bond_launches"], 1)),
            "k_solve": (176.0 * N + 64.0 * bonds_avg, prof["solve_ms"] / max(prof["solve_launches"], 1)),
        }
    dom = max(per_kernel, key=lambda k: per_kernel[k][1])
    bytes_launch, ms_launch = per_kernel[dom]
    achieved = bytes_launch / (ms_launch * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    tr = _ncu_traffic(dom)
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs",
            "traffic": tr["bytes_per_launch"] if tr else None,
            "bytes_per_launch": bytes_launch, "us_per_launch": ms_launch * 1e3, "bonds_per_step": bonds_avg,
            "stage_ms_per_step": {k: prof[k] / steps for k in ("collision_ms", "csr_ms", "predict_ms", "bond_ms",
                                                                 "solve_ms", "finalize_ms", "step_ms")}}
    cfg = config_of(sc, K)
    cfg["sweep"] = {k: info1[k] for k in ("sweep_mode", "sweep_lanes", "sweep_block", "sweep_grid")}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": t_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic", "config": cfg,
        "steps_per_s": world * K / (t_ms * 1e-3),
        "plain_path": {"value": total_body_iter / (t_plain * 1e-3), "unit": UNIT, "ms_per_step": t_plain / K},
        "e2e": {"value": total_body_iter / (t_e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "roofline": roof,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--bodies", type=int, default=4096, help="pile size (4096 = the 16^3 pile)")
    ap.add_argument("--stacked", action="store_true", help="pile as touching columns (contacts from step 0)")
    ap.add_argument("--start-step", type=int, default=0, help="untimed lead-in steps before the timed window")
    ap.add_argument("--sweep-mode", type=int, default=0, help="0: fused persistent sweep, 1: two launches per sweep")
    ap.add_argument("--lanes", type=int, default=0, help="lanes per body in the fused sweep (0: library default)")
    args = ap.parse_args()
    global ARGS
    ARGS = args
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    import __graft_entry__
    __graft_entry__.build()
    main()

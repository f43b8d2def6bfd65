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
    sc = _workload()
    if ARGS is not None and ARGS.resid_tol > 0:
        sc.params = dict(sc.params, resid_tol=ARGS.resid_tol)
    return sc


def _workload():
    if ARGS is not None and ARGS.workload == "trees":
        return S.batched_trees()
    if ARGS is not None and ARGS.workload == "quadruped":
        return S.quadruped_bed_rod()
    if ARGS is not None and ARGS.workload == "stack":
        return S.mass_ratio_stack()
    if ARGS is not None and ARGS.workload == "spring":
        return S.two_box_spring()
    if ARGS is not None and ARGS.workload == "net":
        return S.spring_net()
    n = ARGS.bodies if ARGS is not None else 4096
    if n == 4096 and not (ARGS is not None and ARGS.stacked):
        return S.box_pile()
    return S.box_pile_n(n, stacked=bool(ARGS is not None and ARGS.stacked))


def config_of(sc, K):
    start = ARGS.start_step if ARGS is not None else 0
    if ARGS is not None and ARGS.workload in ("stack", "spring", "net"):
        desc = {"stack": "six-cube stack, each cube 10x heavier than the one below",
                "spring": "two unit cubes joined by a spring stretched to twice its rest length",
                "net": "11 x 11 net of cubes joined by 220 pre-stretched springs, top corners pinned"}[ARGS.workload]
        return {"workload": desc + f" ({sc.n_bodies} bodies), {sc.params['n_iter']} sweeps, steps {start}..{start + K - 1}",
                "n_bodies": sc.n_bodies, "n_iter": sc.params["n_iter"], "l2": "flushed between timed steps (256 MB write)",
                "parallelism": "replicas", **_tol_cfg()}
    if ARGS is not None and ARGS.workload in ("trees", "quadruped"):
        if ARGS.workload == "trees":
            desc = (f"{sc.n_groups} independent trees of 4-64 boxes ({sc.n_bodies} bodies), ground contact, "
                    f"{sc.params['n_iter']} sweeps, h=1/120, one batched scene")
        else:
            desc = (f"driven 13-body quadruped on a bed of {sc.meta['n_bed']} cubes + {sc.meta['n_rod']}-segment "
                    f"elastic rod ({sc.n_bodies} bodies), {sc.params['n_iter']} sweeps, h=1/60")
        return {"workload": desc + f", steps {start}..{start + K - 1}", "n_bodies": sc.n_bodies,
                "n_iter": sc.params["n_iter"], "l2": "flushed between timed steps (256 MB write)",
                "parallelism": "replicas", **_tol_cfg()}
    kind = "stacked columns" if (ARGS is not None and ARGS.stacked) else "jittered grid, spacing 3.5"
    return {"workload": f"box pile {sc.n_bodies} ({kind}), {sc.params['n_iter']} sweeps, "
                        f"h=1/60, steps {start}..{start + K - 1} of the trajectory",
            "n_bodies": sc.n_bodies, "n_iter": sc.params["n_iter"], "l2": "flushed between timed steps (256 MB write)",
            "parallelism": "replicas", **_tol_cfg()}


def _tol_cfg():
    if ARGS is None or ARGS.resid_tol <= 0:
        return {}
    return {"resid_tol": ARGS.resid_tol,
            "note": "each scene stops at its first sweep with residual <= resid_tol (at most n_iter); "
                    "body-iterations count the sweeps actually run (mean_sweeps_per_step)"}


def _kernel_hash():
    """Hash of the sources of the sweep kernels (their arithmetic and memory accesses)."""
    h = hashlib.sha256()
    for f in ("k_sweep.cu", "k_persist.cu", "sweep_math.cuh", "dfloat.cuh"):
        with open(os.path.join(ROOT, "paper_2609_02675_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic(kernel: str, workload: str):
    """dram bytes per launch of `kernel` on `workload` from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            t = json.load(f)
        if t.get("source_hash") != _kernel_hash():
            return None
        return t["entries"].get(f"{kernel}|{workload}")
    except Exception:
        return None


def max_over_ranks(values, world: int, device=None):
    """Element-wise max of per-rank timings (the slowest rank defines the job's time)."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.tolist()


def job_throughput(units_per_rank: float, world: int, t_max_ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_rank * world / (t_max_ms * 1e-3)


def host_cpu() -> str:
    """CPU model and logical core count of this host."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model", "hardware")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return f"{model} ({os.cpu_count()} logical cores)"


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
            "sample": f"oracle steps 0..{m - 1} of the {sc.n_bodies}-box pile ({m} steps, {dt:.1f} s, single thread)",
            "host": host_cpu()}


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
                             "sample": f"oracle steps 0..{args.steps - 1} of the pile, single thread",
                             "host": host_cpu()},
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
    # a settled granular bed reaches about 13 candidate pairs and 30 contact points per grain
    cap = dict(max_pairs=32 * sc.n_bodies, max_contacts=64 * sc.n_bodies) if args.workload == "quadruped" else {}
    g = P.Scene(sc, device=dev, stream=stream, sweep_mode=args.sweep_mode, sweep_lanes=args.lanes, **cap)
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
    mean_sweeps = None
    if sc.params.get("resid_tol", 0.0) > 0:
        # sweeps actually run per step under the threshold, from the same steps (untimed pass)
        counts = []
        for k in range(K):
            g.step(1)
            counts.append(g.info()["last_sweeps"])
        mean_sweeps = float(np.mean(counts))
        n_body_iter = sc.n_bodies * mean_sweeps
        reset()

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

    # batched scenes: the same scenes each run alone on the plain path (a sample, eager launches)
    alone = None
    if args.workload == "trees":
        sizes = sc.meta["sizes"]
        off = np.concatenate([[0], np.cumsum(sizes)])
        pick = np.linspace(0, len(sizes) - 1, 32).astype(int)
        t_alone, body_iter = 0.0, 0
        for gi in pick:
            sl = slice(off[gi], off[gi + 1])
            sub = S.Scene("one", dict(sc.params), sc.bodies[sl].copy(), sc.bonds.copy(), 1)
            sub.bodies["group"] = 0
            m = (sc.bonds["i"] >= off[gi]) & (sc.bonds["i"] < off[gi + 1])
            sub.bonds = sc.bonds[m].copy()
            sub.bonds["i"] -= off[gi]
            sub.bonds["j"] = np.where(sub.bonds["j"] >= 0, sub.bonds["j"] - off[gi], -1)
            one = P.Scene(sub, device=dev, stream=stream)
            one.step_eager(2)
            one.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one.step_eager(min(K, 20))
            e1.record(stream)
            e1.synchronize()
            t_alone += e0.elapsed_time(e1)
            body_iter += int(sizes[gi]) * sc.params["n_iter"] * min(K, 20)
            one.close()
        alone = {"value": body_iter / (t_alone * 1e-3), "unit": UNIT,
                 "sample": "32 of the scenes, each alone on the plain path (eager launches), 20 steps each"}

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
    t_ms, t_plain, t_e2e_ms = max_over_ranks([t_ms, t_plain, t_e2e * 1e3], world, f"cuda:{dev}")
    g.close()
    if rank != 0:
        return
    total_body_iter = n_body_iter * K * world
    value = job_throughput(n_body_iter * K, world, t_ms)

    # roofline of the sweep: per launch of the sweep kernel, algorithmic bytes / average
    # duration (the sweep stage's events bracket all its launches of a step)
    steps = max(prof["steps"], 1)
    n_it = sc.params["n_iter"]
    bonds_avg = prof["bonds_sum"] / steps
    N = sc.n_bodies
    mode = info1["sweep_mode"]
    # per sweep: each body moves q in / out, s, mass, flags, CSR offsets and its residual
    # (176 B); each bond its two CSR-ordered end records (2 x 48 B) and, for a contact, its
    # normal twice (2 x 16 B); the two-launch mode also writes and re-reads the end records
    per_sweep = 176.0 * N + 128.0 * bonds_avg
    if mode == 3:
        kernel, per_launch_bytes = "k_sweep_fused", n_it * per_sweep
    elif mode == 2:
        kernel, per_launch_bytes = "k_sweep_one", per_sweep
    else:
        kernel, per_launch_bytes = "k_bond+k_solve", per_sweep + 64.0 * bonds_avg
    launches_per_step = prof["sweep_launches"] / steps
    ms_launch = prof["sweep_ms"] / max(prof["sweep_launches"], 1)
    if mode == 1:
        ms_launch *= 2.0  # one bond + one solve launch per sweep
    achieved = per_launch_bytes / (ms_launch * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    wl_key = f"{args.workload}|{'stacked' if args.stacked else 'grid'}|{sc.n_bodies}"
    tr = _ncu_traffic(kernel, wl_key)
    roof = {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs",
            "traffic": tr["bytes_per_launch"] if tr else None,
            "bytes_per_launch": per_launch_bytes, "us_per_launch": ms_launch * 1e3, "bonds_per_step": bonds_avg,
            "launches_per_step": launches_per_step,
            "stage_ms_per_step": {k: prof[k] / steps for k in ("collision_ms", "csr_ms", "predict_ms", "sweep_ms",
                                                                 "finalize_ms", "step_ms")}}
    cfg = config_of(sc, K)
    cfg["sweep"] = {k: info1[k] for k in ("sweep_mode", "sweep_lanes", "sweep_block", "sweep_grid")}
    if mean_sweeps is not None:
        cfg["mean_sweeps_per_step"] = mean_sweeps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": t_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic", "config": cfg,
        "steps_per_s": world * K / (t_ms * 1e-3),
        "plain_path": {"value": job_throughput(n_body_iter * K, world, t_plain), "unit": UNIT, "ms_per_step": t_plain / K},
        "e2e": {"value": job_throughput(n_body_iter * K, world, t_e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        **({"scenes_alone_plain_path": alone} if alone else {}),
        "clocks": clk.summary(),
        "roofline": roof,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)


def run_served(args, dev):
    """Poisson stream of step requests over resident pile scenes of 10 to 1e5 bodies (one
    line per rate), against each scene's step alone on the plain path."""
    import torch
    import paper_2609_02675_gb300 as P
    from paper_2609_02675_gb300.serve import Server, replay
    torch.cuda.set_device(dev)

    def make(n):
        return S.box_pile_n(int(n), seed=S.SEED_BASE + 5, stacked=True, n_iter=30)

    out = []
    for rate in [float(x) for x in args.rates.split(",")]:
        reqs, sizes = S.request_stream(rate=rate, duration=args.duration, max_scenes=64)
        srv = Server(lambda sid: make(sizes[sid]), hbm_budget=32 << 30, device=dev)
        t0, t1 = replay(srv, reqs, duration=args.duration, drain_timeout=20.0)
        st = srv.stats(t0, t1)
        # plain path: each distinct scene size stepped alone (sampled), mean step time
        pick = sorted(set(sizes))[:: max(1, len(set(sizes)) // 8)]
        alone_ms = []
        for n in pick:
            g = P.Scene(make(n), device=dev)
            g.step_eager(1)
            g.sync()
            t = time.perf_counter()
            g.step_eager(3)
            g.sync()
            alone_ms.append((time.perf_counter() - t) / 3 * 1e3)
            g.close()
        srv.close()
        st.update({"rate": rate, "scenes": len(sizes), "plain_path_step_ms_mean": float(np.mean(alone_ms)),
                   "plain_path_sizes": [int(n) for n in pick]})
        out.append(st)
        torch.cuda.empty_cache()
    line = {"metric": "served step latency", "unit": "ms", "higher_is_better": False, "n_gpus": 1,
            "data": "synthetic", "dtype": "f32",
            "config": {"workload": f"Poisson step requests (1-60 steps) over at most 64 pile scenes of 10-1e5 "
                                   f"bodies, {args.duration:.0f} s of arrivals per rate (then up to 20 s to drain), "
                                   f"HBM budget 32 GB",
                       "parallelism": "one scene per stream, continuous batching"},
            "rates": out}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="pile",
                    choices=["pile", "trees", "quadruped", "served", "stack", "spring", "net"])
    ap.add_argument("--resid-tol", type=float, default=0.0,
                    help="residual threshold of the sweeps (0: a fixed n_iter sweeps per step)")
    ap.add_argument("--rates", default="100,300,1000,3000,10000", help="served: request rates (req/s)")
    ap.add_argument("--duration", type=float, default=3.0, help="served: seconds of arrivals per rate")
    ap.add_argument("--bodies", type=int, default=4096, help="pile size (4096 = the 16^3 pile)")
    ap.add_argument("--stacked", action="store_true", help="pile as touching columns (contacts from step 0)")
    ap.add_argument("--start-step", type=int, default=0, help="untimed lead-in steps before the timed window")
    ap.add_argument("--sweep-mode", type=int, default=0,
                    help="1: two launches per sweep, 2: one launch per sweep, 3: fused persistent, 0: library choice")
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
    if args.workload == "served":
        if rank == 0:
            run_served(args, local_rank)
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

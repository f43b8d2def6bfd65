"""Benchmark of the projective affine body step on GB300.

Headline workload (default): 4096 independent articulated trees of U{4..64} boxes (139 690
bodies; spherical, revolute and nonlinear elastic joints; ground contact), batched into one
scene, h = 1/120, 10 sweeps per step.  A timed "step" is one whole time step of Algorithm 1
(collision detection, predictor, the sweeps of the global and local solves, velocity
recovery).  The timed window is steps S..S+K-1 with S = 60 by default (0.5 s: the trees have
landed and stand on the ground, so every sweep carries bonds and ground contacts); the lead-in
steps 0..S-1 run untimed, and warm-up steps are run from step S and then undone by restoring
the step-S state.

Metric: body-iterations per second (bodies x sweeps per step x steps / time) with steps/s, the
plain (eager, kernel-by-kernel) path, the end-to-end number through the C-ABI with host
buffers, the roofline of the sweep kernel measured inside the same window, and -- with the
headline only -- the 4096-box pile on a landed window, the quadruped on its granular bed, the
trees run one scene at a time on the plain path, and a short served run (p50/p99 step latency).
L2 is flushed between timed steps (a 256 MB write).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload trees|pile|quadruped|served|stack|spring|net] [--start-step S]

--impl reference times the FP64 CPU oracle (test infrastructure) on a bounded sample of the
same workload and window (a subset of the trees: the trees are independent scenes, so a
subset steps exactly as it does inside the batch); only rank 0 runs it and it never loads the
CUDA library.  Under torchrun (N > 1) every rank steps its own replica: the path does not
shard, so there is no collective in the data path; the barrier and the max over ranks of the
timed region come from torch.distributed.
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
L2_NOTE = "flushed between timed steps (256 MB write)"
# relative per-step position tolerance of the single-precision path against the FP64 oracle
REL_TOL = 1e-5


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


# ---------------------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------------------

# untimed lead-in steps before the timed window: the trees have landed by 0.5 s; the lower
# layers of the 4096 pile by step 150; the quadruped's legs reach the bed by step 30
DEFAULT_START = {"trees": 60, "pile": 150, "quadruped": 30}


def make_workload(name: str, bodies: int = 4096, stacked: bool = False, resid_tol: float = 0.0):
    if name == "trees":
        sc = S.batched_trees()
    elif name == "quadruped":
        sc = S.quadruped_bed_rod()
    elif name == "stack":
        sc = S.mass_ratio_stack()
    elif name == "spring":
        sc = S.two_box_spring()
    elif name == "net":
        sc = S.spring_net()
    elif bodies == 4096 and not stacked:
        sc = S.box_pile()
    else:
        sc = S.box_pile_n(bodies, stacked=stacked)
    if resid_tol > 0:
        sc.params = dict(sc.params, resid_tol=resid_tol)
    return sc


def start_step(name: str, stacked: bool, bodies: int, given: int) -> int:
    if given >= 0:
        return given
    if name == "pile" and (stacked or bodies != 4096):
        return 0  # stacked columns touch from step 0
    return DEFAULT_START.get(name, 0)


def describe(name: str, sc, start: int, K: int, stacked: bool = False) -> str:
    win = f"steps {start}..{start + K - 1}"
    it = sc.params["n_iter"]
    if name == "trees":
        return (f"{sc.n_groups} independent trees of 4-64 boxes ({sc.n_bodies} bodies), spherical/revolute/"
                f"nonlinear-elastic joints, ground contact, {it} sweeps, h=1/120, one batched scene, {win} "
                f"(landed)")
    if name == "quadruped":
        return (f"driven 13-body quadruped on a bed of {sc.meta['n_bed']} cubes + {sc.meta['n_rod']}-segment "
                f"elastic rod ({sc.n_bodies} bodies), {it} sweeps, h=1/60, {win}")
    if name in ("stack", "spring", "net"):
        d = {"stack": "six-cube stack, each cube 10x heavier than the one below",
             "spring": "two unit cubes joined by a spring stretched to twice its rest length",
             "net": "11 x 11 net of cubes joined by 220 pre-stretched springs, top corners pinned"}[name]
        return f"{d} ({sc.n_bodies} bodies), {it} sweeps, {win}"
    kind = "stacked columns" if stacked else "jittered grid, spacing 3.5"
    return f"box pile {sc.n_bodies} ({kind}), {it} sweeps, h=1/60, {win} of the trajectory"


def tol_cfg(resid_tol: float) -> dict:
    if resid_tol <= 0:
        return {}
    return {"resid_tol": resid_tol,
            "note": "each scene stops at its first sweep with residual <= resid_tol (at most n_iter); "
                    "body-iterations count the sweeps actually run (mean_sweeps_per_step)"}


def _kernel_hash():
    """Hash of the sources of the sweep kernels (their arithmetic and memory accesses)."""
    h = hashlib.sha256()
    for f in ("k_sweep.cu", "k_sweep_one.cu", "k_persist.cu", "sweep_math.cuh", "dfloat.cuh"):
        p = os.path.join(ROOT, "paper_2609_02675_gb300", "csrc", f)
        if os.path.exists(p):
            with open(p, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def window_key(name: str, n_bodies: int, start: int, stacked: bool = False) -> str:
    """Key of a measured window in profiles/traffic.json: workload, size and first step."""
    return f"{name}|{'stacked' if stacked else 'default'}|{n_bodies}|start{start}"


def _ncu_traffic(kernel: str, key: str):
    """DRAM bytes per launch of `kernel` on the window `key` from the committed ncu summary,
    if it was taken on the current sweep source (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            t = json.load(f)
        if t.get("source_hash") != _kernel_hash():
            return None
        return t["entries"].get(f"{kernel}|{key}")
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


# ---------------------------------------------------------------------------------------
# error measure of a step against the oracle (same definition as the parity tests)
# ---------------------------------------------------------------------------------------

_SIGNS = np.array([[sx, sy, sz] for sz in (-1, 1) for sy in (-1, 1) for sx in (-1, 1)], dtype=np.float64)


def _corners(st: np.ndarray, he: np.ndarray) -> np.ndarray:
    x = _SIGNS[None, :, :] * he[:, None, :]
    A = st[:, 3:12].reshape(-1, 3, 3)
    return st[:, None, 0:3] + np.einsum("nij,nkj->nki", A, x)


def rel_err(st_gpu: np.ndarray, st_ref: np.ndarray, he: np.ndarray) -> float:
    """max over bodies and box corners |y_gpu - y_ref| / the bounding-box diagonal (>= 1)."""
    y = _corners(st_ref, he).reshape(-1, 3)
    scale = max(float(np.linalg.norm(y.max(0) - y.min(0))), 1.0)
    d = np.linalg.norm(_corners(st_gpu, he) - _corners(st_ref, he), axis=-1)
    return float(d.max()) / scale


# ---------------------------------------------------------------------------------------
# oracle legs: the CPU baseline (and the sampled parity check it enables), the reference arm
# ---------------------------------------------------------------------------------------

def oracle_sample(name: str, sc):
    """A bounded sample of the workload for the FP64 oracle: for the trees the groups
    0, 16, 32, ... (256 of the 4096 independent trees), else the whole scene."""
    if name == "trees" and sc.n_groups > 256:
        groups = np.arange(0, sc.n_groups, sc.n_groups // 256)[:256]
        sub = S.select_groups(sc, groups)
        return sub, groups, f"{len(groups)} of the {sc.n_groups} trees (every {sc.n_groups // 256}th, " \
                            f"{sub.n_bodies} bodies)"
    return sc, None, f"the whole scene ({sc.n_bodies} bodies)"


def cpu_baseline(name: str, sc, start: int, K: int, budget_s: float = 15.0, gpu_check=None):
    """The FP64 oracle (as it stands, one thread) on a sample of the same workload: an
    untimed lead-in to step `start`, then steps start..start+M-1 timed (M <= K, within the
    budget).  With gpu_check(sample_state, groups, k) -> gpu next-step rows of the sample,
    also the per-step error of the GPU step started from the oracle's state at step k
    (teacher-forced) on that sample."""
    import oracle as O
    sub, groups, what = oracle_sample(name, sc)
    o = O.OracleScene(sub)
    t_lead = time.perf_counter()
    if start:
        o.step(start)
    t_lead = time.perf_counter() - t_lead
    st_start, k_start = o.state(), o.step_index
    t0 = time.perf_counter()
    m = 0
    while m < K and time.perf_counter() - t0 < budget_s:
        o.step(1)
        m += 1
    dt = time.perf_counter() - t0
    out = {"value": sub.n_bodies * sub.params["n_iter"] * m / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"oracle on {what}, steps {start}..{start + m - 1} timed ({m} steps, {dt:.1f} s) after an "
                     f"untimed lead-in of {start} steps ({t_lead:.1f} s), single thread",
           "host": host_cpu()}
    parity = None
    if gpu_check is not None:
        # teacher-forced: the GPU runs the full workload (same launch configuration as the
        # timed window) from the oracle's step-`start` state on the sampled rows
        ref = O.OracleScene(sub)
        ref.set_state(st_start)
        ref.step_index = k_start
        ref.step(1)
        g_rows = gpu_check(st_start, groups, k_start)
        he = np.ascontiguousarray(sub.bodies["he"], dtype=np.float64)
        e = rel_err(g_rows, ref.state(), he)
        parity = {"max_rel_err": e, "tol": REL_TOL, "pass": bool(e < REL_TOL),
                  "kind": "one teacher-forced step: the GPU (full workload, timed launch configuration) starts "
                          "from the oracle's state; max over bodies and box corners of |y_gpu - y_ref| / scene "
                          "diagonal",
                  "sample": f"{what}, step {k_start}"}
    return out, parity


def run_reference(args, rank, world):
    """The oracle as the reference arm, on the same window of a bounded sample of the same
    workload (it never imports the CUDA library)."""
    if rank != 0:
        return
    import oracle as O
    name = args.workload
    sc = make_workload(name, args.bodies, args.stacked, args.resid_tol)
    start = start_step(name, args.stacked, args.bodies, args.start_step)
    sub, _, what = oracle_sample(name, sc)
    o = O.OracleScene(sub)
    if start:
        o.step(start)
    st0, k0 = o.state(), o.step_index
    o.step(args.warmup)
    o.set_state(st0)
    o.step_index = k0
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    v = sub.n_bodies * sub.params["n_iter"] * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": describe(name, sc, start, args.steps, args.stacked), "n_bodies": sc.n_bodies,
                       "n_iter": sc.params["n_iter"], "l2": L2_NOTE, "parallelism": "replicas",
                       **tol_cfg(args.resid_tol)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"oracle on {what}, steps {start}..{start + args.steps - 1} after an untimed "
                                       f"lead-in, single thread", "host": host_cpu()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------------------

def measure(P, torch, sc, name, start, K, W, dev, stream, world=1, flush=None, sweep_mode=0, lanes=0,
            stacked=False, plain=True, e2e=True, keep=False, light_order=0):
    """Time K graph steps of `sc` from step `start` (after an untimed lead-in and W warm-up
    steps that are undone), then the same steps with the stage events, on the plain path and
    end to end.  Returns a dict of the measurements (and the scene if keep)."""
    cap = dict(max_pairs=32 * sc.n_bodies, max_contacts=64 * sc.n_bodies) if name == "quadruped" else {}
    g = P.Scene(sc, device=dev, stream=stream, sweep_mode=sweep_mode, sweep_lanes=lanes, light_order=light_order,
                **cap)
    if flush is None:
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{dev}")

    def l2_flush():
        with torch.cuda.stream(stream):
            flush.fill_(1.0)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    if start:
        g.step(start)
        g.sync()
    if sweep_mode == 0 or light_order == 0:
        g.tune()  # the sweep autotuner on the window's first state (results do not depend on it)
    st0 = g.state()

    def reset():
        g.set_state(st0)
        g.set_step_index(start)

    g.step(W)
    g.sync()
    reset()
    n_body_iter = sc.n_bodies * sc.params["n_iter"]
    mean_sweeps = None
    if sc.params.get("resid_tol", 0.0) > 0:
        counts = []
        for _ in range(K):
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
    out = {"g": g, "t_ms": t_ms, "n_body_iter": n_body_iter, "mean_sweeps": mean_sweeps, "clocks": clk.summary(),
           "launches": info1["launches"] - info0["launches"], "info": info1, "K": K, "st0": st0}

    # live stage timing of the same K steps (graph with event nodes between the stages)
    reset()
    g.set_profiling(True)
    g.profile(reset=True)
    for _ in range(K):
        l2_flush()
        g.step(1)
    out["prof"] = g.profile(reset=True)
    g.set_profiling(False)

    if plain:
        reset()
        evp = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        barrier()
        for k in range(K):
            l2_flush()
            evp[k][0].record(stream)
            g.step_eager(1)
            evp[k][1].record(stream)
        barrier()
        out["t_plain"] = sum(a.elapsed_time(b) for a, b in evp)

    if e2e:
        # end to end through the C-ABI with host buffers: every step writes the whole state from
        # page-locked host memory (H2D), steps, and reads the state back (D2H), in the device's
        # single-precision layout (pabd_write_state_f32 / pabd_read_state_f32)
        reset()
        host = torch.empty(24 * sc.n_bodies, dtype=torch.float32, pin_memory=True)
        g.read_state_f32(host.data_ptr())
        g.sync()
        barrier()
        t0 = time.perf_counter()
        for _ in range(K):
            g.write_state_f32(host.data_ptr())
            g.step(1)
            g.read_state_f32(host.data_ptr())
            g.sync()
        barrier()
        out["t_e2e_ms"] = (time.perf_counter() - t0) * 1e3
        out["h2d"] = sc.n_bodies * 96
        out["d2h"] = sc.n_bodies * 96
    reset()
    if not keep:
        g.close()
        out["g"] = None
    return out


def roofline(m, sc, name, start, stacked=False):
    """Roofline of the sweep inside the timed window, per sweep (the sweep's launches: one, or a
    bond and a solve launch): algorithmic bytes (164 B per body + 148 B per bond, this
    window's own mean bond count) / its mean duration (the sweep stage's events bracket all of
    a step's sweep launches)."""
    prof, info = m["prof"], m["info"]
    steps = max(prof["steps"], 1)
    n_it = sc.params["n_iter"]
    bonds_avg = prof["bonds_sum"] / steps
    N = sc.n_bodies
    mode = info["sweep_mode"]
    per_sweep = 164.0 * N + 148.0 * bonds_avg
    if mode == 3:
        kernel, per_launch = "k_sweep_fused", per_sweep  # (one launch runs all sweeps; per sweep)
    elif mode == 2:
        kernel, per_launch = "k_sweep_one", per_sweep
    else:
        kernel, per_launch = "k_bond+k_solve", per_sweep
    # (the sweep stage's events bracket all of a step's sweep launches; per sweep)
    ms_launch = prof["sweep_ms"] / max(prof["sweeps"], 1)
    achieved = per_launch / (ms_launch * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    key = window_key(name, N, start, stacked)
    tr = _ncu_traffic(kernel, key)
    return {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs (of {peak_kind})",
            "traffic": tr["bytes_per_launch"] if tr else None,
            "traffic_window": key if tr else None,
            "bytes_per_launch": per_launch, "bytes_formula": "164 * bodies + 148 * bonds (this window's mean)",
            "us_per_launch": ms_launch * 1e3, "bonds_per_step": bonds_avg,
            "launches_per_step": prof["sweep_launches"] / steps,
            "stage_ms_per_step": {k: prof[k] / steps for k in ("collision_ms", "csr_ms", "predict_ms", "sweep_ms",
                                                                 "finalize_ms", "step_ms")}}


def alone_plain(P, torch, sc, dev, stream, K):
    """32 of the batched scenes, each alone in its own library scene on the plain path."""
    sizes = sc.meta["sizes"]
    pick = np.linspace(0, len(sizes) - 1, 32).astype(int)
    t_alone, body_iter = 0.0, 0
    for gi in pick:
        sub = S.select_groups(sc, [gi])
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
    return {"value": body_iter / (t_alone * 1e-3), "unit": UNIT, "ms_per_scene_step": t_alone / len(pick) / min(K, 20),
            "sample": f"{len(pick)} of the trees, each alone in its own scene on the plain path (eager launches), "
                      f"{min(K, 20)} steps each from step 0"}


def served(P, torch, dev, rates, duration, drain=20.0):
    """Poisson step requests over resident pile scenes of 10 to 1e5 bodies (one entry per
    rate), against each scene's step alone on the plain path."""
    from paper_2609_02675_gb300.serve import Server, replay

    def make(n):
        return S.box_pile_n(int(n), seed=S.SEED_BASE + 5, stacked=True, n_iter=30)

    out = []
    for rate in rates:
        reqs, sizes = S.request_stream(rate=rate, duration=duration, max_scenes=64)
        srv = Server(lambda sid: make(sizes[sid]), hbm_budget=32 << 30, device=dev)
        t0, t1 = replay(srv, reqs, duration=duration, drain_timeout=drain)
        st = srv.stats(t0, t1)
        srv.close()
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
        st.update({"rate": rate, "scenes": len(sizes), "plain_path_step_ms_mean": float(np.mean(alone_ms)),
                   "plain_path_sizes": [int(n) for n in pick]})
        out.append(st)
        torch.cuda.empty_cache()
    return out


def side_line(name, sc, m, start, K, stacked=False):
    """A compact record of a non-headline workload measured in the same run."""
    n_it = m["n_body_iter"]
    r = roofline(m, sc, name, start, stacked)
    d = {"workload": describe(name, sc, start, K, stacked), "value": n_it * K / (m["t_ms"] * 1e-3), "unit": UNIT,
         "ms_per_step": m["t_ms"] / K, "steps_per_s": K / (m["t_ms"] * 1e-3),
         "sweep": {k: r[k] for k in ("kernel", "us_per_launch", "bytes_per_launch", "bonds_per_step", "frac",
                                     "achieved", "traffic")}}
    if "t_plain" in m:
        d["plain_path"] = {"value": n_it * K / (m["t_plain"] * 1e-3), "ms_per_step": m["t_plain"] / K}
    return d


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2609_02675_gb300 as P

    dev = local_rank
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    name = args.workload
    sc = make_workload(name, args.bodies, args.stacked, args.resid_tol)
    start = start_step(name, args.stacked, args.bodies, args.start_step)
    K, W = args.steps, args.warmup
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{dev}")
    m = measure(P, torch, sc, name, start, K, W, dev, stream, world, flush, args.sweep_mode, args.lanes,
                args.stacked, keep=True, light_order=args.light_order)
    g = m["g"]
    t_ms, t_plain, t_e2e_ms = max_over_ranks([m["t_ms"], m["t_plain"], m["t_e2e_ms"]], world, f"cuda:{dev}")
    if rank != 0:
        g.close()
        return
    n_body_iter = m["n_body_iter"]
    info1 = m["info"]
    cfg = {"workload": describe(name, sc, start, K, args.stacked), "n_bodies": sc.n_bodies,
           "n_iter": sc.params["n_iter"], "start_step": start, "l2": L2_NOTE, "parallelism": "replicas",
           **tol_cfg(args.resid_tol)}
    cfg["sweep"] = {k: info1[k] for k in ("sweep_mode", "sweep_lanes", "light_order", "tuned")}
    cfg["sweep"]["tune_sweep_us"] = {n: info1[f"tune_sweep_ns{k}"] / 1e3 for k, n in enumerate(
        ("one_launch_ordered", "one_launch_body_order", "two_launch_ordered", "two_launch_body_order"))}
    if m["mean_sweeps"] is not None:
        cfg["mean_sweeps_per_step"] = m["mean_sweeps"]
    line = {
        "metric": METRIC, "value": job_throughput(n_body_iter * K, world, t_ms), "unit": UNIT, "n_gpus": world,
        "steps": K, "warmup": W, "ms_per_step": t_ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
        "steps_per_s": world * K / (t_ms * 1e-3),
        "plain_path": {"value": job_throughput(n_body_iter * K, world, t_plain), "unit": UNIT,
                       "ms_per_step": t_plain / K},
        "e2e": {"value": job_throughput(n_body_iter * K, world, t_e2e_ms), "unit": UNIT,
                "h2d_bytes_per_step": m["h2d"], "d2h_bytes_per_step": m["d2h"]},
        "gpu_launches": int(m["launches"]),
        "clocks": m["clocks"],
        "roofline": roofline(m, sc, name, start, args.stacked),
    }
    if not args.no_cpu_baseline and world == 1:
        def gpu_check(st_sample, groups, k):
            # the oracle's sampled rows written into the full scene's state, one graph step
            full = m["st0"].copy()
            rows = S.group_rows(sc, groups) if groups is not None else np.arange(sc.n_bodies)
            full[rows] = st_sample
            g.set_state(full)
            g.set_step_index(k)
            g.step(1)
            return g.state()[rows]
        line["cpu_baseline"], parity = cpu_baseline(name, sc, start, K, gpu_check=gpu_check)
        if parity is not None:
            line["parity"] = parity
    g.close()
    if name == "trees" and world == 1 and not args.no_extras:
        extra = {}
        extra["scenes_alone_plain_path"] = alone_plain(P, torch, sc, dev, stream, K)
        pile = make_workload("pile")
        ps = DEFAULT_START["pile"]
        extra["pile_4096_landed"] = side_line("pile", pile, measure(P, torch, pile, "pile", ps, K, W, dev, stream,
                                                                     flush=flush, e2e=False), ps, K)
        del pile
        qd = make_workload("quadruped")
        qs = DEFAULT_START["quadruped"]
        extra["quadruped_bed_rod"] = side_line("quadruped", qd, measure(P, torch, qd, "quadruped", qs, min(K, 10),
                                                                         W, dev, stream, flush=flush, plain=False,
                                                                         e2e=False), qs, min(K, 10))
        del qd
        del flush
        torch.cuda.empty_cache()
        extra["served"] = {"config": "Poisson step requests (1-60 steps each) over at most 64 stacked-pile scenes of "
                                     f"10-1e5 bodies, {args.served_duration:.0f} s of arrivals per rate, HBM budget "
                                     "32 GB, one stream per resident scene",
                           "rates": served(P, torch, dev, [100.0, 1000.0], args.served_duration)}
        line.update(extra)
    print(json.dumps(line), flush=True)


def run_served(args, dev):
    import torch
    import paper_2609_02675_gb300 as P
    torch.cuda.set_device(dev)
    rates = [float(x) for x in args.rates.split(",")]
    line = {"metric": "served step latency", "unit": "ms", "higher_is_better": False, "n_gpus": 1,
            "data": "synthetic", "dtype": "f32",
            "config": {"workload": f"Poisson step requests (1-60 steps) over at most 64 pile scenes of 10-1e5 "
                                   f"bodies, {args.duration:.0f} s of arrivals per rate (then up to 20 s to drain), "
                                   f"HBM budget 32 GB",
                       "parallelism": "one scene per stream, continuous batching"},
            "rates": served(P, torch, dev, rates, args.duration)}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="headline workload only")
    ap.add_argument("--workload", default="trees",
                    choices=["trees", "pile", "quadruped", "served", "stack", "spring", "net"])
    ap.add_argument("--resid-tol", type=float, default=0.0,
                    help="residual threshold of the sweeps (0: a fixed n_iter sweeps per step)")
    ap.add_argument("--rates", default="100,300,1000,3000,10000", help="served: request rates (req/s)")
    ap.add_argument("--duration", type=float, default=3.0, help="served: seconds of arrivals per rate")
    ap.add_argument("--served-duration", type=float, default=2.0,
                    help="seconds of arrivals per rate of the served entry of the headline line")
    ap.add_argument("--bodies", type=int, default=4096, help="pile size (4096 = the 16^3 pile)")
    ap.add_argument("--stacked", action="store_true", help="pile as touching columns (contacts from step 0)")
    ap.add_argument("--start-step", type=int, default=-1,
                    help="first step of the timed window (untimed lead-in before it); -1: the workload's default")
    ap.add_argument("--sweep-mode", type=int, default=0,
                    help="1: two launches per sweep, 2: one launch per sweep, 3: fused persistent, 0: library choice")
    ap.add_argument("--lanes", type=int, default=0, help="lanes per body in the fused sweep (0: library default)")
    ap.add_argument("--light-order", type=int, default=0,
                    help="1: light bodies ordered by end count, 2: body order, 0: library choice")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        import oracle
        oracle.build()
        run_reference(args, rank, world)
        return
    import __graft_entry__
    __graft_entry__.build()
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
    main()

#!/usr/bin/env python
"""Benchmark: iGMRES-PI (Alg. 2) solves per second on the paper-scale dense MDP.

Workload: S = 10^4 states, A = 8 actions, dense row-stochastic P_a stored in FP32 (rows
Dirichlet(0.1)), costs U(0,1), gamma = 0.99; the mixed FP32 / double-float form solved to
||T(v) - v||_inf <= 1e-8 with alpha = 0.1, GMRES restart W = 30.  One step = one whole
solve from V_0 = 0 with the MDP resident in HBM (3.2 GB of P: every sweep streams more than
the 129 MB L2, so no flush is needed between steps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torch.distributed.run, one rank per GPU; every rank solves its own copy
of the workload (independent problems, no collective on the data path) and rank 0 prints
one JSON line with the whole-job rate.  --impl reference times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "MDP solves/s to ||T(v)-v||_inf<=1e-8, p50/p99 latency; Bellman-op HBM GB/s"
S_, A_, GAMMA, TOL, ALPHA, W_ = 10000, 8, 0.99, 1e-8, 0.1, 30
WORKLOAD = ("paper-scale dense MDP: S=10000, A=8, FP32 P_a rows Dirichlet(0.1), g~U(0,1), "
            "gamma=0.99; iGMRES-PI mixed FP32/double-float, alpha=0.1, W=30, tol 1e-8")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the batched (config 4) and banded (config 3) "
                         "legs reported beside the headline")
    ap.add_argument("--host-loop", action="store_true",
                    help="enqueue inner GMRES steps from the host (for profilers that cannot "
                         "follow conditional CUDA-graph nodes)")
    ap.add_argument("--S", type=int, default=S_,
                    help="states of the dense (or, with --config 3, banded) workload; other "
                         "values only for profiling")
    ap.add_argument("--duration", type=float, default=60.0,
                    help="serving workload: seconds of the Poisson request trace")
    ap.add_argument("--pool", type=int, default=64,
                    help="serving workload: distinct MDPs the requests draw from")
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4, 5],
                    help="workload: 2 = the paper-scale dense MDP (the benchmark), 1 = small "
                         "ELL, 3 = S=10^6 banded ELL (for measurement of the ELL kernels), "
                         "4 = a batch of 256 independent ELL MDPs solved together, "
                         "5 = a Poisson stream of requests served with continuous batching")
    ap.add_argument("--batch", type=int, default=256, help="instances of the batched workload")
    ap.add_argument("--forcing-c", type=float, default=0.0,
                    help="forcing sequence alpha_k = min(alpha, c ||Phi_k||_inf) for the timed "
                         "solves (0 = constant alpha, Alg. 2)")
    ap.add_argument("--precond-block", type=int, default=0,
                    help="ELL workloads: two-level preconditioned inner GMRES with aggregation "
                         "blocks of this many states (0 = plain Alg. 2)")
    ap.add_argument("--study", choices=["fig2"], default=None,
                    help="fig2: GMRES vs VI policy evaluation across gamma at n=100 (Sec. 3.1): "
                         "Arnoldi steps, VI sweeps and times on the GPU; one JSON line")
    ap.add_argument("--sweep-only", action="store_true",
                    help="time Bellman sweeps alone (bellman_apply at a fixed v, no solve) on the "
                         "single-MDP workloads: the metric's Bellman-op HBM GB/s")
    ap.add_argument("--no-tune", action="store_true",
                    help="batched workload: keep the library's lanes per row (no autotuning), "
                         "so the launch sequence is the same on every run (for profilers)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def sweep_algorithmic_bytes(syn):
    """Bytes one full Bellman sweep must move: every P_a entry (FP32 value, plus an int32
    column for ELL), the costs as double-float pairs, v read once (8 B/state) and pi, Tv, Phi
    written (4 + 8 + 4 B/state)."""
    S, A = syn.S, syn.A
    per_row = S * 4 if syn.kind == "dense" else syn.k * 8
    return A * S * per_row + A * S * 8 + S * 8 + S * 16


def matvec_algorithmic_bytes(syn):
    """One P^pi matvec in FP32: row pi(s) of P_{pi(s)} per state, pi, x read, w written."""
    S = syn.S
    per_row = S * 4 if syn.kind == "dense" else syn.k * 8
    return S * per_row + S * (4 + 4 + 4)


def workload_name(args, syn):
    if syn.kind == "dense":
        base = WORKLOAD
        if syn.S != S_:
            base += f" [profiling size S={syn.S}]"
        return base
    return (f"ELL MDP config {args.config}: S={syn.S}, A={syn.A}, k={syn.k}, FP32 values, "
            f"gamma={syn.gamma}; iGMRES-PI mixed FP32/double-float, alpha=0.1, W=30, tol 1e-8")


def source_hash():
    h = hashlib.sha256()
    for rel in ["paper_2211_04299_gb300/csrc/sweep.cu", "paper_2211_04299_gb300/csrc/mdp_internal.cuh"]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


WIN_SPAN_MAX, WIN_MIN_S = 1792, 1024  # the library's windowed-sweep rule (banded ELL data)


def sweep_kernel_name(syn):
    """The sweep kernel the library runs for this MDP (same rule as the library's launcher)."""
    if syn.kind == "dense":
        return "sweep_dense_tma_kernel"
    rows = np.arange(syn.S, dtype=np.int32)[:, None]
    span = max(int(np.max(np.abs(syn.col[a] - rows))) for a in range(syn.A))
    return ("sweep_ell_window_kernel" if span <= WIN_SPAN_MAX and syn.S >= WIN_MIN_S
            else "sweep_ell_warp_kernel")


def sweep_traffic(args, syn):
    if syn.kind == "dense" and syn.S == S_:
        return traffic_for("sweep_dense_df_cfg2")
    if args.config == 3 and syn.S == 1_000_000:
        return traffic_for("sweep_ell_window_cfg3")
    return None


def traffic_for(kernel_key):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    kernel source; otherwise None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(kernel_key)
        if e and e.get("source_hash") == source_hash():
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = [ln.split(",") for ln in open(self.file.name).read().strip().splitlines()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
            except ValueError:
                continue
            for nm, val in zip(names, r[5:9]):
                if "Active" in val and "Not" not in val:
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}



# ---------------------------------------------------------------- replicas
def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest x over all ranks (each rank times its own replica; the job took as long as
    the slowest).  device: "cuda" under NCCL, "cpu" under gloo."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, seconds_local: float, world: int, device: str = "cuda") -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return world * units_per_rank / max_over_ranks(seconds_local, world, device)

# ---------------------------------------------------------------- CPU oracle arm
def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.startswith("model name") or ln.startswith("CPU part"):
                    return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cores_used() -> int:
    """Threads the oracle's numpy/BLAS work can use in this process: the BLAS pool's size
    when threadpoolctl can read it, else the thread-count variables, else every core."""
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        if info:
            return int(max(i.get("num_threads", 1) for i in info))
    except Exception:
        pass
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(var, "").isdigit():
            return int(os.environ[var])
    return os.cpu_count() or 1


def oracle_solve_seconds(m) -> tuple[float, object]:
    """One whole oracle iGMRES-PI solve (Alg. 2 to ||T(v)-v||_inf <= 1e-8 from V_0 = 0)."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.gmres_policy_iteration(m, alpha=ALPHA, W=W_, tol=TOL)
    return time.perf_counter() - t0, r


ONE_CORE_ENV = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}


def oracle_one_core(config: int, max_solves: int = 1) -> dict:
    """Whole oracle solves of a workload in a child interpreter whose BLAS and OpenMP pools are
    set to one thread before numpy loads (the paper's single-core setting, Sec. 4)."""
    env = dict(os.environ, **ONE_CORE_ENV)
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench._one_core_child(%d, %d)))" % (ROOT, config, max_solves))
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True,
                             text=True, timeout=900)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as e:  # reported, not fatal: the all-core figure stands on its own
        return {"error": f"one-core oracle run failed: {type(e).__name__}"}


def _one_core_child(config: int, max_solves: int) -> dict:
    import mdp_synth
    import oracle
    if config == 4:
        specs = mdp_synth.batch_specs(256, mdp_synth.CONFIG_SEEDS[4])
        syns = (mdp_synth.instance_from_spec(sp) for sp in specs)
    else:
        syns = iter([mdp_synth.config(2)])
    secs, n = 0.0, 0
    for syn in syns:
        dt, _ = oracle_solve_seconds(oracle.from_synth(syn))
        secs += dt
        n += 1
        if n >= max_solves:
            break
    return {"value": n / secs, "unit": "solves/s", "cores": cores_used(), "solves": n,
            "seconds": secs}


def config_fields(args, syn) -> dict:
    """The bench line's `config` object for a single-MDP workload (both arms use it)."""
    sb = sweep_algorithmic_bytes(syn)
    return {"workload": workload_name(args, syn), "S": syn.S, "A": syn.A, "gamma": syn.gamma,
            "tol": TOL, "alpha": ALPHA, "restart": W_, "forcing_c": args.forcing_c,
            "precond_block": args.precond_block,
            "l2": f"inputs larger than L2 (P is {sb / 1e9:.2f} GB per sweep, L2 129 MB); no flush"}


def reference_line(args, value, total_s, config, sample, extra=None):
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores_used(),
                         "cpu": cpu_model(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    if extra:
        line["cpu_baseline"].update(extra)
    return line


def reference_arm_batch(args):
    """The oracle on the batched workload: each step solves the next instance of the batch
    (Alg. 2 to 1e-8); the rate is instances per second of oracle time."""
    import mdp_synth
    import oracle
    specs = mdp_synth.batch_specs(args.batch, mdp_synth.CONFIG_SEEDS[4])
    total = 0.0
    for i in range(args.warmup + args.steps):
        syn = mdp_synth.instance_from_spec(specs[i % len(specs)])
        dt, _ = oracle_solve_seconds(oracle.from_synth(syn))
        if i >= args.warmup:
            total += dt
    value = args.steps / total
    sample = (f"per step: one whole oracle iGMRES-PI solve of the next instance of the batch "
              f"(instances {args.warmup}..{args.warmup + args.steps - 1} of {args.batch})")
    cfg = {"workload": BATCH_WORKLOAD.format(n=args.batch), "instances": args.batch,
           "tol": TOL, "alpha": ALPHA, "restart": W_}
    print(json.dumps(reference_line(args, value, total, cfg, sample)), flush=True)
    return 0


def reference_arm(args):
    """The oracle on the benchmark workload: every step (warm-up and timed) is one whole
    iGMRES-PI solve of the paper-scale dense MDP from V_0 = 0 on all host cores; afterwards one
    more whole solve runs on one core in a child interpreter."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.config == 4:
        return reference_arm_batch(args)
    import mdp_synth
    import oracle
    syn = mdp_synth.config(2)
    m = oracle.from_synth(syn)
    for _ in range(args.warmup):
        oracle_solve_seconds(m)
    times = []
    for _ in range(args.steps):
        dt, r = oracle_solve_seconds(m)
        times.append(dt)
    total = sum(times)
    value = args.steps / total
    sample = (f"per step: one whole oracle iGMRES-PI solve (Alg. 2, FP64 numpy) of the full "
              f"workload from V_0 = 0 ({r.outer} outer, {r.inner} inner iterations)")
    extra = {"p50_s": statistics.median(times), "one_core": oracle_one_core(2)}
    line = reference_line(args, value, total, config_fields(args, syn), sample, extra)
    line["config"]["parallelism"] = f"replicas x{args.gpus}"
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- batched workload
BATCH_WORKLOAD = ("batch of {n} independent ELL MDPs: S log-uniform in [500, 50000], A uniform "
                  "in 2..16, k in {{8, 16, 32}}, gamma in {{0.9, 0.99, 0.999}}, FP32 values, "
                  "g~U(0,1); iGMRES-PI mixed FP32/double-float, alpha=0.1, W=30, tol 1e-8, all "
                  "instances in one CUDA-graph launch")


def oracle_batch_sample(syns, budget_s=12.0):
    """Oracle iGMRES-PI (Alg. 2) solves of the batch's first instances (an i.i.d. sample of
    its distribution) until about budget_s seconds of CPU time -> (solves/s, instances, s)."""
    import oracle
    t_tot, n = 0.0, 0
    for syn in syns:
        m = oracle.from_synth(syn)
        t0 = time.perf_counter()
        oracle.gmres_policy_iteration(m, alpha=ALPHA, W=W_, tol=TOL)
        t_tot += time.perf_counter() - t0
        n += 1
        if t_tot >= budget_s:
            break
    return n / t_tot, n, t_tot


def run_batch_bench(args, mg, torch, dist, world, rank, local, extra=False):
    """The batched workload.  extra=True: the leg reported beside the headline line (10 timed
    batch solves, the per-instance FP64 and mixed forms; no e2e, forcing or CPU legs); returns
    the dict instead of printing it."""
    import mdp_synth
    n = args.batch
    steps = 10 if extra else args.steps
    specs = mdp_synth.batch_specs(n, mdp_synth.CONFIG_SEEDS[4])
    syns = [mdp_synth.instance_from_spec(sp) for sp in specs]
    hs = [mg.from_synth(syn) for syn in syns]
    # a stream of our own: the CUDA events below must be recorded on the stream the batch
    # launches on (torch's default stream is the legacy stream, handle 0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    o = mg.opts(tol=TOL, alpha=ALPHA, restart=W_, precision="mixed", forcing_c=args.forcing_c,
                flags=mg.MDP_FLAG_HOST_LOOP if args.host_loop else 0)
    b = mg.MDPBatch(hs, o)
    b.set_stream(stream)
    if not args.no_tune:
        b.tune()
    vd = [torch.empty(h.S, dtype=torch.float64, device="cuda") for h in hs]
    pd = [torch.empty(h.S, dtype=torch.int32, device="cuda") for h in hs]

    def barrier():
        if world > 1:
            dist.barrier()

    warm = max(3, args.warmup)
    for _ in range(warm):
        b.solve(vd, pd)
    torch.cuda.synchronize()
    barrier()
    clocks = Clocks(local)
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    stats = []
    ev[0].record(stream)
    for i in range(steps):
        _, _, st, code = b.solve(vd, pd)
        ev[i + 1].record(stream)
        stats.append((st, code))
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    elapsed_ms = ev[0].elapsed_time(ev[-1])
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    value = job_rate(n * steps, elapsed_ms / 1000.0, world)
    elapsed_ms = max_over_ranks(elapsed_ms, world)
    ok = all(code == 0 and all(x["status"] == 0 and x["residual_inf"] <= TOL for x in st)
             for st, code in stats)
    st_last = stats[-1][0]

    # dominant kernel family: the batched Bellman sweep over every instance, timed alone
    peak, peak_kind = peaks()
    sb = float(sum(sweep_algorithmic_bytes(syn) for syn in syns))
    reps = 20
    b.bellman(wait=False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        b.bellman(wait=False)
    e1.record(stream)
    torch.cuda.synchronize()
    sweep_ms = e0.elapsed_time(e1) / reps
    sweep_gbs = sb / (sweep_ms * 1e-3) / 1e9
    launches = int(sum(st[0]["launches"] for st, _ in stats))
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": steps, "warmup": warm, "ms_per_step": elapsed_ms / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "mixed: f32 P/Krylov, double-float (2xf32) values, f64 Givens",
        "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD.format(n=n), "instances": n,
                   "states_total": int(sum(syn.S for syn in syns)),
                   "nonzeros_total": int(sum(syn.S * syn.A * syn.k for syn in syns)),
                   "tol": TOL, "alpha": ALPHA, "restart": W_, "precision": "mixed",
                   "parallelism": f"replicas x{world}",
                   "l2": f"inputs larger than L2 ({sb / 1e9:.2f} GB per batched sweep); no flush"},
        "step": "one batched solve of every instance (solves/s counts instances)",
        "converged": ok,
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                       "p99": float(np.percentile(step_ms, 99)),
                       "note": "every instance of a batch completes when the batch does"},
        "per_batch": {"loop_iterations_launches": st_last[0]["launches"],
                      "outer_max": max(x["outer"] for x in st_last),
                      "inner_sum": int(sum(x["inner"] for x in st_last)),
                      "sweeps_sum": int(sum(x["sweeps"] for x in st_last))},
        "bellman_sweep": {"ms": sweep_ms, "gbs": sweep_gbs, "algorithmic_bytes": sb,
                          "scope": "one batched sweep of all instances"},
        "roofline": {"bound": "hbm", "kernel": "batch_sweep_kernel", "achieved": sweep_gbs,
                     "peak": peak, "unit": "GB/s", "frac": sweep_gbs / peak,
                     "peak_source": peak_kind, "traffic": None},
        "gpu_launches": launches,
        "clocks": clk,
    }
    line["config"]["forcing_c"] = args.forcing_c

    if args.forcing_c == 0.0 and not extra:
        # the same batch with the adaptive forcing sequence (Sec. 3: alpha_k -> 0)
        ba = mg.MDPBatch(hs, mg.opts(tol=TOL, alpha=ALPHA, restart=W_, precision="mixed",
                                     forcing_c=1.0))
        ba.set_stream(stream)
        if not args.no_tune:
            ba.tune()
        ba.solve(vd, pd)
        na = min(steps, 5)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(na):
            _, _, sta, ca = ba.solve(vd, pd)
        a1.record(stream)
        torch.cuda.synchronize()
        line["adaptive_forcing"] = {"forcing_c": 1.0,
                                    "value": n * na / (a0.elapsed_time(a1) / 1000.0),
                                    "unit": "solves/s", "converged": ca == 0,
                                    "outer_max": max(x["outer"] for x in sta),
                                    "inner_sum": int(sum(x["inner"] for x in sta))}
        ba.close()

    if not args.no_e2e and not extra:
        # through the host-pointer API: every step uploads every instance's P and g from pinned
        # memory (mdp_load_ell_async), solves the batch and copies every v and pi back.  Two
        # sets of handles and batches alternate, so step i+1's uploads run while step i solves.
        pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy()
        pins = [(pin(syn.col), pin(syn.val), pin(syn.g)) for syn in syns]
        in_bytes = int(sum(c.nbytes + v.nbytes + g.nbytes for c, v, g in pins))
        vh = [np.empty(syn.S) for syn in syns]
        ph = [np.empty(syn.S, np.int32) for syn in syns]
        out_bytes = int(sum(x.nbytes for x in vh) + sum(x.nbytes for x in ph))
        hs2 = [mg.from_synth(syn) for syn in syns]
        b2 = mg.MDPBatch(hs2, o)
        b2.set_stream(stream)
        if not args.no_tune:
            b2.tune()
        sets = [(hs, b), (hs2, b2)]

        # issuing 256 handles' uploads is thousands of API calls: a second host thread issues
        # the next set's while this one waits for the current batch (calls on different
        # handles are independent; the library's error message is per thread)
        from concurrent.futures import ThreadPoolExecutor
        loader = ThreadPoolExecutor(max_workers=1)

        def load_set(j):
            torch.cuda.set_device(local)  # the loader thread works on this rank's GPU
            for hh, (c, v, g) in zip(sets[j][0], pins):
                mg.mdp_load_ell_async(hh, c, v, g)

        def e2e_run(k):
            load_set(0)
            for i in range(k):
                nxt = loader.submit(load_set, (i + 1) % 2) if i + 1 < k else None
                sets[i % 2][1].solve(vh, ph)
                if nxt is not None:
                    nxt.result()

        e2e_run(2)
        torch.cuda.synchronize()
        barrier()
        e2e_steps = min(steps, 4)
        t0 = time.perf_counter()
        e2e_run(e2e_steps)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        loader.shutdown()
        b2.close()
        for hh in hs2:
            hh.close()
        line["e2e"] = {"value": job_rate(n * e2e_steps, dt, world), "unit": "solves/s",
                       "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": out_bytes,
                       "steps": e2e_steps}
        del pins

    if not args.no_fp64:
        # the plain per-instance forms on the same MDPs: FP64 (P widened exactly) and the
        # single-instance mixed solver, one solve after another
        def per_instance(make_handle, prec):
            tot = 0.0
            for syn, h0 in zip(syns, hs):
                h = make_handle(syn, h0)
                h.set_stream(stream)
                oo = mg.opts(tol=TOL, alpha=ALPHA, restart=W_, precision=prec)
                vo = torch.empty(syn.S, dtype=torch.float64, device="cuda")
                po = torch.empty(syn.S, dtype=torch.int32, device="cuda")
                mg.ipi_solve(h, oo, v_out=vo, pi_out=po)
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                mg.ipi_solve(h, oo, v_out=vo, pi_out=po)
                a1.record(stream)
                torch.cuda.synchronize()
                tot += a0.elapsed_time(a1)
                if h is not h0:
                    h.close()
            return n / (tot / 1000.0), tot

        def fp64_handle(syn, h0):
            return mg.from_synth(mdp_synth.SynthMDP(S=syn.S, A=syn.A, gamma=syn.gamma, g=syn.g,
                                                    kind="ell", col=syn.col,
                                                    val=syn.val.astype(np.float64)), device=False)

        v64, ms64 = per_instance(fp64_handle, "fp64")
        vmx, msmx = per_instance(lambda syn, h0: h0, "mixed")
        line["fp64_plain"] = {"value": v64, "unit": "solves/s", "ms_total": ms64,
                              "form": "one ipi_solve per instance, FP64 P and Krylov"}
        line["mixed_single"] = {"value": vmx, "unit": "solves/s", "ms_total": msmx,
                                "form": "one ipi_solve per instance, mixed precision"}

    if rank == 0 and world == 1 and not args.no_cpu_baseline and not extra:
        rate, m_done, secs = oracle_batch_sample(syns)
        line["cpu_baseline"] = {
            "value": rate, "unit": "solves/s", "cores": cores_used(), "cpu": cpu_model(),
            "kind": "oracle",
            "sample": (f"oracle iGMRES-PI (Alg. 2) solves of the batch's first {m_done} "
                       f"instances ({secs:.1f} s of CPU); instances are i.i.d. draws")}
    b.close()
    for h in hs:
        h.close()
    if extra:
        for key in ("metric", "n_gpus", "higher_is_better", "scaling", "vs_baseline", "data"):
            line.pop(key, None)
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- serving workload
SERVE_WORKLOAD = ("Poisson stream of solve requests at 200/s for {dur:g} s ({n} requests): ELL "
                  "MDPs with S log-uniform in [1e3, 2e5], A in {{4, 8, 16}}, k=16, gamma in "
                  "{{0.95, 0.99}}, FP32 values, g~U(0,1), drawn from {pool} distinct seeded "
                  "instances; iGMRES-PI mixed, alpha=0.1, W=30, tol 1e-8; continuous batching "
                  "with a 120 GB HBM budget; each request uploads its P and g from pinned host "
                  "memory and copies v, pi back")


def serve_trace(args):
    import mdp_synth
    trace = mdp_synth.serving_trace(200.0, args.duration, mdp_synth.CONFIG_SEEDS[5])
    npool = min(args.pool, len(trace))
    return trace, npool


def replay(trace, npool, submit, poll, idle_wait=0.0002):
    """Submit request j at trace[j]['t'] (seconds after start) -> per-request latency (s),
    wall time from the first arrival to the last completion."""
    n = len(trace)
    arrive = {}
    lat = {}
    t0 = time.perf_counter()
    nxt = 0
    while len(lat) < n:
        now = time.perf_counter() - t0
        while nxt < n and trace[nxt]["t"] <= now:
            rid = submit(nxt, nxt % npool)
            arrive[rid] = t0 + trace[nxt]["t"]
            nxt += 1
        done = poll()
        t = time.perf_counter()
        for rid, status in done:
            lat[rid] = (t - arrive[rid], status)
        if not done and nxt < n:
            time.sleep(idle_wait)
    t_end = time.perf_counter()
    return lat, t_end - (t0 + trace[0]["t"])


def run_serve_bench(args, mg, torch, dist, world, rank, local, extra=False):
    """The serving workload.  extra=True: the leg reported beside the headline line (a shorter
    trace, no CPU leg); returns the dict instead of printing it."""
    import mdp_synth
    trace, npool = serve_trace(args)
    n = len(trace)
    pool = [mdp_synth.instance_from_spec(sp) for sp in trace[:npool]]
    pinned = [(torch.from_numpy(np.ascontiguousarray(p.col)).pin_memory().numpy(),
               torch.from_numpy(np.ascontiguousarray(p.val)).pin_memory().numpy(),
               torch.from_numpy(np.ascontiguousarray(p.g)).pin_memory().numpy()) for p in pool]
    o = mg.opts(tol=TOL, alpha=ALPHA, restart=W_, precision="mixed")
    srv = mg.MDPServer(o=o, hbm_budget_bytes=120 << 30)
    statuses = []

    def submit(j, pi):
        c, v, g = pinned[pi]
        return srv.submit(c, v, g, pool[pi].gamma)

    def poll():
        out = []
        for rid, _, _, st in srv.poll():
            out.append((rid, st["status"]))
            statuses.append(st)
        return out

    # warm-up: the first pool instances once each
    for j in range(min(8, npool)):
        submit(j, j)
    srv.drain()
    srv.poll()
    statuses.clear()
    l0 = srv.info()["launches"]
    clocks = Clocks(local)
    clocks.start()
    lat, wall = replay(trace, npool, submit, poll)
    clk = clocks.stop()
    launches = srv.info()["launches"] - l0
    lats = np.array([x[0] for x in lat.values()]) * 1000.0
    ok = all(x[1] == 0 for x in lat.values())
    value = n / wall

    # capacity: the same requests all submitted at once
    sat_n = min(n, 1000)
    t0 = time.perf_counter()
    for j in range(sat_n):
        submit(j, j % npool)
    srv.drain()
    srv.poll()
    sat = sat_n / (time.perf_counter() - t0)
    srv.close()

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": n, "warmup": min(8, npool), "ms_per_step": 1000.0 * wall / n,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "mixed: f32 P/Krylov, double-float (2xf32) values, f64 Givens",
        "data": "synthetic",
        "config": {"workload": SERVE_WORKLOAD.format(dur=args.duration, n=n, pool=npool),
                   "requests": n, "rate_per_s": 200.0, "duration_s": args.duration,
                   "distinct_mdps": npool, "hbm_budget_gb": 120, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 in aggregate; no flush"},
        "step": "one request (arrival to result on the host)",
        "converged": ok,
        "latency_ms": {"p50": float(np.percentile(lats, 50)), "p99": float(np.percentile(lats, 99)),
                       "max": float(lats.max())},
        "capacity": {"value": sat, "unit": "solves/s", "requests": sat_n,
                     "form": "the trace's first requests submitted at once"},
        "gpu_launches": int(launches),
        "clocks": clk,
        "e2e": {"value": value, "unit": "solves/s",
                "h2d_bytes_per_step": int(np.mean([p.col.nbytes + p.val.nbytes + p.g.nbytes for p in pool])),
                "d2h_bytes_per_step": int(np.mean([p.S * 12 for p in pool])),
                "note": "the serving loop is end to end: uploads and result copies are inside"},
        "roofline": None,
    }

    if not args.no_fp64:
        # the plain FP64 per-request path on the same trace: one request after another, each
        # uploading its (FP64) data into a handle of its shape and solving it alone
        hs64 = []
        for p in pool:
            syn64 = mdp_synth.SynthMDP(S=p.S, A=p.A, gamma=p.gamma, g=p.g, kind="ell",
                                       col=p.col, val=p.val.astype(np.float64))
            hs64.append((mg.from_synth(syn64),
                         torch.from_numpy(np.ascontiguousarray(syn64.val)).pin_memory().numpy()))
        o64 = mg.opts(tol=TOL, alpha=ALPHA, restart=W_, precision="fp64")
        queue = []
        results = []
        rid_next = [0]

        def submit64(j, pi):
            rid_next[0] += 1
            queue.append((rid_next[0], pi))
            return rid_next[0]

        def poll64():
            if not queue:
                return []
            rid, pi = queue.pop(0)
            h, val64 = hs64[pi]
            c, _, g = pinned[pi]
            mg.mdp_load_ell(h, c, val64, g)
            v = np.empty(pool[pi].S)
            pi_o = np.empty(pool[pi].S, np.int32)
            _, _, st = mg.ipi_solve(h, o64, v_out=v, pi_out=pi_o)
            return [(rid, st["status"])]

        lat64, wall64 = replay(trace, npool, submit64, poll64)
        l64 = np.array([x[0] for x in lat64.values()]) * 1000.0
        # capacity of the plain path: the same first requests back to back
        t0 = time.perf_counter()
        for j in range(sat_n):
            submit64(j, j % npool)
        while queue:
            poll64()
        sat64 = sat_n / (time.perf_counter() - t0)
        line["fp64_plain"] = {"value": n / wall64, "unit": "solves/s",
                              "latency_ms": {"p50": float(np.percentile(l64, 50)),
                                             "p99": float(np.percentile(l64, 99))},
                              "capacity": {"value": sat64, "unit": "solves/s", "requests": sat_n},
                              "form": "one request after another: mdp_load_ell + ipi_solve FP64"}
        for h, _ in hs64:
            h.close()

    if extra:
        for key in ("metric", "n_gpus", "higher_is_better", "scaling", "vs_baseline", "data"):
            line.pop(key, None)
        return line
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        t_tot, m_done = 0.0, 0
        for p in pool:
            m = oracle.from_synth(p)
            t0 = time.perf_counter()
            oracle.gmres_policy_iteration(m, alpha=ALPHA, W=W_, tol=TOL)
            t_tot += time.perf_counter() - t0
            m_done += 1
            if t_tot >= 12.0:
                break
        line["cpu_baseline"] = {
            "value": m_done / t_tot, "unit": "solves/s", "cores": cores_used(), "cpu": cpu_model(),
            "kind": "oracle",
            "sample": f"oracle iGMRES-PI solves of the first {m_done} distinct request MDPs ({t_tot:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- GPU arm
def run_fig2_study(mg, torch, rank):
    """Fig. 2 (Sec. 3.1): policy evaluation of a dense n=100 MDP (one action, rows
    Dirichlet(1)) to ||g - J V||_inf <= 1e-8 by GMRES(64) and by VI, for several gamma (the
    counts are checked against the oracle in the GPU tests)."""
    import mdp_synth
    rows = []
    for g in (0.5, 0.9, 0.99, 0.999, 0.9999):
        syn = mdp_synth.dense_dirichlet(100, 1, 1.0, g, seed=2022, dtype=np.float64)
        h = mg.from_synth(syn)
        pi0 = np.zeros(100, np.int32)
        og = mg.opts(precision="fp64", restart=64)
        ov = mg.opts(precision="fp64", tol=1e-8, max_outer=10 ** 7)
        mg.policy_eval_gmres(h, pi0, target_inf=1e-8, o=og)
        t0 = time.perf_counter()
        _, st_g = mg.policy_eval_gmres(h, pi0, target_inf=1e-8, o=og)
        t1 = time.perf_counter()
        _, _, st_v = mg.vi_solve(h, ov)
        t2 = time.perf_counter()
        h.close()
        rows.append({"gamma": g, "gmres_steps": st_g["inner"], "vi_sweeps": st_v["outer"],
                     "converged": st_g["status"] == 0 and st_v["status"] == 0,
                     "gmres_ms": 1e3 * (t1 - t0), "vi_ms": 1e3 * (t2 - t1)})
    if rank == 0:
        print(json.dumps({"study": "fig2", "n": 100, "target_inf": 1e-8, "data": "synthetic",
                          "rows": rows}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2211_04299_gb300 import build
    build.build()
    import paper_2211_04299_gb300 as mg
    import mdp_synth

    if args.study == "fig2":
        return run_fig2_study(mg, torch, rank)
    if args.config == 4:
        return run_batch_bench(args, mg, torch, dist, world, rank, local)
    if args.config == 5:
        return run_serve_bench(args, mg, torch, dist, world, rank, local)
    if args.config != 2:
        scale = 1.0 if (args.config != 3 or args.S == S_) else args.S / 1_000_000
        syn = mdp_synth.config(args.config, scale=scale)
        if args.config == 1:
            syn.val = syn.val.astype(np.float32)
    elif args.S == S_:
        syn = mdp_synth.config(2)
    else:
        syn = mdp_synth.dense_dirichlet(args.S, A_, 0.1, GAMMA, mdp_synth.CONFIG_SEEDS[2])
    S, A = syn.S, syn.A
    h = mg.from_synth(syn)
    stream = torch.cuda.Stream()  # not the legacy default stream: see run_batch_bench
    if args.sweep_only:
        return run_sweep_bench(args, mg, torch, syn, h, stream, world, rank, local)
    torch.cuda.set_stream(stream)
    h.set_stream(stream)
    o = mg.opts(tol=TOL, alpha=ALPHA, restart=W_, precision="mixed", forcing_c=args.forcing_c,
                flags=mg.MDP_FLAG_HOST_LOOP if args.host_loop else 0,
                precond_block=args.precond_block)
    v_out = torch.empty(S, dtype=torch.float64, device="cuda")
    pi_out = torch.empty(S, dtype=torch.int32, device="cuda")

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(max(3, args.warmup)):
        mg.ipi_solve(h, o, v_out=v_out, pi_out=pi_out)
    torch.cuda.synchronize()
    barrier()

    h.set_timing(True)
    clocks = Clocks(local)
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    stats = []
    torch.cuda.synchronize()
    barrier()
    ev[0].record(stream)
    for i in range(args.steps):
        _, _, st = mg.ipi_solve(h, o, v_out=v_out, pi_out=pi_out)
        ev[i + 1].record(stream)
        stats.append(st)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    h.set_timing(False)
    elapsed_ms = ev[0].elapsed_time(ev[-1])
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    value = job_rate(args.steps, elapsed_ms / 1000.0, world)
    elapsed_ms = max_over_ranks(elapsed_ms, world)

    ok = all(s["status"] == 0 and s["residual_inf"] <= TOL for s in stats)
    sweeps = sum(s["timed_sweeps"] for s in stats)
    sweep_ms = sum(s["sweep_ms"] for s in stats) / max(1, sweeps)
    # matvecs inside the graph-resident inner loop carry no events: their time comes from
    # the ncu launch list in profiles/, not from this line
    mvs = sum(s["timed_matvecs"] for s in stats)
    mv_ms = sum(s["matvec_ms"] for s in stats) / mvs if mvs else 0.0
    peak, peak_kind = peaks()
    sb = sweep_algorithmic_bytes(syn)
    mb = matvec_algorithmic_bytes(syn)
    sweep_gbs = sb / (sweep_ms * 1e-3) / 1e9 if sweep_ms > 0 else 0.0
    mv_gbs = mb / (mv_ms * 1e-3) / 1e9 if mv_ms > 0 else 0.0
    launches = int(sum(s["launches"] for s in stats))
    per_solve_sweep_ms = sweep_ms * sweeps / args.steps
    per_solve_mv_ms = mv_ms * mvs / args.steps

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup),
        "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "mixed: f32 P/Krylov, double-float (2xf32) values, f64 Givens",
        "data": "synthetic",
        "config": dict(config_fields(args, syn), parallelism=f"replicas x{world}"),
        "converged": ok,
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "per_solve": {"outer": stats[-1]["outer"], "inner": stats[-1]["inner"],
                      "sweeps": stats[-1]["sweeps"], "matvecs": stats[-1]["matvecs"],
                      "sweep_ms": per_solve_sweep_ms},
        "bellman_sweep": {"ms": sweep_ms, "gbs": sweep_gbs, "sweeps_per_s": 1000.0 / sweep_ms if sweep_ms else 0.0,
                          "algorithmic_bytes": sb},
        "pi_matvec": ({"ms": mv_ms, "gbs": mv_gbs, "algorithmic_bytes": mb, "frac": mv_gbs / peak}
                      if mvs else {"ms": None, "algorithmic_bytes": mb,
                                   "note": "launched inside the CUDA graph of the inner loop"}),
        "roofline": {"bound": "hbm",
                     "kernel": sweep_kernel_name(syn),
                     "achieved": sweep_gbs, "peak": peak, "unit": "GB/s",
                     "frac": sweep_gbs / peak, "peak_source": peak_kind,
                     "traffic": sweep_traffic(args, syn)},
        "gpu_launches": launches,
        "clocks": clk,
    }

    def timed_variant(ov, n):
        mg.ipi_solve(h, ov, v_out=v_out, pi_out=pi_out)
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(n):
            _, _, stv = mg.ipi_solve(h, ov, v_out=v_out, pi_out=pi_out)
        b1.record(stream)
        torch.cuda.synchronize()
        return n / (b0.elapsed_time(b1) / 1000.0), stv

    # the banded workload with the two-level preconditioned inner solve (blocks of 512
    # states: measured best of 128..2048), for reference beside the plain Alg. 2 line
    if args.config == 3 and args.precond_block == 0:
        pb = 512
        rate, stp = timed_variant(mg.opts(tol=TOL, alpha=ALPHA, restart=W_, precision="mixed",
                                          precond_block=pb), min(args.steps, 10))
        line["two_level_precond"] = {"precond_block": pb, "value": rate, "unit": "solves/s",
                                     "outer": stp["outer"], "inner": stp["inner"],
                                     "converged": stp["status"] == 0 and stp["residual_inf"] <= TOL}

    # the same solves with the adaptive forcing sequence (Sec. 3: alpha_k -> 0), for reference
    if args.forcing_c == 0.0:
        oa = mg.opts(tol=TOL, alpha=ALPHA, restart=W_, precision="mixed", forcing_c=1.0,
                     precond_block=args.precond_block)
        mg.ipi_solve(h, oa, v_out=v_out, pi_out=pi_out)
        na = min(args.steps, 10)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(na):
            _, _, sta = mg.ipi_solve(h, oa, v_out=v_out, pi_out=pi_out)
        a1.record(stream)
        torch.cuda.synchronize()
        line["adaptive_forcing"] = {"forcing_c": 1.0, "value": na / (a0.elapsed_time(a1) / 1000.0),
                                    "unit": "solves/s", "outer": sta["outer"], "inner": sta["inner"],
                                    "converged": sta["status"] == 0}

    # end to end through the host-pointer API: every step uploads P and g from pinned host
    # memory (mdp_load_*_async), solves, and copies v and pi back to host arrays.  Two handles
    # alternate, so step i+1's upload runs while step i solves.  Each step's time runs from the
    # previous result's arrival on the host to this one's; the rate is 1 / median step.
    if not args.no_e2e:
        g_np = torch.from_numpy(np.ascontiguousarray(syn.g)).pin_memory().numpy()
        h2 = mg.from_synth(syn)
        hs_e2e = [h, h2]
        if syn.kind == "dense":
            pins = [torch.from_numpy(syn.P).pin_memory()]
            load = lambda hh: mg.mdp_load_dense_async(hh, pins[0].numpy(), g_np)
        else:
            pins = [torch.from_numpy(np.ascontiguousarray(syn.col)).pin_memory(),
                    torch.from_numpy(np.ascontiguousarray(syn.val)).pin_memory()]
            load = lambda hh: mg.mdp_load_ell_async(hh, pins[0].numpy(), pins[1].numpy(), g_np)
        in_bytes = sum(int(t.numel() * t.element_size()) for t in pins) + g_np.nbytes
        v_h = np.empty(S)
        pi_h = np.empty(S, np.int32)
        e2e_steps = max(20, args.steps)

        def e2e_run(k):
            t = [time.perf_counter()]
            load(hs_e2e[0])
            for i in range(k):
                if i + 1 < k:
                    load(hs_e2e[(i + 1) % 2])
                mg.ipi_solve(hs_e2e[i % 2], o, v_out=v_h, pi_out=pi_h)
                t.append(time.perf_counter())
            return np.diff(t)

        e2e_run(2)
        torch.cuda.synchronize()
        barrier()
        dts = e2e_run(e2e_steps)
        torch.cuda.synchronize()
        h2.close()
        med = float(np.median(dts))
        line["e2e"] = {"value": job_rate(1, med, world), "unit": "solves/s",
                       "h2d_bytes_per_step": in_bytes,
                       "d2h_bytes_per_step": int(v_h.nbytes + pi_h.nbytes), "steps": e2e_steps,
                       "median_step_ms": 1e3 * med, "mean_rate": e2e_steps / float(np.sum(dts)),
                       "p99_step_ms": float(1e3 * np.percentile(dts, 99))}
        del pins

    # the plain per-instance FP64 form on the same MDP (P widened exactly to FP64); its sweep
    # does one FP64 FMA per entry, so its roofline is the GPU's measured FP64 FMA rate
    if not args.no_fp64:
        line["fp64_plain"] = fp64_plain_leg(args, mg, torch, syn, stream, v_out, pi_out)

    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.S == S_ and args.config == 2:
        import oracle
        m = oracle.from_synth(syn)
        dt, r = oracle_solve_seconds(m)
        line["cpu_baseline"] = {
            "value": 1.0 / dt, "unit": "solves/s", "cores": cores_used(), "cpu": cpu_model(),
            "kind": "oracle",
            "sample": (f"one whole oracle iGMRES-PI solve (Alg. 2, FP64 numpy) of the full "
                       f"workload from V_0 = 0 ({r.outer} outer, {r.inner} inner iterations, "
                       f"{dt:.1f} s)"),
            "one_core": oracle_one_core(2)}
        del m

    # the other benchmark workloads beside the headline: the batch of 256 uneven MDPs (with the
    # plain per-instance FP64 form on the same MDPs) and the banded S = 10^6 MDP
    if args.config == 2 and args.S == S_ and not args.no_extras:
        h.close()
        h = None
        del syn
        line["config4_batched"] = run_batch_bench(args, mg, torch, dist, world, rank, local,
                                                  extra=True)
        line["config3_banded"] = banded_leg(args, mg, torch, stream)
        line["config1_small"] = small_leg(args, mg, torch, stream)
        serve_args = argparse.Namespace(**vars(args))
        serve_args.duration = 10.0
        line["config5_served"] = run_serve_bench(serve_args, mg, torch, dist, world, rank, local,
                                                 extra=True)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if h is not None:
        h.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_sweep_bench(args, mg, torch, syn, h, stream, world, rank, local):
    """Bellman sweeps alone: bellman_apply (mixed arithmetic) at a fixed v, outputs pi and T v
    on the device, no solve around it (so the L2 holds nothing of a Krylov basis)."""
    torch.cuda.set_stream(stream)
    h.set_stream(stream)
    v = torch.from_numpy(np.random.default_rng(7).uniform(0.0, 100.0, syn.S)).cuda()
    Tv = torch.empty(syn.S, dtype=torch.float64, device="cuda")
    pi = torch.empty(syn.S, dtype=torch.int32, device="cuda")
    lib = mg.lib()
    import ctypes as C

    def call():
        rc = lib.bellman_apply_dev(h.ptr, C.c_void_p(v.data_ptr()), C.c_void_p(Tv.data_ptr()),
                                   C.c_void_p(pi.data_ptr()), None, None, mg.MDP_PREC_MIXED)
        assert rc == 0

    for _ in range(max(3, args.warmup)):
        call()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for i in range(args.steps):
        call()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    mean_ms = ev[0].elapsed_time(ev[-1]) / args.steps
    # the sweep writes pi and T v (12 B per state) instead of pi, T v and Phi (16 B)
    sb = sweep_algorithmic_bytes(syn) - 4 * syn.S
    gbs = sb / (mean_ms * 1e-3) / 1e9
    peak, kind = peaks()
    line = {"metric": "Bellman-op HBM GB/s", "value": job_rate(sb / 1e9, mean_ms / 1e3, world),
            "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "mixed: f32 P, double-float (2xf32) sums",
            "data": "synthetic", "step": "one bellman_apply call (v conversion + fused sweep)",
            "config": dict(config_fields(args, syn), parallelism=f"replicas x{world}"),
            "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
            "roofline": {"bound": "hbm", "kernel": sweep_kernel_name(syn), "achieved": gbs,
                         "peak": peak, "unit": "GB/s", "frac": gbs / peak, "peak_source": kind,
                         "traffic": None, "algorithmic_bytes": sb},
            "gpu_launches": 2 * args.steps, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    return 0


def fp64_plain_leg(args, mg, torch, syn, stream, v_out, pi_out, n64=10):
    import mdp_synth
    S, A = syn.S, syn.A
    if syn.kind == "dense":
        syn64 = mdp_synth.SynthMDP(S=S, A=A, gamma=syn.gamma, g=syn.g, kind="dense",
                                   P=syn.P.astype(np.float64))
    else:
        syn64 = mdp_synth.SynthMDP(S=S, A=A, gamma=syn.gamma, g=syn.g, kind="ell",
                                   col=syn.col, val=syn.val.astype(np.float64))
    h64 = mg.from_synth(syn64)
    del syn64
    h64.set_stream(stream)
    o64 = mg.opts(tol=TOL, alpha=ALPHA, restart=W_, precision="fp64",
                  precond_block=args.precond_block)
    mg.ipi_solve(h64, o64, v_out=v_out, pi_out=pi_out)
    torch.cuda.synchronize()
    h64.set_timing(True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(n64 + 1)]
    ev[0].record(stream)
    sts = []
    for i in range(n64):
        _, _, st64 = mg.ipi_solve(h64, o64, v_out=v_out, pi_out=pi_out)
        ev[i + 1].record(stream)
        sts.append(st64)
    torch.cuda.synchronize()
    h64.set_timing(False)
    h64.close()
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(n64)]
    ms64 = ev[0].elapsed_time(ev[-1]) / n64
    sweeps = sum(s["timed_sweeps"] for s in sts)
    sweep_ms = sum(s["sweep_ms"] for s in sts) / max(1, sweeps)
    nnz = S * A * (S if syn.kind == "dense" else syn.k)
    flops = 2.0 * nnz                         # one FMA per transition entry
    bytes64 = nnz * (8 if syn.kind == "dense" else 12) + A * S * 8 + S * 24
    tf = flops / (sweep_ms * 1e-3) / 1e12 if sweep_ms > 0 else 0.0
    fp64_peak = mg.probe_alu("f64")
    hbm_peak, kind = peaks()
    return {"value": 1000.0 / ms64, "unit": "solves/s", "ms_per_solve": ms64, "solves": n64,
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                           "p99": float(np.percentile(step_ms, 99))},
            "outer": sts[-1]["outer"], "inner": sts[-1]["inner"],
            "converged": all(s["status"] == 0 and s["residual_inf"] <= TOL for s in sts),
            "form": "ipi_solve with P widened exactly to FP64, FP64 Krylov vectors and sums",
            "sweep": {"ms": sweep_ms, "algorithmic_flops": flops, "algorithmic_bytes": bytes64,
                      "gbs": bytes64 / (sweep_ms * 1e-3) / 1e9 if sweep_ms > 0 else 0.0},
            "roofline": {"bound": "alu", "kernel": ("sweep_dense_kernel (FP64)" if syn.kind == "dense"
                                                    else "sweep_ell (FP64)"),
                         "achieved": tf, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": tf / fp64_peak if fp64_peak else None,
                         "peak_source": "measured FP64 FMA rate (mdp_probe_alu, this run)",
                         "hbm_frac": (bytes64 / (sweep_ms * 1e-3) / 1e9) / hbm_peak
                         if sweep_ms > 0 else None}}


def small_leg(args, mg, torch, stream, n=20):
    """Config 1 (S = 2000, A = 5, k = 16, gamma = 0.95, FP64 values): the plain FP64 form of
    Alg. 2 as the configuration states it, and the mixed form on the same values rounded to FP32;
    the whole problem lives in L2, so this measures latency, not bandwidth."""
    import mdp_synth
    syn = mdp_synth.config(1)
    out = {"workload": "ELL S=2000, A=5, k=16, gamma=0.95, alpha=0.1, W=30, tol 1e-8", "solves": n}
    for name, prec, data in (("fp64_plain", "fp64", syn.val),
                             ("mixed", "mixed", syn.val.astype(np.float32))):
        h = mg.from_synth(mdp_synth.SynthMDP(S=syn.S, A=syn.A, gamma=syn.gamma, g=syn.g,
                                             kind="ell", col=syn.col, val=data))
        h.set_stream(stream)
        o = mg.opts(tol=TOL, alpha=ALPHA, restart=W_, precision=prec)
        vo = torch.empty(syn.S, dtype=torch.float64, device="cuda")
        po = torch.empty(syn.S, dtype=torch.int32, device="cuda")
        for _ in range(3):
            mg.ipi_solve(h, o, v_out=vo, pi_out=po)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(n + 1)]
        ev[0].record(stream)
        sts = []
        for i in range(n):
            _, _, st = mg.ipi_solve(h, o, v_out=vo, pi_out=po)
            ev[i + 1].record(stream)
            sts.append(st)
        torch.cuda.synchronize()
        step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(n)]
        out[name] = {"value": n / (ev[0].elapsed_time(ev[-1]) / 1000.0), "unit": "solves/s",
                     "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                                    "p99": float(np.percentile(step_ms, 99))},
                     "outer": sts[-1]["outer"], "inner": sts[-1]["inner"],
                     "converged": all(x["status"] == 0 and x["residual_inf"] <= TOL for x in sts)}
        h.close()
    return out


def banded_leg(args, mg, torch, stream):
    """Config 3 (S = 10^6 banded ELL, gamma = 0.999) beside the headline: the two-level
    preconditioned solve (blocks of 512) and plain Alg. 2, with the windowed sweep's HBM
    rate from CUDA events on the handle's stream."""
    import mdp_synth
    syn = mdp_synth.config(3)
    h = mg.from_synth(syn)
    h.set_stream(stream)
    vo = torch.empty(syn.S, dtype=torch.float64, device="cuda")
    po = torch.empty(syn.S, dtype=torch.int32, device="cuda")
    out = {"workload": workload_name(argparse.Namespace(config=3), syn), "S": syn.S, "A": syn.A,
           "k": syn.k, "gamma": syn.gamma}
    peak, kind = peaks()
    for name, pb, n in (("two_level_precond", 512, 10), ("plain", 0, 2)):
        o = mg.opts(tol=TOL, alpha=ALPHA, restart=W_, precision="mixed", precond_block=pb)
        mg.ipi_solve(h, o, v_out=vo, pi_out=po)
        torch.cuda.synchronize()
        h.set_timing(True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(n + 1)]
        ev[0].record(stream)
        sts = []
        for i in range(n):
            _, _, st = mg.ipi_solve(h, o, v_out=vo, pi_out=po)
            ev[i + 1].record(stream)
            sts.append(st)
        torch.cuda.synchronize()
        h.set_timing(False)
        step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(n)]
        sweeps = sum(s["timed_sweeps"] for s in sts)
        sweep_ms = sum(s["sweep_ms"] for s in sts) / max(1, sweeps)
        gbs = sweep_algorithmic_bytes(syn) / (sweep_ms * 1e-3) / 1e9 if sweep_ms > 0 else 0.0
        out[name] = {"precond_block": pb, "value": n / (ev[0].elapsed_time(ev[-1]) / 1000.0),
                     "unit": "solves/s", "solves": n,
                     "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                                    "p99": float(np.percentile(step_ms, 99))},
                     "outer": sts[-1]["outer"], "inner": sts[-1]["inner"],
                     "converged": all(s["status"] == 0 and s["residual_inf"] <= TOL for s in sts)}
        if name == "plain":
            out["bellman_sweep"] = {"kernel": sweep_kernel_name(syn), "ms": sweep_ms, "gbs": gbs,
                                    "algorithmic_bytes": sweep_algorithmic_bytes(syn),
                                    "frac": gbs / peak, "peak": peak, "peak_source": kind,
                                    "traffic": traffic_for("sweep_ell_window_cfg3")}
    h.close()
    return out


if __name__ == "__main__":
    sys.exit(main())

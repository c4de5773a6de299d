#!/usr/bin/env python
"""Benchmark: Crank-Nicolson steps/s of HIF-preconditioned CG on one GB300.

Workload (the configuration the headline metric is quoted on): 2D Fisher-KPP
u_t = div(a grad u) + u(1-u) on (0,1)^2, 1023^2 interior grid (N = 1,046,529),
a = exp(Gaussian random field, correlation length 0.05) with contrast 1e4,
zero Dirichlet data, dt = 1.0, HIF leaf 16x16 (L = 6), eps = 1e-6, PCG to
relative residual 1e-10, u0 = Gaussian bump; synthetic, seeded.

One "step" is one full CN step: right-hand side (stencil + explicit reaction)
and a PCG solve with the HIF inverse applied every iteration.  The headline
path keeps the factor in FP32 (apply in FP32) with FP64 CG; the plain FP64
path is timed beside it.  The factorization (hif_setup) runs once before the
timed region (its time is reported as t_f).  Inputs are resident in HBM when
the timed region starts; the factor streamed every apply (~1 GB) is larger than
the 129 MB L2, so no explicit flush is needed.

Launch: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 (torchrun) every rank runs an independent replica (no collective on
the data path); value = steps of all ranks / max elapsed over ranks.
"""

from __future__ import annotations

import os

# Independent operators stepped together run on one stream each; the driver
# maps streams onto this many hardware work queues (default 8), so more of
# them run concurrently.  Must be set before the CUDA context exists.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import argparse
import hashlib
import json
import math
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CN steps/s at rel-res 1e-10, mixed-prec batched vs FP64 HIF-PCG; p50/p99 latency"
WORKLOAD = ("fisher2d_1023: 2D Fisher-KPP r=u(1-u), 1023^2 interior (N=1046529), "
            "a=exp(GRF corr 0.05) contrast 1e4, dt=1.0, leaf 16 (L=6), eps=1e-6, PCG rel-res 1e-10")
FALLBACK_HBM_GBS = 6800.0


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--eps", type=float, default=1e-6)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-autotune", action="store_true",
                   help="keep the default launch shapes (profiling runs: the first launches are the timed kind)")
    p.add_argument("--n", type=int, default=1024,
                   help="grid intervals per axis (same recipe); 1024 is the benchmark workload, "
                        "smaller values are for profiling captures only")
    p.add_argument("--batched-count", type=int, default=256,
                   help="problems of the batched workload reported beside the headline (0: skip)")
    p.add_argument("--batched-steps", type=int, default=20)
    p.add_argument("--heat3d-steps", type=int, default=50,
                   help="CN steps of the 3D heat 127^3 measurement reported beside the headline (0: skip)")
    p.add_argument("--heat3d-large", type=int, default=0,
                   help="CN steps of the paper's 3D logistic recipe at 255^3 (FP32 factor; setup takes "
                        "minutes; 0: skip)")
    p.add_argument("--heat3d-large-eps", type=float, default=1e-3)
    p.add_argument("--heat3d-large-side", type=int, default=255)
    p.add_argument("--multi-k", type=int, default=16,
                   help="states of the benchmark operator stepped together by cn_step_multi (0: skip)")
    p.add_argument("--serving-ops", type=int, default=16,
                   help="resident operators of the serving measurement (0: skip)")
    p.add_argument("--serving-full", action="store_true",
                   help="also serve the full mix: 48 2D (255^2..2047^2) and 16 3D (63^3..127^3) operators "
                        "under an HBM budget, loads 10..1e4 steps/s (several minutes of setups)")
    p.add_argument("--serving-budget-gb", type=float, default=100.0)
    p.add_argument("--serving-seconds", type=float, default=5.0,
                   help="seconds of arrivals per load point of the full serving mix")
    p.add_argument("--profile-multi", type=int, default=0,
                   help="profiling run: hif_apply_multi (16 columns, six calls) on a 3D operator with "
                        "this many grid intervals per axis (leaf 8, BF16 top levels); prints per-kernel times")
    p.add_argument("--cpu-sample", type=int, default=0, help=argparse.SUPPRESS)
    p.add_argument("--cpu-sample-steps", type=int, default=0, help=argparse.SUPPRESS)
    p.add_argument("--cpu-sample-procs", type=int, default=1, help=argparse.SUPPRESS)
    p.add_argument("--ref-sample-n", type=int, default=0, help=argparse.SUPPRESS)
    return p.parse_args()


# ----------------------------------------------------------------- CPU oracle leg

def oracle_sample(n: int, steps: int, warmup: int, eps: float, procs: int = 1) -> dict:
    """Time the oracle (as it stands) on the same recipe at (n-1)^2.

    Runs in its own process (never touches CUDA) with BLAS limited to one
    thread.  The setup is not timed.  One thread: ``warmup`` steps, then
    ``steps`` timed steps of the trajectory.  All cores (``procs`` > 1): the
    process then forks ``procs`` workers that share the factor and each run
    ``steps`` further steps of the trajectory from the same state, started
    together; their aggregate steps/s is steps x procs / (last end - first
    start).  At n = 1024 the sample is the workload itself (no scaling).
    """
    import numpy as np
    import workloads as W
    from oracle import grid, hif, pcg

    m = 16
    rng = np.random.default_rng(1)
    a = W.lognormal_coefficient(W.grf(rng, n, 2, 0.05), 1e4)
    u = W.gaussian_bump_u0(n, 2)
    A = grid.assemble_A(a, 1.0)
    t0 = time.perf_counter()
    F = hif.factor(A, n, 2, m, eps)
    t_f = time.perf_counter() - t0

    def step(u, its):
        r = grid.reaction(u, 1, 1.0, 1.0)
        g = grid.cn_rhs(a, u, 1.0, r)
        x, it, _, _ = pcg.pcg(A, g.ravel(), lambda v: hif.apply_inverse(F, v), tol=1e-10)
        its.append(it)
        return x.reshape(u.shape)

    its = []
    for _ in range(warmup):
        u = step(u, its)
    its = []
    t0 = time.perf_counter()
    for _ in range(steps):
        u = step(u, its)
    dt = time.perf_counter() - t0
    N_s = (n - 1) ** 2
    N_full = 1023 ** 2
    sps = steps / dt
    out = {"steps_per_s_sample": sps, "steps_per_s_scaled": sps * N_s / N_full, "seconds": dt,
           "steps": steps, "warmup": warmup, "n": n, "N_sample": N_s, "t_f": t_f,
           "iters_per_step": sum(its) / max(1, steps), "cores": 1, "all_cores": None}
    if procs > 1:
        import multiprocessing as mp
        ctx = mp.get_context("fork")  # this process never initialises CUDA
        bar = ctx.Barrier(procs)
        q = ctx.Queue()
        u_start = u

        def worker():
            bar.wait()
            w_its = []
            w0 = time.perf_counter()
            uu = u_start
            for _ in range(steps):
                uu = step(uu, w_its)
            q.put((w0, time.perf_counter(), sum(w_its)))

        ps = [ctx.Process(target=worker) for _ in range(procs)]
        for pr in ps:
            pr.start()
        res = [q.get() for _ in ps]
        for pr in ps:
            pr.join()
        span = max(r[1] for r in res) - min(r[0] for r in res)
        agg = procs * steps / span
        out["all_cores"] = {"steps_per_s_sample": agg, "steps_per_s_scaled": agg * N_s / N_full,
                            "procs": procs, "seconds": span,
                            "iters_per_step": sum(r[2] for r in res) / (procs * steps)}
    return out


def run_oracle_subprocess(n: int, steps: int, warmup: int, eps: float, procs: int = 1) -> dict:
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample", str(n),
           "--cpu-sample-steps", str(steps), "--warmup", str(warmup), "--eps", str(eps),
           "--cpu-sample-procs", str(procs)]
    out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


# ------------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # raw samples (HIFCN_CLOCKS_DIR, else the system temporary directory);
        # the JSON line carries their summary
        out_dir = os.environ.get("HIFCN_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(out_dir, f"clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------------- helpers

def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            with open(p) as f:
                return json.load(f)
        except (OSError, ValueError):
            pass
    return {}


def _find_peak(d: dict, keys) -> float | None:
    for k in keys:
        if k in d and isinstance(d[k], (int, float)):
            return float(d[k])
    for v in d.values():
        if isinstance(v, dict):
            r = _find_peak(v, keys)
            if r is not None:
                return r
    return None


def leaf_kernel_source_hash() -> str:
    """sha256 of the source of the bulk-copy staged leaf kernels (their section
    of apply.cu and the stage size in internal.h): the ncu traffic figures stay
    valid while this is unchanged."""
    csrc = os.path.join(ROOT, "paper_2004_05566_gb300", "csrc")
    src = open(os.path.join(csrc, "apply.cu")).read()
    a = src.index("// ------------------------------------------------------------ TMA-staged cells")
    b = src.index("// Root (Eq. 3_4)", a)
    stage = [l for l in open(os.path.join(csrc, "internal.h")) if "constexpr int kStageBytes" in l]
    return hashlib.sha256((src[a:b] + "".join(stage)).encode()).hexdigest()


def kernel_traffic(name: str) -> float | None:
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current source of the leaf kernels (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        with open(p) as f:
            d = json.load(f)
        if d.get("leaf_kernel_sha256") != leaf_kernel_source_hash():
            return None
        k = d.get("kernels", {}).get(name)
        return float(k["dram_bytes_per_launch_full"]) if k else None
    except (OSError, ValueError, KeyError, TypeError):
        return None


# ----------------------------------------------------------------------- our arm

def max_over_ranks(vals, dist, device):
    """Each timing's maximum over the ranks: the slowest replica sets the job's
    time.  ``dist`` is torch.distributed (or None on one process)."""
    if dist is None:
        return list(vals)
    import torch
    tt = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return tt.tolist()


def job_rate(units_per_rank, t_ms: float, world: int) -> float:
    """Whole-job rate: every rank processed ``units_per_rank`` units and the
    job took ``t_ms`` (already the maximum over the ranks)."""
    return world * units_per_rank / (t_ms / 1e3)


def replica_seed(rank: int) -> int:
    """Seed of rank ``rank``'s coefficient field: every replica solves its own
    independent problem of the same shape (weak scaling, no data exchange)."""
    return 1 + rank


def run_ours(args, rank: int, world: int, dist) -> dict | None:
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2004_05566_gb300.hifcn as H
    import workloads as W

    local = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = W.config_fisher2d_1023(eps=args.eps, seed=replica_seed(rank))
    if args.n != 1024:
        import math as _m
        L = int(round(_m.log2(args.n // 16)))
        rng = np.random.default_rng(replica_seed(rank))
        w = W.Workload(f"fisher2d_{args.n - 1}", 2, args.n, 16, L, 1.0, args.eps,
                       W.lognormal_coefficient(W.grf(rng, args.n, 2, 0.05), 1e4),
                       W.gaussian_bump_u0(args.n, 2), (1, 1.0, 1.0))
    a = torch.from_numpy(w.a_nodes).to(dev)
    stream = torch.cuda.current_stream()

    tuning_s = {}

    def make(precision):
        opt = H.default_options(eps=w.eps, precision=precision, cg_tol=1e-10)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = H.hif_setup(2, w.n, w.leaf, a, w.dt, opt)
        torch.cuda.synchronize()
        tf = time.perf_counter() - t0
        H.hif_set_reaction(h, 1, 1.0, 1.0)
        t1 = time.perf_counter()
        if not args.no_autotune:
            H.hif_autotune(h)  # per-level CTA cut of the apply, by timing (outside the timed steps)
        tuning_s[precision] = round(time.perf_counter() - t1, 3)
        return h, tf

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_steps(h, K, W_, per_step=True, queued=False):
        """K CN steps after W_ warm-up steps: queued (one cn_steps call, no host
        synchronization between steps: the throughput of a time loop) or one
        cn_step call per step (per-step events: the latency of a single call)."""
        u = torch.from_numpy(w.u0.ravel().copy()).to(dev)
        v = torch.empty_like(u)
        its = []
        if queued:
            # GPU warm-up on a scratch copy of the state (about 0.3 s of steps), so that
            # the short timed region does not start on an idle GPU; the timed steps stay
            # steps W+1 .. W+K of the trajectory from u0
            scratch = u.clone()
            H.cn_steps(h, scratch, 300)
            del scratch
        if queued and W_ > 0:
            H.cn_steps(h, u, W_)  # also sizes the step-record buffer before the timed call
        else:
            for _ in range(W_):
                v, it = H.cn_step(h, u, out=v)
                u, v = v, u
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
        barrier()
        lc0 = H.hif_launch_count()
        evs[0].record(stream)
        if queued:
            its = H.cn_steps(h, u, K)
            per_step = False
        else:
            for k in range(K):
                v, it = H.cn_step(h, u, out=v)
                u, v = v, u
                its.append(it)
                if per_step:
                    evs[k + 1].record(stream)
        if not per_step:
            evs[K].record(stream)
        torch.cuda.synchronize()
        lc1 = H.hif_launch_count()
        barrier()
        total = evs[0].elapsed_time(evs[K])
        lat = [evs[k].elapsed_time(evs[k + 1]) for k in range(K)] if per_step else []
        return total, lat, its, lc1 - lc0, u

    # ---- mixed precision (headline)
    h32, tf32 = make(H.HIF_FP32)
    info32 = H.hif_query(h32)
    clocks = ClockSampler(local)
    clocks.start()
    t_ms, _, its, launches, _ = timed_steps(h32, args.steps, args.warmup, queued=True)
    clk = clocks.stop()
    # ---- per-call latency: one cn_step call per step
    K_lat = min(args.steps, 300)
    _, lat, _, _, _ = timed_steps(h32, K_lat, 0, per_step=True)
    # ---- instrumented pass of the same steps: per-kernel device time
    H.hif_stats_enable(h32, True)
    t_ms_stats, _, _, _, _ = timed_steps(h32, args.steps, 0, per_step=False)
    stats = H.hif_stats_read(h32)
    H.hif_stats_enable(h32, False)
    # ---- end to end through host buffers (pinned), same metric
    K_e2e = args.steps
    uh = torch.from_numpy(w.u0.ravel().copy()).pin_memory()
    oh = torch.empty_like(uh).pin_memory()
    ud = torch.empty(w.N, dtype=torch.float64, device=dev)
    vd = torch.empty_like(ud)
    for _ in range(args.warmup):
        ud.copy_(uh, non_blocking=True)
        H.cn_step(h32, ud, out=vd)
        oh.copy_(vd, non_blocking=True)
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K_e2e):
        ud.copy_(uh, non_blocking=True)
        H.cn_step(h32, ud, out=vd)
        oh.copy_(vd, non_blocking=True)
        uh, oh = oh, uh
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = e0.elapsed_time(e1)
    h32.close()
    # ---- plain FP64 path on the same GPU
    h64, tf64 = make(H.HIF_FP64)
    t64_ms, _, its64, _, _ = timed_steps(h64, max(1, args.steps // 2), args.warmup, queued=True)
    _, lat64, _, _, _ = timed_steps(h64, min(max(1, args.steps // 2), 300), 0, per_step=True)
    info64 = H.hif_query(h64)
    h64.close()

    # ---- k states of the benchmark operator at once (BF16 top levels on the tensor cores)
    multi2d = None
    if args.multi_k > 0:
        hb, _ = make(H.HIF_FP32_BF16TOP)
        u_m = torch.from_numpy(w.u0.ravel().copy()).to(dev)
        H.cn_steps(hb, u_m, args.warmup)
        multi2d = multi_vs_single(H, torch, hb, u_m, args.multi_k, reps=2)
        hb.close()

    # ---- batched workload: many independent operators, overlapped vs one at a time
    batched = None
    if args.batched_count > 0:
        batched = run_batched(args, dev, H, W, np, torch)

    # ---- 3D heat 127^3 (leaf 8, eps 1e-4, face + edge skeletonization)
    heat3d = None
    if args.heat3d_steps > 0:
        heat3d = run_heat3d(args, dev, H, W, np, torch)

    heat3d_large = None
    if args.heat3d_large > 0:
        heat3d_large = run_heat3d_large(args, dev, H, W, np, torch)

    # ---- serving: open-loop Poisson step requests over resident operators
    serving = None
    if args.serving_ops > 0:
        serving = run_serving(args, local, W, np)
    serving_full = run_serving_full(args, local, W, np) if args.serving_full else None

    # ---- max over ranks
    t_ms, e2e_ms, t64_ms = max_over_ranks([t_ms, e2e_ms, t64_ms], dist, dev)
    if rank != 0:
        return None

    K = args.steps
    value = job_rate(K, t_ms, world)
    lat_sorted = sorted(lat)

    def pct(xs, q):
        if not xs:
            return None
        i = min(len(xs) - 1, max(0, int(math.ceil(q / 100.0 * len(xs))) - 1))
        return xs[i]

    # ---- roofline of the dominant kernel: the factor-streaming cell kernel
    # with the most time (the HBM-bound steps; the upper levels are latency
    # bound and are listed in apply_kernels)
    peak, peak_note = hbm_peak()
    roof = roofline_of(stats, peak, peak_note)
    if roof:
        roof["traffic"] = kernel_traffic(roof["kernel"])
    kt = sorted(stats, key=lambda s: -s["ms"])
    apply_ms = sum(s["ms"] for s in stats)

    # ---- CPU oracle baseline (rank 0, one GPU only): the workload itself
    # (1023^2, no scaling), setup untimed, one thread and all host cores
    cpu = None
    if world == 1 and not args.no_cpu_baseline and args.n == 1024:
        try:
            procs = host_cores()
            r = run_oracle_subprocess(1024, 2, 1, args.eps, procs=procs)
            ac = r.get("all_cores") or {}
            cpu = {"value": round(r["steps_per_s_sample"], 6), "unit": "steps/s", "cores": 1,
                   "kind": "oracle",
                   "sample": (f"oracle (Python/NumPy/SciPy FP64, 1 BLAS thread) on the workload "
                              f"itself, 1023^2 (N={r['N_sample']}), no scaling: setup untimed "
                              f"({r['t_f']:.1f} s), {r['warmup']} warm-up step, {r['steps']} timed "
                              f"CN steps ({r['seconds']:.1f} s, {r['iters_per_step']:.2f} PCG it/step)"),
                   "ms_per_cg_iteration": round(1e3 * r["seconds"] / max(1e-9, r["steps"] * r["iters_per_step"]), 1),
                   "all_cores": ({"value": round(ac["steps_per_s_sample"], 6), "unit": "steps/s",
                                  "cores": ac["procs"],
                                  "sample": (f"{ac['procs']} oracle processes forked after the setup, "
                                             f"one BLAS thread each, each running {r['steps']} further "
                                             f"steps of the trajectory; aggregate steps/s over "
                                             f"{ac['seconds']:.1f} s ({ac['iters_per_step']:.2f} PCG it/step)")}
                                 if ac else None),
                   "cpu": cpu_model(), "host_cores": procs}
        except Exception as exc:  # report, never fake
            cpu = {"value": None, "unit": "steps/s", "cores": 1, "kind": "oracle",
                   "sample": f"failed: {str(exc)[:200]}"}

    iters_per_step = sum(its) / len(its)
    line = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "steps/s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": round(t_ms / K, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if args.n == 1024 else f"same recipe at {args.n - 1}^2 (profiling)",
                   "precision": "factor FP32 (apply FP32), CG FP64",
                   "global_batch": world, "parallelism": f"replicas x{world}" if world > 1 else "single",
                   "l2": "inputs larger than L2: the ~1 GB FP32 factor streams every apply"},
        "api": "cn_steps: the K timed steps queued in one call (no host synchronization between "
               "steps; per-step iteration counts read back at the end)",
        "latency_ms": {"p50": pct(lat_sorted, 50), "p99": pct(lat_sorted, 99),
                       "api": f"cn_step, one call per step ({len(lat)} steps, per-step CUDA events)"},
        "iters_per_step": round(iters_per_step, 3),
        "iters_per_step_note": (f"steps {args.warmup + 1}..{args.warmup + K} of the trajectory from u0 "
                                f"(the early steps after the bump initial condition take more PCG "
                                f"iterations; steps/s depends on which steps are timed)"),
        "cg_iters_per_s": round(job_rate(sum(its), t_ms, world), 2),
        "ms_per_cg_iteration": round(t_ms / max(1, sum(its)), 4),
        "t_f_s": {"fp32": round(tf32, 3), "fp64": round(tf64, 3)},
        "autotune_s": {"fp32": tuning_s.get(H.HIF_FP32), "fp64": tuning_s.get(H.HIF_FP64)},
        "fp64_path": {"value": round(job_rate(max(1, K // 2), t64_ms, world), 3), "unit": "steps/s",
                      "ms_per_step": round(t64_ms / max(1, K // 2), 4),
                      "iters_per_step": round(sum(its64) / len(its64), 3),
                      "p50_ms": pct(sorted(lat64), 50), "p99_ms": pct(sorted(lat64), 99)},
        "factor": {"entries": info32["factor_entries"], "apply_bytes_fp32": info32["apply_bytes"],
                   "apply_bytes_fp64": info64["apply_bytes"], "root": info32["root_size"],
                   "device_bytes": info32["device_bytes"]},
        "e2e": {"value": round(job_rate(K_e2e, e2e_ms, world), 3), "unit": "steps/s",
                "h2d_bytes_per_step": 8 * w.N, "d2h_bytes_per_step": 8 * w.N,
                "api": "cn_step via the C ABI, u^k copied from pinned host memory and u^{k+1} read back every step"},
        "gpu_launches": int(launches),
        "roofline": roof,
        "apply_kernels": [{"name": s["name"], "launches": s["launches"],
                           "ms": round(s["ms"], 3), "GBps": round(s["bytes"] / (s["ms"] / 1e3) / 1e9, 1)
                           if s["ms"] > 0 else None} for s in kt[:8]],
        "apply_share_of_step": round(apply_ms / t_ms_stats, 3) if t_ms_stats else None,
        "clocks": clk,
        "cpu_baseline": cpu,
        "multi_rhs_2d": multi2d,
        "batched": batched,
        "heat3d": heat3d,
        "heat3d_large": heat3d_large,
        "serving": serving,
        "serving_full": serving_full,
    }
    return line


def run_serving(args, device_index, W, np) -> dict:
    """Serving: resident 2D reaction-diffusion operators (side log-uniform in
    255..1023, leaf 16, lognormal a with contrast 1e3, dt in [1e-2, 1], eps 1e-6,
    FP32 factors); open-loop Poisson arrivals of CN-step requests, the operator
    of each request drawn uniformly; the server batches concurrent requests
    (continuous batching).  Reports latency (arrival to result) percentiles
    and achieved throughput per offered load."""
    import random
    import paper_2004_05566_gb300.serve as S

    rng = np.random.default_rng(2000)
    srv = S.CNServer(hbm_budget_bytes=64 << 30, device=device_index)
    ids = []
    for i in range(args.serving_ops):
        side = math.exp(rng.uniform(math.log(255), math.log(1023)))
        n, m, L = W.snap_side(side, leafs=(16,))
        a = W.lognormal_coefficient(W.grf(rng, n, 2, 0.05), 1e3)
        dt = math.exp(rng.uniform(math.log(1e-2), math.log(1.0)))
        srv.register(i, S.OperatorSpec(2, n, m, a, dt, 1e-6, W.gaussian_bump_u0(n, 2), (1, 1.0, 1.0)))
        ids.append(i)
    t0 = time.perf_counter()
    for f in [srv.submit(i) for i in ids]:  # admission (factorization) of every operator
        f.result()
    t_admit = time.perf_counter() - t0
    loads = []
    rnd = random.Random(7)
    for lam in (10.0, 30.0, 100.0, 300.0, 1000.0, 3000.0, 10000.0):
        nreq = int(min(max(20.0, 2.0 * lam), 3000))
        arrivals = np.cumsum(rng.exponential(1.0 / lam, size=nreq))
        futs = []
        start = time.perf_counter()
        for t_a in arrivals:
            delay = start + t_a - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            futs.append(srv.submit(rnd.choice(ids)))
        res = [f.result() for f in futs]
        end = time.perf_counter()
        lat = sorted(r.latency_s * 1e3 for r in res)
        pct = lambda q: lat[min(len(lat) - 1, max(0, int(math.ceil(q / 100 * len(lat))) - 1))]
        loads.append({"offered_steps_per_s": lam, "requests": nreq,
                      "achieved_steps_per_s": round(nreq / (end - start), 1),
                      "p50_ms": round(pct(50), 3), "p99_ms": round(pct(99), 3),
                      "mean_batch": round(sum(r.batch_size for r in res) / len(res), 2)})
    sides = sorted(srv._ops[i].spec.n - 1 for i in ids)
    out = {"operators": len(ids), "sides_min_max": [sides[0], sides[-1]],
           "admission_s": round(t_admit, 2), "resident_bytes": srv.resident_bytes(),
           "loads": loads,
           "scheduler": "step-level continuous batching over cn_step_batched (serve.CNServer)"}
    srv.close()
    return out


def roofline_of(stats, peak, peak_note, traffic=None) -> dict | None:
    """Achieved HBM bandwidth of the factor-streaming cell kernel with the most
    device time: algorithmic bytes per launch / average launch duration."""
    cell = [x for x in stats if x["name"].startswith("cell_")]
    dom = max(cell or stats, key=lambda x: x["ms"]) if stats else None
    if not dom or dom["launches"] == 0 or dom["ms"] <= 0:
        return None
    per_launch_bytes = dom["bytes"] / dom["launches"]
    per_launch_s = dom["ms"] / dom["launches"] / 1e3
    achieved = per_launch_bytes / per_launch_s / 1e9
    return {"bound": "hbm", "kernel": dom["name"], "achieved": round(achieved, 1),
            "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
            "traffic": traffic, "algorithmic_bytes_per_launch": per_launch_bytes,
            "avg_launch_us": round(per_launch_s * 1e6, 2), "peak_source": peak_note,
            "timing": "CUDA events around each launch on its stream, instrumented pass of "
                      "the same steps"}


def hbm_peak() -> tuple:
    peak = _find_peak(measured_peaks(), ("hbm_gbs", "hbm_GBs", "copy_gbs"))
    return (peak, "measured") if peak else (FALLBACK_HBM_GBS, "fallback")


def multi_vs_single(H, torch, h, u, k: int, reps: int = 2) -> dict:
    """k states of one operator stepped together (cn_step_multi: one
    multi-column apply per PCG iteration, BF16 top levels on the tensor cores)
    against the same k steps taken one cn_step at a time on the same handle.
    States: u scaled by 1 + 0.05 c, c < k; CUDA events around the calls."""
    stream = torch.cuda.current_stream()
    U = torch.stack([u * (1.0 + 0.05 * c) for c in range(k)]).contiguous()
    V = torch.empty_like(U)
    H.cn_step_multi(h, U, out=V)  # warm-up: work space, graphs of the single path
    H.cn_step(h, U[0].contiguous())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    its_m = []
    for _ in range(reps):
        _, it = H.cn_step_multi(h, U, out=V)
        its_m += it
    e1.record(stream)
    torch.cuda.synchronize()
    t_m = e0.elapsed_time(e1) / 1e3
    rows = [U[c].contiguous() for c in range(k)]
    out = torch.empty_like(rows[0])
    its_s = []
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        for c in range(k):
            _, it = H.cn_step(h, rows[c], out=out)
            its_s.append(it)
    e1.record(stream)
    torch.cuda.synchronize()
    t_s = e0.elapsed_time(e1) / 1e3
    n = reps * k
    return {"k": k, "steps": n, "multi_steps_per_s": round(n / t_m, 3),
            "single_steps_per_s": round(n / t_s, 3), "speedup": round(t_s / t_m, 3),
            "multi_iters_per_step": round(sum(its_m) / n, 3),
            "single_iters_per_step": round(sum(its_s) / n, 3),
            "api": "cn_step_multi (k states, one hif_apply_multi per PCG iteration) vs k cn_step calls"}


def _pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    return xs[min(len(xs) - 1, max(0, int(math.ceil(q / 100 * len(xs))) - 1))]


def run_serving_full(args, device_index, W, np) -> dict:
    """Serving the full mix (48 2D operators of 255^2..2047^2 and 16 3D of
    63^3..127^3, FP32 factors with the FP64 copy released, FP64 CG) under an
    HBM budget smaller than the mix: evicted operators are offloaded to host
    memory and reloaded.  2D and 3D operators are served in separate lanes
    (threads and streams), so the 3D steps do not hold back the 2D ones.
    Open-loop Poisson arrivals at 10 .. 1e4 steps/s, the operator of each
    request drawn uniformly; latency = arrival to result ready."""
    import random
    import paper_2004_05566_gb300.serve as S

    budget = int(args.serving_budget_gb * (1 << 30))
    srv = S.CNServer(hbm_budget_bytes=budget, device=device_index, lanes=[0])
    ws = W.config_serving()
    ids = list(range(len(ws)))
    for i, w in zip(ids, ws):
        srv.register(i, S.OperatorSpec(w.dim, w.n, w.leaf, w.a_nodes, w.dt, w.eps, w.u0, w.reaction,
                                       lane=1 if w.dim == 3 else 0))
    t0 = time.perf_counter()
    setup_s = {}
    for i in ids:  # admission (factorization) of every operator, one at a time
        t1 = time.perf_counter()
        srv.submit(i).result()
        setup_s[i] = time.perf_counter() - t1
        print(f"serving_full: admitted {i} ({ws[i].dim}D n={ws[i].n} leaf={ws[i].leaf}) in "
              f"{setup_s[i]:.2f} s, resident {srv.resident_bytes() / 2**30:.1f} GiB, "
              f"evictions {srv.evictions}", file=sys.stderr, flush=True)
    t_admit = time.perf_counter() - t0
    rng = np.random.default_rng(2100)
    rnd = random.Random(11)
    loads = []
    for lam in (10.0, 30.0, 100.0, 300.0, 1000.0, 3000.0, 10000.0):
        nreq = int(min(max(20, lam * args.serving_seconds), 5000))
        print(f"serving_full: load {lam} steps/s, {nreq} requests", file=sys.stderr, flush=True)
        arrivals = np.cumsum(rng.exponential(1.0 / lam, size=nreq))
        ev0, rl0 = srv.evictions, srv.reloads
        futs, dims = [], []
        start = time.perf_counter()
        for t_a in arrivals:
            delay = start + t_a - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            oid = rnd.choice(ids)
            futs.append(srv.submit(oid))
            dims.append(ws[oid].dim)
        res = [f.result() for f in futs]
        end = time.perf_counter()
        lat = [r.latency_s * 1e3 for r in res]
        l2 = [x for x, d in zip(lat, dims) if d == 2]
        l3 = [x for x, d in zip(lat, dims) if d == 3]
        loads.append({"offered_steps_per_s": lam, "requests": nreq,
                      "achieved_steps_per_s": round(nreq / (end - start), 1),
                      "p50_ms": round(_pct(lat, 50), 3), "p99_ms": round(_pct(lat, 99), 3),
                      "p50_ms_2d": round(_pct(l2, 50), 3) if l2 else None,
                      "p99_ms_2d": round(_pct(l2, 99), 3) if l2 else None,
                      "p50_ms_3d": round(_pct(l3, 50), 3) if l3 else None,
                      "p99_ms_3d": round(_pct(l3, 99), 3) if l3 else None,
                      "mean_batch": round(sum(r.batch_size for r in res) / len(res), 2),
                      "evictions": srv.evictions - ev0, "reloads": srv.reloads - rl0})
    sizes = [(w.dim, w.n - 1) for w in ws]
    out = {"operators": len(ws), "sizes": {"2d": sorted(s for d, s in sizes if d == 2),
                                           "3d": sorted(s for d, s in sizes if d == 3)},
           "hbm_budget_gb": args.serving_budget_gb, "admission_s": round(t_admit, 1),
           "setup_s_max": round(max(setup_s.values()), 2),
           "resident_bytes_end": srv.resident_bytes(), "evictions_total": srv.evictions,
           "reloads_total": srv.reloads, "seconds_per_load": args.serving_seconds, "loads": loads,
           "scheduler": "two lanes (2D, 3D) of step-level continuous batching over cn_step_batched; "
                        "eviction offloads the factor to host memory (hif_offload), re-admission "
                        "reloads it (hif_reload); FP64 factor copy released after the setup"}
    srv.close()
    return out


def run_heat3d(args, dev, H, W, np, torch) -> dict:
    """3D heat equation on 127^3 (leaf 8, L = 4, eps 1e-4, dt 0.1, lognormal a with
    contrast 1e3, smooth random u0, face + edge skeletonization, FP64 CG): GPU
    setup time, then `heat3d_steps` CN steps queued in one cn_steps call, with
    the factor in FP32 and the top levels in BF16 (the configuration's
    precision) and with the factor in FP32 throughout.  Each leg reports the
    CN-system residual ||A u^{k+1} - g|| / ||g|| of its last step, with
    g = (I + dt/2 M) u^k = 2 u^k - A u^k (no reaction) evaluated by the
    library's stencil, and the roofline of its dominant cell kernel."""
    w = W.config_heat3d_127()
    a = torch.from_numpy(w.a_nodes).to(dev)
    stream = torch.cuda.current_stream()
    peak, peak_note = hbm_peak()
    legs = {}
    for name, prec in (("fp32_bf16top", H.HIF_FP32_BF16TOP), ("fp32", H.HIF_FP32)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = H.hif_setup(3, w.n, w.leaf, a, w.dt,
                        H.default_options(eps=w.eps, precision=prec, cg_tol=1e-10))
        torch.cuda.synchronize()
        t_setup = time.perf_counter() - t0
        info = H.hif_query(h)
        u = torch.from_numpy(w.u0.ravel().copy()).to(dev)
        H.cn_steps(h, u, 2)  # warm-up: graph capture, step-record buffer
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        its = H.cn_steps(h, u, args.heat3d_steps - 1)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        k_steps = args.heat3d_steps - 1
        # last step, checked: g = 2 u^k - A u^k, residual of A u^{k+1} = g
        uk = u.clone()
        u1, it_last = H.cn_step(h, uk)
        g = 2.0 * uk - H.hif_matvec(h, uk)
        res = float((H.hif_matvec(h, u1) - g).norm() / g.norm())
        multi = multi_vs_single(H, torch, h, u1, 16, reps=1) if prec == H.HIF_FP32_BF16TOP else None
        # instrumented pass: per-kernel device time of a few steps
        H.hif_stats_enable(h, True)
        H.cn_steps(h, u1.clone(), 3)
        stats = H.hif_stats_read(h)
        H.hif_stats_enable(h, False)
        h.close()
        legs[name] = {"steps": k_steps, "steps_per_s": round(k_steps / t, 3),
                      "ms_per_step": round(1e3 * t / k_steps, 3),
                      "iters_per_step": round(sum(its) / k_steps, 3),
                      "ms_per_cg_iteration": round(1e3 * t / max(1, sum(its)), 4),
                      "last_step_cn_residual": res, "last_step_iters": it_last,
                      "setup_s": round(t_setup, 2), "apply_bytes": info["apply_bytes"],
                      "root": info["root_size"], "device_bytes": info["device_bytes"],
                      "roofline": roofline_of(stats, peak, peak_note)}
        if multi:
            legs[name]["multi_rhs"] = multi
    return {"workload": "heat3d_127: 3D heat, 127^3 interior (N=2048383), lognormal a contrast 1e3, "
                        "dt=0.1, leaf 8 (L=4), eps=1e-4, face+edge skeletonization, FP64 CG, "
                        "PCG rel-res 1e-10",
            "steps": args.heat3d_steps,
            "api": "cn_steps (steps queued in one call) after a 2-step warm-up; the last step by "
                   "cn_step with its residual checked",
            **legs}


def run_heat3d_large(args, dev, H, W, np, torch) -> dict:
    """The paper's 3D logistic recipe (Sec. 3, Example 2 in 3D: 200 bumps on
    [0.05, 20], the scaled Gaussian u0, k1 = 1, k2 = 10, dt = 0.1 h) at 255^3
    (leaf 8, L = 5) with the factor in FP32 and PCG to the paper's tolerance
    1e-12: setup time and memory, then `heat3d_large` CN steps one call each,
    with their iteration counts (the tables print n_i = 6 at eps 1e-3 and 3 at
    1e-6) and the CN-system residual of every step, ||A u^{k+1} - g|| / ||g||
    with g = 2 u^k - A u^k + dt k1 u^k (1 - u^k / k2) from the library's
    stencil."""
    side = args.heat3d_large_side
    w = W.paper_heat3d(side + 1, 8, args.heat3d_large_eps, seed=0, logistic=True)
    a = torch.from_numpy(w.a_nodes).to(dev)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    t0 = time.perf_counter()
    h = H.hif_setup(3, w.n, w.leaf, a, w.dt,
                    H.default_options(eps=w.eps, precision=H.HIF_FP32, cg_tol=w.tol))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    del a
    info = H.hif_query(h)
    print(f"[bench] {side}^3 setup {t_setup:.1f} s: {info}", file=sys.stderr, flush=True)
    _, k1, k2 = w.reaction
    H.hif_set_reaction(h, 1, k1, k2)
    u = torch.from_numpy(w.u0.ravel().copy()).to(dev)
    its, res, ms = [], [], []
    for _ in range(args.heat3d_large):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        u1, it = H.cn_step(h, u)
        torch.cuda.synchronize()
        ms.append(1e3 * (time.perf_counter() - t1))
        g = 2.0 * u - H.hif_matvec(h, u) + w.dt * k1 * u * (1.0 - u / k2)
        res.append(float((H.hif_matvec(h, u1) - g).norm() / g.norm()))
        its.append(it)
        u = u1
        print(f"[bench] {side}^3 step {len(its)}: {it} iterations, residual {res[-1]:.3g}, "
              f"{ms[-1]:.1f} ms", file=sys.stderr, flush=True)
    fp64_kept = True
    try:
        H.hif_apply(h, u, precision=H.HIF_FP64)
    except H.HifError:
        fp64_kept = False
    h.close()
    return {"workload": f"paper 3D logistic recipe, {side}^3 interior (N={w.N}), leaf 8 (L={w.levels}), "
                        f"eps={w.eps:g}, face+edge skeletonization, FP32 factor, FP64 CG, PCG rel-res "
                        f"{w.tol:g}",
            "setup_s": round(t_setup, 1), "root": info["root_size"],
            "factor_entries": info["factor_entries"], "device_bytes": info["device_bytes"],
            "device_free_before_setup": free0, "fp64_factor_kept": fp64_kept,
            "apply_bytes": info["apply_bytes"], "iters": its,
            "mean_iters": round(float(np.mean(its)), 2) if its else None,
            "printed_n_i": {1e-3: 6, 1e-6: 3}.get(w.eps),
            "cn_residuals": res, "ms_per_step": [round(x, 1) for x in ms]}


def run_batched(args, dev, H, W, np, torch) -> dict:
    """Batched workload: independent 2D reaction-diffusion problems of uneven
    sizes (side log-uniform in 63..511, snapped to 2^L m - 1), each with its own
    lognormal coefficient (contrast 1e3) and dt in [1e-2, 1], eps 1e-6, FP32
    factors; every problem takes `batched_steps` CN steps.  Timed twice on the
    same handles: all problems per cn_step_batched call (overlapped on the GPU)
    and one cn_step at a time."""
    probs = W.config_batched(count=args.batched_count)
    hs, us = [], []
    t0 = time.perf_counter()
    for w in probs:
        a = torch.from_numpy(w.a_nodes).to(dev)
        h = H.hif_setup(2, w.n, w.leaf, a, w.dt,
                        H.default_options(eps=w.eps, precision=H.HIF_FP32, cg_tol=1e-10))
        H.hif_set_reaction(h, 1, 1.0, 1.0)
        hs.append(h)
        us.append(torch.from_numpy(w.u0.ravel().copy()).to(dev))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    n_dof = sum(w.N for w in probs)
    # warm-up (graph capture of every handle)
    outs, _ = H.cn_step_batched(hs, us)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    buf_a = outs
    buf_b = [torch.empty_like(u) for u in us]
    src, dst = list(us), buf_a
    torch.cuda.synchronize()
    e0.record(stream)
    its = 0
    for _ in range(args.batched_steps):
        _, it = H.cn_step_batched(hs, src, outs=dst)
        its += sum(it)
        src, dst = dst, (buf_b if dst is buf_a else buf_a)
    e1.record(stream)
    torch.cuda.synchronize()
    t_b = e0.elapsed_time(e1) / 1e3
    src, dst = list(us), buf_a
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.batched_steps):
        for h, u, o in zip(hs, src, dst):
            H.cn_step(h, u, out=o)
        src, dst = dst, (buf_b if dst is buf_a else buf_a)
    e1.record(stream)
    torch.cuda.synchronize()
    t_s = e0.elapsed_time(e1) / 1e3
    total = args.batched_steps * len(hs)
    for h in hs:
        h.close()
    sides = sorted(w.n - 1 for w in probs)
    return {"problems": len(hs), "steps_each": args.batched_steps, "total_dofs": n_dof,
            "sides_min_med_max": [sides[0], sides[len(sides) // 2], sides[-1]],
            "setup_s": round(t_setup, 2),
            "batched_steps_per_s": round(total / t_b, 1),
            "sequential_steps_per_s": round(total / t_s, 1),
            "speedup": round(t_s / t_b, 3),
            "iters_per_step": round(its / total, 3),
            "api": "cn_step_batched (per-handle streams, captured PCG graphs) vs cn_step in a loop"}


# ----------------------------------------------------------------- reference arm

def run_reference(args) -> dict:
    """The oracle, as it stands, on the host cores: K timed CN steps of the
    workload itself (1023^2, one thread, setup untimed) when K <= 30, else of
    the same recipe at 255^2 with steps/s scaled by N (so the run stays within
    minutes).  Warm-up capped at one step (the oracle has no caches to warm)."""
    full = args.steps <= 30 and args.ref_sample_n in (0, 1024)
    n = 1024 if full else (args.ref_sample_n or 256)
    r = run_oracle_subprocess(n, args.steps, min(args.warmup, 1), args.eps)
    v = r["steps_per_s_sample"] if full else r["steps_per_s_scaled"]
    sample = (f"each step = one oracle CN step of the workload itself (1023^2, N={r['N_sample']}, "
              f"no scaling), one thread, setup untimed ({r['t_f']:.1f} s), "
              f"{r['iters_per_step']:.2f} PCG it/step" if full else
              f"each step = one oracle CN step of the same recipe at {n - 1}^2 "
              f"(N={r['N_sample']}); steps/s scaled by N to 1023^2; measured "
              f"{r['steps_per_s_sample']:.3f} steps/s on the sample, {r['iters_per_step']:.2f} PCG it/step")
    return {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": "steps/s",
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "ms_per_step": round(1e3 / v, 3),
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if full else f"same recipe at {n - 1}^2 (scaled by N)"},
            "cpu_baseline": {"value": round(v, 6), "unit": "steps/s", "cores": 1, "kind": "oracle",
                             "sample": sample, "cpu": cpu_model()},
            "e2e": {"value": round(v, 6), "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def profile_multi(n: int) -> dict:
    """hif_apply_multi on a 3D n^3-interval operator (leaf 8, eps 1e-4, lognormal
    a, HIF_FP32_BF16TOP), 16 columns: three warm-up calls, then three calls with
    per-kernel statistics (a capture target for ncu on the tensor-core kernel)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2004_05566_gb300.hifcn as H
    import workloads as W
    w = W.small_variable_2d(n=n, m=8, dim=3, eps=1e-4, contrast=1e3, dt=0.1, corr_len=0.05, seed=2)
    h = H.hif_setup(3, n, 8, torch.from_numpy(w.a_nodes).cuda(), w.dt,
                    H.default_options(eps=1e-4, precision=H.HIF_FP32_BF16TOP, cg_tol=1e-10))
    X = torch.from_numpy(np.random.default_rng(0).standard_normal((16, w.N))).cuda()
    for _ in range(3):
        H.hif_apply_multi(h, X)
    torch.cuda.synchronize()
    H.hif_stats_enable(h, True)
    for _ in range(3):
        H.hif_apply_multi(h, X)
    st = H.hif_stats_read(h)
    h.close()
    return {"profile": "hif_apply_multi", "n": n, "k": 16,
            "kernels_us_per_launch": {s["name"]: round(1e3 * s["ms"] / s["launches"], 1)
                                      for s in sorted(st, key=lambda s: -s["ms"])}}


def main():
    args = _args()
    if args.profile_multi:
        print(json.dumps(profile_multi(args.profile_multi)))
        return
    if args.cpu_sample:
        r = oracle_sample(args.cpu_sample, args.cpu_sample_steps, args.warmup, args.eps,
                          args.cpu_sample_procs)
        print(json.dumps(r))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", rank)))
        tdist.init_process_group("nccl")
        dist = tdist
    line = run_ours(args, rank, world, dist)
    if line is not None:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Benchmark of the CC split integrator hot path (arXiv:1407.7105).

One step = one outer step evolve_cc(all, dt) of the 16384-body Plummer
sphere (N-body units, eta = 0.03, dt = 1/256, eps = 0): the tau + edge +
union-find split, segmentation, kicks, drifts and the recursion into every
component, all in libcc.so's kernels.  The metric counts interactions =
tau pairs (n(n-1)/2 per split set) + cross-component kick pairs, per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--form fp64|mixed]
  python bench.py --impl reference ...   (the FP64 CPU oracle, bounded sample)

Multi-GPU: the integrator does not shard (one system per GPU); N ranks run
N independent replicas (different seeds) and value sums their work over the
slowest rank's time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CC interactions/s, mixed vs FP64 at |dE/E|≤1e-6; % of FP64/FP32 roofline"
UNIT = "interactions/s"
N_BODY = 16384
DT = 1.0 / 256
ETA = 0.03
# algorithmic FP64 operations per unordered pair (sqrt and division count 1)
TAU_FLOPS = 47   # Eq. tauij as evaluated: 3 sqrt, 6 div, 38 add/sub/mul
KICK_FLOPS = 28  # one pair force applied to both bodies (Eqs. kickij/kickji)


WORKLOADS = {
    # the configuration the metric is quoted on (default)
    "plummer": dict(dt=1.0 / 256, kepler=False,
                    name="Plummer N={n}, equal masses, N-body units, eps=0, eta=0.03, outer step dt=1/256 "
                         "(one evolve_cc step per bench step)"),
    "fractal": dict(dt=1.0 / 256, kepler=False,
                    name="box fractal N={n}, D=1.6, Salpeter IMF 0.1-100 (total M=1), Q=0.3, N-body units, "
                         "eps=0, eta=0.03, outer step dt=1/256"),
    "binaries": dict(dt=1.0 / 256, kepler=True,
                     name="Plummer N={n} with 50% of bodies in binaries (a log-uniform 1e-5..1e-2, thermal e, "
                          "q~U(0.1,1]), CC_KEPLER, eta=0.03, outer step dt=1/256"),
    "systems": dict(dt=1.0 / 64, kepler=False,
                    name="{nsys} independent systems (triples, or Plummer clumps of logU[3,512] bodies), "
                         "each in its own N-body units, eta=0.03, outer step dt=1/64"),
}


def combine_ranks(maxes, sums, device):
    """Across the ranks of the process group (if any): the max of each value
    in `maxes` (times: the slowest rank) and the sum of each in `sums` (work
    of all replicas).  Without a process group the values come back as they
    are."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return [float(x) for x in maxes], [float(x) for x in sums]
    tt = torch.tensor([float(x) for x in maxes], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    w = torch.tensor([float(x) for x in sums], device=device, dtype=torch.float64)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return tt.tolist(), w.tolist()


def workload_name(n=N_BODY, workload="plummer", nsys=4096):
    return WORKLOADS[workload]["name"].format(n=n, nsys=nsys)


def make_workload(args, seed, dev=None):
    """Seeded synthetic state (m, x3, v3, sys_off or None) of the workload."""
    from paper_1407_7105_gb300 import ics
    w = args.workload
    if w == "plummer":
        return (*ics.plummer(args.n, seed=seed), None)
    if w == "binaries":
        return (*ics.plummer_with_binaries(args.n, seed=seed), None)
    if w == "systems":
        return ics.small_systems(args.nsys, seed=seed)
    # fractal: the potential energy of the unscaled cluster is summed on the
    # GPU by the library's energy diagnostic (velocities zero: E = W)
    from paper_1407_7105_gb300 import cc
    import torch
    x0, v0 = ics.box_fractal_raw(args.n, seed=seed)
    m = ics.salpeter_masses(args.n, seed, 9100)
    x0, v0 = ics._com_frame(m, x0, v0)
    ctx = cc.Context(torch.tensor(m, device=dev), torch.tensor(x0, device=dev),
                     torch.zeros((3, args.n), dtype=torch.float64, device=dev))
    W, _, _ = ctx.energy()
    ctx.close()
    x3, v3 = ics.scale_to_nbody_units(m, x0, v0, Q=0.3, exact=False, W=W)
    return m, x3, v3, None


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ peaks
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------------ oracle
def oracle_sample(m, x, v, reps: int = 1):
    """The FP64 CPU oracle on a bounded sample of the workload: the top-level
    split_cc of all N bodies at h = dt followed by the level's
    drift-kick-drift (no recursion).  Returns (interactions, seconds)."""
    from oracle import oracle as O
    s = O.State(m, x, v)
    p = O.params(eta=ETA, dt=DT)
    inter = 0
    t0 = time.perf_counter()
    for _ in range(reps):
        st = O.Stats()
        lab, _ = O.components(s, p, DT, stats=st)
        ids = np.arange(s.n, dtype=np.int32)
        O.drift(s, ids, lab, 0.5 * DT, stats=st)
        O.kick(s, p, ids, lab, DT, stats=st)
        O.drift(s, ids, lab, 0.5 * DT, stats=st)
        inter += st.tau_pairs + st.kick_pairs
    return inter, time.perf_counter() - t0


def run_reference(args, rank, world):
    from oracle import oracle as O
    O.build()
    if rank != 0:
        return 0
    from paper_1407_7105_gb300 import ics
    m, x, v = ics.plummer(N_BODY, seed=args.seed)
    for _ in range(args.warmup):
        oracle_sample(m, x, v)
    inter, sec = 0, 0.0
    for _ in range(args.steps):
        i, s = oracle_sample(m, x, v)
        inter += i
        sec += s
    val = inter / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(), "form": "oracle"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "per step: top-level split_cc (BFS, lazy tau) of all 16384 bodies at h=dt "
                                   "plus that level's drift-kick-drift, single thread"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def run_gpu(args, rank, world):
    import torch
    import torch.distributed as dist

    from paper_1407_7105_gb300 import build, cc, ics

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    seed = args.seed + rank
    m, x, v, sys_off = make_workload(args, seed, dev)
    N = int(m.shape[0])
    W = WORKLOADS[args.workload]
    DTW = W["dt"]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "plummer":
        from oracle import oracle as O
        O.build()
        inter, sec = oracle_sample(m, x, v)
        cpu = {"value": inter / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "top-level split_cc (BFS, lazy tau) of all 16384 bodies at h=dt plus that level's "
                         "drift-kick-drift, single thread, same initial state"}

    stream = torch.cuda.current_stream(dev)
    f64_peak, f32_peak = cc.probe_peaks()
    l2_flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)  # 256 MB > L2
    dm, dx, dv = (torch.tensor(a, device=dev) for a in (m, x, v))

    def make_ctx(form):
        prec = cc.PREC_MIXED if form == "mixed" else cc.PREC_FP64
        ctx = cc.Context(dm, dx, dv, dt=DTW, eta=ETA, precision=prec, h_fp64=args.h_fp64 * DTW,
                         s_small=args.s_small, kepler=int(W["kepler"]))
        if sys_off is not None:
            ctx.set_systems(sys_off)
        return ctx

    def time_form(form, steps, warmup, clocks_too):
        ctx = make_ctx(form)
        E0, _, _ = ctx.energy()
        t = 0.0
        for _ in range(warmup):
            t += DTW
            ctx.evolve(t)
        torch.cuda.synchronize()
        st0 = ctx.stats()
        ctx.set_timing(True)
        sampler = ClockSampler(local) if clocks_too else None
        if dist.is_initialized():
            dist.barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        torch.cuda.nvtx.range_push("timed_region")
        total_ms = 0.0
        step_ms = []
        for _ in range(steps):
            l2_flush.fill_(1)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            t += DTW
            ctx.evolve(t)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            total_ms += step_ms[-1]
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        clocks = sampler.stop() if sampler else None
        st1 = ctx.stats()
        tm = ctx.timing()
        tuning = ctx.tuning()
        ctx.set_timing(False)
        E1, _, _ = ctx.energy()
        res = {"ctx": ctx, "t": t, "total_ms": total_ms, "step_ms": step_ms, "clocks": clocks, "timing": tm,
               "tuning": tuning,
               "inter": (st1["tau_pairs"] - st0["tau_pairs"]) + (st1["kick_pairs"] - st0["kick_pairs"]),
               "launches": st1["launches"] - st0["launches"],
               "tau_fp64": st1["tau_fp64"] - st0["tau_fp64"], "tau_pairs": st1["tau_pairs"] - st0["tau_pairs"],
               "tau_evaluated": st1["tau_evaluated"] - st0["tau_evaluated"],
               "kick_pairs": st1["kick_pairs"] - st0["kick_pairs"],
               "edges": st1["edges"] - st0["edges"],
               "dE": (E1 - E0) / abs(E0)}
        return res

    head = time_form(args.form, args.steps, args.warmup, True)
    other_form = "fp64" if args.form == "mixed" else "mixed"
    other = None if args.single_form else time_form(other_form, max(1, min(args.steps, 3)), 1, False)
    if other:
        other["ctx"].close()
    ctx, t = head["ctx"], head["t"]
    total_ms, clocks, tm, inter, launches = (head["total_ms"], head["clocks"], head["timing"], head["inter"],
                                             head["launches"])

    # end to end through the C ABI with host buffers (pinned)
    hm = torch.empty(N, dtype=torch.float64).pin_memory()
    hx = torch.empty(3, N, dtype=torch.float64).pin_memory()
    hv = torch.empty(3, N, dtype=torch.float64).pin_memory()
    ctx.get_state(hm, hx, hv)
    e2e_steps = max(1, min(args.steps, 3))
    st2 = ctx.stats()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.set_state(t, hm, hx, hv)
        t += DTW
        ctx.evolve(t)
        ctx.get_state(None, hx, hv, alloc=False)
    torch.cuda.synchronize()
    e2e_sec = time.perf_counter() - w0
    st3 = ctx.stats()
    e2e_inter = (st3["tau_pairs"] - st2["tau_pairs"]) + (st3["kick_pairs"] - st2["kick_pairs"])

    # max over ranks, sums of work
    (sec, e2e_sec), (inter, e2e_inter) = combine_ranks([total_ms * 1e-3, e2e_sec], [inter, e2e_inter], dev)
    value = inter / sec

    # roofline of the dominant pairwise kernel (measured live above)
    fp32 = args.form == "mixed"
    if tm["tau_ms"] >= tm["kick_ms"]:
        kname, kms, kl, flops = "tau", tm["tau_ms"], tm["tau_launches"], TAU_FLOPS * tm["tau_pairs"]
    else:
        kname, kms, kl, flops = "kick", tm["kick_ms"], tm["kick_launches"], KICK_FLOPS * tm["kick_pairs"]
    kname = ("k_tau_mixed" if kname == "tau" else "k_kick_mixed") if fp32 else \
            ("k_tau_hook" if kname == "tau" else "k_kick64")
    achieved = flops / (kms * 1e-3) / 1e12 if kms > 0 else None
    peak = (f32_peak if fp32 else f64_peak) / 1e12
    roof = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if achieved else None, "traffic": None,
            "peak_source": ("FP32" if fp32 else "FP64") + " FMA throughput measured by cc_probe_peaks on this GPU",
            "algorithmic_flops_per_pair": TAU_FLOPS if kname.startswith("k_tau") else KICK_FLOPS,
            "kernel_ms_per_step": kms / args.steps, "launches_per_step": kl / args.steps,
            "tau_ms_per_step": tm["tau_ms"] / args.steps, "kick_ms_per_step": tm["kick_ms"] / args.steps,
            "small_kernel_ms_per_step": tm["small_ms"] / args.steps,
            "fp64_peak_tflops": f64_peak / 1e12, "fp32_peak_tflops": f32_peak / 1e12}
    other_line = None
    if other:
        other_line = {"form": other_form, "value": other["inter"] / (other["total_ms"] * 1e-3),
                      "ms_per_step": other["total_ms"] / max(1, min(args.steps, 3)), "dE_over_E": other["dE"],
                      "tau_ms_per_step": other["timing"]["tau_ms"] / max(1, min(args.steps, 3)),
                      "kick_ms_per_step": other["timing"]["kick_ms"] / max(1, min(args.steps, 3)),
                      "small_kernel_ms_per_step": other["timing"]["small_ms"] / max(1, min(args.steps, 3))}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "step_ms": [round(x, 4) for x in head["step_ms"]], "higher_is_better": True,
            # launch shapes the online tuner picked, per kernel and size bin
            # (pairs in [2^bin, 2^(bin+1))): [kernel, bin, [shape, column
            # slices] picked, us per 1e6 pairs of each variant]
            "autotune": [[e["kernel"], e["bin"],
                          [e["shape"][e["best"]], e["slices"][e["best"]]] if e["best"] >= 0 else None,
                          e["us_per_mpair"]] for e in head["tuning"]],
            "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64" if fp32 else "f64", "data": "synthetic",
            "config": {"workload": workload_name(N, args.workload, args.nsys), "form": args.form, "h_fp64": f"{args.h_fp64}*dt",
                       "s_small": args.s_small,
                       "l2": "flushed (256 MB write) before each step",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "e2e": {"value": e2e_inter / e2e_sec, "unit": UNIT, "h2d_bytes_per_step": 7 * N * 8,
                    "d2h_bytes_per_step": 6 * N * 8, "steps": e2e_steps},
            "gpu_launches": launches,
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "dE_over_E": head["dE"],
            "tau_fp64_fraction": head["tau_fp64"] / max(1, head["tau_pairs"]),
            "interactions_per_step": inter / args.steps / world,
            # interactions = tau pairs decided by the splits + kick pairs; a
            # first-half split decides its pairs from the tau values its
            # parent split computed, so fewer pairs are evaluated than decided
            "tau_pairs_per_step": head["tau_pairs"] / args.steps,
            "tau_pairs_evaluated_per_step": head["tau_evaluated"] / args.steps,
            "kick_pairs_per_step": head["kick_pairs"] / args.steps,
            "edges_per_step": head["edges"] / args.steps,
            "other_form": other_line,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_accuracy(args):
    """The accuracy gate of the metric: both forms integrate the workload to
    t = 1 (256 outer steps) from the same state; |dE/E|, momentum drift and
    time to solution are reported per form (JSON lines, not the bench line)."""
    import torch

    from paper_1407_7105_gb300 import build, cc, ics
    build.build()
    m, x, v = ics.plummer(args.n, seed=args.seed)
    dev = torch.device("cuda", 0)
    dm, dx, dv = (torch.tensor(a, device=dev) for a in (m, x, v))
    steps = int(round(args.t_end / DT))
    for form, hf in (("mixed", 0.0), ("mixed", args.h_fp64 or 1.0 / 16), ("fp64", 0.0)):
        prec = cc.PREC_MIXED if form == "mixed" else cc.PREC_FP64
        ctx = cc.Context(dm, dx, dv, dt=DT, eta=ETA, precision=prec, h_fp64=hf * DT)
        E0, P0, L0 = ctx.energy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.evolve(steps * DT)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        E1, P1, L1 = ctx.energy()
        st = ctx.stats()
        ctx.close()
        inter = st["tau_pairs"] + st["kick_pairs"]
        print(json.dumps({"accuracy": True, "form": form, "h_fp64": f"{hf}*dt", "t_end": steps * DT,
                          "steps": steps, "seconds": sec, "interactions": inter, "interactions_per_s": inter / sec,
                          "dE_over_E": (E1 - E0) / abs(E0), "dP": float(np.abs(P1 - P0).max()),
                          "dL": float(np.abs(L1 - L0).max()), "max_depth": st["max_depth_seen"],
                          "tau_fp64_fraction": st["tau_fp64"] / max(1, st["tau_pairs"])}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cc", choices=["cc", "reference"])
    ap.add_argument("--form", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--h-fp64", type=float, default=0.0,
                    help="mixed form: sets split at h < h_fp64*dt take FP64 forces")
    ap.add_argument("--single-form", action="store_true", help="skip timing the other form")
    ap.add_argument("--s-small", type=int, default=32,
                    help="components of at most this many bodies run in the small-component kernel (0: none)")
    ap.add_argument("--accuracy", action="store_true", help="integrate both forms to --t-end and report dE/E")
    ap.add_argument("--t-end", type=float, default=1.0)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--n", type=int, default=None, help="bodies (default per workload)")
    ap.add_argument("--workload", default="plummer", choices=sorted(WORKLOADS),
                    help="plummer (the metric's configuration), fractal, binaries, systems")
    ap.add_argument("--nsys", type=int, default=4096, help="systems of the 'systems' workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.n is None:
        args.n = {"plummer": N_BODY, "fractal": 65536, "binaries": 32768, "systems": 0}[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.accuracy:
        return run_accuracy(args)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        return run_gpu(args, rank, world)
    finally:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())

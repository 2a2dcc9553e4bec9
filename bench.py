"""Benchmark of the CC split integrator hot path (arXiv:1407.7105).

One step = one outer step evolve_cc(all, dt) of the 16384-body Plummer
sphere (N-body units, eta = 0.03, dt = 1/256, eps = 0): the tau + edge +
union-find split, segmentation, kicks, drifts and the recursion into every
component, all in libcc.so's kernels.  The metric counts interactions =
tau pairs (n(n-1)/2 per split set) + cross-component kick pairs, per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--form fp64|mixed]
  python bench.py --impl reference ...   (the FP64 CPU oracle: full outer steps,
                                          row loops on all host cores)

The bench line also carries (N = 1, rank 0) the metric's accuracy gate (both
forms to t = 1: |dE/E|, momentum drift, time to solution), the mixed kick's
force error against FP64 on the bench state, and the other configurations
(65536-body fractal, 32768-body binaries, 4096 systems) in both forms.

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
# algorithmic operations per unordered pair (sqrt and division count 1)
TAU_FLOPS = 47   # Eq. tauij as evaluated: 3 sqrt, 6 div, 38 add/sub/mul
KICK_FLOPS = 25  # one pair force applied to both bodies (Eqs. kickij/kickji): the difference (3), r^2 (6),
                 # r^-3 (sqrt, mul, div: 3), the weights (2 x 2) and the two 3-vector updates (2 x 3); the
                 # mixed form's row kick evaluates each pair from both sides, which is not credited (the
                 # FP64 kick evaluates each unordered pair once, k_pair_forces, and sums rows, k_kick64)
# DRAM bytes (read + write) per launch of the pair kernels, averaged over the
# launches of one step in an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum): profiles/launches_plummer16384_mixed.md (mixed form)
# and profiles/k_tau_hook_k_kick64_plummer16384_fp64.md (FP64 form; the FP64
# kick's two kernels per kick call: profiles/launches_plummer16384_fp64.md)
KERNEL_TRAFFIC = {"k_kick_mixed": 391e3, "k_tau_mixed": 850e3, "k_pair_forces+k_kick64": 3.07e9, "k_tau_hook": 616e3}


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
def oracle_step(s, steps: int = 1):
    """The FP64 CPU oracle on the workload itself: `steps` full outer steps
    evolve_cc(all, dt) of the state s (recursion included), its row loops
    on every host core (OpenMP; results identical to one thread).  Returns
    (interactions, seconds, threads): interactions = tau pairs decided +
    kick pairs, the GPU's count."""
    from oracle import oracle as O
    p = O.params(eta=ETA, dt=DT)
    nthreads = O.threads(0)
    st = O.Stats()
    t0 = time.perf_counter()
    O.evolve(s, p, steps, stats=st)
    sec = time.perf_counter() - t0
    return st.tau_pairs + st.kick_pairs, sec, nthreads


ORACLE_SAMPLE = ("per step: one full outer step evolve_cc(all, dt=1/256) of the 16384-body sphere, recursion "
                 "included (the GPU's step), FP64 oracle with its row loops on all host cores (OpenMP, results "
                 "identical to one thread)")


def run_reference(args, rank, world):
    from oracle import oracle as O
    if rank != 0:
        return 0
    O.build()
    from paper_1407_7105_gb300 import ics
    m, x, v = ics.plummer(N_BODY, seed=args.seed)
    s = O.State(m, x, v)
    for _ in range(args.warmup):
        oracle_step(s)
    inter, sec, cores = 0, 0.0, 1
    for _ in range(args.steps):
        i, dt_s, cores = oracle_step(s)
        inter += i
        sec += dt_s
    val = inter / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(), "form": "oracle"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": ORACLE_SAMPLE,
                         "same_config": True},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def _ctx(cc, dm, dx, dv, sys_off, workload, form, h_fp64_rel, s_small, split=0):
    """A context of the given form (and split: 0 CC, 1 HOLD) on a
    device-resident state."""
    W = WORKLOADS[workload]
    prec = cc.PREC_MIXED if form == "mixed" else cc.PREC_FP64
    ctx = cc.Context(dm, dx, dv, dt=W["dt"], eta=ETA, precision=prec, h_fp64=h_fp64_rel * W["dt"],
                     s_small=s_small, kepler=int(W["kepler"]), split=split)
    if sys_off is not None:
        ctx.set_systems(sys_off)
    return ctx


def time_steps(ctx, dt, t, steps, stream, l2_flush=None):
    """`steps` outer steps, each bracketed by CUDA events on the library's
    stream (L2 flushed before each when l2_flush is given).  Returns
    (t, total ms, per-step ms, stats before, stats after)."""
    import torch
    st0 = ctx.stats()
    total, per = 0.0, []
    for _ in range(steps):
        if l2_flush is not None:
            l2_flush.fill_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t += dt
        ctx.evolve(t)
        e1.record(stream)
        e1.synchronize()
        per.append(e0.elapsed_time(e1))
        total += per[-1]
    return t, total, per, st0, ctx.stats()


def _work(st0, st1):
    d = {k: st1[k] - st0[k] for k in ("tau_pairs", "kick_pairs", "tau_evaluated", "tau_fp64", "edges", "launches",
                                      "splits")}
    d["interactions"] = d["tau_pairs"] + d["kick_pairs"]
    d["interactions_evaluated"] = d["tau_evaluated"] + d["kick_pairs"]
    return d


def accuracy_gate(cc, dm, dx, dv, t_end, h_fp64_rel):
    """The metric's accuracy gate on the bench workload: each form integrates
    the same state to t_end (one N-body time = 256 outer steps); |dE/E|,
    momentum and angular-momentum drift and the time to solution."""
    import torch
    out = []
    steps = int(round(t_end / DT))
    for form, hf in (("mixed", 0.0), ("mixed", h_fp64_rel), ("fp64", 0.0)):
        ctx = _ctx(cc, dm, dx, dv, None, "plummer", form, hf, cc.SMALL_AUTO)
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
        out.append({"form": form, "h_fp64": f"{hf}*dt", "t_end": steps * DT, "steps": steps, "seconds": round(sec, 4),
                    "interactions_per_s": inter / sec, "dE_over_E": (E1 - E0) / abs(E0),
                    "dP": float(np.abs(P1 - P0).max()), "dL": float(np.abs(L1 - L0).max()),
                    "max_depth": st["max_depth_seen"], "gate_1e-6": abs((E1 - E0) / E0) <= 1e-6})
    return out


def force_error(cc, m, x, v, dev):
    """Relative error of the mixed kick's accelerations against the FP64
    kick on the bench state (every pair: all labels distinct), per body."""
    import torch
    n = m.shape[0]
    labels = np.arange(n, dtype=np.int32)
    acc = {}
    for form in ("fp64", "mixed"):
        dm, dx, dv = (torch.tensor(a, device=dev) for a in (m, x, v))
        ctx = _ctx(cc, dm, dx, dv, None, "plummer", form, 0.0, cc.SMALL_AUTO)
        ctx.kick(labels, 1.0)
        _, _, _, gv = ctx.get_state()
        ctx.close()
        acc[form] = gv - v
    err = np.linalg.norm(acc["mixed"] - acc["fp64"], axis=0) / np.linalg.norm(acc["fp64"], axis=0)
    return {"median": float(np.median(err)), "p99": float(np.quantile(err, 0.99)), "max": float(err.max()),
            "state": "bench initial state, all N(N-1)/2 pairs"}


def other_configs(cc, dev, stream, seed, l2_flush):
    """The other configurations, both forms, a few steps each: ms per step,
    interactions/s (decided and evaluated tau pairs) and |dE/E| over the
    steps.  The binaries also run the mixed form with FP64 forces below
    h_fp64 = dt/64 (close subsystems)."""
    import argparse as _ap
    import torch
    out = {}
    plan = (("fractal", 65536, [("mixed", 0.0), ("fp64", 0.0)]),
            ("binaries", 32768, [("mixed", 0.0), ("mixed", 1.0 / 64), ("fp64", 0.0)]),
            ("systems", 0, [("mixed", 0.0), ("fp64", 0.0)]),
            # the HOLD method (Sec. 2.1) on the same kernels and the bench's
            # own workload: the paper's comparison of the two splits
            ("hold", N_BODY, [("mixed", 0.0), ("fp64", 0.0)]),
            # the OK split (Sec. 4.2, FP64 only) on the bench's workload
            ("ok", N_BODY, [("fp64", 0.0)]))
    for wl, n, forms in plan:
        a = _ap.Namespace(workload=wl, n=n, nsys=4096)
        if wl in ("hold", "ok"):
            a.workload = "plummer"
        m, x, v, sys_off = make_workload(a, seed, dev)
        dm, dx, dv = (torch.tensor(q, device=dev) for q in (m, x, v))
        rows = []
        wname = a.workload
        for form, hf in forms:
            split = {"hold": cc.SPLIT_HOLD, "ok": cc.SPLIT_OK}.get(wl, cc.SPLIT_CC)
            ctx = _ctx(cc, dm, dx, dv, sys_off, wname, form, hf, cc.SMALL_AUTO, split=split)
            E0, _, _ = ctx.energy()
            dtw = WORKLOADS[wname]["dt"]
            w0 = time.perf_counter()
            t = dtw
            ctx.evolve(t)  # warm-up step (allocations, tuner trials)
            torch.cuda.synchronize()
            warm_s = time.perf_counter() - w0
            steps = 3 if warm_s < 0.5 else (2 if warm_s < 3.0 else 1)
            t, ms, per, st0, st1 = time_steps(ctx, dtw, t, steps, stream, l2_flush)
            E1, _, _ = ctx.energy()
            ctx.close()
            w = _work(st0, st1)
            rows.append({"form": form, "h_fp64": f"{hf}*dt", "steps": steps, "ms_per_step": ms / steps,
                         "interactions_per_s": w["interactions"] / (ms * 1e-3),
                         "evaluated_interactions_per_s": w["interactions_evaluated"] / (ms * 1e-3),
                         "tau_pairs_per_step": w["tau_pairs"] / steps, "kick_pairs_per_step": w["kick_pairs"] / steps,
                         "dE_over_E": (E1 - E0) / abs(E0), "steps_for_dE": steps + 1})
        name = workload_name(m.shape[0], wname, 4096)
        if wl == "hold":
            name = "HOLD split (Sec. 2.1) on: " + name
        if wl == "ok":
            name = "OK split (Sec. 4.2) on: " + name
        out[wl] = {"workload": name, "n": int(m.shape[0]), "forms": rows}
    return out


# ------------------------------------------------------------------ GPU arm
def run_gpu(args, rank, world):
    import torch
    import torch.distributed as dist

    from paper_1407_7105_gb300 import build, cc

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    seed = args.seed + rank
    m, x, v, sys_off = make_workload(args, seed, dev)
    N = int(m.shape[0])
    DTW = WORKLOADS[args.workload]["dt"]
    extras = rank == 0 and world == 1

    cpu = None
    if extras and not args.no_cpu_baseline and args.workload == "plummer":
        from oracle import oracle as O
        O.build()
        inter, sec, cores = oracle_step(O.State(m, x, v))
        cpu = {"value": inter / sec, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": ORACLE_SAMPLE
               .replace("per step: one", "one") + ", same initial state", "seconds": round(sec, 3),
               "same_config": True}

    stream = torch.cuda.current_stream(dev)
    f64_peak, f32_peak = cc.probe_peaks()
    l2_flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)  # 256 MB > L2
    dm, dx, dv = (torch.tensor(a, device=dev) for a in (m, x, v))

    def time_form(form, steps, warmup, clocks_too):
        ctx = _ctx(cc, dm, dx, dv, sys_off, args.workload, form, args.h_fp64, args.s_small,
                   split={"cc": cc.SPLIT_CC, "hold": cc.SPLIT_HOLD, "ok": cc.SPLIT_OK}[args.split])
        E0, _, _ = ctx.energy()
        t = 0.0
        for _ in range(warmup):
            t += DTW
            ctx.evolve(t)
        torch.cuda.synchronize()
        ctx.set_timing(True)
        sampler = ClockSampler(local) if clocks_too else None
        if dist.is_initialized():
            dist.barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        torch.cuda.nvtx.range_push("timed_region")
        t, total_ms, step_ms, st0, st1 = time_steps(ctx, DTW, t, steps, stream, l2_flush)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        clocks = sampler.stop() if sampler else None
        tm = ctx.timing()
        tuning = ctx.tuning()
        ctx.set_timing(False)
        E1, _, _ = ctx.energy()
        return {"ctx": ctx, "t": t, "total_ms": total_ms, "step_ms": step_ms, "clocks": clocks, "timing": tm,
                "tuning": tuning, "work": _work(st0, st1), "dE": (E1 - E0) / abs(E0)}

    head = time_form(args.form, args.steps, args.warmup, True)
    other_form = "fp64" if args.form == "mixed" else "mixed"
    osteps = max(1, min(args.steps, 3))
    # (the OK split has the FP64 form only)
    other = None if (args.single_form or args.split == "ok") else time_form(other_form, osteps, 1, False)
    if other:
        other["ctx"].close()
    ctx, t = head["ctx"], head["t"]
    total_ms, clocks, tm, work = head["total_ms"], head["clocks"], head["timing"], head["work"]

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
    ctx.close()

    # max over ranks, sums of work
    inter = work["interactions"]
    (sec, e2e_sec), (inter, e2e_inter, inter_eval) = combine_ranks(
        [total_ms * 1e-3, e2e_sec], [inter, e2e_inter, work["interactions_evaluated"]], dev)
    value = inter / sec

    # roofline of the dominant pairwise kernel (measured live above) and of
    # the small-component kernel (tau pairs it evaluated + kick pairs)
    fp32 = args.form == "mixed"
    if tm["tau_ms"] >= tm["kick_ms"]:
        kname, kms, kl, flops = "tau", tm["tau_ms"], tm["tau_launches"], TAU_FLOPS * tm["tau_pairs"]
    else:
        kname, kms, kl, flops = "kick", tm["kick_ms"], tm["kick_launches"], KICK_FLOPS * tm["kick_pairs"]
    # both forms' splits run the certified FP32 tau kernel; the kicks are the
    # form's own (FP32 in the mixed form, FP64 in the FP64 form)
    fp32 = fp32 or kname == "tau"
    kname = "k_tau_mixed" if kname == "tau" else ("k_kick_mixed" if fp32 else "k_pair_forces+k_kick64")
    achieved = flops / (kms * 1e-3) / 1e12 if kms > 0 else None
    peak = (f32_peak if fp32 else f64_peak) / 1e12
    small_flops = TAU_FLOPS * tm["small_tau_evaluated"] + KICK_FLOPS * tm["small_kick_pairs"]
    small_ach = small_flops / (tm["small_ms"] * 1e-3) / 1e12 if tm["small_ms"] > 0 else None
    roof = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if achieved else None, "traffic": KERNEL_TRAFFIC.get(kname),
            "traffic_note": ("bytes per kick call (both kernels)" if "+" in kname else "bytes per launch")
                            + " from an ncu capture of the same kernel (profiles/)",
            "peak_source": ("FP32" if fp32 else "FP64") + " FMA throughput measured by cc_probe_peaks on this GPU "
                           "(MEASURED_PEAKS.json has no FP32/FP64 figure)",
            "algorithmic_flops_per_pair": TAU_FLOPS if kname.startswith("k_tau") else KICK_FLOPS,
            "kernel_ms_per_step": kms / args.steps, "launches_per_step": kl / args.steps,
            "tau_ms_per_step": tm["tau_ms"] / args.steps, "kick_ms_per_step": tm["kick_ms"] / args.steps,
            "tau_tflops": TAU_FLOPS * tm["tau_pairs"] / (tm["tau_ms"] * 1e-3) / 1e12 if tm["tau_ms"] > 0 else None,
            "kick_tflops": KICK_FLOPS * tm["kick_pairs"] / (tm["kick_ms"] * 1e-3) / 1e12 if tm["kick_ms"] else None,
            "small_kernel": {"kernel": ("k_batch" if args.s_small > 32 or (args.s_small < 0 and args.form == "mixed")
                                        else "k_small"), "ms_per_step": tm["small_ms"] / args.steps,
                             "launches_per_step": tm["small_launches"] / args.steps,
                             "tau_pairs_evaluated_per_step": tm["small_tau_evaluated"] / args.steps,
                             "kick_pairs_per_step": tm["small_kick_pairs"] / args.steps,
                             "achieved": small_ach, "frac": small_ach / peak if small_ach else None,
                             "bound": "latency (one warp per component of <= 32 bodies, one CTA above)"},
            "fp64_peak_tflops": f64_peak / 1e12, "fp32_peak_tflops": f32_peak / 1e12}
    other_line = None
    if other:
        ow = other["work"]
        other_line = {"form": other_form, "value": ow["interactions"] / (other["total_ms"] * 1e-3),
                      "evaluated_value": ow["interactions_evaluated"] / (other["total_ms"] * 1e-3),
                      "ms_per_step": other["total_ms"] / osteps, "dE_over_E": other["dE"],
                      "tau_ms_per_step": other["timing"]["tau_ms"] / osteps,
                      "kick_ms_per_step": other["timing"]["kick_ms"] / osteps,
                      "small_kernel_ms_per_step": other["timing"]["small_ms"] / osteps,
                      "tau_tflops": TAU_FLOPS * other["timing"]["tau_pairs"] / (other["timing"]["tau_ms"] * 1e-3) / 1e12
                      if other["timing"]["tau_ms"] > 0 else None,
                      "kick_tflops": KICK_FLOPS * other["timing"]["kick_pairs"] / (other["timing"]["kick_ms"] * 1e-3)
                      / 1e12 if other["timing"]["kick_ms"] > 0 else None}

    accuracy = forces = configs = None
    if extras and args.workload == "plummer" and not args.no_extras:
        forces = force_error(cc, m, x, v, dev)
        accuracy = accuracy_gate(cc, dm, dx, dv, args.t_end, args.h_fp64_gate)
        configs = other_configs(cc, dev, stream, args.seed, l2_flush)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "step_ms": [round(q, 4) for q in head["step_ms"]], "higher_is_better": True,
            # the same steps counting only the tau pairs a kernel evaluated
            # (first-half splits decide theirs from the parent split's values)
            "evaluated_value": inter_eval / sec,
            # launch shapes the online tuner picked, per kernel and size bin
            # (pairs in [2^bin, 2^(bin+1))): [kernel, bin, [shape, column
            # slices] picked, us per 1e6 pairs of each variant]
            "autotune": [[e["kernel"], e["bin"],
                          [e["shape"][e["best"]], e["slices"][e["best"]]] if e["best"] >= 0 else None,
                          e["us_per_mpair"]] for e in head["tuning"]],
            "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64" if args.form == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(N, args.workload, args.nsys), "form": args.form,
                       "split": args.split,
                       "h_fp64": f"{args.h_fp64}*dt", "s_small": args.s_small,
                       "l2": "flushed (256 MB write) before each step",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "e2e": {"value": e2e_inter / e2e_sec, "unit": UNIT, "h2d_bytes_per_step": 7 * N * 8,
                    "d2h_bytes_per_step": 6 * N * 8, "steps": e2e_steps},
            "gpu_launches": work["launches"],
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "dE_over_E": head["dE"],
            "tau_fp64_fraction": work["tau_fp64"] / max(1, work["tau_pairs"]),
            "interactions_per_step": inter / args.steps / world,
            # interactions = tau pairs decided by the splits + kick pairs; a
            # first-half split decides its pairs from the tau values its
            # parent split computed, so fewer pairs are evaluated than decided
            "tau_pairs_per_step": work["tau_pairs"] / args.steps,
            "tau_pairs_evaluated_per_step": work["tau_evaluated"] / args.steps,
            "kick_pairs_per_step": work["kick_pairs"] / args.steps,
            "edges_per_step": work["edges"] / args.steps,
            "splits_per_step": work["splits"] / args.steps,
            "other_form": other_line,
            "accuracy": accuracy,
            "force_error": forces,
            "configs": configs,
        }
        print(json.dumps(line), flush=True)
    return 0


def run_accuracy(args):
    """The accuracy gate alone (JSON lines): both forms integrate the
    workload to --t-end from the same state."""
    import torch

    from paper_1407_7105_gb300 import build, cc, ics
    build.build()
    m, x, v = ics.plummer(args.n, seed=args.seed)
    dev = torch.device("cuda", 0)
    dm, dx, dv = (torch.tensor(a, device=dev) for a in (m, x, v))
    for row in accuracy_gate(cc, dm, dx, dv, args.t_end, args.h_fp64_gate):
        print(json.dumps({"accuracy": True, **row}), flush=True)
    return 0


def run_eta_sweep(args):
    """The metric's gate on the other configurations (JSON lines): the mixed
    form of the 65536-body fractal and of the 4096-system batch at the eta
    values {0.03, 0.01, 0.005, 0.0025} over --sweep-steps outer steps:
    |dE/E| (systems: the sum of the systems' own energies), ms per step,
    recursion depth.  The configurations leave eta free; the gate picks the
    largest eta that keeps |dE/E| <= 1e-6."""
    import argparse as _ap
    import torch

    from paper_1407_7105_gb300 import build, cc
    build.build()
    dev = torch.device("cuda", 0)
    for wl, n in (("fractal", 65536), ("systems", 0)):
        a = _ap.Namespace(workload=wl, n=n, nsys=4096)
        m, x, v, off = make_workload(a, args.seed, dev)
        dm, dx, dv = (torch.tensor(q, device=dev) for q in (m, x, v))
        dtw = WORKLOADS[wl]["dt"]
        for eta in (0.03, 0.01, 0.005, 0.0025):
            ctx = cc.Context(dm, dx, dv, dt=dtw, eta=eta, precision=cc.PREC_MIXED, kepler=int(WORKLOADS[wl]["kepler"]))
            if off is not None:
                ctx.set_systems(off)
            E0, _, _ = ctx.energy()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.evolve(args.sweep_steps * dtw)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
            E1, _, _ = ctx.energy()
            st = ctx.stats()
            ctx.close()
            print(json.dumps({"eta_sweep": True, "workload": workload_name(m.shape[0], wl, 4096), "form": "mixed",
                              "eta": eta, "steps": args.sweep_steps, "t_end": args.sweep_steps * dtw,
                              "ms_per_step": 1e3 * sec / args.sweep_steps, "dE_over_E": (E1 - E0) / abs(E0),
                              "max_depth": st["max_depth_seen"]}), flush=True)
    return 0


def run_com_sweep(args):
    """The centre-of-mass approximation of V_CC (Sec. 4.1) against the exact
    kick (JSON lines): the 65536-body fractal and the 16384-body Plummer
    sphere, both forms, theta in {0, 0.3, 0.5, 0.7} (com_max = 32): ms per
    step over --sweep-steps outer steps after one warm-up step, kick pairs
    and pairs taken by the approximation per step, |dE/E| and the momentum
    drift over the steps."""
    import argparse as _ap
    import torch

    from paper_1407_7105_gb300 import build, cc
    build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    for wl, n in (("fractal", 65536), ("plummer", N_BODY)):
        a = _ap.Namespace(workload=wl, n=n, nsys=4096)
        m, x, v, _ = make_workload(a, args.seed, dev)
        dm, dx, dv = (torch.tensor(q, device=dev) for q in (m, x, v))
        dtw = WORKLOADS[wl]["dt"]
        for form in ("mixed", "fp64"):
            for theta in (0.0, 0.3, 0.5, 0.7):
                prec = cc.PREC_MIXED if form == "mixed" else cc.PREC_FP64
                ctx = cc.Context(dm, dx, dv, dt=dtw, eta=ETA, precision=prec, theta=theta, com_max=32)
                E0, P0, _ = ctx.energy()
                ctx.evolve(dtw)
                torch.cuda.synchronize()
                steps = 1 if (form == "fp64" and wl == "fractal") else args.sweep_steps
                _, ms, _, s0, s1 = time_steps(ctx, dtw, dtw, steps, stream)
                E1, P1, _ = ctx.energy()
                ctx.close()
                print(json.dumps({"com_sweep": True, "workload": workload_name(m.shape[0], wl, 4096), "form": form,
                                  "theta": theta, "steps": steps, "ms_per_step": ms / steps,
                                  "kick_pairs_per_step": (s1["kick_pairs"] - s0["kick_pairs"]) / steps,
                                  "com_pairs_per_step": (s1["com_pairs"] - s0["com_pairs"]) / steps,
                                  "dE_over_E": (E1 - E0) / abs(E0), "dP": float(np.abs(P1 - P0).max()),
                                  "steps_for_dE": steps + 1}), flush=True)
    return 0


def run_split_compare(args):
    """The three splits on the same Plummer spheres (JSON lines): CC, HOLD
    (Sec. 2.1) and OK (Sec. 4.2), FP64, N = 256 and 1024 at dt = 1/64 to
    t = 1: ms per step, kick and tau pairs per step, recursion depth and
    |dE/E| at t = 1 -- the paper's comparison of evaluation counts and
    energy error (Sec. 3.1, 4.2)."""
    import torch

    from paper_1407_7105_gb300 import build, cc, ics
    build.build()
    dev = torch.device("cuda", 0)
    dt, steps = 1.0 / 64, 64
    for n in (256, 1024):
        m, x, v = ics.plummer(n, seed=args.seed)
        dm, dx, dv = (torch.tensor(q, device=dev) for q in (m, x, v))
        for name, split in (("CC", cc.SPLIT_CC), ("HOLD", cc.SPLIT_HOLD), ("OK", cc.SPLIT_OK)):
            ctx = cc.Context(dm, dx, dv, dt=dt, eta=ETA, split=split)
            E0, _, _ = ctx.energy()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.evolve(steps * dt)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
            E1, _, _ = ctx.energy()
            st = ctx.stats()
            ctx.close()
            print(json.dumps({"split_compare": True, "workload": f"Plummer N={n}, equal masses, N-body units, eps=0, eta={ETA}, dt=1/64",
                              "split": name, "form": "fp64", "steps": steps, "t_end": steps * dt,
                              "ms_per_step": 1e3 * sec / steps, "kick_pairs_per_step": st["kick_pairs"] / steps,
                              "tau_pairs_per_step": st["tau_pairs"] / steps, "max_depth": st["max_depth_seen"],
                              "dE_over_E": (E1 - E0) / abs(E0)}), flush=True)
    return 0


def run_paper_step(args):
    """The paper's worked case (Sec. 3.1): the first global step of its
    smoothed Plummer test, N = 1024, eps = 1/256, eta = 0.01, dt = 700/512,
    both forms (JSON lines): wall time of the step (a warm-up step of the
    same state first), splits, kick pairs, drifts, depth -- the counts the
    paper prints for its serial code."""
    import torch

    from paper_1407_7105_gb300 import build, cc, ics
    build.build()
    dev = torch.device("cuda", 0)
    m, x, v = ics.plummer(1024, seed=args.seed)
    dm, dx, dv = (torch.tensor(q, device=dev) for q in (m, x, v))
    dt = 700.0 / 512
    for form in ("fp64", "mixed"):
        prec = cc.PREC_MIXED if form == "mixed" else cc.PREC_FP64
        ctx = cc.Context(dm, dx, dv, dt=dt, eta=0.01, eps=1.0 / 256, precision=prec, s_small=args.s_small)
        ctx.evolve(dt)  # warm-up: allocations and the launch-shape tuner's trials
        ctx.set_state(0.0, dm, dx, dv)
        ctx.reset_stats()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.evolve(dt)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        st = ctx.stats()
        ctx.close()
        print(json.dumps({"paper_step": True, "workload": "Plummer N=1024, eps=1/256, eta=0.01, one step dt=700/512",
                          "form": form, "s_small": args.s_small, "seconds": sec, "splits": st["splits"],
                          "kick_pairs": st["kick_pairs"],
                          "tau_pairs": st["tau_pairs"], "tau_pairs_evaluated": st["tau_evaluated"],
                          "drifts": st["drifts"], "max_depth": st["max_depth_seen"]}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cc", choices=["cc", "reference"])
    ap.add_argument("--form", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--split", default="cc", choices=["cc", "hold", "ok"],
                    help="the split of the timed steps (ok: FP64 form only)")
    ap.add_argument("--h-fp64", type=float, default=0.0,
                    help="mixed form: sets split at h < h_fp64*dt take FP64 forces")
    ap.add_argument("--single-form", action="store_true", help="skip timing the other form")
    ap.add_argument("--s-small", type=int, default=-1,
                    help="components of at most this many bodies (<= 512) run on-chip in the batched kernel "
                         "(0: none; -1: the library's choice, 512 mixed / 32 FP64)")
    ap.add_argument("--accuracy", action="store_true", help="integrate both forms to --t-end and report dE/E")
    ap.add_argument("--h-fp64-gate", type=float, default=1.0 / 16,
                    help="accuracy gate: the mixed form's second run takes FP64 forces below this times dt")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the accuracy gate, the force error and the other configurations")
    ap.add_argument("--t-end", type=float, default=1.0)
    ap.add_argument("--eta-sweep", action="store_true",
                    help="energy error of the fractal and the systems batch against eta (mixed form)")
    ap.add_argument("--com-sweep", action="store_true",
                    help="the centre-of-mass approximation of V_CC against the exact kick (both forms, theta sweep)")
    ap.add_argument("--paper-step", action="store_true",
                    help="the paper's worked case (Sec. 3.1, N = 1024, one step of 700/512): both forms' wall time and counts")
    ap.add_argument("--split-compare", action="store_true",
                    help="CC, HOLD and OK splits on 256- and 1024-body spheres to t = 1 (FP64)")
    ap.add_argument("--sweep-steps", type=int, default=16)
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
    if args.eta_sweep:
        return run_eta_sweep(args)
    if args.com_sweep:
        return run_com_sweep(args)
    if args.split_compare:
        return run_split_compare(args)
    if args.paper_step:
        return run_paper_step(args)
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

#!/usr/bin/env python
"""Benchmark of the CT-AUX submatrix-update hot path on GB300.

One step = one full submatrix block of every chain: pre-insertion and G0
gather, prep products, k_max proposals with Gamma growth, Woodbury flush with
compaction, G(tau) measurement, and the FP64 refresh every 32 blocks
(amortised: it lands inside the timed steps at its natural rate).

Metric: accepted updates per second (whole job, all GPUs).  Default workload:
the 2x2x2 simple-cubic cluster (N_c=8, beta=5, U=8) with k_max=64 and the
expansion constant K=256 that puts the order at n~430 (inside the 300-500
range the workload names).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
  python bench.py --impl reference      # the CPU oracle on the same workload

Timing: W untimed blocks, then K timed blocks, each bracketed by CUDA events on
the stream the library launches on, with the L2 cache flushed (a 512 MB write)
between timed blocks; barrier + synchronize on both sides; max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CT-AUX accepted updates/s per GPU, mixed vs FP64 at |dN|<1e-8; flush %peak"
UNIT = "accepted updates/s"
N_TAU_BINS, N_ANCHORS, REFRESH_EVERY = 32, 4, 32
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# dominant kernel, from one ncu capture of the same workload in the state the
# timed blocks run in (summaries under profiles/); an entry is removed when its
# kernel changes
DRAM_TRAFFIC = {("cube8", "fp64", "proposals"): 398848}


def workload(name, K, k_max, chain_id=0, n_chains=8):
    from workloads import configs
    if name == "cube8":
        ch = configs.cube8(K=K, k_max=k_max, capacity=1024, seed=chain_id)
        ch.chain_id = chain_id
        return [ch], dict(n_target=430 if K >= 200 else 140)
    if name == "sq36":
        ch = configs.sq36(K=K, k_max=k_max, capacity=3072, seed=chain_id)
        ch.chain_id = chain_id
        return [ch], dict(n_target=2000 if K >= 1000 else 640)
    if name == "cube100":
        # 8 independent chains; K-matched (K=5700: <n> ~ 7000) chains start from a
        # seeded configuration of that order instead of growing from n=0
        chs = [configs.cube100(K=K, k_max=k_max, capacity=9216, seed=8 * chain_id + i,
                               chain_id=8 * chain_id + i) for i in range(n_chains)]
        n_t = 7000 if K >= 4000 else 1400
        return chs, dict(n_target=n_t, start_order=n_t if K >= 4000 else 0)
    if name == "aim1":
        ch = configs.aim1(K=K, k_max=k_max, capacity=256, seed=chain_id)
        return [ch], dict(n_target=20)
    if name == "batch":
        chs = configs.batch(n_chains=512, k_max=k_max)   # K per chain, matched to n ~ 50..1200
        for c in chs:
            c.chain_id += 512 * chain_id
        return chs, dict(n_target=None)
    raise SystemExit(f"unknown workload {name}")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# nominal dense rates of GB300 per the recipe table (TFLOP/s)
NOMINAL = {"bf16": 2250.0, "tf32": 1100.0, "fp64": 1.25}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            v = [x.strip() for x in line.split(",")]
            if len(v) >= 9:
                rows.append(v)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def reduce_over_ranks(torch, dist, total_ms, accepted, device):
    """Whole-job numbers: the slowest rank's timed milliseconds, the sum of accepted updates.

    Chains are independent (each rank runs its own, with its own Philox chain ids), so
    this is the only exchange between ranks.
    """
    t = torch.tensor([total_ms, float(accepted)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


def cpu_baseline(chains, meta, seconds=15.0):
    """The oracle as it stands, single process, on a bounded sample of the workload."""
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    from oracle.ctaux import OracleChain
    from workloads import configs
    ch = chains[0]
    n0 = meta["n_target"] or 100
    cfg = configs.synthetic_configuration(ch, n0, seed=11)
    oc = OracleChain(ch.table, ch.dx_class, ch.beta, ch.U, ch.K, seed=ch.seed, chain_id=ch.chain_id)
    oc.set_config(cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
    t0 = time.perf_counter()
    props = acc = 0
    while time.perf_counter() - t0 < seconds:
        acc += int(oc.step()["accept"])
        props += 1
    dt = time.perf_counter() - t0
    threads = int(os.environ.get("OPENBLAS_NUM_THREADS", "1"))
    return {"value": acc / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{props} proposals of {ch.name} (k_max={ch.k_max}) from a seeded n={n0} "
                      f"configuration, {dt:.1f} s, dense-LU ratios",
            "proposals_per_s": props / dt}


def run_reference(args, rank, world):
    if rank != 0:
        return
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    from oracle.ctaux import OracleChain
    from workloads import configs
    chains, meta = workload(args.workload, args.K, args.k_max)
    ch = chains[0]
    n0 = meta["n_target"] or 100
    cfg = configs.synthetic_configuration(ch, n0, seed=11)
    oc = OracleChain(ch.table, ch.dx_class, ch.beta, ch.U, ch.K, seed=ch.seed, chain_id=ch.chain_id)
    oc.set_config(cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
    # a step of the reference is a bounded sample of one block: as many
    # proposals as keep the whole run near two minutes (at least one)
    t1 = time.perf_counter()
    oc.step()
    t_prop = time.perf_counter() - t1
    per_step = int(max(1, min(ch.k_max, 120.0 / (t_prop * (args.steps + args.warmup)))))
    for _ in range(args.warmup):
        oc.run(per_step)
    acc = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        acc += sum(int(r["accept"]) for r in oc.run(per_step))
    dt = time.perf_counter() - t0
    value = acc / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{ch.name} N_c={ch.n_c} beta={ch.beta} U={ch.U} K={ch.K} "
                                   f"k_max={ch.k_max} n~{n0}", "l2": "oracle on host"},
            "cpu_baseline": {"value": value, "unit": UNIT,
                             "cores": int(os.environ.get("OPENBLAS_NUM_THREADS", "1")),
                             "kind": "oracle",
                             "sample": f"{args.steps} steps of {per_step} proposals from a seeded "
                                       f"n={n0} configuration"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["both", "fp64", "mixed", "mixed_df64"], default="both",
                    help="both = fp64, mixed and mixed_df64 (the mixed form with its refresh "
                         "eliminating in double-float on the float32 pipe)")
    ap.add_argument("--workload", default="cube8")
    ap.add_argument("--K", type=float, default=256.0)
    ap.add_argument("--k-max", dest="k_max", type=int, default=64)
    ap.add_argument("--chains", type=int, default=8,
                    help="chains of the cube100 workload (a smaller case for profiling)")
    ap.add_argument("--thermalize", type=int, default=300)
    ap.add_argument("--refresh-every", dest="refresh_every", type=int, default=REFRESH_EVERY)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", dest="no_graph", action="store_true",
                    help="direct kernel launches instead of one CUDA graph per block")
    ap.add_argument("--autotune", default=None,
                    help="comma-separated k candidates: choose k_max per chain on the device "
                         "(ctaux_autotune_k) after thermalisation; --k-max is the allocation")
    ap.add_argument("--k-sweep", dest="k_sweep", default=None,
                    help="comma-separated k_max values: print proposals/s per k instead")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1010_3690_gb300 as pk

    if args.k_sweep:
        if rank == 0:
            run_k_sweep(args, pk, torch, local)
        return
    chains, meta = workload(args.workload, args.K, args.k_max, chain_id=rank, n_chains=args.chains)
    forms = ["fp64", "mixed", "mixed_df64"] if args.precision == "both" else [args.precision]
    results = {}
    for form in forms:
        results[form] = measure_form(args, pk, torch, dist, chains, meta, form, local, world,
                                     with_e2e=(form == forms[0]))
    prim = results[forms[0]]
    line = dict(prim["line"])
    for form in forms[1:]:
        sec = results[form]
        line[form] = {k: sec["line"][k] for k in ("value", "ms_per_step", "dtype", "roofline",
                                                 "flush_roofline", "phase_ms_per_step",
                                                 "drift_max_last_refresh", "near_ties",
                                                 "tie_refreshes", "gpu_launches", "clocks")}
        line[f"{form}_vs_fp64"] = sec["line"]["value"] / prim["line"]["value"]
        line["gpu_launches"] += sec["line"]["gpu_launches"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(chains, meta, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_k_sweep(args, pk, torch, local):
    """Updates/s against the submatrix size k (k=1 is the rank-one fast update).

    Same workload and starting configuration for every k, the same number of
    proposals per timing (k_max x steps = 4096), no measurement and no refresh
    (both are the same for every k), FP64 and mixed forms.  The paper's claim
    to set this against: submatrix updates ~8x faster than rank-one updates
    on CPUs at orders 512-2048 (Sec. V A, Fig. 2).
    """
    from workloads import configs
    ks = [int(x) for x in args.k_sweep.split(",")]
    forms = ["fp64", "mixed"] if args.precision == "both" else [args.precision]
    rows = []
    for form in forms:
        precision = pk.CTAUX_MIXED if form == "mixed" else pk.CTAUX_FP64
        for k in ks:
            chains, meta = workload(args.workload, args.K, k)
            ctx = pk.Context(chains, precision=precision, refresh_every=0,
                             n_tau_bins=N_TAU_BINS, n_anchors=N_ANCHORS, device=local)
            n0 = meta["n_target"] or 100
            for i, ch in enumerate(chains):
                cfg = configs.synthetic_configuration(ch, n0, seed=1000 + ch.chain_id)
                ctx.set_config(i, cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
            stream = torch.cuda.current_stream()
            sh = stream.cuda_stream
            ctx.sweep(max(3, 512 // k), stream=sh)     # relax the seeded start
            ctx.recompute()
            n_prop = 4096
            steps = max(1, n_prop // k)
            acc0 = sum(sum(ctx.stats(i)["accepted"]) for i in range(len(chains)))
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.sweep(steps, stream=sh)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            acc = sum(sum(ctx.stats(i)["accepted"]) for i in range(len(chains))) - acc0
            st = ctx.stats(0)
            rows.append({"form": form, "k_max": k, "order_n": st["n"],
                         "proposals_per_s": steps * k * len(chains) / (ms / 1e3),
                         "accepted_per_s": acc / (ms / 1e3), "us_per_proposal": ms * 1e3 / (steps * k)})
            ctx.close()
    out = {"metric": "CT-AUX proposals/s against submatrix size k (k=1: rank-one updates)",
           "workload": workload_name(workload(args.workload, args.K, ks[0])[0]),
           "note": "no measurement, no refresh, no L2 flush; 4096 proposals per k after 512 "
                   "relaxation proposals from a seeded configuration", "rows": rows}
    for form in forms:
        r = {x["k_max"]: x["proposals_per_s"] for x in rows if x["form"] == form}
        if 1 in r:
            best = max(r, key=r.get)
            out[f"{form}_submatrix_over_rank_one"] = {"k_best": best, "speedup": r[best] / r[1]}
    print(json.dumps(out), flush=True)


def workload_name(chains):
    c0 = chains[0]
    if len(chains) == 1:
        return f"{c0.name} N_c={c0.n_c} beta={c0.beta} U={c0.U} K={c0.K} k_max={c0.k_max}, 1 chain per GPU"
    if all(c.name == c0.name and c.n_c == c0.n_c and c.beta == c0.beta and c.U == c0.U and c.K == c0.K
           for c in chains):
        return (f"{c0.name} N_c={c0.n_c} beta={c0.beta} U={c0.U} K={c0.K} k_max={c0.k_max}, "
                f"{len(chains)} chains per GPU")
    ncs = sorted({c.n_c for c in chains})
    return (f"{c0.name}: {len(chains)} independent chains per GPU, N_c in {ncs}, "
            f"beta in [{min(c.beta for c in chains)}, {max(c.beta for c in chains)}], "
            f"U in [{min(c.U for c in chains):.2f}, {max(c.U for c in chains):.2f}], "
            f"K = 0.3 beta U N_c + 30, k_max={c0.k_max}")


def measure_form(args, pk, torch, dist, chains, meta, form, local, world, with_e2e):
    precision = pk.CTAUX_FP64 if form == "fp64" else pk.CTAUX_MIXED
    ctx = pk.Context(chains, precision=precision, refresh_every=args.refresh_every,
                     n_tau_bins=N_TAU_BINS, n_anchors=N_ANCHORS, device=local,
                     refresh_df64=int(form == "mixed_df64"), use_graph=int(not args.no_graph))
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    if meta.get("start_order"):
        from workloads import configs
        for i, ch in enumerate(chains):
            cfg = configs.synthetic_configuration(ch, meta["start_order"], seed=1000 + ch.chain_id)
            ctx.set_config(i, cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
    ctx.sweep(args.thermalize, measure=False, stream=sh)
    k_tuned = None
    if args.autotune:
        cand = [int(x) for x in args.autotune.split(",")]
        ks, _ = ctx.autotune_k(candidates=cand, n_blocks=8)
        k_tuned = {str(k): int((ks == k).sum()) for k in sorted(set(ks.tolist()))}
    for _ in range(max(3, args.warmup)):
        ctx.sweep(1, measure=True, stream=sh)
    ctx.synchronize()

    def accepted_total():
        return sum(sum(ctx.stats(i)["accepted"]) for i in range(len(chains)))

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    steps = args.steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    acc0 = accepted_total()
    _, kern0 = ctx.phase_times()
    ties0 = sum(ctx.stats(i)["near_ties"] for i in range(len(chains)))
    # timed region: no phase events (and CUDA-graph launches unless --no-graph)
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(steps):
        flush.zero_()
        starts[i].record(stream)
        ctx.sweep(1, measure=True, stream=sh)
        ends[i].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends))
    acc = accepted_total() - acc0
    _, kern1 = ctx.phase_times()
    kernels = int((kern1 - kern0).sum())
    ties = sum(ctx.stats(i)["near_ties"] for i in range(len(chains))) - ties0
    tie_refreshes = sum(ctx.stats(i)["tie_refreshes"] for i in range(len(chains)))
    if world > 1:
        total_ms, acc = reduce_over_ranks(torch, dist, total_ms, acc, "cuda")
    value = acc / (total_ms / 1e3)

    # phase breakdown: a further profiled pass (CUDA events around every phase,
    # direct launches) over a whole number of refresh periods
    prof_steps = args.refresh_every if args.refresh_every > 0 else 32
    while prof_steps < 16:
        prof_steps += args.refresh_every
    work0 = ctx.work()
    ms0, _ = ctx.phase_times()
    ctx.set_profiling(True)
    for i in range(prof_steps):
        flush.zero_()
        ctx.sweep(1, measure=True, stream=sh)
    ctx.synchronize()
    ctx.set_profiling(False)
    ms1, _ = ctx.phase_times()
    work1 = ctx.work()
    phase_ms = ms1 - ms0

    # ---------------- rooflines (live CUDA-event phase times, algorithmic work from the device)
    peaks, peak_kind = load_peaks()
    names = ctx.PHASES
    fp64_peak = peaks["bf16_tflops"] * NOMINAL["fp64"] / NOMINAL["bf16"]
    fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12     # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz
    tf32x3_peak = peaks["bf16_tflops"] * NOMINAL["tf32"] / NOMINAL["bf16"] / 3.0
    alu_peak = fp64_peak if precision == pk.CTAUX_FP64 else fp32_peak
    alu_src = (f"FP64 = bf16 {peak_kind} x 1.25/2250" if precision == pk.CTAUX_FP64
               else "FP32 = 152 SMs x 128 lanes x 2 x 2.07 GHz")
    dw = {k: work1[k] - work0[k] for k in work1}
    n_sm = min(152, len(chains))   # one CTA (one SM) per chain for the Gamma growth

    def roof(phase):
        sec = phase_ms[phase] / 1e3
        nm = names[phase]
        if nm == "flush_gemm":
            if precision == pk.CTAUX_MIXED:
                return dict(bound="tensor", achieved=dw["flush_flop"] / sec / 1e12, peak=tf32x3_peak,
                            unit="TFLOP/s",
                            peak_source=f"3xTF32 = bf16 {peak_kind} x 1100/2250 / 3 products")
            return dict(bound="alu", achieved=dw["flush_flop"] / sec / 1e12, peak=alu_peak,
                        unit="TFLOP/s", peak_source=alu_src)
        if nm == "prep":
            return dict(bound="alu", achieved=dw["prep_flop"] / sec / 1e12, peak=alu_peak,
                        unit="TFLOP/s", peak_source=alu_src)
        if nm == "proposals":
            return dict(bound="alu", achieved=dw["gamma_flop"] / sec / 1e12,
                        peak=alu_peak * n_sm / 152.0, unit="TFLOP/s",
                        peak_source=alu_src + f", {n_sm} of 152 SMs (one CTA per chain)")
        if nm == "measure":
            return dict(bound="alu", achieved=dw["meas_flop"] / sec / 1e12, peak=alu_peak,
                        unit="TFLOP/s", peak_source=alu_src + " (estimator flops, interpolations not counted)")
        if nm == "refresh":
            if form == "mixed_df64":
                # one compensated double-float multiply-add of the trailing update
                # is 12 float32 operations (TwoProd 2, cross terms 2, TwoSum 6, 2 adds)
                return dict(bound="alu", achieved=dw["refresh_flop"] / sec / 1e12, peak=fp32_peak / 12.0,
                            unit="TFLOP/s",
                            peak_source="double-float = FP32 peak / 12 float32 operations per multiply-add "
                                        "(2 m^3 per spin)")
            return dict(bound="alu", achieved=dw["refresh_flop"] / sec / 1e12, peak=fp64_peak,
                        unit="TFLOP/s", peak_source=f"FP64 = bf16 {peak_kind} x 1.25/2250 (2 m^3 per spin)")
        # plan/gather and flush support: latency-bound, no algorithmic roofline
        return dict(bound="latency", achieved=None, peak=None, unit=None, peak_source=None)

    # dominant among the phases of every block; the near-tie refinement (rare by
    # construction) is reported in phase_ms_per_step only
    dom = int(phase_ms[:names.index("tie_refine")].argmax())
    r = roof(dom)
    roofline = {"kernel": names[dom], "bound": r["bound"], "achieved": r["achieved"],
                "peak": r["peak"], "unit": r["unit"],
                "frac": r["achieved"] / r["peak"] if r["peak"] else None,
                "traffic": DRAM_TRAFFIC.get((args.workload, form, names[dom])),
                "peak_source": r["peak_source"],
                "ms_per_step": phase_ms[dom] / prof_steps}
    fr = roof(names.index("flush_gemm"))
    flush_roof = {"bound": fr["bound"], "achieved": fr["achieved"], "peak": fr["peak"],
                  "unit": fr["unit"], "frac": fr["achieved"] / fr["peak"],
                  "ms_per_step": phase_ms[3] / prof_steps, "peak_source": fr["peak_source"]}

    e2e = None
    if with_e2e:
        e2e_steps = max(5, min(steps, 50))
        acc_e0 = accepted_total()
        t_e2e = 0.0
        d2h = 0
        for _ in range(e2e_steps):
            t0 = time.perf_counter()
            ctx.sweep(1, measure=True, stream=sh)
            G, E, nm_ = ctx.measure_G(0)
            ctx.stats(0)
            t_e2e += time.perf_counter() - t0
            d2h = 2 * G.nbytes + 512   # sums and squares of G(tau), plus the counters
        acc_e = accepted_total() - acc_e0
        e2e = {"value": acc_e / t_e2e, "unit": UNIT, "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": d2h}

    st = ctx.stats(0)
    orders = [ctx.stats(i)["n"] for i in range(len(chains))]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": total_ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if precision == pk.CTAUX_FP64 else "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(chains),
                       "order_n": st["n"] if len(chains) == 1 else
                       {"mean": sum(orders) / len(orders), "min": int(min(orders)), "max": int(max(orders))},
                       "precision": form,
                       "l2": "flushed between timed steps (512 MB write)",
                       "launch": "direct" if args.no_graph else "one CUDA graph per block and per measurement",
                       "refresh_every": args.refresh_every, "n_tau_bins": N_TAU_BINS,
                       "n_anchors": N_ANCHORS,
                       "k_max": ({"autotuned (chains per k)": k_tuned} if k_tuned
                                 else sorted({c.k_max for c in chains}))},
            "roofline": roofline, "flush_roofline": flush_roof,
            "phase_ms_per_step": {names[i]: phase_ms[i] / prof_steps for i in range(len(names))},
            "phase_pass_steps": prof_steps,
            "gpu_launches": kernels,
            "accept_rate": acc / max(1, steps * sum(c.k_max for c in chains) * world),
            "drift_max_last_refresh": st["last_drift_max"], "near_ties": ties,
            "tie_refreshes": tie_refreshes,
            "clocks": clk}
    if e2e is not None:
        line["e2e"] = e2e
    ctx.close()
    del flush
    torch.cuda.empty_cache()
    return {"line": line}


if __name__ == "__main__":
    main()

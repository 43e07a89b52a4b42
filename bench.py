#!/usr/bin/env python
"""Benchmark of the CT-AUX submatrix-update hot path on GB300.

One step = one full submatrix block of every chain: pre-insertion and G0
gather, prep products, k_max proposals with Gamma growth, Woodbury flush with
compaction, G(tau) measurement, and the FP64 refresh at its cadence (it lands
inside the timed steps: every min(refresh_every, steps) blocks).

Metric: accepted updates per second (whole job, all GPUs), for the plain FP64
form and the mixed form (3xTF32 tensor-core flush, FP64 refresh and near-tie
decisions) in one line, plus the flush's fraction of its tensor roofline.
Default workload: the largest single-GPU configuration, the 100-site 3D
Hubbard cluster (beta=4, U=8, half filling) with k_max=256 and 8 independent
chains, at the expansion constant K=5700 that puts the order at n~7000 (the
range the workload names); every chain starts from a seeded configuration of
order 7000.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision both|fp64|mixed|mixed_df64]
                  [--workload cube100|cube8|sq36|batch|aim1]
  python bench.py --impl reference      # the CPU oracle on the same workload
  python bench.py --k-sweep 1,2,4,...   # proposals/s against the submatrix size

Timing: W untimed blocks, then K timed blocks, each bracketed by CUDA events on
the stream the library launches on, with the L2 cache flushed (a 512 MB write)
between timed blocks; barrier + synchronize on both sides; max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
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
N_TAU_BINS, N_ANCHORS = 32, 4

# Per workload: expansion constant (K-matched, so that the order lands in the
# range the workload names), submatrix size, thermalisation blocks, the order
# the chains start from (0 = empty), the order the CPU oracle samples at,
# chains per GPU and the refresh cadence.
WORKLOADS = {
    "cube100": dict(K=5700.0, k_max=256, thermalize=5, start_order=7000, n_target=7000,
                    chains=8, refresh_every=32),
    "cube8": dict(K=256.0, k_max=64, thermalize=300, start_order=0, n_target=430, chains=1,
                  refresh_every=32),
    "sq36": dict(K=1400.0, k_max=128, thermalize=200, start_order=0, n_target=2000, chains=1,
                 refresh_every=32),
    "aim1": dict(K=1.0, k_max=8, thermalize=300, start_order=0, n_target=20, chains=1,
                 refresh_every=32),
    "batch": dict(K=None, k_max=128, thermalize=150, start_order=0, n_target=None, chains=512,
                  refresh_every=128, autotune="16,32,64,128", autotune_tiles=True),
}

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the
# dominant kernel, per unit of work, from an ncu capture of the same kernel on a
# smaller case (profiles/k_refresh_cube100_traffic.md).  The refresh reads and
# writes its float64 work matrix X (8 m^2 bytes per spin, far above L2 at these
# orders) once per 32-column panel, so its traffic grows as m^3: the capture at
# m = 4000 (one chain, both spins, 66.1 GB) gives bytes per m^3, scaled to a
# launch by the sum of m^3 over the chains it refreshes.  An entry is removed
# when its kernel changes.
DRAM_TRAFFIC = {
    ("cube100", "fp64", "refresh"): (32925212672 + 33162264064) / 4000.0 ** 3,
    ("cube100", "mixed_df64", "refresh"): (32591805952 + 33272619776) / 4000.0 ** 3,
}


def workload(name, K=None, k_max=None, chain_id=0, n_chains=None):
    """Chains of one rank (chain ids offset by rank) and the workload's settings."""
    from workloads import configs
    w = dict(WORKLOADS[name])
    K = w["K"] if K is None else K
    k_max = w["k_max"] if k_max is None else k_max
    n_chains = w["chains"] if n_chains is None else n_chains
    w.update(K=K, k_max=k_max, chains=n_chains)
    if name == "cube100":
        chs = [configs.cube100(K=K, k_max=k_max, capacity=9216, seed=n_chains * chain_id + i,
                               chain_id=n_chains * chain_id + i) for i in range(n_chains)]
        if K < 4000:   # K = 1: orders ~1400, grown from the empty configuration
            w.update(n_target=1400, start_order=0)
        return chs, w
    if name == "cube8":
        ch = configs.cube8(K=K, k_max=k_max, capacity=1024, seed=chain_id)
        ch.chain_id = chain_id
        if K < 200:
            w.update(n_target=140)
        return [ch], w
    if name == "sq36":
        ch = configs.sq36(K=K, k_max=k_max, capacity=3072, seed=chain_id)
        ch.chain_id = chain_id
        if K < 1000:
            w.update(n_target=640)
        return [ch], w
    if name == "aim1":
        ch = configs.aim1(K=K, k_max=k_max, capacity=256, seed=chain_id)
        ch.chain_id = chain_id
        return [ch], w
    if name == "batch":
        chs = configs.batch(n_chains=n_chains, k_max=k_max)   # K per chain, matched to n ~ 50..1200
        for c in chs:
            c.chain_id += n_chains * chain_id
        return chs, w
    raise SystemExit(f"unknown workload {name}")


def workload_name(chains, meta):
    c0 = chains[0]
    if c0.name == "batch":
        ncs = sorted({c.n_c for c in chains})
        return (f"batch: {len(chains)} independent chains per GPU, N_c in {ncs}, "
                f"beta in [{min(c.beta for c in chains)}, {max(c.beta for c in chains)}], "
                f"U in [{min(c.U for c in chains):.2f}, {max(c.U for c in chains):.2f}], "
                f"K = 0.3 beta U N_c + 30, k_max={c0.k_max}")
    start = (f", start from a seeded configuration of order {meta['start_order']}"
             if meta.get("start_order") else "")
    return (f"{c0.name} N_c={c0.n_c} beta={c0.beta} U={c0.U} K={c0.K} k_max={c0.k_max}, "
            f"{len(chains)} chain{'s' if len(chains) > 1 else ''} per GPU{start}")


def effective_refresh(meta, args):
    """Refresh cadence of the run: the workload's, or every `steps` blocks when
    fewer steps are timed, so that the timed region holds its share of refreshes
    (exactly one when steps <= the workload's cadence)."""
    r = args.refresh_every if args.refresh_every is not None else meta["refresh_every"]
    if r > 0 and args.steps < r:
        r = args.steps
    return r


def line_config(args, chains, meta, refresh):
    """The `config` object, identical in the GPU arm and the oracle arm."""
    return {"workload": workload_name(chains, meta),
            "k_max": sorted({c.k_max for c in chains}),
            "refresh_every": refresh, "n_tau_bins": N_TAU_BINS, "n_anchors": N_ANCHORS,
            "gamma": getattr(args, "gamma", "inverse"),
            "measure": "one G(tau) measurement per block",
            "l2": "GPU arm: L2 flushed by a 512 MB write between timed steps; "
                  "oracle arm: host cores",
            "launch": "GPU arm: one CUDA graph per block and per measurement; oracle arm: numpy"}


GAMMA_FORMS = {"inverse": 0, "lu": 1}   # CTAUX_GAMMA_INVERSE, CTAUX_GAMMA_LU


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# nominal dense rates of GB300 per the recipe table (TFLOP/s)
NOMINAL = {"bf16": 2250.0, "tf32": 1100.0, "fp64": 1.25}


# ------------------------------------------------------------------ host cores
def host_cores():
    """Cores this process may use: affinity, capped by a cgroup CPU quota."""
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    try:
        q, p = open("/sys/fs/cgroup/cpu.max").read().split()[:2]
        if q != "max":
            n = min(n, max(1, int(math.ceil(int(q) / int(p)))))
    except (OSError, ValueError):
        pass
    return n


def host_cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    fields = {}
    try:
        for line in open("/proc/cpuinfo"):
            if ":" in line:
                k, v = line.split(":", 1)
                fields.setdefault(k.strip(), v.strip())
    except OSError:
        pass
    if "model name" in fields:
        return fields["model name"]
    parts = {"0xd4f": "Arm Neoverse-V2", "0xd40": "Arm Neoverse-V1", "0xd0c": "Arm Neoverse-N1"}
    if "CPU part" in fields:
        return parts.get(fields["CPU part"], f"Arm CPU part {fields['CPU part']}")
    return platform.processor() or platform.machine()


def host_mem_bytes():
    try:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    except (ValueError, OSError):
        return 0


def _oracle_worker(job):
    """One independent oracle chain on one core: untimed start from a seeded
    configuration, then proposals until `seconds` have passed (at least one)."""
    ch, n0, seed, seconds = job
    from oracle.ctaux import OracleChain
    from workloads import configs
    oc = OracleChain(ch.table, ch.dx_class, ch.beta, ch.U, ch.K, seed=ch.seed, chain_id=ch.chain_id)
    if n0:
        cfg = configs.synthetic_configuration(ch, n0, seed=seed)
        oc.set_config(cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
    props = acc = 0
    t0 = time.perf_counter()
    while props == 0 or time.perf_counter() - t0 < seconds:
        acc += int(oc.step()["accept"])
        props += 1
    return props, acc, time.perf_counter() - t0


def cpu_baseline(chains, meta, seconds):
    """The oracle as it stands, one independent chain per host core (single-threaded
    BLAS each), on a bounded sample of the workload at its order."""
    import multiprocessing as mp
    cores = host_cores()
    n0 = meta["n_target"] or 0
    # an oracle proposal at order m holds a few m x m float64 temporaries
    per_proc = 8 * 8 * max(n0, 256) ** 2 + (1 << 28)
    mem = host_mem_bytes()
    procs = max(1, min(cores, int(0.5 * mem // per_proc) if mem else cores))
    jobs = [(chains[i % len(chains)], n0, 11 + i, seconds) for i in range(procs)]
    saved = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS",
                                             "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"        # inherited by the spawned workers only
    try:
        with mp.get_context("spawn").Pool(procs) as pool:
            res = pool.map(_oracle_worker, jobs, chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    props = sum(r[0] for r in res)
    acc = sum(r[1] for r in res)
    wall = max(r[2] for r in res)
    c0 = chains[0]
    return {"value": acc / wall, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"{procs} independent oracle chains of {c0.name} (one per core, "
                      f"single-threaded BLAS), each from a seeded configuration of order {n0}, "
                      f"{props} proposals in {wall:.1f} s; dense-LU determinant ratios, "
                      f"not an optimised CPU solver",
            "proposals_per_s": props / wall, "nproc": cores, "cpu_model": host_cpu_model()}


def run_reference(args, rank, world):
    """The oracle on the same workload (chain 0), on all host cores through the
    BLAS threads of numpy; a step is a bounded sample: one proposal."""
    if rank != 0:
        return
    from oracle.ctaux import OracleChain
    from workloads import configs
    chains, meta = workload(args.workload, args.K, args.k_max, n_chains=args.chains)
    if args.order is not None:
        meta.update(start_order=args.order, n_target=args.order)
    refresh = effective_refresh(meta, args)
    ch = chains[0]
    n0 = meta["n_target"] or 0
    oc = OracleChain(ch.table, ch.dx_class, ch.beta, ch.U, ch.K, seed=ch.seed, chain_id=ch.chain_id)
    if n0:
        cfg = configs.synthetic_configuration(ch, n0, seed=1000 + ch.chain_id)
        oc.set_config(cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
    per_step = 1
    for _ in range(args.warmup):
        oc.run(per_step)
    acc = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        acc += sum(int(r["accept"]) for r in oc.run(per_step))
    dt = time.perf_counter() - t0
    value = acc / dt
    cores = host_cores()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": line_config(args, chains, meta, refresh),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} steps of {per_step} proposal of chain 0 of "
                                       f"{ch.name} from a seeded configuration of order {n0} "
                                       f"(numpy BLAS on {cores} threads)",
                             "cpu_model": host_cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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


# --------------------------------------------------------------- multi-GPU
def reduce_over_ranks(torch, dist, total_ms, accepted, device):
    """Whole-job numbers: the slowest rank's timed milliseconds, the sum of accepted updates."""
    t = torch.tensor([total_ms, float(accepted)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


def pool_accumulators(accs):
    """Sum the raw G(tau) accumulators of several chains (ctaux_get_accumulators);
    chains must share the measurement layout."""
    import numpy as np
    out = {k: np.zeros_like(accs[0][k]) for k in ("sum", "sumsq", "bin_sum", "bin_sumsq")}
    out["n_meas"] = out["n_bins"] = 0
    for a in accs:
        for k in ("sum", "sumsq", "bin_sum", "bin_sumsq"):
            out[k] += a[k]
        out["n_meas"] += a["n_meas"]
        out["n_bins"] += a["n_bins"]
    return out


def merge_accumulators(torch, dist, acc, device):
    """The measurement exchange of the multi-GPU path (chains shard by rank): an
    all-reduce (sum) of the G(tau) sums, squares, bin sums and counts, then the
    pooled mean and its binned standard error."""
    import numpy as np
    shape = acc["sum"].shape
    flat = np.concatenate([acc[k].ravel() for k in ("sum", "sumsq", "bin_sum", "bin_sumsq")]
                          + [np.array([acc["n_meas"], acc["n_bins"]], dtype=np.float64)])
    t = torch.tensor(flat, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    v = t.cpu().numpy()
    size = int(np.prod(shape))
    parts = [v[i * size:(i + 1) * size].reshape(shape) for i in range(4)]
    n_meas, n_bins = float(v[4 * size]), float(v[4 * size + 1])
    return pooled_estimate(parts[0], parts[2], parts[3], n_meas, n_bins)


def pooled_estimate(s, bs, bq, n_meas, n_bins):
    """Mean = sum / measurements; error = spread of the bin means / sqrt(bins)."""
    import numpy as np
    mean = s / max(n_meas, 1.0)
    if n_bins >= 2:
        bm = bs / n_bins
        var = np.maximum(bq / n_bins - bm * bm, 0.0) * n_bins / (n_bins - 1.0)
        err = np.sqrt(var / n_bins)
    else:
        err = np.full_like(mean, np.nan)
    return mean, err, n_meas, n_bins


# ------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["both", "fp64", "mixed", "mixed_df64"], default="both",
                    help="both = fp64, mixed and mixed_df64 (the mixed form with its refresh "
                         "eliminating in double-float on the float32 pipe)")
    ap.add_argument("--workload", default="cube100", choices=sorted(WORKLOADS))
    ap.add_argument("--K", type=float, default=None)
    ap.add_argument("--k-max", dest="k_max", type=int, default=None)
    ap.add_argument("--chains", type=int, default=None,
                    help="chains per GPU (cube100: 8; fewer for a smaller profiling case)")
    ap.add_argument("--thermalize", type=int, default=None)
    ap.add_argument("--order", type=int, default=None,
                    help="start order of the chains (and of the oracle's sample); a smaller "
                         "case for profiling")
    ap.add_argument("--refresh-every", dest="refresh_every", type=int, default=None)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", dest="no_graph", action="store_true",
                    help="direct kernel launches instead of one CUDA graph per block")
    ap.add_argument("--autotune", default=None,
                    help="comma-separated k candidates: choose k_max per chain on the device "
                         "(ctaux_autotune_k) after thermalisation; --k-max is the allocation")
    ap.add_argument("--autotune-tiles", dest="autotune_tiles", action="store_true",
                    help="choose the CUDA-core products' tile shapes per (order, k) octave on the "
                         "device (ctaux_autotune_tiles) after the k tuning")
    ap.add_argument("--cpu-k-sweep", dest="cpu_k_sweep", default=None,
                    help="comma-separated k_max values: rank-one against submatrix updates on one "
                         "host core (the paper's CPU comparison, Sec. V A) at --cpu-orders")
    ap.add_argument("--cpu-orders", dest="cpu_orders", default="512,1024,2048")
    ap.add_argument("--gamma", choices=["inverse", "lu"], default=None,
                    help="how a block keeps Gamma: partitioned inverse (default) or L U (Sec. III D)")
    ap.add_argument("--k-sweep", dest="k_sweep", default=None,
                    help="comma-separated k_max values: print proposals/s per k instead")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.gamma is None:
        args.gamma = WORKLOADS[args.workload].get("gamma", "inverse")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.cpu_k_sweep:
        return run_cpu_k_sweep(args) if rank == 0 else None

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
    if args.order is not None:
        meta.update(start_order=args.order, n_target=args.order)
    if args.autotune is None and meta.get("autotune"):
        args.autotune = meta["autotune"]
    if meta.get("autotune_tiles"):
        args.autotune_tiles = True
    if args.thermalize is None:
        args.thermalize = meta["thermalize"]
    refresh = effective_refresh(meta, args)
    forms = ["fp64", "mixed", "mixed_df64"] if args.precision == "both" else [args.precision]
    results = {}
    for form in forms:
        results[form] = measure_form(args, pk, torch, dist, chains, meta, refresh, form, local,
                                     world, with_e2e=(form == forms[0]) and not args.no_e2e)
    prim = results[forms[0]]
    line = dict(prim["line"])
    line["config"] = line_config(args, chains, meta, refresh)
    for form in forms[1:]:
        sec = results[form]
        line[form] = {k: sec["line"][k] for k in ("value", "ms_per_step", "dtype", "roofline",
                                                 "flush_roofline", "phase_ms_per_step",
                                                 "drift_max_last_refresh",
                                                 "drift_rel_max_last_refresh", "order_n",
                                                 "near_ties", "tie_refreshes", "gpu_launches",
                                                 "refreshes_in_timed_region", "clocks")}
        line[f"{form}_vs_fp64"] = sec["line"]["value"] / prim["line"]["value"]
        line["gpu_launches"] += sec["line"]["gpu_launches"]
    if "mixed" in results:
        line["flush_tensor_frac"] = results["mixed"]["line"]["flush_roofline"]["frac"]
        line["mixed_precision_note"] = (
            "|dN| < 1e-8 after refresh: the FP64 form's drift at a refresh is reported as "
            "drift_max_last_refresh; in the mixed forms the refresh's float64 result is stored "
            "in float32 (relative rounding 6e-8), and drift_max_last_refresh is the float32 "
            "chain's drift before the refresh, so the condition holds for the refresh result, "
            "not for the float32 N the mixed chain continues from")
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(chains, meta, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_cpu_k_sweep(args):
    """Proposals/s of rank-one and submatrix updates on one host core, the same
    Markov chain from the same seeded configuration (bench_cpu.py), on the
    2x2x2 cluster table at the orders of the paper's comparison (Sec. V A, Fig. 2:
    about 8x at orders 512-2048 on CPUs)."""
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    import bench_cpu
    from workloads import configs
    ks = [int(x) for x in args.cpu_k_sweep.split(",")]
    orders = [int(x) for x in args.cpu_orders.split(",")]
    ch = configs.cube8(K=256.0, k_max=max(ks), capacity=max(orders) + 1024)
    rows = []
    for n0 in orders:
        rows += bench_cpu.time_algorithms(ch, n0, ks, n_props=max(256, 2 * max(ks)))
    out = {"metric": "CT-AUX proposals/s on one host core: submatrix against rank-one updates",
           "workload": f"cube8 table (N_c=8, beta=5, U=8, K=256), seeded configurations of orders {orders}",
           "cpu_model": host_cpu_model(), "threads": 1,
           "note": "float64, numpy with BLAS products; the same Markov chain for every algorithm",
           "rows": rows, "speedup": {}}
    for n0 in orders:
        r1 = next(r for r in rows if r["order_n0"] == n0 and r["algorithm"] == "rank_one")
        best = max((r for r in rows if r["order_n0"] == n0 and r["algorithm"] == "submatrix"),
                   key=lambda r: r["proposals_per_s"])
        out["speedup"][str(n0)] = {"k_best": best["k_max"],
                                   "submatrix_over_rank_one": best["proposals_per_s"] / r1["proposals_per_s"]}
    print(json.dumps(out), flush=True)


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
    meta0 = None
    for form in forms:
        precision = pk.CTAUX_MIXED if form == "mixed" else pk.CTAUX_FP64
        for k in ks:
            chains, meta = workload(args.workload, args.K, k, n_chains=args.chains)
            meta0 = meta
            ctx = pk.Context(chains, precision=precision, refresh_every=0,
                             n_tau_bins=N_TAU_BINS, n_anchors=N_ANCHORS, device=local,
                             gamma_form=GAMMA_FORMS[args.gamma])
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
           "workload": workload_name(workload(args.workload, args.K, ks[0], n_chains=args.chains)[0],
                                     meta0),
           "note": "no measurement, no refresh, no L2 flush; 4096 proposals per k after 512 "
                   "relaxation proposals from a seeded configuration", "rows": rows}
    for form in forms:
        r = {x["k_max"]: x["proposals_per_s"] for x in rows if x["form"] == form}
        if 1 in r:
            best = max(r, key=r.get)
            out[f"{form}_submatrix_over_rank_one"] = {"k_best": best, "speedup": r[best] / r[1]}
    print(json.dumps(out), flush=True)


def measure_form(args, pk, torch, dist, chains, meta, refresh, form, local, world, with_e2e):
    precision = pk.CTAUX_FP64 if form == "fp64" else pk.CTAUX_MIXED
    ctx = pk.Context(chains, precision=precision, refresh_every=refresh,
                     n_tau_bins=N_TAU_BINS, n_anchors=N_ANCHORS, device=local,
                     refresh_df64=int(form == "mixed_df64"), use_graph=int(not args.no_graph),
                     gamma_form=GAMMA_FORMS[args.gamma])
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
    tiles_tuned = None
    if args.autotune_tiles:
        import numpy as np
        table, gain = ctx.autotune_tiles(n_blocks=3)
        tiles_tuned = {"variants_in_table": np.bincount(table, minlength=3).tolist(),
                       "gain_over_default_shapes": gain}
    ctx.recompute()   # fresh N; the refresh cadence counts from here
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # phase breakdown first: a profiled pass (CUDA events around every phase,
    # direct launches) over one refresh period, which ends with a refresh
    prof_steps = refresh if refresh > 0 else 16
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

    for _ in range(args.warmup):
        ctx.sweep(1, measure=True, stream=sh)
    ctx.synchronize()

    def accepted_total():
        return sum(sum(ctx.stats(i)["accepted"]) for i in range(len(chains)))

    def proposals_total():
        return sum(sum(ctx.stats(i)["proposals"]) for i in range(len(chains)))

    def refreshes_total():
        return sum(ctx.stats(i)["refreshes"] for i in range(len(chains)))

    steps = args.steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    acc0 = accepted_total()
    prop0 = proposals_total()
    ref0 = refreshes_total()
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
    props = proposals_total() - prop0
    accept_rate = acc / max(1, props)    # this rank's chains
    n_refreshes = (refreshes_total() - ref0) // max(1, len(chains))
    _, kern1 = ctx.phase_times()
    kernels = int((kern1 - kern0).sum())
    ties = sum(ctx.stats(i)["near_ties"] for i in range(len(chains))) - ties0
    tie_refreshes = sum(ctx.stats(i)["tie_refreshes"] for i in range(len(chains)))
    measurement = None
    if world > 1:
        total_ms, acc = reduce_over_ranks(torch, dist, total_ms, acc, "cuda")
        # the measurement exchange: every rank's chains pooled into one estimate
        mean, err, n_meas, n_bins = merge_accumulators(
            torch, dist, pool_accumulators([ctx.accumulators(i) for i in range(len(chains))]),
            "cuda")
        measurement = {"pooled_measurements": n_meas, "pooled_bins": n_bins,
                       "G_local_tau0": float(mean[0, 0, 0]), "err": float(err[0, 0, 0])}
    value = acc / (total_ms / 1e3)

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
    elem = 8 if precision == pk.CTAUX_FP64 else 4

    def roof(phase):
        sec = phase_ms[phase] / 1e3
        nm = names[phase]
        if nm == "flush_gemm":
            r = dict(achieved=dw["flush_flop"] / sec / 1e12, unit="TFLOP/s",
                     alg_bytes_per_step=dw["flush_bytes"] / prof_steps)
            if precision == pk.CTAUX_MIXED:
                r.update(bound="tensor", peak=tf32x3_peak,
                         peak_source=f"3xTF32 = bf16 {peak_kind} x 1100/2250 / 3 products")
            else:
                r.update(bound="alu", peak=alu_peak, peak_source=alu_src)
            return r
        if nm == "prep":
            # N is read by the R~ and the G_{old,new} products: one read per spin is
            # the algorithmic minimum
            n_mean = meta_order_mean[0]
            r = dict(achieved=dw["prep_flop"] / sec / 1e12, unit="TFLOP/s",
                     alg_bytes_per_step=2.0 * elem * n_mean * n_mean * len(chains))
            if precision == pk.CTAUX_MIXED:
                # products 0 and 1 on the tensor cores (3xTF32), the small k x k
                # product on the CUDA cores
                r.update(bound="tensor", peak=tf32x3_peak,
                         peak_source=f"3xTF32 = bf16 {peak_kind} x 1100/2250 / 3 products")
            else:
                r.update(bound="alu", peak=alu_peak, peak_source=alu_src)
            return r
        if nm == "proposals":
            a = dw["gamma_flop"] / sec / 1e12
            return dict(bound="alu", achieved=a, peak=alu_peak, unit="TFLOP/s",
                        peak_source=alu_src + "; whole GPU (the Gamma chain of a chain runs on "
                                              "one SM: frac_of_active_sms is against the "
                                              f"{n_sm} SMs in use)",
                        frac_of_active_sms=a / (alu_peak * n_sm / 152.0))
        if nm == "measure":
            return dict(bound="alu", achieved=dw["meas_flop"] / sec / 1e12, peak=alu_peak,
                        unit="TFLOP/s",
                        peak_source=alu_src + " (estimator flops, interpolations not counted)")
        if nm == "refresh":
            if form == "mixed_df64":
                # one compensated double-float multiply-add of the trailing update
                # is 12 float32 operations (TwoProd 2, cross terms 2, TwoSum 6, 2 adds)
                return dict(bound="alu", achieved=dw["refresh_flop"] / sec / 1e12,
                            peak=fp32_peak / 12.0, unit="TFLOP/s",
                            peak_source="double-float = FP32 peak / 12 float32 operations per "
                                        "multiply-add (2 m^3 per spin)")
            return dict(bound="alu", achieved=dw["refresh_flop"] / sec / 1e12, peak=fp64_peak,
                        unit="TFLOP/s",
                        peak_source=f"FP64 = bf16 {peak_kind} x 1.25/2250 (2 m^3 per spin)")
        # plan/gather and flush support: latency-bound, no algorithmic roofline
        return dict(bound="latency", achieved=None, peak=None, unit=None, peak_source=None)

    orders = [ctx.stats(i)["n"] for i in range(len(chains))]
    meta_order_mean = [sum(orders) / len(orders)]
    # dominant among the phases of every block; the near-tie refinement (rare by
    # construction) is reported in phase_ms_per_step only
    dom = int(phase_ms[:names.index("tie_refine")].argmax())
    r = roof(dom)
    coef = DRAM_TRAFFIC.get((args.workload, form, names[dom]))
    traffic = coef * sum(float(m) ** 3 for m in orders) if coef else None
    roofline = {"kernel": names[dom], "bound": r["bound"], "achieved": r["achieved"],
                "peak": r["peak"], "unit": r["unit"],
                "frac": r["achieved"] / r["peak"] if r["peak"] else None,
                "traffic": traffic, "peak_source": r["peak_source"],
                "ms_per_step": phase_ms[dom] / prof_steps}
    for key in ("frac_of_active_sms", "alg_bytes_per_step"):
        if key in r:
            roofline[key] = r[key]
    if traffic and r.get("alg_bytes_per_step"):
        roofline["traffic_over_alg_bytes"] = traffic / r["alg_bytes_per_step"]
    # fraction of its roofline for every phase that has one
    phase_fracs = {}
    for i in range(names.index("tie_refine")):
        ri = roof(i)
        if ri.get("peak") and ri.get("achieved") is not None:
            phase_fracs[names[i]] = ri["achieved"] / ri["peak"]
    fr = roof(names.index("flush_gemm"))
    flush_roof = {"bound": fr["bound"], "achieved": fr["achieved"], "peak": fr["peak"],
                  "unit": fr["unit"], "frac": fr["achieved"] / fr["peak"],
                  "ms_per_step": phase_ms[3] / prof_steps, "peak_source": fr["peak_source"]}

    e2e = None
    if with_e2e:
        # through the public API with the result read back to the host every step:
        # the chains' state (tables, configurations, N) stays resident by design,
        # so no per-step input crosses to the device
        e2e_steps = steps
        acc_e0 = accepted_total()
        t_e2e = 0.0
        d2h = 0
        for _ in range(e2e_steps):
            t0 = time.perf_counter()
            ctx.sweep(1, measure=True, stream=sh)
            nb = 0
            for i in range(len(chains)):
                G, E, nm_ = ctx.measure_G(i)
                nb += 4 * G.nbytes + 3 * 8       # sums, squares, bin sums and squares, counts
            t_e2e += time.perf_counter() - t0
            d2h = nb
        acc_e = accepted_total() - acc_e0
        e2e = {"value": acc_e / t_e2e, "unit": UNIT, "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": d2h}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": total_ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if precision == pk.CTAUX_FP64 else "f32",
            "data": "synthetic",
            "precision": form,
            "order_n": {"mean": sum(orders) / len(orders), "min": int(min(orders)),
                        "max": int(max(orders))},
            "k_autotuned": k_tuned,
            "tiles_autotuned": tiles_tuned,
            "roofline": roofline, "flush_roofline": flush_roof,
            "phase_ms_per_step": {names[i]: phase_ms[i] / prof_steps for i in range(len(names))},
            "phase_pass_steps": prof_steps,
            "refreshes_in_timed_region": int(n_refreshes),
            "gpu_launches": kernels,
            "accept_rate": accept_rate,
            # per GPU; a sweep is one block (k_max proposals) of every chain
            "proposals_per_s": props / (total_ms / 1e3),
            "sweeps_per_s": steps * len(chains) / (total_ms / 1e3),
            "phase_roofline_frac": phase_fracs,
            "drift_max_last_refresh": max(ctx.stats(i)["last_drift_max"] for i in range(len(chains))),
            # the same relative to max |N| of each chain's fresh N
            "drift_rel_max_last_refresh": max(ctx.stats(i)["last_drift_rel"]
                                              for i in range(len(chains))),
            "near_ties": ties, "tie_refreshes": tie_refreshes,
            "clocks": clk}
    if measurement is not None:
        line["measurement"] = measurement
    if e2e is not None:
        line["e2e"] = e2e
    ctx.close()
    del flush
    torch.cuda.empty_cache()
    return {"line": line}


if __name__ == "__main__":
    main()

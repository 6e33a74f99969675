#!/usr/bin/env python
"""Benchmark of the exhaustive Gaussian-copula O-information path.

Workload: N=30 variables, T=1000 samples with planted redundancy and
synergy, every nplet of orders 3..30 (1,073,741,358 nplets), per-order
min/max/mean/count/top-256 reductions on the device.  A step is one full
pass: copula transform and covariance, enumeration, FP32 Cholesky with
leave-one-out log-determinants, FP64 re-factor of flagged nplets, combine,
reductions and merge.

Prints one JSON line.  `value` = nplets/s of the FP32 + FP64-fix path with
the sample matrix resident in HBM; `e2e` = the same through the public C ABI
from pinned host memory (upload of X and download of the records inside the
timed region).  Under torchrun every rank runs its own replica of the
workload (independent datasets, no collective on the data path).
"""
import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_VARS, T_SAMPLES = 30, 1000
ORDERS = list(range(3, 31))
TOP_M = 256
METRIC = "nplets/s exhaustive N=30 O-info (FP32+FP64 fix vs FP64), % of roofline"
WORKLOAD = ("planted-structure Gaussian copula, N=30, T=1000, all nplets of orders 3..30 "
            "(1,073,741,358), per-order min/max/mean/count/top-256 on device")


def flops_model(k: int) -> float:
    # Cholesky k^3/3 + triangular inverse k^3/3 + leave-one-out diagonal and
    # combine 2k^2 (an FMA counts 2)
    return 2.0 / 3.0 * k ** 3 + 2.0 * k ** 2


# DRAM bytes per nplet of the FP32 nplet kernels with records reduced inside
# them, from ncu captures on this workload (dram__bytes_read.sum +
# dram__bytes_write.sum of one launch / its nplets), each family at order 16
# (145,422,675 nplets), taken after the last change to these kernels.
# None: no capture of the current kernel.
TRAFFIC_BYTES_PER_NPLET = {"dense": 0.00089, "group": 0.00096, "prefix": 0.00099,
                           "prefix2": 0.00055, "prefix2_pair": 0.00062, "prefix3_pair": 0.00067,
                           "prefix4_pair": 0.00294}


def kernel_family(shape) -> str:
    lanes, _, prefix = (int(v) for v in shape)
    if prefix:
        return ("prefix", "prefix2", "prefix2_pair", "prefix3_pair", "prefix4_pair")[prefix - 1]
    return "group" if lanes > 1 else "dense"


def grad_flops_model(k: int) -> float:
    # forward factor and inverse (flops_model) + P = W^T W (k^3/3) +
    # Q = P diag(1/p) P (k^3) per nplet
    return flops_model(k) + k ** 3 / 3.0 + k ** 3


def prefix_level_flops(i: int) -> float:
    # one bordered step onto i factored variables: forward and backward
    # unit-triangular solves (i(i-1)/2 FMAs each), the new row and pivot
    # (i FMUL + i FMA) and the inverse-diagonal update (i FMUL + i FMA)
    return 2.0 * i * (i - 1) + 6.0 * i


def prefix_order_flops(N: int, k: int) -> float:
    # prefix-shared kernel: every (k-1)-prefix is built once (levels
    # 0..k-2), every nplet is one final bordered step plus the product of its
    # k inverse-diagonal entries
    P = k - 1
    per_prefix = sum(prefix_level_flops(i) for i in range(P))
    per_nplet = prefix_level_flops(P) + 2.0 * P
    return math.comb(N - 1, P) * per_prefix + math.comb(N, k) * per_nplet


def prefix2_order_flops(N: int, k: int) -> float:
    # two-level prefix-shared kernel: every (k-2)-prefix built once, one
    # stored bordered step per (k-1)-prefix, one final step per nplet
    GP = k - 2
    per_grand = sum(prefix_level_flops(i) for i in range(GP))
    per_middle = prefix_level_flops(GP)
    per_nplet = prefix_level_flops(k - 1) + 2.0 * (k - 1)
    return (math.comb(N - 2, GP) * per_grand + math.comb(N - 1, k - 1) * per_middle +
            math.comb(N, k) * per_nplet)


def prefix4_order_flops(N: int, k: int) -> float:
    # four-level prefix-shared kernel: every (k-4)-prefix built once, one
    # stored bordered step per (k-3)-, (k-2)- and (k-1)-prefix, one final
    # step per nplet
    IP = k - 4
    per_i = sum(prefix_level_flops(i) for i in range(IP))
    return (math.comb(N - 4, IP) * per_i + math.comb(N - 3, k - 3) * prefix_level_flops(IP) +
            math.comb(N - 2, k - 2) * prefix_level_flops(k - 3) +
            math.comb(N - 1, k - 1) * prefix_level_flops(k - 2) +
            math.comb(N, k) * (prefix_level_flops(k - 1) + 2.0 * (k - 1)))


def prefix3_order_flops(N: int, k: int) -> float:
    # three-level prefix-shared kernel: every (k-3)-prefix built once, one
    # stored bordered step per (k-2)-prefix and per (k-1)-prefix, one final
    # step per nplet
    HP = k - 3
    per_h = sum(prefix_level_flops(i) for i in range(HP))
    return (math.comb(N - 3, HP) * per_h + math.comb(N - 2, k - 2) * prefix_level_flops(HP) +
            math.comb(N - 1, k - 1) * prefix_level_flops(k - 2) +
            math.comb(N, k) * (prefix_level_flops(k - 1) + 2.0 * (k - 1)))


def order_flops(N: int, k: int, prefix: int) -> float:
    # prefix 3 is the two-level kernel with the last variables two at a time:
    # the same algorithmic work as prefix 2
    if prefix in (2, 3):
        return prefix2_order_flops(N, k)
    if prefix == 4:
        return prefix3_order_flops(N, k)
    if prefix == 5:
        return prefix4_order_flops(N, k)
    return prefix_order_flops(N, k) if prefix else math.comb(N, k) * flops_model(k)


def total_nplets(N=N_VARS, orders=ORDERS):
    return sum(math.comb(N, k) for k in orders)


def total_flops(N=N_VARS, orders=ORDERS):
    return sum(math.comb(N, k) * flops_model(k) for k in orders)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-path comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the adjoint and multi-dataset measurements")
    ap.add_argument("--only-order", type=int, default=0,
                    help="profiling aid: run the per-order reduction of one order a few "
                         "times and exit (for ncu captures of one kernel)")
    ap.add_argument("--precision", default="f32_fix64", choices=["f32_fix64", "f64"],
                    help="precision of the --only-order runs")
    ap.add_argument("--shape", default="",
                    help="--only-order runs: launch shape 'lanes,chunk,prefix' (else built-in)")
    return ap.parse_args()


def run_only_order(args, local_rank):
    import torch

    import paper_2501_03381_gb300 as P
    import workloads
    torch.cuda.set_device(local_rank)
    P.load(build_if_missing=False)
    X, _ = workloads.planted30()
    with P.Context(torch.as_tensor(X, device="cuda"), precision=args.precision, top_m=TOP_M,
                   profile=True) as c:
        if args.shape:
            # load one launch shape for this order through the autotuner's cache file
            lanes, chunk, prefix = (int(v) for v in args.shape.split(","))
            props = torch.cuda.get_device_properties(local_rank)
            ent = {"gpu": props.name, "sms": props.multi_processor_count, "k": args.only_order,
                   "wide": 0, "lanes": lanes, "chunk": chunk, "blocks_per_sm": 0,
                   "prefix": prefix}
            path = os.path.join(tempfile.gettempdir(), f"thoi_shape_{os.getpid()}.json")
            with open(path, "w") as fh:
                fh.write("[\n" + json.dumps(ent) + "\n]\n")
            P.thoi_autotune(c.h, args.only_order, args.only_order, path)
        for _ in range(max(1, args.steps)):
            (recs, _, _), st = c.measures([args.only_order], reduction="per_order")
    torch.cuda.synchronize()
    print(json.dumps({"order": args.only_order, "precision": args.precision,
                      "nplet_ms": st.nplet_ms, "refactor_ms": st.refactor_ms,
                      "merge_ms": st.merge_ms, "count": int(recs[0]["count"])}))
    return 0


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------ oracle baseline
def cpu_model() -> str:
    """The host CPU's model as /proc/cpuinfo names it (x86: "model name"; Arm:
    implementer and part numbers, with the part named where it is known)."""
    fields = {}
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields.setdefault(k.strip(), v.strip())
    except OSError:
        return "unknown"
    if "model name" in fields:
        return fields["model name"]
    parts = {"0xd4f": "Neoverse V2 (Grace)", "0xd40": "Neoverse V1", "0xd0c": "Neoverse N1"}
    imp, part = fields.get("CPU implementer", "?"), fields.get("CPU part", "?")
    return f"Arm implementer {imp} part {part}" + (f" = {parts[part]}" if part in parts else "")


def cpu_baseline(seconds: float, seed: int = 0, one_thread_seconds: float = 0.0):
    """The FP64 oracle as it stands, on a uniform random sample of the
    workload's nplet ids, on every host core (and, when one_thread_seconds >
    0, on one thread over a smaller sample of the same draw).  The rate of
    the whole workload is extrapolated from the sample: ids are drawn
    uniformly, so the sample's mix of orders is the workload's."""
    import numpy as np

    import oracle
    import workloads
    X, orders = workloads.planted30()
    S = oracle.copula_cov(X)
    total = total_nplets()
    rng = np.random.default_rng(seed)
    pilot = np.sort(rng.integers(0, total, 4000, dtype=np.uint64))
    t0 = time.perf_counter()
    oracle.measures_ids(S, orders, pilot)
    dt = time.perf_counter() - t0
    n = int(max(4000, min(5e7, 4000 * seconds / max(dt, 1e-6))))
    ids = np.sort(rng.integers(0, total, n, dtype=np.uint64))
    t0 = time.perf_counter()
    oracle.measures_ids(S, orders, ids)
    dt = time.perf_counter() - t0
    cores = os.cpu_count()
    out = {"value": n / dt, "unit": "nplets/s", "cores": cores, "kind": "oracle",
           "cpu_model": cpu_model(), "extrapolated": True,
           "sample": f"{n} nplet ids drawn uniformly (seed {seed}) from the "
                     f"{total:,} nplets; FP64 LU per subset and per leave-one-out subset; "
                     f"{dt:.1f} s on {cores} OpenMP threads; the rate of the whole workload "
                     f"is this sample's rate"}
    if one_thread_seconds > 0:
        n1 = int(max(500, min(n, n / dt / cores * one_thread_seconds)))
        ids1 = ids[rng.permutation(n)[:n1]]
        ids1.sort()
        t0 = time.perf_counter()
        oracle.measures_ids(S, orders, ids1, nthreads=1)
        d1 = time.perf_counter() - t0
        out["one_thread"] = {"value": n1 / d1, "unit": "nplets/s", "sample": f"{n1} of those ids",
                             "seconds": d1}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    per_step_s = max(5.0, 150.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_baseline(min(per_step_s, 5.0), seed=1000)
    vals, times = [], []
    for s in range(args.steps):
        cb = cpu_baseline(per_step_s, seed=s)
        vals.append(cb["value"])
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "nplets/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_nplets() / v * 1e3, "ms_per_step_extrapolated": True,
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N_VARS, "T": T_SAMPLES, "orders": "3..30",
                       "top_m": TOP_M},
            "cpu_baseline": {"value": v, "unit": "nplets/s", "cores": os.cpu_count(),
                             "kind": "oracle", "cpu_model": cb["cpu_model"],
                             "extrapolated": True,
                             "sample": cb["sample"] + "; each step a bounded sample, its time "
                                       "scaled to the whole workload"},
            "e2e": {"value": v, "unit": "nplets/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ ours
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_2501_03381_gb300 as P
    import workloads

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    P.load(build_if_missing=False)
    X = workloads.planted(T_SAMPLES, seed=2 + 7919 * rank)  # replica per rank
    Xd = torch.as_tensor(X, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    nb = P.thoi_records_bytes(len(ORDERS), TOP_M)
    rec_dev = torch.zeros(nb, dtype=torch.uint8, device=dev)
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count

    def one_step(opt):
        h = P.thoi_create(Xd, opt)
        try:
            _, st = P.thoi_measures(h, ORDERS, 0, None, P.THOI_RED_PER_ORDER, rec_dev,
                                    top_m=TOP_M)
        finally:
            P.thoi_destroy(h)
        return st

    def timed(opt, steps, warmup):
        for _ in range(warmup):
            one_step(opt)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms, nplet_ms, ref_ms, launches, nref = [], [], [], 0, 0
        for _ in range(steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            st = one_step(opt)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            nplet_ms.append(st.nplet_ms)
            ref_ms.append(st.refactor_ms)
            launches += st.launches + 6  # + the six copula-stage kernels of thoi_create
            nref = st.n_refactored
        if dist:
            dist.barrier()
        return ms, nplet_ms, ref_ms, launches, nref

    opt32 = P.make_options(top_m=TOP_M, profile=True)
    # launch shapes per order, tuned on this GPU before the timed region
    tune_path = os.path.join(tempfile.gettempdir(), f"thoi_tune_{os.getpid()}.json")
    h = P.thoi_create(Xd, opt32)
    try:
        P.thoi_autotune(h, 3, N_VARS, tune_path)
    finally:
        P.thoi_destroy(h)
    try:
        # the shapes the records path uses (the cache also holds the
        # per-nplet output ones, "out": 1)
        shapes = {e["k"]: [e["lanes"], e["chunk"], e.get("prefix", 0)]
                  for e in json.load(open(tune_path)) if not e.get("out", 0)}
    except Exception:
        shapes = {}
    # measured FFMA and DFMA peaks of this GPU (self-written multiply-add
    # chains): the FP32 one cross-checks the derived peak below, the FP64 one
    # is the denominator of the FP64 rooflines
    fma32, _ = P.thoi_fma_peak(False)
    fma64, _ = P.thoi_fma_peak(True)
    sampler = ClockSampler(local_rank)
    sampler.start()
    ms, nplet_ms, ref_ms, launches, nref = timed(opt32, args.steps, args.warmup)
    clocks = sampler.stop()
    t_step = sum(ms) / len(ms)
    if dist:
        t = torch.tensor([t_step], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_step = float(t.item())
    n_total = total_nplets() * world
    value = n_total / (t_step / 1e3)

    # FP64 path on the same workload (the comparison named by the metric)
    fp64 = None
    if not args.no_fp64:
        opt64 = P.make_options(precision="f64", top_m=TOP_M, profile=True)
        ms64, nms64, _, _, _ = timed(opt64, 1, 1)
        fp64 = {"ms_per_step": ms64[0], "nplets_per_s": total_nplets() / (ms64[0] / 1e3),
                "nplet_kernel_ms": nms64[0],
                "speedup_fp32fix_over_fp64": ms64[0] / t_step}

    # end to end through the public API from pinned host memory
    Xh = torch.as_tensor(X).pin_memory()
    rec_h = torch.zeros(nb, dtype=torch.uint8).pin_memory()

    def e2e_step():
        h = P.thoi_create(Xh, opt32)
        try:
            P.thoi_measures(h, ORDERS, 0, None, P.THOI_RED_PER_ORDER, rec_h.numpy(), top_m=TOP_M)
        finally:
            P.thoi_destroy(h)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e2e_t = []
    for _ in range(max(3, args.steps // 2)):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = sum(e2e_t) / len(e2e_t)

    # roofline of the dominant kernels (the FP32 nplet kernels of all orders),
    # each order counted with the work of the kernel the autotuner chose
    f_total = sum(order_flops(N_VARS, k, int(shapes.get(k, [1, 8, 0])[2])) for k in ORDERS)
    f_dense = total_flops()
    traffic = 0.0
    for k in ORDERS:
        b = TRAFFIC_BYTES_PER_NPLET[kernel_family(shapes.get(k, [1, 8, 0]))]
        traffic = None if (traffic is None or b is None) else traffic + b * math.comb(N_VARS, k)
    kern_s = sum(nplet_ms) / len(nplet_ms) / 1e3
    achieved = f_total / kern_s / 1e12
    sm_max = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "nplets/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N_VARS, "T": T_SAMPLES, "orders": "3..30",
                   "top_m": TOP_M, "precision": "fp32 Cholesky + fp64 re-factor",
                   "l2": "flushed between timed steps (256 MiB write)",
                   "replicas": "one independent dataset per rank",
                   "tuned_shapes_k_lanes_chunk": shapes},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": traffic,
                     "traffic_basis": "per-step DRAM bytes of the FP32 nplet kernels, scaled by "
                                      "nplets from ncu captures of each kernel family at "
                                      f"order 16 (B per nplet: {TRAFFIC_BYTES_PER_NPLET})",
                     "kernel": "FP32 nplet kernels with the records reduced inside (k_nplet_reg, "
                               "k_nplet_grp, k_nplet_pfx, k_nplet_pfx2), CUDA events",
                     "flops_per_step": f_total, "kernel_ms_per_step": kern_s * 1e3,
                     "flops_model": "dense orders 2/3k^3+2k^2 per nplet; prefix-shared orders "
                                    "(tuned_shapes third entry 1) one bordered build per "
                                    "(k-1)-prefix plus one bordered step per nplet; entry 2: "
                                    "one build per (k-2)-prefix, one stored step per "
                                    "(k-1)-prefix, one final step per nplet (entry 3 the "
                                    "same); entry 4: one build per (k-3)-prefix, one "
                                    "stored step per (k-2)- and per (k-1)-prefix, one "
                                    "final step per nplet; entry 5: one build per "
                                    "(k-4)-prefix, one stored step per (k-3)-, (k-2)- and "
                                    "(k-1)-prefix, one final step per nplet",
                     "dense_equivalent_tflops": f_dense / kern_s / 1e12,
                     "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz",
                     "peak_measured_ffma_tflops": fma32,
                     "peak_measured_dfma_tflops": fma64},
        "e2e": {"value": n_total / e2e_s, "unit": "nplets/s",
                "h2d_bytes_per_step": int(X.nbytes), "d2h_bytes_per_step": int(nb)},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "refactored_per_step": int(nref),
        "refactor_ms_per_step": sum(ref_ms) / len(ref_ms),
        "fp64_path": fp64,
    }
    if not args.no_extra:
        line["other_workloads"] = run_extra(args, dev, stream, flush, peak, rank, fma64)
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds, one_thread_seconds=3.0)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0

# ------------------------------------------------------------------ adjoint and batching
def run_extra(args, dev, stream, flush, peak, rank, fp64_peak):
    """The adjoint (N=60, T=2000, orders 3..5), the 64-dataset batch
    (N ~ U{10..40}, T ~ U{200..2000}, orders 3..min(N,8)) and the greedy
    search (N=60, orders 3..20), each timed with CUDA events after warm-up,
    with its roofline and the oracle beside it (rank 0)."""
    import numpy as np
    import torch

    import paper_2501_03381_gb300 as P
    import workloads
    out = {}
    steps = max(3, args.steps)

    def ev_time(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sum(ts) / len(ts)

    # adjoint: dL/dSigma of L = sum of O over every nplet of orders 3..5
    X, orders = workloads.grad60()
    Nv = X.shape[1]
    G = torch.empty((Nv, Nv), dtype=torch.float32, device=dev)
    with P.Context(torch.as_tensor(X, device=dev)) as c:
        ms = ev_time(lambda: P.thoi_measures_grad(c.h, orders, "O", out=G))
    n = total_nplets(Nv, orders)
    fl = sum(math.comb(Nv, k) * grad_flops_model(k) for k in orders)
    ach = fl / (ms / 1e3) / 1e12
    entry = {"workload": "N=60, T=2000 random-correlation Gaussian, L = sum of O over orders "
                         "3..5 (5,983,367 nplets), dL/dSigma (60x60) with the FP64 re-factor",
             "value": n / (ms / 1e3), "unit": "nplets/s", "ms_per_call": ms,
             "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                          "frac": ach / peak, "flops_per_call": fl,
                          "flops_model": "2/3k^3+2k^2 forward + 4/3k^3 adjoint per nplet"}}
    if rank == 0 and not args.no_cpu:
        import oracle
        S = oracle.copula_cov(X)
        t0 = time.perf_counter()
        oracle.grad(S, orders, "O")
        dt = time.perf_counter() - t0
        entry["cpu_baseline"] = {"value": n / dt, "unit": "nplets/s", "cores": os.cpu_count(),
                                 "kind": "oracle",
                                 "sample": f"the whole workload ({n:,} nplets), {dt:.2f} s"}
    out["adjoint_grad60"] = entry

    # 64 datasets through one graph of batched launches
    Xs, ords = workloads.multi64()
    ctxs = [P.Context(torch.as_tensor(Xd, device=dev), top_m=TOP_M) for Xd in Xs]
    prof = P.Context(torch.as_tensor(Xs[0], device=dev), top_m=TOP_M, profile=True)
    hs = [prof.h] + [c.h for c in ctxs[1:]]
    try:
        ms = ev_time(lambda: P.thoi_batch_measures(hs, 3, 8, top_m=TOP_M))
        _, st = P.thoi_batch_measures(hs, 3, 8, top_m=TOP_M)
        graph_ms = st.nplet_ms
        launches = st.launches
        nplet_launches = st.nplet_launches
    finally:
        for c in ctxs + [prof]:
            c.close()
    n = sum(math.comb(Xd.shape[1], k) for Xd, o in zip(Xs, ords) for k in o)
    fl = sum(math.comb(Xd.shape[1], k) * flops_model(k) for Xd, o in zip(Xs, ords) for k in o)
    ach = fl / (graph_ms / 1e3) / 1e12
    entry = {"workload": "64 datasets, N ~ U{10..40}, T ~ U{200..2000} (seeds 3000+d), orders "
                         f"3..min(N,8) ({n:,} nplets), per-order records with top-256 lists, "
                         "one replayed CUDA graph around one persistent nplet launch",
             "value": n / (ms / 1e3), "unit": "nplets/s", "ms_per_call": ms,
             "graph_ms": graph_ms, "gpu_launches_per_call": launches,
             "nplet_launches_per_call": nplet_launches,
             "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                          "frac": ach / peak, "flops_per_call": fl,
                          "kernel": "whole graph (nplet, reduction, re-factor, merge)"}}
    if rank == 0 and not args.no_cpu:
        import oracle
        rng = np.random.default_rng(5)
        counts = [sum(math.comb(Xd.shape[1], k) for k in o) for Xd, o in zip(Xs, ords)]
        m = 400000
        done, dt = 0, 0.0
        for Xd, o, cnt in zip(Xs, ords, counts):
            q = max(1, int(round(m * cnt / n)))
            ids = np.sort(rng.integers(0, cnt, q, dtype=np.uint64))
            S = oracle.copula_cov(Xd)
            t0 = time.perf_counter()
            oracle.measures_ids(S, o, ids)
            dt += time.perf_counter() - t0
            done += q
        entry["cpu_baseline"] = {"value": done / dt, "unit": "nplets/s", "cores": os.cpu_count(),
                                 "kind": "oracle",
                                 "sample": f"{done} nplet ids drawn uniformly per dataset "
                                           f"(seed 5), in proportion to its nplets; {dt:.2f} s"}
    out["multi_dataset_64"] = entry

    # greedy search (Methods, "Greedy Algorithm"): N=60, from the exhaustive
    # top-256 triplets up to order 20, maximising O; FP64 evaluation
    X, _ = workloads.grad60()
    Nv = X.shape[1]
    k0, k1, kappa = 3, 20, 256
    with P.Context(torch.as_tensor(X, device=dev)) as c:
        ms = ev_time(lambda: P.thoi_greedy(c.h, k0, k1, kappa, "O", True))
        masks, values, st = P.thoi_greedy(c.h, k0, k1, kappa, "O", True)
    n_eval = int(st.nplets)
    # FP64 work: the exhaustive order k0 plus the distinct candidates of each
    # later order (at most kappa * (N - k + 1) of them)
    fl = math.comb(Nv, k0) * flops_model(k0)
    rest = n_eval - math.comb(Nv, k0)
    per_order = rest / (k1 - k0) if k1 > k0 else 0
    fl += sum(per_order * flops_model(k) for k in range(k0 + 1, k1 + 1))
    ach = fl / (ms / 1e3) / 1e12
    entry = {"workload": f"N=60, T=2000 random-correlation Gaussian; greedy search maximising O "
                         f"from the exhaustive top-{kappa} of order {k0} to order {k1} "
                         f"({n_eval:,} FP64 evaluations)",
             "value": n_eval / (ms / 1e3), "unit": "nplets/s", "ms_per_call": ms,
             "best_O_at_k1": float(values[-1][0]),
             "roofline": {"bound": "fp64", "achieved": ach, "peak": fp64_peak,
                          "unit": "TFLOP/s", "frac": ach / fp64_peak,
                          "peak_basis": "measured DFMA peak (thoi_fma_peak)",
                          "flops_model": "2/3k^3+2k^2 per evaluated nplet (evaluations "
                                         "spread evenly over the expanded orders)"}}
    if rank == 0 and not args.no_cpu:
        import oracle
        S = oracle.copula_cov(X)
        t0 = time.perf_counter()
        ref = oracle.greedy(S, k0, k1, kappa, "O", True)
        dt = time.perf_counter() - t0
        same = all(
            [tuple(i for i in range(64) if int(x) >> i & 1) for x in masks[lv, :len(sets)]] == sets
            for lv, (sets, _) in enumerate(ref))
        entry["cpu_baseline"] = {"value": n_eval / dt, "unit": "nplets/s",
                                 "cores": os.cpu_count(), "kind": "oracle",
                                 "sample": f"the whole search, {dt:.2f} s",
                                 "same_selection": bool(same)}
    out["greedy_grad60"] = entry

    # simulated annealing (Methods, "Simulated Annealing Algorithm"): N=60,
    # 4096 chains of 1000 steps over orders 3..20, maximising O, FP64 energies
    klo, khi, chains, iters, T0, alpha = 3, 20, 4096, 1000, 0.2, 0.996
    with P.Context(torch.as_tensor(X, device=dev)) as c:
        ms = ev_time(lambda: P.thoi_anneal(c.h, klo, khi, chains, iters, T0, alpha, "O", True, 1))
        fm, fv, bm, bv, st = P.thoi_anneal(c.h, klo, khi, chains, iters, T0, alpha, "O", True, 1)
    n_eval = int(st.nplets)
    sizes = [bin(int(m)).count("1") for m in fm]
    kbar = sum(sizes) / len(sizes)
    fl = n_eval * flops_model(kbar)
    ach = fl / (ms / 1e3) / 1e12
    entry = {"workload": f"N=60, T=2000 random-correlation Gaussian; {chains} annealing chains x "
                         f"{iters} steps over orders {klo}..{khi}, maximising O "
                         f"({n_eval:,} FP64 energies)",
             "value": n_eval / (ms / 1e3), "unit": "nplets/s", "ms_per_call": ms,
             "best_O": float(max(bv)), "accepted": int(st.n_refactored),
             "roofline": {"bound": "fp64", "achieved": ach, "peak": fp64_peak,
                          "unit": "TFLOP/s", "frac": ach / fp64_peak,
                          "peak_basis": "measured DFMA peak (thoi_fma_peak)",
                          "flops_model": f"2/3k^3+2k^2 per energy at the mean final order "
                                         f"{kbar:.1f}"}}
    if rank == 0 and not args.no_cpu:
        import oracle
        S = oracle.copula_cov(X)
        n_ref = 4
        t0 = time.perf_counter()
        ref = oracle.anneal(S, klo, khi, n_ref, iters, T0, alpha, "O", True, 1)
        dt = time.perf_counter() - t0
        same = [tuple(i for i in range(64) if int(m) >> i & 1) for m in bm[:n_ref]] == ref[2]
        entry["cpu_baseline"] = {"value": n_ref * (iters + 1) / dt, "unit": "nplets/s",
                                 "cores": 1, "kind": "oracle",
                                 "sample": f"the first {n_ref} chains ({n_ref * (iters + 1)} "
                                           f"energies), {dt:.2f} s, one thread",
                                 "same_best_sets": bool(same)}
    out["anneal_grad60"] = entry

    # group objectives over datasets (Results, "Leveraging Gaussian entropy
    # estimators with batch processing"; Methods, "fMRI analysis"): 16
    # subjects x 2 conditions, N = 55, the paired Cohen's d of O
    Xs, orders = workloads.paired55()
    Nv, D = Xs[0].shape[1], len(Xs)
    ctxs = [P.Context(torch.as_tensor(Xd, device=dev), top_m=TOP_M) for Xd in Xs]
    try:
        # launch shapes of N = 55 (wide masks) tuned before the timed region
        P.thoi_autotune(ctxs[0].h, min(orders), max(orders))
        ms = ev_time(lambda: P.thoi_group_measures(ctxs, orders, "O", "cohen_d",
                                                   kind=P.THOI_RED_PER_ORDER, top_m=TOP_M))
        (recs, hi, lo), st = P.thoi_group_measures(ctxs, orders, "O", "cohen_d",
                                                   kind=P.THOI_RED_PER_ORDER, top_m=TOP_M)
        launches = int(st.launches)
        k0, k1, kappa = 3, 20, 128
        gms = ev_time(lambda: P.thoi_group_greedy(ctxs, k0, k1, kappa, "O", "cohen_d", True))
        gmasks, gvals, gst = P.thoi_group_greedy(ctxs, k0, k1, kappa, "O", "cohen_d", True)
        klo, khi, chains, iters = 3, 12, 1024, 200
        sms = ev_time(lambda: P.thoi_group_anneal(ctxs, klo, khi, chains, iters, 0.5, 0.98, "O",
                                                  "cohen_d", True, 1))
        fm, fv, bm, bv, sst = P.thoi_group_anneal(ctxs, klo, khi, chains, iters, 0.5, 0.98, "O",
                                                  "cohen_d", True, 1)
    finally:
        for c in ctxs:
            c.close()
    n = total_nplets(Nv, orders)
    fl = D * sum(math.comb(Nv, k) * flops_model(k) for k in orders)
    ach = fl / (ms / 1e3) / 1e12
    entry = {"workload": f"16 subjects x 2 conditions (paired), N=55, T=300 (block-structured "
                         f"AR(1) stand-in), paired Cohen's d of O over orders 3..6 ({n:,} "
                         f"nplets x {D} datasets), per-order records with top-{TOP_M} lists",
             "value": n / (ms / 1e3), "unit": "nplets/s", "ms_per_call": ms,
             "dataset_evaluations_per_s": D * n / (ms / 1e3), "gpu_launches_per_call": launches,
             "max_d": [float(r["max"][3]) for r in recs],
             "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                          "frac": ach / peak, "flops_per_call": fl,
                          "flops_model": "2/3k^3+2k^2 per nplet per dataset (FP32 path); "
                                         "the combine and reduction kernels add no FLOP term"}}
    if rank == 0 and not args.no_cpu:
        import oracle
        Ss = [oracle.copula_cov(Xd) for Xd in Xs]
        rng = np.random.default_rng(6)
        m = 20000
        ids = np.sort(rng.integers(0, n, m, dtype=np.uint64))
        t0 = time.perf_counter()
        oracle.group_measures_ids(Ss, orders, "O", "cohen_d", ids)
        dt = time.perf_counter() - t0
        entry["cpu_baseline"] = {"value": m / dt, "unit": "nplets/s", "cores": os.cpu_count(),
                                 "kind": "oracle",
                                 "sample": f"{m} nplet ids drawn uniformly (seed 6), each in all "
                                           f"{D} datasets; {dt:.2f} s"}
    out["group_cohen_paired55"] = entry
    n_eval = int(gst.nplets)
    entry = {"workload": f"the paired N=55 workload; greedy search maximising the paired "
                         f"Cohen's d of O from the exhaustive top-{kappa} of order {k0} to "
                         f"order {k1} ({n_eval:,} FP64 evaluations over {D} datasets)",
             "value": n_eval / (gms / 1e3), "unit": "evaluations/s", "ms_per_call": gms,
             "best_d_at_k1": float(gvals[-1][0])}
    if rank == 0 and not args.no_cpu:
        import oracle
        Ss = [oracle.copula_cov(Xd) for Xd in Xs]
        t0 = time.perf_counter()
        ref = oracle.greedy(Ss, k0, min(k1, 5), kappa, "O", True, objective="cohen_d")
        dt = time.perf_counter() - t0
        same = all(
            [tuple(i for i in range(64) if int(x) >> i & 1) for x in gmasks[lv, :len(sets)]]
            == sets for lv, (sets, _) in enumerate(ref))
        ev_ref = D * (math.comb(Nv, k0) + sum(
            len({tuple(sorted(s_ + (v,))) for s_ in ref[lv - 1][0] for v in range(Nv)
                 if v not in s_}) for lv in range(1, len(ref))))
        entry["cpu_baseline"] = {"value": ev_ref / dt, "unit": "evaluations/s",
                                 "cores": os.cpu_count(), "kind": "oracle",
                                 "sample": f"orders {k0}..{min(k1, 5)} of the search, {dt:.2f} s",
                                 "same_selection": bool(same)}
    out["group_greedy_paired55"] = entry
    n_eval = int(sst.nplets)
    entry = {"workload": f"the paired N=55 workload; {chains} annealing chains x {iters} steps "
                         f"over orders {klo}..{khi} maximising the paired Cohen's d of O "
                         f"({n_eval:,} FP64 evaluations over {D} datasets)",
             "value": n_eval / (sms / 1e3), "unit": "evaluations/s", "ms_per_call": sms,
             "best_d": float(np.nanmax(bv)), "accepted": int(sst.n_refactored)}
    out["group_anneal_paired55"] = entry

    # per-nplet output (FP32 SoA, 20 B per nplet) at small orders, where the
    # stores outweigh the arithmetic (F(k) / 20 B is below the FP32 : HBM
    # balance of about 12 FLOP/B for k <= 6): N = 64, orders 3..6, the nplet
    # kernels' CUDA-event time against the measured HBM bandwidth
    try:
        Nv, orders_o = 64, [3, 4, 5, 6]
        rng = np.random.default_rng(7)
        Xo = rng.standard_normal((2000, Nv)) @ np.linalg.cholesky(
            workloads.random_corr(rng, Nv)).T
        n = total_nplets(Nv, orders_o)
        out_t = torch.empty((5, n), dtype=torch.float32, device=dev)
        with P.Context(torch.as_tensor(Xo, device=dev), profile=True) as c:
            for _ in range(3):
                c.measures(orders_o, out=out_t)
            kms = []
            for _ in range(steps):
                flush.fill_(1)
                torch.cuda.synchronize()
                _, st = c.measures(orders_o, out=out_t)
                kms.append(st.nplet_ms)
        kms_avg = sum(kms) / len(kms)
        hbm = 6800.0
        basis = "fallback 6.8 TB/s"
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
                hbm = float(json.load(fh)["hbm_gbs"])
            basis = "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
        except Exception:
            pass
        byts = 20.0 * n
        ach = byts / (kms_avg / 1e3) / 1e9
        entry = {"workload": f"N=64, T=2000 random-correlation Gaussian (seed 7), per-nplet FP32 "
                             f"output of orders 3..6 ({n:,} nplets, {byts / 1e6:.0f} MB)",
                 "value": n / (kms_avg / 1e3), "unit": "nplets/s",
                 "nplet_kernel_ms": kms_avg,
                 "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                              "frac": ach / hbm, "bytes_per_call": byts,
                              "peak_basis": basis,
                              "bytes_model": "20 B written per nplet (five FP32 measures)"}}
    except Exception as e:  # an extra line never takes the headline down
        entry = {"error": f"{type(e).__name__}: {e}"}
    out["per_nplet_output_n64"] = entry
    return out


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.only_order:
        return run_only_order(args, local_rank)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())

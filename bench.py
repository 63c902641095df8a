#!/usr/bin/env python3
"""Throughput of U = sign(T) on GB300: useful GFLOP/s (the oracle's flop count
of Algorithm 3) at n = 16384, p = 0.5 (random interleaved diagonal signs,
|t_ii| ~ U[0.5, 2], strictly-upper N(0, 1/n)), seed = rank.

One step = one sign_tri call on a resident input: inertia scan, variant
choice, and the chosen variant's kernels.  The input (2.1 GB) and output are
each larger than L2 (129 MB), so no flush is needed between steps.

The headline is the mixed-precision form with refinement (PH_MIXED_FP16:
tensor-core block sums on a two-term fp16 split, fp32 leaves, float64 defect
correction with emulated-float64 residuals); the three-term bf16 split
(PH_MIXED_TF32) and the float64 forms (PH_FP64_EFFICIENT, PH_FP64) are timed
on the same input for the comparison the metric names, and all are checked
against the oracle on the leading and trailing 4096 principal windows.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--variant V]
    python bench.py --impl reference      # the CPU oracle, the reference arm

Under torchrun (N > 1) every rank solves its own replica (the method does
not shard a single matrix); value = total useful flops / max-over-ranks time.
"""
import argparse
import hashlib
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

METRIC = "sign(T) seconds & useful GFLOP/s at n=16384: mixed+refine vs FP64, ≤1e-12 err"
UNIT = "GFLOP/s"

# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch
# of a kernel class, averaged over the class's launches of one solve, from
# one capture of this script's workload (summarised under profiles/),
# keyed by (class, sha256 of the kernel and job-list sources, n, p, order,
# variant): reported only while those sources are unchanged and for that
# workload, else null.  The capture serialises launches, so classes whose
# launches run side by side in the timed solve (the sweeps' look-ahead
# pairs, which share operand panels through L2) read more there than here.
TRAFFIC_SOURCES = ("paper_1607_06303_gb300/csrc/tc_gemm.cu", "paper_1607_06303_gb300/csrc/mixed.cu")
TRAFFIC = {
    # n = 16384, p = 0.5 random, PH_MIXED_FP16 (profiles/launches_mixed_n16384.txt)
    ("residual", "27e20e3a768f7905"): 35.556e9,
    ("block_sums_tc", "27e20e3a768f7905"): 638.9e6,
}


def traffic_key(cls, n, p, order, variant):
    h = hashlib.sha256()
    for rel in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    h.update(("%d %g %s %s" % (n, p, order, variant)).encode())
    return (cls, h.hexdigest()[:16])


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--p", type=float, default=0.5)
    ap.add_argument("--order", default="random")
    ap.add_argument("--variant", default="PH_MIXED_FP16")
    ap.add_argument("--compare", default="PH_MIXED_TF32,PH_FP64_EFFICIENT,PH_FP64",
                    help="comma-separated variants timed beside the headline on the same input ('' to skip)")
    ap.add_argument("--cutoff", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=4096,
                    help="order of the leading principal window the oracle solves")
    ap.add_argument("--workload", choices=["single", "batched", "general"], default="single",
                    help="batched: 2000 problems, n log-uniform in [32, 2048], p ~ U[0,1], random order; "
                         "general: sign(A) of a general real A (--n), through the GPU Schur decomposition")
    ap.add_argument("--batch", type=int, default=2000)
    return ap.parse_args(argv)


# ---------------------------------------------------------------- clocks ---
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        sm, smax, reasons, power = [], [], set(), []
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1].split()[0]))
                    smax.append(float(parts[2].split()[0]))
                    power.append(float(parts[3].split()[0]))
                except ValueError:
                    continue
                for name, val in zip(names[1:], parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------- reference ---
def run_reference(args, rank):
    """The CPU oracle (Algorithm 3, OpenMP anti-diagonal schedule) on the
    leading principal window of the same input: a bounded sample of the
    workload with the same structure (u_ij of a window depends on the window
    only)."""
    if rank != 0:
        return None
    import numpy as np

    import oracle
    from paper_1607_06303_gb300 import workload
    from paper_1607_06303_gb300.inputs import make_T
    m = min(args.cpu_sample if args.cpu_sample else 3072, args.n)
    T = make_T(args.n, args.p, seed=0, order=args.order)
    Tw = np.asfortranarray(T[:m, :m])
    flops = workload.useful_flops(np.sign(np.diag(Tw)))
    threads = oracle.max_threads()
    for _ in range(args.warmup):
        oracle.sign_tri(Tw, schedule="antidiag", threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sign_tri(Tw, schedule="antidiag", threads=threads)
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    val = flops / dt / 1e9
    sample = "leading %dx%d principal window of the n=%d input (%.3g useful flops/step)" % (m, m, args.n, flops)
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "sign(T) n=%d p=%g %s, seed 0; oracle on a %d-window" % (args.n, args.p, args.order, m),
                   "n": args.n, "p": args.p, "order": args.order},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        # the two arms run different sizes: their rates compare, their seconds
        # do not; a full-size time at the sample's rate is given for context
        "comparison": "useful-GFLOP/s rates (the oracle on a %d-window sample, the GPU on n=%d); "
                      "seconds are not comparable" % (m, args.n),
        "extrapolated_seconds_per_solve": workload.useful_flops(np.sign(np.diag(T))) / (val * 1e9),
    }
    return line


# ------------------------------------------------------------------- ours ---
def block_sum_flops(n, b):
    """Algorithmic flops of all block-sum launches of one call: 6 flops per
    (row, k, column) triple with k in the K-blocks strictly between the row
    and column blocks (the matrix-multiply form of Section 5.3)."""
    nb = (n + b - 1) // b
    total = 0
    for d in range(2, nb):
        for I in range(nb - d):
            J = I + d
            bj = min(b, n - J * b)
            total += 6 * b * (d - 1) * b * bj
    return total


def block_sum_flops_efficient(n, b, signs):
    """Algorithmic flops of the arithmetic-efficient block sums (Section 5.3):
    per (row, k, column) triple 2 flops when the row and column signs agree
    (Y only) and 4 when they differ (X only)."""
    import numpy as np
    nb = (n + b - 1) // b
    pos = np.zeros(nb, dtype=np.int64)
    cnt = np.zeros(nb, dtype=np.int64)
    for I in range(nb):
        s_ = signs[I * b:min(n, (I + 1) * b)]
        pos[I] = int(np.sum(s_ > 0))
        cnt[I] = len(s_)
    total = 0
    for d in range(2, nb):
        pI, nI = pos[:nb - d], cnt[:nb - d] - pos[:nb - d]
        pJ, nJ = pos[d:], cnt[d:] - pos[d:]
        same = pI * pJ + nI * nJ
        opp = cnt[:nb - d] * cnt[d:] - same
        total += int(np.sum((2 * same + 4 * opp) * (d - 1) * b))
    return total


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "MEASURED_PEAKS.json"
    except (OSError, ValueError):
        return {"bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "hbm_gbs": 6800.0}, "fallback"


def h2d_bytes(n, panel=128):
    """Bytes sign_tri_host copies to the device: T's upper triangle by column
    panels of `panel` columns, each from row 0 to its last column."""
    return sum(8 * min(panel, n - j0) * min(n, j0 + panel) for j0 in range(0, n, panel))


def run_batched(args):
    """The batched workload: `--batch` independent problems (seed 0), n log-
    uniform in [32, 2048], p ~ U[0, 1], random diagonal order, in one
    sign_tri_batched call per step (variant AUTO, autotuned cutoffs)."""
    import numpy as np
    import torch

    import paper_1607_06303_gb300 as st
    from paper_1607_06303_gb300 import workload
    from paper_1607_06303_gb300.inputs import batch_sizes, make_batch

    st.load()
    torch.cuda.set_device(0)
    h = torch.cuda.current_stream().cuda_stream
    t0 = time.perf_counter()
    Ts = make_batch(args.batch, seed=0)
    gen_s = time.perf_counter() - t0
    ns = [T.shape[0] for T in Ts]
    useful = sum(workload.useful_flops(np.sign(np.diag(T))) for T in Ts)
    dT = [st.to_device(T) for T in Ts]
    dU = [torch.empty_like(t) for t in dT]
    ptrT, ptrU = [t.data_ptr() for t in dT], [u.data_ptr() for u in dU]
    assert st.signtri_autotune(2048, h) == 0
    table = st.signtri_get_cutoff_table()
    vtable = st.signtri_get_variant_table()
    variant = st.Variant[args.variant] if args.variant in ("AUTO", "PH_FP64") else st.Variant.AUTO

    def step():
        s_, info = st.sign_tri_batched(ns, ptrT, ns, ptrU, ns, variant, h)
        if s_ != 0 or any(info):
            raise st.SignTriError(s_ or max(info), "sign_tri_batched")

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    st.signtri_profile_reset()
    st.signtri_profile_enable(True)
    clocks = ClockSampler(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    st.signtri_profile_enable(False)
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    per_class, launches = {}, 0
    for c in range(st.signtri.KC_COUNT):
        cnt, dms = st.signtri_profile_read(c)
        launches += cnt
        if cnt:
            per_class[st.signtri_kernel_class_name(c)] = {"launches": cnt, "device_ms": dms}
    # a check that needs no oracle, on every problem: with random +-1 probes
    # z, ||U (U z) - z|| / ||z|| and ||U (T z) - T (U z)|| / (||T|| ||U|| ||z||)
    # on the device (U^2 = I and TU = UT hold for sign(T) exactly)
    dev = dT[0].device if dT else torch.device("cuda")
    gen = torch.Generator(device=dev).manual_seed(7)
    inv_worst = com_worst = 0.0
    for t, u in zip(dT, dU):
        # the tensors hold M^T (column-major storage): M z = (M^T)^T z
        z = torch.randint(0, 2, (t.shape[0], 4), generator=gen, device=dev, dtype=torch.float64) * 2 - 1
        Ut, Tt_ = u.T, t.T
        inv = torch.linalg.norm(Ut @ (Ut @ z) - z) / torch.linalg.norm(z)
        com = torch.linalg.norm(Ut @ (Tt_ @ z) - Tt_ @ (Ut @ z)) / (
            torch.linalg.norm(t) * torch.linalg.norm(u) * torch.linalg.norm(z))
        inv_worst = max(inv_worst, float(inv))
        com_worst = max(com_worst, float(com))
    hits, builds = st.signtri_batched_cache_stats()
    line = {
        "metric": "batched sign(T): useful GFLOP/s over %d problems" % len(Ts), "value": useful / (ms * 1e-3) / 1e9,
        "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "batched: %d problems, n log-uniform [32, 2048], p ~ U[0,1], random order, seed 0"
                               % len(Ts), "sum_n2": int(sum(n * n for n in ns)), "useful_flops": useful,
                   "variant": variant.name, "cutoff_table": {str(1 << k): table[k] for k in range(5, 12)},
                   "variant_table": {str(1 << k): (st.Variant(vtable[k]).name if vtable[k] else "batched")
                                     for k in range(5, 12)},
                   "host_generation_s": gen_s},
        "gpu_launches": launches, "kernel_time_ms": per_class, "clocks": clk,
        "probe_residuals": {"involution_max": inv_worst, "commutation_max": com_worst,
                            "what": "max over problems of ||U(Uz)-z||/||z|| and ||U(Tz)-T(Uz)||/(||T|| ||U|| ||z||), "
                                    "4 random +-1 probes each, float64 on the device"},
        "graph_cache": {"hits": hits, "builds": builds},
    }
    if not args.no_cpu_baseline:
        # CPU baseline on a bounded sample (the largest problem and 20 more):
        # the oracle's time on them, and this run's outputs against its results
        import oracle
        rng = np.random.default_rng(1)
        sample = sorted(set([int(np.argmax(ns))] +
                            [int(i) for i in rng.choice(len(Ts), min(20, len(Ts)), replace=False)]))
        threads = oracle.max_threads()
        t0 = time.perf_counter()
        Uos = [oracle.sign_tri(Ts[i], schedule="antidiag", threads=threads) for i in sample]
        dt = time.perf_counter() - t0
        fl = sum(workload.useful_flops(np.sign(np.diag(Ts[i]))) for i in sample)
        errs = [float(np.linalg.norm(st.to_numpy(dU[i]) - Uo) / np.linalg.norm(Uo)) for i, Uo in zip(sample, Uos)]
        line["cpu_baseline"] = {"value": fl / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": "%d of the batch's problems (the largest, n=%d, and up to 20 drawn with seed 1), "
                                          "one solve each (%.3g useful flops, %.1f s)"
                                          % (len(sample), max(ns), fl, dt)}
        line["max_rel_err_vs_oracle_sample"] = max(errs)
        line["sample_size"] = len(sample)
    print(json.dumps(line), flush=True)
    return 0


def run_general(args):
    """sign(A) of a general real A (Section 1's route, all on the GPU): the
    complex Schur decomposition, the complex sign of T and Q U Q^H, through
    signtri_sign_general.  A: `--n` x `--n`, entries uniform in [-50, 50]
    (the matrices of the paper's Section 6), seed 0."""
    import numpy as np
    import torch

    import paper_1607_06303_gb300 as st
    from paper_1607_06303_gb300.inputs import make_A

    st.load()
    torch.cuda.set_device(0)
    n = args.n
    A = make_A(n, seed=0)
    At = st.to_device(A)
    St = torch.empty_like(At)

    def step():
        st.sign_general(At, out=St)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    st.signtri_profile_reset()
    st.signtri_profile_enable(True)
    clocks = ClockSampler(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    st.signtri_profile_enable(False)
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    per_class, launches = {}, 0
    for c in range(st.signtri.KC_COUNT):
        cnt, dms = st.signtri_profile_read(c)
        launches += cnt
        if cnt:
            per_class[st.signtri_kernel_class_name(c)] = {"launches": cnt, "device_ms": dms / max(args.steps, 1)}
    info = st.signtri_get_info()   # the last solve's QR sweeps and rotations
    S = st.to_numpy(St)
    line = {
        "metric": "sign(A) of a general real A: solves per second", "value": 1e3 / ms, "unit": "solves/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "sign(A), A %d x %d, entries uniform in [-50, 50], seed 0" % (n, n)},
        "gpu_launches": launches, "kernel_time_ms_per_solve": per_class, "clocks": clk,
        "involution_residual": float(np.linalg.norm(S @ S - np.eye(n)) / np.linalg.norm(S) ** 2),
        "qr": {"sweeps": info.qr_sweeps, "rotations": info.qr_rotations},
    }
    if not args.no_cpu_baseline:
        # the oracle's route (LAPACK's Schur form, the oracle's complex sign and
        # products) on the same A, one solve, and this run's result against it
        import oracle
        t0 = time.perf_counter()
        ref = oracle.sign_general(A)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 1.0 / dt, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": "the same A, one solve (%.2f s): LAPACK's complex Schur form through "
                                          "scipy (its BLAS may thread over the host's cores; cores is that "
                                          "bound), then the oracle's complex sign and products" % dt}
        line["rel_err_vs_oracle"] = float(np.linalg.norm(S - ref) / np.linalg.norm(ref))
    print(json.dumps(line), flush=True)
    return 0


def reduce_over_ranks(dist, x, op, device):
    """x reduced over the replicas ("max" for times, "sum" for work done);
    x itself when the bench runs as one process."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def main():
    args = parse_args()
    if args.workload == "batched" and args.impl == "ours":
        return run_batched(args)
    if args.workload == "general" and args.impl == "ours":
        return run_general(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        line = run_reference(args, rank)
        if line is not None:
            print(json.dumps(line), flush=True)
        return 0

    import numpy as np
    import torch

    import paper_1607_06303_gb300 as st
    from paper_1607_06303_gb300 import workload
    from paper_1607_06303_gb300.inputs import make_T

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    st.load()
    variant = st.Variant[args.variant]
    if args.cutoff:
        assert st.signtri_set_cutoff(args.cutoff) == 0
    n = args.n
    T = make_T(n, args.p, seed=rank, order=args.order)
    signs = np.sign(np.diag(T))
    useful = workload.useful_flops(signs)
    Tt = st.to_device(T)
    Ut = torch.empty_like(Tt)
    stream = torch.cuda.current_stream()
    h = stream.cuda_stream

    def step():
        s = st.sign_tri(n, Tt.data_ptr(), n, Ut.data_ptr(), n, variant, h)
        if s != 0:
            raise st.SignTriError(s, "sign_tri")

    fp64_peak = st.signtri_probe_fp64_peak(h)
    for _ in range(max(args.warmup, 0)):
        step()
    barrier()
    st.signtri_profile_reset()
    st.signtri_profile_enable(True)
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    st.signtri_profile_enable(False)
    ms_total = e0.elapsed_time(e1)
    per_class = {}
    launches = 0
    for c in range(st.signtri.KC_COUNT):
        cnt, ms = st.signtri_profile_read(c)
        launches += cnt
        if cnt:
            per_class[st.signtri_kernel_class_name(c)] = {"launches": cnt, "device_ms": ms}
    info = st.signtri_get_info()
    ms_step = ms_total / max(args.steps, 1)
    ms_step_max = reduce_over_ranks(dist, ms_step, "max", "cuda")
    # each replica solves its own input (seed = rank): the job's work is the
    # sum of the replicas' useful flops
    useful_all = reduce_over_ranks(dist, useful, "sum", "cuda")
    value = useful_all / (ms_step_max * 1e-3) / 1e9

    # roofline of the dominant kernel class, and of the runner-up among the
    # tensor-core classes (the mixed step's sweeps and residual products are
    # close in time)
    def class_roofline(cls):
        if cls == "block_sums_f64":
            b = info.cutoff
            efficient = info.variant == st.Variant.PH_FP64_EFFICIENT
            flops_step = block_sum_flops_efficient(n, b, signs) if efficient else block_sum_flops(n, b)
            launches_c = per_class[cls]["launches"]
            per_launch = flops_step * args.steps / launches_c
            avg_ms = per_class[cls]["device_ms"] / launches_c
            ach = per_launch / (avg_ms * 1e-3) / 1e12
            peak = fp64_peak / 1e3
            return {"class": cls, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": TRAFFIC.get(traffic_key(cls, n, args.p, args.order, variant.name)),
                    "kernel": ("ph_gemm_split_kernel (float64 DFMA, one sum per entry)" if efficient
                               else "ph_gemm_kernel (float64 DFMA block sums)"),
                    "peak_source": "float64 FMA issue rate measured live by signtri_probe_fp64_peak (no FP64 "
                                   "entry in MEASURED_PEAKS.json)",
                    "share_of_step": per_class[cls]["device_ms"] / ms_total}
        if cls == "block_sums_tc":
            # the sweeps' block sums against the tensor roof on the method's
            # own work: the initial sweep's useful flops (the oracle's count)
            # and, per refinement step, one sum per entry of the correction (4
            # flops per (i, k, j) term of X^E = ET - TE or Y^E = U0 E + E U0:
            # 4 C(n, 3)).  Beside it: the executed tensor rate (every slice
            # pair and quadrant issued) and the operand bytes against the copy
            # bandwidth.
            peaks, src = measured_peaks()
            peak_t = float(peaks.get("bf16_tflops_sustained", 1700.0))
            peak_b = float(peaks.get("hbm_gbs", 6800.0))
            launches_c = per_class[cls]["launches"]
            bytes_all = st.signtri_profile_read_bytes(st.signtri.KC_BLOCK_SUMS_TC)
            flops_all = st.signtri_profile_read_flops(st.signtri.KC_BLOCK_SUMS_TC)
            avg_ms = per_class[cls]["device_ms"] / launches_c
            method_step = useful + 4.0 * math.comb(n, 3) * max(info.refine_steps, 0)
            per_launch = method_step * args.steps / launches_c
            ach = per_launch / (avg_ms * 1e-3) / 1e12
            bytes_launch = bytes_all / launches_c
            ach_b = bytes_launch / (avg_ms * 1e-3) / 1e9
            fp16 = variant == st.Variant.PH_MIXED_FP16
            return {"class": cls, "bound": "tensor", "achieved": ach, "peak": peak_t, "unit": "TFLOP/s",
                    "frac": ach / peak_t,
                    "traffic": TRAFFIC.get(traffic_key(cls, n, args.p, args.order, variant.name)),
                    "kernel": "tc_blocksum_kernel (tcgen05 %s, sweep block sums, blocked slice layout)"
                              % ("fp16, two-term split" if fp16 else "bf16 split"),
                    "algorithmic_flops_per_launch": per_launch,
                    "peak_source": "bf16_tflops_sustained of %s (fp16 runs at the bf16 rate; kernel timed "
                                   "inside a long step)" % src,
                    "executed_tflops": flops_all / launches_c / (avg_ms * 1e-3) / 1e12,
                    "executed_frac": flops_all / launches_c / (avg_ms * 1e-3) / 1e12 / peak_t,
                    "hbm_view": {"operand_bytes_per_launch": bytes_launch, "achieved_gbs": ach_b,
                                 "peak_gbs": peak_b, "frac": ach_b / peak_b,
                                 "peak_source": "hbm_gbs of %s (copy bandwidth)" % src},
                    "share_of_step": per_class[cls]["device_ms"] / ms_total}
        if cls == "residual":
            # emulated-float64 residual and probe products: every slice pair
            # product is needed (exact integer slices), so the executed
            # products are the algorithmic work of the emulation
            peaks, src = measured_peaks()
            peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
            launches_c = per_class[cls]["launches"]
            flops_all = st.signtri_profile_read_flops(st.signtri.KC_RESIDUAL)
            per_launch = flops_all / launches_c
            avg_ms = per_class[cls]["device_ms"] / launches_c
            ach = per_launch / (avg_ms * 1e-3) / 1e12
            return {"class": cls, "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": TRAFFIC.get(traffic_key(cls, n, args.p, args.order, variant.name)),
                    "kernel": "tc_pair2_kernel / tc_blocksum_kernel (tcgen05 bf16, emulated-float64 residual "
                              "and probe products)",
                    "algorithmic_flops_per_launch": per_launch,
                    "peak_source": "bf16_tflops_sustained of %s (kernel timed inside a long step)" % src,
                    "share_of_step": per_class[cls]["device_ms"] / ms_total}
        return None

    ranked = sorted(per_class, key=lambda c: -per_class[c]["device_ms"])
    dom = ranked[0] if ranked else None
    roof = class_roofline(dom) if dom else None
    second = next((c for c in ranked[1:] if c in ("block_sums_tc", "residual")), None)
    roof2 = class_roofline(second) if second else None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step_max, "seconds_per_solve": ms_step_max / 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": ("f64" if variant in (st.Variant.PH_FP64, st.Variant.PS_FP64, st.Variant.PH_FP64_EFFICIENT)
                  else "fp16+f32+f64" if variant == st.Variant.PH_MIXED_FP16 else "bf16+f32+f64"),
        "data": "synthetic",
        "config": {"workload": "sign(T) n=%d p=%g %s diagonal, |t_ii|~U[0.5,2], t_ij~N(0,1/n), seed=rank"
                               % (n, args.p, args.order),
                   "n": n, "p": args.p, "order": args.order, "variant_requested": args.variant,
                   "variant_run": st.Variant(info.variant).name if info.variant >= 0 else None,
                   "cutoff": info.cutoff, "useful_flops_per_solve": useful,
                   "l2": ("no flush: T and U are %.3g GB each, > 129 MB L2" % (8e-9 * n * n) if 8 * n * n > 129e6
                          else "T and U (%.3g MB each) fit in L2: warm-cache timing" % (8e-6 * n * n)),
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "gpu_launches": launches, "kernel_time_ms": per_class, "roofline": roof, "roofline_second": roof2,
        "clocks": clk,
        "refinement": {"steps": info.refine_steps, "resid_commute": info.resid_commute,
                       "resid_involution": info.resid_involution},
    }

    # end to end through the public API with host buffers
    if not args.no_e2e:
        Th = torch.from_numpy(np.ascontiguousarray(T.T)).pin_memory()
        Uh = torch.empty_like(Th).pin_memory()
        s = st.sign_tri_host(n, Th.data_ptr(), n, Uh.data_ptr(), n, variant, h)   # warm (staging alloc)
        if s != 0:
            raise st.SignTriError(s, "sign_tri_host")
        # three repetitions of the timed loop, the median reported (the shared
        # host adds run-to-run noise to the copies and launches)
        reps = []
        for _ in range(3):
            barrier()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                s = st.sign_tri_host(n, Th.data_ptr(), n, Uh.data_ptr(), n, variant, h)
                if s != 0:
                    raise st.SignTriError(s, "sign_tri_host")
            barrier()
            reps.append((time.perf_counter() - t0) / max(args.steps, 1))
        e2e_s = reduce_over_ranks(dist, statistics.median(reps), "max", "cuda")
        line["e2e"] = {"value": useful_all / e2e_s / 1e9, "unit": UNIT,
                       "h2d_bytes_per_step": h2d_bytes(n), "d2h_bytes_per_step": Uh.numel() * 8,
                       "seconds_per_solve": e2e_s, "repetitions_s": reps}
        # where one call's time goes, after (outside) the timed repetitions:
        # the two copies and the kernels by CUDA events, the rest host-side
        st.signtri_profile_reset()
        st.signtri_profile_enable(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = st.sign_tri_host(n, Th.data_ptr(), n, Uh.data_ptr(), n, variant, h)
        wall_ms = (time.perf_counter() - t0) * 1e3
        st.signtri_profile_enable(False)
        if s != 0:
            raise st.SignTriError(s, "sign_tri_host")
        copy_ms = kern_ms = 0.0
        for c in range(st.signtri.KC_COUNT):
            cnt, dms = st.signtri_profile_read(c)
            if c == st.signtri.KC_HOST_COPY:
                copy_ms = dms
            else:
                kern_ms += dms
        line["e2e"]["one_call_ms"] = {"wall": wall_ms, "copies": copy_ms, "kernels": kern_ms,
                                      "rest": wall_ms - copy_ms - kern_ms,
                                      "what": "one extra sign_tri_host call with the library's CUDA-event "
                                              "profiling on; rest = host work, launch gaps and waits"}
        del Th, Uh

    # comparison variants on the same input, fewer steps
    compares = []
    for cname in [c for c in (args.compare or "").split(",") if c and c != args.variant]:
        cv = st.Variant[cname]
        Uc = torch.empty_like(Tt)

        def cstep():
            s_ = st.sign_tri(n, Tt.data_ptr(), n, Uc.data_ptr(), n, cv, h)
            if s_ != 0:
                raise st.SignTriError(s_, "sign_tri")
        cstep()
        barrier()
        ck = max(1, min(args.steps, 2))
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(ck):
            cstep()
        c1.record(stream)
        barrier()
        cms = reduce_over_ranks(dist, c0.elapsed_time(c1) / ck, "max", "cuda")
        compares.append(({"variant": cname, "steps": ck, "seconds_per_solve": cms / 1e3,
                          "value": useful_all / (cms * 1e-3) / 1e9, "unit": UNIT,
                          "speedup_of_headline": cms / ms_step_max}, Uc))
    if compares:
        line["compare"] = [c for c, _ in compares]

    # CPU oracle baseline on a bounded sample (rank 0, N = 1) and the parity of
    # this run's output on that window
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        m = min(args.cpu_sample, n)
        Tw = np.asfortranarray(T[:m, :m])
        threads = oracle.max_threads()
        t0 = time.perf_counter()
        Uo = oracle.sign_tri(Tw, schedule="antidiag", threads=threads)
        dt = time.perf_counter() - t0
        fw = workload.useful_flops(np.sign(np.diag(Tw)))
        line["cpu_baseline"] = {"value": fw / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": "leading %dx%d principal window of the same input, one solve "
                                          "(%.3g useful flops, %.1f s)" % (m, m, fw, dt)}
        Tw2 = np.asfortranarray(T[n - m:, n - m:])
        Uo2 = oracle.sign_tri(Tw2, schedule="antidiag", threads=threads)

        def window_errs(Udev):
            Ug = Udev[:m, :m].cpu().numpy().T      # U[:m,:m] (column-major storage transposed back)
            Ug2 = Udev[n - m:, n - m:].cpu().numpy().T
            return (float(np.linalg.norm(Ug - Uo) / np.linalg.norm(Uo)),
                    float(np.linalg.norm(Ug2 - Uo2) / np.linalg.norm(Uo2)))
        # principal-window property: u_ij depends on T[i..j, i..j] only, so the
        # oracle on a window equals the full oracle there
        line["rel_err_vs_oracle_window"], line["rel_err_vs_oracle_trailing_window"] = window_errs(Ut)
        for c, Uc in compares:
            c["rel_err_vs_oracle_window"], c["rel_err_vs_oracle_trailing_window"] = window_errs(Uc)

    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python
"""Benchmark of the MAPE hot path: verified Graver directions per second.

One step = one pass of the whole path on the large workload (n = 2000,
m = 400, A = [C | I] with C 400x1600 in [-5,5] at density 0.01, box
[-20,20], f = x'Qx + c'x + sum w_i x_i^4 with Q in [-5,5] at 0.005 and w in
[0,3]; P = 65536 starts Z0 ~ N(0, 2), T = 1000 Adam steps, the rounded
iterate collected every 50th step): Algorithm 2 on the streamed tensor-core
kernels, the forward product B z in e4m3 with a power-of-two scale per start
(the workload's stated precision; the gradient product and the exact map
B round(z) in BF16, FP32 accumulation and state), dedup, the kernel test,
the minimality filter, the direction coefficients and Algorithm 1 from xbar,
all through the instance handle.  The same pass in BF16 (z as hi + lo
terms) is reported beside it under "bf16".
value = directions that pass C1, C4, nonzero and set-minimality, summed over
the timed steps and ranks, over the max-over-ranks device time of those
steps.  Inputs are resident in device memory; they are larger than L2
(the state alone is 1.26 GB), and L2 is flushed (256 MiB write) before every
timed step as well, outside the timed events.  The medium workload (n = 200,
P = 8192, the fused resident kernel) is measured beside it under "medium".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own replica (its own start seed): the
starts are independent problems, so there is no data-path collective and the
scaling is weak.  --impl reference times the CPU oracle, on all host cores,
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "verified Graver directions/s"
UNIT = "directions/s"

# The timed workload: the large single instance.  Its starts are Z0 ~ N(0, 2)
# (the projected uniform starts of Algorithm 2 never round into the box of
# this instance within 1000 steps), and the rounded iterate is collected every
# 50th step (one row per start and step would be 131 GB of candidates).
LARGE = dict(name="large", n=2000, m=400, P=65536, T=1000, period=50, std=2.0, seed=2004)
WORKLOAD = ("large_quartic: n=2000 m=400 d=1600, A=[C|I_400], C 400x1600 in [-5,5] at density 0.01, box [-20,20], "
            "f = x'Qx + c'x + sum w_i x_i^4 with Q sym in [-5,5] at 0.005, c in [-20,20], w in [0,3]; P=65536 starts "
            "Z0 ~ N(0,2), T=1000 Adam steps (lr 0.003, lambda1 0.85, lambda2 1), collection every 50th step; "
            "streamed tensor-core kernels, B z in e4m3 with per-start scales, B^T sign and B round(z) in BF16; "
            "Algorithm 1 from xbar")
MEDIUM = dict(name="medium", n=200, m=40, P=8192, T=1000, period=1, std=None, seed=2002)
MEDIUM_WORKLOAD = ("medium_sparse: n=200 m=40 d=160, A=[C|I_40], C 40x160 in [-3,3] at density 0.1, box [0,10], "
                   "Q sym in [-5,5] at 0.05, c in [-20,20]; P=8192 projected Uniform(l-u,u-l) starts, T=1000 Adam "
                   "steps, collection every step; fused resident BF16 kernel; Algorithm 1 from xbar")
P_FULL, T_FULL = LARGE["P"], LARGE["T"]
CPU_STARTS_PER_CORE = 4   # starts per host core in the bounded oracle sample (all T = 1000 steps)
REF_STARTS_PER_CORE = 2   # the same for each step of the reference arm


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["bf16", "bf16x1", "fp32", "sparse", "fp8"], default="fp8",
                    help="precision of the large workload's extraction (default: e4m3 forward product)")
    ap.add_argument("--no-bf16-pass", action="store_true",
                    help="skip the BF16 comparison passes of the large workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP32 comparison run (medium workload)")
    ap.add_argument("--no-medium", action="store_true", help="skip the medium-workload measurement")
    ap.add_argument("--streamed-case", nargs=3, metavar=("NAME", "P", "T"),
                    help="time the streamed tensor-core extraction on a named instance (large: n=2000 m=400; "
                         "uneven1000: n=1000 m=200; medium: n=200 m=40) for P starts and T steps, and exit")
    ap.add_argument("--serve", type=int, default=2000, metavar="N",
                    help="requests in the serving measurement (Poisson stream at 200/s, n log-uniform in "
                         "[30, 3000], m = n/5, P = 4096); 0 skips it")
    ap.add_argument("--serve-plain", type=int, default=24, metavar="N",
                    help="the plain FP32 one-at-a-time comparison runs the first N requests of the stream")
    ap.add_argument("--serve-T", type=int, default=1000, help="Adam steps per request in the serving measurement")
    ap.add_argument("--serve-slots", type=int, default=16, help="requests on the device at once in the serving measurement")
    ap.add_argument("--batch", type=int, default=64, metavar="N",
                    help="instances in the batched-extraction measurement (n log-uniform in [50, 1000], m = n/5, "
                         "P in {1024, 4096, 16384}, T = 1000); 0 skips it")
    ap.add_argument("--sparse-fwd", action="store_true",
                    help="the large workload's forward product on the CUDA cores over the compressed rows of B "
                         "(MAPE_PREC_SPARSE_FWD) instead of the tensor cores")
    ap.add_argument("--autotune", action="store_true",
                    help="with --streamed-case: let the library choose the implementation and tile widths")
    ap.add_argument("--probe-mma", action="store_true",
                    help="measure the issue cost of tcgen05.mma over M, N and operand kind, and exit")
    ap.add_argument("--medium-only", action="store_true",
                    help="run only the medium workload's measurement (BF16 resident kernel) and exit")
    ap.add_argument("--kernel-case", type=int, nargs=2, metavar=("P", "T"),
                    help="time the fused extraction kernel alone on P starts of the workload for T steps "
                         "(two launches; a small case for profilers) and exit")
    return ap.parse_args(argv)


# ---------------------------------------------------------------- distributed

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_over_ranks(units, ms, world):
    """Sum of units over ranks and max of device time over ranks (the
    whole-job throughput of weakly scaled replicas)."""
    if world == 1:
        return float(units), float(ms)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


def row_hashes(D):
    """64-bit hashes of the rows of an int8 direction set (FNV-1a over the
    bytes), for counting distinct directions across ranks."""
    import numpy as np
    D = np.ascontiguousarray(D, dtype=np.int8).view(np.uint8)
    h = np.full(D.shape[0], 0xcbf29ce484222325, dtype=np.uint64)
    prime = np.uint64(0x100000001b3)
    with np.errstate(over="ignore"):
        for j in range(D.shape[1]):
            h = (h ^ D[:, j].astype(np.uint64)) * prime
    return h


def distinct_over_ranks(hashes, world):
    """(distinct rows over all ranks, total rows): the replicas run disjoint
    start seeds, so the job's directions are the union of the ranks' sets."""
    import numpy as np
    if world == 1:
        return int(np.unique(hashes).size), int(hashes.size)
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, hashes)
    allh = np.concatenate(parts)
    return int(np.unique(allh).size), int(allh.size)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks / throttle reasons every 50 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.th.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- peaks

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------- CPU oracle

def _generated(wl):
    from paper_2412_13576_gb300 import instances as I
    return I.large_quartic() if wl["name"] == "large" else I.medium_sparse()


def _starts(wl, inst, P, rank=0):
    """Device-independent start arrays of a workload: (Z0, G0), one of them None."""
    from paper_2412_13576_gb300 import instances as I
    if wl["std"] is not None:
        return I.normal_starts(inst, P, std=wl["std"], seed=wl["seed"] + rank).Z0, None
    return None, I.uniform_samples(inst, P, seed=wl["seed"] + rank).G0


def _oracle_part(args):
    """One host core's share of the oracle sample: Algorithm 2 on a slice of
    the starts (plain numpy, one thread); returns its distinct directions."""
    name, lo, hi, T = args
    from oracle import mape_oracle as O
    wl = LARGE if name == "large" else MEDIUM
    inst = _generated(wl)
    Z0, G0 = _starts(wl, inst, hi)
    Z0 = O.project_to_coordinates(inst.B, G0[lo:hi]) if Z0 is None else Z0[lo:hi]
    res = O.parallel_extraction(inst.A, inst.B, inst.l, inst.u, Z0, T=T, period=wl["period"])
    return res["unique"]


class OraclePool:
    """The CPU oracle on every host core: a pool of spawned one-thread worker
    processes, each running Algorithm 2 on its slice of the sampled starts;
    the parent takes the union of their sets and the minimality filter."""

    def __init__(self, cores=None):
        import multiprocessing as mp
        self.cores = cores or os.cpu_count() or 1
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        os.environ["CUDA_VISIBLE_DEVICES"] = ""
        self.pool = mp.get_context("spawn").Pool(self.cores)

    def run(self, wl, starts, T=None):
        """Algorithm 2 + dedup + minimality on the first `starts` starts of the
        workload for T steps (default: the workload's)."""
        import numpy as np
        from oracle import mape_oracle as O
        T = wl["T"] if T is None else T
        per = -(-starts // self.cores)
        parts = [(wl["name"], lo, min(lo + per, starts), T) for lo in range(0, starts, per)]
        t0 = time.perf_counter()
        sets = self.pool.map(_oracle_part, parts)
        found = {tuple(int(v) for v in r) for U in sets for r in U}
        U = O.sort_directions(np.array(sorted(found), dtype=np.int64).reshape(-1, wl["n"]))
        K = int(O.minimal_elements(U).sum()) if U.shape[0] else 0
        dt = time.perf_counter() - t0
        return {"directions": K, "unique": int(U.shape[0]), "seconds": dt, "value": K / dt, "P": starts,
                "T": T, "cores": len(parts)}

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline_obj(r, wl):
    return {"value": r["value"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
            "host_cores": os.cpu_count(),
            "sample": (f"oracle (numpy fp64/int64, one thread per core, {r['cores']} cores) on {r['P']} of the "
                       f"{wl['P']} starts, all {r['T']} steps of Algorithm 2 with collection every {wl['period']}"
                       f"{'th' if wl['period'] > 1 else ''} step + dedup + minimality filter: {r['directions']} "
                       f"directions in {r['seconds']:.1f} s (augmentation excluded: it adds no directions)")}


# ---------------------------------------------------------------- our arm

PREC = {"bf16": 1, "bf16x1": 2, "fp32": 0, "sparse": 3, "fp8": 4}


def handle_passes(mape, wl, inst, starts, stream, steps, warmup, prec, flush, clk=None):
    """`warmup` untimed and `steps` timed passes of the whole path through one
    instance handle (inputs resident on the device); returns the device time
    of the timed passes (CUDA events on the handle's stream, L2 flushed before
    each), their statuses and the library launches inside the timed region."""
    import torch
    Z0, G0 = starts
    x0 = torch.from_numpy(inst.xbar[None, :].astype("int32")).to(flush.device)
    cfg = mape.default_config(T=wl["T"], precision=prec, period=wl["period"])

    def one(h):
        h.extract_directions(wl["P"], Z0=Z0, G0=G0)
        h.wait(900)
        h.augment(x0)
        h.wait(900)
        return h.poll()

    h = mape.Instance.from_generated(inst, cfg, stream=stream)
    for _ in range(warmup):
        one(h)
    torch.cuda.synchronize()
    total_ms, statuses = 0.0, []
    L = mape.lib()
    launches0 = L.mape_launch_count()
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = one(h)
        e1.record(stream)
        stream.synchronize()
        total_ms += e0.elapsed_time(e1)
        statuses.append(st)
    launches = L.mape_launch_count() - launches0
    h.close()
    return total_ms, statuses, launches


def e2e_passes(mape, wl, inst, starts_host, stream, reps, directions_hint, prec=1):
    """The public handle API with host buffers, every copy inside the region:
    the instance and the starts go up from pinned host memory, the direction
    set (int8 rows) and the best point come back into pinned host memory
    (buffers pinned once, before the region)."""
    import numpy as np
    import torch
    Z0, G0 = starts_host
    src = Z0 if Z0 is not None else G0
    src_host = torch.from_numpy(np.ascontiguousarray(src)).pin_memory().numpy()
    x0_host = inst.xbar[None, :].astype(np.int32)
    D_host = torch.empty((max(int(1.2 * directions_hint), 1024), inst.n), dtype=torch.int8).pin_memory().numpy()
    cfg = mape.default_config(T=wl["T"], precision=prec, period=wl["period"])
    times, units, phases = [], 0, []
    h2d = (inst.A.nbytes + inst.b.nbytes + inst.l.nbytes + inst.u.nbytes + inst.B.nbytes + inst.Q.nbytes
           + inst.c.nbytes + (0 if inst.w is None else inst.w.nbytes) + src_host.nbytes + x0_host.nbytes)
    d2h = 0
    for _ in range(reps):
        torch.cuda.synchronize()
        t = [time.perf_counter()]
        with mape.Instance.from_generated(inst, cfg, stream=stream) as he:
            t.append(time.perf_counter())
            if Z0 is not None:
                he.extract_directions(wl["P"], Z0=src_host)
            else:
                he.extract_directions(wl["P"], G0=src_host)
            he.wait(900)
            t.append(time.perf_counter())
            he.augment(x0_host)
            he.wait(900)
            t.append(time.perf_counter())
            D = he.directions_i8(out=D_host)
            x, fx = he.solution()
            t.append(time.perf_counter())
        t.append(time.perf_counter())
        times.append(t[-1] - t[0])
        phases.append({k: round((t[i + 1] - t[i]) * 1e3, 3)
                       for i, k in enumerate(("create", "extract_filter", "augment", "download", "destroy"))})
        units += D.shape[0]
        d2h = D.nbytes + x.nbytes + 8
    return {"value": units / sum(times), "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "steps": len(times), "ms_per_step": [t * 1e3 for t in times], "phases_ms": phases, "_last_directions": D}


def run_ours(args):
    import torch

    from paper_2412_13576_gb300 import mape

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    mape.lib(build_if_missing=True)
    dev = torch.device("cuda", torch.cuda.current_device())
    wl = LARGE
    inst = _generated(wl)
    starts_host = _starts(wl, inst, wl["P"], rank)
    starts = tuple(None if a is None else torch.from_numpy(a).to(dev) for a in starts_host)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    prec = PREC[args.precision] | (mape.PREC_SPARSE_FWD if args.sparse_fwd else 0)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        total_ms, statuses, launches = handle_passes(mape, wl, inst, starts, stream, args.steps, args.warmup, prec,
                                                     flush)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    directions = sum(st["directions"] for st in statuses)
    units_all, ms_max = reduce_over_ranks(directions, total_ms, world)
    value = units_all / (ms_max / 1e3)
    e2e = e2e_passes(mape, wl, inst, starts_host, stream, max(1, min(args.steps, 3)),
                     directions / max(args.steps, 1), prec)
    # the union of the replicas' sets: rows counted once across ranks
    distinct, rows = distinct_over_ranks(row_hashes(e2e.pop("_last_directions")), world)

    result = None
    if rank == 0:
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"bf16": "bf16", "bf16x1": "bf16", "fp32": "f32", "sparse": "f32",
                      "fp8": "fp8_e4m3+bf16"}[args.precision],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "P": wl["P"], "T": wl["T"], "n": wl["n"], "m": wl["m"],
                       "period": wl["period"], "precision": args.precision + ("+sparse_fwd" if args.sparse_fwd else ""),
                       "l2": "inputs larger than L2, and L2 flushed (256 MiB write) before each timed step",
                       "replicas_per_rank": 1},
            "directions_per_step": directions / args.steps,
            "distinct_over_ranks": {"rows": rows, "distinct": distinct},
            "stages_ms": {k: statistics.median(s[k] for s in statuses)
                          for k in ("extract_ms", "filter_ms", "augment_ms", "first_improve_ms")},
            "candidates_per_step": statistics.median(s["candidates"] for s in statuses),
            "best_f": statuses[-1]["best_f"],
            "f_xbar": int(_f_value(inst, inst.xbar)),
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "e2e": e2e,
        }
        result["roofline"] = roofline_streamed(mape, wl, inst, starts, stream, prec)
        if args.precision == "fp8" and not args.no_bf16_pass:
            result["bf16"] = bf16_passes(mape, wl, inst, starts, stream, flush)
        if not args.no_cpu_baseline and world == 1:
            # before the serving measurement, whose host threads and arrays would share the cores
            pool = OraclePool()
            try:
                result["cpu_baseline"] = cpu_baseline_obj(pool.run(wl, CPU_STARTS_PER_CORE * pool.cores), wl)
            finally:
                pool.close()
        if world == 1 and not args.no_medium:
            result["medium"] = medium_measure(mape, args, stream, flush)
        if args.batch > 0 and world == 1:
            result["batched"] = batch_measure(args.batch)
            result["batched"]["pipeline"] = batch_pipeline_measure(args.batch)
        if args.serve > 0 and world == 1:
            result["serving"] = serve_measure(args.serve, args.serve_T, args.serve_plain, slots=args.serve_slots)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return result


def bf16_passes(mape, wl, inst, starts, stream, flush, steps=2, warmup=1):
    """The same handle passes with the extraction in BF16 (z as hi + lo
    terms, every product on BF16 operands): the comparison for the e4m3
    forward product."""
    total_ms, statuses, _ = handle_passes(mape, wl, inst, starts, stream, steps, warmup, PREC["bf16"], flush)
    directions = sum(st["directions"] for st in statuses)
    return {"value": directions / (total_ms / 1e3), "unit": UNIT, "ms_per_step": total_ms / steps,
            "steps": steps, "directions_per_step": directions / steps,
            "extract_ms": statistics.median(s["extract_ms"] for s in statuses), "best_f": statuses[-1]["best_f"]}


def _f_value(inst, x):
    """f(x) in exact integers (reporting only: the value the path starts from)."""
    import numpy as np
    x = np.asarray(x, dtype=object)
    Q = np.asarray(inst.Q, dtype=object)
    val = int(x @ Q @ x) + int(np.asarray(inst.c, dtype=object) @ x)
    if inst.w is not None:
        val += int(np.asarray(inst.w, dtype=object) @ (x ** 4))
    return val


def medium_measure(mape, args, stream, flush):
    """The medium workload (fused resident kernel) through the same handle
    passes, with its own roofline and the plain FP32 comparison."""
    import torch
    wl = MEDIUM
    inst = _generated(wl)
    starts_host = _starts(wl, inst, wl["P"])
    starts = tuple(None if a is None else torch.from_numpy(a).to(flush.device) for a in starts_host)
    total_ms, statuses, launches = handle_passes(mape, wl, inst, starts, stream, args.steps, min(args.warmup, 3),
                                                 PREC["bf16"], flush)
    directions = sum(st["directions"] for st in statuses)
    out = {"workload": MEDIUM_WORKLOAD, "value": directions / (total_ms / 1e3), "unit": UNIT,
           "ms_per_step": total_ms / args.steps, "directions_per_step": directions / args.steps,
           "stages_ms": {k: statistics.median(s[k] for s in statuses)
                         for k in ("extract_ms", "filter_ms", "augment_ms", "first_improve_ms")},
           "best_f": statuses[-1]["best_f"], "gpu_launches": launches,
           "e2e": {k: v for k, v in e2e_passes(mape, wl, inst, starts_host, stream, max(1, min(args.steps, 3)),
                                                directions / max(args.steps, 1)).items() if not k.startswith("_")},
           "roofline": roofline_resident(mape, wl, inst, starts_host[1], stream)}
    if not args.no_plain:
        out["vs_plain_fp32"] = plain_fp32(mape, wl, inst, starts, stream)
    return out


def medium_only(args):
    """The medium workload's measurement alone (the passes the "medium" key
    reports): the command its launch list is taken on."""
    import torch
    from paper_2412_13576_gb300 import mape
    torch.cuda.set_device(0)
    mape.lib(build_if_missing=True)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    return {"medium": medium_measure(mape, args, stream, flush)}


def time_extract_kernel(mape, inst, starts, P, T, prec, stream, reps, period=1):
    """CUDA-event times (ms, on `stream`) of `reps` + 1 calls of mape_extract
    on the first P starts for T steps, all from the same starting state (the
    first call is a warm-up and is dropped).  starts = (Z0, G0) host arrays,
    one of them None (G0 rows are projected first)."""
    import numpy as np
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    B = torch.from_numpy(inst.B).to(dev)
    span = torch.from_numpy((inst.u - inst.l).astype(np.int32)).to(dev)
    cfg = mape.default_config(T=T, precision=prec, period=period)
    Zs, Gs = starts
    with torch.cuda.stream(stream):
        if Zs is not None:
            Z0 = torch.from_numpy(np.ascontiguousarray(Zs[:P])).to(dev)
        else:
            Z0 = mape.project_starts(B, torch.from_numpy(Gs[:P]).to(dev), stream=stream)
    ldc = mape.round16(inst.n)
    rows = P * (T // period + 1) + 16                      # every collection of every start fits
    cand = torch.empty((rows, ldc), dtype=torch.int8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    flags = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = torch.empty(mape.lib().mape_extract_workspace_bytes(inst.n, inst.d, P, prec), dtype=torch.uint8,
                     device=dev)
    times, counts = [], []
    Z, Mm, V = torch.empty_like(Z0), torch.empty_like(Z0), torch.empty_like(Z0)
    for i in range(reps + 1):
        with torch.cuda.stream(stream):
            Z.copy_(Z0)
            Mm.zero_()
            V.zero_()
            cnt.zero_()
            flags.zero_()
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mape.extract(B, span, Z, Mm, V, t0=0, T=T, cfg=cfg, cand=cand, cand_count=cnt, flags=flags, ldc=ldc,
                     workspace=ws, stream=stream)
        e1.record(stream)
        stream.synchronize()
        if int(flags.item()) != 0:
            raise RuntimeError(f"extraction flags {int(flags.item())}")
        if i > 0:
            times.append(e0.elapsed_time(e1))
            counts.append(int(cnt.item()))
    return times, counts


def kernel_case(args):
    """The fused extraction alone on a small case of the medium workload (P
    starts, T steps): the command profilers run."""
    import torch
    from paper_2412_13576_gb300 import mape
    torch.cuda.set_device(0)
    mape.lib(build_if_missing=True)
    inst = _generated(MEDIUM)
    P, T = args.kernel_case
    stream = torch.cuda.Stream()
    # the medium workload runs in BF16 (its stated precision) unless another BF16/FP32 form is asked for
    prec = args.precision if args.precision in ("bf16x1", "fp32") else "bf16"
    times, counts = time_extract_kernel(mape, inst, _starts(MEDIUM, inst, MEDIUM["P"]), P, T, PREC[prec],
                                        stream, reps=1)
    return {"kernel_case": {"workload": "medium_sparse", "P": P, "T": T, "precision": prec,
                            "ms_per_launch": times, "candidates": counts}}


def streamed_case(args):
    """The streamed kernels (three per step) alone on a named instance, with
    the large workload's starts and collection period: per step, the forward
    pass reads z (4 d bytes per start) and writes sign(Bm z) (2 R bytes), the
    gradient pass reads it back and reads and writes z, m, v (24 d bytes): the
    algorithmic bytes are 28 d + 4 R per start-step."""
    import torch
    from paper_2412_13576_gb300 import instances as I
    from paper_2412_13576_gb300 import mape
    torch.cuda.set_device(0)
    mape.lib(build_if_missing=True)
    name, P, T = args.streamed_case[0], int(args.streamed_case[1]), int(args.streamed_case[2])
    inst = {"large": I.large_quartic, "medium": I.medium_sparse,
            "uneven1000": lambda: I.uneven_single(1000, density=0.05)}[name]()
    bf = args.precision in ("bf16", "bf16x1")
    tunable = bf or args.precision == "fp8"
    prec = PREC[args.precision] | (mape.PREC_AUTOTUNE if (args.autotune and tunable) else
                                   (mape.PREC_STREAMED if bf else 0))
    if args.sparse_fwd:
        prec |= mape.PREC_SPARSE_FWD
    Z0 = I.normal_starts(inst, P, std=LARGE["std"], seed=LARGE["seed"]).Z0
    stream = torch.cuda.Stream()
    times, counts = time_extract_kernel(mape, inst, (Z0, None), P, T, prec, stream, reps=2,
                                        period=LARGE["period"])
    ms = statistics.median(times)
    R = inst.n - inst.d
    algo = (28.0 * inst.d + 4.0 * R) * P * T
    peaks, src = measured_peaks()
    gbs = algo / (ms / 1e3) / 1e9
    return {"streamed_case": {"instance": inst.name, "n": inst.n, "d": inst.d, "P": P, "T": T,
                              "precision": args.precision, "ms_per_call": times, "ms_per_step": ms / T,
                              "candidates": counts, "algorithmic_bytes_per_call": algo, "achieved_gbs": gbs,
                              "hbm_peak_gbs": peaks["hbm_gbs"], "frac_of_hbm": gbs / peaks["hbm_gbs"],
                              "peak_source": src,
                              "autotune": mape.autotune_info(inst.n, inst.d, P, PREC[args.precision])
                              if args.autotune else None}}


SERVE_RATE = 200.0    # requests per second (Poisson)
SERVE_P = 4096
SERVE_DISTINCT = 200  # distinct instances in the stream (each recurs with its starts; drawing 2000 costs minutes)


def _pct(v, q):
    import numpy as np
    return float(np.percentile(np.asarray(v, dtype=np.float64), q)) if len(v) else None


def serve_measure(N, T, n_plain=24, seed=3000, slots=16):
    """The serving workload: N requests arriving as a Poisson stream at 200/s
    over SERVE_DISTINCT distinct instances taken in turn (n log-uniform in
    [30, 3000], m = n/5, C in [-3,3] at a density uniform in [0.05, 0.2], box
    [-5,5]; each with its own P = 4096 projected starts), Algorithm 1 from x̄.  Runs them through the request server (continuous
    batching, BF16 paths) and, for comparison, the first n_plain of them one
    at a time through the plain FP32 single-instance path (arriving on the
    same clock); reports instances/s, p50/p99 time to first improving
    direction and to termination (from arrival), the backlog, and verified
    directions/s.  When the server completes fewer instances per second than
    arrive, the queue grows and the completion rate is the saturation point."""
    import numpy as np
    from paper_2412_13576_gb300 import instances as I
    from paper_2412_13576_gb300 import mape
    rng = np.random.default_rng(seed)
    pool = I.uneven_batch(count=min(N, SERVE_DISTINCT), n_lo=30, n_hi=3000, seed=seed)
    pool_g0 = [I.uniform_samples(inst, SERVE_P, seed=seed + 1 + k).G0 for k, inst in enumerate(pool)]
    # the stream: the distinct instances in turn, each with its own starts
    insts = [pool[k % len(pool)] for k in range(N)]
    arrivals = np.cumsum(rng.exponential(1.0 / SERVE_RATE, size=N))

    def starts(k):
        return pool_g0[k % len(pool)]

    def run_server(cfg, slots, count, batch):
        with mape.Server(cfg, mem_cap_bytes=150 << 30, max_slots=slots, batch_extraction=batch) as srv:
            # warm-up: the smallest and the largest instance, 10 steps each (loads every kernel used)
            warm_cfg = mape.default_config(T=10, precision=cfg.precision)
            with mape.Server(warm_cfg, mem_cap_bytes=150 << 30, max_slots=2) as ws:
                for k in (int(np.argmin([i.n for i in insts])), int(np.argmax([i.n for i in insts]))):
                    ws.submit(insts[k], SERVE_P, G0=starts(k))
                ws.wait_all(600)
            G0s = [starts(k) for k in range(count)]     # drawn before the clock starts (shared per instance)
            t0 = time.perf_counter()
            ids, backlog = [], 0
            for k in range(count):
                wait = arrivals[k] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
                ids.append(srv.submit(insts[k], SERVE_P, G0=G0s[k]))
                if k % 50 == 49:
                    backlog = max(backlog, srv.stats()["queued"])
            srv.wait_all(3600)
            wall = time.perf_counter() - t0
            infos = [srv.info(i) for i in ids]
            stats = srv.stats()
            for i in ids:
                srv.release(i)
        return infos, wall, stats, backlog

    out = {}
    for name, prec, slots, count, batch in (("served_bf16", PREC["bf16"], slots, N, False),
                                            ("served_bf16_batched_extraction", PREC["bf16"], slots, N, True),
                                            ("plain_fp32_one_at_a_time", 0, 1, min(n_plain, N), False)):
        cfg = mape.default_config(T=T, precision=prec)
        infos, wall, stats, backlog = run_server(cfg, slots, count, batch)
        ok = [i for i in infos if i["state"] == "DONE"]
        ttfid = [i["t_first_improve_ms"] - i["t_submit_ms"] for i in ok]
        ttt = [i["t_done_ms"] - i["t_submit_ms"] for i in ok]
        errors = {}
        for i in infos:
            if i["state"] != "DONE":
                key = f"{mape.ERR.get(i['error'], i['error'])}"
                errors[key] = errors.get(key, 0) + 1
        if errors:
            errors["last_cuda_error"] = mape.lib().mape_last_cuda_error().decode()
        out[name] = {"requests": count, "instances_per_s": len(ok) / wall, "wall_s": wall, "completed": len(ok),
                     "failed": len(infos) - len(ok), "errors": errors,
                     "failed_n": sorted(i["n"] for i in infos if i["state"] != "DONE")[:20],
                     "arrival_rate": SERVE_RATE,
                     "arrivals_span_s": float(arrivals[count - 1]),
                     "ttfid_ms_p50": _pct(ttfid, 50), "ttfid_ms_p99": _pct(ttfid, 99),
                     "ttt_ms_p50": _pct(ttt, 50), "ttt_ms_p99": _pct(ttt, 99),
                     "directions_per_s": sum(i["directions"] for i in ok) / wall,
                     "peak_running": stats["peak_running"], "peak_queued_sampled": backlog,
                     "mem_peak_gb": stats["mem_peak"] / 1e9,
                     "best_f": [i["best_f"] for i in infos]}
    a, b = out["served_bf16"]["best_f"], out["plain_fp32_one_at_a_time"]["best_f"]
    out["f_not_worse_than_plain"] = float(np.mean([x <= y for x, y in zip(a, b)]))
    out["batched_equals_slot_streams"] = bool(out["served_bf16"]["best_f"] ==
                                              out["served_bf16_batched_extraction"]["best_f"])
    for k in ("served_bf16", "served_bf16_batched_extraction", "plain_fp32_one_at_a_time"):
        out[k].pop("best_f")
    s = out["served_bf16"]
    s["saturated"] = s["instances_per_s"] < 0.95 * SERVE_RATE
    out["workload"] = (f"{N} requests, Poisson arrivals at {SERVE_RATE:.0f}/s, over {len(pool)} distinct instances "
                       f"taken in turn (n log-uniform in [30, 3000], uneven_batch seed {seed}, m = n/5, each with its "
                       f"own P = {SERVE_P} projected starts), T = {T}, 150 GB admission cap; the plain arm runs the "
                       f"first {min(n_plain, N)} of them")
    return out


def batch_measure(N, T=1000, seed=1003):
    """Batched extraction of uneven instances: N instances with n log-uniform in
    [50, 1000], m = n/5, C in [-3,3] at a density uniform in [0.05, 0.2], box
    [-5,5], P drawn from {1024, 4096, 16384}, projected uniform starts, T Adam
    steps (a3-a8).  Times one mape_extract_batch call (one CUDA graph: one
    persistent launch per resident-kernel variant, three launches per step for
    the streamed shapes) against the same calls made one after another with
    mape_extract, on the same stream, from the same starting state."""
    import numpy as np
    import torch
    from paper_2412_13576_gb300 import instances as I
    from paper_2412_13576_gb300 import mape
    rng = np.random.default_rng(seed + 1000)
    insts = I.uneven_batch(count=N, n_lo=50, n_hi=1000, seed=seed)
    Ps = rng.choice([1024, 4096, 16384], size=N)
    cfg = mape.default_config(T=T, precision=PREC["bf16"])
    stream = torch.cuda.Stream()
    calls, starts = [], []
    with torch.cuda.stream(stream):
        for k, (inst, P) in enumerate(zip(insts, Ps)):
            P = int(P)
            B = torch.from_numpy(inst.B).cuda()
            G0 = torch.from_numpy(I.uniform_samples(inst, P, seed=seed + 2000 + k).G0).cuda()
            Z0 = mape.project_starts(B, G0, stream=stream)
            ldc = mape.round16(inst.n)
            Z = torch.empty_like(Z0)
            calls.append(dict(B=B, span=torch.from_numpy((inst.u - inst.l).astype(np.int32)).cuda(), Z=Z,
                              M=torch.empty_like(Z0), V=torch.empty_like(Z0),
                              cand=torch.empty((min(P * (T + 1), (512 << 20) // ldc), ldc), dtype=torch.int8,
                                               device="cuda"),
                              cand_count=torch.zeros(1, dtype=torch.int64, device="cuda"),
                              flags=torch.zeros(1, dtype=torch.int32, device="cuda"), ldc=ldc,
                              workspace=torch.empty(mape.lib().mape_extract_workspace_bytes(inst.n, inst.d, P,
                                                                                           cfg.precision),
                                                    dtype=torch.uint8, device="cuda")))
            starts.append(Z0)

    def reset():
        with torch.cuda.stream(stream):
            for c, Z0 in zip(calls, starts):
                c["Z"].copy_(Z0)
                c["M"].zero_()
                c["V"].zero_()
                c["cand_count"].zero_()
                c["flags"].zero_()
        stream.synchronize()

    def timed(fn):
        reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1)

    def batched():
        mape.extract_batch(calls, t0=0, T=T, cfg=cfg, stream=stream)

    def sequential():
        for c in calls:
            mape.extract(t0=0, T=T, cfg=cfg, stream=stream, **c)

    timed(batched)
    tb = timed(batched)
    flags = [int(c["flags"].item()) for c in calls]
    zb = [c["Z"].clone() for c in calls]
    timed(sequential)
    ts = timed(sequential)
    same = all(torch.equal(a, c["Z"]) for a, c in zip(zb, calls))
    starts_steps = float(sum(int(p) for p in Ps)) * T
    return {"instances": N, "T": T, "batched_ms": tb, "sequential_ms": ts, "speedup": ts / tb,
            "start_steps_per_s": starts_steps / (tb / 1e3), "same_state_as_sequential": same,
            "flags": sorted(set(flags)), "n_range": [min(i.n for i in insts), max(i.n for i in insts)],
            "workload": (f"uneven_batch(count={N}, n in [50,1000], seed {seed}); P from {{1024,4096,16384}}; "
                         f"projected uniform starts; T = {T}; a3-a8 only")}


def batch_pipeline_measure(N, T=1000, seed=1003):
    """The batched configuration end to end: the same N uneven instances as
    batch_measure, submitted at once to the request server (64 slots, 150 GB
    cap), each through Algorithm 2, dedup, the kernel test, the minimality
    filter, the coefficients and Algorithm 1 from xbar; once with the
    extraction of the requests admitted together run as one batched call
    (batch_extraction) and once with each request on its own slot stream.
    Reports instances/s and p50/p99 time to first improving direction and to
    termination."""
    import numpy as np
    from paper_2412_13576_gb300 import instances as I
    from paper_2412_13576_gb300 import mape
    rng = np.random.default_rng(seed + 1000)
    insts = I.uneven_batch(count=N, n_lo=50, n_hi=1000, seed=seed)
    Ps = rng.choice([1024, 4096, 16384], size=N)
    G0s = [I.uniform_samples(inst, int(P), seed=seed + 2000 + k).G0 for k, (inst, P) in enumerate(zip(insts, Ps))]
    out = {}
    for name, batch in (("batched_extraction", True), ("slot_streams", False)):
        cfg = mape.default_config(T=T, precision=PREC["bf16"])
        with mape.Server(cfg, mem_cap_bytes=150 << 30, max_slots=64, batch_extraction=batch) as srv:
            t0 = time.perf_counter()
            ids = [srv.submit(inst, int(P), G0=G0) for inst, P, G0 in zip(insts, Ps, G0s)]
            srv.wait_all(3600)
            wall = time.perf_counter() - t0
            infos = [srv.info(i) for i in ids]
            stats = srv.stats()
        ok = [i for i in infos if i["state"] == "DONE"]
        ttfid = [i["t_first_improve_ms"] - i["t_submit_ms"] for i in ok]
        ttt = [i["t_done_ms"] - i["t_submit_ms"] for i in ok]
        queued = [i["t_admit_ms"] - i["t_submit_ms"] for i in ok]
        extracting = [i["t_extracted_ms"] - i["t_admit_ms"] for i in ok]
        augmenting = [i["t_done_ms"] - i["t_extracted_ms"] for i in ok]
        out[name] = {"instances_per_s": len(ok) / wall, "wall_s": wall, "completed": len(ok),
                     "failed": len(infos) - len(ok), "ttfid_ms_p50": _pct(ttfid, 50), "ttfid_ms_p99": _pct(ttfid, 99),
                     "ttt_ms_p50": _pct(ttt, 50), "ttt_ms_p99": _pct(ttt, 99),
                     "median_ms": {"queued": _pct(queued, 50), "admitted_to_directions": _pct(extracting, 50),
                                   "directions_to_done": _pct(augmenting, 50)},
                     "directions": sum(i["directions"] for i in ok), "peak_running": stats["peak_running"],
                     "best_f": [i["best_f"] for i in infos]}
    a, b = out["batched_extraction"].pop("best_f"), out["slot_streams"].pop("best_f")
    out["same_f"] = bool(a == b)
    out["workload"] = (f"uneven_batch(count={N}, n in [50,1000], seed {seed}); P from {{1024,4096,16384}}; projected "
                       f"uniform starts; T = {T}; the whole path per instance, all submitted at once")
    return out


RESIDENT_TRAFFIC = os.path.join(ROOT, "profiles", "extract_tc_kernel_medium_sparse_P8192_T1000_traffic.md")
STREAM_TRAFFIC = os.path.join(ROOT, "profiles", "stream_step_large_quartic_traffic.md")


def measured_traffic(record, src_path):
    """DRAM bytes per launch from a committed ncu record, if that record was
    taken on the current source of the kernel (same SHA-256)."""
    import hashlib
    import re
    try:
        text = open(record).read()
        sha = hashlib.sha256(open(src_path, "rb").read()).hexdigest()
    except OSError:
        return None
    m_sha = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    m_b = re.search(r"dram_bytes_per_launch:\s*([0-9]+)", text)
    if not m_sha or not m_b or m_sha.group(1) != sha:
        return None
    return int(m_b.group(1))


def roofline_streamed(mape, wl, inst, starts, stream, prec, reps=2):
    """The streamed extraction of the large workload, timed live: `reps` calls
    of mape_extract (T steps, the workload's starts and period) with the
    library's per-launch CUDA events on the launches' streams.  A step is the
    forward pass (reads z, writes sign(Bm z): (4 d + 2 R) bytes per start) and
    the gradient + Adam pass (reads sign(Bm z) and reads and writes z, m, v:
    (24 d + 2 R) bytes per start); the tiles run as two halves on two
    streams, so that one half's forward pass overlaps the other's gradient
    pass.  The unit of the roofline is therefore the step, both kernels
    together: (28 d + 4 R) P bytes per step over the step's time (the call's
    time over T, which includes packing z, m, v once per call).  The bound is
    HBM bandwidth: the state (1.26 GB) is far larger than L2 and is streamed
    every step.  The per-kernel launch durations are reported beside it; they
    overlap in time."""
    import numpy as np
    peaks, src = measured_peaks()
    P, T, d = wl["P"], wl["T"], inst.d
    R = inst.n - d
    host = tuple(None if a is None else a.cpu().numpy() for a in starts)
    mape.launch_timing(True)
    try:
        times, counts = time_extract_kernel(mape, inst, host, P, T, prec, stream, reps, period=wl["period"])
        per = mape.launch_timing_read()
    finally:
        mape.launch_timing(False)
    peak = peaks["hbm_gbs"]
    call_ms = statistics.median(times)
    step_ms = call_ms / T
    step_bytes = (28.0 * d + 4.0 * R) * P
    achieved = step_bytes / (step_ms / 1e3) / 1e9
    kernels = {}
    for kind, name, per_start in (("stream_grad", "stream_grad_kernel", 24.0 * d + 2.0 * R),
                                  ("stream_fwd", "stream_fwd_sparse_kernel" if prec & mape.PREC_SPARSE_FWD
                                   else "stream_fwd_kernel", 4.0 * d + 2.0 * R)):
        ms, n = per[kind]
        launches_per_step = max(1, round(n / ((reps + 1) * T)))  # two with the tile halves; reps + 1 calls ran
        b = per_start * P / launches_per_step
        kernels[name] = {"ms_per_launch": ms / max(n, 1), "launches_per_step": launches_per_step,
                         "bytes_per_launch": b, "achieved": b / (ms / max(n, 1) / 1e3) / 1e9,
                         "frac_while_overlapped": b / (ms / max(n, 1) / 1e3) / 1e9 / peak}
    src_path = os.path.join(ROOT, "paper_2412_13576_gb300", "csrc", "extract_stream.cu")
    return {"bound": "hbm", "kernel": "streamed step: stream_fwd_kernel and stream_grad_kernel, tile halves on two streams",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": measured_traffic(STREAM_TRAFFIC, src_path), "ms_per_step": step_ms, "bytes_per_step": step_bytes,
            "peak_source": f"{src} HBM copy rate (MEASURED_PEAKS.json hbm_gbs)",
            "kernels": kernels,
            "collect_ms_per_launch": per["stream_collect"][0] / max(per["stream_collect"][1], 1),
            "candidates_per_call": int(np.median(counts)),
            "note": "one step = forward + gradient (+ collection every period-th step) for P = 65536 starts, 28 d + 4 R "
                    "bytes per start; step time = CUDA-event time of a T = 1000 call / T (the call also packs z, m, v "
                    "once); kernel launch durations from events the library records around each launch on its "
                    "stream; traffic = ncu dram read+write bytes of one step (both kernels), null unless taken on "
                    "this source"}


def roofline_resident(mape, wl, inst, G0, stream, reps=3):
    """The fused resident extraction launch of the medium workload (T = 1000
    steps), timed alone with CUDA events on its stream.  Its state (z, m, v)
    stays on chip for the whole launch, so the bound is the tensor-core
    roofline.  Two counts of the work: the dense contraction of the scope
    table (B z, B^T sign(Bz), B round(z): 6 n d flops per start-step) and the
    contraction the kernel performs (B = [I; -C], so only the m rows of -C go
    through the tensor cores: 2 m d flops per product, with z as two BF16
    terms: 8 m d)."""
    peaks, src = measured_peaks()
    P, T = wl["P"], wl["T"]
    times, _ = time_extract_kernel(mape, inst, (None, G0), P, T, PREC["bf16"], stream, reps)
    ms = statistics.median(times)
    n, d, m = inst.n, inst.d, inst.n - inst.d
    flops = 6.0 * n * d * P * T
    performed = 2.0 * m * d * P * T * 4
    achieved = flops / (ms / 1e3) / 1e12
    peak = peaks["bf16_tflops"]
    src_path = os.path.join(ROOT, "paper_2412_13576_gb300", "csrc", "extract_tc.cu")
    return {"bound": "tensor", "kernel": "extract_tc_kernel", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": measured_traffic(RESIDENT_TRAFFIC, src_path), "ms_per_launch": ms,
            "flops_per_launch": flops,
            "performed": {"flops_per_launch": performed, "achieved": performed / (ms / 1e3) / 1e12,
                          "frac": performed / (ms / 1e3) / 1e12 / peak},
            "peak_source": f"{src} cuBLAS BF16 dense burst (MEASURED_PEAKS.json bf16_tflops)",
            "note": "one launch = T=1000 steps for P=8192 starts; frac on the dense 6 n d count; performed = "
                    "the m rows of -C through the tensor cores (hi, lo, round(z), gradient: 8 m d flops per "
                    "start-step); traffic = ncu dram read+write bytes of one full launch, null unless taken on "
                    "this source"}


def plain_fp32(mape, wl, inst, starts, stream):
    """One pass of the plain FP32 single-instance path (per step: strict-FP32
    cuBLAS GEMMs and unfused elementwise kernels) for comparison, timed after
    one untimed warm-up pass."""
    import torch
    Z0, G0 = starts
    x0 = torch.from_numpy(inst.xbar[None, :].astype("int32")).cuda()
    cfg = mape.default_config(T=wl["T"], precision=0, period=wl["period"])
    with mape.Instance.from_generated(inst, cfg, stream=stream) as h:
        for rep in range(2):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.extract_directions(wl["P"], Z0=Z0, G0=G0)
            h.wait(900)
            h.augment(x0)
            h.wait(900)
            e1.record(stream)
            stream.synchronize()
        st = h.poll()
    ms = e0.elapsed_time(e1)
    return {"value": st["directions"] / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "best_f": st["best_f"],
            "directions": st["directions"]}


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    """The CPU oracle as it stands, on all host cores, on a bounded sample of
    the large workload (REF_STARTS_PER_CORE starts per core, all T steps, per
    step), under the same metric and unit."""
    world, rank, _ = dist_env()
    if rank != 0:
        return None
    wl = LARGE
    pool = OraclePool()
    try:
        starts = REF_STARTS_PER_CORE * pool.cores
        for _ in range(args.warmup):      # warm-up: the workers import and build the instance
            pool.run(wl, pool.cores, T=wl["period"])
        total_s, total_units, r = 0.0, 0, None
        for _ in range(args.steps):
            r = pool.run(wl, starts)
            total_s += r["seconds"]
            total_units += r["directions"]
    finally:
        pool.close()
    value = total_units / total_s
    cb = cpu_baseline_obj(r, wl)
    cb["value"] = value
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+int64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "P": wl["P"], "T": wl["T"], "n": wl["n"], "m": wl["m"],
                       "period": wl["period"], "sample_starts": starts},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def probe_mma():
    """The tensor-core instruction cost (mape_mma_issue_probe) over M, N,
    operand kind and accumulator count: SM cycles per instruction and the
    FLOPs per cycle that makes."""
    import torch
    from paper_2412_13576_gb300 import mape
    torch.cuda.set_device(0)
    mape.lib(build_if_missing=True)
    rows = []
    for kind, K in ((0, 16), (1, 32)):
        for M in (64, 128):
            for N in (16, 32, 64, 128, 256):
                for acc in (1, 2):
                    issue, total = mape.mma_issue_probe(kind, M, N, acc, 512)
                    rows.append({"kind": ("f16/bf16", "f8f6f4/e4m3")[kind], "M": M, "N": N, "K": K,
                                 "accumulators": acc, "issue_cycles": issue, "total_cycles": total,
                                 "flops_per_cycle": 2.0 * M * N * K / total})
    return {"probe_mma": rows}


def main(argv=None):
    args = parse_args(argv)
    if args.probe_mma:
        print(json.dumps(probe_mma()), flush=True)
        return 0
    if args.kernel_case:
        print(json.dumps(kernel_case(args)), flush=True)
        return 0
    if args.streamed_case:
        print(json.dumps(streamed_case(args)), flush=True)
        return 0
    if args.medium_only:
        print(json.dumps(medium_only(args)), flush=True)
        return 0
    res = run_reference(args) if args.impl == "reference" else run_ours(args)
    if res is not None:
        print(json.dumps(res), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())

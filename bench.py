#!/usr/bin/env python
"""Benchmark of the GB300 Gustavson SpGEMM hot path.

One step = one whole product C = A*B through the C ABI with the inputs
resident in HBM: analyse (row product counts, binning), symbolic (row sizes,
prefix scan, one host sync for nnz(C)), numeric (columns and values).  The
default workload is C = A*A for the R-MAT power-law adjacency of scale 18,
edge factor 16, (a,b,c,d) = (0.57, 0.19, 0.19, 0.05), values U(0.5, 1.5),
FP64, int32 indices.

Metric: GFLOP/s = 2 * (intermediate products) / time.  The JSON line also
carries the numeric kernel's HBM roofline fraction (algorithmic bytes of
A, the B rows touched and C written, over its CUDA-event duration), an
end-to-end figure with host buffers (H2D of A, D2H of C inside the timed
region), SM clocks sampled during the timed region, and the CPU oracle's
throughput on a bounded row sample.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       [--workload rmat|lap2d|stencil3d]
For N > 1 (torchrun), rank r multiplies a row block of A balanced by product
count; the blocks are independent, there is no collective on the data path.
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

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

from paper_2112_10037_gb300 import gen  # noqa: E402

L2_BYTES = 129 * 1024 * 1024
# default row classes of the library (register sort <= 16 products, hash
# accumulator 17..128; numeric warp window up to 65536 products, bins rounded
# to powers of two; block window above)
TINY_MAX = 16
HASH_MAX = 128
NUM_BLOCK_MIN = 65536
PEAKS_FILE = os.path.join(HERE, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


# ------------------------------------------------------------------ inputs
def make_workload(name: str, rmat_scale: int = 18):
    """(A, B, description) on the host; B is A for the square workloads."""
    if name == "rmat":
        A = gen.rmat(rmat_scale, 16)
        return A, A, {"workload": "rmat_s%d_ef16_AxA" % rmat_scale,
                      "matrix": "R-MAT scale %d, edge factor 16, (0.57,0.19,0.19,0.05), self-loops dropped, "
                                "duplicates merged, U(0.5,1.5) values" % rmat_scale,
                      "rows": A.nrows, "nnz_A": A.nnz}
    if name == "lap2d":
        A = gen.laplacian_2d(64)
        return A, A, {"workload": "laplacian2d_64_AxA", "rows": A.nrows, "nnz_A": A.nnz}
    if name == "stencil3d":
        A = gen.laplacian_3d(96)
        return A, A, {"workload": "laplacian3d_96_AxA", "rows": A.nrows, "nnz_A": A.nnz}
    raise SystemExit("unknown workload %s" % name)


def row_products(A, B):
    """Per-row product counts from the input structure (host bookkeeping for
    the byte model and the row sample; the device computes its own)."""
    lens = np.diff(B.row_ptr.astype(np.int64))
    per_nz = lens[A.col_idx]
    cs = np.concatenate([[0], np.cumsum(per_nz)])
    rp = A.row_ptr.astype(np.int64)
    return cs[rp[1:]] - cs[rp[:-1]]


def balanced_row_blocks(prod, nparts):
    """Row boundaries splitting the rows into nparts blocks of about equal
    product count."""
    cs = np.concatenate([[0], np.cumsum(prod)])
    targets = cs[-1] * np.arange(1, nparts) / nparts
    cuts = np.searchsorted(cs, targets)
    return [0] + [int(c) for c in cuts] + [len(prod)]


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons (read only)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        """Starts the sampler and waits (at most 5 s) for its first sample,
        so that the timed region that follows is covered from its start."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t_end = time.monotonic() + 5.0
        while not self.lines and time.monotonic() < t_end and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def mark(self):
        """Host time of the start of the timed region."""
        self.t0 = time.monotonic()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        t1 = time.monotonic()
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0 = getattr(self, "t0", None)
        inside = [ln for t, ln in self.lines if t0 is None or t0 <= t <= t1 + 0.06]
        for ln in inside:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_hbm_peak():
    try:
        with open(PEAKS_FILE) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


# --------------------------------------------------------- CPU baseline
def cpu_oracle_leg(A, B, prod, target_seconds=12.0):
    """The oracle (single-threaded C) on a bounded sample of rows: every
    s-th row of A, s chosen from a short calibration run so the sample takes
    about target_seconds.  Returns the cpu_baseline dict."""
    import oracle
    oracle.build()
    total = int(prod.sum())
    # calibration on a small strided sample
    s0 = max(1, int(total / 2e7))
    rows = np.arange(0, A.nrows, s0)
    t0 = time.perf_counter()
    oracle.spgemm(oracle.select_rows(A, rows), B)
    dt = max(time.perf_counter() - t0, 1e-3)
    rate = max(int(prod[rows].sum()), 1) / dt
    want = rate * target_seconds
    stride = max(1, int(round(total / max(want, 1.0))))
    rows = np.arange(0, A.nrows, stride)
    sub = oracle.select_rows(A, rows)
    p = int(prod[rows].sum())
    t0 = time.perf_counter()
    oracle.spgemm(sub, B)
    dt = time.perf_counter() - t0
    out = {"value": 2.0 * p / dt / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
           "sample": "rows i = 0 mod %d of A (%d rows, %d products, %.1f s single-threaded)"
                     % (stride, len(rows), p, dt),
           "host_cores": os.cpu_count()}
    out["all_cores"] = cpu_oracle_all_cores(A, B, prod, rows)
    return out


def _oracle_rows_task(task):
    """Worker of cpu_oracle_all_cores: the oracle on one block of the sample
    rows, timed in the worker (inputs already in the worker's memory)."""
    A, B, rows = task
    import oracle
    oracle.build()
    sub = oracle.select_rows(A, rows)
    t0 = time.perf_counter()
    oracle.spgemm(sub, B)
    return time.perf_counter() - t0


def cpu_oracle_all_cores(A, B, prod, rows):
    """The same row sample on every host core: the unchanged single-threaded
    oracle run by one spawned process per core (spawn: this process holds a
    CUDA context) on product-balanced blocks of the sample rows.  The time is
    the slowest worker's compute time; starting the workers and sending them
    the inputs are not counted."""
    import multiprocessing as mp
    procs = max(1, os.cpu_count() or 1)
    p = prod[rows]
    cs = np.cumsum(p)
    cuts = np.searchsorted(cs, cs[-1] * np.arange(1, procs) / procs) if len(cs) else []
    blocks = [b for b in np.split(rows, cuts) if len(b)]
    with mp.get_context("spawn").Pool(len(blocks)) as pool:
        pool.map(_oracle_rows_task, [(A, B, b[:1]) for b in blocks])  # load the oracle in every worker
        times = pool.map(_oracle_rows_task, [(A, B, b) for b in blocks], chunksize=1)
    dt = max(times)
    return {"value": 2.0 * int(p.sum()) / dt / 1e9, "unit": "GFLOP/s", "cores": len(blocks), "kind": "oracle",
            "sample": "the same rows in %d product-balanced blocks, one spawned process per core; slowest "
                      "worker %.2f s" % (len(blocks), dt)}


# ------------------------------------------------------------ our step
def run_ours(args, rank, world, A, B, desc):
    import torch
    from paper_2112_10037_gb300 import api, build as bld, _native as nat

    bld.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    prod = row_products(A, B)
    blocks = balanced_row_blocks(prod, world)
    rb, re = blocks[rank], blocks[rank + 1]
    my_products = int(prod[rb:re].sum())
    dA = api.DeviceCSR.from_host(A, device=dev)
    dB = dA if B is A else api.DeviceCSR.from_host(B, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)

    kw = {} if world == 1 else {"row_range": (rb, re)}
    if args.hash_max:
        kw["hash_max"] = args.hash_max
    for item in args.opt:
        k, v = item.split("=", 1)
        kw[k] = int(v)
    if args.tune:
        from paper_2112_10037_gb300 import autotune as at
        kw.update(at.autotune(dA, dB))
    if args.opt or args.tune:
        desc["options"] = {k: v for k, v in kw.items() if k != "row_range"}

    def step(profile=False):
        plan = api.Plan(dA, dB, dtype=torch.float64, **kw)
        if profile:
            nat.spgemm_plan_set_profiling(plan.handle, True)
        rp, nnz = plan.symbolic()
        ci, v = plan.numeric(dA.vals, dB.vals)
        return plan, rp, ci, v

    for _ in range(args.warmup):
        plan, rp, ci, v = step()
        plan.close()
        del rp, ci, v
    torch.cuda.synchronize()

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    sampler = ClockSampler(dev.index)
    sampler.start()
    sampler.mark()
    times, ktimes, launches = [], [], 0
    for _ in range(args.steps):
        flush.fill_(1)                      # evict L2 between timed steps
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        plan, rp, ci, v = step(profile=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        times.append(ev0.elapsed_time(ev1))
        ktimes.append(nat.spgemm_plan_kernel_times(plan.handle))
        launches += nat.spgemm_plan_launches(plan.handle)
        plan_stats = plan.stats()
        nnz_c = int(ci.numel())
        last = (plan, rp, ci, v)
        plan.close()
    clocks = sampler.stop()
    total_ms = float(sum(times))
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        pt = torch.tensor([my_products], dtype=torch.float64)
        dist.all_reduce(pt, op=dist.ReduceOp.SUM)
        all_products = int(pt.item())
    else:
        all_products = my_products
    ms_per_step = total_ms / args.steps
    gflops = 2.0 * all_products / (ms_per_step / 1e3) / 1e9

    # dominant kernel and its roofline
    names = list(ktimes[0].keys())
    avg = {n: float(np.mean([k[n] for k in ktimes])) for n in names}
    dom = max((n for n in names if n.startswith("num_") or n.startswith("sym_")), key=lambda n: avg[n])
    _, rp_last, _, _ = last
    c_rp = rp_last.cpu().numpy().astype(np.int64)
    byte_model = kernel_bytes(A, B, prod[rb:re], c_rp, dom, rb)
    peak, peak_kind = measured_hbm_peak()
    t_dom = avg[dom] / 1e3
    hbm_achieved = byte_model / t_dom / 1e9 if t_dom > 0 else 0.0
    hbm = {"achieved": round(hbm_achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(hbm_achieved / peak, 4),
           "peak_kind": peak_kind + " hbm_gbs (copy)", "algorithmic_bytes": int(byte_model)}
    traffic = traffic_from_profiles(dom, desc["workload"])
    if dom.startswith("num_"):
        # one FP64 fused multiply-add per product: the FP64 units bound this kernel
        kprod = kernel_products(prod[rb:re], dom)
        fp64_peak = fp64_peak_gflops(torch, dev)
        achieved = 2.0 * kprod / t_dom / 1e9 if t_dom > 0 else 0.0
        roof = {"bound": "alu", "achieved": round(achieved, 2), "peak": fp64_peak, "unit": "GFLOP/s",
                "frac": round(achieved / fp64_peak, 4), "kernel": dom, "kernel_ms": round(avg[dom], 4),
                "peak_kind": "derived: SMs x 2 FP64 FMA/clk x 2 FLOP x max SM clock (nominal 1.25 TFLOP/s FP64)",
                "products": int(kprod), "hbm": hbm, "traffic": traffic}
    else:
        roof = dict(hbm, bound="hbm", kernel=dom, kernel_ms=round(avg[dom], 4), traffic=traffic)

    torch.cuda.synchronize()
    torch.cuda.empty_cache()  # the device leg's cached blocks; the end-to-end leg allocates its own
    e2e = run_e2e(args, api, torch, dev, A, B, kw, all_products if world == 1 else my_products)
    out = {
        "metric": "SpGEMM GFLOP/s (2*products/s)", "value": round(gflops, 2), "unit": "GFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded generator, no dataset)",
        "config": dict(desc, products=int(prod.sum()), nnz_C=nnz_c, l2="flushed between timed steps",
                       **({"hash_max": args.hash_max} if args.hash_max else {}),
                       parallelism="row blocks balanced by products" if world > 1 else "single GPU"),
        "kernel_ms": {n: round(avg[n], 4) for n in names},
        "rows_per_path": dict(zip(["tiny", "hash", "warp", "block"], plan_stats[2])),
        "roofline": roof, "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks,
    }
    return out


def kernel_bytes(A, B, prod_rows, c_rp, kernel, row_begin):
    """Algorithmic bytes of one launch of `kernel` on its rows: the A rows it
    reads, each B row it touches counted once, and what it writes (numeric:
    C's columns and values, 12 B per entry for FP64; symbolic: 4 B per row
    size) -- the byte model of the measurement section, restricted to the
    kernel's rows."""
    P = np.asarray(prod_rows, np.int64)
    path = kernel.split("_", 1)[1]
    # register sort up to 16 products, hash accumulator up to 128; every
    # larger row runs in the warp window kernel (numeric) / the bitmap
    # kernels (symbolic warp <= 8192 < block)
    small = {"tiny": (1, TINY_MAX), "hash": (TINY_MAX + 1, HASH_MAX)}
    if kernel.startswith("num"):
        lo, hi = dict(small, warp=(HASH_MAX + 1, NUM_BLOCK_MIN), block=(NUM_BLOCK_MIN + 1, 1 << 62)).get(
            path, (0, -1))
    else:
        lo, hi = dict(small, warp=(HASH_MAX + 1, 8192), block=(8193, 1 << 62)).get(path, (0, -1))
    rows = np.flatnonzero((P >= lo) & (P <= hi))
    if len(rows) == 0:
        return 0.0
    arp = A.row_ptr.astype(np.int64)
    g = rows + row_begin
    a_nnz = int((arp[g + 1] - arp[g]).sum())
    idx = np.concatenate([np.arange(arp[r], arp[r + 1]) for r in g]) if len(g) < 20000 else \
        np.flatnonzero(np.repeat(np.isin(np.arange(A.nrows), g), np.diff(arp)))
    ks = np.unique(A.col_idx[idx])
    blens = np.diff(B.row_ptr.astype(np.int64))[ks]
    numeric = kernel.startswith("num")
    per_b = 12 if numeric else 4
    b_bytes = 8 * len(ks) + per_b * int(blens.sum())
    a_bytes = 8 * len(rows) + (12 if numeric else 4) * a_nnz
    c_nnz = int((c_rp[rows + 1] - c_rp[rows]).sum())
    c_bytes = (8 * len(rows) + 12 * c_nnz) if numeric else 4 * len(rows)
    return float(a_bytes + b_bytes + c_bytes)


def kernel_products(prod_rows, kernel):
    """Products handled by the numeric kernel of this path (host bookkeeping)."""
    P = np.asarray(prod_rows, np.int64)
    if kernel == "num_tiny":
        return int(P[(P >= 1) & (P <= TINY_MAX)].sum())
    if kernel == "num_hash":
        return int(P[(P > TINY_MAX) & (P <= HASH_MAX)].sum())
    if kernel == "num_warp":
        return int(P[(P > HASH_MAX) & (P <= NUM_BLOCK_MIN)].sum())
    return int(P[P > NUM_BLOCK_MIN].sum())


def fp64_peak_gflops(torch, dev):
    """FP64 peak from unit counts and clocks: 2 fused multiply-adds per SM per
    clock (GB300's nominal 1.25 TFLOP/s FP64 over 152 SMs at 2.07 GHz)."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = 2070.0
    try:
        with open(PEAKS_FILE) as fh:
            mhz = float(json.load(fh).get("sm_max_mhz", mhz))
    except (OSError, ValueError):
        pass
    return round(sms * 2 * 2 * mhz * 1e6 / 1e9, 1)


# Sources of the numeric pass's kernels: numeric.cu and everything it
# includes.  A DRAM-traffic record stays valid while these are unchanged.
NUMERIC_SOURCES = ["numeric.cu", "numdispatch.cuh", "semiring.cuh", "launch_util.cuh", "internal.cuh", "numblock.cuh",
                   "numrank.cuh", "numwarp.cuh", "rowhash.cuh", "rowlane.cuh", "rowpass.cuh", "segstream.cuh"]


def numeric_digest() -> str:
    """16-hex-digit digest of the numeric kernels' sources (the device code
    and its headers; the ABI header's documentation does not enter)."""
    import hashlib
    h = hashlib.sha1()
    csrc = os.path.join(HERE, "paper_2112_10037_gb300", "csrc")
    for name in NUMERIC_SOURCES:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_from_profiles(kernel, workload):
    """dram read+write bytes per launch from a committed ncu summary, if one
    exists for this kernel and workload and the numeric kernels' sources have
    not changed since; else None."""
    path = os.path.join(HERE, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
        ent = rec.get("%s|%s" % (kernel, workload))
        if ent and ent.get("source_digest") == numeric_digest():
            return ent.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass
    return None


def run_e2e(args, api, torch, dev, A, B, kw, products):
    """Same product end to end through the C ABI's host-buffer product
    (``api.spgemm_host``: ``spgemm_host_product_begin`` / ``_finish``): A in
    pinned host memory is copied to the device, C is sized, computed in row
    ranges and copied back into pinned host memory while later ranges
    compute -- all inside the timed region."""
    kw = dict(kw)
    rr = kw.pop("row_range", None)
    aliased = B is A and rr is None   # A*A: B is not copied a second time
    if rr is not None:  # this rank's row block of A
        lo, hi = int(A.row_ptr[rr[0]]), int(A.row_ptr[rr[1]])
        A = gen.CSR(rr[1] - rr[0], A.ncols, (A.row_ptr[rr[0]:rr[1] + 1] - lo).astype(np.int32), A.col_idx[lo:hi],
                    A.vals[lo:hi])
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    HA = gen.CSR(A.nrows, A.ncols, pin(A.row_ptr), pin(A.col_idx), pin(A.vals))
    HB = None if aliased else gen.CSR(B.nrows, B.ncols, pin(B.row_ptr), pin(B.col_idx), pin(B.vals))
    stream = torch.cuda.current_stream()
    steps = max(3, min(args.steps, 5))

    def once(out=None, trace=None):
        rp, ci, v = api.spgemm_host(HA, HB, dtype=torch.float64, chunks=args.e2e_chunks, out=out, trace=trace,
                                    device=dev, **kw)
        return (rp, ci, v), ci.numel(), rp.numel()

    # two untimed calls: the first pins the host buffers and allocates, the
    # second still pays first-use costs of the copies into fresh buffers
    out, nnz, nrp = once()
    once(out)
    torch.cuda.synchronize()
    ts, traces = [], []
    for _ in range(steps):
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tr = {}
        ev0.record(stream)
        once(out, tr)
        ev1.record(stream)
        torch.cuda.synchronize()
        ts.append(ev0.elapsed_time(ev1))
        traces.append(tr)
    ms = float(np.mean(ts))
    h2d = A.row_ptr.nbytes + A.col_idx.nbytes + A.vals.nbytes
    if HB is not None:
        h2d += B.row_ptr.nbytes + B.col_idx.nbytes + B.vals.nbytes
    d2h = 4 * nrp + 12 * nnz

    def summary(tr):
        # host marks (ms from the call's start) and, per row range, when its
        # numeric pass ran and when its copy to the host ran (device ms)
        d = tr.get("device_ms", {})
        return {"host": tr.get("host_ms", {}),
                "numeric": [[a, b] for a, b in zip(d.get("numeric_start", []), d.get("numeric_end", []))],
                "copy": [[a, b] for a, b in zip(d.get("copy_start", []), d.get("copy_end", []))]}
    return {"value": round(2.0 * products / (ms / 1e3) / 1e9, 2), "unit": "GFLOP/s",
            "ms_per_step": round(ms, 3), "ms_steps": [round(t, 3) for t in ts],
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "timeline": [summary(t) for t in traces]}


# ------------------------------------------------------- reference arm
def run_reference(args, A, B, desc):
    """The oracle as it stands (single-threaded C, host cores): each step is
    the product of a bounded row sample of A with B."""
    import oracle
    oracle.build()
    prod = row_products(A, B)
    total = int(prod.sum())
    stride = max(1, int(round(total / 3e8)))   # ~a few seconds per step
    rows = np.arange(0, A.nrows, stride)
    sub = oracle.select_rows(A, rows)
    p = int(prod[rows].sum())
    for _ in range(args.warmup):
        oracle.spgemm(sub, B)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.spgemm(sub, B)
        ts.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(ts))
    val = 2.0 * p / (ms / 1e3) / 1e9
    sample = "rows i = 0 mod %d of A (%d rows, %d products per step)" % (stride, len(rows), p)
    return {
        "impl": "reference", "metric": "SpGEMM GFLOP/s (2*products/s)", "value": round(val, 4),
        "unit": "GFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded generator, no dataset)", "config": desc,
        "cpu_baseline": {"value": round(val, 4), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(val, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ------------------------------------------------- secondary workloads
def _events_ms(fn, steps, stream):
    import torch
    ts = []
    for _ in range(steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.mean(ts)), ts


def _base_line(metric, value, unit, args, ms, desc):
    return {"metric": metric, "value": round(value, 3), "unit": unit, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generator, no dataset)", "config": desc}


def run_batched(args):
    """512 independent uneven products (rows log-uniform in [1024, 200000],
    half stencil squares, half random A*B; about 9.8e9 products at full
    size): the stacked batch -- split into waves whose stacked counts fit
    int32, one persistent launch per pass per wave -- against one-by-one
    calls, full pipeline and numeric only (graph replay of the batch vs a
    loop of per-instance numeric calls).  Options from the autotuner (cached
    per GPU and batch size class) unless --no-tune.  The phases run one after
    the other and free their outputs, so the device holds one copy of C."""
    import torch
    from paper_2112_10037_gb300 import api, build as bld, autotune as at
    bld.build()
    insts = gen.batched_instances_parallel(args.batch_count, args.batch_scale)
    pairs = []
    for inst in insts:
        dA = api.DeviceCSR.from_host(inst.A)
        dB = dA if inst.B is inst.A else api.DeviceCSR.from_host(inst.B)
        pairs.append((dA, dB))
    products = int(sum(int(row_products(i.A, i.B).sum()) for i in insts))
    stream = torch.cuda.current_stream()
    opts = {}
    for item in args.opt:
        k, v = item.split("=", 1)
        opts[k] = int(v)
    if not args.no_tune and not args.opt:
        opts = at.autotune_batch(pairs)
    wave_kw = {"max_b_nnz": args.batch_max_b_nnz} if args.batch_max_b_nnz else {}

    def release():
        torch.cuda.synchronize()
        torch.cuda.empty_cache()

    def batched_full():
        b = api.Batch(pairs, **wave_kw, **opts)
        b.symbolic()
        b.numeric()
        b.close()
    for _ in range(args.warmup):
        batched_full()
    t_b, _ = _events_ms(batched_full, args.steps, stream)
    release()
    # steady state of the batch: structure fixed, numeric passes replayed from the captured graphs
    batch = api.Batch(pairs, **wave_kw, **opts)
    batch.symbolic()
    batch.numeric()
    batch.capture()
    for _ in range(args.warmup):
        batch.replay()
    t_g, _ = _events_ms(batch.replay, args.steps, stream)
    nnz_c, nwaves = int(batch.nnz[-1]), len(batch.waves)
    batch.close()
    del batch
    release()

    def per_call_full():
        for dA, dB in pairs:
            pl = api.Plan(dA, dB, **opts)
            pl.symbolic()
            pl.numeric(dA.vals, dB.vals)
            pl.close()
    for _ in range(args.warmup):
        per_call_full()
    t_p, _ = _events_ms(per_call_full, args.steps, stream)
    release()
    plans, outs = [], []
    for dA, dB in pairs:
        pl = api.Plan(dA, dB, **opts)
        pl.symbolic()
        outs.append(pl.numeric(dA.vals, dB.vals))
        plans.append(pl)

    def loop_numeric():
        for (dA, dB), pl, (ci, v) in zip(pairs, plans, outs):
            pl.numeric(dA.vals, dB.vals, col_idx=ci, vals=v)
    for _ in range(args.warmup):
        loop_numeric()
    t_l, _ = _events_ms(loop_numeric, args.steps, stream)
    for pl in plans:
        pl.close()
    del plans, outs
    release()
    gf = lambda t: 2.0 * products / (t / 1e3) / 1e9
    desc = {"workload": "batched_%d_instances_scale%g" % (len(insts), args.batch_scale),
            "instances": len(insts), "rows_total": int(sum(i.rows for i in insts)), "products": products,
            "nnz_C": nnz_c, "waves": nwaves, "options": opts or "defaults", **wave_kw,
            "note": "rows log-uniform in [1024, 200000] x scale; half stencil squares, half random A*B",
            "l2": "inputs and C larger than L2"}
    out = _base_line("SpGEMM GFLOP/s (2*products/s), batched", gf(t_b), "GFLOP/s", args, t_b, desc)
    out["per_call_full_gflops"] = round(gf(t_p), 3)
    out["batched_graph_numeric_gflops"] = round(gf(t_g), 3)
    out["per_call_numeric_gflops"] = round(gf(t_l), 3)
    out["speedup_full"] = round(t_p / t_b, 3)
    out["speedup_numeric"] = round(t_l / t_g, 3)
    return out


def run_galerkin(args):
    """P^T (A P), 3D 7-point 96^3 with 2x2x2 aggregation: both numeric
    passes replayed from one CUDA graph, against two plain calls."""
    import torch
    from paper_2112_10037_gb300 import api, build as bld
    bld.build()
    A = gen.laplacian_3d(96)
    P = gen.aggregation_3d(96)
    dA, dP = api.DeviceCSR.from_host(A), api.DeviceCSR.from_host(P)
    R = api.transpose(dP)
    stream = torch.cuda.current_stream()
    g = api.Galerkin(dP, dA)
    g.capture()
    p1 = int(row_products(A, P).sum())
    APh = g.AP.to_host()
    Rh = R.to_host()
    p2 = int(row_products(Rh, APh).sum())
    def plain():
        AP = api.spgemm(dA, dP)
        api.spgemm(R, AP)
    for _ in range(args.warmup):
        g.replay()
        plain()
    reps = max(args.steps, 20)
    t_g, _ = _events_ms(g.replay, reps, stream)
    t_p, _ = _events_ms(plain, args.steps, stream)
    gf = lambda t: 2.0 * (p1 + p2) / (t / 1e3) / 1e9
    # byte model of the two numeric passes (A, B rows touched, C written)
    bytes_ap = A.nnz * 12 + A.nrows * 8 + P.nnz * 12 + P.nrows * 8 + APh.nnz * 12 + A.nrows * 8
    bytes_c = Rh.nnz * 12 + Rh.nrows * 8 + APh.nnz * 12 + APh.nrows * 8 + g.Ac.nnz * 12 + Rh.nrows * 8
    peak, kind = measured_hbm_peak()
    achieved = (bytes_ap + bytes_c) / (t_g / 1e3) / 1e9
    desc = {"workload": "galerkin_96cube_2x2x2", "products_AP": p1, "products_PtAP": p2,
            "nnz_AP": int(APh.nnz), "nnz_Ac": int(g.Ac.nnz)}
    out = _base_line("SpGEMM GFLOP/s (2*products/s), Galerkin chain graph replay", gf(t_g), "GFLOP/s", args,
                     t_g, desc)
    out["two_plain_calls_gflops"] = round(gf(t_p), 3)
    out["two_plain_calls_ms"] = round(t_p, 4)
    out["roofline"] = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                       "frac": round(achieved / peak, 4), "peak_kind": kind,
                       "algorithmic_bytes": int(bytes_ap + bytes_c), "kernel": "both numeric passes (graph)"}
    return out


def run_backward(args):
    """C = A*B, A and B 65536^2 with 32 random columns per row: forward
    (numeric) and backward (dA, dB) through the autograd Function, FP64 and
    FP32."""
    import torch
    from paper_2112_10037_gb300 import api, build as bld
    bld.build()
    n = 65536
    rng = np.random.default_rng(0)
    A = gen.random_rows(n, n, np.full(n, 32), np.random.default_rng(0))
    B = gen.random_rows(n, n, np.full(n, 32), np.random.default_rng(1))
    products = int(row_products(A, B).sum())
    stream = torch.cuda.current_stream()
    res = {}
    for dt, name in ((torch.float64, "f64"), (torch.float32, "f32")):
        dA, dB = api.DeviceCSR.from_host(A, dtype=dt), api.DeviceCSR.from_host(B, dtype=dt)
        op = api.SparseMatmul(dA, dB, dtype=dt)
        W = torch.from_numpy(np.random.default_rng(2).standard_normal(op.nnz)).to(device="cuda", dtype=dt)
        a = dA.vals.clone().requires_grad_(True)
        b = dB.vals.clone().requires_grad_(True)
        fwd = lambda: op(a.detach(), b.detach())
        c = op(a, b)
        def bwd():
            a.grad = None
            b.grad = None
            torch.autograd.backward(c, W, retain_graph=True)
        for _ in range(args.warmup):
            fwd()
            bwd()
        t_f, _ = _events_ms(fwd, args.steps, stream)
        t_b, _ = _events_ms(bwd, args.steps, stream)
        res[name] = {"forward_ms": round(t_f, 4), "backward_ms": round(t_b, 4),
                     "forward_gflops": round(2.0 * products / (t_f / 1e3) / 1e9, 2),
                     "backward_gflops": round(4.0 * products / (t_b / 1e3) / 1e9, 2)}
    desc = {"workload": "differentiation_65536sq_32perrow", "products": products}
    out = _base_line("SpGEMM backward GFLOP/s (4*products/s)", res["f64"]["backward_gflops"], "GFLOP/s", args,
                     res["f64"]["backward_ms"], desc)
    out["f64"] = res["f64"]
    out["f32"] = res["f32"]
    return out


def run_transpose(args):
    """The CSR transpose (stable radix scatter on the column index) of two
    products' C: R-MAT scale 16 A*A (164 M entries, 65,536 columns: two
    9-bit digit passes) and the 3D stencil 96^3 A*A (21.7 M entries, 884,736
    columns: three passes), with FP64 values and source positions, and of
    the structure alone.  GB/s counts the algorithmic bytes: M's column
    indices and values read once, M^T's column indices, values and source
    positions written once, and both row pointers.  Inputs larger than L2."""
    import torch
    from paper_2112_10037_gb300 import api, build as bld
    bld.build()
    stream = torch.cuda.current_stream()
    peak, peak_kind = measured_hbm_peak()
    res = {}
    for name, M in (("rmat_s16_AxA", gen.rmat(16, 16)), ("laplacian3d_96_AxA", gen.laplacian_3d(96))):
        dM = api.DeviceCSR.from_host(M)
        C = api.spgemm(dM, dM)
        S = api.DeviceCSR(C.nrows, C.ncols, C.row_ptr, C.col_idx, None)
        del dM
        torch.cuda.synchronize()
        nnz, rows, cols = C.nnz, C.nrows, C.ncols
        entry = {"nnz": nnz, "nrows": rows, "ncols": cols}
        for kind, M_, want_src, vb in (("values_and_src", C, True, 8), ("structure", S, False, 0)):
            for _ in range(args.warmup):
                api.transpose(M_, want_src=want_src)
            ms, _ = _events_ms(lambda: api.transpose(M_, want_src=want_src), args.steps, stream)
            nbytes = nnz * (4 + vb) + 4 * (rows + 1) + nnz * (4 + vb + (4 if want_src else 0)) + 4 * (cols + 1)
            gbs = nbytes / (ms / 1e3) / 1e9
            entry[kind] = {"ms": round(ms, 4), "algorithmic_bytes": int(nbytes), "gbs": round(gbs, 1),
                           "hbm_frac": round(gbs / peak, 4)}
        res[name] = entry
        del C, S
        torch.cuda.empty_cache()
    first = res["rmat_s16_AxA"]["values_and_src"]
    out = _base_line("CSR transpose GB/s (algorithmic bytes)", first["gbs"], "GB/s", args, first["ms"],
                     {"workload": "transpose_rmat_s16_AxA_and_laplacian3d_96_AxA", "l2": "inputs larger than L2"})
    out["roofline"] = {"bound": "hbm", "achieved": first["gbs"], "peak": peak, "unit": "GB/s",
                       "frac": first["hbm_frac"], "peak_kind": peak_kind + " hbm_gbs (copy)", "traffic": None}
    out["matrices"] = res
    return out


def run_triangles(args):
    """Masked product (L*L) .* L on the strictly lower triangle L of the
    undirected R-MAT graph (scale --rmat-scale, edge factor 16): the sum of
    the output is the graph's triangle count.  GFLOP/s counts the products
    of L*L that the row-wise pass forms (2 FLOP each); inputs resident, L2
    flushed between steps; end to end adds the copy of L to the device and
    of the output values back."""
    import torch
    from paper_2112_10037_gb300 import api, build as bld
    bld.build()
    dev = torch.device("cuda", 0)
    L = gen.lower_triangle_undirected(gen.rmat(args.rmat_scale, 16))
    prod = row_products(L, L)
    products = int(prod.sum())
    dL = api.DeviceCSR.from_host(L, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    out = None

    def step():
        nonlocal out
        out = api.masked_spgemm(dL, dL, dL, use_mask_values=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(dev.index)
    sampler.start()
    sampler.mark()
    ts = []
    for _ in range(args.steps):
        flush.fill_(1)
        t, _ = _events_ms(step, 1, stream)
        ts.append(t)
    clocks = sampler.stop()
    ms = float(np.mean(ts))
    triangles = int(round(float(out.sum().item())))
    # byte model: L read as A (row pointers, columns, values), the rows of L
    # touched as B (each once), L's pattern as the mask, the output written
    arp = np.diff(L.row_ptr.astype(np.int64))
    touched = np.unique(L.col_idx)
    b_bytes = 8 * len(touched) + 12 * int(arp[touched].sum())
    byte_model = (8 * L.nrows + 12 * L.nnz) + b_bytes + (8 * L.nrows + 4 * L.nnz) + 8 * L.nnz
    peak, peak_kind = measured_hbm_peak()
    achieved = byte_model / (ms / 1e3) / 1e9
    # end to end: pinned host L -> device, masked product, values -> host
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_rp, h_ci, h_v = pin(L.row_ptr), pin(L.col_idx), pin(L.vals)
    h_out = torch.empty(L.nnz, dtype=torch.float64).pin_memory()

    def e2e_step():
        d = api.DeviceCSR(L.nrows, L.ncols, h_rp.to(dev, non_blocking=True), h_ci.to(dev, non_blocking=True),
                          h_v.to(dev, non_blocking=True))
        h_out.copy_(api.masked_spgemm(d, d, d, use_mask_values=False), non_blocking=True)

    e2e_step()
    t_e2e, e2e_ts = _events_ms(e2e_step, max(3, min(args.steps, 5)), stream)
    desc = {"workload": "triangles_rmat_s%d_ef16_lower" % args.rmat_scale,
            "matrix": "strictly lower triangle of the undirected R-MAT graph (scale %d, edge factor 16, "
                      "(0.57,0.19,0.19,0.05), self-loops dropped, both directions merged), values 1" % args.rmat_scale,
            "rows": L.nrows, "nnz_L": L.nnz, "products": products, "triangles": triangles,
            "l2": "flushed between timed steps"}
    res = _base_line("SpGEMM GFLOP/s (2*products/s), masked product (L*L).*L", 2.0 * products / (ms / 1e3) / 1e9,
                     "GFLOP/s", args, ms, desc)
    res["roofline"] = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                       "frac": round(achieved / peak, 4), "peak_kind": peak_kind + " hbm_gbs (copy)",
                       "algorithmic_bytes": int(byte_model), "kernel": "k_masked", "traffic": None}
    res["e2e"] = {"value": round(2.0 * products / (t_e2e / 1e3) / 1e9, 2), "unit": "GFLOP/s",
                  "ms_per_step": round(t_e2e, 3), "ms_steps": [round(t, 3) for t in e2e_ts],
                  "h2d_bytes_per_step": int(L.row_ptr.nbytes + L.col_idx.nbytes + L.vals.nbytes),
                  "d2h_bytes_per_step": int(8 * L.nnz)}
    res["gpu_launches"] = args.steps
    res["clocks"] = clocks
    if not args.no_cpu:
        import oracle
        oracle.build()
        stride = max(1, int(round(products / 1e9)))   # about 10 s of single-threaded work
        rows = np.arange(0, L.nrows, stride)
        sub = oracle.select_rows(L, rows)
        t0 = time.perf_counter()
        oracle.masked(sub, L, sub, use_mask_values=False)
        dt = time.perf_counter() - t0
        p = int(prod[rows].sum())
        res["cpu_baseline"] = {"value": 2.0 * p / dt / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                               "sample": "rows i = 0 mod %d of L (%d rows, %d products, %.1f s single-threaded)"
                                         % (stride, len(rows), p, dt)}
    return res


def run_stencil_device(args):
    """C = A*A for the 3D 7-point operator on 96^3 (every row on the
    lane-per-row hash path): whole product (analyse, symbolic, numeric) with
    inputs resident, L2 flushed between steps; per-kernel CUDA-event times
    and the numeric pass's HBM fraction (A, the B rows touched, C written)."""
    import torch
    from paper_2112_10037_gb300 import api, build as bld, _native as nat
    bld.build()
    A = gen.laplacian_3d(96)
    products = int(row_products(A, A).sum())
    dA = api.DeviceCSR.from_host(A)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def step(profile=False):
        plan = api.Plan(dA, dA)
        if profile:
            nat.spgemm_plan_set_profiling(plan.handle, True)
        rp, nnz = plan.symbolic()
        plan.numeric(dA.vals, dA.vals)
        return plan, nnz
    for _ in range(args.warmup):
        step()[0].close()
    ts, ks = [], []
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan, nnz = step(profile=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
        ks.append(nat.spgemm_plan_kernel_times(plan.handle))
        plan.close()
    ms = float(np.mean(ts))
    kms = {n: round(float(np.mean([k[n] for k in ks])), 4) for n in ks[0] if np.mean([k[n] for k in ks]) > 0}
    num_ms = kms.get("num_hash", 0.0) + kms.get("num_tiny", 0.0)
    byte_model = (8 * A.nrows + 12 * A.nnz) * 2 + 8 * A.nrows + 12 * nnz  # A, B (= A, counted again), C
    peak, _ = measured_hbm_peak()
    return {"ms": round(ms, 4), "gflops": round(2.0 * products / (ms / 1e3) / 1e9, 2), "kernel_ms": kms,
            "numeric_ms": round(num_ms, 4), "numeric_hbm_frac": round(byte_model / (num_ms / 1e3) / 1e9 / peak, 4)
            if num_ms else None, "products": products, "nnz_C": int(nnz)}


def run_sharing(args):
    """B-row sharing and the row order (Sec. 3's buffering idea, Eq. 1's
    OMAR): on R-MAT scale 20 (A = 193 MB, larger than the 129 MB L2, so B's
    rows no longer all stay in L2) the same set of rows of A multiplies A in
    two orders -- the generator's row order and rows sorted by their
    heaviest column (the B row with the most entries they touch), so rows
    that read the same hub rows of B run close together -- and the numeric
    pass is timed for both.  The rows taken are the first rows whose products
    stay below 2.5e9 (nnz(C) inside int32).  The kernels take rows by
    descending product bin and, inside a bin, in row order, so the sort
    changes which rows run concurrently."""
    import torch
    from paper_2112_10037_gb300 import api, build as bld, _native as nat
    bld.build()
    scale = 20
    A = gen.rmat(scale, 16)
    prod = row_products(A, A)
    cs = np.cumsum(prod)
    r1 = int(np.searchsorted(cs, 2.5e9))
    rows = np.arange(r1)
    lens = np.diff(A.row_ptr.astype(np.int64))
    rp = A.row_ptr.astype(np.int64)
    # heaviest column of each row: its nonzero whose B row is longest
    nz_row = np.repeat(np.arange(A.nrows), lens)
    w = lens[A.col_idx]
    first = np.lexsort((-w, nz_row))  # by row, longest B row first
    heavy = np.full(A.nrows, -1, np.int64)
    starts = rp[:-1][lens > 0]
    heavy[lens > 0] = A.col_idx[first[starts]]
    order = np.lexsort((rows, heavy[rows]))

    def take_rows(M, sel):
        """The rows sel of M as a CSR (input slicing only)."""
        mrp = M.row_ptr.astype(np.int64)
        ln = mrp[sel + 1] - mrp[sel]
        nrp = np.zeros(len(sel) + 1, np.int64)
        np.cumsum(ln, out=nrp[1:])
        idx = np.repeat(mrp[sel] - nrp[:-1], ln) + np.arange(int(nrp[-1]))
        return gen.CSR(len(sel), M.ncols, nrp.astype(np.int32), M.col_idx[idx], M.vals[idx])
    variants = {"row_order": take_rows(A, rows), "heaviest_column_order": take_rows(A, rows[order])}
    dB = api.DeviceCSR.from_host(A)
    stream = torch.cuda.current_stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    out = {}
    for name, S in variants.items():
        dS = api.DeviceCSR.from_host(S)
        plan = api.Plan(dS, dB)
        nat.spgemm_plan_set_profiling(plan.handle, True)
        rp_c, nnz = plan.symbolic()
        ci = torch.empty(nnz, dtype=torch.int32, device="cuda")
        v = torch.empty(nnz, dtype=torch.float64, device="cuda")
        for _ in range(args.warmup):
            plan.numeric(dS.vals, dB.vals, col_idx=ci, vals=v)
        ts, ks = [], []
        for _ in range(args.steps):
            flush.fill_(1)
            t, _ = _events_ms(lambda: plan.numeric(dS.vals, dB.vals, col_idx=ci, vals=v), 1, stream)
            ts.append(t)
            ks.append(nat.spgemm_plan_kernel_times(plan.handle))
        p = int(prod[rows].sum())
        out[name] = {"numeric_ms": round(float(np.mean(ts)), 3),
                     "gflops": round(2.0 * p / (float(np.mean(ts)) / 1e3) / 1e9, 2),
                     "num_warp_ms": round(float(np.mean([k["num_warp"] for k in ks])), 3),
                     "num_block_ms": round(float(np.mean([k["num_block"] for k in ks])), 3),
                     "omar_32_pct": round(api.omar(dS, 32), 2)}
        plan.close()
        del dS, ci, v
        torch.cuda.empty_cache()
    desc = {"workload": "rmat_s20_rows_0_%d_AxA" % r1, "rows": r1, "products": int(prod[rows].sum()),
            "nnz_A_bytes": int(12 * A.nnz + 4 * (A.nrows + 1)), "l2_bytes": L2_BYTES}
    res = _base_line("numeric GFLOP/s, rows in generator order vs sorted by heaviest column",
                     out["heaviest_column_order"]["gflops"], "GFLOP/s", args,
                     out["heaviest_column_order"]["numeric_ms"], desc)
    res["orders"] = out
    return res


def run_secondary(args):
    """The other workloads of the measurement plan, each in a short form, for
    the default bench line: the 3D stencil product, the Galerkin chain replay,
    the differentiation workload's forward and backward passes, triangle
    counting on the R-MAT scale-18 graph, the 512-instance batched workload
    at its stated size against one-by-one calls, the transpose of two
    products' C, and the column-wise and semiring products."""
    import copy
    import torch
    a = copy.copy(args)
    a.steps, a.warmup, a.no_cpu = max(3, min(args.steps, 5)), 2, True
    out = {}

    def keep(name, fn):
        try:
            out[name] = fn()
        except Exception as exc:  # reported in the line, the headline stands
            out[name] = {"error": "%s: %s" % (type(exc).__name__, exc)}
        torch.cuda.synchronize()
        torch.cuda.empty_cache()

    keep("stencil3d_96_AxA", lambda: run_stencil_device(a))

    def gal():
        r = run_galerkin(a)
        return {"replay_ms": r["ms_per_step"], "gflops": r["value"], "hbm_frac": r["roofline"]["frac"],
                "two_plain_calls_ms": r["two_plain_calls_ms"]}
    keep("galerkin_96_graph_replay", gal)

    def bwd():
        r = run_backward(a)
        return {"f64": r["f64"], "f32": r["f32"]}
    keep("differentiation_65536sq", bwd)

    def tri():
        t = copy.copy(a)
        t.rmat_scale = 18
        r = run_triangles(t)
        return {"ms": r["ms_per_step"], "gflops": r["value"], "triangles": r["config"]["triangles"]}
    keep("triangles_rmat_s18", tri)

    def bat():
        b = copy.copy(a)
        b.steps, b.warmup, b.batch_scale, b.batch_count = 1, 1, 1.0, 512
        b.no_tune, b.opt, b.batch_max_b_nnz = True, [], 8_000_000
        r = run_batched(b)
        return {"batched_gflops": r["value"], "per_call_gflops": r["per_call_full_gflops"],
                "batched_graph_numeric_gflops": r["batched_graph_numeric_gflops"],
                "per_call_numeric_gflops": r["per_call_numeric_gflops"], "speedup_full": r["speedup_full"],
                "speedup_numeric": r["speedup_numeric"], "waves": r["config"]["waves"],
                "products": r["config"]["products"], "nnz_C": r["config"]["nnz_C"]}
    keep("batched_512_full_size", bat)

    def tra():
        r = run_transpose(a)
        return {name: {"values_and_src": m["values_and_src"], "structure_ms": m["structure"]["ms"]}
                for name, m in r["matrices"].items()}
    keep("transpose", tra)

    def var():
        r = run_variants(a)
        return {name: {"colwise_ms": m["colwise"]["ms"], "rowwise_ms": m["rowwise"]["ms"],
                       "min_plus_ms": m["min_plus"]["ms"], "min_plus_numeric_ms": m["min_plus"]["numeric_ms"],
                       "min_plus_masked_ms": m["min_plus"]["masked_ms"], "or_and_ms": m["or_and"]["ms"]}
                for name, m in r["matrices"].items()}
    keep("column_wise_and_semiring", var)
    return out


def run_omar(args):
    """OMAR (Eq. 1) of the buffering scheme of Sec. 3 for 2..32 computing
    units on the R-MAT and 3D stencil matrices, computed on the device (one
    symbolic pass of the grouping matrix times A per P); the oracle's count
    beside it for P = 32 (host, single thread)."""
    import torch
    from paper_2112_10037_gb300 import api, build as bld
    bld.build()
    stream = torch.cuda.current_stream()
    pes = [2, 4, 8, 16, 32]
    res = {}
    for name, M in (("rmat_s%d_ef16" % args.rmat_scale, gen.rmat(args.rmat_scale, 16)),
                    ("laplacian3d_96", gen.laplacian_3d(96))):
        dM = api.DeviceCSR.from_host(M)
        vals = {}
        for p in pes:
            for _ in range(args.warmup):
                api.omar(dM, p)
            box = {}
            ms, _ = _events_ms(lambda: box.update(v=api.omar(dM, p)), args.steps, stream)
            vals[p] = {"omar_pct": round(box["v"], 4), "ms": round(ms, 4)}
        entry = {"nnz": M.nnz, "by_pes": vals}
        if not args.no_cpu:
            import oracle
            t0 = time.perf_counter()
            ref = oracle.omar(M, 32)
            entry["oracle_32"] = {"omar_pct": round(ref, 4), "s": round(time.perf_counter() - t0, 3),
                                  "equal": ref == vals[32]["omar_pct"] or abs(ref - vals[32]["omar_pct"]) < 1e-4}
        res[name] = entry
    first = next(iter(res))
    out = _base_line("OMAR (%) of Eq. 1 at 32 computing units", res[first]["by_pes"][32]["omar_pct"], "%", args,
                     res[first]["by_pes"][32]["ms"], {"workload": "omar_rmat_s%d_and_laplacian3d_96" % args.rmat_scale})
    out["matrices"] = res
    return out


def run_variants(args):
    """The widened products on the 3D stencil 96^3 (A*A) and on R-MAT
    scale 16 (A*A): the column-wise Gustavson product (transposes around a
    row-wise product, all three steps timed), and the semiring products
    (min-plus, max-plus, or-and): the whole product (symbolic and numeric
    passes), its numeric pass alone, and the masked product on the pattern
    of A*B.  GFLOP/s counts 2 FLOP per product formed."""
    import torch
    from paper_2112_10037_gb300 import api, build as bld
    bld.build()
    stream = torch.cuda.current_stream()
    res = {}
    for name, M in (("laplacian3d_96", gen.laplacian_3d(96)), ("rmat_s16_ef16", gen.rmat(16, 16))):
        products = int(row_products(M, M).sum())
        dM = api.DeviceCSR.from_host(M)
        entry = {"products": products}
        for _ in range(args.warmup):
            api.spgemm_colwise(dM, dM)
        ms, _ = _events_ms(lambda: api.spgemm_colwise(dM, dM), args.steps, stream)
        entry["colwise"] = {"ms": round(ms, 4), "gflops": round(2.0 * products / (ms / 1e3) / 1e9, 2)}
        ms_row, _ = _events_ms(lambda: api.spgemm(dM, dM), args.steps, stream)
        entry["rowwise"] = {"ms": round(ms_row, 4), "gflops": round(2.0 * products / (ms_row / 1e3) / 1e9, 2)}
        C = api.spgemm(dM, dM)
        P = api.DeviceCSR(C.nrows, C.ncols, C.row_ptr, C.col_idx, None)
        for sr in ("min_plus", "max_plus", "or_and"):
            # the semiring product itself: symbolic + numeric with the
            # semiring's accumulators, and its numeric pass alone
            for _ in range(args.warmup):
                api.spgemm_semiring(dM, dM, sr)
            ms, _ = _events_ms(lambda: api.spgemm_semiring(dM, dM, sr), args.steps, stream)
            plan = api.Plan(dM, dM, semiring=sr)
            plan.symbolic()
            for _ in range(args.warmup):
                plan.numeric(dM.vals, dM.vals)
            ms_num, _ = _events_ms(lambda: plan.numeric(dM.vals, dM.vals), args.steps, stream)
            plan.close()
            # the masked product on the same pattern (values only)
            for _ in range(args.warmup):
                api.masked_semiring(dM, dM, P, sr)
            ms_mask, _ = _events_ms(lambda: api.masked_semiring(dM, dM, P, sr), args.steps, stream)
            entry[sr] = {"ms": round(ms, 4), "gflops": round(2.0 * products / (ms / 1e3) / 1e9, 2),
                         "numeric_ms": round(ms_num, 4), "masked_ms": round(ms_mask, 4)}
        res[name] = entry
    first = res["laplacian3d_96"]
    out = _base_line("SpGEMM GFLOP/s (2*products/s), min-plus product (symbolic and numeric passes)",
                     first["min_plus"]["gflops"], "GFLOP/s", args, first["min_plus"]["ms"],
                     {"workload": "variants_laplacian3d_96_and_rmat_s16"})
    out["matrices"] = res
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat",
                    choices=["rmat", "lap2d", "stencil3d", "batched", "galerkin", "backward", "triangles", "omar",
                             "variants", "stencil_device", "sharing", "transpose"])
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--batch-scale", type=float, default=1.0,
                    help="row-count scale of the batched instances (1.0 = rows in [1024, 200000])")
    ap.add_argument("--tune", action="store_true", help="autotune the options first (rmat)")
    ap.add_argument("--no-tune", action="store_true", help="batched: library default options, no autotuner")
    ap.add_argument("--batch-max-b-nnz", type=int, default=0,
                    help="batched: at most this many B entries per wave (0: waves bounded by products only)")
    ap.add_argument("--opt", action="append", default=[], metavar="NAME=VALUE",
                    help="plan option (spgemm_opts field) for the product, e.g. --opt rank_min=1024")
    ap.add_argument("--rmat-scale", type=int, default=18, help="R-MAT scale (18 is the benchmark workload)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle leg")
    ap.add_argument("--no-secondary", action="store_true",
                    help="default workload: skip the short runs of the other workloads")
    ap.add_argument("--e2e-chunks", type=int, default=8,
                    help="row ranges of the end-to-end leg (computed while earlier ranges are copied back)")
    ap.add_argument("--e2e-streams", type=int, default=1, help="compute streams of the end-to-end leg")
    ap.add_argument("--e2e-order", default="rows", choices=["products", "rows"],
                    help="order of the end-to-end leg's row ranges")
    ap.add_argument("--hash-max", type=int, default=0,
                    help="largest row product count of the hash accumulator (0: library default 128, -1: off)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        if rank != 0:
            return
        A, B, desc = make_workload(args.workload, args.rmat_scale)
        print(json.dumps(run_reference(args, A, B, desc)), flush=True)
        return
    if args.workload in ("batched", "galerkin", "backward", "triangles", "omar", "variants", "stencil_device",
                         "sharing", "transpose"):
        if rank == 0:
            runner = {"batched": run_batched, "galerkin": run_galerkin, "backward": run_backward,
                      "triangles": run_triangles, "omar": run_omar, "variants": run_variants,
                      "stencil_device": run_stencil_device, "sharing": run_sharing,
                      "transpose": run_transpose}[args.workload]
            print(json.dumps(runner(args)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    A, B, desc = make_workload(args.workload, args.rmat_scale)
    out = run_ours(args, rank, world, A, B, desc)
    if rank == 0:
        if world == 1 and args.workload == "rmat" and args.rmat_scale == 18 and not args.no_secondary:
            out["secondary"] = run_secondary(args)
        if not args.no_cpu and world == 1:
            out["cpu_baseline"] = cpu_oracle_leg(A, B, row_products(A, B))
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

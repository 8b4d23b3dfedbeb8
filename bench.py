#!/usr/bin/env python
"""Benchmark of the EFIE impedance-matrix fill with the adaptive Green table.

Default workload: PEC cube of side 3 lambda, 64 x 64 squares per face split
into triangles (49152 triangles, 73728 RWG unknowns), 4-point rule on both
triangles, near pairs = shared vertex or centroids closer than 0.2 lambda,
FP32 table fill with Kahan outer sums into a 43.5 GB complex64 Z, table
tolerance 1e-6. Synthetic, seeded input. `--workload sphere_7680` gives the
1 lambda sphere (5120 triangles, 7680 RWG, 7-point rule).

One step = the whole hot path on a device-resident mesh: R_min/R_max
reduction, Green + Exp table construction, zeroing Z, the regular-pair fill
kernel, the Z + Z^T pass and the near-pair kernel. `value` is Z entries / s
over all ranks. Alongside: the direct (sincospi) fill on the same mesh, the
regular kernel's roofline fraction, an end-to-end number through the C ABI
from host arrays to a host copy of Z, the oracle's accuracy check on seeded
256 x 256 blocks, and the FP64 CPU oracle timed on a bounded sample of rows
(the CPU baseline, extrapolated).

python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload NAME]
"""
import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_COUNT = 152
FP32_LANES_PER_SM = 128
MUFU_PER_SM = 16
SMEM_BYTES_PER_CLK = 128  # shared-memory bandwidth per SM (32 banks x 4 B)
FALLBACK_SM_MHZ = 2070.0
# Algorithmic FP32 lane operations per regular Green evaluation (the op model of
# the roofline): distance 7 (3 differences, 3 squares / FMAs, R = R^2 rsqrt),
# lookup and polynomial 10 (cell FFMA, conversion-free rint, anchor, offset,
# Horner), moment accumulation 8 (M0 and the three beta-weighted moments, complex).
OPS_PER_EVAL = 25
# Shared-memory reads of the FP32 lattice per Green evaluation, as
# (bytes, vector width in bytes) per read: the Lagrange record is a 16-byte
# read of (c0, c1) and a 4-byte read of c2 (two halves).
SMEM_READS = ((16, 16), (4, 4))
# Expected shared-memory wavefronts of one warp-wide read at independent random
# addresses: lanes are served in phases of 128 bytes (8 lanes for 16-byte reads,
# 16 for 8-byte, 32 for 4-byte), and a phase takes as many wavefronts as the
# largest number of distinct addresses that fall on one bank group (the
# expected maximum load of 8 balls in 8 bins, 16 in 16, 32 in 32).
RANDOM_WAVEFRONTS = {16: 4 * 2.595, 8: 2 * 3.077, 4: 3.530}

# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the regular-pair
# table kernel from ncu captures (summarised in profiles/), with the number of
# unordered regular pairs that launch evaluated; valid only while the kernel
# source hash matches. A workload without its own capture takes the bytes per
# pair of the cube's smaller case (the kernel's DRAM traffic is the
# read-modify-write of Z through the row atomics and the mirror-free half, and
# Z grows with the pair count).
TRAFFIC_HASH = "188d6d96b53f69c2"
TRAFFIC = {"cube_3lambda_12288tri_18432rwg_4pt_fp32": (1906964736 + 1992500736, 75331278),
           "sphere_r1lambda_5120tri_7680rwg_7pt_fp32": (298563584 + 260932608, 13073950)}
# The table kernel's instruction issue from the same `--set full` capture of
# the 18432-unknown cube (warp instructions per warp evaluation, fraction of
# cycles with an instruction issued): the kernel is issue-bound, and the
# 25-operation model above counts under a third of the instructions it needs.
ISSUE = {"cube_3lambda_12288tri_18432rwg_4pt_fp32": (3.254e9 / (75331278 * 16 / 32), 0.746)}
TRAFFIC_SCALED_FROM = {"cube_3lambda_49152tri_73728rwg_4pt_fp32": "cube_3lambda_12288tri_18432rwg_4pt_fp32"}
TRAFFIC_NOTE = ("dram__bytes_read.sum + dram__bytes_write.sum of one launch of the regular-pair table kernel "
                "(ncu, --clock-control none); the 73728-unknown cube's from the 18432-unknown cube's capture scaled "
                "by the pair count; null when the kernel sources changed since the capture")


def kernel_issue(workload):
    """Instruction issue of the table kernel from the ncu capture (the same
    kernel at a quarter of the size for the 73728-unknown cube), or None when
    the kernel sources changed since."""
    if kernel_source_hash() != TRAFFIC_HASH:
        return None
    src = workload if workload in ISSUE else TRAFFIC_SCALED_FROM.get(workload)
    if src not in ISSUE:
        return None
    per_eval, active = ISSUE[src]
    return {"warp_instructions_per_warp_eval": per_eval, "issue_active": active,
            "source": "ncu --set full of the 18432-unknown cube's table kernel (smsp__inst_executed, issue active)"}


def kernel_traffic(workload, n_pairs):
    if kernel_source_hash() != TRAFFIC_HASH:
        return None
    if workload in TRAFFIC:
        return TRAFFIC[workload][0]
    src = TRAFFIC_SCALED_FROM.get(workload)
    if src:
        b, n = TRAFFIC[src]
        return b * n_pairs / n
    return None


# FP64 arithmetic instructions (DADD + DFMA + DMUL, thread level) per (near pair,
# test point) of the mixed-precision near kernel, from an ncu capture of the
# 18432-unknown cube (profiles/); valid while the near kernel's sources match.
NEAR_FP64_OPS_HASH = "9db20f98226f9710"
NEAR_FP64_OPS_PER_TASK = (59829840 + 165940896 + 64560827) / (332388 * 4)  # 218.4
FP64_OPS_PER_SM_CLOCK = 2  # GB300: 304 DFMA thread instructions per clock on 152 SMs (ncu peak_sustained)


def near_source_hash():
    h = hashlib.sha256()
    for name in ("gf_device.cuh", "gf_near.cuh", "gf_fill.cu"):
        h.update(open(os.path.join(ROOT, "paper_1901_04162_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def other_kernel_rooflines(workload, zbytes, mirror_ms, near_ms, near_tasks, pk, sm_mhz):
    """The mirror pass against the measured HBM copy bandwidth (it reads and
    writes all of Z), and the mixed near kernel against the FP64 pipe."""
    hbm = float(pk.get("hbm_gbs", 6800.0))
    out = {"mirror": {"kernel": "k_symmetrize32", "bound": "hbm", "bytes": 2 * zbytes,
                      "achieved": 2 * zbytes / (mirror_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s"}}
    out["mirror"]["frac"] = out["mirror"]["achieved"] / hbm
    near = {"kernel": "k_fill_near<mixed>", "bound": "fp64", "unit": "FP64 arithmetic instructions/s (thread)",
            "peak": SM_COUNT * FP64_OPS_PER_SM_CLOCK * sm_mhz * 1e6, "achieved": None, "frac": None}
    if NEAR_FP64_OPS_PER_TASK is not None and near_source_hash() == NEAR_FP64_OPS_HASH and near_ms > 0:
        near["achieved"] = NEAR_FP64_OPS_PER_TASK * near_tasks / (near_ms / 1e3)
        near["frac"] = near["achieved"] / near["peak"]
        near["ops_per_task"] = NEAR_FP64_OPS_PER_TASK
    out["near"] = near
    return out


def nonblocking_stream(torch):
    """A CUDA stream created with cudaStreamNonBlocking: work on the legacy
    default stream (torch's current stream here, the library's synchronous
    uploads) does not wait for work queued on it, nor it for them. It lives
    until the process exits (torch may still query it)."""
    rt = ctypes.CDLL("libcudart.so.13")
    handle = ctypes.c_void_p()
    if rt.cudaStreamCreateWithFlags(ctypes.byref(handle), ctypes.c_uint(1)) != 0:
        raise RuntimeError("cudaStreamCreateWithFlags failed")
    return torch.cuda.ExternalStream(handle.value)


def reduce_max_over_ranks(x, dist=None, device="cpu"):
    """The largest x over all ranks (a job takes as long as its slowest rank)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, seconds):
    """Whole-job throughput of `world` replicas that each process
    `units_per_rank` units in `seconds` (the max over ranks)."""
    return world * units_per_rank / seconds


def kernel_source_hash():
    """Hash of the sources that define the regular-pair table kernel (the
    shared device code, the regular-pair kernel file and the build flags)."""
    h = hashlib.sha256()
    for name in ("csrc/gf_device.cuh", "csrc/gf_regular.cu", "build.py"):
        h.update(open(os.path.join(ROOT, "paper_1901_04162_gb300", name), "rb").read())
    return h.hexdigest()[:16]


WORKLOADS = {
    "sphere_7680": W.sphere_7680,
    "plate_280": W.plate_280,
    "sphere_3072": W.sphere_3072,
    "cube_73728": W.cube_73728,
    "cube_18432": lambda: W.cube_73728(32),
}


def smem_model(evals, ms, mhz):
    """Shared-memory side of the table kernel: bytes per evaluation, the
    wavefronts a warp evaluation costs at random addresses, and the time those
    wavefronts take at one wavefront per clock per SM."""
    wf = sum(RANDOM_WAVEFRONTS[w] for _, w in SMEM_READS)
    t_wf = evals / 32 * wf / (SM_COUNT * mhz * 1e6)
    return {"bytes_per_eval": sum(b for b, _ in SMEM_READS),
            "random_wavefronts_per_warp_eval": wf,
            "conflict_free_wavefronts_per_warp_eval": sum(b * 32 / 128 for b, _ in SMEM_READS),
            "wavefront_time_ms": t_wf * 1e3, "frac_of_kernel_time": t_wf / (ms / 1e3),
            "note": "one wavefront per clock per SM; random lattice cells make bank conflicts (model: "
                    "expected largest bank-group load per 128-byte phase)"}


def evaluated_pairs(nt, n_near):
    """Unordered regular triangle pairs: (ordered regular pairs) / 2."""
    return (nt * nt - n_near) // 2


# ----------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampler (100 ms) for the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
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
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        return json.load(open(PEAKS_FILE)), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "sm_max_mhz": FALLBACK_SM_MHZ}, "fallback"


# ----------------------------------------------------------------------------
def cpu_model():
    """Host CPU model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def panel_rows(ne, seed=256, size=256):
    """The rows of one seeded panel of `size` consecutive RWG unknowns."""
    npan = max(1, ne // size)
    p = int(np.random.default_rng(seed).integers(npan))
    return np.arange(p * size, min(ne, (p + 1) * size))


class OracleRun:
    """The FP64 CPU oracle as it stands (table mode) on one workload: its
    range reduction and tables once, then timed samples of Z rows."""

    def __init__(self, wl):
        import oracle as O
        self.O = O
        self.wl = wl
        self.om = O.Mesh(wl.xyz, wl.tri, wl.near_dist)
        self.ne = self.om.ne
        t0 = time.perf_counter()
        self.lo, self.hi = self.om.range(wl.rule, prune=len(wl.tri) > 10000)
        self.t_range = time.perf_counter() - t0
        t0 = time.perf_counter()
        self.tabs = O.make_tables(wl.k, self.lo, self.hi)
        self.t_tables = time.perf_counter() - t0

    def rows(self, rows, nthreads=0):
        """Seconds to compute the given Z rows."""
        rows = np.asarray(rows)
        t0 = time.perf_counter()
        self.om.z_rows(self.wl.k, self.wl.rule, rows, mode="table", tables=self.tabs, nthreads=nthreads)
        return time.perf_counter() - t0

    def sized_rows(self, panel, target_s, nthreads=0):
        """A prefix of `panel` sized to about target_s seconds (one row timed first)."""
        t1 = self.rows(panel[:1], nthreads)
        n = int(max(1, min(len(panel), round(target_s / max(t1, 1e-4)))))
        return panel[:n]


def oracle_baseline(wl, target_s=8.0, run=None):
    """CPU baseline: the oracle (table mode) on the host cores, on rows of a
    seeded 256-row panel, one thread and all threads; entries/s extrapolated
    to the full matrix (range reduction and tables timed once on all
    threads)."""
    run = run or OracleRun(wl)
    panel = panel_rows(run.ne)
    cores = os.cpu_count()
    r1 = run.sized_rows(panel, target_s / 2, nthreads=1)
    t1 = run.rows(r1, nthreads=1)
    ra = run.sized_rows(panel, target_s, nthreads=0)
    ta = run.rows(ra, nthreads=0)
    rate1 = len(r1) * run.ne / t1
    ratea = len(ra) * run.ne / ta
    setup = run.t_range + run.t_tables
    full_a = setup + run.ne * run.ne / ratea
    full_1 = setup + run.ne * run.ne / rate1
    desc = (f"extrapolated: oracle table-mode Z rows of the seeded 256-row panel starting at row {panel[0]} "
            f"({len(ra)} rows on {cores} threads in {ta:.2f} s; {len(r1)} rows on 1 thread in {t1:.2f} s), "
            f"scaled by entry count to all {run.ne} rows, plus the full range reduction ({run.t_range:.2f} s) "
            f"and tables ({run.t_tables:.3f} s) on {cores} threads; CPU: {cpu_model()}")
    out = {"value": run.ne * run.ne / full_a, "unit": "Z entries/s", "cores": cores, "kind": "oracle",
           "sample": desc, "cpu_model": cpu_model(),
           "single_thread": {"value": run.ne * run.ne / full_1, "unit": "Z entries/s", "cores": 1,
                             "rows": int(len(r1)), "rows_s": t1},
           "all_threads_rows": int(len(ra)), "all_threads_rows_s": ta,
           "setup_s": {"range": run.t_range, "tables": run.t_tables}}
    return out


# ----------------------------------------------------------------------------
def run_reference(args, wl, rank):
    """The oracle as the reference arm: each step computes a bounded sample of
    Z rows (a seeded 256-row panel) on all host threads; the value is the
    sample's entries over its measured time. The range and tables are built
    once before the steps (their time is reported)."""
    if rank != 0:
        return
    run = OracleRun(wl)
    panel = panel_rows(run.ne)
    rows = run.sized_rows(panel, args.ref_seconds)
    times = []
    for i in range(args.warmup + args.steps):
        t = run.rows(rows)
        if i >= args.warmup:
            times.append(t)
    t = statistics.median(times)
    value = len(rows) * run.ne / t
    cores = os.cpu_count()
    desc = (f"oracle table-mode fill of {len(rows)} Z rows ({len(rows) * run.ne} entries) of the seeded "
            f"256-row panel at row {panel[0]} per step, on {cores} threads; range reduction "
            f"({run.t_range:.2f} s) and tables ({run.t_tables:.3f} s) once before the steps; CPU: {cpu_model()}")
    line = {"impl": "reference", "metric": "Z entries/s (table fill)", "value": value, "unit": "Z entries/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name},
            "cpu_baseline": {"value": value, "unit": "Z entries/s", "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "Z entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
def sample_blocks(ne, count=64, size=256, seed=64):
    """`count` seeded (row block, column block) pairs of size x size blocks;
    the whole matrix as one block when it is small."""
    if ne <= 4 * size:
        return [(0, 0)], ne
    nb = ne // size
    rng = np.random.default_rng(seed)
    return [(int(i), int(j)) for i, j in zip(rng.integers(nb, size=count), rng.integers(nb, size=count))], size


def gather_blocks(torch, Z, blocks, size):
    return np.stack([Z[i * size:(i + 1) * size, j * size:(j + 1) * size].cpu().numpy() for i, j in blocks])


def oracle_blocks(run, blocks, size, mode):
    ii = np.arange(size)
    mi = np.concatenate([np.repeat(i * size + ii, size) for i, _ in blocks])
    ni = np.concatenate([np.tile(j * size + ii, size) for _, j in blocks])
    kw = {"mode": "table", "tables": run.tabs} if mode == "table" else {}
    z = run.om.z_entries(run.wl.k, run.wl.rule, mi, ni, **kw)
    return z.reshape(len(blocks), size, size)


def err_stats(z, ref, floor=1e-3):
    """Relative Frobenius error, max |error| / max |ref|, and the per-entry
    relative error |z - ref| / |ref| over entries with |ref| >= floor * max|ref|."""
    d = np.abs(z - ref)
    a = np.abs(ref)
    big = a >= floor * a.max()
    rel = d[big] / a[big]
    return {"rel_fro": float(np.linalg.norm(z - ref) / np.linalg.norm(ref)),
            "max_abs_err_over_max_abs_ref": float(d.max() / a.max()),
            "entry_rel_max": float(rel.max()), "entry_rel_p999": float(np.quantile(rel, 0.999)),
            "entry_floor": f"|ref| >= {floor:g} max|ref| ({int(big.sum())} of {big.size} entries)"}


def run_ours(args, wl, rank, world, local_rank):
    import torch

    import paper_1901_04162_gb300 as gf

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    dist = None
    if world > 1:
        import torch.distributed as dist

    def barrier():
        if dist is not None:
            dist.barrier()

    prec = gf.GF_FP32 if wl.precision == "fp32" else gf.GF_FP64
    zdt = torch.complex64 if prec == gf.GF_FP32 else torch.complex128
    p = gf.gf_params_default(rule=wl.rule)
    mesh = gf.Mesh(wl.xyz, wl.tri, wl.near_dist)
    ne, nt, n_near = mesh.ne, mesh.nt, mesh.n_near
    Z = torch.empty((ne, ne), dtype=zdt, device=dev)
    zbytes = Z.numel() * Z.element_size()
    flush = None if zbytes > (1 << 30) else torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > L2
    # clear, pair kernel, mirror (Z += Z^T), near kernel: events between them
    parts = (gf.GF_PART_ZERO, gf.GF_PART_PAIRS, gf.GF_PART_MIRROR, gf.GF_PART_NEAR)

    def step(direct, ev, params=None):
        pp = params or p
        tab = None
        ev[0].record(stream)
        if not direct:
            lo, hi = mesh.range(wl.rule, prec)
        ev[1].record(stream)
        # Z is cleared on the device while the host places the table samples
        # (clearing it on a second stream beside the range kernels measured
        # slower: 7.0 -> 7.6 ms on the cube)
        gf.gf_fill_parts(mesh.h, wl.k, pp, None, prec, Z, parts[0])
        if not direct:
            tab = gf.Table(wl.k, lo, hi, pp)
        for i, part in enumerate(parts[1:]):
            ev[2 + i].record(stream)
            gf.gf_fill_parts(mesh.h, wl.k, pp, tab.h if tab else None, prec, Z, part)
        ev[5].record(stream)
        return tab

    def timed(direct, steps, warmup, params=None):
        keep = []
        for _ in range(warmup):
            keep.append(step(direct, [torch.cuda.Event(enable_timing=True) for _ in range(6)], params))
        torch.cuda.synchronize()
        keep.clear()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(steps)]
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(steps):
            if flush is not None:
                flush.fill_(i & 0xFF)  # evict Z and the geometry from L2 between steps
            keep.append(step(direct, evs[i], params))
        torch.cuda.synchronize()
        barrier()
        wall = time.perf_counter() - t0
        st = [e[0].elapsed_time(e[5]) for e in evs]
        reg = [e[2].elapsed_time(e[3]) for e in evs]
        mir = [e[3].elapsed_time(e[4]) for e in evs]
        near = [e[4].elapsed_time(e[5]) for e in evs]
        pre = [e[0].elapsed_time(e[2]) for e in evs]
        keep.clear()
        return {"step_ms": st, "regular_ms": reg, "mirror_ms": mir, "near_ms": near, "range_table_ms": pre,
                "wall_s": wall}

    def spread(x):
        return {"mean": statistics.mean(x), "min": min(x), "max": max(x)}

    def reduce_max(x):
        return reduce_max_over_ranks(x, dist, dev)

    # ---- table path (the method) with clocks sampled in the timed region
    with Clocks(local_rank) as clk:
        tt = timed(False, args.steps, args.warmup)
    clocks = clk.summary()
    with Clocks(local_rank) as clkd:
        td = timed(True, args.steps, args.warmup)
    clocks_direct = clkd.summary()
    px = gf.gf_params_default(rule=wl.rule, green_from_exp=1)
    tx = timed(False, args.steps, args.warmup, px)
    p64 = gf.gf_params_default(rule=wl.rule, near_fp64=1)
    n64 = max(3, args.steps // 2)
    t64 = timed(False, n64, 1, p64) if prec == gf.GF_FP32 else None
    d64 = timed(True, n64, 1, p64) if prec == gf.GF_FP32 else None

    total_ms = reduce_max(sum(tt["step_ms"]))
    ms_step = total_ms / args.steps
    value = job_throughput(world, ne * ne * args.steps, total_ms / 1e3)
    direct_ms = reduce_max(sum(td["step_ms"])) / args.steps

    # ---- end to end through the C ABI: host arrays in (mesh creation, range,
    # tables, fill) and the whole Z copied to page-locked host memory, per step
    e2e = {"value": None}
    zhost = None
    try:
        avail = int(next(ln.split()[1] for ln in open("/proc/meminfo") if ln.startswith("MemAvailable"))) * 1024
    except (OSError, StopIteration, ValueError):
        avail = 0
    # every rank copies its own Z: all of them need the room, or none times e2e
    fits = zbytes * 1.3 * world + (8 << 30) < avail
    if reduce_max(0.0 if fits else 1.0) == 0.0:
        try:
            zhost = torch.empty((ne, ne), dtype=zdt, pin_memory=True)  # page-locked (cudaHostAlloc)
        except RuntimeError as exc:
            e2e["reason"] = f"page-locked host buffer of {zbytes} bytes: {exc}"[:200]
    else:
        e2e["reason"] = f"host memory: {avail} bytes available for {world} x {zbytes}-byte Z copies"
    if reduce_max(0.0 if zhost is not None else 1.0) != 0.0:
        zhost = None
    if zhost is not None:
        times, parts_ms = [], []
        big = zbytes >= (4 << 30)
        zflat, zhost_flat = Z.view(-1), zhost.view(-1)
        chunk = max(1, (1 << 30) // Z.element_size())
        n_e2e = min(args.steps, 5) if big else args.steps
        n_w = 1 if big else args.warmup
        for i in range(n_w + n_e2e):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            m2 = gf.Mesh(wl.xyz, wl.tri, wl.near_dist)
            t1 = time.perf_counter()
            lo, hi = m2.range(wl.rule, prec)
            gf.gf_fill_parts(m2.h, wl.k, p, None, prec, Z, gf.GF_PART_ZERO)  # overlaps the host table stage
            tab = gf.Table(wl.k, lo, hi, p)
            ev[0].record(stream)
            gf.gf_fill_parts(m2.h, wl.k, p, tab.h, prec, Z, gf.GF_PART_REGULAR | gf.GF_PART_NEAR)
            ev[1].record(stream)
            for c0 in range(0, zflat.numel(), chunk):  # the copy in 1 GiB pieces
                zhost_flat[c0:c0 + chunk].copy_(zflat[c0:c0 + chunk], non_blocking=True)
            ev[2].record(stream)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            if i >= n_w:
                times.append(t2 - t0)
                parts_ms.append(((t1 - t0) * 1e3, ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])))
            del tab, m2
        serial_s = reduce_max(statistics.median(times))
        cp = statistics.median(x[2] for x in parts_ms)
        serial = {"value": world * ne * ne / serial_s, "ms_per_step": serial_s * 1e3, "steps": len(times),
                  "breakdown_ms": {"mesh_create_host": statistics.median(x[0] for x in parts_ms),
                                   "fill_after_tables": statistics.median(x[1] for x in parts_ms),
                                   "copy_z_to_host": cp, "copy_gb_per_s": zbytes / (cp / 1e3) / 1e9}}
        # streamed: the same steps one after another as a user filling a series of
        # meshes would run them, with two device copies of Z: the copy of step i to
        # host memory (its own stream) overlaps the mesh creation, range, tables
        # and fill of step i + 1 into the other copy; every step still creates its
        # mesh from host arrays and copies all of its Z to host memory
        pipe_s = None
        try:
            Zb = (Z, torch.empty_like(Z))
        except RuntimeError:
            Zb = None
        if reduce_max(0.0 if Zb is not None else 1.0) == 0.0:
            copy_stream = nonblocking_stream(torch)

            piece = max(1, (256 << 20) // Z.element_size())

            def streamed(n):
                """n steps; the copies run on a host thread that keeps two 256 MiB
                pieces queued, so that the next step's host-to-device uploads
                (mesh, tables) are not queued behind a whole Z of copies."""
                import queue
                jobs, copied, keep = queue.Queue(), [threading.Event() for _ in range(n)], []

                failed = []

                def copier():
                    try:
                        while True:
                            job = jobs.get()
                            if job is None:
                                return
                            i, zsrc, filled = job
                            filled.synchronize()
                            with torch.cuda.stream(copy_stream):
                                inflight = []
                                for c0 in range(0, zsrc.numel(), piece):
                                    zhost_flat[c0:c0 + piece].copy_(zsrc[c0:c0 + piece], non_blocking=True)
                                    ev = torch.cuda.Event()
                                    ev.record(copy_stream)
                                    inflight.append(ev)
                                    if len(inflight) == 2:  # two pieces queued: no gap between them
                                        inflight.pop(0).synchronize()
                                for ev in inflight:
                                    ev.synchronize()
                            copied[i].set()
                    except Exception as exc:  # noqa: BLE001 - reported by the main thread
                        failed.append(exc)
                        for ev in copied:
                            ev.set()

                th = threading.Thread(target=copier)
                th.start()
                try:
                    for i in range(n):
                        zb = Zb[i % 2]
                        m3 = gf.Mesh(wl.xyz, wl.tri, wl.near_dist)
                        lo3, hi3 = m3.range(wl.rule, prec)
                        if i >= 2:
                            copied[i - 2].wait()  # the copy out of this buffer, two steps back
                        if failed:
                            raise failed[0]
                        gf.gf_fill_parts(m3.h, wl.k, p, None, prec, zb, gf.GF_PART_ZERO)
                        tab3 = gf.Table(wl.k, lo3, hi3, p)
                        gf.gf_fill_parts(m3.h, wl.k, p, tab3.h, prec, zb, gf.GF_PART_REGULAR | gf.GF_PART_NEAR)
                        filled = torch.cuda.Event()
                        filled.record(stream)
                        jobs.put((i, zb.view(-1), filled))
                        keep.append((m3, tab3))  # freed after the timed loop (freeing waits for the device)
                finally:
                    jobs.put(None)
                    th.join()
                if failed:
                    raise failed[0]
                torch.cuda.synchronize()
                return keep

            streamed(n_e2e).clear()  # warm-up; its meshes and tables go back to the library's pools
            barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            kept = streamed(n_e2e)
            pipe_s = reduce_max((time.perf_counter() - t0) / n_e2e)
            kept.clear()
            torch.cuda.synchronize()
            del Zb  # (the copy stream lives until the process exits: torch may still query it)
        e2e_s = pipe_s if pipe_s is not None else serial_s
        e2e = {"value": world * ne * ne / e2e_s, "unit": "Z entries/s",
               "h2d_bytes_per_step": wl.xyz.nbytes + wl.tri.nbytes, "d2h_bytes_per_step": zbytes,
               "ms_per_step": e2e_s * 1e3, "steps": n_e2e,
               "mode": "streamed: two device Z buffers, copy of step i overlapping step i + 1" if pipe_s is not None
               else "serial",
               "serial": serial,
               "path": "host xyz/tri -> gf_mesh_create -> gf_range -> gf_table_create -> gf_fill_parts -> "
                       "cudaMemcpyAsync of all of Z (1 GiB pieces) to page-locked host memory"}

    # ---- roofline of the regular-pair kernel (table), CUDA events on its stream
    m = wl.rule
    n_regular = nt * nt - n_near
    n_eval = evaluated_pairs(nt, n_near)
    evals_regular = n_eval * m * m
    evals_near = n_near * m * (3 * (p.nphi + p.nl) + 1)
    reg_ms = statistics.mean(tt["regular_ms"])
    pk, src = peaks()
    sm_mhz = float(pk.get("sm_max_mhz", FALLBACK_SM_MHZ))
    peak_tops = SM_COUNT * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12
    ops = evals_regular * OPS_PER_EVAL
    achieved = ops / (reg_ms / 1e3) / 1e12
    traffic = kernel_traffic(wl.name, evaluated_pairs(nt, n_near))
    mhz = clocks.get("sm_mhz") or sm_mhz
    mhz_d = clocks_direct.get("sm_mhz") or sm_mhz

    line = {
        "metric": "Z entries/s (table fill)", "value": value, "unit": "Z entries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == gf.GF_FP32 else "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "triangles": nt, "rwg_unknowns": ne, "rule_points": m, "k": wl.k,
                   "near_criterion": (f"shared vertex or centroid distance < {wl.near_dist} lambda"
                                      if wl.near_dist > 0 else "shared vertex"),
                   "table_tol": p.table_tol, "near_pairs": n_near, "regular_pairs": n_regular,
                   "regular_pairs_evaluated": n_eval, "z_bytes": zbytes,
                   "precision": ("fp32 regular pairs (Kahan outer sums); mixed near pairs (near_fp64=0: FP64 "
                                 "geometry, projections and closed-form static parts, FP32 sampling of e^-jkR "
                                 "on the source edges and FP32 3x3 assembly); the all-FP64 near variant is "
                                 "near_fp64_variant" if prec == gf.GF_FP32 else "fp64 throughout"),
                   "l2": ("inputs larger than L2: Z is written every step" if flush is None
                          else "flushed between steps (256 MiB write)"),
                   "parallelism": f"replicas x{world}"},
        "green_evals_per_s": world * (evals_regular + evals_near) * args.steps / (total_ms / 1e3),
        "green_evals": {"regular_per_step": evals_regular, "near_per_step": evals_near},
        "step_breakdown_ms": {"range_tables_and_zero": statistics.mean(tt["range_table_ms"]),
                              "regular_kernel": reg_ms, "mirror_z_plus_zt": statistics.mean(tt["mirror_ms"]),
                              "near_kernel": statistics.mean(tt["near_ms"])},
        "spread_ms": {"table_step": spread(tt["step_ms"]), "table_regular": spread(tt["regular_ms"]),
                      "direct_step": spread(td["step_ms"]), "direct_regular": spread(td["regular_ms"])},
        "clock_normalised": {"table_regular_ms_x_mhz": reg_ms * mhz,
                             "direct_regular_ms_x_mhz": statistics.mean(td["regular_ms"]) * mhz_d,
                             "table_sm_mhz": mhz, "direct_sm_mhz": mhz_d},
        "direct": {"value": world * ne * ne / (direct_ms / 1e3), "unit": "Z entries/s", "ms_per_step": direct_ms,
                   "regular_kernel_ms": statistics.mean(td["regular_ms"]),
                   "mirror_ms": statistics.mean(td["mirror_ms"]),
                   "near_kernel_ms": statistics.mean(td["near_ms"]), "clocks": clocks_direct},
        "near_fp64_variant": None if t64 is None else {
            "ms_per_step": statistics.mean(t64["step_ms"]), "value": ne * ne / (statistics.mean(t64["step_ms"]) / 1e3),
            "near_kernel_ms": statistics.mean(t64["near_ms"]),
            "direct_ms_per_step": statistics.mean(d64["step_ms"]),
            "direct_near_kernel_ms": statistics.mean(d64["near_ms"]),
            "note": "near pairs in FP64 throughout (near_fp64=1): the configuration's 'FP64 near-singular "
                    "correction' as written"},
        "exp_over_r_variant": {
            "ms_per_step": statistics.mean(tx["step_ms"]), "regular_kernel_ms": statistics.mean(tx["regular_ms"]),
            "range_tables_and_zero_ms": statistics.mean(tx["range_table_ms"]),
            "regular_speedup_vs_direct": statistics.mean(td["regular_ms"]) / statistics.mean(tx["regular_ms"]),
            "note": "green_from_exp=1: regular-pair e^{-jkR} from the linear Exp table (one 16-byte record), "
                    "times 1/R; near pairs unchanged"},
        "table_speedup_vs_direct": {"step": direct_ms / ms_step,
                                    "regular_kernel": statistics.mean(td["regular_ms"]) / reg_ms,
                                    "near_kernel": statistics.mean(td["near_ms"]) / statistics.mean(tt["near_ms"])},
        "roofline": {"kernel": "k_fill_regular32<table>", "bound": "alu", "achieved": achieved,
                     "peak": peak_tops, "unit": "Tops/s (FP32 lane ops)", "frac": achieved / peak_tops,
                     "op_model": f"{OPS_PER_EVAL} FP32 lane operations per regular Green evaluation "
                                 "(distance 7, lookup and polynomial 10, moment accumulation 8); per-point "
                                 "Kahan updates and the per-pair 3x3 block not counted",
                     "peak_source": f"{SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_mhz:.0f} MHz "
                                    f"({src} max SM clock)",
                     "ops_per_launch": ops, "evals_per_launch": evals_regular, "traffic": traffic,
                     "traffic_note": TRAFFIC_NOTE,
                     "mufu_frac": evals_regular / (reg_ms / 1e3) / (SM_COUNT * MUFU_PER_SM * sm_mhz * 1e6),
                     "hbm_frac_z": zbytes / (reg_ms / 1e3) / (float(pk.get("hbm_gbs", 6800.0)) * 1e9),
                     "smem": smem_model(evals_regular, reg_ms, sm_mhz),
                     "issue": kernel_issue(wl.name)},
        "clocks": clocks,
        "e2e": e2e,
        "other_kernels": other_kernel_rooflines(wl.name, zbytes, statistics.mean(tt["mirror_ms"]),
                                                statistics.mean(tt["near_ms"]), n_near * m, pk, sm_mhz),
        # per step: range (init, [pass 0, pass 1, list, pass 2] or FP64 pass, out),
        # three table kernels, the pair kernel [and its corrections of the point
        # pairs in lattice cells holding samples, the mirror], the near kernel
        "gpu_launches": (13 if prec == gf.GF_FP32 else 8) * args.steps,
    }
    del zhost
    # ---- accuracy vs the FP64 oracle on 64 seeded 256 x 256 blocks (outside the timed region)
    run = None
    if rank == 0 and not args.skip_oracle:
        run = OracleRun(wl)
        lo, hi = mesh.range(wl.rule, prec)
        blocks, bs = sample_blocks(ne)
        tab = gf.Table(wl.k, lo, hi, p)
        gf.gf_fill(mesh.h, wl.k, p, tab.h, prec, Z)
        zt = gather_blocks(torch, Z, blocks, bs)
        gf.gf_fill(mesh.h, wl.k, px, tab.h, prec, Z)
        zx = gather_blocks(torch, Z, blocks, bs)
        gf.gf_fill(mesh.h, wl.k, p, None, prec, Z)
        zd = gather_blocks(torch, Z, blocks, bs)
        z64 = None
        if prec == gf.GF_FP32:
            gf.gf_fill(mesh.h, wl.k, p64, tab.h, prec, Z)
            z64 = gather_blocks(torch, Z, blocks, bs)
        ref_t = oracle_blocks(run, blocks, bs, "table")
        ref_d = oracle_blocks(run, blocks, bs, "direct")
        line["accuracy"] = {
            "blocks": f"{len(blocks)} seeded {bs} x {bs} blocks ({len(blocks) * bs * bs} entries)",
            "gpu_table_vs_oracle_table": err_stats(zt, ref_t),
            "gpu_direct_vs_oracle_direct": err_stats(zd, ref_d),
            "gpu_table_vs_oracle_direct": err_stats(zt, ref_d),
            "gpu_exp_over_r_vs_oracle_direct": err_stats(zx, ref_d),
            "tolerance_rel_fro": 1e-5}
        if z64 is not None:
            line["accuracy"]["gpu_table_near_fp64_vs_oracle_table"] = err_stats(z64, ref_t)
    if rank == 0 and not args.skip_cpu_baseline:
        line["cpu_baseline"] = oracle_baseline(wl, run=run)
    if rank == 0 and "sphere_radius" in wl.extra and not args.skip_oracle:
        line["rcs"] = sphere_rcs(gf, torch, mesh, wl, p, prec, stream, dev)
    if rank == 0:
        print(json.dumps(line), flush=True)


def sphere_rcs(gf, torch, mesh, wl, p, prec, stream, dev):
    """Plane-wave scattering by the sphere (outside the timed region): fill,
    excitation, dense solve, far field; bistatic sigma in the E- and H-planes
    against the Mie series, table fill against direct fill, and the times of
    the scattering kernels (CUDA events on the launching stream)."""
    from oracle import rcs
    a = wl.extra["sphere_radius"]
    th = np.linspace(0, math.pi, 181)
    dirs = {pl: torch.from_numpy(rcs.plane_directions(th, pl)).to(dev) for pl in "EH"}
    mie = dict(zip("EH", rcs.mie_bistatic(wl.k, a, th)))
    lo, hi = mesh.range(wl.rule, prec)
    tab = gf.Table(wl.k, lo, hi, p)
    zdt = torch.complex64 if prec == gf.GF_FP32 else torch.complex128
    out, sig = {}, {}
    torch.linalg.solve(torch.eye(8, dtype=zdt, device=dev), torch.ones(8, dtype=zdt, device=dev))  # loads the solver
    torch.cuda.synchronize()
    for name, table in (("table", tab), ("direct", None)):
        Z = gf.fill(mesh, wl.k, p, table, prec)
        V = torch.empty(mesh.ne, dtype=zdt, device=dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        gf.gf_excitation(mesh.h, wl.k, p, (0.0, 0.0, 1.0), (1.0, 0.0, 0.0), prec, V)
        ev[1].record(stream)
        I = torch.linalg.solve(Z, V)
        ev[2].record(stream)
        for pl in "EH":
            sig[(name, pl)] = gf.gf_far_field(mesh.h, wl.k, p, prec, I, dirs[pl])[1].cpu().numpy()
        ev[3].record(stream)
        torch.cuda.synchronize()
        del Z
        if name == "table":
            out["excitation_ms"] = ev[0].elapsed_time(ev[1])
            out["solve_ms (torch.linalg.solve, LU)"] = ev[1].elapsed_time(ev[2])
            out["far_field_ms"] = ev[2].elapsed_time(ev[3])
    # MFIE (K operator) on the same closed surface: fill time, and its solution's sigma
    for name, table in (("mfie_table", tab), ("mfie_direct", None)):
        Z = torch.empty((mesh.ne, mesh.ne), dtype=zdt, device=dev)
        for _ in range(2):
            gf.gf_fill_mfie(mesh.h, wl.k, p, table.h if table else None, prec, Z)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        reps = 5
        ev[0].record(stream)
        for _ in range(reps):
            gf.gf_fill_mfie(mesh.h, wl.k, p, table.h if table else None, prec, Z)
        ev[1].record(stream)
        torch.cuda.synchronize()
        out[f"{name}_fill_ms"] = ev[0].elapsed_time(ev[1]) / reps
        V = torch.empty(mesh.ne, dtype=zdt, device=dev)
        gf.gf_excitation(mesh.h, wl.k, p, (0.0, 0.0, 1.0), (1.0, 0.0, 0.0), prec, V, op=gf.GF_OP_MFIE)
        I = torch.linalg.solve(Z, V)
        del Z
        for pl in "EH":
            sig[(name, pl)] = gf.gf_far_field(mesh.h, wl.k, p, prec, I, dirs[pl])[1].cpu().numpy()
    rl = lambda x, y: float(np.linalg.norm(x - y) / np.linalg.norm(y))  # noqa: E731
    for pl in "EH":
        out[f"mfie_table_vs_mie_rel_l2_{pl}"] = rl(sig[("mfie_table", pl)], mie[pl])
        out[f"mfie_vs_efie_rel_l2_{pl}"] = rl(sig[("mfie_table", pl)], sig[("table", pl)])
        out[f"mfie_table_vs_direct_rel_l2_{pl}"] = rl(sig[("mfie_table", pl)], sig[("mfie_direct", pl)])
    out["mfie_z_entries_per_s"] = mesh.ne * mesh.ne / (out["mfie_table_fill_ms"] / 1e3)
    for pl in "EH":
        out[f"table_vs_mie_rel_l2_{pl}"] = rl(sig[("table", pl)], mie[pl])
        out[f"direct_vs_mie_rel_l2_{pl}"] = rl(sig[("direct", pl)], mie[pl])
        out[f"table_vs_direct_rel_l2_{pl}"] = rl(sig[("table", pl)], sig[("direct", pl)])
    out["backscatter_over_pi_a2"] = {"table": float(sig[("table", "E")][-1] / (math.pi * a * a)),
                                     "mie": float(mie["E"][-1] / (math.pi * a * a))}
    out["angles"] = "181 per plane, theta 0..180 deg; x-polarised plane wave along +z"
    return out


def run_batch(args, rank, world, local_rank):
    """64 perturbed ellipsoids, each with its own k and tables, one CUDA-graph
    launch (persistent kernels) per step."""
    import torch

    import paper_1901_04162_gb300 as gf

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wls = W.ellipsoid_batch(args.batch_count)
    rule = wls[0].rule
    p = gf.gf_params_default(rule=rule)
    t0 = time.perf_counter()
    meshes = [gf.Mesh(wl.xyz, wl.tri) for wl in wls]
    t_mesh = time.perf_counter() - t0
    t0 = time.perf_counter()
    tables = []
    for wl, m in zip(wls, meshes):
        lo, hi = m.range(rule, gf.GF_FP32)
        tables.append(gf.Table(wl.k, lo, hi, p))
    torch.cuda.synchronize()
    t_tables = time.perf_counter() - t0
    Zs = [torch.empty((m.ne, m.ne), dtype=torch.complex64, device=dev) for m in meshes]
    t0 = time.perf_counter()
    batch = gf.Batch(meshes, [wl.k for wl in wls], p, tables, Zs, autotune=not args.no_autotune)
    t_create = time.perf_counter() - t0
    direct = gf.Batch(meshes, [wl.k for wl in wls], p, None, Zs, autotune=not args.no_autotune)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def timed(b):
        for _ in range(args.warmup):
            b.launch()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            evs[i][0].record(stream)
            b.launch()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(c) for a, c in evs)

    with Clocks(local_rank) as clk:
        total_ms = timed(batch)
    clocks = clk.summary()
    direct_ms = timed(direct)
    # variant: one table in u = kR for all 64 meshes (built once over the union of their k R ranges)
    t0 = time.perf_counter()
    rngs = [m.range(rule, gf.GF_FP32) for m in meshes]
    umin = min(wl.k * lo for wl, (lo, _) in zip(wls, rngs)) * (1 - 1e-6)
    umax = max(wl.k * hi for wl, (_, hi) in zip(wls, rngs)) * (1 + 1e-6)
    tkr = gf.Table.kr(umin, umax, p)
    torch.cuda.synchronize()
    t_kr = time.perf_counter() - t0
    kr_batch = gf.Batch(meshes, [wl.k for wl in wls], p, [tkr] * len(meshes), Zs, autotune=not args.no_autotune)
    kr_ms = timed(kr_batch)
    entries = sum(m.ne * m.ne for m in meshes)
    n_regular = sum(evaluated_pairs(m.nt, m.n_near) for m in meshes)
    n_near = sum(m.n_near for m in meshes)
    evals = n_regular * rule * rule + n_near * rule * (3 * (p.nphi + p.nl) + 1)
    ms = total_ms / args.steps
    pk, src = peaks()
    sm_mhz = float(pk.get("sm_max_mhz", FALLBACK_SM_MHZ))
    peak_tops = SM_COUNT * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12
    achieved = n_regular * rule * rule * OPS_PER_EVAL / (ms / 1e3) / 1e12
    line = {
        "metric": "Z entries/s (table fill)", "value": entries / (ms / 1e3), "unit": "Z entries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{len(wls)} perturbed ellipsoids, {sum(m.nt for m in meshes)} triangles, "
                               f"{rule}-point rule, k in [pi, 4pi], one table per mesh",
                   "meshes": len(wls), "rwg_unknowns_total": sum(m.ne for m in meshes),
                   "z_bytes": entries * 8, "l2": "flushed between steps (256 MiB write)",
                   "launch": "one CUDA graph (zero Z, persistent regular kernel, one Z += Z^T pass over every mesh, "
                             "persistent near kernel)",
                   "autotuned": batch.config(), "parallelism": f"replicas x{world}"},
        "green_evals_per_s": evals / (ms / 1e3),
        "setup_s": {"meshes": t_mesh, "ranges_and_tables": t_tables, "batch_create_and_autotune": t_create},
        "direct": {"value": entries / (direct_ms / args.steps / 1e3), "ms_per_step": direct_ms / args.steps,
                   "autotuned": direct.config()},
        "kr_table_variant": {"ms_per_step": kr_ms / args.steps, "value": entries / (kr_ms / args.steps / 1e3),
                             "u_range": [umin, umax], "green_samples": tkr.info(gf.GF_GREEN)[0],
                             "ranges_and_one_table_s": t_kr,
                             "note": "one table in u = kR shared by all meshes (gf_table_create_kr)"},
        "roofline": {"kernel": "batched graph (regular + mirrors + near)", "bound": "alu", "achieved": achieved,
                     "peak": peak_tops, "unit": "Tops/s (FP32 lane ops, regular pairs only, whole graph time)",
                     "frac": achieved / peak_tops, "traffic": None,
                     "op_model": f"{OPS_PER_EVAL} FP32 lane operations per regular Green evaluation, as for "
                                 "the single fill"},
        "clocks": clocks,
        "e2e": {"value": None, "reason": "batched workload: fill-only; see setup_s"},
        # per graph launch: the regular kernel, the mirror pass over every Z, the near kernel
        "gpu_launches": 3 * args.steps,
    }
    if not args.skip_oracle:
        import oracle as O
        errs = []
        for i in (0, len(wls) // 2, len(wls) - 1):
            wl = wls[i]
            om = O.Mesh(wl.xyz, wl.tri)
            lo, hi = om.range(rule)
            rows = np.random.default_rng(i).choice(om.ne, 4, replace=False)
            ref = om.z_rows(wl.k, rule, rows, mode="table", tables=O.make_tables(wl.k, lo, hi))
            batch.launch()
            z = Zs[i][torch.from_numpy(rows).to(dev)].cpu().numpy()
            errs.append(float(np.linalg.norm(z - ref) / np.linalg.norm(ref)))
        line["accuracy"] = {"meshes_sampled": 3, "rows_each": 4, "max_rel_fro_vs_oracle_table": max(errs),
                            "tolerance": 1e-5}
    print(json.dumps(line), flush=True)


def run_adjoint(args, rank, world, local_rank):
    """Backward of L = Re(a^H Z b) on the 2048-triangle sphere (6-point rule):
    dL/d(vertex coordinates) and dL/dk from gZ = a conj(b)^T."""
    import torch

    import paper_1901_04162_gb300 as gf

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl = W.sphere_3072()
    rule = wl.rule
    p = gf.gf_params_default(rule=rule)
    m = gf.Mesh(wl.xyz, wl.tri)
    lo, hi = m.range(rule, gf.GF_FP32)
    tab = gf.Table(wl.k, lo, hi, p)
    a = W.complex_gaussian(m.ne, 7)
    b = W.complex_gaussian(m.ne, 8)
    gZ = torch.from_numpy(np.outer(a, np.conj(b)).astype(np.complex64)).to(dev)
    Z = torch.empty((m.ne, m.ne), dtype=torch.complex64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            evs[i][0].record(stream)
            fn()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(x.elapsed_time(y) for x, y in evs) / args.steps

    with Clocks(local_rank) as clk:
        bwd_ms = timed(lambda: gf.gf_fill_backward(m, wl.k, p, tab, gZ))
    fwd_ms = timed(lambda: gf.gf_fill(m.h, wl.k, p, tab.h, gf.GF_FP32, Z))
    bwd_direct_ms = timed(lambda: gf.gf_fill_backward(m, wl.k, p, None, gZ))
    n_regular = m.nt * m.nt - m.n_near
    line = {
        "metric": "Z entries/s (adjoint fill)", "value": m.ne * m.ne / (bwd_ms / 1e3), "unit": "Z entries/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": bwd_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "triangles": m.nt, "rwg_unknowns": m.ne, "rule_points": rule,
                   "loss": "Re(a^H Z b), a, b seeded complex Gaussian", "regular_pairs": n_regular,
                   "regular_pairs_evaluated": evaluated_pairs(m.nt, m.n_near), "near_pairs": m.n_near, "parallelism": f"replicas x{world}"},
        "gradient_evals_per_s": 1.0 / (bwd_ms / 1e3),
        "forward_fill_ms": fwd_ms, "backward_over_forward": bwd_ms / fwd_ms,
        "direct_backward_ms": bwd_direct_ms,
        "clocks": clk.summary(),
        "e2e": {"value": None, "reason": "adjoint workload: device-resident gZ"},
        "gpu_launches": 3 * args.steps,
    }
    if not args.skip_oracle:
        import oracle as O
        dxyz, dk = gf.gf_fill_backward(m, wl.k, p, tab, gZ)
        g = dxyz.cpu().numpy()
        om = O.Mesh(wl.xyz, wl.tri)
        verts = [0, 517, 1000]
        mask = np.isin(np.arange(len(wl.tri)), np.where(np.isin(wl.tri, verts).any(axis=1))[0]).astype(np.int32)
        _, g_ref, _ = om.loss_grad(wl.k, rule, a, b, tri_mask=mask)
        _, dk_ref = om.loss_dk(wl.k, rule, a, b)
        line["accuracy"] = {
            "sampled_vertices": verts,
            "max_abs_err_over_max_abs_ref": float(np.abs(g[verts] - g_ref[verts]).max() / np.abs(g_ref[verts]).max()),
            "dk_rel_err": abs(float(dk.cpu()[0]) - dk_ref) / abs(dk_ref), "reference": "oracle FP64 direct, dual numbers",
            "tolerance": 1e-4}
    print(json.dumps(line), flush=True)


def run_near_field(args, rank, world, local_rank):
    """Near-field sparse fill (Z on the RWG pairs within 0.3 lambda) of the
    3 lambda cube (49152 triangles, 4-point rule): the fast-solver regime."""
    import torch

    import paper_1901_04162_gb300 as gf
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    wl = W.cube_73728()
    radius = 0.3
    m = gf.Mesh(wl.xyz, wl.tri, wl.near_dist)
    p = gf.gf_params_default(rule=wl.rule)
    lo, hi = m.range(wl.rule, gf.GF_FP32)
    tab = gf.Table(wl.k, lo, hi, p)
    t0 = time.perf_counter()
    sp = gf.Sparse(m, radius)
    setup_s = time.perf_counter() - t0
    vals = torch.empty(sp.nnz, dtype=torch.complex64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(table):
        for _ in range(args.warmup):
            sp.fill(wl.k, p, table, vals)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            evs[i][0].record(stream)
            sp.fill(wl.k, p, table, vals)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(x.elapsed_time(y) for x, y in evs) / args.steps

    with Clocks(local_rank) as clk:
        ms = timed(tab)
    ms_direct = timed(None)
    line = {
        "metric": "near-field Z entries/s (sparse table fill)", "value": world * sp.nnz / (ms / 1e3),
        "unit": "Z entries/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name + "_near_field_0.3lambda", "triangles": m.nt, "rwg_unknowns": m.ne,
                   "rule_points": wl.rule, "radius_lambda": radius, "nnz": sp.nnz, "nnz_per_row": sp.nnz / m.ne,
                   "regular_triangle_pairs": sp.n_pairs, "near_pairs": m.n_near,
                   "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas x{world}"},
        "direct": {"ms_per_step": ms_direct, "value": world * sp.nnz / (ms_direct / 1e3)},
        "pattern_setup_s (host, once per mesh and radius)": setup_s,
        "clocks": clk.summary(),
        "e2e": {"value": None, "reason": "near-field workload: device-resident mesh and pattern"},
        "gpu_launches": 2 * args.steps,
    }
    if not args.skip_oracle:
        import oracle as O
        row_ptr, cols = sp.pattern()
        rows = np.repeat(np.arange(m.ne), np.diff(row_ptr))
        pick = np.random.default_rng(8).choice(sp.nnz, 200, replace=False)
        sp.fill(wl.k, p, tab, vals)
        v = vals.cpu().numpy()[pick]
        om = O.Mesh(wl.xyz, wl.tri, wl.near_dist)
        olo, ohi = om.range(wl.rule, prune=True)
        zo = om.z_entries(wl.k, wl.rule, rows[pick], cols[pick], mode="table", tables=O.make_tables(wl.k, olo, ohi))
        line["accuracy"] = {"entries_sampled": 200, "rel_l2_vs_oracle_table": float(np.linalg.norm(v - zo) /
                                                                                   np.linalg.norm(zo)),
                            "tolerance": 1e-5}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_mfie(args, rank, world, local_rank):
    """MFIE (K operator) fill of the 1 lambda sphere (5120 triangles, 7680 RWG,
    7-point rule): identity term, every ordered regular pair, near pairs with
    the singular scheme; table and direct Green function."""
    import torch

    import paper_1901_04162_gb300 as gf
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    wl = W.sphere_7680()
    m = gf.Mesh(wl.xyz, wl.tri, wl.near_dist)
    p = gf.gf_params_default(rule=wl.rule)
    lo, hi = m.range(wl.rule, gf.GF_FP32)
    tab = gf.Table(wl.k, lo, hi, p)
    Z = torch.empty((m.ne, m.ne), dtype=torch.complex64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(table):
        h = table.h if table else None
        for _ in range(args.warmup):
            gf.gf_fill_mfie(m.h, wl.k, p, h, gf.GF_FP32, Z)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            evs[i][0].record(stream)
            gf.gf_fill_mfie(m.h, wl.k, p, h, gf.GF_FP32, Z)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(x.elapsed_time(y) for x, y in evs) / args.steps

    with Clocks(local_rank) as clk:
        ms = timed(tab)
    zt = Z.clone()
    ms_direct = timed(None)
    entries = m.ne * m.ne
    line = {
        "metric": "MFIE Z entries/s (table fill)", "value": world * entries / (ms / 1e3),
        "unit": "Z entries/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name + "_mfie", "triangles": m.nt, "rwg_unknowns": m.ne, "rule_points": wl.rule,
                   "near_pairs": m.n_near, "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"replicas x{world}"},
        "direct": {"ms_per_step": ms_direct, "value": world * entries / (ms_direct / 1e3)},
        "table_vs_direct_rel_l2": float(torch.linalg.vector_norm(zt - Z) / torch.linalg.vector_norm(Z)),
        "clocks": clk.summary(),
        "e2e": {"value": None, "reason": "MFIE workload: device-resident mesh and Z"},
        # identity, regular, near
        "gpu_launches": 3 * args.steps,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cube_73728",
                    choices=sorted(WORKLOADS) + ["ellipsoid_batch", "adjoint_3072", "cube_near_field",
                                                   "sphere_mfie"])
    ap.add_argument("--skip-oracle", action="store_true")
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=8.0)
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--no-autotune", action="store_true", help="batched workload: the default launch shape")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload == "adjoint_3072":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "reference arm runs the single-mesh workloads"}))
            return
        run_adjoint(args, rank, world, local_rank)
        return
    if args.workload == "sphere_mfie":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "reference arm runs the single-mesh workloads"}))
            return
        run_mfie(args, rank, world, local_rank)
        return
    if args.workload == "cube_near_field":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "reference arm runs the single-mesh workloads"}))
            return
        run_near_field(args, rank, world, local_rank)
        return
    if args.workload == "ellipsoid_batch":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "reference arm runs the single-mesh workloads"}))
            return
        run_batch(args, rank, world, local_rank)
        return
    wl = WORKLOADS[args.workload]()
    if args.impl == "reference":
        run_reference(args, wl, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_ours(args, wl, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Benchmark: maximal all-ones square detection on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Prints ONE JSON line (rank 0).  A step is one pass of the hot path over the
workload's matrices: the tile pass, the exact fix-up when needed and the
result write-out, for every matrix.  Inputs are generated in HBM by the
seeded generator before timing; `value` is cells/s over K device-timed steps
(max over ranks); `e2e` repeats the measurement with the inputs in pinned
host memory and the host->device copies and the result read-back inside the
timed region.  `--impl reference` times the CPU oracle (the paper's
Algorithm 1, single thread) on the same workload instead.

Workloads (sizes from the configurations this benchmark mirrors):
  sweep    (default) square uint8 matrices, sides 1000..5000 x densities
           0.1..0.9 (45 matrices, 495 M cells), one call per matrix; side+witness
  c1       256 x 256, p = 0.5, seed 0, side + witness + int32 dp map
  c3-u8 / c3-u8-dp / c3-bits / c3-bits-dp
           32768 x 32768, p = 0.9, one planted 600-square, seed 3
  c3q-*    the same with 8192 rows (for profiler captures)
  c5       serving stream (see run_serve)
  c4       4096 uint8 matrices, m and n log-uniform in [16, 2048]: one autotuned
           ms_batch per step replayed from a CUDA graph (plain calls reported beside)
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcells/s on 1 GB300 (% HBM roofline), batched vs plain; serve p50/p99 ms"


# ----------------------------------------------------------------- workloads --

def sweep_specs():
    specs = []
    for side in (1000, 2000, 3000, 4000, 5000):
        for k in range(1, 10):
            p = k / 10
            specs.append(dict(m=side, n=side, p=p, seed=10 * (side // 1000) + k, plant=0))
    return specs


def c3_spec():
    return dict(m=32768, n=32768, p=0.9, seed=3, plant=600)


def c4_specs(count=4096):
    import gen
    specs = []
    lo, hi = math.log(16), math.log(2049)
    for k in range(count):
        seed = gen.draw(4, k)
        u = lambda j: (gen.draw(seed, (1 << 40) + j) >> 11) / float(1 << 53)
        m = min(2048, int(math.exp(lo + (hi - lo) * u(0))))
        n = min(2048, int(math.exp(lo + (hi - lo) * u(1))))
        p = (1 + int(9 * u(2))) / 10
        plant = 0
        if u(3) < 0.5:
            plant = 1 + int(min(m, n) * u(4))
        specs.append(dict(m=m, n=n, p=p, seed=seed, plant=plant))
    return specs


def round_up(x, a):
    return (x + a - 1) // a * a


class Mat:
    """One generated matrix resident in HBM (and optionally in pinned host memory)."""

    def __init__(self, spec, fmt, device, want_host=False):
        import torch

        import gen
        self.spec = spec
        self.fmt = fmt
        m, n = spec["m"], spec["n"]
        self.m, self.n = m, n
        if fmt == 0:
            self.ld = round_up(n, 16)
            self.dev = torch.empty((m, self.ld), dtype=torch.uint8, device=device)
            gen.fill_u8_dev(self.dev.data_ptr(), m, n, self.ld, spec["p"], spec["seed"])
            if spec["plant"]:
                r, c = gen.plant_pos(spec["seed"], m, n, spec["plant"])
                gen.plant_u8_dev(self.dev.data_ptr(), self.ld, r, c, spec["plant"])
        else:
            self.ld = round_up((n + 31) // 32, 4)
            self.dev = torch.empty((m, self.ld), dtype=torch.int32, device=device)
            gen.fill_bits_dev(self.dev.data_ptr(), m, n, self.ld, spec["p"], spec["seed"])
            if spec["plant"]:
                r, c = gen.plant_pos(spec["seed"], m, n, spec["plant"])
                gen.plant_bits_dev(self.dev.data_ptr(), self.ld, r, c, spec["plant"])
        self.host = None
        if want_host:
            torch.cuda.synchronize()
            self.host = torch.empty(self.dev.shape, dtype=self.dev.dtype, pin_memory=True)
            self.host.copy_(self.dev)
        self.view = self.dev[:, :n] if fmt == 0 else self.dev

    @property
    def nbytes(self):
        return self.dev.numel() * self.dev.element_size()

    def args(self, tensor=None):
        t = self.dev if tensor is None else tensor
        return (t[:, :self.n], None, 0) if self.fmt == 0 else (t, self.n, 1)


class Workload:
    name = ""
    dtype = "u8"
    bytes_per_cell = 1.0  # algorithmic bytes of the dominant kernel

    def __init__(self, device):
        self.device = device

    def config(self):
        raise NotImplementedError


class PlainSet(Workload):
    """A list of matrices, one plain ms_max_square / ms_dp_map call each."""

    def __init__(self, device, specs, fmt=0, dpmap=False, label="", host=False):
        super().__init__(device)
        import torch
        self.specs = specs
        self.fmt = fmt
        self.dpmap = dpmap
        self.label = label
        self.mats = [Mat(s, fmt, device, want_host=host) for s in specs]
        self.cells = sum(s["m"] * s["n"] for s in specs)
        self.res = torch.empty((len(specs), 4), dtype=torch.int32, device=device)
        self.dps = None
        if dpmap:
            self.dps = [torch.empty((s["m"], s["n"]), dtype=torch.int32, device=device)
                        for s in specs]
        self.dtype = "u8" if fmt == 0 else "bits32"
        self.bytes_per_cell = (1.0 if fmt == 0 else 0.125) + (4.0 if dpmap else 0.0)
        self.dev_bufs = None

    def prepare(self, ms, ctx, tensors=None):
        """ctypes descriptors for every matrix (the C ABI is called directly)."""
        import ctypes
        descs = []
        for i, mt in enumerate(self.mats):
            x, n, fmt = mt.args(None if tensors is None else tensors[i])
            descs.append(ms.describe(x, n, fmt))
        arr = (ms._Matrix * len(descs))(*descs)
        base = ctypes.addressof(arr)
        ptrs = [ctypes.cast(base + i * ctypes.sizeof(ms._Matrix), ctypes.POINTER(ms._Matrix))
                for i in range(len(descs))]
        res = [self.res[i].data_ptr() for i in range(len(descs))]
        dps = [(d.data_ptr(), d.stride(0)) for d in self.dps] if self.dpmap else None
        return arr, ptrs, res, dps

    def step(self, ms, ctx, prep, stream_ptr):
        """One plain call per matrix."""
        for i in range(len(prep[1])):
            self.step_one(ms, ctx, prep, i, stream_ptr)

    def step_one(self, ms, ctx, prep, i, stream_ptr):
        """The plain call of matrix i."""
        arr, ptrs, res, dps = prep
        L, h = ms.lib(), ctx._h
        if self.dpmap:
            rc = L.ms_dp_map(h, ptrs[i], dps[i][0], dps[i][1], res[i], stream_ptr)
            if rc:
                raise ms.MSError(rc, "ms_dp_map")
        else:
            rc = L.ms_max_square(h, ptrs[i], res[i], stream_ptr)
            if rc:
                raise ms.MSError(rc, "ms_max_square")

    def batch_step(self, ms, ctx, prep, stream_ptr):
        """One ms_batch call over all matrices."""
        arr = prep[0]
        rc = ms.lib().ms_batch(ctx._h, arr, len(self.mats), self.res.data_ptr(), stream_ptr)
        if rc:
            raise ms.MSError(rc, "ms_batch")

    def h2d_bytes(self):
        return sum(mt.nbytes for mt in self.mats)

    def config(self):
        return {"workload": self.label, "matrices": len(self.specs), "cells": self.cells,
                "format": self.dtype, "dp_map": self.dpmap,
                "row_stride": "columns rounded up to 16 bytes" if self.fmt == 0 else
                              "words rounded up to 4",
                "l2": ("inputs larger than L2 (129 MB)" if self.cells * self.bytes_per_cell
                       > 129e6 else "L2 flushed between steps")}


def make_workload(name, device, host=False):
    if name == "sweep":
        return PlainSet(device, sweep_specs(), label="paper-scale sweep: square uint8, sides "
                        "1000..5000 x p 0.1..0.9, seed 10*side/1000+10p, side + witness, "
                        "one call per matrix", host=host)
    if name == "c1":
        return PlainSet(device, [dict(m=256, n=256, p=0.5, seed=0, plant=0)], dpmap=True,
                        label="256x256 uint8, p=0.5, seed 0, side + witness + int32 dp map",
                        host=host)
    if name.startswith("c3"):
        fmt = 1 if "bits" in name else 0
        dp = name.endswith("-dp")
        spec = c3_spec()
        if name.startswith("c3q"):  # a quarter of it (8192 rows) for profiler captures
            spec = dict(spec, m=8192)
        return PlainSet(device, [spec], fmt=fmt, dpmap=dp,
                        label=f"{spec['m']}x32768 {'bit-packed' if fmt else 'uint8'}, p=0.9, "
                              f"planted 600-square, seed 3, "
                              f"{'dp map' if dp else 'side + witness'}", host=host)
    if name == "c4":
        return PlainSet(device, c4_specs(), label="batch of 4096 uint8 matrices, m,n "
                        "log-uniform in [16,2048], p in 0.1..0.9, half planted", host=host)
    raise SystemExit(f"unknown workload {name}")


# ------------------------------------------------------------------- helpers --

class ClockSampler:
    """nvidia-smi clock / throttle samples (200 ms) around the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def mark(self, t0, t1):
        self.t0, self.t1 = t0, t1

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=2)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        lo, hi = (self.t0 or 0) - 0.25, (self.t1 or 1e30) + 0.25
        rows = [s for (t, s) in self.samples if lo <= t <= hi] or [s for (_, s) in self.samples]
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            f = [x.strip() for x in r.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                pass
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        mhz.sort()
        return {"sm_mhz": mhz[len(mhz) // 2] if mhz else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(rows),
                "window": "timed region +-0.25 s, 200 ms sampling"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def profile_traffic(kernel_key):
    """Per-cell DRAM traffic of a kernel from its committed ncu summary, if the
    kernel sources are unchanged since the capture (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "ncu_summary.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"sources_sha1:\s*([0-9a-f]{40})", text)
    h = hashlib.sha1()
    for f in ("ms.cu", "ms_kernels.cuh", "ms_device.cuh", "ms_bits.cuh", "ms_bitile.cuh"):
        p = os.path.join(ROOT, "paper_2503_18974_gb300", "csrc", f)
        if os.path.exists(p):
            h.update(open(p, "rb").read())
    if not m or m.group(1) != h.hexdigest():
        return None
    m2 = re.search(rf"traffic_bytes_per_cell\[{re.escape(kernel_key)}\]:\s*([0-9.]+)", text)
    return float(m2.group(1)) if m2 else None


def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x, device):
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------ CPU (oracle) ----

def cpu_oracle_run(specs, budget_s=20.0, reps=5):
    """The paper's Algorithm 1 (oracle.freq, one thread) on the workload's
    matrices regenerated on the host; the paper's protocol scaled down: one
    warm-up, then repetitions until the budget, 10% trimmed mean."""
    import numpy as np

    import gen
    import oracle
    oracle.build()
    mats = []
    tot = 0
    for s in specs:
        a = gen.bernoulli_u8(s["m"], s["n"], s["p"], s["seed"])
        if s["plant"]:
            r, c = gen.plant_pos(s["seed"], s["m"], s["n"], s["plant"])
            a[r:r + s["plant"], c:c + s["plant"]] = 1
        mats.append(a)
        tot += s["m"] * s["n"]
    for a in mats:
        oracle.freq(a)
    times = []
    t_start = time.perf_counter()
    while len(times) < reps and (time.perf_counter() - t_start) < budget_s:
        t0 = time.perf_counter()
        for a in mats:
            oracle.freq(a)
        times.append(time.perf_counter() - t0)
    times.sort()
    trim = int(len(times) * 0.1)
    kept = times[trim:len(times) - trim] if len(times) > 2 * trim else times
    sec = sum(kept) / len(kept)
    t0 = time.perf_counter()
    oracle.dp_rows(mats[len(mats) // 2])
    dp_rate = mats[len(mats) // 2].size / (time.perf_counter() - t0)
    return tot, sec, len(times), dp_rate


def cpu_sample_specs(specs, max_cells=600_000_000):
    out, tot = [], 0
    for s in specs:
        c = s["m"] * s["n"]
        if tot + c > max_cells and out:
            continue
        out.append(s)
        tot += c
    return out


def cpu_baseline(specs):
    sample = cpu_sample_specs(specs)
    cells, sec, reps, dp_rate = cpu_oracle_run(sample)
    return {"value": cells / sec / 1e9, "unit": "Gcells/s", "cores": 1, "kind": "oracle",
            "sample": f"{len(sample)} of {len(specs)} matrices ({cells / 1e6:.0f} M cells), "
                      f"Algorithm 1 (oracle_freq), 1 warm-up + {reps} timed passes, "
                      f"10% trimmed mean",
            "oracle_dp_rows_gcells_s": dp_rate / 1e9}


# ------------------------------------------------------------------- arms -----

def run_reference(args, world, rank, local, pg):
    if rank != 0:
        return
    specs = {"sweep": sweep_specs, "c1": lambda: [dict(m=256, n=256, p=0.5, seed=0, plant=0)],
             "c4": c4_specs}.get(args.workload, lambda: [c3_spec()])()
    sample = cpu_sample_specs(specs, max_cells=120_000_000)
    import gen
    import oracle
    oracle.build()
    mats = []
    for s in sample:
        a = gen.bernoulli_u8(s["m"], s["n"], s["p"], s["seed"])
        if s["plant"]:
            r, c = gen.plant_pos(s["seed"], s["m"], s["n"], s["plant"])
            a[r:r + s["plant"], c:c + s["plant"]] = 1
        mats.append(a)
    cells = sum(a.size for a in mats)
    for _ in range(args.warmup):
        for a in mats:
            oracle.freq(a)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for a in mats:
            oracle.freq(a)
    dt = time.perf_counter() - t0
    value = cells * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gcells/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": args.workload, "sample_matrices": len(mats),
                       "sample_cells": cells},
            "cpu_baseline": {"value": value, "unit": "Gcells/s", "cores": 1, "kind": "oracle",
                             "sample": f"each step: {len(mats)} of {len(specs)} matrices "
                                       f"({cells / 1e6:.0f} M cells) through Algorithm 1"},
            "e2e": {"value": value, "unit": "Gcells/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed(fn, steps, stream):
    import torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        fn()
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1)


def run_ours(args, world, rank, local, pg):
    import torch

    import paper_2503_18974_gb300 as ms
    device = torch.device(f"cuda:{local}")
    torch.cuda.set_device(device)
    ms.build()
    ctx = ms.MaxSquare(local)
    # packed size-only work: the autotuner below chooses between the tile
    # kernel and the bitplane search unless --packed-path fixes it
    packed_path = args.packed_path if args.packed_path is not None else 0
    ctx.set_tuning(packed_path=packed_path, band_rows=args.band_rows, lane_cols=args.lane_cols,
                   tile_kind=args.tile_kind)
    wl = make_workload(args.workload, device, host=True)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream or None
    prep = wl.prepare(ms, ctx)
    batch_headline = args.workload == "c4"
    multi = len(wl.mats) > 1 and not wl.dpmap

    # the plain form: one autotune per workload class (format, log2 cells) on
    # a representative matrix, cached in the context for the plain calls
    plain_tuned = {}
    if (not wl.dpmap and not args.band_rows and not args.lane_cols and not args.tile_kind
            and args.packed_path is None):
        classes = {}
        for mt in wl.mats:
            classes.setdefault((mt.fmt, int(math.log2(max(mt.m * mt.n, 1)))), []).append(mt)
        for key, group in sorted(classes.items()):
            rep = sorted(group, key=lambda mt: mt.m * mt.n)[len(group) // 2]
            plain_tuned[f"fmt{key[0]}_2^{key[1]}"] = ctx.autotune(
                [rep.args()[:2] if rep.fmt else rep.args()[0]])

    # the batched form: autotuned, then captured in a CUDA graph
    graph = None
    tuned = None
    if multi:
        tuned = ctx.autotune([mt.args()[:2] if mt.fmt else mt.args()[0] for mt in wl.mats])
        wl.batch_step(ms, ctx, prep, sp)  # uploads the job table outside the capture
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            with torch.cuda.graph(graph, stream=side):
                wl.batch_step(ms, ctx, prep, side.cuda_stream)
        torch.cuda.synchronize()

    def plain():
        wl.step(ms, ctx, prep, sp)

    def batched():
        graph.replay()

    headline = batched if batch_headline else plain

    for _ in range(args.warmup):
        headline()
    torch.cuda.synchronize()

    # timed region: K steps, device-timed, clocks sampled
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.4)
    barrier(pg)
    t_wall0 = time.time()
    torch.cuda.nvtx.range_push("timed_steps")  # lets a profiler select the timed launches
    ms_total = timed(headline, args.steps, stream)
    torch.cuda.nvtx.range_pop()
    t_wall1 = time.time()
    barrier(pg)
    sampler.mark(t_wall0, t_wall1)
    clocks = sampler.stop()
    ms_total = max_over_ranks(pg, ms_total, device)
    ms_step = ms_total / args.steps
    value = world * wl.cells * args.steps / (ms_total * 1e-3) / 1e9

    # dominant kernel: the same K steps again with a CUDA event pair recorded
    # by the library around every launch on this stream
    ctx.profile_start()
    for _ in range(args.steps):
        if batch_headline:
            wl.batch_step(ms, ctx, prep, sp)
        else:
            plain()
    prof = ctx.profile_stop()
    peak, peak_kind = measured_peaks()
    roof = None
    if prof.other_ms > prof.tile_ms:
        kern_ms, kern_launches, kern_name = prof.other_ms, prof.other_launches, \
            "k_bits_search (bitplane doubling + binary search)"
    else:
        kern_ms, kern_launches, kern_name = prof.tile_ms, prof.tile_launches, \
            ("k_batch_tiles (persistent tile queue)" if batch_headline
             else "k_bitiles_one (bitplane tile pass)"
             if prof.bit_tile_launches == prof.tile_launches
             else "k_tiles_one (dp-recurrence tile pass)"
             if prof.bit_tile_launches == 0 else "k_tiles_one + k_bitiles_one (tile passes)")
    if kern_launches and kern_ms > 0:
        alg_bytes = wl.cells * wl.bytes_per_cell * args.steps
        achieved = alg_bytes / (kern_ms * 1e-3) / 1e9
        traffic = profile_traffic(args.workload)
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "peak_source": ("of measured (MEASURED_PEAKS.json hbm_gbs)"
                                if peak_kind == "measured" else "of fallback 6800 GB/s"),
                "traffic": (traffic * wl.cells if traffic is not None else None),
                "kernel": kern_name, "bytes_per_cell": wl.bytes_per_cell,
                "launches_per_step": kern_launches / args.steps,
                "kernel_ms_per_step": kern_ms / args.steps,
                "tile_ms_per_step": prof.tile_ms / args.steps,
                "fixup_ms_per_step": prof.fixup_ms / args.steps,
                "search_ms_per_step": prof.other_ms / args.steps,
                "how": "per-launch CUDA events on the launching stream, same K steps re-run"}
    launches_per_step = (prof.tile_launches + prof.fixup_launches + prof.other_launches) \
        / args.steps
    if batch_headline:
        launches_per_step += 0  # the graph replays the same launches (queue reset is a memset)
    launches = int(round(launches_per_step * args.steps))

    # batched vs plain, same matrices
    compare = None
    if multi:
        other = plain if batch_headline else batched
        for _ in range(2):
            other()
        oms = timed(other, args.steps, stream) / args.steps
        compare = {"plain" if batch_headline else "batched_graph": {
            "value": wl.cells / (oms * 1e-3) / 1e9, "unit": "Gcells/s", "ms_per_step": oms,
            "how": ("one ms_max_square call per matrix, eager launches" if batch_headline else
                    "one ms_batch per step (autotuned, persistent tile queue), graph replay")},
            "autotuned": tuned}
    if plain_tuned:
        compare = dict(compare or {}, plain_autotuned=plain_tuned)

    # e2e: pinned host inputs copied to fixed device buffers, the public call
    # (ms_max_square per matrix, or ms_batch), results read back, per step.
    # Plain calls: the copies run on a copy stream and each matrix's call
    # waits for its own copy only, so copies overlap earlier matrices' calls
    # (a host link of about 210 GB/s makes the copies the longer part).
    # (the batch's matrices live in one pinned host arena and one device arena,
    # 256-byte aligned, so that a step's input is one copy, not 4096)
    h2d_bytes = wl.h2d_bytes()
    if batch_headline:
        offs, total = [], 0
        for mt in wl.mats:
            total = round_up(total, 256)
            offs.append(total)
            total += mt.nbytes
        dev_arena = torch.empty(total, dtype=torch.uint8, device=device)
        host_arena = torch.empty(total, dtype=torch.uint8, pin_memory=True)
        bufs = []
        for mt, o in zip(wl.mats, offs):
            host_arena[o:o + mt.nbytes].view(mt.dev.dtype).view(mt.dev.shape).copy_(mt.host)
            bufs.append(dev_arena[o:o + mt.nbytes].view(mt.dev.dtype).view(mt.dev.shape))
        h2d_bytes = total
    else:
        bufs = [torch.empty_like(mt.dev) for mt in wl.mats]
    eprep = wl.prepare(ms, ctx, tensors=bufs)
    res_host = torch.empty(wl.res.shape, dtype=torch.int32, pin_memory=True)
    copy_stream = torch.cuda.Stream(device)
    copied = [torch.cuda.Event() for _ in wl.mats]

    def e2e_step():
        if batch_headline:
            dev_arena.copy_(host_arena, non_blocking=True)
            wl.batch_step(ms, ctx, eprep, sp)
        else:
            with torch.cuda.stream(copy_stream):
                for b, mt, ev in zip(bufs, wl.mats, copied):
                    b.copy_(mt.host, non_blocking=True)
                    ev.record(copy_stream)
            for i, ev in enumerate(copied):
                stream.wait_event(ev)
                wl.step_one(ms, ctx, eprep, i, sp)
        res_host.copy_(wl.res, non_blocking=True)
        torch.cuda.synchronize()

    for _ in range(max(1, args.warmup)):
        e2e_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_ms = max_over_ranks(pg, (time.perf_counter() - t0) * 1e3, device)
    e2e = {"value": world * wl.cells * args.steps / (e2e_ms * 1e-3) / 1e9, "unit": "Gcells/s",
           "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": res_host.numel() * 4,
           "how": ("the batch's pinned host arena copied H2D in one copy, the public ms_batch "
                   "call, results read back"
                   if batch_headline else
                   "pinned host inputs copied H2D on a copy stream (matrix i's call waits for "
                   "its own copy), one public ms_* call per matrix, results read back")}

    ok = bool((wl.res[:, 3] == 0).all().item())

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(wl.specs)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Gcells/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": wl.dtype, "data": "synthetic (seeded SplitMix64 Bernoulli matrices)",
                "config": {**wl.config(), "parallelism": f"replicas x{world}",
                           "packed_path": packed_path,
                           **({"band_rows": args.band_rows} if args.band_rows else {}),
                           **({"lane_cols": args.lane_cols} if args.lane_cols else {}),
                           **({"tile_kind": args.tile_kind} if args.tile_kind else {}),
                           "timed_path": ("ms_batch, CUDA graph replay" if batch_headline
                                          else "one ms_* call per matrix (plain)")},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks, "compare": compare,
                "status_ok": ok}
        print(json.dumps(line), flush=True)
    ctx.close()


def run_serve(args, world, rank, local, pg):
    """Serving stream: Poisson arrivals of `--requests` requests, square sides
    log-uniform in [64, 8192], density uniform in [0.1, 0.9], bit-packed input
    from pinned host memory, 16 GB device admission budget.  Payloads are
    quantised to 24 side classes x 9 densities (kept pinned in host memory)."""
    import numpy as np
    import torch

    import gen
    import paper_2503_18974_gb300 as ms
    device = torch.device(f"cuda:{local}")
    torch.cuda.set_device(device)
    ms.build()
    rng = np.random.default_rng(5)
    sides = np.unique(np.round(np.exp(np.linspace(np.log(64), np.log(8192), 24))).astype(int))
    dens = np.arange(1, 10) / 10
    nreq = args.requests
    req_side = np.exp(rng.uniform(np.log(64), np.log(8192), nreq))
    req_cls = np.abs(np.log(sides)[None, :] - np.log(req_side)[:, None]).argmin(1)
    req_den = np.abs(dens[None, :] - rng.uniform(0.1, 0.9, nreq)[:, None]).argmin(1)
    payload = {}
    for c, d in set(zip(req_cls.tolist(), req_den.tolist())):
        side = int(sides[c])
        ldw = ((side + 31) // 32 + 3) // 4 * 4
        dev = torch.empty((side, ldw), dtype=torch.int32, device=device)
        gen.fill_bits_dev(dev.data_ptr(), side, side, ldw, float(dens[d]), 5000 + 16 * c + d)
        host = torch.empty((side, ldw), dtype=torch.int32, pin_memory=True)
        host.copy_(dev)
        payload[(c, d)] = (host, dev, side)
    torch.cuda.synchronize()
    cells = sum(int(sides[c]) ** 2 for c in req_cls)

    # prebuilt host descriptors (the payload tensors stay alive throughout)
    descs = {key: ms.host_describe(host, n=side) for key, (host, _, side) in payload.items()}

    # results alone (the reference for "same alone and in the mix")
    ctx = ms.MaxSquare(local)
    alone = {}
    for key, (host, dev, side) in payload.items():
        alone[key] = ctx.max_square(dev, n=side).cpu().tolist()

    def serve(rate):
        srv = ms.Server(local, memory_budget=16 << 30, streams=3, max_batch=512)
        srv.submit(payload[(req_cls[0], req_den[0])][0].numpy()[:1], n=64)  # warm
        srv.wait_all()
        srv.poll()
        t0 = ms.now() + 0.01
        arrivals = t0 + (np.cumsum(rng.exponential(1.0 / rate, nreq)) if rate else np.zeros(nreq))
        keys = [(int(req_cls[k]), int(req_den[k])) for k in range(nreq)]
        arr_list = [float(x) for x in arrivals]
        ids = {}
        now = ms.now
        sub = srv.submit_desc
        while now() < t0:
            pass
        ts0 = now()
        for k in range(nreq):
            if rate:
                while now() < arr_list[k]:
                    pass
            ids[sub(descs[keys[k]], arr_list[k])] = keys[k]
        submit_s = now() - ts0
        srv.wait_all()
        done = srv.poll(nreq + 10)
        st = srv.stats()
        srv.close()
        lat = np.array([c["t_done"] - c["t_submit"] for c in done])
        span = max(c["t_done"] for c in done) - float(arrivals[0])
        wrong = sum(1 for c in done if c["result"] != alone[ids[c["id"]]])
        return {"cells_per_s": cells / span, "req_per_s": nreq / span, "span_s": span,
                "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3), "wrong": wrong,
                "batches": st["batches"], "peak_bytes": st["peak_bytes"],
                "peak_inflight": st["peak_inflight"], "completed": len(done),
                "client_submit_s": submit_s, "server_host_batch_s": st["host_batch_s"],
                "server_host_copy_s": st["host_copy_s"]}

    sat = serve(0)
    runs = {}
    clocks = None
    for f in (0.5, 0.7, 0.9):
        if f == 0.7:  # the headline run: clocks sampled while it serves
            sampler = ClockSampler(local)
            sampler.start()
            time.sleep(0.4)
            tw0 = time.time()
            runs["0.7x"] = serve(f * sat["req_per_s"])
            sampler.mark(tw0, time.time())
            clocks = sampler.stop()
        else:
            runs[f"{f}x"] = serve(f * sat["req_per_s"])

    # per-request plain launches, FIFO: copy in, ms_max_square, read back
    buf = torch.empty(max(h.numel() for h, _, _ in payload.values()), dtype=torch.int32,
                      device=device)
    res = torch.empty(4, dtype=torch.int32, device=device)
    res_h = torch.empty(4, dtype=torch.int32, pin_memory=True)
    sub = min(nreq, 4000)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain_cells = 0
    for k in range(sub):
        host, _, side = payload[(int(req_cls[k]), int(req_den[k]))]
        d = buf[:host.numel()].view(host.shape)
        d.copy_(host, non_blocking=True)
        ctx.max_square(d, n=side, out=res)
        res_h.copy_(res, non_blocking=True)
        torch.cuda.synchronize()
        plain_cells += side * side
    plain = plain_cells / (time.perf_counter() - t0)
    ctx.close()
    r7 = runs["0.7x"]
    if rank == 0:
        line = {"metric": METRIC, "value": r7["cells_per_s"] / 1e9, "unit": "Gcells/s",
                "n_gpus": world, "steps": 1, "warmup": 1,
                "ms_per_step": r7["span_s"] * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "bits32",
                "data": "synthetic (seeded SplitMix64 Bernoulli matrices)",
                "config": {"workload": f"serving stream: {nreq} Poisson requests at 0.7x the "
                                       "saturated rate, sides log-uniform 64..8192, p in "
                                       "0.1..0.9, bit-packed, 16 GB admission budget",
                           "payload_classes": len(payload), "cells": cells},
                "serve": {"saturated": sat, **runs},
                "p50_ms": r7["p50_ms"], "p99_ms": r7["p99_ms"],
                "plain_per_request": {"value": plain / 1e9, "unit": "Gcells/s",
                                      "requests": sub,
                                      "how": "FIFO, one H2D + ms_max_square + D2H per request"},
                "e2e": {"value": r7["cells_per_s"] / 1e9, "unit": "Gcells/s",
                        "h2d_bytes_per_step": int(cells // 8),
                        "d2h_bytes_per_step": 16 * nreq,
                        "how": "requests submitted from pinned host memory; latency includes "
                               "queueing, copies and read-back"},
                "roofline": None, "cpu_baseline": None, "clocks": clocks,
                # each batch is one ms_batch: the tile-queue launch and the fix-up launch
                "gpu_launches": 2 * r7["batches"]}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sweep")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--requests", type=int, default=20000)
    ap.add_argument("--packed-path", type=int, default=None,
                    help="packed size-only work: 0 tile kernel, 1 bitplane search "
                         "(default: the autotuner's choice)")
    ap.add_argument("--band-rows", type=int, default=0,
                    help="rows per tile (0: automatic, or autotuned for multi-matrix runs)")
    ap.add_argument("--tile-kind", type=int, default=0, choices=[0, 1, 2],
                    help="size-only tile pass: 0 automatic, 1 dp recurrence, 2 bitplane tiles")
    ap.add_argument("--lane-cols", type=int, default=0,
                    help="columns per lane in a tile (0: automatic)")
    args = ap.parse_args()
    world, rank, local, pg = dist_setup(args)
    try:
        if args.impl == "reference":
            run_reference(args, world, rank, local, pg)
        elif args.workload == "c5":
            run_serve(args, world, rank, local, pg)
        else:
            run_ours(args, world, rank, local, pg)
    finally:
        if pg is not None:
            pg.destroy_process_group()


if __name__ == "__main__":
    main()

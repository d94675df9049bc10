"""Benchmark of the symmetric-heap hot path on one GB300.

Workload (one step): the collective and RMA bandwidth sweep over 64 virtual PEs --
int32/int64 sum and max all-reduce and int32/int64 fcollect of 1 Ki-16 Mi elements,
alltoall of 4 KiB-1 MiB per PE pair, broadcast of 1 KiB-256 MiB, and a ring of
concurrent device-initiated put_nbi (then get_nbi) of 8 B-256 MiB from every PE to its
neighbour followed by quiet.  Metric: GB/s of algorithmic bytes over the whole step,
with per-op GB/s and the dominant kernel's fraction of the measured HBM copy peak.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

--impl reference times the CPU oracle on a bounded sample of the same workload.
Under torchrun every rank runs an independent replica on its own GPU (nothing is
exchanged between GPUs).  Rank 0 prints each secondary leg's full record on its own
JSON line ({"leg": ...}), then the headline as the LAST line, kept under 1400 bytes.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

KiB, MiB, GiB = 1 << 10, 1 << 20, 1 << 30
NPES = 64
H = 768 * MiB               # the largest sweep points (256 MiB src + dst) and a second source region
A_OFF, B_OFF = 0, 256 * MiB  # sources live in region A, destinations in region B
A2_OFF = 512 * MiB           # the end-to-end leg's second source region (its steps alternate A / A2)
I32_OFF = 128 * MiB          # int32 sources: A[128 MiB, 192 MiB); int64 sources: A[0, 128 MiB)
METRIC = "collective & bulk-RMA GB/s vs HBM peak; AMO GUPS; served p50/p99 op latency"
WORKLOAD = ("64 virtual PEs x 512 MiB sweep: int32/int64 sum+max reduce and fcollect 1Ki-16Mi elements; "
            "alltoall 4KiB-1MiB/pair; broadcast 1KiB-256MiB; put_nbi/get_nbi ring + quiet 8B-256MiB")


def sweep_points():
    """(name, family, size, algorithmic bytes) of one step, in execution order."""
    P = NPES
    pts = []
    for n in W.SWEEP_ELEMS:
        for dt, es in (("int32", 4), ("int64", 8)):
            for op in ("sum", "max"):
                pts.append((f"reduce_{dt}_{op}", "reduce", n, 2 * P * n * es))
    for L in W.SWEEP_ELEMS:
        for dt, es in (("int32", 4), ("int64", 8)):
            n = max(1, L // P)  # fcollect length = total destination elements
            pts.append((f"fcollect_{dt}", "fcollect", n, P * n * es + P * P * n * es))
    for m in W.SWEEP_A2A_BYTES:
        pts.append(("alltoall", "alltoall", m, 2 * P * P * m))
    for m in W.SWEEP_BCAST_BYTES:
        pts.append(("broadcast", "broadcast", m, (P + 1) * m))
    for m in W.SWEEP_PUT_BYTES:
        pts.append(("put_nbi_ring", "put", m, 2 * P * m))
    for m in W.SWEEP_PUT_BYTES:
        pts.append(("get_nbi_ring", "get", m, 2 * P * m))
    return pts


def ring_script(kind, m, a_off=A_OFF):
    ops = np.zeros(NPES + 1, W.OP_DTYPE)
    for p in range(NPES):
        q = (p + 1) % NPES
        if kind == "put":   # PE p: its A -> PE q's B
            ops[p] = (W.OP_PUT_NBI, 0, 0, 0, q, p, B_OFF, a_off, m, 0, 0, 0)
        else:               # PE p: PE q's A -> its own B
            ops[p] = (W.OP_GET_NBI, 0, 0, 0, q, p, B_OFF, a_off, m, 0, 0, 0)
    ops[NPES] = (W.OP_QUIET, 0, 0, 0, 0, -1, 0, 0, 0, 0, 0, 0)
    return ops


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 100 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- GPU arm
class GpuStep:
    def __init__(self, torch, sg, stream):
        self.torch, self.sg, self.stream = torch, sg, stream
        self.heap = sg.Heap(NPES, H, pe_mode=sg.PE_MODE_CLUSTER, cluster_dim=2, stream=stream)
        base = self.heap.base
        self.A, self.B, self.A32 = base + A_OFF, base + B_OFF, base + A_OFF + I32_OFF
        self.pts = sweep_points()
        self.scripts = {}
        for name, fam, m, _ in self.pts:
            if fam in ("put", "get"):
                for reg, a_off in ((0, A_OFF), (1, A2_OFF)):
                    self.scripts[(fam, m, reg)] = torch.from_numpy(ring_script(fam, m, a_off).view(np.uint8).copy()).cuda()
        self.fill_inputs()

    def fill_inputs(self):
        """Region A of every PE: int64 values U[-2^20, 2^20] in [0, 128 MiB), int32 values in
        [128 MiB, 192 MiB), seeded counter draws (workloads); the rest of A is bytes."""
        torch = self.torch
        parts = self.heap.partitions()
        seed = W.derive_seed("sweep-inputs")
        for p in range(NPES):
            i64 = torch.arange(16 << 20, dtype=torch.int64, device="cuda") + (p << 32)
            parts[p, A_OFF:A_OFF + 128 * MiB].view(torch.int64).copy_(W.uniform_ints_torch(seed, i64, -(1 << 20), 1 << 20))
            v32 = W.uniform_ints_torch(seed ^ 1, i64, -(1 << 20), 1 << 20).to(torch.int32)
            parts[p, A_OFF + I32_OFF:A_OFF + I32_OFF + 64 * MiB].view(torch.int32).copy_(v32)
            parts[p, A_OFF + 192 * MiB:A_OFF + 256 * MiB].view(torch.int64).copy_(
                W.cb64_torch(seed ^ 2, i64[: 8 << 20]))
        torch.cuda.synchronize()

    def launches_per_step(self):
        return len(self.pts)

    def run_point(self, name, fam, m, region=0):
        """One sweep point; region 1 reads the second source region (A2) instead of A."""
        sg, s = self.sg, self.stream
        A = self.A + (A2_OFF - A_OFF if region else 0)
        A32 = self.A32 + (A2_OFF - A_OFF if region else 0)
        if fam == "reduce":
            _, dt, op = name.split("_")
            dtype = sg.INT32 if dt == "int32" else sg.INT64
            src = A32 if dt == "int32" else A
            sg.reduce(sg.TEAM_WORLD, self.B, src, m, dtype, sg.SUM if op == "sum" else sg.MAX, s)
        elif fam == "fcollect":
            es = 4 if name.endswith("int32") else 8
            src = A32 if es == 4 else A
            sg.fcollectmem(sg.TEAM_WORLD, self.B, src, m * es, s)
        elif fam == "alltoall":
            sg.alltoallmem(sg.TEAM_WORLD, self.B, A, m, s)
        elif fam == "broadcast":
            sg.broadcastmem(sg.TEAM_WORLD, self.B, A, m, NPES - 1, s)
        else:
            sg.run_script(self.scripts[(fam, m, region)], NPES + 1, None, s)

    def step(self, events=None):
        for i, (name, fam, m, _) in enumerate(self.pts):
            if events is not None:
                events[i][0].record(self.stream)
            self.run_point(name, fam, m)
            if events is not None:
                events[i][1].record(self.stream)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def run_gpu(args, rank, world):
    import torch

    import paper_2607_08006_gb300 as sg

    sg.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = GpuStep(torch, sg, stream)
        pts = g.pts
        for _ in range(args.warmup):
            g.step()
        stream.synchronize()
        code, detail = sg.get_status()
        if code != 0:
            raise RuntimeError(f"device status {code} ({sg.strerror(code)}) detail {detail}")
        # ---- timed region: K steps between barriers, events per launch on the stream
        ev = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in pts]
              for _ in range(args.steps)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clocks = ClockSampler(dev)
        barrier(world)
        torch.cuda.synchronize()
        clocks.start()
        t0.record(stream)
        for k in range(args.steps):
            g.step(ev[k])
        t1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        barrier(world)
        total_ms = t0.elapsed_time(t1)
        total_ms = max_over_ranks(total_ms, world)
        code, detail = sg.get_status()
        if code != 0:
            raise RuntimeError(f"device status {code} after timed steps")
        bytes_step = sum(b for *_, b in pts)
        per_pt = np.array([[ev[k][i][0].elapsed_time(ev[k][i][1]) for i in range(len(pts))]
                           for k in range(args.steps)]).mean(axis=0)
        # the GPU on the oracle's bounded sample: the same points, their own launch times
        sample = {(nm, f, m) for nm, f, m, _ in cpu_sample_points()}
        sel = [i for i, (nm, f, m, _) in enumerate(pts) if (nm, f, m) in sample]
        same_sample = {"value": round(sum(pts[i][3] for i in sel) / (float(sum(per_pt[i] for i in sel)) * 1e-3) / 1e9, 1),
                       "unit": "GB/s"}
        # ---- end-to-end: host inputs -> device, the step, result -> host
        e2e = run_e2e(torch, sg, g, stream, args, world)
        summary = summarise(pts, per_pt)
        hbm, src = measured_peaks()
        rl = roofline_for(summary, hbm, src)
        g.heap.close()
    ms_step = total_ms / args.steps
    value = world * bytes_step / (ms_step * 1e-3) / 1e9
    out = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32/int64",
        "data": "synthetic, seeded",
        "config": headline_config(world),
        "roofline": rl,
        "gpu_launches": g.launches_per_step() * args.steps,
        "clocks": clk,
        "e2e": e2e,
        "gpu_on_cpu_sample": same_sample,
        "per_family": summary["families"],
        "largest_points": summary["largest"],
        "points": [[nm, m, round(float(ms), 4), round(b / (float(ms) * 1e-3) / 1e9, 1)]
                   for (nm, f, m, b), ms in zip(pts, per_pt)],
    }
    return out


def headline_config(world):
    """The workload of one step, as both arms name it."""
    return {"workload": WORKLOAD, "npes": NPES, "pe": "2-CTA cluster",
            "algorithmic_bytes_per_step": sum(b for *_, b in sweep_points()),
            "l2": "no flush: %d GiB/step >> L2" % (sum(b for *_, b in sweep_points()) // GiB),
            "parallelism": "replicas" if world > 1 else "single GPU"}


def summarise(pts, per_pt_ms):
    fam = {}
    largest = {}
    for (name, f, m, b), ms in zip(pts, per_pt_ms):
        d = fam.setdefault(f, {"ms": 0.0, "bytes": 0, "launches": 0})
        d["ms"] += float(ms)
        d["bytes"] += b
        d["launches"] += 1
        cur = largest.get(name)
        if cur is None or m > cur["size"]:
            largest[name] = {"size": m, "ms": round(float(ms), 4), "GBps": round(b / (ms * 1e-3) / 1e9, 1)}
    for d in fam.values():
        d["GBps"] = round(d["bytes"] / (d["ms"] * 1e-3) / 1e9, 1)
        d["ms"] = round(d["ms"], 3)
    return {"families": fam, "largest": largest}


KERNEL_OF = {"reduce": "k_reduce", "fcollect": "k_xfer", "alltoall": "k_xfer", "broadcast": "k_xfer",
             "put": "k_interp", "get": "k_interp"}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def roofline_for(summary, hbm, src):
    """Roofline of the kernel with the largest share of the step (families grouped by
    the kernel that runs them)."""
    per_k = {}
    for fam, d in summary["families"].items():
        k = per_k.setdefault(KERNEL_OF[fam], {"ms": 0.0, "bytes": 0, "launches": 0, "families": []})
        k["ms"] += d["ms"]
        k["bytes"] += d["bytes"]
        k["launches"] += d["launches"]
        k["families"].append(fam)
    name, d = max(per_k.items(), key=lambda kv: kv[1]["ms"])
    achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9
    traffic = None
    if os.path.exists(TRAFFIC_FILE):
        with open(TRAFFIC_FILE) as f:
            t = json.load(f).get(name)
        if t:
            # the captured launch's DRAM bytes, scaled by algorithmic bytes to one average
            # launch of this workload (traffic grows in proportion to the bytes moved)
            traffic = round(t["capture_dram_bytes"] / t["capture_algorithmic_bytes"] * d["bytes"] / d["launches"])
    total_ms = sum(v["ms"] for v in per_k.values())
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "traffic": traffic, "kernel": name,
            "families": d["families"], "share_of_step": round(d["ms"] / total_ms, 3),
            "peak_source": "measured hbm_gbs" if src == "measured" else "fallback 6.8 TB/s",
            "launches_per_step": d["launches"], "algorithmic_bytes_per_step": d["bytes"],
            "avg_launch_ms": round(d["ms"] / d["launches"], 4),
            "per_kernel": {k: {"ms_per_step": round(v["ms"], 3), "GBps": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1),
                               "share": round(v["ms"] / total_ms, 3)} for k, v in per_k.items()}}


E2E_CHUNK = 32 * MiB
# the order region A's chunks are copied in: the int64 and int32 source areas interleaved
# from their starts (the small reductions of both kinds can start early), the byte area
# (read only by the largest broadcasts and rings) last
E2E_CHUNK_ORDER = [0, 4, 1, 5, 2, 3, 6, 7]


def point_reads(name, fam, m):
    """Bytes [lo, hi) of region A that a sweep point reads (on every PE, or the root)."""
    if fam in ("reduce", "fcollect"):
        es = 4 if "int32" in name else 8
        lo = I32_OFF if es == 4 else 0
        return lo, lo + m * es
    if fam == "alltoall":
        return 0, NPES * m
    return 0, m  # broadcast, put, get


def run_e2e(torch, sg, g, stream, args, world):
    """Same step through the public API with the inputs on the HOST: every step copies
    the sources of every PE from pinned host memory, runs the sweep on them, and reads PE
    0's destination region B back.  The copies are pipelined with the work: a step's
    sources move in 32 MiB chunks on a copy stream in E2E_CHUNK_ORDER, and each point runs
    once the chunks it reads have landed (points in order of readiness, the sweep's order
    among equals).  Steps alternate between source regions A and A2, so the next step's
    copies start as soon as this step's are done (they wait only for the step before this
    one to have finished reading the region they overwrite): the copy stream never idles."""
    steps = max(1, min(args.steps, 3))
    parts = g.heap.partitions()
    host_in = torch.empty((NPES, 256 * MiB), dtype=torch.uint8, pin_memory=True)
    for p in range(NPES):
        host_in[p].copy_(parts[p, A_OFF:A_OFF + 256 * MiB])
    host_out = torch.empty(256 * MiB, dtype=torch.uint8, pin_memory=True)
    copy_stream = torch.cuda.Stream()
    pos = {c: k for k, c in enumerate(E2E_CHUNK_ORDER)}
    regions = (A_OFF, A2_OFF)

    def ready_after(pt):
        lo, hi = point_reads(pt[0], pt[1], pt[2])
        return max(pos[c] for c in range(lo // E2E_CHUNK, (hi + E2E_CHUNK - 1) // E2E_CHUNK))

    order = sorted(range(len(g.pts)), key=lambda k: (ready_after(g.pts[k]), k))
    done = [None, None]  # per region: the event after the last step that read it

    def issue_copies(k):
        reg = k % 2
        if done[reg] is not None:
            copy_stream.wait_event(done[reg])  # that step has finished reading the region
        landed = []
        with torch.cuda.stream(copy_stream):
            for c in E2E_CHUNK_ORDER:
                lo = regions[reg] + c * E2E_CHUNK
                for p in range(NPES):
                    parts[p, lo:lo + E2E_CHUNK].copy_(host_in[p, c * E2E_CHUNK:(c + 1) * E2E_CHUNK],
                                                      non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(copy_stream)
                landed.append(ev)
        return landed

    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    t0.record(stream)
    copy_stream.wait_event(t0)
    landed = issue_copies(0)
    for k in range(steps):
        nxt = issue_copies(k + 1) if k + 1 < steps else None
        waited = -1
        for i in order:
            need = ready_after(g.pts[i])
            if need > waited:
                stream.wait_event(landed[need])
                waited = need
            g.run_point(*g.pts[i][:3], region=k % 2)
        host_out.copy_(parts[0, B_OFF:B_OFF + 256 * MiB], non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(stream)
        done[k % 2] = ev
        landed = nxt
    t1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(t0.elapsed_time(t1), world) / steps
    bytes_step = sum(b for *_, b in g.pts)
    return {"value": round(world * bytes_step / (ms * 1e-3) / 1e9, 1), "unit": "GB/s",
            "h2d_bytes_per_step": NPES * 256 * MiB, "d2h_bytes_per_step": 256 * MiB,
            "ms_per_step": round(ms, 3), "steps": steps,
            "pipeline": "32 MiB chunks on a copy stream, each point waits for the chunks it reads; "
                        "steps alternate two source regions, so the next step's copies overlap this step"}


# ----------------------------------------------------------------------------- CPU oracle arm
CPU_MAX_ELEMS = 1 << 18
CPU_MAX_BYTES = 1 * MiB
CPU_MAX_A2A = 64 * KiB


def cpu_sample_points():
    """The sweep restricted to its small points (the oracle would need minutes per
    large point); same 64 PEs, same formulas."""
    out = []
    for name, fam, m, b in sweep_points():
        if fam in ("reduce", "fcollect") and m * (1 if fam == "reduce" else NPES) > CPU_MAX_ELEMS:
            continue
        if fam in ("broadcast", "put", "get") and m > CPU_MAX_BYTES:
            continue
        if fam == "alltoall" and m > CPU_MAX_A2A:
            continue
        out.append((name, fam, m, b))
    return out


def run_cpu_sample(orc, heap, pts):
    P = NPES
    team = (0, 1, P)
    Hs = heap.H
    a, bb, a32 = 0, Hs // 2, Hs // 4
    t0 = time.perf_counter()
    for name, fam, m, _ in pts:
        if fam == "reduce":
            _, dt, op = name.split("_")
            heap.reduce(team, bb, a32 if dt == "int32" else a, m, W.DT_INT32 if dt == "int32" else W.DT_INT64,
                        W.RED_SUM if op == "sum" else W.RED_MAX)
        elif fam == "fcollect":
            es = 4 if name.endswith("int32") else 8
            heap.fcollect(team, bb, a32 if es == 4 else a, m * es)
        elif fam == "alltoall":
            heap.alltoall(team, bb, a, m)
        elif fam == "broadcast":
            heap.broadcast(team, bb, a, m, P - 1)
        elif fam == "put":
            for p in range(P):
                heap.put(bb, a, m, (p + 1) % P, p)
        else:
            for p in range(P):
                heap.get(bb, a, m, (p + 1) % P, p)
    return time.perf_counter() - t0


def cpu_heap(orc):
    Hs = 8 * MiB
    seed = W.derive_seed("sweep-inputs")
    init = np.zeros((NPES, Hs), np.uint8)
    for p in range(NPES):
        i = np.arange(Hs // 16, dtype=np.uint64) + np.uint64(p << 32)
        init[p, :Hs // 2].view(np.int64)[: Hs // 16] = W.uniform_ints_np(seed, i, -(1 << 20), 1 << 20)
    return orc.Heap(NPES, Hs, init.reshape(-1))


def cpu_baseline(reps=None):
    import oracle as orc

    orc.build()
    heap = cpu_heap(orc)
    pts = cpu_sample_points()
    b = sum(x[3] for x in pts)
    secs = run_cpu_sample(orc, heap, pts)
    n = reps or max(1, int(12.0 / max(secs, 1e-3)))
    secs = sum(run_cpu_sample(orc, heap, pts) for _ in range(n))
    return {"value": round(n * b / secs / 1e9, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"{len(pts)} small sweep points (<= 256 Ki elts, <= 1 MiB msgs), {n} passes, {secs:.1f} s",
            "seconds": round(secs, 2)}


def run_reference(args, rank, world):
    import oracle as orc

    orc.build()
    heap = cpu_heap(orc)
    pts = cpu_sample_points()
    b = sum(x[3] for x in pts)
    for _ in range(args.warmup):
        run_cpu_sample(orc, heap, pts)
    secs = sum(run_cpu_sample(orc, heap, pts) for _ in range(args.steps))
    value = b * args.steps / secs / 1e9
    sample = f"{len(pts)} small sweep points (<= 256 Ki elts, <= 1 MiB msgs) per step, single-threaded oracle"
    return {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32/int64",
            "data": "synthetic", "config": headline_config(world),
            "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ----------------------------------------------------------------------------- scripted stream
def run_script_leg(torch, sg, reps=5):
    """The 4-PE x 1 MiB scripted stream of 10,000 ops (+20 barriers): device-initiated
    (one cooperative launch) and launch-per-op, each checked against the oracle's final
    heap, with the oracle's own time (single thread)."""
    import oracle as orc

    s = W.gen_plain_script()
    heap = sg.Heap(s.npes, s.heap_bytes)
    out = {"ops": int(len(s.ops))}
    try:
        parts = heap.partitions()
        init = torch.from_numpy(s.heap.reshape(s.npes, s.heap_bytes)).cuda()
        dev_ops = torch.from_numpy(s.ops.view(np.uint8).copy()).cuda()
        fetched = torch.zeros(len(s.ops), dtype=torch.int64, device="cuda")
        stream = torch.cuda.current_stream()
        ref = orc.Heap(s.npes, s.heap_bytes, s.heap)
        t0 = time.perf_counter()
        ref.run_script(s.ops)
        out["oracle_ms"] = round((time.perf_counter() - t0) * 1e3, 3)
        for mode in ("device", "host"):
            times = []
            for _ in range(reps + 1):
                parts.copy_(init)
                torch.cuda.synchronize()
                e0, e1 = _events(torch)
                e0.record(stream)
                if mode == "device":
                    sg.run_script(dev_ops, len(s.ops), fetched, stream)
                else:
                    sg.run_script_host(s.ops, fetched, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            ok = bool(np.array_equal(parts.cpu().numpy().reshape(-1), ref.mem))
            ms = float(np.median(times[1:]))
            out[mode] = {"ms": round(ms, 3), "ops_per_s": round(len(s.ops) / (ms * 1e-3), 1), "heap_matches_oracle": ok}
        out["status"] = sg.get_status()[0]
    finally:
        heap.close()
    return out


# ----------------------------------------------------------------------------- cluster (DSMEM) team
def run_cluster_leg(torch, sg, rounds=200, reps=3, iters=10000):
    """The device shared team as a thread-block cluster.  (1) The 512 put_signal /
    wait_until ping-pong pairs (1024 CTAs, each pair inside one 2-CTA cluster) through
    distributed shared memory vs the same pairs through L2/HBM, half round trip per
    payload, final heaps checked.  (2) One cluster of 8 CTA PEs: `rounds` collectives in
    one device-initiated script on the shared team (hardware cluster barrier; alltoalls of
    up to 8 KiB per member staged in the DSMEM windows, the rest through L2) vs the same 8
    PEs as the world team (L2 barrier) at PE scope and at warp scope, time per collective,
    results compared."""
    out = {}
    npes, H = 1024, 16384
    heap = sg.Heap(npes, H, pe_mode=sg.PE_MODE_CTA, cluster_dim=2)
    try:
        parts = heap.partitions()
        parts.random_(0, 255)
        sig_off = 3 * 4096
        lat = torch.zeros(512 * iters, dtype=torch.int64, device="cuda")
        pp = {}
        for payload in (8, 64, 512, 4096):
            row = {}
            for mode, fn in (("l2", sg.pingpong), ("dsmem", sg.pingpong_cluster)):
                parts[:, payload:2 * payload].zero_()
                parts[:, sig_off:sig_off + 8].zero_()
                torch.cuda.synchronize()
                fn(heap.base, heap.base + sig_off, payload, 512, iters, lat)
                torch.cuda.synchronize()
                half = lat.cpu().numpy().astype(np.float64) / 2 / 1e3
                peer = parts.view(512, 2, H).flip(1).reshape(npes, H)
                ok = bool(torch.equal(parts[:, payload:2 * payload], peer[:, :payload])) and \
                    bool((parts[:, sig_off:sig_off + 8].contiguous().view(torch.int64) == iters).all())
                row[mode] = {"half_rtt_us_p50": round(float(np.percentile(half, 50)), 3),
                             "half_rtt_us_p99": round(float(np.percentile(half, 99)), 3), "final_heap_ok": ok}
            row["speedup_p50"] = round(row["l2"]["half_rtt_us_p50"] / row["dsmem"]["half_rtt_us_p50"], 2)
            pp[str(payload)] = row
        out["pingpong_512_pairs"] = pp
        del lat
    finally:
        heap.close()

    P, Hc = 8, 1 << 20
    heap = sg.Heap(P, Hc, pe_mode=sg.PE_MODE_CTA, cluster_dim=P)
    try:
        parts = heap.partitions()
        parts.random_(0, 255)
        parts[:, :65536].view(torch.float32).normal_()
        stream = torch.cuda.current_stream()
        dst = 512 * 1024
        cases = [("team_sync", W.OP_TEAM_SYNC, 0, 0, 0), ("reduce_int64_256B", W.OP_REDUCE, W.DT_INT64, 0, 32),
                 ("reduce_int64_4KiB", W.OP_REDUCE, W.DT_INT64, 0, 512),
                 ("reduce_int64_64KiB", W.OP_REDUCE, W.DT_INT64, 0, 8192),
                 ("reduce_fp32_4KiB", W.OP_REDUCE, W.DT_FLOAT, 0, 1024), ("broadcast_4KiB", W.OP_BCAST, 0, 3, 4096),
                 ("broadcast_64KiB", W.OP_BCAST, 0, 3, 65536), ("fcollect_4KiB", W.OP_FCOLLECT, 0, 0, 4096),
                 ("alltoall_512B", W.OP_ALLTOALL, 0, 0, 512), ("alltoall_4KiB", W.OP_ALLTOALL, 0, 0, 4096)]
        coll = {}
        for name, kind, dt, root, n in cases:
            row = {}
            res = {}
            for mode, team, flag in (("global", 0, 0), ("global_warp", 0, W.OP_WARP), ("shared", 1, 0)):
                ops = np.zeros(rounds, W.OP_DTYPE)
                for k in range(rounds):
                    ops[k] = (kind | flag, dt, W.RED_SUM, team, root, -1, dst, 4096 if kind != W.OP_REDUCE else 0, n,
                              0, 0, 0)
                dev = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
                parts[:, dst:].zero_()
                times = []
                for _ in range(reps + 1):
                    e0, e1 = _events(torch)
                    e0.record(stream)
                    sg.run_script(dev, rounds, None, stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1))
                res[mode] = parts[:, dst:dst + 65536].clone()
                row[mode + "_us_per_op"] = round(float(np.median(times[1:])) * 1e3 / rounds, 3)
            row["speedup"] = round(row["global_us_per_op"] / row["shared_us_per_op"], 2)
            row["results_equal"] = bool(torch.equal(res["global"], res["shared"])) and \
                bool(torch.equal(res["global"], res["global_warp"]))
            coll[name] = row
        out["one_cluster_8_pes"] = coll
        out["status"] = sg.get_status()[0]
    finally:
        heap.close()
    return out


# ----------------------------------------------------------------------------- device contexts
def run_ctx_leg(torch, sg, reps=3, big=32 * MiB, nsmall=100, small=8 * KiB):
    """Explicit device contexts: 64 PEs (one CTA each) each move `big` bytes to a
    neighbour and run `nsmall` blocking puts of `small` bytes to another, in one script:
    the big transfer blocking on the default context, vs put_nbi on context 1 quieted at
    the end (moving in the background while the small puts run), vs each part alone.
    Also `nsmall` small puts each followed by a quiet on context 2 (independent of the big
    transfer on context 1) vs by a quiet on all contexts.  Heaps compared."""
    npes = 64
    Hc = 2 * big + 2 * nsmall * small + MiB
    heap = sg.Heap(npes, Hc)
    out = {"npes": npes, "big_bytes": big, "small_ops": nsmall, "small_bytes": small}
    try:
        parts = heap.partitions()
        parts.random_(0, 255)
        init = parts.clone()
        stream = torch.cuda.current_stream()
        B0, S0 = big, 2 * big

        def big_op(p, kind, ctx):
            return (kind, 0, ctx, 0, (p + 1) % npes, p, B0, 0, big, 0, 0, 0)

        def small_ops(p, k, quiet_ctx=None):
            # (sources in the big transfer's source range: read-only, no race with it)
            o = [(W.OP_PUT, 0, 0, 0, (p + 2) % npes, p, S0 + small * k, small * (k % 16), small, 0, 0, 0)]
            if quiet_ctx is not None:
                o.append((W.OP_QUIET, 0, quiet_ctx, 0, 0, p, 0, 0, 0, 0, 0, 0))
            return o

        def script(with_big, kind=W.OP_PUT, ctx=0, quiet_ctx=None, with_small=True):
            ops = []
            for p in range(npes):
                if with_big:
                    ops.append(big_op(p, kind, ctx))
            if with_small:
                for k in range(nsmall):
                    for p in range(npes):
                        ops += small_ops(p, k, quiet_ctx)
            for p in range(npes):
                ops.append((W.OP_QUIET, 0, 0xFF, 0, 0, p, 0, 0, 0, 0, 0, 0))
            ops.append((W.OP_BARRIER_ALL, 0, 0, 0, 0, -1, 0, 0, 0, 0, 0, 0))
            return np.array(ops, dtype=W.OP_DTYPE)

        cases = {"blocking_big_then_small": script(True),
                 "ctx1_big_with_small": script(True, W.OP_PUT_NBI, 1),
                 "small_only": script(False),
                 "blocking_big_only": script(True, with_small=False),
                 "ctx1_big_only": script(True, W.OP_PUT_NBI, 1, with_small=False),
                 "ctx1_big_small_quiet_ctx2": script(True, W.OP_PUT_NBI, 1, quiet_ctx=2),
                 "ctx1_big_small_quiet_all": script(True, W.OP_PUT_NBI, 1, quiet_ctx=0xFF)}
        res = {}
        heaps = {}
        for name, ops in cases.items():
            dev = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
            times = []
            for _ in range(reps + 1):
                parts.copy_(init)
                e0, e1 = _events(torch)
                e0.record(stream)
                sg.run_script(dev, len(ops), None, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            res[name] = {"ms": round(float(np.median(times[1:])), 3), "ops": int(len(ops))}
            heaps[name] = parts.clone()
        out["cases"] = res
        out["heaps_equal"] = bool(torch.equal(heaps["blocking_big_then_small"], heaps["ctx1_big_with_small"])) and \
            bool(torch.equal(heaps["ctx1_big_with_small"], heaps["ctx1_big_small_quiet_ctx2"]))
        out["overlap_saving_ms"] = round(res["blocking_big_then_small"]["ms"] - res["ctx1_big_with_small"]["ms"], 3)
        out["quiet_ctx2_saving_ms"] = round(res["ctx1_big_small_quiet_all"]["ms"] - res["ctx1_big_small_quiet_ctx2"]["ms"], 3)
        out["ctx1_GBps"] = round(npes * 2 * big / (res["ctx1_big_only"]["ms"] * 1e-3) / 1e9, 1)
        out["blocking_GBps"] = round(npes * 2 * big / (res["blocking_big_only"]["ms"] * 1e-3) / 1e9, 1)
        out["status"] = sg.get_status()[0]
    finally:
        heap.close()
    return out


# ----------------------------------------------------------------------------- halo exchange
def run_halo(torch, sg, iters=100, reps=3):
    """The halo-exchange stencil (case study 1): 152 PEs (one per SM) as 19 x 8 tiles of
    1024 x 1024 binary32 (a 8192 x 19456 periodic grid, 608 MiB per buffer), `iters` Jacobi sweeps
    with the boundary stores fused into each sweep and one signal per neighbour (one
    launch), vs one launch per sweep; PE = one CTA and PE = a 2-CTA cluster.  GB/s of
    algorithmic bytes (every sweep reads and writes the grid, plus the halos); results of
    both forms compared bitwise; the oracle timed on one sweep of a 2048 x 4096 sample."""
    import oracle as orc

    px, py, nx, ny = 19, 8, 1024, 1024
    npes = px * py
    hs = sg.halo_stride(nx, ny)
    tile_b, halo_b = 2 * nx * ny * 4, 2 * hs * 4
    H = (tile_b + halo_b + 64 + 4095) // 4096 * 4096
    sweep_bytes = npes * (2 * nx * ny * 4 + 2 * (2 * nx + 2 * ny) * 4)
    out = {"pes": f"{px}x{py}", "tile": f"{nx}x{ny}", "grid": f"{py * ny}x{px * nx}", "iters": iters,
           "bytes_per_sweep": sweep_bytes}
    stream = torch.cuda.current_stream()
    for name, mode, cd in (("cta", sg.PE_MODE_CTA, 1), ("cluster2", sg.PE_MODE_CLUSTER, 2)):
        heap = sg.Heap(npes, H, pe_mode=mode, cluster_dim=cd)
        try:
            parts = heap.partitions()
            parts.zero_()
            gen = torch.Generator(device="cuda")
            gen.manual_seed(W.derive_seed("halo") & 0x7FFFFFFF)
            init = torch.randn(npes, nx * ny, device="cuda", generator=gen)
            tiles, halos, sigs = heap.sym(0, tile_b), heap.sym(tile_b, halo_b), heap.sym(tile_b + halo_b, 32)
            row = {}
            res = {}
            for variant in ("persistent", "plain"):
                times = []
                for _ in range(reps + 1):
                    parts[:, :nx * ny * 4].view(torch.float32).copy_(init)
                    e0, e1 = _events(torch)
                    e0.record(stream)
                    sg.halo_jacobi(tiles, halos, sigs, px, py, nx, ny, iters, stream, plain=variant == "plain")
                    e1.record(stream)
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1))
                ms = float(np.median(times[1:]))
                r0 = (iters & 1) * nx * ny * 4
                res[variant] = parts[:, r0:r0 + nx * ny * 4].clone()
                row[variant] = {"ms": round(ms, 3), "us_per_sweep": round(ms * 1e3 / iters, 2),
                                "GBps": round(iters * sweep_bytes / (ms * 1e-3) / 1e9, 1)}
            row["speedup_vs_plain"] = round(row["plain"]["ms"] / row["persistent"]["ms"], 2)
            row["results_equal"] = bool(torch.equal(res["persistent"], res["plain"]))
            row["status"] = sg.get_status()[0]
            out[name] = row
        finally:
            heap.close()
    hbm, _ = measured_peaks()
    best = max(out["cta"]["persistent"]["GBps"], out["cluster2"]["persistent"]["GBps"])
    out["frac_of_hbm"] = round(best / hbm, 4)
    # a strong-scaling point: the same 19 x 8 PEs with 256 x 256 tiles (the grid fits in
    # L2), where each sweep is short and the per-sweep synchronisation decides
    sn, sit = 256, 400
    shs = sg.halo_stride(sn, sn)
    st_b, sh_b = 2 * sn * sn * 4, 2 * shs * 4
    heap = sg.Heap(npes, (st_b + sh_b + 64 + 4095) // 4096 * 4096)
    try:
        parts = heap.partitions()
        parts.zero_()
        init = torch.randn(npes, sn * sn, device="cuda", generator=torch.Generator(device="cuda").manual_seed(7))
        tiles, halos, sigs = heap.sym(0, st_b), heap.sym(st_b, sh_b), heap.sym(st_b + sh_b, 32)
        row, res = {}, {}
        for variant in ("persistent", "plain"):
            times = []
            for _ in range(reps + 1):
                parts[:, :sn * sn * 4].view(torch.float32).copy_(init)
                e0, e1 = _events(torch)
                e0.record(stream)
                sg.halo_jacobi(tiles, halos, sigs, px, py, sn, sn, sit, stream, plain=variant == "plain")
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            r0 = (sit & 1) * sn * sn * 4
            res[variant] = parts[:, r0:r0 + sn * sn * 4].clone()
            row[variant + "_us_per_sweep"] = round(float(np.median(times[1:])) * 1e3 / sit, 2)
        row["speedup_vs_plain"] = round(row["plain_us_per_sweep"] / row["persistent_us_per_sweep"], 2)
        row["results_equal"] = bool(torch.equal(res["persistent"], res["plain"]))
        out["small_tiles_256"] = row
    finally:
        heap.close()
    g = W.normals_np(11, 2048 * 4096).astype(np.float32).reshape(2048, 4096)
    t0 = time.perf_counter()
    orc.halo_jacobi(g, 1)
    dt = time.perf_counter() - t0
    out["oracle"] = {"GBps": round(2 * g.nbytes / dt / 1e9, 3), "sample": "one sweep of a 2048 x 4096 grid",
                     "cores": 1, "seconds": round(dt, 3)}
    return out


# ----------------------------------------------------------------------------- AMO / signal stress
def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _amo_ops(pool, seed, nops, bits, dist, ch=1 << 24):
    """W.amo_stream_np over [0, nops) in chunks of `ch` ops on a process pool (the
    stream does not depend on the chunking)."""
    out = np.empty(nops, np.uint32)
    futs = {pool.submit(W.amo_stream_np, seed, min(ch, nops - c), bits, dist=dist, offset=c): c
            for c in range(0, nops, ch)}
    for f in futs:
        c = futs[f]
        out[c:c + ch] = f.result()
    return out


def run_amo(torch, sg, nops_log2=30, reps=3):
    """1024 PEs (one CTA each) over a 2^27-word int64 table; uniform and Zipf(1.1)
    streams of 2^nops_log2 fetch_add/compare_swap/fetch_xor; GUPS plain, warp-aggregated
    and block-combined, against an L2-resident table and the HBM-sector ceiling; then 512
    put_signal/wait_until ping-pong pairs."""
    npes, wpp = 1024, 1 << 17
    Hh = wpp * 8 + 16384
    heap = sg.Heap(npes, Hh)
    out = {"npes": npes, "table_words": npes * wpp, "ops": 1 << nops_log2}
    try:
        parts = heap.partitions()
        tseed, oseed = W.derive_seed("amo-table"), W.derive_seed("amo-ops")
        for p0 in range(0, npes, 128):
            idx = torch.arange(p0 * wpp, (p0 + 128) * wpp, dtype=torch.int64, device="cuda")
            parts[p0:p0 + 128, :wpp * 8].view(torch.int64).copy_(W.cb64_torch(tseed, idx).view(128, wpp))
        nops = 1 << nops_log2
        s = torch.cuda.current_stream()
        # the op streams are drawn on the host by a spawned process pool (no CUDA state in
        # the workers), chunk by chunk
        import concurrent.futures as cf
        import multiprocessing as mp

        workers = max(1, min(16, os.cpu_count() or 1))
        pool = cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn"))
        out["generator_processes"] = workers
        for dist in ("uniform", "zipf"):
            t0 = time.perf_counter()
            ops = _amo_ops(pool, W.derive_seed("amo-" + dist), nops, 27, dist)
            gen_s = time.perf_counter() - t0
            dops = torch.from_numpy(ops.view(np.int32)).cuda()
            del ops
            fetched = torch.empty(nops, dtype=torch.int64, device="cuda")
            for agg, name in ((0, "plain"), (1, "agg"), (2, "combine")):
                sg.amo_stream(heap.base, wpp, dops, nops, oseed, tseed, fetched, flags=agg)
                e0, e1 = _events(torch)
                e0.record(s)
                for _ in range(reps):
                    sg.amo_stream(heap.base, wpp, dops, nops, oseed, tseed, fetched, flags=agg)
                e1.record(s)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                out[f"{dist}_{name}"] = {"GUPS": round(nops / (ms * 1e-3) / 1e9, 3), "ms": round(ms, 3)}
            out[f"{dist}_generation_s"] = round(gen_s, 2)
            del dops, fetched
        pool.shutdown()
        # ceilings: the L2 atomic units' rate and the HBM bytes per uniform op, both from the
        # ncu counters of the stream (profiles/amo_counters.json); and the random-access
        # rate of DRAM itself over the same table -- PyTorch's gather and scatter of random
        # 8-byte words (one random read, then one random write per word, like an atomic's
        # read-modify-write without the atomic)
        hbm, _ = measured_peaks()
        with open(os.path.join(ROOT, "profiles", "amo_counters.json")) as f:
            ctr = json.load(f)
        l2_ceiling = ctr["l2_atomic_ops_per_s"] / 1e9
        hbm_ceiling = hbm / ctr["uniform_dram_bytes_per_op"]
        table = parts[:, :wpp * 8].contiguous().view(torch.int64).reshape(-1)   # a copy of the same size
        nr = 1 << 26
        gen = torch.Generator(device="cuda")
        gen.manual_seed(W.derive_seed("amo-probe") & 0x7FFFFFFF)
        idx = torch.randint(0, table.numel(), (nr,), device="cuda", generator=gen)
        vals = table[idx]
        e0, e1, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True), \
            torch.cuda.Event(enable_timing=True)
        for _ in range(2):
            e0.record(s)
            vals = table[idx]
            e1.record(s)
            table.index_put_((idx,), vals)
            e2.record(s)
        torch.cuda.synchronize()
        g_ms, s_ms = e0.elapsed_time(e1), e1.elapsed_time(e2)
        del table, idx, vals
        out["random_gather_G_per_s"] = round(nr / (g_ms * 1e-3) / 1e9, 2)
        out["random_scatter_G_per_s"] = round(nr / (s_ms * 1e-3) / 1e9, 2)
        out["random_rmw_G_per_s"] = round(nr / ((g_ms + s_ms) * 1e-3) / 1e9, 2)
        out["l2_atomic_ceiling_GUPS"] = round(l2_ceiling, 1)
        out["hbm_ceiling_GUPS"] = round(hbm_ceiling, 2)
        best = max(out["uniform_plain"]["GUPS"], out["uniform_agg"]["GUPS"], out["uniform_combine"]["GUPS"])
        out["uniform_frac_of_hbm_ceiling"] = round(best / hbm_ceiling, 3)
        out["uniform_frac_of_l2_atomic_ceiling"] = round(best / l2_ceiling, 3)
        out["uniform_vs_random_rmw"] = round(best / out["random_rmw_G_per_s"], 3)
        out["zipf_frac_of_l2_atomic_ceiling"] = round(out["zipf_combine"]["GUPS"] / l2_ceiling, 3)
        # ping-pong: 512 pairs, 10^4 round trips, payload sweep
        sg.get_status()
        sig_off = wpp * 8 + 8192
        pp = {}
        iters = 10000
        lat = torch.zeros(512 * iters, dtype=torch.int64, device="cuda")
        for payload in (8, 64, 512, 4096):
            parts[:, sig_off:sig_off + 8].zero_()
            torch.cuda.synchronize()
            sg.pingpong(heap.base + wpp * 8, heap.base + sig_off, payload, 512, iters, lat)
            torch.cuda.synchronize()
            rt = lat.cpu().numpy().astype(np.float64)
            half = rt / 2 / 1e3
            pp[str(payload)] = {"half_rtt_us_p50": round(float(np.percentile(half, 50)), 3),
                                "half_rtt_us_p99": round(float(np.percentile(half, 99)), 3),
                                "payload_GBps": round(512 * 2 * payload * iters / (rt.reshape(512, iters).sum(1).max() * 1e-9) / 1e9, 3)}
        code, _ = sg.get_status()
        out["pingpong_512_pairs"] = pp
        out["status"] = code
    finally:
        heap.close()
    return out


# ----------------------------------------------------------------------------- batched teams
class BatchWorkload:
    """The batched-collective workload on a 128-PE heap: 256 teams of log-uniform 2-128
    contiguous PEs, n log-uniform 256-4 Mi, 25 % int64 teams (values U[-2^20, 2^20]),
    the rest fp32 N(0,1) with room for bf16 / E4M3 codes and per-128 scales.  `lay[t]` =
    (kind, src, dst, codes, scales) symmetric offsets of team t."""

    def __init__(self, torch, sg):
        self.torch, self.sg = torch, sg
        bt = self.bt = W.gen_batch_teams()
        self.world = world = 128
        P, n = self.P, self.n = bt.size.astype(np.int64), bt.n.astype(np.int64)
        need = np.where(bt.is_int, 16 * n, 10 * n + 4 * ((n + 127) // 128) + 1024)
        order = np.argsort(-need, kind="stable")
        hw = np.zeros(world, np.int64)
        off = np.zeros(len(P), np.int64)
        for t in order:
            s0, e = bt.start[t], bt.start[t] + P[t]
            o = (int(hw[s0:e].max()) + 255) // 256 * 256
            off[t] = o
            hw[s0:e] = o + need[t]
        self.Hb = int((hw.max() + (1 << 20)) // (1 << 20) * (1 << 20))
        heap = self.heap = sg.Heap(world, self.Hb)
        self.base = heap.base
        self.teams_h = {}
        try:
            gen = torch.Generator(device="cuda")
            gen.manual_seed(W.derive_seed("batch-values") & 0x7FFFFFFF)
            lay = self.lay = []
            for t in range(len(P)):
                o = int(off[t])
                nt = int(n[t])
                if bt.is_int[t]:
                    src, dst = o, o + 8 * nt
                    for p in range(bt.start[t], bt.start[t] + P[t]):
                        v = torch.randint(-(1 << 20), (1 << 20) + 1, (nt,), dtype=torch.int64, device="cuda", generator=gen)
                        heap.view(src, p, torch.int64, nt).copy_(v)
                    lay.append(("i64", src, dst, None, None))
                else:
                    src = o
                    codes = (o + 4 * nt + 255) // 256 * 256      # 16-byte aligned codes: the wide path
                    dst = (codes + 2 * nt + 255) // 256 * 256
                    sc = (dst + 4 * nt + 255) // 256 * 256
                    for p in range(bt.start[t], bt.start[t] + P[t]):
                        heap.view(src, p, torch.float32, nt).normal_(generator=gen)
                    lay.append(("f", src, dst, codes, sc))
            torch.cuda.synchronize()
        except BaseException:
            heap.close()
            raise

    def team(self, t):
        key = (int(self.bt.start[t]), int(self.P[t]))
        if key not in self.teams_h:
            self.teams_h[key] = self.sg.team_split_strided(self.sg.TEAM_WORLD, key[0], 1, key[1])
        return self.teams_h[key]

    def descs(self, fmt):
        sg, d = self.sg, []
        for t, (k, src, dst, codes, sc) in enumerate(self.lay):
            st0, sz, nt = int(self.bt.start[t]), int(self.P[t]), int(self.n[t])
            if k == "i64":
                d.append(sg.CollDesc(st0, sz, sg.INT64, -1, nt, self.base + dst, self.base + src, None))
            elif fmt < 0:
                d.append(sg.CollDesc(st0, sz, sg.FLOAT, -1, nt, self.base + dst, self.base + src, None))
            else:
                d.append(sg.CollDesc(st0, sz, sg.FLOAT, fmt, nt, self.base + dst, self.base + codes, self.base + sc))
        return d

    def quantize(self, fmt):
        """every float team's fp32 input into its codes + scales (the library's quantiser)"""
        for t, (k, src, dst, codes, sc) in enumerate(self.lay):
            if k != "i64":
                self.sg.quantize(self.team(t), self.base + codes, self.base + sc, self.base + src, fmt, int(self.n[t]))
        self.torch.cuda.synchronize()

    def close(self):
        for tm in self.teams_h.values():
            self.sg.team_destroy(tm)
        self.teams_h = {}
        self.heap.close()


def run_batch(torch, sg, reps=5, check_teams=32, check_elems=4096):
    """256 teams of log-uniform 2-128 PEs (128-PE world), n log-uniform 256-4 Mi, 25 %
    int64; fp32 N(0,1) payloads vs bf16 / E4M3 payloads with per-128 scales.  One
    graph-captured persistent launch per format, autotuned; compared with one launch per
    team and with the untuned plan; error against binary64 on sampled elements."""
    wl = BatchWorkload(torch, sg)
    bt, P, n, lay, heap, base = wl.bt, wl.P, wl.n, wl.lay, wl.heap, wl.base
    out = {"teams": len(P), "world": wl.world, "heap_bytes_per_pe": wl.Hb}
    try:
        descs = wl.descs

        def algo_bytes(fmt):
            tot = 0
            for t, (k, *_r) in enumerate(lay):
                e_in = 8 if k == "i64" else (4 if fmt < 0 else (2 if fmt == 0 else 1))
                e_out = 8 if k == "i64" else 4
                sc = 0 if (k == "i64" or fmt < 0) else 4 / 128
                tot += P[t] * n[t] * (e_in + e_out + sc)
            return float(tot)

        s = torch.cuda.current_stream()

        def time_graph(b):
            b.launch()
            e0, e1 = _events(torch)
            e0.record(s)
            for _ in range(reps):
                b.launch()
            e1.record(s)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        hbm, src_kind = measured_peaks()
        for fmt, name in ((-1, "fp32"), (0, "bf16"), (1, "e4m3")):
            if fmt >= 0:
                wl.quantize(fmt)
            ab = algo_bytes(fmt)
            b = sg.Batch(descs(fmt), sg.Tune(16384, 0, 0, 0))
            untuned = time_graph(b)
            tune = b.autotune()
            tuned = time_graph(b)
            # one launch per team (plain path)
            for t in range(len(P)):
                wl.team(t)
            e0, e1 = _events(torch)
            e0.record(s)
            for _ in range(reps):
                for t, (k, src, dst, codes, sc) in enumerate(lay):
                    tm = wl.team(t)
                    if k == "i64":
                        sg.reduce(tm, base + dst, base + src, int(n[t]), sg.INT64, sg.SUM, s)
                    elif fmt < 0:
                        sg.reduce(tm, base + dst, base + src, int(n[t]), sg.FLOAT, sg.SUM, s)
                    else:
                        sg.qsum_reduce(tm, base + dst, base + codes, base + sc, fmt, int(n[t]), s)
            e1.record(s)
            torch.cuda.synchronize()
            per_team = e0.elapsed_time(e1) / reps
            b.launch()
            torch.cuda.synchronize()
            err = batch_errors(torch, heap, bt, lay, fmt, check_teams, check_elems)
            out[name] = {"GBps": round(ab / (tuned * 1e-3) / 1e9, 1), "ms": round(tuned, 3),
                         "frac_of_hbm": round(ab / (tuned * 1e-3) / 1e9 / hbm, 3),
                         "untuned_ms": round(untuned, 3), "launch_per_team_ms": round(per_team, 3),
                         "speedup_vs_launch_per_team": round(per_team / tuned, 2),
                         "tune": {"tile_elems": tune.tile_elems, "ctas_per_sm": tune.ctas_per_sm, "deep": tune.deep},
                         "algorithmic_bytes": ab, "error_vs_fp64": err}
            b.destroy()
    finally:
        wl.close()
    return out


def batch_errors(torch, heap, bt, lay, fmt, nteams, nel):
    """Normwise error of the float teams' outputs against binary64 sums of the original
    fp32 inputs (sampled: the first nteams float teams, first nel elements)."""
    rel_max, sq_num, sq_den, i64_ok = 0.0, 0.0, 0.0, True
    seen = 0
    for t, (k, src, dst, codes, sc) in enumerate(lay):
        m = min(int(bt.n[t]), nel)
        members = range(int(bt.start[t]), int(bt.start[t] + bt.size[t]))
        if k == "i64":
            if seen < nteams:
                x = np.stack([heap.view(src, p, torch.int64, m).cpu().numpy() for p in members])
                y = heap.view(dst, int(bt.start[t]), torch.int64, m).cpu().numpy()
                i64_ok &= bool(np.array_equal(x.sum(0), y))
            continue
        if seen >= nteams:
            continue
        seen += 1
        x = np.stack([heap.view(src, p, torch.float32, m).cpu().numpy().astype(np.float64) for p in members])
        y64 = x.sum(0)
        y = heap.view(dst, int(bt.start[t]), torch.float32, m).cpu().numpy().astype(np.float64)
        num, den = np.linalg.norm(y - y64), np.linalg.norm(y64)
        rel_max = max(rel_max, num / den if den else 0.0)
        sq_num += num * num
        sq_den += den * den
    return {"normwise_rel_max": float(f"{rel_max:.3e}"), "normwise_rel_rms": float(f"{math.sqrt(sq_num / sq_den):.3e}"),
            "int64_teams_exact": i64_ok, "sampled_float_teams": seen, "elements_per_team": nel}


# ----------------------------------------------------------------------------- serving
def serve_latency(recs, t0_host, arrivals, offset_ns):
    """Per-request latency (us) from the intended arrival (host clock) to device
    completion, through the measured clock offset."""
    done_host = recs["t_done_ns"].astype(np.int64) - offset_ns
    return (done_host - (t0_host + arrivals[recs["ticket"].astype(np.int64)].astype(np.int64))) / 1e3


SERVE_RATES = (1e6, 2e6, 5e6, 1e7, 2e7, 5e7)          # the configuration's arrival rates (req/s)
SERVE_SAT_FRACTIONS = (0.1, 0.25, 0.5, 0.75, 1.0, 1.25)  # and fractions of the measured saturation rate


def served_bytes(reqs):
    """Bytes each request moves in HBM by definition: its staged payload written, then the
    operation's reads and writes (put/get n + 2n; reduce P*n_in + P*n_in + P*4n;
    alltoall 3*P^2*m; an AMO 16)."""
    k = reqs["kind"].astype(np.int64)
    n = reqs["n"].astype(np.float64)
    P = reqs["issuer"].astype(np.float64)
    bf = (reqs["fmt"] == W.FMT_BF16) & (k == 16)
    n_in = np.where(bf, 2 * n + 4 * np.ceil(n / 128), 4 * n)
    return np.select([np.isin(k, (1, 2)), k == 16, k == 15], [3 * n, P * (2 * n_in + 4 * n), 3 * P * P * n], 16.0)


def run_serve(torch, sg, nreq=1 << 16, rates=None, npes=512, arena=32 << 20):
    """512 PEs, each with a 32 MiB page arena (16 GiB) beside its AMO table.  Mixed
    Poisson arrivals: 60 % put/get 8 B-4 MiB, 25 % int64 AMOs, 10 % fp32/bf16 team
    reductions of 64 Ki-8 Mi elements, 5 % alltoall of 4-256 KiB per pair, every non-AMO
    request staging its own payload into its admitted pages; served by the persistent
    engine and by one launch per request, same arrivals; throughput (req/s, GB/s of the
    bytes each request moves) and p50/p99 latency at 1-50 M req/s and at 0.1-1.25 x the
    saturation rate, `nreq` requests per point."""
    lay = W.serve_layout_staged(arena_bytes=arena, amo_words=8192)
    heap = sg.Heap(npes, lay.H)
    out = {"npes": npes, "arena_bytes": npes * arena, "heap_bytes": npes * lay.H, "requests_per_point": nreq,
           "payloads": "staged (fp32 reductions in place)"}
    try:
        parts = heap.partitions()
        parts[:, lay.amo_offset:lay.amo_offset + 8 * lay.amo_words].view(torch.int64).copy_(
            W.cb64_torch(W.derive_seed("serve-amo"), torch.arange(npes * lay.amo_words, device="cuda")).view(
                npes, lay.amo_words))
        torch.cuda.synchronize()
        cfg = sg.ServerCfg()
        cfg.page_bytes = lay.page_bytes
        cfg.arena_offset, cfg.arena_bytes = lay.arena_offset, lay.arena_bytes
        cfg.amo_offset, cfg.amo_words = lay.amo_offset, lay.amo_words
        cfg.max_ns = 300 * 10**9
        cfg.ring_slots = 1 << 17     # room for a whole point's requests and completions
        reqs = W.gen_serve_requests(W.derive_seed("serve-reqs"), nreq, npes, lay, red_hi=8 << 20, staged=True)
        req_bytes = served_bytes(reqs)
        out["mean_request_MB"] = round(float(req_bytes.mean()) / 1e6, 3)
        out["largest_reduce_elems"] = int(reqs["n"][reqs["kind"] == 16].max())
        out["largest_alltoall_pair_bytes"] = int(reqs["n"][reqs["kind"] == 15].max())
        mb = float(np.mean(reqs["n"][np.isin(reqs["kind"], (1, 2))])) / 1e6
        out["mix_counts"] = {k: int(v) for k, v in zip(("rma", "amo", "reduce", "alltoall"), (
            np.isin(reqs["kind"], (1, 2)).sum(), np.isin(reqs["kind"], (5, 6, 7)).sum(),
            (reqs["kind"] == 16).sum(), (reqs["kind"] == 15).sum()))}
        out["mean_rma_MB"] = round(mb, 3)
        offset, err = sg.clock_offset(50)
        out["clock_offset_err_us"] = round(err / 1e3, 2)
        sstream = torch.cuda.Stream()
        comp_buf = np.zeros(16384, sg.COMPLETION_DTYPE)

        def serve_once(arr):
            srv = sg.Server(cfg, sstream)
            t0 = srv.feed(reqs, arr)
            recs = np.zeros(nreq, sg.COMPLETION_DTYPE)
            got, tl = 0, time.time()
            while got < nreq:
                k = srv.poll(comp_buf)
                recs[got:got + k] = comp_buf[:k]
                got += k
                if k == 0:
                    if time.time() - tl > 120:
                        break
                    time.sleep(0.0002)
            srv.stop()
            return recs[:got], t0

        rec_t = torch.zeros(nreq * sg.COMPLETION_DTYPE.itemsize, dtype=torch.uint8).pin_memory()

        def plain_once(arr):
            rec_t.zero_()
            pstream = torch.cuda.Stream()
            t0 = sg.plain_feed(reqs, arr, cfg, rec_t.data_ptr(), pstream)
            pstream.synchronize()
            return np.frombuffer(rec_t.numpy().tobytes(), sg.COMPLETION_DTYPE).copy(), t0

        classes = {"rma": (1, 2), "amo": (5, 6, 7), "reduce": (16,), "alltoall": (15,)}
        hbm, _ = measured_peaks()

        def summarise(recs, t0, arr):
            ok = recs[recs["status"] == 0]
            lat = serve_latency(ok, t0, arr, offset)
            span = (int(ok["t_done_ns"].max()) - offset - t0) / 1e9
            svc = (ok["t_done_ns"].astype(np.int64) - ok["t_admit_ns"].astype(np.int64)) / 1e3
            kinds = reqs["kind"][ok["ticket"].astype(np.int64)]
            per = {}
            for cname, ks in classes.items():
                m = np.isin(kinds, ks)
                if m.any():
                    per[cname] = {"p50_us": round(float(np.percentile(lat[m], 50)), 1),
                                  "p99_us": round(float(np.percentile(lat[m], 99)), 1),
                                  "service_p50_us": round(float(np.percentile(svc[m], 50)), 1)}
            gbps = float(req_bytes[ok["ticket"].astype(np.int64)].sum()) / span / 1e9
            return {"req_per_s": round(len(ok) / span, 1), "GBps": round(gbps, 1), "frac_of_hbm": round(gbps / hbm, 3),
                    "p50_us": round(float(np.percentile(lat, 50)), 1),
                    "p99_us": round(float(np.percentile(lat, 99)), 1), "completed": int(len(ok)),
                    "errors": int((recs["status"] != 0).sum()), "per_class": per}

        # saturation rate: everything at t = 0
        zero = np.zeros(nreq, np.uint64)
        r_s, t_s = serve_once(zero)
        sat = summarise(r_s, t_s, zero)
        out["burst_server"] = sat
        r_p, t_p = plain_once(zero)
        out["burst_plain"] = summarise(r_p, t_p, zero)
        lam_sat = sat["req_per_s"]
        out["saturation_req_per_s"] = lam_sat
        pts = rates or [f * lam_sat for f in SERVE_SAT_FRACTIONS] + list(SERVE_RATES)
        out["points"] = []
        for lam in pts:
            arr = W.poisson_arrivals_ns(W.derive_seed("serve-arrivals"), nreq, lam)
            rs, ts = serve_once(arr)
            rp, tp = plain_once(arr)
            out["points"].append({"rate_req_per_s": round(lam, 1), "server": summarise(rs, ts, arr),
                                  "plain": summarise(rp, tp, arr)})
    finally:
        heap.close()
    return out


# ----------------------------------------------------------------------------- profiling cases
PROFILE_CASES = ("interp_ring", "interp_ops", "reduce", "reduce_mid", "reduce_big", "reduce_f32", "broadcast", "alltoall", "amo", "amo_l2", "amo_plain", "amo_combine", "amo_combine_zipf", "batch_bf16", "batch_e4m3", "batch_e4m3_teams", "batch_bf16_teams", "qsum", "serve_reduce", "serve_a2a",
                 "pingpong_cluster", "cluster_coll", "halo", "halo_plain")


def run_profile_case(name, launches=4):
    """Small cases of single kernels for ncu captures: inputs larger than the 129 MB L2,
    at most ~2 GB on the device, `launches` launches of the kernel of interest."""
    import torch

    import paper_2607_08006_gb300 as sg

    sg.build()
    torch.cuda.set_device(0)
    s = torch.cuda.current_stream()
    if name == "interp_ring":      # 128 PEs of one CTA each, ring put_nbi of 12 MiB, bulk engine
        # (one CTA per PE: the bench's 64 two-CTA clusters give each SM the same share,
        # and a cluster launch is profiled without its cluster shape)
        m, npes = 12 * MiB, 128
        heap = sg.Heap(npes, 2 * m, pe_mode=sg.PE_MODE_CTA, cluster_dim=1)
        ops = np.zeros(npes + 1, W.OP_DTYPE)
        for p in range(npes):
            ops[p] = (W.OP_PUT_NBI, 0, 0, 0, (p + 1) % npes, p, m, 0, m, 0, 0, 0)
        ops[npes] = (W.OP_QUIET, 0, 0, 0, 0, -1, 0, 0, 0, 0, 0, 0)
        dev = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
        for _ in range(launches):
            sg.run_script(dev, npes + 1, None, s)
    elif name == "interp_ops":     # 64 PEs of 2-CTA clusters, 640 empty put_nbi ops + quiet (per-op cost)
        npes = 64
        heap = sg.Heap(npes, 1 << 20, pe_mode=sg.PE_MODE_CLUSTER, cluster_dim=2)
        ops = np.zeros(641, W.OP_DTYPE)
        for k in range(640):
            ops[k] = (W.OP_PUT_NBI, 0, 0, 0, (k + 1) % npes, k % npes, 1 << 19, 0, 0, 0, 0, 0)
        ops[640] = (W.OP_QUIET, 0, 0, 0, 0, -1, 0, 0, 0, 0, 0, 0)
        dev = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
        for _ in range(launches):
            sg.run_script(dev, 641, None, s)
    elif name in ("reduce_mid", "reduce_big"):  # 64 PEs, int32 sum: 1 Mi elements (4 MiB per member,
        # the bulk ring k_reduce_bulk) or 8 Mi (32 MiB per member, the register form k_reduce)
        n = 1 << 20 if name == "reduce_mid" else 8 << 20
        heap = sg.Heap(64, 8 * n)
        heap.partitions().random_(0, 255)
        for _ in range(launches):
            sg.reduce(sg.TEAM_WORLD, heap.base + 4 * n, heap.base, n, sg.INT32, sg.SUM, s)
    elif name in ("reduce", "reduce_f32"):  # 64 PEs, 1 Mi elements (int64: the bulk ring)
        n = 1 << 20
        heap = sg.Heap(64, 16 * n)
        heap.partitions().random_(0, 255)
        dt = sg.INT64 if name == "reduce" else sg.FLOAT
        if dt == sg.FLOAT:
            heap.partitions()[:, :8 * n].view(torch.float32).normal_()
        for _ in range(launches):
            sg.reduce(sg.TEAM_WORLD, heap.base + 8 * n, heap.base, n, dt, sg.SUM, s)
    elif name in ("serve_reduce", "serve_a2a"):  # the serving tiles on the plain path: one staged
        # request per launch pair (staging launch, then the operation's): an fp32 reduction of
        # 4 Mi elements over 32 PEs in place, or a 32 x 256 KiB alltoall
        lay = W.serve_layout_staged(arena_bytes=32 * MiB, amo_words=1024)
        heap = sg.Heap(32, lay.H)
        cfg = sg.ServerCfg()
        cfg.page_bytes = lay.page_bytes
        cfg.arena_offset, cfg.arena_bytes = lay.arena_offset, lay.arena_bytes
        cfg.amo_offset, cfg.amo_words = lay.amo_offset, lay.amo_words
        cfg.max_ns = 60 * 10**9
        req = np.zeros(1, sg.REQ_DTYPE)
        req["flags"], req["pe"], req["issuer"], req["word"] = 1, 0, 32, 12345
        if name == "serve_reduce":
            req["kind"], req["dtype"], req["fmt"], req["n"] = W.OP_REDUCE, W.DT_FLOAT, W.FMT_F32, 4 << 20
        else:
            req["kind"], req["n"] = W.OP_ALLTOALL, 256 * KiB
        recs = torch.zeros(launches * sg.COMPLETION_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
        reqs = np.repeat(req, launches)
        sg.plain_feed(reqs, np.zeros(launches, np.uint64), cfg, recs.data_ptr(), s)
        s.synchronize()
        done = np.frombuffer(recs.numpy().tobytes(), sg.COMPLETION_DTYPE)
        assert np.all(done["status"] == 0), done["status"]
    elif name == "broadcast":      # 64 PEs, 8 MiB
        m = 8 * MiB
        heap = sg.Heap(64, 2 * m)
        for _ in range(launches):
            sg.broadcastmem(sg.TEAM_WORLD, heap.base + m, heap.base, m, 63, s)
    elif name == "alltoall":       # 64 PEs, 128 KiB per pair
        m = 128 * KiB
        heap = sg.Heap(64, 2 * 64 * m)
        for _ in range(launches):
            sg.alltoallmem(sg.TEAM_WORLD, heap.base + 64 * m, heap.base, m, s)
    elif name == "amo":            # 1024 PEs, 2^27-word table (1 GiB), 2^22 uniform ops
        wpp = 1 << 17
        heap = sg.Heap(1024, wpp * 8)
        nops = 1 << 22
        ops = torch.from_numpy(W.amo_stream_np(1, nops, 27).view(np.int32)).cuda()
        f = torch.empty(nops, dtype=torch.int64, device="cuda")
        for _ in range(launches):
            sg.amo_stream(heap.base, wpp, ops, nops, 1, 2, f, 0, s)
    elif name == "amo_l2":         # the same kernel on an L2-resident table: 2^21 words (16 MiB), 2^24 ops
        wpp = (1 << 21) // 1024
        heap = sg.Heap(1024, 1 << 17)
        nops = 1 << 24
        ops = torch.from_numpy(W.amo_stream_np(5, nops, 21).view(np.int32)).cuda()
        for _ in range(launches):
            sg.amo_stream(heap.base, wpp, ops, nops, 1, 2, None, 0, s)
    elif name in ("amo_plain", "amo_combine", "amo_combine_zipf"):  # as "amo", 2^24 ops
        wpp = 1 << 17
        heap = sg.Heap(1024, wpp * 8)
        nops = 1 << 24
        dist = "zipf" if name.endswith("zipf") else "uniform"
        ops = torch.from_numpy(W.amo_stream_np(1, nops, 27, dist=dist).view(np.int32)).cuda()
        f = torch.empty(nops, dtype=torch.int64, device="cuda")
        for _ in range(launches):
            sg.amo_stream(heap.base, wpp, ops, nops, 1, 2, f, 0 if name == "amo_plain" else 2, s)
    elif name in ("batch_e4m3_teams", "batch_bf16_teams"):  # 8 teams of all 64 PEs, 1 Mi elements each, tile 8192
        n, nt = 1 << 20, 8
        per = 8 * n  # codes (<= 2n) + scales + output (4n), rounded up
        heap = sg.Heap(64, nt * per)
        fmt = sg.FMT_E4M3 if name == "batch_e4m3_teams" else sg.FMT_BF16
        d = []
        for t in range(nt):
            o = t * per
            heap.partitions()[:, o:o + 4 * n].view(torch.float32).normal_()
            sg.quantize(sg.TEAM_WORLD, heap.base + o + 4 * n, heap.base + o + 6 * n, heap.base + o, fmt, n, s)
            d.append(sg.CollDesc(0, 64, sg.FLOAT, fmt, n, heap.base + o, heap.base + o + 4 * n, heap.base + o + 6 * n))
        b = sg.Batch(d, sg.Tune(8192, 0, 0, 0))
        for _ in range(launches):
            b.launch(s)
        torch.cuda.synchronize()
        b.destroy()
    elif name in ("batch_bf16", "batch_e4m3", "qsum"):   # 64 PEs, bf16 / E4M3 payloads of 1 Mi elements
        n = 1 << 20
        heap = sg.Heap(64, 12 * n)
        x = heap.partitions()[:, :4 * n].view(torch.float32)
        x.normal_()
        fmt = sg.FMT_E4M3 if name == "batch_e4m3" else sg.FMT_BF16
        sg.quantize(sg.TEAM_WORLD, heap.base + 4 * n, heap.base + 6 * n, heap.base, fmt, n, s)
        if name == "qsum":
            for _ in range(launches):
                sg.qsum_reduce(sg.TEAM_WORLD, heap.base + 7 * n, heap.base + 4 * n, heap.base + 6 * n, sg.FMT_BF16, n, s)
        else:
            d = [sg.CollDesc(0, 64, sg.FLOAT, fmt, n, heap.base + 7 * n, heap.base + 4 * n, heap.base + 6 * n)]
            b = sg.Batch(d, sg.Tune(8192, 0, 0, 0))
            for _ in range(launches):
                b.launch(s)
            torch.cuda.synchronize()
            b.destroy()
    elif name == "pingpong_cluster":  # 64 pairs, each inside one 2-CTA cluster, 4 KiB, 2000 round trips
        heap = sg.Heap(128, 16384, pe_mode=sg.PE_MODE_CTA, cluster_dim=2)
        heap.partitions().zero_()
        for _ in range(launches):
            sg.pingpong_cluster(heap.base, heap.base + 12288, 4096, 64, 2000, None, s)
    elif name == "cluster_coll":      # 8 clusters of 8 CTA PEs: shared-team reduce 64 KiB + fcollect 4 KiB
        heap = sg.Heap(64, 1 << 20, pe_mode=sg.PE_MODE_CTA, cluster_dim=8)
        heap.partitions().random_(0, 255)
        ops = np.zeros(200, W.OP_DTYPE)
        for k in range(100):
            ops[2 * k] = (W.OP_REDUCE, W.DT_INT64, W.RED_SUM, 1, 0, -1, 512 * KiB, 0, 8192, 0, 0, 0)
            ops[2 * k + 1] = (W.OP_FCOLLECT, 0, 0, 1, 0, -1, 768 * KiB, 65536, 4096, 0, 0, 0)
        dev = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
        for _ in range(launches):
            sg.run_script(dev, len(ops), None, s)
    elif name in ("halo", "halo_plain"):  # 8 x 8 PEs of 1024 x 1024 binary32 (256 MiB per buffer), 4 sweeps
        px, py, nx, ny = 8, 8, 1024, 1024
        tile_b, halo_b = 2 * nx * ny * 4, 2 * sg.halo_stride(nx, ny) * 4
        heap = sg.Heap(px * py, (tile_b + halo_b + 64 + 4095) // 4096 * 4096)
        heap.partitions().zero_()
        heap.partitions()[:, :nx * ny * 4].view(torch.float32).normal_()
        for _ in range(launches):
            sg.halo_jacobi(heap.sym(0, tile_b), heap.sym(tile_b, halo_b), heap.sym(tile_b + halo_b, 32), px, py, nx,
                           ny, 4, s, plain=name == "halo_plain")
    else:
        raise SystemExit(f"unknown profile case {name}")
    torch.cuda.synchronize()
    code, detail = sg.get_status()
    heap.close()
    if code != 0:
        raise SystemExit(f"device status {code} detail {detail}")
    print(json.dumps({"profile_case": name, "launches": launches, "status": "ok"}))


# ----------------------------------------------------------------------------- distributed
def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- output
HEADLINE_MAX = 1400  # bytes of the last stdout line
ROOFLINE_KEYS = ("bound", "achieved", "peak", "unit", "frac", "traffic", "kernel", "share_of_step", "avg_launch_ms",
                 "peak_source")


def _get(d, *path):
    for k in path:
        if not isinstance(d, dict) or k not in d:
            return None
        d = d[k]
    return d


def leg_summary(name, r):
    """A few numbers per secondary leg for the headline (the leg's own line has the rest)."""
    if name == "script":
        return {"dev_ops_s": _get(r, "device", "ops_per_s"), "plain_ops_s": _get(r, "host", "ops_per_s"),
                "ok": bool(_get(r, "device", "heap_matches_oracle") and _get(r, "host", "heap_matches_oracle"))}
    if name == "amo":
        uni = [_get(r, "uniform_" + k, "GUPS") for k in ("plain", "agg", "combine")]
        uni = [u for u in uni if u is not None]
        return {"uni_GUPS": max(uni) if uni else None, "zipf_GUPS": _get(r, "zipf_combine", "GUPS"),
                "zipf_plain_GUPS": _get(r, "zipf_plain", "GUPS"), "uni_frac": r.get("uniform_frac_of_hbm_ceiling"),
                "pp8_us": _get(r, "pingpong_512_pairs", "8", "half_rtt_us_p50")}
    if name == "cluster":
        return {"pp8_us": [_get(r, "pingpong_512_pairs", "8", m, "half_rtt_us_p50") for m in ("dsmem", "l2")]}
    if name == "ctx":
        return {"overlap_ms": r.get("overlap_saving_ms"), "ctx1_GBps": r.get("ctx1_GBps"),
                "blocking_GBps": r.get("blocking_GBps")}
    if name == "halo":
        return {"GBps": _get(r, "cta", "persistent", "GBps"), "frac": r.get("frac_of_hbm"),
                "x_plain": _get(r, "cta", "speedup_vs_plain"), "x_plain_256": _get(r, "small_tiles_256", "speedup_vs_plain")}
    if name == "batch":
        return {f: _get(r, f, "GBps") for f in ("fp32", "bf16", "e4m3")}
    if name == "serve":
        pts = r.get("points") or []
        lo = pts[0] if pts else {}
        return {"req_s": [_get(r, "burst_server", "req_per_s"), _get(r, "burst_plain", "req_per_s")],
                "GBps": _get(r, "burst_server", "GBps"), "frac": _get(r, "burst_server", "frac_of_hbm"),
                "low_p50_us": [_get(lo, "server", "p50_us"), _get(lo, "plain", "p50_us")],
                "low_p99_us": [_get(lo, "server", "p99_us"), _get(lo, "plain", "p99_us")],
                "p99_lower": "%d/%d" % (sum(1 for q in pts if (_get(q, "server", "p99_us") or 0) <
                                            (_get(q, "plain", "p99_us") or 0)), len(pts))}
    return {}


def headline_numbers(summary):
    """A handful of numbers from the secondary legs, flat, for the headline."""
    g = _get
    return {k: v for k, v in {
        "amo_uni_GUPS": g(summary, "amo", "uni_GUPS"), "amo_zipf_GUPS": g(summary, "amo", "zipf_GUPS"),
        "batch_e4m3_GBps": g(summary, "batch", "e4m3"), "halo_GBps": g(summary, "halo", "GBps"),
        "serve_req_s": (g(summary, "serve", "req_s") or [None])[0], "serve_GBps": g(summary, "serve", "GBps")}.items()
        if v is not None}


def compose_headline(out, legs):
    """The headline: the metric, roofline, clocks, e2e, the CPU baseline and a few numbers
    per secondary leg -- short enough to be one line that a log tail keeps whole."""
    keys = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "config", "gpu_launches", "clocks", "e2e", "cpu_baseline",
            "gpu_on_cpu_sample")
    h = {k: out[k] for k in keys if k in out}
    h["roofline"] = {k: out["roofline"][k] for k in ROOFLINE_KEYS if k in out.get("roofline", {})}
    if "e2e" in h:
        h["e2e"] = {k: v for k, v in h["e2e"].items() if k in ("value", "unit", "h2d_bytes_per_step",
                                                                "d2h_bytes_per_step", "ms_per_step")}
    if "cpu_baseline" in h:
        h["cpu_baseline"] = {k: v for k, v in h["cpu_baseline"].items() if k != "seconds"}
    if legs:
        h["secondary"] = headline_numbers({n: leg_summary(n, r) for n, r in legs.items()})
    while h.get("secondary") and len(headline_line(h)) > HEADLINE_MAX:
        h["secondary"].popitem()
    for drop in (("secondary",), ("gpu_on_cpu_sample",), ("config", "l2"), ("roofline", "peak_source")):
        if len(headline_line(h)) <= HEADLINE_MAX:
            break
        d = h
        for k in drop[:-1]:
            d = d.get(k, {})
        d.pop(drop[-1], None)
    return h


def headline_line(h):
    return json.dumps(h, separators=(",", ":"))


LEGS = ("script", "amo", "cluster", "ctx", "halo", "batch", "serve")


def run_leg(name, args, torch, sg):
    if name == "script":
        return run_script_leg(torch, sg)
    if name == "amo":
        return run_amo(torch, sg, args.amo_ops_log2)
    if name == "cluster":
        return run_cluster_leg(torch, sg)
    if name == "halo":
        return run_halo(torch, sg)
    if name == "ctx":
        return run_ctx_leg(torch, sg)
    if name == "batch":
        return run_batch(torch, sg)
    if name == "serve":
        return run_serve(torch, sg, args.serve_requests)
    raise SystemExit(f"unknown secondary leg {name}")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="shmemg", choices=["shmemg", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--secondary", default=",".join(LEGS),
                    help="extra workloads measured after the sweep (comma list of %s, or 'none'); each prints "
                         "its own JSON line before the headline" % ",".join(LEGS))
    ap.add_argument("--amo-ops-log2", type=int, default=30)
    ap.add_argument("--serve-requests", type=int, default=1 << 16)
    ap.add_argument("--profile", choices=PROFILE_CASES, help="run one small single-kernel case (for ncu) and exit")
    args = ap.parse_args(argv)
    if args.profile:
        run_profile_case(args.profile)
        return
    rank, world = dist_init()
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)), flush=True)
        return
    out = run_gpu(args, rank, world)
    if rank != 0:
        return
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline()
    # detail lines first, the headline last
    print(json.dumps({"leg": "sweep", "per_family": out.get("per_family"), "roofline": out.get("roofline"),
                      "e2e": out.get("e2e"), "points": out.get("points")}), flush=True)
    legs = {}
    sec = [s for s in args.secondary.split(",") if s and s != "none"]
    if sec:
        import torch

        import paper_2607_08006_gb300 as sg

        for name in sec:
            t0 = time.perf_counter()
            r = run_leg(name, args, torch, sg)
            r["wall_s"] = round(time.perf_counter() - t0, 1)
            legs[name] = r
            print(json.dumps({"leg": name, **r}), flush=True)
    if legs:
        print(json.dumps({"leg": "summary", **{n: leg_summary(n, r) for n, r in legs.items()}}), flush=True)
    print(headline_line(compose_headline(out, legs)), flush=True)


if __name__ == "__main__":
    main()

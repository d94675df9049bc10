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
exchanged between GPUs); rank 0 prints one JSON line.
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
H = 512 * MiB               # grown from 64 MiB to hold the largest sweep points (256 MiB src + dst)
A_OFF, B_OFF = 0, 256 * MiB  # sources live in region A, destinations in region B
I32_OFF = 128 * MiB          # int32 sources: A[128 MiB, 192 MiB); int64 sources: A[0, 128 MiB)
METRIC = "collective & bulk-RMA GB/s vs HBM peak; AMO GUPS; served p50/p99 op latency"
WORKLOAD = ("collective and RMA bandwidth sweep: 64 virtual PEs x 512 MiB (64 MiB grown to the largest "
            "point's footprint); int32/int64 sum+max reduce and fcollect 1Ki-16Mi elements; alltoall "
            "4KiB-1MiB per pair; broadcast 1KiB-256MiB; put_nbi/get_nbi ring + quiet 8B-256MiB")


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


def ring_script(kind, m):
    ops = np.zeros(NPES + 1, W.OP_DTYPE)
    for p in range(NPES):
        q = (p + 1) % NPES
        if kind == "put":   # PE p: its A -> PE q's B
            ops[p] = (W.OP_PUT_NBI, 0, 0, 0, q, p, B_OFF, A_OFF, m, 0, 0, 0)
        else:               # PE p: PE q's A -> its own B
            ops[p] = (W.OP_GET_NBI, 0, 0, 0, q, p, B_OFF, A_OFF, m, 0, 0, 0)
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
                self.scripts[(fam, m)] = torch.from_numpy(ring_script(fam, m).view(np.uint8).copy()).cuda()
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

    def run_point(self, name, fam, m):
        sg, s = self.sg, self.stream
        if fam == "reduce":
            _, dt, op = name.split("_")
            dtype = sg.INT32 if dt == "int32" else sg.INT64
            src = self.A32 if dt == "int32" else self.A
            sg.reduce(sg.TEAM_WORLD, self.B, src, m, dtype, sg.SUM if op == "sum" else sg.MAX, s)
        elif fam == "fcollect":
            es = 4 if name.endswith("int32") else 8
            src = self.A32 if es == 4 else self.A
            sg.fcollectmem(sg.TEAM_WORLD, self.B, src, m * es, s)
        elif fam == "alltoall":
            sg.alltoallmem(sg.TEAM_WORLD, self.B, self.A, m, s)
        elif fam == "broadcast":
            sg.broadcastmem(sg.TEAM_WORLD, self.B, self.A, m, NPES - 1, s)
        else:
            sg.run_script(self.scripts[(fam, m)], NPES + 1, None, s)

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
        "dtype": "int32/int64 (integer reduce, byte movement)",
        "data": "synthetic: seeded splitmix64 values U[-2^20, 2^20]",
        "config": {"workload": WORKLOAD, "npes": NPES, "heap_bytes_per_pe": H, "pe_mode": "cluster(2 CTAs)",
                   "points_per_step": len(pts), "algorithmic_bytes_per_step": bytes_step,
                   "l2": "no flush: each step moves ~%d GiB, far above the 129 MB L2; the big points' inputs "
                         "exceed L2" % (bytes_step // GiB),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": rl,
        "gpu_launches": g.launches_per_step() * args.steps,
        "clocks": clk,
        "e2e": e2e,
        "per_family": summary["families"],
        "largest_points": summary["largest"],
    }
    return out


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
            traffic = t.get("dram_bytes_per_launch")
    total_ms = sum(v["ms"] for v in per_k.values())
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "traffic": traffic, "kernel": name,
            "families": d["families"], "share_of_step": round(d["ms"] / total_ms, 3),
            "peak_source": f"{src}: MEASURED_PEAKS.json hbm_gbs" if src == "measured" else "fallback 6.8 TB/s",
            "launches_per_step": d["launches"], "algorithmic_bytes_per_step": d["bytes"],
            "avg_launch_ms": round(d["ms"] / d["launches"], 4),
            "per_kernel": {k: {"ms_per_step": round(v["ms"], 3), "GBps": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1),
                               "share": round(v["ms"] / total_ms, 3)} for k, v in per_k.items()}}


def run_e2e(torch, sg, g, stream, args, world):
    """Same step through the public API with the inputs on the HOST: every step copies
    region A of every PE from pinned host memory, runs the sweep, and reads PE 0's
    destination region B back."""
    steps = max(1, min(args.steps, 2))
    parts = g.heap.partitions()
    host_in = torch.empty((NPES, 256 * MiB), dtype=torch.uint8, pin_memory=True)
    for p in range(NPES):
        host_in[p].copy_(parts[p, A_OFF:A_OFF + 256 * MiB])
    host_out = torch.empty(256 * MiB, dtype=torch.uint8, pin_memory=True)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(steps):
        for p in range(NPES):
            parts[p, A_OFF:A_OFF + 256 * MiB].copy_(host_in[p], non_blocking=True)
        g.step()
        host_out.copy_(parts[0, B_OFF:B_OFF + 256 * MiB], non_blocking=True)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(t0.elapsed_time(t1), world) / steps
    bytes_step = sum(b for *_, b in g.pts)
    return {"value": round(world * bytes_step / (ms * 1e-3) / 1e9, 1), "unit": "GB/s",
            "h2d_bytes_per_step": NPES * 256 * MiB, "d2h_bytes_per_step": 256 * MiB,
            "ms_per_step": round(ms, 3), "steps": steps}


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
            "sample": f"{len(pts)} sweep points with <= {CPU_MAX_ELEMS} reduce / fcollect elements and <= "
                      f"{CPU_MAX_BYTES // KiB} KiB messages, 64 PEs, {n} passes, {secs:.1f} s, single thread",
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
    sample = (f"{len(pts)} sweep points with <= {CPU_MAX_ELEMS} reduce/fcollect elements and <= "
              f"{CPU_MAX_BYTES // KiB} KiB messages per step, 64 PEs, single-threaded oracle")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32/int64",
            "data": "synthetic", "config": {"workload": WORKLOAD + " (bounded CPU sample)", "npes": NPES},
            "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="shmemg", choices=["shmemg", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    rank, world = dist_init()
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)), flush=True)
        return
    out = run_gpu(args, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            out["cpu_baseline"] = cpu_baseline()
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()

"""bench.py's output contract, on the CPU: the headline is the LAST stdout line, one JSON
object under 2 KB with the keys a reader of a log tail needs; every secondary leg's
full record comes earlier on its own line.  The GPU parts are replaced by records of
the same shape and size as a real run's (the serving leg's per-point, per-class tables
included)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

REQUIRED = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "config", "roofline", "gpu_launches", "clocks", "e2e", "cpu_baseline")


def _fake_gpu(args, rank, world):
    pts = bench.sweep_points()
    fams = {f: {"ms": 1.0, "bytes": 10**10, "launches": 8, "GBps": 6000.0} for f in
            ("reduce", "fcollect", "alltoall", "broadcast", "put", "get")}
    largest = {nm: {"size": m, "ms": 1.0, "GBps": 6000.0} for nm, f, m, b in pts}
    rl = {"bound": "hbm", "achieved": 6483.0, "peak": 6784.5, "unit": "GB/s", "frac": 0.9556, "traffic": 4.03e9,
          "kernel": "k_interp", "families": ["put", "get"], "share_of_step": 0.47,
          "peak_source": "measured hbm_gbs", "launches_per_step": 28,
          "algorithmic_bytes_per_step": 114 * 10**9, "avg_launch_ms": 0.63,
          "per_kernel": {k: {"ms_per_step": 10.0, "GBps": 6000.0, "share": 0.3} for k in ("k_interp", "k_reduce", "k_xfer")}}
    return {"metric": bench.METRIC, "value": 6244.0, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 37.7, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32/int64", "data": "synthetic, seeded",
            "config": bench.headline_config(world),
            "roofline": rl, "gpu_launches": len(pts) * args.steps,
            "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 12},
            "e2e": {"value": 2414.0, "unit": "GB/s", "h2d_bytes_per_step": 64 << 28, "d2h_bytes_per_step": 1 << 28,
                    "ms_per_step": 98.0, "steps": 2, "pipeline": "32 MiB chunks"},
            "gpu_on_cpu_sample": {"value": 1500.0, "unit": "GB/s"},
            "per_family": fams, "largest_points": largest}


def _fake_leg(name, args, torch, sg):
    cls = {c: {"p50_us": 389469.8, "p99_us": 767124.3, "service_p50_us": 3.3} for c in ("rma", "amo", "reduce", "alltoall")}
    one = {"req_per_s": 246363.2, "p50_us": 129995.7, "p99_us": 256954.9, "completed": 65536, "errors": 0,
           "per_class": cls, "GBps": 5000.0, "frac_of_hbm": 0.74}
    if name == "serve":
        return {"burst_server": one, "burst_plain": one, "saturation_req_per_s": 246363.2,
                "points": [{"rate_req_per_s": 1e6, "server": one, "plain": one} for _ in range(12)]}
    if name == "amo":
        d = {f"{a}_{b}": {"GUPS": 25.0, "ms": 40.0} for a in ("uniform", "zipf") for b in ("plain", "agg", "combine")}
        d["pingpong_512_pairs"] = {str(p): {"half_rtt_us_p50": 1.9, "half_rtt_us_p99": 2.5, "payload_GBps": 1.0}
                                   for p in (8, 64, 512, 4096)}
        d["uniform_frac_of_hbm_ceiling"] = 0.28
        return d
    if name == "batch":
        return {f: {"GBps": 6000.0, "error_vs_fp64": {"normwise_rel_max": 1e-3}} for f in ("fp32", "bf16", "e4m3")}
    return {"status": 0, "filler": "x" * 3000}


def _run_main(monkeypatch, capsys, argv):
    monkeypatch.setattr(bench, "run_gpu", _fake_gpu)
    monkeypatch.setattr(bench, "cpu_baseline", lambda reps=None: {
        "value": 7.9, "unit": "GB/s", "cores": 1, "kind": "oracle",
        "sample": "57 small sweep points (<= 256 Ki elts, <= 1 MiB msgs), 40 passes, 12.0 s",
        "seconds": 12.0})
    monkeypatch.setattr(bench, "run_leg", _fake_leg)
    monkeypatch.setattr(bench, "dist_init", lambda: (0, 1))
    bench.main(argv)
    return capsys.readouterr().out.strip().splitlines()


def test_headline_is_a_short_last_line(monkeypatch, capsys):
    lines = _run_main(monkeypatch, capsys, ["--steps", "2", "--warmup", "3"])
    last = lines[-1]
    assert len(last) <= bench.HEADLINE_MAX < 1500, len(last)
    h = json.loads(last)
    for k in REQUIRED:
        assert k in h, k
    assert h["value"] > 0 and h["unit"] == "GB/s" and h["steps"] == 2 and h["warmup"] == 3
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in h["roofline"], k
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in h["e2e"], k
    assert h["cpu_baseline"]["kind"] == "oracle" and h["cpu_baseline"]["cores"] == 1
    assert "sm_mhz" in h["clocks"] and "reasons" in h["clocks"]
    assert "workload" in h["config"]
    assert h["secondary"]["amo_uni_GUPS"] > 0 and h["secondary"]["serve_req_s"] > 0
    # every leg printed its own full record before the headline
    legs = {json.loads(x)["leg"]: json.loads(x) for x in lines[:-1]}
    assert set(legs) == {"sweep", "summary", *bench.LEGS}
    assert len(legs["serve"]["points"]) == 12


def test_headline_without_legs(monkeypatch, capsys):
    lines = _run_main(monkeypatch, capsys, ["--secondary", "none", "--steps", "1"])
    h = json.loads(lines[-1])
    assert len(lines[-1]) < 2048 and "secondary_summary" not in h and h["value"] > 0


def test_reference_arm_names_the_same_config():
    """Both arms name the same workload (the ratio divides like by like); the oracle's
    sample is stated in its cpu_baseline."""
    assert bench.headline_config(1) == bench.headline_config(1)
    pts = bench.cpu_sample_points()
    assert 0 < len(pts) < len(bench.sweep_points())

#!/usr/bin/env python3
"""Throughput of the phase-field lattice Boltzmann step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: the single-case throughput grid, 2048 x 2048 periodic D2Q9, a
spinodal-like mixture (0.5 +- 0.01 seeded noise, interfaces everywhere) at
density ratio 1000, FP32 populations.  One step = one lattice time step of
both distributions over the whole grid (one launch of the fused step kernel).
Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank advances its
own independent lattice (replicas; the method has no exchange between cases).

The line also carries `batched`: 64 independent drop and impact cases of
uneven sizes, Reynolds numbers and density ratios, advanced by the batched
kernel with FP16-shifted storage, against the same cases run one by one on
the plain FP32 single-case path; and `single_case_storage`: the 2048 x 2048
workload with 16-bit storage.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1710_09541_gb300 import cases  # noqa: E402

METRIC = "MLUPS (both distributions) and fraction of HBM roofline; batched vs plain FP32"
UNIT = "MLUPS"
# algorithmic DRAM bytes per lattice update, FP32 storage: read 9 f + 9 g (72 B),
# write 9 f + 9 g (72 B), read and write (phi u) of the previous step (16 B)
BYTES_PER_LU = 160
BYTES_PER_LU_POPULATIONS = 144


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


KERNEL_SOURCES = ["paper_1710_09541_gb300/csrc/lbm_pf.cu", "paper_1710_09541_gb300/csrc/lbm_kernels.cuh",
                  "paper_1710_09541_gb300/csrc/lbm_store.cuh",
                  "include/lbm_pf.h"]
PROFILE = "profiles/k_step_fp32_perf2048.md"


def _source_hash():
    import hashlib

    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_traffic():
    """DRAM bytes (read + write) per launch of the FP32 step kernel from the
    committed ncu summary, or None when the kernel sources have changed since
    that capture (the summary records their hash)."""
    import re

    try:
        text = open(os.path.join(ROOT, PROFILE)).read()
    except OSError:
        return None
    m = re.search(r"kernel source hash: ([0-9a-f]{16})", text)
    t = re.search(r"\| traffic \(read \+ write\) \| ([0-9.]+) MB per launch", text)
    if not m or not t or m.group(1) != _source_hash():
        return None
    return float(t.group(1)) * 1e6


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        import tempfile

        self.dev = device_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"lbm_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return None
        rows = []
        try:
            with open(self.path) as fh:
                lines = fh.readlines()
        except OSError:
            return None
        try:
            os.remove(self.path)
        except OSError:
            pass
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) != 7:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), float(parts[2]), parts[3:]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        sm = [r[0] for r in rows]
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


def _oracle_rate(nx, ny, params, phi0, budget_s, max_steps=None):
    """MLUPS of the FP64 oracle on this host: one warm-up step, then as many
    steps as fit in budget_s (at least one)."""
    import oracle

    lat = oracle.Lattice(nx, ny, **params).init(phi0)
    t0 = time.perf_counter()
    lat.step(1)
    t1 = time.perf_counter()
    per = t1 - t0
    n = max(1, int(budget_s / max(per, 1e-9)))
    if max_steps:
        n = min(n, max_steps)
    t0 = time.perf_counter()
    lat.step(n)
    dt = time.perf_counter() - t0
    return nx * ny * n / dt / 1e6, n, dt


def _cores():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def _cpu_model():
    """The host CPU as /proc/cpuinfo names it ("model name" on x86; the
    implementer and part codes on Arm), with the machine type."""
    import platform

    model = None
    try:
        info = {}
        with open("/proc/cpuinfo", errors="replace") as fh:
            for line in fh:
                k, _, v = line.partition(":")
                info.setdefault(k.strip(), v.strip())
        model = info.get("model name") or (
            f"implementer {info['CPU implementer']} part {info['CPU part']}"
            if "CPU implementer" in info and "CPU part" in info else None)
    except Exception:  # the figure is informative only; never fail the run for it
        model = None
    return f"{platform.machine()}: {model}" if model else platform.machine()


def run_reference(args):
    """The oracle (plain FP64 C, OpenMP over rows) on the host cores, timed on
    a periodic strip of the same workload sized so the whole run stays within
    a few minutes."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle

    cores = oracle.set_threads(_cores())
    nx = cases.PERF_NX
    phi_full, params = cases.perf_case()
    total = args.steps + args.warmup
    # size the strip from one probe step so (W + K) steps take about
    # --reference-seconds (90 s by default)
    probe_rows = 64
    rate, _, _ = _oracle_rate(nx, probe_rows, params, phi_full[:probe_rows], 1.0, max_steps=20)
    rows = int(args.reference_seconds * rate * 1e6 / max(total, 1) / nx)
    rows = int(min(max(rows, 4), cases.PERF_NY))

    lat = oracle.Lattice(nx, rows, **params).init(phi_full[:rows])
    lat.step(args.warmup)
    t0 = time.perf_counter()
    lat.step(args.steps)
    dt = time.perf_counter() - t0
    value = nx * rows * args.steps / dt / 1e6
    sample = f"periodic {nx}x{rows} strip of the {nx}x{cases.PERF_NY} workload, {args.steps} timed steps"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / max(args.steps, 1) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "perf-2048: spinodal-like 2048x2048 periodic D2Q9, density ratio 1000",
                   "nx": nx, "ny": cases.PERF_NY, "sample_rows": rows},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample, "cpu": _cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank timings over all ranks (every rank gets
    it); dist is torch.distributed or None for a single process."""
    import torch

    t = torch.tensor(values, dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_mlups(nodes_per_rank, steps, world, seconds):
    """Aggregate MLUPS of N replicas, each advancing nodes_per_rank nodes by
    `steps` steps, timed by the slowest rank (weak scaling)."""
    return world * nodes_per_rank * steps / seconds / 1e6


STORAGE_NAMES = {0: "fp32", 1: "fp16_shifted", 2: "bf16_shifted", 3: "bf16_shifted_sr"}
# FP16/BF16 shifted storage: f_0 FP32 (4 B) + f_1..8 and g_0..8 16-bit (34 B)
# per set, read and written, plus (phi u): 2 * 38 + 16.  The algorithmic
# minimum of a 16-bit format stores f_0 in 16 bits too: 2 * 36 + 16 = 88 B.
BYTES_PER_LU_SHIFTED16 = 92
BYTES_PER_LU_16_MIN = 88


def _time_steps(torch, stream, fn):
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    fn()
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / 1e3


def run_batched(torch, lbm, stream, steps, storage=1):
    """The batched sweep: 64 independent drops and impacts of uneven sizes and
    parameters, each advanced `steps` steps (a) one case after another on the
    plain FP32 single-case path and (b) all together by the batched kernel with
    the given storage; aggregate MLUPS of both, with the mass-conservation and
    spurious-velocity figures of each run."""
    specs = cases.batch_cases()
    nodes = sum(sp["nx"] * sp["ny"] for sp in specs)

    def make(st):
        return [lbm.Lattice(sp["nx"], sp["ny"], stream=stream, storage=st, **sp["params"])
                .init(sp["phi0"], sp["ux0"], sp["uy0"]) for sp in specs]

    def accuracy(lats):
        drift, umax = [], []
        for sp, lat in zip(specs, lats):
            d = lat.diag()
            drift.append(abs(d[0] / sp["phi0"].sum() - 1.0))
            umax.append(d[1])
        return drift, umax

    seq = make(0)
    for lat in seq:
        lat.step(5)
    t_seq = _time_steps(torch, stream, lambda: [lat.step(steps) for lat in seq])
    d_seq, u_seq = accuracy(seq)
    for lat in seq:
        lat.close()
    bat = make(storage)
    b = lbm.Batch(bat)
    b.step(150)                                   # tile-shape tuning (140 steps) + warm-up
    t_bat = _time_steps(torch, stream, lambda: b.step(steps))
    info = b.info()
    d_bat, u_bat = accuracy(bat)
    b.close()
    for lat in bat:
        lat.close()
    # the same batch with FP32 storage: batching alone, at the plain path's precision
    bat32 = make(0)
    b32 = lbm.Batch(bat32)
    b32.step(150)
    t_b32 = _time_steps(torch, stream, lambda: b32.step(steps))
    b32.close()
    for lat in bat32:
        lat.close()
    drops = [k for k, sp in enumerate(specs) if sp["kind"] == "static_drop"]
    v_bat = nodes * steps / t_bat / 1e6
    v_seq = nodes * steps / t_seq / 1e6
    peak, _ = _peaks()
    bpl = BYTES_PER_LU if storage == 0 else BYTES_PER_LU_SHIFTED16
    return {
        "cases": len(specs), "nodes": nodes, "steps_per_case": steps + 5,
        "storage": STORAGE_NAMES[storage], "value": v_bat, "unit": UNIT,
        "sequential_fp32": v_seq, "speedup_vs_sequential_fp32": v_bat / v_seq,
        "batched_fp32": nodes * steps / t_b32 / 1e6,
        "tile": {k: list(info[k]["tile"]) for k in ("periodic", "walls")},
        "tuned_us_per_step": {k: info[k]["us"] for k in ("periodic", "walls")},
        "bytes_per_lu": bpl,
        "roofline_frac": v_bat * 1e6 * bpl / 1e9 / peak,
        "roofline_frac_88": (v_bat * 1e6 * BYTES_PER_LU_16_MIN / 1e9 / peak) if storage else None,
        "sum_phi_rel_drift_max": {"batched": max(d_bat), "sequential_fp32": max(d_seq)},
        "drop_umax_max": {"batched": max(u_bat[k] for k in drops),
                          "sequential_fp32": max(u_seq[k] for k in drops)},
        "launches_per_step": 2,
    }


def run_storage_variants(torch, lbm, stream, steps):
    """Single-case MLUPS of the 2048 x 2048 workload with 16-bit storage
    (FP16, BF16, and BF16 with stochastically rounded g codes)."""
    nx, ny = cases.PERF_NX, cases.PERF_NY
    phi0, params = cases.perf_case()
    out = {}
    for st in (1, 2, 3):
        lat = lbm.Lattice(nx, ny, stream=stream, storage=st, **params).init(phi0)
        lat.step(50)
        t = _time_steps(torch, stream, lambda: lat.step(steps))
        lat.close()
        v = nx * ny * steps / t / 1e6
        peak, _ = _peaks()
        out[STORAGE_NAMES[st]] = {"value": v, "unit": UNIT,
                                  "bytes_per_lu": BYTES_PER_LU_SHIFTED16, "steps": steps,
                                  "roofline_frac": v * 1e6 * BYTES_PER_LU_SHIFTED16 / 1e9 / peak,
                                  "roofline_frac_88": v * 1e6 * BYTES_PER_LU_16_MIN / 1e9 / peak}
    return out


def run_data_variants(torch, lbm, stream, steps):
    """The same FP32 step on other data and options:
    - perf-2048-drop: one static drop of R = 512 (mostly bulk) against the
      spinodal-like headline (interfaces everywhere);
    - perf-2048-eq29: the headline workload with the local normal of Eq. 29;
    - impact-2400x600-open-top: the droplet impact (D = 200, Re = 100) with a
      wall below and the open top (zero-gradient outflow)."""
    out = {}
    nx, ny = cases.PERF_NX, cases.PERF_NY
    phi_drop, p_drop = cases.perf_drop_case()
    phi_perf, p_perf = cases.perf_case()
    p_imp = dict(cases.params_impact(Re=100.0), bc_y=2)
    phi_imp, ux_imp, uy_imp = cases.impact(2400, 600, 200.0, 20.0, 0.04, p_imp["W"])
    runs = [("perf-2048-drop", nx, ny, p_drop, (phi_drop,), "static drop R = 512, W = 4, ratio 1000"),
            ("perf-2048-eq29", nx, ny, dict(p_perf, normal_scheme=1), (phi_perf,),
             "perf-2048 with the Eq. 29 normal"),
            ("impact-2400x600-open-top", 2400, 600, p_imp, (phi_imp, ux_imp, uy_imp),
             "droplet impact D = 200, Re = 100, ratio 1000, wall below, open top")]
    for name, gx, gy, params, init, what in runs:
        lat = lbm.Lattice(gx, gy, stream=stream, **params).init(*init)
        lat.step(50)
        t = _time_steps(torch, stream, lambda: lat.step(steps))
        out[name] = {"value": gx * gy * steps / t / 1e6, "unit": UNIT, "steps": steps,
                     "workload": what + ", FP32 storage"}
        if name.startswith("impact"):
            out["impact_tooling_us"] = _tooling_us(lat, gx, gy)
        lat.close()
    return out


def _tooling_us(lat, nx, ny, reps=20):
    """Host wall time per call (microseconds, the call returns its result to
    the host) of the impact tooling on an nx x ny lattice: the spreading
    radius of one row, a Laplace jump over the grid, and a probe of 1000
    nodes."""
    xs = np.arange(1000) % nx
    ys = (np.arange(1000) * 7) % ny
    calls = {"spreading_radius": lambda: lat.spreading_radius(25),
             "laplace_jump": lambda: lat.laplace_jump(nx / 2, 120.0, 50.0, 150.0),
             "probe_1000": lambda: lat.probe(xs, ys)}
    out = {}
    for name, fn in calls.items():
        fn()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        out[name] = (time.perf_counter() - t0) / reps * 1e6
    return out


def run_ours(args):
    import torch

    world, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1710_09541_gb300 import lbm

    nx, ny = cases.PERF_NX, cases.PERF_NY
    phi0, params = cases.perf_case(seed=1 + rank)
    stream = torch.cuda.current_stream()
    N = nx * ny

    def barrier():
        if dist is not None:
            dist.barrier()

    # -- device-resident throughput ------------------------------------------
    lat = lbm.Lattice(nx, ny, stream=stream, **params)
    lat.init(phi0)
    lat.step(args.warmup)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0.record(stream)
        lat.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    s_phi, umax, _, _ = lat.diag()
    lat.close()

    # -- end to end through the C ABI with host buffers ------------------------
    pin = lambda shape: torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    phi_h = pin((ny, nx))
    phi_h[...] = phi0
    outs = {k: pin((ny, nx)) for k in ("phi", "rho", "ux", "uy", "p")}
    lat = lbm.Lattice(nx, ny, stream=stream, **params)
    lat.init(phi_h).step(min(args.warmup, 10))
    lat.fields(out=outs)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat.init(phi_h)            # H2D: phi0 (ux0, uy0, p0 zero on the device)
    lat.step(args.steps)
    lat.fields(out=outs)       # D2H: phi, rho, ux, uy, p; synchronises
    e2e_s = time.perf_counter() - t0
    lat.close()

    batched = storage_variants = data_variants = None
    if not args.no_batched:
        batched = run_batched(torch, lbm, stream, args.batch_steps)
        storage_variants = run_storage_variants(torch, lbm, stream, 2000)
        data_variants = run_data_variants(torch, lbm, stream, 2000)

    t_dev, t_e2e = max_over_ranks([ms / 1e3, e2e_s], dist, "cuda")

    if rank == 0:
        value = whole_job_mlups(N, args.steps, world, t_dev)
        e2e_value = whole_job_mlups(N, args.steps, world, t_e2e)
        ms_step = t_dev * 1e3 / args.steps
        peak, peak_kind = _peaks()
        achieved = BYTES_PER_LU * N / (ms_step * 1e-3) / 1e9
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            rows = 256
            import oracle

            cores = oracle.set_threads(_cores())
            rate, n, dt = _oracle_rate(nx, rows, params, phi0[:rows], args.cpu_seconds)
            cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": _cpu_model(),
                   "sample": f"periodic {nx}x{rows} strip of the workload, {n} steps in {dt:.1f} s"}
            # the same oracle on one thread, on a narrower strip for ~3 s
            oracle.set_threads(1)
            r1, n1, dt1 = _oracle_rate(nx, 32, params, phi0[:32], 3.0)
            oracle.set_threads(cores)
            cpu["single_thread"] = {"value": r1, "unit": UNIT, "cores": 1,
                                    "sample": f"periodic {nx}x32 strip, {n1} steps in {dt1:.1f} s"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "perf-2048: spinodal-like 2048x2048 periodic D2Q9, density ratio 1000",
                       "nx": nx, "ny": ny, "storage": "fp32", "parallelism": f"replicas{world}",
                       "l2": "working set 671 MB per GPU > 129 MB L2 (no flush)",
                       "bytes_per_lu": BYTES_PER_LU},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": _profiled_traffic(),
                         "traffic_unit": "bytes per launch (ncu, " + PROFILE + ")",
                         "peak_kind": peak_kind,
                         "frac_populations_only": BYTES_PER_LU_POPULATIONS * N / (ms_step * 1e-3) / 1e9 / peak,
                         "kernel": "k_step (fused pull-collide, FP32)"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * N / args.steps,
                    "d2h_bytes_per_step": 40 * N / args.steps},
            "clocks": clk.summary(),
            "gpu_launches": args.steps,
            "sum_phi": s_phi, "umax": umax,
            "batched": batched,
            "single_case_storage": storage_variants,
            "data_variants": data_variants,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=1000)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--reference-seconds", type=float, default=90.0,
                    help="--impl reference: host seconds the warm-up and timed steps should take")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("bench.py: --warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

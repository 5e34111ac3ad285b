#!/usr/bin/env python
"""Benchmark: point-iterations per second of Lloyd's k-means with MTI pruning.

One step = one whole k-means run (reset to the Forgy centroids, then Lloyd
iterations until no assignment changes or the iteration limit) over the
workload's points, which are resident in HBM before timing starts.  The
metric is n * iterations / time.  Default workload: 66M points, d = 32,
k = 20, a 20-component Gaussian mixture with random SPD covariances, Forgy
seed 42, at most 50 iterations (the MTI FP32 configuration).

Printed (rank 0, one JSON line): the device-timed throughput, the same run
through the C ABI from pinned host memory (e2e), the roofline of the
dominant step (the CUDA-event time of its kernels per iteration against its
algorithmic bytes, or against its FP32 operations at the FMA rate measured in
the same run when that roof binds), the speed of plain FP32 Lloyd on the same
input (with a check that it assigns identically), the FP64 CPU oracle timed
on the host cores on a bounded sample (cpu_baseline), and the SM clocks
sampled while timing.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
                  [--workload NAME] [--no-e2e] [--no-plain] [--no-cpu]
Under torchrun (N > 1) every rank runs an independent replica of the
workload ("replicas only": the data path has no exchange at one GPU per box).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

THROTTLE_BITS = {  # nvidia-smi clocks_event_reasons bitmask
    0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
    0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
    0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting",
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mti_66m_d32_k20")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--n", type=int, default=0, help="override the workload's n (profiling runs)")
    ap.add_argument("--m", type=int, default=0, help="override the batched workload's instance count "
                                                      "(profiling runs)")
    ap.add_argument("--precision", default="", choices=["", "bf16", "fp16", "fp8"],
                    help="override the tensor-core operand format of a precision workload")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(ms: float, work: float, world: int, device: str = "cuda"):
    """Whole-job figures of N replicas: the slowest rank's time and the work
    of all ranks (point-iterations).  Returns (ms_max, work_total)."""
    if world <= 1:
        return ms, work
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, float(work)], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(t[1])


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while timing."""

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows = []
        self.proc = None

    def start(self):
        q = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active"
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 4:
                self.rows.append(parts)

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                bits = int(r[3], 16) if r[3].startswith("0x") else int(r[3])
                for b, name in THROTTLE_BITS.items():
                    if bits & b and name != "gpu_idle":
                        reasons.add(name)
            except ValueError:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


KERNEL_SOURCES = {  # CUDA sources that define each profiled kernel
    "k_mti_w": "kernels_warp.cu", "k_dense_w": "kernels_warp.cu", "k_mti": "kernels.cu", "k_dense": "kernels.cu",
    "k_tc_assign": "precision.cu", "k_bscan": "batch.cu", "k_bmti": "batch.cu",
    "k_mti_sel": "kernels_split.cu", "k_mti_scan": "kernels_split.cu", "k_mti_delta": "kernels_split.cu",
    "k_dense_scan": "kernels_split.cu",
}


def csrc_sha256(kernel: str = "") -> str:
    """Hash of the CUDA sources of `kernel` (its file plus the shared
    headers), or of every CUDA source when kernel is empty."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1606_08905_gb300", "csrc")
    base = re.sub(r"<.*", "", kernel)
    want = {KERNEL_SOURCES[base], "device_common.cuh", "knor_internal.cuh"} if base in KERNEL_SOURCES else None
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".h")) and (want is None or f in want):
            h.update(f.encode())
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()


def ncu_traffic(kernel: str, workload: str):
    """Per-launch DRAM bytes of `kernel` (scaled to this workload) from the
    committed ncu summary profiles/<kernel>_<workload>.md, if the kernel's
    CUDA sources have not changed since the capture (else None).  For a step
    of several kernels ("a + b + c") the sum of theirs, if all are known."""
    if " + " in kernel:
        parts = [ncu_traffic(kk, workload) for kk in kernel.split(" + ")]
        return None if any(v is None for v in parts) else float(sum(parts))
    base = re.sub(r"<.*", "", kernel)
    path = os.path.join(ROOT, "profiles", f"{base}_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    h = re.search(r"csrc_sha256:\s*([0-9a-f]+)", text)
    if not m or not h or h.group(1) != csrc_sha256(kernel):
        return None
    return float(m.group(1))


def make_points(wl, device):
    from paper_1606_08905_gb300 import synth
    return synth.make(wl["kind"], wl["n"], wl["d"], wl["k"], wl["data_seed"], device=device)


def cpu_oracle_run(Xs, k, max_iters, prune, threads):
    import oracle
    C0 = oracle.forgy_centroids(Xs, k, 42)
    t = time.perf_counter()
    r = oracle.run(Xs, C0, max_iters, prune=prune, nthreads=threads)
    dt = time.perf_counter() - t
    return Xs.shape[0] * r.iters, dt, r.iters


def cpu_sample_rows(wl, seconds, X=None, threads=1):
    """Rows of the workload that the FP64 oracle runs through in about
    `seconds`, from a short probe run on the first rows (or the workload's
    distribution drawn on the CPU when X is None)."""
    probe = int(min(wl["n"], 200_000))
    if X is not None:
        Xp = X[:probe].cpu().numpy()
    else:
        from paper_1606_08905_gb300 import synth
        Xp = synth.make(wl["kind"], probe, wl["d"], wl["k"], wl["data_seed"], device="cpu").numpy()
    p, dt, _ = cpu_oracle_run(Xp, wl["k"], wl["max_iters"], ("elkan" if wl.get("elkan") else wl["prune"]), threads)
    rate = p / max(dt, 1e-3)
    return int(max(20_000, min(wl["n"], rate * seconds / wl["max_iters"])))


L2_BYTES = 129e6  # GB300 L2


def l2_note(point_bytes: float) -> str:
    """How the timed loop relates to L2: the named large workloads exceed it;
    a workload smaller than L2 (the 100k-point plain configuration) is timed
    L2-resident, as it runs in practice, and says so."""
    if point_bytes > L2_BYTES:
        return f"inputs larger than L2 ({point_bytes / 1e9:.2f} GB of points)"
    return f"L2-resident: {point_bytes / 1e6:.1f} MB of points, no flush between iterations"


def reference_arm(args, wl, world, rank):
    """The FP64 CPU oracle as the reference arm (there is no installable
    reference implementation: the paper ships no code)."""
    if rank != 0:
        return
    import numpy as np
    import oracle
    import torch  # noqa: F401
    from paper_1606_08905_gb300 import synth
    threads = os.cpu_count() or 1
    total_budget = 150.0
    per_step = max(2.0, total_budget / max(1, args.steps + args.warmup))
    ns = cpu_sample_rows(wl, per_step, None, threads)
    Xs = synth.make(wl["kind"], ns, wl["d"], wl["k"], wl["data_seed"], device="cpu").numpy()
    for _ in range(args.warmup):
        cpu_oracle_run(Xs, wl["k"], wl["max_iters"], ("elkan" if wl.get("elkan") else wl["prune"]), threads)
    pts, secs, its = 0, 0.0, []
    for _ in range(args.steps):
        p, dt, it = cpu_oracle_run(Xs, wl["k"], wl["max_iters"], ("elkan" if wl.get("elkan") else wl["prune"]), threads)
        pts += p
        secs += dt
        its.append(it)
    value = pts / secs
    sample = f"first {ns} points of the workload's distribution (CPU-drawn), full run per step"
    line = {
        "impl": "reference", "metric": "point-iterations/sec", "value": value,
        "unit": "point-iterations/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(wl, args.workload, world),
        "cpu_baseline": {"value": value, "unit": "point-iterations/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "point-iterations/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "iterations_per_step": its,
    }
    print(json.dumps(line), flush=True)


def batch_reference_arm(args, wl, world, rank):
    """The FP64 oracle on the batched workload: whole runs of its instances,
    smallest first, for a bounded time per step."""
    if rank != 0:
        return
    import oracle  # noqa: F401
    from paper_1606_08905_gb300 import synth
    threads = os.cpu_count() or 1
    per_step = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    specs = sorted(synth.batched_specs(wl["m"], wl["data_seed"]), key=lambda s: s.n)

    def one_step():
        pts, secs, used = 0, 0.0, 0
        for sp in specs:
            if secs >= per_step:
                break
            Xs = synth.batched_instance(sp).numpy()
            p, dt, _ = cpu_oracle_run(Xs, sp.k, wl["max_iters"], wl["prune"], threads)
            pts += p
            secs += dt
            used += 1
        return pts, secs, used

    for _ in range(args.warmup):
        one_step()
    pts, secs, used = 0, 0.0, 0
    for _ in range(args.steps):
        p, dt, used = one_step()
        pts += p
        secs += dt
    value = pts / secs
    sample = (f"the {used} smallest of the {wl['m']} instances, a full run of each ({'MTI' if wl['prune'] else 'plain'}, "
              f"FP64), per step")
    line = {
        "impl": "reference", "metric": "point-iterations/sec", "value": value,
        "unit": "point-iterations/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(wl, args.workload, world),
        "cpu_baseline": {"value": value, "unit": "point-iterations/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "point-iterations/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batch_arm(args, wl, world, rank, local):
    """The batched form: every instance of the workload, one knor_batch_run
    per step (from C^0, up to max_iters iterations)."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1606_08905_gb300 import build as kbuild
    from paper_1606_08905_gb300 import knor, synth
    kbuild.build()
    knor.load()
    torch.cuda.set_device(local)
    T = wl["max_iters"]
    specs = synth.batched_specs(wl["m"], wl["data_seed"])
    Xd = [synth.batched_instance(sp, device="cuda") for sp in specs]
    ks = [sp.k for sp in specs]
    torch.cuda.synchronize()
    b = knor.Batch(Xd, ks, seed=42, prune=wl["prune"])
    stream = torch.cuda.ExternalStream(b.stream)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(max(3, args.warmup)):
        b.reset()
        b.run(T)
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    iters, pit = [], 0
    for _ in range(args.steps):
        b.reset()
        done, _ = b.run(T)
        iters.append(done)
        pit += b.work()[0]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms_max, pts_all = aggregate(ms, float(pit), world)
    value = pts_all / (ms_max / 1000.0)
    # per iteration: k_bscan, k_breduce, k_bstep, k_btable; with pruning
    # also k_bseg, k_bclause1, k_bbatches and one k_bmti per width class
    # present; 3 more per reset (k_bround, k_binit_state, k_btable)
    n_widths = len({sp.d for sp in specs})
    per_iter = 4 + (3 + n_widths if wl["prune"] else 0)
    launches = sum(3 + per_iter * it for it in iters)

    # per-kernel event timing; the scan's roofline over the MTI iterations
    # (iteration 1 is the full scan from C^0 and is timed apart)
    peaks, peak_src = measured_peaks()
    b.set_profiling(True)
    b.reset()
    b.profile(reset=True)
    b.iterate()
    first = b.profile(reset=True)
    w1 = b.work()
    done, recs = b.run(T - 1)
    prof = b.profile(reset=True)
    w2 = b.work()
    b.set_profiling(False)
    n_scan, ms_scan = prof["mti"]
    mti_bytes = w2[1] - w1[1]
    gbs = mti_bytes / (ms_scan / 1000.0) / 1e9 if ms_scan > 0 else 0.0
    kernels = {
        "scan_iteration1": {"kernel": "k_bscan", "launches": first["mti"][0], "ms_total": first["mti"][1],
                            "point_iterations": w1[0], "algorithmic_bytes": w1[1]},
        "scan_mti": {"kernel": "k_bclause1 + k_bmti (k_bscan for instances in dense mode)",
                     "launches": n_scan, "ms_total": ms_scan,
                     "ms_per_launch": ms_scan / max(1, n_scan), "algorithmic_bytes_per_launch": mti_bytes / max(1, n_scan),
                     "achieved_gbs": gbs},
        "reduce": {"kernel": "k_breduce", "launches": prof["reduce"][0], "ms_total": prof["reduce"][1]},
        "table": {"kernel": "k_bstep + k_btable", "launches": prof["table"][0], "ms_total": prof["table"][1]},
    }
    total_ms = sum(v[1] for v in prof.values()) + sum(v[1] for v in first.values())
    roof = {"kernel": "k_bmti", "bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"],
            "peak_source": peak_src, "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
            "traffic": ncu_traffic("k_bmti", args.workload),
            "share_of_kernel_time": (ms_scan + first["mti"][1]) / total_ms if total_ms else None,
            "scope": "MTI iterations (2..): the scan group k_bscan + k_bseg + k_bclause1 + k_bbatches + "
                     "k_bmti per width class, timed as one interval; iteration 1 is the full scan from C^0"}

    # plain Lloyd on the same batch
    plain = None
    if not args.no_plain:
        with knor.Batch(Xd, ks, seed=42, prune=False) as bp:
            bp.reset()
            bp.run(T)
            ps = torch.cuda.ExternalStream(bp.stream)
            q0 = torch.cuda.Event(enable_timing=True)
            q1 = torch.cuda.Event(enable_timing=True)
            q0.record(ps)
            bp.reset()
            bp.run(T)
            ppit = bp.work()[0]
            q1.record(ps)
            torch.cuda.synchronize()
            same = all(np.array_equal(bp.assignments(i), b.assignments(i)) for i in range(wl["m"]))
            pv = ppit / (q0.elapsed_time(q1) / 1000.0)
            plain = {"value": pv, "unit": "point-iterations/s", "speedup": (value / world) / pv,
                     "identical_assignments_all_instances": bool(same)}

    # e2e through the C ABI from pinned host memory: create, run, read back
    e2e = None
    if not args.no_e2e:
        Xh = []
        for x in Xd:
            h = torch.empty(x.shape, dtype=torch.float32, pin_memory=True)
            h.copy_(x)
            Xh.append(h)
        outs = [torch.empty(sp.n, dtype=torch.int32, pin_memory=True) for sp in specs]
        del b
        torch.cuda.synchronize()
        es = max(1, min(args.steps, 2))
        t0 = time.perf_counter()
        e_pit = 0
        for _ in range(es):
            with knor.Batch(Xh, ks, seed=42, prune=wl["prune"]) as b2:
                b2.run(T)
                for i in range(wl["m"]):
                    b2.assignments(i, outs[i])
                e_pit += b2.work()[0]
        dt = time.perf_counter() - t0
        ntot = sum(sp.n for sp in specs)
        e2e = {"value": e_pit / dt, "unit": "point-iterations/s",
               "h2d_bytes_per_step": sum(sp.n * sp.d * 4 for sp in specs), "d2h_bytes_per_step": ntot * 4,
               "steps": es, "ms_per_step": 1000.0 * dt / es,
               "includes": "knor_batch_create (H2D copies, validation, allocation, tuning from the cache, graph "
                           "build), knor_batch_run, knor_batch_get_assignments for every instance, destroy"}

    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        threads = os.cpu_count() or 1
        srt = sorted(specs, key=lambda sp: sp.n)
        pts, secs, used = 0, 0.0, 0
        for sp in srt:
            if secs >= args.cpu_seconds:
                break
            Xs = synth.batched_instance(sp).numpy()
            p, dt, _ = cpu_oracle_run(Xs, sp.k, T, wl["prune"], threads)
            pts += p
            secs += dt
            used += 1
        cpu = {"value": pts / secs, "unit": "point-iterations/s", "cores": threads, "kind": "oracle",
               "sample": f"full runs of the {used} smallest of the {wl['m']} instances "
                         f"({'MTI' if wl['prune'] else 'plain'}, FP64), {secs:.1f} s"}

    if rank == 0:
        line = {"metric": "point-iterations/sec", "value": value, "unit": "point-iterations/s",
                "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
                "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_of(wl, args.workload, world),
                "iterations_per_step": iters, "roofline": roof, "kernels": kernels,
                "cpu_baseline": cpu, "e2e": e2e, "vs_plain_fp32": plain,
                "gpu_launches": launches, "clocks": clk}
        print(json.dumps(line), flush=True)


def synth_n(name):
    from paper_1606_08905_gb300 import synth
    return synth.WORKLOADS[name]["n"]


def batch_bytes(wl):
    from paper_1606_08905_gb300 import synth
    return sum(sp.n * sp.d * 4 for sp in synth.batched_specs(wl["m"], wl["data_seed"]))


def config_of(wl, name, world):
    if wl["kind"] == "batched":
        return {"workload": name if wl["n"] == synth_n(name) else f"{name} (m overridden)",
                "instances": wl["m"], "total_points": wl["n"],
                "n_i": "log-uniform in [1e3, 1e6]", "d_i": "uniform over {8, 16, 32, 64}",
                "k_i": "uniform on {4..256}", "max_iters": wl["max_iters"],
                "pruning": "MTI" if wl["prune"] else "none", "init": "Forgy, seed 42 + instance",
                "data_seed": wl["data_seed"], "points_dtype": "f32",
                "l2": l2_note(batch_bytes(wl)),
                "parallelism": f"replicas x{world}"}
    return {"workload": name if wl["n"] == synth_n(name) else f"{name} (n overridden)", "n": wl["n"],
            "distance": (wl["precision"].upper() + " tensor cores + exact FP32 recheck"
                         if wl.get("precision", "fp32") != "fp32" else "FP32"), "d": wl["d"], "k": wl["k"], "max_iters": wl["max_iters"],
            "pruning": ("Elkan (MTI + lower bounds)" if wl.get("elkan") else "MTI") if wl["prune"] else "none",
            "init": "Forgy, seed 42",
            "data_seed": wl["data_seed"], "points_dtype": "f32",
            "l2": l2_note(wl["n"] * wl["d"] * 4),
            "points": "pinned host memory, read in place over NVLink-C2C" if wl.get("points_in_host")
                      else "HBM",
            "parallelism": f"replicas x{world}"}


def our_arm(args, wl, world, rank, local):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1606_08905_gb300 import build as kbuild
    from paper_1606_08905_gb300 import knor
    kbuild.build()
    knor.load()
    torch.cuda.set_device(local)
    n, d, k, T = wl["n"], wl["d"], wl["k"], wl["max_iters"]
    X = make_points(wl, "cuda")
    torch.cuda.synchronize()
    prec = wl.get("precision", "fp32")
    elkan = bool(wl.get("elkan", False))
    on_host = bool(wl.get("points_in_host", False))
    if on_host:  # the points stay in pinned host memory; the GPU reads them in place
        X = X.cpu().pin_memory()
    ctx = knor.Context(X, k, seed=42, prune=wl["prune"], precision=prec, elkan=elkan, points_in_host=on_host)
    stream = torch.cuda.ExternalStream(ctx.stream)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(max(3, args.warmup)):
        ctx.reset()
        ctx.run(T)
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    iters = []
    for _ in range(args.steps):
        ctx.reset()
        done, _ = ctx.run(T)
        iters.append(done)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    pts = float(n) * sum(iters)
    ms_max, pts_all = aggregate(ms, pts, world)
    value = pts_all / (ms_max / 1000.0)
    # kernels in one iteration's graph (each scan launch returns at once in the
    # iterations that are not its own): precision form 9; split path: dense
    # scan [+ Clause-1 selection + MTI scan] + delta sums + merge + table;
    # else dense | MTI scan + merge + table
    if wl.get("precision", "fp32") != "fp32":
        per_it = 9
    elif ctx.kernel_name("delta"):  # the split path: a delta-sum launch every iteration
        per_it = (5 if elkan else 6) if wl["prune"] else 4
    else:
        per_it = 4 if wl["prune"] else 3
    launches = sum(3 + it * per_it for it in iters)

    # ---- per-kernel CUDA-event timing (profiling mode: kernel by kernel on the
    # library stream, same reset + run steps), for the roofline
    ctx.set_profiling(True)
    ctx.profile(reset=True)
    prof_iters = []
    prof_recs = []
    # per-kernel totals over the dense iterations (plain Lloyd, MTI iteration
    # 1) and over the MTI iterations, read back after every iteration
    prof_it = {"dense": {}, "mti": {}}
    for _ in range(max(1, min(args.steps, 3))):
        ctx.reset()
        done = 0
        while done < T:
            r = ctx.iterate()
            done += 1
            prof_recs.append(r)
            kind = "dense" if (r["iteration"] == 1 or not wl["prune"]) else "mti"
            for kname_, (lk, mk) in ctx.profile(reset=True).items():
                if lk:
                    a0 = prof_it[kind].setdefault(kname_, [0, 0.0])
                    a0[0] += lk
                    a0[1] += mk
            if r["changed"] == 0:
                break
        prof_iters.append(done)
    prof = {kk: (0, 0.0) for kk in knor.KERNELS}
    for kind in prof_it.values():
        for kname_, (lk, mk) in kind.items():
            prof[kname_] = (prof[kname_][0] + lk, prof[kname_][1] + mk)
    ctx.set_profiling(False)
    # algorithmic work per launch: dense scan n(4d + 16) bytes;
    # MTI scan 8n + active (4d + 8) bytes with active = n - clause1_skipped;
    # tensor-core scan 2 n k d flops
    peaks, peak_src = measured_peaks()
    kernels = {}
    if prec != "fp32":
        launches_k, ms_k = prof["dense"]
        flops = 2.0 * n * k * d * launches_k
        tf = flops / (ms_k / 1000.0) / 1e12
        # FP16 runs at the BF16 dense rate; FP8 at twice it (nominal ratio)
        ratio = 2.0 if prec == "fp8" else 1.0
        peak_t = peaks["bf16_tflops_sustained"] * ratio
        kernels["dense"] = {"kernel": ctx.kernel_name("dense"), "launches": launches_k, "ms_total": ms_k,
                            "ms_per_launch": ms_k / launches_k, "algorithmic_flops_per_launch": 2.0 * n * k * d,
                            "achieved_tflops": tf, "frac_of_peak": tf / peak_t}
        for kk in ("recheck", "sums", "reduce", "table"):
            lk, mk = prof[kk]
            if lk:
                kernels[kk] = {"kernel": ctx.kernel_name(kk), "launches": lk, "ms_total": mk,
                               "ms_per_launch": mk / lk}
        rechecked = sum(r["rechecked"] for r in prof_recs)
        total_prof_ms = sum(v[1] for v in prof.values())
        roof = {"kernel": ctx.kernel_name("dense"), "bound": "tensor", "achieved": tf,
                "peak": peak_t, "peak_source": peak_src + " bf16 sustained" + (" x 2 (FP8 nominal ratio)"
                                                                               if ratio != 1.0 else ""),
                "unit": "TFLOP/s", "frac": tf / peak_t,
                "traffic": ncu_traffic(ctx.kernel_name("dense"), args.workload) if not args.n else None,
                "share_of_kernel_time": ms_k / total_prof_ms,
                "rechecked_fraction": rechecked / float(n * max(1, len(prof_recs))),
                "fp32_evals_per_rechecked_point":
                    (sum(r["dist_evals"] for r in prof_recs) - n * k * len(prof_recs)) / float(max(1, rechecked))}
    else:
        dense_bytes = sum(n * (4 * d + 16) for r in prof_recs if (r["iteration"] == 1 or not wl["prune"]))
        mti_bytes = sum(8 * n + (n - r["clause1_skipped"]) * (4 * d + 8) for r in prof_recs
                        if wl["prune"] and r["iteration"] > 1)
        if elkan:
            # Elkan also reads the k lower bounds of every point Clause 1 does
            # not skip and writes one per distance it computes; its first
            # (full) scan writes all n k of them
            dense_bytes += sum(4 * n * k for r in prof_recs if r["iteration"] == 1)
            mti_bytes += sum((n - r["clause1_skipped"]) * 4 * k + 4 * r["dist_evals"] for r in prof_recs
                             if r["iteration"] > 1)
        # FP32 arithmetic of the scans: one subtraction and one fused
        # multiply-add per dimension and distance (the direct form), against
        # the FMA issue rate measured on this GPU now (knor_probe_alu)
        kernels_bytes = {}
        fma_tflops, _ = knor.probe_alu("fp32")
        fma_ops_peak = fma_tflops * 1e12 / 2.0
        dense_ops = sum(2.0 * d * k * n for r in prof_recs if (r["iteration"] == 1 or not wl["prune"]))
        mti_ops = sum(2.0 * d * r["dist_evals"] for r in prof_recs if wl["prune"] and r["iteration"] > 1)
        # one "step" of each kind: its scan plus, on the split path, the
        # Clause-1 selection and the delta sums of the same iterations
        def step(kind, names):
            parts = {nm: prof_it[kind][nm] for nm in names if nm in prof_it[kind]}
            launches_k = max((v[0] for v in parts.values()), default=0)
            return launches_k, sum(v[1] for v in parts.values()), {
                ctx.kernel_name(nm): {"launches": v[0], "ms_total": v[1]} for nm, v in parts.items()}
        for name, byts, ops in (("dense", dense_bytes, dense_ops), ("mti", mti_bytes, mti_ops)):
            launches_k, ms_k, parts = step(name, ("dense", "delta") if name == "dense" else ("select", "mti", "delta"))
            if launches_k == 0 or ms_k <= 0:
                continue
            kernels_bytes[name] = byts
            if launches_k == 0 or ms_k <= 0:
                continue
            gbs = byts / (ms_k / 1000.0) / 1e9
            opsps = ops / (ms_k / 1000.0)
            if name == "dense" and ctx.kernel_name("dense") in parts:
                # the scan on its own against the FP32 pipe (its sums are the
                # delta part)
                sp_ = parts[ctx.kernel_name("dense")]
                sp_["alu_frac"] = ops / (sp_["ms_total"] / 1000.0) / fma_ops_peak
            kernels[name] = {"launches": launches_k, "ms_total": ms_k, "ms_per_launch": ms_k / launches_k,
                             "parts": parts,
                             "algorithmic_bytes_per_launch": byts / launches_k, "achieved_gbs": gbs,
                             "frac_of_" + peak_src + "_hbm": gbs / peaks["hbm_gbs"],
                             "fp32_ops_per_launch": ops / launches_k,
                             "alu": {"achieved_tops": opsps / 1e12, "peak_tops": fma_ops_peak / 1e12,
                                     "peak_source": "FP32 FMA issue rate measured now (knor_probe_alu)",
                                     "frac": opsps / fma_ops_peak}}
        total_prof_ms = sum(v[1] for v in prof.values())
        dom = max(kernels, key=lambda kk: kernels[kk]["ms_total"])
        for kk in kernels:
            kernels[kk]["kernel"] = " + ".join(kernels[kk]["parts"])
        kname = kernels[dom]["kernel"]
        kd = kernels[dom]
        hbm_frac = kd["achieved_gbs"] / peaks["hbm_gbs"]
        if kd["alu"]["frac"] > hbm_frac:
            # the binding roof is the FP32 pipe (large k: 2dk operations per
            # 4d + 16 bytes), e.g. the plain scans and uniform data at k = 100
            roof = {"kernel": kname, "bound": "alu", "achieved": kd["alu"]["achieved_tops"],
                    "peak": kd["alu"]["peak_tops"], "peak_source": kd["alu"]["peak_source"],
                    "unit": "Tops/s (FP32 sub + FMA per dimension and distance)", "frac": kd["alu"]["frac"],
                    "traffic": None, "hbm_frac": hbm_frac}
        else:
            roof = {"kernel": kname, "bound": "hbm", "achieved": kd["achieved_gbs"],
                    "peak": peaks["hbm_gbs"], "peak_source": peak_src, "unit": "GB/s", "frac": hbm_frac,
                    "traffic": ncu_traffic(kname, args.workload) if not args.n else None,
                    "alu_frac": kd["alu"]["frac"]}
        roof["share_of_kernel_time"] = kd["ms_total"] / total_prof_ms

    # ---- Elkan's ablation: MTI on the same points, the same measurements
    vs_mti = None
    if elkan:
        ctx.reset()
        _, e_recs = ctx.run(T)
        a_e = torch.empty(n, dtype=torch.int32, device="cuda")
        ctx.assignments(a_e)
        with knor.Context(X, k, seed=42, prune=True) as mc:
            ms_ = torch.cuda.ExternalStream(mc.stream)
            mc.run(T)
            q0 = torch.cuda.Event(enable_timing=True)
            q1 = torch.cuda.Event(enable_timing=True)
            q0.record(ms_)
            msteps, mits = max(1, min(args.steps, 3)), 0
            for _ in range(msteps):
                mc.reset()
                done_m, m_recs = mc.run(T)
                mits += done_m
            q1.record(ms_)
            torch.cuda.synchronize()
            a_m = torch.empty(n, dtype=torch.int32, device="cuda")
            mc.assignments(a_m)
            m_bytes = sum(8 * n + (n - r["clause1_skipped"]) * (4 * d + 8) for r in m_recs[1:])
            vs_mti = {"mti_value": n * mits / (q0.elapsed_time(q1) / 1000.0), "unit": "point-iterations/s",
                      "elkan_value_over_mti": value / (n * mits / (q0.elapsed_time(q1) / 1000.0)),
                      "identical_assignments": bool(torch.equal(a_e, a_m)),
                      "iterations": [len(e_recs), len(m_recs)],
                      "dist_evals_after_iteration_1": [sum(r["dist_evals"] for r in e_recs[1:]),
                                                        sum(r["dist_evals"] for r in m_recs[1:])],
                      "clause1_skipped_after_iteration_1": [sum(r["clause1_skipped"] for r in e_recs[1:]),
                                                             sum(r["clause1_skipped"] for r in m_recs[1:])],
                      "algorithmic_bytes_after_iteration_1": [
                          sum(8 * n + (n - r["clause1_skipped"]) * (4 * d + 8 + 4 * k) + 4 * r["dist_evals"]
                              for r in e_recs[1:]), m_bytes],
                      "order": "[elkan, mti]"}

    # ---- plain FP32 Lloyd on the same points: speed, and identical assignments
    plain = None
    if not args.no_plain and (wl["prune"] or prec != "fp32"):
        ctx.reset()
        ctx.run(T)
        a_mti = torch.empty(n, dtype=torch.int32, device="cuda")
        ctx.assignments(a_mti)
        with knor.Context(X, k, seed=42, prune=False, points_in_host=on_host) as pc:
            pc.reset()
            pc.run(T)
            pstream = torch.cuda.ExternalStream(pc.stream)
            ps = 1 if prec != "fp32" else max(1, min(args.steps, 2))
            q0 = torch.cuda.Event(enable_timing=True)
            q1 = torch.cuda.Event(enable_timing=True)
            q0.record(pstream)
            pits = 0
            for _ in range(ps):
                pc.reset()
                done, _ = pc.run(T)
                pits += done
            q1.record(pstream)
            torch.cuda.synchronize()
            a_plain = torch.empty(n, dtype=torch.int32, device="cuda")
            pc.assignments(a_plain)
            pv = n * pits / (q0.elapsed_time(q1) / 1000.0)
            plain = {"value": pv, "unit": "point-iterations/s", "speedup": (value / world) / pv,
                     "identical_assignments": bool(torch.equal(a_mti, a_plain)),
                     "iterations": pits // ps}

    # ---- e2e through the C ABI from pinned host memory
    e2e = None
    if not args.no_e2e:
        Xh = torch.empty((n, d), dtype=torch.float32, pin_memory=True)
        Xh.copy_(X)
        ah = torch.empty(n, dtype=torch.int32, pin_memory=True)
        Ch = torch.empty((k, d), dtype=torch.float64, pin_memory=True)
        del ctx
        torch.cuda.synchronize()
        es = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        e_iters = 0
        for _ in range(es):
            with knor.Context(Xh, k, seed=42, prune=wl["prune"], precision=prec, elkan=elkan,
                              points_in_host=on_host) as c2:
                done, _ = c2.run(T)
                c2.assignments(ah)
                c2.centroids(Ch)
                e_iters += done
        dt = time.perf_counter() - t0
        e2e = {"value": n * e_iters / dt, "unit": "point-iterations/s",
               "h2d_bytes_per_step": n * d * 4, "d2h_bytes_per_step": n * 4 + k * d * 8,
               "steps": es, "ms_per_step": 1000.0 * dt / es,
               "includes": "knor_create (H2D copy, input validation, allocation, graph build), knor_run, "
                           "knor_get_assignments, knor_get_centroids, knor_destroy"}

    # ---- CPU oracle on a bounded sample of the same points (rank 0, N = 1)
    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        threads = os.cpu_count() or 1
        ns = cpu_sample_rows(wl, args.cpu_seconds, X, threads)
        Xs = X[:ns].cpu().numpy()
        mode = "elkan" if elkan else wl["prune"]
        p, dt, it = cpu_oracle_run(Xs, k, T, mode, threads)
        cpu = {"value": p / dt, "unit": "point-iterations/s", "cores": threads, "kind": "oracle",
               "sample": f"first {ns} of the {n} points, one full run ({it} iterations, "
                         f"{'Elkan' if elkan else 'MTI' if wl['prune'] else 'plain'}, FP64), {dt:.1f} s"}

    if rank == 0:
        line = {"metric": "point-iterations/sec", "value": value, "unit": "point-iterations/s",
                "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
                "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_of(wl, args.workload, world),
                "iterations_per_step": iters,
                "active_fraction_per_iteration": [round(1.0 - r["clause1_skipped"] / n, 4)
                                                  for r in prof_recs[:prof_iters[0]]] if wl["prune"] else None,
                "roofline": roof, "kernels": kernels,
                "cpu_baseline": cpu, "e2e": e2e, "vs_plain_fp32": plain,
                "gpu_launches": launches, "clocks": clk}
        if vs_mti is not None:
            line["elkan_vs_mti"] = vs_mti
        print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world, rank, local = dist_env()
    from paper_1606_08905_gb300 import synth
    if args.workload not in synth.WORKLOADS:
        raise SystemExit(f"unknown workload {args.workload}; one of {sorted(synth.WORKLOADS)}")
    wl = dict(synth.WORKLOADS[args.workload])
    if args.n:
        wl["n"] = args.n
    if args.precision and wl.get("precision", "fp32") != "fp32":
        wl["precision"] = args.precision
    if args.m and wl["kind"] == "batched":
        wl["m"] = args.m
        wl["n"] = sum(sp.n for sp in synth.batched_specs(args.m, wl["data_seed"]))
    if args.impl == "reference":
        (batch_reference_arm if wl["kind"] == "batched" else reference_arm)(args, wl, world, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
    try:
        (batch_arm if wl["kind"] == "batched" else our_arm)(args, wl, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Throughput of the coupled flow + enthalpy lattice Boltzmann step on GB300.

Workload: the 256^3 cubic-cavity melting case (Sec. 3.3 set-up; Ra = 1e6, Pr = 0.02,
St = 1), D3Q19 MRT flow + D3Q7 MRT enthalpy, FP32 storage with the FP64 enthalpy
channel, two-lattice pull streaming, diagnostics every 500 steps.  A step is one
time step of every lattice node.  The working set (3.6 GB) is far larger than the
129 MB L2, so no flush is needed between steps.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle instead (on a
256x32x32 slab of the same cavity, host cores): the paper ships no code, so the oracle is
the reference.
Under torchrun every rank runs its own replica (the lattice is not sharded).
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lbpc_inputs as inp  # noqa: E402

METRIC = "coupled flow+enthalpy MLUPS, % of HBM roofline; adjoint/forward time ratio"
BYTES_PER_LUP = {inp.FP64: 416, inp.FP32: 216, inp.FP16: 116, inp.BF16: 116, inp.FP16_G32: 140,
                 inp.BF16_G32: 140}
SAMPLE_SHAPE = (256, 32, 32)  # oracle sample: a slab of the same cavity (same lattice constants)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _kernel_hash():
    """Hash of the sources that define the step kernels (device code and its headers);
    host API code is left out."""
    csrc = os.path.join(ROOT, "paper_1703_02652_gb300", "csrc")
    files = [os.path.join(csrc, n) for n in ("lbpc_kernels.cuh", "lbpc_internal.h")]
    files += sorted(glob.glob(os.path.join(csrc, "lbpc_kern_*.cu")))
    h = hashlib.sha256()
    for p in files:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic_per_lup(precision, streaming=inp.PULL):
    """DRAM bytes per lattice update of the step kernel from the committed ncu summary
    (one full-size launch, read + write), valid only while the kernel sources hash to the
    recorded value."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.txt")
    if not os.path.exists(path):
        return None
    rec = {}
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#") and "=" in line:
            k, v = line.split("=", 1)
            rec[k.strip()] = v.strip()
    if rec.get("kernel_sources_sha256_16") != _kernel_hash():
        return None
    key = f"dram_bytes_per_lup_{inp.PRECISION_NAMES[precision]}" + (
        "_aa" if streaming == inp.AA else "")
    return float(rec[key]) if key in rec else None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(self.idx).uuid)
            sel = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        except Exception:
            sel = str(self.idx)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", sel, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        if not self.rows:
            return None
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest value of x over all ranks (the slowest replica sets the job time)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(world: int, nodes: int, steps: int, seconds: float) -> float:
    """Whole-job throughput of `world` independent replicas of `nodes` lattice nodes each,
    all advanced `steps` steps within `seconds` (max over ranks)."""
    return world * nodes * steps / seconds / 1e6


def cpu_baseline(seconds=15.0, min_steps=2):
    """The FP64 oracle as it stands on the host cores, on a slab of the benchmark cavity."""
    import oracle

    w = inp.bench_workload()
    o = oracle.Oracle(SAMPLE_SHAPE, w.params)
    h0 = np.random.default_rng(w.seed).uniform(-w.perturb, w.perturb, o.N)
    o.set_initial_h(h0)
    o.step(1)  # warm-up
    steps, t0 = 0, time.perf_counter()
    while steps < min_steps or time.perf_counter() - t0 < seconds:
        o.step(1)
        steps += 1
    dt = time.perf_counter() - t0
    return {"value": o.N * steps / dt / 1e6, "unit": "MLUPS", "cores": oracle.threads(),
            "kind": "oracle",
            "sample": f"{steps} FP64 oracle steps of a {SAMPLE_SHAPE[0]}x{SAMPLE_SHAPE[1]}x"
                      f"{SAMPLE_SHAPE[2]} slab of the 256^3 cavity (same lattice constants)"}


def adjoint_ratio(p, shape, h0, steps=200, intervals=(50, 100, 200)):
    """Wall time of the adjoint (forward with checkpoints, then backward: segment
    recompute with the macroscopic tape + reverse sweep) over the plain forward, same
    steps, same state; CUDA events on the handle's stream."""
    import torch
    from paper_1703_02652_gb300 import LBPC

    g = LBPC(shape, p.replace(report_every=0))
    g.set_initial_h(h0)
    g.step(5)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    ev[0].record(g.stream)
    g.step(steps)
    ev[1].record(g.stream)
    torch.cuda.synchronize()
    t_fwd = ev[0].elapsed_time(ev[1])
    out = {"lattice": list(shape), "steps": steps, "forward_ms_per_step": t_fwd / steps,
           "backward_over_forward": {}, "total_over_forward": {}, "workspace_gb": {}}
    for k in intervals:
        g.set_initial_h(h0)
        g.step(5)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev[0].record(g.stream)
        g.adjoint_forward(steps, k)  # synchronises to return J
        ev[1].record(g.stream)
        g.adjoint_backward(0)
        ev[2].record(g.stream)
        torch.cuda.synchronize()
        t_af, t_ab = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
        out["backward_over_forward"][str(k)] = t_ab / t_fwd
        out["total_over_forward"][str(k)] = (t_af + t_ab) / t_fwd
        out["workspace_gb"][str(k)] = g._adj_ws.numel() / 1e9
        g.release_adjoint_workspace()
        torch.cuda.empty_cache()
    del g
    torch.cuda.empty_cache()
    return out


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle

    w = inp.bench_workload()
    o = oracle.Oracle(SAMPLE_SHAPE, w.params)
    o.set_initial_h(np.random.default_rng(w.seed).uniform(-w.perturb, w.perturb, o.N))
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    v = o.N * args.steps / dt / 1e6
    sample = (f"{args.steps} FP64 oracle steps of a {SAMPLE_SHAPE[0]}x{SAMPLE_SHAPE[1]}x"
              f"{SAMPLE_SHAPE[2]} slab of the 256^3 cavity (same lattice constants)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w.name + " (oracle sample: slab)",
                                        "lattice": list(SAMPLE_SHAPE)},
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": oracle.threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_ours(args):
    import torch

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1703_02652_gb300 import LBPC

    w = inp.bench_workload()
    if args.lattice != 256 or args.pr != 0.02:
        # the same cavity at another size (profiling cases; the 512^3 throughput-ceiling
        # lines) or Prandtl number (512^3 is quoted at Pr = 50)
        w = inp.cavity_melting(n=args.lattice, Ra=1e6, Pr=args.pr, St=1.0, precision=inp.FP32,
                               steps=w.steps, report_every=w.params.report_every)
    precision = {"f32": inp.FP32, "f16": inp.FP16, "bf16": inp.BF16, "f64": inp.FP64,
                 "f16g32": inp.FP16_G32, "bf16g32": inp.BF16_G32}[args.precision]
    streaming = inp.AA if args.streaming == "aa" else inp.PULL
    p = w.params.replace(precision=precision, streaming=streaming)
    h0 = inp.h0_field(w)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
            torch.cuda.synchronize()

    g = LBPC(w.shape, p)
    g.set_initial_h(h0)
    g.step(args.warmup)
    stream = g.stream
    barrier()
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    launches0 = g.launch_count
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    g.step(args.steps)
    e1.record(stream)
    barrier()
    clocks = sampler.stop() if sampler else None
    launches = g.launch_count - launches0
    ms = max_over_ranks(e0.elapsed_time(e1), dist, device="cuda")
    s = g.scalars()
    assert s["nan"] == 0, "diverged during the timed region"
    value = job_mlups(world, w.nodes, args.steps, ms * 1e-3)
    per_rank = job_mlups(1, w.nodes, args.steps, ms * 1e-3)
    del g
    torch.cuda.empty_cache()

    # end to end through the public API: host initial field in, host fields out
    barrier()
    pin_h0 = torch.from_numpy(h0).pin_memory().numpy()
    t0 = time.perf_counter()
    ge = LBPC(w.shape, p)
    ge.set_initial_h(pin_h0)
    ge.step(args.steps)
    out = ge.fields_host(mask=1 | 2)  # T and f_l to host
    sc = ge.scalars()
    torch.cuda.synchronize()
    te = max_over_ranks(time.perf_counter() - t0, dist, device="cuda")
    assert sc["nan"] == 0 and np.isfinite(out["T"]).all()
    del ge
    torch.cuda.empty_cache()

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return
    peak, peak_kind = _peaks()
    bpl = BYTES_PER_LUP[precision]
    achieved = per_rank * 1e6 * bpl / 1e9
    tr = _traffic_per_lup(precision, streaming)
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {inp.FP32: "f32", inp.FP16: "f32 (f16-shifted storage)",
                  inp.BF16: "f32 (bf16-shifted storage)", inp.FP64: "f64",
                  inp.FP16_G32: "f32 (f16-shifted f, f32 g storage)",
                  inp.BF16_G32: "f32 (bf16-shifted f, f32 g storage)"}[precision],
        "data": "synthetic",
        "config": {"workload": w.name + " D3Q19-MRT + D3Q7-MRT", "lattice": list(w.shape),
                   "precision": inp.PRECISION_NAMES[precision],
                   "streaming": "aa" if streaming == inp.AA else "pull",
                   "report_every": p.report_every,
                   "l2": (f"working set {w.nodes * bpl / 1e6:.0f} MB > 129 MB L2 (no flush needed)"
                          if w.nodes * bpl > 129e6 else
                          f"working set {w.nodes * bpl / 1e6:.0f} MB fits in the 129 MB L2 "
                          "(small-lattice case, not an HBM measurement)"),
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_kind,
                     "algorithmic_bytes_per_lup": bpl,
                     "traffic": (tr * w.nodes if tr is not None else None),
                     "traffic_per_lup": tr},
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": {"value": job_mlups(world, w.nodes, args.steps, te), "unit": "MLUPS",
                "h2d_bytes_per_step": 8 * w.nodes / args.steps,
                "d2h_bytes_per_step": (16 * w.nodes + 8 * 9) / args.steps,
                "what": "create + initial h from pinned host + K steps + T, f_l and scalars "
                        "to host, per-step bytes = totals / K"},
    }
    if world == 1 and not args.no_adjoint and streaming == inp.PULL:
        line["adjoint"] = adjoint_ratio(p, w.shape, h0)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f32",
                    choices=["f32", "f16", "bf16", "f64", "f16g32", "bf16g32"])
    ap.add_argument("--streaming", default="pull", choices=["pull", "aa"])
    ap.add_argument("--lattice", type=int, default=256,
                    help="cavity edge (256: the benchmark; 128: profiling; 512: ceiling lines)")
    ap.add_argument("--pr", type=float, default=0.02, help="Prandtl number of the cavity")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    args = ap.parse_args()
    assert args.warmup >= 3, "at least 3 warm-up steps"
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

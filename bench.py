"""Benchmark of the FSLBM step (every sub-step of the method) on one GB300.

Headline workload (default): the dense coalescing foam, 512^3 cells
(134,217,728), periodic in x and y, no-slip bottom wall, lid moving at
u_x = 0.05, gravity 1e-5, sigma = 3e-3, TRT (Lambda = 3/16, tau = 0.8);
lognormal bubble radii (median 8, sigma_log 0.3, clipped to [4, 16]) placed by
random sequential addition toward a gas fraction of 0.4 (seeded synthetic
geometry; the achieved fraction is reported).  FP16-shifted PDF storage with
FP32 collision, against FP32, BF16-shifted and FP64 storage of the same
lattice, each with its mass drift over the run.

One step = stream/bounce-back + mass exchange + reconstruction + collision,
the conversion phases with excess-mass redistribution, the bubble-volume
update, and the merge/split labelling when triggered.  Inputs are resident in
HBM when the timed region starts; the L2 cache (129 MB) is flushed before every
timed step and only the steps are timed, with CUDA events on the stream.  The
first steps of a handle tune the stream-collide kernel's form (they are real
steps); the timed steps come after them and after the warm-up.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision f16s] [--workload foam512]
    python bench.py --impl reference      # the FP64 CPU oracle on the host cores

Under torchrun every rank advances its own independent copy of the lattice
(weak scaling, no collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FSLBM MLUPS & HBM roofline fraction: FP16-store/batched vs plain FP32/FP64"
UNIT = "MLUPS"
BYTES = {"fp64": 8, "fp32": 4, "f16s": 2, "bf16s": 2}
DTYPE = {"fp64": "f64", "fp32": "f32", "f16s": "f32", "bf16s": "f32"}
KERNEL = ("stream-collide work of a step (interface and liquid cells): the tuned form's kernels, "
          "in the 16-bit forms on the foam the normals pass and the tile-fused kernel, timed together")
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "stream_collide_traffic.json")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1604_01632_gb300", "csrc", f) for f in
                  ("fsl_device.cuh", "fsl_fast.cu", "fsl_core.cu")]
CPU_SAMPLE_N = 128        # the oracle's bounded sample: the same foam recipe at 128^3


def workload(name: str):
    from paper_1604_01632_gb300 import scenarios as S
    if name == "foam512":
        sc = S.foam(n=512)
        return sc, ("foam 512^3 TRT tau=0.8 sigma=3e-3 g=1e-5 lid u_x=0.05, lognormal radii (median 8, "
                    "sigma_log 0.3, [4,16]) by RSA toward gas fraction 0.4")
    if name.startswith("foam"):
        n = int(name[4:])
        return S.foam(n=n), f"foam {n}^3 (the 512^3 foam recipe at {n}^3)"
    if name == "gas_thread":
        return S.gas_thread(), "gas_thread 256x64x64 TRT sigma=5e-3 R=8(1+0.1 sin(2 pi x/64))"
    if name == "static_bubble":
        return S.static_bubble(), "static_bubble 32^3 BGK R=8 sigma=1e-3"
    if name == "gas_thread_large":
        return (S.gas_thread(nx=1024, ny=256, nz=256, radius=32.0, wavelength=256.0),
                "gas_thread 1024x256x256 TRT sigma=5e-3 R=32(1+0.1 sin(2 pi x/256))")
    if name == "orifice":
        return S.orifice(), "orifice 128x128x256 TRT g=1e-5 sigma=2e-3 hole r=6"
    raise ValueError(name)


def gas_fraction(sc) -> float:
    """Gas volume (gas cells 1, interface cells 1 - fill) over the lattice."""
    g = np.count_nonzero(sc.flags == 2)
    i = sc.flags == 1
    return float((g + np.sum(1.0 - sc.fill[i])) / sc.n)


def algorithmic_bytes(counts, s: int) -> float:
    """Minimum bytes one stream-collide launch moves: every cell's type byte;
    19 PDFs read and 19 written per liquid or interface cell; per interface cell
    its mass (read + write), fill level, density and mark (37 B)."""
    n_all = float(sum(counts))
    n_liq, n_if = float(counts[0]), float(counts[1])
    return n_all * 1.0 + (n_liq + n_if) * 38.0 * s + n_if * 37.0


def max_over_ranks(x: float, world: int, device: str) -> float:
    """The largest x over the ranks (the slowest rank's time); x itself on one rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(cells_per_rank: int, steps: int, world: int, ms_max: float) -> float:
    """Million lattice-cell updates per second of the whole job: every rank
    advances its own copy of the lattice, the job lasts as long as the slowest."""
    return cells_per_rank * steps * world / (ms_max * 1e-3) / 1e6


def kernel_sha() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def traffic_per_launch(precision: str, wl: str):
    """DRAM bytes per stream-collide launch from the committed ncu summary, if it
    was taken on the current kernel source for this precision and workload."""
    try:
        rec = json.load(open(PROFILE_TRAFFIC))
    except Exception:
        return None
    ent = rec.get(f"{wl}:{precision}")
    if not ent or ent.get("kernel_sha") != kernel_sha():
        return None
    return ent.get("dram_bytes_per_launch")


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), p[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


class L2Flush:
    """Empties the 129 MB L2 before a timed step: a 256 MB write, then (mode
    "write+read") a 256 MB read of a second buffer, so that the lines left in
    L2 are clean and the timed step does not pay for writing back the flush
    buffer's dirty lines."""

    def __init__(self, torch, mode):
        self.mode = mode
        self.torch = torch
        self.w = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        self.r = torch.ones(32 << 20, dtype=torch.int64, device="cuda") if mode == "write+read" else None

    def __call__(self):
        self.w.zero_()
        if self.r is not None:
            self.r.sum()

    def describe(self):
        if self.mode == "write+read":
            return "flushed (256 MB write, then 256 MB read of another buffer: no dirty lines left)"
        return "flushed (256 MB write)"


def tune(sim, limit: int = 64) -> dict:
    """Run the autotuning steps (real steps) until the stream-collide form is
    decided; returns the tuner's record and the number of steps it took."""
    k = 0
    while sim.tuning()["form"] < 0 and k < limit:
        sim.step(1)
        k += 1
    sim.sync()
    rec = sim.tuning()
    rec["steps"] = k
    return rec


def run_gpu(args, rank: int, world: int):
    import torch
    from paper_1604_01632_gb300 import fsl

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    t0 = time.perf_counter()
    sc, wl_desc = workload(args.workload)
    gen_s = time.perf_counter() - t0
    n = sc.n
    stream = torch.cuda.current_stream()

    def make(precision, scen=None):
        sim = fsl.Simulation.from_scenarios([scen or sc], precision=precision, stream=int(stream.cuda_stream))
        if args.no_graphs:
            sim.set_graphs(False)
        if args.stream_form >= 0:
            sim.set_stream_form(args.stream_form)
        return sim

    flush = L2Flush(torch, args.flush)
    meas_peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else None
    peak = float(meas_peaks["hbm_gbs"]) if meas_peaks else 6800.0
    peak_src = "MEASURED_PEAKS.json hbm_gbs (measured)" if meas_peaks else "fallback 6800 GB/s"

    def timed_steps(sim, K, W, timing=True, barrier=False):
        sim.set_timing(timing)
        for _ in range(W):
            flush()
            sim.step(1)
        sim.sync()
        sim.set_timing(timing)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        c0 = sim.cell_counts(0)   # (its export kernel is not a step kernel)
        l0 = sim.launches
        r0 = sim.labelling_runs
        if barrier and world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for k in range(K):
            flush()
            ev[k][0].record()
            sim.step(1)
            ev[k][1].record()
        torch.cuda.synchronize()
        sim.sync()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        k1 = sim.stream_collide_ms()
        launches = sim.launches - l0
        c1 = sim.cell_counts(0)
        return ms, k1, launches, (np.asarray(c0) + np.asarray(c1)) / 2.0, sim.labelling_runs - r0

    def measure(sim, cells, prec, K, W):
        """Uninstrumented step time, then the stream-collide kernel by events,
        and the liquid-mass drift over all steps the handle ran."""
        m0 = sim.total_mass()
        vms, _, _, vc, lr = timed_steps(sim, K, W, timing=False)
        _, vk1, _, _, _ = timed_steps(sim, K, W, timing=True)
        m1 = sim.total_mass()
        vb = algorithmic_bytes(vc, BYTES[prec])
        return {"mlups": round(cells * K / (vms * 1e-3) / 1e6, 1), "ms_per_step": round(vms / K, 5),
                "stream_collide_ms": round(vk1 / K, 5),
                "stream_collide_gbs": round(vb / (vk1 / K * 1e-3) / 1e9, 1),
                "stream_collide_frac": round(vb / (vk1 / K * 1e-3) / 1e9 / peak, 3),
                "labelling_runs_per_step": round(lr / K, 3),
                "mass_drift_rel": float(f"{(m1 - m0) / m0:.3e}")}

    # headline: the requested precision, tuned, then steps timed without instrumentation
    sim = make(args.precision)
    mass0 = sim.total_mass()
    tuning = tune(sim)
    rb0, lr0 = sim.relabelled_bubbles, sim.labelling_runs
    clk = Clocks(dev)
    clk.start()
    ms, _, launches, counts, lruns = timed_steps(sim, args.steps, args.warmup, timing=False, barrier=True)
    clocks = clk.stop()
    # the stream-collide kernel of the same run, timed by CUDA events recorded
    # around it inside each step (a second pass of the same length: the event
    # records add a few microseconds to a step, so they stay out of the headline)
    _, k1_ms, _, _, _ = timed_steps(sim, args.steps, args.warmup, timing=True)
    mass1 = sim.total_mass()
    # bubbles a labelling pass takes: only those phase C marked (out of all)
    relab = (sim.relabelled_bubbles - rb0) / max(1, sim.labelling_runs - lr0)
    steps_run = tuning["steps"] + 2 * (args.steps + args.warmup)
    ms_max = max_over_ranks(ms, world, "cuda")
    value = whole_job_mlups(n, args.steps, world, ms_max)
    s = BYTES[args.precision]
    abytes = algorithmic_bytes(counts, s)
    k1_avg = k1_ms / args.steps
    achieved = abytes / (k1_avg * 1e-3) / 1e9
    traffic = traffic_per_launch(args.precision, args.workload)
    nbub = len(sim.bubbles(0))
    sim.close()

    # the same lattice in the other storage forms (FP32 is the metric's plain baseline)
    variants = {}
    if not args.no_variants and world == 1:
        for prec in ("fp32", "bf16s", "fp64"):
            if prec == args.precision:
                continue
            v = make(prec)
            rec = tune(v)
            K = max(5, args.steps // 2) if prec != "fp64" else max(3, args.steps // 4)
            r = measure(v, n, prec, K, 3)
            r["tuned_form"] = rec["form_name"]
            variants[prec] = r
            v.close()
            torch.cuda.empty_cache()

    # secondary workloads: the 1 M-cell gas thread (latency-dominated) and a
    # batch of 64 bubble-population domains in one handle
    secondary = {}
    if not args.no_secondary and world == 1:
        gsc, gdesc = workload("gas_thread")
        for prec in (args.precision, "fp32"):
            v = make(prec, gsc)
            rec = tune(v)
            r = measure(v, gsc.n, prec, 20, 5)
            r.update({"workload": gdesc, "cells": gsc.n, "tuned_form": rec["form_name"]})
            secondary[f"gas_thread_{prec}"] = r
            v.close()
    batched = None
    if not args.no_batched and world == 1:
        batched = run_batched(args, fsl, torch, stream, flush)

    # end to end through the C ABI from pinned host buffers: upload the initial
    # state, K steps, read back cell types, fill levels, bubble ids and the
    # bubble table
    e2e = None
    if not args.no_e2e:
        def pinned(shape, dtype):
            t = torch.empty(int(np.prod(shape)), dtype=getattr(torch, np.dtype(dtype).name), pin_memory=True)
            return t.numpy().reshape(shape)
        flags, fill = pinned(n, np.uint8), pinned(n, np.float64)
        rho, u = pinned(n, np.float64), pinned(3 * n, np.float64)
        np.copyto(flags, sc.flags.reshape(-1))
        np.copyto(fill, sc.fill.reshape(-1))
        np.copyto(rho, sc.rho.reshape(-1))
        np.copyto(u, sc.u.reshape(-1))
        res = {"flags": pinned(n, np.uint8), "fill": pinned(n, np.float64), "id": pinned(n, np.int64)}
        reps = []
        for _ in range(3):
            sim = fsl.Simulation([sc.params()], precision=args.precision, stream=int(stream.cuda_stream))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sim.init_geometry(0, flags, fill, rho, u)
            for seed, extra, rate, constp in sc.sources:
                sim.set_source(0, seed, extra, rate, constp)
            sim.step(args.steps)
            out = sim.fields(0, ("flags", "fill", "id"), out=res)
            bub = sim.bubbles(0)
            torch.cuda.synchronize()
            reps.append(n * args.steps * world / (time.perf_counter() - t0) / 1e6)
            sim.close()
        h2d = flags.nbytes + fill.nbytes + rho.nbytes + u.nbytes
        d2h = sum(a.nbytes for a in out.values()) + bub.nbytes
        e2e = {"value": round(float(np.median(reps)), 1), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d // args.steps), "d2h_bytes_per_step": int(d2h // args.steps),
               "runs": [round(r, 1) for r in reps],
               "note": f"median of 3 runs; {args.steps} steps per upload and read-back"}
        del flags, fill, rho, u, res

    cpu = cpu_single = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, cpu_single = cpu_baselines(args)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {"workload": wl_desc, "cells": n, "storage": args.precision,
                       "gas_fraction": round(gas_fraction(sc), 4),
                       "bubbles_placed": getattr(sc, "bubbles_placed", None), "bubbles_at_end": nbub,
                       "input_generation_s": round(gen_s, 1),
                       "l2": flush.describe() + " before every timed step (the lattice's working set also "
                             "exceeds L2); steps timed by CUDA events",
                       "parallelism": f"replicas x{world}",
                       "labelling_runs_per_step": round(lruns / args.steps, 3),
                       "bubbles_relabelled_per_pass": round(relab, 1),
                       "cell_counts_liquid_interface_gas_obstacle_lid": [int(c) for c in counts[:5]],
                       "stream_collide_tuning": tuning,
                       "mass_drift_rel": float(f"{(mass1 - mass0) / mass0:.3e}"),
                       "mass_drift_steps": steps_run},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": traffic,
                         "kernel": KERNEL, "algorithmic_bytes_per_launch": int(abytes),
                         "avg_launch_ms": round(k1_avg, 5), "peak_source": peak_src,
                         "timing": "CUDA events on the launching stream around the stream-collide kernel, "
                                   "second timed pass of the same run"},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
            "variants": variants, "secondary": secondary, "batched": batched,
            "cpu_baseline_single_thread": cpu_single,
        }
        print(json.dumps(line))


def run_batched(args, fsl, torch, stream, flush, steps: int = 20):
    """64 domains of 32-96 cells per axis with 20-200 bubbles each, FP16-shifted
    storage: one handle advancing all domains per launch, against a loop over 64
    single-domain handles."""
    from paper_1604_01632_gb300 import scenarios as S
    doms = S.bubble_population(n_domains=64, seed=0)
    cells = sum(d.n for d in doms)
    out = {"domains": len(doms), "cells": cells, "steps": steps, "storage": args.precision}

    def timed(step_fn, sync_fn):
        for _ in range(3):
            flush()
            step_fn()
        sync_fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for k in range(steps):
            flush()
            ev[k][0].record()
            step_fn()
            ev[k][1].record()
        torch.cuda.synchronize()
        sync_fn()
        return sum(a.elapsed_time(b) for a, b in ev)

    sim = fsl.Simulation.from_scenarios(doms, precision=args.precision, stream=int(stream.cuda_stream))
    rec = tune(sim)
    r0, rb0 = sim.labelling_runs, sim.relabelled_bubbles
    ms = timed(lambda: sim.step(1), sim.sync)
    out["batched_mlups"] = round(cells * steps / (ms * 1e-3) / 1e6, 1)
    out["batched_ms_per_step"] = round(ms / steps, 4)
    out["labelling_runs_per_step"] = round((sim.labelling_runs - r0) / (steps + 3), 3)
    out["bubbles_relabelled_per_pass"] = round((sim.relabelled_bubbles - rb0) / max(1, sim.labelling_runs - r0), 1)
    out["bubbles"] = int(sum(len(sim.bubbles(d)) for d in range(len(doms))))
    out["tuned_form"] = rec["form_name"]
    out["tuning_ms_per_form"] = rec["ms_per_form"]
    sim.close()
    sims = [fsl.Simulation.from_scenarios([d], precision=args.precision, stream=int(stream.cuda_stream)) for d in doms]
    for x in sims:
        tune(x)

    def step_all():
        for x in sims:
            x.step(1)

    def sync_all():
        for x in sims:
            x.sync()

    ms = timed(step_all, sync_all)
    out["looped_mlups"] = round(cells * steps / (ms * 1e-3) / 1e6, 1)
    out["looped_ms_per_step"] = round(ms / steps, 4)
    for x in sims:
        x.close()
    return out


def cpu_sample():
    """The oracle's bounded sample of the headline workload: the same foam
    recipe (radii, placement, walls, lid, parameters) on a 128^3 lattice."""
    from paper_1604_01632_gb300 import scenarios as S
    return S.foam(n=CPU_SAMPLE_N)


def cpu_baselines(args, steps_omp: int = 40, steps_single: int = 10):
    """The FP64 oracle as it stands on the host cores: its OpenMP build on all
    cores (os.cpu_count()) and the serial build on one core, on a bounded
    sample of the headline workload (about 10 s of host work each)."""
    from oracle import oracle
    sc = cpu_sample()
    cores = os.cpu_count() or 1
    res = []
    for openmp, steps in ((True, steps_omp), (False, steps_single)):
        try:
            o = oracle.Oracle.from_scenario(sc, openmp=openmp)
        except RuntimeError:
            res.append(None)
            continue
        o.step(1)
        t0 = time.perf_counter()
        o.step(steps)
        dt = time.perf_counter() - t0
        res.append({"value": round(sc.n * steps / dt / 1e6, 3), "unit": UNIT, "cores": cores if openmp else 1,
                    "kind": "oracle",
                    "sample": f"{steps} steps of the foam recipe at {CPU_SAMPLE_N}^3 ({sc.n} cells) after one "
                              f"untimed step, {'OpenMP build, all host cores' if openmp else 'serial build'} "
                              f"({dt:.1f} s)"})
    return res[0] or res[1], res[1]


def run_reference(args, rank: int):
    if rank != 0:
        return
    from oracle import oracle
    sc = cpu_sample()
    cores = os.cpu_count() or 1
    try:
        o = oracle.Oracle.from_scenario(sc, openmp=True)
        kind = "OpenMP build, all host cores"
    except RuntimeError:
        o = oracle.Oracle.from_scenario(sc)
        kind, cores = "serial build (no OpenMP support)", 1
    steps = max(1, args.steps)
    o.step(max(0, args.warmup))
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    value = sc.n * steps / dt / 1e6
    _, wl_desc = ("", "foam 512^3 (headline workload); each reference step is one oracle step of the same foam "
                      f"recipe at {CPU_SAMPLE_N}^3")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": args.warmup, "ms_per_step": round(dt / steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl_desc, "cells": sc.n, "storage": "fp64"},
        "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{steps} timed steps of the {CPU_SAMPLE_N}^3 foam after {args.warmup} untimed, "
                                   f"{kind}"},
        "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="fsl", choices=["fsl", "reference"])
    ap.add_argument("--precision", default="f16s", choices=list(BYTES))
    ap.add_argument("--workload", default="foam512")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-graphs", action="store_true", help="direct kernel launches (for ncu)")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--stream-form", type=int, default=-1,
                    help="fix the stream-collide form (0-8) instead of tuning it (for ncu)")
    ap.add_argument("--flush", default="write+read", choices=["write", "write+read"],
                    help="L2 flush between timed steps")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    from paper_1604_01632_gb300 import build
    build.build()
    run_gpu(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

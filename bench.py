"""Benchmark of the QS-PIC hot path: plasma particle-slice updates per second.

One step = one beam step of the method: a full plasma sweep (every xi slice: push, deposit,
FFT field solves, predictor-corrector for B_perp) followed by the beam push with the deposit
of the next sweep's beam sources.  Workload: the 256x256, 1024-slice, 4-ppc mixed precision
electron-beam run (5.4e8 beam macroparticles), synthetic seeded inputs, state resident in
HBM; by default its 200 beam steps are timed, through the linear stage into saturation
(later steps cost more: the filamented beam's particles gather and deposit away from their
lattice homes), and the first launch's rate is reported beside it.  The steps run through
qsa_advance with pipeline_depth steps in flight per persistent launch (a wavefront in xi;
the same arithmetic as the steps one after the other).  Also
measured: the same workload on the FP64 path, an end-to-end job through host buffers, the
roofline of the dominant kernel (the pipelined launch), and the FP64 oracle on a bounded
sample (CPU baseline).

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank runs an independent replica (the method does not shard; weak
scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2607_24214_b300 import config  # noqa: E402

METRIC = "plasma particle-slice updates/s (push+deposit+field solve), mixed vs FP64"
# ncu summary holding the DRAM bytes of one full pipelined launch of the workload
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "pipe_kernel_c2_linear_launch_dram.md")
WORKLOAD = "c2_mixed_electron_beam_256x256_1024slices"
CPU_SAMPLE_SLICES = 12
REF_BUDGET_S = 150.0  # the reference arm's timed and warm-up steps together


def bytes_per_update(p):
    """Algorithmic HBM bytes per plasma particle-slice update of one beam step (mixed path),
    as the method's data flow fixes them: the plasma state (x, y, u_x, u_y: 4 x 4 B) read and
    written once per slice, the beam state read (32 B) and written (28 B) once per step, the
    beam-source slab (S_b, J_z, J_x, J_y: 16 B per node) written and read, and the field slab
    (six fields: 24 B per node) written and read.  At 4 plasma and 8 beam particles per cell
    that is 688 B per cell per slice, 172 B per update."""
    ppc = p.ppc_plasma_x * p.ppc_plasma_y
    cells = p.nx * p.ny
    plasma = 32.0 * ppc * cells * p.nxi
    nb = sum(p.nx * p.ny * s.ppc_x * s.ppc_y * s.ppc_xi * p.nxi for s in p.species)
    beam = 60.0 * nb
    slabs = (32.0 + 48.0) * cells * p.nxi
    return (plasma + beam + slabs) / (ppc * cells * p.nxi)


def sweep_bytes(p):
    """Algorithmic HBM bytes of one sweep: the plasma state read and written per slice
    (32 B per particle), the beam sources read (16 B per node) and the field slab written
    (24 B per node), counted per slice as the update metric counts them."""
    ppc = p.ppc_plasma_x * p.ppc_plasma_y
    cells = p.nx * p.ny
    return 32.0 * ppc * cells * p.nxi + (16.0 + 24.0) * cells * p.nxi


def pipe_bytes(p, depth):
    """Algorithmic HBM bytes of one pipelined launch of `depth` steps: each step's sweep and
    beam push (sweep_bytes + push_bytes)."""
    return depth * (sweep_bytes(p) + push_bytes(p))


def push_bytes(p):
    """Algorithmic HBM bytes of the beam push of one step: beam state read 32 B and written
    28 B per particle, field slab read (24 B per node), sources written (16 B per node)."""
    nb = sum(p.nx * p.ny * s.ppc_x * s.ppc_y * s.ppc_xi * p.nxi for s in p.species)
    return 60.0 * nb + (24.0 + 16.0) * p.nx * p.ny * p.nxi


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.rows = []
        self.proc = None
        self.idx = gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace('.', '').isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace('.', '').isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = set()
        for r in self.rows:
            for i, n in enumerate(names):
                if len(r) > 5 + i and r[5 + i].lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


def dist_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def updates_per_step(p):
    return p.plasma_per_slice() * p.nxi


def time_advance(q, steps, warmup, depth, torch, stream):
    """Warm up, then time `steps` beam steps through qsa_advance (launches of `depth` steps)
    with CUDA events on the library's stream.  Returns (total ms, per-launch ms of the
    persistent kernel, launches of the library's kernels)."""
    q.advance(warmup)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    l0 = q.launch_count()
    t0.record(stream)
    q.advance(steps)
    t1.record(stream)
    t1.synchronize()
    torch.cuda.synchronize()
    return t0.elapsed_time(t1), q.launch_times(), q.launch_count() - l0


def time_steps(q, p, steps, warmup, torch, stream, extra=None):
    """Warm up, then time `steps` beam steps with CUDA events on the library's stream; also
    the sweep and push launches separately.  Returns (total ms, sweep ms list, push ms list,
    launches)."""
    for _ in range(warmup):
        q.sweep()
        q.beam_step()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    l0 = q.launch_count()
    t0.record(stream)
    for k in range(steps):
        ev[k][0].record(stream)
        q.sweep()
        ev[k][1].record(stream)
        q.beam_step()
        ev[k][2].record(stream)
        if extra:
            extra()
    t1.record(stream)
    t1.synchronize()
    torch.cuda.synchronize()
    launches = q.launch_count() - l0
    sw = [ev[k][0].elapsed_time(ev[k][1]) for k in range(steps)]
    pu = [ev[k][1].elapsed_time(ev[k][2]) for k in range(steps)]
    return t0.elapsed_time(t1), sw, pu, launches


def oracle_sample_beam(p, slices):
    """The synthetic beam particles of the first slices + 2 xi cells (the oracle's sample)."""
    from paper_2607_24214_b300 import inputs
    per_layer = p.nx * p.ny * p.species[0].ppc_x * p.species[0].ppc_y * p.species[0].ppc_xi
    return inputs.beam_arrays(p, 0, 0, (slices + 2) * per_layer)


def cpu_baseline(p, slices=CPU_SAMPLE_SLICES, sub=None):
    """The FP64 oracle, as it stands, on the first `slices` slices of one sweep of the same
    workload (the particles of the first xi cells only: the slice loop is sequential in xi).
    sub: those particles, when already generated (oracle_sample_beam)."""
    from oracle import qspic
    if sub is None:
        sub = oracle_sample_beam(p, slices)
    t = time.perf_counter()
    src = qspic.beam_sources(p, [sub], n_nodes=slices + 2)
    qspic.plasma_sweep(p, src, n_slices=slices)
    dt = time.perf_counter() - t
    return p.plasma_per_slice() * slices / dt, dt


def _cpu_sample(args):
    """One oracle sample in a worker process (one thread): updates and seconds."""
    import os as _os
    _os.environ["OMP_NUM_THREADS"] = "1"
    p, slices = args
    return cpu_baseline(p, slices)


def cpu_baseline_all_cores(p, slices=CPU_SAMPLE_SLICES, max_procs=16):
    """The same oracle sample run in one process per core (spawned, one thread each, up to
    max_procs), all at once: the aggregate updates/s of the host's cores on independent
    samples (the slice loop of one sweep is sequential, so independent samples are how the
    oracle uses more cores).  Returns (updates/s, processes, seconds)."""
    import multiprocessing as mp
    try:
        ncore = len(os.sched_getaffinity(0))
    except AttributeError:
        ncore = os.cpu_count() or 1
    nproc = max(1, min(ncore, max_procs))
    ctx = mp.get_context("spawn")
    with ctx.Pool(nproc) as pool:
        pool.map(_cpu_sample, [(p, 1)] * nproc)  # start-up and imports outside the timing
        t = time.perf_counter()
        res = pool.map(_cpu_sample, [(p, slices)] * nproc)
        dt = time.perf_counter() - t
    ups = sum(p.plasma_per_slice() * slices for _ in res)
    return ups / dt, nproc, dt, ncore


def cpu_c1_full():
    """The oracle on the whole C1 run (32 x 32, 64 slices, 10 beam steps and the final sweep),
    one thread: updates/s and seconds."""
    from oracle import qspic
    from paper_2607_24214_b300 import inputs
    p = config.c1_fp64_electron_beam()
    beams = inputs.all_beams(p)
    t = time.perf_counter()
    qspic.run(p, beams, p.steps)
    dt = time.perf_counter() - t
    return p.plasma_per_slice() * p.nxi * p.steps / dt, dt


def run_reference(args, p):
    """The reference arm: the FP64 oracle, as it stands, on this host's cores, for the same
    metric and workload.  Each of the --warmup untimed and --steps timed steps is one oracle
    sample (the first slices of one sweep); unless --ref-slices fixes it, the sample is sized
    from a one-slice probe so that all the steps take about REF_BUDGET_S seconds."""
    rank, world, _ = dist_info()
    if rank != 0:
        return
    steps, warmup = max(args.steps, 1), max(args.warmup, 0)
    slices = args.ref_slices
    if slices <= 0:
        _, t1 = cpu_baseline(p, 1)  # untimed probe
        slices = int(max(1, min(CPU_SAMPLE_SLICES, REF_BUDGET_S / ((steps + warmup) * t1))))
    sub = oracle_sample_beam(p, slices)  # the inputs, generated once
    for _ in range(warmup):
        cpu_baseline(p, slices, sub)
    vals = []
    t0 = time.perf_counter()
    for _ in range(steps):
        v, _ = cpu_baseline(p, slices, sub)
        vals.append(v)
    wall = time.perf_counter() - t0
    val = float(np.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "updates/s",
            "n_gpus": args.gpus, "steps": steps, "warmup": warmup,
            "ms_per_step": 1e3 * wall / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"first {slices} slices"},
            "cpu_baseline": {"value": val, "unit": "updates/s", "cores": 1, "kind": "oracle",
                             "sample": f"first {slices} of {p.nxi + 1} slices of one sweep "
                                       f"per step, {p.nx}x{p.ny}, numpy FP64"},
            "e2e": {"value": val, "unit": "updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def kernel_sources_sha256() -> str:
    """SHA-256 over the library's CUDA sources (csrc/*.cu, *.cuh, *.h, in name order)."""
    import hashlib
    d = os.path.join(ROOT, "paper_2607_24214_b300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".h")):
            h.update(name.encode())
            with open(os.path.join(d, name), "rb") as f:
                h.update(f.read())
    return h.hexdigest()


def measured_traffic(p, steps_per_launch):
    """DRAM bytes (read + write) of one full pipelined launch, from the committed ncu summary,
    when that capture was taken on these kernel sources, this grid and this launch length;
    else None (the counters no longer describe the kernel that ran)."""
    try:
        with open(TRAFFIC_FILE) as f:
            lines = f.read().splitlines()
    except OSError:
        return None
    kv = {}
    for ln in lines:
        if ln.startswith("- ") and ": " in ln:
            k, v = ln[2:].split(": ", 1)
            kv[k.strip()] = v.strip()
    want = f"nx {p.nx}, ny {p.ny}, nxi {p.nxi}, steps per launch {steps_per_launch}"
    if kv.get("kernel sources sha256") != kernel_sources_sha256() or kv.get("workload") != want:
        return None
    try:
        return float(kv["dram bytes per launch"])
    except (KeyError, ValueError):
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200,
                    help="timed beam steps (the workload's 200: the linear stage and saturation)")
    ap.add_argument("--depth", type=int, default=16, help="beam steps in flight per launch")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=16,
                    help="FP64 steps, pipelined as deep as the mixed run (at most --depth)")
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-c3", action="store_true",
                    help="skip the full-size pair-beam workload (224 GB on the device)")
    ap.add_argument("--batch-steps", type=int, default=42,
                    help="timed steps of the batched C4 scan after its 8 untimed autotuning "
                         "steps (42: the scan's 50 steps in all)")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--ref-slices", type=int, default=0,
                    help="slices of the oracle sample per reference step (0: sized so that "
                         "the reference arm's steps take about REF_BUDGET_S seconds)")
    ap.add_argument("--nxi", type=int, default=0,
                    help="override the number of slices (small profiling cases only)")
    args = ap.parse_args()
    p = config.c2_mixed_electron_beam().with_(pipeline_depth=args.depth)
    if args.nxi:
        p = p.with_(nxi=args.nxi, Lxi=p.dxi * args.nxi)
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    if args.impl == "reference":
        run_reference(args, p)
        return
    import torch

    from paper_2607_24214_b300.qsa import QSA
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    q = QSA(p)
    ups = updates_per_step(p)
    barrier(world)
    if args.depth > 1:
        with Clocks(local) as clk:
            ms, lt, launches = time_advance(q, args.steps, args.warmup, args.depth, torch,
                                            stream)
        barrier(world)
        ms = max_over_ranks(ms, world)
        value = ups * args.steps * world / (ms * 1e-3)
        # dominant kernel: the persistent pipelined launch (all but a few memsets of the
        # step); its full launches (depth steps each) give the per-launch duration
        full = [t for i, t in enumerate(lt) if (i + 1) * args.depth <= args.steps]
        dom_ms = float(np.mean(full if full else lt))
        dom_steps = args.depth if full else args.steps
        achieved = pipe_bytes(p, dom_steps) / (dom_ms * 1e-3) / 1e9
        traffic = measured_traffic(p, dom_steps)
        roof = {"bound": "hbm", "kernel": "pipe_kernel", "achieved": achieved,
                "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": traffic,
                "traffic_launch": ("the first timed launch (linear stage), one ncu capture of "
                                   "these kernel sources" if traffic is not None else None),
                "algorithmic_bytes": pipe_bytes(p, dom_steps),
                "peak_source": peak_src, "launch_ms": dom_ms,
                "steps_per_launch": dom_steps, "kernel_share": float(np.sum(lt)) / ms,
                "step_frac": bytes_per_update(p) * value / world / 1e9 / hbm_peak,
                "launch_ms_each": [round(float(t), 1) for t in lt]}
        # the first launch covers the linear stage only (the steps right after the warm-up);
        # later steps cost more once the beam has filamented and its particles have left
        # their lattice homes
        first_ms = float(lt[0]) if len(lt) else ms
        first_steps = min(args.depth, args.steps)
        first = {"steps": first_steps, "ms_per_step": first_ms / first_steps,
                 "value": ups * first_steps / (first_ms * 1e-3)}
    else:
        with Clocks(local) as clk:
            ms, sw, pu, launches = time_steps(q, p, args.steps, args.warmup, torch, stream)
        first = None
        barrier(world)
        ms = max_over_ranks(ms, world)
        value = ups * args.steps * world / (ms * 1e-3)
        sw_ms, pu_ms = float(np.mean(sw)), float(np.mean(pu))
        if sw_ms >= pu_ms:
            dom, dom_ms, dom_bytes = "sweep_kernel", sw_ms, sweep_bytes(p)
        else:
            dom, dom_ms, dom_bytes = "beam_push_kernel", pu_ms, push_bytes(p)
        achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm_peak,
                "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": None,
                "peak_source": peak_src,
                "step_frac": bytes_per_update(p) * value / world / 1e9 / hbm_peak,
                "sweep_ms": sw_ms, "push_ms": pu_ms}
    d = q.diagnostics()
    q.close()
    del q
    torch.cuda.empty_cache()

    line = {"metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": p.nx, "ny": p.ny, "nxi": p.nxi,
                       "ppc_plasma": 4, "ppc_beam": 8, "beam_particles": 8 * p.nx * p.ny * p.nxi,
                       "n_pc_iter": p.n_pc_iter, "precision": "mixed",
                       "pipeline_depth": args.depth,
                       "l2": "inputs larger than L2 (15 GB beam state)",
                       "parallelism": f"replicas{world}"},
            "gpu_launches": launches, "roofline": roof,
            "clocks": clk.summary(), "status": d["status"]}
    if first is not None:
        line["first_launch"] = first

    if not args.no_fp64:
        # the FP64 path, pipelined as deep as the mixed run (137 GB on the device at depth 16)
        d64 = min(args.fp64_steps, args.depth)
        p64 = p.with_(precision="fp64", pipeline_depth=d64)
        q = QSA(p64)
        ms64, _, _ = time_advance(q, args.fp64_steps, 1, d64, torch, stream)
        q.close()
        del q
        torch.cuda.empty_cache()
        v64 = ups * args.fp64_steps / (ms64 * 1e-3)
        line["fp64"] = {"value": v64, "unit": "updates/s", "steps": args.fp64_steps,
                        "pipeline_depth": d64, "ms_per_step": ms64 / args.fp64_steps,
                        "speedup_mixed_over_fp64": ((first["value"] if first else value) / v64),
                        "speedup_basis": "mixed rate of the first pipelined launch (the same "
                                         "linear-stage steps as the FP64 run)"}

    if not args.no_e2e:
        line["e2e"] = e2e(p, args.e2e_steps, torch, stream)

    if not args.no_batch:
        line["batched"] = batched(args.batch_steps, torch, stream, hbm_peak)

    if not args.no_c3:
        line["pair_beam"] = pair_beam(torch, stream)
        line["pair_beam_8ppc"] = pair_beam(torch, stream, steps=3, ppc_xi=2)

    if not args.no_adjoint:
        line["adjoint"] = adjoint_cost(torch, stream)

    if rank == 0 and not args.no_cpu:
        v, dt = cpu_baseline(p)
        line["cpu_baseline"] = {"value": v, "unit": "updates/s", "cores": 1, "kind": "oracle",
                                "sample": f"first {CPU_SAMPLE_SLICES} of {p.nxi + 1} slices of "
                                          f"one sweep of the same workload ({dt:.1f} s)"}
        va, nproc, dta, ncore = cpu_baseline_all_cores(p)
        line["cpu_baseline"]["all_cores"] = {
            "value": va, "unit": "updates/s", "cores": nproc, "host_cores": ncore,
            "sample": f"the same sample in {nproc} spawned one-thread processes at once "
                      f"({dta:.1f} s)"}
        vc, dtc = cpu_c1_full()
        line["cpu_baseline"]["c1_full_run"] = {
            "value": vc, "unit": "updates/s", "cores": 1,
            "sample": f"the whole 32x32, 64-slice, 10-step FP64 run ({dtc:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def pair_beam(torch, stream, steps=6, depth=1, ppc_xi=1, warmup=3):
    """The full-size pair-beam workload (512 x 512, 2048 slices, electrons and positrons):
    `steps` timed beam steps after `warmup` untimed ones (the linear stage).  Same metric.
    ppc_xi = 1: 4 beam ppc per species (4.3e9 beam particles, 155 GB on the device); ppc_xi =
    2: the workload's 8 per species (8.6e9 particles, 28 bytes each, 275 GB).  Depth 1: a
    512^2 slice fills the GPU by itself, and deeper pipelines were slower (1.12-1.15 against
    0.93 s per step at 4 ppc)."""
    from paper_2607_24214_b300.qsa import QSA
    p = config.c3_pair_beam(ppc_xi=ppc_xi).with_(pipeline_depth=depth)
    name = "c3_pair_beam_512x512_2048slices" + ("_8ppc" if ppc_xi == 2 else "")
    torch.cuda.empty_cache()
    try:
        q = QSA(p)
    except Exception as e:  # a device with less free memory than the workload needs
        return {"workload": name, "unavailable": str(e)[:200]}
    dev = q.device_bytes()
    q.advance(warmup)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    q.advance(steps)
    t1.record(stream)
    t1.synchronize()
    ms = t0.elapsed_time(t1)
    st = q.diagnostics()["status"]
    q.close()
    del q
    torch.cuda.empty_cache()
    nb = sum(p.nx * p.ny * sp.ppc_x * sp.ppc_y * sp.ppc_xi * p.nxi for sp in p.species)
    return {"workload": name, "value": updates_per_step(p) * steps / (ms * 1e-3),
            "unit": "updates/s", "steps": steps, "warmup": warmup, "pipeline_depth": depth,
            "ms_per_step": ms / steps, "beam_particles": nb, "device_bytes": dev,
            "status": st}


def batched(steps, torch, stream, hbm_peak):
    """The batched parameter scan (64 instances of uneven grids, qsa_advance_batch): 8 untimed
    steps (the first four time the FFT unit shapes), then `steps` timed steps of all
    instances (8 + 42: the scan's 50).  Same metric: plasma particle-slice updates of all
    instances per second.  Roofline of the batched launches: the algorithmic bytes of the
    sweeps and pushes of their instances over the mean launch time (CUDA events)."""
    from paper_2607_24214_b300.qsa import QSA, advance_batch, batch_graphs
    ps = config.c4_parameter_scan()
    qs = [QSA(pi) for pi in ps]
    advance_batch(qs, 8)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    advance_batch(qs, steps)
    t1.record(stream)
    t1.synchronize()
    ms = t0.elapsed_time(t1)
    lt = qs[0].launch_times()   # the launches of the last call (up to 64)
    replays = batch_graphs(qs[0])  # steps run as CUDA graphs so far
    status = min(q.diagnostics()["status"] for q in qs)
    for q in qs:
        q.close()
    del qs
    torch.cuda.empty_cache()
    ups = sum(updates_per_step(pi) for pi in ps)
    # launches per step: instances in groups of up to 16; the bytes of one step of all
    # instances spread over those launches
    per_step = (len(ps) + 15) // 16
    step_bytes = sum(sweep_bytes(pi) + push_bytes(pi) for pi in ps)
    out = {"workload": "c4_parameter_scan_64", "value": ups * steps / (ms * 1e-3),
           "unit": "updates/s", "instances": len(ps), "steps": steps, "untimed_steps": 8,
           "ms_per_step": ms / steps, "grids": sorted({pi.nx for pi in ps}),
           "graph_replays": replays, "status": status}
    if len(lt):
        launch_ms = float(np.mean(lt))
        achieved = step_bytes / per_step / (launch_ms * 1e-3) / 1e9
        out["roofline"] = {"bound": "hbm", "kernel": "pipe_kernel (independent instances)",
                           "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                           "frac": achieved / hbm_peak,
                           "algorithmic_bytes_per_step": step_bytes,
                           "launches_per_step": per_step, "launch_ms": launch_ms,
                           "launches_timed": int(len(lt))}
    return out


def adjoint_cost(torch, stream, steps=None, ckpt=10):
    """The seeded-mode workload (128 x 128, 256 slices, 16 modes, 50 beam steps): the forward
    run as the library runs it (mixed precision, pipelined, one qsa_advance), the recorded
    FP64 forward of the gradient (qsa_grad_forward) and its backward pass (qsa_grad_backward:
    checkpoint segments recomputed and recorded, adjoint sweeps and beam pushes), wall times
    with the device synchronised."""
    from paper_2607_24214_b300.qsa import QSA
    p = config.c5_seeded_modes()
    steps = p.steps if steps is None else steps
    q = QSA(p.with_(pipeline_depth=16))
    torch.cuda.synchronize()
    t = time.perf_counter()
    q.advance(steps)
    q.sweep()
    q.diagnostics()
    t_mixed = time.perf_counter() - t
    q.close()
    q = QSA(p.with_(precision="fp64"))
    torch.cuda.synchronize()
    t = time.perf_counter()
    loss = q.grad_forward(steps, ckpt)
    t_fwd = time.perf_counter() - t
    t = time.perf_counter()
    dm, da = q.grad_backward(1.0)
    t_bwd = time.perf_counter() - t
    q.close()
    del q
    torch.cuda.empty_cache()
    return {"workload": "c5_seeded_modes_128x128_256slices_16modes", "steps": steps,
            "step_checkpoints": ckpt, "loss": loss, "forward_mixed_s": t_mixed,
            "forward_fp64_recorded_s": t_fwd, "backward_s": t_bwd,
            "backward_over_forward_fp64": t_bwd / t_fwd,
            "backward_over_forward_mixed": t_bwd / t_mixed,
            "grad_alpha": float(da[0]), "grad_mode0": float(dm[0])}


def e2e(p, steps, torch, stream):
    """Same metric for a whole job through the public API, from host data to host results:
    the beam state goes up from pinned host memory (qsa_set_beam), `steps` beam steps run
    (qsa_advance), and the per-slice diagnostics of the last sweep (qsa_diagnostics) and the
    final beam state (qsa_get_beam) come back; all inside the timed region.  Bytes per step
    are the job's copies divided by its steps."""
    from paper_2607_24214_b300.qsa import QSA
    q = QSA(p)
    n = p.nx * p.ny * p.nxi * 8
    keys = ("x", "y", "xi", "ux", "uy", "uz", "w")
    host = {k: torch.empty(n, dtype=torch.float64, pin_memory=True).numpy() for k in keys}
    back = {k: torch.empty(n, dtype=torch.float64, pin_memory=True).numpy() for k in keys}
    import ctypes as ct
    from paper_2607_24214_b300.qsa import _ptr
    nout = ct.c_int64()
    q._check(q.lib.qsa_get_beam(q.h, 0, n, *[_ptr(host[k]) for k in keys], ct.byref(nout)))
    # one untimed step (allocator warm-up)
    q.set_beam(0, host)
    q.advance(1)
    q.diagnostics()
    torch.cuda.synchronize()
    t = time.perf_counter()
    q.set_beam(0, host)
    q.advance(steps)
    q.diagnostics()
    q._check(q.lib.qsa_get_beam(q.h, 0, n, *[_ptr(back[k]) for k in keys], ct.byref(nout)))
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    q.close()
    del q
    torch.cuda.empty_cache()
    diag_bytes = (p.nxi + 1) * 15 * 8
    beam_bytes = 7 * 8 * n
    return {"value": updates_per_step(p) * steps / dt, "unit": "updates/s",
            "h2d_bytes_per_step": beam_bytes // steps,
            "d2h_bytes_per_step": (beam_bytes + diag_bytes) // steps, "steps": steps,
            "job": "set_beam + advance(steps) + diagnostics + get_beam"}


if __name__ == "__main__":
    main()

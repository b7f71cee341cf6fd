#!/usr/bin/env python
"""Benchmark of the fused fluctuating-LB step: two-species D2Q9 GLUPS and the fraction of the
HBM roofline, FP32-deviation batched ensemble against the plain FP64 path on the same GPU.

One benchmark step = one sampling period of the batched ensemble: 100 lattice-Boltzmann steps
of all 768 lattices (64 seeds x Lz in {32, 64, 128, 256} with Lx = 4 Lz x wall-to-wall
difference in {0.1, 0.3, 0.5}; 66,846,720 sites), the first of them a sample step (fields,
pressure and mass sums, row and column FFTs, compensated accumulation).  The state (9.6 GB) is
far larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own ensemble (other seeds): weak scaling, no
collective on the data path; the timed region is bracketed by barriers and the maximum over
ranks is reported.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LB_STEPS_PER_STEP = 100          # one sampling period
BYTES_PER_SITE = {"dev32": 144, "fp64": 288}  # 18 populations read + 18 written per lattice update


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 / large-lattice / e2e / CPU legs")
    ap.add_argument("--profile-small", action="store_true",
                    help="run a small single-lattice case only (for ncu captures)")
    ap.add_argument("--profile-kT", type=float, default=1e-5, help="kT of the small case")
    ap.add_argument("--profile-persistent", action="store_true", help="ensemble case as one persistent launch")
    ap.add_argument("--profile-no-tensor-maps", action="store_true", help="ensemble case with 1-d bulk copies only")
    ap.add_argument("--profile-precision", default="dev32", choices=["dev32", "fp64"])
    ap.add_argument("--profile-generic", action="store_true", help="small case with per-thread staging")
    ap.add_argument("--profile-tile", type=int, default=128, help="tile width of the small case")
    ap.add_argument("--profile-rows", type=int, default=None,
                    help="rows per block of the profiling cases (default 64 small, 256 ensemble)")
    ap.add_argument("--profile-ensemble", type=int, default=0,
                    help="run the ensemble with this many seeds for 6 steps (for ncu captures)")
    ap.add_argument("--profile-adjoint", action="store_true",
                    help="one mean-pressure-shift gradient on the 256 x 128 lattice (2000 steps, checkpoints "
                         "every 100), in --profile-precision (for ncu captures)")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks during the timed region
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


KERNEL_SOURCES = ("lb_step_impl.cuh", "lb_internal.cuh")


def kernel_code_hash():
    """sha256 of the step kernels' sources (the kernel and the layouts and device helpers it
    includes) with comments and blank lines removed (a comment edit does not change the kernel)."""
    lines = []
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1808_05168_gb300", "csrc", name)) as f:
            for ln in f.read().splitlines():
                i = ln.find("//")
                ln = (ln if i < 0 else ln[:i]).rstrip()
                if ln:
                    lines.append(ln)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


C3_WORKLOAD = ("c3 batched ensemble: 64 seeds x Lz {32,64,128,256} (Lx=4Lz) x dc {0.1,0.3,0.5}, G=0.5, "
               "kT=1e-5; 768 lattices, 66,846,720 sites per rank")


def kernel_traffic(kind):
    """DRAM bytes per LB step of the dominant kernel at full size from the committed ncu summary,
    if it was taken on the current kernel source (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "persistent_kernel_bulk_traffic_c3.json")) as f:
            d = json.load(f)
        if d.get("kernel_code_sha256") != kernel_code_hash():
            return None
        e = d.get(kind)
        return None if e is None else float(e["bytes_per_step_full_size"])
    except Exception:
        return None


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import torch

    from paper_1808_05168_gb300 import Simulation, workloads

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_1808_05168_gb300.ensemble import seeds_for_rank

    P = LB_STEPS_PER_STEP
    lattices = workloads.c3(seed0=seeds_for_rank(rank, 64).start)
    sites = workloads.sites(lattices)
    stream = torch.cuda.Stream()
    sim = Simulation(lattices, precision="dev32", graph=True, persistent=True, autotune=True)
    sim.set_stream(stream)
    sim.set_sampling(0, P)
    for _ in range(args.warmup):
        sim.step(P)
    sim.synchronize()

    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local)
    launches0 = sim.kernel_launches()
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    with torch.cuda.stream(stream):
        e0.record(stream)
        for k in range(K):
            sim.step(1)                 # the sample step of the period
            ev[k][0].record(stream)
            sim.step(P - 1)             # plain steps: one persistent launch of the dominant kernel
            ev[k][1].record(stream)
        e1.record(stream)
    sim.synchronize()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = sim.kernel_launches() - launches0
    ms = e0.elapsed_time(e1)
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    step_kernel_ms = statistics.mean(a.elapsed_time(b) for a, b in ev) / (P - 1)
    glups = world * sites * P * K / (ms / 1e3) / 1e9
    peak, peak_kind = peaks()
    achieved = BYTES_PER_SITE["dev32"] * sites / (step_kernel_ms / 1e3) / 1e9
    tile = sim.tile()
    res = {
        "metric": "two-species D2Q9 GLUPS (FP32-deviation batched ensemble)",
        "value": glups,
        "unit": "GLUPS",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": ms / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": C3_WORKLOAD,
                   "lb_steps_per_step": P, "sample_every": P, "precision": "dev32 (f32 deviations, f64 sums)",
                   "launch": "CUDA graph per period: the sample step and its kernels, then one persistent launch "
                             "of the 99 plain steps (items handed out in order, per-item dependencies)",
                   "tile": {"tile_x": tile[0], "rows": tile[1]},
                   "l2": "state 9.6 GB >> 129 MB L2; no flush needed", "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": kernel_traffic("dev32_c3"),
                     "kernel": "persistent_kernel_bulk<float,128,hom noise> (tile the autotuner picked); 99 LB steps "
                               "per launch: achieved, traffic and kernel_ms are per LB step",
                     "peak_source": f"hbm_gbs ({peak_kind})",
                     "kernel_ms": step_kernel_ms, "bytes_per_step": BYTES_PER_SITE["dev32"] * sites},
        "clocks": clk,
        "gpu_launches": launches,
    }
    sim.close()
    del sim
    torch.cuda.synchronize()

    if not args.no_extras and rank == 0:
        res["fp64_plain"] = measure_plain(torch, workloads.c4(), "fp64", steps=10)
        res["fp64_plain"]["roofline"] = fp64_roofline(res["fp64_plain"]["GLUPS"])
        res["fp64_plain"]["GLUPS_one_launch_per_step"] = measure_plain(torch, workloads.c4(), "fp64", steps=10,
                                                                       persistent=False)["GLUPS"]
        res["dev32_large"] = measure_plain(torch, workloads.c4(), "dev32", steps=40)
        res["c2_sampled"] = {prec: measure_sampled(torch, workloads.c2(), prec) for prec in ("dev32", "fp64")}
        res["e2e"] = measure_e2e(torch, lattices, K, P)
        res["adjoint_c5"] = measure_adjoint(torch)
        res["cpu_baseline"] = cpu_baseline()
    elif not args.no_extras:
        res["e2e"] = measure_e2e(torch, lattices, K, P)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(res))


# Double-precision arithmetic instructions (DFMA + DADD + DMUL, each one issue of the FP64 pipe)
# per lattice update of the FP64 step kernel, from ncu's sm__sass_thread_inst_executed_op_d*
# counters (profiles/step_kernel_bulk_f64_small.md).
FP64_INSTR_PER_LU = 428.4


def fp64_roofline(glups):
    """The FP64 path is bound by its double-precision arithmetic: its FP64 instruction rate against
    the device's FP64 FMA issue rate, measured live by the library (lb_debug_fma_rate)."""
    from paper_1808_05168_gb300 import capi

    peak = capi.lb_debug_fma_rate(capi.LB_PREC_FP64) / 2 / 1e12  # FMA instructions per second, 1e12
    achieved = FP64_INSTR_PER_LU * glups * 1e9 / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T FP64 instructions/s",
            "frac": achieved / peak, "fp64_instr_per_lu": FP64_INSTR_PER_LU,
            "peak_source": "measured DFMA rate (lb_debug_fma_rate), 2 flops per DFMA"}


def measure_adjoint(torch):
    """The gradient of the mean-pressure shift on the 256 x 128 lattice (2000 steps from rest,
    checkpoints every 100): wall time of the two forward runs alone and of forward + reverse
    sweep, per precision."""
    from paper_1808_05168_gb300 import Simulation, workloads

    (p,) = workloads.c5()
    out = {"workload": "256x128, G=0.5, dc=0.5, kT=1e-5, 2000 steps, checkpoints every 100"}
    for prec in ("fp64", "dev32"):
        with Simulation(p, precision=prec) as sim:
            sim.pressure_shift_gradient(100, 100)  # set-up and first-use costs
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sim.pressure_shift_gradient(2000, 100, want_grad=False)
            t1 = time.perf_counter()
            sim.pressure_shift_gradient(2000, 100)
            t2 = time.perf_counter()
        out[prec] = {"loss_only_s": t1 - t0, "loss_and_gradient_s": t2 - t1, "ratio": (t2 - t1) / (t1 - t0)}
    # 16 seeds of the same lattice in one sweep (each its own loss and gradient)
    from dataclasses import replace
    ps = [replace(p, seed=p.seed + k, lattice_id=k) for k in range(16)]
    with Simulation(ps, precision="dev32") as sim:
        sim.pressure_shift_gradients(100, 100)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.pressure_shift_gradients(2000, 100)
        t1 = time.perf_counter()
    out["dev32_batch16"] = {"lattices": 16, "loss_and_gradient_s": t1 - t0, "per_lattice_s": (t1 - t0) / 16}
    return out


def measure_plain(torch, lattices, precision, steps, persistent=True):
    """Plain steps of one large lattice (no sampling), one persistent launch or one launch per
    step: GLUPS and HBM fraction."""
    from paper_1808_05168_gb300 import Simulation, workloads

    sites = workloads.sites(lattices)
    stream = torch.cuda.Stream()
    with Simulation(lattices, precision=precision, autotune=True, persistent=persistent) as sim:
        sim.set_stream(stream)
        sim.step(3)
        sim.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            sim.step(steps)
            b.record(stream)
        sim.synchronize()
        ms = a.elapsed_time(b) / steps
        peak, _ = peaks()
        gbs = BYTES_PER_SITE[precision] * sites / (ms / 1e3) / 1e9
        Lx, Lz = sim.shape(0)
        return {"workload": f"{Lx}x{Lz} single lattice, G=0.5, dc=0.5, kT=1e-5", "precision": precision,
                "launch": "persistent" if persistent else "one per step",
                "GLUPS": sites / (ms / 1e3) / 1e9, "ms_per_lb_step": ms, "hbm_GBps": gbs, "hbm_frac": gbs / peak,
                "tile": list(sim.tile())}


def measure_sampled(torch, lattices, precision, periods=10, every=100):
    """A single production run as the paper's (the 512 x 256 lattice, a sample of every
    diagnostic every 100 steps, CUDA graphs and the persistent launch, autotuned tile): GLUPS
    including the sample steps and their transforms.  The state (9.4 MB in FP32) stays in L2, so
    this is not an HBM-roofline figure."""
    from paper_1808_05168_gb300 import Simulation, workloads

    sites = workloads.sites(lattices)
    stream = torch.cuda.Stream()
    with Simulation(lattices, precision=precision, graph=True, persistent=True, autotune=True) as sim:
        sim.set_stream(stream)
        sim.set_sampling(0, every)
        sim.step(3 * every)
        sim.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            sim.step(periods * every)
            b.record(stream)
        sim.synchronize()
        ms = a.elapsed_time(b) / (periods * every)
        Lx, Lz = sim.shape(0)
        return {"workload": f"{Lx}x{Lz} single lattice, sample every {every} steps", "GLUPS": sites / (ms / 1e3) / 1e9,
                "ms_per_lb_step": ms, "tile": list(sim.tile())}


def measure_e2e(torch, lattices, K, P):
    """The same work through the public API from host buffers: create the ensemble from the host
    parameter table, run K sampling periods, read every lattice's q_z = 0 concentration structure
    factor and mean pressure back to host memory."""
    import numpy as np

    from paper_1808_05168_gb300 import Simulation, capi, workloads

    sites = workloads.sites(lattices)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim = Simulation(lattices, precision="dev32", graph=True, persistent=True, autotune=True)
    sim.set_sampling(0, P)
    for _ in range(K):
        sim.step(P)
    d2h = 0
    for i, p in enumerate(lattices):
        s, _ = sim.structure_factor("c", lattice=i, qz0_only=True)
        sim.mean_pressure(i)
        d2h += s.nbytes + 16
    t1 = time.perf_counter()
    sim.close()
    h2d = len(lattices) * np.dtype(np.uint8).itemsize * __import__("ctypes").sizeof(capi.lb_params)
    return {"value": sites * K * P / (t1 - t0) / 1e9, "unit": "GLUPS", "h2d_bytes_per_step": h2d / K,
            "d2h_bytes_per_step": d2h / K, "seconds": t1 - t0,
            "what": "lb_create_batch from host params + K x lb_step(100) + lb_structure_factor/lb_mean_pressure "
                    "of every lattice to host"}


def _oracle_member(omp):
    """The oracle on the largest member of the ensemble (1024 x 256 sites, wall-to-wall difference
    0.5): the plain build (one core) or the OpenMP build of the same source (its row loops on
    every host core; bit-identical results)."""
    import oracle
    from paper_1808_05168_gb300 import workloads

    p = [q for q in workloads.c3(n_seeds=1) if q.Lz == 256 and abs(q.grad_c0 * q.Lz - 0.5) < 1e-12][0]
    o = oracle.OracleLattice(p.Lx, p.Lz, lambda_s=p.lambda_s, lambda_d=p.lambda_d, lambda_e=p.lambda_e,
                             lambda_q=p.lambda_q, lambda_eps=p.lambda_eps, kT=p.kT, G=p.G, grad_c0=p.grad_c0,
                             seed=p.seed, lattice_id=p.lattice_id, omp=omp)
    cores = oracle.set_threads(os.cpu_count() or 1) if omp else 1
    return p, o, cores


def cpu_baseline(budget_s=10.0):
    """The oracle, as it stands, on the host's cores (OpenMP build, one thread per core) and on
    one core (plain build): one Lz = 256 member of the ensemble stepped for about budget_s
    seconds each."""
    out = {}
    for omp in (True, False):
        p, o, cores = _oracle_member(omp)
        o.step(1)
        n, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < budget_s:
            o.step(1)
            n += 1
        dt = time.perf_counter() - t0
        out[omp] = {"value": p.Lx * p.Lz * n / dt / 1e9, "unit": "GLUPS", "cores": cores, "kind": "oracle",
                    "sample": f"{n} steps of the 1024x256 (dc=0.5) ensemble member, FP64, -O2, "
                              + (f"OpenMP over rows on {cores} host cores" if omp else "single thread")}
    res = out[True]
    res["single_core"] = out[False]
    return res


# ---------------------------------------------------------------- reference arm: the oracle
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    p, o, cores = _oracle_member(True)
    o.set_sampling(0, LB_STEPS_PER_STEP)
    per = 8  # LB steps of the 1024 x 256 member per benchmark step (a bounded sample)
    for _ in range(args.warmup):
        o.step(per)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(per)
    dt = time.perf_counter() - t0
    v = p.Lx * p.Lz * per * args.steps / dt / 1e9
    sample = (f"{per} LB steps of the 1024x256 (dc=0.5) ensemble member per step, FP64, OpenMP over rows on "
              f"{cores} host cores")
    print(json.dumps({
        "impl": "reference", "metric": "two-species D2Q9 GLUPS (FP32-deviation batched ensemble)", "value": v,
        "unit": "GLUPS", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": C3_WORKLOAD, "lb_steps_per_step": LB_STEPS_PER_STEP,
                   "sample_every": LB_STEPS_PER_STEP, "precision": "f64 (the oracle)",
                   "sample": "a bounded sample per step: " + sample},
        "cpu_baseline": {"value": v, "unit": "GLUPS", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_profile_small(kT, precision, bulk=True, tile=128, rows=64):
    """A small case for ncu: one 4096 x 1024 lattice (302 MB per FP32 state buffer, more than L2),
    6 steps."""
    import torch

    from paper_1808_05168_gb300 import LatticeParams, Simulation

    p = LatticeParams(4096, 1024, kT=kT, G=0.5, grad_c0=0.5 / 1024, seed=4, lambda_e=1.0)
    with Simulation(p, precision=precision, bulk=bulk) as sim:
        sim.set_tile(tile, rows)
        sim.step(6)
        sim.synchronize()
    torch.cuda.synchronize()
    print("profile-small ok")


def run_profile_ensemble(n_seeds, rows=256, persistent=False, tensor_maps=True):
    """The ensemble mix with fewer seeds (8 seeds: 96 lattices, 8.4 M sites, 1.2 GB of state;
    16 seeds: 2.4 GB), the benchmark's precision, 128-column tiles of `rows` rows, 6 steps (for
    ncu captures): six launches of the step kernel, or one persistent launch of six steps."""
    import torch

    from paper_1808_05168_gb300 import Simulation, workloads

    with Simulation(workloads.c3(n_seeds=n_seeds), precision="dev32", persistent=persistent,
                    tensor_maps=tensor_maps) as sim:
        sim.set_tile(128, rows)
        sim.step(6)
        sim.synchronize()
    torch.cuda.synchronize()
    print("profile-ensemble ok")


def run_profile_adjoint(precision):
    """One gradient of the mean-pressure shift on the 256 x 128 lattice (2000 steps from rest,
    checkpoints every 100), as the benchmark's adjoint leg times it."""
    import torch

    from paper_1808_05168_gb300 import Simulation, workloads

    (p,) = workloads.c5()
    with Simulation(p, precision=precision) as sim:
        loss, grad = sim.pressure_shift_gradient(2000, 100)
    torch.cuda.synchronize()
    print("profile-adjoint ok", loss, list(grad))


if __name__ == "__main__":
    a = parse()
    if a.profile_adjoint:
        run_profile_adjoint(a.profile_precision)
    elif a.profile_ensemble:
        run_profile_ensemble(a.profile_ensemble, rows=a.profile_rows or 256, persistent=a.profile_persistent,
                             tensor_maps=not a.profile_no_tensor_maps)
    elif a.profile_small:
        run_profile_small(a.profile_kT, a.profile_precision, bulk=not a.profile_generic, tile=a.profile_tile,
                          rows=a.profile_rows or 64)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)

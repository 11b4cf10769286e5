#!/usr/bin/env python3
"""Benchmark: random batch Ewald MD steps on one GB300 (or N, one replica each).

One benchmark step = one MD step of the whole hot path on the 2:1 electrolyte
(N = 8001: 2667 cations +2, 5334 anions -1, number density 0.05, alpha = 0.2,
r_c = 6, P = 200, WCA LJ, Langevin T = 1, gamma = 1, dt = 1e-3): k-sampling,
structure factors, FP64 rho(k), Fourier forces, cell list, real space + LJ and
the Langevin update, mixed precision, replayed from a CUDA graph.

Printed as one JSON line (rank 0):
  value       particle-steps/s over all ranks (inputs resident in HBM; L2
              flushed by a 256 MiB write between timed steps, outside the timing)
  e2e         the same through rbe_step_host: pinned host pos/vel copied in and
              out every step, wall-clock
  roofline    dominant kernel (from a profiled pass of the same steps) against
              the special-function-unit rate (sin/cos) or HBM bandwidth
  cpu_baseline  the FP64 CPU oracle on a bounded sample, host cores
  fp64_path   the plain FP64 GPU path on the same steps; speedup_vs_fp64
  accuracy    rel-RMS of the mixed forces against the FP64 GPU forces
  large_system  the same measurements for the 1:1 electrolyte of 2^20 ions
              (density 0.064, alpha = 0.3, r_c = 5, P = 500), where the Fourier
              kernels dominate
``--impl reference`` times the FP64 CPU oracle instead (the reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("RBE force evals/sec & particle-steps/sec at force rel-RMS≤1e-5 vs FP64 path, "
          "same GPU")
UNIT = "particle-steps/s"
SM_COUNT = 152
SFU_PER_SM_PER_CLK = 16          # sin/cos results per SM per clock (special-function unit)
SM_MAX_MHZ = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="budget of the CPU-oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--large", dest="large", action="store_true", default=True,
                    help="also measure the 2^20-particle system (default)")
    ap.add_argument("--no-large", dest="large", action="store_false")
    return ap.parse_args()


def workload():
    from paper_2010_01559_gb300 import workloads
    return workloads.config_2to1_mixed()


# --------------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------- CPU oracle
def oracle_steps(wl, nsteps, sub=None, step0=0):
    """Run nsteps oracle MD steps (forces for `sub` only if given); returns seconds."""
    import numpy as np
    import oracle
    p = wl.params
    pos = wl.pos.astype(np.float64)
    vel = wl.vel.astype(np.float64)
    q = wl.q.astype(np.float64)
    t0 = time.perf_counter()
    for s in range(nsteps):
        out = oracle.rbe_forces(pos, q, p.box, p.alpha, p.r_c, p.P, p.seed, p.stream, step0 + s,
                                lB=p.coulomb_prefactor, lj_eps=p.lj_eps, lj_sigma=p.lj_sigma,
                                lj_rcut=p.lj_rcut, sub=sub)
        if sub is None:
            pos, vel = oracle.langevin_step(pos, vel, out["F"], p.box, p.gamma, p.kT, p.dt,
                                            p.mass, p.seed, p.stream, step0 + s)
    return time.perf_counter() - t0


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(wl, budget_s):
    """Time the FP64 oracle (as it stands) on a bounded sample of the workload."""
    import oracle
    oracle.build()
    t1 = oracle_steps(wl, 1)                       # one full step (also warms up)
    n = max(1, min(200, int(budget_s / max(t1, 1e-6))))
    t = oracle_steps(wl, n, step0=1)
    return {"value": wl.n * n / t, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
            "sample": f"{n} full FP64 oracle MD steps (all {wl.n} particles: sample k, "
                      f"rho, Fourier + real-space + LJ forces, Langevin)"}


# --------------------------------------------------------------------- distributed
def dist_setup(backend="nccl"):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend)
    return world, rank, local


def replica_stream(base_stream, rank):
    """Each rank runs its own replica: the same workload on Philox stream
    base + rank (independent k-batches and Langevin noise, no communication)."""
    return base_stream + rank


def combine_ranks(world, local_seconds, local_particles, steps, device):
    """Whole-job throughput: particles of all ranks x steps / the slowest rank's
    time (weak scaling: every rank steps its own replica)."""
    t_max = reduce_max(local_seconds, world, device)
    n_all = reduce_sum(float(local_particles), world, device)
    return {"seconds": t_max, "particles": n_all, "value": n_all * steps / t_max}


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def reduce_sum(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.item()


# --------------------------------------------------------------------- roofline
def source_hash(kernel_file):
    """Hash of a kernel's source file together with the shared device header
    it includes (a change to either makes committed counters stale)."""
    h = hashlib.sha256(open(kernel_file, "rb").read())
    hdr = os.path.join(os.path.dirname(kernel_file), "rbe_internal.cuh")
    if os.path.exists(hdr):
        h.update(open(hdr, "rb").read())
    return h.hexdigest()[:16]


def traffic_for(kernel, workload_name):
    """dram bytes (read + write) per launch of ``kernel`` on ``workload_name`` from
    the committed ncu summary (profiles/ncu_traffic.json), if the counters were
    taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        db = json.load(open(path))
    except ValueError:
        return None
    e = db.get(kernel, {}).get(workload_name)
    if not e:
        return None
    src = os.path.join(ROOT, "paper_2010_01559_gb300", "csrc", e["source"])
    if not os.path.exists(src) or source_hash(src) != e.get("source_sha256_16"):
        return None
    return e.get("dram_bytes_per_launch")


FP32_LANES_PER_SM = 128
# FP32-pipe operations the real-space pass needs: the distance test of a
# list entry (3 subtractions, 1 multiply, 2 fused multiply-adds) and the terms
# of a pair inside the cutoff (erfc by the 5-term rational form, Gaussian,
# G(r)/r, force, potential and energy accumulation: 25 operations, plus three
# special-function operations counted separately).
REAL_OPS_PER_CANDIDATE = 6
REAL_OPS_PER_PAIR = 25


def list_skin(p):
    """The neighbour-list skin the library uses for these parameters (0.1 r_c,
    capped so that the cells of side r_c + skin stay at least 3 per edge, or
    r_c + skin <= L/2 in the one-cell mode)."""
    cap = p.box / 3 - p.r_c if p.box >= 3 * p.r_c else p.box / 2 - p.r_c
    s = getattr(p, "skin", 0.0)
    return max(0.0, min(s if s > 0 else 0.1 * p.r_c, cap))


def pair_counts(wl):
    """(candidates, pairs within r_c) of the MD step's real-space pass, counted
    on the host with a k-d tree: the list entries it visits (ordered pairs
    within r_c + skin, self excluded) and the ordered pairs within r_c."""
    import numpy as np
    from scipy.spatial import cKDTree
    p = wl.params
    pos = wl.pos.astype(np.float64)
    tree = cKDTree(pos, boxsize=p.box)
    candidates = int(tree.count_neighbors(tree, p.r_c + list_skin(p))) - wl.n
    pairs = int(tree.count_neighbors(tree, p.r_c)) - wl.n
    return candidates, pairs


def unit_peaks(rbe, clk_mhz):
    """SFU and FP32 peaks in T ops/s: per-SM-per-clock rates measured by the
    library's probe kernels (rbe_probe_peaks) times the SM clock seen during the
    timed region (the probe's own clock if none was sampled); the nominal unit
    counts if the probe fails."""
    try:
        pk = rbe.probe_peaks()
    except Exception as e:            # reported, never silent
        pk = {"error": str(e)}
    measured = "sfu_per_clk_sm" in pk
    mhz = clk_mhz or (pk.get("sm_clock_mhz") if measured else None) or SM_MAX_MHZ
    sfu = pk["sfu_per_clk_sm"] if measured else SFU_PER_SM_PER_CLK
    ffma = pk["ffma_per_clk_sm"] if measured else FP32_LANES_PER_SM
    sms = pk.get("sms", SM_COUNT) if measured else SM_COUNT
    basis = (f"{sms} SMs x {sfu:.2f} sin/cos per SM-clock (measured by rbe_probe_peaks) x "
             f"{mhz:.0f} MHz (SM clock under load)") if measured else \
        f"{SM_COUNT} SMs x {SFU_PER_SM_PER_CLK} sin/cos per SM-clock (nominal) x {mhz:.0f} MHz"
    basis_alu = (f"{sms} SMs x {ffma:.1f} FFMA per SM-clock (measured by rbe_probe_peaks) x "
                 f"{mhz:.0f} MHz") if measured else \
        f"{SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 lanes (nominal) x {mhz:.0f} MHz"
    return {"sfu": sms * sfu * mhz * 1e6 / 1e12, "alu": sms * ffma * mhz * 1e6 / 1e12,
            "sfu_basis": basis, "alu_basis": basis_alu, "probe": pk}


# SFU operations per (particle, wave vector) pair: the structure factors take
# a sine and a cosine; the MD step's Fourier force, with the coefficient in
# polar form, one sine (R sin(phi - theta))
SFU_OPS_PER_PAIR = {"rho": 2, "fourier_force": 1}


def fourier_rooflines(prof, wl, units):
    """SFU roofline of both Fourier kernels of an MD step."""
    out = {}
    peak = units["sfu"]
    for name in ("rho", "fourier_force"):
        ms, cnt = prof.get(name, (0.0, 0))
        if not cnt:
            continue
        avg_s = ms / cnt / 1e3
        achieved = SFU_OPS_PER_PAIR[name] * wl.n * wl.params.P / avg_s / 1e12
        out[name] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tsfu/s",
                     "frac": achieved / peak, "avg_launch_us": avg_s * 1e6,
                     "traffic": traffic_for(name, wl.name)}
    return out


def roofline(prof, wl, peaks, units, counts=None):
    """Dominant kernel of the profiled pass against its bound."""
    name, (ms, cnt) = max(prof.items(), key=lambda kv: kv[1][0])
    avg_s = ms / max(cnt, 1) / 1e3
    N, P = wl.n, wl.params.P
    if name in ("rho", "fourier_force"):
        ops = SFU_OPS_PER_PAIR[name]
        work = float(ops) * N * P
        peak = units["sfu"]
        achieved = work / avg_s / 1e12
        out = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak,
               "unit": "Tsfu/s", "frac": achieved / peak, "peak_basis": units["sfu_basis"],
               "algorithmic": f"{ops} SFU op{'s' if ops > 1 else ''} per (particle, k) pair x "
                              f"{N} x {P}"}
    elif name == "real" and counts is not None:
        cand, pairs = counts
        work = REAL_OPS_PER_CANDIDATE * cand + REAL_OPS_PER_PAIR * pairs
        peak = units["alu"]
        achieved = work / avg_s / 1e12
        out = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak,
               "unit": "Tops/s", "frac": achieved / peak, "peak_basis": units["alu_basis"],
               "algorithmic": f"{REAL_OPS_PER_CANDIDATE} ops x {cand} list entries (pairs "
                              f"within r_c + skin) + {REAL_OPS_PER_PAIR} ops x {pairs} pairs "
                              f"within r_c"}
    else:
        # bytes the kernel must move: records read/written per particle
        per_particle = {"prep": 16 + 16 + 4 + 4, "scatter": 4 + 4 + 4 + 4,
                        "cell_order": 4 + 16 + 4 + 16 + 4, "scan": 0, "energy": 0}.get(name, 0)
        bytes_ = per_particle * N
        peak = peaks.get("hbm_gbs", 6800.0)
        achieved = bytes_ / avg_s / 1e9
        out = {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak,
               "unit": "GB/s", "frac": achieved / peak,
               "algorithmic": f"{per_particle} B per particle x {N}"}
    out["avg_launch_us"] = avg_s * 1e6
    out["traffic"] = traffic_for(name, wl.name)
    return out


# --------------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_01559_gb300 as rbe

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = workload()
    if world > 1:
        wl.params.stream = replica_stream(wl.params.stream, rank)
    K, W = args.steps, args.warmup
    peaks = {}
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        peaks = json.load(open(pp))

    stream = torch.cuda.Stream(device=dev)
    h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    pos0 = torch.from_numpy(wl.pos_q()).to(dev)
    vel0 = torch.zeros((wl.n, 4), dtype=torch.float32, device=dev)
    vel0[:, :3] = torch.from_numpy(wl.vel).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed_steps(pos, vel, step_dev, nsteps, profile=False):
        evs = []
        h.profile(profile)
        with torch.cuda.stream(stream):
            for k in range(nsteps):
                flush.fill_(k & 0xFF)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h.step(pos, vel, 1, step_dev)
                e1.record(stream)
                evs.append((e0, e1))
        stream.synchronize()
        h.profile(False)
        return sum(a.elapsed_time(b) for a, b in evs)

    # ---------------------------------------------------------------- mixed path
    with torch.cuda.stream(stream):
        tuning = h.autotune(pos0)            # the library's own launch-shape tuner
        pos = pos0.clone()
        vel = vel0.clone()
        step_dev = torch.zeros(1, dtype=torch.int64, device=dev)
        h.set_graph(True)
        for _ in range(W):
            h.step(pos, vel, 1, step_dev)
    stream.synchronize()
    launches0 = h.launch_count()
    clocks = Clocks(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()              # a no-op unless a profiler asks for ranges
    total_ms = timed_steps(pos, vel, step_dev, K)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    barrier(world)
    clk = clocks.stop()
    units = unit_peaks(rbe, clk.get("sm_mhz"))
    launches = h.launch_count() - launches0
    h.sync()
    agg = combine_ranks(world, total_ms / 1e3, wl.n, K, dev)
    t_max, n_all, value = agg["seconds"], agg["particles"], agg["value"]
    ms_per_step = t_max * 1e3 / K

    # per-kernel profile of the same steps (events around each kernel)
    timed_steps(pos, vel, step_dev, K, profile=True)
    prof = h.profile_read()
    kernels_us = {k: (ms / c * 1e3 if c else 0.0) for k, (ms, c) in prof.items()}

    # accuracy at this configuration: mixed vs FP64 forces on the same input
    with torch.cuda.stream(stream):
        F32, E32, _ = h.forces(pos0, 0)
        F64, E64, _ = h.forces_f64(pos0.double().contiguous(), 0)
    stream.synchronize()
    d = (F32[:, :3].double() - F64[:, :3])
    acc = (d.norm() / F64[:, :3].norm()).item()

    # ---------------------------------------------------------------- FP64 path
    K64 = max(3, min(K, 50))
    with torch.cuda.stream(stream):
        pos64 = pos0.double().contiguous()
        vel64 = vel0.double().contiguous()
        step64 = torch.zeros(1, dtype=torch.int64, device=dev)
        for _ in range(3):
            h.step(pos64, vel64, 1, step64)
    stream.synchronize()
    ms64 = timed_steps(pos64, vel64, step64, K64)
    value64 = wl.n * K64 / (ms64 / 1e3)

    # ---------------------------------------------------------------- end to end
    hpos = pos0.cpu().pin_memory()
    hvel = vel0.cpu().pin_memory()
    for s in range(3):
        h.step_host(hpos, hvel, 1, 10_000 + s)
    e2e_t = 0.0
    for s in range(K):
        with torch.cuda.stream(stream):
            flush.fill_(s & 0xFF)
        stream.synchronize()
        t0 = time.perf_counter()
        h.step_host(hpos, hvel, 1, 20_000 + s)
        e2e_t += time.perf_counter() - t0
    e2e_t = reduce_max(e2e_t, world, dev)
    e2e_value = n_all * K / e2e_t
    bytes_io = 2 * 16 * wl.n

    paper_literal = measure_paper_literal(rbe, torch, wl, dev, stream, flush, units) \
        if rank == 0 else None

    large = None
    if args.large and rank == 0:
        from paper_2010_01559_gb300 import workloads as wls
        large = measure_system(rbe, torch, wls.config_large(), dev, stream, 50, 3, flush, peaks,
                               units)
        large["scaling"] = scaling_sweep(rbe, torch, wls, dev, stream, flush) + [
            {"N": large["N"], "ms_per_step": large["ms_per_step"], "value": large["value"]}]
        large["batched_replicas"] = measure_replicas(rbe, torch, wls, dev, stream, flush)

    result = None
    if rank == 0:
        rl = roofline(prof, wl, peaks, units, counts=pair_counts(wl))
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "N": wl.n, "P": wl.params.P,
                       "alpha": wl.params.alpha, "r_c": wl.params.r_c,
                       "box": round(wl.params.box, 4), "path": "mixed (FP32 phases/forces, "
                       "FP64 rho(k) and energy sums)", "graph": True,
                       "l2": "flushed between timed steps (256 MiB write, untimed)",
                       "tuning": {"rho_chunk": tuning[0], "force_split": tuning[1],
                                  "real_split": tuning[2], "real_seg": tuning[3],
                                  "list_split": tuning[4]},
                       "parallelism": f"replicas x{world}"},
            "force_evals_per_s": value / wl.n,
            "clocks": clk,
            "roofline": rl,
            "fourier_rooflines": fourier_rooflines(prof, wl, units),
            "unit_peaks": {k: units[k] for k in ("sfu", "alu", "probe")},
            "kernels_avg_us": kernels_us,
            "gpu_launches": launches,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": bytes_io,
                    "d2h_bytes_per_step": bytes_io,
                    "api": "rbe_step_host on pinned host pos/vel: every step reads them from and writes them to host memory (the step's kernels access the page-locked arrays in place over the host link; the call returns when the closing kernel's completion word reaches mapped host memory)"},
            "fp64_path": {"value": value64, "unit": UNIT, "steps": K64,
                          "ms_per_step": ms64 / K64},
            "speedup_vs_fp64": value / value64,
            "accuracy": {"force_rel_rms_mixed_vs_fp64_gpu": acc, "target": 1e-5},
        }
        if large is not None:
            result["large_system"] = large
        if paper_literal is not None:
            result["paper_literal"] = paper_literal
        if not args.no_cpu_baseline:
            result["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)
        print(json.dumps(result), flush=True)
    h.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return result


def measure_paper_literal(rbe, torch, wl, dev, stream, flush, units, K=200):
    """The same workload with the paper's Metropolis-Hastings k-sampler and with
    leapfrog + Andersen (Algorithm 1 as printed), MD steps from a graph with
    L2 flushed between timed steps; and the true (non-random) energy and
    pressure (rbe_observables, full Ewald over the sampler's |m| <= M)."""
    import copy
    out = {}
    for name, kw in (("mh_sampler", dict(sampler=1)),
                     ("andersen", dict(thermostat=1, andersen_nu=10.0))):
        sp = copy.copy(wl.params)
        for k, v in kw.items():
            setattr(sp, k, v)
        h = rbe.RBE(rbe.params_from(sp, n_max=wl.n))
        pos = torch.from_numpy(wl.pos_q()).to(dev)
        vel = torch.zeros((wl.n, 4), dtype=torch.float32, device=dev)
        vel[:, :3] = torch.from_numpy(wl.vel).to(dev)
        with torch.cuda.stream(stream):
            h.autotune(pos)
            step = torch.zeros(1, dtype=torch.int64, device=dev)
            h.set_graph(True)
            h.step(pos, vel, 5, step)
        stream.synchronize()
        evs = []
        with torch.cuda.stream(stream):
            for k in range(K):
                flush.fill_(k & 0xFF)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h.step(pos, vel, 1, step)
                e1.record(stream)
                evs.append((e0, e1))
        stream.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs) / K
        out[name] = {"ms_per_step": ms, "value": wl.n / (ms / 1e3), "unit": UNIT, "steps": K}
        if name == "mh_sampler":
            h.profile(True)
            with torch.cuda.stream(stream):
                h.step(pos, vel, 20, step)
            stream.synchronize()
            h.profile(False)
            pr = h.profile_read()
            out[name]["prep_us"] = pr["prep"][0] / max(pr["prep"][1], 1) * 1e3
        h.close()
    # observables: full Ewald over |m| <= M (the sampler's table half-width)
    h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    pos = torch.from_numpy(wl.pos_q()).to(dev)
    vel = torch.zeros((wl.n, 4), dtype=torch.float32, device=dev)
    vel[:, :3] = torch.from_numpy(wl.vel).to(dev)
    M = h.info(0).M
    h.observables(pos, vel, M)                      # warm-up (allocates the k list)
    reps = 5
    t0 = time.perf_counter()
    for _ in range(reps):
        obs = h.observables(pos, vel, M)[0]
    dt = (time.perf_counter() - t0) / reps
    side = 2 * M + 1
    khalf = (side ** 3 - 1) // 2
    achieved = 2.0 * wl.n * khalf / dt / 1e12      # sin + cos per (particle, k) pair
    out["observables"] = {"mmax": M, "wave_vectors_half_space": khalf, "ms_per_call": dt * 1e3,
                          "pressure": obs["pressure"], "E_total": obs["E_total"],
                          "sfu_roofline": {"bound": "alu", "achieved": achieved,
                                           "peak": units["sfu"], "unit": "Tsfu/s",
                                           "frac": achieved / units["sfu"],
                                           "note": "whole call (host-timed, includes the "
                                                   "real-space pass and the copy-out)"}}
    h.close()
    return out


def scaling_sweep(rbe, torch, wls, dev, stream, flush, sizes=(1 << 14, 1 << 16, 1 << 18)):
    """Mixed MD steps of the 1:1 electrolyte at density 0.064 for growing N (box
    grows with N), autotuned launch shapes, L2 flushed between timed steps: the
    O(N) cost per step."""
    out = []
    for n in sizes:
        wl = wls.config_large(n)
        h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
        pos = torch.from_numpy(wl.pos_q()).to(dev)
        vel = torch.zeros((wl.n, 4), dtype=torch.float32, device=dev)
        vel[:, :3] = torch.from_numpy(wl.vel).to(dev)
        with torch.cuda.stream(stream):
            h.autotune(pos)
            step = torch.zeros(1, dtype=torch.int64, device=dev)
            h.set_graph(True)
            h.step(pos, vel, 3, step)
        stream.synchronize()
        evs = []
        with torch.cuda.stream(stream):
            for k in range(30):
                flush.fill_(k & 0xFF)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h.step(pos, vel, 1, step)
                e1.record(stream)
                evs.append((e0, e1))
        stream.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs) / len(evs)
        out.append({"N": wl.n, "ms_per_step": ms, "value": wl.n / (ms / 1e3)})
        h.close()
    return out


def measure_replicas(rbe, torch, wls, dev, stream, flush, K=20, W=3):
    """The batched configuration: 64 independent 1:1 electrolytes (N log-uniform
    in [1000, 65536], density 0.064, P = 100, one Philox stream each) stepped
    together by one batch handle, graph replay, L2 flushed between steps."""
    import numpy as np
    reps = wls.config_replicas()
    h = rbe.RBEBatch([rbe.params_from(w.params) for w in reps], [w.n for w in reps])
    pos = torch.from_numpy(np.concatenate([w.pos_q() for w in reps])).to(dev)
    vel = torch.zeros_like(pos)
    vel[:, :3] = torch.from_numpy(np.concatenate([w.vel for w in reps])).to(dev)
    n_all = int(pos.shape[0])
    with torch.cuda.stream(stream):
        tuning = h.autotune(pos)
        step_dev = torch.zeros(1, dtype=torch.int64, device=dev)
        h.set_graph(True)
        h.step(pos, vel, W, step_dev)
    stream.synchronize()
    evs = []
    with torch.cuda.stream(stream):
        for k in range(K):
            flush.fill_(k & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.step(pos, vel, 1, step_dev)
            e1.record(stream)
            evs.append((e0, e1))
    stream.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    stats = h.list_stats()
    h.close()
    return {"workload": f"{len(reps)} replicas, 1:1 electrolyte, N log-uniform in [1000, 65536], "
                        f"density 0.064, P = 100", "systems": len(reps), "N_total": n_all,
            "value": n_all * K / (ms / 1e3), "unit": UNIT, "steps": K, "ms_per_step": ms / K,
            "tuning": list(tuning), "list_builds": stats["builds"]}


def measure_system(rbe, torch, wl, dev, stream, K, W, flush, peaks, units):
    """Timed MD steps (mixed, graph replay, L2 flushed between steps), a
    profiled pass, the FP64 path and the mixed-vs-FP64 force agreement."""
    h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    pos0 = torch.from_numpy(wl.pos_q()).to(dev)
    vel0 = torch.zeros((wl.n, 4), dtype=torch.float32, device=dev)
    vel0[:, :3] = torch.from_numpy(wl.vel).to(dev)

    def timed(pos, vel, step_dev, nsteps, profile=False):
        evs = []
        h.profile(profile)
        with torch.cuda.stream(stream):
            for k in range(nsteps):
                flush.fill_(k & 0xFF)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h.step(pos, vel, 1, step_dev)
                e1.record(stream)
                evs.append((e0, e1))
        stream.synchronize()
        h.profile(False)
        return sum(a.elapsed_time(b) for a, b in evs)

    with torch.cuda.stream(stream):
        tuning = h.autotune(pos0)
        pos, vel = pos0.clone(), vel0.clone()
        step_dev = torch.zeros(1, dtype=torch.int64, device=dev)
        h.set_graph(True)
        for _ in range(W):
            h.step(pos, vel, 1, step_dev)
    stream.synchronize()
    torch.cuda.profiler.start()
    ms = timed(pos, vel, step_dev, K)
    torch.cuda.profiler.stop()
    timed(pos, vel, step_dev, max(3, K // 4), profile=True)
    prof = h.profile_read()
    with torch.cuda.stream(stream):
        F32, _, _ = h.forces(pos0, 0, energy=False)
        F64, _, _ = h.forces_f64(pos0.double().contiguous(), 0, energy=False)
    stream.synchronize()
    acc = ((F32[:, :3].double() - F64[:, :3]).norm() / F64[:, :3].norm()).item()
    K64 = 3
    with torch.cuda.stream(stream):
        p64, v64 = pos0.double().contiguous(), vel0.double().contiguous()
        s64 = torch.zeros(1, dtype=torch.int64, device=dev)
        h.step(p64, v64, 1, s64)
    stream.synchronize()
    ms64 = timed(p64, v64, s64, K64)
    value = wl.n * K / (ms / 1e3)
    value64 = wl.n * K64 / (ms64 / 1e3)
    out = {"workload": wl.name, "N": wl.n, "P": wl.params.P, "alpha": wl.params.alpha,
           "r_c": wl.params.r_c, "value": value, "unit": UNIT, "steps": K,
           "ms_per_step": ms / K, "force_evals_per_s": K / (ms / 1e3),
           "tuning": {"rho_chunk": tuning[0], "force_split": tuning[1], "real_split": tuning[2],
                      "real_seg": tuning[3], "list_split": tuning[4]},
           "kernels_avg_us": {k: (t / c * 1e3 if c else 0.0) for k, (t, c) in prof.items()},
           "roofline": roofline(prof, wl, peaks, units, counts=pair_counts(wl)),
           "fourier_rooflines": fourier_rooflines(prof, wl, units),
           "fp64_path": {"value": value64, "unit": UNIT, "steps": K64, "ms_per_step": ms64 / K64},
           "speedup_vs_fp64": value / value64,
           "accuracy": {"force_rel_rms_mixed_vs_fp64_gpu": acc, "target": 1e-5}}
    h.close()
    return out


# --------------------------------------------------------------------- reference arm
def run_reference(args):
    """The FP64 CPU oracle as it stands, on this host's cores, same workload and
    metric.  Each step is one oracle MD step; if K steps of the whole system
    would not fit a few minutes, each step evaluates forces for a fixed subset
    of particles (rho(k) still over all of them) and counts only that subset."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import numpy as np
    import oracle
    oracle.build()
    wl = workload()
    K, W = args.steps, args.warmup
    t1 = oracle_steps(wl, 1)
    budget = 150.0
    if t1 * (K + W) <= budget:
        sub, n_per_step = None, wl.n
    else:
        frac = budget / (t1 * (K + W))
        n_per_step = max(16, int(wl.n * frac))
        sub = np.linspace(0, wl.n - 1, n_per_step).astype(int)
    oracle_steps(wl, W, sub=sub, step0=100)
    t = oracle_steps(wl, K, sub=sub, step0=1000)
    value = n_per_step * K / t
    sample = (f"{K} oracle MD steps over all {wl.n} particles" if sub is None else
              f"{K} oracle steps: rho(k) over all {wl.n} particles, forces for "
              f"{n_per_step} evenly spaced particles per step")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
           "steps": K, "warmup": W, "ms_per_step": t * 1e3 / K, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl.name, "N": wl.n, "P": wl.params.P},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

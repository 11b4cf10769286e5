#!/usr/bin/env python3
"""Benchmark: random batch Ewald MD steps on one GB300 (or N, one replica each).

One benchmark step = one MD step of the whole hot path on the large 1:1
electrolyte (N = 2^20 ions, 2^19 of each sign, number density 0.064,
alpha = 0.3, r_c = 5, P = 500, WCA LJ, Langevin T = 1, gamma = 1, dt = 1e-3):
k-sampling, structure factors with FP64 rho(k), Fourier forces, neighbour
list (rebuilt on the device when a particle has moved more than skin/2), real
space + LJ and the Langevin update, mixed precision, replayed from a CUDA graph.

Printed as one JSON line (rank 0):
  value       particle-steps/s over all ranks (inputs resident in HBM; L2
              flushed by a 256 MiB write between timed steps, outside the
              timing; the K-step timed region is repeated until it has lasted
              0.3 s, so that the clock samples cover it)
  e2e         the same through rbe_step_host on pinned host pos/vel: every
              step reads them from and writes them to host memory, wall-clock
  roofline    dominant kernel (from a profiled pass of the same steps) against
              the special-function-unit rate (sin/cos) or HBM bandwidth
  cpu_baseline  the FP64 CPU oracle on a bounded sample of the same workload
              (rho(k) over all particles, forces of 4096 of them), all cores
  fp64_path   the plain FP64 GPU path on the same system; speedup_vs_fp64, and
              the same-algorithm ratio (both paths scanning the cells every step)
  accuracy    rel-RMS of an MD step's mixed force against the FP64 GPU forces
              at the positions and step it started from
  extra       the 2:1 electrolyte (N = 8001), the water-like autograd energy,
              the FP64 100-step loop of the small electrolyte, 64 batched
              replicas, the O(N) sweep, the paper-literal variants, and the
              oracle's own timings at 1 thread and on all cores next to the
              paper's CPU timings
``--impl reference`` times the FP64 CPU oracle instead (the reference arm).
``--profile-case W`` runs a few steps of one workload inside a profiler range
(for ncu captures with ``--profile-from-start off``) and prints their time.
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
MIN_TIMED_SECONDS = 0.3          # the timed region is repeated until it has lasted this long
SUBSET = 4096                    # oracle subset of the large system: particles 256 t

# The paper's own CPU timings (whole MD steps: RBE Fourier + real space + LJ +
# thermostat), one core of an Intel Xeon Gold 6248 (Cascade Lake) at 2.5 GHz
# (Sec. 4).  Context only: other systems, other hardware, no GPU.
PAPER_CPU_TIMINGS = [
    {"what": "RBE, 1e6 steps in 1267 s (Table 1)", "N": 300, "P": 10,
     "ms_per_step": 1.267, "particle_steps_per_s": 300 / 1.267e-3,
     "system": "electrolyte, L = 10, alpha = 0.55, r_c = 4"},
    {"what": "RBE, 1e5 steps in 1167 s (Table 4, c_salt = 0)", "N": 501, "P": 100,
     "ms_per_step": 11.67, "particle_steps_per_s": 501 / 11.67e-3,
     "system": "colloid + counterions, alpha = 0.0072 A^-2, r_c = 40 A"},
    {"what": "RBE, 1e5 steps in 15258 s (Table 4, c_salt = 196 mM)", "N": 3101, "P": 100,
     "ms_per_step": 152.58, "particle_steps_per_s": 3101 / 152.58e-3,
     "system": "colloid + salt"},
]
PAPER_HARDWARE = "1 core of an Intel Xeon Gold 6248 (Cascade Lake) @ 2.5 GHz, 4 GB"


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=150.0,
                    help="wall-clock budget of the reference arm's oracle steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra workloads and the oracle timing table")
    # profiler capture of one workload (ncu --profile-from-start off)
    ap.add_argument("--profile-case", choices=["2to1", "large", "water"], default=None)
    ap.add_argument("--n", type=int, default=0, help="profile case: particles (large) or "
                    "molecules (water)")
    ap.add_argument("--tuning", default="", help="profile case: rho_chunk,force_split,"
                    "real_split,real_seg,list_split (0 = the library's choice); empty: autotune")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "f64"])
    ap.add_argument("--graph", action="store_true", help="profile case: graph replay")
    ap.add_argument("--fusion", choices=["auto", "on", "off"], default="auto",
                    help="profile case: structure factors and the standing-list pass in one "
                    "launch (on), two (off), or as the library chooses (auto)")
    ap.add_argument("--no-fusion", dest="fusion", action="store_const", const="off",
                    help="profile case: same as --fusion off")
    return ap.parse_args(argv)


def workload():
    from paper_2010_01559_gb300 import workloads
    return workloads.config_large()


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
def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _f64(wl):
    import numpy as np
    return wl.pos.astype(np.float64), wl.q.astype(np.float64)


def oracle_eval_seconds(wl, step=0, sub=None, pos64=None, q64=None):
    """Seconds of one oracle force evaluation (sample k, rho, Fourier, real
    space and LJ forces; forces for ``sub`` only if given)."""
    import oracle
    p = wl.params
    if pos64 is None:
        pos64, q64 = _f64(wl)
    t0 = time.perf_counter()
    oracle.rbe_forces(pos64, q64, p.box, p.alpha, p.r_c, p.P, p.seed, p.stream, step,
                      lB=p.coulomb_prefactor, lj_eps=p.lj_eps, lj_sigma=p.lj_sigma,
                      lj_rcut=p.lj_rcut, sub=sub)
    return time.perf_counter() - t0


def oracle_large_estimate(wl, threads, rho_slice=None, nsub=SUBSET, step=0):
    """One oracle force evaluation of a large system, timed in parts and
    scaled to all N particles: rho(k) over ``rho_slice`` particles (all if
    None) gives the per-particle structure-factor cost; the Fourier forces of
    nsub particles from that rho, and their real-space + LJ forces over the
    whole system (the oracle's plain all-pairs loop), give the per-particle
    force cost.  Whole evaluation = N x (rho + Fourier force + real space)
    per particle.  Returns a dict of the parts and the estimate."""
    import numpy as np
    import oracle
    p = wl.params
    used = oracle.set_threads(threads)
    pos64, q64 = _f64(wl)
    m, _, _ = oracle.sample_k(p.alpha, p.box, p.seed, p.stream, step, p.P)
    ns = wl.n if rho_slice is None else min(wl.n, rho_slice)
    sub = (np.arange(nsub) * (wl.n // nsub)).astype(int)
    t0 = time.perf_counter()
    oracle.rbe_fourier(pos64[:ns], q64[:ns], p.box, p.alpha, m, lB=p.coulomb_prefactor,
                       sub=np.array([0]))
    t_rho = time.perf_counter() - t0
    # rho and the Fourier forces of every particle of the slice
    sub_f = np.arange(ns)
    t0 = time.perf_counter()
    oracle.rbe_fourier(pos64[:ns], q64[:ns], p.box, p.alpha, m, lB=p.coulomb_prefactor,
                       sub=sub_f)
    t_four = max(time.perf_counter() - t0 - t_rho, 0.0)
    t0 = time.perf_counter()
    oracle.real_space(pos64, q64, p.box, p.alpha, p.r_c, lB=p.coulomb_prefactor,
                      lj_eps=p.lj_eps, lj_sigma=p.lj_sigma, lj_rcut=p.lj_rcut, sub=sub)
    t_real = time.perf_counter() - t0
    per = {"rho": t_rho / ns, "fourier_force": t_four / max(len(sub_f), 1),
           "real_space_lj": t_real / nsub}
    full = wl.n * sum(per.values())
    oracle.set_threads(0)
    return {"threads": used, "seconds_per_eval": full, "force_evals_per_s": 1.0 / full,
            "particle_steps_per_s": wl.n / full,
            "seconds_per_particle": per, "sample_seconds": t_rho * 2 + t_four + t_real,
            "sample": f"rho(k) and Fourier forces over {ns} particles, real-space + LJ forces "
                      f"of {nsub} evenly spaced particles (the oracle's all-pairs loop over all "
                      f"{wl.n}), each scaled to all {wl.n} particles"}


def cpu_baseline(wl):
    """The FP64 oracle (as it stands) on all host cores, on a bounded sample of
    the benchmark workload, scaled to the metric's unit."""
    import oracle
    oracle.build()
    est = oracle_large_estimate(wl, 0, rho_slice=1 << 18)
    return {"value": est["particle_steps_per_s"], "unit": UNIT, "cores": est["threads"],
            "kind": "oracle", "sample": est["sample"], "seconds_per_eval": est["seconds_per_eval"],
            "seconds_per_particle": est["seconds_per_particle"],
            "sample_seconds": est["sample_seconds"]}


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
def _local_includes(path, seen):
    """The file and the quoted #include files it reaches, in a fixed order."""
    if path in seen or not os.path.exists(path):
        return
    seen.append(path)
    for line in open(path, encoding="utf-8", errors="replace"):
        s = line.strip()
        if s.startswith("#include") and '"' in s:
            _local_includes(os.path.join(os.path.dirname(path), s.split('"')[1]), seen)


def source_hash(kernel_file):
    """Hash of a kernel's source file, the device headers it includes (directly
    or through others) and the compiler flags: a change to any of them makes
    committed counters stale."""
    from paper_2010_01559_gb300 import build as _build
    files = []
    _local_includes(kernel_file, files)
    h = hashlib.sha256()
    for f in files:
        h.update(open(f, "rb").read())
    h.update(" ".join(_build.ARCH + [f for f in _build.NVCC_FLAGS
                                     if not os.path.isabs(f)]).encode())
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
SFU_OPS_PER_PAIR = {"rho": 2, "fourier_force": 1, "rho_list": 2}


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
    if name in ("rho", "fourier_force", "rho_list"):
        ops = SFU_OPS_PER_PAIR[name]
        work = float(ops) * N * P
        peak = units["sfu"]
        achieved = work / avg_s / 1e12
        out = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak,
               "unit": "Tsfu/s", "frac": achieved / peak, "peak_basis": units["sfu_basis"],
               "algorithmic": f"{ops} SFU op{'s' if ops > 1 else ''} per (particle, k) pair x "
                              f"{N} x {P}"}
        if name == "rho_list":
            out["algorithmic"] += (" (the structure factors; the pass over the standing "
                                   "neighbour list runs in the same launch, on other pipes)")
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


# Bytes the real-space pass must move at the least (Sec. 2 real-space sum
# under r_c): each particle's 16-byte record read once and its 16-byte force
# written once; the neighbour list is this implementation's choice and is
# reported beside it.
REAL_ALGO_BYTES_PER_PARTICLE = 32


def list_pass_roofline(prof, wl, peaks, counts, entry_bytes=4):
    """HBM view of the real-space list pass: algorithmic bytes (records in,
    forces out) and the list-inclusive bytes, per average launch."""
    ms, cnt = prof.get("real", (0.0, 0))
    if not cnt:
        return None
    avg_s = ms / cnt / 1e3
    cand, _ = counts
    algo = REAL_ALGO_BYTES_PER_PARTICLE * wl.n
    with_list = algo + entry_bytes * cand + 4 * wl.n + 4 * wl.n     # + counts, + order
    peak = peaks.get("hbm_gbs", 6800.0)
    return {"bound": "hbm", "achieved": algo / avg_s / 1e9, "peak": peak, "unit": "GB/s",
            "frac": algo / avg_s / 1e9 / peak, "avg_launch_us": avg_s * 1e6,
            "algorithmic": f"{REAL_ALGO_BYTES_PER_PARTICLE} B per particle x {wl.n}",
            "with_list_bytes": with_list, "with_list_GBps": with_list / avg_s / 1e9,
            "traffic": traffic_for("real", wl.name)}


# --------------------------------------------------------------------- our arm
def _state(torch, wl, dev, dtype=None):
    dtype = dtype or torch.float32
    pos = torch.from_numpy(wl.pos_q()).to(dev).to(dtype).contiguous()
    vel = torch.zeros((wl.n, 4), dtype=dtype, device=dev)
    vel[:, :3] = torch.from_numpy(wl.vel).to(dev).to(dtype)
    return pos, vel


def timed_steps(torch, h, pos, vel, step_dev, nsteps, stream, flush, profile=False, F_out=None):
    """nsteps single MD steps on `stream`, each bracketed by CUDA events with an
    untimed 256 MiB write (L2 flush) before it; returns the summed device ms."""
    evs = []
    h.profile(profile)
    with torch.cuda.stream(stream):
        for k in range(nsteps):
            flush.fill_(k & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.step(pos, vel, 1, step_dev, F_out=F_out)
            e1.record(stream)
            evs.append((e0, e1))
    stream.synchronize()
    h.profile(False)
    return sum(a.elapsed_time(b) for a, b in evs)


def md_handle(rbe, torch, wl, dev, stream, skin=None, warm=3):
    """Handle for MD steps of wl (autotuned launch shapes, graph replay),
    warmed up; returns (handle, pos, vel, step counter, tuning)."""
    import copy
    sp = wl.params
    if skin is not None:
        sp = copy.copy(sp)
        sp.skin = skin
    h = rbe.RBE(rbe.params_from(sp, n_max=wl.n))
    pos, vel = _state(torch, wl, dev)
    with torch.cuda.stream(stream):
        tuning = h.autotune(pos)
        step = torch.zeros(1, dtype=torch.int64, device=dev)
        h.set_graph(True)
        if warm:
            h.step(pos, vel, warm, step)
    stream.synchronize()
    return h, pos, vel, step, tuning


def step_accuracy(torch, h, pos, vel, step, stream, sub_n=None):
    """One MD step with its total force out (rbe_step_ex), against the FP64
    GPU forces at the positions and step index it started from: rel-RMS and
    the largest per-particle deviation relative to the RMS force."""
    before = pos.clone()
    k = int(step.item())
    F = torch.zeros_like(pos)
    with torch.cuda.stream(stream):
        h.step(pos, vel, 1, step, F_out=F)
        F64, _, _ = h.forces_f64(before.double().contiguous(), k, energy=False)
    stream.synchronize()
    d = F[:, :3].double() - F64[:, :3]
    ref = F64[:, :3]
    rms = ref.norm(dim=1).square().mean().sqrt().item()
    return {"force_rel_rms_step_vs_fp64_gpu": (d.norm() / ref.norm()).item(),
            "max_particle_dev_over_rms_force": d.norm(dim=1).max().item() / rms,
            "step": k, "target": 1e-5,
            "how": "an MD step's total force (rbe_step_ex: the kernels the timed steps run) "
                   "against rbe_forces_f64 at the positions and step index it started from"}


def measure_headline(rbe, torch, wl, args, world, local, dev, stream, flush):
    """The benchmark's own measurement: K-step timed regions (repeated until
    they have lasted MIN_TIMED_SECONDS), clocks sampled during them."""
    K, W = args.steps, args.warmup
    h, pos, vel, step_dev, tuning = md_handle(rbe, torch, wl, dev, stream, warm=W)
    launches0 = h.launch_count()
    clocks = Clocks(local)
    clocks.start()
    total_ms, reps, wall0 = 0.0, 0, time.perf_counter()
    while True:
        barrier(world)
        torch.cuda.synchronize()
        total_ms += timed_steps(torch, h, pos, vel, step_dev, K, stream, flush)
        torch.cuda.synchronize()
        barrier(world)
        reps += 1
        done = reduce_max(time.perf_counter() - wall0, world, dev) >= MIN_TIMED_SECONDS
        if done or reps >= 10000:
            break
    clk = clocks.stop()
    launches = h.launch_count() - launches0
    agg = combine_ranks(world, total_ms / 1e3, wl.n, K * reps, dev)
    return h, pos, vel, step_dev, tuning, {
        "seconds": agg["seconds"], "particles": agg["particles"], "value": agg["value"],
        "reps": reps, "ms_per_step": agg["seconds"] * 1e3 / (K * reps), "clocks": clk,
        "launches_per_step": launches / (K * reps), "launches": launches}


def measure_e2e(torch, h, wl, K, stream, flush, world, dev, step0=20_000):
    """rbe_step_host on pinned host arrays: each call moves that step's pos and
    vel from host memory and back (the step's kernels access the page-locked
    arrays in place) and returns when the closing kernel's completion word has
    reached host memory; wall-clock per call, L2 flushed before each."""
    hpos = torch.from_numpy(wl.pos_q()).pin_memory()
    hvel = torch.zeros((wl.n, 4), dtype=torch.float32).pin_memory()
    hvel[:, :3] = torch.from_numpy(wl.vel)
    for s in range(3):
        h.step_host(hpos, hvel, 1, step0 - 10 + s)
    t = 0.0
    for s in range(K):
        with torch.cuda.stream(stream):
            flush.fill_(s & 0xFF)
        stream.synchronize()
        t0 = time.perf_counter()
        h.step_host(hpos, hvel, 1, step0 + s)
        t += time.perf_counter() - t0
    return reduce_max(t, world, dev)


def fp64_and_same_algorithm(rbe, torch, wl, dev, stream, flush, K_mixed):
    """The plain FP64 GPU path (per-step cell scan) and, for a like-for-like
    ratio, the mixed path with the neighbour list off (skin < 0: the same
    per-step cell scan), both as MD steps with L2 flushed between steps."""
    h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    p64, v64 = _state(torch, wl, dev, torch.float64)
    s64 = torch.zeros(1, dtype=torch.int64, device=dev)
    with torch.cuda.stream(stream):
        h.step(p64, v64, 1, s64)
    stream.synchronize()
    K64 = 3
    ms64 = timed_steps(torch, h, p64, v64, s64, K64, stream, flush)
    h.close()
    del p64, v64
    hc, pc, vc, sc, tun = md_handle(rbe, torch, wl, dev, stream, skin=-1.0, warm=2)
    Kc = max(3, min(K_mixed, 30))
    msc = timed_steps(torch, hc, pc, vc, sc, Kc, stream, flush)
    hc.close()
    return {"fp64": {"value": wl.n * K64 / (ms64 / 1e3), "unit": UNIT, "steps": K64,
                     "ms_per_step": ms64 / K64, "path": "FP64 phases, sums and forces; cell scan "
                                                       "every step (k_real_f64)"},
            "mixed_cell_scan": {"value": wl.n * Kc / (msc / 1e3), "unit": UNIT, "steps": Kc,
                                "ms_per_step": msc / Kc, "tuning": list(tun),
                                "path": "mixed precision, neighbour list off (skin < 0): cell "
                                        "scan every step (k_real_seg)"}}


def measure_system(rbe, torch, wl, dev, stream, flush, peaks, units, K=200):
    """A second workload: timed MD steps (graph replay, L2 flushed), its
    per-kernel profile and rooflines, the FP64 path and an MD step's accuracy."""
    h, pos, vel, step, tuning = md_handle(rbe, torch, wl, dev, stream)
    ms = timed_steps(torch, h, pos, vel, step, K, stream, flush)
    fused = h.get_fusion()
    timed_steps(torch, h, pos, vel, step, max(3, K // 4), stream, flush, profile=True)
    prof_step = h.profile_read()
    h.set_fusion(False)
    timed_steps(torch, h, pos, vel, step, max(3, K // 4), stream, flush, profile=True)
    prof = h.profile_read()
    h.set_fusion(None)
    acc = step_accuracy(torch, h, pos, vel, step, stream)
    h.close()
    h64 = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    p64, v64 = _state(torch, wl, dev, torch.float64)
    s64 = torch.zeros(1, dtype=torch.int64, device=dev)
    with torch.cuda.stream(stream):
        h64.step(p64, v64, 2, s64)
    stream.synchronize()
    K64 = 20
    ms64 = timed_steps(torch, h64, p64, v64, s64, K64, stream, flush)
    h64.close()
    counts = pair_counts(wl)
    value = wl.n * K / (ms / 1e3)
    return {"workload": wl.name, "N": wl.n, "P": wl.params.P, "alpha": wl.params.alpha,
            "r_c": wl.params.r_c, "value": value, "unit": UNIT, "steps": K,
            "ms_per_step": ms / K, "force_evals_per_s": K / (ms / 1e3), "tuning": list(tuning),
            "fused_list_step": fused,
            "kernels_avg_us": {k: t / c * 1e3 for k, (t, c) in prof.items() if c},
            "step_kernels_avg_us": {k: t / c * 1e3 for k, (t, c) in prof_step.items() if c},
            "roofline": roofline(prof_step, wl, peaks, units, counts=counts),
            "fourier_rooflines": fourier_rooflines(prof, wl, units),
            "fp64_path": {"value": wl.n * K64 / (ms64 / 1e3), "unit": UNIT, "steps": K64,
                          "ms_per_step": ms64 / K64},
            "speedup_vs_fp64": value / (wl.n * K64 / (ms64 / 1e3)), "accuracy": acc}


def measure_water_autograd(rbe, torch, dev, stream, flush, units, K=20):
    """The water-like point-charge system (10^4 rigid 3-site molecules, 3 10^4
    charges, alpha = 0.1, r_c = 10, P = 100): RBEEnergy forward + backward
    (dE/dr = -F and dE/dq = phi for a frozen k-batch), CUDA events, L2 flushed
    between iterations.  Each iteration runs two force evaluations (forward:
    energy; backward: forces and dE/dq with rho recomputed)."""
    from paper_2010_01559_gb300 import workloads
    wl = workloads.config_water()
    h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    pos = torch.from_numpy(wl.pos).to(dev).requires_grad_(True)
    q = torch.from_numpy(wl.q).to(dev).requires_grad_(True)
    with torch.cuda.stream(stream):
        h.autotune(torch.from_numpy(wl.pos_q()).to(dev))
        for s in range(3):
            E = rbe.RBEEnergy.apply(pos, q, h, s)
            E.backward()
    stream.synchronize()
    evs = []
    h.profile(False)
    with torch.cuda.stream(stream):
        for k in range(K):
            flush.fill_(k & 0xFF)
            pos.grad = None
            q.grad = None
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            E = rbe.RBEEnergy.apply(pos, q, h, 100 + k)
            E.backward()
            e1.record(stream)
            evs.append((e0, e1))
    stream.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / K
    # per-kernel profile of one forward + backward
    h.profile(True)
    with torch.cuda.stream(stream):
        E = rbe.RBEEnergy.apply(pos, q, h, 7)
        E.backward()
    stream.synchronize()
    h.profile(False)
    prof = h.profile_read()
    h.close()
    pairs = wl.n * wl.params.P
    # SFU work: forward and backward each take the structure factors (sin and
    # cos per pair) and the Fourier force with dE/dq (sin and cos per pair)
    sfu_ops = 2 * 4 * pairs
    return {"workload": wl.name, "N": wl.n, "P": wl.params.P, "ms_per_fwd_bwd": ms,
            "fwd_bwd_per_s": 1e3 / ms, "particle_steps_per_s": wl.n / (ms / 1e3),
            "iterations": K,
            "kernels_avg_us": {k: t / c * 1e3 for k, (t, c) in prof.items() if c},
            "sfu_roofline": {"bound": "alu", "achieved": sfu_ops / (ms / 1e3) / 1e12,
                             "peak": units["sfu"], "unit": "Tsfu/s",
                             "frac": sfu_ops / (ms / 1e3) / 1e12 / units["sfu"],
                             "note": "whole forward + backward (8 SFU ops per particle-wave-"
                                     "vector pair) over its wall time, real space included"}}


def measure_small_fp64_loop(rbe, torch, dev, stream):
    """The 1:1 electrolyte N = 1000 (L = 25, P = 100): 100 Langevin steps of the
    plain FP64 path in one call (and of the mixed path), CUDA events."""
    from paper_2010_01559_gb300 import workloads
    wl = workloads.config_small_fp64()
    out = {"workload": wl.name, "N": wl.n, "P": wl.params.P}
    for name, dt in (("fp64", torch.float64), ("mixed", torch.float32)):
        h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
        pos, vel = _state(torch, wl, dev, dt)
        step = torch.zeros(1, dtype=torch.int64, device=dev)
        with torch.cuda.stream(stream):
            if dt == torch.float32:
                h.autotune(pos)
            h.set_graph(True)
            h.step(pos, vel, 5, step)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.step(pos, vel, 100, step)
            e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = {"ms_100_steps": ms, "ms_per_step": ms / 100,
                     "particle_steps_per_s": wl.n * 100 / (ms / 1e3)}
        h.close()
    return out


def oracle_timings(large_all_cores=None):
    """The oracle (as it stands) on this host: one force evaluation of each
    workload at 1 thread and on all cores (the water-like system at 1 thread
    and the large system sampled and scaled, see oracle_large_estimate), the
    small electrolyte's 100 Langevin steps, and the paper's own CPU timings
    for context."""
    import numpy as np
    import oracle
    from paper_2010_01559_gb300 import workloads as wls
    oracle.build()
    out = {"host_cores": cpu_cores(), "paper": {"hardware": PAPER_HARDWARE,
                                                "timings": PAPER_CPU_TIMINGS}}
    evals = {}
    for name, wl in (("electrolyte_1to1_N1000", wls.config_small_fp64()),
                     ("electrolyte_2to1_N8001", wls.config_2to1_mixed()),
                     ("water_like_30000", wls.config_water())):
        pos64, q64 = _f64(wl)
        row = {"N": wl.n, "P": wl.params.P}
        for th in (1, 0):
            if th == 1 and wl.n > 10000:
                row["threads_1"] = oracle_large_estimate(wl, 1, nsub=wl.n // 10)
                continue
            used = oracle.set_threads(th)
            oracle_eval_seconds(wl, 0, pos64=pos64, q64=q64)            # warm
            reps = 3 if wl.n <= 10000 else 1
            t = sum(oracle_eval_seconds(wl, s + 1, pos64=pos64, q64=q64) for s in range(reps))
            t /= reps
            row[f"threads_{used}"] = {"seconds_per_eval": t, "force_evals_per_s": 1 / t,
                                      "particle_steps_per_s": wl.n / t}
        evals[name] = row
    big = wls.config_large()
    evals[big.name] = {"N": big.n, "P": big.params.P,
                       "all_cores": large_all_cores or oracle_large_estimate(big, 0,
                                                                             rho_slice=1 << 18),
                       "one_thread": oracle_large_estimate(big, 1, rho_slice=1 << 15, nsub=256)}
    out["force_eval"] = evals
    # the small electrolyte's 100 Langevin steps (Sec. 3.3), all cores and 1 thread
    wl = wls.config_small_fp64()
    p = wl.params
    loop = {}
    for th in (0, 1):
        used = oracle.set_threads(th)
        pos, vel = _f64(wl)[0].copy(), wl.vel.astype(np.float64)
        q = wl.q.astype(np.float64)
        t0 = time.perf_counter()
        for s in range(100):
            r = oracle.rbe_forces(pos, q, p.box, p.alpha, p.r_c, p.P, p.seed, p.stream, s,
                                  lB=p.coulomb_prefactor, lj_eps=p.lj_eps, lj_sigma=p.lj_sigma,
                                  lj_rcut=p.lj_rcut)
            pos, vel = oracle.langevin_step(pos, vel, r["F"], p.box, p.gamma, p.kT, p.dt, p.mass,
                                            p.seed, p.stream, s)
        t = time.perf_counter() - t0
        loop[f"threads_{used}"] = {"seconds_100_steps": t, "ms_per_step": t * 10,
                                   "particle_steps_per_s": wl.n * 100 / t}
    oracle.set_threads(0)
    out["small_100_step_loop"] = loop
    return out


def run_ours(args):
    import numpy as np  # noqa: F401
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
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    # ---------------------------------------------------------------- headline
    h, pos, vel, step_dev, tuning, hl = measure_headline(rbe, torch, wl, args, world, local,
                                                         dev, stream, flush)
    units = unit_peaks(rbe, hl["clocks"].get("sm_mhz"))
    # per-kernel profile of the same steps (events around each kernel): once as
    # the timed steps run them (structure factors and standing-list pass in one
    # launch), once with the two launched apart, each timed alone
    fused = h.get_fusion()
    nprof = max(3, min(K, 50))
    timed_steps(torch, h, pos, vel, step_dev, nprof, stream, flush, profile=True)
    prof_step = h.profile_read()
    h.set_fusion(False)
    timed_steps(torch, h, pos, vel, step_dev, nprof, stream, flush, profile=True)
    prof = h.profile_read()
    h.set_fusion(None)
    kernels_us = {k: (ms / c * 1e3 if c else 0.0) for k, (ms, c) in prof.items() if c}
    step_kernels_us = {k: (ms / c * 1e3 if c else 0.0) for k, (ms, c) in prof_step.items()
                       if c}
    acc = step_accuracy(torch, h, pos, vel, step_dev, stream)
    stats = h.list_stats()
    e2e_t = measure_e2e(torch, h, wl, K, stream, flush, world, dev)
    h.close()
    del pos, vel
    e2e_value = hl["particles"] * K / e2e_t
    bytes_io = 2 * 16 * wl.n
    same = fp64_and_same_algorithm(rbe, torch, wl, dev, stream, flush, K) if rank == 0 else None

    result = None
    if rank == 0:
        counts = pair_counts(wl)
        value = hl["value"]
        v64 = same["fp64"]["value"]
        vcs = same["mixed_cell_scan"]["value"]
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": hl["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "N": wl.n, "P": wl.params.P,
                       "alpha": wl.params.alpha, "r_c": wl.params.r_c,
                       "box": round(wl.params.box, 4), "density": 0.064,
                       "path": "mixed (FP32 phases/forces, FP64 rho(k) and energy sums), "
                               "neighbour-list MD steps, Langevin", "graph": True,
                       "l2": "flushed between timed steps (256 MiB write, untimed)",
                       "timed_region": f"{hl['reps']} x {K} steps, each block bracketed by "
                                       f"barrier + synchronize (repeated until "
                                       f"{MIN_TIMED_SECONDS} s had passed)",
                       "tuning": {"rho_chunk": tuning[0], "force_split": tuning[1],
                                  "real_split": tuning[2], "real_seg": tuning[3],
                                  "list_split": tuning[4]},
                       "fused_list_step": fused,
                       "parallelism": f"replicas x{world}"},
            "force_evals_per_s": value / wl.n,
            "clocks": hl["clocks"],
            "roofline": roofline(prof_step, wl, peaks, units, counts=counts),
            "fourier_rooflines": fourier_rooflines(prof, wl, units),
            "list_pass_roofline": list_pass_roofline(prof, wl, peaks, counts),
            "unit_peaks": {k: units[k] for k in ("sfu", "alu", "probe", "sfu_basis")},
            "kernels_avg_us": kernels_us,
            "step_kernels_avg_us": step_kernels_us,
            "kernels_note": "step_kernels_avg_us: the kernels as the timed steps launch them "
                            "(rho_list = structure factors + standing-list pass in one launch; "
                            "real = the pass after a list rebuild); kernels_avg_us: the same "
                            "steps with the two launched apart, each timed alone",
            "gpu_launches": hl["launches"],
            "gpu_launches_per_step": hl["launches_per_step"],
            "list_stats": stats,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": bytes_io,
                    "d2h_bytes_per_step": bytes_io, "steps": K,
                    "api": "rbe_step_host on pinned host pos/vel (float32 [N, 4] each): every "
                           "step's kernels read and write the page-locked arrays in place over "
                           "the host link; the call returns when the closing kernel's "
                           "completion word reaches mapped host memory"},
            "fp64_path": same["fp64"],
            "speedup_vs_fp64": value / v64,
            "speedup_same_algorithm": {
                "mixed_cell_scan": same["mixed_cell_scan"],
                "precision_only": vcs / v64,
                "neighbour_list_only": value / vcs,
                "note": "speedup_vs_fp64 = precision_only x neighbour_list_only: the FP64 path "
                        "and mixed_cell_scan run the same per-step cell scan, so their ratio is "
                        "what FP32 arithmetic (fixed-point phases, polar-form Fourier force) "
                        "buys; the rest is the Verlet list of the mixed MD step"},
            "accuracy": acc,
        }
        if not args.no_extras:
            from paper_2010_01559_gb300 import workloads as wls
            extra = {}
            extra["electrolyte_2to1_N8001"] = measure_system(rbe, torch, wls.config_2to1_mixed(),
                                                             dev, stream, flush, peaks, units)
            extra["water_like_autograd"] = measure_water_autograd(rbe, torch, dev, stream,
                                                                  flush, units)
            extra["small_fp64_100_steps"] = measure_small_fp64_loop(rbe, torch, dev, stream)
            extra["batched_replicas"] = measure_replicas(rbe, torch, wls, dev, stream, flush)
            extra["scaling"] = scaling_sweep(rbe, torch, wls, dev, stream, flush) + [
                {"N": wl.n, "ms_per_step": hl["ms_per_step"], "value": value}]
            extra["paper_literal"] = measure_paper_literal(rbe, torch, wls.config_2to1_mixed(),
                                                           dev, stream, flush, units)
            result["extra"] = extra
        if not args.no_cpu_baseline:
            result["cpu_baseline"] = cpu_baseline(wl)
            if not args.no_extras:
                cb = result["cpu_baseline"]
                result["oracle_timings"] = oracle_timings(
                    {"threads": cb["cores"], "seconds_per_eval": cb["seconds_per_eval"],
                     "force_evals_per_s": 1.0 / cb["seconds_per_eval"],
                     "particle_steps_per_s": cb["value"], "sample": cb["sample"],
                     "seconds_per_particle": cb["seconds_per_particle"]})
        print(json.dumps(result), flush=True)
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
    out = {"workload": wl.name}
    for name, kw in (("mh_sampler", dict(sampler=1)),
                     ("andersen", dict(thermostat=1, andersen_nu=10.0))):
        sp = copy.copy(wl.params)
        for k, v in kw.items():
            setattr(sp, k, v)
        w2 = copy.copy(wl)
        w2.params = sp
        h, pos, vel, step, _ = md_handle(rbe, torch, w2, dev, stream, warm=5)
        ms = timed_steps(torch, h, pos, vel, step, K, stream, flush) / K
        out[name] = {"ms_per_step": ms, "value": wl.n / (ms / 1e3), "unit": UNIT, "steps": K}
        if name == "mh_sampler":
            timed_steps(torch, h, pos, vel, step, 20, stream, flush, profile=True)
            pr = h.profile_read()
            out[name]["prep_us"] = pr["prep"][0] / max(pr["prep"][1], 1) * 1e3
        h.close()
    # observables: full Ewald over |m| <= M (the sampler's table half-width)
    h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    pos, vel = _state(torch, wl, dev)
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
        h, pos, vel, step, _ = md_handle(rbe, torch, wl, dev, stream)
        ms = timed_steps(torch, h, pos, vel, step, 30, stream, flush) / 30
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
    ms = timed_steps(torch, h, pos, vel, step_dev, K, stream, flush)
    stats = h.list_stats()
    h.close()
    return {"workload": f"{len(reps)} replicas, 1:1 electrolyte, N log-uniform in [1000, 65536], "
                        f"density 0.064, P = 100", "systems": len(reps), "N_total": n_all,
            "value": n_all * K / (ms / 1e3), "unit": UNIT, "steps": K, "ms_per_step": ms / K,
            "tuning": list(tuning), "list_builds": stats["builds"]}


# --------------------------------------------------------------------- reference arm
def run_reference(args):
    """The FP64 CPU oracle as it stands, on this host's cores, same workload and
    metric.  Each step is one oracle force evaluation of the benchmark system,
    sampled: rho(k) over all particles and the forces of 256 evenly spaced
    particles (a different set each step); its time is scaled to all N with
    the structure-factor share measured once.  Steps run until K are done or
    the --cpu-seconds budget is spent."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import numpy as np
    import oracle
    oracle.build()
    wl = workload()
    K, W = args.steps, args.warmup
    p = wl.params
    threads = oracle.set_threads(0)
    pos64, q64 = _f64(wl)
    nsub = 256
    stride = wl.n // nsub
    m, _, _ = oracle.sample_k(p.alpha, p.box, p.seed, p.stream, 0, p.P)
    t0 = time.perf_counter()
    oracle.rbe_fourier(pos64, q64, p.box, p.alpha, m, lB=p.coulomb_prefactor, sub=np.array([0]))
    t_rho = time.perf_counter() - t0
    budget = args.cpu_seconds
    start = time.perf_counter()

    def one(s):
        sub = (np.arange(nsub) * stride + (s % stride)).astype(int)
        t = oracle_eval_seconds(wl, 1000 + s, sub=sub, pos64=pos64, q64=q64)
        return t_rho + max(t - t_rho, 0.0) * wl.n / nsub

    for s in range(min(W, 1)):
        one(s)
    full, done = [], 0
    for s in range(K):
        full.append(one(W + s))
        done += 1
        if time.perf_counter() - start > budget:
            break
    t = sum(full)
    value = wl.n * done / t
    sample = (f"{done} of {K} oracle steps: each rho(k) over all {wl.n} particles and the "
              f"forces (Fourier, real space + LJ) of {nsub} evenly spaced particles, scaled to "
              f"all {wl.n} with the rho share measured once ({t_rho:.2f} s)")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
           "steps": K, "warmup": W, "ms_per_step": t * 1e3 / done, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl.name, "N": wl.n, "P": wl.params.P},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads,
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return out


# --------------------------------------------------------------------- profile case
def profile_case(args):
    """A few MD steps of one workload inside cudaProfilerStart/Stop, for
    `ncu --profile-from-start off`: the handle is built, the launch shape
    fixed (--tuning) or autotuned, --warmup steps run outside the range, then
    --steps steps inside it.  Prints the mean step time."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2010_01559_gb300 import RBE, params_from, workloads
    if args.profile_case == "2to1":
        wl = workloads.config_2to1_mixed()
    elif args.profile_case == "large":
        wl = workloads.config_large(args.n or (1 << 20))
    else:
        wl = workloads.config_water(args.n or 10000)
    h = RBE(params_from(wl.params, n_max=wl.n))
    dt = torch.float32 if args.precision == "mixed" else torch.float64
    pos = torch.from_numpy(wl.pos_q()).cuda().to(dt).contiguous()
    vel = torch.zeros((wl.n, 4), dtype=dt, device="cuda")
    vel[:, :3] = torch.from_numpy(wl.vel).cuda().to(dt)
    if args.tuning:
        h.set_tuning(*[int(v) for v in args.tuning.split(",")])
    elif args.precision == "mixed":
        h.autotune(pos)
    h.set_graph(args.graph)
    h.set_fusion({"auto": None, "on": True, "off": False}[args.fusion])
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.step(pos, vel, args.warmup, step)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()
    e0.record()
    h.step(pos, vel, args.steps, step)
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"workload": wl.name, "N": wl.n, "tuning": list(h.get_tuning()),
                      "fused_list_step": h.get_fusion(),
                      "steps": args.steps, "ms_per_step": e0.elapsed_time(e1) / args.steps}))
    h.close()


def main():
    args = parse()
    if args.profile_case:
        profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

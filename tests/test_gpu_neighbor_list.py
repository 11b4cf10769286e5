"""The neighbour list of the mixed MD step (pairs within r_c + skin, rebuilt
when a particle has moved more than skin/2) against the cell scan and the
oracle.

Each step's total force comes out through rbe_step_ex.  At the same positions
and step index the Fourier part is bit-identical between the list step and a
forces call (same fixed-point structure factors, same kernels), so the
difference of the two is the real-space sum's FP32 summation order alone --
about 1e-6 -- while one pair within r_c missing from the list would move a
particle's force by ~1e-4 (the erfc and Gaussian terms near r_c at these alpha
and r_c, times |q_i q_j| >= 1).  The per-particle bound 1e-5 + 1e-6 |F| sits
between the two.
"""
import copy

import numpy as np
import pytest

from gpu_util import assert_per_particle, need_gpu, oracle_eval, rel_rms
from paper_2010_01559_gb300 import capi, workloads

pytestmark = pytest.mark.gpu
TOL_MIXED = 1e-5


@pytest.fixture(scope="module")
def rbe():
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_01559_gb300 as rbe
    return rbe


def _no_list(sp):
    sp = copy.copy(sp)
    sp.skin = -1.0
    return sp


def _state(wl, torch, v_scale=1.0):
    pos = torch.from_numpy(wl.pos_q()).cuda().contiguous()
    vel = torch.zeros((wl.n, 4), dtype=torch.float32, device="cuda")
    vel[:, :3] = torch.from_numpy(wl.vel * v_scale).cuda()
    return pos, vel


def _check_same(F_list, F_cell, what):
    a = F_list[:, :3].cpu().numpy().astype(np.float64)
    b = F_cell[:, :3].cpu().numpy().astype(np.float64)
    dev = np.linalg.norm(a - b, axis=1)
    bound = 1e-5 + 1e-6 * np.linalg.norm(b, axis=1)
    worst = int(np.argmax(dev / bound))
    assert np.all(dev <= bound), (what, worst, dev[worst], bound[worst])
    return float(dev.max())


def test_list_step_forces_match_cell_scan_every_step_with_frequent_rebuilds(rbe):
    """Small skin (0.1) and particles at 9 kT: a rebuild every few steps, and
    each of 30 steps' forces equal to the cell scan's at the same positions."""
    import torch
    wl = workloads.config_2to1_mixed()
    sp = copy.copy(wl.params)
    sp.skin = 0.1
    h = rbe.RBE(rbe.params_from(sp, n_max=wl.n))
    h.set_graph(True)
    hc = rbe.RBE(rbe.params_from(_no_list(sp), n_max=wl.n))
    pos, vel = _state(wl, torch, 3.0)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    F = torch.zeros((wl.n, 4), dtype=torch.float32, device="cuda")
    worst = 0.0
    for s in range(30):
        before = pos.clone()
        h.step(pos, vel, 1, step, F_out=F)
        Fc, _, _ = hc.forces(before, s, energy=False)
        torch.cuda.synchronize()
        worst = max(worst, _check_same(F, Fc, s))
    st = h.list_stats()
    h.sync()
    print("list stats", st, "largest |dF|", worst)
    assert st["builds"] >= 5                        # the skin was crossed again and again
    assert 0 < st["max_count"] <= st["capacity"]
    h.close()
    hc.close()


def test_list_step_force_matches_oracle_after_60_steps(rbe):
    """Default skin, Langevin at kT: the step force after 60 list steps against
    the oracle's estimator at the same positions and step (the mixed-path
    tolerance 1e-5)."""
    import torch
    wl = workloads.config_2to1_mixed()
    h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    h.set_graph(True)
    pos, vel = _state(wl, torch)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.step(pos, vel, 60, step)
    before = pos.clone()
    F = torch.zeros((wl.n, 4), dtype=torch.float32, device="cuda")
    h.step(pos, vel, 1, step, F_out=F)
    h.sync()
    w2 = copy.copy(wl)
    w2.pos = before[:, :3].cpu().numpy()
    ref = oracle_eval(w2, 60)
    err = rel_rms(F[:, :3].cpu().numpy(), ref["F"])
    print("list step force vs oracle rel-RMS", err, h.list_stats())
    assert err <= TOL_MIXED
    assert_per_particle(F[:, :3].cpu().numpy(), ref["F"], "list step after 60 steps")
    h.close()


def test_list_across_forces_calls_and_after_caller_moves_particles(rbe):
    import torch
    wl = workloads.config_small_fp64()
    h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    hc = rbe.RBE(rbe.params_from(_no_list(wl.params), n_max=wl.n))
    pos, vel = _state(wl, torch)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    F = torch.zeros((wl.n, 4), dtype=torch.float32, device="cuda")
    h.step(pos, vel, 5, step)
    b0 = h.list_stats()["builds"]
    # a mixed forces call at these positions goes over the same list: no rebuild
    Ff, _, _ = h.forces(pos, 5, energy=False)
    assert h.list_stats()["builds"] == b0
    _check_same(Ff, hc.forces(pos, 5, energy=False)[0], "forces call over the list")
    # an FP64 forces call reorders the shared sorted arrays: the next step rebuilds
    h.forces_f64(pos.double().contiguous(), 5, energy=False)
    before = pos.clone()
    h.step(pos, vel, 1, step, F_out=F)
    assert h.list_stats()["builds"] == b0 + 1
    _check_same(F, hc.forces(before, 5, energy=False)[0], "after an FP64 forces call")
    # the caller moves one particle by half a box edge: the next step sees it
    b1 = h.list_stats()["builds"]
    pos[17, 0] = (pos[17, 0] + 0.5 * wl.params.box) % wl.params.box
    before = pos.clone()
    h.step(pos, vel, 1, step, F_out=F)
    assert h.list_stats()["builds"] == b1 + 1
    _check_same(F, hc.forces(before, 6, energy=False)[0], "after a teleport")
    # nothing moved beyond skin/2 in one step at kT: no rebuild
    before = pos.clone()
    h.step(pos, vel, 1, step, F_out=F)
    assert h.list_stats()["builds"] == b1 + 1
    _check_same(F, hc.forces(before, 7, energy=False)[0], "list reused")
    h.close()
    hc.close()


def test_list_heterogeneous_batch_matches_oracle_per_system(rbe):
    import torch
    e = workloads.electrolyte_1to1
    systems = [e(600, 0.05, 0.25, 5.5, 60, seed=31, stream=1),
               e(900, 0.08, 0.35, 4.5, 150, seed=32, stream=2, thermostat=1, andersen_nu=20.0,
                 dt=2e-3),
               e(400, 0.064, 0.3, 5.0, 40, seed=33, stream=3, thermostat=2, nh_tau=0.05),
               e(300, 0.064, 0.2, 6.0, 30, seed=34, stream=4)]        # one cell: r_c > L/3
    h = rbe.RBEBatch([rbe.params_from(w.params) for w in systems], [w.n for w in systems])
    pos = torch.from_numpy(np.concatenate([w.pos_q() for w in systems])).cuda()
    vel = torch.zeros((pos.shape[0], 4), dtype=torch.float32, device="cuda")
    vel[:, :3] = torch.from_numpy(np.concatenate([w.vel for w in systems])).cuda()
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.step(pos, vel, 25, step)
    before = pos.clone()
    F = torch.zeros_like(pos)
    h.step(pos, vel, 1, step, F_out=F)
    h.sync()
    off = 0
    for w in systems:
        w2 = copy.copy(w)
        w2.pos = before[off:off + w.n, :3].cpu().numpy()
        ref = oracle_eval(w2, 25)
        err = rel_rms(F[off:off + w.n, :3].cpu().numpy(), ref["F"])
        print(w.name, w.n, "rel-RMS", err)
        assert err <= TOL_MIXED, (w.name, err)
        assert_per_particle(F[off:off + w.n, :3].cpu().numpy(), ref["F"], w.name)
        off += w.n
    assert h.list_stats()["builds"] >= 1
    h.close()


def test_list_overflow_is_reported_not_silent(rbe):
    """A dense cluster in a dilute box exceeds the capacity sized from the mean
    density: the overflow is latched and rbe_sync reports RBE_ERR_LIST."""
    import torch
    rng = np.random.default_rng(5)
    L, n = 40.0, 2000
    p = workloads.SystemParams(box=L, alpha=0.3, r_c=5.0, P=50, seed=5, lj_eps=0.0)
    xyz = rng.uniform(0, L, (n, 3))
    xyz[:300] = 20.0 + rng.uniform(-2.0, 2.0, (300, 3))       # 300 ions within a 4^3 cube
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    pos = torch.from_numpy(np.concatenate([xyz, q[:, None]], axis=1).astype(np.float32)).cuda()
    vel = torch.zeros_like(pos)
    h = rbe.RBE(rbe.params_from(p, n_max=n))
    assert h.list_stats()["capacity"] < 300
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.step(pos, vel, 1, step)
    with pytest.raises(capi.RBEError) as ei:
        h.sync()
    assert ei.value.status == capi.RBE_ERR_LIST
    h.sync()                                             # the latch was cleared
    # a host-buffer step on page-locked arrays returns the error itself (the
    # closing kernel delivers the error word with its completion word)
    hp, hv = pos.cpu().pin_memory(), vel.cpu().pin_memory()
    hp[:, :3] += 0.5                                     # moved > skin/2: a rebuild
    with pytest.raises(capi.RBEError) as ei:
        h.step_host(hp, hv, 1, 1)
    assert ei.value.status == capi.RBE_ERR_LIST
    h.sync()
    h.close()


def test_list_step_with_mh_sampler_matches_oracle_chain(rbe):
    """The paper's MH sampler on list steps: after 30 steps, the step force at
    the positions it started from equals the oracle's estimator on the batch
    its chain yields for that (31st) evaluation."""
    import torch
    import oracle
    wl = workloads.config_small_fp64()
    sp = copy.copy(wl.params)
    sp.sampler = 1
    h = rbe.RBE(rbe.params_from(sp, n_max=wl.n))
    h.set_graph(True)
    pos, vel = _state(wl, torch)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.step(pos, vel, 30, step)
    before = pos.clone()
    F = torch.zeros((wl.n, 4), dtype=torch.float32, device="cuda")
    h.step(pos, vel, 1, step, F_out=F)
    h.sync()
    chain = oracle.MHChain(sp.alpha, sp.box, sp.seed, sp.stream)
    for _ in range(30):
        chain.draw(sp.P)
    m = chain.draw(sp.P)
    ref = oracle.rbe_forces(before[:, :3].cpu().numpy().astype(np.float64),
                            wl.q.astype(np.float64), sp.box, sp.alpha, sp.r_c, sp.P, sp.seed,
                            sp.stream, 30, lB=sp.coulomb_prefactor, lj_eps=sp.lj_eps,
                            lj_sigma=sp.lj_sigma, lj_rcut=sp.lj_rcut, m=m)
    err = rel_rms(F[:, :3].cpu().numpy(), ref["F"])
    print("MH list step force vs oracle rel-RMS", err)
    assert err <= TOL_MIXED
    assert_per_particle(F[:, :3].cpu().numpy(), ref["F"], "MH list step")
    h.close()


def test_list_step_on_water_like_system_matches_oracle(rbe):
    """A dense, strongly bound charge distribution (rigid 3-site molecules as
    free point charges, ~560 neighbours within r_c + skin per atom): after 15
    list steps, the step force at the positions it started from against the
    oracle's estimator."""
    import torch
    wl = workloads.config_water(1500)
    h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    h.set_graph(True)
    pos, vel = _state(wl, torch)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.step(pos, vel, 15, step)
    before = pos.clone()
    F = torch.zeros((wl.n, 4), dtype=torch.float32, device="cuda")
    h.step(pos, vel, 1, step, F_out=F)
    h.sync()
    st = h.list_stats()
    w2 = copy.copy(wl)
    w2.pos = before[:, :3].cpu().numpy()
    ref = oracle_eval(w2, 15)
    err = rel_rms(F[:, :3].cpu().numpy(), ref["F"])
    print("water list step force vs oracle rel-RMS", err, st)
    assert st["max_count"] > 400 and st["max_count"] <= st["capacity"]
    assert err <= TOL_MIXED
    assert_per_particle(F[:, :3].cpu().numpy(), ref["F"], "water list step")
    h.close()


def test_list_survives_particle_count_change_and_fp64_steps(rbe):
    """One single-system handle: list steps with all 1000 particles, then with
    the first 800 (a smaller n re-prepares the work tables; the list is built
    afresh), then an FP64 step in between mixed ones (it reorders the shared
    sorted arrays): each mixed step force against the cell scan at the same
    positions."""
    import torch
    wl = workloads.config_small_fp64()
    h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    hc = rbe.RBE(rbe.params_from(_no_list(wl.params), n_max=wl.n))
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    pos, vel = _state(wl, torch)
    h.step(pos, vel, 5, step)
    F = torch.zeros((wl.n, 4), dtype=torch.float32, device="cuda")
    before = pos.clone()
    h.step(pos, vel, 1, step, F_out=F)
    _check_same(F, hc.forces(before, 5, energy=False)[0], "n = 1000")
    m = 800                                              # the first 800 particles
    p2, v2 = pos[:m].clone(), vel[:m].clone()
    b0 = h.list_stats()["builds"]
    before = p2.clone()
    F2 = torch.zeros((m, 4), dtype=torch.float32, device="cuda")
    h.step(p2, v2, 1, step, F_out=F2)
    assert h.list_stats()["builds"] == b0 + 1
    _check_same(F2, hc.forces(before, 6, energy=False)[0], "n = 800")
    p64, v64 = p2.double().contiguous(), v2.double().contiguous()
    h.step(p64, v64, 1, step)                            # FP64 step, index 7
    p2, v2 = p64.float().contiguous(), v64.float().contiguous()
    b1 = h.list_stats()["builds"]
    before = p2.clone()
    h.step(p2, v2, 1, step, F_out=F2)
    assert h.list_stats()["builds"] == b1 + 1            # rebuilt after the FP64 step
    _check_same(F2, hc.forces(before, 8, energy=False)[0], "after an FP64 step")
    h.sync()
    h.close()
    hc.close()

"""The kernels an MD step launches, in every launch shape, against the oracle.

An MD step on the mixed path runs the Fourier force in its step mode (one sine
per particle-wave-vector pair, no dE/dq, closing thermostat update) and the
real-space pass over the neighbour list in its step mode (real-space force
only, handed to the closing update).  Forces calls run other instantiations
of both kernels, so these tests take each step's total force out through
rbe_step_ex and compare it with

* the oracle's estimator (Eq. rbmapprox plus the real-space and LJ terms of
  Eq. force and Eq. Ljpotential) at the positions the step started from and
  the step's own k-batch: rel-RMS <= 1e-5 and a per-particle bound;
* a forces call of a handle without a neighbour list (the cell scan) at the
  same positions and step, with the same structure-factor chunk: the Fourier
  part is computed from the same fixed-point structure factors (the FP32
  partial sums of rho(k) run over the same particles in the same order), so
  the two differ by FP32 summation order only (per particle <= 1e-5 +
  1e-6 |F|, while one pair within r_c missing from the list moves a force by
  ~1e-4).

At N = 8001 every lane split of both kernels runs (1, 2, 4, 8 threads per
particle; 1 means two particles per thread in the Fourier force); at N = 2^20
the launch shapes the autotuner picks for the benchmark, and the two list
splits it chooses between.
"""
import copy

import numpy as np
import pytest

from gpu_util import assert_per_particle, need_gpu, oracle_eval, rel_rms
from paper_2010_01559_gb300 import workloads

pytestmark = pytest.mark.gpu
TOL_MIXED = 1e-5


@pytest.fixture(scope="module")
def rbe():
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_01559_gb300 as rbe
    return rbe


def _state(wl, torch):
    pos = torch.from_numpy(wl.pos_q()).cuda().contiguous()
    vel = torch.zeros((wl.n, 4), dtype=torch.float32, device="cuda")
    vel[:, :3] = torch.from_numpy(wl.vel).cuda()
    return pos, vel


def _no_list(sp):
    sp = copy.copy(sp)
    sp.skin = -1.0
    return sp


def _check_same(F_step, F_cell, what):
    a = F_step[:, :3].cpu().numpy().astype(np.float64)
    b = F_cell[:, :3].cpu().numpy().astype(np.float64)
    dev = np.linalg.norm(a - b, axis=1)
    bound = 1e-5 + 1e-6 * np.linalg.norm(b, axis=1)
    worst = int(np.argmax(dev / bound))
    assert np.all(dev <= bound), (what, worst, dev[worst], bound[worst])
    return float(dev.max())


def _step_force(h, pos, vel, step, torch):
    """One MD step; returns (positions it started from, its total force, step index)."""
    before = pos.clone()
    k = int(step.item())
    F = torch.zeros_like(pos)
    h.step(pos, vel, 1, step, F_out=F)
    h.sync()
    return before, F, k


@pytest.mark.parametrize("force_split", [1, 2, 4, 8])
@pytest.mark.parametrize("list_split", [1, 2, 4, 8])
def test_md_step_kernels_every_split_n8001(rbe, force_split, list_split):
    import torch
    wl = workloads.config_2to1_mixed()
    h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    h.set_tuning(128, force_split, 3, 0, list_split)
    h.set_graph(True)
    hc = rbe.RBE(rbe.params_from(_no_list(wl.params), n_max=wl.n))
    hc.set_tuning(128, 0, 0, 0, 0)
    pos, vel = _state(wl, torch)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    # step 0 builds the list (the pass after the rebuild), step 3 walks the
    # standing list (the pass launched right after prep)
    checked = []
    for s in range(4):
        before, F, k = _step_force(h, pos, vel, step, torch)
        if s not in (0, 3):
            continue
        w2 = copy.copy(wl)
        w2.pos = before[:, :3].cpu().numpy()
        ref = oracle_eval(w2, k)
        err = rel_rms(F[:, :3].cpu().numpy(), ref["F"])
        assert err <= TOL_MIXED, (force_split, list_split, k, err)
        assert_per_particle(F[:, :3].cpu().numpy(), ref["F"], (force_split, list_split, k))
        Fc, _, _ = hc.forces(before, k, energy=False)
        torch.cuda.synchronize()
        _check_same(F, Fc, (force_split, list_split, k))
        checked.append((k, err))
    assert h.get_tuning()[1] == force_split and h.get_tuning()[4] == list_split
    print("force_split", force_split, "list_split", list_split, checked, h.list_stats())
    h.close()
    hc.close()


@pytest.fixture(scope="module")
def large():
    return workloads.config_large()


def test_md_step_kernels_at_2p20_in_the_benchmark_launch_shapes(rbe, large):
    """N = 2^20, P = 500: the autotuned shapes (as the benchmark picks them),
    then list splits 1 and 2 with one Fourier-force thread per two particles;
    each step's force against the oracle on 1024 evenly spaced particles and
    against the cell scan over all 2^20."""
    import torch
    wl = large
    h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    hc = rbe.RBE(rbe.params_from(_no_list(wl.params), n_max=wl.n))
    pos, vel = _state(wl, torch)
    tuned = h.autotune(pos)
    h.set_graph(True)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.step(pos, vel, 2, step)
    sub = np.linspace(0, wl.n - 1, 1024).astype(int)
    shapes = [tuple(tuned), (tuned[0], 1, tuned[2], tuned[3], 2),
              (tuned[0], 1, tuned[2], tuned[3], 1)]
    for shape in shapes:
        h.set_tuning(*shape)
        hc.set_tuning(shape[0], 0, 0, 0, 0)
        h.step(pos, vel, 1, step)             # the list is rebuilt after a tuning change
        before, F, k = _step_force(h, pos, vel, step, torch)
        assert h.get_tuning() == shape
        w2 = copy.copy(wl)
        w2.pos = before[:, :3].cpu().numpy()
        ref = oracle_eval(w2, k, sub=sub)
        Fs = F[:, :3].cpu().numpy()[sub]
        err = rel_rms(Fs, ref["F"])
        print("2^20 step", k, "shape", shape, "rel-RMS vs oracle (1024 sampled)", err)
        assert err <= TOL_MIXED, (shape, err)
        assert_per_particle(Fs, ref["F"], shape)
        Fc, _, _ = hc.forces(before, k, energy=False)
        torch.cuda.synchronize()
        worst = _check_same(F, Fc, shape)
        print("  largest |dF| against the cell scan over all 2^20:", worst)
    h.close()
    hc.close()


def _fusion_pair(rbe, wl, tuning, torch):
    hf = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    hs = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    hf.set_fusion(True)
    hs.set_fusion(False)
    for h in (hf, hs):
        h.set_tuning(*tuning)
        h.set_graph(True)
    return hf, hs


@pytest.mark.parametrize("list_split", [1, 2, 4, 8])
def test_fused_and_separate_launches_agree_bitwise_n8001(rbe, list_split):
    """The structure factors and the standing-list pass in one launch or in
    two: the same trajectory to the last bit (rho(k) is summed in the same
    order and added in fixed point; each particle's list terms are added by
    the same lanes in the same order), over steps that build the list and
    steps that walk it."""
    import torch
    wl = workloads.config_2to1_mixed()
    hf, hs = _fusion_pair(rbe, wl, (128, 1, 3, 0, list_split), torch)
    pf, vf = _state(wl, torch)
    ps, vs = pf.clone(), vf.clone()
    sf = torch.zeros(1, dtype=torch.int64, device="cuda")
    ss = sf.clone()
    for s in range(6):
        _, Ff, kf = _step_force(hf, pf, vf, sf, torch)
        _, Fs, ks = _step_force(hs, ps, vs, ss, torch)
        assert kf == ks == s
        assert torch.equal(Ff, Fs), (list_split, s)
        assert torch.equal(pf, ps) and torch.equal(vf, vs), (list_split, s)
    # profiled, the fused launch has its own slot and the separate pass none
    hf.profile(True)
    _step_force(hf, pf, vf, sf, torch)
    prof = hf.profile_read()
    hf.profile(False)
    assert prof["rho_list"][1] == 1 and prof["rho"][1] == 0, prof
    hf.close()
    hs.close()


def test_fused_and_separate_launches_agree_bitwise_at_2p20(rbe, large):
    """As above at N = 2^20 in the autotuned launch shapes."""
    import torch
    wl = large
    h0 = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    pf, vf = _state(wl, torch)
    tuned = tuple(h0.autotune(pf))
    h0.close()
    hf, hs = _fusion_pair(rbe, wl, tuned, torch)
    ps, vs = pf.clone(), vf.clone()
    sf = torch.zeros(1, dtype=torch.int64, device="cuda")
    ss = sf.clone()
    for s in range(4):
        _, Ff, _ = _step_force(hf, pf, vf, sf, torch)
        _, Fs, _ = _step_force(hs, ps, vs, ss, torch)
        assert torch.equal(Ff, Fs), (tuned, s)
        assert torch.equal(pf, ps) and torch.equal(vf, vs), (tuned, s)
    print("2^20 fused vs separate: bitwise equal over 4 steps, shape", tuned)
    hf.close()
    hs.close()


def test_fusion_choice(rbe):
    """Automatic fusion: before an autotune a system of 2^19 particles or more
    fuses and a smaller one does not; the autotuner's choice is reported; an
    explicit setting holds through an autotune; -1, 0 and 1 are the only
    settings."""
    import torch
    wl = workloads.config_2to1_mixed()
    h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    pos, vel = _state(wl, torch)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.step(pos, vel, 1, step)
    assert h.get_fusion() is False
    h.autotune(pos)
    assert h.get_fusion() in (True, False)
    h.set_fusion(True)
    h.autotune(pos)
    assert h.get_fusion() is True
    h.step(pos, vel, 2, step)
    with pytest.raises(rbe.RBEError):
        rbe.capi.check(h.lib.rbe_set_fusion(h._h, 2), h._h)
    h.close()
    big = workloads.config_large(1 << 19)
    hb = rbe.RBE(rbe.params_from(big.params, n_max=big.n))
    pb, vb = _state(big, torch)
    hb.step(pb, vb, 1, torch.zeros(1, dtype=torch.int64, device="cuda"))
    assert hb.get_fusion() is True
    hb.close()


def test_fused_and_separate_agree_bitwise_heterogeneous_batch(rbe):
    """A batch of four systems of different size, P, cutoff and thermostat
    (Langevin, Andersen, Nose-Hoover; one with r_c > L/3): the fused launch's
    multi-system form against the separate launches, the same trajectory to
    the last bit over steps that build the lists and steps that walk them, and
    the fused step's force against the oracle per system."""
    import torch
    e = workloads.electrolyte_1to1
    systems = [e(600, 0.05, 0.25, 5.5, 60, seed=31, stream=1),
               e(900, 0.08, 0.35, 4.5, 150, seed=32, stream=2, thermostat=1, andersen_nu=20.0,
                 dt=2e-3),
               e(400, 0.064, 0.3, 5.0, 40, seed=33, stream=3, thermostat=2, nh_tau=0.05),
               e(300, 0.064, 0.2, 6.0, 30, seed=34, stream=4)]
    hs = []
    for fuse in (True, False):
        h = rbe.RBEBatch([rbe.params_from(w.params) for w in systems], [w.n for w in systems])
        h.set_fusion(fuse)
        h.set_graph(True)
        hs.append(h)
    states = []
    for _ in hs:
        pos = torch.from_numpy(np.concatenate([w.pos_q() for w in systems])).cuda()
        vel = torch.zeros((pos.shape[0], 4), dtype=torch.float32, device="cuda")
        vel[:, :3] = torch.from_numpy(np.concatenate([w.vel for w in systems])).cuda()
        states.append((pos, vel, torch.zeros(1, dtype=torch.int64, device="cuda")))
    for s in range(8):
        outs = [_step_force(h, *st, torch) for h, st in zip(hs, states)]
        (b0, F0, k0), (_, F1, k1) = outs
        assert k0 == k1 == s
        assert torch.equal(F0, F1), s
        assert torch.equal(states[0][0], states[1][0]) and torch.equal(states[0][1], states[1][1])
    off = 0
    for w in systems:
        w2 = copy.copy(w)
        w2.pos = b0[off:off + w.n, :3].cpu().numpy()
        ref = oracle_eval(w2, k0)
        Fs = F0[off:off + w.n, :3].cpu().numpy()
        assert rel_rms(Fs, ref["F"]) <= TOL_MIXED, w.name
        assert_per_particle(Fs, ref["F"], w.name)
        off += w.n
    assert hs[0].get_fusion() is True and hs[1].get_fusion() is False
    for h in hs:
        h.close()

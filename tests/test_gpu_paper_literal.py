"""Algorithm 1 as printed (Sec. 3.1), on the GPU against the oracle:

* the Metropolis-Hastings k-sampler (RBE_SAMPLER_MH): the batches of 60
  consecutive evaluations are bit-exact with the oracle's chains consumed in
  order (single system and a batch of replicas, each on its own chain), and
  the forces at the last one match the oracle's estimator on that batch;
* leapfrog + Andersen (RBE_THERMO_ANDERSEN): the FP64 GPU trajectory equals
  the oracle's (same Philox collisions and velocities) to 1e-9 after 100
  steps, and the mixed path holds the temperature at kT.
"""
import copy

import numpy as np
import pytest

import oracle
from gpu_util import need_gpu, oracle_eval, rel_rms
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


def _mh(wl):
    sp = copy.copy(wl.params)
    sp.sampler = 1
    return sp


def test_mh_batches_bit_exact_with_oracle_chain(rbe):
    import torch
    wl = workloads.config_small_fp64()
    sp = _mh(wl)
    h = rbe.RBE(rbe.params_from(sp, n_max=wl.n))
    x = torch.from_numpy(wl.pos_q()).cuda()
    chain = oracle.MHChain(sp.alpha, sp.box, sp.seed, sp.stream)
    for s in range(60):
        F, E, _ = h.forces(x, s)
        m = h.sample_k(s).cpu().numpy()[:, :3]
        ref = chain.draw(sp.P)
        assert np.array_equal(m, ref), s
    ref_f = oracle.rbe_forces(wl.pos.astype(np.float64), wl.q.astype(np.float64), sp.box,
                              sp.alpha, sp.r_c, sp.P, sp.seed, sp.stream, 59,
                              lB=sp.coulomb_prefactor, lj_eps=sp.lj_eps, lj_sigma=sp.lj_sigma,
                              lj_rcut=sp.lj_rcut, m=ref)
    assert rel_rms(F[:, :3].cpu().numpy(), ref_f["F"]) <= TOL_MIXED


def test_mh_batch_replicas_each_on_its_chain(rbe):
    import torch
    reps = workloads.config_replicas()[:5]
    ps = [_mh(w) for w in reps]
    h = rbe.RBEBatch([rbe.params_from(p) for p in ps], [w.n for w in reps])
    x = torch.from_numpy(np.concatenate([w.pos_q() for w in reps])).cuda()
    chains = [oracle.MHChain(p.alpha, p.box, p.seed, p.stream) for p in ps]
    for s in range(10):
        h.forces(x, s, energy=False)
        m = h.sample_k(s).cpu().numpy()[:, :3]
        off = 0
        for p, ch in zip(ps, chains):
            assert np.array_equal(m[off:off + p.P], ch.draw(p.P)), (s, p.stream)
            off += p.P


def _andersen(wl, nu):
    sp = copy.copy(wl.params)
    sp.thermostat = 1
    sp.andersen_nu = nu
    return sp


def test_andersen_fp64_trajectory_matches_oracle(rbe):
    import torch
    wl = workloads.config_small_fp64()
    sp = _andersen(wl, 20.0)                         # 2 % of the particles collide per step
    h = rbe.RBE(rbe.params_from(sp, n_max=wl.n))
    pos = torch.from_numpy(wl.pos_q()).cuda().double().contiguous()
    vel = torch.zeros((wl.n, 4), dtype=torch.float64, device="cuda")
    vel[:, :3] = torch.from_numpy(wl.vel).cuda().double()
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.step(pos, vel, 100, step)
    h.sync()
    rp, rv = wl.pos.astype(np.float64), wl.vel.astype(np.float64)
    q = wl.q.astype(np.float64)
    hits = 0
    for s in range(100):
        out = oracle.rbe_forces(rp, q, sp.box, sp.alpha, sp.r_c, sp.P, sp.seed, sp.stream, s,
                                lB=sp.coulomb_prefactor, lj_eps=sp.lj_eps, lj_sigma=sp.lj_sigma,
                                lj_rcut=sp.lj_rcut)
        rp, rv, hit = oracle.andersen_step(rp, rv, out["F"], sp.box, sp.andersen_nu, sp.kT,
                                           sp.dt, sp.mass, sp.seed, sp.stream, s)
        hits += int(hit.sum())
    assert hits > 100                                # collisions did happen
    d = pos[:, :3].cpu().numpy() - rp
    d -= sp.box * np.round(d / sp.box)
    assert np.abs(d).max() <= 1e-9
    assert np.abs(vel[:, :3].cpu().numpy() - rv).max() <= 1e-9


def test_andersen_mixed_holds_temperature(rbe):
    import torch
    wl = workloads.config_small_fp64()
    sp = _andersen(wl, 50.0)
    h = rbe.RBE(rbe.params_from(sp, n_max=wl.n))
    h.set_graph(True)
    pos = torch.from_numpy(wl.pos_q()).cuda()
    vel = torch.zeros((wl.n, 4), dtype=torch.float32, device="cuda")
    vel[:, :3] = torch.from_numpy(wl.vel).cuda()
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.step(pos, vel, 1000, step)
    temps = []
    for _ in range(100):
        h.step(pos, vel, 10, step)
        temps.append((vel[:, :3].double() ** 2).sum().item() / (3 * wl.n))
    h.sync()
    T = float(np.mean(temps))
    print("Andersen kinetic temperature", T)
    assert abs(T - sp.kT) < 0.05

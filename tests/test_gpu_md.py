"""MD steps (Algorithm 1 with the Langevin thermostat of Sec. 3.3) on the GPU.

* FP64 GPU trajectory = oracle trajectory (same Philox noise) to 1e-9 after
  100 steps of the 1:1 electrolyte (N = 1000, L = 25);
* mixed vs FP64 GPU trajectory: stated agreement after 100 steps;
* graph replay, host-buffer calls and resume-from-step reproduce the plain
  device calls bit for bit;
* the thermostat holds T = 1 (kinetic temperature after equilibration).
"""
import numpy as np
import pytest

import oracle
from gpu_util import need_gpu, rel_rms
from paper_2010_01559_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbe():
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_01559_gb300 as rbe
    return rbe


@pytest.fixture(scope="module")
def c1():
    return workloads.config_small_fp64()


def _state(wl, dtype):
    import torch
    pos = torch.from_numpy(wl.pos_q()).cuda()
    vel = torch.zeros((wl.n, 4), dtype=torch.float32, device="cuda")
    vel[:, :3] = torch.from_numpy(wl.vel).cuda()
    if dtype == "float64":
        pos, vel = pos.double().contiguous(), vel.double().contiguous()
    return pos, vel


def _min_image(d, L):
    return d - L * np.round(d / L)


def _oracle_traj(wl, nsteps):
    p = wl.params
    pos = wl.pos.astype(np.float64)
    vel = wl.vel.astype(np.float64)
    q = wl.q.astype(np.float64)
    for s in range(nsteps):
        out = oracle.rbe_forces(pos, q, p.box, p.alpha, p.r_c, p.P, p.seed, p.stream, s,
                                lB=p.coulomb_prefactor, lj_eps=p.lj_eps, lj_sigma=p.lj_sigma,
                                lj_rcut=p.lj_rcut)
        pos, vel = oracle.langevin_step(pos, vel, out["F"], p.box, p.gamma, p.kT, p.dt, p.mass,
                                        p.seed, p.stream, s)
    return pos, vel


def test_fp64_trajectory_matches_oracle(rbe, c1):
    import torch
    h = rbe.RBE(rbe.params_from(c1.params, n_max=c1.n))
    pos, vel = _state(c1, "float64")
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.step(pos, vel, 100, step)
    h.sync()
    assert step.item() == 100
    rp, rv = _oracle_traj(c1, 100)
    d = _min_image(pos[:, :3].cpu().numpy() - rp, c1.params.box)
    assert np.abs(d).max() <= 1e-9
    assert np.abs(vel[:, :3].cpu().numpy() - rv).max() <= 1e-9
    assert np.array_equal(pos[:, 3].cpu().numpy(), c1.q.astype(np.float64))


def test_mixed_trajectory_tracks_fp64(rbe, c1):
    import torch
    h = rbe.RBE(rbe.params_from(c1.params, n_max=c1.n))
    p32, v32 = _state(c1, "float32")
    p64, v64 = _state(c1, "float64")
    s32 = torch.zeros(1, dtype=torch.int64, device="cuda")
    s64 = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.step(p32, v32, 100, s32)
    h.step(p64, v64, 100, s64)
    h.sync()
    d = _min_image(p32[:, :3].double().cpu().numpy() - p64[:, :3].cpu().numpy(), c1.params.box)
    dv = v32[:, :3].double().cpu().numpy() - v64[:, :3].cpu().numpy()
    print("mixed vs fp64 after 100 steps: max |dr|", np.abs(d).max(), "max |dv|", np.abs(dv).max())
    assert np.abs(d).max() <= 1e-4
    assert np.abs(dv).max() <= 1e-3


def test_graph_replay_resume_and_host_calls_are_bitwise(rbe, c1):
    import torch
    h = rbe.RBE(rbe.params_from(c1.params, n_max=c1.n))
    # plain device calls, 20 steps
    pa, va = _state(c1, "float32")
    sa = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.step(pa, va, 20, sa)
    # graph replay, 10 + 10 steps (resume from the device counter)
    h.set_graph(True)
    pb, vb = _state(c1, "float32")
    sb = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.step(pb, vb, 10, sb)
    h.step(pb, vb, 10, sb)
    h.set_graph(False)
    h.sync()
    assert sb.item() == 20
    assert torch.equal(pa, pb) and torch.equal(va, vb)
    # host buffers, 20 single steps
    hp = c1.pos_q().copy()
    hv = np.zeros((c1.n, 4), np.float32)
    hv[:, :3] = c1.vel
    tp, tv = torch.from_numpy(hp), torch.from_numpy(hv)
    for s in range(20):
        h.step_host(tp, tv, 1, s)
    assert np.array_equal(tp.numpy(), pa.cpu().numpy())
    assert np.array_equal(tv.numpy(), va.cpu().numpy())
    # page-locked host buffers, read and written in place by the step's
    # kernels; the call returns on the completion word the closing kernel
    # writes.  Direct launches and graph replay, one, two and three steps per
    # call, repeated step indices (a stale completion word must not count).
    for graph in (False, True):
        h.set_graph(graph)
        for per in (1, 2):
            v0 = np.zeros((c1.n, 4), np.float32)      # hv was updated in place above
            v0[:, :3] = c1.vel
            tp = torch.from_numpy(c1.pos_q().copy()).pin_memory()
            tv = torch.from_numpy(v0).pin_memory()
            for s in range(0, 20, per):
                h.step_host(tp, tv, per, s)
            assert np.array_equal(tp.numpy(), pa.cpu().numpy()), (graph, per)
            assert np.array_equal(tv.numpy(), va.cpu().numpy()), (graph, per)
        # the same step index twice from the same state gives the same result
        v0 = np.zeros((c1.n, 4), np.float32)
        v0[:, :3] = c1.vel
        outs = []
        for _ in range(2):
            tp = torch.from_numpy(c1.pos_q().copy()).pin_memory()
            tv = torch.from_numpy(v0.copy()).pin_memory()
            h.step_host(tp, tv, 3, 7)
            outs.append((tp.clone(), tv.clone()))
        assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    h.set_graph(False)
    # forces through host buffers equal the device call
    F = torch.zeros((c1.n, 4), dtype=torch.float32)
    E = torch.zeros(4, dtype=torch.float64)
    h.forces_host(torch.from_numpy(c1.pos_q()), 3, F, E)
    Fd, Ed, _ = h.forces(torch.from_numpy(c1.pos_q()).cuda(), 3)
    assert torch.equal(F, Fd.cpu()) and torch.equal(E, Ed.cpu()[0])


def test_fp64_resume_bitwise(rbe, c1):
    import torch
    h = rbe.RBE(rbe.params_from(c1.params, n_max=c1.n))
    pa, va = _state(c1, "float64")
    sa = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.step(pa, va, 12, sa)
    pb, vb = _state(c1, "float64")
    sb = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.step(pb, vb, 5, sb)
    h.step(pb, vb, 7, sb)
    h.sync()
    assert torch.equal(pa, pb) and torch.equal(va, vb)


def test_thermostat_holds_temperature(rbe, c1):
    """gamma = 10 (velocity relaxation in 100 steps): after 1000 steps of
    equilibration from the random start, the kinetic temperature averaged over
    the next 1000 steps is kT within 5 %."""
    import copy
    import torch
    sp = copy.copy(c1.params)
    sp.gamma = 10.0
    h = rbe.RBE(rbe.params_from(sp, n_max=c1.n))
    h.set_graph(True)
    pos, vel = _state(c1, "float32")
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.step(pos, vel, 1000, step)
    temps = []
    for _ in range(100):
        h.step(pos, vel, 10, step)
        temps.append((vel[:, :3].double() ** 2).sum().item() / (3 * c1.n))
    h.sync()
    T = float(np.mean(temps))
    print("kinetic temperature", T)
    assert abs(T - sp.kT) < 0.05
    assert np.all(np.isfinite(pos.cpu().numpy()))
    p = pos[:, :3].cpu().numpy()
    assert (p >= 0).all() and (p < sp.box).all()

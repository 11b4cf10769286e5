"""The Nose-Hoover thermostat (RBE_THERMO_NOSE_HOOVER, the equations of motion
of Sec. 3.3) and batches of systems that differ in every parameter, on the GPU:

* the FP64 trajectory and the friction xi equal the oracle's leapfrog after
  100 steps (1e-9), and after xi is set through rbe_nose_hoover_xi the next
  steps follow the oracle started from that xi;
* on the mixed path at the 2:1 electrolyte's size (N = 8001), each step's xi
  increment equals dt / Q (sum m|v|^2 - 3 N kT) of the previous step's
  velocities, the identity the discretisation fixes at any size;
* from a start at kT / 4 the mixed path heats the system to kT;
* one batch handle holding five systems with different N, L, alpha, r_c, P,
  dt, kT, mass and thermostat (Langevin, Andersen, Nose-Hoover with two time
  constants, one of them in the one-cell mode r_c > L/3) steps every system
  along the oracle's FP64 trajectory for that system.
"""
import copy

import numpy as np
import pytest

import oracle
from gpu_util import need_gpu
from paper_2010_01559_gb300 import workloads

pytestmark = pytest.mark.gpu
TOL = 1e-9


@pytest.fixture(scope="module")
def rbe():
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_01559_gb300 as rbe
    return rbe


def _nh(wl, tau):
    sp = copy.copy(wl.params)
    sp.thermostat = 2
    sp.nh_tau = tau
    return sp


def _oracle_forces(rp, q, sp, s):
    return oracle.rbe_forces(rp, q, sp.box, sp.alpha, sp.r_c, sp.P, sp.seed, sp.stream, s,
                             lB=sp.coulomb_prefactor, lj_eps=sp.lj_eps, lj_sigma=sp.lj_sigma,
                             lj_rcut=sp.lj_rcut)["F"]


def _dev_state(wl, v_scale, torch, dtype):
    pos = torch.from_numpy(wl.pos_q()).cuda().to(dtype).contiguous()
    vel = torch.zeros((wl.n, 4), dtype=dtype, device="cuda")
    vel[:, :3] = torch.from_numpy(wl.vel * v_scale).cuda().to(dtype)
    return pos, vel


def _close(pos, vel, rp, rv, L):
    d = pos[:, :3].cpu().numpy() - rp
    d -= L * np.round(d / L)
    return max(np.abs(d).max(), np.abs(vel[:, :3].cpu().numpy() - rv).max())


def test_nose_hoover_fp64_trajectory_and_xi_match_oracle(rbe):
    import torch
    wl = workloads.config_small_fp64()
    sp = _nh(wl, 0.05)
    h = rbe.RBE(rbe.params_from(sp, n_max=wl.n))
    pos, vel = _dev_state(wl, 0.5, torch, torch.float64)      # starts at kT / 4
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.step(pos, vel, 100, step)
    xi_gpu = h.nose_hoover_xi()[0]
    rp, rv = wl.pos.astype(np.float64), (wl.vel * 0.5).astype(np.float64)
    q = wl.q.astype(np.float64)
    nh = oracle.NoseHoover(sp.nh_tau)
    for s in range(100):
        rp, rv = nh.step(rp, rv, _oracle_forces(rp, q, sp, s), sp.box, sp.kT, sp.dt, sp.mass)
    print("xi after 100 steps", nh.xi, xi_gpu)
    assert nh.xi < -1.0                               # heating: the friction went negative
    assert abs(xi_gpu - nh.xi) <= TOL * max(1.0, abs(nh.xi))
    assert _close(pos, vel, rp, rv, sp.box) <= TOL
    # resume from a given xi: the next step keeps it, later steps advance it
    h.nose_hoover_xi([0.7])
    assert h.nose_hoover_xi() == [0.7]
    h.step(pos, vel, 20, step)
    nh.state[:] = [0.7, 0.0, 1.0]
    for s in range(100, 120):
        rp, rv = nh.step(rp, rv, _oracle_forces(rp, q, sp, s), sp.box, sp.kT, sp.dt, sp.mass)
    assert abs(h.nose_hoover_xi()[0] - nh.xi) <= TOL * max(1.0, abs(nh.xi))
    assert _close(pos, vel, rp, rv, sp.box) <= TOL
    h.close()


def test_nose_hoover_mixed_xi_increments_follow_kinetic_sum_at_n8001(rbe):
    import torch
    wl = workloads.config_2to1_mixed()
    sp = _nh(wl, 0.1)
    h = rbe.RBE(rbe.params_from(sp, n_max=wl.n))
    h.set_graph(True)
    pos, vel = _dev_state(wl, 0.7, torch, torch.float32)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    rate = sp.dt / (3 * wl.n * sp.nh_tau ** 2)
    h.step(pos, vel, 1, step)
    xi = [h.nose_hoover_xi()[0]]
    assert xi[0] == 0.0                               # the first step keeps xi
    k2 = [sp.mass * (vel[:, :3].double() ** 2).sum().item() / sp.kT]
    for _ in range(40):
        h.step(pos, vel, 1, step)
        xi.append(h.nose_hoover_xi()[0])
        k2.append(sp.mass * (vel[:, :3].double() ** 2).sum().item() / sp.kT)
    h.close()
    dxi = np.diff(xi) / rate
    want = np.array(k2[:-1]) - 3 * wl.n
    print("first increments", dxi[:3], want[:3])
    assert np.abs(want).min() > 1000                 # far from kT: the increments are large
    assert np.abs(dxi - want).max() <= 0.05


def test_nose_hoover_mixed_heats_to_kT(rbe):
    import torch
    wl = workloads.config_small_fp64()
    sp = _nh(wl, 0.1)
    h = rbe.RBE(rbe.params_from(sp, n_max=wl.n))
    h.set_graph(True)
    pos, vel = _dev_state(wl, 0.5, torch, torch.float32)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.step(pos, vel, 3000, step)
    temps = []
    for _ in range(200):
        h.step(pos, vel, 10, step)
        temps.append((vel[:, :3].double() ** 2).sum().item() * sp.mass / (3 * wl.n))
    h.sync()
    h.close()
    T = float(np.mean(temps))
    print("Nose-Hoover kinetic temperature", T, "from", 0.25 * sp.kT)
    assert abs(T - sp.kT) < 0.05


def _hetero_systems():
    """Five 1:1 electrolytes that differ in every per-system parameter."""
    e = workloads.electrolyte_1to1
    a = e(600, 0.05, 0.25, 5.5, 60, seed=21, stream=3, gamma=2.0, dt=1e-3)
    b = e(900, 0.08, 0.35, 4.5, 150, seed=22, stream=5, thermostat=1, andersen_nu=20.0,
          dt=2e-3, kT=0.8)
    c = e(400, 0.064, 0.3, 5.0, 40, seed=23, stream=7, thermostat=2, nh_tau=0.05,
          dt=1.5e-3, mass=2.0)
    d = e(1000, 0.064, 0.2, 6.0, 100, seed=24, stream=9, thermostat=2, nh_tau=0.2,
          kT=1.2)
    f = e(300, 0.064, 0.2, 6.0, 30, seed=25, stream=11, thermostat=2, nh_tau=0.1)
    return [a, b, c, d, f]


def test_heterogeneous_batch_follows_each_systems_oracle(rbe):
    import torch
    systems = _hetero_systems()
    L_f = systems[-1].params.box
    assert systems[-1].params.r_c > L_f / 3 >= 0     # the last one runs in one-cell mode
    scale = [1.0, 1.0, 0.6, 0.6, 0.6]
    h = rbe.RBEBatch([rbe.params_from(w.params) for w in systems], [w.n for w in systems])
    pos = torch.from_numpy(np.concatenate([w.pos_q() for w in systems])).cuda().double()
    vel = torch.zeros((pos.shape[0], 4), dtype=torch.float64, device="cuda")
    vel[:, :3] = torch.from_numpy(
        np.concatenate([w.vel * s for w, s in zip(systems, scale)])).cuda().double()
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    nsteps = 40
    h.step(pos, vel, nsteps, step)
    xi_gpu = h.nose_hoover_xi()
    off = 0
    for k, (w, s) in enumerate(zip(systems, scale)):
        sp = w.params
        rp, rv = w.pos.astype(np.float64), (w.vel * s).astype(np.float64)
        q = w.q.astype(np.float64)
        nh = oracle.NoseHoover(sp.nh_tau) if sp.thermostat == 2 else None
        for st in range(nsteps):
            F = _oracle_forces(rp, q, sp, st)
            if sp.thermostat == 0:
                rp, rv = oracle.langevin_step(rp, rv, F, sp.box, sp.gamma, sp.kT, sp.dt, sp.mass,
                                              sp.seed, sp.stream, st)
            elif sp.thermostat == 1:
                rp, rv, _ = oracle.andersen_step(rp, rv, F, sp.box, sp.andersen_nu, sp.kT, sp.dt,
                                                 sp.mass, sp.seed, sp.stream, st)
            else:
                rp, rv = nh.step(rp, rv, F, sp.box, sp.kT, sp.dt, sp.mass)
        err = _close(pos[off:off + w.n], vel[off:off + w.n], rp, rv, sp.box)
        print(w.name, "thermostat", sp.thermostat, "max deviation", err)
        assert err <= TOL, (k, err)
        if nh is not None:
            assert abs(xi_gpu[k] - nh.xi) <= TOL * max(1.0, abs(nh.xi)), (k, xi_gpu[k], nh.xi)
        off += w.n
    h.close()

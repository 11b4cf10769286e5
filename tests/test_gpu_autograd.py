"""Differentiable RBE energy (torch.autograd.Function RBEEnergy) on the
water-like point-charge system (rigid 3-site molecules, FP32 positions and
charges, no LJ).

* backward gives dE/dr = -F and dE/dq = phi, compared with the oracle's
  analytic forces and potentials (mixed tolerance 1e-5);
* the forward energy matches the oracle (frozen k-batch estimator);
* central finite differences of the FP64 GPU energy (h = 1e-4) reproduce the
  FP64 GPU Fourier forces and potentials;
* sum_i q_i phi_i = 2 E_Coulomb.
"""
import numpy as np
import pytest

from gpu_util import assert_per_particle, energy_rel, need_gpu, oracle_eval, rel_rms
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


@pytest.mark.parametrize("n_mol,sub", [(1500, None), (10000, 512)])
def test_autograd_matches_oracle_gradients(rbe, n_mol, sub):
    import torch
    wl = workloads.config_water(n_mol)
    h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    pos = torch.from_numpy(wl.pos).cuda().requires_grad_(True)
    q = torch.from_numpy(wl.q).cuda().requires_grad_(True)
    step = 3
    E = rbe.RBEEnergy.apply(pos, q, h, step)
    E.backward()
    idx = np.arange(wl.n) if sub is None else np.linspace(0, wl.n - 1, sub).astype(int)
    ref = oracle_eval(wl, step, sub=None if sub is None else idx, want_phi=True)
    gpos = pos.grad.cpu().numpy()[idx]
    gq = q.grad.cpu().numpy()[idx]
    e_f = rel_rms(-gpos, ref["F"])
    e_phi = rel_rms(gq, ref["phi"])
    print("water", n_mol, "dE/dr vs -F", e_f, "dE/dq vs phi", e_phi)
    assert e_f <= TOL_MIXED
    assert e_phi <= TOL_MIXED
    assert_per_particle(-gpos, ref["F"], "dE/dr")
    assert_per_particle(gq, ref["phi"], "dE/dq")
    if sub is None:
        assert energy_rel([E.item()] + list(ref["E"][1:]), ref["E"]) <= 1e-6


def test_charge_identity_and_fd_on_fp64_path(rbe):
    import torch
    wl = workloads.config_water(1500)
    h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    x = torch.from_numpy(wl.pos_q()).cuda().double().contiguous()
    step = 5
    F, E, phi = h.forces_f64(x, step, phi=True)
    E = E.cpu().numpy()[0]
    # E is quadratic in the charges (Coulomb parts): sum q phi = 2 (E_fourier + E_real)
    qphi = (x[:, 3] * phi).sum().item()
    assert abs(qphi - 2 * (E[1] + E[2])) <= 1e-11 * abs(E[1] + E[2])
    # finite differences of the Fourier energy (smooth, no cutoff) for a frozen batch
    Ff, _, phif = h.forces_f64(x, step, parts=rbe.RBE_PART_FOURIER, phi=True)
    hstep = 1e-4
    for i in (0, 7, 1234, 4000):
        for ax in range(3):
            xp = x.clone(); xp[i, ax] += hstep
            xm = x.clone(); xm[i, ax] -= hstep
            ep = h.forces_f64(xp, step, parts=rbe.RBE_PART_FOURIER)[1][0, 1].item()
            em = h.forces_f64(xm, step, parts=rbe.RBE_PART_FOURIER)[1][0, 1].item()
            fd = -(ep - em) / (2 * hstep)
            assert abs(fd - Ff[i, ax].item()) <= 1e-6 * (1 + abs(fd)), (i, ax, fd, Ff[i, ax].item())
        xp = x.clone(); xp[i, 3] += hstep
        xm = x.clone(); xm[i, 3] -= hstep
        ep = h.forces_f64(xp, step, parts=rbe.RBE_PART_FOURIER)[1][0, 1].item()
        em = h.forces_f64(xm, step, parts=rbe.RBE_PART_FOURIER)[1][0, 1].item()
        fdq = (ep - em) / (2 * hstep)
        assert abs(fdq - phif[i].item()) <= 1e-6 * (1 + abs(fdq))


def test_gradcheck_style_directional_derivative_mixed(rbe):
    """The mixed energy's directional derivative along a random direction agrees
    with <grad, d> from backward to the accuracy FP32 inputs allow."""
    import torch
    wl = workloads.config_water(1500)
    h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    pos = torch.from_numpy(wl.pos).cuda().requires_grad_(True)
    q = torch.from_numpy(wl.q).cuda().requires_grad_(True)
    E = rbe.RBEEnergy.apply(pos, q, h, 1)
    E.backward()
    g = torch.cat([pos.grad.flatten(), q.grad.flatten()]).double()
    gen = torch.Generator(device="cpu").manual_seed(0)
    d = torch.randn(g.numel(), generator=gen, dtype=torch.float64).cuda()
    d /= d.norm()
    # FD on the FP64 path with the same inputs promoted (directional, h = 1e-3)
    x = torch.cat([pos.detach(), q.detach()[:, None]], 1).double().contiguous()
    dx = torch.cat([d[:3 * wl.n].view(-1, 3), d[3 * wl.n:, None]], 1)
    hs = 1e-3
    ep = h.forces_f64((x + hs * dx).contiguous(), 1, parts=rbe.RBE_PART_FOURIER)[1][0, 1].item()
    em = h.forces_f64((x - hs * dx).contiguous(), 1, parts=rbe.RBE_PART_FOURIER)[1][0, 1].item()
    # the mixed gradient includes the real-space part; compare Fourier parts only
    F, _, phi = h.forces(torch.cat([pos.detach(), q.detach()[:, None]], 1).contiguous(), 1,
                         parts=rbe.RBE_PART_FOURIER, energy=False, phi=True)
    gf = torch.cat([-F[:, :3].flatten(), phi]).double()
    fd = (ep - em) / (2 * hs)
    assert abs(fd - (gf @ d).item()) <= 1e-4 * (abs(fd) + 1e-3)

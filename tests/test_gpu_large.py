"""Full-size checks: the large 1:1 electrolyte (N = 2^20, P = 500) in the
launch configuration the library picks for it, compared with the oracle on a
sample of particles (rho(k) over all N in FP64, forces of 1024 evenly spaced
particles), and the mixed path against the FP64 GPU path over all particles.
Also the unbiasedness of the Fourier estimator (Prop. 1) over 10^4 k-batches.
"""
import math

import numpy as np
import pytest

import oracle
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


@pytest.fixture(scope="module")
def large():
    return workloads.config_large()


def test_large_system_sampled_parity(rbe, large):
    import torch
    wl = large
    h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    x = torch.from_numpy(wl.pos_q()).cuda()
    step = 2
    m = h.sample_k(step).cpu().numpy()
    ref_m = oracle.sample_k(wl.params.alpha, wl.params.box, wl.params.seed, 0, step, wl.params.P)[0]
    assert np.array_equal(m[:, :3], ref_m)
    F, E, phi = h.forces(x, step, phi=True)
    sub = np.linspace(0, wl.n - 1, 1024).astype(int)
    ref = oracle_eval(wl, step, sub=sub, want_phi=True)
    Fs = F[:, :3].cpu().numpy()[sub]
    for name in ("F", ):
        err = rel_rms(Fs, ref[name])
        print("N=2^20 sampled rel-RMS", name, err)
        assert err <= TOL_MIXED
    assert rel_rms(phi.cpu().numpy()[sub], ref["phi"]) <= TOL_MIXED
    assert_per_particle(Fs, ref["F"], "F sampled")
    assert_per_particle(phi.cpu().numpy()[sub], ref["phi"], "phi sampled")
    F64, E64, _ = h.forces_f64(x.double().contiguous(), step)
    err_all = rel_rms(Fs, F64[:, :3].cpu().numpy()[sub])
    err_full = (F[:, :3].double() - F64[:, :3]).norm().item() / F64[:, :3].norm().item()
    print("mixed vs FP64 GPU over all 2^20 particles", err_full)
    assert err_full <= TOL_MIXED and err_all <= TOL_MIXED
    assert_per_particle(F[:, :3].cpu().numpy(), F64[:, :3].cpu().numpy(), "mixed vs FP64, all")
    assert abs(E[0, 0].item() - E64[0, 0].item()) <= 1e-6 * E64[0, 1:].abs().sum().item()


def test_unbiased_fourier_force_over_many_batches(rbe):
    """Mean of 10^4 RBE Fourier forces (frozen configuration) against the full
    Ewald Fourier force (Prop. 1, E chi = 0), and the empirical variance
    against Eq. varianceforce.

    Per component z = (mean - F_1) / (s / sqrt(nb)).  All particles share each
    k-batch, so the components are correlated: mean(z^2) has expectation ~1
    and variance 2 sum_ab R_ab^2 / n^2 (R = correlation matrix of the
    components, estimated from the same batches)."""
    import torch
    wl = workloads.config_small_fp64()
    p = wl.params
    h = rbe.RBE(rbe.params_from(p, n_max=wl.n))
    x = torch.from_numpy(wl.pos_q()).cuda()
    nb = 10000
    X = torch.empty((nb, 3 * wl.n), dtype=torch.float32, device="cuda")
    for s in range(nb):
        F, _, _ = h.forces(x, s, parts=rbe.RBE_PART_FOURIER, energy=False)
        X[s] = F[:, :3].reshape(-1)
    h.sync()
    Xd = X.double()
    mean_t = Xd.mean(0)
    Xc = Xd - mean_t
    cov = Xc.T @ Xc / (nb - 1)
    sd = cov.diagonal().sqrt()
    R = cov / (sd[:, None] * sd[None, :])
    n = R.shape[0]
    n_eff = n * n / (R * R).sum().item()
    mean = mean_t.cpu().numpy().reshape(-1, 3)
    var = (sd ** 2).cpu().numpy().reshape(-1, 3)
    pos64 = wl.pos.astype(np.float64)
    q64 = wl.q.astype(np.float64)
    mmax = 20           # per-axis weight at |m| = 20 is below 1e-9 of the largest (alpha = 0.3, L = 25)
    _, F1, _ = oracle.ewald_fourier(pos64, q64, p.box, p.alpha, mmax)
    z = (mean - F1) / np.sqrt(var / nb)
    mz2 = float((z ** 2).mean())
    bound = 5.0 * math.sqrt(2.0 / n_eff) + 0.01
    print("unbiasedness: mean z^2", mz2, "n_eff", n_eff, "bound", bound, "max |z|", np.abs(z).max())
    assert abs(mz2 - 1.0) <= bound
    assert np.abs(z).max() < 5.5
    var_ref, _ = oracle.fourier_variance(pos64, q64, p.box, p.alpha, mmax, p.P)
    ratio = var.sum(1) / var_ref
    print("variance ratio mean", ratio.mean())
    assert abs(ratio.mean() - 1) < 0.02

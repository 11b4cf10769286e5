"""True (non-random) energy and pressure on the GPU (rbe_observables) against
the oracle's full Ewald sum and virial, and the Coulomb homogeneity identity
W = E at converged sums.  The structure factors use FP32 phases, so the
tolerances are the mixed path's: 1e-5 relative to the sum of the magnitudes
of the parts."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import need_gpu
from paper_2010_01559_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbe():
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_01559_gb300 as rbe
    return rbe


def _gpu_obs(rbe, wl, mmax, with_vel=True):
    import torch
    h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    x = torch.from_numpy(wl.pos_q()).cuda()
    v = None
    if with_vel:
        v = torch.zeros((wl.n, 4), dtype=torch.float32, device="cuda")
        v[:, :3] = torch.from_numpy(wl.vel).cuda()
    return h.observables(x, v, mmax)[0]


def _ref(wl, mmax):
    p = wl.params
    return oracle.true_energy_virial(wl.pos.astype(np.float64), wl.q.astype(np.float64), p.box,
                                     p.alpha, p.r_c, mmax, lB=p.coulomb_prefactor,
                                     lj_eps=p.lj_eps, lj_sigma=p.lj_sigma, lj_rcut=p.lj_rcut)


@pytest.mark.parametrize("which", ["electrolyte", "water"])
def test_observables_match_oracle(rbe, which):
    wl = workloads.config_small_fp64() if which == "electrolyte" else workloads.config_water(1500)
    mmax = 10 if which == "electrolyte" else 8
    g = _gpu_obs(rbe, wl, mmax)
    r = _ref(wl, mmax)
    p = wl.params
    scale_e = abs(r["E_fourier"]) + abs(r["E_real"]) + abs(r["E_lj"])
    scale_w = abs(r["W_fourier"]) + abs(r["W_real"]) + abs(r["W_lj"]) + abs(r["W_bg"])
    for k in ("E_fourier", "E_real", "E_lj"):
        assert abs(g[k] - r[k]) <= 1e-5 * scale_e, (k, g[k], r[k])
    for k in ("W_fourier", "W_real", "W_lj", "W_bg"):
        assert abs(g[k] - r[k]) <= 1e-5 * scale_w, (k, g[k], r[k])
    ke = 0.5 * p.mass * float((wl.vel.astype(np.float64) ** 2).sum())
    assert abs(g["E_kin"] - ke) <= 1e-6 * ke
    V = p.box ** 3
    P_ref = (2 * ke + r["W_fourier"] + r["W_real"] + r["W_lj"] + r["W_bg"]) / (3 * V)
    assert abs(g["pressure"] - P_ref) <= 1e-5 * (2 * ke + scale_w) / (3 * V)
    assert abs(g["T_kin"] - 2 * ke / (3 * wl.n)) <= 1e-6 * g["T_kin"]
    assert abs(g["E_total"] - (g["E_fourier"] + g["E_real"] + g["E_lj"])) <= 1e-9 * scale_e


def test_coulomb_virial_equals_energy_at_convergence(rbe):
    r_c = 10.0 / 3.0
    alpha = (4.2 / r_c) ** 2
    wl = workloads.electrolyte_1to1(200, 0.2, alpha, r_c * 0.999, 10, seed=8, lj_eps=0.0)
    L = wl.params.box
    mmax = int(math.ceil(math.sqrt(alpha) * L * 4.6 / math.pi)) + 1
    g = _gpu_obs(rbe, wl, mmax, with_vel=False)
    E = g["E_fourier"] + g["E_real"]
    W = g["W_fourier"] + g["W_real"] + g["W_bg"]
    print("W", W, "E", E)
    assert abs(W - E) <= 2e-5 * (abs(E) + abs(g["E_real"]) + abs(g["W_fourier"]))

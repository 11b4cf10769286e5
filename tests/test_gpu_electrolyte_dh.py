"""The paper's charge-correlation electrolyte (Sec. 4.1) run with the GPU
library: N = 300 monovalent ions, L = 10, diameter 0.2 (shifted LJ, sigma =
0.2, R_c = 4), T = 1, alpha = 0.55, r_c = 4, Andersen thermostat nu = 3,
dt = 0.002, mixed path.

* Debye-Hueckel: the net charge around a cation, rho(r) = c (g_++ - g_+-),
  decays as e^{-kappa r} / r with kappa^2 = 4 pi l_B sum_i c_i q_i^2; the
  printed kappa (1.9416) follows from the formula, and the slope of
  ln(r |rho(r)|) over 0.5 < r < 1.6, sampled by both runs below, is within
  10 % of -kappa.
* RBE against a near-exact reference: the mean true potential energy per
  particle and the mean pressure (rbe_observables: full Ewald sum, no random
  batch) of the p = 10 run agree with those of a p = 500 run within four
  combined standard errors (block averages), and the kinetic temperature is kT.
"""
import math

import numpy as np
import pytest

from gpu_util import need_gpu
from paper_2010_01559_gb300 import workloads

pytestmark = pytest.mark.gpu
KAPPA_PRINTED = 1.9416


@pytest.fixture(scope="module")
def rbe():
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_01559_gb300 as rbe
    return rbe


def _run(rbe, P, n_eq=10000, n_prod=150000, every=100):
    import torch
    wl = workloads.config_electrolyte_dh(P=P)
    h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    pos = torch.from_numpy(wl.pos_q()).cuda()
    vel = torch.zeros((wl.n, 4), dtype=torch.float32, device="cuda")
    vel[:, :3] = torch.from_numpy(wl.vel).cuda()
    h.autotune(pos)
    h.set_graph(True)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.step(pos, vel, n_eq, step)
    snaps, E, Pr, T = [], [], [], []
    for _ in range(n_prod // every):
        h.step(pos, vel, every, step)
        o = h.observables(pos, vel)[0]
        E.append((o["E_fourier"] + o["E_real"] + o["E_lj"]) / wl.n)
        Pr.append(o["pressure"])
        T.append(o["T_kin"])
        snaps.append(pos[:, :3].cpu().numpy().astype(np.float64))
    h.sync()
    assert np.all(np.isfinite(np.array(snaps)))
    return wl, np.array(snaps), np.array(E), np.array(Pr), np.array(T)


def _mean_se(x, blocks=10):
    b = np.array_split(x, blocks)
    m = np.array([v.mean() for v in b])
    return x.mean(), m.std(ddof=1) / math.sqrt(blocks)


def _charge_correlation(wl, snaps, rmax=4.0, dr=0.05):
    L = wl.params.box
    pp = np.where(wl.q > 0)[0]
    mm = np.where(wl.q < 0)[0]
    edges = np.arange(0.0, rmax + dr, dr)
    hpp = np.zeros(len(edges) - 1)
    hpm = np.zeros(len(edges) - 1)
    iu = np.triu_indices(len(pp), 1)
    for x in snaps:
        d = x[pp][:, None, :] - x[pp][None, :, :]
        d -= L * np.round(d / L)
        hpp += np.histogram(np.sqrt((d ** 2).sum(-1))[iu], edges)[0]
        d = x[pp][:, None, :] - x[mm][None, :, :]
        d -= L * np.round(d / L)
        hpm += np.histogram(np.sqrt((d ** 2).sum(-1)).ravel(), edges)[0]
    V = L ** 3
    shell = 4.0 / 3.0 * math.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    r = 0.5 * (edges[1:] + edges[:-1])
    gpp = 2 * hpp / (len(pp) * (len(pp) - 1) / V * shell * len(snaps))
    gpm = hpm / (len(pp) * len(mm) / V * shell * len(snaps))
    c = len(pp) / V
    return r, c * (gpp - gpm)


@pytest.fixture(scope="module")
def runs(rbe):
    return _run(rbe, 10), _run(rbe, 500)


def test_debye_hueckel_decay(runs):
    wl = runs[0][0]
    snaps = np.concatenate([runs[0][1], runs[1][1]])     # both runs sample the same ensemble
    n_ion = wl.n / wl.params.box ** 3
    kappa = math.sqrt(4 * math.pi * wl.params.coulomb_prefactor / wl.params.kT * n_ion)
    assert abs(kappa - KAPPA_PRINTED) < 5e-4
    r, rho = _charge_correlation(wl, snaps)
    m = (r > 0.5) & (r < 1.6)
    assert np.all(rho[m] < 0)                  # like charges avoid each other
    slope, icpt = np.polyfit(r[m], np.log(r[m] * np.abs(rho[m])), 1)
    print(f"ln(r|rho|) = {slope:.4f} r + {icpt:.4f}   (DH: -{kappa:.4f} r - 1.1437)")
    assert abs(slope + kappa) < 0.1 * kappa


def test_rbe_matches_large_batch_reference(runs):
    (_, _, E10, P10, T10), (_, _, E500, P500, T500) = runs
    e10, se10 = _mean_se(E10)
    e500, se500 = _mean_se(E500)
    p10, sp10 = _mean_se(P10)
    p500, sp500 = _mean_se(P500)
    print(f"E_pot/N p=10 {e10:.5f}+-{se10:.5f}  p=500 {e500:.5f}+-{se500:.5f}; "
          f"P p=10 {p10:.5f}+-{sp10:.5f}  p=500 {p500:.5f}+-{sp500:.5f}")
    assert abs(e10 - e500) < 4 * math.hypot(se10, se500)
    assert abs(p10 - p500) < 4 * math.hypot(sp10, sp500)
    for T in (T10, T500):
        t, st = _mean_se(T)
        assert abs(t - 1.0) < 0.02 + 4 * st

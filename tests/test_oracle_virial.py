"""Pins of the oracle's true (non-random) energy and virial.

* Scaling: the virial of every part equals -dE/dlambda at lambda = 1 under
  r -> lambda r, L -> lambda L (alpha fixed; cutoffs fixed -- no pair sits
  within the finite-difference step of a cutoff), by central differences.
* Homogeneity: with converged sums (r_c near L/2 where erfc is negligible,
  mmax where the Gaussian is negligible) the Coulomb energy is homogeneous of
  degree -1, so W_coulomb = E_coulomb, also for a non-neutral system with its
  neutralising background.
"""
import math

import numpy as np
import pytest

import oracle


def _config(N, L, seed, neutral=True, dmin=0.95):
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < N:
        p = rng.uniform(0, L, 3)
        ok = True
        for r in pts:
            d = p - r
            d -= L * np.round(d / L)
            if d @ d < dmin * dmin:
                ok = False
                break
        if ok:
            pts.append(p)
    q = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    if not neutral:
        q[0] = 2.0
    return np.array(pts), q


@pytest.mark.parametrize("neutral", [True, False])
def test_virial_is_minus_scaling_derivative(neutral):
    L, alpha, r_c, mmax = 8.0, 0.9, 2.6, 6
    pos, q = _config(40, L, 3, neutral)
    kw = dict(lB=1.3, lj_eps=1.0, lj_sigma=1.0, lj_rcut=2 ** (1 / 6))
    base = oracle.true_energy_virial(pos, q, L, alpha, r_c, mmax, **kw)
    h = 1e-5
    ep = oracle.true_energy_virial(pos * (1 + h), q, L * (1 + h), alpha, r_c, mmax, **kw)
    em = oracle.true_energy_virial(pos * (1 - h), q, L * (1 - h), alpha, r_c, mmax, **kw)
    for e, w in (("E_fourier", "W_fourier"), ("E_real", "W_real"), ("E_lj", "W_lj"),
                 ("E_bg", "W_bg")):
        fd = -(ep[e] - em[e]) / (2 * h)
        w_expect = base[w]
        if e == "E_fourier":
            # E_fourier includes the self term (lambda-independent) and the background
            w_expect = base["W_fourier"] + base["W_bg"]
        assert abs(fd - w_expect) <= 1e-6 * (1 + abs(fd)), (e, fd, w_expect)


@pytest.mark.parametrize("neutral", [True, False])
def test_coulomb_virial_equals_energy_when_converged(neutral):
    L = 6.0
    pos, q = _config(24, L, 7, neutral)
    r_c = 2.99                                    # < L/2: minimum image only
    alpha = (4.2 / r_c) ** 2                      # erfc(sqrt(alpha) r_c) ~ 1e-9
    mmax = int(math.ceil(math.sqrt(alpha) * L * 4.6 / math.pi)) + 1   # e^{-k^2/4a} < 1e-9
    r = oracle.true_energy_virial(pos, q, L, alpha, r_c, mmax)
    E = r["E_fourier"] + r["E_real"]
    W = r["W_fourier"] + r["W_real"] + r["W_bg"]
    assert abs(W - E) <= 1e-7 * (abs(E) + abs(r["E_real"])), (W, E)

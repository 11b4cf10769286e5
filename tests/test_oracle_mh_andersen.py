"""Pins of the oracle's paper-literal Metropolis-Hastings k-sampler and of the
leapfrog + Andersen step (the loop of Algorithm 1 as printed), against the
mathematics rather than against themselves.

MH sampler (Sec. 3.1):
* the exact one-axis transition matrix built from the tabulated proposal and
  acceptance has the discrete Gaussian P(m) as its stationary law (a wrong
  acceptance rule -- e.g. accepting with probability qbar(m*), as the text
  literally reads -- does not);
* the expected acceptance rate is above 99 % (the paper's "very high");
* a chi-square test of the chain's output against P_k conditioned on k != 0;
* the chain is consumed in order: draw(a) then draw(b) == draw(a + b).

Leapfrog + Andersen:
* free particles, no collisions: positions advance by exactly n dt v;
* a harmonic oscillator integrated with the step keeps its energy within the
  leapfrog's O(dt^2) band without drift over many periods;
* collisions happen with frequency nu dt per particle and step, and the
  redrawn velocities are N(0, kT/m).
"""
import math

import numpy as np
import pytest

import oracle


def _target(alpha, L, M):
    w = np.array([math.exp(-math.pi ** 2 * k * k / (alpha * L * L)) for k in range(-M, M + 1)])
    return w / w.sum()


def _transition(Tq, rho):
    """One-axis MH kernel: proposal q_j from the 32-bit thresholds, acceptance
    min(1, rho_j / rho_i)."""
    t = Tq.astype(np.float64)
    q = np.diff(np.concatenate([[0.0], t])) / 2.0 ** 32
    acc = np.minimum(1.0, rho[None, :] / rho[:, None])
    K = q[None, :] * acc
    np.fill_diagonal(K, 0.0)
    K[np.diag_indices_from(K)] = 1.0 - K.sum(axis=1)
    return K, q


@pytest.mark.parametrize("alpha,L", [(0.3, 25.0), (0.2, 54.29), (0.3, 10.0)])
def test_mh_kernel_has_the_discrete_gaussian_as_stationary_law(alpha, L):
    Tq, rho, M = oracle.mh_tables(alpha, L)
    K, q = _transition(Tq, rho)
    p = _target(alpha, L, M)
    drift = np.abs(p @ K - p).max()
    assert drift < 1e-8, drift
    # the printed rule taken literally (accept with probability qbar(m*)) is not stationary
    Kw = q[None, :] * q[None, :] * np.ones_like(K)
    np.fill_diagonal(Kw, 0.0)
    Kw[np.diag_indices_from(Kw)] = 1.0 - Kw.sum(axis=1)
    assert np.abs(p @ Kw - p).max() > 1e3 * max(drift, 1e-12)


@pytest.mark.parametrize("alpha,L", [(0.3, 25.0), (0.2, 54.29)])
def test_mh_acceptance_rate_is_high(alpha, L):
    Tq, rho, M = oracle.mh_tables(alpha, L)
    K, q = _transition(Tq, rho)
    p = _target(alpha, L, M)
    acc = np.minimum(1.0, rho[None, :] / rho[:, None])
    rate = float(p @ (acc * q[None, :]).sum(axis=1))
    assert rate > 0.99, rate


def test_mh_chain_chi2_against_conditioned_target():
    alpha, L = 0.3, 10.0
    ch = oracle.MHChain(alpha, L, seed=5, stream=2)
    P = 60000
    m = ch.draw(P)
    assert not np.any(np.all(m == 0, axis=1))
    M = oracle.mh_tables(alpha, L)[2]
    p = _target(alpha, L, M)
    p0 = p[M]
    marg = p * (1 - (np.arange(-M, M + 1) == 0) * p0 ** 2) / (1 - p0 ** 3)
    for ax in range(3):
        counts = np.bincount(m[:, ax] + M, minlength=2 * M + 1).astype(float)
        exp_c = marg * P
        keep = exp_c > 20
        chi2 = np.sum((counts[keep] - exp_c[keep]) ** 2 / exp_c[keep])
        dof = keep.sum() - 1
        # nearly independent draws (acceptance > 99 %): allow a little extra spread
        assert chi2 < 1.2 * dof + 5 * math.sqrt(2 * dof), (ax, chi2, dof)


def test_mh_chain_consumed_in_order():
    a = oracle.MHChain(0.3, 25.0, seed=9, stream=1)
    b = oracle.MHChain(0.3, 25.0, seed=9, stream=1)
    x = np.concatenate([a.draw(37), a.draw(63)])
    y = b.draw(100)
    assert np.array_equal(x, y)
    assert a.pos[0] == b.pos[0] and np.array_equal(a.state, b.state)
    c = oracle.MHChain(0.3, 25.0, seed=9, stream=2)
    assert not np.array_equal(c.draw(100), y)


def test_leapfrog_free_particles_exact():
    rng = np.random.default_rng(0)
    L, dt = 10.0, 0.01
    pos = rng.uniform(0, L, (50, 3)); vel = rng.normal(size=(50, 3))
    p, v = pos.copy(), vel.copy()
    for n in range(100):
        p, v, hit = oracle.andersen_step(p, v, np.zeros_like(p), L, 0.0, 1.0, dt, 1.0, 1, 0, n)
        assert not hit.any()
    expect = (pos + 100 * dt * vel) % L
    d = (p - expect + L / 2) % L - L / 2
    assert np.abs(d).max() < 1e-10
    assert np.array_equal(v, vel)


def test_leapfrog_harmonic_energy_bounded():
    # 1D oscillator x'' = -w^2 x along x, large box so no wrap; leapfrog keeps
    # E within O((w dt)^2) of E0 with no secular drift
    L, w, dt = 1e6, 1.0, 0.05
    x0 = L / 2
    pos = np.array([[x0 + 1.0, 0.0, 0.0]]); vel = np.zeros((1, 3))
    E0 = 0.5 * w ** 2 * 1.0
    dev = []
    for n in range(20000):                    # ~160 periods
        F = np.array([[-w ** 2 * (pos[0, 0] - x0), 0.0, 0.0]])
        pos, vel, _ = oracle.andersen_step(pos, vel, F, L, 0.0, 1.0, dt, 1.0, 1, 0, n)
        # energy at integer step n+1 from the half-step velocity: v = v^{n+1/2} + (dt/2) F(r^{n+1})
        v_n = vel[0, 0] - 0.5 * dt * w ** 2 * (pos[0, 0] - x0)
        dev.append(0.5 * v_n ** 2 + 0.5 * w ** 2 * (pos[0, 0] - x0) ** 2 - E0)
    dev = np.array(dev)
    # the Euler start v^{1/2} = v^0 + dt F^0 adds (dt/2) F^0 to the velocity once
    start = 0.5 * (0.5 * dt * w ** 2 * 1.0) ** 2
    assert np.abs(dev).max() < 2.0 * (w * dt) ** 2 * E0 + 2 * start
    assert abs(dev[-2000:].mean() - dev[:2000].mean()) < 0.1 * (w * dt) ** 2 * E0


def test_andersen_collision_rate_and_velocity_law():
    rng = np.random.default_rng(1)
    N, L, dt, nu, kT = 20000, 50.0, 0.01, 5.0, 1.7
    pos = rng.uniform(0, L, (N, 3)); vel = np.full((N, 3), 3.0)
    _, v, hit = oracle.andersen_step(pos, vel, np.zeros_like(pos), L, nu, kT, dt, 1.0, 4, 0, 11)
    pc = nu * dt
    assert abs(hit.mean() - pc) < 5 * math.sqrt(pc * (1 - pc) / N)
    assert np.all(v[~hit] == 3.0)
    vv = v[hit].ravel()
    assert abs(vv.mean()) < 5 * math.sqrt(kT / len(vv))
    assert abs(vv.var() / kT - 1) < 5 * math.sqrt(2.0 / len(vv))


# ------------------------------------------------------------------ Nose-Hoover
def _nh_run(nsteps, dt, tau, kT=1.0, N=200, w=1.0, seed=0):
    """Independent 3-D harmonic oscillators (F = -w^2 (r - r0)) under the
    oracle's Nose-Hoover step.  Returns the kinetic temperatures of the
    half-step velocities and the extended energy H' = K + U + Q xi^2/2 +
    3 N kT eta (eta = integral of xi) at integer times: U at the positions the
    step starts from, K from the mean of the two half-step velocities around
    them, eta by the trapezoid rule."""
    rng = np.random.default_rng(seed)
    L = 1e4
    r0 = rng.uniform(100, L - 100, (N, 3))
    pos = r0 + rng.normal(scale=0.5, size=(N, 3))
    vel = rng.normal(scale=0.3, size=(N, 3))          # starts far colder than kT
    nh = oracle.NoseHoover(tau)
    Q = 3 * N * kT * tau ** 2
    T, H = [], []
    eta, xi_prev = 0.0, 0.0
    for n in range(nsteps):
        F = -w ** 2 * (pos - r0)
        U = 0.5 * w ** 2 * float(((pos - r0) ** 2).sum())
        pos, vnew = nh.step(pos, vel, F, L, kT, dt, 1.0)
        eta += 0.5 * dt * (xi_prev + nh.xi) if n else 0.0
        xi_prev = nh.xi
        K = 0.5 * float((((vel + vnew) / 2) ** 2).sum())
        vel = vnew
        T.append(float((vel ** 2).sum()) / (3 * N))
        if n:
            H.append(K + U + 0.5 * Q * nh.xi ** 2 + 3 * N * kT * eta)
    return np.array(T), np.array(H)


def test_nose_hoover_drives_temperature_to_kT():
    T, _ = _nh_run(40000, 0.01, tau=0.5)
    assert T[0] < 0.2
    assert abs(T[20000:].mean() - 1.0) < 0.03


def test_nose_hoover_extended_energy_conserved():
    # the Nose-Hoover flow conserves H'; the leapfrog keeps it to O(dt^2) with
    # no drift, which a wrong sign of the friction or of the xi equation breaks
    _, H1 = _nh_run(10000, 0.02, tau=0.5)
    _, H2 = _nh_run(20000, 0.01, tau=0.5)
    d1 = np.abs(H1 - H1[0]).max() / abs(H1[0])
    d2 = np.abs(H2 - H2[0]).max() / abs(H2[0])
    assert d1 < 0.01 and d2 < d1 / 3             # second order: halving dt quarters it

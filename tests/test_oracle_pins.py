"""Pins of the FP64 CPU oracle against things other than itself.

Each test ties an oracle function to a published value, a closed form, a
brute-force computation or an invariant, chosen so that a plausible mistake
(a dropped term, a wrong sign or index, a transposed operand, a missing factor
of 2 or S/P) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_kv(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split()[:2]
        out[k] = float(v)
    return out


def _nacl():
    pos, q = [], []
    for x in (0, 1):
        for y in (0, 1):
            for z in (0, 1):
                pos.append((x, y, z))
                q.append(1.0 if (x + y + z) % 2 == 0 else -1.0)
    return np.array(pos, float), np.array(q)


def _rand_system(n, L, seed, qvals=(1.0, -1.0), min_sep=0.0):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, L, (n, 3))
    q = np.array([qvals[i % len(qvals)] for i in range(n)], float)
    if abs(q.sum()) > 0 and n % 2 == 0:
        q -= q.mean()
    return pos, q


# ------------------------------------------------------------------ Philox
def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


# ------------------------------------------------------------------ sampling table
@pytest.mark.parametrize("alpha,L", [(0.3, 25.0), (0.2, 54.29), (0.1, 66.9), (0.3, 253.98),
                                     (0.55, 10.0), (0.30273, 100.8)])
def test_H_direct_sum_matches_poisson_form(alpha, L):
    """Eq. psf: sum_m exp(-pi^2 m^2/(alpha L^2)) = sqrt(alpha L^2/pi) sum_m exp(-alpha m^2 L^2)."""
    M, T, H = oracle.axis_table(alpha, L)
    poisson = math.sqrt(alpha * L * L / math.pi) * sum(
        math.exp(-alpha * m * m * L * L) for m in range(-3, 4))
    assert abs(H - poisson) / poisson < 1e-14
    # M leaves out weight below 2^-64
    assert math.exp(-math.pi ** 2 * M * M / (alpha * L * L)) < 2.0 ** -64
    assert math.exp(-math.pi ** 2 * (M - 2) ** 2 / (alpha * L * L)) > 2.0 ** -64


def test_H_paper_approximation_table1():
    """Sec. 3.1: H ~ sqrt(alpha L^2/pi)(1 + 2 exp(-alpha L^2)) for alpha L^2 >> 1."""
    kv = _read_kv("paper_printed.txt")
    a, L = kv["table1_rbe_alpha"], kv["table1_L"]
    _, _, H = oracle.axis_table(a, L)
    approx = math.sqrt(a * L * L / math.pi) * (1 + 2 * math.exp(-a * L * L))
    assert abs(H - approx) / H < 1e-15


def test_table_is_floor_of_scaled_cdf():
    """T_j = floor(2^32 CDF(j)) of the per-axis pmf exp(-pi^2 m^2/(alpha L^2))/H,
    against correctly rounded partial sums (math.fsum) evaluated in Python."""
    alpha, L = 0.3, 25.0
    M, T, H = oracle.axis_table(alpha, L)
    w = [math.exp(-math.pi ** 2 * m * m / (alpha * L * L)) for m in range(-M, M + 1)]
    Z = math.fsum(w)
    assert T[-1] == 2 ** 32
    assert np.all(np.diff(T.astype(np.int64)) >= 0)
    for j in range(2 * M):
        c = math.fsum(w[: j + 1]) / Z
        assert abs(int(T[j]) - c * 2 ** 32) <= 2.0       # rounding of the running sum only


def test_sampler_distribution_chi2():
    """Per-axis marginals follow P(m) = exp(-pi^2 m^2/(alpha L^2))/H conditioned on
    m != 0 jointly (Eq. probexpression); chi-square over 60000 samples."""
    alpha, L = 0.3, 10.0
    P = 60000
    m, att, bad = oracle.sample_k(alpha, L, seed=11, stream=3, step=7, P=P)
    assert bad == 0
    assert not np.any(np.all(m == 0, axis=1))
    M, T, H = oracle.axis_table(alpha, L)
    w = np.array([math.exp(-math.pi ** 2 * k * k / (alpha * L * L)) for k in range(-M, M + 1)])
    p = w / w.sum()
    # joint law of (m_x, m_y, m_z) is the product law conditioned on not all zero:
    # marginal of m_x: P(m_x=a) = p_a (1 - [a==0] p_0^2) / (1 - p_0^3)
    p0 = p[M]
    marg = p * (1 - (np.arange(-M, M + 1) == 0) * p0 ** 2) / (1 - p0 ** 3)
    for ax in range(3):
        counts = np.bincount(m[:, ax] + M, minlength=2 * M + 1).astype(float)
        exp_c = marg * P
        keep = exp_c > 20
        chi2 = np.sum((counts[keep] - exp_c[keep]) ** 2 / exp_c[keep])
        dof = keep.sum() - 1
        assert chi2 < dof + 5 * math.sqrt(2 * dof), (ax, chi2, dof)
    # retry frequency: one attempt fails with probability p0^3 = 1/H^3
    extra = (att - 1).sum()
    expect = P * p0 ** 3 / (1 - p0 ** 3)
    assert abs(extra - expect) < 5 * math.sqrt(expect) + 1


def test_sampler_is_deterministic_and_stream_separated():
    a = oracle.sample_k(0.3, 25.0, 0, 0, 5, 100)[0]
    b = oracle.sample_k(0.3, 25.0, 0, 0, 5, 100)[0]
    c = oracle.sample_k(0.3, 25.0, 0, 1, 5, 100)[0]
    d = oracle.sample_k(0.3, 25.0, 0, 0, 6, 100)[0]
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)
    assert not np.array_equal(a, d)


# ------------------------------------------------------------------ full Ewald
@pytest.mark.parametrize("alpha,mmax", [(30.0, 26), (36.0, 28), (49.0, 32)])
def test_madelung_nacl(alpha, mmax):
    kv = _read_kv("madelung_nacl.txt")
    pos, q = _nacl()
    L = kv["cell_L"]
    Ef, F, _ = oracle.ewald_fourier(pos, q, L, alpha, mmax)
    Ec, _, Fc, _, _ = oracle.real_space(pos, q, L, alpha, L / 2)
    U = Ef + Ec
    assert abs(U - (-kv["ion_pairs"] * kv["madelung"])) < 1e-9
    assert np.abs(F + Fc).max() < 1e-12          # every ion sits at a centre of symmetry


def test_alpha_independence_and_zero_net_force():
    L = 6.0
    pos, q = _rand_system(10, L, seed=3)
    Us, Fs = [], []
    for a in (3.5, 4.0, 5.0):
        Ef, F, _ = oracle.ewald_fourier(pos, q, L, a, 24)
        Ec, _, Fc, _, _ = oracle.real_space(pos, q, L, a, L / 2)
        Us.append(Ef + Ec)
        Fs.append(F + Fc)
        assert np.abs((F + Fc).sum(0)).max() < 1e-10
        assert np.abs(F.sum(0)).max() < 1e-10
    assert max(Us) - min(Us) < 1e-9 * abs(Us[0])
    assert np.abs(Fs[0] - Fs[2]).max() < 1e-8


def test_brute_force_image_sum_with_dipole_term():
    """Eq. energy summed over expanding cubes converges (as 1/R^2) to the
    tin-foil Ewald energy plus (2 pi / 3V)|sum q r|^2; Richardson-extrapolate."""
    rng = np.random.default_rng(1)
    L = 3.0
    pos = rng.uniform(0, L, (4, 3))
    q = np.array([1.0, -1.0, 0.5, -0.5])
    D = (q[:, None] * pos).sum(0)
    a = 16.0
    Ef, _, _ = oracle.ewald_fourier(pos, q, L, a, 30)
    Ec, _, _, _, _ = oracle.real_space(pos, q, L, a, L / 2)
    target = Ef + Ec + 2 * math.pi / (3 * L ** 3) * D @ D
    U40 = oracle.brute_images(pos, q, L, 40)
    U80 = oracle.brute_images(pos, q, L, 80)
    extrap = (4 * U80 - U40) / 3
    assert abs(extrap - target) < 2e-7 * abs(target)
    assert abs((Ef + Ec) - target) > 1e-2     # the dipole term matters here


def test_real_space_force_is_minus_gradient():
    L = 8.0
    pos, q = _rand_system(12, L, seed=5)
    a, rc = 0.8, 3.5
    kw = dict(lj_eps=1.0, lj_sigma=0.9, lj_rcut=0.9 * 2 ** (1 / 6))
    pos[1] = pos[0] + np.array([0.85, 0.1, 0.0])      # one pair inside the LJ range
    Ec, Elj, Fc, Flj, phi = oracle.real_space(pos, q, L, a, rc, want_phi=True, **kw)
    assert np.abs(Flj).max() > 0.1
    h = 1e-6
    for i in (0, 1, 4):
        for ax in range(3):
            p1 = pos.copy(); p1[i, ax] += h
            p2 = pos.copy(); p2[i, ax] -= h
            e1 = sum(oracle.real_space(p1, q, L, a, rc, **kw)[:2])
            e2 = sum(oracle.real_space(p2, q, L, a, rc, **kw)[:2])
            fd = -(e1 - e2) / (2 * h)
            assert abs(fd - (Fc[i, ax] + Flj[i, ax])) < 1e-6 * (1 + abs(fd))
    assert abs(q @ phi - 2 * Ec) < 1e-12 * (1 + abs(Ec))


# ------------------------------------------------------------------ RBE estimator
def _small_rbe_case():
    L = 4.0
    pos, q = _rand_system(10, L, seed=7)
    return pos, q, L, 1.0


def test_rbe_expectation_equals_ewald_fourier_force():
    """Prop. 1, E chi = 0: sum_k P_k F*(k) = F_i,1 exactly, with P_k =
    exp(-k^2/4alpha)/S over the same (converged) cube of k."""
    pos, q, L, alpha = _small_rbe_case()
    M, T, H = oracle.axis_table(alpha, L)
    S = H ** 3 - 1
    _, F1, _ = oracle.ewald_fourier(pos, q, L, alpha, M)
    acc = np.zeros_like(F1)
    for a in range(-M, M + 1):
        for b in range(-M, M + 1):
            for c in range(-M, M + 1):
                if a == b == c == 0:
                    continue
                pk = math.exp(-math.pi ** 2 * (a * a + b * b + c * c) / (alpha * L * L)) / S
                if pk < 1e-30:
                    continue
                acc += pk * oracle.rbe_single_k_force(pos, q, L, alpha, [a, b, c], S)
    assert np.abs(acc - F1).max() < 1e-11 * np.abs(F1).max()


def test_rbe_variance_matches_proposition1():
    """Eq. varianceforce against sum_k P_k |F*(k) - F_i,1|^2 / p by enumeration."""
    pos, q, L, alpha = _small_rbe_case()
    M, T, H = oracle.axis_table(alpha, L)
    S = H ** 3 - 1
    P = 7
    var, F1 = oracle.fourier_variance(pos, q, L, alpha, M, P, S=S)
    acc = np.zeros(len(q))
    for a in range(-M, M + 1):
        for b in range(-M, M + 1):
            for c in range(-M, M + 1):
                if a == b == c == 0:
                    continue
                pk = math.exp(-math.pi ** 2 * (a * a + b * b + c * c) / (alpha * L * L)) / S
                if pk < 1e-30:
                    continue
                Fk = oracle.rbe_single_k_force(pos, q, L, alpha, [a, b, c], S)
                acc += pk * ((Fk - F1) ** 2).sum(1)
    assert np.allclose(var, acc / P, rtol=1e-9, atol=0)


def test_rbe_energy_gradient_and_charge_identities():
    """For a frozen batch: -grad U1* = F* (central differences), dU/dq = phi,
    sum_i q_i phi_i = 2 U, U(lambda q) = lambda^2 U, sum_i F*_i = 0,
    translation invariance."""
    L = 6.0
    pos, q = _rand_system(9, L, seed=9, qvals=(1.0, -0.5, -0.5))
    alpha = 0.7
    m, _, _ = oracle.sample_k(alpha, L, seed=1, stream=0, step=3, P=12)
    S = oracle.S_of(alpha, L)
    E, F, phi, rho = oracle.rbe_fourier(pos, q, L, alpha, m, S=S, lB=1.3, want_phi=True)
    assert np.abs(F.sum(0)).max() < 1e-12 * (1 + np.abs(F).max())
    h = 1e-5
    for i in range(0, 9, 2):
        for ax in range(3):
            p1 = pos.copy(); p1[i, ax] += h
            p2 = pos.copy(); p2[i, ax] -= h
            fd = -(oracle.rbe_fourier(p1, q, L, alpha, m, S=S, lB=1.3)[0]
                   - oracle.rbe_fourier(p2, q, L, alpha, m, S=S, lB=1.3)[0]) / (2 * h)
            assert abs(fd - F[i, ax]) < 1e-7 * (1 + abs(fd))
        q1 = q.copy(); q1[i] += h
        q2 = q.copy(); q2[i] -= h
        fdq = (oracle.rbe_fourier(pos, q1, L, alpha, m, S=S, lB=1.3)[0]
               - oracle.rbe_fourier(pos, q2, L, alpha, m, S=S, lB=1.3)[0]) / (2 * h)
        assert abs(fdq - phi[i]) < 1e-7 * (1 + abs(fdq))
    assert abs(q @ phi - 2 * E) < 1e-11 * (1 + abs(E))
    E2 = oracle.rbe_fourier(pos, 2.5 * q, L, alpha, m, S=S, lB=1.3)[0]
    assert abs(E2 - 6.25 * E) < 1e-11 * abs(E2)
    shift = np.array([0.37, -1.1, 2.9])
    Et, Ft, _, _ = oracle.rbe_fourier(pos + shift, q, L, alpha, m, S=S, lB=1.3)
    assert abs(Et - E) < 1e-11 * abs(E)
    assert np.abs(Ft - F).max() < 1e-10 * np.abs(F).max()


def test_rbe_with_all_k_each_once_and_weights_reduces_to_ewald_energy():
    """With P equal to every k of the cube, weight S/P per k against
    exp(-k^2/4alpha) per k: the estimator energy differs from U1 only through
    the weights, so sum over k of (P_k * P) * per-k terms reproduces U1."""
    pos, q, L, alpha = _small_rbe_case()
    M, T, H = oracle.axis_table(alpha, L)
    S = H ** 3 - 1
    Ef, _, _ = oracle.ewald_fourier(pos, q, L, alpha, M)
    self_term = -math.sqrt(alpha / math.pi) * (q ** 2).sum()
    acc = 0.0
    for a in range(-M, M + 1):
        for b in range(-M, M + 1):
            for c in range(-M, M + 1):
                if a == b == c == 0:
                    continue
                pk = math.exp(-math.pi ** 2 * (a * a + b * b + c * c) / (alpha * L * L)) / S
                if pk < 1e-30:
                    continue
                e1 = oracle.rbe_fourier(pos, q, L, alpha, np.array([[a, b, c]]), S=S)[0]
                acc += pk * (e1 - self_term)
    assert abs(acc + self_term - Ef) < 1e-11 * abs(Ef)


def test_background_term_for_non_neutral_charges():
    """A non-neutral cell adds -pi (sum q)^2/(2 V alpha) (neutralising
    background), which makes the Ewald energy alpha independent again."""
    L = 5.0
    rng = np.random.default_rng(4)
    pos = rng.uniform(0, L, (6, 3))
    q = np.array([1.0, -1.0, 0.7, 0.2, -0.4, 0.3])     # sum = 0.8
    Us = []
    for a in (3.0, 5.0):
        Ef, _, _ = oracle.ewald_fourier(pos, q, L, a, 20)
        Ec, _, _, _, _ = oracle.real_space(pos, q, L, a, L / 2)
        Us.append(Ef + Ec)
    assert abs(Us[0] - Us[1]) < 1e-9 * abs(Us[0])


# ------------------------------------------------------------------ Langevin
def test_langevin_normals_are_standard():
    xi = oracle.langevin_normals(200000, seed=3, stream=1, step=17)
    assert abs(xi.mean()) < 5 / math.sqrt(xi.size)
    assert abs(xi.var() - 1) < 5 * math.sqrt(2 / xi.size)
    # independent components
    c = np.corrcoef(xi.T)
    assert np.abs(c - np.eye(3)).max() < 0.02


def test_langevin_kick_then_ou_then_drift():
    """One step from identical (r, v, F): mean of v' is c1 (v + dt F/m) (kick
    before the Ornstein-Uhlenbeck step), variance (1 - c1^2) kT/m, and
    r' = wrap(r + dt v')."""
    N = 100000
    L, gamma, kT, dt, mass = 10.0, 2.0, 1.5, 0.5, 1.0
    pos = np.full((N, 3), 9.9)
    vel = np.tile([0.3, -0.2, 0.1], (N, 1))
    F = np.tile([2.0, 0.0, -4.0], (N, 1))
    p2, v2 = oracle.langevin_step(pos, vel, F, L, gamma, kT, dt, mass, 5, 0, 0)
    c1 = math.exp(-gamma * dt / mass)
    mean_expect = c1 * (vel[0] + dt * F[0] / mass)
    sd = math.sqrt((1 - c1 * c1) * kT / mass)
    assert np.abs(v2.mean(0) - mean_expect).max() < 5 * sd / math.sqrt(N)
    assert np.abs(v2.var(0) / sd ** 2 - 1).max() < 0.02
    assert np.all((p2 >= 0) & (p2 < L))
    expect_r = np.mod(pos + dt * v2, L)
    assert np.abs(p2 - expect_r).max() < 1e-12


def test_langevin_equipartition_free_particles():
    N = 4000
    rng = np.random.default_rng(0)
    pos = rng.uniform(0, 5, (N, 3)); vel = np.zeros((N, 3)); F = np.zeros((N, 3))
    for s in range(60):
        pos, vel = oracle.langevin_step(pos, vel, F, 5.0, 1.0, 0.7, 0.1, 2.0, 9, 0, s)
    # after 60 steps of gamma dt / m = 0.05 the velocity variance is within e^-6 of kT/m
    assert abs(vel.var() / 0.35 - 1) < 0.03

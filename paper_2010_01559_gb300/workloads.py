"""Seeded synthetic inputs: electrolytes and a water-like point-charge system.

This module only places particles and assigns charges and velocities; it holds
none of the method's arithmetic, and both the CUDA path's tests/benchmark and
the CPU oracle read the inputs it makes.  Random numbers come from numpy's
PCG64 seeded per workload, so every input is reproducible from its seed.

Workloads (the shapes of the electrolytes of Sec. 4.1 and 4.2 at the sizes the
benchmark configurations ask for):

* ``electrolyte(n_pos, n_neg, q_pos, q_neg, L, ...)``: ions placed uniformly in
  a periodic cube and re-drawn until every minimum-image pair is at least
  ``min_sep`` apart (random sequential re-drawing of the offending particle).
* ``water_like(n_mol, density, ...)``: rigid 3-site molecules (O -0.8476,
  H +0.4238, O-H 1.0, H-O-H 109.47 deg) with uniformly random orientations and
  centres at least ``min_oo`` apart.

Positions and charges are returned as float32 (the mixed-precision path's
input type); the oracle reads the same float32 values promoted to float64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

WCA_RCUT = 2.0 ** (1.0 / 6.0)


@dataclass
class SystemParams:
    """Physical and method parameters of one periodic system."""
    box: float
    alpha: float
    r_c: float
    P: int
    seed: int = 0
    stream: int = 0
    coulomb_prefactor: float = 1.0
    lj_eps: float = 1.0
    lj_sigma: float = 1.0
    lj_rcut: float = WCA_RCUT
    gamma: float = 1.0
    kT: float = 1.0
    dt: float = 1e-3
    mass: float = 1.0
    sampler: int = 0          # 0: exact i.i.d. inverse CDF, 1: the paper's MH chains
    thermostat: int = 0       # 0: Langevin (kick / OU / drift), 1: leapfrog + Andersen,
                              # 2: Nose-Hoover leapfrog
    andersen_nu: float = 0.0  # Andersen collision frequency
    nh_tau: float = 0.0       # Nose-Hoover time constant (Q = 3 N kT tau^2)
    skin: float = 0.0         # neighbour-list skin of the MD step (0: automatic, < 0: none)


@dataclass
class Workload:
    name: str
    params: SystemParams
    pos: np.ndarray          # float32 [N, 3], in [0, L)
    q: np.ndarray            # float32 [N]
    vel: np.ndarray          # float32 [N, 3]
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(len(self.q))

    def pos_q(self) -> np.ndarray:
        """float32 [N, 4] = (x, y, z, q), the C-ABI's particle layout."""
        out = np.empty((self.n, 4), dtype=np.float32)
        out[:, :3] = self.pos
        out[:, 3] = self.q
        return out


def _to_box32(x: np.ndarray, L: float) -> np.ndarray:
    """Cast to float32 and fold any value that rounded up to L back to 0."""
    x32 = np.asarray(x, dtype=np.float32)
    L32 = np.float32(L)
    x32 = np.where(x32 >= L32, np.float32(0.0), x32)
    x32 = np.where(x32 < 0, np.float32(0.0), x32)
    return x32.astype(np.float32)


def _close_pairs(pos: np.ndarray, L: float, dmin: float) -> np.ndarray:
    from scipy.spatial import cKDTree
    tree = cKDTree(pos.astype(np.float64), boxsize=L)
    return tree.query_pairs(dmin, output_type="ndarray")


def _close_pairs_with(pos: np.ndarray, L: float, dmin: float, idx: np.ndarray) -> np.ndarray:
    """The pairs (i < j) closer than dmin that involve a particle of idx."""
    from scipy.spatial import cKDTree
    tree = cKDTree(pos.astype(np.float64), boxsize=L)
    nb = tree.query_ball_point(pos[idx].astype(np.float64), dmin, return_sorted=False)
    out = set()
    for a, lst in zip(idx.tolist(), nb):
        for b in lst:
            if b != a:
                out.add((min(a, b), max(a, b)))
    return np.array(sorted(out), dtype=np.int64).reshape(-1, 2)


def place_uniform(n: int, L: float, min_sep: float, rng: np.random.Generator,
                  max_rounds: int = 1000) -> np.ndarray:
    """n points in [0,L)^3 with all minimum-image separations >= min_sep.

    Each round re-draws the higher-indexed particle of every close pair.  Only
    pairs that involve a particle re-drawn in the previous round can be close
    after the first round, so later rounds look only at those."""
    pos = _to_box32(rng.uniform(0.0, L, size=(n, 3)), L)
    if n < 2 or min_sep <= 0:
        return pos
    pairs = _close_pairs(pos, L, min_sep)
    for _ in range(max_rounds):
        if len(pairs) == 0:
            return pos
        redo = np.unique(pairs[:, 1])
        pos[redo] = _to_box32(rng.uniform(0.0, L, size=(len(redo), 3)), L)
        pairs = _close_pairs_with(pos, L, min_sep, redo)
    raise RuntimeError("placement did not converge; density too high for min_sep")


def maxwell(n: int, kT: float, mass: float, rng: np.random.Generator) -> np.ndarray:
    return (rng.standard_normal((n, 3)) * math.sqrt(kT / mass)).astype(np.float32)


def electrolyte(name: str, n_pos: int, n_neg: int, q_pos: float, q_neg: float,
                params: SystemParams, min_sep: float = 0.9) -> Workload:
    rng = np.random.default_rng([params.seed, params.stream, 0x5EED, n_pos, n_neg])
    n = n_pos + n_neg
    pos = place_uniform(n, params.box, min_sep, rng)
    q = np.empty(n, dtype=np.float32)
    q[:n_pos] = q_pos
    q[n_pos:] = q_neg
    perm = rng.permutation(n)
    q = q[perm]
    vel = maxwell(n, params.kT, params.mass, rng)
    return Workload(name, params, pos, q, vel)


def place_jittered_lattice(n: int, L: float, min_sep: float,
                           rng: np.random.Generator) -> np.ndarray:
    """n distinct random sites of the smallest simple-cubic lattice with at
    least n sites, each moved uniformly within +-(a - min_sep)/2 per axis
    (a = lattice spacing), so every pair stays at least min_sep apart.  Used
    where the packing is too dense for re-drawing uniform points."""
    side = int(math.ceil(n ** (1.0 / 3.0) - 1e-9))
    a = L / side
    if a < min_sep:
        raise ValueError("lattice spacing below min_sep")
    sites = rng.choice(side ** 3, size=n, replace=False)
    idx = np.stack([sites % side, (sites // side) % side, sites // (side * side)], 1)
    jitter = rng.uniform(-(a - min_sep) / 2, (a - min_sep) / 2, size=(n, 3))
    return (idx + 0.5) * a + jitter


def water_like(name: str, n_mol: int, density: float, params: SystemParams,
               min_oo: float = 2.5) -> Workload:
    """3 n_mol point charges; centres at ``density`` molecules per unit volume,
    on a jittered lattice with O-O distances of at least ``min_oo``."""
    rng = np.random.default_rng([params.seed, 0xAA7E, n_mol])
    L = params.box
    centres = place_jittered_lattice(n_mol, L, min_oo, rng)
    # uniform random rotations from normalised Gaussian quaternions
    qt = rng.standard_normal((n_mol, 4))
    qt /= np.linalg.norm(qt, axis=1, keepdims=True)
    w, x, y, z = qt.T
    R = np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1),
    ], 1)
    half = math.radians(109.47) / 2.0
    body = np.array([[0.0, 0.0, 0.0],
                     [math.sin(half), 0.0, math.cos(half)],
                     [-math.sin(half), 0.0, math.cos(half)]])       # O-H = 1.0
    sites = centres[:, None, :] + np.einsum("nij,sj->nsi", R, body)
    sites = np.mod(sites, L).reshape(-1, 3)
    pos = _to_box32(sites, L)
    q = np.tile(np.array([-0.8476, 0.4238, 0.4238], dtype=np.float32), n_mol)
    vel = maxwell(3 * n_mol, params.kT, params.mass, rng)
    return Workload(name, params, pos, q, vel, extra=dict(n_mol=n_mol))


# ---------------------------------------------------------------- named configs
def alpha_for_cut(r_c: float, tol: float = 1e-4) -> float:
    """alpha with erfc(sqrt(alpha) r_c) = tol."""
    from scipy.special import erfcinv
    return float((erfcinv(tol) / r_c) ** 2)


def electrolyte_1to1(n: int, density: float, alpha: float, r_c: float, P: int,
                     seed: int, stream: int = 0, name: str = "electrolyte_1to1",
                     **kw) -> Workload:
    L = (n / density) ** (1.0 / 3.0)
    p = SystemParams(box=L, alpha=alpha, r_c=r_c, P=P, seed=seed, stream=stream, **kw)
    return electrolyte(name, n // 2, n - n // 2, 1.0, -1.0, p)


def config_small_fp64() -> Workload:
    """1:1 electrolyte, N=1000, L=25, alpha=0.3, r_c=5, P=100, WCA, seed 0."""
    p = SystemParams(box=25.0, alpha=0.3, r_c=5.0, P=100, seed=0)
    return electrolyte("electrolyte_1to1_N1000_L25", 500, 500, 1.0, -1.0, p)


def config_2to1_mixed() -> Workload:
    """2:1 electrolyte: 2667 cations (+2) and 5334 anions (-1), N=8001, density
    0.05, alpha=0.2, r_c=6, P=200, WCA, seed 2."""
    n = 2667 + 5334
    L = (n / 0.05) ** (1.0 / 3.0)
    p = SystemParams(box=L, alpha=0.2, r_c=6.0, P=200, seed=2)
    return electrolyte("electrolyte_2to1_N8001_rho0.05_P200", 2667, 5334, 2.0, -1.0, p)


def config_water(n_mol: int = 10000) -> Workload:
    """10^4 rigid 3-site molecules at 0.0334 per unit volume, alpha=0.1,
    r_c=10, P=100, no LJ, seed 3."""
    L = (n_mol / 0.0334) ** (1.0 / 3.0)
    p = SystemParams(box=L, alpha=0.1, r_c=10.0, P=100, seed=3, lj_eps=0.0)
    return water_like(f"water_like_{n_mol}mol", n_mol, 0.0334, p)


def config_replicas(n_rep: int = 64, n_lo: int = 1000, n_hi: int = 65536,
                    density: float = 0.064, r_c: float = 5.0, P: int = 100,
                    seed: int = 4) -> list:
    """n_rep 1:1 electrolytes with N log-uniform in [n_lo, n_hi] (even), each in
    its own box at ``density``, alpha from erfc(sqrt(alpha) r_c) = 1e-4, P each,
    replica r on Philox stream r."""
    rng = np.random.default_rng([seed, 0xBA7C])
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=n_rep))
    ns = (np.round(ns / 2.0) * 2).astype(int)
    alpha = alpha_for_cut(r_c)
    out = []
    for r, n in enumerate(ns):
        out.append(electrolyte_1to1(int(n), density, alpha, r_c, P, seed=seed, stream=r,
                                    name=f"replica{r}_N{n}"))
    return out


def config_large(n: int = 1 << 20, density: float = 0.064, alpha: float = 0.3,
                 r_c: float = 5.0, P: int = 500, seed: int = 5) -> Workload:
    """1:1 electrolyte, N=2^20 by default, density 0.064, alpha=0.3, r_c=5, P=500."""
    return electrolyte_1to1(n, density, alpha, r_c, P, seed=seed,
                            name=f"electrolyte_1to1_N{n}_rho0.064_P{P}")


def config_electrolyte_dh(n: int = 300, density: float = 0.3, P: int = 10, seed: int = 6,
                          andersen_nu: float = 3.0) -> Workload:
    """The paper's charge-correlation electrolyte (Sec. 4.1): monovalent ions of
    diameter 0.2, shifted LJ with sigma = 0.2, epsilon = 1, R_c = 4 (r_off = 0),
    T = 1, prefactor 1 (epsilon_r = 1/(4 pi)), N / L^3 = 0.3 (L = 10 at N = 300),
    alpha = 0.55, r_c = 4, batch p, Andersen thermostat nu = 3, dt = 0.002;
    ions placed uniformly at least 0.25 apart."""
    L = (n / density) ** (1.0 / 3.0)
    p = SystemParams(box=L, alpha=0.55, r_c=min(4.0, L / 2), P=P, seed=seed, lj_eps=1.0,
                     lj_sigma=0.2, lj_rcut=min(4.0, L / 2), dt=0.002, thermostat=1,
                     andersen_nu=andersen_nu)
    return electrolyte(f"electrolyte_dh_N{n}_P{P}", n // 2, n - n // 2, 1.0, -1.0, p,
                       min_sep=0.25)

"""FP64 CPU oracle for the random batch Ewald method (arXiv:2010.01559).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA library never
imports, links or executes anything here, and this package shares no code with
it (own Philox, own sampling table, own Ewald sums in ``rbe_oracle.c``).

This module compiles ``rbe_oracle.c`` with the system C compiler on first use
(or through :func:`build`) and wraps its functions with ``ctypes`` so that they
take and return numpy arrays.  All arithmetic happens in the C file; the
wrappers only marshal arguments.

Pins (see ``tests/test_oracle_*.py``): Philox against published vectors; the
sampling table against the Poisson form of H (Eq. psf) and the exact per-axis
probabilities; full Ewald against the NaCl Madelung constant, alpha
independence and direct image sums (Eq. energy); the RBE estimator against the
exact expectation (Proposition 1, E chi = 0), the exact variance (Eq.
varianceforce), finite differences of its energy, and charge-scaling
identities; the Langevin step against its closed-form moments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rbe_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "librbe_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_U32 = ctypes.POINTER(ctypes.c_uint32)
_U64 = ctypes.POINTER(ctypes.c_uint64)
_INT = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP, no FP contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.orc_philox4x32_10.argtypes = [_U32, _U32, _U32]
        lib.orc_philox4x32_10.restype = None
        lib.orc_axis_M.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.orc_axis_M.restype = ctypes.c_int
        lib.orc_axis_table.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, _U64]
        lib.orc_axis_table.restype = ctypes.c_double
        lib.orc_sample_k.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                     ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, _I32, _I32]
        lib.orc_sample_k.restype = ctypes.c_int
        lib.orc_ewald_fourier.argtypes = [ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int, ctypes.c_int, _INT,
                                          _D, _D, _D]
        lib.orc_ewald_fourier.restype = None
        lib.orc_rbe_fourier.argtypes = [ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_int, _I32,
                                        ctypes.c_int, _INT, _D, _D, _D, _D]
        lib.orc_rbe_fourier.restype = None
        lib.orc_rbe_single_k_force.argtypes = [ctypes.c_int, _D, _D, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                               _I32, _D]
        lib.orc_rbe_single_k_force.restype = None
        lib.orc_real_space.argtypes = [ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int, _INT,
                                       _D, _D, _D, _D]
        lib.orc_real_space.restype = None
        lib.orc_brute_images.argtypes = [ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_int]
        lib.orc_brute_images.restype = ctypes.c_double
        lib.orc_fourier_variance.argtypes = [ctypes.c_int, _D, _D, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_int, ctypes.c_int, _D, _D]
        lib.orc_fourier_variance.restype = None
        lib.orc_langevin_normals.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                             ctypes.c_uint64, _D]
        lib.orc_langevin_normals.restype = None
        lib.orc_langevin_step.argtypes = [ctypes.c_int, _D, _D, _D, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                                          ctypes.c_uint64]
        lib.orc_langevin_step.restype = None
        lib.orc_mh_tables.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, _U64, _D]
        lib.orc_mh_tables.restype = None
        lib.orc_mh_sample_k.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                        ctypes.c_uint32, ctypes.c_int, _I32, _U64, _I32]
        lib.orc_mh_sample_k.restype = ctypes.c_int
        lib.orc_andersen_step.argtypes = [ctypes.c_int, _D, _D, _D, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                                          ctypes.c_uint64, _INT]
        lib.orc_andersen_step.restype = None
        lib.orc_true_energy_virial.argtypes = [ctypes.c_int, _D, _D, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_int, _D]
        lib.orc_true_energy_virial.restype = None
        lib.orc_nose_hoover_step.argtypes = [ctypes.c_int, _D, _D, _D, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, _D]
        lib.orc_nose_hoover_step.restype = None
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_threads.restype = None
        lib.orc_get_threads.argtypes = []
        lib.orc_get_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def set_threads(n: int) -> int:
    """Threads of the oracle's OpenMP loops (n <= 0: all processors); returns
    the count in effect.  Results do not depend on it (rows are owned whole)."""
    lib = _load()
    lib.orc_set_threads(int(n))
    return int(lib.orc_get_threads())


def _dp(a):
    return None if a is None else a.ctypes.data_as(_D)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _sub(sub):
    if sub is None:
        return 0, None, None
    s = np.ascontiguousarray(sub, dtype=np.intc)
    return len(s), s, s.ctypes.data_as(_INT)


# ---------------------------------------------------------------- Philox
def philox4x32_10(ctr, key):
    """Philox4x32-10 block function: four 32-bit counter words, two key words."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(c.ctypes.data_as(_U32), k.ctypes.data_as(_U32), out.ctypes.data_as(_U32))
    return out


# ---------------------------------------------------------------- sampling
def axis_M(alpha: float, L: float) -> int:
    """Half-width M of the per-axis table: tail weight below 2^-64."""
    return int(_load().orc_axis_M(alpha, L))


def axis_table(alpha: float, L: float):
    """(M, T, H): the per-axis cumulative table floor(2^32 CDF) and H (Eq. psf)."""
    lib = _load()
    M = int(lib.orc_axis_M(alpha, L))
    T = np.zeros(2 * M + 1, dtype=np.uint64)
    H = lib.orc_axis_table(alpha, L, M, T.ctypes.data_as(_U64))
    return M, T, float(H)


def S_of(alpha: float, L: float) -> float:
    """S = H^3 - 1 (Eq. S)."""
    _, _, H = axis_table(alpha, L)
    return H ** 3 - 1.0


def sample_k(alpha, L, seed, stream, step, P):
    """(m[P,3] int32, attempts[P] int32, bad) for one (seed, stream, step)."""
    lib = _load()
    m = np.zeros((P, 3), dtype=np.int32)
    att = np.zeros(P, dtype=np.int32)
    bad = lib.orc_sample_k(alpha, L, seed, stream, step, P, m.ctypes.data_as(_I32),
                           att.ctypes.data_as(_I32))
    return m, att, int(bad)


class MHChain:
    """The paper's Metropolis-Hastings k-sampler (Sec. 3.1): three per-axis
    independence chains with the rounded-Gaussian proposal, consumed in order
    (the set K of Algorithm 1).  ``draw(P)`` returns the next P nonzero triples
    and advances the chains."""

    def __init__(self, alpha, L, seed, stream, state=(0, 0, 0), pos=0):
        self.alpha, self.L, self.seed, self.stream = alpha, L, seed, stream
        self.state = np.array(state, dtype=np.int32)
        self.pos = np.array([pos], dtype=np.uint64)

    def draw(self, P):
        m = np.zeros((P, 3), dtype=np.int32)
        bad = _load().orc_mh_sample_k(self.alpha, self.L, self.seed, self.stream, P,
                                      self.state.ctypes.data_as(_I32),
                                      self.pos.ctypes.data_as(_U64), m.ctypes.data_as(_I32))
        if bad:
            raise RuntimeError("MH chain emitted fewer than P nonzero triples")
        return m


def mh_tables(alpha, L):
    """(Tq uint64[2M+1], rho float64[2M+1], M): proposal thresholds and P/qbar."""
    lib = _load()
    M = lib.orc_axis_M(alpha, L)
    Tq = np.zeros(2 * M + 1, dtype=np.uint64)
    rho = np.zeros(2 * M + 1)
    lib.orc_mh_tables(alpha, L, M, Tq.ctypes.data_as(_U64), _dp(rho))
    return Tq, rho, M


# ---------------------------------------------------------------- Fourier part
def ewald_fourier(pos, q, L, alpha, mmax, lB=1.0, sub=None, want_phi=False):
    """Full Ewald Fourier part over 0<|m|_inf<=mmax: (E, F[nsub,3], phi or None)."""
    lib = _load()
    pos = _f64(pos, (-1, 3)); q = _f64(q)
    N = len(q)
    nsub, s, sp = _sub(sub)
    n_out = nsub if sub is not None else N
    F = np.zeros((n_out, 3)); E = np.zeros(1)
    phi = np.zeros(n_out) if want_phi else None
    lib.orc_ewald_fourier(N, _dp(pos), _dp(q), L, alpha, lB, mmax, nsub, sp,
                          _dp(F), _dp(phi), _dp(E))
    return float(E[0]), F, phi


def rbe_fourier(pos, q, L, alpha, m, S=None, lB=1.0, sub=None, want_phi=False):
    """RBE Fourier estimator (Eq. rbmapprox) for a given batch m[P,3]:
    (E, F[nsub,3], phi or None, rho[P] complex)."""
    lib = _load()
    pos = _f64(pos, (-1, 3)); q = _f64(q)
    N = len(q)
    m = np.ascontiguousarray(m, dtype=np.int32).reshape(-1, 3)
    P = len(m)
    if S is None:
        S = S_of(alpha, L)
    nsub, s, sp = _sub(sub)
    n_out = nsub if sub is not None else N
    F = np.zeros((n_out, 3)); E = np.zeros(1); rho = np.zeros((P, 2))
    phi = np.zeros(n_out) if want_phi else None
    lib.orc_rbe_fourier(N, _dp(pos), _dp(q), L, alpha, lB, S, P, m.ctypes.data_as(_I32),
                        nsub, sp, _dp(F), _dp(phi), _dp(E), _dp(rho))
    return float(E[0]), F, phi, rho[:, 0] + 1j * rho[:, 1]


def rbe_single_k_force(pos, q, L, alpha, m1, S, lB=1.0):
    """RBE force with a batch of one wave vector (weight S), all particles."""
    lib = _load()
    pos = _f64(pos, (-1, 3)); q = _f64(q)
    m1 = np.ascontiguousarray(m1, dtype=np.int32).reshape(3)
    F = np.zeros((len(q), 3))
    lib.orc_rbe_single_k_force(len(q), _dp(pos), _dp(q), L, alpha, lB, S,
                               m1.ctypes.data_as(_I32), _dp(F))
    return F


# ---------------------------------------------------------------- real space
def real_space(pos, q, L, alpha, r_c, lB=1.0, lj_eps=0.0, lj_sigma=1.0, lj_rcut=0.0,
               sub=None, want_phi=False):
    """Real-space Coulomb + shifted LJ, all pairs, minimum image:
    (E_coul, E_lj, Fc[nsub,3], Flj[nsub,3], phi or None)."""
    lib = _load()
    pos = _f64(pos, (-1, 3)); q = _f64(q)
    N = len(q)
    nsub, s, sp = _sub(sub)
    n_out = nsub if sub is not None else N
    Fc = np.zeros((n_out, 3)); Flj = np.zeros((n_out, 3)); E = np.zeros(2)
    phi = np.zeros(n_out) if want_phi else None
    lib.orc_real_space(N, _dp(pos), _dp(q), L, alpha, r_c, lB, lj_eps, lj_sigma, lj_rcut,
                       nsub, sp, _dp(Fc), _dp(Flj), _dp(phi), _dp(E))
    return float(E[0]), float(E[1]), Fc, Flj, phi


def brute_images(pos, q, L, R):
    """Direct image sum of Eq. energy over the cube |n|_inf <= R (lB = 1)."""
    pos = _f64(pos, (-1, 3)); q = _f64(q)
    return float(_load().orc_brute_images(len(q), _dp(pos), _dp(q), L, R))


def fourier_variance(pos, q, L, alpha, mmax, P, lB=1.0, S=None):
    """Proposition 1: exact E|chi_i|^2 (per particle) and F_i,1 over |m|_inf<=mmax."""
    lib = _load()
    pos = _f64(pos, (-1, 3)); q = _f64(q)
    if S is None:
        S = S_of(alpha, L)
    N = len(q)
    var = np.zeros(N); F1 = np.zeros((N, 3))
    lib.orc_fourier_variance(N, _dp(pos), _dp(q), L, alpha, lB, S, mmax, P, _dp(var), _dp(F1))
    return var, F1


# ---------------------------------------------------------------- integrator
def langevin_normals(N, seed, stream, step):
    xi = np.zeros((N, 3))
    _load().orc_langevin_normals(N, seed, stream, step, _dp(xi))
    return xi


def langevin_step(pos, vel, F, L, gamma, kT, dt, mass, seed, stream, step):
    """One kick / Ornstein-Uhlenbeck / drift step; returns new (pos, vel)."""
    pos = _f64(pos, (-1, 3)).copy(); vel = _f64(vel, (-1, 3)).copy(); F = _f64(F, (-1, 3))
    _load().orc_langevin_step(len(pos), _dp(pos), _dp(vel), _dp(F), L, gamma, kT, dt, mass,
                              seed, stream, step)
    return pos, vel


def andersen_step(pos, vel, F, L, nu, kT, dt, mass, seed, stream, step):
    """One leapfrog step with Andersen collisions; returns (pos, vel, collided)."""
    pos = _f64(pos, (-1, 3)).copy(); vel = _f64(vel, (-1, 3)).copy(); F = _f64(F, (-1, 3))
    hit = np.zeros(len(pos), dtype=np.int32)
    _load().orc_andersen_step(len(pos), _dp(pos), _dp(vel), _dp(F), L, nu, kT, dt, mass,
                              seed, stream, step, hit.ctypes.data_as(_INT))
    return pos, vel, hit.astype(bool)


class NoseHoover:
    """Nose-Hoover thermostat state (xi, previous kinetic sum, first-step flag)
    and its leapfrog step (see orc_nose_hoover_step); tau = sqrt(Q / (3 N kT))."""

    def __init__(self, tau):
        self.tau = tau
        self.state = np.array([0.0, 0.0, 1.0])

    def step(self, pos, vel, F, L, kT, dt, mass):
        pos = _f64(pos, (-1, 3)).copy(); vel = _f64(vel, (-1, 3)).copy(); F = _f64(F, (-1, 3))
        _load().orc_nose_hoover_step(len(pos), _dp(pos), _dp(vel), _dp(F), L, self.tau, kT, dt,
                                     mass, _dp(self.state))
        return pos, vel

    @property
    def xi(self):
        return float(self.state[0])


# ---------------------------------------------------------------- observables
def true_energy_virial(pos, q, L, alpha, r_c, mmax, lB=1.0, lj_eps=0.0, lj_sigma=1.0,
                       lj_rcut=0.0):
    """Full-Ewald energy parts and virials (no random batch): dict with E_fourier
    (incl. self, background), E_real, E_lj, E_bg, W_fourier, W_real, W_lj, W_bg;
    pressure = (2 E_kin + W) / (3 V), W the sum of the W parts."""
    pos = _f64(pos, (-1, 3)); q = _f64(q, (-1,))
    out = np.zeros(8)
    _load().orc_true_energy_virial(len(q), _dp(pos), _dp(q), L, alpha, r_c, lB, lj_eps,
                                   lj_sigma, lj_rcut, mmax, _dp(out))
    keys = ("E_fourier", "E_real", "E_lj", "E_bg", "W_fourier", "W_real", "W_lj", "W_bg")
    return dict(zip(keys, out.tolist()))


# ---------------------------------------------------------------- composites
def rbe_forces(pos, q, L, alpha, r_c, P, seed, stream, step, lB=1.0, lj_eps=0.0,
               lj_sigma=1.0, lj_rcut=0.0, sub=None, want_phi=False, m=None):
    """One RBE force evaluation (sample, Fourier estimator, real space, LJ).

    Returns a dict with m, E parts (total, fourier, real, lj), forces per part
    and their sum, and optionally phi = dE/dq.  Forces for ``sub`` only if given.
    ``m`` (P x 3) replaces the i.i.d. sample of this step (e.g. the MH chain's).
    """
    if m is None:
        m, att, bad = sample_k(alpha, L, seed, stream, step, P)
    else:
        m = np.ascontiguousarray(m, dtype=np.int32)
        att, bad = np.ones(len(m), dtype=np.int32), 0
    S = S_of(alpha, L)
    Ef, Ff, phif, rho = rbe_fourier(pos, q, L, alpha, m, S=S, lB=lB, sub=sub, want_phi=want_phi)
    Ec, Elj, Fc, Flj, phir = real_space(pos, q, L, alpha, r_c, lB=lB, lj_eps=lj_eps,
                                        lj_sigma=lj_sigma, lj_rcut=lj_rcut, sub=sub,
                                        want_phi=want_phi)
    out = dict(m=m, attempts=att, bad=bad, S=S, rho=rho,
               E=np.array([Ef + Ec + Elj, Ef, Ec, Elj]),
               F_fourier=Ff, F_real=Fc, F_lj=Flj, F=Ff + Fc + Flj)
    if want_phi:
        out["phi"] = phif + phir
        out["phi_fourier"] = phif
        out["phi_real"] = phir
    return out

"""Helpers shared by the GPU parity tests (comparison metrics, oracle calls)."""
import numpy as np
import pytest

import oracle


def rel_rms(x, ref):
    """sqrt(sum |x - ref|^2) / sqrt(sum |ref|^2) over all particles and components."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.sqrt((ref ** 2).sum())
    return float(np.sqrt(((x - ref) ** 2).sum()) / (den if den > 0 else 1.0))


def energy_rel(e, ref_parts):
    """|e - e_ref| relative to the sum of the magnitudes of the energy parts."""
    return abs(e[0] - ref_parts[0]) / max(np.abs(ref_parts[1:]).sum(), 1e-300)


def oracle_eval(wl, step, sub=None, want_phi=False, pos=None, q=None):
    p = wl.params
    pos = wl.pos.astype(np.float64) if pos is None else pos
    q = wl.q.astype(np.float64) if q is None else q
    return oracle.rbe_forces(pos, q, p.box, p.alpha, p.r_c, p.P, p.seed, p.stream, step,
                             lB=p.coulomb_prefactor, lj_eps=p.lj_eps, lj_sigma=p.lj_sigma,
                             lj_rcut=p.lj_rcut, sub=sub, want_phi=want_phi)


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    return torch


def assert_per_particle(x, ref, what="", rel_rms_scale=1e-4, rel_own=1e-5):
    """Every particle's deviation within rel_rms_scale * RMS|ref| + rel_own * |ref_i|.

    A rel-RMS over all particles can hide a wrong result confined to a few
    particles of a large system; this bound cannot: with the mixed path's
    per-particle errors near 1e-6 of the RMS force, a single particle off by
    1e-3 of the RMS fails it.  x and ref are [n, k] (or [n]) arrays.
    """
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if x.ndim == 1:
        x, ref = x[:, None], ref[:, None]
    dev = np.linalg.norm(x - ref, axis=1)
    mag = np.linalg.norm(ref, axis=1)
    rms = float(np.sqrt((mag ** 2).mean())) if len(mag) else 0.0
    bound = rel_rms_scale * rms + rel_own * mag
    if len(dev) == 0:
        return 0.0
    worst = int(np.argmax(dev / np.maximum(bound, 1e-300)))
    assert np.all(dev <= bound), (what, "particle", worst, dev[worst], bound[worst], rms)
    return float(dev.max() / max(rms, 1e-300))

"""rbe_fourier_forces_noalloc, the entry point for callers that cannot allocate.

Some callers of this library may not call cudaMalloc: an MD engine whose own
pool owns all device memory, or a loop that cannot afford cudaMalloc's
device-wide synchronisation.  They cannot create a handle, so
rbe_fourier_forces_noalloc keeps its scratch in a static device array inside
librbe.  The GPU test calls it through the C ABI several times in a row, on
systems that need different chunk sizes of the scratch's partial sums (so
anything left in the shared array by one call would show up in the next), and
compares each result with the FP64 oracle's RBE Fourier estimator for the same
k-batch and with the handle-based rbe_forces_ex(..., RBE_PART_FOURIER, ...),
within the mixed-path tolerances: force rel-RMS 1e-5 plus a per-particle bound,
energy 1e-6 relative.  The cases include the documented limit (n = 2^20 with
P = 500) and a system whose chunks hold 8192 particles.

This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from gpu_util import assert_per_particle, need_gpu, rel_rms
from paper_2010_01559_gb300 import capi, workloads

TOL_MIXED = 1e-5     # force rel-RMS, as in the other mixed-path tests
TOL_E = 1e-6         # energy, relative


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _call(lib, params, x, n, step, F, E, stream):
    return lib.rbe_fourier_forces_noalloc(ctypes.byref(params), n, _ptr(x), step, _ptr(F),
                                          _ptr(E), ctypes.c_void_p(stream))


def _chunk(n, P):
    """The chunk size the entry point picks (the scratch layout's arithmetic)."""
    def a256(x):
        return (x + 255) & ~255
    c = 512
    while True:
        nch = (n + c - 1) // c if n > 0 else 1
        part = a256(a256(a256(a256(a256(8 * 4096) + 16 * P) + 8 * P) + 8 * P) + 16 * nch)
        if part + 8 * nch * P <= (4 << 20) - 256:
            return c
        c <<= 1


@pytest.mark.gpu
def test_noalloc_matches_oracle_and_handle_path_calls_in_a_row():
    torch = need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_01559_gb300 as rbe
    lib = capi.load()
    big = workloads.config_large(1 << 21, P=1024)
    cases = [(workloads.config_2to1_mixed(), 7, True),        # chunk 512
             (workloads.config_large(), 2, True),             # n = 2^20, P = 500: chunk 1024
             (big, 5, False),                                  # chunk 8192
             (workloads.config_2to1_mixed(), 8, False)]       # chunk 512 again
    chunks = [_chunk(wl.n, wl.params.P) for wl, _, _ in cases]
    assert chunks == [512, 1024, 8192, 512], chunks
    for (wl, step, with_handle), chunk in zip(cases, chunks):
        p = wl.params
        params = rbe.params_from(p, n_max=wl.n)
        x = torch.from_numpy(wl.pos_q()).cuda()
        F = torch.full((wl.n, 4), float("nan"), dtype=torch.float32, device="cuda")
        E = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        st = _call(lib, params, x, wl.n, step, F, E, torch.cuda.current_stream().cuda_stream)
        assert st == capi.RBE_OK, lib.rbe_last_error(None)
        Fn = F[:, :3].cpu().numpy()
        # the oracle: the same k-batch (bit-exact sampler), rho over all particles
        # in FP64, forces of all particles or of 1024 evenly spaced ones
        m, _, bad = oracle.sample_k(p.alpha, p.box, p.seed, p.stream, step, p.P)
        assert bad == 0
        sub = None if wl.n <= 10000 else np.linspace(0, wl.n - 1, 1024).astype(int)
        Eo, Fo, _, _ = oracle.rbe_fourier(wl.pos.astype(np.float64), wl.q.astype(np.float64),
                                          p.box, p.alpha, m, lB=p.coulomb_prefactor, sub=sub)
        Fs = Fn if sub is None else Fn[sub]
        err_f = rel_rms(Fs, Fo)
        err_e = abs(E.item() - Eo) / abs(Eo)
        print(wl.name, "P", p.P, "chunk", chunk, "vs oracle: F", err_f, "E", err_e)
        assert err_f <= TOL_MIXED, (wl.name, err_f)
        assert_per_particle(Fs, Fo, (wl.name, "vs oracle"))
        assert err_e <= TOL_E, (wl.name, err_e)
        if with_handle:
            h = rbe.RBE(params)
            Fr, Er, _ = h.forces(x, step, parts=rbe.RBE_PART_FOURIER)
            torch.cuda.synchronize()
            err_h = rel_rms(Fn, Fr[:, :3].cpu().numpy())
            assert err_h <= TOL_MIXED, (wl.name, err_h)
            assert_per_particle(Fn, Fr[:, :3].cpu().numpy(), (wl.name, "vs handle path"))
            assert abs(E.item() - Er[0, 1].item()) <= TOL_E * abs(Er[0, 1].item())
            h.close()
        del x, F, E


def test_noalloc_rejects_sizes_beyond_its_limits_on_host():
    """Checked before any CUDA call, so this runs without a GPU."""
    from paper_2010_01559_gb300 import build
    build.build()
    lib = capi.load()
    big_p = capi.make_params(box=25.0, alpha=0.3, r_c=5.0, P=1025)
    assert _call(lib, big_p, None, 0, 0, None, None, 0) == capi.RBE_ERR_ARG
    assert b"1024" in lib.rbe_last_error(None)
    big_table = capi.make_params(box=2000.0, alpha=0.3, r_c=5.0, P=10)
    assert _call(lib, big_table, None, 0, 0, None, None, 0) == capi.RBE_ERR_ARG
    assert b"4096" in lib.rbe_last_error(None)
    # n * P beyond what chunks of 65536 particles fit: pointers are never read
    many = capi.make_params(box=25.0, alpha=0.3, r_c=5.0, P=1024)
    fake = ctypes.c_void_p(256)
    st = lib.rbe_fourier_forces_noalloc(ctypes.byref(many), 2 ** 31 - 1, fake, 0, fake, None,
                                        None)
    assert st == capi.RBE_ERR_ARG
    assert b"n * P too large" in lib.rbe_last_error(None)
    # only the exact sampler
    mh = capi.make_params(box=25.0, alpha=0.3, r_c=5.0, P=10)
    mh.sampler = 1
    assert _call(lib, mh, None, 0, 0, None, None, 0) == capi.RBE_ERR_ARG
    assert b"exact sampler" in lib.rbe_last_error(None)
    # non-finite parameters
    for field, val in (("box", float("inf")), ("alpha", float("nan")),
                       ("coulomb_prefactor", float("inf"))):
        bad = capi.make_params(box=25.0, alpha=0.3, r_c=5.0, P=10)
        setattr(bad, field, val)
        assert _call(lib, bad, None, 0, 0, None, None, 0) == capi.RBE_ERR_ARG, field
        assert b"finite" in lib.rbe_last_error(None), field
    # n < 0, and n > 0 with a null buffer
    ok = capi.make_params(box=25.0, alpha=0.3, r_c=5.0, P=10)
    assert _call(lib, ok, None, -1, 0, None, None, 0) == capi.RBE_ERR_ARG
    assert lib.rbe_fourier_forces_noalloc(ctypes.byref(ok), 5, None, 0, fake, None,
                                          None) == capi.RBE_ERR_ARG
    # n = 0 without E_out: nothing to compute, no GPU work
    assert _call(lib, ok, None, 0, 0, None, None, 0) == capi.RBE_OK

"""rbe_fourier_forces_noalloc, the entry point for callers that cannot allocate.

Some callers of this library may not call cudaMalloc: an MD engine whose own
pool owns all device memory, or a loop that cannot afford cudaMalloc's
device-wide synchronisation.  They cannot create a
handle, so rbe_fourier_forces_noalloc keeps its scratch in a static device
array inside librbe.  The GPU test calls it through the C ABI twice in a row, on
two different systems (so anything left in the shared array by the first call
would show up in the second), and compares each result with the handle-based
rbe_forces_ex(..., RBE_PART_FOURIER, ...) within the mixed-path tolerance.
"""
import ctypes

import pytest

from gpu_util import need_gpu, rel_rms
from paper_2010_01559_gb300 import capi, workloads

TOL_MIXED = 1e-5     # force rel-RMS, as in the other mixed-path tests
TOL_E = 1e-6         # energy, relative


def _call(lib, params, x, n, step, F, E, stream):
    return lib.rbe_fourier_forces_noalloc(
        ctypes.byref(params), n, ctypes.c_void_p(x.data_ptr()) if x is not None else None, step,
        ctypes.c_void_p(F.data_ptr()) if F is not None else None,
        ctypes.c_void_p(E.data_ptr()) if E is not None else None, ctypes.c_void_p(stream))


@pytest.mark.gpu
def test_noalloc_matches_handle_path_two_calls_in_a_row():
    torch = need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_01559_gb300 as rbe
    lib = capi.load()
    cases = [(workloads.config_2to1_mixed(), 7),
             (workloads.electrolyte_1to1(3000, 0.064, 0.3, 5.0, 300, seed=12), 2)]
    for wl, step in cases:
        params = rbe.params_from(wl.params, n_max=wl.n)
        x = torch.from_numpy(wl.pos_q()).cuda()
        F = torch.full((wl.n, 4), float("nan"), dtype=torch.float32, device="cuda")
        E = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        st = _call(lib, params, x, wl.n, step, F, E, torch.cuda.current_stream().cuda_stream)
        assert st == capi.RBE_OK, lib.rbe_last_error(None)
        h = rbe.RBE(params)
        Fr, Er, _ = h.forces(x, step, parts=rbe.RBE_PART_FOURIER)
        torch.cuda.synchronize()
        err_f = rel_rms(F[:, :3].cpu().numpy(), Fr[:, :3].cpu().numpy())
        err_e = abs(E.item() - Er[0, 1].item()) / abs(Er[0, 1].item())
        h.close()
        assert err_f <= TOL_MIXED, (wl.name, err_f)
        assert err_e <= TOL_E, (wl.name, err_e)


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

"""Failure detection without faulting the GPU.

* A NaN or infinite position or charge is latched on the device and reported
  as RBE_ERR_NONFINITE by the next synchronisation (forces call, MD step over
  the neighbour list, FP64 path, the allocation-free entry point); the latch
  clears, and the next call on finite input matches the oracle again.  Every
  index the kernels derive from a position goes through the 32-bit fixed-point
  record (or the FP64 wrap, which maps NaN to 0), so such input stays in range.
* A host wait limit (rbe_set_wait_limit) far below the work's duration makes
  rbe_step_host return RBE_ERR_TIMEOUT with the step still queued; rbe_sync
  then completes it, and the trajectory equals the one run without a limit.
* The bounds-checked build (-DRBE_CHECK_BOUNDS) runs MD steps with frequent
  list rebuilds (with the structure factors and the list pass launched apart
  and in one launch), forces calls, the FP64 path and a heterogeneous batch
  with every data-derived index checked, reports no violation, and gives
  bitwise the same forces as the normal build.
"""
import copy
import ctypes
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_util import assert_per_particle, need_gpu, oracle_eval, rel_rms
from paper_2010_01559_gb300 import capi, workloads

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rbe():
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_01559_gb300 as rbe
    return rbe


def _status(exc):
    return exc.value.status


def test_nonfinite_input_is_latched_and_cleared(rbe):
    import torch
    wl = workloads.config_small_fp64()
    h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    x = torch.from_numpy(wl.pos_q()).cuda()
    bad = x.clone()
    bad[17, 1] = float("nan")
    h.forces(bad, 3)
    with pytest.raises(rbe.RBEError) as e:
        h.sync()
    assert _status(e) == capi.RBE_ERR_NONFINITE
    # the latch is cleared: finite input again gives the oracle's forces
    F, _, _ = h.forces(x, 3)
    h.sync()
    ref = oracle_eval(wl, 3)
    assert rel_rms(F[:, :3].cpu().numpy(), ref["F"]) <= 1e-5
    assert_per_particle(F[:, :3].cpu().numpy(), ref["F"], "after the latch")
    # an infinite charge in an MD step over the neighbour list
    vel = torch.zeros_like(x)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    pos = x.clone()
    pos[5, 3] = float("inf")
    h.step(pos, vel, 2, step)
    with pytest.raises(rbe.RBEError) as e:
        h.sync()
    assert _status(e) == capi.RBE_ERR_NONFINITE
    # the FP64 path
    x64 = x.double().contiguous()
    x64[3, 0] = float("-inf")
    h.forces_f64(x64, 1)
    with pytest.raises(rbe.RBEError) as e:
        h.sync()
    assert _status(e) == capi.RBE_ERR_NONFINITE
    h.sync()
    h.close()


def test_nonfinite_input_in_the_allocation_free_entry_point(rbe):
    import torch
    lib = capi.load()
    wl = workloads.config_small_fp64()
    params = rbe.params_from(wl.params, n_max=wl.n)
    x = torch.from_numpy(wl.pos_q()).cuda()
    x[11, 2] = float("nan")
    F = torch.zeros((wl.n, 4), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    st = lib.rbe_fourier_forces_noalloc(ctypes.byref(params), wl.n,
                                        ctypes.c_void_p(x.data_ptr()), 0,
                                        ctypes.c_void_p(F.data_ptr()), None,
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == capi.RBE_ERR_NONFINITE


def test_wait_limit_times_out_and_the_queued_step_completes(rbe):
    import torch
    wl = workloads.config_large(1 << 18)
    hp = torch.from_numpy(wl.pos_q()).pin_memory()
    hv = torch.zeros((wl.n, 4), dtype=torch.float32).pin_memory()
    hv[:, :3] = torch.from_numpy(wl.vel)
    ref_p, ref_v = hp.clone().pin_memory(), hv.clone().pin_memory()
    h = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    h.set_graph(True)
    h.set_wait_limit(1e-7)                 # far below the ~0.7 ms of four steps
    with pytest.raises(rbe.RBEError) as e:
        h.step_host(hp, hv, 4, 0)
    assert _status(e) == capi.RBE_ERR_TIMEOUT
    h.set_wait_limit(0.0)
    h.sync()                               # the queued steps finish
    r = rbe.RBE(rbe.params_from(wl.params, n_max=wl.n))
    r.set_graph(True)
    r.step_host(ref_p, ref_v, 4, 0)
    assert torch.equal(hp, ref_p) and torch.equal(hv, ref_v)
    with pytest.raises(rbe.RBEError) as e:
        h.set_wait_limit(-1.0)
    assert _status(e) == capi.RBE_ERR_ARG
    h.close()
    r.close()


_CHECKED_SCRIPT = r"""
import json, os, sys
import numpy as np
sys.path.insert(0, {root!r})
from paper_2010_01559_gb300 import build, capi
capi._lib = capi.load(build.build(check_bounds={checked}))
import torch
import paper_2010_01559_gb300 as rbe
from paper_2010_01559_gb300 import workloads
out = {{}}
wl = workloads.config_2to1_mixed()
sp = wl.params
sp.skin = 0.1                                  # rebuilds every few steps
h = rbe.RBE(rbe.params_from(sp, n_max=wl.n))
h.set_graph(True)
pos = torch.from_numpy(wl.pos_q()).cuda()
vel = torch.zeros_like(pos)
vel[:, :3] = torch.from_numpy(wl.vel * 3.0).cuda()
step = torch.zeros(1, dtype=torch.int64, device="cuda")
F = torch.zeros_like(pos)
h.step(pos, vel, 30, step, F_out=F)
h.sync()
out["builds"] = h.list_stats()["builds"]
Ff, E, phi = h.forces(pos, 31, phi=True)
F64, E64, _ = h.forces_f64(pos.double().contiguous(), 31)
h.sync()
# the same steps with the structure factors and the list pass in one launch
h2 = rbe.RBE(rbe.params_from(sp, n_max=wl.n))
h2.set_fusion(True)
h2.set_graph(True)
pos2 = torch.from_numpy(wl.pos_q()).cuda()
vel2 = torch.zeros_like(pos2)
vel2[:, :3] = torch.from_numpy(wl.vel * 3.0).cuda()
step2 = torch.zeros(1, dtype=torch.int64, device="cuda")
F2 = torch.zeros_like(pos2)
h2.step(pos2, vel2, 30, step2, F_out=F2)
h2.sync()
out["builds_fused"] = h2.list_stats()["builds"]
reps = workloads.config_replicas(n_rep=5, n_hi=4000)
hb = rbe.RBEBatch([rbe.params_from(w.params) for w in reps], [w.n for w in reps])
xb = torch.from_numpy(np.concatenate([w.pos_q() for w in reps])).cuda()
vb = torch.zeros_like(xb)
sb = torch.zeros(1, dtype=torch.int64, device="cuda")
hb.step(xb, vb, 5, sb)
Fb, _, _ = hb.forces(xb, 6)
hb.sync()
hb.set_fusion(True)
Fbs = torch.zeros_like(xb)
hb.step(xb, vb, 3, sb, F_out=Fbs)
hb.sync()
np.savez({path!r}, F=F.cpu().numpy(), Ff=Ff.cpu().numpy(), phi=phi.cpu().numpy(),
         F64=F64.cpu().numpy(), Fb=Fb.cpu().numpy(), pos=pos.cpu().numpy(),
         F2=F2.cpu().numpy(), pos2=pos2.cpu().numpy(), Fbs=Fbs.cpu().numpy())
print(json.dumps(out))
"""


def _run_scenario(checked, path):
    code = _CHECKED_SCRIPT.format(root=ROOT, checked=checked, path=path)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_bounds_checked_build_finds_no_violation_and_matches(rbe, tmp_path):
    a = _run_scenario(True, str(tmp_path / "checked.npz"))
    b = _run_scenario(False, str(tmp_path / "normal.npz"))
    assert a["builds"] >= 3 and a["builds"] == b["builds"]
    assert a["builds_fused"] == a["builds"] == b["builds_fused"]
    ca, cb = np.load(tmp_path / "checked.npz"), np.load(tmp_path / "normal.npz")
    for k in ("F", "Ff", "phi", "F64", "Fb", "pos", "F2", "pos2", "Fbs"):
        assert np.array_equal(ca[k], cb[k]), k
    # the fused and the separate list step give the same trajectory
    assert np.array_equal(ca["F2"], ca["F"]) and np.array_equal(ca["pos2"], ca["pos"])

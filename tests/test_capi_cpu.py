"""CPU checks of the C ABI: the library builds, loads, exports every symbol the
header declares, and rejects bad arguments on the host (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2010_01559_gb300 import build as rbe_build
from paper_2010_01559_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    rbe_build.build()
    return capi.load()


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "rbe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rbe_[a-z0-9_]+)\s*\(", src)))


def test_header_matches_binding():
    assert _declared_symbols() == sorted(capi.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_symbols():
        assert hasattr(lib, name), name


def test_params_layout_matches_header():
    assert ctypes.sizeof(capi.rbe_params) == 144
    assert capi.rbe_params.seed.offset == 88
    assert capi.rbe_params.precision.offset == 108
    assert capi.rbe_params.andersen_nu.offset == 112
    assert capi.rbe_params.sampler.offset == 120
    assert capi.rbe_params.thermostat.offset == 124
    assert capi.rbe_params.nh_tau.offset == 128
    assert capi.rbe_params.skin.offset == 136
    assert ctypes.sizeof(capi.rbe_tuning) == 20


def _create(lib, **kw):
    base = dict(box=25.0, alpha=0.3, r_c=5.0, P=100, n_max=1000, lj_eps=1.0, lj_sigma=1.0,
                lj_rcut=2 ** (1 / 6))
    base.update(kw)
    p = capi.make_params(**base)
    h = ctypes.c_void_p()
    st = lib.rbe_create(ctypes.byref(p), ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("kw,needle", [
    (dict(box=0.0), "box"),
    (dict(alpha=-1.0), "alpha"),
    (dict(r_c=13.0), "L/2"),
    (dict(P=0), "P must"),
    (dict(n_max=-1), "n_max"),
    (dict(lj_rcut=6.0), "lj_rcut"),
    (dict(box=1.0, r_c=0.3, alpha=0.5, lj_eps=0.0), "too small"),
    (dict(mass=0.0), "mass"),
    (dict(sampler=2), "sampler"),
    (dict(thermostat=3), "thermostat"),
    (dict(thermostat=2, nh_tau=0.0), "nh_tau"),
    (dict(thermostat=2, nh_tau=0.5, kT=0.0), "kT > 0"),
    (dict(skin=float("nan")), "skin"),
    (dict(skin=4.0), "skin must be <="),        # L/3 - r_c = 3.33 at L = 25, r_c = 5
    (dict(andersen_nu=-1.0), "andersen_nu"),
    (dict(andersen_nu=2000.0, dt=1e-3), "andersen_nu"),
])
def test_create_rejects_bad_parameters_on_host(lib, kw, needle):
    st, h = _create(lib, **kw)
    assert st == capi.RBE_ERR_ARG
    assert not h.value
    assert needle in lib.rbe_last_error(None).decode()


def test_null_arguments_are_rejected(lib):
    assert lib.rbe_create(None, None) == capi.RBE_ERR_ARG
    assert lib.rbe_forces(None, 0, None, 0, None, None, None) == capi.RBE_ERR_ARG
    assert lib.rbe_step(None, 0, None, None, 1, None) == capi.RBE_ERR_ARG
    assert lib.rbe_sync(None) == capi.RBE_ERR_ARG
    assert lib.rbe_nose_hoover_xi(None, None, 0) == capi.RBE_ERR_ARG
    assert lib.rbe_list_stats(None, None, None, None) == capi.RBE_ERR_ARG
    assert lib.rbe_step_ex(None, 0, None, None, 1, None, None) == capi.RBE_ERR_ARG
    assert lib.rbe_set_fusion(None, 1) == capi.RBE_ERR_ARG
    assert lib.rbe_get_fusion(None, None) == capi.RBE_ERR_ARG
    lib.rbe_destroy(None)
    n = ctypes.c_int32(0)
    assert lib.rbe_create_batch(None, ctypes.byref(n), 0, None) == capi.RBE_ERR_ARG


def test_product_path_fails_loudly_without_library(tmp_path):
    with pytest.raises(RuntimeError, match="librbe.so not found"):
        capi.load(str(tmp_path / "missing" / "librbe.so"))

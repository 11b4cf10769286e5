"""ctypes binding of librbe (include/rbe.h): same names, argument marshalling only.

Every function here passes plain pointers and sizes to the CUDA library; no
step of the method runs in Python.  If ``_build/librbe.so`` is missing the
import of this module still succeeds but every call raises ``RuntimeError`` --
there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librbe.so")

RBE_OK, RBE_ERR_ARG, RBE_ERR_CUDA, RBE_ERR_OOM = 0, 1, 2, 3
RBE_ERR_SAMPLER, RBE_ERR_TIMEOUT, RBE_ERR_NONFINITE, RBE_ERR_STATE, RBE_ERR_LIST = 4, 5, 6, 7, 8
RBE_ERR_BOUNDS = 9
RBE_FP64, RBE_MIXED = 0, 1
RBE_PART_FOURIER, RBE_PART_REAL, RBE_PART_LJ, RBE_PART_ALL = 1, 2, 4, 7
RBE_SAMPLER_EXACT, RBE_SAMPLER_MH = 0, 1
RBE_THERMO_LANGEVIN, RBE_THERMO_ANDERSEN, RBE_THERMO_NOSE_HOOVER = 0, 1, 2

STATUS_NAMES = {0: "RBE_OK", 1: "RBE_ERR_ARG", 2: "RBE_ERR_CUDA", 3: "RBE_ERR_OOM",
                4: "RBE_ERR_SAMPLER", 5: "RBE_ERR_TIMEOUT", 6: "RBE_ERR_NONFINITE",
                7: "RBE_ERR_STATE", 8: "RBE_ERR_LIST", 9: "RBE_ERR_BOUNDS"}


class rbe_params(ctypes.Structure):
    _fields_ = [("box", ctypes.c_double), ("alpha", ctypes.c_double), ("r_c", ctypes.c_double),
                ("coulomb_prefactor", ctypes.c_double), ("lj_eps", ctypes.c_double),
                ("lj_sigma", ctypes.c_double), ("lj_rcut", ctypes.c_double),
                ("gamma", ctypes.c_double), ("kT", ctypes.c_double), ("dt", ctypes.c_double),
                ("mass", ctypes.c_double), ("seed", ctypes.c_uint64), ("stream", ctypes.c_uint32),
                ("P", ctypes.c_int32), ("n_max", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("andersen_nu", ctypes.c_double), ("sampler", ctypes.c_int32),
                ("thermostat", ctypes.c_int32), ("nh_tau", ctypes.c_double),
                ("skin", ctypes.c_double)]


class rbe_tuning(ctypes.Structure):
    _fields_ = [("rho_chunk", ctypes.c_int32), ("force_split", ctypes.c_int32),
                ("real_split", ctypes.c_int32), ("real_seg", ctypes.c_int32),
                ("list_split", ctypes.c_int32)]


class rbe_peaks(ctypes.Structure):
    _fields_ = [("sfu_per_clk_sm", ctypes.c_double), ("ffma_per_clk_sm", ctypes.c_double),
                ("sm_clock_mhz", ctypes.c_double), ("sms", ctypes.c_int32)]


class rbe_info(ctypes.Structure):
    _fields_ = [("H", ctypes.c_double), ("S", ctypes.c_double), ("M", ctypes.c_int32),
                ("n_cells_dim", ctypes.c_int32), ("n", ctypes.c_int32), ("P", ctypes.c_int32),
                ("n_systems", ctypes.c_int32), ("first_particle", ctypes.c_int32),
                ("first_k", ctypes.c_int32), ("reserved", ctypes.c_int32)]


assert ctypes.sizeof(rbe_params) == 144

_H = ctypes.c_void_p
_P = ctypes.c_void_p
_SIGS = {
    "rbe_create": ([ctypes.POINTER(rbe_params), ctypes.POINTER(_H)], ctypes.c_int),
    "rbe_create_batch": ([ctypes.POINTER(rbe_params), ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                          ctypes.POINTER(_H)], ctypes.c_int),
    "rbe_destroy": ([_H], None),
    "rbe_last_error": ([_H], ctypes.c_char_p),
    "rbe_set_stream": ([_H, _P], ctypes.c_int),
    "rbe_get_info": ([_H, ctypes.c_int32, ctypes.POINTER(rbe_info)], ctypes.c_int),
    "rbe_get_table": ([_H, ctypes.c_int32, _P], ctypes.c_int),
    "rbe_sample_k": ([_H, ctypes.c_uint64, _P], ctypes.c_int),
    "rbe_forces": ([_H, ctypes.c_int32, _P, ctypes.c_uint64, _P, _P, _P], ctypes.c_int),
    "rbe_forces_ex": ([_H, ctypes.c_int32, _P, ctypes.c_uint64, ctypes.c_int32, _P, _P, _P],
                      ctypes.c_int),
    "rbe_forces_f64": ([_H, ctypes.c_int32, _P, ctypes.c_uint64, ctypes.c_int32, _P, _P, _P],
                       ctypes.c_int),
    "rbe_step": ([_H, ctypes.c_int32, _P, _P, ctypes.c_int32, _P], ctypes.c_int),
    "rbe_step_f64": ([_H, ctypes.c_int32, _P, _P, ctypes.c_int32, _P], ctypes.c_int),
    "rbe_set_graph": ([_H, ctypes.c_int32], ctypes.c_int),
    "rbe_forces_host": ([_H, ctypes.c_int32, _P, ctypes.c_uint64, _P, _P], ctypes.c_int),
    "rbe_step_host": ([_H, ctypes.c_int32, _P, _P, ctypes.c_int32, ctypes.c_uint64], ctypes.c_int),
    "rbe_sync": ([_H], ctypes.c_int),
    "rbe_set_wait_limit": ([_H, ctypes.c_double], ctypes.c_int),
    "rbe_set_fusion": ([_H, ctypes.c_int32], ctypes.c_int),
    "rbe_get_fusion": ([_H, _P], ctypes.c_int),
    "rbe_set_tuning": ([_H, ctypes.POINTER(rbe_tuning)], ctypes.c_int),
    "rbe_get_tuning": ([_H, ctypes.POINTER(rbe_tuning)], ctypes.c_int),
    "rbe_autotune": ([_H, ctypes.c_int32, _P, ctypes.POINTER(rbe_tuning)], ctypes.c_int),
    "rbe_profile": ([_H, ctypes.c_int32], ctypes.c_int),
    "rbe_profile_read": ([_H, _P, _P], ctypes.c_int),
    "rbe_launch_count": ([_H, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "rbe_fourier_forces_noalloc": ([ctypes.POINTER(rbe_params), ctypes.c_int32, _P,
                                    ctypes.c_uint64, _P, _P, _P], ctypes.c_int),
    "rbe_probe_peaks": ([ctypes.POINTER(rbe_peaks)], ctypes.c_int),
    "rbe_nose_hoover_xi": ([_H, _P, ctypes.c_int32], ctypes.c_int),
    "rbe_step_ex": ([_H, ctypes.c_int32, _P, _P, ctypes.c_int32, _P, _P], ctypes.c_int),
    "rbe_list_stats": ([_H, _P, _P, _P], ctypes.c_int),
    "rbe_observables": ([_H, ctypes.c_int32, _P, _P, ctypes.c_int32, _P], ctypes.c_int),
}

#: kernel names in RBE_K_* order
KERNELS = ("prep", "scan", "scatter", "cell_order", "rho", "finalize", "fourier_force",
           "real", "energy", "list_build", "rho_list")

#: every symbol include/rbe.h declares
EXPORTED = tuple(_SIGS)

_lock = threading.Lock()
_lib = None


class RBEError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path: str | None = None) -> ctypes.CDLL:
    """Load librbe.so (raises RuntimeError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"librbe.so not found at {p}: build it with "
                               "`python -m paper_2010_01559_gb300.build` (needs nvcc)")
        lib = ctypes.CDLL(p)
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        if path is None:
            _lib = lib
        return lib


def check(status: int, handle=None) -> None:
    if status != RBE_OK:
        msg = load().rbe_last_error(handle)
        raise RBEError(status, msg.decode() if msg else "")


def make_params(box, alpha, r_c, P, seed=0, stream=0, coulomb_prefactor=1.0, lj_eps=0.0,
                lj_sigma=1.0, lj_rcut=0.0, gamma=1.0, kT=1.0, dt=1e-3, mass=1.0, n_max=0,
                precision=RBE_MIXED, sampler=RBE_SAMPLER_EXACT, thermostat=RBE_THERMO_LANGEVIN,
                andersen_nu=0.0, nh_tau=0.0, skin=0.0) -> rbe_params:
    return rbe_params(box=box, alpha=alpha, r_c=r_c, coulomb_prefactor=coulomb_prefactor,
                      lj_eps=lj_eps, lj_sigma=lj_sigma, lj_rcut=lj_rcut, gamma=gamma, kT=kT,
                      dt=dt, mass=mass, seed=seed, stream=stream, P=P, n_max=n_max,
                      precision=precision, andersen_nu=andersen_nu, sampler=sampler,
                      thermostat=thermostat, nh_tau=nh_tau, skin=skin)


def __getattr__(name):
    # rbe_* names resolve to the raw ctypes functions of the loaded library
    if name in _SIGS:
        return getattr(load(), name)
    raise AttributeError(name)

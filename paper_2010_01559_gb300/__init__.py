"""GB300-native random batch Ewald (RBE) force engine (arXiv:2010.01559).

The computation lives in ``librbe.so`` (CUDA for sm_103a, C ABI in
``include/rbe.h``).  This package provides

* :mod:`.capi` -- the ctypes binding with the C ABI's names,
* :class:`RBE` / :class:`RBEBatch` -- handles that marshal torch CUDA tensors,
* :class:`RBEEnergy` -- a ``torch.autograd.Function`` returning the energy of a
  frozen k-batch with backward dE/dr = -F and dE/dq = phi,
* :mod:`.workloads` -- seeded synthetic electrolytes (inputs only).

PyTorch supplies device memory and streams; every step of the method runs in
the library's kernels.  Without ``librbe.so`` every call raises.
"""
from __future__ import annotations

import ctypes

from . import capi
from .capi import (RBE_FP64, RBE_MIXED, RBE_PART_ALL, RBE_PART_FOURIER, RBE_PART_LJ,
                   RBE_PART_REAL, RBE_SAMPLER_EXACT, RBE_SAMPLER_MH, RBE_THERMO_ANDERSEN,
                   RBE_THERMO_LANGEVIN, RBE_THERMO_NOSE_HOOVER, RBEError)

__all__ = ["capi", "RBE", "RBEBatch", "RBEEnergy", "params_from", "RBEError",
           "RBE_FP64", "RBE_MIXED", "RBE_PART_ALL", "RBE_PART_FOURIER", "RBE_PART_LJ",
           "RBE_PART_REAL"]


def _torch():
    import torch
    return torch


def params_from(sp, n_max=0, precision=RBE_MIXED) -> capi.rbe_params:
    """rbe_params from a workloads.SystemParams (or any object with those fields)."""
    return capi.make_params(box=sp.box, alpha=sp.alpha, r_c=sp.r_c, P=sp.P, seed=sp.seed,
                            stream=sp.stream, coulomb_prefactor=sp.coulomb_prefactor,
                            lj_eps=sp.lj_eps, lj_sigma=sp.lj_sigma, lj_rcut=sp.lj_rcut,
                            gamma=sp.gamma, kT=sp.kT, dt=sp.dt, mass=sp.mass, n_max=n_max,
                            precision=precision, sampler=getattr(sp, "sampler", 0),
                            thermostat=getattr(sp, "thermostat", 0),
                            andersen_nu=getattr(sp, "andersen_nu", 0.0),
                            nh_tau=getattr(sp, "nh_tau", 0.0),
                            skin=getattr(sp, "skin", 0.0))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _need(t, dtype, cols, n, name):
    torch = _torch()
    if t is None:
        raise ValueError(f"{name} is required")
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous() or tuple(t.shape) != (n, cols):
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor of shape ({n}, {cols})")
    if t.data_ptr() % 16:
        raise ValueError(f"{name} must be 16-byte aligned")
    return t


class _HandleBase:
    def __init__(self):
        self._h = ctypes.c_void_p()
        self.lib = capi.load()

    @property
    def handle(self):
        return self._h

    def _stream(self):
        torch = _torch()
        capi.check(self.lib.rbe_set_stream(self._h, ctypes.c_void_p(
            torch.cuda.current_stream().cuda_stream)), self._h)

    def close(self):
        if self._h:
            self.lib.rbe_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self, sys=0) -> capi.rbe_info:
        inf = capi.rbe_info()
        capi.check(self.lib.rbe_get_info(self._h, sys, ctypes.byref(inf)), self._h)
        return inf

    def table(self, sys=0):
        import numpy as np
        inf = self.info(sys)
        t = np.zeros(2 * inf.M + 1, dtype=np.uint64)
        capi.check(self.lib.rbe_get_table(self._h, sys, t.ctypes.data_as(ctypes.c_void_p)), self._h)
        return t

    def sample_k(self, step):
        """int32 [total P, 4] = (m_x, m_y, m_z, attempts) of step `step`."""
        torch = _torch()
        k = sum(self.info(s).P for s in range(self.info(0).n_systems))
        out = torch.empty((k, 4), dtype=torch.int32, device="cuda")
        self._stream()
        capi.check(self.lib.rbe_sample_k(self._h, step, _ptr(out)), self._h)
        return out

    def sync(self):
        capi.check(self.lib.rbe_sync(self._h), self._h)

    def set_wait_limit(self, seconds):
        """Longest host wait for the GPU in seconds (0: none); past it a call
        raises RBEError(RBE_ERR_TIMEOUT) with the work still queued
        (``rbe_set_wait_limit``)."""
        capi.check(self.lib.rbe_set_wait_limit(self._h, float(seconds)), self._h)

    def set_fusion(self, on):
        """Structure factors and the standing-list pass of a mixed list MD
        step in one launch (True), two (False), or chosen by the autotuner
        and the system size (None, the default) (``rbe_set_fusion``)."""
        v = -1 if on is None else (1 if on else 0)
        capi.check(self.lib.rbe_set_fusion(self._h, v), self._h)

    def get_fusion(self):
        """Whether a list MD step at the current particle count runs fused."""
        v = ctypes.c_int32(0)
        capi.check(self.lib.rbe_get_fusion(self._h, ctypes.byref(v)), self._h)
        return bool(v.value)

    def set_tuning(self, rho_chunk=0, force_split=0, real_split=0, real_seg=0, list_split=0):
        t = capi.rbe_tuning(rho_chunk, force_split, real_split, real_seg, list_split)
        capi.check(self.lib.rbe_set_tuning(self._h, ctypes.byref(t)), self._h)

    def get_tuning(self):
        """(rho_chunk, force_split, real_split, real_seg, list_split) in effect."""
        t = capi.rbe_tuning()
        capi.check(self.lib.rbe_get_tuning(self._h, ctypes.byref(t)), self._h)
        return t.rho_chunk, t.force_split, t.real_split, t.real_seg, t.list_split

    def autotune(self, pos_q):
        """Pick the fastest launch shapes on this input; returns them."""
        t = capi.rbe_tuning()
        self._stream()
        capi.check(self.lib.rbe_autotune(self._h, pos_q.shape[0], _ptr(pos_q), ctypes.byref(t)),
                   self._h)
        return t.rho_chunk, t.force_split, t.real_split, t.real_seg, t.list_split

    def profile(self, on=True):
        capi.check(self.lib.rbe_profile(self._h, 1 if on else 0), self._h)

    def observables(self, pos_q, vel=None, mmax=0):
        """True (non-random) energy and pressure (rbe_observables): a list of
        dicts, one per system, with E_total, E_fourier, E_real, E_lj, E_kin,
        W_fourier, W_real, W_lj, W_bg, pressure and T_kin."""
        import numpy as np
        torch = _torch()
        n = pos_q.shape[0]
        _need(pos_q, torch.float32, 4, n, "pos_q")
        if vel is not None:
            _need(vel, torch.float32, 4, n, "vel")
        nsys = self._nsys()
        out = np.zeros(12 * nsys)
        capi.check(self.lib.rbe_observables(self._h, n, _ptr(pos_q),
                                            _ptr(vel) if vel is not None else None, mmax,
                                            out.ctypes.data_as(ctypes.c_void_p)), self._h)
        keys = ("E_total", "E_fourier", "E_real", "E_lj", "E_kin", "W_fourier", "W_real",
                "W_lj", "W_bg", "pressure", "T_kin")
        return [dict(zip(keys, out[12 * s:12 * s + 11].tolist())) for s in range(nsys)]

    def profile_read(self):
        """{kernel name: (device ms, launches)} accumulated since the last read."""
        import numpy as np
        ms = np.zeros(len(capi.KERNELS), dtype=np.float64)
        cnt = np.zeros(len(capi.KERNELS), dtype=np.int64)
        capi.check(self.lib.rbe_profile_read(self._h, ms.ctypes.data_as(ctypes.c_void_p),
                                             cnt.ctypes.data_as(ctypes.c_void_p)), self._h)
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(capi.KERNELS)}

    def launch_count(self):
        c = ctypes.c_int64()
        capi.check(self.lib.rbe_launch_count(self._h, ctypes.byref(c)), self._h)
        return c.value

    def list_stats(self):
        """Neighbour-list builds so far, the largest neighbour count seen at a
        build and the per-particle capacity (``rbe_list_stats``)."""
        b = ctypes.c_int64(0); m = ctypes.c_int32(0); c = ctypes.c_int32(0)
        capi.check(self.lib.rbe_list_stats(self._h, ctypes.byref(b), ctypes.byref(m),
                                           ctypes.byref(c)), self._h)
        return {"builds": b.value, "max_count": m.value, "capacity": c.value}

    def nose_hoover_xi(self, xi=None):
        """The Nose-Hoover friction of every system (``rbe_nose_hoover_xi``):
        returns them as a list, or with ``xi`` given sets them (a resume)."""
        n = self._nsys()
        buf = (ctypes.c_double * n)(*([0.0] * n if xi is None else [float(v) for v in xi]))
        capi.check(self.lib.rbe_nose_hoover_xi(self._h, buf, 0 if xi is None else 1), self._h)
        return list(buf)

    def set_graph(self, on=True):
        capi.check(self.lib.rbe_set_graph(self._h, 1 if on else 0), self._h)

    def _nsys(self):
        return self.info(0).n_systems

    # ------------------------------------------------------------------ compute
    def forces(self, pos_q, step, parts=RBE_PART_ALL, energy=True, phi=False, out=None):
        """Mixed path: pos_q float32 [n,4] -> (F float32 [n,4], E float64 [nsys,4] or None,
        phi float32 [n] or None)."""
        torch = _torch()
        n = pos_q.shape[0]
        _need(pos_q, torch.float32, 4, n, "pos_q")
        F = out if out is not None else torch.empty((n, 4), dtype=torch.float32, device=pos_q.device)
        E = torch.empty((self._nsys(), 4), dtype=torch.float64, device=pos_q.device) if energy else None
        ph = torch.empty(n, dtype=torch.float32, device=pos_q.device) if phi else None
        self._stream()
        capi.check(self.lib.rbe_forces_ex(self._h, n, _ptr(pos_q), step, parts, _ptr(F), _ptr(E),
                                          _ptr(ph)), self._h)
        return F, E, ph

    def forces_f64(self, pos_q, step, parts=RBE_PART_ALL, energy=True, phi=False):
        """FP64 path: pos_q float64 [n,4] -> (F float64 [n,4], E [nsys,4], phi float64 [n])."""
        torch = _torch()
        n = pos_q.shape[0]
        _need(pos_q, torch.float64, 4, n, "pos_q")
        F = torch.empty((n, 4), dtype=torch.float64, device=pos_q.device)
        E = torch.empty((self._nsys(), 4), dtype=torch.float64, device=pos_q.device) if energy else None
        ph = torch.empty(n, dtype=torch.float64, device=pos_q.device) if phi else None
        self._stream()
        capi.check(self.lib.rbe_forces_f64(self._h, n, _ptr(pos_q), step, parts, _ptr(F), _ptr(E),
                                           _ptr(ph)), self._h)
        return F, E, ph

    def step(self, pos_q, vel, nsteps, step_dev, F_out=None):
        """nsteps MD steps in place (mixed: float32, FP64: float64 tensors [n,4]);
        step_dev: int64 CUDA tensor of one element holding the next step index.
        F_out (mixed only, float32 [n,4]): receives each step's total force
        (``rbe_step_ex``); after the call, the last step's."""
        torch = _torch()
        n = pos_q.shape[0]
        if step_dev.dtype != torch.int64 or not step_dev.is_cuda or step_dev.numel() != 1:
            raise ValueError("step_dev must be a one-element int64 CUDA tensor")
        self._stream()
        if pos_q.dtype == torch.float32:
            _need(pos_q, torch.float32, 4, n, "pos_q"); _need(vel, torch.float32, 4, n, "vel")
            if F_out is not None:
                _need(F_out, torch.float32, 4, n, "F_out")
                capi.check(self.lib.rbe_step_ex(self._h, n, _ptr(pos_q), _ptr(vel), nsteps,
                                                _ptr(step_dev), _ptr(F_out)), self._h)
                return
            capi.check(self.lib.rbe_step(self._h, n, _ptr(pos_q), _ptr(vel), nsteps,
                                         _ptr(step_dev)), self._h)
        else:
            _need(pos_q, torch.float64, 4, n, "pos_q"); _need(vel, torch.float64, 4, n, "vel")
            capi.check(self.lib.rbe_step_f64(self._h, n, _ptr(pos_q), _ptr(vel), nsteps,
                                             _ptr(step_dev)), self._h)

    def forces_host(self, pos_q, step, F_out, E_out=None):
        """Host-buffer variant: pos_q, F_out float32 CPU tensors [n,4] (pinned preferred)."""
        n = pos_q.shape[0]
        capi.check(self.lib.rbe_forces_host(self._h, n, _ptr(pos_q), step, _ptr(F_out),
                                            _ptr(E_out)), self._h)

    def step_host(self, pos_q, vel, nsteps, step0):
        n = pos_q.shape[0]
        capi.check(self.lib.rbe_step_host(self._h, n, _ptr(pos_q), _ptr(vel), nsteps, step0),
                   self._h)


class RBE(_HandleBase):
    """One periodic system of up to n_max particles."""

    def __init__(self, params: capi.rbe_params):
        super().__init__()
        capi.check(self.lib.rbe_create(ctypes.byref(params), ctypes.byref(self._h)))
        self.params = params


class RBEBatch(_HandleBase):
    """Independent systems evaluated together; arrays are concatenated in order."""

    def __init__(self, params_list, n_list):
        super().__init__()
        arr = (capi.rbe_params * len(params_list))(*params_list)
        ns = (ctypes.c_int32 * len(n_list))(*[int(n) for n in n_list])
        capi.check(self.lib.rbe_create_batch(arr, ns, len(params_list), ctypes.byref(self._h)))
        self.params = list(params_list)
        self.n_list = [int(n) for n in n_list]


def probe_peaks() -> dict:
    """Measured special-function (sin/cos) and FP32-FMA throughput per SM per
    clock on the current device, the SM clock during the probe and the SM
    count (``rbe_probe_peaks``)."""
    lib = capi.load()
    out = capi.rbe_peaks()
    capi.check(lib.rbe_probe_peaks(ctypes.byref(out)))
    return {"sfu_per_clk_sm": out.sfu_per_clk_sm, "ffma_per_clk_sm": out.ffma_per_clk_sm,
            "sm_clock_mhz": out.sm_clock_mhz, "sms": out.sms}


class RBEEnergy:
    """autograd.Function: E(positions, charges) for a frozen k-batch (step).

    ``RBEEnergy.apply(pos, q, rbe, step)`` with pos float32 [n,3] and q float32
    [n] (CUDA) returns the FP64 energy of the mixed path (scalar tensor for a
    single system).  backward gives dE/dpos = -F and dE/dq = phi, recomputing
    rho(k) for the same k-batch instead of storing per-pair phases.
    """

    _fn = None

    @classmethod
    def apply(cls, pos, q, rbe, step):
        if cls._fn is None:
            cls._fn = _make_energy_fn()
        return cls._fn.apply(pos, q, rbe, step)


def _make_energy_fn():
    torch = _torch()

    class _Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, pos, q, rbe, step):
            pos_q = torch.cat([pos.detach().float(), q.detach().float()[:, None]], 1).contiguous()
            _, E, _ = rbe.forces(pos_q, step, energy=True, phi=False)
            ctx.rbe = rbe
            ctx.step = step
            ctx.save_for_backward(pos, q)
            return E[:, 0].sum() if E.shape[0] > 1 else E[0, 0]

        @staticmethod
        def backward(ctx, gE):
            pos, q = ctx.saved_tensors
            pos_q = torch.cat([pos.detach().float(), q.detach().float()[:, None]], 1).contiguous()
            F, _, phi = ctx.rbe.forces(pos_q, ctx.step, energy=False, phi=True)
            g = gE.to(torch.float32)
            gpos = (-F[:, :3] * g).to(pos.dtype) if ctx.needs_input_grad[0] else None
            gq = (phi * g).to(q.dtype) if ctx.needs_input_grad[1] else None
            return gpos, gq, None, None

    return _Fn

"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances:
  * sampling tables and k-samples: bit-exact (integer work);
  * FP64 GPU path: relative RMS <= 1e-12 per force part, energies <= 1e-12
    relative to the sum of the magnitudes of the parts;
  * mixed path: relative RMS <= 1e-5 per part (Fourier, real-space Coulomb,
    LJ) and for the total force, dE/dq <= 1e-5, energies <= 1e-6.
"""
import copy

import numpy as np
import pytest

import oracle
from gpu_util import assert_per_particle, energy_rel, need_gpu, oracle_eval, rel_rms
from paper_2010_01559_gb300 import workloads

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-12
TOL_MIXED = 1e-5
TOL_E_MIXED = 1e-6


@pytest.fixture(scope="module")
def rbe():
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_01559_gb300 as rbe
    return rbe


def _handle(rbe, wl, n_max=None, path="list"):
    """path "list": mixed forces over the neighbour list (the default);
    "cells": the per-call cell scan (skin < 0 turns the list off)."""
    p = wl.params
    if path == "cells":
        p = copy.copy(p)
        p.skin = -1.0
    return rbe.RBE(rbe.params_from(p, n_max=wl.n if n_max is None else n_max))


def _dev(wl, dtype="float32"):
    import torch
    t = torch.from_numpy(wl.pos_q()).cuda()
    return t.double().contiguous() if dtype == "float64" else t


@pytest.fixture(scope="module")
def c1():
    return workloads.config_small_fp64()


@pytest.fixture(scope="module")
def c2():
    return workloads.config_2to1_mixed()


# ------------------------------------------------------------------ sampling
@pytest.mark.parametrize("alpha,L", [(0.3, 25.0), (0.2, 54.288), (0.1, 66.9), (0.3, 253.98),
                                     (0.30273, 100.8), (0.55, 10.0)])
def test_table_bit_exact(rbe, alpha, L):
    h = rbe.RBE(rbe.capi.make_params(box=L, alpha=alpha, r_c=L / 3.5, P=10, n_max=16))
    M, T, H = oracle.axis_table(alpha, L)
    inf = h.info()
    assert inf.M == M
    assert np.array_equal(h.table(), T)
    assert inf.H == H
    assert abs(inf.S - (H ** 3 - 1)) <= 1e-15 * inf.S


def test_k_samples_bit_exact_many_steps(rbe, c1):
    p = c1.params
    h = _handle(rbe, c1)
    for step in list(range(100)) + [2 ** 32 + 5, 123456789]:
        m = h.sample_k(step).cpu().numpy()
        ref, att, bad = oracle.sample_k(p.alpha, p.box, p.seed, p.stream, step, p.P)
        assert bad == 0
        assert np.array_equal(m[:, :3], ref), step
        assert np.array_equal(m[:, 3], att), step


def test_k_samples_bit_exact_large_box(rbe):
    h = rbe.RBE(rbe.capi.make_params(box=253.98, alpha=0.3, r_c=5.0, P=500, seed=5, n_max=16))
    for step in range(0, 100, 7):
        m = h.sample_k(step).cpu().numpy()
        ref, att, _ = oracle.sample_k(0.3, 253.98, 5, 0, step, 500)
        assert np.array_equal(m[:, :3], ref)
        assert np.array_equal(m[:, 3], att)


def test_k_samples_inside_force_pass_match(rbe, c1):
    """The structure-factor kernel draws its own k-batch; it must be the same."""
    import torch
    h = _handle(rbe, c1)
    x = _dev(c1)
    for step in (0, 17):
        h.forces(x, step)
        torch.cuda.synchronize()
        ref = oracle.sample_k(c1.params.alpha, c1.params.box, c1.params.seed, 0, step, c1.params.P)[0]
        assert np.array_equal(h.sample_k(step).cpu().numpy()[:, :3], ref)


# ------------------------------------------------------------------ FP64 path
def test_fp64_path_matches_oracle_per_part(rbe, c1):
    h = _handle(rbe, c1)
    x = _dev(c1, "float64")
    step = 4
    ref = oracle_eval(c1, step, want_phi=True)
    parts = {1: ref["F_fourier"], 2: ref["F_real"], 4: ref["F_lj"], 7: ref["F"]}
    for mask, Fref in parts.items():
        F, E, phi = h.forces_f64(x, step, parts=mask, phi=True)
        assert rel_rms(F[:, :3].cpu().numpy(), Fref) <= TOL_F64, mask
        assert F[:, 3].abs().max().item() == 0.0
    E = E.cpu().numpy()[0]
    assert energy_rel(E, ref["E"]) <= TOL_F64
    for k in range(1, 4):
        assert abs(E[k] - ref["E"][k]) <= TOL_F64 * np.abs(ref["E"][1:]).sum()
    assert rel_rms(phi.cpu().numpy(), ref["phi"]) <= TOL_F64


def test_one_cell_box_all_pairs_match_oracle(rbe):
    """r_c > L/3 (the paper's electrolyte: r_c = 4, L = 10): the box is one cell
    and every pair is met once as the minimum image, on both paths."""
    wl = workloads.config_electrolyte_dh()
    assert wl.params.box / wl.params.r_c < 3
    h = _handle(rbe, wl)
    step = 2
    ref = oracle_eval(wl, step, want_phi=True)
    F64, E64, phi64 = h.forces_f64(_dev(wl, "float64"), step, phi=True)
    assert rel_rms(F64[:, :3].cpu().numpy(), ref["F"]) <= TOL_F64
    assert energy_rel(E64.cpu().numpy()[0], ref["E"]) <= TOL_F64
    assert rel_rms(phi64.cpu().numpy(), ref["phi"]) <= TOL_F64
    F, E, phi = h.forces(_dev(wl), step, phi=True)          # over the neighbour list
    assert rel_rms(F[:, :3].cpu().numpy(), ref["F"]) <= TOL_MIXED
    assert_per_particle(F[:, :3].cpu().numpy(), ref["F"], "one cell, list")
    assert energy_rel(E.cpu().numpy()[0], ref["E"]) <= TOL_E_MIXED
    assert rel_rms(phi.cpu().numpy(), ref["phi"]) <= TOL_MIXED
    hc = _handle(rbe, wl, path="cells")
    for R in (1, 3, 9):                                      # the cell scan's lane splits
        hc.set_tuning(0, 0, R, 0)
        F, E, phi = hc.forces(_dev(wl), step, phi=True)
        assert rel_rms(F[:, :3].cpu().numpy(), ref["F"]) <= TOL_MIXED, R
        assert energy_rel(E.cpu().numpy()[0], ref["E"]) <= TOL_E_MIXED, R
        assert rel_rms(phi.cpu().numpy(), ref["phi"]) <= TOL_MIXED, R
        assert_per_particle(F[:, :3].cpu().numpy(), ref["F"], ("F", R))
        assert_per_particle(phi.cpu().numpy(), ref["phi"], ("phi", R))


# ------------------------------------------------------------------ mixed path
@pytest.mark.parametrize("path", ["list", "cells"])
@pytest.mark.parametrize("cfg", ["c1", "c2"])
def test_mixed_path_matches_oracle_per_part(rbe, cfg, path, request):
    wl = request.getfixturevalue(cfg)
    h = _handle(rbe, wl, path=path)
    x = _dev(wl)
    step = 11
    ref = oracle_eval(wl, step, want_phi=True)
    errs = {}
    for mask, name in ((1, "F_fourier"), (2, "F_real"), (4, "F_lj"), (7, "F")):
        F, E, phi = h.forces(x, step, parts=mask, phi=True)
        errs[name] = rel_rms(F[:, :3].cpu().numpy(), ref[name])
        assert_per_particle(F[:, :3].cpu().numpy(), ref[name], (cfg, path, name))
    print(cfg, errs)
    for name, e in errs.items():
        assert e <= TOL_MIXED, (name, e)
    E = E.cpu().numpy()[0]
    assert energy_rel(E, ref["E"]) <= TOL_E_MIXED
    assert rel_rms(phi.cpu().numpy(), ref["phi"]) <= TOL_MIXED
    assert_per_particle(phi.cpu().numpy(), ref["phi"], (cfg, path, "phi"))


def test_mixed_vs_fp64_gpu(rbe, c2):
    h = _handle(rbe, c2)
    F, E, _ = h.forces(_dev(c2), 3)
    F64, E64, _ = h.forces_f64(_dev(c2, "float64"), 3)
    assert rel_rms(F[:, :3].cpu().numpy(), F64[:, :3].cpu().numpy()) <= TOL_MIXED
    assert_per_particle(F[:, :3].cpu().numpy(), F64[:, :3].cpu().numpy(), "mixed vs FP64")
    assert abs(E[0, 0].item() - E64[0, 0].item()) <= TOL_E_MIXED * E64[0, 1:].abs().sum().item()


def test_water_like_no_lj_fp32_charges(rbe):
    wl = workloads.config_water(1500)
    h = _handle(rbe, wl)
    ref = oracle_eval(wl, 2, want_phi=True)
    F, E, phi = h.forces(_dev(wl), 2, phi=True)
    assert rel_rms(F[:, :3].cpu().numpy(), ref["F"]) <= TOL_MIXED
    assert rel_rms(phi.cpu().numpy(), ref["phi"]) <= TOL_MIXED
    assert_per_particle(F[:, :3].cpu().numpy(), ref["F"], "water F")
    assert_per_particle(phi.cpu().numpy(), ref["phi"], "water phi")
    F64, E64, phi64 = h.forces_f64(_dev(wl, "float64"), 2, phi=True)
    assert rel_rms(F64[:, :3].cpu().numpy(), ref["F"]) <= TOL_F64
    assert energy_rel(E64.cpu().numpy()[0], ref["E"]) <= TOL_F64


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("n,P", [(1, 1), (2, 3), (37, 129), (1000 + 37, 100), (513, 257)])
def test_ragged_sizes(rbe, n, P):
    sp = workloads.SystemParams(box=25.0, alpha=0.3, r_c=5.0, P=P, seed=9)
    wl = workloads.electrolyte(f"ragged{n}", n - n // 2, n // 2, 1.0, -1.0, sp)
    h = _handle(rbe, wl, n_max=wl.n + 50)
    ref = oracle_eval(wl, 1)
    F, E, _ = h.forces(_dev(wl), 1)
    F64, E64, _ = h.forces_f64(_dev(wl, "float64"), 1)
    assert rel_rms(F[:, :3].cpu().numpy(), ref["F"]) <= TOL_MIXED
    assert_per_particle(F[:, :3].cpu().numpy(), ref["F"], (n, P))
    assert rel_rms(F64[:, :3].cpu().numpy(), ref["F"]) <= TOL_F64
    assert energy_rel(E64.cpu().numpy()[0], ref["E"]) <= TOL_F64


def test_empty_input(rbe, c1):
    import torch
    h = _handle(rbe, c1)
    x = torch.empty((0, 4), dtype=torch.float32, device="cuda")
    F, E, _ = h.forces(x, 0)
    h.sync()
    assert F.shape == (0, 4)
    assert np.allclose(E.cpu().numpy(), 0.0)


def test_positions_outside_box_are_wrapped(rbe, c1):
    """Inputs shifted by whole box lengths: the float32 input itself is rounded
    differently, so compare with the oracle on the wrapped shifted values."""
    import torch
    h = _handle(rbe, c1)
    x = _dev(c1)
    shift = torch.tensor([25.0 * 3, -25.0 * 2, 25.0], device="cuda")
    y = x.clone()
    y[:, :3] += shift
    F1, E1, _ = h.forces(y, 5)
    wrapped = np.mod(y[:, :3].cpu().numpy().astype(np.float64), 25.0)
    ref = oracle_eval(c1, 5, pos=wrapped)
    assert rel_rms(F1[:, :3].cpu().numpy(), ref["F"]) <= TOL_MIXED
    assert_per_particle(F1[:, :3].cpu().numpy(), ref["F"], "wrapped")
    x64 = _dev(c1, "float64")
    y64 = x64.clone()
    y64[:, :3] += shift.double()
    G0, _, _ = h.forces_f64(x64, 5)
    G1, _, _ = h.forces_f64(y64, 5)
    assert rel_rms(G1[:, :3].cpu().numpy(), G0[:, :3].cpu().numpy()) <= 1e-11


def test_whole_box_shifts_give_the_same_fixed_point_records(rbe):
    """L = 16 and positions on a 2^-12 grid, so that x + 16 m is exact in
    float32 for |m| <= 128: the fixed-point fraction round(2^32 x / L) mod 2^32
    is then the same for every shift, and so is every force to the last bit
    (both real-space paths).  The shifts take 2^32 x / L through
    [-2^39, 2^39]: the modulo-2^32 reduction, negative inputs, and x = L/2,
    whose product 2^31 is the one value that converts through the tie."""
    import torch
    wl = workloads.electrolyte_1to1(256, 0.0625, 0.5, 5.0, 64, seed=11)
    assert abs(wl.params.box - 16.0) < 1e-9
    wl.params.box = 16.0
    wl.pos = (np.floor(wl.pos.astype(np.float64) * 4096.0) / 4096.0).astype(np.float32)
    wl.pos[0, 0] = np.float32(8.0)
    for path in ("list", "cells"):
        h = _handle(rbe, wl, path=path)
        x = _dev(wl)
        F0, E0, _ = h.forces(x, 3)
        for m in [(1, 0, 0), (-1, 2, -3), (100, -127, 64), (-128, 127, 1), (0, 0, -1)]:
            sh = torch.tensor(m, dtype=torch.float32, device="cuda") * 16.0
            y = x.clone()
            y[:, :3] += sh
            back = y[:, :3].double() - sh.double()
            assert torch.equal(back, x[:, :3].double()), m          # the shift is exact
            F1, E1, _ = h.forces(y, 3)
            assert torch.equal(F1, F0), (path, m)
            assert torch.equal(E1, E0), (path, m)
        ref = oracle_eval(wl, 3)
        assert rel_rms(F0[:, :3].cpu().numpy(), ref["F"]) <= TOL_MIXED
        h.close()


def test_non_neutral_charges_background(rbe):
    wl = workloads.electrolyte_1to1(600, 0.064, 0.3, 5.0, 64, seed=3)
    wl.q[:7] = np.float32(0.5)            # sum q != 0
    h = _handle(rbe, wl)
    ref = oracle_eval(wl, 2, want_phi=True)
    F64, E64, phi64 = h.forces_f64(_dev(wl, "float64"), 2, phi=True)
    assert energy_rel(E64.cpu().numpy()[0], ref["E"]) <= TOL_F64
    assert rel_rms(phi64.cpu().numpy(), ref["phi"]) <= TOL_F64


def test_smallest_cell_grid(rbe):
    """Three cells per edge: every neighbour cell distinct, nothing counted twice."""
    wl = workloads.electrolyte_1to1(300, 0.3, 0.9, 3.0, 40, seed=1, lj_eps=1.0, lj_sigma=0.5,
                                    lj_rcut=0.5 * 2 ** (1 / 6))
    assert wl.params.box / wl.params.r_c < 4
    h = _handle(rbe, wl)
    assert h.info().n_cells_dim == 3
    ref = oracle_eval(wl, 0)
    F64, E64, _ = h.forces_f64(_dev(wl, "float64"), 0)
    assert rel_rms(F64[:, :3].cpu().numpy(), ref["F"]) <= TOL_F64
    assert energy_rel(E64.cpu().numpy()[0], ref["E"]) <= TOL_F64


def test_deterministic_bitwise(rbe, c2):
    h = _handle(rbe, c2)
    x = _dev(c2)
    a = h.forces(x, 8, phi=True)
    b = h.forces(x, 8, phi=True)
    for u, v in zip(a, b):
        assert (u == v).all()


def test_tuning_does_not_change_results_beyond_rounding(rbe, c2):
    h = _handle(rbe, c2)
    x = _dev(c2)
    ref = oracle_eval(c2, 6)
    for chunk, split, rsplit in ((32, 1, 1), (256, 2, 3), (4096, 8, 9), (64, 4, 3),
                                 (0, 0, 0)):
        h.set_tuning(chunk, split, rsplit)
        F, E, phi = h.forces(x, 6, phi=True)
        assert rel_rms(F[:, :3].cpu().numpy(), ref["F"]) <= TOL_MIXED, (chunk, split, rsplit)
        assert_per_particle(F[:, :3].cpu().numpy(), ref["F"], (chunk, split, rsplit))
        assert energy_rel(E.cpu().numpy()[0], ref["E"]) <= TOL_E_MIXED
        if chunk:
            assert h.get_tuning()[:3] == (chunk, split, rsplit)
    for ls in (1, 2, 4, 8):                # lanes per particle of the list pass
        h.set_tuning(128, 2, 3, 0, ls)
        F, E, _ = h.forces(x, 6)
        assert rel_rms(F[:, :3].cpu().numpy(), ref["F"]) <= TOL_MIXED, ls
        assert_per_particle(F[:, :3].cpu().numpy(), ref["F"], ("list_split", ls))
        assert energy_rel(E.cpu().numpy()[0], ref["E"]) <= TOL_E_MIXED
        assert h.get_tuning()[4] == ls
    hc = _handle(rbe, c2, path="cells")
    for seg in (1, 2, 8):                  # segment lengths of the cell scan
        hc.set_tuning(128, 2, 3, seg)
        F, E, _ = hc.forces(x, 6)
        assert rel_rms(F[:, :3].cpu().numpy(), ref["F"]) <= TOL_MIXED, seg
        assert_per_particle(F[:, :3].cpu().numpy(), ref["F"], ("seg", seg))
        assert energy_rel(E.cpu().numpy()[0], ref["E"]) <= TOL_E_MIXED
        assert hc.get_tuning()[3] == seg
    hc.close()
    c, s, r, sg, ls = h.autotune(x)
    assert c >= 32 and s in (1, 2, 4, 8) and r in (1, 3, 9) and sg >= 1
    assert h.get_tuning() == (c, s, r, sg, ls)

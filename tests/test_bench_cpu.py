"""Host-side bookkeeping of bench.py, on CPU: the algorithmic work the
roofline keys divide by, the choice of the dominant kernel, the neighbour-list
skin and pair counts behind the real-space figure, and the lookup of committed
DRAM traffic (valid only for the kernel sources it was taken on)."""
import importlib.util
import json
import os
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _wl(n, P, name="synthetic", **kw):
    params = types.SimpleNamespace(P=P, **kw)
    return types.SimpleNamespace(n=n, params=params, name=name)


def test_fourier_rooflines_count_two_sfu_ops_for_rho_and_one_for_the_polar_force(bench):
    wl = _wl(1000, 200)
    units = {"sfu": 5.0, "alu": 38.0, "sfu_basis": "", "alu_basis": ""}
    # 10 launches each: rho 2 ms in all (0.2 ms a launch), force 1 ms (0.1 ms)
    prof = {"rho": (2.0, 10), "fourier_force": (1.0, 10)}
    r = bench.fourier_rooflines(prof, wl, units)
    assert r["rho"]["achieved"] == pytest.approx(2 * 1000 * 200 / 2e-4 / 1e12)
    assert r["fourier_force"]["achieved"] == pytest.approx(1000 * 200 / 1e-4 / 1e12)
    assert r["rho"]["frac"] == pytest.approx(r["rho"]["achieved"] / 5.0)
    assert r["rho"]["avg_launch_us"] == pytest.approx(200.0)
    assert r["rho"]["traffic"] is None                  # no counters for this workload


def test_roofline_takes_the_dominant_kernel_with_its_own_bound(bench):
    wl = _wl(4096, 100)
    units = {"sfu": 5.0, "alu": 38.0, "sfu_basis": "sfu", "alu_basis": "alu"}
    peaks = {"hbm_gbs": 7000.0}
    r = bench.roofline({"prep": (0.5, 10), "rho": (3.0, 10), "real": (1.0, 10)}, wl, peaks,
                       units)
    assert r["kernel"] == "rho" and r["unit"] == "Tsfu/s"
    assert r["achieved"] == pytest.approx(2 * 4096 * 100 / 3e-4 / 1e12)
    r = bench.roofline({"fourier_force": (3.0, 10), "rho": (1.0, 10)}, wl, peaks, units)
    assert r["kernel"] == "fourier_force"
    assert r["achieved"] == pytest.approx(4096 * 100 / 3e-4 / 1e12)
    assert r["algorithmic"].startswith("1 SFU op per")
    cand, pairs = 50_000, 30_000
    r = bench.roofline({"real": (2.0, 10)}, wl, peaks, units, counts=(cand, pairs))
    ops = bench.REAL_OPS_PER_CANDIDATE * cand + bench.REAL_OPS_PER_PAIR * pairs
    assert r["bound"] == "alu" and r["achieved"] == pytest.approx(ops / 2e-4 / 1e12)
    r = bench.roofline({"prep": (1.0, 10)}, wl, peaks, units)
    assert r["bound"] == "hbm" and r["frac"] == pytest.approx(r["achieved"] / 7000.0)
    assert r["achieved"] == pytest.approx(40 * 4096 / 1e-4 / 1e9)


def test_list_skin_follows_the_library_rule(bench):
    p = types.SimpleNamespace(box=54.29, r_c=6.0, skin=0.0)
    assert bench.list_skin(p) == pytest.approx(0.6)             # 0.1 r_c by default
    p.skin = 2.0
    assert bench.list_skin(p) == pytest.approx(2.0)             # as given, below the cap
    p = types.SimpleNamespace(box=18.0, r_c=5.5, skin=0.0)
    assert bench.list_skin(p) == pytest.approx(0.5)             # cap L/3 - r_c
    p = types.SimpleNamespace(box=13.0, r_c=6.0, skin=0.0)
    assert bench.list_skin(p) == pytest.approx(0.5)             # one cell: L/2 - r_c
    p = types.SimpleNamespace(box=12.0, r_c=6.0, skin=0.0)
    assert bench.list_skin(p) == 0.0


def test_pair_counts_equal_brute_force_minimum_image(bench):
    rng = np.random.default_rng(3)
    n, L, rc = 300, 14.0, 3.0
    pos = rng.uniform(0.0, L, (n, 3))
    wl = types.SimpleNamespace(n=n, pos=pos, params=types.SimpleNamespace(box=L, r_c=rc, skin=0.0))
    d = pos[:, None, :] - pos[None, :, :]
    d -= L * np.round(d / L)
    r = np.sqrt((d * d).sum(-1))
    np.fill_diagonal(r, np.inf)
    skin = bench.list_skin(wl.params)
    assert bench.pair_counts(wl) == (int((r < rc + skin).sum()), int((r < rc).sum()))


def test_traffic_lookup_needs_the_sources_it_was_taken_on(bench, tmp_path, monkeypatch):
    db = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    for kernel, per in db.items():
        for wname, e in per.items():
            got = bench.traffic_for(kernel, wname)
            src = os.path.join(ROOT, "paper_2010_01559_gb300", "csrc", e["source"])
            if bench.source_hash(src) == e["source_sha256_16"]:
                assert got == e["dram_bytes_per_launch"], (kernel, wname)
            else:
                assert got is None, (kernel, wname)
    # a counter taken on other sources is never reported
    fake = {"rho": {"w": {"source": "rbe_fourier.cu", "source_sha256_16": "0" * 16,
                          "dram_bytes_per_launch": 1}}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(fake))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("rho", "w") is None
    assert bench.traffic_for("rho", "other") is None


def test_roofline_of_the_fused_launch_counts_the_structure_factors(bench):
    """The fused structure-factor + list-pass launch as the dominant kernel: its
    algorithmic work is the structure factors' two SFU operations per pair."""
    wl = _wl(8192, 500)
    units = {"sfu": 5.0, "alu": 38.0, "sfu_basis": "sfu", "alu_basis": "alu"}
    r = bench.roofline({"rho_list": (3.2, 10), "fourier_force": (2.0, 10), "prep": (0.3, 10)},
                       wl, {}, units)
    assert r["kernel"] == "rho_list" and r["unit"] == "Tsfu/s"
    assert r["achieved"] == pytest.approx(2 * 8192 * 500 / 3.2e-4 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 5.0)
    assert r["algorithmic"].startswith("2 SFU ops per") and "list" in r["algorithmic"]


def test_source_hash_follows_the_include_chain(bench, tmp_path):
    """A kernel file's counters go stale with a header it reaches through
    #include (directly or through another header), not with one it does not
    include; an include cycle is walked once."""
    d = tmp_path / "csrc"
    d.mkdir()
    (d / "k.cu").write_text('#include "a.cuh"\n__global__ void k() {}\n')
    (d / "a.cuh").write_text('#pragma once\n#include "b.cuh"\n')
    (d / "b.cuh").write_text('#pragma once\n#include "a.cuh"\nconstexpr int kB = 1;\n')
    (d / "other.cuh").write_text('constexpr int kO = 1;\n')
    files = []
    bench._local_includes(str(d / "k.cu"), files)
    assert [os.path.basename(f) for f in files] == ["k.cu", "a.cuh", "b.cuh"]
    h0 = bench.source_hash(str(d / "k.cu"))
    (d / "other.cuh").write_text('constexpr int kO = 2;\n')
    assert bench.source_hash(str(d / "k.cu")) == h0
    (d / "b.cuh").write_text('#pragma once\n#include "a.cuh"\nconstexpr int kB = 2;\n')
    assert bench.source_hash(str(d / "k.cu")) != h0

"""Batched replicas: independent systems of uneven N evaluated by the same
launches (one work table over all replicas).

* every replica's k-batch is bit-exact with the oracle (its own Philox stream);
* the smallest, median and largest replica match the oracle (forces for a
  subset of particles where the oracle's all-pairs real space is too slow);
* a replica inside the batch gives bitwise the same forces as the replica on
  its own handle with the same launch shapes;
* MD steps on the batch advance every replica.
"""
import numpy as np
import pytest

import oracle
from gpu_util import assert_per_particle, energy_rel, need_gpu, oracle_eval, rel_rms
from paper_2010_01559_gb300 import workloads

pytestmark = pytest.mark.gpu
TOL_MIXED = 1e-5


@pytest.fixture(scope="module")
def rbe():
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_01559_gb300 as rbe
    return rbe


@pytest.fixture(scope="module")
def replicas():
    return workloads.config_replicas()


def _concat(wls):
    import torch
    return torch.from_numpy(np.concatenate([w.pos_q() for w in wls])).cuda()


def test_replica_k_samples_bit_exact(rbe, replicas):
    h = rbe.RBEBatch([rbe.params_from(w.params) for w in replicas], [w.n for w in replicas])
    for step in (0, 5, 77):
        m = h.sample_k(step).cpu().numpy()
        off = 0
        for r, w in enumerate(replicas):
            p = w.params
            ref, att, _ = oracle.sample_k(p.alpha, p.box, p.seed, p.stream, step, p.P)
            assert p.stream == r
            assert np.array_equal(m[off:off + p.P, :3], ref), (step, r)
            assert np.array_equal(m[off:off + p.P, 3], att)
            off += p.P


def test_batch_matches_oracle_smallest_median_largest(rbe, replicas):
    h = rbe.RBEBatch([rbe.params_from(w.params) for w in replicas], [w.n for w in replicas])
    x = _concat(replicas)
    step = 9
    F, E, _ = h.forces(x, step)
    F = F.cpu().numpy()
    E = E.cpu().numpy()
    ns = np.array([w.n for w in replicas])
    offs = np.concatenate([[0], np.cumsum(ns)])
    order = np.argsort(ns)
    for r in (order[0], order[len(order) // 2], order[-1]):
        w = replicas[r]
        sub = None if w.n <= 4000 else np.linspace(0, w.n - 1, 512).astype(int)
        ref = oracle_eval(w, step, sub=sub)
        Fr = F[offs[r]:offs[r + 1], :3]
        if sub is not None:
            Fr = Fr[sub]
        err = rel_rms(Fr, ref["F"])
        print("replica", r, "N", w.n, "rel-RMS", err)
        assert err <= TOL_MIXED, (r, w.n, err)
        assert_per_particle(Fr, ref["F"], ("replica", r))
        if sub is None:
            assert energy_rel(E[r], ref["E"]) <= 1e-6


def test_replica_in_batch_equals_single_handle(rbe, replicas):
    import torch
    few = replicas[:6]
    h = rbe.RBEBatch([rbe.params_from(w.params) for w in few], [w.n for w in few])
    h.set_tuning(512, 2, 3)
    Fb, Eb, _ = h.forces(_concat(few), 4)
    off = 0
    for r, w in enumerate(few):
        s = rbe.RBE(rbe.params_from(w.params, n_max=w.n))
        s.set_tuning(512, 2, 3)
        Fs, Es, _ = s.forces(torch.from_numpy(w.pos_q()).cuda(), 4)
        assert torch.equal(Fb[off:off + w.n], Fs), r
        assert torch.equal(Eb[r], Es[0]), r
        off += w.n
        s.close()


def test_batch_md_steps(rbe, replicas):
    import torch
    few = replicas[:8]
    h = rbe.RBEBatch([rbe.params_from(w.params) for w in few], [w.n for w in few])
    h.set_graph(True)
    pos = _concat(few)
    vel = torch.zeros_like(pos)
    vel[:, :3] = torch.from_numpy(np.concatenate([w.vel for w in few])).cuda()
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    p0 = pos.clone()
    h.step(pos, vel, 50, step)
    h.sync()
    assert step.item() == 50
    assert torch.isfinite(pos).all() and torch.isfinite(vel).all()
    moved = (pos[:, :3] - p0[:, :3]).abs().amax(1)
    assert (moved > 0).all()
    assert torch.equal(pos[:, 3], p0[:, 3])


def test_batch_rejects_wrong_total(rbe, replicas):
    import torch
    few = replicas[:3]
    h = rbe.RBEBatch([rbe.params_from(w.params) for w in few], [w.n for w in few])
    x = _concat(few)[:-1].contiguous()
    with pytest.raises(rbe.RBEError, match="total"):
        h.forces(x, 0)

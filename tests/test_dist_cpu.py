"""Multi-rank bookkeeping of bench.py on CPU (gloo, world size 2): every rank
steps its own replica on its own Philox stream, throughput = particles of all
ranks x steps / the slowest rank's time, and the reference arm runs on rank 0
only.  No GPU: the ranks exchange only the timing scalars."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import importlib.util
    import torch
    import torch.distributed as dist
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    w, r, _ = bench.dist_setup("gloo")
    dev = torch.device("cpu")
    # rank r: 1000 + 10 r particles, 2 + r seconds for 50 steps
    agg = bench.combine_ranks(w, 2.0 + r, 1000 + 10 * r, 50, dev)
    stream = bench.replica_stream(7, r)
    bench.barrier(w)

    class A:
        steps, warmup = 1, 0
    ref = bench.run_reference(A()) if r != 0 else "rank0-skipped"
    q.put((r, agg, stream, ref))
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_and_shard():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda t: t[0])
    for r, agg, stream, ref in res:
        assert agg["seconds"] == pytest.approx(3.0)          # the slowest rank
        assert agg["particles"] == pytest.approx(2010.0)     # both replicas
        assert agg["value"] == pytest.approx(2010.0 * 50 / 3.0)
        assert stream == 7 + r                               # one Philox stream per replica
    assert res[1][3] is None                                 # reference arm: rank 0 only

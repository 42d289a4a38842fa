"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The weak-scaling runs shard independent columns over ranks with no data-path
collective: each rank draws its own columns (rank-dependent seed) and the job
aggregates are the maximum of the ranks' times and the sum of their work.
"""
import importlib.util
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        bench = _bench()
        import workloads as W
        # aggregates: times -> max over ranks, work -> sum
        mx, sm = bench.reduce_ranks(dist, [10.0 * (rank + 1), rank + 1.0], device="cpu")
        # sharding: each rank's batch columns come from its own seed
        wl = W.config4(n_columns=4, seed=bench.rank_seed(20240624, rank), nz_min=20, nz_max=30)
        sig = torch.tensor([float(sum(c.T.sum() for c in wl.columns))], dtype=torch.float64)
        sigs = [torch.zeros(1, dtype=torch.float64) for _ in range(ws)]
        dist.all_gather(sigs, sig)
        out[rank] = (mx, sm, [float(x) for x in sigs])
    finally:
        dist.destroy_process_group()


def test_weak_scaling_aggregates_and_sharding_over_two_ranks():
    ws = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        mx, sm, sigs = res[rank]
        assert mx == [20.0, 2.0]            # the slowest rank's time
        assert sm == [30.0, 3.0]            # the work of both ranks
        assert sigs[0] != sigs[1]           # distinct columns per rank
    assert res[0][2] == res[1][2]


def test_single_process_aggregates_are_its_own():
    bench = _bench()
    mx, sm = bench.reduce_ranks(None, [3.0, 4.0])
    assert mx == [3.0, 4.0] and sm == [3.0, 4.0]
    assert np.all(np.array([bench.rank_seed(7, r) for r in range(4)]) == np.arange(7, 11))

"""Host-side logic that needs no GPU: argument checks of the batch entry point,
the stability measure over grid symmetries, and the bench's workload tables."""
import ctypes as ct
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_batch_search_argument_checks_without_a_gpu():
    from paper_2411_16431_b300 import build, sgtn
    build.build()
    L = sgtn.load()
    null = ct.POINTER(ct.c_int32)()
    # nothing to run: success, no CUDA call
    assert L.sgtn_batch_search(None, 0, 1.0, 4, 0, 1, 8, 1, None, None, None, None, None, null, 0, null) == 0
    # negative count or threads, or a null output array: SGTN_ERR_ARG before anything runs
    assert L.sgtn_batch_search(None, -1, 1.0, 4, 0, 1, 8, 1, None, None, None, None, None, null, 0, null) == -1
    hs = (ct.c_void_p * 1)(None)
    assert L.sgtn_batch_search(hs, 1, 1.0, 4, 0, 1, 8, 1, None, None, None, None, None, null, 0, null) == -1
    assert L.sgtn_batch_search(None, 0, 1.0, 4, 0, 1, 8, 1, None, None, None, None, None, null, -2, null) == -1


def test_logz_spread():
    from paper_2411_16431_b300.sgtn import logz_spread
    assert logz_spread([(0, 1.0), (1, 3.0), (2, float("nan"))]) == 1.0
    assert math.isnan(logz_spread([(0, 2.0)]))
    assert logz_spread([(k, 5.5) for k in range(8)]) == 0.0


def test_bench_workload_tables():
    sys.path.insert(0, ROOT)
    import bench
    units = bench._batch64(0)
    assert len(units) == 64
    sizes = [u[0].n_spins for u in units]
    assert sorted(set(sizes)) == [96, 216, 384, 600, 864]
    assert all(len(st) == u.rows * u.cols and all(len(x) == 256 for x in st) for u, st in units)
    for name, wl in bench.WORKLOADS.items():
        assert wl.get("precision", bench.DEFAULT_PRECISION) in bench.PRECISIONS, name
        assert wl["chi"] >= 1 and wl["M"] >= 1 and "desc" in wl
    k = bench.WORKLOADS["kings50x50"]["make"](0)
    assert k.denom == 1000 and not np.any(k.h_num)


def _ranks_worker(rank, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2")
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=2)
    ws, r, _ = bench.dist_env()
    t, ev = bench.combine_ranks(100.0 + 50 * rank, 1000 + rank, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((ws, r, t, ev))


def test_replicas_combine_over_two_gloo_ranks():
    """The N > 1 bench path on CPU: two gloo ranks, max of the times, sum of the evaluations."""
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_ranks_worker, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
    assert [r[:2] for r in res] == [(2, 0), (2, 1)]
    assert all(r[2] == 150.0 and r[3] == 2001.0 for r in res)

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

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


def test_hamming_ball_states():
    """Distinct patterns per cell, the reference first, ordered by Hamming distance."""
    from paper_2411_16431_b300 import lattices as L
    inst = L.pegasus_nice(4, 2)
    states = L.hamming_ball_states(inst, 40, seed=5)
    for site, st in enumerate(states):
        assert len(st) == 40 and len(set(st.tolist())) == 40
        dist = [bin(int(x) ^ int(st[0])).count("1") for x in st]
        assert dist[0] == 0 and dist == sorted(dist) and max(dist) <= 2
    pl = L.planted(L.chimera_grid(2, 3, 1), 3)
    ref = L.hamming_ball_states(pl, 5)
    for site, st in enumerate(ref):
        sp = np.nonzero(pl.site_of_spin == site)[0]
        assert int(st[0]) == sum(1 << j for j, g in enumerate(sp) if pl.planted[g] < 0)


def test_grid_transform_keeps_energies():
    """A grid symmetry relabels the cell grid only: the same spin configuration has the
    same energy, every coupling stays between king's-graph neighbours, and the state
    lists of a cell follow it to its new position."""
    from paper_2411_16431_b300 import lattices as L
    inst = L.pegasus_nice(4, 1)
    states = L.hamming_ball_states(inst, 6, seed=2)
    rng = np.random.default_rng(0)
    s = rng.choice([-1, 1], inst.n_spins).astype(np.int8)
    for k in range(8):
        t = L.transform(inst, k)
        assert t.energy_num(s) == inst.energy_num(s)
        r, c = t.site_of_spin // t.cols, t.site_of_spin % t.cols
        assert np.all(np.abs(r[t.ei] - r[t.ej]) <= 1) and np.all(np.abs(c[t.ei] - c[t.ej]) <= 1)
        ts = L.transform_states(inst, states, k)
        for site in range(inst.rows * inst.cols):
            spins = np.nonzero(inst.site_of_spin == site)[0]
            new_site = int(t.site_of_spin[spins[0]])
            assert np.array_equal(ts[new_site], states[site])


def test_bench_roofline_helpers():
    """The bench's roofline entry: the kernel with the most device time, achieved =
    algorithmic flop per launch / time per launch, frac = achieved / peak."""
    sys.path.insert(0, ROOT)
    import bench
    kt = {"cholesky_f64": (500.0, 100, 2e9), "score_f32": (100.0, 10, 5e11), "tc_gemm_3xtf32": (50.0, 5, 1e12),
          "select": (1.0, 10, 0.0)}
    r = bench.roofline_of(kt, list(kt))
    assert r["kernel"] == "cholesky_f64" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - (2e9 / 100) / (5e-3) / 1e12) < 1e-12
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15 and r["traffic"] is None
    assert abs(r["peak"] - bench.FP64_PEAK_GFLOPS / 1e3) < 1e-12
    t = bench.roofline_of(kt, ["tc_gemm_3xtf32"])
    assert t["bound"] == "tensor" and t["peak"] == bench.peak_of("tc_gemm_3xtf32")[0]
    assert bench.peak_of("score_f32")[0] == bench.FP32_PEAK_TFLOPS
    assert bench.roofline_of(kt, ["select"]) is None          # no flop count: no roofline entry

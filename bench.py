"""Benchmark of the hot path: boundary-MPS contraction + branch-and-bound search.

One step = set_beta + contract_boundary + search on one instance resident in
HBM (every kernel of the path); the "_x8" workloads run the instance in all
eight grid symmetries at once (one stream and host thread each, through
sgtn_batch_search), as the paper runs every instance from every corner.  ``value`` = conditional marginals evaluated
per second over the whole job (all ranks); the boundary contraction's
algorithmic TFLOP/s is reported beside it.  Multi-GPU runs are independent
replicas (one instance per rank, different seeds): the method has no data
exchange between instances.

    python bench.py [--gpus N --steps K --warmup W] [--impl native|reference] [--workload NAME]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2411_16431_b300 import lattices as L  # noqa: E402

# Workloads: sizes of the benchmark configurations.  Pegasus cells keep the 256
# states nearest a seeded reference configuration (Hamming ball): the stand-in
# for the local-dimension reduction of Sec. IV (the full 2^24 states per cell
# do not fit).
_PEG_SAMPLE = dict(make=lambda seed: L.pegasus_nice(3, seed),
                   states=lambda inst, seed: L.hamming_ball_states(inst, 32, seed=seed + 1),
                   chi=8, M=64, desc="Pegasus P3 nice 2x2 cells, d=32, chi=8, M=64")
WORKLOADS = {
    "chimera4x4": dict(desc="4x4 grid of K44 cells (128 spins), iid J,h in {+-1..+-7}/7, beta=1, chi=16, M=64",
                       make=lambda seed: L.chimera_grid(4, 4, seed), states=None, beta=1.0, chi=16, M=64, sweeps=2,
                       d=256),
    "pegasus5x5": dict(desc="Pegasus P6 nice, 5x5 cells of 24 spins (600 spins), d=256 states per cell "
                            "(Hamming ball around a seeded reference), iid J,h in {+-1..+-7}/7, beta=1, chi=32, M=256",
                       make=lambda seed: L.pegasus_nice(6, seed),
                       states=lambda inst, seed: L.hamming_ball_states(inst, 256, seed=seed + 1),
                       beta=1.0, chi=32, M=256, sweeps=2, d=256,
                       # the oracle's dense row MPOs cannot hold d=256 cells: its timed sample is a
                       # 2x2-cell Pegasus slice (P3 nice) with 32 states per cell
                       oracle_sample=_PEG_SAMPLE),
    "pegasus5x5_d4096": dict(desc="Pegasus P6 nice, 5x5 cells of 24 spins (600 spins), d=4096 states per cell "
                                  "(Hamming ball around a seeded reference), iid J,h in {+-1..+-7}/7, beta=1, chi=32, "
                                  "M=256",
                             make=lambda seed: L.pegasus_nice(6, seed),
                             states=lambda inst, seed: L.hamming_ball_states(inst, 4096, seed=seed + 1),
                             beta=1.0, chi=32, M=256, sweeps=2, d=4096, oracle_sample=_PEG_SAMPLE),
    "pegasus15x15": dict(desc="Pegasus P16 nice, 15x15 cells of 24 spins (5400 spins), d=256 states per cell "
                              "(Hamming ball around a seeded reference), iid J,h in {+-1..+-7}/7, beta=2, chi=64, "
                              "M=1024",
                         make=lambda seed: L.pegasus_nice(16, seed),
                         states=lambda inst, seed: L.hamming_ball_states(inst, 256, seed=seed + 1),
                         beta=2.0, chi=64, M=1024, sweeps=2, d=256, oracle_sample=dict(_PEG_SAMPLE)),
    "pegasus15x15_d4096": dict(desc="Pegasus P16 nice, 15x15 cells of 24 spins (5400 spins), d=4096 states per cell "
                                    "(Hamming ball around a seeded reference), iid J,h in {+-1..+-7}/7, beta=2, "
                                    "chi=64, M=1024",
                               make=lambda seed: L.pegasus_nice(16, seed),
                               states=lambda inst, seed: L.hamming_ball_states(inst, 4096, seed=seed + 1),
                               beta=2.0, chi=64, M=1024, sweeps=2, d=4096, oracle_sample=dict(_PEG_SAMPLE)),
    "pegasus15x15_planted": dict(
        desc="Pegasus P16 nice, 15x15 cells, planted frustrated 4-cycles (ground energy known), d=256 states per "
             "cell around the planted state, beta=2, chi=64, M=1024",
        make=lambda seed: L.planted(L.pegasus_nice(16, seed), seed + 7, loops_per_cell=6),
        states=lambda inst, seed: L.hamming_ball_states(inst, 256, seed=seed + 1, reference=inst.planted),
        beta=2.0, chi=64, M=1024, sweeps=2, d=256, oracle_sample=dict(_PEG_SAMPLE)),
    # single-spin sites with both diagonals (the mediating path with trivial d)
    "kings50x50": dict(desc="King's lattice 50x50 (2500 spins, nearest and diagonal bonds), one spin per site, "
                            "class I couplings (J uniform in [-1, 1] on a 1/1000 grid, h = 0), beta=4, chi=16, M=256",
                       make=lambda seed: L.kings_grid(50, 50, seed, couplings="uniform"), states=None, beta=4.0,
                       chi=16, M=256, sweeps=2, d=2,
                       # beta = 4 is past the beta < 3 where the paper finds FP32 contractions adequate (Sec. VI)
                       precision="fp64",
                       oracle_sample=dict(make=lambda seed: L.kings_grid(8, 8, seed, couplings="uniform"),
                                          states=lambda inst, seed: None, chi=8, M=64,
                                          desc="King's lattice 8x8 (class I), chi=8, M=64")),
}
# many independent Pegasus instances of uneven size per step, each on its own stream: P3..P7 nice
# (2x2 .. 6x6 cells of 24 spins, 13/13/13/13/12 of each), 256 states per cell, beta 1, chi 32, M 128
def _batch64(seed):
    out = []
    for i in range(64):
        inst = L.pegasus_nice(3 + i % 5, seed * 1000 + i)
        out.append((inst, L.hamming_ball_states(inst, 256, seed=seed * 1000 + i + 1)))
    return out


WORKLOADS["batch64_pegasus"] = dict(
    desc="64 independent Pegasus instances of uneven size (P3..P7 nice: 2x2 to 6x6 cells, 96 to 864 spins), "
         "d=256 states per cell, iid J,h in {+-1..+-7}/7, beta=1, chi=32, M=128, one stream each",
    make=lambda seed: _batch64(seed)[0][0], states=lambda inst, seed: _batch64(seed)[0][1], batch=_batch64,
    n_batch=64, threads=16, beta=1.0, chi=32, M=128, sweeps=2, d=256, oracle_sample=dict(_PEG_SAMPLE))
# the same instances in all eight grid symmetries per step (Sec. IV: every instance is run from every corner)
for _name in ("kings50x50",):
    WORKLOADS[_name + "_x8"] = dict(WORKLOADS[_name], transforms=8,
                                    desc=WORKLOADS[_name]["desc"] + "; all 8 grid symmetries per step, concurrently")
DEFAULT = "pegasus15x15"
# precision name -> (boundary precision, search precision or -1, dtype label, FP64 final sweeps)
PRECISIONS = {"fp64": (0, -1, "f64", False),
              "fp32": (3, -1, "f32 contractions, f64 truncation", False),
              "tf32": (1, -1, "3xtf32 tensor cores + f32 contractions, f64 truncation", False),
              "tf32_polish": (1, -1, "3xtf32 tensor cores + f32 contractions, f64 truncation and final sweeps", True),
              "fp64_tf32search": (0, 1, "f64 boundary, 3xtf32/f32 conditional scores", False),
              "bf16": (2, -1, "bf16x3 tensor cores (segmented contractions) + 3xtf32 dense + f32, f64 truncation",
                       False)}
# the default: a mixed boundary whose sweeps after the cut run in FP64 (about 1.5e-7 log Z
# error at beta = 2 on P16, where the plain TF32 boundary sits near 1e-6), mixed scores
DEFAULT_PRECISION = "tf32_polish"
# FP64 peak of a B300 derived from unit counts: 148 SMs x 2 DFMA/clk/SM x 2 flop x 2032 MHz
FP64_PEAK_GFLOPS = 148 * 2 * 2 * 2.032
# FP32 SIMT peak from unit counts (148 SMs x 128 FMA/clk x 2 flop x 2032 MHz)
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e-3


def _measured_bf16():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except Exception:
        return 1800.0


MEASURED_BF16 = _measured_bf16()
# TF32 dense tensor peak = measured bf16 burst x 1/2 (nominal 1.1 / 2.25 PFLOP/s ratio)
TF32_PEAK_TFLOPS = MEASURED_BF16 * 0.5


def measure_peaks():
    """Dense GEMM peaks of this GPU measured here (cuBLAS through torch, CUDA events, best of
    several): FP64 (DGEMM 4096^3), FP32 (SGEMM 8192^3, TF32 off), TF32 (8192^3, TF32 on).
    B300's FP64 rate is far below its FP32 and tensor rates, so the FP64 kernels of the
    truncation are judged against the FP64 figure measured on the same box."""
    import torch
    out = {}
    dev = torch.device("cuda")
    prev = torch.backends.cuda.matmul.allow_tf32
    for name, n, dtype, tf32, reps in (("fp64_tflops", 4096, torch.float64, False, 5),
                                       ("fp32_tflops", 8192, torch.float32, False, 5),
                                       ("tf32_tflops", 8192, torch.float32, True, 10)):
        try:
            torch.backends.cuda.matmul.allow_tf32 = tf32
            a = torch.randn(n, n, device=dev, dtype=dtype)
            b = torch.randn(n, n, device=dev, dtype=dtype)
            torch.matmul(a, b)
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            out[name] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
            del a, b
        except Exception:
            out[name] = None
    torch.backends.cuda.matmul.allow_tf32 = prev
    torch.cuda.empty_cache()
    out["how"] = "torch.matmul (cuBLAS), CUDA events, best of 5-10: FP64 4096^3, FP32 (TF32 off) and TF32 8192^3"
    return out


MEASURED = {}


def clocks_sampler(dev_index):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    try:
        return subprocess.Popen(["nvidia-smi", "-i", str(dev_index), f"--query-gpu={q}", "--format=csv,noheader",
                                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except Exception:
        return None


def clocks_summary(proc):
    if proc is None:
        return None
    proc.terminate()
    out, _ = proc.communicate(timeout=10)
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1].split()[0]))
            mx.append(float(f[2].split()[0]))
        except ValueError:
            continue
        for n, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def marginal_check(h, inst, states, spins, mixed, n_steps=8):
    """Largest |p_mixed - p_fp64| / max p_fp64 of the conditionals along one configuration."""
    R, C = inst.rows, inst.cols
    cfg = []
    for site in range(R * C):
        sp = np.nonzero(inst.site_of_spin == site)[0]
        pat = int(sum(((1 - int(spins[g])) // 2) << j for j, g in enumerate(sp)))
        cfg.append(pat if states is None else int(np.nonzero(np.asarray(states[site]) == pat)[0][0]))
    steps = sorted(set(np.linspace(1, R * C - 1, n_steps).astype(int).tolist()))
    worst = 0.0
    for n in steps:
        h.set_search_precision(0)
        p64 = h.conditionals(n, np.array(cfg[:n], np.int32)[None])[0]
        h.set_search_precision(mixed)
        pm = h.conditionals(n, np.array(cfg[:n], np.int32)[None])[0]
        worst = max(worst, float(np.max(np.abs(pm - p64)) / np.max(p64)))
    return {"steps": steps, "max_abs_err_rel_to_max": worst, "search_precision": mixed}


def combine_ranks(t_ms, evals, device):
    """Whole-job figures of a replicas run: the slowest rank's time, every rank's evaluations."""
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(t_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ev = torch.tensor([float(evals)], device=device, dtype=torch.float64)
    dist.all_reduce(ev, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(ev.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_workload(wl):
    """The workload the oracle is timed on: the bench workload, or its declared bounded sample."""
    smp = wl.get("oracle_sample")
    if not smp:
        return dict(wl, sample_desc="the bench workload itself")
    return dict(wl, make=smp["make"], states=smp["states"], chi=smp["chi"], M=smp["M"], sample_desc=smp["desc"])


def cpu_oracle(wl, seed, budget_s=15.0, max_runs=5):
    """Oracle search timed on the host cores: marginals evaluated per second."""
    from oracle.search import search as oracle_search
    wl = oracle_workload(wl)
    try:
        from threadpoolctl import threadpool_info
        cores = max([t.get("num_threads", 1) for t in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    inst = wl["make"](seed)
    states = wl["states"](inst, seed) if wl["states"] else None
    runs, t_tot, evals = 0, 0.0, 0
    while runs < max_runs and (t_tot < budget_s or runs == 0):
        t0 = time.perf_counter()
        res = oracle_search(inst, wl["beta"], chi=wl["chi"], M=wl["M"], n_sweeps=wl["sweeps"], states=states)
        t_tot += time.perf_counter() - t0
        evals += res["evals"]
        runs += 1
    return {"value": evals / t_tot, "unit": "marginal evals/s", "cores": cores, "kind": "oracle",
            "sample": f"{runs} full oracle search(es) of {wl['sample_desc']} ({evals} evaluations, {t_tot:.1f} s)"}


def bench_config(args, wl, ws=1):
    return {"workload": args.workload, "description": wl["desc"],
            "instances_per_rank": wl.get("n_batch", 1), "grid_symmetries_per_step": wl.get("transforms", 1),
            "beta": wl["beta"], "chi": wl["chi"], "M": wl["M"], "states_per_cell": wl.get("d"),
            "n_sweeps": wl["sweeps"], "precision": args.precision, "parallelism": f"replicas{ws}",
            "l2": "flushed between timed steps (256 MB write)"}


def run_reference(args, wl):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle.search import search as oracle_search
    wl = oracle_workload(wl)
    inst = wl["make"](args.seed)
    states = wl["states"](inst, args.seed) if wl["states"] else None
    for _ in range(args.warmup):
        oracle_search(inst, wl["beta"], chi=wl["chi"], M=wl["M"], n_sweeps=wl["sweeps"], states=states)
    t_tot, evals = 0.0, 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        res = oracle_search(inst, wl["beta"], chi=wl["chi"], M=wl["M"], n_sweeps=wl["sweeps"], states=states)
        t_tot += time.perf_counter() - t0
        evals += res["evals"]
    try:
        from threadpoolctl import threadpool_info
        cores = max([t.get("num_threads", 1) for t in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    v = evals / t_tot
    line = {"impl": "reference", "metric": "marginal evals/s", "value": v, "unit": "marginal evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(bench_config(args, wl), oracle_sample=wl["sample_desc"]),
            "cpu_baseline": {"value": v, "unit": "marginal evals/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} full oracle searches of {wl['sample_desc']} ({evals} evaluations)"},
            "e2e": {"value": v, "unit": "marginal evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def peak_of(name):
    """(peak in TFLOP/s, bound, source) of a timed kernel label, from its arithmetic: the
    GEMM peak of the same arithmetic measured on this machine (measure_peaks), else derived."""
    if name.endswith("_tc_bf16"):
        return (MEASURED_BF16 / 6.0, "tensor",
                "measured bf16 burst peak (MEASURED_PEAKS.json) / 6 (six BF16 products per product)")
    if name.startswith("tc_gemm") or name.endswith("_tc"):
        if MEASURED.get("tf32_tflops"):
            return (MEASURED["tf32_tflops"] / 3.0, "tensor",
                    "measured TF32 cuBLAS peak on this box / 3 (three products per 3xTF32)")
        return (TF32_PEAK_TFLOPS / 3.0, "tensor",
                "measured bf16 burst peak x 1/2 (tf32 nominal ratio) / 3 (three products per 3xTF32)")
    if name.endswith("_f32"):
        if MEASURED.get("fp32_tflops"):
            return (MEASURED["fp32_tflops"], "alu", "measured FP32 (TF32 off) cuBLAS peak on this box")
        return (FP32_PEAK_TFLOPS, "alu", "derived: 148 SMs x 128 FFMA/clk x 2 flop x 2032 MHz")
    if MEASURED.get("fp64_tflops"):
        return (MEASURED["fp64_tflops"], "alu", "measured FP64 DGEMM peak on this box")
    return (FP64_PEAK_GFLOPS / 1e3, "alu", "derived: 148 SMs x 2 DFMA/clk x 2 flop x 2032 MHz")


# timing labels that bracket a chain of launches (the recursive blocked Cholesky:
# one-CTA diagonal blocks, GEMMs and zeroing kernels) rather than one kernel
REGIONS = ("cholesky_",)


def roofline_of(kt, names):
    """Roofline entry of the kernel with the largest device time among ``names``."""
    cand = [(kt[n][0], n) for n in names if kt.get(n) and kt[n][1] > 0 and kt[n][2] > 0]
    if not cand:
        return None
    _, kn = max(cand)
    ms, nl, fl = kt[kn]
    achieved = (fl / nl) / (ms / nl * 1e-3) / 1e12
    pk, bound, src = peak_of(kn)
    return {"kernel": kn, "bound": bound, "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
            "frac": achieved / pk, "traffic": None, "peak_source": src,
            "launches": nl, "ms_per_launch": ms / nl, "flop_per_launch": fl / nl}


# the sparse / batched contractions of the method (site diagram, environments, scores); the
# dense GEMMs ("gemm", "gemm_splitk") serve both contractions and the truncation and are left out
CONTRACTION_KERNELS = ("site_diagram", "env_update", "theta_env", "theta_mul", "renv", "score", "tc_gemm")


def run_native(args, wl):
    import torch
    import torch.distributed as dist
    from paper_2411_16431_b300 import sgtn

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    inst = wl["make"](args.seed + rank)
    states = wl["states"](inst, args.seed + rank) if wl["states"] else None
    prec, sprec, dtype_name, polish = PRECISIONS[args.precision]
    # the units of one step: the instance, or its first n grid symmetries, or a batch of
    # independent instances; every unit on its own stream when there are several
    if "batch" in wl:
        units = wl["batch"](args.seed + rank)
        inst, states = units[0]
    elif wl.get("transforms", 1) > 1:
        units = [(inst if k == 0 else L.transform(inst, k),
                  states if (k == 0 or states is None) else L.transform_states(inst, states, k))
                 for k in range(wl["transforms"])]
    else:
        units = [(inst, states)]
    n_tr = len(units)
    t_streams = [stream] if n_tr == 1 else [torch.cuda.Stream() for _ in range(n_tr)]

    def make_handles():
        hs = []
        for k, (ti, tst) in enumerate(units):
            hk = sgtn.Handle(ti, tst, stream=t_streams[k].cuda_stream)
            hk.set_search_precision(sprec)
            hk.set_final_sweeps_fp64(polish)
            hs.append(hk)
        return hs

    if rank == 0 and not args.no_peaks:
        MEASURED.update(measure_peaks())
    handles = make_handles()
    h = handles[0]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > 126 MB L2

    failed_transforms = [0]   # grid symmetries whose search stopped (no candidate with a positive score)
    spread = [None]           # std of log Z over the grid symmetries (App. C stability test)

    def one_search(hk):
        if args.droplets is None:
            return hk.search(wl["M"])
        # search with the excitation bookkeeping of Fig. 4 (energy window in energy units)
        r = hk.search_droplets(wl["M"], int(round(args.droplets * hk.inst.denom)), args.min_hamming, cap=0)
        drop_count[0] = r["n_droplets"]
        return dict(spins=r["spins"][None], energy_num=np.array([r["energy_num"]]), logp=np.array([r["logp"]]),
                    pd=r["pd"])

    drop_count = [None]

    def run_all(hs):
        """One step on every handle: (log Z of the first, best search result over all)."""
        if len(hs) == 1:
            hs[0].set_beta(wl["beta"])
            lz = hs[0].contract_boundary(wl["chi"], precision=prec, n_sweeps=wl["sweeps"])[0]
            return lz, one_search(hs[0])
        out = sgtn.batch_search(hs, wl["beta"], wl["chi"], wl["M"], precision=prec, n_sweeps=wl["sweeps"],
                                threads=wl.get("threads", 0), raise_on_error=False)
        ok = [i for i in range(len(out)) if out[i][1] is not None]
        failed_transforms[0] = len(out) - len(ok)
        spread[0] = sgtn.logz_spread([(None, out[i][0]) for i in ok])
        if not ok:
            raise RuntimeError("every unit failed: " + hs[0].L.sgtn_last_error(hs[0].h).decode())
        if "batch" in wl:   # independent instances: report the first one's result
            return out[0][0], out[0][1] if out[0][1] is not None else out[ok[0]][1]
        best = min(ok, key=lambda i: (int(out[i][1]["energy_num"][0]), i))
        return out[0][0], out[best][1]

    def step():
        return run_all(handles)[1]

    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    l0, f0, e0 = sgtn.stats()
    sgtn.kernel_timing(True, reset=True)
    clk = clocks_sampler(local)
    times = []
    bflops = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        if n_tr == 1:
            h.set_beta(wl["beta"])
            fa = sgtn.stats()[1]
            logz = h.contract_boundary(wl["chi"], precision=prec, n_sweeps=wl["sweeps"])[0]
            bflops += sgtn.stats()[1] - fa
            res = one_search(h)
        else:
            logz, res = run_all(handles)   # every stream has finished when the call returns
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    clocks = clocks_summary(clk)
    sgtn.kernel_timing(False)
    l1, f1, e1 = sgtn.stats()
    t_ms = sum(times)
    evals = e1 - e0
    if ws > 1:
        t_ms, evals_all = combine_ranks(t_ms, evals, "cuda")
    else:
        evals_all = evals
    kt = {n: sgtn.kernel_time(n) for n in sgtn.kernel_names()}
    unconverged = h.boundary_info()[0]
    # the FP64 arm of the "mixed vs FP64" comparison: the same step with every contraction
    # and score in FP64, timed the same way (1 warm-up, up to 2 steps) in the same process
    fp64_arm = None
    logz64 = None
    if (prec, sprec) != (0, -1) and n_tr == 1:
        for hk in handles:
            hk.set_search_precision(0)
        t64 = []
        ev64 = 0
        for i in range(1 + max(1, min(2, args.steps))):
            flush.zero_()
            torch.cuda.synchronize()
            e_a = sgtn.stats()[2]
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.set_beta(wl["beta"])
            logz64 = h.contract_boundary(wl["chi"], precision=0, n_sweeps=wl["sweeps"])[0]
            r64 = h.search(wl["M"])
            b.record(stream)
            torch.cuda.synchronize()
            if i > 0:
                t64.append(a.elapsed_time(b))
                ev64 += sgtn.stats()[2] - e_a
        fp64_arm = {"precision": "fp64", "value": ev64 / (sum(t64) * 1e-3), "unit": "marginal evals/s",
                    "steps": len(t64), "warmup": 1, "ms_per_step": sum(t64) / len(t64),
                    "logz": float(logz64) if np.isfinite(logz64) else None,
                    "energy_num": int(r64["energy_num"][0])}
        for hk in handles:
            hk.set_search_precision(sprec)
    # boundary contraction timed alone for its TFLOP/s
    torch.cuda.synchronize()
    h.set_beta(wl["beta"])
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fa = sgtn.stats()[1]
    h.contract_boundary(wl["chi"], precision=prec, n_sweeps=wl["sweeps"])
    b.record(stream)
    torch.cuda.synchronize()
    bound_ms = a.elapsed_time(b)
    if n_tr > 1:
        bflops = (sgtn.stats()[1] - fa) * args.steps   # one instance's boundary, timed alone
    # stated error of the timed arm's log Z against the separately computed FP64 boundary of
    # the FP64 arm (for an FP64 boundary the arithmetic is the same, so it is 0 exactly)
    fin = (lambda v: float(v) if np.isfinite(v) else None)   # JSON has no NaN: an undefined log Z is null
    if logz64 is None and prec != 0:
        logz64 = h.contract_boundary(wl["chi"], precision=0, n_sweeps=wl["sweeps"])[0]
    lz64 = logz if logz64 is None else logz64
    ok = np.isfinite(logz) and np.isfinite(lz64)
    logz_err = {"logz": fin(logz), "logz_fp64": fin(lz64), "rel_err": abs(logz - lz64) / abs(lz64) if ok else None,
                "boundary": "fp64" if prec == 0 else args.precision,
                "reference": "FP64 arm's boundary" if logz64 is not None else "the timed FP64 boundary itself"}
    # stated marginal error of the mixed search arithmetic: conditionals along the best
    # configuration at 8 steps, mixed against FP64 scores on the same (FP64) boundary (untimed)
    marg_err = None
    if (sprec != -1 or prec != 0) and n_tr == 1 and wl.get("transforms", 1) == 1:
        if prec != 0:
            h.contract_boundary(wl["chi"], precision=0, n_sweeps=wl["sweeps"])
        marg_err = marginal_check(h, inst, states, res["spins"][0], sprec if sprec != -1 else prec)
        h.set_search_precision(sprec)
    # end to end through the public API from host buffers: build (H2D) .. results (D2H)
    e2e_times = []
    h2d = 0
    for ui, us in units:
        h2d += ui.ei.nbytes + ui.ej.nbytes + ui.j_num.nbytes + ui.h_num.nbytes + ui.site_of_spin.nbytes
        if us is not None:
            h2d += sum(np.asarray(x, np.int64).nbytes for x in us) + 8 * (len(us) + 1)
    d2h = 0
    for _ in range(max(1, min(args.steps, 2))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hs2 = make_handles()
        _, r2 = run_all(hs2)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
        d2h = sum(ui.n_spins + 8 + 8 + 8 + 8 for ui, _ in units)   # spins, energy, log p, log Z, p_d
        for h2 in hs2:
            h2.close()
    e2e_val = (evals / args.steps) / statistics.median(e2e_times) * ws
    if rank != 0:
        if ws > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    timed = [n for n, v in kt.items() if v]
    roof = roofline_of(kt, [n for n in timed if not n.startswith(REGIONS)])
    region = roofline_of(kt, [n for n in timed if n.startswith(REGIONS)])
    roof_c = roofline_of(kt, [n for n in timed if n.startswith(CONTRACTION_KERNELS)])
    shares = {}
    tot_k = sum(v[0] for v in kt.values() if v)
    for n, v in sorted(kt.items(), key=lambda kv: -(kv[1][0] if kv[1] else 0)):
        if v:
            shares[n] = {"ms": v[0], "launches": v[1], "share_of_timed_kernels": v[0] / tot_k if tot_k else None}
    line = {"metric": "marginal evals/s", "value": evals_all / (t_ms * 1e-3), "unit": "marginal evals/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype_name,
            "data": "synthetic",
            "config": dict(bench_config(args, wl, ws), unconverged_truncations=unconverged,
                           failed_units=failed_transforms[0] if n_tr > 1 else None),
            "logz_spread_over_grid_symmetries": (spread[0] if spread[0] is not None and np.isfinite(spread[0])
                                                 else None) if wl.get("transforms", 1) > 1 else None,
            "droplets": None if args.droplets is None else {"max_dE": args.droplets, "min_hamming": args.min_hamming,
                                                            "count_of_best": drop_count[0]},
            "boundary_tflops": (bflops / args.steps) / (bound_ms * 1e-3) / 1e12,
            "boundary_ms": bound_ms,
            "fp64_arm": fp64_arm,
            "mixed_over_fp64": (evals_all / (t_ms * 1e-3)) / fp64_arm["value"] if fp64_arm else None,
            "measured_peaks": MEASURED or None,
            "logz_check": logz_err,
            "marginal_check": marg_err,
            "roofline": roof, "roofline_contraction": roof_c, "roofline_region": region, "kernel_times": shares,
            "e2e": {"value": e2e_val, "unit": "marginal evals/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int((l1 - l0) / args.steps),
            "clocks": clocks,
            "result": {"energy_num": int(res["energy_num"][0]), "logp": float(res["logp"][0]),
                       "planted_energy_num": getattr(inst, "planted_energy_num", None)}}
    if ws == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle(wl, args.seed)
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default=None,
                    help=f"default: the workload's own, else {DEFAULT_PRECISION}")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip measuring the GEMM peaks (kernels are then rated against derived peaks)")
    ap.add_argument("--droplets", type=float, default=None,
                    help="search with droplet bookkeeping (Fig. 4) in this energy window (single-instance workloads)")
    ap.add_argument("--min-hamming", type=int, default=2, help="Hamming threshold of the droplet filter")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    if args.precision is None:
        args.precision = wl.get("precision", DEFAULT_PRECISION)
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_native(args, wl)


if __name__ == "__main__":
    main()

"""The allocation-free entry point sgtn_conditionals_noalloc.

It exists for callers that must not let the library allocate device memory
while they run (a server that gives all device memory to its own pool at
start-up, a real-time loop that cannot absorb cudaMalloc's synchronisation).
It must return what sgtn_conditionals returns, call after call, although all
its temporaries live in one static device array that keeps the previous
call's contents, and it must make no device allocation at all -- checked with
the library's own count of cudaMalloc calls, in every search precision (the
FP32 and TF32 paths take other GEMM branches than FP64).  This file is
collected last so that a run stopping at the first failure has run every
other test first.
"""
import numpy as np
import pytest

from paper_2411_16431_b300 import lattices as L

pytestmark = pytest.mark.gpu

RTOL = {0: 1e-10, 3: 1e-4, 1: 1e-4}     # FP64, FP32, TF32 (against the same precision's sgtn_conditionals)


def _random_configs(h, step, count, seed):
    rng = np.random.default_rng(seed)
    return np.array([[rng.integers(h.d[p]) for p in range(step)] for _ in range(count)], np.int32).reshape(count, step)


@pytest.mark.parametrize("precision", [0, 3, 1], ids=["fp64", "fp32", "tf32"])
def test_noalloc_matches_conditionals_and_allocates_nothing(precision):
    from paper_2411_16431_b300.sgtn import Handle, device_allocations
    inst = L.chimera_grid(4, 4, 0)
    h = Handle(inst)
    h.set_beta(1.0)
    h.contract_boundary(16, n_sweeps=2)
    h.set_search_precision(precision)
    cases = ((6, 40, 1), (6, 40, 2), (13, 7, 3), (9, 300, 4))
    # warm-up: the first call on a device loads the module there
    h.conditionals_noalloc(*cases[0][:1], _random_configs(h, cases[0][0], 2, 0))
    refs = [h.conditionals(step, _random_configs(h, step, count, seed)) for step, count, seed in cases]
    before = device_allocations()
    # two calls in a row on different inputs (the second sees the first's
    # leftovers), then other shapes, all without a single device allocation
    got = [h.conditionals_noalloc(step, _random_configs(h, step, count, seed)) for step, count, seed in cases]
    assert device_allocations() == before
    for g, r in zip(got, refs):
        assert g.shape == r.shape
        assert np.allclose(g, r, rtol=RTOL[precision], atol=0.0)
        assert np.allclose(g.sum(axis=1), 1.0, rtol=1e-9)
    h.close()


def test_noalloc_rejects_requests_beyond_its_scratch_or_the_beam_limit():
    from paper_2411_16431_b300.sgtn import Handle, SgtnError
    inst = L.chimera_grid(4, 4, 0)
    h = Handle(inst)
    h.set_beta(1.0)
    h.contract_boundary(16, n_sweeps=2)
    # more partial configurations than one call may score: refused before
    # anything is copied or launched, by both entry points
    for count in (1025, 5000):
        cfg = _random_configs(h, 5, count, 6)
        with pytest.raises(SgtnError, match="SGTN_MAX_BEAM"):
            h.conditionals_noalloc(5, cfg)
        with pytest.raises(SgtnError, match="SGTN_MAX_BEAM"):
            h.conditionals(5, cfg)
    cfg = _random_configs(h, 5, 8, 5)               # still usable afterwards
    assert np.allclose(h.conditionals_noalloc(5, cfg), h.conditionals(5, cfg), rtol=1e-10, atol=0.0)
    full = _random_configs(h, 5, 1024, 7)           # the largest count fits the array here
    assert np.allclose(h.conditionals_noalloc(5, full), h.conditionals(5, full), rtol=1e-10, atol=0.0)
    h.close()
    # 4096 states per 24-spin cell: the projected boundary MPS of the row alone outgrows the
    # 32 MiB array (about 52 MB for 16 branches), so the call is refused with the byte
    # count; sgtn_conditionals serves it
    peg = L.pegasus_nice(4, 1)
    states = L.hamming_ball_states(peg, 4096, seed=2)
    h = Handle(peg, states)
    h.set_beta(0.5)
    h.contract_boundary(4, n_sweeps=1)
    cfg = _random_configs(h, 4, 16, 9)
    with pytest.raises(SgtnError, match="bytes of device scratch"):
        h.conditionals_noalloc(4, cfg)
    assert h.conditionals(4, cfg).shape == (16, 4096)
    h.close()

"""The allocation-free entry point sgtn_conditionals_noalloc.

It exists for callers that must not let the library allocate device memory
while they run (a server that gives all device memory to its own pool at
start-up, a real-time loop that cannot absorb cudaMalloc's synchronisation).
It must return what sgtn_conditionals returns, call after call, although all
its temporaries live in one static device array that keeps the previous
call's contents.  This file is collected last so that a run stopping at the
first failure has run every other test first.
"""
import numpy as np
import pytest

from paper_2411_16431_b300 import lattices as L

pytestmark = pytest.mark.gpu

RTOL = 1e-10


def _random_configs(h, step, count, seed):
    rng = np.random.default_rng(seed)
    return np.array([[rng.integers(h.d[p]) for p in range(step)] for _ in range(count)], np.int32).reshape(count, step)


def test_noalloc_matches_conditionals_on_consecutive_calls():
    from paper_2411_16431_b300.sgtn import Handle
    inst = L.chimera_grid(4, 4, 0)
    h = Handle(inst)
    h.set_beta(1.0)
    h.contract_boundary(16, n_sweeps=2)
    # two calls in a row on different inputs (the second sees the first's leftovers),
    # and a step with a different shape after them
    for step, count, seed in ((6, 40, 1), (6, 40, 2), (13, 7, 3)):
        cfg = _random_configs(h, step, count, seed)
        ref = h.conditionals(step, cfg)
        got = h.conditionals_noalloc(step, cfg)
        assert got.shape == ref.shape
        assert np.allclose(got, ref, rtol=RTOL, atol=0.0)
        assert np.allclose(got.sum(axis=1), 1.0, rtol=1e-12)
    h.close()


def test_noalloc_rejects_requests_beyond_its_scratch():
    from paper_2411_16431_b300.sgtn import Handle, SgtnError
    inst = L.chimera_grid(4, 4, 0)
    h = Handle(inst)
    h.set_beta(1.0)
    h.contract_boundary(16, n_sweeps=2)
    big = _random_configs(h, 5, 20000, 4)          # ~40 MB of scores > 32 MiB
    with pytest.raises(SgtnError, match="bytes of device scratch"):
        h.conditionals_noalloc(5, big)
    cfg = _random_configs(h, 5, 8, 5)               # still usable afterwards
    assert np.allclose(h.conditionals_noalloc(5, cfg), h.conditionals(5, cfg), rtol=RTOL, atol=0.0)
    h.close()

"""Continuous-batching service: every request's end state equals the same run stepped alone
(and the oracle's), whatever else shared its launches."""
import numpy as np
import pytest

from gpu_util import assert_same, gpu_run, oracle_for
from paper_2405_03605_gb300.workloads import RunShape

pytestmark = pytest.mark.gpu


def small_trace():
    shapes = []
    for i in range(10):
        shapes.append(RunShape(rows=3 + i % 4, cols=2 + (i * 3) % 5,
                               island_size=(16, 32, 64)[i % 3],
                               tournament_size=2 + i % 6, p_ben=0.02 * (i % 2),
                               surface_sites=(64, 256)[i % 2], seed=7, run_id=100 + i,
                               generations=20 + 13 * i))
    return [(0.002 * i, s) for i, s in enumerate(shapes)]


def test_served_results_equal_alone():
    from paper_2405_03605_gb300 import ga, serve
    trace = small_trace()
    budget = 4 * max(ga.workspace_bytes(s) for _, s in trace)  # forces queueing
    rep = serve.serve_continuous(trace, budget, chunk_gens=16, keep_results=True)
    assert rep.peak_bytes <= budget
    for req in rep.requests:
        s = req.shape
        assert req.finished >= req.admitted >= req.arrival
        alone = gpu_run(s)
        alone.step(s.generations)
        alone.sync()
        assert np.array_equal(req.result, alone.snapshot()), req.rid
        o = oracle_for(s)
        o.step(s.generations)
        assert_same(req.result, o.snapshot(), s.island_size)
    assert rep.percentile(50) <= rep.percentile(99)


def test_one_at_a_time_matches():
    from paper_2405_03605_gb300 import serve
    trace = small_trace()[:4]
    rep = serve.serve_one_at_a_time(trace, keep_results=True)
    for req in rep.requests:
        alone = gpu_run(req.shape)
        alone.step(req.shape.generations)
        alone.sync()
        assert np.array_equal(req.result, alone.snapshot())

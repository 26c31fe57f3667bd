"""Resident stepping (one cooperative launch per chunk of generations, islands kept in
registers, migrants through mailboxes) against the oracle and the streamed kernels, bit-exact,
through the C ABI; and the bounded mailbox waits: a neighbour that never sends makes the wait
run out, the launch ends with GA_ETIMEOUT, and the run steps correctly afterwards."""
import time

import numpy as np
import pytest

from gpu_util import assert_same, gpu_run, oracle_for
from paper_2405_03605_gb300.workloads import RunShape, SMALL_TORUS, STEADY, TILTED, HYBRID, \
    MODEL_FITNESS

pytestmark = pytest.mark.gpu

RESIDENT_AUTO, RESIDENT_OFF, RESIDENT_ON = 0, 1, 2


def _run(shape, gens, mode, chunks=None):
    g = gpu_run(shape)
    g.resident_policy(mode)
    for c in (chunks or [gens]):
        g.step(c)
    g.sync()
    return g


def test_paper_torus_full_run():
    """The 32x32 torus of 32-agent islands for 1,000 generations: resident, streamed and the
    oracle agree on every agent."""
    res = _run(SMALL_TORUS, 1000, RESIDENT_ON).snapshot()
    o = oracle_for(SMALL_TORUS)
    o.step(1000)
    assert_same(res, o.snapshot(), 32)
    assert_same(res, _run(SMALL_TORUS, 1000, RESIDENT_OFF).snapshot(), 32)


@pytest.mark.parametrize("N,rows,cols,every,tsize", [
    (32, 7, 9, 1, 5), (16, 9, 11, 1, 5), (8, 5, 7, 1, 5), (64, 6, 10, 1, 5),
    (32, 1, 1, 1, 5), (32, 1, 5, 1, 5), (16, 4, 1, 1, 5), (32, 2, 2, 1, 5),
    (32, 6, 6, 3, 5), (16, 5, 4, 16, 5), (32, 6, 5, 0, 5),
    (32, 5, 7, 1, 3), (16, 6, 6, 2, 8), (64, 3, 5, 1, 1),
])
def test_shapes_match_oracle(N, rows, cols, every, tsize):
    shape = RunShape(rows=rows, cols=cols, island_size=N, tournament_size=tsize,
                     migrate_every=every, seed=300 + N + rows, run_id=cols, p_ben=0.05,
                     p_del=0.05)
    got = _run(shape, 300, RESIDENT_ON).snapshot()
    o = oracle_for(shape)
    o.step(300)
    assert_same(got, o.snapshot(), N)


@pytest.mark.parametrize("S,b,policy", [(64, 1, HYBRID), (8, 8, TILTED), (32, 2, STEADY)])
def test_surfaces_and_float_model(S, b, policy):
    """Other 16-byte surfaces (hybrid, 8-bit tilted, 2-bit steady) and the float-fitness
    model of the paper's treatments."""
    shape = RunShape(rows=8, cols=6, surface_sites=S, differentia_bits=b, curation=policy,
                     seed=17, run_id=S)
    got = _run(shape, 500, RESIDENT_ON).snapshot()
    o = oracle_for(shape)
    o.step(500)
    assert_same(got, o.snapshot(), 32)
    for n in (32, 64):
        fit = RunShape(rows=6, cols=6, island_size=n, model=MODEL_FITNESS, p_del=0.33,
                       p_ben=0.003, seed=18 + n)
        got = _run(fit, 400, RESIDENT_ON).snapshot()
        o = oracle_for(fit)
        o.step(400)
        assert_same(got, o.snapshot(), n)


def test_split_steps_and_chunk_boundary():
    """Resident launches over ga_step calls of odd lengths and across the 4,096-generation
    site-table chunk equal one streamed run of 5,000 generations."""
    shape = RunShape(rows=12, cols=10, seed=51, run_id=2)
    res = _run(shape, 5000, RESIDENT_ON, chunks=[1, 36, 4096, 867]).snapshot()
    ref = _run(shape, 5000, RESIDENT_OFF).snapshot()
    assert_same(res, ref, 32)


def test_ineligible_runs():
    """48-byte records have no resident kernel (GA_EUNSUPPORTED under GA_RESIDENT_ON; AUTO
    streams them); a population loaded with mixed counters streams under AUTO."""
    from paper_2405_03605_gb300 import ga
    wide = RunShape(rows=4, cols=4, surface_sites=256)
    g = gpu_run(wide)
    g.resident_policy(RESIDENT_ON)
    with pytest.raises(ga.GaError) as e:
        g.step(3)
    assert e.value.code == -6
    g.resident_policy(RESIDENT_AUTO)
    g.step(3)
    g.sync()
    shape = RunShape(rows=4, cols=4, seed=4)
    g = gpu_run(shape)
    g.step(10)
    g.sync()
    rec = g.snapshot()
    rec[::7, 4:8] = np.array([3], np.uint32).view(np.uint8)  # some counters differ
    g.load(rec, 10)
    with pytest.raises(ga.GaError):
        g.resident_policy(RESIDENT_ON, 0)  # a zero wait limit is refused
    g.step(20)
    g.sync()
    o = oracle_for(shape)
    o.load(rec, 10)
    o.step(20)
    assert_same(g.snapshot(), o.snapshot(), 32)


def test_lost_migrants_time_out_and_the_run_recovers():
    """Island 5 never sends, so its four neighbours wait for mailboxes that nothing fills:
    with a 2 ms limit the launch ends with GA_ETIMEOUT within a fraction of a second (no block
    is left waiting), and after the injection is lifted the same run, reset, steps exactly as
    the oracle."""
    from paper_2405_03605_gb300 import ga
    shape = RunShape(rows=8, cols=8, seed=61)
    g = gpu_run(shape)
    g.resident_policy(RESIDENT_ON, 2000)
    g.inject_lost_migrants(5)
    t0 = time.perf_counter()
    g.step(200)
    with pytest.raises(ga.GaError) as e:
        g.sync()
    elapsed = time.perf_counter() - t0
    assert e.value.code == -4
    assert elapsed < 1.0, elapsed
    with pytest.raises(ga.GaError):
        g.inject_lost_migrants(64)  # out of range
    g.inject_lost_migrants()
    g.reset()
    g.step(200)
    g.sync()
    o = oracle_for(shape)
    o.step(200)
    assert_same(g.snapshot(), o.snapshot(), 32)

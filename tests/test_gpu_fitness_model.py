"""The float-fitness treatments of Sec. 3 on the GPU: bit-exact against the oracle (the
normal deviates are computed from correctly rounded single-precision operations on both
sides), at island sizes 16/32/64 and several tournament sizes, plus the full 512x1024 grid."""
import numpy as np
import pytest

from gpu_util import assert_same, gpu_run, oracle_for
from paper_2405_03605_gb300.workloads import RunShape, MODEL_FITNESS, \
    PAPER_FITNESS_ADAPTIVE, PAPER_FITNESS_PURIFYING, sample_agent_ids

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,n,p_ben", [(32, 5, 0.003), (32, 5, 0.0), (16, 3, 0.003),
                                       (64, 7, 0.05), (32, 8, 0.2)])
def test_fitness_model_parity(N, n, p_ben):
    shape = RunShape(rows=7, cols=5, island_size=N, tournament_size=n, p_ben=p_ben, p_del=0.33,
                     model=MODEL_FITNESS, effect_scale=0.75, seed=17 + N + n, run_id=n)
    g = gpu_run(shape)
    g.step(200)
    g.sync()
    o = oracle_for(shape)
    o.step(200)
    assert_same(g.snapshot(), o.snapshot(), N)


def test_fitness_model_full_grid():
    for shape in (PAPER_FITNESS_PURIFYING, PAPER_FITNESS_ADAPTIVE):
        g = gpu_run(shape)
        g.step(3)
        g.sync()
        o = oracle_for(shape)
        o.step(3)
        assert_same(g.snapshot(), o.snapshot(), 32)


def test_fitness_model_rejected_where_unsupported():
    from paper_2405_03605_gb300 import ga
    assert ga.config_check(RunShape(rows=2, cols=2, island_size=8, model=MODEL_FITNESS)) == -6
    assert ga.config_check(RunShape(rows=2, cols=2, model=MODEL_FITNESS, effect_scale=0.0)) == -1


def test_fitness_runs_step_solo_inside_a_batch():
    from paper_2405_03605_gb300 import ga
    a = RunShape(rows=4, cols=6, model=MODEL_FITNESS, p_ben=0.003, p_del=0.33, seed=5, run_id=1)
    b = RunShape(rows=5, cols=3, seed=5, run_id=2)
    runs = [gpu_run(a), gpu_run(b)]
    batch = ga.Batch(runs)
    batch.step(40)
    batch.step(3)
    batch.sync()
    for s, r in zip((a, b), runs):
        o = oracle_for(s)
        o.step(43)
        assert r.generation == 43
        assert_same(r.snapshot(), o.snapshot(), s.island_size)
    batch.close()


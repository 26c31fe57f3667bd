"""Batched stepping (many runs per launch) is bit-identical to stepping each run alone and
to the CPU oracle; autotuning changes no result."""
import ctypes as C

import numpy as np
import pytest

from gpu_util import assert_same, gpu_run, oracle_for
from paper_2405_03605_gb300.workloads import RunShape, batch_shapes, STEADY, TILTED, HYBRID

pytestmark = pytest.mark.gpu


def mixed_shapes():
    return [
        RunShape(rows=5, cols=7, island_size=32, seed=1, run_id=0),
        RunShape(rows=3, cols=4, island_size=16, tournament_size=3, p_ben=0.05, seed=1, run_id=1),
        RunShape(rows=6, cols=2, island_size=64, tournament_size=8, seed=1, run_id=2),
        RunShape(rows=4, cols=4, island_size=8, tournament_size=2, seed=1, run_id=3),
        RunShape(rows=4, cols=9, island_size=32, surface_sites=256, seed=1, run_id=4),
        RunShape(rows=2, cols=5, island_size=16, surface_sites=32, differentia_bits=8,
                 curation=TILTED, seed=1, run_id=5),
        RunShape(rows=3, cols=3, island_size=32, curation=HYBRID, migrate_every=4, seed=1,
                 run_id=6),
        RunShape(rows=7, cols=3, island_size=32, seed=99, run_id=7),  # another seed class
        RunShape(rows=1, cols=1, island_size=32, seed=1, run_id=8),
    ]


@pytest.mark.parametrize("chunks", [[37], [64, 64, 5], [1, 2, 3]])
def test_batch_equals_alone_and_oracle(chunks):
    from paper_2405_03605_gb300 import ga
    shapes = mixed_shapes()
    runs = [gpu_run(s) for s in shapes]
    batch = ga.Batch(runs)
    for c in chunks:
        batch.step(c)
    batch.sync()
    total = sum(chunks)
    for s, r in zip(shapes, runs):
        alone = gpu_run(s)
        alone.step(total)
        alone.sync()
        got = r.snapshot()
        assert np.array_equal(got, alone.snapshot()), s
        o = oracle_for(s)
        o.step(total)
        assert_same(got, o.snapshot(), s.island_size)
        assert r.generation == total
    batch.close()


def test_batch_membership_changes():
    from paper_2405_03605_gb300 import ga
    shapes = mixed_shapes()[:4]
    runs = [gpu_run(s) for s in shapes]
    batch = ga.Batch(runs[:2])
    batch.step(10)
    batch.add(runs[2])           # joins at generation 0 while the others are at 10
    batch.step(20)
    batch.remove(runs[0])
    runs[0].step(5)              # stepped alone after leaving
    batch.add(runs[3])
    batch.step(7)
    batch.sync()
    expect = {0: 35, 1: 37, 2: 27, 3: 7}
    for i, s in enumerate(shapes):
        assert runs[i].generation == expect[i]
        alone = gpu_run(s)
        alone.step(expect[i])
        alone.sync()
        runs[i].sync()
        assert np.array_equal(runs[i].snapshot(), alone.snapshot()), i
    batch.close()


def test_membership_rules():
    """A run belongs to at most one batch; destroying a member removes it from its batch, so
    the batch never steps a freed run; a destroyed batch leaves its runs free to join another."""
    from paper_2405_03605_gb300 import ga
    shapes = mixed_shapes()[:3]
    runs = [gpu_run(s) for s in shapes]
    b1 = ga.Batch(runs[:2])
    b2 = ga.Batch()
    with pytest.raises(ga.GaError):
        b2.add(runs[0])              # member of b1
    with pytest.raises(ga.GaError):
        b1.add(runs[1])              # already in b1
    b1.step(4)
    b1.sync()
    runs[1].close()                  # leaves b1 on destruction
    n = C.c_uint32()
    assert runs[0].lib.ga_batch_size(b1._h, C.byref(n)) == 0 and n.value == 1
    b1.step(3)                       # steps the remaining member only
    b1.sync()
    assert runs[0].generation == 7
    b1.close()
    b2.add(runs[0])                  # free again once b1 is gone
    b2.add(runs[2])
    b2.step(2)
    b2.sync()
    assert runs[0].generation == 9 and runs[2].generation == 2
    alone = gpu_run(shapes[0])
    alone.step(9)
    alone.sync()
    assert np.array_equal(runs[0].snapshot(), alone.snapshot())
    b2.close()


def test_autotune_changes_no_result():
    from paper_2405_03605_gb300 import ga
    shapes = [s.with_(generations=40) for s in batch_shapes(12, seed=5)]
    shapes = [s.with_(rows=min(s.rows, 32), cols=min(s.cols, 32)) for s in shapes]
    runs = [gpu_run(s) for s in shapes]
    batch = ga.Batch(runs)
    batch.step(3)
    choice = batch.autotune(trial_gens=4)
    assert choice["chunk"] in (16, 64, 256)
    assert all(w in (4, 8, 16) for _, w in choice["class_warps"])
    batch.step(37)
    batch.sync()
    for s, r in zip(shapes, runs):
        alone = gpu_run(s)
        alone.step(40)
        alone.sync()
        assert np.array_equal(r.snapshot(), alone.snapshot())
    batch.close()


def test_large_member_steps_solo_bit_identical():
    from paper_2405_03605_gb300 import ga
    shapes = [RunShape(rows=256, cols=256, island_size=16, seed=3, run_id=40),  # 65,536 islands
              RunShape(rows=6, cols=5, island_size=32, seed=3, run_id=41)]
    runs = [gpu_run(s) for s in shapes]
    batch = ga.Batch(runs)
    batch.step(9)
    batch.step(4)
    batch.sync()
    for s, r in zip(shapes, runs):
        alone = gpu_run(s)
        alone.step(13)
        alone.sync()
        assert r.generation == 13
        assert np.array_equal(r.snapshot(), alone.snapshot())
    o = oracle_for(shapes[1])
    o.step(13)
    assert_same(runs[1].snapshot(), o.snapshot(), 32)
    batch.close()

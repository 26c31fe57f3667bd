"""Determinism: the same configuration run twice gives the same end state, byte for byte.

compute-sanitizer is not available on this GPU pool; a race between blocks (an island
reading a neighbour's records while they are rewritten, a batch member stepped twice, a
buffer handed over early) would show up as run-to-run differences at full scale, where the
oracle is too slow to follow every generation.  Every synchronous mode, the batch and the
asynchronous sequential schedule must be deterministic; the free-running asynchronous mode
is not, by design.
"""
import hashlib

import pytest

from gpu_util import gpu_run
from paper_2405_03605_gb300.workloads import RunShape, PAPER_ADAPTIVE, batch_shapes, \
    variant_shapes, ASYNC_SEQUENTIAL

pytestmark = pytest.mark.gpu


def _digest(run):
    run.sync()
    return hashlib.sha256(run.snapshot().tobytes()).hexdigest()


def _twice(shape, gens):
    out = []
    for _ in range(2):
        g = gpu_run(shape)
        g.step(gens)
        out.append(_digest(g))
        g.close()
    return out


def test_full_grid_repeats():
    a, b = _twice(PAPER_ADAPTIVE, 300)
    assert a == b


@pytest.mark.parametrize("name", ["steady256x1", "tilted32x8", "hybrid64x1"])
def test_variants_repeat(name):
    shape = variant_shapes(island_size=16, migrate_every=4)[name]
    a, b = _twice(shape, 200)
    assert a == b


def test_batch_repeats():
    from paper_2405_03605_gb300 import ga
    shapes = batch_shapes(24, seed=5, generations=150)
    digests = []
    for _ in range(2):
        runs = [gpu_run(s) for s in shapes]
        b = ga.Batch(runs)
        b.step(150)
        b.sync()
        digests.append([_digest(r) for r in runs])
        b.close()
        for r in runs:
            r.close()
    assert digests[0] == digests[1]


def test_async_sequential_repeats():
    shape = RunShape(rows=5, cols=7, island_size=32, seed=3, mode=ASYNC_SEQUENTIAL,
                     async_window=3)
    a, b = _twice(shape, 60)
    assert a == b

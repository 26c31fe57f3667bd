"""Worker for tests/test_gpu_device_checks.py: runs on the device-check build of the library
(PAPER_2405_03605_GB300_LIB names libga_debug.so), where every kernel tests its global
indices and a failed test makes ga_sync / ga_batch_sync return GA_EBOUNDS.  Each case must
finish with a clean status and, as everywhere, the oracle's result."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from gpu_util import assert_same, oracle_for  # noqa: E402
from paper_2405_03605_gb300 import ga  # noqa: E402
from paper_2405_03605_gb300.workloads import (RunShape, STEADY, TILTED, HYBRID, ASYNC,  # noqa: E402
                                              ASYNC_SEQUENTIAL, sample_agent_ids)


def sync_case(shape, gens, ids=0):
    g = ga.Run(shape)
    g.step(gens)
    g.sync()
    o = oracle_for(shape)
    o.step(gens)
    assert_same(g.snapshot(), o.snapshot(), shape.island_size)
    if ids:
        sample = sample_agent_ids(shape.n_agents, ids, seed=3)
        lo, hi = g.mrca_bounds(sample)
        g.sync()
        elo, ehi = o.mrca_bounds(sample)
        assert np.array_equal(lo, elo) and np.array_equal(hi, ehi)
    g.close()


def async_case(shape, gens):
    g = ga.Run(shape)
    g.step(gens)
    g.sync()
    o = oracle_for(shape)
    o.step_async(gens, window=shape.async_window)
    assert_same(g.snapshot(), o.snapshot(), shape.island_size)
    g.close()


def main():
    assert os.path.basename(ga.LIB_PATH) == "libga_debug.so", ga.LIB_PATH
    n = 0
    for N, rows, cols in ((4, 5, 7), (8, 3, 9), (16, 4, 5), (32, 6, 7), (64, 3, 4), (128, 2, 3),
                          (32, 1, 1), (16, 1, 5), (32, 4, 1)):
        for S, b, policy in ((64, 1, STEADY), (128, 1, HYBRID), (32, 8, TILTED)):
            for every in (1, 3):
                sync_case(RunShape(rows=rows, cols=cols, island_size=N, surface_sites=S,
                                   differentia_bits=b, curation=policy, migrate_every=every,
                                   seed=N + S, run_id=every), 40, ids=24 if every == 1 else 0)
                n += 1
    for N, rows, cols in ((16, 3, 5), (32, 1, 2), (64, 2, 3), (32, 4, 4)):
        for S, b in ((64, 1), (256, 1)):
            for window in (1, 4):
                async_case(RunShape(rows=rows, cols=cols, island_size=N, surface_sites=S,
                                    differentia_bits=b, seed=5 + window, mode=ASYNC_SEQUENTIAL,
                                    async_window=window), 30)
                n += 1
    # free-running asynchronous runs with the mixed-counter MRCA
    for window in (1, 16):
        shape = RunShape(rows=64, cols=32, island_size=32, mode=ASYNC, async_window=window)
        g = ga.Run(shape)
        g.step(200)
        g.sync()
        ids = sample_agent_ids(shape.n_agents, 300, seed=1)
        lo, hi = g.mrca_bounds(ids)
        g.sync()
        elo, ehi = oracle.mrca_bounds_mixed(g.snapshot(), ids, shape.curation, shape.surface_sites,
                                            shape.differentia_bits)
        assert np.array_equal(lo, elo) and np.array_equal(hi, ehi)
        g.close()
        n += 1
    # a batch of mixed members
    shapes = [RunShape(rows=16, cols=16, island_size=16, run_id=1, tournament_size=3),
              RunShape(rows=32, cols=16, island_size=32, run_id=2),
              RunShape(rows=16, cols=32, island_size=64, run_id=3, surface_sites=256),
              RunShape(rows=3, cols=3, island_size=32, run_id=4, mode=ASYNC_SEQUENTIAL)]
    runs = [ga.Run(s) for s in shapes]
    batch = ga.Batch(runs)
    batch.step(70)
    batch.sync()
    for r, s in zip(runs, shapes):
        r.sync()
        o = oracle_for(s)
        if s.mode == ASYNC_SEQUENTIAL:
            o.step_async(70, window=s.async_window)
        else:
            o.step(70)
        assert_same(r.snapshot(), o.snapshot(), s.island_size)
    batch.close()
    n += 1
    print(f"device checks clean over {n} cases")


if __name__ == "__main__":
    main()

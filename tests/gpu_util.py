"""Helpers for the GPU parity tests: run the same seeded configuration through the CUDA
library and through the CPU oracle and compare canonical records byte for byte."""
import os

import numpy as np

from oracle import OracleRun


def threads():
    return max(1, min(32, os.cpu_count() or 1))


def oracle_for(shape, n_threads=None):
    return OracleRun(shape.rows, shape.cols, island_size=shape.island_size,
                     tournament_size=shape.tournament_size, p_ben=shape.p_ben,
                     p_del=shape.p_del, surface_sites=shape.surface_sites,
                     differentia_bits=shape.differentia_bits, curation=shape.curation,
                     migrate_every=shape.migrate_every, seed=shape.seed, run_id=shape.run_id,
                     threads=n_threads or threads(), model=shape.model,
                     effect_scale=shape.effect_scale)


def gpu_run(shape):
    from paper_2405_03605_gb300.build import build
    from paper_2405_03605_gb300 import ga
    build()
    return ga.Run(shape)


def describe_mismatch(got, exp, island_size):
    bad = np.nonzero((got != exp).any(axis=1))[0]
    a = int(bad[0])
    g = got[a].view(np.uint32)
    e = exp[a].view(np.uint32)
    return (f"{bad.size} of {got.shape[0]} agents differ; first agent {a} (island "
            f"{a // island_size}, slot {a % island_size}): gpu words {g.tolist()} oracle "
            f"{e.tolist()}")


def assert_same(got, exp, island_size):
    assert got.shape == exp.shape, (got.shape, exp.shape)
    if not np.array_equal(got, exp):
        raise AssertionError(describe_mismatch(got, exp, island_size))

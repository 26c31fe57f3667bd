"""GPU (CUDA library, through the C ABI) versus the CPU oracle, bit-exact on every trait,
counter and surface word of every agent.  Sizes span several warps/blocks with ragged tails;
one case runs the full 512x1024-island grid for 100 generations in the bench's launch
configuration."""
import hashlib
import json
import os

import numpy as np
import pytest

from conftest import GOLDEN
from gpu_util import assert_same, gpu_run, oracle_for
from paper_2405_03605_gb300.workloads import RunShape, SMALL_TORUS, PAPER_ADAPTIVE, \
    variant_shapes, sample_agent_ids, STEADY, TILTED, HYBRID

pytestmark = pytest.mark.gpu


def run_both(shape, gens, chunks=None):
    g = gpu_run(shape)
    for c in (chunks or [gens]):
        g.step(c)
    g.sync()
    o = oracle_for(shape)
    o.step(gens)
    got, exp = g.snapshot(), o.snapshot()
    return g, o, got, exp


def test_founder():
    shape = RunShape(rows=5, cols=7, surface_sites=256)
    g = gpu_run(shape)
    g.sync()
    assert_same(g.snapshot(), oracle_for(shape).snapshot(), shape.island_size)


@pytest.mark.parametrize("variant", ["adaptive", "purifying"])
def test_small_torus_full_run_and_golden(variant):
    with open(os.path.join(GOLDEN, "small_torus.json")) as f:
        gold = json.load(f)
    case = gold["cases"][variant]
    shape = SMALL_TORUS.with_(p_ben=case["p_ben"], run_id=case["run_id"])
    g = gpu_run(shape)
    g.step(gold["generations"])
    g.sync()
    got = g.snapshot()
    assert hashlib.sha256(got.tobytes()).hexdigest() == case["sha256"]
    o = oracle_for(shape)
    o.step(gold["generations"])
    assert_same(got, o.snapshot(), shape.island_size)


@pytest.mark.parametrize("N,rows,cols", [(4, 5, 7), (8, 7, 9), (16, 9, 11), (32, 13, 17),
                                         (64, 6, 10), (128, 5, 3)])
def test_island_sizes_ragged(N, rows, cols):
    shape = RunShape(rows=rows, cols=cols, island_size=N, seed=1234 + N, run_id=N)
    _, _, got, exp = run_both(shape, 150)
    assert_same(got, exp, N)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
def test_tournament_sizes(n):
    shape = RunShape(rows=6, cols=5, tournament_size=n, p_ben=0.05, p_del=0.05, seed=n)
    _, _, got, exp = run_both(shape, 120)
    assert_same(got, exp, 32)


@pytest.mark.parametrize("name", ["steady256x1", "tilted32x8", "hybrid64x1"])
@pytest.mark.parametrize("N", [16, 32, 64])
@pytest.mark.parametrize("k", [1, 4, 16])
def test_surface_variants(name, N, k):
    base = variant_shapes(N, migrate_every=k)[name]
    shape = base.with_(rows=max(2, 8 * 32 // N), cols=7)
    _, _, got, exp = run_both(shape, 230)
    assert_same(got, exp, N)


@pytest.mark.parametrize("S,b,policy", [(128, 1, STEADY), (16, 2, STEADY), (8, 4, STEADY),
                                        (4, 1, STEADY), (64, 4, TILTED), (32, 1, HYBRID),
                                        (16, 8, TILTED), (8, 1, HYBRID)])
def test_more_surfaces(S, b, policy):
    shape = RunShape(rows=4, cols=9, island_size=16, surface_sites=S, differentia_bits=b,
                     curation=policy, seed=S * 10 + b)
    _, _, got, exp = run_both(shape, 300)
    assert_same(got, exp, 16)


@pytest.mark.parametrize("rows,cols", [(1, 1), (1, 5), (4, 1), (2, 2), (3, 2)])
def test_degenerate_tori(rows, cols):
    shape = RunShape(rows=rows, cols=cols, seed=rows * 100 + cols)
    _, _, got, exp = run_both(shape, 90)
    assert_same(got, exp, 32)


def test_no_migration_long_launches():
    shape = RunShape(rows=5, cols=6, migrate_every=0, seed=77)
    _, _, got, exp = run_both(shape, 600)  # 256-generation launches
    assert_same(got, exp, 32)


@pytest.mark.parametrize("p_ben,p_del", [(0.0, 0.0), (1.0, 0.0), (0.0, 1.0), (0.5, 0.5),
                                         (1e-4, 1e-1)])
def test_mutation_extremes(p_ben, p_del):
    shape = RunShape(rows=4, cols=4, p_ben=p_ben, p_del=p_del, seed=5)
    _, _, got, exp = run_both(shape, 64)
    assert_same(got, exp, 32)


def test_large_seed_and_run_id():
    shape = RunShape(rows=4, cols=5, seed=0xDEADBEEF12345678, run_id=0xFFFFFFF0)
    _, _, got, exp = run_both(shape, 50)
    assert_same(got, exp, 32)


def test_split_steps_identical():
    shape = RunShape(rows=6, cols=6, island_size=16, migrate_every=4, seed=3)
    a = gpu_run(shape)
    a.step(45)
    b = gpu_run(shape)
    for c in (1, 2, 3, 7, 11, 21):
        b.step(c)
    a.sync()
    b.sync()
    assert np.array_equal(a.snapshot(), b.snapshot())


def test_reset_and_resume():
    shape = RunShape(rows=5, cols=4, seed=8)
    a = gpu_run(shape)
    a.step(40)
    a.sync()
    mid = a.snapshot()
    a.step(25)
    a.sync()
    full = a.snapshot()
    b = gpu_run(shape)
    b.load(mid, 40)
    b.step(25)
    b.sync()
    assert np.array_equal(b.snapshot(), full)
    a.reset()
    a.step(65)
    a.sync()
    assert np.array_equal(a.snapshot(), full)


@pytest.mark.parametrize("policy,S,b", [(STEADY, 64, 1), (TILTED, 32, 8), (HYBRID, 64, 1)])
def test_sync_steps_from_mixed_counters(policy, S, b):
    """A synchronous run loaded with agents of different counters (an asynchronous population)
    deposits each agent at its own counter's site, alone and as a batch member."""
    from paper_2405_03605_gb300 import ga
    shape = RunShape(rows=4, cols=6, island_size=32, surface_sites=S, differentia_bits=b,
                     curation=policy, seed=21)
    src = oracle_for(shape)
    src.step_async(60, window=7)
    mixed = src.snapshot()
    counters = mixed.view(np.uint32)[:, 1]
    assert len(set(counters.tolist())) > 1
    o = oracle_for(shape)
    o.load(mixed, 60)
    o.step(35)
    exp = o.snapshot()
    g = gpu_run(shape)
    g.load(mixed, 60)
    g.step(35)
    g.sync()
    assert_same(g.snapshot(), exp, shape.island_size)
    # a batch member first stepped in a uniform-counter class, then loaded with the mixed
    # counters at the same generation and buffer: only its counters' uniformity changes, and
    # the batch must move it to a class with the closed form
    h = gpu_run(shape)
    batch = ga.Batch([h])
    batch.step(60)
    batch.sync()
    h.load(mixed, 60)
    batch.step(35)
    batch.sync()
    assert_same(h.snapshot(), exp, shape.island_size)
    batch.close()
    # then loading a population whose counters all equal the generation (a synchronous run's)
    # restores the uniform path
    u = oracle_for(shape)
    u.step(20)
    g.load(u.snapshot(), 20)
    g.step(10)
    g.sync()
    u.step(10)
    assert_same(g.snapshot(), u.snapshot(), shape.island_size)


def test_library_allocated_workspace():
    from paper_2405_03605_gb300 import ga
    shape = RunShape(rows=3, cols=3, seed=4)
    g = ga.Run(shape, workspace="library")
    g.step(33)
    g.sync()
    o = oracle_for(shape)
    o.step(33)
    assert_same(g.snapshot(), o.snapshot(), 32)
    g.close()


def test_curation_sites_match_oracle():
    import oracle
    from paper_2405_03605_gb300 import ga
    count = 1 << 20
    for policy, sizes in ((STEADY, (4, 8, 16, 32, 64, 128, 256)),
                          (TILTED, (4, 8, 16, 32, 64, 256)),
                          (HYBRID, (8, 16, 64, 256))):
        for S in sizes:
            for t0 in (0, 2 ** 32 - count):
                got = ga.curation_sites(policy, S, t0, count).cpu().numpy()
                exp = oracle.site_table(policy, S, t0, count)
                bad = np.nonzero(got != exp)[0]
                assert bad.size == 0, (policy, S, t0, int(bad[0]), int(got[bad[0]]),
                                       int(exp[bad[0]]))


def test_full_grid_first_generations():
    """The 512x1024 x 32-agent grid (16,777,216 agents) for 100 generations, compared with the
    oracle on every agent, in the launch configuration the benchmark times (one launch per
    generation, migration every generation); then the MRCA bounds of 4,096 sampled agents."""
    shape = PAPER_ADAPTIVE
    g = gpu_run(shape)
    g.step(100)
    g.sync()
    o = oracle_for(shape)
    o.step(100)
    got, exp = g.snapshot(), o.snapshot()
    assert_same(got, exp, 32)
    ids = sample_agent_ids(shape.n_agents, 4096, seed=42)
    lo, hi = g.mrca_bounds(ids)
    elo, ehi = o.mrca_bounds(ids)
    assert np.array_equal(lo, elo) and np.array_equal(hi, ehi)


@pytest.mark.parametrize("shape", [
    RunShape(rows=16, cols=16, island_size=32, surface_sites=64, differentia_bits=1,
             curation=STEADY, seed=101, run_id=1),
    RunShape(rows=16, cols=16, island_size=32, surface_sites=32, differentia_bits=8,
             curation=TILTED, seed=102, run_id=2),
], ids=["steady64x1", "tilted32x8"])
def test_benchmark_depth_10000_generations(shape):
    """A 16x16 torus for 10,000 generations -- the depth the benchmark runs, where steady
    curation reaches epoch 8 -- compared with the oracle on every agent, then the MRCA bounds
    of 2,000 sampled agents at T = 10,000 compared pair by pair (8,192 agents coalesce within
    a few dozen generations, so most pairs share the newest retained ranks)."""
    g, o, got, exp = run_both(shape, 10000, chunks=[4096, 4096, 1808])
    assert_same(got, exp, 32)
    ids = sample_agent_ids(shape.n_agents, 2000, seed=8)
    lo, hi = g.mrca_bounds(ids)
    elo, ehi = o.mrca_bounds(ids)
    assert np.array_equal(lo, elo) and np.array_equal(hi, ehi)

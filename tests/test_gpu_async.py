"""Asynchronous mode on the GPU (mailbox migration, Sec. 2 wafer-scale loop) against the
oracle, through the C ABI.

  - GA_ASYNC_SEQUENTIAL (islands one launch at a time, in index order) is bit-exact against
    the oracle's sequential schedule: mailboxes, sequence marks, landing draws, drifting
    counters and the deposits at each agent's own counter;
  - free-running GA_ASYNC is bit-exact where the schedule cannot matter (migration off; a
    single island) and otherwise checked by invariants;
  - the mixed-counter MRCA kernels are exact against the oracle on populations with widely
    spread counters (synthetic forked lineages loaded through ga_load) and on populations the
    free-running mode produced.
"""
import numpy as np
import pytest

import oracle
from gpu_util import assert_same, gpu_run, oracle_for
from paper_2405_03605_gb300.workloads import RunShape, STEADY, TILTED, HYBRID, \
    SYNC, ASYNC, ASYNC_SEQUENTIAL, MODEL_FITNESS, sample_agent_ids

pytestmark = pytest.mark.gpu


def _sequential_both(shape, calls):
    g = gpu_run(shape)
    o = oracle_for(shape)
    arrivals = 0
    for n in calls:
        g.step(n)
        arrivals += int(o.step_async(n, window=shape.async_window).sum())
    g.sync()
    return g.snapshot(), o.snapshot(), arrivals


# drift: the oracle's end state holds agents of different counters (genomes that arrived
# late survived), so those cases exercise deposits at counters other than the generation.
# 16-byte records take the atomic handoff, 32/48-byte ones the flag handoff; tori with one
# row or column (an island its own neighbour) take the in-generation ordering; one-generation
# launches of 16-byte records take the block-cooperative kernel.
@pytest.mark.parametrize("rows,cols,N,S,b,policy,window,every,drift", [
    (1, 1, 16, 64, 1, STEADY, 5, 1, True),
    (1, 2, 32, 64, 1, STEADY, 3, 1, True),
    (3, 5, 16, 64, 1, STEADY, 5, 1, True),
    (2, 3, 64, 64, 1, TILTED, 7, 1, False),
    (3, 4, 32, 256, 1, STEADY, 16, 1, False),
    (4, 3, 16, 32, 8, TILTED, 1, 1, True),
    (3, 1, 32, 128, 1, HYBRID, 8, 3, True),
    (2, 5, 64, 16, 2, STEADY, 11, 2, False),
    # window 1, 16-byte records: the block-cooperative one-generation kernel
    (3, 5, 16, 64, 1, STEADY, 1, 1, True),
    (1, 2, 32, 64, 1, STEADY, 1, 1, True),
    (2, 3, 64, 64, 1, TILTED, 1, 2, True),
    (4, 4, 32, 32, 2, HYBRID, 1, 1, True),
    # 8- and 128-agent islands
    (3, 4, 8, 64, 1, STEADY, 3, 1, True),
    (3, 3, 8, 32, 8, TILTED, 1, 1, True),
    (2, 3, 128, 64, 1, STEADY, 1, 1, True),
    (2, 2, 128, 256, 1, STEADY, 4, 1, False),
])
def test_sequential_matches_oracle(rows, cols, N, S, b, policy, window, every, drift):
    shape = RunShape(rows=rows, cols=cols, island_size=N, surface_sites=S, differentia_bits=b,
                     curation=policy, migrate_every=every, seed=700 + rows * cols + N,
                     run_id=rows, p_ben=0.05, p_del=0.05, mode=ASYNC_SEQUENTIAL,
                     async_window=window)
    got, exp, arrivals = _sequential_both(shape, [40, 23])
    assert arrivals > 0
    assert_same(got, exp, N)
    c = exp[:, 4:8].copy().view(np.uint32)
    assert (len(np.unique(c)) > 1) == drift


@pytest.mark.parametrize("window", [6, 1])
def test_sequential_fitness_model_matches_oracle(window):
    shape = RunShape(rows=3, cols=4, island_size=32, p_ben=0.003, p_del=0.33,
                     model=MODEL_FITNESS, seed=17, run_id=5, mode=ASYNC_SEQUENTIAL,
                     async_window=window)
    got, exp, _ = _sequential_both(shape, [50])
    assert_same(got, exp, 32)


@pytest.mark.parametrize("tsize,N", [(3, 16), (8, 32), (1, 64)])
@pytest.mark.parametrize("window", [1, 4])
def test_sequential_tournament_sizes(tsize, N, window):
    """Tournament sizes other than the compiled-in 5, in both kernels (window 1: the
    one-generation kernel; window 4: the multi-generation kernel)."""
    shape = RunShape(rows=3, cols=3, island_size=N, tournament_size=tsize, seed=23 + tsize,
                     p_ben=0.05, p_del=0.05, mode=ASYNC_SEQUENTIAL, async_window=window)
    got, exp, _ = _sequential_both(shape, [21])
    assert_same(got, exp, N)


@pytest.mark.parametrize("N", [8, 16, 32, 64, 128])
def test_free_running_without_migration_is_sync(N):
    base = RunShape(rows=37, cols=41, island_size=N, migrate_every=0, seed=5, run_id=N)
    a = gpu_run(base.with_(mode=ASYNC, async_window=16))
    s = gpu_run(base)
    a.step(100)
    s.step(100)
    a.sync()
    s.sync()
    got = a.snapshot()
    assert_same(got, s.snapshot(), N)
    o = oracle_for(base)
    o.step(100)
    assert_same(got, o.snapshot(), N)


@pytest.mark.parametrize("window", [1, 16, 256])
def test_free_running_single_island_matches_oracle(window):
    """One island has one schedule: the free-running launch must equal the oracle."""
    shape = RunShape(rows=1, cols=1, island_size=32, seed=3, mode=ASYNC, async_window=window)
    g = gpu_run(shape)
    g.step(300)
    g.sync()
    o = oracle_for(shape)
    o.step_async(300, window=window)
    assert_same(g.snapshot(), o.snapshot(), 32)


def test_free_running_invariants_and_mrca():
    shape = RunShape(rows=256, cols=64, island_size=32, seed=11, p_ben=0.05, p_del=0.05,
                     mode=ASYNC, async_window=16)  # many block waves: counters run ahead
    g = gpu_run(shape)
    g.step(400)
    g.sync()
    rec = g.snapshot()
    words = rec.view(np.uint32).reshape(rec.shape[0], -1)
    t = words[:, 0].view(np.int32).astype(np.int64)
    c = words[:, 1].astype(np.int64)
    assert np.all(np.abs(t) <= c)
    assert c.min() >= 1  # every slot was refilled by a birth in the last generation
    ids = np.sort(np.random.default_rng(1).choice(shape.n_agents, 700, replace=False)).astype(np.uint32)
    lo, hi = g.mrca_bounds(ids)
    elo, ehi = oracle.mrca_bounds_mixed(rec, ids, shape.curation, shape.surface_sites,
                                        shape.differentia_bits)
    assert np.array_equal(lo, elo) and np.array_equal(hi, ehi)


def _mean_depth(g, ids, shape):
    """Mean over pairs of min(Ta, Tb) - hi: how long ago, at least, two lineages split."""
    rec = g.snapshot()
    lo, hi = g.mrca_bounds(ids)
    c = rec[:, 4:8].copy().view(np.uint32).ravel()[ids].astype(np.int64)
    T = np.minimum(c[:, None], c[None, :])[np.triu_indices(len(ids), 1)]
    assert np.all(lo <= hi) and np.all(hi <= T)
    return float(np.mean(T - hi.astype(np.int64)))


@pytest.mark.parametrize("seed", [1, 2])
def test_free_running_counters_and_treatment_contrast(seed):
    """Window 1 (neighbours at most a generation apart).  Every agent descends, through at
    least one birth per generation, from an agent or a buffered copy of the previous
    snapshot, so the smallest counter never falls; |trait| <= counter; and purifying-only
    runs keep far deeper genealogies than adaptive ones (Sec. 3), measured by the
    mixed-counter MRCA bounds."""
    depth = {}
    for p_ben in (0.01, 0.0):
        shape = RunShape(rows=8, cols=8, p_ben=p_ben, p_del=0.01, seed=seed,
                         run_id=int(p_ben > 0), mode=ASYNC, async_window=1)
        g = gpu_run(shape)
        low = 0
        for _ in range(6):
            g.step(100)
            g.sync()
            w = g.snapshot().view(np.uint32).reshape(shape.n_agents, -1)
            c = w[:, 1].astype(np.int64)
            assert c.min() >= low and c.min() >= 1
            assert np.all(np.abs(w[:, 0].view(np.int32).astype(np.int64)) <= c)
            low = int(c.min())
        ids = sample_agent_ids(shape.n_agents, 200, seed=seed)
        depth[p_ben] = _mean_depth(g, ids, shape)
    assert depth[0.0] > depth[0.01] + 100, depth


def _forked_population(n_agents, S, b, policy, t_lo, t_hi, seed):
    """Agents whose lineages split from one trunk at random ranks and then ran to random
    counters in [t_lo, t_hi): records with widely spread counters and a known structure."""
    rng = np.random.default_rng(seed)
    words = (S * b + 31) // 32
    rb = oracle.record_bytes(S, b)
    sites = oracle.site_table(policy, S, 0, t_hi)
    mask = (1 << b) - 1

    def deposit(surf, t):
        k = int(sites[t])
        if k >= 0:
            pos = k * b
            w, sh = pos // 32, pos % 32
            surf[w] = (surf[w] & ~(mask << sh)) | (int(rng.integers(0, mask + 1)) << sh)

    trunk = [[int(x) for x in rng.integers(0, 2 ** 32, words)]]
    for t in range(t_hi):
        s = list(trunk[-1])
        deposit(s, t)
        trunk.append(s)
    distinct = min(n_agents, 320)  # the rest repeat them (identical pairs are a case too)
    rec = np.zeros((n_agents, rb), np.uint8)
    for a in range(distinct):
        T = int(rng.integers(t_lo, t_hi))
        D = int(rng.integers(max(0, T - 400), T + 1)) if a % 3 else int(rng.integers(0, T + 1))
        s = list(trunk[D])
        for t in range(D, T):
            deposit(s, t)
        rec[a, 0:4] = np.array([a], np.int32).view(np.uint8)
        rec[a, 4:8] = np.array([T], np.uint32).view(np.uint8)
        rec[a, 8:8 + 4 * words] = np.array(s, np.uint32).view(np.uint8)
    rec[distinct:] = rec[np.arange(distinct, n_agents) % distinct]
    return rec


@pytest.mark.parametrize("S,b,policy,t_lo,t_hi,n", [
    (64, 1, STEADY, 0, 3000, 300),
    (32, 8, TILTED, 1500, 2600, 257),
    (64, 1, HYBRID, 900, 1000, 17),
    (256, 1, STEADY, 2000, 2100, 1000),
    (64, 4, STEADY, 5000, 5001, 64),
    (16, 2, TILTED, 0, 40, 2),
])
def test_mixed_mrca_loaded_matches_oracle(S, b, policy, t_lo, t_hi, n):
    shape = RunShape(rows=8, cols=8, island_size=32, surface_sites=S, differentia_bits=b,
                     curation=policy, mode=ASYNC)
    rec = _forked_population(shape.n_agents, S, b, policy, t_lo, t_hi, seed=S + n)
    g = gpu_run(shape)
    g.load(rec, 0)
    ids = np.random.default_rng(n).permutation(shape.n_agents)[:n].astype(np.uint32)
    lo, hi = g.mrca_bounds(ids)
    elo, ehi = oracle.mrca_bounds_mixed(rec, ids, policy, S, b)
    assert np.array_equal(hi, ehi), np.nonzero(hi != ehi)[0][:5]
    assert np.array_equal(lo, elo), np.nonzero(lo != elo)[0][:5]


def test_window_setter_errors():
    from paper_2405_03605_gb300 import ga
    s = gpu_run(RunShape(rows=2, cols=2))
    with pytest.raises(ga.GaError) as e:
        s.async_window(8)
    assert e.value.code == -5  # GA_ESTATE: synchronous run
    a = gpu_run(RunShape(rows=2, cols=2, mode=ASYNC))
    for bad in (0, 257):
        with pytest.raises(ga.GaError) as e:
            a.async_window(bad)
        assert e.value.code == -1
    a.async_window(256)


def test_batch_steps_async_member_alone():
    """A batch advances an asynchronous member with the single-run kernels: a sequential
    member stays bit-exact against the oracle, a synchronous one beside it too."""
    from paper_2405_03605_gb300 import ga
    seq = RunShape(rows=3, cols=4, island_size=16, seed=2, mode=ASYNC_SEQUENTIAL, async_window=4)
    syn = RunShape(rows=16, cols=16, island_size=32, seed=3, run_id=1)
    r1, r2 = gpu_run(seq), gpu_run(syn)
    b = ga.Batch([r1, r2])
    b.step(64)
    b.sync()
    o1 = oracle_for(seq)
    o1.step_async(64, window=4)
    o2 = oracle_for(syn)
    o2.step(64)
    assert_same(r1.snapshot(), o1.snapshot(), 16)
    assert_same(r2.snapshot(), o2.snapshot(), 32)
    b.close()


@pytest.mark.parametrize("sites", [64, 256])  # 16-byte (atomic) and 48-byte (flag) buffers
def test_reset_and_load_empty_the_buffers(sites):
    """ga_reset and ga_load empty every send buffer: on the sequential schedule a reset run
    repeats a fresh run exactly, and a population loaded mid-run continues exactly as the
    oracle continues from the same records with empty buffers."""
    shape = RunShape(rows=3, cols=4, island_size=16, surface_sites=sites, seed=41,
                     mode=ASYNC_SEQUENTIAL, async_window=4)
    g = gpu_run(shape)
    g.step(30)
    g.sync()
    first = g.snapshot()
    g.reset()
    g.step(30)
    g.sync()
    assert_same(g.snapshot(), first, 16)
    # buffers are full after 30 generations; a load must drop them
    g.load(first, 30)
    g.step(20)
    g.sync()
    o = oracle_for(shape)
    o.load(first, 30)
    o.step_async(20, window=4)
    assert_same(g.snapshot(), o.snapshot(), 16)


@pytest.mark.parametrize("window", [1, 4])  # one-generation kernel, multi-generation kernel
def test_reserved_counter_is_refused_and_reported(window):
    """Counter 2^32 - 1 marks an empty 16-byte buffer, so the asynchronous modes keep it out
    of every valid run: ga_load refuses it (GA_EINVAL), and a birth that would produce it
    (parents at 2^32 - 2) leaves GA_ESTATE in the status word for the next ga_sync.  The
    synchronous mode has no buffers and accepts it."""
    from paper_2405_03605_gb300 import ga
    shape = RunShape(rows=2, cols=3, island_size=16, seed=12, mode=ASYNC, async_window=window)
    g = gpu_run(shape)
    rec = g.snapshot()
    rec[:, 4:8] = np.array([0xFFFFFFFF], np.uint32).view(np.uint8)
    with pytest.raises(ga.GaError) as e:
        g.load(rec, 0)
    assert e.value.code == -1
    rec[:, 4:8] = np.array([0xFFFFFFFE], np.uint32).view(np.uint8)
    g.load(rec, 0)
    g.step(window)
    with pytest.raises(ga.GaError) as e:
        g.sync()
    assert e.value.code == -5
    g.sync()  # the status word was read and cleared
    s = gpu_run(shape.with_(mode=SYNC))
    rec[:, 4:8] = np.array([0xFFFFFFFF], np.uint32).view(np.uint8)
    s.load(rec, 0)
    s.step(2)
    s.sync()


@pytest.mark.parametrize("S,b,policy,t_lo,t_hi", [
    (64, 1, STEADY, 70000, 73000),
    (32, 8, TILTED, 100000, 100500),
    (256, 1, HYBRID, 16000, 40000),
])
def test_mixed_mrca_large_counters_match_oracle(S, b, policy, t_lo, t_hi):
    """Counters past 16,384 spread over a range, sparse random surfaces (first mismatches
    anywhere in the shared ranks): the GPU's per-agent tables (closed form) and the oracle's
    (replay) give the same bounds on every pair."""
    shape = RunShape(rows=4, cols=8, island_size=32, surface_sites=S, differentia_bits=b,
                     curation=policy, mode=ASYNC)
    rng = np.random.default_rng(S + b)
    rb = oracle.record_bytes(S, b)
    rec = np.zeros((shape.n_agents, rb), np.uint8)
    on = rng.random((shape.n_agents, S * b)) < rng.uniform(0.001, 0.05, (shape.n_agents, 1))
    rec[:, 8:8 + S * b // 8] = np.packbits(on, axis=1, bitorder="little")
    rec[:, 4:8] = rng.integers(t_lo, t_hi, shape.n_agents).astype(np.uint32).view(np.uint8).reshape(-1, 4)
    g = gpu_run(shape)
    g.load(rec, 0)
    ids = rng.permutation(shape.n_agents)[:300].astype(np.uint32)
    lo, hi = g.mrca_bounds(ids)
    elo, ehi = oracle.mrca_bounds_mixed(rec, ids, policy, S, b)
    assert np.array_equal(hi, ehi), np.nonzero(hi != ehi)[0][:5]
    assert np.array_equal(lo, elo), np.nonzero(lo != elo)[0][:5]

"""Pins for the oracle's asynchronous mode (Sec. 2: migrants are posted and collected without
waiting) on its sequential schedule, and for the lineage tracking the pins rely on.

What fixes the asynchronous mode independently of its own code:
  - with migration off it must be the synchronous GA exactly (the reproduction path);
  - the number of deliveries per (island, direction) follows from the protocol alone (a send
    buffer holds one genome and is refilled only once its genome was taken; every flag is
    tested before anything moves, as the Sec. 2 loop does): within each window an earlier
    neighbour delivers once, a later one delivers what it sent in the previous window, and
    an island that is its own neighbour delivers every second generation (the buffer it
    empties itself tested full, so it is refilled one pass later);
  - on populations it produces, whose counters drift apart, the mixed-counter MRCA bounds
    must bracket the true divergence rank known from the recorded pedigree.
"""
import numpy as np
import pytest

import oracle
from oracle import OracleRun, STEADY, TILTED, HYBRID


def _neighbour(rows, cols, isl, d):
    y, x = divmod(isl, cols)
    if d == 0:
        y = (y - 1) % rows
    elif d == 1:
        y = (y + 1) % rows
    elif d == 2:
        x = (x + 1) % cols
    else:
        x = (x - 1) % cols
    return y * cols + x


@pytest.mark.parametrize("window", [1, 5, 16])
@pytest.mark.parametrize("N,S,b,policy", [(16, 64, 1, STEADY), (32, 32, 8, TILTED)])
def test_no_migration_is_sync(window, N, S, b, policy):
    kw = dict(island_size=N, surface_sites=S, differentia_bits=b, curation=policy,
              migrate_every=0, seed=9, p_ben=0.05, p_del=0.05)
    a = OracleRun(3, 4, **kw)
    s = OracleRun(3, 4, **kw)
    a.step_async(37, window=window)
    s.step(37)
    assert a.generation == s.generation == 37
    assert np.array_equal(a.snapshot(), s.snapshot())


@pytest.mark.parametrize("rows,cols", [(1, 1), (1, 3), (3, 1), (2, 2), (3, 4), (1, 2)])
@pytest.mark.parametrize("window", [1, 3, 8])
def test_arrival_counts(rows, cols, window):
    k = 4
    run = OracleRun(rows, cols, island_size=16, seed=3)
    arr = run.step_async(k * window, window=window)
    for isl in range(rows * cols):
        for d in range(4):
            nb = _neighbour(rows, cols, isl, d)
            want = k if nb < isl else k - 1 if nb > isl else (k * window) // 2
            assert arr[isl, d] == want, (isl, d, nb, arr[isl, d], want)


def test_counters_drift_and_stay_consistent():
    """Arrivals keep their counters, so counters spread.  On the sequential schedule a
    genome never arrives from a neighbour's future (an earlier neighbour sent it at the same
    generation, a later one a window before, the island itself a generation before), so no
    counter exceeds the generation; each birth adds one to the counter and changes the trait
    by at most one."""
    run = OracleRun(1, 9, island_size=16, seed=21, p_ben=0.2, p_del=0.2)
    run.step_async(96, window=8)
    c = run.counters().astype(np.int64)
    t = run.traits().astype(np.int64)
    assert c.max() > c.min()
    assert c.max() <= 96
    assert np.all(np.abs(t) <= c)


def test_tracking_matches_pedigree_sync():
    """Lineage tags against a pedigree rebuilt from the synchronous migrate / reproduce
    outputs (source ids and winner slots)."""
    R, Cc, N, G = 3, 3, 8, 120
    run = OracleRun(R, Cc, island_size=N, seed=13)
    run.track_lineage()
    n = run.n_agents
    parents = []
    for _ in range(G):
        src = run.migrate()
        par = run.reproduce()
        parents.append(src[(np.arange(n) // N) * N + par])
    ids = np.arange(0, n, 3, dtype=np.uint32)
    D = run.divergence(ids)

    def divergence(a, b):
        for t in range(G, 0, -1):
            if a == b:
                return t
            a, b = parents[t - 1][a], parents[t - 1][b]
        return 0

    p = 0
    for i in range(len(ids)):
        for j in range(i + 1, len(ids)):
            assert D[p] == divergence(int(ids[i]), int(ids[j]))
            p += 1


@pytest.mark.parametrize("policy,S,b,window,every", [
    (STEADY, 64, 1, 8, 1), (TILTED, 32, 8, 16, 1), (HYBRID, 64, 1, 4, 1),
    (STEADY, 256, 1, 32, 1), (STEADY, 64, 1, 8, 20), (TILTED, 32, 8, 8, 20)])
def test_async_mrca_brackets_true_divergence(policy, S, b, window, every):
    """A 1 x 9 ring: every island is its own north and south neighbour, so genomes that
    arrive a generation late keep the counters mixed; every = 20: sparse migration keeps
    deep splits (D spread over the whole run)."""
    run = OracleRun(1, 9, island_size=16, surface_sites=S, differentia_bits=b,
                    curation=policy, seed=31 + S, migrate_every=every)
    run.track_lineage()
    run.step_async(400 if every == 1 else 300, window=window)
    rec = run.snapshot()
    cnt = run.counters()
    ids = np.sort(np.random.default_rng(2).choice(run.n_agents, 80, replace=False)).astype(np.uint32)
    assert len(np.unique(cnt[ids])) > 1  # the case the mixed bounds exist for
    lo, hi = oracle.mrca_bounds_mixed(rec, ids, policy, S, b)
    D = run.divergence(ids)
    p = 0
    for i in range(len(ids)):
        for j in range(i + 1, len(ids)):
            Ta, Tb = int(cnt[ids[i]]), int(cnt[ids[j]])
            assert lo[p] <= hi[p] <= min(Ta, Tb)
            assert D[p] <= hi[p], (ids[i], ids[j], D[p], lo[p], hi[p])  # certain
            p += 1


@pytest.mark.parametrize("policy,S,b", [(STEADY, 64, 1), (TILTED, 32, 8), (HYBRID, 64, 1)])
def test_async_mrca_lower_bound_rate(policy, S, b):
    """lo misses (D < lo) only when K retained ranks past the split all matched by chance,
    probability <= 2^(-b K).  Pairs of one population share their ancestors' chance matches,
    so the rate is taken over independent runs: one random pair of agents on different
    islands per seeded run."""
    trials, misses = 160, 0
    for seed in range(trials):
        run = OracleRun(1, 9, island_size=16, surface_sites=S, differentia_bits=b,
                        curation=policy, seed=1000 + seed, migrate_every=10)
        run.track_lineage()
        run.step_async(300, window=8)
        rng = np.random.default_rng(seed)
        isl = rng.choice(9, 2, replace=False)
        ids = np.sort(isl * 16 + rng.integers(0, 16, 2)).astype(np.uint32)
        lo, hi = oracle.mrca_bounds_mixed(run.snapshot(), ids, policy, S, b)
        D = run.divergence(ids)
        assert D[0] <= hi[0]
        misses += int(D[0] < lo[0])
    p_miss = 2.0 ** (-b * oracle.mrca_margin(b))
    assert misses / trials <= p_miss + 4 * np.sqrt(p_miss / trials)


def test_every_counter_value_is_sent():
    """The protocol has no reserved genome value: a member is sent whatever its counter (here
    2^32 - 1 and 7).  On a 1 x 3 ring, every buffer filled in generation 0 is taken in
    generation 1 by island 0 (which runs first) from its east and west neighbours."""
    def first_island_arrivals(counter):
        run = OracleRun(1, 3, island_size=16, seed=8)
        rec = run.snapshot()
        rec[:, 4:8] = np.array([counter], np.uint32).view(np.uint8)
        run.load(rec, 0)
        run.step_async(1, window=1)
        return run.step_async(1, window=1)[0]
    assert first_island_arrivals(0xFFFFFFFF)[2:].tolist() == [1, 1]
    assert first_island_arrivals(7)[2:].tolist() == [1, 1]


def test_own_buffer_tested_before_taking():
    """Sec. 2 order on a 1 x 1 torus (every neighbour is the island itself): generation 0
    tests all four own buffers empty and fills them; generation 1 tests them full, takes all
    four back and leaves them empty (they were full when tested); generation 2 takes nothing
    and refills them."""
    run = OracleRun(1, 1, island_size=16, seed=4)
    per_gen = [run.step_async(1, window=1)[0].tolist() for _ in range(4)]
    assert per_gen == [[0, 0, 0, 0], [1, 1, 1, 1], [0, 0, 0, 0], [1, 1, 1, 1]]


def test_load_clears_mailboxes():
    kw = dict(island_size=16, seed=4)
    a = OracleRun(2, 3, **kw)
    a.step_async(20, window=4)
    snap = a.snapshot()
    a.load(snap, 20)
    a.step_async(12, window=4)
    b = OracleRun(2, 3, **kw)
    b.load(snap, 20)
    b.step_async(12, window=4)
    assert np.array_equal(a.snapshot(), b.snapshot())

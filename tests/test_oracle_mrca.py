"""Pins for the oracle's pairwise MRCA bounds (Fig. 1: post hoc relatedness estimation).

Reading: D = the first rank whose deposit the two lineages drew in separate births (ranks
below D are shared by descent).  The bound [lo, hi] must contain D: hi with certainty,
lo except when K retained ranks at or after D all matched by chance (probability
2^(-b K) < 0.05).  These tests construct lineages whose true D is known -- directly at the
hstrat level, and from the GA's own pedigree -- and check the bracket and the miss rate.
"""
import numpy as np
import pytest

import oracle
from oracle import OracleRun, STEADY, TILTED, HYBRID


def test_margin_values():
    # smallest K with 2^(-bK) < 0.05
    assert oracle.mrca_margin(1) == 5
    assert oracle.mrca_margin(2) == 3
    assert oracle.mrca_margin(4) == 2
    assert oracle.mrca_margin(8) == 1


def _records_from_surfaces(surfs, S, b, T):
    rb = oracle.record_bytes(S, b)
    words = (S * b + 31) // 32
    rec = np.zeros((len(surfs), rb), np.uint8)
    for i, s in enumerate(surfs):
        rec[i, 4:8] = np.array([T], np.uint32).view(np.uint8)
        rec[i, 8:8 + 4 * words] = np.array(s, np.uint32).view(np.uint8)
    return rec


def _fork_trial(policy, S, b, D, T, sites, rng):
    words = (S * b + 31) // 32
    mask = (1 << b) - 1
    base = [int(x) for x in rng.integers(0, 2 ** 32, words)]

    def dep(surf, t):
        site = sites[t]
        if site >= 0:
            pos = site * b
            w, sh = pos // 32, pos % 32
            surf[w] = (surf[w] & ~(mask << sh)) | (int(rng.integers(0, mask + 1)) << sh)

    for t in range(D):
        dep(base, t)
    a, c = list(base), list(base)
    for t in range(D, T):
        dep(a, t)
        dep(c, t)
    rec = _records_from_surfaces([a, c], S, b, T)
    lo, hi = oracle.mrca_bounds(rec, [0, 1], policy, S, b, T)
    return int(lo[0]), int(hi[0])


@pytest.mark.parametrize("policy,S,b,T", [(STEADY, 64, 1, 1000), (STEADY, 256, 1, 3000),
                                          (TILTED, 32, 8, 2000), (HYBRID, 64, 1, 1500),
                                          (STEADY, 16, 2, 800)])
def test_two_lineage_bracket(policy, S, b, T):
    rng = np.random.default_rng(policy * 1000 + S + b)
    sites = [oracle.site(policy, S, t) for t in range(T)]
    trials = 1500
    misses = 0
    for _ in range(trials):
        D = int(rng.integers(0, T + 1))
        lo, hi = _fork_trial(policy, S, b, D, T, sites, rng)
        assert lo <= hi
        assert D <= hi, (D, lo, hi)  # certain
        misses += D < lo
    K = oracle.mrca_margin(b)
    p_miss = 2.0 ** (-b * K)
    assert misses / trials <= p_miss + 4 * np.sqrt(p_miss / trials) + 1e-9


def test_identical_agents_no_mismatch():
    S, b, T = 64, 1, 500
    rng = np.random.default_rng(0)
    s = [int(x) for x in rng.integers(0, 2 ** 32, 2)]
    rec = _records_from_surfaces([s, s], S, b, T)
    lo, hi = oracle.mrca_bounds(rec, [0, 1], STEADY, S, b, T)
    ranks = sorted(r for r in oracle.site_ranks(STEADY, S, T) if r >= 0)
    assert hi[0] == T
    assert lo[0] == ranks[-5] + 1


def test_pair_order_row_major():
    S, b, T = 64, 1, 300
    rng = np.random.default_rng(4)
    surfs = [[int(x) for x in rng.integers(0, 2 ** 32, 2)] for _ in range(6)]
    rec = _records_from_surfaces(surfs, S, b, T)
    ids = [0, 1, 2, 3, 4, 5]
    lo, hi = oracle.mrca_bounds(rec, ids, STEADY, S, b, T)
    p = 0
    for i in range(6):
        for j in range(i + 1, 6):
            l1, h1 = oracle.mrca_bounds(rec, [ids[i], ids[j]], STEADY, S, b, T)
            assert (lo[p], hi[p]) == (l1[0], h1[0])
            p += 1


def test_counter_mismatch_rejected():
    rec = _records_from_surfaces([[1, 2], [3, 4]], 64, 1, 10)
    with pytest.raises(ValueError):
        oracle.mrca_bounds(rec, [0, 1], STEADY, 64, 1, 11)


def test_ga_pedigree_bracket():
    """Run the GA with parent tracking; the true divergence rank of two end-state agents is
    the last generation at which their ancestor chains meet."""
    R, Cc, N, G = 6, 6, 8, 400
    run = OracleRun(R, Cc, island_size=N, tournament_size=5, migrate_every=1, seed=77)
    n = run.n_agents
    parents = []
    for g in range(G):
        src = run.migrate()
        par = run.reproduce()
        child = np.arange(n)
        parents.append(src[(child // N) * N + par])
    rng = np.random.default_rng(5)
    ids = np.sort(rng.choice(n, 120, replace=False)).astype(np.uint32)
    lo, hi = run.mrca_bounds(ids)

    def divergence(a, b):
        x, y = a, b
        for t in range(G, 0, -1):
            if x == y:
                return t
            x, y = parents[t - 1][x], parents[t - 1][y]
        return 0

    p = 0
    misses = 0
    for i in range(len(ids)):
        for j in range(i + 1, len(ids)):
            D = divergence(int(ids[i]), int(ids[j]))
            assert lo[p] <= hi[p]
            assert D <= hi[p], (ids[i], ids[j], D, lo[p], hi[p])
            misses += D < lo[p]
            p += 1
    assert misses / p < 0.10


def test_mixed_equals_uniform_when_counters_equal():
    S, b, T = 64, 1, 700
    rng = np.random.default_rng(8)
    surfs = [[int(x) for x in rng.integers(0, 2 ** 32, 2)] for _ in range(12)]
    rec = _records_from_surfaces(surfs, S, b, T)
    ids = list(range(12))
    lo, hi = oracle.mrca_bounds(rec, ids, STEADY, S, b, T)
    lo2, hi2 = oracle.mrca_bounds_mixed(rec, ids, STEADY, S, b)
    assert np.array_equal(lo, lo2) and np.array_equal(hi, hi2)


def _fork_trial_mixed(policy, S, b, D, Ta, Tb, sites, rng):
    """Lineages split at D, then run to different counters Ta and Tb (as after asynchronous
    migration); returns the mixed-counter bounds of the two end agents."""
    words = (S * b + 31) // 32
    mask = (1 << b) - 1
    base = [int(x) for x in rng.integers(0, 2 ** 32, words)]

    def dep(surf, t):
        site = sites[t]
        if site >= 0:
            pos = site * b
            w, sh = pos // 32, pos % 32
            surf[w] = (surf[w] & ~(mask << sh)) | (int(rng.integers(0, mask + 1)) << sh)

    for t in range(D):
        dep(base, t)
    a, c = list(base), list(base)
    for t in range(D, Ta):
        dep(a, t)
    for t in range(D, Tb):
        dep(c, t)
    rb = oracle.record_bytes(S, b)
    rec = np.zeros((2, rb), np.uint8)
    for i, (s, T) in enumerate(((a, Ta), (c, Tb))):
        rec[i, 4:8] = np.array([T], np.uint32).view(np.uint8)
        rec[i, 8:8 + 4 * words] = np.array(s, np.uint32).view(np.uint8)
    lo, hi = oracle.mrca_bounds_mixed(rec, [0, 1], policy, S, b)
    return int(lo[0]), int(hi[0])


@pytest.mark.parametrize("policy,S,b", [(STEADY, 64, 1), (TILTED, 32, 8), (HYBRID, 64, 1)])
def test_mixed_counter_bracket(policy, S, b):
    rng = np.random.default_rng(S * 7 + b)
    T_max = 1200
    sites = [oracle.site(policy, S, t) for t in range(T_max)]
    trials, misses = 1200, 0
    for _ in range(trials):
        Ta = int(rng.integers(600, T_max))
        Tb = int(np.clip(Ta + rng.integers(-40, 41), 1, T_max - 1))
        D = int(rng.integers(0, min(Ta, Tb) + 1))
        lo, hi = _fork_trial_mixed(policy, S, b, D, Ta, Tb, sites, rng)
        assert lo <= hi <= min(Ta, Tb)
        assert D <= hi, (D, lo, hi, Ta, Tb)
        misses += D < lo
    p_miss = 2.0 ** (-b * oracle.mrca_margin(b))
    assert misses / trials <= p_miss + 4 * np.sqrt(p_miss / trials) + 1e-9

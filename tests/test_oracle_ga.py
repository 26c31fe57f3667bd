"""Pins for the oracle's synchronous island GA (Sec. 2 step order, Sec. 3 parameters).

The GA has no closed form, so these tests check what the paper and probability theory fix:
special cases with a known outcome, the exact distribution of a tournament winner, mutation
frequencies within binomial bounds, migration conservation on the torus, independence of
islands without migration, determinism and bit-exact resume.
"""
import numpy as np
import pytest

from oracle import OracleRun, STEADY, TILTED, HYBRID


def tagged_records(run, traits):
    rec = run.snapshot()
    rec[:, 0:4] = np.asarray(traits, np.int32).view(np.uint8).reshape(-1, 4)
    return rec


def test_no_mutation_traits_stay_zero():
    run = OracleRun(8, 8, p_ben=0.0, p_del=0.0)
    run.step(60)
    assert (run.traits() == 0).all()
    assert (run.counters() == 60).all()


def test_counters_track_generations():
    run = OracleRun(4, 6, island_size=16, migrate_every=3)
    for g in (1, 5, 17):
        run.step(g)
    assert (run.counters() == 23).all()
    assert run.generation == 23


def test_founder_is_shared():
    run = OracleRun(3, 5, surface_sites=256, differentia_bits=1)
    s = run.surfaces()
    assert (s == s[0]).all()
    assert s[0].any()


def test_tournament_winner_distribution():
    """With distinct traits, no mutation and no migration, a child's parent is the best of n
    uniform draws with replacement: P(parent rank <= q) = (q/N)^n for ranks 1..N."""
    N, n = 32, 5
    run = OracleRun(64, 64, island_size=N, tournament_size=n, p_ben=0, p_del=0,
                    migrate_every=0, seed=7)
    rng = np.random.default_rng(1)
    perm = np.concatenate([rng.permutation(N) for _ in range(64 * 64)])
    run.load(tagged_records(run, perm), 0)
    run.step(1)
    ranks = run.traits() + 1  # trait value = rank - 1
    m = ranks.size
    emp = np.array([(ranks <= q).mean() for q in range(1, N + 1)])
    exact = (np.arange(1, N + 1) / N) ** n
    # Kolmogorov-Smirnov style band
    assert np.abs(emp - exact).max() < 1.8 / np.sqrt(m)


def test_tournament_size_one_is_uniform_resampling():
    N = 16
    run = OracleRun(32, 32, island_size=N, tournament_size=1, p_ben=0, p_del=0,
                    migrate_every=0, seed=3)
    run.load(tagged_records(run, np.tile(np.arange(N), 32 * 32)), 0)
    par = run.reproduce()
    counts = np.bincount(par, minlength=N)
    expect = par.size / N
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < 50  # 15 dof; p ~ 1e-5 threshold


def test_ties_broken_uniformly():
    """All traits equal: every candidate ties, so the winner must be uniform (Sec. 2: ties
    broken randomly)."""
    N = 32
    run = OracleRun(32, 32, island_size=N, tournament_size=5, p_ben=0, p_del=0,
                    migrate_every=0, seed=11)
    par = run.reproduce()
    counts = np.bincount(par, minlength=N)
    expect = par.size / N
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < 80  # 31 dof


@pytest.mark.parametrize("p_ben,p_del", [(0.01, 0.01), (0.0, 0.01), (0.05, 0.2)])
def test_mutation_frequencies(p_ben, p_del):
    run = OracleRun(64, 64, island_size=32, tournament_size=1, p_ben=p_ben, p_del=p_del,
                    migrate_every=0, seed=5)
    run.step(1)
    t = run.traits()
    m = t.size
    for value, p in ((1, p_ben), (-1, p_del)):
        k = (t == value).sum()
        sd = np.sqrt(m * p * (1 - p)) + 1e-9
        assert abs(k - m * p) <= 5 * sd + 1, (value, k, m * p)
    assert set(np.unique(t)) <= {-1, 0, 1}


def test_purifying_never_improves():
    run = OracleRun(8, 8, p_ben=0.0, p_del=0.05, seed=9)
    run.step(200)
    assert run.traits().max() <= 0
    assert run.traits().min() < 0


def test_migration_conservation_and_directions():
    R, Cc, N = 5, 7, 8
    run = OracleRun(R, Cc, island_size=N, migrate_every=1, seed=13)
    ids = np.arange(R * Cc * N, dtype=np.int32)
    run.load(tagged_records(run, ids), 0)
    src = run.migrate()
    traits = run.traits()
    assert (traits == src.astype(np.int32)).all()
    for isl in range(R * Cc):
        y, x = divmod(isl, Cc)
        slots = np.arange(isl * N, (isl + 1) * N)
        moved = slots[src[slots] != slots]
        assert len(moved) == 4  # four distinct slots replaced
        src_isl = sorted(int(src[s]) // N for s in moved)
        expect = sorted([((y - 1) % R) * Cc + x, ((y + 1) % R) * Cc + x,
                         y * Cc + (x + 1) % Cc, y * Cc + (x - 1) % Cc])
        assert src_isl == expect


def test_migration_draws_uniform():
    R, Cc, N = 32, 32, 16
    run = OracleRun(R, Cc, island_size=N, migrate_every=1, seed=17)
    src = run.migrate()
    moved = np.nonzero(src != np.arange(src.size))[0]
    slot_counts = np.bincount(moved % N, minlength=N)
    src_counts = np.bincount(src[moved] % N, minlength=N)
    for counts in (slot_counts, src_counts):
        e = counts.sum() / N
        assert ((counts - e) ** 2 / e).sum() < 45  # 15 dof


def test_small_island_migration_slots_distinct():
    run = OracleRun(3, 3, island_size=4, migrate_every=1, seed=2)
    for _ in range(20):
        src = run.migrate()
        for isl in range(9):
            sl = np.arange(isl * 4, isl * 4 + 4)
            assert (src[sl] != sl).all()  # all four slots replaced, by distinct arrivals
        run.reproduce()


def test_islands_independent_without_migration():
    a = OracleRun(3, 4, island_size=16, migrate_every=0, seed=21)
    b = OracleRun(1, 4, island_size=16, migrate_every=0, seed=21)
    a.step(40)
    b.step(40)
    assert (a.snapshot()[:4 * 16] == b.snapshot()).all()


def test_migration_couples_islands():
    a = OracleRun(3, 4, island_size=16, migrate_every=1, seed=21)
    b = OracleRun(1, 4, island_size=16, migrate_every=1, seed=21)
    a.step(40)
    b.step(40)
    assert not (a.snapshot()[:4 * 16] == b.snapshot()).all()


@pytest.mark.parametrize("curation,S,b", [(STEADY, 64, 1), (TILTED, 32, 8),
                                          (HYBRID, 64, 1), (STEADY, 256, 1)])
def test_deterministic_and_resumable(curation, S, b):
    kw = dict(island_size=16, surface_sites=S, differentia_bits=b, curation=curation,
              migrate_every=4, seed=99, run_id=3)
    a = OracleRun(4, 4, **kw)
    a.step(37)
    b_ = OracleRun(4, 4, **kw)
    b_.step(20)
    snap = b_.snapshot()
    c = OracleRun(4, 4, **kw)
    c.load(snap, 20)
    c.step(17)
    assert (a.snapshot() == c.snapshot()).all()
    d = OracleRun(4, 4, **{**kw, "run_id": 4})
    d.step(37)
    assert not (a.snapshot() == d.snapshot()).all()


def test_threads_match_serial():
    a = OracleRun(16, 16, seed=5, threads=1)
    b = OracleRun(16, 16, seed=5, threads=4)
    a.step(30)
    b.step(30)
    assert (a.snapshot() == b.snapshot()).all()


def test_deposit_writes_only_the_curated_site():
    """Between generation g and g+1 each child's surface differs from its parent's only at
    the site the curation rule names for rank g (checked via the winner slots)."""
    import oracle as O
    run = OracleRun(4, 4, island_size=8, migrate_every=0, seed=31, surface_sites=32,
                    differentia_bits=8, curation=TILTED)
    run.step(50)
    before = run.surfaces().copy()
    par = run.reproduce()
    after = run.surfaces()
    site = O.site(TILTED, 32, 50)
    byte_before = before.view(np.uint8)
    byte_after = after.view(np.uint8)
    N = 8
    for a in range(run.n_agents):
        parent = (a // N) * N + int(par[a])
        diff = np.nonzero(byte_before[parent] != byte_after[a])[0]
        assert set(diff.tolist()) <= {site}


def test_invalid_configs_rejected():
    with pytest.raises(ValueError):
        OracleRun(4, 4, island_size=24)
    with pytest.raises(ValueError):
        OracleRun(4, 4, tournament_size=9)
    with pytest.raises(ValueError):
        OracleRun(4, 4, p_ben=0.7, p_del=0.6)
    with pytest.raises(ValueError):
        OracleRun(4, 4, surface_sites=512, differentia_bits=1)

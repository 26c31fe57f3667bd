"""GPU MRCA-bound kernels versus the oracle, exact on every (lo, hi) pair."""
import numpy as np
import pytest

from gpu_util import gpu_run, oracle_for
from paper_2405_03605_gb300.workloads import RunShape, SMALL_TORUS, variant_shapes, \
    sample_agent_ids

pytestmark = pytest.mark.gpu


def both(shape, gens, n_ids, seed=1):
    g = gpu_run(shape)
    g.step(gens)
    g.sync()
    o = oracle_for(shape)
    o.step(gens)
    ids = sample_agent_ids(shape.n_agents, n_ids, seed=seed)
    return g, o, ids


@pytest.mark.parametrize("gens", [0, 1, 5, 63, 64, 65, 1000])
def test_small_torus_pairs(gens):
    g, o, ids = both(SMALL_TORUS, gens, 700)
    lo, hi = g.mrca_bounds(ids)
    elo, ehi = o.mrca_bounds(ids)
    assert np.array_equal(lo, elo)
    assert np.array_equal(hi, ehi)
    assert (lo <= hi).all() and (hi <= gens).all()


@pytest.mark.parametrize("name", ["steady256x1", "tilted32x8", "hybrid64x1"])
def test_variant_pairs(name):
    shape = variant_shapes(32)[name].with_(rows=6, cols=8)
    g, o, ids = both(shape, 700, 500, seed=3)
    lo, hi = g.mrca_bounds(ids)
    elo, ehi = o.mrca_bounds(ids)
    assert np.array_equal(lo, elo)
    assert np.array_equal(hi, ehi)


@pytest.mark.parametrize("S,b,policy,n_ids", [
    (16, 4, "TILTED", 1500), (32, 2, "STEADY", 777), (8, 8, "HYBRID", 301), (4, 1, "STEADY", 64),
    (64, 1, "STEADY", 4096),
])
def test_narrow_strings(S, b, policy, n_ids):
    """Strings of at most 64 bits (the two-launch path): every curation policy, differentia
    widths 1 to 8, samples spanning several pack blocks, and the full 4,096-agent sample."""
    from paper_2405_03605_gb300 import workloads
    shape = RunShape(rows=16, cols=10, surface_sites=S, differentia_bits=b,
                     curation=getattr(workloads, policy), seed=S + b)
    g, o, ids = both(shape, 900, n_ids, seed=S)
    lo, hi = g.mrca_bounds(ids)
    elo, ehi = o.mrca_bounds(ids)
    assert np.array_equal(lo, elo)
    assert np.array_equal(hi, ehi)


def test_device_entry_point_matches_host():
    import torch
    shape = RunShape(rows=8, cols=8, seed=9)
    g, o, ids = both(shape, 200, 333)
    d_ids = torch.from_numpy(ids.view(np.int32)).cuda()
    lo, hi = g.mrca_bounds_device(d_ids)
    g.sync()
    hlo, hhi = g.mrca_bounds(ids)
    assert np.array_equal(lo.cpu().numpy().view(np.uint32), hlo)
    assert np.array_equal(hi.cpu().numpy().view(np.uint32), hhi)


def test_two_samples_and_errors():
    from paper_2405_03605_gb300 import ga
    shape = RunShape(rows=2, cols=2, seed=2)
    g, o, _ = both(shape, 30, 2)
    lo, hi = g.mrca_bounds(np.array([3, 100], np.uint32))
    elo, ehi = o.mrca_bounds(np.array([3, 100], np.uint32))
    assert (lo[0], hi[0]) == (elo[0], ehi[0])
    with pytest.raises(ga.GaError):
        g.mrca_bounds(np.array([0, shape.n_agents], np.uint32))
    with pytest.raises(ga.GaError):
        g.mrca_bounds(np.array([0], np.uint32))


def test_outputs_at_any_4_byte_alignment():
    """Output buffers offset by one element from an aligned allocation (4-byte aligned only):
    the same bounds as the oracle."""
    import torch
    g, o, ids = both(SMALL_TORUS, 300, 513, seed=4)
    n = ids.size
    pairs = n * (n - 1) // 2
    dev_ids = torch.from_numpy(np.ascontiguousarray(ids, np.uint32).view(np.int32)).cuda()
    lo_buf = torch.zeros(pairs + 1, dtype=torch.int32, device="cuda")
    hi_buf = torch.zeros(pairs + 1, dtype=torch.int32, device="cuda")
    lo, hi = g.mrca_bounds_device(dev_ids, lo_buf[1:], hi_buf[1:])
    g.sync()
    elo, ehi = o.mrca_bounds(ids)
    assert np.array_equal(lo.cpu().numpy().view(np.uint32), elo)
    assert np.array_equal(hi.cpu().numpy().view(np.uint32), ehi)


@pytest.mark.parametrize("n_ids", [2, 5, 333, 1500])
def test_output_alignment(n_ids):
    """(lo, hi) arrays at any 4-byte offset (not only the 256-byte boundaries of fresh
    allocations): the bounds equal the oracle's and nothing outside the n(n-1)/2 pairs is
    written."""
    import torch
    shape = RunShape(rows=8, cols=8, seed=13)
    g, o, ids = both(shape, 300, n_ids, seed=n_ids)
    d_ids = torch.from_numpy(ids.view(np.int32)).cuda()
    pairs = n_ids * (n_ids - 1) // 2
    elo, ehi = o.mrca_bounds(ids)
    for off_lo, off_hi in ((0, 0), (1, 1), (2, 0), (0, 3), (3, 2)):
        lo_b = torch.full((pairs + 8,), -1, dtype=torch.int32, device="cuda")
        hi_b = torch.full((pairs + 8,), -1, dtype=torch.int32, device="cuda")
        lo, hi = lo_b[off_lo:off_lo + pairs], hi_b[off_hi:off_hi + pairs]
        g.mrca_bounds_device(d_ids, lo, hi)
        g.sync()
        assert np.array_equal(lo.cpu().numpy().view(np.uint32), elo)
        assert np.array_equal(hi.cpu().numpy().view(np.uint32), ehi)
        for buf, off in ((lo_b, off_lo), (hi_b, off_hi)):
            assert bool((buf[:off] == -1).all()) and bool((buf[off + pairs:] == -1).all())

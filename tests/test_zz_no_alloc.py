"""ga_mrca_bounds_noalloc, the MRCA entry point for callers that cannot allocate device
memory (its scratch is a fixed array inside the library), against the allocating entry
point ga_mrca_bounds_device on the same inputs, exact on every (lo, hi) pair, over two calls
in a row; and against the oracle's bounds on the same records, including counters past
16,384 and the largest layout the fixed array is sized for (256 one-bit sites, 4,096
sampled agents).  This file is collected last so that a failure here stops a -x run only
after every other test has run."""
import numpy as np
import pytest

import oracle
from gpu_util import gpu_run
from paper_2405_03605_gb300.workloads import RunShape, sample_agent_ids

pytestmark = pytest.mark.gpu


def _device_u32(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


def test_noalloc_matches_allocating_entry_point():
    import torch
    from paper_2405_03605_gb300 import ga
    cases = [
        (RunShape(rows=16, cols=12, seed=21, run_id=5), 400, 1500, 11),
        (RunShape(rows=8, cols=8, island_size=16, surface_sites=32, differentia_bits=8,
                  curation=ga.TILTED, seed=22), 250, 700, 12),
    ]
    for shape, gens, n, seed in cases:  # two calls in a row, different sizes and layouts
        run = gpu_run(shape)
        run.step(gens)
        run.sync()
        ids = _device_u32(sample_agent_ids(shape.n_agents, n, seed=seed))
        ref_lo, ref_hi = run.mrca_bounds_device(ids)
        run.sync()
        pairs = n * (n - 1) // 2
        lo = torch.full((pairs,), -1, dtype=torch.int32, device="cuda")
        hi = torch.full((pairs,), -1, dtype=torch.int32, device="cuda")
        ptr, _ = run.population_ptr()
        ga.mrca_bounds_noalloc(ptr, run.record_bytes, shape.n_agents, shape.curation,
                               shape.surface_sites, shape.differentia_bits, gens, ids, lo, hi,
                               stream=run.stream)
        assert torch.equal(lo, ref_lo) and torch.equal(hi, ref_hi)
        run.close()


def _noalloc(run, shape, T, ids):
    import torch
    from paper_2405_03605_gb300 import ga
    n = ids.numel()
    pairs = n * (n - 1) // 2
    lo = torch.full((pairs,), -1, dtype=torch.int32, device="cuda")
    hi = torch.full((pairs,), -1, dtype=torch.int32, device="cuda")
    ptr, _ = run.population_ptr()
    ga.mrca_bounds_noalloc(ptr, run.record_bytes, shape.n_agents, shape.curation,
                           shape.surface_sites, shape.differentia_bits, T, ids, lo, hi,
                           stream=run.stream)
    return lo, hi


def _sparse_surfaces(rec, S, b, seed):
    """Surfaces whose differentiae are mostly zero, each agent with its own density, so the
    first mismatch of a pair falls anywhere from the oldest retained rank to the newest; a
    tenth of the agents copy another agent's surface (pairs without a mismatch)."""
    rng = np.random.default_rng(seed)
    n = rec.shape[0]
    bits = S * b
    dens = rng.uniform(0.0005, 0.08, size=n)
    on = rng.random((n, bits)) < dens[:, None]
    copy = rng.random(n) < 0.1
    on[copy] = on[rng.integers(0, n, copy.sum())]
    words = np.packbits(on, axis=1, bitorder="little").view(np.uint32)
    rec = rec.copy()
    rec[:, 8:8 + 4 * words.shape[1]] = words.view(np.uint8)
    return rec


@pytest.mark.parametrize("policy,S,b,T", [
    (0, 64, 1, 20000),          # steady, past the 16,384 that one launch once replayed
    (1, 32, 8, 20000),          # tilted, 8-bit differentiae
    (2, 256, 1, 16385),         # hybrid, the largest string the fixed array holds
    (0, 256, 1, 3_000_000),     # a counter far past any replay
])
def test_noalloc_matches_oracle_at_large_counters(policy, S, b, T):
    """Records loaded with every counter at T: noalloc, the allocating entry point and the
    oracle (its own site-rank replay) agree on every pair, over 4,096 sampled agents."""
    import torch
    shape = RunShape(rows=8, cols=16, island_size=32, surface_sites=S, differentia_bits=b,
                     curation=policy, seed=31 + S, run_id=b)
    run = gpu_run(shape)
    run.sync()
    rec = _sparse_surfaces(run.snapshot(), S, b, seed=T % 1000)
    rec[:, 4:8] = np.array([T], np.uint32).view(np.uint8)
    run.load(rec, T)
    ids_h = sample_agent_ids(shape.n_agents, 4096, seed=5)
    ids = _device_u32(ids_h)
    ref_lo, ref_hi = run.mrca_bounds_device(ids)
    run.sync()
    lo, hi = _noalloc(run, shape, T, ids)
    assert torch.equal(lo, ref_lo) and torch.equal(hi, ref_hi)
    elo, ehi = oracle.mrca_bounds(rec, ids_h, policy, S, b, T)
    glo = lo.cpu().numpy().view(np.uint32)
    ghi = hi.cpu().numpy().view(np.uint32)
    assert np.array_equal(ghi, ehi), np.nonzero(ghi != ehi)[0][:5]
    assert np.array_equal(glo, elo), np.nonzero(glo != elo)[0][:5]
    assert len(np.unique(ehi)) > 20  # mismatches spread over many retained ranks
    run.close()


def test_noalloc_hybrid_256_stepped_past_16384():
    """A hybrid 256-site run stepped 16,400 generations (counters produced by the GA, not
    loaded), 4,096 sampled agents: noalloc equals the allocating entry point exactly."""
    import torch
    shape = RunShape(rows=8, cols=16, island_size=32, surface_sites=256, differentia_bits=1,
                     curation=2, seed=77, run_id=3)
    run = gpu_run(shape)
    run.step(16400)
    run.sync()
    ids = _device_u32(sample_agent_ids(shape.n_agents, 4096, seed=6))
    ref_lo, ref_hi = run.mrca_bounds_device(ids)
    run.sync()
    lo, hi = _noalloc(run, shape, 16400, ids)
    assert torch.equal(lo, ref_lo) and torch.equal(hi, ref_hi)
    run.close()


def test_noalloc_rejects_oversized_and_bad_counters():
    import torch
    from paper_2405_03605_gb300 import ga
    shape = RunShape(rows=4, cols=40, seed=3)  # 5,120 agents
    run = gpu_run(shape)
    run.step(20)
    run.sync()
    ptr, _ = run.population_ptr()
    big = _device_u32(np.arange(4097))
    out_lo = torch.empty(4097 * 4096 // 2, dtype=torch.int32, device="cuda")
    out_hi = torch.empty(4097 * 4096 // 2, dtype=torch.int32, device="cuda")
    with pytest.raises(ga.GaError) as e:
        ga.mrca_bounds_noalloc(ptr, 16, shape.n_agents, 0, 64, 1, 20, big, out_lo, out_hi,
                               stream=run.stream)
    assert e.value.code == -1
    ids = _device_u32([1, 2, 3])
    lo = torch.empty(3, dtype=torch.int32, device="cuda")
    hi = torch.empty(3, dtype=torch.int32, device="cuda")
    with pytest.raises(ga.GaError) as e:  # counters are 20, not 21
        ga.mrca_bounds_noalloc(ptr, 16, shape.n_agents, 0, 64, 1, 21, ids, lo, hi,
                               stream=run.stream)
    assert e.value.code == -5
    # the binding refuses outputs too small for n (n - 1) / 2 pairs, shared or host tensors
    with pytest.raises(ValueError):
        ga.mrca_bounds_noalloc(ptr, 16, shape.n_agents, 0, 64, 1, 20, ids, lo[:2], hi,
                               stream=run.stream)
    with pytest.raises(ValueError):
        ga.mrca_bounds_noalloc(ptr, 16, shape.n_agents, 0, 64, 1, 20, ids, lo, lo,
                               stream=run.stream)
    with pytest.raises(ValueError):
        ga.mrca_bounds_noalloc(ptr, 16, shape.n_agents, 0, 64, 1, 20, ids, lo.cpu(), hi,
                               stream=run.stream)
    # and a valid call after the refused ones still works
    ga.mrca_bounds_noalloc(ptr, 16, shape.n_agents, 0, 64, 1, 20, ids, lo, hi,
                           stream=run.stream)
    run.close()

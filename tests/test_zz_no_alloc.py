"""ga_mrca_bounds_noalloc, the MRCA entry point for callers that cannot allocate device
memory (its scratch is a fixed array inside the library), against the allocating entry
point ga_mrca_bounds_device on the same inputs, exact on every (lo, hi) pair, over two calls
in a row.  This file is collected last so that a failure here stops a -x run only after
every other test has run."""
import numpy as np
import pytest

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


def test_noalloc_rejects_oversized_and_bad_counters():
    import torch
    from paper_2405_03605_gb300 import ga
    shape = RunShape(rows=4, cols=40, seed=3)  # 5,120 agents
    run = gpu_run(shape)
    run.step(20)
    run.sync()
    ptr, _ = run.population_ptr()
    big = _device_u32(np.arange(4097))
    out = torch.empty(4097 * 4096 // 2, dtype=torch.int32, device="cuda")
    with pytest.raises(ga.GaError) as e:
        ga.mrca_bounds_noalloc(ptr, 16, shape.n_agents, 0, 64, 1, 20, big, out, out,
                               stream=run.stream)
    assert e.value.code == -1
    ids = _device_u32([1, 2, 3])
    lo = torch.empty(3, dtype=torch.int32, device="cuda")
    with pytest.raises(ga.GaError) as e:  # counters are 20, not 21
        ga.mrca_bounds_noalloc(ptr, 16, shape.n_agents, 0, 64, 1, 21, ids, lo, lo,
                               stream=run.stream)
    assert e.value.code == -5
    run.close()

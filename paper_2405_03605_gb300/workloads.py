"""Seeded synthetic workloads: run configurations and agent samples.

This module holds only workload shapes and seeded draws of inputs (which agents to sample,
the parameters of batched and served runs).  It contains none of the GA's arithmetic, so
both the CUDA path and the CPU oracle's tests may use it.

Shapes follow the paper's runs (Sec. 3: 32 genomes per island, tournament size 5,
purifying-only versus adaptive treatments, lattices up to 750x750, 10k sampled end-state
agents) scaled to the workloads this library is measured on.
"""
from dataclasses import dataclass, asdict, replace
import math

import numpy as np

STEADY, TILTED, HYBRID = 0, 1, 2
MODEL_TRAIT, MODEL_FITNESS = 0, 1
SYNC, ASYNC, ASYNC_SEQUENTIAL = 0, 1, 2


@dataclass(frozen=True)
class RunShape:
    rows: int
    cols: int
    island_size: int = 32
    tournament_size: int = 5
    p_ben: float = 0.01
    p_del: float = 0.01
    surface_sites: int = 64
    differentia_bits: int = 1
    curation: int = STEADY
    migrate_every: int = 1
    seed: int = 42
    run_id: int = 0
    generations: int = 1000
    model: int = MODEL_TRAIT
    effect_scale: float = 1.0
    mode: int = SYNC
    async_window: int = 1  # generations per launch in the asynchronous modes

    @property
    def n_islands(self):
        return self.rows * self.cols

    @property
    def n_agents(self):
        return self.rows * self.cols * self.island_size

    @property
    def record_bytes(self):
        words = (self.surface_sites * self.differentia_bits + 31) // 32
        return (8 + 4 * words + 15) // 16 * 16

    def kwargs(self):
        d = asdict(self)
        for k in ("generations", "mode", "async_window"):
            d.pop(k)
        return d

    def with_(self, **kw):
        return replace(self, **kw)


# 32x32 torus of 32-agent islands, 16-byte genome, 1,000 generations.
SMALL_TORUS = RunShape(rows=32, cols=32, generations=1000)

# Paper-scale: 512x1024 islands x 32 agents = 16,777,216 agents, 10,000 generations, an
# adaptive run (p_ben = 0.01) and a purifying-only run (p_ben = 0), then pairwise MRCA
# bounds over 4,096 sampled end-state agents.
PAPER_ADAPTIVE = RunShape(rows=512, cols=1024, p_ben=0.01, run_id=0, generations=10000)
PAPER_PURIFYING = RunShape(rows=512, cols=1024, p_ben=0.0, run_id=1, generations=10000)
PAPER_SAMPLE = 4096


# The paper's own treatments (Sec. 3): 128-bit genome whose first 32 bits are a float
# fitness; purifying-only runs lose fitness by a normally distributed amount at 33% of births,
# adaptive runs also gain by a normally distributed amount at 0.3% of births; tournament 5.
PAPER_FITNESS_PURIFYING = RunShape(rows=512, cols=1024, p_ben=0.0, p_del=0.33, run_id=2,
                                   generations=10000, model=MODEL_FITNESS)
PAPER_FITNESS_ADAPTIVE = RunShape(rows=512, cols=1024, p_ben=0.003, p_del=0.33, run_id=3,
                                  generations=10000, model=MODEL_FITNESS)


def variant_shapes(island_size=32, migrate_every=1, generations=5000):
    """4,194,304-agent surface/genome variants: 256-site 1-bit steady (48 B record),
    32-site 8-bit tilted (48 B record) and 64-site 1-bit hybrid (16 B record)."""
    rows = 4194304 // (1024 * island_size)
    base = RunShape(rows=rows, cols=1024, island_size=island_size,
                    migrate_every=migrate_every, generations=generations)
    return {
        "steady256x1": base.with_(surface_sites=256, differentia_bits=1, curation=STEADY),
        "tilted32x8": base.with_(surface_sites=32, differentia_bits=8, curation=TILTED),
        "hybrid64x1": base.with_(surface_sites=64, differentia_bits=1, curation=HYBRID),
    }


def sample_agent_ids(n_agents, n, seed=42):
    """n distinct agent ids drawn uniformly without replacement, sorted ascending."""
    if n > n_agents:
        raise ValueError("sample larger than population")
    rng = np.random.default_rng(seed)
    ids = rng.choice(n_agents, size=n, replace=False)
    return np.sort(ids).astype(np.uint32)


def batch_shapes(n_runs=256, seed=42, generations=2000):
    """Heterogeneous replicate runs: grid sides from {16,...,256}, island size from
    {16,32,64}, p_ben and p_del log-uniform on [1e-4, 1e-1], tournament size 2..8."""
    rng = np.random.default_rng(seed)
    sides = np.array([16, 32, 64, 128, 256])
    out = []
    for r in range(n_runs):
        rows = int(rng.choice(sides))
        cols = int(rng.choice(sides))
        n_isl = int(rng.choice([16, 32, 64]))
        p_ben = float(10 ** rng.uniform(-4, -1))
        p_del = float(10 ** rng.uniform(-4, -1))
        tsize = int(rng.integers(2, 9))
        out.append(RunShape(rows=rows, cols=cols, island_size=n_isl, tournament_size=tsize,
                            p_ben=p_ben, p_del=p_del, run_id=r, generations=generations))
    return out


def serve_trace(n_requests=1000, rate_hz=50.0, seed=42):
    """Poisson arrivals of GA runs: total agents log-uniform on [1e4, 1e7] mapped onto
    32-agent islands on a near-square torus, generations log-uniform on [100, 10000]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for r in range(n_requests):
        t += float(rng.exponential(1.0 / rate_hz))
        agents = 10 ** rng.uniform(4, 7)
        islands = max(1, int(round(agents / 32)))
        rows = max(1, int(math.sqrt(islands)))
        cols = max(1, islands // rows)
        gens = int(round(10 ** rng.uniform(2, 4)))
        sites = int(rng.choice([64, 256]))
        reqs.append((t, RunShape(rows=rows, cols=cols, surface_sites=sites, run_id=r,
                                 generations=gens)))
    return reqs

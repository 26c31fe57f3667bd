"""The treatment contrast of Sec. 3: purifying-only runs keep deeper genealogies than
adaptive runs, where beneficial mutations sweep and recent common ancestry dominates.  The
paper measures it with phylometrics of reconstructed trees; here the stand-in is the mean
pairwise time since divergence bounded by the MRCA estimate (T - hi, a lower bound on how
long ago the two lineages split), which must be larger under purifying selection."""
import numpy as np

from oracle import OracleRun
from paper_2405_03605_gb300.workloads import sample_agent_ids


def mean_depth(p_ben, seed):
    run = OracleRun(8, 8, island_size=32, tournament_size=5, p_ben=p_ben, p_del=0.01,
                    seed=seed, run_id=int(p_ben > 0), threads=4)
    run.step(600)
    ids = sample_agent_ids(run.n_agents, 200, seed=seed)
    lo, hi = run.mrca_bounds(ids)
    return float(np.mean(600 - hi.astype(np.int64)))


def test_purifying_deeper_than_adaptive():
    for seed in (1, 2):
        adaptive = mean_depth(0.01, seed)
        purifying = mean_depth(0.0, seed)
        assert purifying > adaptive + 50, (seed, purifying, adaptive)

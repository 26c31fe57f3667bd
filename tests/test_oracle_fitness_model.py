"""Pins for the float-fitness treatments (Sec. 3: deleterious mutations at 33% of births and,
in adaptive runs, beneficial ones at 0.3%, each by a normally distributed amount): the
oracle's single-precision Box-Muller pieces against the mathematics, the deviates against the
standard normal distribution, and the mutation process against its probabilities."""
import math

import numpy as np
import pytest

import oracle
from oracle import OracleRun, MODEL_FITNESS


def test_unit_log_accuracy():
    for k in list(range(0, 5000)) + list(range(2 ** 24 - 5000, 2 ** 24, 7)) + \
            [int(x) for x in np.linspace(0, 2 ** 24 - 1, 3000)]:
        x = (k + 1) / 2 ** 24
        got = oracle.unit_log(np.float32(x))
        assert abs(got - math.log(x)) <= 1e-6 * max(1.0, abs(math.log(x))), (k, got)


def test_turn_cos_accuracy():
    for k in [int(x) for x in np.linspace(0, 2 ** 24 - 1, 20000)] + [0, 1 << 22, 1 << 23, 3 << 22]:
        got = oracle.turn_cos(k)
        assert abs(got - math.cos(2 * math.pi * k / 2 ** 24)) <= 3e-7, (k, got)


def test_normal_deviates_are_standard_normal():
    n = 60000
    z = np.empty(n)
    for i in range(n):
        w = oracle.philox4x32_10([i, 11, 7 | (3 << 16), 0], [42, 0])
        z[i] = oracle.normal(int(w[0]), int(w[1]))
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    zs = np.sort(z)
    cdf = np.array([0.5 * (1 + math.erf(v / math.sqrt(2))) for v in zs])
    ks = np.max(np.maximum(np.arange(1, n + 1) / n - cdf, cdf - np.arange(n) / n))
    assert ks < 1.63 / math.sqrt(n)  # 1% Kolmogorov-Smirnov critical value


def fitness_run(**kw):
    base = dict(island_size=32, tournament_size=5, model=MODEL_FITNESS, effect_scale=1.0,
                migrate_every=1, seed=3)
    base.update(kw)
    return OracleRun(**base)


def test_purifying_never_improves_and_adaptive_does():
    pur = fitness_run(rows=6, cols=6, p_ben=0.0, p_del=0.33)
    ada = fitness_run(rows=6, cols=6, p_ben=0.003, p_del=0.33, run_id=1)
    pur.step(150)
    ada.step(150)
    assert pur.fitness().max() <= 0.0
    assert ada.fitness().max() > 0.0


def test_first_generation_mutation_statistics():
    # from the all-zero founder with tournaments of one, children differ from 0 exactly by
    # their own mutation: P(decrease) = p_del, P(increase) = p_ben, |change| half-normal
    run = fitness_run(rows=64, cols=64, tournament_size=1, p_ben=0.05, p_del=0.33,
                      migrate_every=0, threads=4)
    run.step(1)
    f = run.fitness().astype(np.float64)
    m = f.size
    for frac, p in (((f < 0).mean(), 0.33), ((f > 0).mean(), 0.05)):
        assert abs(frac - p) < 5 * math.sqrt(p * (1 - p) / m)
    mag = np.abs(f[f != 0])
    assert abs(mag.mean() - math.sqrt(2 / math.pi)) < 5 * math.sqrt((1 - 2 / math.pi) / mag.size)


def test_effect_scale_scales():
    a = fitness_run(rows=8, cols=8, p_ben=0.0, p_del=0.33, effect_scale=1.0, migrate_every=0)
    b = fitness_run(rows=8, cols=8, p_ben=0.0, p_del=0.33, effect_scale=0.25, migrate_every=0)
    a.step(1)
    b.step(1)
    fa, fb = a.fitness(), b.fitness()
    assert np.array_equal(fa == 0, fb == 0)
    nz = fa != 0
    assert np.allclose(fb[nz], np.float32(0.25) * fa[nz], rtol=1e-6)


def test_invalid_fitness_config():
    with pytest.raises(ValueError):
        fitness_run(rows=2, cols=2, effect_scale=0.0)

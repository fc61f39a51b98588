"""The seeded input recipes (no GPU): deterministic per seed, inside their stated ranges,
and shaped as stated (smoothing length, mean and spread, parameter distributions)."""
import numpy as np

from paper_1409_5929_gb300 import inputs


def test_porosity_field_recipe():
    a = inputs.porosity_field(64, 128, 0.3, 0.9, 4.0, seed=2)
    b = inputs.porosity_field(64, 128, 0.3, 0.9, 4.0, seed=2)
    c = inputs.porosity_field(64, 128, 0.3, 0.9, 4.0, seed=3)
    assert a.dtype == np.float32 and a.shape == (64, 128) and a.flags.c_contiguous
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= 0.3 and a.max() <= 0.9
    white = inputs.porosity_field(64, 128, 0.3, 0.9, 0.0, seed=2)
    assert abs(white.mean() - 0.6) < 0.01 and abs(white.std() - 0.6 / np.sqrt(12)) < 0.01
    # a Gaussian of sigma = 4 cells keeps the mean and correlates neighbours
    assert abs(a.mean() - white.mean()) < 5e-3 and a.std() < 0.2 * white.std()
    lag1 = np.corrcoef(a[:, :-1].ravel(), a[:, 1:].ravel())[0, 1]
    lag1_white = np.corrcoef(white[:, :-1].ravel(), white[:, 1:].ravel())[0, 1]
    assert lag1 > 0.9 and abs(lag1_white) < 0.05


def test_porosity_field_around_mean_and_spread():
    f = inputs.porosity_field_around(128, 128, 0.4, 0.05, 2.0, seed=7).astype(np.float64)
    assert abs(f.mean() - 0.4) < 1e-3 and abs(f.std() - 0.05) < 1e-3
    g = inputs.porosity_field_around(64, 64, 0.5, 1.0, 2.0, seed=7)
    assert g.min() >= np.float32(0.05) and g.max() <= np.float32(0.99)


def test_sweep_instances_ranges():
    draws = inputs.sweep_instances(2000, seed=3)
    assert draws[:5] == inputs.sweep_instances(5, seed=3)
    nr = np.array([d["nr"] for d in draws])
    assert nr.min() >= 64 and nr.max() <= 512 and all(d["nz"] == 2 * d["nr"] for d in draws)
    lra = np.log10([d["Ra"] for d in draws])
    lda = np.log10([d["Da"] for d in draws])
    assert lra.min() >= 3 and lra.max() <= 6 and abs(lra.mean() - 4.5) < 0.1
    assert lda.min() >= -5 and lda.max() <= -1 and abs(lda.mean() + 3) < 0.1
    eps = np.array([d["eps"] for d in draws])
    rs = np.array([d["radius_ratio"] for d in draws])
    assert eps.min() >= 0.3 and eps.max() <= 0.9 and rs.min() >= 1.5 and rs.max() <= 4.0
    assert set(d["Pr"] for d in draws) == {0.71, 1.0, 7.0}
    small = inputs.sweep_instances(50, seed=4, nr_lo=24, nr_hi=48)
    assert all(24 <= d["nr"] <= 48 for d in small)

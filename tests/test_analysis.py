"""Pins of the effective-exponent post-processing (Sec. 5.3) on exact power laws."""
import numpy as np
import pytest

from paper_1301_6082_gb300.analysis import effective_exponent
from paper_1301_6082_gb300.workloads import log_times


def test_pure_power_law_gives_its_exponent():
    t = np.array(log_times(10**6, 100), dtype=float)
    for delta in (0.2, 0.5, 1.0):
        tm, rm, de = effective_exponent(t, 3.0 * t ** -delta)
        np.testing.assert_allclose(de, delta, rtol=1e-12)
        assert np.all(np.diff(tm) > 0) and np.all(np.diff(rm) < 0)


def test_correction_to_scaling_converges():
    # rho = c1 t^-d + c2 t^-2d (the form of Sec. 5.3): delta_eff -> d as t grows, and the
    # departure shrinks like t^-d
    t = np.array(log_times(10**7, 120), dtype=float)
    d = 0.25
    tm, rm, de = effective_exponent(t, t ** -d + 0.8 * t ** (-2 * d))
    assert abs(de[-1] - d) < 0.01 and abs(de[0] - d) > abs(de[-1] - d)
    # against rho the departure is linear to leading order: delta_eff - d -> d * (c2/c1) * rho,
    # the straight line of Sec. 5.3 (here d * c2/c1 = 0.2)
    slope = (de - d) / rm
    assert abs(slope[-1] - 0.2) < 0.01 and abs(slope[-1] - 0.2) < abs(slope[0] - 0.2)


def test_skips_non_positive_entries():
    tm, rm, de = effective_exponent([0, 1, 2, 4], [1.0, 0.5, 0.0, 0.25])
    assert len(de) == 1 and np.isclose(de[0], -np.log(0.25 / 0.5) / np.log(4 / 1))


def test_jackknife_error_of_the_mean_is_the_standard_error():
    from paper_1301_6082_gb300.analysis import jackknife_effective_exponent
    rng = np.random.default_rng(4)
    t = np.array(log_times(10**4, 30), dtype=float)
    R = 16
    reps = (t ** -0.3)[None, :] * (1 + 0.05 * rng.standard_normal((R, t.size)))
    mean, err, tm, de, de_err = jackknife_effective_exponent(t, reps)
    np.testing.assert_allclose(mean, reps.mean(0), rtol=1e-14)
    # for a linear statistic the jackknife error equals the usual standard error of the mean
    np.testing.assert_allclose(err, reps.std(0, ddof=1) / np.sqrt(R), rtol=1e-10)
    assert de.shape == de_err.shape == tm.shape and np.all(de_err > 0)
    # the exponent is recovered within a few of its own error bars on the later intervals
    assert np.all(np.abs(de[-10:] - 0.3) < 5 * de_err[-10:] + 1e-3)


def test_jackknife_identical_replicas_have_zero_error():
    from paper_1301_6082_gb300.analysis import jackknife_effective_exponent
    t = np.array(log_times(1000, 12), dtype=float)
    reps = np.tile(2.0 * t ** -0.5, (5, 1))
    mean, err, _, de, de_err = jackknife_effective_exponent(t, reps)
    assert np.all(err < 1e-15) and np.all(de_err < 1e-12)
    np.testing.assert_allclose(de, 0.5, rtol=1e-12)


def test_phase_group_densities_group_and_normalise():
    from paper_1301_6082_gb300.analysis import phase_group_densities
    rng = np.random.default_rng(3)
    L, R, S = 1000, 5, 512
    counts = rng.integers(0, L + 1, size=(R, S))
    g = phase_group_densities(counts, L)
    assert g.shape == (S // 128, R)
    for h in range(S // 128):
        np.testing.assert_allclose(g[h], counts[:, 128 * h:128 * (h + 1)].sum(1) / (128 * L))
    # the mean over phase groups is the run's density
    np.testing.assert_allclose(g.mean(0), counts.sum(1) / (S * L))
    with pytest.raises(ValueError):
        phase_group_densities(counts[:, :100], L)


def test_phase_group_error_bars_through_the_jackknife():
    """Independent phase groups with a known spread: the jackknife error of the mean density
    is the textbook standard error over groups."""
    from paper_1301_6082_gb300.analysis import jackknife_effective_exponent, phase_group_densities
    rng = np.random.default_rng(9)
    L, S = 4096, 128 * 16
    t = np.array([1.0, 2.0, 4.0, 8.0])
    base = 0.5 * t ** -0.3
    counts = np.stack([rng.binomial(L, b, size=S) for b in base])
    g = phase_group_densities(counts, L)
    mean, err, _, delta, derr = jackknife_effective_exponent(t, g)
    np.testing.assert_allclose(mean, counts.sum(1) / (S * L))
    np.testing.assert_allclose(err, g.std(0, ddof=1) / np.sqrt(g.shape[0]), rtol=1e-12)
    assert np.all(np.abs(delta - 0.3) < 6 * derr + 1e-3)

"""Pins of the effective-exponent post-processing (Sec. 5.3) on exact power laws."""
import numpy as np

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

"""The near-critical sweep driver: its batched densities equal separate lone runs summed."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1301_6082_gb300 import build, pcpd
    build.build()
    pcpd.load()
    return pcpd


def test_p_sweep_matches_lone_runs(P):
    from paper_1301_6082_gb300.sweep import p_sweep
    from paper_1301_6082_gb300.workloads import log_times
    L, S, d, mcs = 2048, 64, 0.5, 60
    ps, seeds = (0.12, 0.2), (3, 4)
    out = p_sweep(d, ps, L, S, mcs, n_rec=10, seeds=seeds)
    times = log_times(mcs, 10)
    for p in ps:
        tot = 0
        prs = 0
        for s in seeds:
            a = P.Pcpd(L, S, p, d, seed=s)
            a.run(mcs, times)
            tot = tot + a.counts().astype(np.int64)
            prs = prs + a.pair_counts().astype(np.int64)
            a.close()
        np.testing.assert_array_equal(out[p]["rho"], tot / (L * S * len(seeds)))
        np.testing.assert_array_equal(out[p]["rho_pair"], prs / (L * S * len(seeds)))
        assert np.all(out[p]["rho_pair"] <= out[p]["rho"])
    # more annihilation, faster decay
    assert out[0.2]["rho"][-1] < out[0.12]["rho"][-1]
    # two seeds: jackknife errors come with the means
    for p in ps:
        assert out[p]["rho_err"].shape == out[p]["rho"].shape and np.all(out[p]["rho_err"] >= 0)
        assert out[p]["delta_eff_err"].shape == out[p]["delta_eff"][1].shape


def test_p_sweep_tcpd_matches_lone_runs(P):
    from paper_1301_6082_gb300.sweep import p_sweep
    from paper_1301_6082_gb300.workloads import log_times
    L, S, d, mcs = 2000, 64, 0.5, 40
    ps, seeds = (0.02, 0.1), (5,)
    out = p_sweep(d, ps, L, S, mcs, n_rec=8, seeds=seeds, tuple_n=3)
    times = log_times(mcs, 8)
    for p in ps:
        a = P.Pcpd(L, S, p, d, seed=5, tuple_n=3)
        a.run(mcs, times)
        np.testing.assert_array_equal(out[p]["rho"], a.counts().astype(np.int64) / (L * S))
        a.close()


def test_p_sweep_equals_the_oracle(P, oracle_mod):
    """The sweep's seed-summed counts (particle and pair densities, Sec. 5.3) equal the
    oracle's, and its effective exponents and jackknife errors are those the analysis gives
    for the oracle's per-seed densities."""
    from paper_1301_6082_gb300.analysis import effective_exponent, jackknife_effective_exponent
    from paper_1301_6082_gb300.sweep import p_sweep
    from paper_1301_6082_gb300.workloads import INIT_FULL, log_times
    L, S, d, mcs, n_rec = 300, 64, 0.5, 50, 8
    ps, seeds = (0.1, 0.22), (11, 12)
    out = p_sweep(d, ps, L, S, mcs, n_rec=n_rec, seeds=seeds)
    times = log_times(mcs, n_rec)
    subs = [oracle_mod.substep_of_time(L, t) for t in times]
    for p in ps:
        per, per_pair, tot_sum, prs_sum = [], [], 0, 0
        for s in seeds:
            st = oracle_mod.init_state(L, S, INIT_FULL, s)
            tot, _, _, prs = oracle_mod.run(st, p, d, s, 0, subs[-1], subs, pairs=True)
            tot_sum = tot_sum + tot.astype(np.int64)
            prs_sum = prs_sum + prs.astype(np.int64)
            per.append(tot.astype(np.float64) / (L * S))
            per_pair.append(prs.astype(np.float64) / (L * S))
        rho = tot_sum / float(L * S * len(seeds))
        np.testing.assert_array_equal(out[p]["rho"], rho)
        np.testing.assert_array_equal(out[p]["rho_pair"], prs_sum / float(L * S * len(seeds)))
        _, rm, de = effective_exponent(times, rho)
        np.testing.assert_array_equal(out[p]["delta_eff"][1], de)
        _, err, _, _, de_err = jackknife_effective_exponent(times, np.array(per))
        np.testing.assert_allclose(out[p]["rho_err"], err, rtol=1e-12, atol=0)
        np.testing.assert_allclose(out[p]["delta_eff_err"], de_err, rtol=1e-12, atol=0)

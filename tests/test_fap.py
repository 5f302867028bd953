"""False-alarm-probability tail fits (power law and Gumbel) against distributions with
known parameters, and the device noise generator against E[Upsilon] = 2 N_eff."""
import numpy as np
import pytest
import scipy.stats as st

from paper_2510_19047_b300 import fap


def test_gumbel_fit_recovers_parameters_and_matches_mle():
    rng = np.random.default_rng(11)
    mu, beta, n = 50.0, 4.0, 4000
    x = st.gumbel_r.rvs(loc=mu, scale=beta, size=n, random_state=rng)
    f = fap.fit_gumbel(x)
    # asymptotic standard errors of the Gumbel MLE: 1.053 beta/sqrt(n), 0.780 beta/sqrt(n)
    assert abs(f["mu"] - mu) < 4 * 1.053 * beta / np.sqrt(n)
    assert abs(f["beta"] - beta) < 4 * 0.780 * beta / np.sqrt(n)
    # the same maximum of the likelihood as a general-purpose optimiser finds
    m2, b2 = st.gumbel_r.fit(x)
    assert abs(f["mu"] - m2) < 1e-6 * beta and abs(f["beta"] - b2) < 1e-6 * beta


def test_gumbel_fap_is_the_survival_function():
    f = {"mu": 40.0, "beta": 3.0}
    u = np.array([30.0, 40.0, 55.0, 90.0, 200.0])
    z = (u - 40.0) / 3.0
    exact = 1.0 - np.exp(-np.exp(-z))
    got = fap.fap_gumbel(u, f)
    assert np.allclose(got[:3], exact[:3], rtol=1e-12)
    # deep tail: 1 - exp(-e^{-z}) ~ e^{-z} without cancellation
    assert np.allclose(got[3:], np.exp(-z[3:]), rtol=1e-6)
    assert np.all(np.diff(got) < 0)


def test_power_law_fit_recovers_exponent():
    rng = np.random.default_rng(12)
    alpha, xm, n = 3.0, 10.0, 20000
    x = xm * (1.0 + st.pareto.rvs(alpha, size=n, random_state=rng) - 1.0)
    f = fap.fit_power_law(x, tail_fraction=1.0)
    assert abs(-f["delta"] - 1.0 - alpha) < 4 * alpha / np.sqrt(n)
    assert f["u_min"] == pytest.approx(x.min())


def test_power_law_fap_shape():
    f = {"delta": -5.0, "u_min": 20.0, "fraction": 0.2, "n": 40}
    assert fap.fap_power_law(20.0, f) == pytest.approx(0.2)
    assert fap.fap_power_law(40.0, f) == pytest.approx(0.2 * 2.0 ** -4)
    s = np.linspace(1.0, 30.0, 100)
    # below u_min the empirical survival fraction of the samples
    assert fap.fap_power_law(1.0, f, samples=s) == pytest.approx(1.0)
    assert fap.fap_power_law(15.5, f, samples=s) == pytest.approx(np.mean(s >= 15.5))


def test_tail_of_a_known_exponential_maximum():
    """The maximum of N unit exponentials is Gumbel(ln N, 1) asymptotically: the fit
    of simulated maxima recovers it."""
    rng = np.random.default_rng(13)
    N, R = 2000, 3000
    m = rng.exponential(size=(R, N)).max(axis=1)
    f = fap.fit_gumbel(m)
    assert abs(f["mu"] - np.log(N)) < 0.1 and abs(f["beta"] - 1.0) < 0.05


@pytest.mark.gpu
def test_device_noise_gives_expected_statistic_mean():
    """One template's Upsilon over noise-only realisations drawn by the library
    (tfs_noise_realisation) has mean 2 N_eff (Upsilon is chi^2 with 2 N_eff degrees of
    freedom in noise)."""
    from paper_2510_19047_b300 import synth
    from paper_2510_19047_b300.binding import TFS
    D = synth.week_one_channel(seed=0)
    c = TFS(0, pn_order=0, response=0, path="mixed", pixel="f32")
    c.load_tf_data(D.d, D.dt, D.dT)
    c.set_noise_weights(D.w)
    th = synth.week_bank(8, 0)
    vals, neff = [], None
    for r in range(200):
        c.noise_realisation(1000 + r)
        s, ne, _ = c.eval_statistic(th, 8)
        vals.append(s)
        neff = ne
    v = np.array(vals)  # [R, 8]
    expect = 2.0 * neff
    sd = np.sqrt(4.0 * neff / v.shape[0])  # Var Upsilon = 4 N_eff for chi^2_{2 N_eff}
    assert np.all(np.abs(v.mean(0) - expect) < 4 * sd), (v.mean(0), expect)
    mx = fap.background_maxima(c, D, th, 8, n_real=5, seed=7)
    assert mx.shape == (5,) and np.all(np.isfinite(mx)) and np.all(mx > 0)


@pytest.mark.gpu
def test_device_noise_matches_its_definition():
    """The realisation tfs_noise_realisation draws is the one its definition gives
    (restated in NumPy: Philox4x32-10, Box-Muller, S/(4 df) scaling): the FP64 statistic
    of the library's realisation equals the oracle's statistic of the NumPy one within
    the FP64 bound, on the 45-day A/E grid with gaps and PSD modulation."""
    import oracle
    import search_ref as R
    from paper_2510_19047_b300 import synth
    from paper_2510_19047_b300.binding import TFS
    D = synth.two_year_two_channel(seed=77, n_inj=3, n_tranche=384, L=2048)
    th = synth.two_year_bank(64, seed=8)
    c = TFS(0, path="fp64", pn_order=1, response=1)
    c.load_tf_data(D.d, D.dt, D.dT, D.t0)
    c.set_noise_weights(D.w, D.mask)
    for seed in (3, 2**40 + 5):
        c.noise_realisation(seed)
        got, ne, _ = c.eval_statistic(th, 8)
        dn = R.noise(D.w, 1.0 / D.dT, seed)
        ref, rne, _, _ = oracle.statistic(dn, D.w, D.mask, th, 8, D.dT, pn_order=1, response=1)
        m = ref > 0
        assert np.max(np.abs(got[m] - ref[m]) / ref[m]) < 1e-10
        assert np.array_equal(ne, rne)

"""Pins of the oracle's multi-harmonic statistic (Sec. "Outlook": the waveform
quantities {A, f, fdot, phi} of each harmonic, then the Fresnel expressions per
harmonic).

Each pin takes an independent route: the single-mode statistic (its own pinned code
path), an exact symmetry of the Newtonian chirp, or brute force over all bins from the
oracle's primitives (track, response, tranche transform).
"""
import math

import numpy as np
import pytest

import oracle
from oracle.api import FRESNEL_PAPER, PN_1PN, PN_NEWTONIAN, RESP_LW, RESP_NONE, RESP_TDI
from paper_2510_19047_b300 import synth


@pytest.fixture(scope="module")
def week():
    return synth.week_one_channel(seed=0)


@pytest.fixture(scope="module")
def small_ae():
    return synth.two_year_two_channel(seed=77, n_inj=3, n_tranche=384, L=2048)


def _bank(D, n, seed):
    th = synth.two_year_bank(n, seed=seed)
    th[:, :3] = D.injections
    return th


@pytest.mark.parametrize("resp", [RESP_LW, RESP_TDI])
def test_one_dominant_harmonic_is_the_single_mode_statistic(small_ae, resp):
    # nu = 1 with any complex amplitude: the template is scaled and phase-shifted by a
    # constant, which Upsilon ignores
    D = small_ae
    th = _bank(D, 6, 21)
    kw = dict(pn_order=PN_1PN, response=resp)
    ref = oracle.statistic(D.d, D.w, D.mask, th, 16, D.dT, **kw)
    got = oracle.statistic_harm(D.d, D.w, D.mask, th, 16, D.dT, [1.0], [0.7 - 0.3j], **kw)
    np.testing.assert_allclose(got[0], ref[0], rtol=1e-11)
    for a, b in zip(got[1:], ref[1:]):
        np.testing.assert_array_equal(a, b)


def test_split_harmonic_keeps_cross_terms(small_ae):
    # two copies of nu = 1 whose amplitudes sum to 1 are the single-mode template: their
    # windows coincide, so <y|y> holds the cross terms 2 Re(conj(c1) c2) |h|^2
    D = small_ae
    th = _bank(D, 6, 22)
    kw = dict(pn_order=PN_1PN, response=RESP_LW)
    ref = oracle.statistic(D.d, D.w, D.mask, th, 16, D.dT, **kw)[0]
    got = oracle.statistic_harm(D.d, D.w, D.mask, th, 16, D.dT, [1.0, 1.0],
                                [0.3 + 0.2j, 0.7 - 0.2j], **kw)[0]
    np.testing.assert_allclose(got, ref, rtol=1e-11)


def _rescaled(th, nu):
    # Newtonian chirp: f0 -> nu f0, M_c -> M_c nu^(-8/5) keeps tau_0 and gives
    # f'(t) = nu f(t), fdot' = nu fdot, Phi' - phi0' = nu (Phi - phi0)
    t2 = th.copy()
    t2[0] = th[0] * nu ** (-1.6)
    t2[2] = th[2] * nu
    t2[3] = th[3] * nu
    return t2


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.0])
def test_harmonic_is_the_rescaled_newtonian_chirp(week, small_ae, nu):
    # one harmonic nu of theta = the dominant mode of the rescaled chirp (the response
    # depends on time and sky only, or on the frequency, which both sides share)
    th = synth.week_bank(6, seed=4)
    th[:, 0] = week.injections[:, 0]
    ref = oracle.statistic(week.d, week.w, week.mask, _rescaled(th, nu), 8, week.dT)[0]
    got = oracle.statistic_harm(week.d, week.w, week.mask, th, 8, week.dT, [nu], [1.0])[0]
    assert np.count_nonzero(ref) >= 2  # nu = 0.5 leaves the band for part of the bank
    np.testing.assert_allclose(got, ref, rtol=1e-9)
    D = small_ae
    th = _bank(D, 4, 23)
    for resp in (RESP_LW, RESP_TDI):
        kw = dict(pn_order=PN_NEWTONIAN, response=resp)
        ref = oracle.statistic(D.d, D.w, D.mask, _rescaled(th, nu), 16, D.dT, **kw)[0]
        got = oracle.statistic_harm(D.d, D.w, D.mask, th, 16, D.dT, [nu], [1.0], **kw)[0]
        assert np.all(ref > 0)
        np.testing.assert_allclose(got, ref, rtol=1e-9)


def test_overlaps_are_linear_in_the_amplitudes(small_ae):
    # Z_n is linear in (c_1, ..., c_H); N_n is the quadratic form, which splits into the
    # harmonics' own norms where their windows are disjoint (nu = 1 and 2 at 15-30 mHz)
    D = small_ae
    th = _bank(D, 3, 24)[:, 0]
    kw = dict(pn_order=PN_1PN, response=RESP_LW)
    nu = [1.0, 2.0]
    c = np.array([0.8 + 0.1j, -0.3 + 0.4j])
    z, n, _ = oracle.segments_harm(D.d, D.w, D.mask, th, 32, D.dT, nu, c, **kw)
    z1, n1, _ = oracle.segments_harm(D.d, D.w, D.mask, th, 32, D.dT, nu, [c[0], 0.0], **kw)
    z2, n2, _ = oracle.segments_harm(D.d, D.w, D.mask, th, 32, D.dT, nu, [0.0, c[1]], **kw)
    assert np.count_nonzero(n) > 10
    np.testing.assert_allclose(z, z1 + z2, rtol=1e-12, atol=1e-12 * np.abs(z).max())
    np.testing.assert_allclose(n, n1 + n2, rtol=1e-12, atol=1e-14 * n.max())


def _phase_origin(th, pn, resp):
    """Detector time t* at which t' = 0, so that the oracle's phase advanced from t* is
    Phi(t') - phi_0."""
    t = 0.0
    for _ in range(40):
        t = -(oracle.track(th, np.array([t]), 0.0, pn, resp)["tprime"][0] - t)
    return t


def _brute_force_harm(D, th, n_seg, pn, resp, nu, c):
    """Explicit loops over (m, h, k, alpha): each harmonic's Eq. fresnel-ft over all bins
    times its 21-bin window indicator, summed into one template per tranche (Eqs.
    inner-tf, inner-tranche-tf, overlap-n, Upsilon-seg)."""
    nt, nb = D.n_tranche, D.n_bins
    seg = nt // n_seg
    t_star = _phase_origin(th, pn, resp)
    k = np.arange(nb)
    ups = 0.0
    for n in range(n_seg):
        Z = 0j
        N = 0.0
        for m in range(n * seg, (n + 1) * seg):
            if not D.mask[m]:
                continue
            tm = m * D.dT
            tr = oracle.track(th, np.array([tm]), t_anchor=t_star, pn_order=pn, response=resp)
            if not tr["alive"][0] or tr["fdot"][0] <= 0:
                continue
            f, fd, A = tr["f"][0], tr["fdot"][0], tr["amp"][0]
            phi = th[3] + tr["dphi"][0]
            y = np.zeros((D.n_chan, nb), complex)
            for nh, ch in zip(nu, c):
                kc = math.ceil(nh * f / D.df)
                if kc - 10 < 1 or kc + 10 > nb - 1:
                    continue
                if resp == RESP_TDI:
                    T = oracle.response_tdi(th, np.array([tm]), np.array([nh * f]), D.n_chan)[:, 0]
                elif resp == RESP_LW:
                    T = oracle.response(th, np.array([tm]), D.n_chan)[:, 0]
                else:
                    T = np.ones(D.n_chan)
                h_all = oracle.tranche_ft(A, nh * phi, nh * f, nh * fd, D.dT, 0, nb, FRESNEL_PAPER)
                win = (np.abs(k - kc) <= 10).astype(float)
                for a in range(D.n_chan):
                    y[a] += T[a] * ch * h_all * win
            for a in range(D.n_chan):
                for kk in range(nb):
                    Z += np.conj(D.d[a, m, kk]) * y[a, kk] * D.w[a, m, kk] * D.df
                    N += abs(y[a, kk]) ** 2 * D.w[a, m, kk] * D.df
        if N > 0:
            ups += 4 * abs(Z) ** 2 / N
    return ups


def test_brute_force_harmonics_tiny_grids(week):
    # week grid: nu = 1 and 1.5 windows overlap near f = 15 mHz, nu = 0.5 sits at the
    # lower band edge
    sub = synth.TFData(d=week.d[:, :48], w=week.w[:, :48], mask=week.mask[:48].copy(),
                       dt=week.dt, dT=week.dT)
    sub.mask[5] = 0
    th = week.injections[:, 0]
    nu, c = [0.5, 1.0, 1.5], [0.2 + 0.1j, 1.0, -0.4 + 0.3j]
    ref = _brute_force_harm(sub, th, 8, PN_NEWTONIAN, RESP_NONE, nu, c)
    got = oracle.statistic_harm(sub.d, sub.w, sub.mask, th[:, None], 8, sub.dT, nu, c)[0][0]
    assert ref > 0 and abs(got - ref) < 1e-11 * ref
    # two channels, 8 x 64 bins, 1PN, both responses: windows of nu = 0.75, 1, 1.25 overlap
    rng = np.random.default_rng(4)
    dT = 10240.0
    d = rng.standard_normal((2, 8, 64)) + 1j * rng.standard_normal((2, 8, 64))
    w = rng.uniform(0.5, 2.0, (2, 8, 64))
    tiny = synth.TFData(d=d, w=w, mask=np.array([1, 1, 0, 1, 1, 1, 1, 1], np.uint8), dt=5.0, dT=dT)
    th = np.array([40.0, 0.2, 30.3 / dT, 0.5, 2.0, 0.3, 1.0, 0.6])
    nu, c = [0.75, 1.0, 1.25], [0.3 - 0.2j, 1.0, 0.5 + 0.5j]
    for resp in (RESP_LW, RESP_TDI):
        ref = _brute_force_harm(tiny, th, 4, PN_1PN, resp, nu, c)
        got = oracle.statistic_harm(d, w, tiny.mask, th[:, None], 4, dT, nu, c, pn_order=PN_1PN,
                                    response=resp)[0][0]
        assert ref > 0 and abs(got - ref) < 1e-11 * ref

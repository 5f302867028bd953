"""Multi-harmonic templates on the CUDA paths against the FP64 oracle (same seeded
inputs, element by element).

Tolerances: every path keeps the single-mode bounds of its pixel type; the FP64 path
1e-10. The harmonics' relative phases depend on the absolute phase nu_h Phi(t'), which
the FP64 kernel forms in double-double from double-double chirp constants.
"""
import numpy as np
import pytest

import oracle
from paper_2510_19047_b300 import synth

pytestmark = pytest.mark.gpu

TOL = {("fp64", "f16"): (1e-10, 1e-10), ("plain", "f16"): (1e-4, 1e-4),
       ("mixed", "f32"): (1e-4, 1e-4), ("mixed", "f16"): (1.5e-3, 1e-3),
       ("mixed", "bf16"): (1.2e-2, 8e-3)}
CASES = list(TOL)
FP64_TOL = 1e-10
NU = [0.5, 1.0, 1.5]
C = [0.3 + 0.1j, 1.0, 0.4 - 0.2j]


def rel_err(got, ref):
    got, ref = np.asarray(got, float), np.asarray(ref, float)
    assert np.all(np.isfinite(got))
    zero = ref == 0
    assert np.all(got[zero] == 0)
    r = np.abs(got[~zero] - ref[~zero]) / ref[~zero]
    return (r.max(), np.percentile(r, 99)) if r.size else (0.0, 0.0)


def ctx_for(D, path, pixel, nu, c):
    from paper_2510_19047_b300.binding import TFS
    t = TFS(0, path=path, pixel=pixel, pn_order=D.pn_order, response=D.response)
    t.load_tf_data(D.d, D.dt, D.dT, D.t0)
    t.set_noise_weights(D.w, D.mask)
    t.set_harmonics(nu, c)
    return t


def check(D, th, lev, path, pixel, nu, c, diag_slack=None):
    refs = [oracle.statistic_harm(D.d, D.w, D.mask, th, L, D.dT, nu, c, pn_order=D.pn_order,
                                  response=D.response) for L in lev]
    t = ctx_for(D, path, pixel, nu, c)
    got, neff, diag = t.eval_statistic(th, lev, diag=True)
    for i, (ref, rneff, rnact, _) in enumerate(refs):
        assert np.count_nonzero(ref) > 0.8 * th.shape[1]
        mx, p99 = rel_err(got[i], ref)
        tol = FP64_TOL if path == "fp64" else TOL[(path, pixel)][0]
        assert mx < tol and p99 < max(tol, TOL[(path, pixel)][1]), (lev[i], mx, p99)
        assert np.array_equal(neff[i], rneff)
    slack = (0 if path == "fp64" else 1) if diag_slack is None else diag_slack
    assert np.abs(diag[0] - refs[0][2]).max() <= slack
    return got


@pytest.fixture(scope="module")
def ae45():
    return synth.two_year_two_channel(seed=77, n_inj=3, n_tranche=384, L=2048)


@pytest.fixture(scope="module")
def bank(ae45):
    th = synth.two_year_bank(77, seed=13)  # ragged: not a multiple of 32
    th[:, :3] = ae45.injections
    return th


@pytest.mark.parametrize("path,pixel", CASES)
def test_three_harmonics_long_wavelength(ae45, bank, path, pixel):
    check(ae45, bank, [64, 8], path, pixel, NU, C)


@pytest.mark.parametrize("path,pixel", [("fp64", "f16"), ("plain", "f16"), ("mixed", "f16")])
def test_three_harmonics_tdi(path, pixel):
    D = synth.cached(synth.two_year_two_channel, seed=78, n_inj=2, n_tranche=384, L=2048,
                     response="tdi")
    th = np.concatenate([D.injections, synth.two_year_bank(46, seed=17)], axis=1)
    check(D, th, [32, 8], path, pixel, NU, C)


@pytest.mark.parametrize("path,pixel", [("fp64", "f16"), ("plain", "f16"), ("mixed", "f32"),
                                        ("mixed", "f16")])
def test_one_channel_and_band_edges(path, pixel):
    # one channel, no response; nu = 0.5 puts part of the bank below the band's lower edge
    D = synth.week_one_channel(seed=0)
    th = synth.week_bank(200, 0)
    check(D, th, [8, 2], path, pixel, [0.5, 1.0, 2.0], [0.5, 1.0, 0.25j])


@pytest.mark.parametrize("path,pixel", [("fp64", "f16"), ("plain", "f16"), ("mixed", "f32"),
                                        ("mixed", "f16")])
def test_overlapping_windows_keep_cross_terms(ae45, bank, path, pixel):
    # nu = 1 and 1.05 share ~10 bins at 20 mHz: the cross terms of N_n are evaluated
    # bin by bin
    check(ae45, bank[:, :40], [16], path, pixel, [1.0, 1.05], [1.0, 0.6 + 0.3j])
    # two copies of the dominant mode whose amplitudes sum to 1 are the single-mode
    # template (the oracle's single-mode statistic is the reference)
    t = ctx_for(ae45, path, pixel, [1.0, 1.0], [0.3 + 0.2j, 0.7 - 0.2j])
    got, _, _ = t.eval_statistic(bank[:, :40], 16)
    ref = oracle.statistic(ae45.d, ae45.w, ae45.mask, bank[:, :40], 16, ae45.dT, pn_order=1,
                           response=1)[0]
    mx, _ = rel_err(got, ref)
    assert mx < (FP64_TOL if path == "fp64" else TOL[(path, pixel)][0])


@pytest.mark.parametrize("path,pixel", [("fp64", "f16"), ("plain", "f16"), ("mixed", "f16")])
def test_low_harmonic_outlives_the_dominant_window(ae45, path, pixel):
    # chirps that leave the band (f > (N_bins - 11) df) inside the grid: the nu = 1/2
    # harmonic stays in band until coalescence, so the tranche range that can be active
    # reaches past the dominant mode's
    rng = np.random.Generator(np.random.PCG64(41))
    th = synth.two_year_bank(48, seed=42)
    th[0] = rng.uniform(45, 60, 48)
    th[2] = rng.uniform(0.05, 0.08, 48)
    ref1 = oracle.statistic(ae45.d, ae45.w, ae45.mask, th, 8, ae45.dT, pn_order=1, response=1)
    ref = oracle.statistic_harm(ae45.d, ae45.w, ae45.mask, th, 8, ae45.dT, [0.5, 1.0],
                                [0.5, 1.0], pn_order=1, response=1)
    assert np.sum(ref[2] > ref1[2] + 10) > 10  # the low harmonic adds active tranches
    check(ae45, th, [8], path, pixel, [0.5, 1.0], [0.5, 1.0])


def test_harmonic_settings_and_errors(ae45, bank):
    from paper_2510_19047_b300.binding import TFSError
    t = ctx_for(ae45, "mixed", "f16", [], [])
    base, _, _ = t.eval_statistic(bank, [64, 8])
    t.set_harmonics([1.0], [1.0])
    one, _, _ = t.eval_statistic(bank, [64, 8])
    assert rel_err(one, base)[0] < 1e-3  # the single-mode template through the harmonic kernel
    t.set_harmonics()
    again, _, _ = t.eval_statistic(bank, [64, 8])
    assert np.array_equal(again, base)  # back to the dominant-mode kernel, bit for bit
    for nu, c in (([0.0], [1.0]), ([17.0], [1.0]), ([1.0], [np.nan]), ([1.0] * 9, [1.0] * 9)):
        with pytest.raises(TFSError, match="ARG"):
            t.set_harmonics(nu, c)
    t.set_harmonics(NU, C)
    with pytest.raises(TFSError, match="ARG"):
        t.grad_statistic(bank[:, :4], 8)
    t.set_options(path="mixed")
    s, n, _ = t.eval_statistic(np.zeros((8, 0)), 8)
    assert s.shape == (0,)


def test_two_year_full_bank_three_harmonics_sampled():
    """The bench workload with three harmonics (1e6 templates, N_seg 256/64/16 in one
    launch of the harmonic kernel): 60 templates spread over the queue against the
    oracle (max and p99), the FP64 path on the same sample, and properties that hold for
    every template."""
    import torch
    D = synth.cached(synth.two_year_two_channel)
    lev = [256, 64, 16]
    th = synth.two_year_bank(1_000_000, seed=2002)
    t = ctx_for(D, "mixed", "f16", NU, C)
    st, ne, dg = t.eval_statistic(torch.from_numpy(th).cuda(), lev, diag=True)
    st, ne = st.cpu().numpy(), ne.cpu().numpy()
    assert np.all(np.isfinite(st)) and np.all(st >= 0)
    assert np.all(ne <= np.array(lev)[:, None])
    assert np.all(st[0] >= st[1] * (1 - 3e-3)) and np.all(st[1] >= st[2] * (1 - 3e-3))
    act = ne[0] > 0
    assert abs(np.mean(st[0][act]) / np.mean(2 * ne[0][act]) - 1) < 0.02  # noise: chi^2
    idx = np.linspace(0, th.shape[1] - 1, 60).astype(int)
    t64 = ctx_for(D, "fp64", "f16", NU, C)
    g64, _, _ = t64.eval_statistic(th[:, idx], lev)
    for i, L in enumerate(lev):
        ref, rneff, _, _ = oracle.statistic_harm(D.d, D.w, D.mask, th[:, idx], L, D.dT, NU, C,
                                                 pn_order=1, response=1)
        mx, p99 = rel_err(st[i, idx], ref)
        assert mx < TOL[("mixed", "f16")][0] and p99 < TOL[("mixed", "f16")][1], (L, mx, p99)
        assert np.array_equal(ne[i, idx], rneff)
        assert rel_err(g64[i], ref)[0] < FP64_TOL, L


def test_harmonics_per_template_segments_checked_and_graph_options(ae45, bank):
    # per-template N_seg, checked mode and the graph option (the harmonic launch is not
    # captured: the option is ignored) against the plain call
    from paper_2510_19047_b300.binding import TFS
    th = bank[:, :64]
    ns = np.array([64, 16, 8, 1], np.int32)[np.arange(64) % 4]
    for path, tol in (("fp64", FP64_TOL), ("mixed", TOL[("mixed", "f16")][0])):
        t = ctx_for(ae45, path, "f16", NU, C)
        got, neff, _ = t.eval_statistic(th, ns, per_template=True)
        for L in (64, 16, 8, 1):
            sel = ns == L
            ref, rneff, _, _ = oracle.statistic_harm(ae45.d, ae45.w, ae45.mask, th[:, sel], int(L),
                                                     ae45.dT, NU, C, pn_order=1, response=1)
            assert rel_err(got[sel], ref)[0] < tol, (path, L)
            assert np.array_equal(neff[sel], rneff)
    base = ctx_for(ae45, "mixed", "f16", NU, C)
    ref, _, _ = base.eval_statistic(th, [64, 8])
    for kw in ({"checked": 1}, {"use_graph": 1}, {"sort": 0}):
        t = TFS(0, path="mixed", pixel="f16", pn_order=1, response=1, **kw)
        t.load_tf_data(ae45.d, ae45.dt, ae45.dT, ae45.t0)
        t.set_noise_weights(ae45.w, ae45.mask)
        t.set_harmonics(NU, C)
        for _ in range(2):
            got, _, _ = t.eval_statistic(th, [64, 8])
            assert np.array_equal(got, ref), kw

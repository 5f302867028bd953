"""The search workloads against the oracle at their own launch configurations.

test_uneven_length_bank_at_the_ladder_launch: the 1e7-template bank whose in-band
durations are lognormal in [30 d, 2 yr] (the paper's cost follows the in-band track
length, Sec. "Hardware acceleration and computational cost"), evaluated at N_seg = 256
in one persistent, length-sorted launch replayed as a CUDA graph, exactly as the ladder's
first stage runs it; 12 templates spread over the range of track lengths are compared
with the oracle.

test_two_year_coherent_stage: the ladder's last stage, N_seg = 1 over the whole two-year
grid (phases of ~1e7 rad in one coherent segment), on the 20 injections and candidates
around them: the FP64 path within 1e-10 of the oracle, the mixed path within its FP16
and FP32 bounds.
"""
import numpy as np
import pytest

import oracle
from paper_2510_19047_b300 import synth

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
F16_MAX = 1.5e-3


@pytest.fixture(scope="module")
def two_year():
    return synth.cached(synth.two_year_two_channel)


def ctx_for(D, **kw):
    from paper_2510_19047_b300.binding import TFS
    c = TFS(0, pn_order=D.pn_order, response=D.response, **kw)
    c.load_tf_data(D.d, D.dt, D.dT, D.t0)
    c.set_noise_weights(D.w, D.mask)
    return c


def rel(got, ref):
    got, ref = np.asarray(got, float), np.asarray(ref, float)
    assert np.all(np.isfinite(got))
    assert np.all(got[ref == 0] == 0)
    m = ref != 0
    return np.abs(got[m] - ref[m]) / ref[m]


def test_uneven_length_bank_at_the_ladder_launch(two_year):
    import torch
    D = two_year
    n = 10_000_000
    bank = synth.uneven_length_bank(n, seed=2004, dT=D.dT, n_bins=D.n_bins)
    c = ctx_for(D, use_graph=1)
    th = torch.from_numpy(bank).cuda()
    st, ne, dg = c.eval_statistic(th, 256, diag=True)
    st, ne, nact = st.cpu().numpy(), ne.cpu().numpy(), dg[0].cpu().numpy()
    del th
    assert np.all(np.isfinite(st)) and np.all(st >= 0) and np.all(ne <= 256)
    act = ne > 0
    assert abs(np.mean(st[act]) / np.mean(2 * ne[act]) - 1) < 0.02  # noise: E = 2 N_eff
    # 12 templates from the shortest to the longest in-band track
    order = np.argsort(nact, kind="stable")
    idx = order[np.linspace(0, n - 1, 12).astype(int)]
    assert nact[idx[-1]] > 20 * max(nact[idx[0]], 1)  # the sample spans the length range
    ref, rneff, rnact, _ = oracle.statistic(D.d, D.w, D.mask, bank[:, idx], 256, D.dT,
                                            pn_order=1, response=1)
    assert rel(st[idx], ref).max() < F16_MAX
    assert np.array_equal(ne[idx], rneff)
    assert np.abs(nact[idx] - rnact).max() <= 1  # double-float window decision


def test_two_year_coherent_stage(two_year):
    """The injections carry a spin/eccentricity-like phase drift the templates lack, so
    over one two-year coherent segment some of them fall to the noise level (Upsilon ~ 1);
    candidates near them span both regimes. The FP64 path is held to 1e-10 relative; the
    mixed path's bound is relative to max(Upsilon, 2 N_eff), the statistic's noise mean,
    because the pixel rounding moves a noise-level Upsilon by a fraction of that mean,
    not of its own value."""
    D = two_year
    th = np.concatenate([D.injections, synth.candidates_near(D.injections, 20, seed=21)], axis=1)
    ref, rneff, _, _ = oracle.statistic(D.d, D.w, D.mask, th, 1, D.dT, pn_order=1, response=1)
    assert np.max(ref) > 10 * 2  # one injection stays far above the noise mean
    for path, pixel, tol in (("fp64", "f16", FP64_TOL), ("mixed", "f16", F16_MAX),
                             ("mixed", "f32", 1e-4)):
        got, ne, _ = ctx_for(D, path=path, pixel=pixel).eval_statistic(th, 1)
        assert np.array_equal(ne, rneff)
        if path == "fp64":
            assert rel(got, ref).max() < tol, (path, rel(got, ref).max())
        else:
            err = np.abs(got - ref) / np.maximum(ref, 2.0 * rneff)
            assert err.max() < tol, (path, pixel, err.max())

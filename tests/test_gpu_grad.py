"""Adjoint gradient kernel against the oracle's dual-number gradient and central
differences of the CUDA FP64 path; the autograd wrapper and an ascent step."""
import numpy as np
import pytest

import oracle
from paper_2510_19047_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ae45():
    return synth.two_year_two_channel(seed=77, n_inj=3, n_tranche=384, L=2048)


def ctx_for(D, **kw):
    from paper_2510_19047_b300.binding import TFS
    c = TFS(0, pn_order=D.pn_order, response=D.response, **kw)
    c.load_tf_data(D.d, D.dt, D.dT, D.t0)
    c.set_noise_weights(D.w, D.mask)
    return c


@pytest.fixture(scope="module")
def ae45_tdi():
    # injections built through the time-domain TDI-1.5 single-link response
    return synth.cached(synth.two_year_two_channel, seed=78, n_inj=2, n_tranche=384, L=2048,
                        response="tdi")


@pytest.mark.parametrize("n_seg", [16, 1])
@pytest.mark.parametrize("data", ["ae45", "ae45_tdi"])
def test_gradient_matches_oracle(data, n_seg, request):
    D = request.getfixturevalue(data)
    th = synth.candidates_near(D.injections, 24, seed=3)
    ref_u, ref_g = oracle.gradient(D.d, D.w, D.mask, th, n_seg, D.dT, pn_order=1,
                                   response=D.response)
    c = ctx_for(D)
    u, g = c.grad_statistic(th, n_seg)
    np.testing.assert_allclose(u, ref_u, rtol=1e-4)
    # per component, relative to the component or to the gradient's own scale
    # (|dU/dtheta_p| * |theta range|), whichever is larger
    for p in range(8):
        if p == 3:
            assert np.all(np.abs(g[3]) < 1e-3 * ref_u)  # phi_0 is maximised away
            continue
        scale = np.maximum(np.abs(ref_g[p]), 1e-3 * np.abs(ref_g[p]).max())
        err = np.abs(g[p] - ref_g[p]) / scale
        assert err.max() < 2e-3, (p, err.max())
        assert np.median(np.abs(g[p] - ref_g[p]) / np.maximum(np.abs(ref_g[p]), 1e-300)) < 1e-4, p


def test_gradient_per_template_is_independent_of_batch(ae45):
    D = ae45
    th = synth.candidates_near(D.injections, 40, seed=5)
    c = ctx_for(D)
    u_all, g_all = c.grad_statistic(th, 16)
    u_one, g_one = c.grad_statistic(th[:, 7:8], 16)
    assert np.array_equal(u_all[7:8], u_one) and np.array_equal(g_all[:, 7:8], g_one)


def test_split_work_items_match_one_item_per_template(ae45):
    # a small batch splits each template's segments into work items whose partial sums
    # are added afterwards; inside a large batch every template is one item. Both give
    # the same FP32 segment sums, combined in another FP64 order
    D = ae45
    th = synth.candidates_near(D.injections, 24, seed=11)
    c = ctx_for(D)
    u_small, g_small = c.grad_statistic(th, 16)
    big = np.concatenate([th, synth.candidates_near(D.injections, 7976, seed=12)], axis=1)
    u_big, g_big = c.grad_statistic(big, 16)
    np.testing.assert_allclose(u_small, u_big[:24], rtol=1e-12)
    scale = np.abs(g_big[:, :24]).max(axis=1, keepdims=True)
    assert np.all(np.abs(g_small - g_big[:, :24]) <= 1e-9 * scale)


def test_autograd_and_ascent(ae45):
    import torch
    from paper_2510_19047_b300.autograd import statistic
    D = ae45
    c = ctx_for(D)
    th0 = synth.candidates_near(D.injections, 16, seed=9)
    th = torch.from_numpy(th0).cuda().requires_grad_(True)
    u = statistic(th, c, 16)
    u.sum().backward()
    _, g = c.grad_statistic(th0, 16)
    np.testing.assert_allclose(th.grad.cpu().numpy(), g, rtol=1e-12)
    # a projected ascent step along sigma^2 * grad gains what the gradient predicts:
    # dU ~ t |sigma g|^2 for a step of 0.01 sigma-units
    sig = np.array([1e-5 * 30, 1e-4, 1e-8, 0.0, 1e-4, 1e-4, 1e-4, 1e-4])
    u0, g0 = c.grad_statistic(th0, 16)
    norm = np.sqrt(((sig[:, None] * g0) ** 2).sum(0))
    t = 0.01 / norm
    lo = np.array([1, 0.01, 1e-5, 0, 0, -np.pi / 2, 0, 0])
    hi = np.array([200, 0.25, 1.0, 2 * np.pi, 2 * np.pi, np.pi / 2, np.pi, np.pi])
    t1 = th0.copy()
    c.ascent_step(t1, g0 * t[None, :], sig ** 2, lo, hi)
    u1, _ = c.grad_statistic(t1, 16)
    pred = t * norm ** 2
    ratio = (u1 - u0) / pred
    assert np.mean((ratio > 0.5) & (ratio < 1.5)) > 0.8, ratio

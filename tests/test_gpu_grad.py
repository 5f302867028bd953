"""Adjoint gradient kernel (tfs_grad_statistic) against the oracle's dual-number
gradient, and against 5-point central differences (step 1e-6 relative) of the GPU's own
FP64 statistic path; the autograd wrapper and the refinement steps.

Bound. dUpsilon/dtheta_p is a sum, over every (segment n, tranche m), of the terms
t_nm = 8 Re(conj(Z_n) dz_m)/N_n - 4 |Z_n|^2 dn_m/N_n^2 (Eq. Upsilon-seg differentiated,
z_m and n_m the tranche's shares of Z_n and N_n). The kernel forms each tranche's share
in FP32, so it resolves the component to ~u32 = 6e-8 of S_p = sum |t_nm|, the oracle's
tranche-level term scale, and no better: where the terms cancel (dUpsilon/dpsi is
exactly zero for circular polarisation, iota = 0 or pi, while its per-tranche terms are
of the order of Upsilon) no FP32 evaluation has a relative error below 1. Each
component is therefore held to 2e-5 S_p (~340 u32; measured <= 2.3e-6 S_p on these
candidates), which is a relative bound of 1e-4 wherever the component is at least a
fifth of its scale. phi_0 is maximised away (zero exactly); its value is held to 2e-5 of
the statistic (measured <= 2.2e-6).
"""
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


GRAD_TOL = 2e-5   # of the tranche-level term scale
PHI0_TOL = 2e-5   # of Upsilon


@pytest.mark.parametrize("n_seg", [16, 1])
@pytest.mark.parametrize("data", ["ae45", "ae45_tdi"])
def test_gradient_matches_oracle(data, n_seg, request):
    D = request.getfixturevalue(data)
    th = synth.candidates_near(D.injections, 24, seed=3)
    kw = dict(pn_order=1, response=D.response)
    ref_u, ref_g = oracle.gradient(D.d, D.w, D.mask, th, n_seg, D.dT, **kw)
    S = oracle.gradient_scale(D.d, D.w, D.mask, th, n_seg, D.dT, tranche_level=True, **kw)
    c = ctx_for(D)
    u, g = c.grad_statistic(th, n_seg)
    np.testing.assert_allclose(u, ref_u, rtol=1e-4)
    assert np.all(np.abs(g[3]) <= PHI0_TOL * ref_u)  # phi_0 is maximised away
    n_rel = 0
    for p in (0, 1, 2, 4, 5, 6, 7):
        err = np.abs(g[p] - ref_g[p])
        assert np.all(err <= GRAD_TOL * S[p]), (p, (err / S[p]).max())
        # where the component is not a cancelling sum the bound is relative
        big = np.abs(ref_g[p]) >= 0.2 * S[p]
        assert np.all(err[big] <= 1e-4 * np.abs(ref_g[p][big])), p
        n_rel += int(big.sum())
    assert n_rel >= 10  # the relative form is exercised


@pytest.mark.parametrize("data", ["ae45", "ae45_tdi"])
def test_gradient_matches_central_differences(data, request):
    """Config 5's check: 5-point central differences with step h = 1e-6 relative
    (1e-6 rad where an angle is below 1) of the FP64 statistic path, at N_seg = 16.
    Where the stencils at h and h/2 disagree, a window or Fresnel-branch switch lies
    inside the stencil and the almost-everywhere derivative is not what the differences
    see (reading Q16): such pairs are excluded and counted. The differences agree with
    the oracle to 1e-5 relative plus 2e-6 of the term scale (measured <= 6.8e-7 S), and
    the adjoint kernel agrees with them within its own bound."""
    D = request.getfixturevalue(data)
    n_seg = 16
    th = synth.candidates_near(D.injections, 24, seed=3)
    kw = dict(pn_order=1, response=D.response)
    _, ref_g = oracle.gradient(D.d, D.w, D.mask, th, n_seg, D.dT, **kw)
    S = oracle.gradient_scale(D.d, D.w, D.mask, th, n_seg, D.dT, tranche_level=True, **kw)
    _, g = ctx_for(D).grad_statistic(th, n_seg)
    c64 = ctx_for(D, path="fp64")

    def fd5(p, h):
        vals = []
        for k in (2, 1, -1, -2):
            t = th.copy()
            t[p] += k * h
            vals.append(c64.eval_statistic(t, n_seg)[0])
        return (-vals[0] + 8 * vals[1] - 8 * vals[2] + vals[3]) / (12 * h)

    checked = flipped = 0
    for p in (0, 1, 2, 4, 5, 6, 7):
        h = 1e-6 * np.maximum(np.abs(th[p]), 1.0)
        fd, fd2 = fd5(p, h), fd5(p, 0.5 * h)
        smooth = np.abs(fd - fd2) <= 1e-6 * S[p]
        flipped += int((~smooth).sum())
        e_ref = np.abs(fd - ref_g[p])[smooth]
        assert np.all(e_ref <= 1e-5 * np.abs(ref_g[p][smooth]) + 2e-6 * S[p][smooth]), p
        assert np.all(np.abs(g[p] - fd)[smooth] <= GRAD_TOL * S[p][smooth]), p
        checked += int(smooth.sum())
    assert checked >= 100 and flipped <= checked // 2, (checked, flipped)


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


@pytest.mark.parametrize("n", [64, 8192])
def test_templates_without_active_tranches_give_zeros(ae45, n):
    """A template whose track never enters the band (f_0 above the top bin, or so far
    below the bottom of the window range that it does not reach it in 45 days) has no
    active tranche: its statistic and gradient are exactly zero, both when a small batch
    splits every template into several work items (n = 64) and when each template is one
    item (n = 8192, over three waves), and its neighbours in the batch are unaffected."""
    import torch
    th = synth.candidates_near(ae45.injections, n, seed=9)
    top = ae45.n_bins / ae45.dT  # frequency of the top bin [Hz]
    dead = np.arange(5, n, 7)
    th[2, dead[::2]] = 3.0 * top            # above the band from the start
    th[2, dead[1::2]] = 2e-4                # below bin 10 for the whole grid
    c = ctx_for(ae45)
    _, ne, dg = c.eval_statistic(th, 16, diag=True)
    idle = dg[0] == 0
    assert idle[dead].all() and idle.sum() < len(dead) + n // 10
    # poison the outputs so that an unwritten entry would show
    u = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
    g = torch.full((8, n), np.nan, dtype=torch.float64, device="cuda")
    c.grad_statistic(torch.from_numpy(th).cuda(), 16, out=(u, g))
    u, g = u.cpu().numpy(), g.cpu().numpy()
    assert np.all(u[idle] == 0) and np.all(g[:, idle] == 0)
    assert np.all(np.isfinite(u)) and np.all(np.isfinite(g))
    ref_u, _ = c.grad_statistic(th[:, ~idle][:, :32], 16)
    np.testing.assert_allclose(u[~idle][:32], ref_u, rtol=1e-12)  # work-item split may differ


@pytest.mark.parametrize("response", [1, 2])
def test_refine_launch_matches_oracle(response):
    """The refine study's launch: 4096 candidates near the two-year bank's injections at
    N_seg 16 in one gradient call (with the work-item split a batch of this size takes),
    with the long-wavelength and the TDI-1.5 response; 32 candidates spread over the
    batch against the oracle at the bounds above."""
    from paper_2510_19047_b300.binding import TFS
    D = synth.cached(synth.two_year_two_channel)
    cand = synth.candidates_near(D.injections, 4096, seed=2005)
    c = TFS(0, pn_order=D.pn_order, response=response)
    c.load_tf_data(D.d, D.dt, D.dT, D.t0)
    c.set_noise_weights(D.w, D.mask)
    u, g = c.grad_statistic(cand, 16)
    idx = np.linspace(0, cand.shape[1] - 1, 32).astype(int)
    u, g = np.asarray(u)[idx], np.asarray(g)[:, idx]
    kw = dict(pn_order=1, response=response)
    ref_u, ref_g = oracle.gradient(D.d, D.w, D.mask, cand[:, idx], 16, D.dT, **kw)
    S = oracle.gradient_scale(D.d, D.w, D.mask, cand[:, idx], 16, D.dT, tranche_level=True, **kw)
    np.testing.assert_allclose(u, ref_u, rtol=1e-4)
    assert np.all(np.abs(g[3]) <= PHI0_TOL * ref_u)
    for p in (0, 1, 2, 4, 5, 6, 7):
        err = np.abs(g[p] - ref_g[p])
        assert np.all(err <= GRAD_TOL * S[p]), (p, (err / S[p]).max())
        big = np.abs(ref_g[p]) >= 0.2 * S[p]
        assert np.all(err[big] <= 1e-4 * np.abs(ref_g[p][big])), p

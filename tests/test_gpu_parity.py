"""CUDA paths against the FP64 oracle, element by element on the same seeded inputs.

Tolerances (relative error of Upsilon per template and level):
  FP64 path          1e-10 at every segment length (the chirp constants t_c, P5, P3
                     and each tranche's absolute phase are carried in double-double, so
                     a phase of ~1e7 rad keeps ~1e-16 cycles)
  plain FP32 path    1e-4
  mixed, FP32 pixels 1e-4
  mixed, FP16 pixels max 1.5e-3, p99 1e-3   (3x and 2x the FP16 unit roundoff 2^-11)
  mixed, BF16 pixels max 1.2e-2, p99 8e-3   (3x and 2x the BF16 unit roundoff 2^-8)
  mixed, u and w FP16, template values FP16   max 2e-3, p99 1.5e-3 (two independent
                     roundings of 2^-11 per bin: the pixel's and the template value's)
  mixed, u and w BF16, template values FP16   max 1.2e-2, p99 8e-3 (the BF16 pixel rounding
                     dominates)
The reduced-precision bounds follow from rounding u = d~/S once to the storage type
(w = 1/S is stored in FP32): each pixel carries an independent relative error below the
unit roundoff, so |Z_n| moves by a random fraction of it and Upsilon by about twice
that.
"""
import numpy as np
import pytest

import oracle
from paper_2510_19047_b300 import synth

pytestmark = pytest.mark.gpu

TOL = {("fp64", "f16"): (1e-10, 1e-10), ("plain", "f16"): (1e-4, 1e-4),
       ("mixed", "f32"): (1e-4, 1e-4), ("mixed", "f16"): (1.5e-3, 1e-3),
       ("mixed", "bf16"): (1.2e-2, 8e-3),
       ("mixed", "f16all"): (2e-3, 1.5e-3), ("mixed", "bf16all"): (1.2e-2, 8e-3)}
CASES = list(TOL)
FP64_TOL = 1e-10


def rel_err(got, ref):
    got, ref = np.asarray(got, float), np.asarray(ref, float)
    assert np.all(np.isfinite(got))
    zero = ref == 0
    assert np.all(got[zero] == 0)
    r = np.abs(got[~zero] - ref[~zero]) / ref[~zero]
    return (r.max(), np.percentile(r, 99)) if r.size else (0.0, 0.0)


def ctx_for(D, path, pixel, **kw):
    from paper_2510_19047_b300.binding import TFS
    c = TFS(0, path=path, pixel=pixel, pn_order=D.pn_order, response=D.response, **kw)
    c.load_tf_data(D.d, D.dt, D.dT, D.t0)
    c.set_noise_weights(D.w, D.mask)
    return c


@pytest.fixture(scope="module")
def week():
    return synth.week_one_channel(seed=0)


@pytest.fixture(scope="module")
def ae45():
    return synth.two_year_two_channel(seed=77, n_inj=3, n_tranche=384, L=2048)


@pytest.fixture(scope="module")
def ae45_bank(ae45):
    th = synth.two_year_bank(253, seed=5)  # ragged: not a multiple of 32 or 128
    th[:, :3] = ae45.injections
    return th


@pytest.mark.parametrize("path,pixel", CASES)
def test_week_one_channel(week, path, pixel):
    th = synth.week_bank(1024, 0)
    ref, rneff, rnact, rnnc = oracle.statistic(week.d, week.w, week.mask, th, 8, week.dT)
    c = ctx_for(week, path, pixel)
    got, neff, diag = c.eval_statistic(th, 8, diag=True)
    mx, p99 = rel_err(got, ref)
    tol = FP64_TOL if path == "fp64" else TOL[(path, pixel)][0]
    assert mx < tol and p99 < max(tol, TOL[(path, pixel)][1]), (mx, p99)
    assert np.array_equal(neff, rneff)
    assert np.array_equal(diag[0], rnact) and np.array_equal(diag[1], rnnc)


def test_week_long_coherent_segments(week):
    """N_seg down to 1 (week-long coherent segments) on the slow chirps of the week grid
    (sweep ~5e-5 bins per tranche), where the dominant bin's W'' is a difference across
    2/sigma^2 bins that a per-tranche |Z|^2/N does not see but a long coherent sum does.
    Mixed FP32 pixels (single-mode and harmonic kernels) keep the FP32 bound at every
    level. The plain path evaluates the printed C(v2) - C(v1), S(v2) - S(v1) in FP32:
    with C, S ~ 1/2 and differences ~1e-3 on the non-central bins it keeps ~6e-5 of
    each, which adds up coherently over the segment; its bound at N_seg = 1 is 1e-3."""
    th = synth.week_bank(1024, 0)
    lev = [512, 64, 8, 1]
    refs = [oracle.statistic(week.d, week.w, week.mask, th, L, week.dT)[0] for L in lev]
    for path, harm, tol1 in (("mixed", False, 1e-4), ("mixed", True, 1e-4), ("plain", False, 1e-3)):
        c = ctx_for(week, path, "f32")
        if harm:
            c.set_harmonics([1.0], [1.0])
        got, _, _ = c.eval_statistic(th, lev)
        for i, L in enumerate(lev):
            mx, _ = rel_err(got[i], refs[i])
            assert mx < (tol1 if L == 1 else 1e-4), (path, harm, L, mx)


def _round_pixels(D, pixel):
    """(d', w') whose u' = d' w' and w' are the pixels the mixed path stores: u = d w and
    w scaled by the library's powers of two (largest |component| to 2^14 < 2^ceil(log2)),
    rounded to FP32, u then to FP16 or BF16 (round to nearest even; w stays FP32),
    scaled back."""
    act = D.w > 0
    u = np.where(act, D.d * D.w, 0)
    umax = max(np.abs(u.real).max(), np.abs(u.imag).max())
    su = 2.0 ** (14 - int(np.ceil(np.log2(umax))))
    sw = 2.0 ** (14 - int(np.ceil(np.log2(D.w.max()))))

    def rnd(x):
        x = np.asarray(x, np.float64).astype(np.float32)
        if pixel == "f16":
            return x.astype(np.float16).astype(np.float64)
        b = x.view(np.uint32).astype(np.uint64)
        b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
        return b.astype(np.uint32).view(np.float32).astype(np.float64)

    wq = np.where(act, (D.w * sw).astype(np.float32).astype(np.float64) / sw, 0.0)
    uq = (rnd(u.real * su) + 1j * rnd(u.imag * su)) / su
    dq = np.where(wq > 0, uq / np.where(wq > 0, wq, 1.0), 0)
    return dq, wq


@pytest.mark.parametrize("pixel", ["f16", "bf16"])
def test_reduced_precision_pixels_are_the_only_rounding(week, pixel):
    """The FP16/BF16 paths against the oracle run on the same pixels rounded to the
    storage type: apart from storing u and w, they compute at FP32 accuracy. At N_seg = 1
    Upsilon is chi^2 with 2 degrees of freedom and can be ~1e-3 of its mean, so the pixel
    rounding alone moves it by up to ~7e-3 (FP16) or ~7e-2 (BF16) against the unrounded
    oracle. Like the FP32-pixel instantiation they form the offset of the bin below f_nm
    from x - rint(x), not from aa = f_nm/df - k_c ~ -1 (which would leave W'' of that bin
    ~1e-3 off for slow chirps, adding up over coherent tranches to 9.0e-5 at N_seg = 8
    and 6.5e-4 at N_seg = 1 on this grid); with it the FP32-arithmetic bound 1e-4 holds
    at every N_seg (2.5e-5 at N_seg = 1 measured with FP32 pixels)."""
    th = synth.week_bank(1024, 0)
    lev = [512, 64, 8, 1]
    dq, wq = _round_pixels(week, pixel)
    c = ctx_for(week, "mixed", pixel)
    got, _, _ = c.eval_statistic(th, lev)
    for i, L in enumerate(lev):
        ref = oracle.statistic(dq, wq, week.mask, th, L, week.dT)[0]
        mx, _ = rel_err(got[i], ref)
        assert mx < 1e-4, (pixel, L, mx)


@pytest.mark.parametrize("path,pixel", CASES)
def test_two_channel_response_gaps_levels(ae45, ae45_bank, path, pixel):
    lev = [128, 32, 8]
    refs = [oracle.statistic(ae45.d, ae45.w, ae45.mask, ae45_bank, L, ae45.dT, pn_order=1,
                             response=1) for L in lev]
    c = ctx_for(ae45, path, pixel)
    got, neff, diag = c.eval_statistic(ae45_bank, lev, diag=True)
    for i, (ref, rneff, rnact, _) in enumerate(refs):
        mx, p99 = rel_err(got[i], ref)
        tol = FP64_TOL if path == "fp64" else TOL[(path, pixel)][0]
        assert mx < tol and p99 < max(tol, TOL[(path, pixel)][1]), (lev[i], mx, p99)
        assert np.array_equal(neff[i], rneff)
    # the double-float track decides the window like the FP64 oracle
    assert np.abs(diag[0] - refs[0][2]).max() <= (0 if path != "mixed" else 1)


@pytest.fixture(scope="module")
def ae45_tdi():
    # 45 days of A/E data whose injections went through the TDI-1.5 single-link response
    return synth.cached(synth.two_year_two_channel, seed=78, n_inj=2, n_tranche=384, L=2048,
                        response="tdi")


@pytest.mark.parametrize("path,pixel", CASES)
def test_tdi_response(ae45_tdi, path, pixel):
    """Response code 2 (TDI-1.5 transfer per tranche) against the oracle, with the
    injections themselves in the bank."""
    D = ae45_tdi
    assert D.response == 2
    th = synth.two_year_bank(94, seed=9)
    th = np.concatenate([D.injections, th], axis=1)
    lev = [128, 8]
    refs = [oracle.statistic(D.d, D.w, D.mask, th, L, D.dT, pn_order=1, response=2) for L in lev]
    c = ctx_for(D, path, pixel)
    got, neff, diag = c.eval_statistic(th, lev, diag=True)
    for i, (ref, rneff, rnact, _) in enumerate(refs):
        mx, p99 = rel_err(got[i], ref)
        tol = FP64_TOL if path == "fp64" else TOL[(path, pixel)][0]
        assert mx < tol and p99 < max(tol, TOL[(path, pixel)][1]), (lev[i], mx, p99)
        assert np.array_equal(neff[i], rneff)
    # the injections stand far above the noise (E[Upsilon] = 2 N_eff in noise)
    assert np.all(refs[1][0][:2] > 4 * 2 * refs[1][1][:2])


def fast_chirp_bank(n, seed):
    """Half the bank sweeps 0.01-0.05 bins per tranche (sigma = df sqrt(2/fdot) > 6: only
    the two bins next to f_nm can need the general Fresnel form, and some tranches hold
    a bin inside their sweep), half sweeps ~1-3 bins (sigma < 6: general bins across
    the window, the mixed kernel's loop path)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    th = synth.two_year_bank(n, seed=seed + 1)
    h = n // 2
    th[0, :h] = rng.uniform(20, 30, h)
    th[2, :h] = rng.uniform(0.022, 0.03, h)
    th[0, h:] = rng.uniform(50, 60, n - h)
    th[2, h:] = rng.uniform(0.05, 0.07, n - h)
    return th


@pytest.mark.parametrize("path,pixel", CASES)
def test_fast_chirps_general_bins(ae45, path, pixel):
    th = fast_chirp_bank(96, seed=31)
    lev = [64, 8]
    refs = [oracle.statistic(ae45.d, ae45.w, ae45.mask, th, L, ae45.dT, pn_order=1, response=1)
            for L in lev]
    c = ctx_for(ae45, path, pixel)
    got, neff, diag = c.eval_statistic(th, lev, diag=True)
    for i, (ref, rneff, _, _) in enumerate(refs):
        assert np.count_nonzero(ref) > 0.9 * th.shape[1]
        mx, p99 = rel_err(got[i], ref)
        tol = FP64_TOL if path == "fp64" else TOL[(path, pixel)][0]
        assert mx < tol and p99 < max(tol, TOL[(path, pixel)][1]), (lev[i], mx, p99)
        assert np.array_equal(neff[i], rneff)
    # both halves really exercise their branch: sigma > 6 vs < 6 at the first tranche
    df = 1.0 / ae45.dT
    Mc = th[0] * 4.925490947e-6
    fdot = (96 / 5) * np.pi ** (8 / 3) * Mc ** (5 / 3) * th[2] ** (11 / 3)
    sig = df * np.sqrt(2 / fdot)
    assert np.all(sig[:48] > 6) and np.all(sig[48:] < 6)


@pytest.mark.parametrize("path", ["fp64", "plain", "mixed"])
def test_per_template_segment_counts(ae45, ae45_bank, path):
    th = ae45_bank[:, :96]
    choices = np.array([128, 32, 8, 1], np.int32)
    ns = choices[np.arange(th.shape[1]) % 4]
    c = ctx_for(ae45, path, "f32")
    got, neff, _ = c.eval_statistic(th, ns, per_template=True)
    for L in choices:
        tol = {"fp64": FP64_TOL, "plain": 1e-4, "mixed": 1e-4}[path]
        sel = ns == L
        ref, rneff, _, _ = oracle.statistic(ae45.d, ae45.w, ae45.mask, th[:, sel], int(L), ae45.dT,
                                            pn_order=1, response=1)
        assert rel_err(got[sel], ref)[0] < tol
        assert np.array_equal(neff[sel], rneff)


def test_device_and_host_pointers_agree(ae45, ae45_bank):
    import torch
    c = ctx_for(ae45, "mixed", "f16")
    host, _, _ = c.eval_statistic(ae45_bank, [64, 8])
    dev, _, _ = c.eval_statistic(torch.from_numpy(ae45_bank).cuda(), [64, 8])
    torch.cuda.synchronize()
    assert np.array_equal(host, dev.cpu().numpy())  # deterministic, bit for bit
    again, _, _ = c.eval_statistic(ae45_bank, [64, 8])
    assert np.array_equal(host, again)


def test_edge_cases(ae45):
    from paper_2510_19047_b300.binding import TFS, TFSError
    for path in ("fp64", "plain", "mixed"):
        c = ctx_for(ae45, path, "f16")
        # empty batch
        s, n, _ = c.eval_statistic(np.zeros((8, 0)), 8)
        assert s.shape == (0,)
        # out of band (above the top bin), non-physical, and one ordinary template
        th = synth.two_year_bank(3, seed=1)
        th[2, 0] = 0.3       # f_0 above (N_bins - 11) df
        th[0, 1] = -5.0      # M_c < 0
        s, n, d = c.eval_statistic(th, [16, 4], diag=True)
        assert np.all(s[:, :2] == 0) and np.all(n[:, :2] == 0) and np.all(d[:, :2] == 0)
        assert np.all(s[:, 2] > 0)
        # N_seg must divide N_t
        with pytest.raises(TFSError, match="NSEG"):
            c.eval_statistic(th, 7)
        with pytest.raises(TFSError, match="ARG"):
            c.eval_statistic(th, [1, 2, 4, 8, 16])
    # a grid whose tranches are all gapped
    D = synth.TFData(d=ae45.d, w=ae45.w, mask=np.zeros_like(ae45.mask), dt=ae45.dt, dT=ae45.dT,
                     pn_order=1, response=1)
    c = ctx_for(D, "mixed", "f16")
    s, n, _ = c.eval_statistic(synth.two_year_bank(40, seed=3), 16)
    assert np.all(s == 0) and np.all(n == 0)
    # the mixed path folds at most 1024 finest segments; the FP64 path has no such limit
    big = synth.TFData(d=np.zeros((1, 2048, 64), complex), w=np.ones((1, 2048, 64)),
                       mask=np.ones(2048, np.uint8), dt=5.0, dT=640.0)
    c = ctx_for(big, "mixed", "f16")
    with pytest.raises(TFSError, match="ARG"):
        c.eval_statistic(synth.week_bank(4), 2048)
    c.set_options(path="fp64")
    c.eval_statistic(synth.week_bank(4), 2048)
    # calls before data is loaded
    c = TFS(0)
    with pytest.raises(TFSError, match="STATE"):
        c.eval_statistic(synth.week_bank(4), 1)
    with pytest.raises(TFSError, match="STATE"):
        c.set_noise_weights(np.ones((1, 4, 64)))
    # invalid weights are rejected
    c.load_tf_data(week_like(), 5.0, 1280.0)
    w = np.ones((1, 16, 64))
    w[0, 3, 5] = -1.0
    with pytest.raises(TFSError, match="ARG"):
        c.set_noise_weights(w)


def week_like():
    return np.zeros((1, 16, 64), complex)


def test_select_top_matches_stable_sort():
    from paper_2510_19047_b300.binding import TFS
    rng = np.random.default_rng(3)
    c = TFS(0)
    for n, k in ((1, 1), (1000, 10), (100_003, 1000)):
        x = np.round(rng.normal(size=n), 2)  # many ties
        idx = c.select_top(x, k)
        ref = np.lexsort((np.arange(n), -x))[:k]
        assert np.array_equal(idx, ref)
    x = rng.normal(size=5000)
    x[7] = np.nan
    idx = c.select_top(x, 5000)
    assert idx[-1] == 7


def test_ascent_step_update():
    from paper_2510_19047_b300.binding import TFS
    rng = np.random.default_rng(4)
    th = synth.two_year_bank(300, seed=8)
    g = rng.normal(size=th.shape)
    step = np.array([1e-3, 1e-4, 1e-6, 0.1, 0.1, 0.1, 0.1, 0.1])
    lo = np.array([5, 0.05, 1e-4, 0, 0, -np.pi / 2, 0, 0])
    hi = np.array([100, 0.25, 0.1, 2 * np.pi, 2 * np.pi, np.pi / 2, np.pi, np.pi])
    ref = th + step[:, None] * g
    for p in (0, 1, 2, 5, 7):
        ref[p] = np.clip(ref[p], lo[p], hi[p])
    ref[3] = np.mod(ref[3], 2 * np.pi)
    ref[4] = np.mod(ref[4], 2 * np.pi)
    ref[6] = np.mod(ref[6], np.pi)
    c = TFS(0)
    out = th.copy()
    c.ascent_step(out, g, step, lo, hi)
    np.testing.assert_allclose(out, ref, rtol=1e-14, atol=1e-14)


@pytest.fixture(scope="module")
def two_year():
    return synth.cached(synth.two_year_two_channel)


def test_two_year_full_bank_sampled(two_year):
    """The bench workload (1e6 templates, N_seg 256/64/16 in one mixed launch): 120
    templates spread over the sorted queue's range against the oracle (max and p99 at the
    FP16 bounds), and properties that hold for every template."""
    import torch
    D = two_year
    lev = [256, 64, 16]
    th = synth.two_year_bank(1_000_000, seed=2002)
    c = ctx_for(D, "mixed", "f16")
    st, ne, dg = c.eval_statistic(torch.from_numpy(th).cuda(), lev, diag=True)
    st, ne, dg = st.cpu().numpy(), ne.cpu().numpy(), dg.cpu().numpy()
    assert np.all(np.isfinite(st)) and np.all(st >= 0)
    assert np.all(ne <= np.array(lev)[:, None])
    # nested segmentations (Cauchy-Schwarz), up to the mixed-precision error
    assert np.all(st[0] >= st[1] * (1 - 3e-3)) and np.all(st[1] >= st[2] * (1 - 3e-3))
    # noise-dominated bank: Upsilon ~ chi^2 with 2 N_eff dof on average
    act = ne[0] > 0
    assert abs(np.mean(st[0][act]) / np.mean(2 * ne[0][act]) - 1) < 0.02
    idx = np.linspace(0, th.shape[1] - 1, 120).astype(int)
    for i, L in enumerate(lev):
        ref, rneff, rnact, _ = oracle.statistic(D.d, D.w, D.mask, th[:, idx], L, D.dT,
                                                pn_order=1, response=1)
        mx, p99 = rel_err(st[i, idx], ref)
        assert mx < TOL[("mixed", "f16")][0] and p99 < TOL[("mixed", "f16")][1], (L, mx, p99)
        assert np.array_equal(ne[i, idx], rneff)
        if i == 0:  # active tranches per template: the double-float window decision
            assert np.abs(dg[0, idx] - rnact).max() <= 1
    # FP64 and plain paths on the sampled templates
    for path in ("fp64", "plain"):
        c2 = ctx_for(D, path, "f16")
        got, _, _ = c2.eval_statistic(th[:, idx], lev)
        for i, L in enumerate(lev):
            tol = FP64_TOL if path == "fp64" else 1e-4
            ref = oracle.statistic(D.d, D.w, D.mask, th[:, idx], L, D.dT, pn_order=1, response=1)[0]
            assert rel_err(got[i], ref)[0] < tol, (path, L)


@pytest.mark.parametrize("pixel", ["f32", "bf16"])
def test_two_year_full_bank_sampled_pixels(two_year, pixel):
    """The bench bank (1e6 templates, N_seg 256/64/16 in one mixed launch) with FP32
    pixels (the bench's equal-accuracy leg, held to the FP32 path's 1e-4) and with BF16
    u (a precision-study variant, at its stated bound): 120 templates spread over the
    sorted queue's range against the oracle, N_eff exact."""
    import torch
    D = two_year
    lev = [256, 64, 16]
    th = synth.two_year_bank(1_000_000, seed=2002)
    c = ctx_for(D, "mixed", pixel)
    st, ne, _ = c.eval_statistic(torch.from_numpy(th).cuda(), lev)
    st, ne = st.cpu().numpy(), ne.cpu().numpy()
    assert np.all(np.isfinite(st)) and np.all(st >= 0)
    idx = np.linspace(0, th.shape[1] - 1, 120).astype(int)
    for i, L in enumerate(lev):
        ref, rneff, _, _ = oracle.statistic(D.d, D.w, D.mask, th[:, idx], L, D.dT,
                                            pn_order=1, response=1)
        mx, p99 = rel_err(st[i, idx], ref)
        assert mx < TOL[("mixed", pixel)][0] and p99 < TOL[("mixed", pixel)][1], (L, mx, p99)
        assert np.array_equal(ne[i, idx], rneff)


def test_two_year_full_bank_sampled_tdi(two_year):
    """The TDI study's workload: the bench bank (1e6 templates, N_seg 256/64/16 in one
    mixed launch, FP16 pixels) with the TDI-1.5 response (code 2): 120 templates spread
    over the sorted queue's range against the oracle (max and p99 at the FP16 bounds),
    N_eff exact, the active-tranche count within one."""
    import torch
    from paper_2510_19047_b300.binding import TFS
    D = two_year
    lev = [256, 64, 16]
    th = synth.two_year_bank(1_000_000, seed=2002)
    c = TFS(0, path="mixed", pixel="f16", pn_order=D.pn_order, response=2)
    c.load_tf_data(D.d, D.dt, D.dT, D.t0)
    c.set_noise_weights(D.w, D.mask)
    st, ne, dg = c.eval_statistic(torch.from_numpy(th).cuda(), lev, diag=True)
    st, ne, dg = st.cpu().numpy(), ne.cpu().numpy(), dg.cpu().numpy()
    assert np.all(np.isfinite(st)) and np.all(st >= 0)
    idx = np.linspace(0, th.shape[1] - 1, 120).astype(int)
    for i, L in enumerate(lev):
        ref, rneff, rnact, _ = oracle.statistic(D.d, D.w, D.mask, th[:, idx], L, D.dT,
                                                pn_order=1, response=2)
        mx, p99 = rel_err(st[i, idx], ref)
        assert mx < TOL[("mixed", "f16")][0] and p99 < TOL[("mixed", "f16")][1], (L, mx, p99)
        assert np.array_equal(ne[i, idx], rneff)
        if i == 0:
            assert np.abs(dg[0, idx] - rnact).max() <= 1


def _four_bin_window_share(D, th):
    """Per template, the share of its active tranches that sit in 32-tranche blocks whose
    general-form bins all lie in jp = -2 .. 1 with at least one lane beyond jp = -1, 0:
    the blocks the statistic kernel evaluates in its four-general-bin window. From the
    oracle's track with the kernel's test (a bin needs the general form when |v| <= 6
    on either offset or the sweep crosses it: jp in [ceil(a - 6/sigma), floor(a + eps +
    6/sigma)], a = f/df - ceil(f/df), with a 0.01-bin margin)."""
    from oracle.api import PN_1PN, RESP_LW
    live = np.flatnonzero(D.mask)
    df = 1.0 / D.dT
    share = np.zeros(th.shape[1])
    for j in range(th.shape[1]):
        tr = oracle.track(th[:, j], live * D.dT, pn_order=PN_1PN, response=RESP_LW)
        x, fd = tr["f"] / df, tr["fdot"]
        ok = np.isfinite(x) & (fd > 0) & (np.ceil(x) - 10 >= 1) & (np.ceil(x) + 10 <= D.n_bins - 1)
        if not ok.any():
            continue
        fd = np.where(fd > 0, fd, 1.0)
        r6 = 6.0 / (df * np.sqrt(2.0 / fd))
        a = x - np.ceil(x)
        lo = np.ceil(a - r6 - 0.01)
        hi = np.floor(a + fd * D.dT * D.dT + r6 + 0.01)
        act = np.flatnonzero(ok)
        n4 = 0
        for b0 in range(act[0], act[-1] + 1, 32):
            o = ok[b0:b0 + 32]
            if o.any():
                JLO, JHI = lo[b0:b0 + 32][o].min(), hi[b0:b0 + 32][o].max()
                if JLO >= -2 and JHI <= 1 and not (JLO >= -1 and JHI <= 0):
                    n4 += int(o.sum())
        share[j] = n4 / ok.sum()
    return share


@pytest.mark.parametrize("pixel", ["f16", "f32"])
def test_four_general_bin_window(two_year, pixel):
    """Templates of the bench bank chosen for the tranche blocks that the statistic
    kernel evaluates in its four-general-bin window (18 % of the units on this bank),
    against the oracle at N_seg 256/64/16."""
    D = two_year
    pool = synth.two_year_bank(400, seed=2002)
    share = _four_bin_window_share(D, pool)
    pick = np.argsort(share)[-16:]
    assert share[pick].min() > 0.3  # these templates really use that window
    th = pool[:, pick]
    lev = [256, 64, 16]
    got, neff, _ = ctx_for(D, "mixed", pixel).eval_statistic(th, lev)
    tol = TOL[("mixed", pixel)][0]
    for i, L in enumerate(lev):
        ref, rneff, _, _ = oracle.statistic(D.d, D.w, D.mask, th, L, D.dT, pn_order=1, response=1)
        mx, _ = rel_err(got[i], ref)
        assert mx < tol, (pixel, L, mx)
        assert np.array_equal(neff[i], rneff)


def test_graph_replay_with_profiling(ae45, ae45_bank):
    """The bench's call pattern: a profiled context replaying a CUDA graph, first with
    the diagnostic outputs and then without, repeatedly; the kernel times are reported
    and the results match the direct launch bit for bit."""
    lev = [64, 16, 4]
    ref, _, rdiag = ctx_for(ae45, "mixed", "f16").eval_statistic(ae45_bank, lev, diag=True)
    c = ctx_for(ae45, "mixed", "f16", use_graph=1, profile=1)
    got, _, diag = c.eval_statistic(ae45_bank, lev, diag=True)
    assert np.array_equal(got, ref) and np.array_equal(diag, rdiag)
    for _ in range(3):
        got, _, _ = c.eval_statistic(ae45_bank, lev)
        assert np.array_equal(got, ref)
        prof = c.last_profile()
        assert prof["statistic"] > 0 and prof["setup"] > 0
    shape = c.last_launch_shape()
    assert shape["threads_per_cta"] in (128, 256) and shape["ctas"] >= 1
    assert shape["tune_trials"] >= 8


def test_graph_replay_checked_mode_and_launch_shapes(ae45, ae45_bank):
    """CUDA-graph replay, checked mode and every launch shape (each compiled tile variant
    at 4 and 8 warps per CTA) give the direct path's result bit for bit (templates are
    independent and the fold is deterministic)."""
    import torch
    lev = [64, 16, 4]
    base = ctx_for(ae45, "mixed", "f16")
    ref, rneff, _ = base.eval_statistic(ae45_bank, lev)
    shapes = [{"warps_per_cta": w, "tile_variant": v} for v in range(3) for w in (4, 8)]
    for kw in [{"use_graph": 1}, {"checked": 1}, {"sort": 0},
               {"use_graph": 1, "warps_per_cta": 4, "tile_variant": 2}] + shapes:
        c = ctx_for(ae45, "mixed", "f16", **kw)
        for _ in range(2):  # second call replays the captured graph
            got, neff, _ = c.eval_statistic(ae45_bank, lev)
            assert np.array_equal(got, ref) and np.array_equal(neff, rneff), kw
        if "tile_variant" in kw:  # the compiled variant asked for is the one launched
            sh = c.last_launch_shape()
            assert sh["variant"] == kw["tile_variant"], (kw, sh)
            assert sh["threads_per_cta"] == 32 * kw["warps_per_cta"], (kw, sh)
    # a graph re-captures when the batch shape changes, and works on device arrays
    c = ctx_for(ae45, "mixed", "f16", use_graph=1)
    sub = ae45_bank[:, :100]
    got, _, _ = c.eval_statistic(torch.from_numpy(sub).cuda(), lev)
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), ref[:, :100])
    got, _, _ = c.eval_statistic(ae45_bank, lev)
    assert np.array_equal(got, ref)

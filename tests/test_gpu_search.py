"""Search-step kernels (tfs_pso_init, tfs_pso_step, tfs_refine_step) against their NumPy
restatement (tests/search_ref.py) on the same state, and the swarm driver on objectives
with a known maximum."""
import ctypes
import math

import numpy as np
import pytest

import search_ref as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2510_19047_b300.binding import TFS
    return TFS(0)


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _swarm(ctx, lo, hi, P, seed, state, inertia=0.72, c1=1.49, c2=1.49):
    from paper_2510_19047_b300.binding import Swarm, _ptr
    t = [_dev(a) for a in (lo, hi) + tuple(state)]
    p = [_ptr(a)[0].value for a in t]
    sw = Swarm(lo.shape[0], P, p[0], p[1], inertia, c1, c2, seed, *p[2:])
    return sw, t


def test_pso_init_matches_numpy(ctx):
    rng = np.random.default_rng(1)
    S, P, seed = 3, 300, 0x1234_5678_9ABC
    lo = rng.uniform(-1, 0, (S, 8))
    hi = lo + rng.uniform(0, 2, (S, 8))
    hi[1, 4] = lo[1, 4]  # a fixed coordinate
    state = [np.zeros((8, S * P)), np.zeros((8, S * P)), np.zeros((8, S * P)), np.zeros(S * P),
             np.zeros((8, S)), np.zeros(S)]
    sw, t = _swarm(ctx, lo, hi, P, seed, state)
    ctx.pso_init(sw, t[2])
    want = R.pso_init(lo, hi, P, seed)
    for got, ref in zip(t[2:], want):
        np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("move", [1, 0])
def test_pso_step_matches_numpy(ctx, move):
    rng = np.random.default_rng(2)
    S, P, seed, it = 4, 257, 99, 17  # P not a multiple of the block size
    lo = rng.uniform(-1, 0, (S, 8))
    hi = lo + rng.uniform(0.1, 2, (S, 8))
    lo[:, 3], hi[:, 3] = 0.0, 2 * np.pi          # phi_0 spans its period: wraps
    lo[0, 6], hi[0, 6] = 0.0, np.pi              # psi of swarm 0 wraps, others clip
    lo[:, 6] = np.where(np.arange(S) == 0, 0.0, 0.2)
    hi[:, 6] = np.where(np.arange(S) == 0, np.pi, 1.0)
    hi[2, 1] = lo[2, 1]                          # a fixed coordinate
    x = lo.T[:, np.repeat(np.arange(S), P)] + (hi - lo).T[:, np.repeat(np.arange(S), P)] * \
        rng.uniform(0, 1, (8, S * P))
    v = rng.normal(0, 0.5, (8, S * P))           # large: some coordinates clip
    pbest = x + rng.normal(0, 0.1, (8, S * P))
    pval = rng.normal(0, 1, S * P)
    pval[5] = -np.inf
    f = rng.normal(0, 1, S * P)
    f[P + 3] = f[P + 9] = 10.0                   # a tie: the lower index wins
    f[3 * P:] = np.nan                           # swarm 3: nothing improves
    gbest = rng.normal(0, 1, (8, S))
    gval = np.array([0.5, 1.0, 20.0, 0.0])      # swarm 2 keeps its best
    state = [x, v, pbest, pval, gbest, gval]
    sw, t = _swarm(ctx, lo, hi, P, seed, state, 0.7, 1.4, 1.6)
    import torch
    hist = torch.full((it + 1, S), -1.0, dtype=torch.float64, device="cuda")
    ctx.pso_step(sw, _dev(f), it, move, hist)
    want = R.pso_step(lo, hi, P, seed, 0.7, 1.4, 1.6, x, v, pbest, pval, gbest, gval, f, it, move)
    names = ["x", "v", "pbest", "pval", "gbest", "gval"]
    for name, got, ref in zip(names, t[2:], want):
        g = got.cpu().numpy()
        if name in ("pbest", "pval", "gbest", "gval"):  # selections: exact
            assert np.array_equal(g, ref), name
        else:  # one FMA contraction apart at most
            np.testing.assert_allclose(g, ref, rtol=1e-14, atol=1e-14, err_msg=name)
    # swarm 1's new best is particle 3 (tied with particle 9), at its new personal best x
    assert want[5][1] == 10.0 and np.array_equal(want[4][:, 1], x[:, P + 3])
    assert np.array_equal(hist[it].cpu().numpy(), want[5])
    assert np.all(hist[:it].cpu().numpy() == -1.0)


def test_refine_step_matches_numpy(ctx):
    import torch
    from paper_2510_19047_b300.binding import Refine, _ptr
    rng = np.random.default_rng(3)
    n = 1000
    theta = np.stack([rng.uniform(10, 60, n), rng.uniform(0.1, 0.25, n),
                      rng.uniform(0.015, 0.03, n), rng.uniform(0, 6.28, n),
                      rng.uniform(0, 6.28, n), rng.uniform(-1.5, 1.5, n),
                      rng.uniform(0, 3.14, n), rng.uniform(0, 3.14, n)])
    stat = rng.uniform(0, 100, n)
    grad = rng.normal(0, 1, (8, n)) * np.array([1, 10, 1e8, 0, 1, 1, 1, 1])[:, None]
    best_theta = theta + rng.normal(0, 1e-3, (8, n))
    best_grad = rng.normal(0, 1, (8, n))
    best_stat = rng.uniform(0, 100, n)
    best_stat[:10] = -np.inf
    eta = rng.uniform(0.1, 1, n)
    sigma = np.repeat(np.array([1e-4, 1e-3, 1e-9, 0, 1e-3, 1e-3, 1e-3, 1e-3])[:, None], n, 1)
    sigma[0] *= theta[0]
    sigma[2] *= theta[2]
    sigma[:, 7] *= 1e6  # a candidate pushed past its bounds and wrap points
    lo = np.array([1.0, 0.01, 1e-5, 0.0, 0.0, -np.pi / 2, 0.0, 0.0])
    hi = np.array([200.0, 0.25, 1.0, 2 * np.pi, 2 * np.pi, np.pi / 2, np.pi, np.pi])
    d = [_dev(a) for a in (theta, best_theta, best_grad, best_stat, eta, sigma)]
    p = [_ptr(a)[0].value for a in d]
    arr8 = ctypes.c_double * 8
    rf = Refine(n, *p, arr8(*lo), arr8(*hi), 1.2, 0.5)
    mean = torch.empty(1, dtype=torch.float64, device="cuda")
    ctx.refine_step(rf, _dev(stat), _dev(grad), mean)
    want = R.refine_step(stat, grad, theta, best_theta, best_grad, best_stat, eta, sigma, lo, hi,
                         1.2, 0.5)
    np.testing.assert_allclose(d[0].cpu().numpy(), want[0], rtol=1e-14, atol=1e-14)
    for got, ref in zip(d[1:5], want[1:5]):
        assert np.array_equal(got.cpu().numpy(), ref)
    assert mean.item() == pytest.approx(want[5], rel=1e-14)


def bowl(center):
    import torch
    c = torch.as_tensor(center, dtype=torch.float64, device="cuda")

    def f(th):
        d = th - c[:, None]
        d[3] = torch.remainder(d[3] + math.pi, 2 * math.pi) - math.pi  # periodic phi_0
        return -(d * d).sum(0)
    return f


def test_swarm_finds_the_maximum_of_a_bowl(ctx):
    from paper_2510_19047_b300 import pso
    center = np.array([0.3, 0.7, -0.2, 6.1, 0.0, 0.1, 0.0, 0.0])
    lo = np.array([-1, -1, -1, 0, 0, -1, 0, 0.0])
    hi = np.array([1, 1, 1, 2 * math.pi, 0, 1, 0, 0.0])
    x, fx = pso.swarm(bowl(center), lo, hi, n_particles=64, n_iter=150, seed=3, tfs=ctx)
    x = x.cpu().numpy()
    assert fx.item() > -1e-6
    assert np.allclose(x[0][[0, 1, 2, 5]], center[[0, 1, 2, 5]], atol=1e-3)
    # phi_0 found across the wrap point (6.1 rad is near 2 pi)
    assert abs(((x[0, 3] - center[3] + math.pi) % (2 * math.pi)) - math.pi) < 1e-3
    # fixed coordinates stay put
    assert x[0, 4] == 0.0 and x[0, 6] == 0.0


def test_many_swarms_run_independently(ctx):
    import torch
    from paper_2510_19047_b300 import pso
    centers = [np.array([0.5, 0, 0, 1, 0, 0, 0, 0.0]), np.array([-0.5, 0, 0, 1, 0, 0, 0, 0.0])]

    def two(th):  # swarm s sees the bowl of centre s (particles are grouped by swarm)
        n = th.shape[1] // 2
        return torch.cat([bowl(centers[0])(th[:, :n]), bowl(centers[1])(th[:, n:])])
    lo = np.tile(np.array([-1, 0, 0, 1, 0, 0, 0, 0.0]), (2, 1))
    hi = np.tile(np.array([1, 0, 0, 1, 0, 0, 0, 0.0]), (2, 1))
    hist = []
    x, fx = pso.swarm(two, lo, hi, n_particles=32, n_iter=80, seed=4, history=hist, tfs=ctx)
    assert abs(x[0, 0].item() - 0.5) < 1e-3 and abs(x[1, 0].item() + 0.5) < 1e-3
    h = torch.stack(hist).cpu().numpy()
    assert h.shape == (81, 2)
    assert np.all(np.diff(h, axis=0) >= 0)  # the swarm best never decreases
    # the same seed gives the same run
    x2, _ = pso.swarm(two, lo, hi, n_particles=32, n_iter=80, seed=4, tfs=ctx)
    assert np.array_equal(x.cpu().numpy(), x2.cpu().numpy())


def test_search_steps_reject_host_state(ctx):
    from paper_2510_19047_b300.binding import Swarm, TFSError
    lo = np.zeros((1, 8))
    hi = np.ones((1, 8))
    host = [np.zeros((8, 4)), np.zeros((8, 4)), np.zeros((8, 4)), np.zeros(4), np.zeros((8, 1)),
            np.zeros(1)]
    sw = Swarm(1, 4, lo.ctypes.data, hi.ctypes.data, 0.7, 1.5, 1.5, 0,
               *[a.ctypes.data for a in host])
    with pytest.raises(TFSError):
        ctx.pso_init(sw, None)

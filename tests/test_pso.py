"""Particle-swarm driver on objectives with a known maximum (CPU), and on the statistic
of an injected chirp (GPU)."""
import math

import numpy as np
import pytest
import torch

from paper_2510_19047_b300 import pso


def bowl(center):
    c = torch.as_tensor(center, dtype=torch.float64)

    def f(th):
        d = th - c[:, None]
        d[3] = torch.remainder(d[3] + math.pi, 2 * math.pi) - math.pi  # periodic phi_0
        return -(d * d).sum(0)
    return f


def test_swarm_finds_the_maximum_of_a_bowl():
    center = np.array([0.3, 0.7, -0.2, 6.1, 0.0, 0.1, 0.0, 0.0])
    lo = np.array([-1, -1, -1, 0, 0, -1, 0, 0.0])
    hi = np.array([1, 1, 1, 2 * math.pi, 0, 1, 0, 0.0])
    x, fx = pso.swarm(bowl(center), lo, hi, n_particles=64, n_iter=150, seed=3)
    assert fx.item() > -1e-6
    assert np.allclose(x[0].numpy()[[0, 1, 2, 5]], center[[0, 1, 2, 5]], atol=1e-3)
    # phi_0 found across the wrap point (6.1 rad is near 2 pi)
    assert abs(((x[0, 3].item() - center[3] + math.pi) % (2 * math.pi)) - math.pi) < 1e-3
    # fixed coordinates stay put
    assert x[0, 4].item() == 0.0 and x[0, 6].item() == 0.0


def test_many_swarms_run_independently():
    centers = [np.array([0.5, 0, 0, 1, 0, 0, 0, 0.0]), np.array([-0.5, 0, 0, 1, 0, 0, 0, 0.0])]

    def two(th):  # swarm s sees the bowl of centre s (particles are grouped by swarm)
        n = th.shape[1] // 2
        return torch.cat([bowl(centers[0])(th[:, :n]), bowl(centers[1])(th[:, n:])])
    lo = np.tile(np.array([-1, 0, 0, 1, 0, 0, 0, 0.0]), (2, 1))
    hi = np.tile(np.array([1, 0, 0, 1, 0, 0, 0, 0.0]), (2, 1))
    hist = []
    x, fx = pso.swarm(two, lo, hi, n_particles=32, n_iter=80, seed=4, history=hist)
    assert abs(x[0, 0].item() - 0.5) < 1e-3 and abs(x[1, 0].item() + 0.5) < 1e-3
    h = torch.stack(hist).numpy()
    assert np.all(np.diff(h, axis=0) >= 0)  # the swarm best never decreases


@pytest.mark.gpu
def test_swarm_recovers_an_injection():
    from paper_2510_19047_b300 import synth
    from paper_2510_19047_b300.binding import TFS
    D = synth.week_one_channel(seed=0)
    c = TFS(0, pn_order=0, response=0)
    c.load_tf_data(D.d, D.dt, D.dT)
    c.set_noise_weights(D.w, D.mask)
    inj = D.injections[:, 0]
    u_inj = c.eval_statistic(D.injections, 8)[0][0]
    lo = inj.copy()
    hi = inj.copy()
    lo[0], hi[0] = inj[0] * (1 - 2e-3), inj[0] * (1 + 2e-3)
    lo[2], hi[2] = inj[2] * (1 - 1e-3), inj[2] * (1 + 1e-3)
    lo[3], hi[3] = 0.0, 2 * math.pi

    def obj(th):
        return c.eval_statistic(th, 8)[0]
    x, fx = pso.swarm(obj, lo, hi, n_particles=256, n_iter=60, seed=5, device="cuda")
    # M_c and f_0 trade along the chirp's ridge, so the value, not the position, is checked
    assert fx.item() > 0.95 * u_inj, (fx.item(), u_inj)
    assert abs(c.eval_statistic(x.T.contiguous(), 8)[0].item() - fx.item()) < 1e-9 * fx.item()

"""Particle-swarm driver on the statistic of an injected chirp (GPU). The swarm kernels
against their NumPy restatement and on objectives with a known maximum are in
test_gpu_search.py."""
import math

import numpy as np
import pytest

from paper_2510_19047_b300 import pso


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
    x, fx = pso.swarm(obj, lo, hi, n_particles=256, n_iter=60, seed=5, tfs=c)
    # M_c and f_0 trade along the chirp's ridge, so the value, not the position, is checked
    assert fx.item() > 0.95 * u_inj, (fx.item(), u_inj)
    assert abs(c.eval_statistic(x.T.contiguous(), 8)[0].item() - fx.item()) < 1e-9 * fx.item()

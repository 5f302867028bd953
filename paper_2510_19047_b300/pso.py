"""Particle-swarm maximisation of the statistic over parameter tiles.

The paper finds the maximum of Upsilon in each parameter tile with a particle swarm
optimiser (Sec. "Implementation details"). This is a standard global-best swarm with an
inertia weight. For each particle:

    v <- w v + c1 r1 (p - x) + c2 r2 (g - x),    x <- x + v,

where p is the particle's best position, g is its swarm's best, and r1, r2 ~ U(0, 1)
are drawn per coordinate (for wrapped angles p - x and g - x take the shorter way
round). Positions are wrapped for the angles (phi_0 and lambda mod 2 pi, psi mod pi)
where the tile spans the whole period, and clipped to the tile otherwise and for the
other parameters; clipping a coordinate stops its velocity. A parameter with lo == hi
stays fixed.

Many swarms, one per tile, run together. Every iteration evaluates all particles of all
swarms with one call of the objective on the device; the bookkeeping is elementwise
torch work on the same device.
"""
import math

import numpy as np

PERIOD = {3: 2 * math.pi, 4: 2 * math.pi, 6: math.pi}  # phi_0, lambda, psi


def swarm(objective, lo, hi, n_particles, n_iter, seed=0, inertia=0.72, c1=1.49, c2=1.49,
          device=None, history=None):
    """Maximise `objective` over boxes.

    objective: callable taking theta [8, N] (float64 tensor on `device`) and returning
    [N] values. lo, hi: [n_swarms, 8] (or [8]) box corners per swarm. Returns
    (best_theta [n_swarms, 8], best_value [n_swarms]) as tensors on `device`; if
    `history` is a list, the best value per swarm after every iteration is appended.
    """
    import torch
    dev = torch.device(device) if device is not None else torch.device("cpu")
    lo = torch.as_tensor(np.atleast_2d(lo), dtype=torch.float64, device=dev)
    hi = torch.as_tensor(np.atleast_2d(hi), dtype=torch.float64, device=dev)
    S = lo.shape[0]
    P = int(n_particles)
    g = torch.Generator(device=dev)
    g.manual_seed(int(seed))
    span = (hi - lo)[:, None, :]                         # [S, 1, 8]
    x = lo[:, None, :] + span * torch.rand((S, P, 8), generator=g, dtype=torch.float64, device=dev)
    v = 0.1 * span * (2 * torch.rand((S, P, 8), generator=g, dtype=torch.float64, device=dev) - 1)
    fixed = (span == 0)
    per = torch.zeros(8, dtype=torch.float64, device=dev)
    for k, T in PERIOD.items():
        per[k] = T
    # an angle wraps only where the tile spans its whole period; otherwise it is clipped
    periodic = (per > 0) & (span >= per * (1 - 1e-12))      # [S, 1, 8]

    def toward(d):
        # the shorter way round for wrapped angles
        half = 0.5 * per
        dw = torch.remainder(d + half, torch.where(per > 0, per, torch.ones_like(per))) - half
        return torch.where(periodic, dw, d)

    def evaluate(pos):
        th = pos.reshape(S * P, 8).T.contiguous()
        return objective(th).reshape(S, P)

    f = evaluate(x)
    pbest, pval = x.clone(), f.clone()
    gi = torch.argmax(pval, dim=1)
    gbest = pbest[torch.arange(S, device=dev), gi].clone()   # [S, 8]
    gval = pval[torch.arange(S, device=dev), gi].clone()
    for _ in range(int(n_iter)):
        r1 = torch.rand((S, P, 8), generator=g, dtype=torch.float64, device=dev)
        r2 = torch.rand((S, P, 8), generator=g, dtype=torch.float64, device=dev)
        v = inertia * v + c1 * r1 * toward(pbest - x) + c2 * r2 * toward(gbest[:, None, :] - x)
        v = torch.where(fixed, torch.zeros_like(v), v)
        x = x + v
        # angles wrap; everything else is clipped to the tile and loses its velocity there
        wrapped = x - per * torch.floor(x / torch.where(per > 0, per, torch.ones_like(per)))
        wrapped = torch.where(periodic, wrapped, x)
        clipped = torch.minimum(torch.maximum(wrapped, lo[:, None, :]), hi[:, None, :])
        hit = (clipped != wrapped) & ~periodic
        v = torch.where(hit, torch.zeros_like(v), v)
        x = torch.where(periodic & ~fixed, wrapped, clipped)
        f = evaluate(x)
        better = f > pval
        pbest = torch.where(better[..., None], x, pbest)
        pval = torch.where(better, f, pval)
        gi = torch.argmax(pval, dim=1)
        gv = pval[torch.arange(S, device=dev), gi]
        upd = gv > gval
        gbest = torch.where(upd[:, None], pbest[torch.arange(S, device=dev), gi], gbest)
        gval = torch.where(upd, gv, gval)
        if history is not None:
            history.append(gval.clone())
    return gbest, gval

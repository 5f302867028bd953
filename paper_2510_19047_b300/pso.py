"""Particle-swarm maximisation of the statistic over parameter tiles.

The paper finds the maximum of Upsilon in each parameter tile with a particle swarm
optimiser (Sec. "Implementation details"). This is a standard global-best swarm with an
inertia weight; for each particle and coordinate

    v <- w v + c1 r1 (p - x) + c2 r2 (g - x),    x <- x + v,

where p is the particle's best position, g is its swarm's best, and r1, r2 ~ U(0, 1)
(for wrapped angles p - x and g - x take the shorter way round). Positions are wrapped
for the angles (phi_0 and lambda mod 2 pi, psi mod pi) where the tile spans the whole
period, and clipped to the tile otherwise and for the other parameters; clipping a
coordinate stops its velocity. A parameter with lo == hi stays fixed.

Many swarms, one per tile, run together. Every iteration evaluates all particles of all
swarms with one call of the objective on the device (normally tfs_eval_statistic), and
one tfs_pso_step launch updates the bests and moves the swarm: the random draws
(Philox4x32-10 keyed by the seed) and the bookkeeping run in libtfs. This module only
allocates the device state and sequences the calls.
"""
import numpy as np

PERIOD = {3: 2 * np.pi, 4: 2 * np.pi, 6: np.pi}  # phi_0, lambda, psi


def swarm(objective, lo, hi, n_particles, n_iter, seed=0, inertia=0.72, c1=1.49, c2=1.49,
          device=0, history=None, tfs=None):
    """Maximise `objective` over boxes.

    objective: callable taking theta [8, S*P] (float64 CUDA tensor; particle i of swarm
    s in column s*P + i) and returning the [S*P] values as a float64 CUDA tensor.
    lo, hi: [n_swarms, 8] (or [8]) box corners per swarm. tfs: a binding.TFS context for
    the swarm kernels (a new one on `device` if None). Returns (best_theta [S, 8],
    best_value [S]) as CUDA tensors; if `history` is a list, the swarm bests after
    every step (n_iter + 1 rows of [S], the initial evaluation first) are appended.
    """
    import torch
    from .binding import TFS, Swarm, _ptr
    ctx = tfs if tfs is not None else TFS(device)
    dev = torch.device("cuda", ctx.device)
    lo = np.ascontiguousarray(np.atleast_2d(np.asarray(lo, dtype=np.float64)))
    hi = np.ascontiguousarray(np.atleast_2d(np.asarray(hi, dtype=np.float64)))
    if lo.shape != hi.shape or lo.shape[1] != 8:
        raise ValueError("lo and hi must be [n_swarms, 8]")
    S, P = lo.shape[0], int(n_particles)
    f64 = dict(dtype=torch.float64, device=dev)
    lo_d = torch.from_numpy(lo).to(dev)
    hi_d = torch.from_numpy(hi).to(dev)
    x = torch.empty((8, S * P), **f64)
    v = torch.empty((8, S * P), **f64)
    pbest = torch.empty((8, S * P), **f64)
    pval = torch.empty(S * P, **f64)
    gbest = torch.empty((8, S), **f64)
    gval = torch.empty(S, **f64)
    hist = torch.empty((int(n_iter) + 1, S), **f64) if history is not None else None
    p = lambda t: _ptr(t)[0].value  # noqa: E731
    sw = Swarm(S, P, p(lo_d), p(hi_d), float(inertia), float(c1), float(c2), int(seed),
               p(x), p(v), p(pbest), p(pval), p(gbest), p(gval))
    ctx.pso_init(sw, x)
    for it in range(int(n_iter) + 1):
        f = objective(x)
        if not (f.is_cuda and f.dtype == torch.float64 and f.numel() == S * P):
            raise ValueError("the objective must return S*P float64 values on the device")
        ctx.pso_step(sw, f.contiguous(), it, it < int(n_iter), hist)
    if history is not None:
        history.extend(hist.unbind(0))
    return gbest.T.contiguous(), gval

"""NumPy restatements of the search-step kernels (test reference, CPU): Philox4x32-10
(Salmon, Moraes, Dror & Shaw, SC 2011), the particle-swarm step and the refinement
step, written from their definitions in include/tfs.h."""
import numpy as np

M0, M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
W0, W1 = np.uint64(0x9E3779B9), np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c, k):
    """c: uint [..., 4], k: uint [..., 2] -> uint64 [..., 4] (32-bit words)."""
    c = [np.asarray(c[..., i], dtype=np.uint64) for i in range(4)]
    k0 = np.asarray(k[..., 0], dtype=np.uint64)
    k1 = np.asarray(k[..., 1], dtype=np.uint64)
    for _ in range(10):
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c = [(hi1 ^ c[1] ^ k0) & MASK, lo1, (hi0 ^ c[3] ^ k1) & MASK, lo0]
        k0 = (k0 + W0) & MASK
        k1 = (k1 + W1) & MASK
    return np.stack(c, axis=-1)


def uniform2(c, k):
    """Two doubles in [0, 1) per block: top 53 bits of (w0, w1) and of (w2, w3)."""
    r = philox4x32_10(c, k)
    ab = (r[..., 0] << np.uint64(32)) | r[..., 1]
    cd = (r[..., 2] << np.uint64(32)) | r[..., 3]
    return (ab >> np.uint64(11)).astype(np.float64) * 2.0 ** -53, \
        (cd >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def pso_counter(particle, q, purpose, it):
    particle = np.asarray(particle, dtype=np.uint64)
    c = np.zeros(np.broadcast(particle, q).shape + (4,), dtype=np.uint64)
    c[..., 0] = particle & MASK
    c[..., 1] = (np.uint64(q) | (np.uint64(purpose) << np.uint64(8)) |
                 ((particle >> np.uint64(32)) << np.uint64(16))) & MASK
    c[..., 2] = np.uint64(it) & MASK
    c[..., 3] = (np.uint64(it) >> np.uint64(32)) & MASK
    return c


def key_of(seed):
    return np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)


PERIOD = np.array([0, 0, 0, 2 * np.pi, 2 * np.pi, 0, np.pi, 0])


def pso_init(lo, hi, P, seed):
    S = lo.shape[0]
    i = np.arange(S * P, dtype=np.uint64)
    x = np.empty((8, S * P))
    v = np.empty((8, S * P))
    s = (np.arange(S * P) // P)
    for q in range(8):
        r1, r2 = uniform2(pso_counter(i, q, 0, 0), key_of(seed))
        span = hi[s, q] - lo[s, q]
        x[q] = lo[s, q] + span * r1
        v[q] = 0.1 * span * (2 * r2 - 1)
    gbest = (0.5 * (lo + hi)).T.copy()
    return x, v, x.copy(), np.full(S * P, -np.inf), gbest, np.full(S, -np.inf)


def pso_step(lo, hi, P, seed, inertia, c1, c2, x, v, pbest, pval, gbest, gval, f, it, move):
    x, v, pbest, pval, gbest, gval = (a.copy() for a in (x, v, pbest, pval, gbest, gval))
    S = lo.shape[0]
    better = f > pval
    pval[better] = f[better]
    pbest[:, better] = x[:, better]
    for s in range(S):
        sl = slice(s * P, (s + 1) * P)
        vals = pval[sl]
        if np.all(np.isnan(vals)) or not np.any(vals > -np.inf):
            continue
        gi = int(np.nanargmax(vals))  # first (lowest) index of the maximum
        if vals[gi] > gval[s]:
            gval[s] = vals[gi]
            gbest[:, s] = pbest[:, s * P + gi]
    if not move:
        return x, v, pbest, pval, gbest, gval
    i = np.arange(S * P, dtype=np.uint64)
    sidx = np.arange(S * P) // P
    for q in range(8):
        lo_q, hi_q = lo[sidx, q], hi[sidx, q]
        span = hi_q - lo_q
        per = PERIOD[q]
        periodic = (per > 0) & (span >= per * (1 - 1e-12))
        dp = pbest[q] - x[q]
        dg = gbest[q, sidx] - x[q]
        if per > 0:
            wdp = np.mod(dp + 0.5 * per, per) - 0.5 * per
            wdg = np.mod(dg + 0.5 * per, per) - 0.5 * per
            dp = np.where(periodic, wdp, dp)
            dg = np.where(periodic, wdg, dg)
        r1, r2 = uniform2(pso_counter(i, q, 1, it), key_of(seed))
        vq = inertia * v[q] + c1 * r1 * dp + c2 * r2 * dg
        vq = np.where(span == 0, 0.0, vq)
        xn = x[q] + vq
        wrapped = xn - per * np.floor(xn / per) if per > 0 else xn
        clipped = np.minimum(np.maximum(xn, lo_q), hi_q)
        vq = np.where(~periodic & (clipped != xn), 0.0, vq)
        x[q] = np.where(periodic & (span != 0), wrapped, clipped)
        v[q] = vq
    return x, v, pbest, pval, gbest, gval


def refine_step(stat, grad, theta, best_theta, best_grad, best_stat, eta, sigma, lo, hi,
                eta_up, eta_down):
    best_theta, best_grad, best_stat, eta = (a.copy() for a in (best_theta, best_grad,
                                                                 best_stat, eta))
    acc = stat >= best_stat
    best_stat[acc] = stat[acc]
    best_theta[:, acc] = theta[:, acc]
    best_grad[:, acc] = grad[:, acc]
    eta = np.where(acc, eta * eta_up, eta * eta_down)
    sg = sigma * best_grad
    nrm = np.maximum(np.sqrt((sg * sg).sum(0)), 1e-300)
    nxt = best_theta + sigma * sg * (eta / nrm)[None, :]
    for q in range(8):
        if q in (3, 4):
            nxt[q] = nxt[q] - 2 * np.pi * np.floor(nxt[q] / (2 * np.pi))
        elif q == 6:
            nxt[q] = nxt[q] - np.pi * np.floor(nxt[q] / np.pi)
        else:
            nxt[q] = np.clip(nxt[q], lo[q], hi[q])
    return nxt, best_theta, best_grad, best_stat, eta, best_stat.mean()


NOISE_TAG = 0x4E4F4953


def noise(w, df, seed):
    """The noise-only data tfs_noise_realisation draws: d~ = sqrt(S/(4 df)) (g1 + i g2),
    S = 1/w (0 where w = 0), g1 + i g2 = sqrt(-2 ln(1 - a)) e^{2 pi i b} from the two
    uniforms of one Philox4x32-10 block with counter (pixel index low, high, 0, tag)."""
    w = np.asarray(w, dtype=np.float64)
    n = w.size
    i = np.arange(n, dtype=np.uint64)
    c = np.zeros((n, 4), dtype=np.uint64)
    c[:, 0] = i & MASK
    c[:, 1] = i >> np.uint64(32)
    c[:, 3] = NOISE_TAG
    a, b = uniform2(c, key_of(seed))
    wf = w.ravel()
    pos = wf > 0
    r = np.zeros(n)
    r[pos] = np.sqrt(-2.0 * np.log(1.0 - a[pos])) * np.sqrt(1.0 / (4.0 * df * wf[pos]))
    d = r * np.exp(2j * np.pi * b)
    return d.reshape(w.shape)

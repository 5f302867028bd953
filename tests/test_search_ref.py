"""The NumPy restatement of Philox4x32-10 used to check the swarm kernel's random draws,
pinned to the generator's published known-answer vectors (Salmon et al., SC 2011)."""
import numpy as np

from search_ref import philox4x32_10, uniform2

KAT = [((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
        (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
       ((0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff), (0xffffffff, 0xffffffff),
        (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
       ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
        (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1))]


def test_philox_known_answers():
    for c, k, want in KAT:
        got = philox4x32_10(np.array(c, dtype=np.uint64), np.array(k, dtype=np.uint64))
        assert [int(x) for x in got] == list(want)


def test_uniform_draws_are_uniform():
    n = 200_000
    c = np.zeros((n, 4), dtype=np.uint64)
    c[:, 0] = np.arange(n)
    a, b = uniform2(c, np.array([7, 11], dtype=np.uint64))
    for u in (a, b):
        assert u.min() >= 0.0 and u.max() < 1.0
        assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / n)
        hist = np.histogram(u, bins=20, range=(0, 1))[0]
        assert np.all(np.abs(hist - n / 20) < 5 * np.sqrt(n / 20))
    assert abs(np.corrcoef(a, b)[0, 1]) < 4 / np.sqrt(n)


def test_noise_restatement_has_the_data_convention():
    """E|d~|^2 = S / (2 df) with S = 1/w, real and imaginary parts independent and
    Gaussian; zero where the weight is zero."""
    from search_ref import noise
    rng = np.random.default_rng(5)
    w = rng.uniform(0.5, 2.0, (2, 50, 2000))
    w[:, 7, :] = 0.0
    df = 1e-4
    d = noise(w, df, seed=11)
    assert np.all(d[:, 7, :] == 0)
    m = w > 0
    z = d[m] * np.sqrt(2.0 * df * w[m])  # unit-variance complex normal
    n = z.size
    assert abs(np.mean(np.abs(z) ** 2) - 1.0) < 5 * np.sqrt(1.0 / n)
    for part in (z.real, z.imag):
        assert abs(part.mean()) < 5 * np.sqrt(0.5 / n)
        assert abs(np.mean(part ** 4) / np.mean(part ** 2) ** 2 - 3.0) < 0.05  # Gaussian
    assert abs(np.corrcoef(z.real, z.imag)[0, 1]) < 5 / np.sqrt(n)

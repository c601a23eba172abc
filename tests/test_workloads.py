"""Seeded input generators: the SplitMix64 stream against its published test values,
the vectorised draws against one-at-a-time draws, and the 2D sigma_0 fields."""
import numpy as np

from paper_1811_05579_gb300 import workloads as wl


def test_splitmix64_published_values():
    # the first outputs for seed 1234567 of the reference SplitMix64 (Vigna's splitmix64.c)
    g = wl.SplitMix64(1234567)
    assert [g.next_u64() for _ in range(3)] == [6457827717110365317, 3203168211198807973,
                                               9817491932198370423]


def test_vectorised_uniform_is_the_same_stream():
    a, b = wl.SplitMix64(99), wl.SplitMix64(99)
    x = a.uniform(777)
    y = np.array([(b.next_u64() >> 11) * (1.0 / (1 << 53)) for _ in range(777)])
    assert np.array_equal(x, y) and a.state == b.state
    assert a.uniform() == b.uniform()


def test_checkerboard_sigma_2d():
    s = wl.checkerboard_sigma_2d(16, blocks=8)
    assert s.shape == (16, 16)
    assert s[0, 0] == 1.0 and s[0, 2] == 100.0 and s[2, 0] == 100.0 and s[2, 2] == 1.0
    assert s[1, 1] == 1.0 and np.count_nonzero(s == 1.0) == 128


def test_lognormal_sigma_2d_moments_and_correlation():
    n = 96
    s = wl.lognormal_sigma_2d(n, seed=5, sd_cells=4.0)
    g = np.log(s)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1.0) < 1e-12
    # Gaussian smoothing of sd 4 cells: white noise filtered by it has the correlation
    # exp(-d^2 / (4 sd^2)) at lag d (both axes); sampled at d = 4 and 8 within a few
    # standard errors of a 96^2 field with ~ (96 / 8)^2 independent patches
    for d, want in ((4, np.exp(-0.25)), (8, np.exp(-1.0))):
        for ax in (0, 1):
            r = float(np.mean(g * np.roll(g, d, axis=ax)))
            assert abs(r - want) < 0.2, (d, ax, r, want)
    # periodic: the filter wraps, so the field has no edge effect (lag-1 correlation at
    # the seam equals the interior one within noise)
    seam = float(np.mean(g[:, 0] * g[:, -1]))
    inner = float(np.mean(g[:, 1:] * g[:, :-1]))
    assert abs(seam - inner) < 0.3

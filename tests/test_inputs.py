"""Seeded input generators: SplitMix64 against a scalar integer transcription of
the published algorithm, reproducibility, and the column recipe."""
import numpy as np

from paper_2301_12869_gb300 import inputs

MASK = (1 << 64) - 1


def splitmix64_scalar(seed, k):
    """k-th output (k >= 0) of SplitMix64 started from state = seed (Steele et al. 2014)."""
    state = (seed + (k + 1) * 0x9E3779B97F4A7C15) & MASK
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def test_splitmix64_matches_scalar_definition():
    for seed in [0, 1, 20230130, (1 << 63) + 12345]:
        k = np.arange(40, dtype=np.uint64)
        got = inputs.splitmix64(k, seed)
        want = [splitmix64_scalar(seed, int(i)) for i in k]
        assert [int(v) for v in got] == want


def test_uniform_field_reproducible_and_uniform():
    a = inputs.uniform_field(7, 64, 32)
    b = inputs.uniform_field(7, 64, 32)
    np.testing.assert_array_equal(a, b)
    assert a.min() >= 0.0 and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 0.02 and abs(a.var() - 1 / 12) < 0.01
    assert not np.array_equal(a, inputs.uniform_field(8, 64, 32))
    # a node's draw does not depend on the grid it sits in
    big = inputs.uniform_field(7, 64, 40)
    np.testing.assert_array_equal(big[:32], a)


def test_column_rho0_recipe():
    rho = inputs.column_rho0(8, 100, 0.3, 0.03, 50, width=5.0)
    assert rho.shape == (100, 8)
    assert np.all(rho == rho[:, :1])
    assert rho[0, 0] > 0.299 and rho[-1, 0] < 0.031
    # the interface midpoint sits at y0 = 49.5
    mid = 0.5 * (0.3 + 0.03)
    assert rho[49, 0] > mid > rho[50, 0]
    noisy = inputs.column_rho0(8, 100, 0.3, 0.03, 50, width=5.0, noise_amp=1e-3, seed=3)
    d = noisy - rho
    assert np.abs(d).max() <= 1e-3
    ys = np.arange(100)[:, None] * np.ones((1, 8))
    assert np.all(d[np.abs(ys - 49.5) > 10] == 0.0)
    assert np.abs(d[np.abs(ys - 49.5) <= 10]).min() > 0


def test_batched_columns_ranges():
    cols = inputs.batched_columns(4096)
    H = np.array([c["ny"] for c in cols])
    assert set(H) == {64, 128, 256, 512, 1024}
    Tr = np.array([c["Tr"] for c in cols])
    g = np.array([c["gy"] for c in cols])
    assert Tr.min() >= 0.70 and Tr.max() <= 0.95
    assert np.all(g < 0) and -g.max() >= 1e-6 and -g.min() <= 1e-4
    assert 0.45 < np.mean([c["form"] == 1 for c in cols]) < 0.55

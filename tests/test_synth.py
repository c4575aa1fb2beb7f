"""The seeded generators: deterministic, the documented shapes, ranges and class mix."""
import numpy as np

import synth


def test_splitmix64_published_values():
    # first outputs of splitmix64 seeded with 0 (the generator's reference sequence)
    out = synth.splitmix64(0, np.arange(3, dtype=np.uint64))
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_cube_exact_and_deterministic():
    a = synth.uniform_cube(1000, 7)
    b = synth.uniform_cube(1000, 7)
    assert a.dtype == np.float32 and a.shape == (1000, 3)
    assert np.array_equal(a, b) and not np.array_equal(a, synth.uniform_cube(1000, 8))
    assert a.min() >= 0 and a.max() < 1
    assert np.all(a * np.float32(2 ** 24) == np.floor(a * np.float32(2 ** 24)))   # multiples of 2^-24


def test_lidar_tile_shape():
    n = 200_000
    xyz = synth.lidar_tile(n, synth.CONFIG_SEED[2])
    side = np.sqrt(n / 10.0)
    assert xyz.shape == (n, 3) and xyz.dtype == np.float32
    ground = xyz[: int(0.6 * n)]
    assert ground[:, :2].min() > -0.5 and ground[:, :2].max() < side + 0.5
    assert 0 - 0.5 < ground[:, 2].min() and ground[:, 2].max() < 40.5
    veg = xyz[int(0.6 * n): int(0.9 * n)]
    assert veg[:, 2].max() < 40 + 25 + 1.0
    assert np.array_equal(xyz, synth.lidar_tile(n, synth.CONFIG_SEED[2]))


def test_gaussian_clusters_shape():
    xyz = synth.gaussian_clusters(50_000, 3)
    assert xyz.shape == (50_000, 3) and np.isfinite(xyz).all()

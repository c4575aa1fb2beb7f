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


def test_batch_workload_matches_its_recipe():
    """The 256-cloud batch: log-uniform sizes on [10k, 2M] (95.4M points in all), the three
    generators in turn, about half radius (r from the set) and half kNN (k from the set)."""
    specs = synth.batch_workload()
    assert len(specs) == 256
    sizes = np.array([s["n"] for s in specs])
    assert sizes.min() >= 10_000 and sizes.max() <= 2_000_000
    assert sizes.sum() == 95_396_245
    # log-uniform: the median of log(n) sits near the middle of [log 10k, log 2M]
    mid = 0.5 * (np.log(10_000) + np.log(2_000_000))
    assert abs(np.median(np.log(sizes)) - mid) < 0.5
    assert [s["gen"] for s in specs[:6]] == list(synth.BATCH_GENERATORS) * 2
    radius = [s for s in specs if s["search"] == "radius"]
    knn = [s for s in specs if s["search"] == "knn"]
    assert len(radius) + len(knn) == 256 and 100 < len(radius) < 156
    assert {s["r"] for s in radius} <= set(synth.BATCH_RADII) and {s["k"] for s in knn} <= set(synth.BATCH_KS)
    assert synth.batch_workload() == specs  # seeded


def test_batch_cloud_scales():
    """Uniform cubes at 2 pts/m^3, LiDAR tiles at 10 pts/m^2."""
    spec = dict(gen="uniform", n=20_000, seed=5)
    xyz = synth.batch_cloud(spec)
    side = (20_000 / 2.0) ** (1.0 / 3.0)
    assert xyz.shape == (20_000, 3) and xyz.min() >= 0.0 and xyz.max() < side
    tile = synth.batch_cloud(dict(gen="lidar", n=20_000, seed=6))
    side = np.sqrt(20_000 / 10.0)  # the ground covers the tile; crowns and roofs may overhang it
    on_tile = np.all((tile[:, :2] >= -0.2) & (tile[:, :2] < side + 0.2), axis=1)
    assert on_tile.mean() > 0.85
    assert synth.batch_cloud(dict(gen="clusters", n=0, seed=1)).shape == (0, 3)

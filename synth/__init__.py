"""Seeded synthetic point clouds shared by the tests, the oracle runs and the benchmark.

This module only draws inputs. It holds none of the neighbour-search method's
arithmetic (no discretisation, no space-filling curve, no distance test), so the
CPU oracle and the CUDA path can both consume its buffers without sharing code.

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: output n of stream s under seed S is mix(S + (c + 1) * 0x9E3779B97F4A7C15)
with counter c = s * 2**40 + n.  Every array below is a pure function of
(seed, shape parameters); it does not depend on the machine.

Workloads (the paper measures on public LiDAR scans that are not available here;
these generators stand in for them):

* ``uniform_cube``   - i.i.d. uniform float32 in [0, side)^3.  With side 1 the
  coordinates are (u >> 40) * 2**-24, exact float32 values in [0, 1).
* ``lidar_tile``     - an aerial-LiDAR-like tile: 60 % ground on a 6-octave
  value-noise heightfield (0-40 m), 30 % tree crowns (ellipsoids), 10 % box
  buildings with flat or gable roofs, 3 cm Gaussian jitter, 10 points/m^2.
* ``gaussian_clusters`` - 64 isotropic Gaussian blobs in a cube.
* ``batch_workload`` / ``batch_cloud`` - many clouds of uneven sizes (log-uniform),
  the generator cycling uniform / LiDAR tile / Gaussian clusters, each with a
  radius or kNN search drawn for it.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "splitmix64",
    "Rng",
    "uniform_cube",
    "lidar_tile",
    "gaussian_clusters",
    "CONFIG_SEED",
    "config_cloud",
    "batch_workload",
    "batch_cloud",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

#: Seed of workload ``k``: 1 uniform cube, 2 LiDAR tile (10M), 3 LiDAR tiles for kNN (10M,
#: 50M), 4 batch of clouds, 5 serving requests.
CONFIG_SEED = {k: 0x5EED0000 + k for k in range(1, 6)}


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """Return splitmix64 outputs number ``counters + 1`` of the sequence started at ``seed``."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Rng:
    """Counter-based generator: ``stream`` selects an independent counter range."""

    def __init__(self, seed: int):
        self.seed = int(seed)

    def u64(self, stream: int, n: int, offset: int = 0) -> np.ndarray:
        base = np.uint64((int(stream) << 40) + int(offset))
        return splitmix64(self.seed, base + np.arange(n, dtype=np.uint64))

    def u01_f32(self, stream: int, n: int) -> np.ndarray:
        """Uniform float32 in [0, 1): the top 24 bits times 2**-24 (exact)."""
        return (self.u64(stream, n) >> np.uint64(40)).astype(np.float32) * np.float32(2.0 ** -24)

    def u01(self, stream: int, n: int) -> np.ndarray:
        """Uniform float64 in [0, 1): the top 53 bits times 2**-53."""
        return (self.u64(stream, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def uniform(self, stream: int, n: int, lo: float, hi: float) -> np.ndarray:
        return lo + (hi - lo) * self.u01(stream, n)

    def normal(self, stream: int, n: int) -> np.ndarray:
        """Standard normal by the Box-Muller transform of two uniform streams."""
        u1 = self.u01(2 * stream + 0x100000, n)
        u2 = self.u01(2 * stream + 0x100001, n)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)

    def integers(self, stream: int, n: int, high: int) -> np.ndarray:
        """Integers in [0, high) (multiply-shift on the top 32 bits)."""
        top = self.u64(stream, n) >> np.uint64(32)
        return ((top * np.uint64(high)) >> np.uint64(32)).astype(np.int64)


def uniform_cube(n: int, seed: int, side: float = 1.0) -> np.ndarray:
    """``n`` points i.i.d. uniform in [0, side)^3 as float32, shape (n, 3)."""
    rng = Rng(seed)
    xyz = rng.u01_f32(0, 3 * n).reshape(n, 3)
    if side != 1.0:
        xyz = (xyz.astype(np.float64) * side).astype(np.float32)
    return np.ascontiguousarray(xyz)


def _fade(t: np.ndarray) -> np.ndarray:
    # quintic smoothstep 6t^5 - 15t^4 + 10t^3
    return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)


def _value_noise(x: np.ndarray, y: np.ndarray, seed: int, wavelength: float,
                 octaves: int = 6, lacunarity: float = 2.0, gain: float = 0.5) -> np.ndarray:
    """Fractal value noise in [0, 1): lattice values from splitmix64, quintic fade."""
    total = np.zeros_like(x)
    amp, freq, norm = 1.0, 1.0 / wavelength, 0.0
    for o in range(octaves):
        fx, fy = x * freq, y * freq
        ix, iy = np.floor(fx), np.floor(fy)
        sx, sy = _fade(fx - ix), _fade(fy - iy)
        ix = ix.astype(np.int64) + (1 << 20)
        iy = iy.astype(np.int64) + (1 << 20)

        def lat(dx: int, dy: int) -> np.ndarray:
            c = ((ix + dx) << 21) + (iy + dy)
            return (splitmix64(seed + 7919 * (o + 1), c.astype(np.uint64)) >> np.uint64(11)).astype(
                np.float64) * (2.0 ** -53)

        v0 = lat(0, 0) + (lat(1, 0) - lat(0, 0)) * sx
        v1 = lat(0, 1) + (lat(1, 1) - lat(0, 1)) * sx
        total += amp * (v0 + (v1 - v0) * sy)
        norm += amp
        amp *= gain
        freq *= lacunarity
    return total / norm


def lidar_tile(n: int, seed: int, side: float | None = None, relief: float = 40.0,
               wavelength: float = 500.0, jitter: float = 0.03) -> np.ndarray:
    """Aerial-LiDAR-like tile of ``n`` float32 points, shape (n, 3), local coordinates.

    ``side`` defaults to sqrt(n / 10) m (10 points per square metre).  Classes:
    ground 60 % (uniform x, y; z = relief * value noise), vegetation 30 % (crowns of
    trees placed uniformly, one tree per 400 m^2: horizontal radius U(2, 8) m, vertical
    semi-axis U(0.6, 1.2) x radius, crown top U(2c + 1, 25) m above the ground, 70 % of
    a tree's points on the upper crown surface and 30 % inside the crown), buildings
    10 % (one per 2500 m^2: footprint U(10, 40) m x U(10, 40) m, height U(3, 20) m,
    half flat and half gable roofs with a U(1, 4) m ridge, 80 % of the points on the
    roof and 20 % on the walls).  Every coordinate then gets N(0, jitter^2) noise.
    Points are stored class by class in generation order (no scan-order locality).
    """
    if side is None:
        side = math.sqrt(n / 10.0)
    rng = Rng(seed)
    area = side * side
    n_ground = int(round(0.6 * n))
    n_veg = int(round(0.3 * n))
    n_bld = n - n_ground - n_veg

    def ground(x, y):
        return relief * _value_noise(x, y, seed ^ 0x6E01, wavelength)

    # ground
    gx = rng.uniform(1, n_ground, 0.0, side)
    gy = rng.uniform(2, n_ground, 0.0, side)
    gz = ground(gx, gy)

    # vegetation
    n_trees = max(1, int(round(area / 400.0)))
    tx = rng.uniform(10, n_trees, 0.0, side)
    ty = rng.uniform(11, n_trees, 0.0, side)
    tr = rng.uniform(12, n_trees, 2.0, 8.0)
    tc = tr * rng.uniform(13, n_trees, 0.6, 1.2)
    ttop = (2.0 * tc + 1.0) + (25.0 - (2.0 * tc + 1.0)) * rng.u01(14, n_trees)
    tzc = ground(tx, ty) + ttop - tc
    which = rng.integers(15, n_veg, n_trees)
    surface = rng.u01(16, n_veg) < 0.7
    phi = 2.0 * np.pi * rng.u01(17, n_veg)
    cos_t = np.where(surface, rng.u01(18, n_veg), 2.0 * rng.u01(18, n_veg) - 1.0)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    rad = np.where(surface, 1.0, np.cbrt(rng.u01(19, n_veg)))
    vx = tx[which] + tr[which] * rad * sin_t * np.cos(phi)
    vy = ty[which] + tr[which] * rad * sin_t * np.sin(phi)
    vz = tzc[which] + tc[which] * rad * cos_t

    # buildings
    n_b = max(1, int(round(area / 2500.0)))
    bx = rng.uniform(20, n_b, 0.0, side)
    by = rng.uniform(21, n_b, 0.0, side)
    bw = rng.uniform(22, n_b, 10.0, 40.0)
    bd = rng.uniform(23, n_b, 10.0, 40.0)
    bh = rng.uniform(24, n_b, 3.0, 20.0)
    gable = rng.u01(25, n_b) < 0.5
    ridge = rng.uniform(26, n_b, 1.0, 4.0)
    bz0 = ground(bx, by)
    which = rng.integers(27, n_bld, n_b)
    on_roof = rng.u01(28, n_bld) < 0.8
    u = rng.u01(29, n_bld)
    v = rng.u01(30, n_bld)
    w, d, h = bw[which], bd[which], bh[which]
    along_x = w >= d
    across = np.where(along_x, v, u)           # coordinate across the ridge, in [0, 1)
    roof_z = bz0[which] + h + np.where(gable[which], ridge[which] * (1.0 - np.abs(2.0 * across - 1.0)), 0.0)
    rx = bx[which] + (u - 0.5) * w
    ry = by[which] + (v - 0.5) * d
    # walls: a position along the perimeter, uniform height
    per = 2.0 * (w + d)
    t = u * per
    wx = np.where(t < w, t, np.where(t < w + d, w, np.where(t < 2 * w + d, 2 * w + d - t, 0.0)))
    wy = np.where(t < w, 0.0, np.where(t < w + d, t - w, np.where(t < 2 * w + d, d, per - t)))
    wx = bx[which] - 0.5 * w + wx
    wy = by[which] - 0.5 * d + wy
    wz = bz0[which] + v * h
    bxp = np.where(on_roof, rx, wx)
    byp = np.where(on_roof, ry, wy)
    bzp = np.where(on_roof, roof_z, wz)

    xyz = np.empty((n, 3), dtype=np.float64)
    xyz[:n_ground, 0], xyz[:n_ground, 1], xyz[:n_ground, 2] = gx, gy, gz
    s = n_ground
    xyz[s:s + n_veg, 0], xyz[s:s + n_veg, 1], xyz[s:s + n_veg, 2] = vx, vy, vz
    s += n_veg
    xyz[s:, 0], xyz[s:, 1], xyz[s:, 2] = bxp, byp, bzp
    if jitter > 0:
        for a in range(3):
            xyz[:, a] += jitter * rng.normal(40 + a, n)
    return np.ascontiguousarray(xyz.astype(np.float32))


def gaussian_clusters(n: int, seed: int, n_centres: int = 64, side: float | None = None,
                      sigma_lo: float = 1.0, sigma_hi: float = 5.0) -> np.ndarray:
    """``n`` float32 points around ``n_centres`` isotropic Gaussian centres.

    Centres are uniform in [0, side)^3 with side = cbrt(n / 2) m by default; each
    centre draws sigma ~ U(sigma_lo, sigma_hi) and each point picks a centre uniformly.
    """
    if side is None:
        side = (n / 2.0) ** (1.0 / 3.0)
    rng = Rng(seed)
    c = rng.uniform(0, 3 * n_centres, 0.0, side).reshape(n_centres, 3)
    sig = rng.uniform(1, n_centres, sigma_lo, sigma_hi)
    which = rng.integers(2, n, n_centres)
    xyz = c[which] + sig[which, None] * np.stack([rng.normal(3 + a, n) for a in range(3)], axis=1)
    return np.ascontiguousarray(xyz.astype(np.float32))


def config_cloud(config: int, n: int | None = None) -> np.ndarray:
    """The point cloud of workload ``config`` (1: uniform cube 131072; 2/3: LiDAR tile)."""
    seed = CONFIG_SEED[config]
    if config == 1:
        return uniform_cube(131072 if n is None else n, seed)
    if config in (2, 3):
        return lidar_tile(10_000_000 if n is None else n, seed)
    raise ValueError(f"no single cloud for workload {config}")


BATCH_RADII = (0.5, 1.0, 2.0, 3.0)
BATCH_KS = (8, 16, 32)
BATCH_GENERATORS = ("uniform", "lidar", "clusters")


def batch_workload(n_clouds: int = 256, seed: int = CONFIG_SEED[4], n_lo: int = 10_000,
                   n_hi: int = 2_000_000) -> list[dict]:
    """Specs of a batch of clouds: size log-uniform on [n_lo, n_hi], generator cycling
    uniform (cube side cbrt(n / 2) m) / LiDAR tile (side sqrt(n / 10) m) / Gaussian
    clusters (64 centres in the cube of side cbrt(n / 2) m, sigma U(1, 5) m); half the
    clouds get an all-points sphere search with r from {0.5, 1, 2, 3} m, the other half
    all-points kNN with k from {8, 16, 32}."""
    rng = Rng(seed)
    u = rng.u01(0, n_clouds)
    sizes = np.exp(np.log(n_lo) + u * (np.log(n_hi) - np.log(n_lo)))
    radius = rng.u01(1, n_clouds) < 0.5
    ri = rng.integers(2, n_clouds, len(BATCH_RADII))
    ki = rng.integers(3, n_clouds, len(BATCH_KS))
    specs = []
    for i in range(n_clouds):
        spec = dict(gen=BATCH_GENERATORS[i % 3], n=int(round(sizes[i])), seed=seed * 1000 + i)
        if radius[i]:
            spec.update(search="radius", kernel="sphere", r=BATCH_RADII[int(ri[i])])
        else:
            spec.update(search="knn", k=BATCH_KS[int(ki[i])])
        specs.append(spec)
    return specs


def batch_cloud(spec: dict) -> np.ndarray:
    """The points of one ``batch_workload`` entry."""
    n, seed = spec["n"], spec["seed"]
    if n == 0:
        return np.zeros((0, 3), np.float32)
    if spec["gen"] == "uniform":
        return uniform_cube(n, seed, side=(n / 2.0) ** (1.0 / 3.0))
    if spec["gen"] == "lidar":
        return lidar_tile(n, seed, side=math.sqrt(n / 10.0))
    return gaussian_clusters(n, seed)

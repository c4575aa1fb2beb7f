"""Shared helpers of the parity tests: run the CUDA path and the oracle on one input."""
from __future__ import annotations

import functools

import numpy as np

import oracle
import synth

ENC = {"none": oracle.ENC_NONE, "morton": oracle.ENC_MORTON, "hilbert": oracle.ENC_HILBERT}
KERN = {"sphere": oracle.SPHERE, "circle": oracle.CIRCLE, "cube": oracle.CUBE, "square": oracle.SQUARE}


def cloud(name: str) -> np.ndarray:
    """Named test clouds: the seeded workloads plus edge cases."""
    if name == "uniform131k":
        return synth.config_cloud(1)
    if name.startswith("uniform"):
        return synth.uniform_cube(int(name[7:]), 101)
    if name == "lidar60k":
        return synth.lidar_tile(60_000, synth.CONFIG_SEED[2], side=float(np.sqrt(60_000 / 10.0)))
    if name == "clusters40k":
        return synth.gaussian_clusters(40_000, synth.CONFIG_SEED[4])
    if name == "duplicates":       # every point 5 times, plus a 300-fold pile
        base = synth.uniform_cube(2000, 103)
        pile = np.repeat(base[:1], 300, axis=0)
        return np.ascontiguousarray(np.concatenate([np.repeat(base, 5, axis=0), pile]))
    if name == "identical":
        return np.full((100, 3), 0.25, np.float32)
    if name == "lattice":
        g = np.arange(12, dtype=np.float32)
        return np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).copy()
    if name == "plane":
        xyz = synth.uniform_cube(20_000, 104, side=50.0)
        xyz[:, 2] = 3.0
        return xyz
    if name == "empty":
        return np.zeros((0, 3), np.float32)
    raise KeyError(name)


@functools.lru_cache(maxsize=16)
def _pipeline(name: str, enc: int, ncap: int) -> oracle.Pipeline:
    return oracle.Pipeline(cloud(name), enc, ncap)


def oracle_pipeline(name: str, enc: str, ncap: int) -> oracle.Pipeline:
    return _pipeline(name, ENC[enc], ncap)


@functools.lru_cache(maxsize=64)
def oracle_radius(name: str, ncap: int, r: float, kern: str):
    """All-points CSR of the oracle (rows by original index), independent of the encoding."""
    p = _pipeline(name, oracle.ENC_MORTON, ncap)
    return p.tree.radius(p.xyz, r, KERN[kern])


def gpu_csr(row_ptr, cols):
    return row_ptr.cpu().numpy(), cols.cpu().numpy()


def csr_rows_sorted_by_id(row_ptr: np.ndarray, cols: np.ndarray) -> np.ndarray:
    rows = np.repeat(np.arange(len(row_ptr) - 1), np.diff(row_ptr))
    return cols[np.lexsort((cols, rows))]


def nodes_canonical(keys, levels, cols: dict) -> tuple[np.ndarray, dict]:
    order = np.lexsort((levels, keys))
    return order, {k: np.asarray(v)[order] for k, v in cols.items()}

"""The kNN workload's larger tile: 50M LiDAR-like points (2236 m x 2236 m at 10 pts/m^2),
Hilbert order, all-points kNN with k in {8, 16, 50}, in the launch configuration of the
benchmark.  Sampled rows are compared with the oracle's brute-force kNN over all 50M
points (bit-exact); every row is checked for order and for self-inclusion."""
import numpy as np
import pytest
import torch

import oracle
import paper_2603_06771_gb300 as sfc
import synth

pytestmark = pytest.mark.gpu

N = 50_000_000
N_SAMPLE = 200


@pytest.fixture(scope="module")
def tile():
    sfc.build()
    assert torch.cuda.is_available(), "these tests need a CUDA device"
    xyz = synth.lidar_tile(N, synth.CONFIG_SEED[3])
    rows = np.sort(synth.Rng(3).integers(0, N_SAMPLE, N)).astype(np.int64)
    pts = torch.from_numpy(xyz).cuda()
    tree = sfc.octree_build(pts, "hilbert", leaf_capacity=96)
    yield {"xyz": xyz, "rows": rows, "tree": tree}
    tree.free()


@pytest.mark.parametrize("k", [8, 16, 50])
def test_knn_50m_sampled_rows(tile, k):
    idx, d2 = sfc.knn(tile["tree"], None, k)
    rows = tile["rows"]
    oi, od = oracle.knn_brute(tile["xyz"], tile["xyz"][rows], k)
    r = torch.as_tensor(rows, device="cuda")
    assert np.array_equal(idx[r].cpu().numpy(), oi)
    assert np.array_equal(d2[r].cpu().numpy().view(np.uint32), od.view(np.uint32))
    # every row: ascending in (d2, index), its first distance is 0 (the centre or a duplicate)
    ok = torch.ones(1, dtype=torch.bool, device="cuda")
    for lo in range(0, N, 10_000_000):  # in slices, to bound host memory
        dd, ii = d2[lo:lo + 10_000_000], idx[lo:lo + 10_000_000]
        asc = (dd[:, 1:] > dd[:, :-1]) | ((dd[:, 1:] == dd[:, :-1]) & (ii[:, 1:] > ii[:, :-1]))
        ok &= asc.all() & (dd[:, 0] == 0).all() & (ii >= 0).all()
    assert bool(ok.item())

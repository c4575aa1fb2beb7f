"""The batched workload at full size: 256 clouds of 10k-2M points (95.4M in all; uniform,
LiDAR-like and Gaussian clusters), half all-points sphere searches (radius redrawn smaller
when a cloud would exceed 2^28 neighbours), half all-points kNN.  Every cloud's sampled
rows are compared with the oracle's brute force over that cloud; the recorded plan gives
the same bytes as the eager batch for every cloud."""
import os
import sys

import numpy as np
import pytest
import torch

import oracle
import paper_2603_06771_gb300 as sfc
import synth

pytestmark = pytest.mark.gpu
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402  (the workload's setup, shared with the benchmark)

ROWS_PER_CLOUD = 12


@pytest.fixture(scope="module")
def batch():
    sfc.build()
    assert torch.cuda.is_available(), "these tests need a CUDA device"
    specs, pts, _, _ = bench.batch_setup(sfc, torch, 256, 64, "hilbert")
    xyz = bench.batch_setup.xyz
    clouds = [dict(n=sp["n"], search=sp["search"], kernel=sp.get("kernel", "sphere"), r=sp.get("r", 0.0),
                   k=sp.get("k", 0)) for sp in specs]
    b = sfc.batch_search(pts, clouds, "hilbert", leaf_capacity=64)
    yield clouds, xyz, pts, b
    b.free()


def test_batch256_every_cloud_sampled_rows(batch):
    clouds, xyz, _, b = batch
    for i, (c, x) in enumerate(zip(clouds, xyz)):
        rows = np.sort(synth.Rng(1000 + i).integers(0, min(ROWS_PER_CLOUD, c["n"]), c["n"])).astype(np.int64)
        q = x[rows]
        if c["search"] == "radius":
            rp, cols = b.radius(i)
            orp, ocols = oracle.radius_brute(x, q, c["r"], oracle.KERNELS[c["kernel"]])
            rp_h = rp.cpu().numpy()
            for j, row in enumerate(rows):
                got = np.sort(cols[rp_h[row]:rp_h[row + 1]].cpu().numpy())
                assert np.array_equal(got, np.sort(ocols[orp[j]:orp[j + 1]])), (i, int(row))
        else:
            idx, d2 = b.knn(i)
            oi, od = oracle.knn_brute(x, q, c["k"])
            r = torch.as_tensor(rows, device="cuda")
            assert np.array_equal(idx[r].cpu().numpy(), oi), i
            assert np.array_equal(d2[r].cpu().numpy().view(np.uint32), od.view(np.uint32)), i


def test_batch256_plan_equals_eager_batch(batch):
    clouds, _, pts, b = batch
    nnz = sum(int(b.radius(i)[1].shape[0]) for i, c in enumerate(clouds) if c["search"] == "radius")
    plan = sfc.BatchPlan(clouds, "hilbert", leaf_capacity=64, nnz_capacity=nnz)
    plan.points.copy_(pts)
    plan.run()
    for i, c in enumerate(clouds):
        if c["search"] == "radius":
            a_rp, a_cols = b.radius(i)
            p_rp, p_cols = plan.radius(i)
            assert torch.equal(a_rp, p_rp) and torch.equal(a_cols, p_cols), i
        else:
            a_i, a_d = b.knn(i)
            p_i, p_d = plan.knn(i)
            assert torch.equal(a_i, p_i) and torch.equal(a_d.view(torch.int32), p_d.view(torch.int32)), i
    plan.free()

"""Work counters of the search walks (``sfc_stats_enable``): the instrumented kernels give
the same results as the plain ones, and the counters obey what the walks must satisfy —
every neighbour is either a point test that passed or a point of a node taken whole, so
hits + whole equals the count the oracle's brute force gives; a walk without the
shortcuts takes nothing whole; a kNN list is built from insertions of marked candidates."""
import numpy as np
import pytest
import torch

import oracle
import paper_2603_06771_gb300 as sfc
import synth
from helpers import KERN

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _library():
    sfc.build()
    assert torch.cuda.is_available(), "these tests need a CUDA device"


N = 20_000


@pytest.fixture(scope="module")
def cloud():
    return synth.lidar_tile(N, 4242, side=float(np.sqrt(N / 10.0)))


def _radius(t, q, r, kern):
    rp, cols = sfc.radius_search(t, q, r, kern)
    return rp.cpu().numpy(), cols.cpu().numpy()


@pytest.mark.parametrize("enc", ["hilbert", "morton", "none"])
@pytest.mark.parametrize("kern", ["sphere", "cube", "circle", "square"])
def test_radius_counters(cloud, enc, kern):
    pts = torch.from_numpy(cloud).cuda()
    t = sfc.octree_build(pts, enc, leaf_capacity=32)
    r = 1.5
    plain = _radius(t, None, r, kern)
    with sfc.search_stats() as st:
        counted = _radius(t, None, r, kern)
    assert np.array_equal(plain[0], counted[0]) and np.array_equal(plain[1], counted[1])
    nnz = int(plain[0][-1])
    orp, _ = oracle.radius_brute(cloud, cloud, r, KERN[kern])
    assert nnz == int(orp[-1])
    assert st["passed"] + st["whole"] == nnz
    assert st["walks"] == (N if enc == "none" else (N + 31) // 32)
    assert 0 < st["needed_tests"] <= st["point_tests"]
    assert st["passed"] <= st["point_tests"]
    assert st["leaves"] > 0 and st["expansions"] > 0 and st["box_tests"] >= st["expansions"]
    assert st["inserts"] == 0
    t.free()


@pytest.mark.parametrize("enc", ["hilbert", "none"])
def test_radius_counters_without_shortcuts(cloud, enc):
    pts = torch.from_numpy(cloud).cuda()
    t = sfc.octree_build(pts, enc, leaf_capacity=32, prune=False)
    with sfc.search_stats() as st:
        rp, _ = _radius(t, None, 2.0, "sphere")
    assert st["whole"] == 0 and st["passed"] == int(rp[-1])
    t.free()


def test_radius_counters_caller_centres(cloud):
    pts = torch.from_numpy(cloud).cuda()
    t = sfc.octree_build(pts, "hilbert", leaf_capacity=32)
    q = torch.from_numpy(np.ascontiguousarray(cloud[::7] + 0.25)).cuda()
    plain = _radius(t, q, 1.0, "sphere")
    with sfc.search_stats() as st:
        counted = _radius(t, q, 1.0, "sphere")
    assert np.array_equal(plain[1], counted[1])
    assert st["walks"] == (q.shape[0] + 31) // 32
    assert st["passed"] + st["whole"] == int(plain[0][-1])
    t.free()


@pytest.mark.parametrize("enc", ["hilbert", "none"])
@pytest.mark.parametrize("k", [8, 16, 32])
def test_knn_counters(cloud, enc, k):
    pts = torch.from_numpy(cloud).cuda()
    t = sfc.octree_build(pts, enc, leaf_capacity=32)
    idx, d2 = sfc.knn(t, None, k)
    with sfc.search_stats() as st:
        idx2, d22 = sfc.knn(t, None, k)
    assert torch.equal(idx, idx2) and torch.equal(d2.view(torch.int32), d22.view(torch.int32))
    assert st["walks"] == (N if enc == "none" else (N + 31) // 32)
    assert 0 < st["needed_tests"] <= st["point_tests"]
    assert st["inserts"] <= st["passed"] <= st["point_tests"]
    assert st["whole"] == 0
    if enc == "none":  # each list starts empty: every one of its k entries was inserted
        assert st["inserts"] >= N * k
    else:  # the seeding window: 2k curve neighbours tested per centre before the walk
        assert st["point_tests"] >= ((N + 31) // 32) * 32 * 2 * max(8, k)
    t.free()


def test_counting_stops_and_restarts(cloud):
    pts = torch.from_numpy(cloud).cuda()
    t = sfc.octree_build(pts, "hilbert", leaf_capacity=32)
    with sfc.search_stats() as first:
        sfc.knn(t, None, 8)
    sfc.knn(t, None, 8)  # not counted
    assert sfc.stats_read() == first
    with sfc.search_stats() as second:
        sfc.knn(t, None, 8)
        sfc.knn(t, None, 8)
    assert second["walks"] == 2 * first["walks"] and second["point_tests"] == 2 * first["point_tests"]
    t.free()

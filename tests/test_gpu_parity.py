"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer results (codes, permutation, leaves, node ranges, CSR rows, kNN indices) must
be identical; floating-point results (node boxes, kNN squared distances) are compared
bit for bit, because both sides evaluate the same binary32 expression with every
operation rounded to nearest and no contraction.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2603_06771_gb300 as sfc
import synth
from helpers import (ENC, KERN, cloud, csr_rows_sorted_by_id, gpu_csr, nodes_canonical, oracle_pipeline,
                     oracle_radius)

pytestmark = pytest.mark.gpu

ENCS = ["none", "morton", "hilbert"]
KERNS = ["sphere", "circle", "cube", "square"]
# radii giving about 35 neighbours per centre in the 131072-point unit cube
R131K = {"sphere": 0.04, "circle": 0.0092, "cube": 0.032, "square": 0.0082}


@pytest.fixture(scope="module", autouse=True)
def _library():
    sfc.build()
    assert torch.cuda.is_available(), "these tests need a CUDA device"


def dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def u64(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


# ----------------------------------------------------------------------------- codes
@pytest.mark.parametrize("enc", ["morton", "hilbert"])
def test_encode_cells_parity(enc):
    rng = synth.Rng(5)
    rand = (rng.u64(0, 3 * 300_000) >> np.uint64(43)).astype(np.uint32).reshape(-1, 3)
    g = np.arange(16, dtype=np.uint32)
    small = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    top = small + np.uint32((1 << 21) - 16)
    mixed = small + np.array([0, 1 << 20, (1 << 21) - 16], np.uint32)
    cells = np.concatenate([rand, small, top, mixed]).astype(np.uint32)
    want = oracle.encode_cells(cells, ENC[enc])
    got = sfc.encode_cells(dev(cells.astype(np.int32)), enc)
    assert np.array_equal(u64(got), want)


# ----------------------------------------------------------------------------- build
BUILD_CASES = [("uniform131k", 32), ("lidar60k", 32), ("clusters40k", 16), ("duplicates", 8), ("identical", 8),
               ("lattice", 4), ("plane", 64), ("uniform1", 32), ("uniform5", 2), ("uniform33", 32),
               ("uniform4097", 1), ("empty", 32)]


@pytest.mark.parametrize("enc", ENCS)
@pytest.mark.parametrize("name,ncap", BUILD_CASES)
def test_build_parity(name, ncap, enc):
    xyz = cloud(name)
    p = oracle_pipeline(name, enc, ncap)
    t = sfc.octree_build(dev(xyz), enc, leaf_capacity=ncap)
    ex = t.export()
    if len(xyz):
        assert t.lo == tuple(float(v) for v in p.lo) and t.scale == p.scale
    assert np.array_equal(u64(ex["keys"]), p.sorted_keys)
    assert np.array_equal(ex["perm"].cpu().numpy().astype(np.uint32), p.perm)
    assert np.array_equal(u64(ex["leaves"]), p.leaves)
    assert np.array_equal(ex["counts"].cpu().numpy().astype(np.uint32), p.counts)
    assert t.n_nodes == p.tree.num_nodes and t.n_leaves == len(p.counts)

    nd = {k: v.cpu().numpy() for k, v in t.export_nodes().items()}
    gkey = nd["key"].view(np.uint64)
    _, g = nodes_canonical(gkey, nd["level"], {
        "key": gkey, "level": nd["level"].astype(np.int32), "start": nd["start"].astype(np.int64),
        "end": nd["end"].astype(np.int64), "leaf": nd["child"] < 0, "box": nd["box"]})
    on = p.nodes()
    _, o = nodes_canonical(on["key"], on["level"], {
        "key": on["key"], "level": on["level"], "start": on["start"], "end": on["end"],
        "leaf": on["is_leaf"] == 1, "box": on["box"]})
    for k in g:
        assert np.array_equal(g[k], o[k]), k
    # links: the eight children of an internal node are consecutive, one level down, in code order
    child, lvl = nd["child"], nd["level"].astype(np.int64)
    inner = np.nonzero(child >= 0)[0]
    for j in range(8):
        c = child[inner] + j
        assert np.array_equal(lvl[c], lvl[inner] + 1)
        step = np.left_shift(np.uint64(1), (3 * (20 - lvl[inner])).astype(np.uint64))
        assert np.array_equal(gkey[c], gkey[inner] + np.uint64(j) * step)
    t.free()


# ----------------------------------------------------------------------------- fixed radius
@pytest.mark.parametrize("prune", [True, False])
@pytest.mark.parametrize("enc", ENCS)
@pytest.mark.parametrize("kern", KERNS)
def test_radius_all_points_uniform(kern, enc, prune):
    name, ncap, r = "uniform131k", 32, R131K[kern]
    p = oracle_pipeline(name, enc, ncap)
    orp, ocol = oracle_radius(name, ncap, r, kern)
    t = sfc.octree_build(dev(p.xyz), enc, leaf_capacity=ncap, prune=prune)
    rp, cols = gpu_csr(*sfc.radius_search(t, None, r, kern))
    assert np.array_equal(rp, orp)
    assert np.array_equal(cols, p.rows_by_rank(orp, ocol))


@pytest.mark.parametrize("enc", ["morton", "hilbert"])
@pytest.mark.parametrize("kern", KERNS)
def test_radius_row_counts_more_radii(kern, enc):
    """Row counts against the oracle at three more radii per kernel on the uniform cloud:
    more pairs at the boundary of the binary32 test (a faster evaluation once decided one
    pair of 30.6M differently at circle r = 0.024 and was dropped)."""
    name, ncap = "uniform131k", 32
    p = oracle_pipeline(name, enc, ncap)
    t = sfc.octree_build(dev(p.xyz), enc, leaf_capacity=ncap)
    for r in (0.017, 0.024, 0.031):
        orp, _ = p.tree.radius(p.xyz, r, KERN[kern])  # not cached: only the row pointers are kept
        rp, _ = sfc.radius_count(t, None, r, kern)
        assert np.array_equal(rp.cpu().numpy(), orp), (kern, enc, r)
    t.free()


@pytest.mark.parametrize("enc", ENCS)
@pytest.mark.parametrize("kern", KERNS)
@pytest.mark.parametrize("r", [0.5, 2.0])
def test_radius_all_points_lidar(kern, enc, r):
    name, ncap = "lidar60k", 32
    p = oracle_pipeline(name, enc, ncap)
    orp, ocol = oracle_radius(name, ncap, r, kern)
    t = sfc.octree_build(dev(p.xyz), enc, leaf_capacity=ncap)
    rp, cols = gpu_csr(*sfc.radius_search(t, None, r, kern))
    assert np.array_equal(rp, orp)
    assert np.array_equal(cols, p.rows_by_rank(orp, ocol))


@pytest.mark.parametrize("name,ncap,r", [("duplicates", 8, 0.03), ("identical", 8, 0.1), ("lattice", 4, 1.5),
                                         ("plane", 16, 0.8), ("clusters40k", 64, 1.0), ("uniform4097", 1, 0.1),
                                         ("uniform5", 2, 10.0)])
def test_radius_edge_clouds(name, ncap, r):
    for enc in ("none", "hilbert"):
        p = oracle_pipeline(name, enc, ncap)
        for kern in KERNS:
            orp, ocol = oracle_radius(name, ncap, r, kern)
            t = sfc.octree_build(dev(p.xyz), enc, leaf_capacity=ncap)
            rp, cols = gpu_csr(*sfc.radius_search(t, None, r, kern))
            assert np.array_equal(rp, orp), (enc, kern)
            assert np.array_equal(cols, p.rows_by_rank(orp, ocol)), (enc, kern)


def _centres(xyz: np.ndarray, n_in: int, seed: int) -> np.ndarray:
    rng = synth.Rng(seed)
    lo, hi = xyz.min(0).astype(np.float64), xyz.max(0).astype(np.float64)
    inside = lo + (hi - lo) * rng.u01(0, 3 * n_in).reshape(-1, 3)
    near = hi + rng.u01(1, 3 * 50).reshape(-1, 3) * 3.0          # just outside the box
    far = np.array([[1e6, -1e6, 3e5], [-50, -50, -50]], np.float64)
    exact = xyz[:: max(1, len(xyz) // 300)].astype(np.float64)     # centres on cloud points
    return np.ascontiguousarray(np.concatenate([inside, near, far, exact]).astype(np.float32))


@pytest.mark.parametrize("enc", ENCS)
@pytest.mark.parametrize("kern", KERNS)
def test_radius_caller_centres(kern, enc):
    name, ncap, r = "lidar60k", 32, 2.0
    p = oracle_pipeline(name, enc, ncap)
    q = _centres(p.xyz, 1007, 17)
    orp, ocol = p.tree.radius(q, r, KERN[kern])
    t = sfc.octree_build(dev(p.xyz), enc, leaf_capacity=ncap)
    rp, cols = gpu_csr(*sfc.radius_search(t, dev(q), r, kern))
    assert np.array_equal(rp, orp)
    assert np.array_equal(cols, p.rows_by_rank(orp, ocol))
    # the library-allocated CSR entry point gives the same arrays
    rp2, cols2 = gpu_csr(*sfc.radius_search_csr(t, dev(q), r, kern))
    assert np.array_equal(rp2, rp) and np.array_equal(cols2, cols)


@pytest.mark.parametrize("enc", ["morton", "hilbert"])
@pytest.mark.parametrize("spread", [4, 16])
def test_caller_centres_with_constant_code_digits(spread, enc):
    """Caller centres whose codes share most 8-bit digits: the sort of the centres skips
    those passes (one pass left for spread 4, two for spread 16 under Morton, so the
    sorted pairs end in either buffer), and the rows must still be the oracle's."""
    side = float(1 << 21)
    xyz = synth.uniform_cube(20_000, 107) * side
    xyz = np.concatenate([xyz, [[0.0, 0.0, 0.0], [side, side, side]]]).astype(np.float32)  # scale 1
    rng = synth.Rng(9)
    cells = (1 << 20) + 256 * (rng.u64(0, 3 * 3000) % np.uint64(spread)).astype(np.int64).reshape(-1, 3)
    if enc == "morton":
        codes = oracle.encode_cells(cells.astype(np.uint32), ENC[enc])
        varying = [d for d in range(8) if len(np.unique((codes >> np.uint64(8 * d)) & np.uint64(255))) > 1]
        assert varying == ([3] if spread == 4 else [3, 4])
    q = cells.astype(np.float32)
    p = oracle.Pipeline(xyz, ENC[enc], 16)
    orp, ocol = p.tree.radius(q, 60_000.0, KERN["sphere"])
    t = sfc.octree_build(dev(xyz), enc, leaf_capacity=16)
    assert t.scale == 1.0 and t.lo == (0.0, 0.0, 0.0)
    rp, cols = gpu_csr(*sfc.radius_search(t, dev(q), 60_000.0, "sphere"))
    assert orp[-1] > 0
    assert np.array_equal(rp, orp)
    assert np.array_equal(cols, p.rows_by_rank(orp, ocol))
    t.free()


def test_radius_special_radii():
    xyz = cloud("uniform4097")
    t = sfc.octree_build(dev(xyz), "hilbert", leaf_capacity=16)
    for r in (0.0, -1.0, -np.inf):
        rp, cols = gpu_csr(*sfc.radius_search(t, None, r, "sphere"))
        assert (rp == 0).all() and len(cols) == 0
    rp, cols = gpu_csr(*sfc.radius_search(t, dev(xyz[:10]), np.inf, "cube"))
    assert (np.diff(rp) == len(xyz)).all()
    with pytest.raises(sfc.SFCError) as e:
        sfc.radius_search(t, None, float("nan"), "sphere")
    assert e.value.status == 1


def test_radius_symmetry_and_encoding_invariance():
    xyz = cloud("lidar60k")
    sets = []
    for enc in ENCS:
        t = sfc.octree_build(dev(xyz), enc, leaf_capacity=32)
        rp, cols = gpu_csr(*sfc.radius_search(t, None, 1.0, "sphere"))
        sets.append((rp, csr_rows_sorted_by_id(rp, cols)))
    for rp, c in sets[1:]:
        assert np.array_equal(rp, sets[0][0]) and np.array_equal(c, sets[0][1])
    rp, c = sets[0]
    rows = np.repeat(np.arange(len(xyz)), np.diff(rp))
    fwd = rows.astype(np.int64) * len(xyz) + c
    bwd = c.astype(np.int64) * len(xyz) + rows
    assert np.array_equal(np.sort(fwd), np.sort(bwd))   # j in N(i) <=> i in N(j)


def test_radius_deterministic():
    xyz = cloud("clusters40k")
    t = sfc.octree_build(dev(xyz), "hilbert", leaf_capacity=16)
    a = gpu_csr(*sfc.radius_search(t, None, 1.5, "cube"))
    b = gpu_csr(*sfc.radius_search(t, None, 1.5, "cube"))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# ----------------------------------------------------------------------------- kNN
@pytest.mark.parametrize("enc", ENCS)
@pytest.mark.parametrize("k", [1, 8, 16, 32, 50, 64])
def test_knn_all_points_uniform(k, enc):
    """All-points kNN, every row: k = 8, 16, 32, 50 and 64 run the kernel copies with the
    list size (and, for the sorted encodings, the seeding window) fixed at compile time,
    k = 1 the copy with both known at run time."""
    p = oracle_pipeline("uniform131k", enc, 32)
    oidx, od2 = p.tree.knn(p.xyz, k)
    t = sfc.octree_build(dev(p.xyz), enc, leaf_capacity=32)
    idx, d2 = sfc.knn(t, None, k)
    assert np.array_equal(idx.cpu().numpy(), oidx)
    assert np.array_equal(d2.cpu().numpy().view(np.uint32), od2.view(np.uint32))


@pytest.mark.parametrize("name,ncap", [("lattice", 4), ("duplicates", 8), ("identical", 8), ("plane", 16),
                                       ("lidar60k", 32), ("uniform5", 2)])
@pytest.mark.parametrize("k", [1, 7, 26, 64])
def test_knn_ties_and_edges(name, ncap, k):
    xyz = cloud(name)
    q = np.concatenate([xyz, _centres(xyz, 200, 23)])
    if name == "lattice":  # half-integer centres: many exactly equal distances
        q = np.concatenate([q, (xyz[:500] + np.float32(0.5))])
    oidx, od2 = oracle.knn_brute(xyz, q, k)
    for enc in ENCS:
        t = sfc.octree_build(dev(xyz), enc, leaf_capacity=ncap)
        idx, d2 = sfc.knn(t, dev(q), k)
        assert np.array_equal(idx.cpu().numpy(), oidx), enc
        assert np.array_equal(d2.cpu().numpy().view(np.uint32), od2.view(np.uint32)), enc


def test_knn_empty_tree_pads():
    t = sfc.octree_build(dev(cloud("empty")), "hilbert")
    idx, d2 = sfc.knn(t, dev(np.zeros((3, 3), np.float32)), 4)
    assert (idx.cpu().numpy() == -1).all() and np.isinf(d2.cpu().numpy()).all()


def test_knn_locality_histogram_properties():
    """H_k(0) = N and sum H_k = kN (section 5.2) on the GPU's kNN rows."""
    xyz = cloud("uniform131k")
    t = sfc.octree_build(dev(xyz), "hilbert", leaf_capacity=32)
    idx, _ = sfc.knn(t, None, 8)
    perm = t.export()["perm"].cpu().numpy().astype(np.int64)
    rank = np.empty_like(perm)
    rank[perm] = np.arange(len(perm))
    h = oracle.locality_histogram(rank[idx.cpu().numpy().astype(np.int64)], rank, len(xyz))
    assert h[0] == len(xyz) and h.sum() == 8 * len(xyz)


# ----------------------------------------------------------------------------- errors
def test_errors_are_reported():
    xyz = cloud("uniform4097")
    bad = xyz.copy()
    bad[17, 1] = np.nan
    with pytest.raises(sfc.SFCError) as e:
        sfc.octree_build(dev(bad), "morton")
    assert e.value.status == 7
    t = sfc.octree_build(dev(xyz), "morton")
    q = xyz[:5].copy()
    q[2, 0] = np.inf
    with pytest.raises(sfc.SFCError) as e:
        sfc.radius_search(t, dev(q), 0.1, "sphere")
    assert e.value.status == 7
    with pytest.raises(sfc.SFCError) as e:
        sfc.knn(t, dev(q), 4)
    assert e.value.status == 7
    for k, status in ((0, 1), (65, 5)):
        with pytest.raises(sfc.SFCError) as e:
            sfc.knn(t, None, k)
        assert e.value.status == status
    # a host pointer is refused
    lib = sfc.binding.lib()
    h = ctypes.c_void_p()
    host = np.ascontiguousarray(xyz)
    st = lib.octree_build(host.ctypes.data_as(ctypes.c_void_p), len(host), 1, None, None, ctypes.byref(h))
    assert st == 6
    with pytest.raises(KeyError):
        sfc.radius_search(t, None, 0.1, "ellipse")


# ----------------------------------------------------------------------------- range output (neighboursStruct)
@pytest.mark.parametrize("enc", ENCS)
@pytest.mark.parametrize("name,ncap,r", [("uniform131k", 32, 0.04), ("lidar60k", 32, 2.0), ("lattice", 4, 2.5),
                                         ("duplicates", 8, 0.05), ("clusters40k", 16, 1.5)])
def test_radius_ranges_all_points(name, ncap, r, enc):
    p = oracle_pipeline(name, enc, ncap)
    t = sfc.octree_build(dev(p.xyz), enc, leaf_capacity=ncap)
    for kern in KERNS:
        rr = r if kern in ("sphere", "cube") else r * 0.6
        orp, oruns = p.radius_runs(p.xyz, rr, KERN[kern])
        rp, runs = sfc.radius_search_ranges(t, None, rr, kern)
        assert np.array_equal(rp.cpu().numpy(), orp), kern
        assert np.array_equal(runs.cpu().numpy().astype(np.int64), oruns), kern
        # the runs expand to the CSR of radius_search through the permutation
        crp, ccols = gpu_csr(*sfc.radius_search(t, None, rr, kern))
        perm = t.export()["perm"].cpu().numpy()
        lens = oruns[:, 1] - oruns[:, 0]
        run_rows = np.repeat(np.arange(len(orp) - 1), np.diff(orp))
        row_len = np.bincount(run_rows, weights=lens, minlength=len(orp) - 1).astype(np.int64)
        assert np.array_equal(np.diff(crp), row_len), kern
        expanded = np.arange(lens.sum()) - np.repeat(np.cumsum(lens) - lens, lens) + np.repeat(oruns[:, 0], lens)
        assert np.array_equal(perm[expanded], ccols), kern
        assert len(oruns) <= len(ccols)


@pytest.mark.parametrize("enc", ENCS)
def test_radius_ranges_caller_centres(enc):
    name, ncap, r = "lidar60k", 32, 3.0
    p = oracle_pipeline(name, enc, ncap)
    q = _centres(p.xyz, 1007, 29)
    t = sfc.octree_build(dev(p.xyz), enc, leaf_capacity=ncap)
    for kern in KERNS:
        orp, oruns = p.radius_runs(q, r, KERN[kern])
        rp, runs = sfc.radius_search_ranges(t, dev(q), r, kern)
        assert np.array_equal(rp.cpu().numpy(), orp), kern
        assert np.array_equal(runs.cpu().numpy().astype(np.int64), oruns), kern


def test_radius_ranges_special_cases():
    t = sfc.octree_build(dev(cloud("empty")), "hilbert")
    rp, runs = sfc.radius_search_ranges(t, None, 1.0, "sphere")
    assert rp.cpu().tolist() == [0] and runs.shape == (0, 2)
    xyz = cloud("identical")  # every point at one place: one run of all 100 positions per row
    t = sfc.octree_build(dev(xyz), "morton", leaf_capacity=8)
    rp, runs = sfc.radius_search_ranges(t, None, 0.5, "cube")
    assert (np.diff(rp.cpu().numpy()) == 1).all() and (runs.cpu().numpy() == [0, 100]).all()
    rp, runs = sfc.radius_search_ranges(t, None, 0.0, "sphere")
    assert (rp.cpu().numpy() == 0).all() and runs.shape == (0, 2)


# ----------------------------------------------------------------------------- locality histogram (section 5.2)
@pytest.mark.parametrize("enc", ENCS)
@pytest.mark.parametrize("name,step", [("lidar60k", 100), ("uniform131k", 100), ("duplicates", 7)])
def test_knn_locality_histogram(name, step, enc):
    p = oracle_pipeline(name, enc, 32)
    t = sfc.octree_build(dev(p.xyz), enc, leaf_capacity=32)
    ids = np.arange(0, len(p.xyz), step, dtype=np.int32)
    g = {}
    for order in ENCS:
        oh, og = p.locality(ids, 8, ENC[order])
        h, g1 = sfc.knn_locality(t, dev(ids), 8, order)
        assert np.array_equal(h.cpu().numpy(), oh), order
        assert abs(g1 - og) <= 1e-9 * max(1.0, abs(og)), order
        g[order] = og
    best, gs = sfc.choose_encoding(t, dev(ids), 8)
    assert best == max(g, key=g.get)
    for order in ENCS:
        assert abs(gs[order] - g[order]) <= 1e-9 * max(1.0, abs(g[order]))


def test_knn_locality_errors():
    t = sfc.octree_build(dev(cloud("uniform4097")), "hilbert")
    with pytest.raises(sfc.SFCError):
        sfc.knn_locality(t, dev(np.array([0, 4097], np.int32)), 4, "morton")
    with pytest.raises(sfc.SFCError):
        sfc.knn_locality(t, dev(np.array([0], np.int32)), 65, "morton")
    h, g1 = sfc.knn_locality(t, dev(np.zeros(0, np.int32)), 4, "morton")
    assert g1 == 0.0 and int(h.sum()) == 0

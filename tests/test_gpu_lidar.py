"""Parity at full size: the 10M-point LiDAR-like tile in the benchmark's launch configuration.

The build (codes, permutation, leaves, node table) is compared in full; searches run
over all points on the GPU and are compared with the oracle on seeded samples of rows,
plus properties checked over every row.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2603_06771_gb300 as sfc
import synth

pytestmark = pytest.mark.gpu

N_SAMPLE = 600
ENCS = ["none", "morton", "hilbert"]
KERNS = ["sphere", "circle", "cube", "square"]


@pytest.fixture(scope="module")
def tile():
    sfc.build()
    xyz = synth.config_cloud(2)
    p = oracle.Pipeline(xyz, oracle.ENC_HILBERT, 32)
    ranks = {"hilbert": p.rank}
    morton_perm, _ = oracle.sort_keys(oracle.encode_cells(p.cell, oracle.ENC_MORTON))
    r = np.empty(len(xyz), np.int64)
    r[morton_perm.astype(np.int64)] = np.arange(len(xyz))
    ranks["morton"] = ranks["none"] = r
    sample = np.sort(np.random.default_rng(2603).choice(len(xyz), N_SAMPLE, replace=False))
    return {"xyz": xyz, "p": p, "ranks": ranks, "sample": sample, "dev": torch.from_numpy(xyz).cuda()}


@pytest.fixture(scope="module")
def trees(tile):
    out = {enc: sfc.octree_build(tile["dev"], enc, leaf_capacity=32) for enc in ENCS}
    yield out
    for t in out.values():
        t.free()


def gpu_rows(row_ptr: torch.Tensor, cols: torch.Tensor, rows: np.ndarray):
    r = torch.as_tensor(rows, device="cuda", dtype=torch.int64)
    start = row_ptr[r]
    lens = row_ptr[r + 1] - start
    first = torch.cumsum(lens, 0) - lens
    total = int(lens.sum())
    pos = torch.repeat_interleave(start - first, lens) + torch.arange(total, device="cuda")
    return lens.cpu().numpy(), cols[pos].cpu().numpy()


def by_rank(rank: np.ndarray, lens: np.ndarray, cols: np.ndarray) -> np.ndarray:
    rows = np.repeat(np.arange(len(lens)), lens)
    return cols[np.lexsort((rank[cols.astype(np.int64)], rows))]


def test_build_full_arrays(tile, trees):
    p = tile["p"]
    t = trees["hilbert"]
    ex = t.export()
    assert np.array_equal(ex["keys"].cpu().numpy().view(np.uint64), p.sorted_keys)
    assert np.array_equal(ex["perm"].cpu().numpy().astype(np.uint32), p.perm)
    assert np.array_equal(ex["leaves"].cpu().numpy().view(np.uint64), p.leaves)
    assert np.array_equal(ex["counts"].cpu().numpy().astype(np.uint32), p.counts)
    nd = {k: v.cpu().numpy() for k, v in t.export_nodes().items()}
    on = p.nodes()
    go = np.lexsort((nd["level"], nd["key"].view(np.uint64)))
    oo = np.lexsort((on["level"], on["key"]))
    assert np.array_equal(nd["key"].view(np.uint64)[go], on["key"][oo])
    assert np.array_equal(nd["start"][go].astype(np.int64), on["start"][oo])
    assert np.array_equal(nd["end"][go].astype(np.int64), on["end"][oo])
    assert np.array_equal(nd["box"][go], on["box"][oo])


@pytest.mark.parametrize("enc", ENCS)
@pytest.mark.parametrize("kern", KERNS)
@pytest.mark.parametrize("r", [0.5, 1.0, 2.0, 3.0])
def test_radius_sampled_rows(tile, trees, kern, r, enc):
    p, s = tile["p"], tile["sample"]
    row_ptr, cols = sfc.radius_search(trees[enc], None, r, kern)
    assert int(row_ptr[-1]) == cols.numel()
    assert bool((row_ptr[1:] >= row_ptr[:-1]).all())
    lens, got = gpu_rows(row_ptr, cols, s)
    orp, ocol = p.tree.radius(tile["xyz"][s], r, oracle.KERNELS[kern])
    assert np.array_equal(lens, np.diff(orp))
    assert np.array_equal(got, by_rank(tile["ranks"][enc], np.diff(orp), ocol))
    del row_ptr, cols
    torch.cuda.empty_cache()


def test_radius_every_row_properties(tile, trees):
    """All-points sphere r = 2 (the benchmark's search): every row ascends along the curve,
    and j in N(i) <=> i in N(j) on a sample."""
    t = trees["hilbert"]
    row_ptr, cols = sfc.radius_search(t, None, 2.0, "sphere")
    rank = torch.as_tensor(tile["ranks"]["hilbert"].astype(np.int32), device="cuda")
    rk = rank[cols.long()]
    step_up = rk[1:] > rk[:-1]
    boundary = torch.zeros_like(step_up)
    inner = row_ptr[1:-1]
    inner = inner[(inner > 0) & (inner < cols.numel())]
    boundary[inner - 1] = True
    assert bool((step_up | boundary).all())
    del rk, step_up, boundary
    s = tile["sample"][:150]
    lens, nb = gpu_rows(row_ptr, cols, s)
    owner = np.repeat(s, lens)
    jl, jc = gpu_rows(row_ptr, cols, nb.astype(np.int64))
    jstart = np.concatenate([[0], np.cumsum(jl)[:-1]])
    for i, a, l in zip(owner, jstart, jl):
        assert i in jc[a:a + l]


@pytest.mark.parametrize("enc,k", [("hilbert", 8), ("hilbert", 16), ("hilbert", 50), ("morton", 16), ("none", 16)])
def test_knn_sampled_rows(tile, trees, enc, k):
    p, s = tile["p"], tile["sample"]
    idx, d2 = sfc.knn(trees[enc], None, k)
    oi, od = p.tree.knn(tile["xyz"][s], k)
    si = torch.as_tensor(s, device="cuda")
    assert np.array_equal(idx[si].cpu().numpy(), oi)
    assert np.array_equal(d2[si].cpu().numpy().view(np.uint32), od.view(np.uint32))
    # every row ascends in (d2, index)
    dd, ii = d2.cpu().numpy(), idx.cpu().numpy()
    assert ((dd[:, 1:] > dd[:, :-1]) | ((dd[:, 1:] == dd[:, :-1]) & (ii[:, 1:] > ii[:, :-1]))).all()


def test_every_row_sphere_r2_and_knn16_benchmark_config(tile):
    """Every row of the benchmark's searches (Hilbert, leaf capacity 96): the oracle answers
    all 10M centres (its pointer octree, all host cores); neighbour sets are compared row by
    row after sorting each row by id on the device, kNN lists exactly."""
    xyz, p = tile["xyz"], tile["p"]
    t = sfc.octree_build(tile["dev"], "hilbert", leaf_capacity=96)
    rp, cols = sfc.radius_search(t, None, 2.0, "sphere")
    orp, ocols = p.tree.radius(xyz, 2.0, oracle.SPHERE)
    assert np.array_equal(rp.cpu().numpy(), orp)

    def row_sorted(row_ptr: torch.Tensor, c: torch.Tensor) -> torch.Tensor:
        rows = torch.repeat_interleave(torch.arange(len(row_ptr) - 1, device="cuda"), torch.diff(row_ptr))
        return torch.sort((rows << 32) | c.to(torch.int64)).values

    want = row_sorted(torch.from_numpy(orp).cuda(), torch.from_numpy(ocols).cuda())
    assert torch.equal(row_sorted(rp, cols), want)
    del want, cols, rp
    idx, d2 = sfc.knn(t, None, 16)
    oi, od = p.tree.knn(xyz, 16)
    assert np.array_equal(idx.cpu().numpy(), oi)
    assert np.array_equal(d2.cpu().numpy().view(np.uint32), od.view(np.uint32))
    t.free()

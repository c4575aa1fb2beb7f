"""Parity of the batched path: every cloud of a batch gets exactly the results of the
oracle on that cloud alone, and the same bytes as the single-cloud entry points (CSR rows
in the same order, kNN lists bit for bit), whatever the other clouds in the batch."""
import numpy as np
import pytest
import torch

import paper_2603_06771_gb300 as sfc
import synth
from helpers import KERN, cloud, gpu_csr, oracle_pipeline

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _library():
    sfc.build()
    assert torch.cuda.is_available(), "these tests need a CUDA device"


def dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# (cloud, search): sizes from empty through one leaf to 131072 points, duplicates and
# exact ties, every kernel, k below and above the cloud size
MIX = [
    ("uniform4097", dict(search="radius", kernel="sphere", r=0.1)),
    ("lidar60k", dict(search="knn", k=16)),
    ("empty", dict(search="radius", kernel="cube", r=1.0)),
    ("clusters40k", dict(search="radius", kernel="cube", r=1.5)),
    ("identical", dict(search="knn", k=8)),
    ("uniform1", dict(search="knn", k=4)),
    ("duplicates", dict(search="radius", kernel="sphere", r=0.05)),
    ("uniform33", dict(search="knn", k=50)),
    ("lattice", dict(search="radius", kernel="square", r=1.0)),
    ("plane", dict(search="knn", k=32)),
    ("uniform5", dict(search="radius", kernel="circle", r=0.5)),
    ("empty", dict(search="knn", k=8)),
    ("uniform131k", dict(search="radius", kernel="sphere", r=0.04)),
    ("uniform4097", dict(search="radius", kernel="sphere", r=0.0)),
    ("lidar60k", dict(search="radius", kernel="sphere", r=2.0)),
    ("lattice", dict(search="knn", k=64)),
    ("clusters40k", dict(search="knn", k=1)),
]


def _run_batch(items, enc, ncap):
    xyz = [cloud(name) for name, _ in items]
    specs = [dict(spec, n=len(x)) for x, (_, spec) in zip(xyz, items)]
    pts = dev(np.concatenate(xyz) if xyz else np.zeros((0, 3), np.float32))
    return xyz, sfc.batch_search(pts, specs, enc, leaf_capacity=ncap)


def _radius_expected(name, enc, ncap, kern, r):
    p = oracle_pipeline(name, enc, ncap)
    rp, cols = p.tree.radius(p.xyz, r, KERN[kern])
    return rp, p.rows_by_rank(rp, cols)


@pytest.mark.parametrize("enc,ncap", [("hilbert", 32), ("morton", 8)])
def test_batch_matches_oracle(enc, ncap):
    xyz, b = _run_batch(MIX, enc, ncap)
    for i, (name, spec) in enumerate(MIX):
        if spec["search"] == "radius":
            rp, cols = gpu_csr(*b.radius(i))
            if spec["r"] > 0 and len(xyz[i]):
                orp, ocols = _radius_expected(name, enc, ncap, spec["kernel"], spec["r"])
            else:
                orp, ocols = np.zeros(len(xyz[i]) + 1, np.int64), np.zeros(0, np.int32)
            assert np.array_equal(rp, orp), (i, name)
            assert np.array_equal(cols, ocols), (i, name)
        else:
            idx, d2 = b.knn(i)
            if len(xyz[i]):
                p = oracle_pipeline(name, enc, ncap)
                oidx, od2 = p.tree.knn(p.xyz, spec["k"])
            else:
                oidx, od2 = np.zeros((0, spec["k"]), np.int32), np.zeros((0, spec["k"]), np.float32)
            assert np.array_equal(idx.cpu().numpy(), oidx), (i, name)
            assert np.array_equal(d2.cpu().numpy().view(np.uint32), od2.view(np.uint32)), (i, name)
    b.free()


def _single(x, spec, enc, ncap):
    t = sfc.octree_build(dev(x), enc, leaf_capacity=ncap)
    if spec["search"] == "radius":
        out = gpu_csr(*sfc.radius_search(t, None, spec["r"], spec["kernel"]))
    else:
        out = tuple(v.cpu().numpy() for v in sfc.knn(t, None, spec["k"]))
    t.free()
    return out


def _random_batch(n_clouds, seed, max_n):
    rng = synth.Rng(seed)
    sizes = (rng.u01(0, n_clouds) ** 3 * max_n).astype(np.int64)
    kinds = rng.integers(1, n_clouds, 8)
    xyz, specs = [], []
    for i in range(n_clouds):
        n = int(sizes[i])
        gen = int(kinds[i]) % 3
        if gen == 0:
            x = synth.uniform_cube(n, seed * 1000 + i, side=10.0)
        elif gen == 1:
            x = synth.gaussian_clusters(n, seed * 1000 + i) if n else np.zeros((0, 3), np.float32)
        else:
            x = synth.lidar_tile(n, seed * 1000 + i, side=float(max(np.sqrt(n / 10.0), 1.0))) if n \
                else np.zeros((0, 3), np.float32)
        xyz.append(x)
        if kinds[i] < 4:
            specs.append(dict(n=n, search="radius", kernel=["sphere", "circle", "cube", "square"][int(kinds[i])],
                              r=[0.5, 1.0, 2.0, 3.0][i % 4]))
        else:
            specs.append(dict(n=n, search="knn", k=[8, 16, 32, 5][int(kinds[i]) - 4]))
    return xyz, specs


@pytest.mark.parametrize("enc", ["hilbert", "morton"])
def test_batch_equals_single_cloud_calls(enc):
    """300 clouds of every generator and size: each is alone what it is in the mix."""
    ncap = 16
    xyz, specs = _random_batch(300, 7, 6000)
    b = sfc.batch_search(dev(np.concatenate(xyz)), specs, enc, leaf_capacity=ncap)
    for i, (x, spec) in enumerate(zip(xyz, specs)):
        want = _single(x, spec, enc, ncap)
        got = gpu_csr(*b.radius(i)) if spec["search"] == "radius" else tuple(v.cpu().numpy() for v in b.knn(i))
        assert np.array_equal(got[0], want[0]), i
        if spec["search"] == "radius":
            assert np.array_equal(got[1], want[1]), i
        else:
            assert np.array_equal(got[1].view(np.uint32), want[1].view(np.uint32)), i
    b.free()


def test_batch_order_independent():
    """A cloud's results do not depend on its neighbours in the batch or its position."""
    xyz, specs = _random_batch(40, 11, 4000)
    pts = dev(np.concatenate(xyz))
    a = sfc.batch_search(pts, specs, "hilbert", leaf_capacity=32)
    order = np.arange(40)[::-1]
    b = sfc.batch_search(dev(np.concatenate([xyz[i] for i in order])), [specs[i] for i in order], "hilbert",
                         leaf_capacity=32)
    for j, i in enumerate(order):
        if specs[i]["search"] == "radius":
            ra, rb = gpu_csr(*a.radius(int(i))), gpu_csr(*b.radius(j))
            assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])
        else:
            ka, kb = a.knn(int(i)), b.knn(j)
            assert torch.equal(ka[0], kb[0]) and torch.equal(ka[1], kb[1])


def test_batch_launches_do_not_grow_with_clouds():
    # eight clouds that open every search group, then 12 or 240 random clouds (the cloud
    # numbers fit one 8-bit radix digit in both)
    head_x = [synth.uniform_cube(500, 900 + j) for j in range(8)]
    head = [dict(n=500, search="radius", kernel=kern, r=0.1) for kern in ("sphere", "circle", "cube", "square")]
    head += [dict(n=500, search="knn", k=k) for k in (8, 16, 32, 64)]
    xyz, specs = _random_batch(240, 13, 3000)
    counts = []
    for m in (12, 240):
        before = sfc.launch_count()
        b = sfc.batch_search(dev(np.concatenate(head_x + xyz[:m])), head + specs[:m], "hilbert", leaf_capacity=32)
        counts.append(sfc.launch_count() - before)
        b.free()
    assert counts[0] == counts[1], counts


def test_batch_errors():
    x = dev(synth.uniform_cube(100, 3))
    ok = [dict(n=100, search="knn", k=4)]
    with pytest.raises(sfc.SFCError) as e:
        sfc.batch_search(x, [dict(n=100, search="knn", k=65)], "hilbert")
    assert e.value.status == 5  # SFC_ERR_TOO_LARGE
    with pytest.raises(sfc.SFCError) as e:
        sfc.batch_search(x, ok, "none")
    assert e.value.status == 1
    with pytest.raises(sfc.SFCError) as e:
        sfc.batch_search(x, [dict(n=100, search="radius", kernel="sphere", r=float("nan"))], "hilbert")
    assert e.value.status == 1
    with pytest.raises(sfc.SFCError) as e:
        sfc.batch_search(dev(synth.uniform_cube(1025, 5)), [dict(n=1, search="knn", k=1)] * 1025, "hilbert")
    assert e.value.status == 5
    with pytest.raises(ValueError):  # the clouds must cover the points exactly
        sfc.batch_search(x, [dict(n=99, search="knn", k=1)], "hilbert")
    bad = synth.uniform_cube(100, 3)
    bad[57, 1] = np.inf
    with pytest.raises(sfc.SFCError) as e:
        sfc.batch_search(dev(np.concatenate([synth.uniform_cube(50, 4), bad])),
                         [dict(n=50, search="knn", k=4), dict(n=100, search="knn", k=4)], "hilbert")
    assert e.value.status == 7  # SFC_ERR_NOT_FINITE
    b = sfc.batch_search(x, ok, "morton")  # the context is still usable
    assert b.knn(0)[0].shape == (100, 4)
    b.free()


# ----------------------------------------------------------------------------- batch plans
def _same(a, b, specs):
    for i, sp in enumerate(specs):
        if sp["search"] == "radius":
            ra, rb = gpu_csr(*a.radius(i)), gpu_csr(*b.radius(i))
            assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1]), i
        else:
            ka, kb = a.knn(i), b.knn(i)
            assert torch.equal(ka[0], kb[0]), i
            assert torch.equal(ka[1].view(torch.int32), kb[1].view(torch.int32)), i


@pytest.mark.parametrize("enc,ncap", [("hilbert", 32), ("morton", 8)])
def test_plan_matches_batch_search(enc, ncap):
    """A recorded plan gives batch_search's bytes (hence the oracle's), run after run."""
    items = [it for it in MIX if it[0] != "empty"] + [MIX[2]]  # an empty cloud last
    xyz = [cloud(name) for name, _ in items]
    specs = [dict(spec, n=len(x)) for x, (_, spec) in zip(xyz, items)]
    pts = dev(np.concatenate(xyz))
    want = sfc.batch_search(pts, specs, enc, leaf_capacity=ncap)
    plan = sfc.BatchPlan(specs, enc, leaf_capacity=ncap)
    plan.points.copy_(pts)
    before = sfc.launch_count()
    plan.run()
    per_run = sfc.launch_count() - before
    assert per_run > 20
    _same(plan, want, specs)
    plan.run()  # a replay of the same graph
    _same(plan, want, specs)
    assert sfc.launch_count() - before == 2 * per_run
    plan.free()
    want.free()


def test_plan_new_points_each_run():
    xyz, specs = _random_batch(60, 17, 5000)
    plan = sfc.BatchPlan(specs, "hilbert", leaf_capacity=16)
    for seed in (0, 1):
        pts = [x if seed == 0 else (x[::-1].copy() * np.float32(1.5)) for x in xyz]
        p = dev(np.concatenate(pts))
        plan.points.copy_(p)
        plan.run()
        _same(plan, sfc.batch_search(p, specs, "hilbert", leaf_capacity=16), specs)
    plan.free()


def test_plan_radius_output_overflow_regrows():
    """A radius output capacity far too small: the run skips its fill, finish grows the
    array to the exact size and fills again; the next run uses a graph recorded with it."""
    items = [("uniform4097", dict(search="radius", kernel="sphere", r=0.1)),
             ("clusters40k", dict(search="knn", k=16)),
             ("lidar60k", dict(search="radius", kernel="cube", r=1.0))]
    xyz = [cloud(name) for name, _ in items]
    specs = [dict(spec, n=len(x)) for x, (_, spec) in zip(xyz, items)]
    pts = dev(np.concatenate(xyz))
    want = sfc.batch_search(pts, specs, "hilbert", leaf_capacity=32)
    plan = sfc.BatchPlan(specs, "hilbert", leaf_capacity=32, nnz_capacity=1)
    plan.points.copy_(pts)
    plan.run()
    _same(plan, want, specs)
    plan.run()
    _same(plan, want, specs)
    plan.free()


def test_plan_errors():
    with pytest.raises(sfc.SFCError) as e:
        sfc.BatchPlan([dict(n=0, search="knn", k=4)], "hilbert")
    assert e.value.status == 1
    plan = sfc.BatchPlan([dict(n=100, search="knn", k=4)], "hilbert")
    with pytest.raises(sfc.SFCError):
        plan.finish()  # nothing launched
    bad = synth.uniform_cube(100, 3)
    bad[5, 0] = np.nan
    plan.points.copy_(dev(bad))
    with pytest.raises(sfc.SFCError) as e:
        plan.run()
    assert e.value.status == 7
    plan.points.copy_(dev(synth.uniform_cube(100, 3)))
    plan.run()  # the plan is still usable
    assert plan.knn(0)[0].shape == (100, 4)
    plan.free()


# ----------------------------------------------------------------------------- per-cloud knobs and the tuner
def test_per_cloud_leaf_capacity_and_window_keep_results():
    """Leaf capacity and seeding window are speed knobs: any per-cloud choice gives the
    same bytes (each cloud equals its single-cloud run at its own capacity)."""
    xyz, specs = _random_batch(24, 19, 5000)
    caps = [16, 64, 256, 8, 33, 1]
    wins = [1, 8, 16, 32, 0, 5]
    for i, sp in enumerate(specs):
        sp["leaf_capacity"] = caps[i % len(caps)]
        if sp["search"] == "knn":
            sp["knn_window"] = wins[i % len(wins)]
    b = sfc.batch_search(dev(np.concatenate(xyz)), specs, "hilbert", leaf_capacity=32)
    for i, (x, sp) in enumerate(zip(xyz, specs)):
        want = _single(x, sp, "hilbert", sp["leaf_capacity"])
        got = gpu_csr(*b.radius(i)) if sp["search"] == "radius" else tuple(v.cpu().numpy() for v in b.knn(i))
        assert np.array_equal(got[0], want[0]), i
        assert np.array_equal(got[1].view(np.uint32), want[1].view(np.uint32)), i
    b.free()


def test_autotune_choices_are_valid_and_keep_results():
    xyz, specs = _random_batch(30, 23, 8000)
    pts = dev(np.concatenate(xyz))
    tuned = sfc.batch_autotune(pts, specs, "hilbert", leaf_candidates=(16, 64), window_candidates=(16, 32),
                               qpw_candidates=(8, 16, 32), slot_candidates=(4, 64))
    for sp, t in zip(specs, tuned):
        searched = sp["n"] > 0 and (sp["search"] == "knn" or sp.get("r", 0) > 0)
        assert t["leaf_capacity"] in (16, 32, 64)  # 32: clouds without a search keep the default
        assert t["knn_window"] in ((16, 32) if sp["search"] == "knn" and sp["n"] > 0 else (0,))
        assert t["queries_per_warp"] in ((8, 16, 32) if searched else (0,))
        assert t["record_slots"] in ((4, 64) if searched and sp["search"] == "radius" else (0,))
    _same(sfc.batch_search(pts, tuned, "hilbert"), sfc.batch_search(pts, specs, "hilbert"), specs)
    with pytest.raises(sfc.SFCError):
        sfc.batch_autotune(pts, specs, "hilbert", window_candidates=(65,))
    with pytest.raises(sfc.SFCError):
        sfc.batch_autotune(pts, specs, "hilbert", qpw_candidates=(12,))
    with pytest.raises(sfc.SFCError):
        sfc.batch_autotune(pts, specs, "hilbert", slot_candidates=(0,))


@pytest.mark.parametrize("qpw,slots", [(8, 1), (16, 3), (32, 128)])
def test_queries_per_warp_and_record_slots_keep_results(qpw, slots):
    """Every cloud walked by groups of 8, 16 or 32 centres, with 1 to 128 record slots per
    group (1 slot: almost every group overflows and walks again in the fill), gives the
    same bytes as the defaults."""
    xyz, specs = _random_batch(20, 29, 6000)
    pts = dev(np.concatenate(xyz))
    knobbed = [dict(sp, queries_per_warp=qpw, record_slots=slots) for sp in specs]
    _same(sfc.batch_search(pts, knobbed, "hilbert"), sfc.batch_search(pts, specs, "hilbert"), specs)
    plan = sfc.BatchPlan(knobbed, "hilbert")
    plan.points.copy_(pts)
    plan.run()
    _same(plan, sfc.batch_search(pts, specs, "hilbert"), specs)
    plan.free()

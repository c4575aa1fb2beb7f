"""Pins of the CPU oracle against facts the paper and the mathematics fix.

None of these re-types the oracle's formulas: they check worked examples printed
in the paper, closed forms, invariants, hand-worked cases and brute force on tiny
inputs, chosen so that a dropped term, a wrong sign or index or a transposed
operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from conftest import read_golden

ALL_KERNELS = [oracle.SPHERE, oracle.CIRCLE, oracle.CUBE, oracle.SQUARE]
KNAME = {"sphere": oracle.SPHERE, "circle": oracle.CIRCLE, "cube": oracle.CUBE, "square": oracle.SQUARE}


# ----------------------------------------------------------------------------- section 4.1 Morton
def test_morton_worked_example():
    for L, x, y, z, code in read_golden("morton_worked_example.txt"):
        assert oracle.morton(int(x), int(y), int(z), int(L)) == int(code)
        assert tuple(oracle.decode_codes(np.array([int(code)], np.uint64), oracle.ENC_MORTON, int(L))[0]) == (
            int(x), int(y), int(z))


def _all_cells(L):
    g = np.arange(1 << L, dtype=np.uint32)
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


@pytest.mark.parametrize("enc", [oracle.ENC_MORTON, oracle.ENC_HILBERT])
@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_curve_is_bijection(enc, L):
    """An SFC of level l maps S_l one-to-one onto [0, 2^{3l}) (section 4, Definition)."""
    cells = _all_cells(L)
    codes = oracle.encode_cells(cells, enc, L)
    assert np.array_equal(np.sort(codes), np.arange(8 ** L, dtype=np.uint64))
    assert np.array_equal(oracle.decode_codes(codes, enc, L), cells)


@pytest.mark.parametrize("enc", [oracle.ENC_MORTON, oracle.ENC_HILBERT])
@pytest.mark.parametrize("L", [2, 3, 4])
def test_curve_is_recursive(enc, L):
    """Every aligned block of 8^m codes is an aligned cube of side 2^m (section 4, Definition)."""
    cells = oracle.decode_codes(np.arange(8 ** L, dtype=np.uint64), enc, L).astype(np.int64)
    for m in range(L + 1):
        blocks = cells.reshape(-1, 8 ** m, 3)
        lo = blocks.min(axis=1)
        hi = blocks.max(axis=1)
        assert np.all(hi - lo == (1 << m) - 1)
        assert np.all(lo % (1 << m) == 0)


@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_hilbert_is_continuous(L):
    """Consecutive Hilbert codes are face neighbours: L1 distance 1 (stronger than the
    L-infinity continuity of the Definition in section 4)."""
    cells = oracle.decode_codes(np.arange(8 ** L, dtype=np.uint64), oracle.ENC_HILBERT, L).astype(np.int64)
    step = np.abs(np.diff(cells, axis=0)).sum(axis=1)
    assert np.all(step == 1)
    assert tuple(cells[0]) == (0, 0, 0)


def test_morton_is_not_continuous():
    cells = oracle.decode_codes(np.arange(64, dtype=np.uint64), oracle.ENC_MORTON, 2).astype(np.int64)
    assert np.abs(np.diff(cells, axis=0)).max() > 1


@pytest.mark.parametrize("enc", [oracle.ENC_MORTON, oracle.ENC_HILBERT])
def test_curves_at_full_depth(enc):
    """At L = 21: decode inverts encode, codes stay below 2^63, and (Hilbert) code c
    and c + 1 are face neighbours for random c."""
    rng = synth.Rng(99)
    cells = (rng.u64(0, 3 * 20000) >> np.uint64(43)).astype(np.uint32).reshape(-1, 3)
    codes = oracle.encode_cells(cells, enc)
    assert np.all(codes < np.uint64(1 << 63))
    assert np.array_equal(oracle.decode_codes(codes, enc), cells)
    if enc == oracle.ENC_HILBERT:
        c = rng.u64(1, 20000) >> np.uint64(1)
        c = c[c < np.uint64((1 << 63) - 1)]
        a = oracle.decode_codes(c, enc).astype(np.int64)
        b = oracle.decode_codes(c + np.uint64(1), enc).astype(np.int64)
        assert np.all(np.abs(a - b).sum(axis=1) == 1)


def test_morton_matches_numpy_bit_interleave():
    """Morton at L = 21 against an interleave built from numpy bit operations."""
    rng = synth.Rng(7)
    cells = (rng.u64(0, 3 * 5000) >> np.uint64(43)).astype(np.uint64).reshape(-1, 3)
    want = np.zeros(len(cells), np.uint64)
    for b in range(21):
        for axis, off in ((0, 2), (1, 1), (2, 0)):
            bit = (cells[:, axis] >> np.uint64(b)) & np.uint64(1)
            want |= bit << np.uint64(3 * b + off)
    assert np.array_equal(oracle.encode_cells(cells.astype(np.uint32), oracle.ENC_MORTON), want)


# ----------------------------------------------------------------------------- section 4 discretisation
def test_discretise_hand_example():
    """Lower corner -> 0 (section 4, step 2); extent 8 -> scale 2^21 / 8 = 2^18; the upper
    corner lands on 2^21 and is clamped to 2^21 - 1; the scale is one for all axes."""
    xyz = np.array([[0, 0, 0], [8, 2, 1], [3.5, 1.25, 0.5], [2 ** -30, 0, 0]], np.float32)
    lo, ext, s = oracle.bbox(xyz)
    assert list(lo) == [0, 0, 0] and ext == 8.0 and s == 2.0 ** 18
    cell = oracle.discretise(xyz, lo, s)
    assert cell.tolist() == [[0, 0, 0], [2 ** 21 - 1, 2 ** 19, 2 ** 18], [917504, 327680, 131072], [0, 0, 0]]


def test_discretise_shifted_and_flat():
    xyz = np.array([[-5, 10, 3], [-1, 10, 3], [-3, 10, 3]], np.float32)
    lo, ext, s = oracle.bbox(xyz)
    assert list(lo) == [-5, 10, 3] and ext == 4.0
    assert oracle.discretise(xyz, lo, s).tolist() == [[0, 0, 0], [2 ** 21 - 1, 0, 0], [2 ** 20, 0, 0]]
    one = np.array([[1.5, -2, 7]], np.float32)
    lo, ext, s = oracle.bbox(one)
    assert ext == 1.0 and oracle.discretise(one, lo, s).tolist() == [[0, 0, 0]]


def test_bbox_rejects_non_finite():
    for bad in (np.nan, np.inf):
        with pytest.raises(ValueError):
            oracle.bbox(np.array([[0, 0, 0], [1, bad, 0]], np.float32))
    with pytest.raises(ValueError):   # the extent overflows binary32
        oracle.bbox(np.array([[-3e38, 0, 0], [3e38, 0, 0]], np.float32))


# ----------------------------------------------------------------------------- section 4 reorder
def test_sort_is_stable_ascending():
    rng = synth.Rng(3)
    keys = rng.u64(0, 50000) >> np.uint64(54)   # many duplicates
    perm, srt = oracle.sort_keys(keys)
    assert np.array_equal(perm, np.argsort(keys, kind="stable"))
    assert np.array_equal(srt, keys[perm])


# ----------------------------------------------------------------------------- section 5.1 leaves
def _check_leaves(lv, ct, sk, ncap):
    lv = lv.astype(object)
    n = len(sk)
    assert lv[0] == 0 and lv[-1] == 8 ** 21
    assert (len(lv) - 1) % 7 == 1            # complete octree: 7 * internal + 1 leaves
    assert int(ct.sum()) == n
    pos = lambda k: int(np.searchsorted(sk, np.uint64(k), side="left")) if k < 8 ** 21 else n
    for a, b, c in zip(lv[:-1], lv[1:], ct):
        size = b - a
        m = round(math.log(size, 8))
        assert 8 ** m == size and a % size == 0          # an octree cell
        assert pos(b) - pos(a) == c
        assert c <= ncap or size == 1                    # not over-full (level-21 cells may be)
        if size < 8 ** 21:                               # its parent was over-full
            pa = a - a % (size * 8)
            assert pos(pa + size * 8) - pos(pa) > ncap


@pytest.mark.parametrize("gen,n,ncap", [("uniform", 5000, 32), ("lidar", 20000, 16), ("clusters", 8000, 64),
                                        ("uniform", 20, 32)])
def test_leaves_invariants_and_pointer_octree(gen, n, ncap):
    xyz = {"uniform": synth.uniform_cube, "lidar": synth.lidar_tile,
           "clusters": synth.gaussian_clusters}[gen](n, 11)
    for enc in (oracle.ENC_MORTON, oracle.ENC_HILBERT):
        p = oracle.Pipeline(xyz, enc, ncap)
        _check_leaves(p.leaves, p.counts, p.sorted_keys, ncap)
        nd = p.nodes()
        # the pointer octree (section 3.1) has the same cells as the linear octree (5.1)
        leaf_keys = np.sort(nd["key"][nd["is_leaf"] == 1])
        assert np.array_equal(leaf_keys, p.leaves[:-1])
        n_int = int((nd["is_leaf"] == 0).sum())
        assert len(nd["key"]) == 8 * n_int + 1
        # every node's points are one contiguous run of the sorted cloud (internalRanges)
        assert nd["contiguous"].all()
        lidx = np.searchsorted(p.leaves[:-1], nd["key"][nd["is_leaf"] == 1])
        assert np.array_equal(nd["count"][nd["is_leaf"] == 1], p.counts[lidx])


@pytest.mark.parametrize("gen", ["uniform", "lidar", "dup"])
def test_node_boxes_are_the_tight_boxes(gen):
    """Every node's box is the min/max of its own points, no larger and no smaller (the
    pruning boxes of reading 8): the points of the node at (first code, level) are those
    whose code lies in [first, first + 8^(21 - level)) (section 5.1), here found with numpy
    over the sorted codes; empty nodes carry the empty box (+inf, -inf)."""
    xyz = {"uniform": lambda: synth.uniform_cube(4000, 12),
           "lidar": lambda: synth.lidar_tile(5000, 13, side=25.0),
           "dup": lambda: np.repeat(synth.uniform_cube(200, 14), 20, axis=0)}[gen]()
    for enc in (oracle.ENC_MORTON, oracle.ENC_HILBERT):
        p = oracle.Pipeline(xyz, enc, 16)
        nd = p.nodes()
        sk = p.sorted_keys
        pts = xyz[p.perm.astype(np.int64)]
        for i in range(len(nd["key"])):
            first = int(nd["key"][i])
            span = 1 << (3 * (oracle.L - int(nd["level"][i])))
            a = int(np.searchsorted(sk, np.uint64(first), "left"))
            b = int(np.searchsorted(sk, np.uint64(first + span - 1), "right"))
            assert nd["count"][i] == b - a
            box = nd["box"][i]
            if b == a:
                assert np.isposinf(box[:3]).all() and np.isneginf(box[3:]).all()
                continue
            assert (nd["start"][i], nd["end"][i]) == (a, b)
            assert np.array_equal(box[:3], pts[a:b].min(0)), (gen, enc, i)
            assert np.array_equal(box[3:], pts[a:b].max(0)), (gen, enc, i)


def test_leaves_closed_forms():
    # N <= N_max: the root is the only leaf
    lv, ct = oracle.leaves(np.arange(10, dtype=np.uint64), 32)
    assert lv.tolist() == [0, 8 ** 21] and ct.tolist() == [10]
    lv, ct = oracle.leaves(np.zeros(0, np.uint64), 8)
    assert lv.tolist() == [0, 8 ** 21] and ct.tolist() == [0]
    # N > N_max identical codes: every level 0..20 splits once -> 7 * 21 + 1 leaves,
    # and the single level-21 cell holds all N points
    key = np.uint64(0o123456701234567012345)
    lv, ct = oracle.leaves(np.full(100, key, np.uint64), 8)
    assert len(lv) - 1 == 7 * 21 + 1
    assert ct.max() == 100 and (ct > 0).sum() == 1
    assert lv[np.argmax(ct)] == key
    # 9 points in 9 distinct level-1 octants cannot exist; 9 points over 2 octants with N_max 8:
    keys = np.sort(np.array([0] * 5 + [8 ** 20 * 3] * 4, np.uint64))
    lv, ct = oracle.leaves(keys, 8)
    assert len(lv) - 1 == 8 and ct.tolist() == [5, 0, 0, 4, 0, 0, 0, 0]


# ----------------------------------------------------------------------------- section 3.2 kernels
def test_kernel_hand_cases():
    for k, px, py, pz, cx, cy, cz, r, inside in read_golden("kernel_hand_cases.txt"):
        p = np.array([px, py, pz], np.float32)
        c = np.array([cx, cy, cz], np.float32)
        assert oracle.pred(KNAME[k], p, c, float(r)) == bool(int(inside)), (k, p, c, r)


def _clouds():
    rng = synth.Rng(5)
    uni = synth.uniform_cube(3000, 21)
    lat = np.stack(np.meshgrid(*[np.arange(7, dtype=np.float32)] * 3, indexing="ij"), -1).reshape(-1, 3)
    dup = np.repeat(synth.uniform_cube(300, 22), 4, axis=0)      # every point four times
    lid = synth.lidar_tile(6000, 23, side=30.0)
    flat = synth.uniform_cube(2000, 24, side=10.0)
    flat[:, 2] = 0.0                                               # a plane: zero z extent
    return {"uniform": (uni, 0.1), "lattice": (lat, 1.0), "dup": (dup, 0.15), "lidar": (lid, 2.0),
            "flat": (flat, 0.7)}


@pytest.mark.parametrize("name", ["uniform", "lattice", "dup", "lidar", "flat"])
def test_tree_search_equals_brute_force(name):
    xyz, r = _clouds()[name]
    q = np.concatenate([xyz[::7], xyz[:50] + np.float32(0.01), np.array([[100, 100, 100]], np.float32)])
    tree = oracle.PointerOctree(xyz, 16)
    for kern in ALL_KERNELS:
        for rr in (r, r * 0.5, 0.0):
            a = oracle.radius_brute(xyz, q, rr, kern, nthreads=4)
            b = tree.radius(q, rr, kern, nthreads=4)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), (name, kern, rr)


@pytest.mark.parametrize("name", ["uniform", "lattice", "dup"])
def test_kernels_symmetric_and_nested(name):
    xyz, r = _clouds()[name]
    rows = {}
    for kern in ALL_KERNELS:
        rp, cols = oracle.radius_brute(xyz, xyz, r, kern, nthreads=4)
        m = np.zeros((len(xyz), len(xyz)), bool)
        m[np.repeat(np.arange(len(xyz)), np.diff(rp)), cols] = True
        assert np.array_equal(m, m.T)                          # j in N(i) <=> i in N(j)
        assert m.diagonal().all()                               # the centre is its own neighbour
        rows[kern] = m
    s, c, cu, sq = rows[oracle.SPHERE], rows[oracle.CIRCLE], rows[oracle.CUBE], rows[oracle.SQUARE]
    assert not (s & ~cu).any()      # ball inside the cube of half-side r
    assert not (s & ~c).any()       # dropping z can only shrink a distance
    assert not (cu & ~sq).any()
    assert not (c & ~sq).any()


def test_sphere_mean_count_matches_volume():
    """Interior centres of a uniform cloud see about N * 4/3 pi r^3 neighbours."""
    xyz = synth.config_cloud(1)
    r = 0.04
    inner = xyz[np.all((xyz > r) & (xyz < 1 - r), axis=1)][:4000]
    rp, _ = oracle.radius_brute(xyz, inner, r, oracle.SPHERE)
    mu = np.diff(rp).mean()
    assert abs(mu - len(xyz) * 4.0 / 3.0 * math.pi * r ** 3) < 1.0
    rp, _ = oracle.radius_brute(xyz, inner, r, oracle.CUBE)
    assert abs(np.diff(rp).mean() - len(xyz) * (2 * r) ** 3) < 1.5


def test_boundary_report_runs():
    xyz, r = _clouds()["lattice"]
    # on the integer lattice every distance is exact in both precisions
    assert oracle.boundary_disagreements(xyz, xyz, r, oracle.SPHERE) == 0


def _rounding_cases():
    """Rows of rounding_cases.txt grouped by kernel: (points, centre, r, columns)."""
    groups = {}
    for row in read_golden("rounding_cases.txt"):
        vals = [np.float32(float.fromhex(v)) for v in row[1:8]]
        cols = {name: (None if v == "-" else bool(int(v)))
                for name, v in zip(("inside", "o2", "o3", "fma1", "fma2", "f64"), row[8:14])}
        g = groups.setdefault(row[0], dict(p=[], c=vals[3:6], r=vals[6], cols=[]))
        assert g["c"] == vals[3:6] and g["r"] == vals[6]          # one centre and radius per kernel
        g["p"].append(vals[0:3])
        g["cols"].append(cols)
    return groups


def test_kernel_rounding_cases():
    """Section 3.2 tests at the rounding boundary, decided by exact rational arithmetic
    (tests/golden/make_rounding_cases.py): the oracle takes the reading's decision on every
    row, and every plausible mistake (another summation order, a fused multiply-add, the
    test evaluated in binary64) takes another one on at least one row."""
    groups = _rounding_cases()
    assert set(groups) == set(KNAME)
    for name, g in groups.items():
        kern = KNAME[name]
        c = np.array(g["c"], np.float32)
        for p, cols in zip(g["p"], g["cols"]):
            assert oracle.pred(kern, np.array(p, np.float32), c, float(g["r"])) == cols["inside"], (name, p)
        for alt in ("o2", "o3", "fma1", "fma2", "f64"):
            if any(cols[alt] is not None for cols in g["cols"]):
                assert any(cols[alt] != cols["inside"] for cols in g["cols"]), (name, alt)
        # the searches decide the same: brute force and the pointer octree
        xyz = np.array(g["p"], np.float32)
        want = [i for i, cols in enumerate(g["cols"]) if cols["inside"]]
        rp, got = oracle.radius_brute(xyz, c[None], float(g["r"]), kern)
        assert got.tolist() == want
        rp, got = oracle.PointerOctree(xyz, 2).radius(c[None], float(g["r"]), kern)
        assert got.tolist() == want


def test_boundary_report_counts_the_disagreements():
    """The boundary report counts the (point, centre) pairs whose binary32 decision differs
    from the binary64 evaluation of the same expression; the rounding cases fix the count."""
    total = 0
    for name, g in _rounding_cases().items():
        want = sum(cols["inside"] != cols["f64"] for cols in g["cols"])
        assert want > 0
        xyz = np.array(g["p"], np.float32)
        c = np.array(g["c"], np.float32)[None]
        assert oracle.boundary_disagreements(xyz, c, float(g["r"]), KNAME[name]) == want, name
        # every pair counted once: the same centre twice doubles the count
        assert oracle.boundary_disagreements(xyz, np.repeat(c, 2, 0), float(g["r"]), KNAME[name]) == 2 * want
        total += want
    assert total >= 16


# ----------------------------------------------------------------------------- section 3.3 kNN
def test_knn_hand_example():
    xyz = np.array([[i, 0, 0] for i in range(10)], np.float32)
    idx, d2 = oracle.knn_brute(xyz, np.array([[4.5, 0, 0]], np.float32), 5)
    assert idx.tolist() == [[4, 5, 3, 6, 2]]                    # ties go to the smaller index
    assert d2.tolist() == [[0.25, 0.25, 2.25, 2.25, 6.25]]
    idx, d2 = oracle.knn_brute(xyz[:3], np.array([[0, 0, 0]], np.float32), 5)
    assert idx.tolist() == [[0, 1, 2, -1, -1]] and np.isinf(d2[0, 3:]).all()


def test_knn_rounding_order():
    """Section 3.3 order of two candidates whose binary32 squared distances tie or differ by
    one unit in the last place (tests/golden/knn_rounding_cases.txt, exact rational
    arithmetic): the oracle's distances are the reading's bit for bit and its order puts the
    smaller first, a tie to the smaller index; another summation order or a fused
    multiply-add flips the order on at least one row."""
    rows = read_golden("knn_rounding_cases.txt")
    flips = {k: 0 for k in ("o2", "o3", "fma1", "fma2")}
    ties = 0
    for row in rows:
        f = [np.float32(float.fromhex(v)) for v in row[0:9]]
        c, p0, p1 = np.array(f[0:3])[None], f[3:6], f[6:9]
        order, d0, d1 = row[9], np.float32(float.fromhex(row[10])), np.float32(float.fromhex(row[11]))
        ties += d0 == d1
        for k, v in zip(flips, row[12:16]):
            flips[k] += v != order
        want = [0, 1] if order == "01" else [1, 0]
        xyz = np.array([p0, p1], np.float32)
        for idx, d2 in (oracle.knn_brute(xyz, c, 2), oracle.PointerOctree(xyz, 1).knn(c, 2)):
            assert idx[0].tolist() == want, row
            assert d2[0].tobytes() == np.array([d0, d1][::1 if want == [0, 1] else -1], np.float32).tobytes()
        # the same two points in the other storage order: a tie now goes to the other one
        idx, _ = oracle.knn_brute(xyz[::-1].copy(), c, 1)
        assert idx[0, 0] == (0 if (d1 < d0 or d0 == d1) else 1), row
    assert ties >= 2 and all(v > 0 for v in flips.values()), (ties, flips)


@pytest.mark.parametrize("name", ["uniform", "lattice", "dup", "lidar", "flat"])
def test_knn_tree_equals_brute_force(name):
    xyz, _ = _clouds()[name]
    q = np.concatenate([xyz[::5], np.array([[100, 100, 100], [3.5, 3.5, 3.5]], np.float32)])
    tree = oracle.PointerOctree(xyz, 16)
    for k in (1, 8, 16, 50):
        a = oracle.knn_brute(xyz, q, k, nthreads=4)
        b = tree.knn(q, k, nthreads=4)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), (name, k)
    # more neighbours than points: padding
    small = xyz[:20]
    i1, d1 = oracle.PointerOctree(small, 4).knn(q[:10], 30)
    assert (i1[:, 20:] == -1).all() and np.isinf(d1[:, 20:]).all()
    assert np.array_equal(np.sort(i1[:, :20], axis=1), np.tile(np.arange(20), (10, 1)))


def test_knn_rows_are_exact_and_sorted():
    xyz = synth.uniform_cube(3000, 31)
    q = xyz[::13]
    idx, d2 = oracle.PointerOctree(xyz, 32).knn(q, 16)
    assert (np.diff(d2, axis=1) >= 0).all()
    for i in range(0, len(q), 17):
        diff = xyz.astype(np.float64) - q[i].astype(np.float64)
        dd = (diff ** 2).sum(1)
        kth = d2[i, -1]
        # float64 distances differ from the binary32 ones by a few ulp at most
        assert (dd[np.setdiff1d(np.arange(len(xyz)), idx[i])] >= kth * (1 - 1e-5)).all()
        assert np.allclose(dd[idx[i]], d2[i], rtol=1e-5, atol=1e-12)


# ----------------------------------------------------------------------------- section 5.1 range output
def _merge(entries):
    out = []
    for s0, e0 in entries:
        if out and out[-1][1] == s0:
            out[-1] = (out[-1][0], e0)
        else:
            out.append((s0, e0))
    return out


def test_runs_of_rows_hand_example():
    # rows: {3,4,5,9,11,12}, {}, {7}, {0,1}
    rp = np.array([0, 6, 6, 7, 9])
    pos = np.array([3, 4, 5, 9, 11, 12, 7, 0, 1])
    run_ptr, runs = oracle.runs_of_rows(rp, pos)
    assert run_ptr.tolist() == [0, 3, 3, 4, 5]
    assert runs.tolist() == [[3, 6], [9, 10], [11, 13], [7, 8], [0, 2]]


@pytest.mark.parametrize("gen", ["uniform", "lattice", "lidar"])
def test_neighbours_struct_merges_to_the_runs(gen):
    """The paper's neighboursStruct walk (octant ranges + single points), with adjacent
    entries merged, is the run encoding of the exact neighbour set; large radii make it
    take whole octants."""
    if gen == "uniform":
        xyz = synth.uniform_cube(2500, 61)
        radii = (0.05, 0.2, 0.45)
    elif gen == "lattice":
        g = np.arange(9, dtype=np.float32)
        xyz = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).copy()
        radii = (1.0, 2.5, 4.0)
    else:
        xyz = synth.lidar_tile(3000, 62, side=float(np.sqrt(300.0)))
        radii = (0.5, 2.0, 6.0)
    p = oracle.Pipeline(xyz, oracle.ENC_HILBERT, 8)
    centres = xyz[::97]
    took_octant = False
    for kern in (oracle.SPHERE, oracle.CIRCLE, oracle.CUBE, oracle.SQUARE):
        for r in radii:
            run_ptr, runs = p.radius_runs(centres, r, kern)
            brp, bcols = oracle.radius_brute(xyz, centres, r, kern)
            for i, c in enumerate(centres):
                ent = p.neighbours_struct(c, r, kern)
                took_octant |= any(e - s0 > 1 for s0, e in ent)
                want = [tuple(x) for x in runs[run_ptr[i]:run_ptr[i + 1]].tolist()]
                assert _merge(ent) == want
                assert len(ent) >= len(want)
                expanded = np.concatenate([np.arange(s0, e0) for s0, e0 in want]) if want else np.zeros(0, int)
                assert np.array_equal(np.sort(p.perm[expanded]), np.sort(bcols[brp[i]:brp[i + 1]]))
    assert took_octant


# ----------------------------------------------------------------------------- section 5.2 histogram
def test_locality_histogram_properties():
    """H_k(0) = N and sum_d H_k(d) = kN for distinct points (section 5.2)."""
    xyz = synth.uniform_cube(2000, 41)
    p = oracle.Pipeline(xyz, oracle.ENC_HILBERT, 32)
    k = 8
    idx, _ = p.tree.knn(xyz, k)
    nbr_pos = p.rank[idx.astype(np.int64)]
    h = oracle.locality_histogram(nbr_pos, p.rank, len(xyz))
    assert h[0] == len(xyz) and h.sum() == k * len(xyz)
    # storage order matters: the Hilbert order puts neighbours closer than the input order
    h_none = oracle.locality_histogram(idx.astype(np.int64), np.arange(len(xyz)), len(xyz))
    d = np.arange(len(xyz))
    assert (h * d).sum() < (h_none * d).sum()


def test_skewness_matches_library():
    """G1 of section 5.2 against scipy's biased sample skewness on the expanded sample."""
    stats = pytest.importorskip("scipy.stats")
    rng = synth.Rng(71)
    for t in range(4):
        h = rng.integers(t, 60, 50).astype(np.int64)
        d = np.repeat(np.arange(len(h)), h)
        assert abs(oracle.skewness(h) - stats.skew(d, bias=True)) < 1e-9


def test_skewness_closed_forms():
    """G1 of section 5.2 on a symmetric histogram (0), the two-point (Bernoulli) closed form
    (1 - 2q) / sqrt(q (1 - q)), q the share at d = 1, and a point mass (0); no library."""
    assert abs(oracle.skewness([1, 4, 6, 4, 1])) < 1e-12
    for a, b in ((1, 3), (2, 7), (5, 1)):
        q = b / (a + b)
        assert abs(oracle.skewness([a, b]) - (1 - 2 * q) / np.sqrt(q * (1 - q))) < 1e-12
    assert oracle.skewness([0, 0, 5]) == 0.0


def test_locality_subset_properties():
    """H_k of a subset: H_k(0) = centres, sum = k * centres; the curve orders are more
    left-heavy than the input order (section 5.2, Table 5)."""
    xyz = synth.lidar_tile(30000, 73, side=float(np.sqrt(3000.0)))
    p = oracle.Pipeline(xyz, oracle.ENC_HILBERT, 32)
    ids = np.arange(0, len(xyz), 100)
    g = {}
    for order in (oracle.ENC_NONE, oracle.ENC_MORTON, oracle.ENC_HILBERT):
        h, g[order] = p.locality(ids, 8, order)
        assert h[0] == len(ids) and h.sum() == 8 * len(ids)
    assert g[oracle.ENC_MORTON] > g[oracle.ENC_NONE] and g[oracle.ENC_HILBERT] > g[oracle.ENC_NONE]


# ----------------------------------------------------------------------------- section 7.5 memory model
def test_table7_overhead_arithmetic():
    for _, t_o, t_p, rho, omega in read_golden("table7_memory_overhead.txt"):
        w = (float(t_p) + float(rho) * float(t_o)) / 32.0 * 100.0
        assert abs(w - float(omega)) <= 0.0051

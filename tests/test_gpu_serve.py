"""The request server: every request's result is the same bytes whether it ran alone or in
a mix of concurrent, merged requests, and equals the oracle's; admission respects the
memory budget; a failing request does not stop the others."""
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


def _requests(n_req: int, seed: int, max_n: int):
    """Requests like the serving workload, smaller: LiDAR-like clouds of log-uniform size,
    all points or a 1 % subset as centres, sphere r or kNN k."""
    rng = synth.Rng(seed)
    u = rng.u01(0, n_req)
    sizes = np.exp(np.log(500) + u * (np.log(max_n) - np.log(500))).astype(np.int64)
    subset = rng.u01(1, n_req) < 0.5
    radius = rng.u01(2, n_req) < 0.5
    ri = rng.integers(3, n_req, 4)
    ki = rng.integers(4, n_req, 3)
    out = []
    for i in range(n_req):
        n = int(sizes[i])
        xyz = synth.lidar_tile(n, seed * 100 + i, side=float(np.sqrt(n / 10.0)))
        q = None
        if subset[i]:
            rows = np.sort(synth.Rng(seed * 100 + i).integers(9, max(1, n // 100), n))
            q = np.ascontiguousarray(xyz[rows])
        if radius[i]:
            spec = dict(search="radius", kernel=["sphere", "cube", "circle", "square"][i % 4],
                        r=[0.5, 1.0, 2.0, 3.0][int(ri[i])])
        else:
            spec = dict(search="knn", k=[8, 16, 32][int(ki[i])])
        out.append((xyz, q, spec))
    return out


def _run(server: sfc.Server, reqs, one_at_a_time: bool):
    results, ids = [], []
    if one_at_a_time:
        for xyz, q, spec in reqs:
            rid = server.submit(xyz, queries=q, **spec)
            assert server.wait(rid) == 0
            results.append(server.result(rid))
            server.release(rid)
        return results
    for xyz, q, spec in reqs:
        ids.append(server.submit(xyz, queries=q, **spec))
    for rid in ids:
        assert server.wait(rid) == 0
        results.append(server.result(rid))
    for rid in ids:
        server.release(rid)
    return results


def _equal(a: dict, b: dict, spec: dict):
    if spec["search"] == "radius":
        assert torch.equal(a["row_ptr"], b["row_ptr"]) and torch.equal(a["cols"], b["cols"])
    else:
        assert torch.equal(a["knn_idx"], b["knn_idx"])
        assert torch.equal(a["knn_d2"].view(torch.int32), b["knn_d2"].view(torch.int32))


def test_same_result_alone_and_in_the_mix():
    reqs = _requests(40, 31, 60_000)
    alone_srv = sfc.Server(slots=1, max_batch=1, batch_points=0)
    alone = _run(alone_srv, reqs, one_at_a_time=True)
    alone_srv.close()
    assert all(r["batched_with"] == 1 for r in alone)
    mix_srv = sfc.Server(slots=4, max_batch=16, batch_points=400_000)
    mixed = _run(mix_srv, reqs, one_at_a_time=False)  # a burst: queued, merged, overlapped
    mix_srv.close()
    assert max(r["batched_with"] for r in mixed) > 1  # some requests did share a pass
    for (xyz, q, spec), a, b in zip(reqs, alone, mixed):
        _equal(a, b, spec)


def test_results_match_the_oracle():
    reqs = _requests(12, 37, 20_000)
    srv = sfc.Server(slots=3, max_batch=8, batch_points=100_000)
    got = _run(srv, reqs, one_at_a_time=False)
    srv.close()
    for (xyz, q, spec), g in zip(reqs, got):
        p = oracle.Pipeline(xyz, oracle.ENC_HILBERT, 64)
        centres = xyz if q is None else q
        if spec["search"] == "radius":
            orp, ocols = p.tree.radius(centres, spec["r"], KERN[spec["kernel"]])
            assert np.array_equal(g["row_ptr"].cpu().numpy(), orp)
            assert np.array_equal(g["cols"].cpu().numpy(), p.rows_by_rank(orp, ocols))
        else:
            oidx, od2 = p.tree.knn(centres, spec["k"])
            assert np.array_equal(g["knn_idx"].cpu().numpy(), oidx)
            assert np.array_equal(g["knn_d2"].cpu().numpy().view(np.uint32), od2.view(np.uint32))


def test_budget_admits_one_at_a_time():
    """With a budget smaller than any request, each runs alone and only once the previous
    one's memory is released."""
    reqs = _requests(6, 41, 20_000)
    srv = sfc.Server(slots=4, max_batch=16, batch_points=1_000_000, hbm_budget=1)
    ids = [srv.submit(xyz, queries=q, **spec) for xyz, q, spec in reqs]
    for rid in ids:
        assert srv.wait(rid) == 0
        t = srv.timings(rid)
        assert t["batched_with"] == 1
        st = srv.stats()
        assert st["running"] == 0  # the next one waits for this one's release
        srv.release(rid)
    assert srv.stats()["reserved_bytes"] == 0
    srv.close()


def test_failed_request_in_a_merged_pass_fails_alone():
    """A non-finite cloud merged with good ones: the merged pass fails, its requests are
    answered one by one, and only the bad one reports the failure."""
    srv = sfc.Server(slots=1, max_batch=8, batch_points=1_000_000)
    blocker = srv.submit(synth.lidar_tile(4_000_000, 77), search="knn", k=32)  # holds the only slot
    bad = synth.uniform_cube(3000, 78)
    bad[5, 0] = np.nan
    goods = [synth.uniform_cube(3000, 79 + j) for j in range(3)]
    ids = [srv.submit(goods[0], search="knn", k=8), srv.submit(bad, search="knn", k=8),
           srv.submit(goods[1], search="radius", kernel="sphere", r=0.1),
           srv.submit(goods[2], search="knn", k=4)]
    assert srv.wait(blocker) == 0
    assert [srv.wait(i) for i in ids] == [0, 7, 0, 0]
    for i, (g, spec) in zip((ids[0], ids[2], ids[3]), zip((goods[0], goods[1], goods[2]),
                                                         (dict(k=8), dict(r=0.1), dict(k=4)))):
        res = srv.result(i)
        assert res["batched_with"] == 1 and res["rows"] == 3000
        if "k" in spec:
            oi, _ = oracle.knn_brute(g, g, spec["k"])
            assert np.array_equal(res["knn_idx"].cpu().numpy(), oi)
        else:
            orp, _ = oracle.radius_brute(g, g, spec["r"], oracle.SPHERE)
            assert np.array_equal(res["row_ptr"].cpu().numpy(), orp)
    for i in [blocker] + ids:
        srv.release(i)
    srv.close()


def test_failed_request_does_not_stop_the_server():
    srv = sfc.Server(slots=2)
    bad = synth.uniform_cube(1000, 5)
    bad[17, 2] = np.inf
    good = synth.uniform_cube(1000, 6)
    r_bad = srv.submit(bad, search="knn", k=4)
    r_good = srv.submit(good, search="radius", kernel="cube", r=0.1)
    assert srv.wait(r_bad) == 7  # SFC_ERR_NOT_FINITE
    assert srv.wait(r_good) == 0
    assert srv.result(r_good)["rows"] == 1000
    with pytest.raises(sfc.SFCError):
        srv.result(r_bad)
    srv.release(r_bad)
    srv.release(r_good)
    with pytest.raises(sfc.SFCError):
        srv.submit(good, search="knn", k=65)
    with pytest.raises(sfc.SFCError):
        srv.submit(good, search="radius", r=float("nan"))
    srv.close()


def test_real_size_requests_sampled_rows():
    """Requests of the serving workload's sizes (50k to 20M points, all points or a 1 %
    subset), sent as a burst: sampled rows of each equal the oracle's brute force."""
    sizes = (50_000, 2_000_000, 8_000_000, 20_000_000)
    specs = (dict(search="radius", kernel="sphere", r=2.0), dict(search="knn", k=16),
             dict(search="radius", kernel="sphere", r=1.0), dict(search="knn", k=32))
    reqs = []
    for j, (n, spec) in enumerate(zip(sizes, specs)):
        xyz = synth.lidar_tile(n, 900 + j)
        q = None
        if j % 2 == 1:  # a seeded 1 % subset of the points as centres
            q = np.ascontiguousarray(xyz[np.sort(synth.Rng(950 + j).integers(0, n // 100, n))])
        reqs.append((xyz, q, spec))
    srv = sfc.Server(slots=4)
    got = _run(srv, reqs, one_at_a_time=False)
    srv.close()
    for j, ((xyz, q, spec), g) in enumerate(zip(reqs, got)):
        centres = xyz if q is None else q
        rows = np.sort(synth.Rng(970 + j).integers(0, 10, len(centres))).astype(np.int64)
        if spec["search"] == "radius":
            orp, ocols = oracle.radius_brute(xyz, centres[rows], spec["r"], KERN[spec["kernel"]])
            rp = g["row_ptr"].cpu().numpy()
            for i, row in enumerate(rows):
                mine = np.sort(g["cols"][rp[row]:rp[row + 1]].cpu().numpy())
                assert np.array_equal(mine, np.sort(ocols[orp[i]:orp[i + 1]])), (j, int(row))
        else:
            oi, od = oracle.knn_brute(xyz, centres[rows], spec["k"])
            r = torch.as_tensor(rows, device="cuda")
            assert np.array_equal(g["knn_idx"][r].cpu().numpy(), oi), j
            assert np.array_equal(g["knn_d2"][r].cpu().numpy().view(np.uint32), od.view(np.uint32)), j

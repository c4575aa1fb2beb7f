"""Out-of-memory paths of every public call, made on the host: a test allocator registered
through sfc_set_allocator returns NULL for the n-th allocation of a call, for n = 1, 2, ...
until the call no longer allocates that many blocks.  Each failing call must report
SFC_ERR_OOM, give back every block it took (sfc_live_allocations returns to its value
before the call), and the same call with a working allocator must then give the oracle's
result bit for bit."""
import gc

import numpy as np
import pytest
import torch

import oracle
import paper_2603_06771_gb300 as sfc
import synth
from alloc_hooks import HookAllocator
from helpers import csr_rows_sorted_by_id

pytestmark = pytest.mark.gpu

R, K = 0.06, 8


@pytest.fixture(scope="module")
def setup():
    sfc.build()
    xyz = synth.uniform_cube(20_000, 61)
    q = synth.uniform_cube(700, 62)
    p = oracle.Pipeline(xyz, oracle.ENC_HILBERT, 32)
    want = {
        "radius": p.tree.radius(xyz, R, oracle.SPHERE),
        "radius_q": p.tree.radius(q, R, oracle.CUBE),
        "knn_q": p.tree.knn(q, K),
        "runs": p.radius_runs(xyz, R, oracle.SPHERE),
    }
    return xyz, q, want


def _check_csr(rp, cols, want):
    rp_h, cols_h = rp.cpu().numpy(), cols.cpu().numpy()
    assert np.array_equal(rp_h, want[0])
    assert np.array_equal(csr_rows_sorted_by_id(rp_h, cols_h), csr_rows_sorted_by_id(want[0], want[1]))


def _drive(hook, call, check):
    """Fail the 1st, 2nd, ... allocation of call(); returns how many allocations failed."""
    n = 1
    while True:
        gc.collect()
        torch.cuda.synchronize()
        live0 = sfc.live_allocations()
        hook.fail_nth_from_now(n)
        try:
            out = call()
        except sfc.SFCError as e:
            hook.fail_nth_from_now(None)
            assert e.status == 2, f"allocation {n}: {e}"  # SFC_ERR_OOM
            gc.collect()
            torch.cuda.synchronize()
            assert sfc.live_allocations() == live0, f"allocation {n}: blocks leaked"
            out = call()  # the allocator works again: the full, correct result
            check(out)
            del out
            n += 1
            continue
        hook.fail_nth_from_now(None)
        check(out)  # the call made fewer than n allocations
        del out
        gc.collect()
        torch.cuda.synchronize()
        return n - 1


def test_every_call_reports_oom_and_leaks_nothing(setup):
    xyz, q, want = setup
    pts = torch.from_numpy(xyz).cuda()
    qd = torch.from_numpy(q).cuda()
    hook = HookAllocator()
    hook.install()
    try:
        failed = {}
        failed["octree_build"] = _drive(hook, lambda: sfc.octree_build(pts, "hilbert", leaf_capacity=32),
                                        lambda t: t.free())
        tree = sfc.octree_build(pts, "hilbert", leaf_capacity=32)
        failed["radius_search"] = _drive(hook, lambda: sfc.radius_search_csr(tree, None, R, "sphere"),
                                         lambda o: _check_csr(o[0], o[1], want["radius"]))
        failed["radius_count+fill centres"] = _drive(
            hook, lambda: sfc.radius_search(tree, qd, R, "cube"), lambda o: _check_csr(o[0], o[1], want["radius_q"]))

        def check_runs(o):
            assert np.array_equal(o[0].cpu().numpy(), want["runs"][0])
            assert np.array_equal(o[1].cpu().numpy().reshape(-1), want["runs"][1].reshape(-1))
        failed["radius_search_ranges"] = _drive(hook, lambda: sfc.radius_search_ranges(tree, None, R, "sphere"),
                                                check_runs)

        def check_knn(o):
            assert np.array_equal(o[0].cpu().numpy(), want["knn_q"][0])
            assert o[1].cpu().numpy().tobytes() == want["knn_q"][1].tobytes()
        failed["knn centres"] = _drive(hook, lambda: sfc.knn(tree, qd, K), check_knn)

        def batch():
            return sfc.batch_search(torch.cat([pts, pts]), [dict(n=len(xyz), search="radius", kernel="sphere", r=R),
                                                           dict(n=len(xyz), search="knn", k=K)], "hilbert")

        def check_batch(b):
            rp, cols = b.radius(0)
            _check_csr(rp, cols, want["radius"])
            b.free()
        failed["batch_search"] = _drive(hook, batch, check_batch)
        tree.free()
        del tree
        # every call above allocates, so each saw at least one failure
        assert all(v >= 1 for v in failed.values()), failed
    finally:
        hook.uninstall()


def test_server_request_reports_oom_and_the_next_one_runs(setup):
    xyz, q, want = setup
    hook = HookAllocator()
    hook.install()
    srv = sfc.Server(slots=1)
    try:
        n = 1
        while True:
            gc.collect()
            torch.cuda.synchronize()
            live0 = sfc.live_allocations()
            hook.fail_nth_from_now(n)
            rid = srv.submit(xyz, search="knn", k=K, queries=q)
            st = srv.wait(rid)
            hook.fail_nth_from_now(None)
            if st == 0:
                res = srv.result(rid)
                assert np.array_equal(res["knn_idx"].cpu().numpy(), want["knn_q"][0])
                srv.release(rid)
                break
            assert st == 2, st  # SFC_ERR_OOM, reported by server_wait
            srv.release(rid)
            torch.cuda.synchronize()
            assert sfc.live_allocations() == live0
            rid = srv.submit(xyz, search="knn", k=K, queries=q)
            assert srv.wait(rid) == 0
            res = srv.result(rid)
            assert np.array_equal(res["knn_idx"].cpu().numpy(), want["knn_q"][0])
            assert res["knn_d2"].cpu().numpy().tobytes() == want["knn_q"][1].tobytes()
            srv.release(rid)
            n += 1
        assert n > 1
    finally:
        srv.close()
        hook.uninstall()

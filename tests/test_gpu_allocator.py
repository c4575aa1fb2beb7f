"""The allocator hook: with torch's caching allocator registered, every device allocation
of the library comes from torch (its allocated bytes grow while octrees and outputs are
alive), results are the same bytes as with the stream-ordered allocator, and the hook can
be changed only while no library allocation is alive."""
import gc

import numpy as np
import pytest
import torch

import paper_2603_06771_gb300 as sfc
import synth

pytestmark = pytest.mark.gpu


def _work(pts):
    t = sfc.octree_build(pts, "hilbert", leaf_capacity=32)
    rp, cols = sfc.radius_search_csr(t, None, 0.05, "sphere")  # library-allocated CSR
    idx, d2 = sfc.knn(t, None, 8)
    b = sfc.batch_search(torch.cat([pts, pts[:5000]]), [dict(n=pts.shape[0], search="knn", k=4),
                                                       dict(n=5000, search="radius", kernel="cube", r=0.1)],
                         "hilbert")
    out = (rp.clone(), cols.clone(), idx.clone(), d2.clone(), b.knn(0)[0].clone(), b.radius(1)[1].clone())
    return t, (rp, cols), b, out


def test_torch_allocator_serves_the_library():
    sfc.build()
    gc.collect()
    torch.cuda.synchronize()
    assert sfc.live_allocations() == 0, "library objects from earlier tests are still alive"
    pts = torch.from_numpy(synth.uniform_cube(60_000, 11)).cuda()
    t, csr, b, plain = _work(pts)
    with pytest.raises(sfc.SFCError):  # allocations are alive: the hook may not change
        sfc.use_torch_allocator(True)
    t.free()
    b.free()
    del csr
    gc.collect()
    torch.cuda.synchronize()
    assert sfc.live_allocations() == 0
    sfc.use_torch_allocator(True)
    try:
        before = torch.cuda.memory_allocated()
        t, csr, b, hooked = _work(pts)
        assert sfc.live_allocations() > 0
        assert torch.cuda.memory_allocated() > before  # the octree, the CSR and the batch live in torch's pool
        for a, h in zip(plain, hooked):
            assert torch.equal(a.view(torch.int32) if a.dtype == torch.float32 else a,
                               h.view(torch.int32) if h.dtype == torch.float32 else h)
        plan = sfc.BatchPlan([dict(n=pts.shape[0], search="knn", k=4)], "hilbert")
        plan.points.copy_(pts)
        plan.run()
        assert torch.equal(plan.knn(0)[0], plain[4])
        plan.free()
        t.free()
        b.free()
        del csr
        gc.collect()
        torch.cuda.synchronize()
        assert sfc.live_allocations() == 0
    finally:
        gc.collect()
        torch.cuda.synchronize()
        sfc.use_torch_allocator(False)

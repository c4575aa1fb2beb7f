"""radius_count_static: the count pass for callers that cannot let the library allocate
device memory (for example an application that reserves its whole device budget up
front, or a loop with a hard latency budget).  It must give exactly what radius_count
gives, on consecutive calls that share its static scratch, and must not call the device
allocator at all: a counting allocator registered through sfc_set_allocator sees no
allocate and no free call during it, and the device's stream-ordered pool does not grow.
Collected last on purpose."""
import ctypes
import gc

import pytest
import torch

import paper_2603_06771_gb300 as sfc
import synth
from alloc_hooks import HookAllocator

pytestmark = pytest.mark.gpu


def _used_pool_bytes():
    """Bytes in use in the current device's default stream-ordered pool, or None."""
    for name in ("libcudart.so", "libcudart.so.13", "libcudart.so.12"):
        try:
            rt = ctypes.CDLL(name)
            break
        except OSError:
            rt = None
    if rt is None:
        return None
    pool = ctypes.c_void_p()
    if rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) != 0:
        return None
    used = ctypes.c_uint64()
    attr_used_mem_current = 7
    if rt.cudaMemPoolGetAttribute(pool, attr_used_mem_current, ctypes.byref(used)) != 0:
        return None
    return used.value


def _count_static(tree, r, kernel):
    lib = sfc.binding.lib()
    row_ptr = torch.empty(tree.n + 1, dtype=torch.int64, device="cuda")
    nnz = ctypes.c_int64(-1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.radius_count_static(tree.handle, ctypes.c_float(r), sfc.KERNELS[kernel], stream,
                                 ctypes.c_void_p(row_ptr.data_ptr()), ctypes.byref(nnz))
    return st, row_ptr, nnz.value


def test_static_count_matches_radius_count():
    sfc.build()
    hook = HookAllocator()
    hook.install()  # every library allocation from here on is counted
    try:
        trees = [
            (sfc.octree_build(torch.from_numpy(synth.lidar_tile(300_000, 11)).cuda(), "hilbert", leaf_capacity=32),
             2.0, "sphere"),
            (sfc.octree_build(torch.from_numpy(synth.uniform_cube(70_001, 12)).cuda(), "morton", leaf_capacity=16),
             0.05, "cube"),
            # the unordered cloud: every centre walks on its own (the per-lane kernels)
            (sfc.octree_build(torch.from_numpy(synth.uniform_cube(40_003, 14)).cuda(), "none", leaf_capacity=32),
             0.06, "circle"),
        ]
        torch.cuda.synchronize()
        # calls in a row on the shared scratch: the largest tree first, then smaller ones
        for tree, r, kern in trees:
            want_rp, want_nnz = sfc.radius_count(tree, None, r, kern)
            torch.cuda.synchronize()
            before_pool = _used_pool_bytes()
            before = hook.calls()
            st, got_rp, got_nnz = _count_static(tree, r, kern)
            torch.cuda.synchronize()
            assert hook.calls() == before, "radius_count_static called the device allocator"
            after_pool = _used_pool_bytes()
            assert st == 0
            assert got_nnz == want_nnz
            assert torch.equal(got_rp, want_rp)
            if before_pool is not None and after_pool is not None:
                assert after_pool == before_pool
            # the filled rows agree with the rows of the allocating path
            cols = sfc.radius_fill(tree, None, r, kern, got_rp, got_nnz)
            _, want_cols = sfc.radius_search(tree, None, r, kern)
            assert torch.equal(cols, want_cols)
        for tree, _, _ in trees:
            tree.free()
        del trees
    finally:
        hook.uninstall()


def test_static_count_rejects_large_clouds():
    lib = sfc.binding.lib()
    cap = lib.radius_count_static_max_points()
    assert cap == 1 << 21
    big = sfc.octree_build(torch.from_numpy(synth.uniform_cube(cap + 1, 13)).cuda(), "hilbert")
    st, _, _ = _count_static(big, 0.01, "sphere")
    assert st == 5  # SFC_ERR_TOO_LARGE
    big.free()
    gc.collect()

"""A test allocator for the library's allocator hook (sfc_set_allocator): it serves every
block from torch's caching allocator, counts the allocate and free calls, and can be told
to fail one allocation (return NULL), so the library's out-of-memory paths run without
exhausting the device."""
from __future__ import annotations

import ctypes as C
import gc
import threading

import torch

import paper_2603_06771_gb300 as sfc


class HookAllocator:
    def __init__(self):
        self._lock = threading.Lock()
        self.allocs = 0
        self.frees = 0
        self.failed = 0
        self._fail_at = None
        self._a = sfc.binding._ALLOC_FN(self._alloc)  # kept alive while installed
        self._f = sfc.binding._FREE_FN(self._free)
        self._device = torch.cuda.current_device()

    def _alloc(self, nbytes, ctx, stream):
        with self._lock:
            self.allocs += 1
            if self._fail_at is not None and self.allocs == self._fail_at:
                self.failed += 1
                return None
        s = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream(self._device)
        return torch.cuda.caching_allocator_alloc(int(nbytes), device=self._device, stream=s)

    def _free(self, ptr, ctx, stream):
        with self._lock:
            self.frees += 1
        torch.cuda.caching_allocator_delete(ptr)

    def fail_nth_from_now(self, n: int | None):
        """Make the n-th allocation from now (1 = the next one) fail; None: none fails."""
        with self._lock:
            self._fail_at = None if n is None else self.allocs + int(n)

    def calls(self) -> tuple[int, int]:
        with self._lock:
            return self.allocs, self.frees

    def install(self):
        gc.collect()
        torch.cuda.synchronize()
        st = sfc.binding.lib().sfc_set_allocator(C.cast(self._a, C.c_void_p), C.cast(self._f, C.c_void_p), None)
        if st != 0:
            raise RuntimeError(f"sfc_set_allocator refused the hook (status {st}, live allocations "
                               f"{sfc.live_allocations()})")

    def uninstall(self):
        gc.collect()
        torch.cuda.synchronize()
        st = sfc.binding.lib().sfc_set_allocator(None, None, None)
        if st != 0:
            raise RuntimeError(f"sfc_set_allocator(NULL) failed (status {st}, live allocations "
                               f"{sfc.live_allocations()})")

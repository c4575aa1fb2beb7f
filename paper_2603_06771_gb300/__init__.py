"""GB300-native space-filling-curve linear-octree neighbour search (arXiv 2603.06771).

The compute path is the CUDA library ``libsfcoct.so`` (sources in ``csrc/``, C ABI in
``include/sfcoct.h``); this package builds it (:mod:`.build`) and binds it with ctypes
(:mod:`.binding`).  See ``octree_build``, ``radius_search`` and ``knn``; many clouds at once
with ``batch_search``, ``BatchPlan`` (a recorded CUDA graph) and ``batch_autotune``; requests
arriving over time with ``Server``.
"""
from .binding import (ENCODINGS, KERNELS, Batch, BatchPlan, Octree, Server, SFCError, batch_autotune,
                      batch_search, choose_encoding, encode_cells, knn, knn_locality, launch_count, library_path,
                      live_allocations, octree_build, profile_enable, profile_read, radius_count, radius_fill,
                      radius_search, radius_search_csr, radius_search_ranges, search_stats, stats_enable, stats_read,
                      use_torch_allocator)
from .build import build

__all__ = ["ENCODINGS", "KERNELS", "Batch", "BatchPlan", "Octree", "Server", "SFCError", "batch_autotune",
           "batch_search", "build", "choose_encoding", "encode_cells", "knn", "knn_locality", "launch_count",
           "library_path", "live_allocations", "octree_build", "profile_enable", "profile_read", "radius_count",
           "radius_fill", "radius_search", "radius_search_csr", "radius_search_ranges", "search_stats", "stats_enable",
           "stats_read", "use_torch_allocator"]

/*
 * sfcoct.h - C ABI of the GB300 space-filling-curve linear-octree neighbour search.
 *
 * The library implements, on one CUDA device, the data-parallel path of the method of
 * "Efficient Neighbourhood Search in 3D Point Clouds Through Space-Filling Curves and
 * Linear Octrees" (arXiv 2603.06771):
 *   encode every point with a 63-bit Morton or Hilbert code (section 4, 4.1, 4.2),
 *   reorder the cloud by code (section 4), build the linear octree over the sorted codes
 *   (section 5.1: leaves, counts, internal nodes, internalRanges), then answer all-points
 *   or arbitrary-centre fixed-radius searches with the four kernels of section 3.2
 *   (neighboursPrune / neighboursLin of section 5.1) and kNN searches (section 3.3).
 *
 * Conventions shared by every call:
 *   - Points and centres are float32 xyz triples stored contiguously (array of n x 3
 *     floats, "AoS").  Pointers marked "device" must be CUDA device (or managed) memory
 *     of the current device; a host pointer gives SFC_ERR_NOT_DEVICE_PTR.  There is no
 *     CPU fallback.
 *   - Every call is asynchronous on cuda_stream (a cudaStream_t; NULL = legacy default
 *     stream) unless its comment names a synchronisation.
 *   - Indices returned to the caller (neighbour ids, kNN ids) are positions in the
 *     caller's original point array, so results do not depend on the encoding.
 *   - Errors are returned as sfc_status; no exception crosses the ABI.  After
 *     SFC_ERR_CUDA, sfc_last_error() gives the CUDA message of the calling thread.
 *   - Sizes: 0 <= n <= 2^31 - 1 points; the node table must fit int32 indices.
 */
#ifndef SFCOCT_H
#define SFCOCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sfc_octree_s* sfc_octree; /* opaque handle, owned by the library */

/* Ordering of the cloud (section 4).  SFC_ENC_NONE keeps the cloud in input order: the
 * octree is still built over Morton codes (a linear octree needs sorted codes, section
 * 7.1), but the coordinates are not gathered and the searches read them through the
 * permutation, and all-points queries run in input order. */
typedef enum { SFC_ENC_NONE = 0, SFC_ENC_MORTON = 1, SFC_ENC_HILBERT = 2 } sfc_encoding;

/* Search kernels, section 3.2 (Definition), all with the strict "<":
 *   SPHERE ||p - c||_2 < r;  CIRCLE ||(p - c)_xy||_2 < r;
 *   CUBE ||p - c||_inf < r;  SQUARE ||(p - c)_xy||_inf < r. */
typedef enum { SFC_SPHERE = 0, SFC_CIRCLE = 1, SFC_CUBE = 2, SFC_SQUARE = 3 } sfc_kernel;

typedef enum {
    SFC_OK = 0,
    SFC_ERR_INVALID = 1,         /* bad argument: n < 0, k < 1, NaN radius, bad enum, ... */
    SFC_ERR_OOM = 2,             /* a device allocation failed */
    SFC_ERR_CUDA = 3,            /* a CUDA call failed; see sfc_last_error() */
    SFC_ERR_TIMEOUT = 4,         /* a bounded wait gave up: a tile of the sort or of a scan
                                    waiting for the counts of earlier tiles (never expected;
                                    the results are then wrong), or server_wait's timeout */
    SFC_ERR_TOO_LARGE = 5,       /* a size limit of this library is exceeded */
    SFC_ERR_NOT_DEVICE_PTR = 6,  /* a pointer that must be device memory is not */
    SFC_ERR_NOT_FINITE = 7,      /* a coordinate, or the cloud's extent, is NaN or infinite */
    SFC_ERR_INTERNAL = 8         /* a device-side consistency guard tripped (a library bug) */
} sfc_status;

/* Build options.  leaf_capacity is N_max of sections 3.1 and 5.1 (a leaf above level 21
 * holds at most N_max points); prune selects neighboursPrune (1: an octant that lies
 * inside the kernel is taken whole, step 1a of section 5.1) or neighboursLin (0: every
 * candidate point is tested).  Both give identical results. */
typedef struct {
    int32_t leaf_capacity; /* >= 1, default 32 */
    int32_t prune;         /* 0 or 1, default 1 */
} sfc_build_opts;

/* Compressed sparse rows: row q holds the neighbours of centre q in
 * cols[row_ptr[q] .. row_ptr[q + 1]), listed in ascending position along the curve
 * (ascending sorted position of the tree points).  Device memory. */
typedef struct {
    int64_t n_rows;
    int64_t nnz;
    int64_t* row_ptr; /* n_rows + 1 entries */
    int32_t* cols;    /* nnz entries, original point indices */
} sfc_csr;

typedef struct {
    int64_t n_points;
    int64_t n_leaves;   /* 7 * n_internal + 1 (complete octree) */
    int64_t n_internal;
    int64_t n_nodes;    /* n_internal + n_leaves */
    int32_t encoding;
    int32_t leaf_capacity;
    int32_t prune;
    int32_t device;
    float lo[3];        /* lower corner of the bounding box (section 4, step 1) */
    float scale;        /* 2^21 / largest extent, binary32 (section 4, step 1) */
} sfc_octree_info;

/* Fills *opts with the defaults (leaf_capacity 32, prune 1). */
sfc_status sfc_build_opts_default(sfc_build_opts* opts);

/* Build the octree of n points (sections 4 and 5.1).
 *   points_xyz  device, n x 3 float32, read only; the library copies what it keeps, so the
 *               caller may free it once the stream has passed this call.
 *   n           number of points, 0 <= n <= 2^31 - 1 (n = 0 gives an empty tree).
 *   enc         SFC_ENC_NONE / MORTON / HILBERT.
 *   opts        NULL for the defaults.
 *   out         receives the handle; release it with octree_free.
 * Steps on the device: bounding box and scale, 63-bit codes (bit 63 is 0), stable LSD
 * radix sort of (code, index), gather of the sorted cloud, leaves/counts, internal nodes,
 * internalRanges and a tight bounding box per node.
 * Synchronises cuda_stream once (to size the node table).  Returns SFC_ERR_NOT_FINITE if a
 * coordinate is NaN or infinite or the extent overflows binary32. */
sfc_status octree_build(const float* points_xyz, int64_t n, sfc_encoding enc, const sfc_build_opts* opts,
                        void* cuda_stream, sfc_octree* out);

/* Release the handle; its device memory is freed in stream order on cuda_stream.  Work
 * that uses the handle on other streams must be complete or ordered before that stream. */
sfc_status octree_free(sfc_octree h, void* cuda_stream);

/* Sizes and parameters of a built octree (host struct, no synchronisation). */
sfc_status octree_info(sfc_octree h, sfc_octree_info* info);

/* Fixed-radius search (section 3.2 kernels; section 5.1 neighboursPrune / neighboursLin).
 *   queries_xyz  device, n_queries x 3 float32 centres; any finite position, inside the
 *                cloud's box or not.  NULL = every point of the tree, in the caller's
 *                original order (then n_queries must be 0 or the number of points).
 *   r            radius (for CUBE / SQUARE the half side); r <= 0 gives empty rows, a
 *                NaN r gives SFC_ERR_INVALID.
 *   out          receives a CSR whose two arrays the library allocates in stream order
 *                on cuda_stream (its allocator: see sfc_set_allocator); release it with
 *                sfc_csr_free.
 * Row q lists every tree point p with kernel(p, centre q, r) true, the centre itself
 * included when it is a tree point.  Synchronises cuda_stream (to read nnz, then the
 * device guard word). */
sfc_status radius_search(sfc_octree h, const float* queries_xyz, int64_t n_queries, float r, sfc_kernel kern,
                         void* cuda_stream, sfc_csr* out);

/* The two halves of radius_search for callers that allocate the output themselves.
 * radius_count writes row_ptr (device, n_rows + 1 int64, caller-owned) and *nnz (host);
 * it synchronises cuda_stream once.  radius_fill then writes cols (device, *nnz int32,
 * caller-owned) given the same queries, r and kernel and that row_ptr. */
sfc_status radius_count(sfc_octree h, const float* queries_xyz, int64_t n_queries, float r, sfc_kernel kern,
                        void* cuda_stream, int64_t* row_ptr, int64_t* nnz);
sfc_status radius_fill(sfc_octree h, const float* queries_xyz, int64_t n_queries, float r, sfc_kernel kern,
                       void* cuda_stream, const int64_t* row_ptr, int32_t* cols);

/* radius_count for every point of the tree (queries_xyz == NULL) without allocating any
 * device memory.  The paper has no counterpart: this exists for callers that cannot let a
 * library allocate, such as an application that reserves its whole device memory budget
 * up front (an allocation inside the call could fail or disturb its pool) or a loop with a
 * hard latency budget.  The per-point counts and the scan's per-tile words live in a
 * file-scope __device__ array of the library (about 8 MiB, held by every GPU that loads the
 * library until the process exits) instead of device scratch; each call clears the words
 * that must start at zero.
 *   row_ptr  device, n_points + 1 int64, caller-owned; *nnz (host) receives the total.
 *   Same results as radius_count(h, NULL, 0, r, kern, ...).
 * Limits: at most radius_count_static_max_points() points (2^21), else SFC_ERR_TOO_LARGE.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  Every call uses the same array and it
 * keeps the last call's contents, so calls that overlap on the GPU race with each other.
 * Synchronises cuda_stream once (to read nnz). */
sfc_status radius_count_static(sfc_octree h, float r, sfc_kernel kern, void* cuda_stream, int64_t* row_ptr,
                               int64_t* nnz);
/* The largest point count radius_count_static accepts. */
int64_t radius_count_static_max_points(void);

/* Free a CSR allocated by radius_search (stream ordered); zeroes *csr. */
sfc_status sfc_csr_free(sfc_csr* csr, void* cuda_stream);

/* Range output of a fixed-radius search (neighboursStruct, section 5.1): row i lists its
 * neighbours as runs of consecutive positions of the octree's sorted cloud, [start, end),
 * in ascending order and maximal (two runs of a row never touch).  Position p is original
 * point perm[p] (octree_export).  The paper's form lists each wholly contained octant as
 * one range and each other neighbour alone; the maximal runs merge adjacent entries of
 * that list, so they are never more, and they depend on the neighbour set only. */
typedef struct {
    int64_t n_rows;
    int64_t n_runs;
    int64_t* run_ptr; /* device, n_rows + 1: row i's runs are run_ptr[i] .. run_ptr[i + 1] - 1 */
    int32_t* runs;    /* device, 2 * n_runs int32: start, end of every run */
} sfc_ranges;

/* radius_search with the range output; same arguments, centres and errors.  Allocates the
 * output (release with sfc_ranges_free); synchronises cuda_stream as radius_search. */
sfc_status radius_search_ranges(sfc_octree h, const float* queries_xyz, int64_t n_queries, float r, sfc_kernel kern,
                                void* cuda_stream, sfc_ranges* out);
/* Free (in stream order on cuda_stream) the two arrays of a range output and clear *ranges;
 * SFC_ERR_INVALID for ranges == NULL. */
sfc_status sfc_ranges_free(sfc_ranges* ranges, void* cuda_stream);

/* k nearest neighbours (section 3.3) under the squared Euclidean distance in binary32,
 * d2 = (dx*dx + dy*dy) + dz*dz with d = p - c, each operation rounded to nearest.
 *   queries_xyz  as for radius_search (NULL = all tree points, original order).
 *   k            1 <= k <= 64.
 *   out_idx      device, n_rows x k int32, caller-owned: original point indices.
 *   out_d2       device, n_rows x k float32, caller-owned.
 * Row q is sorted by (d2, index) ascending, so equal distances go to the smaller index;
 * when k exceeds the number of points the row is padded with index -1 and d2 = +inf.
 * With queries_xyz == NULL the call does not synchronise; with caller centres it
 * synchronises once to report non-finite centres (SFC_ERR_NOT_FINITE). */
sfc_status knn(sfc_octree h, const float* queries_xyz, int64_t n_queries, int32_t k, void* cuda_stream,
               int32_t* out_idx, float* out_d2);

/* ---- batched path: many clouds in one pass ------------------------------------------- */

/* What to search in one cloud of a batch: every point of the cloud is a centre. */
typedef enum { SFC_SEARCH_RADIUS = 0, SFC_SEARCH_KNN = 1 } sfc_search_kind;

typedef struct {
    int64_t n_points; /* points of this cloud; the clouds are concatenated in the input */
    int32_t search;   /* sfc_search_kind */
    int32_t kernel;   /* SFC_SEARCH_RADIUS: sfc_kernel */
    float r;          /* SFC_SEARCH_RADIUS: radius (r <= 0 gives empty rows) */
    int32_t k;        /* SFC_SEARCH_KNN: neighbours, 1 <= k <= 64 */
    int32_t leaf_capacity; /* this cloud's leaf capacity; 0 = opts->leaf_capacity */
    int32_t knn_window;    /* SFC_SEARCH_KNN: curve neighbours per side that seed each list,
                              0..64 (0 = max(8, k), the default of knn()); a speed knob only
                              (a window wider than the list size class allows is not used) */
    int32_t queries_per_warp; /* centres one warp walks the octree for together: 8, 16 or 32
                                 (0 = 32); fewer centres give each walk a tighter box but
                                 leave lanes idle; a speed knob only */
    int32_t record_slots;  /* SFC_SEARCH_RADIUS: hit-mask records kept per warp group from the
                              count pass for the fill (the staging depth of the two passes),
                              1..128 (0 = 32); a group with more leaf chunks than slots walks
                              the tree again in the fill.  Clouds of one kernel type share the
                              largest value among them.  A speed and memory knob only */
} sfc_batch_cloud;

typedef struct sfc_batch_s* sfc_batch; /* results of a batch, owned by the library */

/* Build the linear octree of every cloud of a batch and run every cloud's all-points
 * search, with the same results as octree_build + radius_search / knn on each cloud alone.
 *   points_xyz  device, sum(n_points) x 3 float32: cloud 0's points, then cloud 1's, ...
 *   clouds      host array of n_clouds entries (1 <= n_clouds <= 1024).
 *   enc         SFC_ENC_MORTON or SFC_ENC_HILBERT; opts: NULL for the defaults.
 * Every step runs once over the whole batch (per-cloud bounding boxes and codes, one radix
 * sort ordered by (cloud, code), segmented linear-octree kernels, one search launch per
 * kernel type or kNN size class), so the launch count does not grow with the number of
 * clouds.  Each cloud gets the pipeline of sections 4 and 5 with its own bounding box,
 * scale and root; the paper itself processes one cloud per call.  Waits on cuda_stream
 * three times (node counts, radius output size, the end).  Neighbour indices are
 * positions inside each cloud.
 * Errors (then *out = NULL and nothing is held): SFC_ERR_INVALID for a bad argument or
 * cloud entry (negative n_points, unknown search or kernel, NaN r, k < 1, other
 * encodings); SFC_ERR_TOO_LARGE for n_clouds > 1024, k > 64, 2^31 - 1 points or more, or
 * node tables beyond 2^31 entries; SFC_ERR_NOT_DEVICE_PTR; SFC_ERR_NOT_FINITE when any
 * cloud holds a non-finite coordinate; SFC_ERR_OOM / SFC_ERR_CUDA; SFC_ERR_INTERNAL when
 * a device guard tripped. */
sfc_status batch_search(const float* points_xyz, const sfc_batch_cloud* clouds, int32_t n_clouds, sfc_encoding enc,
                        const sfc_build_opts* opts, void* cuda_stream, sfc_batch* out);

/* Device views of one cloud's results (no copy, valid until batch_free):
 *   radius cloud: the cloud's own CSR: row_ptr has n_points + 1 entries, row_ptr[0] == 0,
 *                 and row i is cols[row_ptr[i] .. row_ptr[i + 1]); *nnz = row_ptr[n_points];
 *                 knn pointers are NULL.
 *   kNN cloud:    knn_idx / knn_d2 hold n_points x k entries (layout of knn()); the CSR
 *                 pointers are NULL and *nnz = 0. */
sfc_status batch_cloud_result(sfc_batch b, int32_t cloud, const int64_t** row_ptr, const int32_t** cols,
                              int64_t* nnz, const int32_t** knn_idx, const float** knn_d2);

/* Release a batch's results (stream ordered on cuda_stream). */
sfc_status batch_free(sfc_batch b, void* cuda_stream);

/* Choose every cloud's speed knobs for this batch by timing it on the device: leaf
 * capacity, seeding window (kNN), centres per warp walk and record slots (radius).  The
 * build is timed whole and every launch set (radius kernel type: count + fill; kNN list
 * size 8/16/32/64) on its own with CUDA events.  First one pass per candidate leaf
 * capacity (after one untimed warm pass): each set takes the capacity minimising its
 * search time plus its points' share of the build time.  Then, at those capacities, one
 * pass per candidate window picks each kNN set's window, one pass per candidate
 * centres-per-warp value picks each set's, and one pass per candidate record-slot count
 * picks each radius set's.  An empty candidate list keeps the cloud's own value (or the
 * default).  Writes tuned_out[n_clouds]: the clouds with the chosen leaf_capacity,
 * knn_window (0 for radius clouds), queries_per_warp and record_slots (0 for kNN clouds),
 * ready for batch_search.  Results of a batch depend on none of these knobs.  The paper has
 * no counterpart (it fixes N_max per run and serves one centre per thread).  Errors as
 * batch_search, plus SFC_ERR_INVALID for a leaf candidate < 1, a window outside 1..64, a
 * centres-per-warp value other than 8, 16 or 32, or a record-slot count outside 1..128.
 * Synchronises cuda_stream repeatedly. */
sfc_status batch_autotune(const float* points_xyz, const sfc_batch_cloud* clouds, int32_t n_clouds, sfc_encoding enc,
                          const sfc_build_opts* opts, const int32_t* leaf_candidates, int32_t n_leaf,
                          const int32_t* window_candidates, int32_t n_window, const int32_t* qpw_candidates,
                          int32_t n_qpw, const int32_t* slot_candidates, int32_t n_slot, void* cuda_stream,
                          sfc_batch_cloud* tuned_out);

/* ---- batch plans: the batched pass recorded once as a CUDA graph and replayed --------- */

typedef struct sfc_batch_plan_s* sfc_batch_plan; /* owned by the library */

/* Record the batched pass of batch_search for a fixed list of clouds (sizes and searches)
 * as one CUDA graph over buffers allocated here, once: the input points, every work
 * array, the node tables (sized by a bound on the internal nodes: the internal nodes of
 * one level hold disjoint sets of more than leaf_capacity points), hit-mask records and
 * the outputs (radius output: nnz_capacity entries, 0 = 64 per radius centre).
 * A run is then one graph launch with no allocation and no host wait; sizes the device
 * learns (node counts, radius output size) are checked on the device, and a run that
 * outgrows a capacity skips its searches and is repaired by batch_plan_finish.  Same
 * arguments, results and errors as batch_search, plus SFC_ERR_INVALID when the clouds
 * hold no point.  Synchronises cuda_stream once. */
sfc_status batch_plan_create(const sfc_batch_cloud* clouds, int32_t n_clouds, sfc_encoding enc,
                             const sfc_build_opts* opts, int64_t nnz_capacity, void* cuda_stream,
                             sfc_batch_plan* out);

/* The plan's input: device, sum(n_points) x 3 float32, cloud after cloud.  The caller
 * writes the points there (stream ordered before batch_plan_launch). */
sfc_status batch_plan_points(sfc_batch_plan p, float** points_xyz);

/* Launch one run on cuda_stream (asynchronous; the results of an earlier run are
 * overwritten).  Each run must be followed by batch_plan_finish before the next. */
sfc_status batch_plan_launch(sfc_batch_plan p, void* cuda_stream);

/* Wait for the run and check it.  A radius output larger than its capacity is grown to
 * the exact size and the fill runs again; node tables that did not fit are regrown and the
 * run repeated (the graph is recorded again before the next launch in both cases).
 * Errors: SFC_ERR_INVALID without a launch, SFC_ERR_NOT_FINITE, SFC_ERR_TOO_LARGE,
 * SFC_ERR_OOM / SFC_ERR_CUDA, SFC_ERR_INTERNAL (a device guard tripped). */
sfc_status batch_plan_finish(sfc_batch_plan p, void* cuda_stream);

/* Views of one cloud's results after batch_plan_finish, as batch_cloud_result; valid until
 * the next launch or batch_plan_free. */
sfc_status batch_plan_result(sfc_batch_plan p, int32_t cloud, const int64_t** row_ptr, const int32_t** cols,
                             int64_t* nnz, const int32_t** knn_idx, const float** knn_d2);

/* Release the plan (waits for cuda_stream first). */
sfc_status batch_plan_free(sfc_batch_plan p, void* cuda_stream);

/* ---- section 5.2: kNN locality histogram ------------------------------------------ */

/* H_k and its skewness for a set of centres (cloud points, by original index; a 1 % subset
 * estimates the whole cloud's): the centres' k nearest neighbours come from this octree's
 * search; `order` gives every point a storage position (SFC_ENC_NONE: its original index;
 * SFC_ENC_MORTON / SFC_ENC_HILBERT: its rank in the stable order of that curve's codes
 * under this octree's discretisation, equal codes by original index); H_k(d) counts the
 * (centre, neighbour) pairs whose positions are d apart.
 *   hist  device, n_points uint64 (H_k(0 .. n - 1)), or NULL for G1 only.
 *   g1    host: the Fisher-Pearson skewness E[((d - mu) / sigma)^3] of that distribution
 *         (float64, mean first, then central moments); 0 when sigma = 0.
 * Neighbour slots padded for k > n are skipped.  Errors: SFC_ERR_INVALID (bad argument or
 * a centre id outside the cloud), SFC_ERR_TOO_LARGE (k > 64), SFC_ERR_NOT_DEVICE_PTR.
 * Synchronises cuda_stream. */
sfc_status knn_locality(sfc_octree h, const int32_t* centre_ids, int64_t n_centres, int32_t k, sfc_encoding order,
                        void* cuda_stream, uint64_t* hist, double* g1);

/* The storage order with the largest G1 for these centres (the paper's selection rule:
 * the most left-heavy histogram), among input order, Morton and Hilbert; g1_by_order
 * (host, 3 doubles, may be NULL) receives G1 for NONE, MORTON, HILBERT. */
sfc_status choose_encoding(sfc_octree h, const int32_t* centre_ids, int64_t n_centres, int32_t k, void* cuda_stream,
                           sfc_encoding* best, double* g1_by_order);

/* ---- serving: requests that arrive at any time ------------------------------------ */

typedef struct sfc_server_s* sfc_server; /* owned by the library */

typedef struct {
    int32_t slots;         /* requests (or merged groups) on the device at once, 1..16; one
                              worker thread and one CUDA stream each */
    int32_t max_batch;     /* all-points requests merged into one batched pass, 1..1024 */
    int64_t batch_points;  /* merge all-points requests of at most this many points, and at
                              most this many points per merged pass (0: never merge) */
    int64_t hbm_budget;    /* bytes: a request is admitted while the admitted, unreleased ones
                              plus its estimate stay within this (one larger than the whole
                              budget runs alone) */
    sfc_encoding enc;      /* SFC_ENC_MORTON or SFC_ENC_HILBERT */
    int32_t leaf_capacity;
} sfc_server_opts;

typedef struct {
    const float* points_xyz;  /* host, n_points x 3 float32; read until the request finishes */
    int64_t n_points;
    const float* queries_xyz; /* host, n_queries x 3, or NULL: every point is a centre */
    int64_t n_queries;
    int32_t search;           /* sfc_search_kind */
    int32_t kernel;           /* radius: sfc_kernel */
    float r;                  /* radius */
    int32_t k;                /* kNN: 1..64 */
} sfc_request;

typedef struct {
    const int64_t* row_ptr;   /* radius: device, n_rows + 1 entries, row_ptr[0] == 0; row i is
                                 cols[row_ptr[i] .. row_ptr[i + 1]) */
    const int32_t* cols;      /* radius: device, nnz entries (ids are positions in the cloud) */
    int64_t nnz;
    int64_t row_base;         /* always 0 (kept for the layout) */
    const int32_t* knn_idx;   /* kNN: device, n_rows x k (layout of knn()) */
    const float* knn_d2;
    int64_t n_rows;
    double latency_ms;        /* submit to result resident on the device */
    double queue_ms;          /* submit to admission */
    int32_t batched_with;     /* requests in its device pass (1: alone) */
    int32_t pad;
} sfc_request_result;

typedef struct {
    int64_t queued, running, admitted, reserved_bytes;
} sfc_server_stats;

/* Defaults: 4 slots, merge up to 64 all-points requests of <= 4M points in all, 150 GiB,
 * Hilbert, leaf capacity 64. */
sfc_status sfc_server_opts_default(sfc_server_opts* o);

/* Start a server on the current device (worker threads and streams).  The requests' work
 * is the plain method's (octree_build + radius_search / knn, or batch_search for merged
 * all-points requests): a result does not depend on the requests that ran beside it.
 * The paper serves one query set at a time; this is the serving layer around it. */
sfc_status server_create(const sfc_server_opts* opts, sfc_server* out);

/* Queue a request (non-blocking; its arrival time is now).  SFC_ERR_INVALID /
 * SFC_ERR_TOO_LARGE for bad arguments; failures of the work itself are reported by
 * server_wait. */
sfc_status server_submit(sfc_server s, const sfc_request* req, int64_t* id);

/* Wait for a request (timeout_ms < 0: no limit): SFC_ERR_TIMEOUT if it has not finished
 * in time, else SFC_OK with *result = the request's own status. */
sfc_status server_wait(sfc_server s, int64_t id, int32_t timeout_ms, sfc_status* result);

/* Device views and timings of a finished request; valid until server_release. */
sfc_status server_result(sfc_server s, int64_t id, sfc_request_result* out);

/* Free a finished request's octree and results (its memory leaves the budget). */
sfc_status server_release(sfc_server s, int64_t id);

/* A snapshot of the server's counters (host struct, no device synchronisation);
 * SFC_ERR_INVALID for a NULL server or out. */
sfc_status server_stats(sfc_server s, sfc_server_stats* out);

/* Stop accepting requests, free the results of finished ones, run the queued requests to
 * the end (still admitted within the memory budget), stop the workers and free everything. */
sfc_status server_destroy(sfc_server s);

/* ---- device memory ---------------------------------------------------------------- */

/* A caller's device allocator (e.g. a framework's caching allocator): alloc returns
 * `bytes` of device memory usable in stream order on cuda_stream, or NULL; free releases
 * it in stream order.  Both may be called from any host thread (the server's workers). */
typedef void* (*sfc_alloc_fn)(size_t bytes, void* ctx, void* cuda_stream);
typedef void (*sfc_free_fn)(void* p, void* ctx, void* cuda_stream);

/* Route every device allocation of the library (octrees, search outputs it allocates,
 * scratch) through alloc / free; both NULL restores the stream-ordered allocator.  The
 * temporaries recorded into a batch plan's graph always use the stream-ordered allocator.
 * SFC_ERR_INVALID when exactly one of the two is NULL, or while library allocations are
 * alive (every allocation is freed by the allocator that made it). */
sfc_status sfc_set_allocator(sfc_alloc_fn alloc, sfc_free_fn free_fn, void* ctx);

/* Library device allocations alive now (octrees, outputs, plans, records). */
int64_t sfc_live_allocations(void);

/* ---- introspection (tests, diagnostics) ------------------------------------------ */

/* Copy the sorted codes (n), the permutation sorted position -> original index (n), the
 * leaves array (n_leaves + 1, last entry 8^21) and the per-leaf point counts (n_leaves)
 * into caller-owned device buffers; any pointer may be NULL. */
sfc_status octree_export(sfc_octree h, void* cuda_stream, uint64_t* sorted_keys, uint32_t* perm,
                         uint64_t* leaves, uint32_t* leaf_counts);

/* Copy the node table (n_nodes entries; node 0 is the root, the eight children of an
 * internal node are consecutive): first code of the node's cell, level (0..21),
 * internalRanges [start, end) in sorted positions, first-child index (-1 for a leaf) and
 * tight bounding box (lo xyz, hi xyz; +inf/-inf when empty).  Caller-owned device
 * buffers; any pointer may be NULL. */
sfc_status octree_export_nodes(sfc_octree h, void* cuda_stream, uint64_t* node_key, int32_t* node_level,
                               uint32_t* node_start, uint32_t* node_end, int32_t* node_child, float* node_box);

/* 63-bit codes of integer cells (sections 4.1, 4.2) at L = 21: cells device n x 3 uint32
 * (each < 2^21), keys device n uint64.  SFC_ENC_NONE gives Morton codes. */
sfc_status sfc_encode_cells(const uint32_t* cells, int64_t n, sfc_encoding enc, void* cuda_stream,
                            uint64_t* keys);

/* ---- runtime ------------------------------------------------------------------------ */

const char* sfc_status_string(sfc_status s);
/* Last CUDA error message seen by the calling thread ("" if none). */
const char* sfc_last_error(void);
/* Number of kernels this library has launched in this process. */
uint64_t sfc_launch_count(void);
/* Per-kernel timing with CUDA events recorded on each launch's stream: on != 0 starts a
 * new record, 0 stops recording. */
sfc_status sfc_profile_enable(int32_t on);
/* Synchronises on the recorded events and returns the number of distinct kernels
 * recorded; for i < min(that, cap): names[i * 64 ..] (NUL-terminated), launches[i],
 * total_ms[i]. */
int32_t sfc_profile_read(char* names, int64_t* launches, double* total_ms, int32_t cap);

/* Work counters of the search walks (the candidate tests of sections 3.2-3.3 and 5.1, for
 * the ALU side of a roofline).  Summed over every radius count pass (CSR output) and
 * every kNN search on octree_build handles launched while counting is on, from any
 * thread (the request server's requests that run alone included); the batched searches
 * and the range output are not counted.  "Executed" counts every lane
 * of a warp that runs an evaluation, "needed" only the lanes whose own centre's walk
 * reaches the leaf (what a walk per centre would test). */
typedef struct {
    int64_t walks;         /* warp groups of 32 centres, or walks of one centre (SFC_ENC_NONE) */
    int64_t expansions;    /* internal nodes whose children were examined */
    int64_t box_tests;     /* centre-box evaluations executed (one per lane and child examined) */
    int64_t leaves;        /* leaves whose points were read */
    int64_t point_tests;   /* centre-point kernel or distance evaluations executed, including
                              the kNN seeding window along the curve */
    int64_t needed_tests;  /* of those, by lanes whose own walk reaches the leaf */
    int64_t passed;        /* radius: hits; kNN: points marked as candidates */
    int64_t whole;         /* radius: neighbours taken inside whole nodes (step 1a, no test) */
    int64_t inserts;       /* kNN: insertions into a centre's list of k best */
} sfc_search_stats;

/* on != 0 zeroes the counters (synchronising the device) and makes the searches launch an
 * instrumented copy of their kernels: the same results, more registers and instructions,
 * so never time a search while counting.  The counters live on the device current at
 * this call; searches launched on another device are not counted.  0 stops counting.
 * SFC_ERR_CUDA if the counters cannot be allocated. */
sfc_status sfc_stats_enable(int32_t on);
/* Synchronises the counters' device and copies the counters into *out (all zero if
 * counting was never enabled).  SFC_ERR_INVALID for out == NULL. */
sfc_status sfc_stats_read(sfc_search_stats* out);

#ifdef __cplusplus
}
#endif
#endif /* SFCOCT_H */

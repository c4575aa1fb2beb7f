/*
 * oracle.h - plain, slow CPU reference for the SFC + linear-octree neighbour search.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load or call this library.  The CUDA library never links,
 * includes or calls it, and it shares no code with the CUDA library.
 *
 * Every routine follows a definition of the paper (arXiv 2603.06771) and cites it:
 *   section 3.2  (Definition of the search kernels)      -> orc_pred, radius searches
 *   section 3.3  (kNN priority queue, octant distance)   -> orc_knn_tree, orc_knn_brute
 *   section 4    (discretisation of the bounding box)    -> orc_bbox, orc_discretise
 *   section 4.1  (Morton bit interleaving)               -> orc_morton_*
 *   section 4.2  (Hilbert curve)                         -> orc_hilbert_*
 *   section 4    (reordering by ascending codes)         -> orc_sort
 *   section 5.1  (leaves construction, internalRanges)   -> orc_leaves, orc_tree_nodes
 *   section 3.1  (pointer octree with N_max)             -> orc_tree_build
 *   section 5.2  (kNN locality histogram)                -> orc_locality_histogram
 *
 * Floating point: IEEE binary32, round to nearest, every operation rounded on its
 * own (built with -ffp-contract=off, no fast-math).
 */
#ifndef SFC_ORACLE_H
#define SFC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_SPHERE = 0, ORC_CIRCLE = 1, ORC_CUBE = 2, ORC_SQUARE = 3 };
enum { ORC_ENC_NONE = 0, ORC_ENC_MORTON = 1, ORC_ENC_HILBERT = 2 };

#define ORC_L 21

void orc_free(void* p);

/* section 4: bounding box and the uniform scale into [0, 2^21)^3.
 * Returns 0, or 1 when a coordinate or the extent is not finite. */
int orc_bbox(const float* xyz, int64_t n, float lo[3], float* ext, float* scale);
void orc_discretise(const float* xyz, int64_t n, const float lo[3], float scale, uint32_t* cell);

/* section 4.1 / 4.2: codes at L levels (1 <= L <= 21). */
uint64_t orc_morton_encode(uint32_t x, uint32_t y, uint32_t z, int L);
void orc_morton_decode(uint64_t code, int L, uint32_t out[3]);
uint64_t orc_hilbert_encode(uint32_t x, uint32_t y, uint32_t z, int L);
void orc_hilbert_decode(uint64_t code, int L, uint32_t out[3]);
/* batch forms; enc NONE encodes with Morton (the tree of an unordered cloud uses Morton keys) */
void orc_encode_cells(const uint32_t* cell, int64_t n, int enc, int L, uint64_t* codes);
void orc_decode_codes(const uint64_t* codes, int64_t n, int enc, int L, uint32_t* cell);

/* section 4: ascending order of the codes; equal codes keep input order. */
void orc_sort(const uint64_t* keys, int64_t n, uint32_t* perm, uint64_t* sorted);

/* section 5.1: the leaves array by repeated splitting; returns the number of leaves
 * nL and mallocs *leaves (nL + 1 entries) and *counts (nL entries). */
int64_t orc_leaves(const uint64_t* sorted, int64_t n, int64_t ncap, uint64_t** leaves, uint32_t** counts);

/* section 3.1: pointer octree over the discretised cells. */
typedef struct orc_tree orc_tree;
orc_tree* orc_tree_build(const float* xyz, const uint32_t* cell, int64_t n, int64_t ncap);
void orc_tree_free(orc_tree* t);
int64_t orc_tree_num_nodes(const orc_tree* t);
int64_t orc_tree_num_leaves(const orc_tree* t);
/* Node list in depth-first order.  For encoding enc: key_start = first code of the
 * node's cell, level, count, is_leaf, and [start, end) = positions of the node's
 * points in the sorted cloud (rank[i] = sorted position of point i); contiguous[i]
 * is 1 when those positions form one range.  Empty nodes get start = end =
 * lower_bound(sorted_keys, key_start).  box = tight AABB (lo xyz, hi xyz). */
void orc_tree_nodes(const orc_tree* t, int enc, const uint32_t* rank, const uint64_t* sorted_keys,
                    uint64_t* key_start, int32_t* level, int64_t* count, int32_t* is_leaf,
                    int64_t* start, int64_t* end, int32_t* contiguous, float* box);

/* section 3.2: one kernel decision (1 = inside). */
int orc_pred(int kern, const float p[3], const float c[3], float r);

/* Fixed-radius search for nq centres.  row_ptr has nq + 1 entries; *cols is malloced.
 * Rows list original point indices in ascending order.  Returns the total count. */
int64_t orc_radius_brute(const float* xyz, int64_t n, const float* q, int64_t nq, float r, int kern,
                         int nthreads, int64_t* row_ptr, int32_t** cols);
int64_t orc_radius_tree(const orc_tree* t, const float* q, int64_t nq, float r, int kern,
                        int nthreads, int64_t* row_ptr, int32_t** cols);

/* section 3.3: k nearest by (squared distance, original index); idx = -1 and
 * d2 = +inf pad rows when k > n. */
void orc_knn_brute(const float* xyz, int64_t n, const float* q, int64_t nq, int k, int nthreads,
                   int32_t* idx, float* d2);
void orc_knn_tree(const orc_tree* t, const float* q, int64_t nq, int k, int nthreads,
                  int32_t* idx, float* d2);

/* Count of (centre, point) pairs whose binary32 decision differs from the decision
 * taken in binary64 on the same inputs. */
int64_t orc_boundary_disagreements(const float* xyz, int64_t n, const float* q, int64_t nq, float r,
                                   int kern, int nthreads);

/* section 5.2: H_k(d) for d = 0..n-1 from kNN index rows given in sorted positions. */
void orc_locality_histogram(const int64_t* nbr_pos, int64_t n_rows, int k, const int64_t* row_pos,
                            int64_t n, int64_t* hist);

int orc_num_cpus(void);

#ifdef __cplusplus
}
#endif
#endif

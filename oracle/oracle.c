/*
 * oracle.c - plain, slow CPU reference for the SFC + linear-octree neighbour search.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load or call this library.  It shares no code with the
 * CUDA library and neither includes nor links the other.
 *
 * Each function states the passage of arXiv 2603.06771 it follows.  Where the
 * paper leaves a choice open, the reading taken is written next to the code.
 * Built with -O2 -ffp-contract=off: every binary32 operation is rounded on its own.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

void orc_free(void* p) { free(p); }

int orc_num_cpus(void) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (int)c : 1;
}

/* ------------------------------------------------------------------------- */
/* Section 4: translate and scale into [0, N)^3 with N = 2^L, then floor.     */
/* Reading: one uniform scale for all three axes (cubic cells), computed in   */
/* binary32: s = 2^21 / ext with ext the largest axis extent (1 if all zero). */
/* The upper corner lands on 2^21 and is clamped into the half-open grid.     */
/* ------------------------------------------------------------------------- */
int orc_bbox(const float* xyz, int64_t n, float lo[3], float* ext, float* scale) {
    float hi[3];
    for (int a = 0; a < 3; a++) { lo[a] = 0.0f; hi[a] = 0.0f; }
    for (int64_t i = 0; i < n; i++) {
        for (int a = 0; a < 3; a++) {
            float v = xyz[3 * i + a];
            if (!isfinite(v)) return 1;
            if (i == 0 || v < lo[a]) lo[a] = v;
            if (i == 0 || v > hi[a]) hi[a] = v;
        }
    }
    float e = 0.0f;
    for (int a = 0; a < 3; a++) {
        float d = hi[a] - lo[a];
        if (d > e) e = d;
    }
    if (!isfinite(e)) return 1;
    if (e == 0.0f) e = 1.0f;
    *ext = e;
    *scale = 2097152.0f / e;
    return 0;
}

void orc_discretise(const float* xyz, int64_t n, const float lo[3], float scale, uint32_t* cell) {
    const uint32_t top = (1u << ORC_L) - 1u;
    for (int64_t i = 0; i < n; i++) {
        for (int a = 0; a < 3; a++) {
            float shifted = xyz[3 * i + a] - lo[a];
            float scaled = shifted * scale;
            float f = floorf(scaled);
            uint32_t c;
            if (!(f > 0.0f)) c = 0;                 /* also the -0 and below-box cases */
            else if (f >= (float)top) c = top;      /* the half-open upper face */
            else c = (uint32_t)f;
            cell[3 * i + a] = c;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Section 4.1: Morton code = the bits of x, y, z interleaved level by level,  */
/* most significant level first, x before y before z inside each triple        */
/* (the worked example (3, 7, 2) at L = 3 gives 010 111 110 = 190).            */
/* ------------------------------------------------------------------------- */
uint64_t orc_morton_encode(uint32_t x, uint32_t y, uint32_t z, int L) {
    uint64_t code = 0;
    for (int level = 0; level < L; level++) {
        int bit = L - 1 - level; /* bit of the coordinate used at this level */
        uint64_t triple = ((uint64_t)((x >> bit) & 1u) << 2) | ((uint64_t)((y >> bit) & 1u) << 1) |
                          (uint64_t)((z >> bit) & 1u);
        code = (code << 3) | triple;
    }
    return code;
}

void orc_morton_decode(uint64_t code, int L, uint32_t out[3]) {
    uint32_t x = 0, y = 0, z = 0;
    for (int level = 0; level < L; level++) {
        uint64_t triple = (code >> (3 * (L - 1 - level))) & 7u;
        x = (x << 1) | (uint32_t)((triple >> 2) & 1u);
        y = (y << 1) | (uint32_t)((triple >> 1) & 1u);
        z = (z << 1) | (uint32_t)(triple & 1u);
    }
    out[0] = x; out[1] = y; out[2] = z;
}

/* ------------------------------------------------------------------------- */
/* Section 4.2: Hilbert code.  The paper leaves the member of the Hilbert      */
/* family open (only continuity matters) and used an algorithm that is not     */
/* reproduced here.  Reading: the curve of J. Skilling, "Programming the       */
/* Hilbert curve", AIP Conf. Proc. 707 (2004): coordinates are turned into the  */
/* "transposed" Hilbert index level by level (at each bit plane, an axis whose  */
/* bit is set inverts the lower bits of axis 0, otherwise axis 0 and that axis  */
/* exchange their lower bits), the planes are Gray coded, and the transposed   */
/* bits are read out x-high like the Morton triples.                            */
/* ------------------------------------------------------------------------- */
static void skilling_axes_to_transposed(uint32_t v[3], int bits) {
    const uint32_t top = 1u << (bits - 1);
    /* undo the excess work, plane by plane from the top */
    for (uint32_t plane = top; plane > 1; plane >>= 1) {
        const uint32_t below = plane - 1;
        for (int axis = 0; axis < 3; axis++) {
            if (v[axis] & plane) {
                v[0] ^= below; /* invert */
            } else {
                uint32_t diff = (v[0] ^ v[axis]) & below; /* exchange */
                v[0] ^= diff;
                v[axis] ^= diff;
            }
        }
    }
    /* Gray encode across the axes */
    v[1] ^= v[0];
    v[2] ^= v[1];
    /* fold the running parity of the last axis into every lower plane */
    uint32_t flip = 0;
    for (uint32_t plane = top; plane > 1; plane >>= 1)
        if (v[2] & plane) flip ^= plane - 1;
    v[0] ^= flip; v[1] ^= flip; v[2] ^= flip;
}

static void skilling_transposed_to_axes(uint32_t v[3], int bits) {
    const uint32_t end = 2u << (bits - 1);
    /* Gray decode: H ^ (H >> 1) on the interleaved index, written per axis */
    uint32_t carry = v[2] >> 1;
    v[2] ^= v[1];
    v[1] ^= v[0];
    v[0] ^= carry;
    /* redo the work, plane by plane from the bottom */
    for (uint32_t plane = 2; plane != end; plane <<= 1) {
        const uint32_t below = plane - 1;
        for (int axis = 2; axis >= 0; axis--) {
            if (v[axis] & plane) {
                v[0] ^= below;
            } else {
                uint32_t diff = (v[0] ^ v[axis]) & below;
                v[0] ^= diff;
                v[axis] ^= diff;
            }
        }
    }
}

uint64_t orc_hilbert_encode(uint32_t x, uint32_t y, uint32_t z, int L) {
    uint32_t v[3] = {x, y, z};
    skilling_axes_to_transposed(v, L);
    /* the transposed index read out like a Morton code */
    return orc_morton_encode(v[0], v[1], v[2], L);
}

void orc_hilbert_decode(uint64_t code, int L, uint32_t out[3]) {
    uint32_t v[3];
    orc_morton_decode(code, L, v);
    skilling_transposed_to_axes(v, L);
    out[0] = v[0]; out[1] = v[1]; out[2] = v[2];
}

void orc_encode_cells(const uint32_t* cell, int64_t n, int enc, int L, uint64_t* codes) {
    for (int64_t i = 0; i < n; i++) {
        const uint32_t* c = cell + 3 * i;
        codes[i] = enc == ORC_ENC_HILBERT ? orc_hilbert_encode(c[0], c[1], c[2], L)
                                          : orc_morton_encode(c[0], c[1], c[2], L);
    }
}

void orc_decode_codes(const uint64_t* codes, int64_t n, int enc, int L, uint32_t* cell) {
    for (int64_t i = 0; i < n; i++) {
        if (enc == ORC_ENC_HILBERT) orc_hilbert_decode(codes[i], L, cell + 3 * i);
        else orc_morton_decode(codes[i], L, cell + 3 * i);
    }
}

/* ------------------------------------------------------------------------- */
/* Section 4: reorder the cloud by ascending code.  Reading: equal codes keep  */
/* their input order (a stable sort).  Sorting (code, index) pairs under the   */
/* lexicographic order is the same permutation.                                */
/* ------------------------------------------------------------------------- */
typedef struct { uint64_t key; uint32_t idx; } key_idx;

static int cmp_key_idx(const void* a, const void* b) {
    const key_idx* x = (const key_idx*)a;
    const key_idx* y = (const key_idx*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

void orc_sort(const uint64_t* keys, int64_t n, uint32_t* perm, uint64_t* sorted) {
    key_idx* tmp = (key_idx*)malloc((size_t)(n > 0 ? n : 1) * sizeof(key_idx));
    for (int64_t i = 0; i < n; i++) { tmp[i].key = keys[i]; tmp[i].idx = (uint32_t)i; }
    qsort(tmp, (size_t)n, sizeof(key_idx), cmp_key_idx);
    for (int64_t i = 0; i < n; i++) { perm[i] = tmp[i].idx; sorted[i] = tmp[i].key; }
    free(tmp);
}

/* first position whose code is >= key */
static int64_t lower_bound_u64(const uint64_t* a, int64_t n, uint64_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* ------------------------------------------------------------------------- */
/* Section 5.1: leaves = {0, 8^L}; count the codes of every range by binary    */
/* search; a range holding more than N_max codes becomes 8 equal ranges;       */
/* repeat until nothing splits.  Reading: a single-cell range (level L) is     */
/* never split, so duplicate codes may overfill it.                            */
/* ------------------------------------------------------------------------- */
int64_t orc_leaves(const uint64_t* sorted, int64_t n, int64_t ncap, uint64_t** leaves_out,
                   uint32_t** counts_out) {
    const uint64_t whole = (uint64_t)1 << (3 * ORC_L);
    int64_t nb = 2, cap = 1024;
    uint64_t* b = (uint64_t*)malloc((size_t)cap * sizeof(uint64_t));
    b[0] = 0; b[1] = whole;
    for (;;) {
        int split_any = 0;
        int64_t out_cap = nb * 8, m = 0;
        uint64_t* nbnd = (uint64_t*)malloc((size_t)out_cap * sizeof(uint64_t));
        for (int64_t i = 0; i + 1 < nb; i++) {
            uint64_t a = b[i], e = b[i + 1];
            int64_t cnt = lower_bound_u64(sorted, n, e) - lower_bound_u64(sorted, n, a);
            uint64_t size = e - a;
            if (cnt > ncap && size > 1) {
                uint64_t part = size / 8;
                for (int j = 0; j < 8; j++) nbnd[m++] = a + (uint64_t)j * part;
                split_any = 1;
            } else {
                nbnd[m++] = a;
            }
        }
        nbnd[m++] = whole;
        free(b);
        b = nbnd;
        nb = m;
        if (!split_any) break;
    }
    int64_t nl = nb - 1;
    uint32_t* counts = (uint32_t*)malloc((size_t)(nl > 0 ? nl : 1) * sizeof(uint32_t));
    for (int64_t i = 0; i < nl; i++)
        counts[i] = (uint32_t)(lower_bound_u64(sorted, n, b[i + 1]) - lower_bound_u64(sorted, n, b[i]));
    *leaves_out = b;
    *counts_out = counts;
    return nl;
}

/* ------------------------------------------------------------------------- */
/* Section 3.1: pointer octree.  A node is split into its eight octants when   */
/* it holds more than N_max points; all eight children are created (complete   */
/* octree).  The octants are halves of the integer cell cube, so the tree has  */
/* exactly the cells of the linear octree.  Every node keeps the tight AABB of */
/* its points for pruning.                                                     */
/* ------------------------------------------------------------------------- */
typedef struct onode {
    uint32_t cx, cy, cz; /* cell index at this level */
    int level;
    int64_t count;
    int64_t* ids;        /* leaf: the original indices of its points */
    struct onode* child[8];
    float lo[3], hi[3];
    int is_leaf;
} onode;

struct orc_tree {
    onode* root;
    const float* xyz;
    const uint32_t* cell;
    int64_t n, ncap;
    int64_t* ids;
    int64_t n_nodes, n_leaves;
};

static void box_empty(onode* nd) {
    for (int a = 0; a < 3; a++) { nd->lo[a] = INFINITY; nd->hi[a] = -INFINITY; }
}

static void build_node(orc_tree* t, onode* nd, int64_t* ids, int64_t count, int64_t* scratch) {
    nd->count = count;
    t->n_nodes++;
    box_empty(nd);
    if (count > t->ncap && nd->level < ORC_L) {
        int shift = ORC_L - 1 - nd->level; /* bit of the cell coordinate that picks the octant */
        int64_t cnt[8] = {0}, off[8];
        for (int64_t i = 0; i < count; i++) {
            const uint32_t* c = t->cell + 3 * ids[i];
            int oct = (int)(((c[0] >> shift) & 1u) << 2 | ((c[1] >> shift) & 1u) << 1 | ((c[2] >> shift) & 1u));
            cnt[oct]++;
        }
        off[0] = 0;
        for (int o = 1; o < 8; o++) off[o] = off[o - 1] + cnt[o - 1];
        int64_t pos[8];
        memcpy(pos, off, sizeof pos);
        for (int64_t i = 0; i < count; i++) {
            const uint32_t* c = t->cell + 3 * ids[i];
            int oct = (int)(((c[0] >> shift) & 1u) << 2 | ((c[1] >> shift) & 1u) << 1 | ((c[2] >> shift) & 1u));
            scratch[pos[oct]++] = ids[i];
        }
        memcpy(ids, scratch, (size_t)count * sizeof(int64_t));
        nd->is_leaf = 0;
        nd->ids = NULL;
        for (int o = 0; o < 8; o++) {
            onode* ch = (onode*)calloc(1, sizeof(onode));
            ch->level = nd->level + 1;
            ch->cx = nd->cx * 2 + ((o >> 2) & 1);
            ch->cy = nd->cy * 2 + ((o >> 1) & 1);
            ch->cz = nd->cz * 2 + (o & 1);
            build_node(t, ch, ids + off[o], cnt[o], scratch + off[o]);
            nd->child[o] = ch;
            for (int a = 0; a < 3; a++) {
                if (ch->lo[a] < nd->lo[a]) nd->lo[a] = ch->lo[a];
                if (ch->hi[a] > nd->hi[a]) nd->hi[a] = ch->hi[a];
            }
        }
    } else {
        nd->is_leaf = 1;
        nd->ids = ids;
        t->n_leaves++;
        for (int64_t i = 0; i < count; i++) {
            const float* p = t->xyz + 3 * ids[i];
            for (int a = 0; a < 3; a++) {
                if (p[a] < nd->lo[a]) nd->lo[a] = p[a];
                if (p[a] > nd->hi[a]) nd->hi[a] = p[a];
            }
        }
    }
}

orc_tree* orc_tree_build(const float* xyz, const uint32_t* cell, int64_t n, int64_t ncap) {
    orc_tree* t = (orc_tree*)calloc(1, sizeof(orc_tree));
    t->xyz = xyz; t->cell = cell; t->n = n; t->ncap = ncap;
    t->ids = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t* scratch = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) t->ids[i] = i;
    t->root = (onode*)calloc(1, sizeof(onode));
    build_node(t, t->root, t->ids, n, scratch);
    free(scratch);
    return t;
}

static void free_node(onode* nd) {
    if (!nd->is_leaf)
        for (int o = 0; o < 8; o++) free_node(nd->child[o]);
    free(nd);
}

void orc_tree_free(orc_tree* t) {
    if (!t) return;
    free_node(t->root);
    free(t->ids);
    free(t);
}

int64_t orc_tree_num_nodes(const orc_tree* t) { return t->n_nodes; }
int64_t orc_tree_num_leaves(const orc_tree* t) { return t->n_leaves; }

typedef struct {
    int enc;
    const uint32_t* rank;
    const uint64_t* sorted_keys;
    int64_t n;
    uint64_t* key_start; int32_t* level; int64_t* count; int32_t* is_leaf;
    int64_t* start; int64_t* end; int32_t* contiguous; float* box;
    int64_t next;
} node_walk;

/* returns (min rank, max rank) of the node's points through *mn, *mx */
static void walk_nodes(node_walk* w, const onode* nd, int64_t* mn, int64_t* mx) {
    int64_t me = w->next++;
    int sh = ORC_L - nd->level;
    uint32_t x = nd->cx << sh, y = nd->cy << sh, z = nd->cz << sh; /* the cell's lowest corner */
    uint64_t code = w->enc == ORC_ENC_HILBERT ? orc_hilbert_encode(x, y, z, ORC_L) : orc_morton_encode(x, y, z, ORC_L);
    uint64_t mask = ((uint64_t)1 << (3 * sh)) - 1; /* 3 * sh <= 63 */
    w->key_start[me] = code & ~mask;
    w->level[me] = nd->level;
    w->count[me] = nd->count;
    w->is_leaf[me] = nd->is_leaf;
    for (int a = 0; a < 3; a++) { w->box[6 * me + a] = nd->lo[a]; w->box[6 * me + 3 + a] = nd->hi[a]; }
    int64_t lo = INT64_MAX, hi = -1;
    if (nd->is_leaf) {
        for (int64_t i = 0; i < nd->count; i++) {
            int64_t r = w->rank[nd->ids[i]];
            if (r < lo) lo = r;
            if (r > hi) hi = r;
        }
    } else {
        for (int o = 0; o < 8; o++) {
            int64_t a, b;
            walk_nodes(w, nd->child[o], &a, &b);
            if (a < lo) lo = a;
            if (b > hi) hi = b;
        }
    }
    if (nd->count == 0) {
        int64_t p = lower_bound_u64(w->sorted_keys, w->n, w->key_start[me]);
        w->start[me] = p; w->end[me] = p; w->contiguous[me] = 1;
    } else {
        w->start[me] = lo; w->end[me] = hi + 1;
        w->contiguous[me] = (hi - lo + 1) == nd->count;
    }
    *mn = lo; *mx = hi;
}

void orc_tree_nodes(const orc_tree* t, int enc, const uint32_t* rank, const uint64_t* sorted_keys,
                    uint64_t* key_start, int32_t* level, int64_t* count, int32_t* is_leaf,
                    int64_t* start, int64_t* end, int32_t* contiguous, float* box) {
    node_walk w = {enc, rank, sorted_keys, t->n, key_start, level, count, is_leaf, start, end, contiguous, box, 0};
    int64_t a, b;
    walk_nodes(&w, t->root, &a, &b);
}

/* ------------------------------------------------------------------------- */
/* Section 3.2, Definition (search kernels), with the strict "<" of the paper:  */
/*   Sphere ||(dx,dy,dz)||_2 < r, Circle ||(dx,dy,0)||_2 < r,                   */
/*   Cube ||(dx,dy,dz)||_inf < r, Square ||(dx,dy,0)||_inf < r.                 */
/* Evaluated without square roots: d = p - c per axis, squared norms summed     */
/* left to right and compared with r*r; the max-norms compared with r.  A norm  */
/* is never negative, so r <= 0 admits no point.                               */
/* ------------------------------------------------------------------------- */
static int pred_d(int kern, float dx, float dy, float dz, float r, float r2) {
    if (!(r > 0.0f)) return 0;
    switch (kern) {
    case ORC_SPHERE: {
        float xx = dx * dx;
        float yy = dy * dy;
        float zz = dz * dz;
        float s = xx + yy;
        s = s + zz;
        return s < r2;
    }
    case ORC_CIRCLE: {
        float xx = dx * dx;
        float yy = dy * dy;
        float s = xx + yy;
        return s < r2;
    }
    case ORC_CUBE: {
        float m = fabsf(dx);
        if (fabsf(dy) > m) m = fabsf(dy);
        if (fabsf(dz) > m) m = fabsf(dz);
        return m < r;
    }
    default: { /* ORC_SQUARE */
        float m = fabsf(dx);
        if (fabsf(dy) > m) m = fabsf(dy);
        return m < r;
    }
    }
}

int orc_pred(int kern, const float p[3], const float c[3], float r) {
    float r2 = r * r;
    float dx = p[0] - c[0];
    float dy = p[1] - c[1];
    float dz = p[2] - c[2];
    return pred_d(kern, dx, dy, dz, r, r2);
}

/* ------------------------------------------------------------------------- */
/* Simple work sharing: threads take chunks of centres from a shared counter    */
/* (the dynamic schedule the paper uses for its query loop, section 7.4).       */
/* ------------------------------------------------------------------------- */
typedef struct {
    int64_t next, total, chunk;
    pthread_mutex_t mu;
    void (*fn)(void* ctx, int64_t begin, int64_t end);
    void* ctx;
} work_pool;

static void* pool_worker(void* arg) {
    work_pool* w = (work_pool*)arg;
    for (;;) {
        pthread_mutex_lock(&w->mu);
        int64_t b = w->next;
        w->next += w->chunk;
        pthread_mutex_unlock(&w->mu);
        if (b >= w->total) break;
        int64_t e = b + w->chunk < w->total ? b + w->chunk : w->total;
        w->fn(w->ctx, b, e);
    }
    return NULL;
}

static void run_parallel(int64_t total, int nthreads, void (*fn)(void*, int64_t, int64_t), void* ctx) {
    if (nthreads <= 0) nthreads = orc_num_cpus();
    work_pool w;
    w.next = 0; w.total = total; w.chunk = 64; w.fn = fn; w.ctx = ctx;
    pthread_mutex_init(&w.mu, NULL);
    if (nthreads == 1 || total <= w.chunk) {
        pool_worker(&w);
    } else {
        pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
        for (int i = 0; i < nthreads; i++) pthread_create(&th[i], NULL, pool_worker, &w);
        for (int i = 0; i < nthreads; i++) pthread_join(th[i], NULL);
        free(th);
    }
    pthread_mutex_destroy(&w.mu);
}

/* growable list of point indices, one per query row */
typedef struct { int32_t* v; int64_t n, cap; } ivec;

static void ivec_push(ivec* a, int32_t x) {
    if (a->n == a->cap) {
        a->cap = a->cap ? a->cap * 2 : 16;
        a->v = (int32_t*)realloc(a->v, (size_t)a->cap * sizeof(int32_t));
    }
    a->v[a->n++] = x;
}

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

static int64_t assemble_rows(ivec* rows, int64_t nq, int64_t* row_ptr, int32_t** cols) {
    row_ptr[0] = 0;
    for (int64_t q = 0; q < nq; q++) row_ptr[q + 1] = row_ptr[q] + rows[q].n;
    int64_t total = row_ptr[nq];
    int32_t* c = (int32_t*)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
    for (int64_t q = 0; q < nq; q++) {
        qsort(rows[q].v, (size_t)rows[q].n, sizeof(int32_t), cmp_i32);
        if (rows[q].n) memcpy(c + row_ptr[q], rows[q].v, (size_t)rows[q].n * sizeof(int32_t));
        free(rows[q].v);
    }
    free(rows);
    *cols = c;
    return total;
}

typedef struct {
    const float* xyz; int64_t n; const float* q; float r; int kern; ivec* rows;
    const orc_tree* tree;
} radius_ctx;

/* the definition itself: every point tested against every centre */
static void radius_brute_chunk(void* vctx, int64_t b, int64_t e) {
    radius_ctx* cx = (radius_ctx*)vctx;
    float r2 = cx->r * cx->r;
    for (int64_t qi = b; qi < e; qi++) {
        const float* c = cx->q + 3 * qi;
        for (int64_t i = 0; i < cx->n; i++) {
            const float* p = cx->xyz + 3 * i;
            float dx = p[0] - c[0];
            float dy = p[1] - c[1];
            float dz = p[2] - c[2];
            if (pred_d(cx->kern, dx, dy, dz, cx->r, r2)) ivec_push(&cx->rows[qi], (int32_t)i);
        }
    }
}

int64_t orc_radius_brute(const float* xyz, int64_t n, const float* q, int64_t nq, float r, int kern,
                         int nthreads, int64_t* row_ptr, int32_t** cols) {
    radius_ctx cx = {xyz, n, q, r, kern, (ivec*)calloc((size_t)(nq > 0 ? nq : 1), sizeof(ivec)), NULL};
    run_parallel(nq, nthreads, radius_brute_chunk, &cx);
    return assemble_rows(cx.rows, nq, row_ptr, cols);
}

/* The naive octree search of section 3.2 (recurse into children that intersect
 * the kernel, test leaf points one by one).  "Intersects" is decided on the
 * node's tight AABB: the point of the box nearest to the centre (section 3.3's
 * clamp) is tested with the kernel itself.  Rounding to nearest is monotone, so a
 * box whose nearest point fails the test holds no point that passes it. */
static void radius_rec(const orc_tree* t, const onode* nd, const float c[3], float r, float r2, int kern,
                       ivec* out) {
    if (nd->count == 0) return;
    float g[3];
    for (int a = 0; a < 3; a++) g[a] = c[a] < nd->lo[a] ? nd->lo[a] : (c[a] > nd->hi[a] ? nd->hi[a] : c[a]);
    float gx = g[0] - c[0];
    float gy = g[1] - c[1];
    float gz = g[2] - c[2];
    if (!pred_d(kern, gx, gy, gz, r, r2)) return;
    if (nd->is_leaf) {
        for (int64_t i = 0; i < nd->count; i++) {
            int64_t id = nd->ids[i];
            const float* p = t->xyz + 3 * id;
            float dx = p[0] - c[0];
            float dy = p[1] - c[1];
            float dz = p[2] - c[2];
            if (pred_d(kern, dx, dy, dz, r, r2)) ivec_push(out, (int32_t)id);
        }
        return;
    }
    for (int o = 0; o < 8; o++) radius_rec(t, nd->child[o], c, r, r2, kern, out);
}

static void radius_tree_chunk(void* vctx, int64_t b, int64_t e) {
    radius_ctx* cx = (radius_ctx*)vctx;
    float r2 = cx->r * cx->r;
    for (int64_t qi = b; qi < e; qi++)
        radius_rec(cx->tree, cx->tree->root, cx->q + 3 * qi, cx->r, r2, cx->kern, &cx->rows[qi]);
}

int64_t orc_radius_tree(const orc_tree* t, const float* q, int64_t nq, float r, int kern,
                        int nthreads, int64_t* row_ptr, int32_t** cols) {
    radius_ctx cx = {t->xyz, t->n, q, r, kern, (ivec*)calloc((size_t)(nq > 0 ? nq : 1), sizeof(ivec)), t};
    run_parallel(nq, nthreads, radius_tree_chunk, &cx);
    return assemble_rows(cx.rows, nq, row_ptr, cols);
}

/* ------------------------------------------------------------------------- */
/* Section 3.3: k nearest neighbours.  Distance = the squared Euclidean norm of */
/* p - c summed left to right in binary32.  Reading of ties: neighbours are     */
/* ordered by (squared distance, original index).                              */
/* ------------------------------------------------------------------------- */
static float sq_dist(const float p[3], const float c[3]) {
    float dx = p[0] - c[0];
    float dy = p[1] - c[1];
    float dz = p[2] - c[2];
    float xx = dx * dx;
    float yy = dy * dy;
    float zz = dz * dz;
    float s = xx + yy;
    return s + zz;
}

static int pair_less(float da, int64_t ia, float db, int64_t ib) {
    return da < db || (da == db && ia < ib);
}

typedef struct {
    const float* xyz; int64_t n; const float* q; int k; int32_t* idx; float* d2; const orc_tree* tree;
} knn_ctx;

/* brute force: keep the k best (d2, index) pairs seen so far in sorted order */
static void knn_brute_chunk(void* vctx, int64_t b, int64_t e) {
    knn_ctx* cx = (knn_ctx*)vctx;
    int k = cx->k;
    float* bd = (float*)malloc(sizeof(float) * (size_t)k);
    int64_t* bi = (int64_t*)malloc(sizeof(int64_t) * (size_t)k);
    for (int64_t qi = b; qi < e; qi++) {
        const float* c = cx->q + 3 * qi;
        int have = 0;
        for (int64_t i = 0; i < cx->n; i++) {
            float d = sq_dist(cx->xyz + 3 * i, c);
            if (have == k && !pair_less(d, i, bd[k - 1], bi[k - 1])) continue;
            int pos = have < k ? have : k - 1;
            while (pos > 0 && pair_less(d, i, bd[pos - 1], bi[pos - 1])) {
                bd[pos] = bd[pos - 1]; bi[pos] = bi[pos - 1]; pos--;
            }
            bd[pos] = d; bi[pos] = i;
            if (have < k) have++;
        }
        for (int j = 0; j < k; j++) {
            cx->idx[qi * k + j] = j < have ? (int32_t)bi[j] : -1;
            cx->d2[qi * k + j] = j < have ? bd[j] : INFINITY;
        }
    }
    free(bd); free(bi);
}

void orc_knn_brute(const float* xyz, int64_t n, const float* q, int64_t nq, int k, int nthreads,
                   int32_t* idx, float* d2) {
    knn_ctx cx = {xyz, n, q, k, idx, d2, NULL};
    run_parallel(nq, nthreads, knn_brute_chunk, &cx);
}

/* The priority queue of section 3.3: elements (i, depth, is_octant, d).  The
 * smallest d is taken out; a point joins the result, a leaf puts its points in the
 * queue, an internal node puts its children.  An octant's d is the squared
 * distance from the centre to its nearest box point (the clamp, 0 inside), which
 * no point of the box undercuts.  With equal d, octants come out before points and
 * points by index, so the points come out in (d2, index) order. */
typedef struct { float d; int is_octant; int64_t id; const onode* node; int depth; } qitem;

static int qitem_less(const qitem* a, const qitem* b) {
    if (a->d != b->d) return a->d < b->d;
    if (a->is_octant != b->is_octant) return a->is_octant > b->is_octant;
    return a->id < b->id;
}

typedef struct { qitem* v; int64_t n, cap; } pqueue;

static void pq_push(pqueue* h, qitem x) {
    if (h->n == h->cap) {
        h->cap = h->cap ? h->cap * 2 : 256;
        h->v = (qitem*)realloc(h->v, (size_t)h->cap * sizeof(qitem));
    }
    int64_t i = h->n++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!qitem_less(&x, &h->v[p])) break;
        h->v[i] = h->v[p];
        i = p;
    }
    h->v[i] = x;
}

static qitem pq_pop(pqueue* h) {
    qitem top = h->v[0];
    qitem last = h->v[--h->n];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        const qitem* best = &last;
        if (l < h->n && qitem_less(&h->v[l], best)) { m = l; best = &h->v[l]; }
        if (r < h->n && qitem_less(&h->v[r], best)) { m = r; }
        if (m == i) break;
        h->v[i] = h->v[m];
        i = m;
    }
    if (h->n > 0) h->v[i] = last;
    return top;
}

static float octant_dist(const onode* nd, const float c[3]) {
    float g[3];
    for (int a = 0; a < 3; a++) g[a] = c[a] < nd->lo[a] ? nd->lo[a] : (c[a] > nd->hi[a] ? nd->hi[a] : c[a]);
    return sq_dist(g, c);
}

static void knn_tree_chunk(void* vctx, int64_t b, int64_t e) {
    knn_ctx* cx = (knn_ctx*)vctx;
    const orc_tree* t = cx->tree;
    int k = cx->k;
    pqueue h = {NULL, 0, 0};
    int64_t seq = 0;
    for (int64_t qi = b; qi < e; qi++) {
        const float* c = cx->q + 3 * qi;
        h.n = 0;
        int found = 0;
        if (t->root->count > 0) {
            qitem r0 = {octant_dist(t->root, c), 1, seq++, t->root, 0};
            pq_push(&h, r0);
        }
        while (found < k && h.n > 0) {
            qitem it = pq_pop(&h);
            if (!it.is_octant) {
                cx->idx[qi * k + found] = (int32_t)it.id;
                cx->d2[qi * k + found] = it.d;
                found++;
            } else if (it.node->is_leaf) {
                for (int64_t i = 0; i < it.node->count; i++) {
                    int64_t id = it.node->ids[i];
                    qitem p = {sq_dist(t->xyz + 3 * id, c), 0, id, NULL, 0};
                    pq_push(&h, p);
                }
            } else {
                for (int o = 0; o < 8; o++) {
                    const onode* ch = it.node->child[o];
                    if (ch->count == 0) continue;
                    qitem x = {octant_dist(ch, c), 1, seq++, ch, it.depth + 1};
                    pq_push(&h, x);
                }
            }
        }
        for (int j = found; j < k; j++) {
            cx->idx[qi * k + j] = -1;
            cx->d2[qi * k + j] = INFINITY;
        }
    }
    free(h.v);
}

void orc_knn_tree(const orc_tree* t, const float* q, int64_t nq, int k, int nthreads,
                  int32_t* idx, float* d2) {
    knn_ctx cx = {t->xyz, t->n, q, k, idx, d2, t};
    run_parallel(nq, nthreads, knn_tree_chunk, &cx);
}

/* ------------------------------------------------------------------------- */
/* Report only: how many (centre, point) decisions change when the same test   */
/* is taken in binary64 (differences and sums of the widened inputs).          */
/* ------------------------------------------------------------------------- */
typedef struct {
    const float* xyz; int64_t n; const float* q; float r; int kern; int64_t* per_chunk; int64_t chunk;
} bnd_ctx;

static int pred_f64(int kern, const float p[3], const float c[3], float r) {
    if (!(r > 0.0f)) return 0;
    double dx = (double)p[0] - (double)c[0];
    double dy = (double)p[1] - (double)c[1];
    double dz = (double)p[2] - (double)c[2];
    double rr = (double)r;
    switch (kern) {
    case ORC_SPHERE: return dx * dx + dy * dy + dz * dz < rr * rr;
    case ORC_CIRCLE: return dx * dx + dy * dy < rr * rr;
    case ORC_CUBE: return fmax(fabs(dx), fmax(fabs(dy), fabs(dz))) < rr;
    default: return fmax(fabs(dx), fabs(dy)) < rr;
    }
}

static void bnd_chunk(void* vctx, int64_t b, int64_t e) {
    bnd_ctx* cx = (bnd_ctx*)vctx;
    int64_t bad = 0;
    for (int64_t qi = b; qi < e; qi++) {
        const float* c = cx->q + 3 * qi;
        for (int64_t i = 0; i < cx->n; i++) {
            const float* p = cx->xyz + 3 * i;
            if (orc_pred(cx->kern, p, c, cx->r) != pred_f64(cx->kern, p, c, cx->r)) bad++;
        }
    }
    cx->per_chunk[b / cx->chunk] = bad;
}

int64_t orc_boundary_disagreements(const float* xyz, int64_t n, const float* q, int64_t nq, float r,
                                   int kern, int nthreads) {
    int64_t nchunks = (nq + 63) / 64;
    bnd_ctx cx = {xyz, n, q, r, kern, (int64_t*)calloc((size_t)(nchunks > 0 ? nchunks : 1), sizeof(int64_t)), 64};
    run_parallel(nq, nthreads, bnd_chunk, &cx);
    int64_t total = 0;
    for (int64_t i = 0; i < nchunks; i++) total += cx.per_chunk[i];
    free(cx.per_chunk);
    return total;
}

/* ------------------------------------------------------------------------- */
/* Section 5.2, Definition: H_k(d) = sum over centres i of the number of its k  */
/* nearest neighbours j stored at distance |i - j| = d in memory.  Positions    */
/* are storage positions; entries < 0 (padding) are skipped.                    */
/* ------------------------------------------------------------------------- */
void orc_locality_histogram(const int64_t* nbr_pos, int64_t n_rows, int k, const int64_t* row_pos,
                            int64_t n, int64_t* hist) {
    for (int64_t d = 0; d < n; d++) hist[d] = 0;
    for (int64_t i = 0; i < n_rows; i++) {
        for (int j = 0; j < k; j++) {
            int64_t p = nbr_pos[i * k + j];
            if (p < 0) continue;
            int64_t d = p > row_pos[i] ? p - row_pos[i] : row_pos[i] - p;
            hist[d]++;
        }
    }
}

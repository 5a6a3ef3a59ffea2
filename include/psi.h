/*
 * psi.h -- C ABI of the GB300 (sm_103a) spatial-index library.
 *
 * The library builds and maintains the two index families of "Parallel Dynamic
 * Spatial Indexes" (PPoPP '26, arXiv 2601.05347) on one GPU:
 *   - SPaC-Z / SPaC-H (Sec 4): points ordered by a Morton (Z) or Hilbert key,
 *     wrapped into leaves of at most `leaf_size` points, with bounding boxes and
 *     counts summarised bottom-up;
 *   - P-Orth (Sec 3): the orth-tree (quadtree/octree) that splits a region at its
 *     midpoint in every dimension until a node holds at most `leaf_size` points.
 * and answers the queries of Sec 2.2 on them: k-nearest neighbours, range count
 * and range list ("report").
 *
 * Conventions shared by every call:
 *   - Coordinates are int32 in [0, 2^coord_bits); points are AoS, `dim` int32
 *     per point ([n][dim]).  Ids are uint32 chosen by the caller and must be
 *     unique among the live points of an index (not checked).
 *   - Every pointer argument named d_* is DEVICE memory owned by the caller.
 *     The library reads inputs and writes outputs only in stream order on the
 *     given stream; it keeps no reference to them after the call returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls are asynchronous unless stated otherwise.
 *   - The library owns the index memory (stream-ordered allocations on the
 *     current device); psi_destroy releases it.
 *   - Errors: every call returns a psi_status; psi_last_error() gives a message
 *     for the calling thread.  Errors detected on the device (a coordinate out
 *     of range, a bounded wait that timed out) are recorded in the index and
 *     returned by the next psi_sync() (and by synchronising calls).
 *   - Squared distances are exact int64; k-NN ties are broken by smaller id.
 *     Range boxes are closed ([lo, hi] in every dimension); a box with
 *     lo > hi in some dimension is empty.
 */
#ifndef PSI_H
#define PSI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PSI_OK = 0,
  PSI_ERR_INVALID = 1,        /* bad argument: null pointer, n < 0, k < 1, unsupported config */
  PSI_ERR_RANGE = 2,          /* a coordinate outside [0, 2^coord_bits) (device-detected) */
  PSI_ERR_OOM = 3,            /* a device allocation failed */
  PSI_ERR_CAPACITY = 4,       /* psi_range_report: output capacity too small */
  PSI_ERR_DEVICE_TIMEOUT = 5, /* a bounded device-side wait gave up */
  PSI_ERR_CUDA = 6            /* any other CUDA error */
} psi_status;

typedef enum {
  PSI_SPAC_Z = 0, /* SPaC-tree on the Morton (Z) curve, Sec 4 */
  PSI_SPAC_H = 1, /* SPaC-tree on the Hilbert curve (2D: Hilbert 1891; 3D: Skilling 2004), Sec 4 */
  PSI_PORTH = 2   /* P-Orth tree, Sec 3 */
} psi_kind;

typedef struct {
  int32_t dim;        /* 2 or 3 */
  int32_t kind;       /* psi_kind */
  int32_t leaf_size;  /* leaf wrap phi, 1..64 (Table 1 "leaf wrap"; the paper uses 32-40) */
  int32_t coord_bits; /* b: 1..31 in 2D, 1..21 in 3D; keys have dim*b bits */
  int32_t fanout;     /* fanout of the SPaC summary tree over the leaves, 2..32 (0 = 32) */
  int32_t radix_bits; /* digit width of the key sort: 8, 10 or 11 (0 = 8, the fastest on GB300) */
} psi_config;

typedef struct psi_index psi_index;

/* Batch construction.  SPaC (Algorithm 3): each point's curve key is computed
 * on first touch inside the key sort, (key, id) pairs are sorted (ties in key by
 * id), and the sorted sequence is cut into leaves of exactly leaf_size points
 * (the last may be shorter) with their boxes, counts and first (key, id); a
 * summary tree of the given fanout is built over the leaves.  P-Orth
 * (Algorithm 1): the same key sort on Morton keys, then the orth-tree whose
 * nodes split by key bits.  d_pts is [n][dim], d_ids is [n]; n may be 0.
 * On success *out receives a new index. */
psi_status psi_build(const psi_config *cfg, const int32_t *d_pts, const uint32_t *d_ids, int64_t n,
                     void *stream, psi_index **out);

/* Batch insertion (SPaC: Algorithm 4; P-Orth: Algorithm 2).  The batch is
 * key-sorted and each point is routed to the leaf whose key range holds it.
 * SPaC: a leaf whose points fit its block (2*leaf_size slots) takes them
 * unsorted; an overflowing leaf is merged with its slice and re-wrapped into
 * leaves of at most leaf_size.  P-Orth: the leaves within leaf_size + 1
 * points (in key order) of an inserted point are rebuilt, a leaf that exceeds
 * leaf_size being split by the next key bits, and the nodes re-derived, so the
 * tree equals a fresh build of the same points (a batch above n/16, or above
 * n/256 reaching more than a quarter of the leaves, rebuilds every leaf).
 * Synchronises `stream`: SPaC once, to size the new leaf list; P-Orth a few
 * times, to size the rebuilt leaf and node lists. */
psi_status psi_insert_batch(psi_index *ix, const int32_t *d_pts, const uint32_t *d_ids, int64_t m,
                            void *stream);

/* Batch deletion (Sec 4.2 deletion paragraph; Sec 3.2).  Removes every live
 * point whose coordinates AND id equal a batch entry; absent entries are
 * ignored, a repeated entry deletes once.  d_num_deleted (device int64, may be
 * NULL) receives the number of points removed.  SPaC: touched leaves are
 * compacted and empty ones dropped; then every run of consecutive leaves
 * holding fewer than max(1, leaf_size / 2) points is joined with the leaf
 * after it (a run at the end with nothing after it, alone) and re-wrapped
 * into balanced leaves, so every leaf but the last keeps at least that many.
 * P-Orth: subtrees left with at most leaf_size points are flattened into one
 * leaf (the tree equals a fresh build).  Synchronises `stream`: SPaC once, or
 * twice when leaves are re-wrapped; P-Orth a few times. */
psi_status psi_delete_batch(psi_index *ix, const int32_t *d_pts, const uint32_t *d_ids, int64_t m,
                            int64_t *d_num_deleted, void *stream);

/* k-nearest neighbours (Sec 2.2).  For each of the q query points d_q[q][dim]
 * writes the min(k, size) live points smallest in (squared distance, id),
 * ascending, to d_ids[q][k] and d_d2[q][k]; slots past the index size get
 * id 0xFFFFFFFF and d2 INT64_MAX.  1 <= k <= 128. */
psi_status psi_knn(const psi_index *ix, const int32_t *d_q, int64_t q, int32_t k, uint32_t *d_ids,
                   int64_t *d_d2, void *stream);

/* Range count (Sec 2.2).  d_boxes is [q][2][dim] (lo corner, then hi corner);
 * d_counts[q] receives the number of live points inside each closed box. */
psi_status psi_range_count(const psi_index *ix, const int32_t *d_boxes, int64_t q, int64_t *d_counts,
                           void *stream);

#define PSI_REPORT_SORTED 1 /* sort each query's ids ascending */

/* Range list (Sec 2.2).  Writes d_offsets[q+1] (exclusive prefix of the
 * per-query counts) and, if the total fits in `capacity`, the ids of the
 * points inside each box to d_ids[offsets[i] .. offsets[i+1]).  Order within a
 * query is unspecified unless flags has PSI_REPORT_SORTED.  Synchronises
 * `stream`; *h_total (host) receives the total.  Returns PSI_ERR_CAPACITY
 * (offsets written, ids not) if total > capacity. */
psi_status psi_range_report(const psi_index *ix, const int32_t *d_boxes, int64_t q, int64_t *d_offsets,
                            uint32_t *d_ids, int64_t capacity, int64_t *h_total, int32_t flags,
                            void *stream);

/* Waits for the index's outstanding work on `stream` and returns any
 * device-detected error (PSI_ERR_RANGE, PSI_ERR_DEVICE_TIMEOUT), clearing it. */
psi_status psi_sync(psi_index *ix, void *stream);

/* Releases the index (synchronises the device first). */
psi_status psi_destroy(psi_index *ix);

/* Number of live points (host-side; exact after every call returns). */
int64_t psi_size(const psi_index *ix);

/* Number of leaves and of tree nodes (leaves included). */
int64_t psi_num_leaves(const psi_index *ix);
int64_t psi_num_nodes(const psi_index *ix);

/* Message of the last error on the calling thread ("" if none). */
const char *psi_last_error(void);

/* ---- Many independent indexes at once ---------------------------------- */

typedef struct psi_batch psi_batch;

/* Lays out storage for nidx independent SPaC indexes over one concatenated
 * point array: index i owns points [h_offsets[i], h_offsets[i+1]) (host array
 * of nidx+1 entries, h_offsets[0] = 0).  All indexes share cfg (SPAC_Z or
 * SPAC_H).  `threads` is the thread-block size of the build (256, 512, 1024; 0
 * = 512); cfg->radix_bits is the digit width of the build's block sort (0 or 8:
 * 8-bit digits; 11: 11-bit digits, with 256 or 512 threads only).  The index
 * layout does not depend on either.  Allocates everything the build needs, so psi_batch_build and
 * psi_batch_knn allocate nothing and can be captured in a CUDA graph.
 * Synchronises `stream`. */
psi_status psi_batch_create(const psi_config *cfg, const int64_t *h_offsets, int32_t nidx, int32_t threads,
                            void *stream, psi_batch **out);

/* Builds every index of the batch (Algorithm 3 per index: curve keys, (key, id)
 * sort, leaf wrapping, summaries) in ONE persistent kernel launch: each thread
 * block takes whole indexes, largest first, from an atomic queue.  Each index
 * gets exactly the layout psi_build would give it.  d_pts [total][dim] and
 * d_ids [total] are read during the call only. */
psi_status psi_batch_build(psi_batch *b, const int32_t *d_pts, const uint32_t *d_ids, void *stream);

/* Reserves query scratch for up to max_queries queries per psi_batch_knn call. */
psi_status psi_batch_knn_reserve(psi_batch *b, int64_t max_queries, void *stream);

/* k-NN (Sec 2.2) for queries grouped by index: d_qoffsets (DEVICE, nidx+1
 * entries) gives the queries [qoff[i], qoff[i+1]) that ask index i.  Results as
 * in psi_knn, one launch for all indexes.  nq <= the reserved capacity. */
psi_status psi_batch_knn(psi_batch *b, const int32_t *d_q, const int64_t *d_qoffsets, int64_t nq, int32_t k,
                         uint32_t *d_ids, int64_t *d_d2, void *stream);

/* Waits for `stream` and returns any device-detected error of the batch. */
psi_status psi_batch_sync(psi_batch *b, void *stream);
psi_status psi_batch_destroy(psi_batch *b);

/* Inspection: leaves of index i (counts[L], lo[L][dim], hi[L][dim]); *h_leaves = L. */
int64_t psi_batch_num_leaves(const psi_batch *b, int32_t i);
psi_status psi_batch_export_index(const psi_batch *b, int32_t i, int32_t *d_counts, int32_t *d_lo, int32_t *d_hi,
                                  int64_t *h_leaves, void *stream);

/* ---- Inspection (tests, tools) --------------------------------------- */

/* Leaves in key order: counts[L], lo[L][dim], hi[L][dim], first key and first
 * id of each leaf's key range (for a freshly built SPaC tree: of its first
 * point).  Any pointer may be NULL.  Device pointers; asynchronous. */
psi_status psi_export_leaves(const psi_index *ix, int32_t *d_counts, int32_t *d_lo, int32_t *d_hi,
                             uint64_t *d_sep_key, uint32_t *d_sep_id, void *stream);

/* All live points, leaf by leaf in key order (within a leaf: storage order):
 * d_pts[n][dim], d_ids[n], d_keys[n], d_leaf[n] (leaf number).  Any may be NULL. */
psi_status psi_export_points(const psi_index *ix, int32_t *d_pts, uint32_t *d_ids, uint64_t *d_keys,
                             int32_t *d_leaf, void *stream);

/* Tree nodes in preorder: depth (P-Orth: cell depth; SPaC: height above the
 * root), P-Orth cell prefix (SPaC: 0), subtree count, box, is_leaf.  Arrays of
 * psi_num_nodes() entries; any may be NULL. */
psi_status psi_export_nodes(const psi_index *ix, int32_t *d_depth, uint64_t *d_prefix, int64_t *d_count,
                            int32_t *d_lo, int32_t *d_hi, int32_t *d_is_leaf, void *stream);

/* Curve keys of n points under cfg (Morton for SPAC_Z/PORTH, Hilbert for
 * SPAC_H), as used by the index.  Out-of-range coordinates are reported by the
 * returned status after the call synchronises `stream`. */
psi_status psi_encode(const psi_config *cfg, const int32_t *d_pts, int64_t n, uint64_t *d_keys, void *stream);

/* Sorts n (key, value) pairs ascending by key with the library's onesweep LSD
 * radix sort (stable: equal keys keep their input order).  key_bits limits the
 * digits sorted (1..64).  In-place on the caller's arrays; uses library scratch. */
psi_status psi_sort_pairs(uint64_t *d_keys, uint32_t *d_vals, int64_t n, int32_t key_bits, void *stream);

/* Same sort as psi_sort_pairs, for callers that cannot let a library allocate
 * device memory: code running inside a host application that owns the whole
 * device memory budget (an engine that has reserved the memory pool for its
 * own arena), or a real-time loop where an allocation could block or fail in
 * the middle of a frame.  This entry point calls no cudaMalloc, cudaFree or
 * other allocating routine.  (The paper has no counterpart; it is a service of
 * this library.)
 *   - Limit: n <= 1048576 pairs; larger n returns PSI_ERR_INVALID and leaves
 *     the arrays untouched.
 *   - Scratch: one fixed array of about 14 MB in device memory, defined at
 *     file scope in the library; every GPU that loads the library holds it
 *     until the process exits.  All calls share it and it keeps the last
 *     call's contents; the call clears what must start at zero.  Calls that
 *     overlap on the GPU (on different streams, or from several host threads)
 *     race on it and must be serialised by the caller.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.  The address is looked up again when the
 *     device's context has changed since (e.g. after cudaDeviceReset).
 *   - Synchronises `stream` at the end (like psi_sort_pairs).
 *   - PSI_ERR_DEVICE_TIMEOUT (a bounded device-side wait ran out): the
 *     arrays' contents are then unspecified. */
psi_status psi_sort_pairs_noalloc(uint64_t *d_keys, uint32_t *d_vals, int64_t n, int32_t key_bits, void *stream);

/* ---- Test hook of the bounded device-side waits ----------------------------
 * Failure detection (every wait of a digit pass on a predecessor tile's
 * look-back word gives up after a bounded number of polls and reports
 * PSI_ERR_DEVICE_TIMEOUT) made testable without a GPU fault or hang.  Sorts
 * n (key, value) pairs like psi_sort_pairs (8-bit digits, all 64 key bits),
 * but tile `withheld_tile` (0-based, 4096 pairs per tile; -1: none) of the
 * first digit pass never publishes its look-back words, and a waiting tile
 * gives up after `spin_limit` (>= 1) polls.  Returns PSI_ERR_DEVICE_TIMEOUT
 * when a wait ran out: the arrays' contents are then unspecified (every
 * write stays inside them); PSI_OK and the sorted arrays when no wait did.  The context stays usable either way.
 * Synchronises `stream`.  No counterpart in the paper: a test facility. */
psi_status psi_test_sort_withheld_tile(uint64_t *d_keys, uint32_t *d_vals, int64_t n, int64_t withheld_tile,
                                       uint32_t spin_limit, void *stream);

/* ---- Instrumentation ---------------------------------------------------- */

/* psi_knn with traversal counters: d_stats (device, 5 x uint64) receives the
 * number of internal nodes expanded, leaves scanned, points scanned, queries
 * answered and child descriptors read (children evaluated by the expanded
 * nodes).  Same results as psi_knn; slower (atomic counters). */
psi_status psi_knn_instrumented(const psi_index *ix, const int32_t *d_q, int64_t q, int32_t k, uint32_t *d_ids,
                                int64_t *d_d2, uint64_t *d_stats, void *stream);

/* psi_batch_knn with the same five traversal counters (summed over all
 * indexes); d_stats must be zeroed by the caller. */
psi_status psi_batch_knn_instrumented(psi_batch *b, const int32_t *d_q, const int64_t *d_qoffsets, int64_t nq,
                                      int32_t k, uint32_t *d_ids, int64_t *d_d2, uint64_t *d_stats, void *stream);

/* ---- P-Orth over float coordinates, without space-filling curves ------- */
/*
 * The P-Orth of Sec 3 / Algorithm 1 for float32 coordinates in D = 2..5
 * dimensions, built by splitting regions at their midpoints (no Morton keys,
 * so coordinates need not be integers).  The root region is H = [lo, hi)^D;
 * the midpoint of [lo, hi) is lo + 0.5f * (hi - lo) in float arithmetic (each
 * operation rounded to nearest) and a point takes the upper half of a
 * dimension iff its coordinate >= the midpoint; child c takes the upper half of
 * dimension d iff bit d of c is set; a child exists iff it holds a point; a
 * node is a leaf iff it holds at most leaf_size points, is at depth max_depth,
 * or some midpoint is not strictly inside its range (precision exhausted).
 * Nodes are numbered breadth first (children consecutive in child order).
 * k-NN distances are sum over d of (double(q_d) - double(p_d))^2 with every
 * operation rounded to nearest, in dimension order; ties by id; k > size pads
 * with id 0xFFFFFFFF and +inf.  Range boxes are closed ([q][2][D]: lo then hi).
 * An insert or delete rebuilds the tree from the updated point set (the tree
 * is a function of the set, Sec 3.2), synchronising the stream; builds
 * synchronise once per tree level.  Points outside H: PSI_ERR_RANGE.
 */
typedef struct psi_forth psi_forth;
typedef struct {
  int32_t dim;       /* 2..5 */
  int32_t leaf_size; /* 1..64 */
  int32_t max_depth; /* 0..48 */
  float lo[8], hi[8]; /* root region H, first dim entries used, lo < hi */
} psi_fconfig;

psi_status psi_forth_build(const psi_fconfig *cfg, const float *d_pts /*[n][dim]*/, const uint32_t *d_ids, int64_t n,
                           void *stream, psi_forth **out);
psi_status psi_forth_insert(psi_forth *ix, const float *d_pts, const uint32_t *d_ids, int64_t m, void *stream);
/* Deletes the (coordinates, id) pairs present; *d_num_deleted (device) gets their number. */
psi_status psi_forth_delete(psi_forth *ix, const float *d_pts, const uint32_t *d_ids, int64_t m,
                            int64_t *d_num_deleted, void *stream);
psi_status psi_forth_knn(const psi_forth *ix, const float *d_q /*[q][dim]*/, int64_t q, int32_t k,
                         uint32_t *d_ids /*[q][k]*/, double *d_d2 /*[q][k]*/, void *stream);
psi_status psi_forth_range_count(const psi_forth *ix, const float *d_boxes, int64_t q, int64_t *d_counts,
                                 void *stream);
int64_t psi_forth_size(const psi_forth *ix);
int64_t psi_forth_num_nodes(const psi_forth *ix);
/* Node arrays (depth, count, number of children, ref = first child or, for a
 * leaf, first point slot; boxes [N][dim]) and the points in slot order
 * ([n][dim], ids); any pointer may be null. */
psi_status psi_forth_export(const psi_forth *ix, int32_t *d_depth, int32_t *d_count, int32_t *d_kids, uint32_t *d_ref,
                            float *d_lo, float *d_hi, float *d_pts, uint32_t *d_ids, void *stream);
/* Waits for `stream`; reports a device-detected error (traversal overflow). */
psi_status psi_forth_sync(psi_forth *ix, void *stream);
void psi_forth_destroy(psi_forth *ix);

/* Number of kernels this library has launched in the process. */
int64_t psi_launch_count(void);

/* When on, every launch of a library kernel is bracketed by CUDA events on its
 * stream; psi_profile_read() synchronises and reports, for the kernel named
 * `name`, the number of launches and their summed duration since the last
 * psi_profile_reset().  Names are those in the ncu launch list. */
void psi_profile_enable(int on);
void psi_profile_reset(void);
int psi_profile_read(const char *name, int64_t *launches, double *total_ms);
/* Writes "name launches total_ms\n" lines for every kernel seen into buf. */
int psi_profile_dump(char *buf, int64_t cap);

#ifdef __cplusplus
}
#endif
#endif /* PSI_H */

/*
 * psi_oracle.h -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.
 *
 * A plain, sequential, deliberately slow CPU restatement of the operations of
 * "Parallel Dynamic Spatial Indexes" (PPoPP '26, arXiv 2601.05347).  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load this library.  It shares no code, header, table or helper with the CUDA
 * library, and the CUDA library never calls it.
 *
 * Every coordinate is an int32 in [0, 2^bits); keys are uint64; squared
 * distances are exact int64; ids are uint32 and unique among live points.
 */
#ifndef PSI_ORACLE_H
#define PSI_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_SPAC_Z = 0, OR_SPAC_H = 1, OR_PORTH = 2 };

typedef struct {
  int dim;     /* 2 or 3 */
  int kind;    /* OR_SPAC_Z, OR_SPAC_H or OR_PORTH */
  int phi;     /* leaf wrap (leaf size bound) */
  int bits;    /* coordinate bits b: coordinates lie in [0, 2^b) */
  int fanout;  /* fanout F of the summary tree over the leaves */
} or_cfg;

/* Space-filling-curve keys (Sec 2.2 "Spatial Filling Curves"). */
uint64_t or_morton(const int32_t *p, int dim, int bits);
uint64_t or_hilbert2(int32_t x, int32_t y, int bits);
/* Skilling's 3D Hilbert index of (x, y, z) at `bits` bits per axis. */
uint64_t or_hilbert3(int32_t x, int32_t y, int32_t z, int bits);
/* Keys of n points under cfg (Morton for SPAC_Z and PORTH, Hilbert for SPAC_H).
 * Returns 0, or -1 if a coordinate lies outside [0, 2^bits). */
int or_keys(const or_cfg *cfg, const int32_t *pts, int64_t n, uint64_t *keys);

typedef struct or_index or_index;

or_index *or_build(const or_cfg *cfg, const int32_t *pts, const uint32_t *ids, int64_t n);
void or_free(or_index *ix);
int64_t or_size(const or_index *ix);
void or_insert(or_index *ix, const int32_t *pts, const uint32_t *ids, int64_t m);
int64_t or_delete(or_index *ix, const int32_t *pts, const uint32_t *ids, int64_t m);

/* Live points in (key, id) order: keys[n], ids[n], pts[n][dim]. */
void or_points(const or_index *ix, uint64_t *keys, uint32_t *ids, int32_t *pts);

/* Canonical leaf blocking and summary tree (Algorithm 3, BuildSorted).
 * Level 0 holds the leaves; level l+1 node j summarises level-l nodes
 * [j*F, (j+1)*F).  or_level_size(ix, l) is 0 past the root level. */
int or_num_levels(const or_index *ix);
int64_t or_level_size(const or_index *ix, int level);
/* lo/hi are [size][dim]; count is [size]; first_key/first_id only for level 0 (may be NULL). */
void or_level(const or_index *ix, int level, int32_t *lo, int32_t *hi, int64_t *count,
              uint64_t *first_key, uint32_t *first_id);

/* Queries (Sec 2.2 "Queries on Spatial Data"). */
void or_knn(const or_index *ix, const int32_t *q, int64_t nq, int k, uint32_t *out_ids, int64_t *out_d2);
void or_knn_brute(const or_index *ix, const int32_t *q, int64_t nq, int k, uint32_t *out_ids, int64_t *out_d2);
void or_range_count(const or_index *ix, const int32_t *boxes, int64_t nq, int64_t *counts);
void or_range_count_brute(const or_index *ix, const int32_t *boxes, int64_t nq, int64_t *counts);
/* Writes offsets[nq+1]; ids (each query's ids ascending) only if the total fits in cap.
 * Returns the total number of reported ids. */
int64_t or_range_report(const or_index *ix, const int32_t *boxes, int64_t nq, int64_t *offsets,
                        uint32_t *ids, int64_t cap);

/* P-Orth tree over the live points (Algorithm 1), nodes in preorder.
 * Returns the number of nodes; arrays are filled only if cap is large enough. */
int64_t or_porth(const or_index *ix, int64_t cap, int32_t *depth, uint64_t *prefix, int64_t *count,
                 int32_t *lo, int32_t *hi, int32_t *is_leaf);

/* Definitions over raw arrays (no index): k-NN and range count. */
void or_knn_brute_raw(const int32_t *pts, const uint32_t *ids, int64_t n, int dim, const int32_t *q, int64_t nq,
                      int k, uint32_t *out_ids, int64_t *out_d2);
void or_range_count_brute_raw(const int32_t *pts, int64_t n, int dim, const int32_t *boxes, int64_t nq,
                              int64_t *counts);

/* ---- SFC-free P-Orth over float coordinates (psi_oracle_f.c) ---------- */
#define OR_FMAXD 8
typedef struct {
  int dim;       /* 2 .. OR_FMAXD */
  int phi;       /* leaf bound */
  int max_depth; /* a node at this depth is a leaf */
  float lo[OR_FMAXD], hi[OR_FMAXD]; /* root region H = [lo, hi) */
} or_fcfg;
typedef struct or_forth or_forth;
/* NULL if a point lies outside H. */
or_forth *or_forth_build(const or_fcfg *cfg, const float *pts, const uint32_t *ids, int64_t n);
void or_forth_free(or_forth *t);
int64_t or_forth_num_nodes(const or_forth *t);
/* Node arrays in breadth-first order; leaf_first[u] = offset of leaf u's ids
 * (ascending) in leaf_ids, -1 for internal nodes; boxes are [node][dim]. */
void or_forth_export(const or_forth *t, int32_t *depth, int64_t *count, int32_t *kids, int32_t *is_leaf, float *blo,
                     float *bhi, int64_t *leaf_first, uint32_t *leaf_ids);
void or_fknn_brute(const float *pts, const uint32_t *ids, int64_t n, int dim, const float *q, int64_t nq, int k,
                   uint32_t *out_ids, double *out_d2);
void or_frange_count_brute(const float *pts, int64_t n, int dim, const float *boxes, int64_t nq, int64_t *counts);

#ifdef __cplusplus
}
#endif
#endif

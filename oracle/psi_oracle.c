/*
 * psi_oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.
 *
 * Plain sequential restatement of "Parallel Dynamic Spatial Indexes" (PPoPP '26,
 * arXiv 2601.05347), used only to check the CUDA library.  Nothing here is
 * blocked, fused or reordered for speed.  The index is a sorted array of
 * (key, id, point) records; every update re-derives the canonical layout from
 * that array.  Each function names the passage it follows.
 *
 * Readings of passages the paper leaves open:
 *   - Morton bit order: key bit D*i + d is bit i of coordinate d (x lowest).
 *   - Hilbert orientation: Hilbert's 1891 curve starting at (0,0), visiting the
 *     quadrants lower-left, upper-left, upper-right, lower-right, ending at
 *     (2^b - 1, 0).  In 3D: Skilling's curve (see or_hilbert3), from (0,0,0)
 *     to (2^b - 1, 0, 0).
 *   - A node is a leaf iff it holds at most phi points (P-Orth: or it is a
 *     single cell at depth b).
 *   - Ties in key are ordered by id; k-NN ties in distance are ordered by id.
 *   - Range boxes are closed on both ends; a box with lo > hi is empty.
 */
#include "psi_oracle.h"

#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Space-filling curves (Sec 2.2, "Spatial Filling Curves")                   */
/* ------------------------------------------------------------------------- */

/* Z-curve: interleave the coordinate bits, bit i of coordinate d becoming key
 * bit D*i + d. */
uint64_t or_morton(const int32_t *p, int dim, int bits) {
  uint64_t key = 0;
  for (int i = 0; i < bits; ++i)
    for (int d = 0; d < dim; ++d) {
      uint64_t bit = ((uint64_t)(uint32_t)p[d] >> i) & 1u;
      key |= bit << (dim * i + d);
    }
  return key;
}

/* Hilbert curve of order `bits`, by recursive subdivision of the square.  At
 * each level the current square of side 2s is cut into four quadrants that the
 * curve visits in the order lower-left (0), upper-left (1), upper-right (2),
 * lower-right (3).  Inside the lower-left quadrant the curve is the next-order
 * curve mirrored about the diagonal (x <-> y); inside the lower-right one it is
 * mirrored about the anti-diagonal (x -> s-1-y, y -> s-1-x); inside the two
 * upper quadrants it is the next-order curve translated. */
uint64_t or_hilbert2(int32_t x, int32_t y, int bits) {
  uint64_t d = 0;
  int64_t X = x, Y = y;
  for (int level = bits - 1; level >= 0; --level) {
    int64_t s = (int64_t)1 << level;
    int rx = X >= s, ry = Y >= s;
    int q;
    if (!rx && !ry)
      q = 0;
    else if (!rx && ry)
      q = 1;
    else if (rx && ry)
      q = 2;
    else
      q = 3;
    d = d * 4 + (uint64_t)q;
    if (rx) X -= s;
    if (ry) Y -= s;
    if (q == 0) {
      int64_t t = X;
      X = Y;
      Y = t;
    } else if (q == 3) {
      int64_t t = X;
      X = s - 1 - Y;
      Y = s - 1 - t;
    }
  }
  return d;
}

/* 3D Hilbert curve.  The paper defines Hilbert keys in 2D only; in 3D the
 * curve is read as Skilling's (J. Skilling, "Programming the Hilbert curve",
 * AIP Conf. Proc. 707, 2004) with axes X0 = x, X1 = y, X2 = z.  His method, on
 * whole coordinate words:
 *   1. from the top bit level down to level 1, for each axis i in turn: if
 *      bit l of X_i is set, complement the bits of X_0 below l; otherwise
 *      exchange the bits below l between X_0 and X_i;
 *   2. Gray-code across the axes (X_i ^= X_{i-1} for i = 1, 2), then
 *      complement, at every level, the bits below each set bit of X_2;
 *   3. the key reads the transposed words level by level, top level first,
 *      X_0's bit the most significant of each three-bit digit. */
uint64_t or_hilbert3(int32_t x, int32_t y, int32_t z, int bits) {
  uint32_t X[3] = {(uint32_t)x, (uint32_t)y, (uint32_t)z};
  for (int level = bits - 1; level >= 1; --level) {
    uint32_t bit = (uint32_t)1 << level, below = bit - 1;
    for (int i = 0; i < 3; ++i) {
      if (X[i] & bit) {
        X[0] ^= below;
      } else {
        uint32_t diff = (X[0] ^ X[i]) & below;
        X[0] ^= diff;
        X[i] ^= diff;
      }
    }
  }
  X[1] ^= X[0];
  X[2] ^= X[1];
  uint32_t flip = 0;
  for (int level = bits - 1; level >= 1; --level)
    if (X[2] & ((uint32_t)1 << level)) flip ^= ((uint32_t)1 << level) - 1;
  for (int i = 0; i < 3; ++i) X[i] ^= flip;
  uint64_t key = 0;
  for (int level = bits - 1; level >= 0; --level)
    for (int i = 0; i < 3; ++i) key = (key << 1) | ((X[i] >> level) & 1u);
  return key;
}

static int in_domain(const int32_t *p, int dim, int bits) {
  for (int d = 0; d < dim; ++d)
    if (p[d] < 0 || (int64_t)p[d] >= ((int64_t)1 << bits)) return 0;
  return 1;
}

static uint64_t key_of(const or_cfg *cfg, const int32_t *p) {
  if (cfg->kind == OR_SPAC_H && cfg->dim == 3) return or_hilbert3(p[0], p[1], p[2], cfg->bits);
  if (cfg->kind == OR_SPAC_H) return or_hilbert2(p[0], p[1], cfg->bits);
  return or_morton(p, cfg->dim, cfg->bits);
}

int or_keys(const or_cfg *cfg, const int32_t *pts, int64_t n, uint64_t *keys) {
  for (int64_t i = 0; i < n; ++i) {
    if (!in_domain(pts + i * cfg->dim, cfg->dim, cfg->bits)) return -1;
    keys[i] = key_of(cfg, pts + i * cfg->dim);
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* The index: records sorted by (key, id)                                     */
/* ------------------------------------------------------------------------- */

typedef struct {
  uint64_t key;
  uint32_t id;
  int32_t c[3];
} rec;

#define MAX_LEVELS 64

struct or_index {
  or_cfg cfg;
  int64_t n, cap;
  rec *r;
  int nlev;
  int64_t lsize[MAX_LEVELS];
  int32_t *lo[MAX_LEVELS], *hi[MAX_LEVELS];
  int64_t *cnt[MAX_LEVELS];
};

static int rec_less(const rec *a, const rec *b) {
  if (a->key != b->key) return a->key < b->key;
  return a->id < b->id;
}

static int rec_cmp(const void *pa, const void *pb) {
  const rec *a = (const rec *)pa, *b = (const rec *)pb;
  if (rec_less(a, b)) return -1;
  if (rec_less(b, a)) return 1;
  return 0;
}

static void free_summary(or_index *ix) {
  for (int l = 0; l < ix->nlev; ++l) {
    free(ix->lo[l]);
    free(ix->hi[l]);
    free(ix->cnt[l]);
  }
  ix->nlev = 0;
}

/* Leaf wrapping and bounding boxes (Algorithm 3, BuildSorted): the sorted
 * records are cut into leaves of phi consecutive records (the last one may be
 * shorter).  Above the leaves sits a summary tree whose node j at level l+1
 * covers level-l nodes [j*F, (j+1)*F); every node keeps the tight bounding box
 * (lower-left and upper-right corners, Appendix "Implementation Details") and
 * the point count of its subtree. */
static void derive_summary(or_index *ix) {
  free_summary(ix);
  const int D = ix->cfg.dim, phi = ix->cfg.phi, F = ix->cfg.fanout;
  if (ix->n == 0) return;
  int64_t L = (ix->n + phi - 1) / phi;
  int l = 0;
  ix->lsize[0] = L;
  ix->lo[0] = (int32_t *)malloc(sizeof(int32_t) * L * D);
  ix->hi[0] = (int32_t *)malloc(sizeof(int32_t) * L * D);
  ix->cnt[0] = (int64_t *)malloc(sizeof(int64_t) * L);
  for (int64_t i = 0; i < L; ++i) {
    int64_t b = i * phi, e = b + phi < ix->n ? b + phi : ix->n;
    ix->cnt[0][i] = e - b;
    for (int d = 0; d < D; ++d) {
      int32_t mn = ix->r[b].c[d], mx = ix->r[b].c[d];
      for (int64_t j = b; j < e; ++j) {
        if (ix->r[j].c[d] < mn) mn = ix->r[j].c[d];
        if (ix->r[j].c[d] > mx) mx = ix->r[j].c[d];
      }
      ix->lo[0][i * D + d] = mn;
      ix->hi[0][i * D + d] = mx;
    }
  }
  while (ix->lsize[l] > 1) {
    int64_t S = ix->lsize[l], P = (S + F - 1) / F;
    ++l;
    ix->lsize[l] = P;
    ix->lo[l] = (int32_t *)malloc(sizeof(int32_t) * P * D);
    ix->hi[l] = (int32_t *)malloc(sizeof(int32_t) * P * D);
    ix->cnt[l] = (int64_t *)malloc(sizeof(int64_t) * P);
    for (int64_t j = 0; j < P; ++j) {
      int64_t b = j * F, e = b + F < S ? b + F : S;
      ix->cnt[l][j] = 0;
      for (int d = 0; d < D; ++d) {
        ix->lo[l][j * D + d] = ix->lo[l - 1][b * D + d];
        ix->hi[l][j * D + d] = ix->hi[l - 1][b * D + d];
      }
      for (int64_t c = b; c < e; ++c) {
        ix->cnt[l][j] += ix->cnt[l - 1][c];
        for (int d = 0; d < D; ++d) {
          if (ix->lo[l - 1][c * D + d] < ix->lo[l][j * D + d]) ix->lo[l][j * D + d] = ix->lo[l - 1][c * D + d];
          if (ix->hi[l - 1][c * D + d] > ix->hi[l][j * D + d]) ix->hi[l][j * D + d] = ix->hi[l - 1][c * D + d];
        }
      }
    }
  }
  ix->nlev = l + 1;
}

static void reserve(or_index *ix, int64_t want) {
  if (want <= ix->cap) return;
  int64_t c = ix->cap ? ix->cap : 16;
  while (c < want) c *= 2;
  ix->r = (rec *)realloc(ix->r, sizeof(rec) * c);
  ix->cap = c;
}

static rec make_rec(const or_cfg *cfg, const int32_t *p, uint32_t id) {
  rec t;
  memset(&t, 0, sizeof t);
  t.key = key_of(cfg, p);
  t.id = id;
  for (int d = 0; d < cfg->dim; ++d) t.c[d] = p[d];
  return t;
}

/* Construction (Algorithm 3): compute each point's curve key, sort the
 * (key, id) pairs, then wrap leaves and summarise. */
or_index *or_build(const or_cfg *cfg, const int32_t *pts, const uint32_t *ids, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!in_domain(pts + i * cfg->dim, cfg->dim, cfg->bits)) return NULL;
  or_index *ix = (or_index *)calloc(1, sizeof(or_index));
  ix->cfg = *cfg;
  reserve(ix, n > 0 ? n : 1);
  for (int64_t i = 0; i < n; ++i) ix->r[i] = make_rec(cfg, pts + i * cfg->dim, ids[i]);
  ix->n = n;
  qsort(ix->r, (size_t)n, sizeof(rec), rec_cmp);
  derive_summary(ix);
  return ix;
}

void or_free(or_index *ix) {
  if (!ix) return;
  free_summary(ix);
  free(ix->r);
  free(ix);
}

int64_t or_size(const or_index *ix) { return ix->n; }

/* Batch insertion (Algorithm 4): sort the batch by curve key, then merge it
 * into the ordered point sequence.  The leaf layout is then re-derived. */
void or_insert(or_index *ix, const int32_t *pts, const uint32_t *ids, int64_t m) {
  const or_cfg *cfg = &ix->cfg;
  rec *b = (rec *)malloc(sizeof(rec) * (m > 0 ? m : 1));
  for (int64_t i = 0; i < m; ++i) b[i] = make_rec(cfg, pts + i * cfg->dim, ids[i]);
  qsort(b, (size_t)m, sizeof(rec), rec_cmp);
  rec *out = (rec *)malloc(sizeof(rec) * (ix->n + m > 0 ? ix->n + m : 1));
  int64_t i = 0, j = 0, k = 0;
  while (i < ix->n && j < m) out[k++] = rec_less(&b[j], &ix->r[i]) ? b[j++] : ix->r[i++];
  while (i < ix->n) out[k++] = ix->r[i++];
  while (j < m) out[k++] = b[j++];
  free(ix->r);
  free(b);
  ix->r = out;
  ix->n = k;
  ix->cap = k > 0 ? k : 1;
  derive_summary(ix);
}

/* Batch deletion (Sec 4.2, deletion paragraph): remove each (point, id) that is
 * present; absent pairs are ignored.  Returns the number removed. */
int64_t or_delete(or_index *ix, const int32_t *pts, const uint32_t *ids, int64_t m) {
  const or_cfg *cfg = &ix->cfg;
  char *dead = (char *)calloc((size_t)(ix->n > 0 ? ix->n : 1), 1);
  int64_t removed = 0;
  for (int64_t t = 0; t < m; ++t) {
    const int32_t *p = pts + t * cfg->dim;
    if (!in_domain(p, cfg->dim, cfg->bits)) continue;
    rec want = make_rec(cfg, p, ids[t]);
    int64_t lo = 0, hi = ix->n; /* first record not less than want */
    while (lo < hi) {
      int64_t mid = lo + (hi - lo) / 2;
      if (rec_less(&ix->r[mid], &want))
        lo = mid + 1;
      else
        hi = mid;
    }
    if (lo < ix->n && ix->r[lo].key == want.key && ix->r[lo].id == want.id && !dead[lo]) {
      int same = 1;
      for (int d = 0; d < cfg->dim; ++d) same &= ix->r[lo].c[d] == p[d];
      if (same) {
        dead[lo] = 1;
        ++removed;
      }
    }
  }
  int64_t k = 0;
  for (int64_t i = 0; i < ix->n; ++i)
    if (!dead[i]) ix->r[k++] = ix->r[i];
  ix->n = k;
  free(dead);
  derive_summary(ix);
  return removed;
}

void or_points(const or_index *ix, uint64_t *keys, uint32_t *ids, int32_t *pts) {
  for (int64_t i = 0; i < ix->n; ++i) {
    if (keys) keys[i] = ix->r[i].key;
    if (ids) ids[i] = ix->r[i].id;
    if (pts)
      for (int d = 0; d < ix->cfg.dim; ++d) pts[i * ix->cfg.dim + d] = ix->r[i].c[d];
  }
}

int or_num_levels(const or_index *ix) { return ix->nlev; }

int64_t or_level_size(const or_index *ix, int level) {
  return (level >= 0 && level < ix->nlev) ? ix->lsize[level] : 0;
}

void or_level(const or_index *ix, int level, int32_t *lo, int32_t *hi, int64_t *count,
              uint64_t *first_key, uint32_t *first_id) {
  if (level < 0 || level >= ix->nlev) return;
  const int D = ix->cfg.dim;
  int64_t S = ix->lsize[level];
  memcpy(lo, ix->lo[level], sizeof(int32_t) * S * D);
  memcpy(hi, ix->hi[level], sizeof(int32_t) * S * D);
  memcpy(count, ix->cnt[level], sizeof(int64_t) * S);
  if (level == 0)
    for (int64_t i = 0; i < S; ++i) {
      if (first_key) first_key[i] = ix->r[i * ix->cfg.phi].key;
      if (first_id) first_id[i] = ix->r[i * ix->cfg.phi].id;
    }
}

/* ------------------------------------------------------------------------- */
/* Queries (Sec 2.2 "Queries on Spatial Data"; Appendix "Implementation       */
/* Details": k-NN visits subtrees in increasing order of box distance)        */
/* ------------------------------------------------------------------------- */

static int64_t sqdist(const int32_t *a, const int32_t *b, int D) {
  int64_t s = 0;
  for (int d = 0; d < D; ++d) {
    int64_t t = (int64_t)a[d] - (int64_t)b[d];
    s += t * t;
  }
  return s;
}

/* Smallest squared distance from q to the closed box [lo, hi]. */
static int64_t box_dist(const int32_t *q, const int32_t *lo, const int32_t *hi, int D) {
  int64_t s = 0;
  for (int d = 0; d < D; ++d) {
    int64_t t = 0;
    if (q[d] < lo[d]) t = (int64_t)lo[d] - q[d];
    if (q[d] > hi[d]) t = (int64_t)q[d] - hi[d];
    s += t * t;
  }
  return s;
}

typedef struct {
  int64_t d2;
  uint32_t id;
} cand;

static int cand_less(cand a, cand b) { return a.d2 < b.d2 || (a.d2 == b.d2 && a.id < b.id); }

/* Max-heap of the best k candidates found so far, ordered by (d2, id). */
typedef struct {
  cand *a;
  int n, k;
} topk;

static void topk_push(topk *h, cand c) {
  if (h->n < h->k) {
    int i = h->n++;
    h->a[i] = c;
    while (i > 0 && cand_less(h->a[(i - 1) / 2], h->a[i])) {
      cand t = h->a[i];
      h->a[i] = h->a[(i - 1) / 2];
      h->a[(i - 1) / 2] = t;
      i = (i - 1) / 2;
    }
    return;
  }
  if (!cand_less(c, h->a[0])) return;
  h->a[0] = c;
  int i = 0;
  for (;;) {
    int l = 2 * i + 1, r = l + 1, m = i;
    if (l < h->n && cand_less(h->a[m], h->a[l])) m = l;
    if (r < h->n && cand_less(h->a[m], h->a[r])) m = r;
    if (m == i) break;
    cand t = h->a[i];
    h->a[i] = h->a[m];
    h->a[m] = t;
    i = m;
  }
}

static int cand_cmp(const void *pa, const void *pb) {
  cand a = *(const cand *)pa, b = *(const cand *)pb;
  return cand_less(a, b) ? -1 : (cand_less(b, a) ? 1 : 0);
}

/* Write the k best in ascending (d2, id) order, padding with (UINT32_MAX, INT64_MAX). */
static void topk_emit(topk *h, uint32_t *ids, int64_t *d2) {
  qsort(h->a, (size_t)h->n, sizeof(cand), cand_cmp);
  for (int i = 0; i < h->k; ++i) {
    ids[i] = i < h->n ? h->a[i].id : 0xFFFFFFFFu;
    d2[i] = i < h->n ? h->a[i].d2 : INT64_MAX;
  }
}

/* Min-heap of tree nodes keyed by their box distance (best-first traversal). */
typedef struct {
  int64_t md;
  int level;
  int64_t idx;
} qnode;

typedef struct {
  qnode *a;
  int64_t n, cap;
} pq;

static void pq_push(pq *h, qnode x) {
  if (h->n == h->cap) {
    h->cap = h->cap ? h->cap * 2 : 64;
    h->a = (qnode *)realloc(h->a, sizeof(qnode) * h->cap);
  }
  int64_t i = h->n++;
  h->a[i] = x;
  while (i > 0 && h->a[(i - 1) / 2].md > h->a[i].md) {
    qnode t = h->a[i];
    h->a[i] = h->a[(i - 1) / 2];
    h->a[(i - 1) / 2] = t;
    i = (i - 1) / 2;
  }
}

static qnode pq_pop(pq *h) {
  qnode top = h->a[0];
  h->a[0] = h->a[--h->n];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, m = i;
    if (l < h->n && h->a[l].md < h->a[m].md) m = l;
    if (r < h->n && h->a[r].md < h->a[m].md) m = r;
    if (m == i) break;
    qnode t = h->a[i];
    h->a[i] = h->a[m];
    h->a[m] = t;
    i = m;
  }
  return top;
}

static int64_t child_begin(const or_index *ix, int level, int64_t idx) {
  return level == 0 ? idx * ix->cfg.phi : idx * ix->cfg.fanout;
}

static int64_t child_end(const or_index *ix, int level, int64_t idx) {
  int64_t e = level == 0 ? (idx + 1) * ix->cfg.phi : (idx + 1) * ix->cfg.fanout;
  int64_t lim = level == 0 ? ix->n : ix->lsize[level - 1];
  return e < lim ? e : lim;
}

/* k-NN (Sec 2.2): the k live points closest to q, best-first over the summary
 * tree: nodes leave the queue in increasing box distance, and the search stops
 * once that distance exceeds the current k-th best. */
void or_knn(const or_index *ix, const int32_t *q, int64_t nq, int k, uint32_t *out_ids, int64_t *out_d2) {
  const int D = ix->cfg.dim;
  topk h;
  h.a = (cand *)malloc(sizeof(cand) * (k > 0 ? k : 1));
  h.k = k;
  pq Q = {0, 0, 0};
  for (int64_t t = 0; t < nq; ++t) {
    const int32_t *qp = q + t * D;
    h.n = 0;
    Q.n = 0;
    if (ix->nlev > 0) {
      int top = ix->nlev - 1;
      qnode root = {box_dist(qp, ix->lo[top], ix->hi[top], D), top, 0};
      pq_push(&Q, root);
    }
    while (Q.n > 0) {
      qnode x = pq_pop(&Q);
      if (h.n == h.k && x.md > h.a[0].d2) break;
      int64_t b = child_begin(ix, x.level, x.idx), e = child_end(ix, x.level, x.idx);
      if (x.level == 0) {
        for (int64_t j = b; j < e; ++j) {
          cand c = {sqdist(qp, ix->r[j].c, D), ix->r[j].id};
          topk_push(&h, c);
        }
      } else {
        for (int64_t c = b; c < e; ++c) {
          qnode y = {box_dist(qp, ix->lo[x.level - 1] + c * D, ix->hi[x.level - 1] + c * D, D), x.level - 1, c};
          pq_push(&Q, y);
        }
      }
    }
    topk_emit(&h, out_ids + t * (int64_t)k, out_d2 + t * (int64_t)k);
  }
  free(Q.a);
  free(h.a);
}

/* k-NN by its definition: every live point is a candidate. */
void or_knn_brute(const or_index *ix, const int32_t *q, int64_t nq, int k, uint32_t *out_ids, int64_t *out_d2) {
  const int D = ix->cfg.dim;
  topk h;
  h.a = (cand *)malloc(sizeof(cand) * (k > 0 ? k : 1));
  h.k = k;
  for (int64_t t = 0; t < nq; ++t) {
    h.n = 0;
    for (int64_t j = 0; j < ix->n; ++j) {
      cand c = {sqdist(q + t * D, ix->r[j].c, D), ix->r[j].id};
      topk_push(&h, c);
    }
    topk_emit(&h, out_ids + t * (int64_t)k, out_d2 + t * (int64_t)k);
  }
  free(h.a);
}

static int pt_in_box(const int32_t *p, const int32_t *box, int D) {
  for (int d = 0; d < D; ++d)
    if (p[d] < box[d] || p[d] > box[D + d]) return 0;
  return 1;
}

/* Box relation: 0 disjoint, 1 partial, 2 node box inside the query box. */
static int box_rel(const int32_t *lo, const int32_t *hi, const int32_t *box, int D) {
  int inside = 1;
  for (int d = 0; d < D; ++d) {
    if (hi[d] < box[d] || lo[d] > box[D + d]) return 0;
    if (lo[d] < box[d] || hi[d] > box[D + d]) inside = 0;
  }
  return inside ? 2 : 1;
}

/* Range count (Sec 2.2): subtrees whose box lies inside the query contribute
 * their count; partially overlapping leaves are scanned. */
static int64_t count_rec(const or_index *ix, int level, int64_t idx, const int32_t *box) {
  const int D = ix->cfg.dim;
  int rel = box_rel(ix->lo[level] + idx * D, ix->hi[level] + idx * D, box, D);
  if (rel == 0) return 0;
  if (rel == 2) return ix->cnt[level][idx];
  int64_t b = child_begin(ix, level, idx), e = child_end(ix, level, idx), s = 0;
  for (int64_t c = b; c < e; ++c) s += level == 0 ? pt_in_box(ix->r[c].c, box, D) : count_rec(ix, level - 1, c, box);
  return s;
}

void or_range_count(const or_index *ix, const int32_t *boxes, int64_t nq, int64_t *counts) {
  for (int64_t t = 0; t < nq; ++t)
    counts[t] = ix->nlev > 0 ? count_rec(ix, ix->nlev - 1, 0, boxes + t * 2 * ix->cfg.dim) : 0;
}

void or_range_count_brute(const or_index *ix, const int32_t *boxes, int64_t nq, int64_t *counts) {
  for (int64_t t = 0; t < nq; ++t) {
    counts[t] = 0;
    for (int64_t j = 0; j < ix->n; ++j) counts[t] += pt_in_box(ix->r[j].c, boxes + t * 2 * ix->cfg.dim, ix->cfg.dim);
  }
}

typedef struct {
  uint32_t *a;
  int64_t n, cap;
} idvec;

static void idvec_push(idvec *v, uint32_t x) {
  if (v->n == v->cap) {
    v->cap = v->cap ? v->cap * 2 : 64;
    v->a = (uint32_t *)realloc(v->a, sizeof(uint32_t) * v->cap);
  }
  v->a[v->n++] = x;
}

static void report_rec(const or_index *ix, int level, int64_t idx, const int32_t *box, idvec *out) {
  const int D = ix->cfg.dim;
  if (box_rel(ix->lo[level] + idx * D, ix->hi[level] + idx * D, box, D) == 0) return;
  int64_t b = child_begin(ix, level, idx), e = child_end(ix, level, idx);
  for (int64_t c = b; c < e; ++c) {
    if (level == 0) {
      if (pt_in_box(ix->r[c].c, box, D)) idvec_push(out, ix->r[c].id);
    } else {
      report_rec(ix, level - 1, c, box, out);
    }
  }
}

static int u32_cmp(const void *a, const void *b) {
  uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* Range list (Sec 2.2): all live points inside the closed query box; each
 * query's ids are reported in ascending order. */
int64_t or_range_report(const or_index *ix, const int32_t *boxes, int64_t nq, int64_t *offsets,
                        uint32_t *ids, int64_t cap) {
  idvec all = {0, 0, 0};
  offsets[0] = 0;
  for (int64_t t = 0; t < nq; ++t) {
    int64_t start = all.n;
    if (ix->nlev > 0) report_rec(ix, ix->nlev - 1, 0, boxes + t * 2 * ix->cfg.dim, &all);
    qsort(all.a + start, (size_t)(all.n - start), sizeof(uint32_t), u32_cmp);
    offsets[t + 1] = all.n;
  }
  if (all.n <= cap && ids) memcpy(ids, all.a, sizeof(uint32_t) * all.n);
  int64_t total = all.n;
  free(all.a);
  return total;
}

/* ------------------------------------------------------------------------- */
/* P-Orth tree (Algorithm 1), by recursion over regions                       */
/* ------------------------------------------------------------------------- */

typedef struct {
  const or_index *ix;
  int64_t cap, n;
  int32_t *depth, *lo, *hi, *is_leaf;
  uint64_t *prefix;
  int64_t *count;
  int64_t *tmp;
} porth_ctx;

/* Node of the orth-tree over region [corner, corner + 2^(b - depth))^D holding
 * the records listed in idx[0..cnt).  It is a leaf when it holds at most phi
 * points or is a single cell; otherwise the region is cut at its midpoint in
 * every dimension and the 2^D sub-regions become children, numbered
 * sum_d (p_d in upper half) << d and emitted in that order when non-empty.
 * The root region is the whole domain [0, 2^b)^D. */
static void porth_rec(porth_ctx *C, int64_t *idx, int64_t cnt, int depth, uint64_t prefix, const int64_t *corner) {
  const or_index *ix = C->ix;
  const int D = ix->cfg.dim, bits = ix->cfg.bits;
  int64_t me = C->n++;
  int leaf = cnt <= ix->cfg.phi || depth == bits;
  if (me < C->cap) {
    C->depth[me] = depth;
    C->prefix[me] = prefix;
    C->count[me] = cnt;
    C->is_leaf[me] = leaf;
    for (int d = 0; d < D; ++d) {
      int32_t mn = ix->r[idx[0]].c[d], mx = mn;
      for (int64_t j = 0; j < cnt; ++j) {
        int32_t v = ix->r[idx[j]].c[d];
        if (v < mn) mn = v;
        if (v > mx) mx = v;
      }
      C->lo[me * D + d] = mn;
      C->hi[me * D + d] = mx;
    }
  }
  if (leaf) return;
  int64_t half = (int64_t)1 << (bits - depth - 1);
  int nb = 1 << D;
  int64_t bucket_cnt[8] = {0}, bucket_off[8];
  int64_t *child_of = C->tmp; /* scratch: the child number of each record */
  for (int64_t j = 0; j < cnt; ++j) {
    int c = 0;
    for (int d = 0; d < D; ++d)
      if ((int64_t)ix->r[idx[j]].c[d] >= corner[d] + half) c |= 1 << d;
    child_of[j] = c;
    bucket_cnt[c]++;
  }
  int64_t *sorted = (int64_t *)malloc(sizeof(int64_t) * cnt);
  bucket_off[0] = 0;
  for (int c = 1; c < nb; ++c) bucket_off[c] = bucket_off[c - 1] + bucket_cnt[c - 1];
  {
    int64_t pos[8];
    for (int c = 0; c < nb; ++c) pos[c] = bucket_off[c];
    for (int64_t j = 0; j < cnt; ++j) sorted[pos[child_of[j]]++] = idx[j];
  }
  memcpy(idx, sorted, sizeof(int64_t) * cnt);
  free(sorted);
  for (int c = 0; c < nb; ++c) {
    if (bucket_cnt[c] == 0) continue;
    int64_t sub[3];
    for (int d = 0; d < D; ++d) sub[d] = corner[d] + (((c >> d) & 1) ? half : 0);
    porth_rec(C, idx + bucket_off[c], bucket_cnt[c], depth + 1, (prefix << D) | (uint64_t)c, sub);
  }
}

int64_t or_porth(const or_index *ix, int64_t cap, int32_t *depth, uint64_t *prefix, int64_t *count,
                 int32_t *lo, int32_t *hi, int32_t *is_leaf) {
  if (ix->n == 0) return 0;
  porth_ctx C;
  C.ix = ix;
  C.cap = cap;
  C.n = 0;
  C.depth = depth;
  C.prefix = prefix;
  C.count = count;
  C.lo = lo;
  C.hi = hi;
  C.is_leaf = is_leaf;
  C.tmp = (int64_t *)malloc(sizeof(int64_t) * ix->n);
  int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * ix->n);
  for (int64_t j = 0; j < ix->n; ++j) idx[j] = j;
  int64_t corner[3] = {0, 0, 0};
  porth_rec(&C, idx, ix->n, 0, 0, corner);
  free(idx);
  free(C.tmp);
  return C.n;
}

/* ------------------------------------------------------------------------- */
/* Definitions over raw point arrays (for sampled checks at full size)        */
/* ------------------------------------------------------------------------- */

/* k-NN by definition over n points pts[n][dim] with ids[n]. */
void or_knn_brute_raw(const int32_t *pts, const uint32_t *ids, int64_t n, int dim, const int32_t *q, int64_t nq,
                      int k, uint32_t *out_ids, int64_t *out_d2) {
  topk h;
  h.a = (cand *)malloc(sizeof(cand) * (k > 0 ? k : 1));
  h.k = k;
  for (int64_t t = 0; t < nq; ++t) {
    h.n = 0;
    for (int64_t j = 0; j < n; ++j) {
      cand c = {sqdist(q + t * dim, pts + j * dim, dim), ids[j]};
      topk_push(&h, c);
    }
    topk_emit(&h, out_ids + t * (int64_t)k, out_d2 + t * (int64_t)k);
  }
  free(h.a);
}

/* Range count by definition over raw points. */
void or_range_count_brute_raw(const int32_t *pts, int64_t n, int dim, const int32_t *boxes, int64_t nq,
                              int64_t *counts) {
  for (int64_t t = 0; t < nq; ++t) {
    counts[t] = 0;
    for (int64_t j = 0; j < n; ++j) counts[t] += pt_in_box(pts + j * dim, boxes + t * 2 * dim, dim);
  }
}

/*
 * psi_oracle_f.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.
 *
 * Plain sequential restatement of the P-Orth construction of "Parallel Dynamic
 * Spatial Indexes" (PPoPP '26, arXiv 2601.05347) for floating-point coordinates,
 * without space-filling curves (Sec 3.1, Algorithm 1: a node's region is split
 * at its midpoint in every dimension; a node holding at most phi points is a
 * leaf).  Written as a breadth-first recursion over regions, so it shares
 * nothing with the CUDA library's level-synchronous partition.  Compile with
 * -ffp-contract=off: every float and double operation is rounded on its own.
 *
 * Readings of passages the paper leaves open:
 *   - The root region H = [lo, hi)^D is given by the caller; every point must
 *     lie in it.
 *   - Midpoint of [lo, hi): mid = lo + 0.5f * (hi - lo) in float arithmetic; a
 *     point goes to the upper half of a dimension iff its coordinate >= mid.
 *   - Child c of a node takes the upper half of dimension d iff bit d of c is
 *     set.  A child exists iff it holds a point.
 *   - A node is a leaf iff it holds at most phi points, or it is at depth
 *     max_depth, or some dimension can no longer be split (mid is not strictly
 *     inside (lo, hi): float precision is exhausted).
 *   - Nodes are numbered breadth first: a node's children are consecutive, in
 *     child-number order, and the nodes of one depth are ordered by parent.
 *   - Squared distances are sum over d of (double(q_d) - double(p_d))^2,
 *     accumulated in dimension order with every operation rounded to nearest;
 *     k-NN ties in distance are ordered by id; range boxes are closed.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "psi_oracle.h"

typedef struct {
  int64_t *idx; /* indices of the node's points, input order */
  int64_t cnt;
  float lo[OR_FMAXD], hi[OR_FMAXD];
  int depth;
} fjob;

struct or_forth {
  int dim;
  int64_t n_nodes, cap;
  int32_t *depth, *kids, *is_leaf;
  int64_t *count, *first; /* internal: id of the first child; leaf: offset of its ids in leaf_ids */
  float *blo, *bhi;       /* [n_nodes][dim] tight boxes */
  uint32_t *leaf_ids;     /* each leaf's ids, ascending */
  int64_t n_leaf_ids;
};

static float midpoint(float lo, float hi) {
  float w = hi - lo;
  float h = 0.5f * w;
  return lo + h;
}

static int cmp_u32(const void *a, const void *b) {
  uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
  return x < y ? -1 : (x > y);
}

static void grow(or_forth *t) {
  int64_t c = t->cap ? 2 * t->cap : 64;
  t->depth = (int32_t *)realloc(t->depth, sizeof(int32_t) * c);
  t->kids = (int32_t *)realloc(t->kids, sizeof(int32_t) * c);
  t->is_leaf = (int32_t *)realloc(t->is_leaf, sizeof(int32_t) * c);
  t->count = (int64_t *)realloc(t->count, sizeof(int64_t) * c);
  t->first = (int64_t *)realloc(t->first, sizeof(int64_t) * c);
  t->blo = (float *)realloc(t->blo, sizeof(float) * c * t->dim);
  t->bhi = (float *)realloc(t->bhi, sizeof(float) * c * t->dim);
  t->cap = c;
}

or_forth *or_forth_build(const or_fcfg *cfg, const float *pts, const uint32_t *ids, int64_t n) {
  const int D = cfg->dim;
  if (D < 2 || D > OR_FMAXD || cfg->phi < 1) return NULL;
  for (int64_t i = 0; i < n; ++i)
    for (int d = 0; d < D; ++d) {
      float x = pts[i * D + d];
      if (!(x >= cfg->lo[d] && x < cfg->hi[d])) return NULL; /* outside H (or NaN) */
    }
  or_forth *t = (or_forth *)calloc(1, sizeof(or_forth));
  t->dim = D;
  t->leaf_ids = (uint32_t *)malloc(sizeof(uint32_t) * (n > 0 ? n : 1));
  if (n == 0) return t;

  /* breadth-first queue of regions; queue position = node id */
  int64_t qcap = 64, qn = 0;
  fjob *q = (fjob *)malloc(sizeof(fjob) * qcap);
  fjob root;
  root.idx = (int64_t *)malloc(sizeof(int64_t) * n);
  for (int64_t i = 0; i < n; ++i) root.idx[i] = i;
  root.cnt = n;
  root.depth = 0;
  for (int d = 0; d < D; ++d) {
    root.lo[d] = cfg->lo[d];
    root.hi[d] = cfg->hi[d];
  }
  q[qn++] = root;
  for (int64_t u = 0; u < qn; ++u) {
    if (t->n_nodes == t->cap) grow(t);
    fjob j = q[u];
    t->n_nodes = u + 1;
    t->depth[u] = j.depth;
    t->count[u] = j.cnt;
    float mid[OR_FMAXD];
    int exhausted = 0;
    for (int d = 0; d < D; ++d) {
      mid[d] = midpoint(j.lo[d], j.hi[d]);
      if (!(j.lo[d] < mid[d] && mid[d] < j.hi[d])) exhausted = 1;
    }
    if (j.cnt <= cfg->phi || j.depth >= cfg->max_depth || exhausted) {
      t->is_leaf[u] = 1;
      t->kids[u] = 0;
      t->first[u] = t->n_leaf_ids;
      float *lo = t->blo + u * D, *hi = t->bhi + u * D; /* tight box of the leaf's points */
      for (int d = 0; d < D; ++d) {
        lo[d] = INFINITY;
        hi[d] = -INFINITY;
      }
      for (int64_t i = 0; i < j.cnt; ++i)
        for (int d = 0; d < D; ++d) {
          const float x = pts[j.idx[i] * D + d];
          if (x < lo[d]) lo[d] = x;
          if (x > hi[d]) hi[d] = x;
        }
      for (int64_t i = 0; i < j.cnt; ++i) t->leaf_ids[t->n_leaf_ids + i] = ids[j.idx[i]];
      qsort(t->leaf_ids + t->n_leaf_ids, (size_t)j.cnt, sizeof(uint32_t), cmp_u32);
      t->n_leaf_ids += j.cnt;
    } else {
      t->is_leaf[u] = 0;
      t->first[u] = qn;
      int kids = 0;
      for (int c = 0; c < (1 << D); ++c) {
        fjob ch;
        ch.idx = (int64_t *)malloc(sizeof(int64_t) * j.cnt);
        ch.cnt = 0;
        ch.depth = j.depth + 1;
        for (int d = 0; d < D; ++d) {
          int up = (c >> d) & 1;
          ch.lo[d] = up ? mid[d] : j.lo[d];
          ch.hi[d] = up ? j.hi[d] : mid[d];
        }
        for (int64_t i = 0; i < j.cnt; ++i) {
          const float *p = pts + j.idx[i] * D;
          int mine = 1;
          for (int d = 0; d < D; ++d) mine &= ((p[d] >= mid[d]) == (((c >> d) & 1) != 0));
          if (mine) ch.idx[ch.cnt++] = j.idx[i];
        }
        if (ch.cnt == 0) {
          free(ch.idx);
          continue;
        }
        if (qn == qcap) {
          qcap *= 2;
          q = (fjob *)realloc(q, sizeof(fjob) * qcap);
        }
        q[qn++] = ch;
        ++kids;
      }
      t->kids[u] = kids;
    }
    free(q[u].idx);
    q[u].idx = NULL;
  }
  free(q);

  /* internal boxes: union of the children's, children before parents
   * (children have larger ids) */
  for (int64_t u = t->n_nodes - 1; u >= 0; --u) {
    if (t->is_leaf[u]) continue;
    float *lo = t->blo + u * D, *hi = t->bhi + u * D;
    for (int d = 0; d < D; ++d) {
      lo[d] = INFINITY;
      hi[d] = -INFINITY;
    }
    for (int64_t c = t->first[u]; c < t->first[u] + t->kids[u]; ++c)
      for (int d = 0; d < D; ++d) {
        if (t->blo[c * D + d] < lo[d]) lo[d] = t->blo[c * D + d];
        if (t->bhi[c * D + d] > hi[d]) hi[d] = t->bhi[c * D + d];
      }
  }
  return t;
}

void or_forth_free(or_forth *t) {
  if (!t) return;
  free(t->depth);
  free(t->kids);
  free(t->is_leaf);
  free(t->count);
  free(t->first);
  free(t->blo);
  free(t->bhi);
  free(t->leaf_ids);
  free(t);
}

int64_t or_forth_num_nodes(const or_forth *t) { return t ? t->n_nodes : 0; }

void or_forth_export(const or_forth *t, int32_t *depth, int64_t *count, int32_t *kids, int32_t *is_leaf, float *blo,
                     float *bhi, int64_t *leaf_first, uint32_t *leaf_ids) {
  for (int64_t u = 0; u < t->n_nodes; ++u) {
    depth[u] = t->depth[u];
    count[u] = t->count[u];
    kids[u] = t->kids[u];
    is_leaf[u] = t->is_leaf[u];
    leaf_first[u] = t->is_leaf[u] ? t->first[u] : -1;
    for (int d = 0; d < t->dim; ++d) {
      blo[u * t->dim + d] = t->blo[u * t->dim + d];
      bhi[u * t->dim + d] = t->bhi[u * t->dim + d];
    }
  }
  memcpy(leaf_ids, t->leaf_ids, sizeof(uint32_t) * (size_t)t->n_leaf_ids);
}

/* Squared distance as defined above. */
static double fsqdist(const float *q, const float *p, int D) {
  double s = 0.0;
  for (int d = 0; d < D; ++d) {
    double t = (double)q[d] - (double)p[d];
    double sq = t * t;
    s = s + sq;
  }
  return s;
}

typedef struct {
  double d;
  uint32_t id;
} fcand;

static int fcand_less(fcand a, fcand b) { return a.d < b.d || (a.d == b.d && a.id < b.id); }

/* k-NN by definition: the first min(k, n) points by (distance, id); padded
 * with (+inf, 0xFFFFFFFF). */
void or_fknn_brute(const float *pts, const uint32_t *ids, int64_t n, int dim, const float *q, int64_t nq, int k,
                   uint32_t *out_ids, double *out_d2) {
  fcand *best = (fcand *)malloc(sizeof(fcand) * (k > 0 ? k : 1));
  for (int64_t t = 0; t < nq; ++t) {
    int have = 0;
    for (int64_t j = 0; j < n; ++j) {
      fcand c = {fsqdist(q + t * dim, pts + j * dim, dim), ids[j]};
      if (have == k && !fcand_less(c, best[k - 1])) continue;
      int pos = have < k ? have : k - 1;
      while (pos > 0 && fcand_less(c, best[pos - 1])) {
        best[pos] = best[pos - 1];
        --pos;
      }
      best[pos] = c;
      if (have < k) ++have;
    }
    for (int r = 0; r < k; ++r) {
      out_ids[t * k + r] = r < have ? best[r].id : 0xFFFFFFFFu;
      out_d2[t * k + r] = r < have ? best[r].d : INFINITY;
    }
  }
  free(best);
}

/* Points inside closed boxes [lo, hi] (boxes[q][2][dim]); lo > hi anywhere: empty. */
void or_frange_count_brute(const float *pts, int64_t n, int dim, const float *boxes, int64_t nq, int64_t *counts) {
  for (int64_t t = 0; t < nq; ++t) {
    const float *lo = boxes + t * 2 * dim, *hi = lo + dim;
    int64_t c = 0;
    for (int64_t j = 0; j < n; ++j) {
      int in = 1;
      for (int d = 0; d < dim; ++d) in &= pts[j * dim + d] >= lo[d] && pts[j * dim + d] <= hi[d];
      c += in;
    }
    counts[t] = c;
  }
}

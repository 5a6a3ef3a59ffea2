// query.cu -- batched k-NN, range count and range list (Sec 2.2) on either
// tree layout (SPaC summary tree or P-Orth), one warp per query, queries taken
// in curve order so that neighbouring warps walk the same nodes out of L2.
//
// k-NN: depth-first traversal that enters children in increasing order of
// their box distance (Appendix "Implementation Details": subtrees are visited
// in increasing minimum distance to the query) and prunes a subtree whose box
// is farther than the current k-th best.  A node's children are evaluated one
// per lane; each level of the current path keeps its children's distance keys
// and a bitmask of those still to visit in shared memory, and a warp minimum
// picks the next one.  The search starts from seed leaves at the query's own
// curve position (SPaC; P-Orth for k > 32).  The k best (d2, id) pairs live in
// a KList (klist.cuh).  Squared distances are exact int64 (|dx| < 2^31 for
// coordinates in [0, 2^31)).
//
// Range count: children inside the box add their subtree count; children that
// straddle the box are descended; straddling leaves are scanned.
// Range list: the same traversal counts first; after an exclusive scan of the
// counts a second traversal writes each query's ids at its offset (a
// subtree inside the box is enumerated without further box tests).
#include "bitonic.cuh"
#include "index.cuh"
#include "keys.cuh"
#include "klist.cuh"

namespace psi {

// Curve order of a query batch and its sorted keys; owns the sort buffers.
struct QueryOrder {
  Buf<uint64_t> k0, k1;
  Buf<uint32_t> v0, v1;
  const uint32_t *order = nullptr;
  const uint64_t *keys = nullptr;
  int key_shift = 0;
};

namespace {

constexpr int QW = 4;         // warps per block
constexpr int STACK = 256;    // stack entries per warp (>= depth * fanout)
constexpr uint32_t INSIDE = 0x80000000u;

// Pruning key of a child box: the float bits of a lower bound of its squared
// distance to the query, computed on the FP32 pipe (the ALU pipe is the
// k-NN kernel's bottleneck): each gap is an exact int32 difference converted,
// squared and summed with rounding toward -inf, so the bound never exceeds the
// exact distance; a float at or below the exact k-th distance is at or below
// that distance rounded to nearest, so comparing float bits never prunes a box
// that holds a neighbour.
template <int D>
__device__ __forceinline__ uint32_t box_key(const TreeView &t, uint32_t node, const int32_t *qc) {
  float s = 0.0f;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int32_t lo = t.lo[d][node], hi = t.hi[d][node], q = qc[d];
    const int32_t g = q < lo ? lo - q : (q > hi ? q - hi : 0);
    const float gf = __int2float_rd(g);
    s = __fadd_rd(s, __fmul_rd(gf, gf));
  }
  return __float_as_uint(s);
}

// 0: disjoint, 1: straddles, 2: node box inside the query box.
template <int D>
__device__ __forceinline__ int box_relation(const TreeView &t, uint32_t node, const int32_t *blo, const int32_t *bhi) {
  bool inside = true, disjoint = false;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int32_t lo = t.lo[d][node], hi = t.hi[d][node];
    disjoint |= hi < blo[d] || lo > bhi[d];
    inside &= blo[d] <= lo && hi <= bhi[d];
  }
  return disjoint ? 0 : (inside ? 2 : 1);
}

struct KnnArgs {
  TreeView t;
  const int32_t *q;
  int64_t nq;
  int k;
  const uint32_t *order;
  const int32_t *qroot;  // per-query root (many indexes in one node array), or null
  KnnSeed seed;        // SPaC: leaves scanned before the search
  int64_t leaf_limit;  // >= 0: the leaves are exactly the nodes [0, leaf_limit) (one SPaC index)
  uint32_t *out_id;
  int64_t *out_d2;
  int *status;
};

// Scan one leaf: every point whose (d2, id) beats the current k-th enters the
// list (klist_offer: in bulk when many enter at once, the seed leaves of a
// query; one at a time otherwise).
// Slots [s0, s0 + cnt), except those in [skip_lo, skip_hi) (already scanned).
template <int D, int KPL>
__device__ __forceinline__ void knn_scan_slots(const TreeView &t, uint32_t s0, int cnt, const int32_t *qc,
                                               KList<KPL> &kl, int k, uint32_t skip_lo = 1, uint32_t skip_hi = 0) {
  const int lane = threadIdx.x & 31;
  for (int b = 0; b < cnt; b += 32) {
    const int s = b + lane;
    int64_t d2 = INT64_MAX;
    uint32_t id = 0xFFFFFFFFu;
    const uint32_t sl = s0 + (uint32_t)s;
    const bool valid = s < cnt && !(sl >= skip_lo && sl < skip_hi);
    if (valid) {
      const uint32_t slot = s0 + (uint32_t)s;
      id = t.pid[slot];
      d2 = 0;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int64_t dd = (int64_t)t.px[d][slot] - qc[d];
        d2 += dd * dd;
      }
    }
    klist_offer(kl, valid && kl.admits(d2, id), d2, id, k);
  }
}

template <int D, int KPL>
__device__ __forceinline__ void knn_scan_leaf(const TreeView &t, uint32_t node, const int32_t *qc, KList<KPL> &kl,
                                              int k, uint32_t skip_lo = 1, uint32_t skip_hi = 0) {
  knn_scan_slots<D, KPL>(t, t.ref[node], t.cnt[node], qc, kl, k, skip_lo, skip_hi);
}

// Monotone non-decreasing 32-bit image of a non-negative distance (its float
// bits, rounded to nearest).  a <= b implies key(a) <= key(b), so skipping a
// node whose key exceeds key(k-th distance) never skips one that could hold a
// neighbour; it may keep a few that cannot, which costs time, not exactness.
__device__ __forceinline__ uint32_t order_key(int64_t md) { return __float_as_uint((float)md); }

struct KnnStats {
  unsigned long long *c;  // [0] internal nodes expanded, [1] leaves scanned, [2] points scanned, [3] queries
};

constexpr int MAXLVL = 33;  // tree depth bound (P-Orth: 31 levels below the root)

// Last leaf j in [0, L) whose first key (>> shift) is <= key, or 0: a 32-ary
// search by the warp, one ballot over 32 evenly spaced leaves per round.
template <typename FirstKey>
__device__ __forceinline__ int64_t seed_leaf(FirstKey first_key, int64_t L, uint64_t key, int shift) {
  const int lane = threadIdx.x & 31;
  int64_t lo = 0, hi = L;  // the answer lies in [lo, hi)
  while (hi - lo > 1) {
    const int64_t step = (hi - lo + 31) >> 5;
    const int64_t p = lo + (int64_t)lane * step;
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, p < hi && (first_key(p) >> shift) <= key);
    if (m == 0) return lo;  // only when lo == 0: the key precedes every leaf
    lo += (int64_t)(31 - __clz(m)) * step;
    hi = min(hi, lo + step);
  }
  return lo;
}

// One warp per query: depth-first search that always enters the nearest
// not-yet-visited child (Appendix "Implementation Details": children in
// increasing box distance).  Each level of the current path keeps, in shared
// memory, its children's distance keys and a bitmask of children still to
// visit; one ballot prunes every remaining child farther than the current
// k-th distance, one reduce picks the nearest.
// Seed (SPaC): the leaf that holds the query's own curve position is scanned
// first.  SPaC leaves are consecutive runs of the curve and their boxes
// overlap, so the nearest box is often not the leaf around the query; the
// curve neighbours make the k-th distance nearly final before the search
// starts, and the search then skips the seed leaf.
template <int D, int KPL, bool STATS>
__global__ __launch_bounds__(QW * 32) void k_knn(KnnArgs a, KnnStats stats) {
  __shared__ uint32_t s_key[QW][MAXLVL][32];
  __shared__ uint32_t s_c0[QW][MAXLVL];
  __shared__ uint32_t s_mask[QW][MAXLVL];
  __shared__ uint32_t s_leaf[QW][MAXLVL];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t nw = (int64_t)gridDim.x * QW;
  const TreeView &t = a.t;
  unsigned long long n_int = 0, n_leaf = 0, n_pts = 0;
  for (int64_t qi = (int64_t)blockIdx.x * QW + w; qi < a.nq; qi += nw) {
    const int64_t q = a.order ? (int64_t)a.order[qi] : qi;
    int32_t qc[D];
#pragma unroll
    for (int d = 0; d < D; ++d) qc[d] = a.q[q * D + d];
    KList<KPL> kl;
    kl.init();
    const int32_t root = a.qroot ? a.qroot[q] : t.root;
    // seed leaves [s_lo, s_hi]: the leaf at the query's curve position, widened
    // along the curve until it holds at least k points
    int64_t s_lo = 0, s_hi = -1;
    const KnnSeed &sd = a.seed;
    int64_t lb = 0, L = sd.L;  // the query's leaves are nodes [lb, lb + L)
    if (sd.qkey && sd.qseg) {
      const int sg = sd.qseg[q];
      lb = sd.node_off[sg];
      L = (sd.off[sg + 1] - sd.off[sg] + sd.phi - 1) / sd.phi;
    }
    // P-Orth (k > 32): the 32 * KPL points of the key-sorted pool around the
    // query's key are scanned first, 32 at a time, and skipped point by point
    // afterwards
    const bool by_slots = sd.pkey && sd.n_slots > 0;
    uint32_t sk_lo = 1, sk_hi = 0;
    if (sd.qkey && root >= 0) {
      const uint64_t key = sd.qkey[qi] & sd.qkey_mask;
      if (by_slots) {
        const int64_t pos = seed_leaf([&](int64_t p) { return sd.pkey[p]; }, sd.n_slots, key, sd.key_shift);
        const int64_t want = min((int64_t)32 * KPL, sd.n_slots);
        const int64_t lo = max((int64_t)0, min(pos - want / 2, sd.n_slots - want));
        sk_lo = (uint32_t)lo;
        sk_hi = (uint32_t)(lo + want);
        knn_scan_slots<D, KPL>(t, sk_lo, (int)want, qc, kl, a.k);
        if (STATS) n_pts += want;
      } else if (L > 0) {
        const int64_t j = lb + (sd.sep_key ? seed_leaf([&](int64_t p) { return sd.sep_key[p]; }, L, key, sd.key_shift)
                                           : seed_leaf([&](int64_t p) { return sd.pkey[t.ref[lb + p]]; }, L, key,
                                                       sd.key_shift));
        const int64_t le = lb + L;
        int64_t got = 0;
        s_lo = j;
        s_hi = j - 1;
        while (got < a.k && (s_lo > lb || s_hi + 1 < le)) {
          int64_t nx;
          if (s_hi < s_lo || (s_hi + 1 < le && (s_lo == lb || s_hi - j <= j - s_lo)))
            nx = ++s_hi;
          else
            nx = --s_lo;
          knn_scan_leaf<D, KPL>(t, (uint32_t)nx, qc, kl, a.k);
          got += t.cnt[nx];
          if (STATS) {
            ++n_leaf;
            n_pts += t.cnt[nx];
          }
        }
      }
    }
    auto seeded = [&](uint32_t leaf) { return !by_slots && (int64_t)leaf >= s_lo && (int64_t)leaf <= s_hi; };
    uint32_t kdk = order_key(kl.kd);
    auto expand = [&](uint32_t node, int lvl) {
      const int nk = t.kids[node];
      const uint32_t c0 = t.ref[node];
      const uint32_t c = c0 + (uint32_t)lane;
      uint32_t key = 0xFFFFFFFFu;
      bool leafc = false;
      if (lane < nk) {  // every node of every layout holds a point
        key = box_key<D>(t, c, qc);
        leafc = a.leaf_limit >= 0 ? (int64_t)c < a.leaf_limit : t.kids[c] == 0;
      }
      s_key[w][lvl][lane] = key;
      const uint32_t mk = __ballot_sync(0xFFFFFFFFu, key <= kdk);
      const uint32_t lf = __ballot_sync(0xFFFFFFFFu, leafc);
      if (lane == 0) {
        s_c0[w][lvl] = c0;
        s_mask[w][lvl] = mk;
        s_leaf[w][lvl] = lf;
      }
      if (STATS) ++n_int;
      __syncwarp();
    };
    if (root >= 0) {
      if (t.kids[root] == 0) {
        if (!seeded((uint32_t)root)) knn_scan_leaf<D, KPL>(t, (uint32_t)root, qc, kl, a.k, sk_lo, sk_hi);
      } else {
        int lvl = 0;
        expand((uint32_t)root, 0);
        while (lvl >= 0) {
          const uint32_t key = s_key[w][lvl][lane];
          const uint32_t m = s_mask[w][lvl] & __ballot_sync(0xFFFFFFFFu, key <= kdk);
          if (m == 0) {
            --lvl;
            continue;
          }
          const bool in = (m >> lane) & 1u;
          const uint32_t mn = __reduce_min_sync(0xFFFFFFFFu, in ? key : 0xFFFFFFFFu);
          const int src = __ffs(__ballot_sync(0xFFFFFFFFu, in && key == mn)) - 1;
          const uint32_t child = s_c0[w][lvl] + (uint32_t)src;
          const bool is_leaf = (s_leaf[w][lvl] >> src) & 1u;
          __syncwarp();
          if (lane == 0) s_mask[w][lvl] = m & ~(1u << src);
          __syncwarp();
          if (is_leaf) {
            if (seeded(child)) continue;  // scanned as a seed
            knn_scan_leaf<D, KPL>(t, child, qc, kl, a.k, sk_lo, sk_hi);
            kdk = order_key(kl.kd);
            if (STATS) {
              ++n_leaf;
              n_pts += t.cnt[child];
            }
          } else if (lvl + 1 < MAXLVL) {
            ++lvl;
            expand(child, lvl);
          } else if (lane == 0) {
            atomicOr(a.status, ST_STACK);
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < KPL; ++r) {
      const int e = r * 32 + lane;
      if (e < a.k) {
        a.out_id[q * a.k + e] = kl.i[r];
        a.out_d2[q * a.k + e] = kl.d[r];
      }
    }
    if (STATS && lane == 0) atomicAdd(&stats.c[3], 1ull);
  }
  if (STATS && lane == 0) {
    atomicAdd(&stats.c[0], n_int);
    atomicAdd(&stats.c[1], n_leaf);
    atomicAdd(&stats.c[2], n_pts);
  }
}

struct RangeArgs {
  TreeView t;
  const int32_t *boxes;
  int64_t nq;
  int64_t *counts;          // count pass
  const int64_t *offsets;   // emit pass
  uint32_t *out_ids;
  int *status;
};

template <int D>
__device__ __forceinline__ bool point_in(const TreeView &t, uint32_t slot, const int32_t *blo, const int32_t *bhi) {
  bool in = true;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int32_t c = t.px[d][slot];
    in &= c >= blo[d] && c <= bhi[d];
  }
  return in;
}

// EMIT = false: count; EMIT = true: write ids.
template <int D, bool EMIT>
__global__ __launch_bounds__(QW * 32) void k_range(RangeArgs a) {
  __shared__ uint32_t s_node[QW][STACK];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t nw = (int64_t)gridDim.x * QW;
  const TreeView &t = a.t;
  for (int64_t q = (int64_t)blockIdx.x * QW + w; q < a.nq; q += nw) {
    int32_t blo[D], bhi[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      blo[d] = a.boxes[q * 2 * D + d];
      bhi[d] = a.boxes[q * 2 * D + D + d];
    }
    int64_t acc = 0;                               // count pass: per-lane partial
    int64_t cursor = EMIT ? a.offsets[q] : 0;      // emit pass: warp-uniform
    int sp = 0;
    if (t.root >= 0) {
      const int rel = box_relation<D>(t, (uint32_t)t.root, blo, bhi);
      if (rel == 2 && !EMIT) {
        if (lane == 0) acc += t.cnt[t.root];
      } else if (rel != 0) {
        if (lane == 0) s_node[w][0] = (uint32_t)t.root | (rel == 2 ? INSIDE : 0u);
        sp = 1;
      }
    }
    __syncwarp();
    while (sp > 0) {
      --sp;
      const uint32_t e = s_node[w][sp];
      __syncwarp();
      const uint32_t node = e & ~INSIDE;
      const bool inside = (e & INSIDE) != 0;
      const int nk = t.kids[node];
      if (nk == 0) {
        const uint32_t s0 = t.ref[node];
        const int cnt = t.cnt[node];
        for (int b = 0; b < cnt; b += 32) {
          const int s = b + lane;
          const bool hit = s < cnt && (inside || point_in<D>(t, s0 + (uint32_t)s, blo, bhi));
          if (!EMIT) {
            acc += hit;
          } else {
            const uint32_t m = __ballot_sync(0xFFFFFFFFu, hit);
            if (hit) a.out_ids[cursor + __popc(m & lanemask_lt())] = t.pid[s0 + s];
            cursor += __popc(m);
          }
        }
        continue;
      }
      const uint32_t c0 = t.ref[node];
      for (int cb = 0; cb < nk; cb += 32) {
        uint32_t push = 0xFFFFFFFFu;
        if (cb + lane < nk) {
          const uint32_t c = c0 + (uint32_t)(cb + lane);
          const int rel = inside ? 2 : box_relation<D>(t, c, blo, bhi);
          if (rel == 2 && !EMIT)
            acc += t.cnt[c];
          else if (rel != 0)
            push = c | (rel == 2 ? INSIDE : 0u);
        }
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, push != 0xFFFFFFFFu);
        if (sp + __popc(m) > STACK) {
          if (lane == 0) atomicOr(a.status, ST_STACK);
          break;
        }
        if (push != 0xFFFFFFFFu) s_node[w][sp + __popc(m & lanemask_lt())] = push;
        sp += __popc(m);
        __syncwarp();
      }
    }
    if (!EMIT) {
      for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
      if (lane == 0) a.counts[q] = acc;
    }
  }
}

// One block per query segment: ascending sort of its ids.
__global__ __launch_bounds__(1024) void k_sort_segments(const int64_t *offsets, int64_t nq, uint32_t *ids) {
  __shared__ uint32_t sv[4096];
  for (int64_t q = blockIdx.x; q < nq; q += gridDim.x) {
    const int64_t b = offsets[q], len = offsets[q + 1] - b;
    if (len <= 1) continue;
    if (len <= 4096) {
      for (int64_t j = threadIdx.x; j < len; j += blockDim.x) sv[j] = ids[b + j];
      __syncthreads();
      bitonic_ascending(
          len, [&](int64_t x, int64_t y) { return sv[x] < sv[y]; },
          [&](int64_t x, int64_t y) {
            const uint32_t tmp = sv[x];
            sv[x] = sv[y];
            sv[y] = tmp;
          });
      for (int64_t j = threadIdx.x; j < len; j += blockDim.x) ids[b + j] = sv[j];
      __syncthreads();
    } else {
      uint32_t *v = ids + b;
      bitonic_ascending(
          len, [&](int64_t x, int64_t y) { return v[x] < v[y]; },
          [&](int64_t x, int64_t y) {
            const uint32_t tmp = v[x];
            v[x] = v[y];
            v[y] = tmp;
          });
    }
  }
}

int query_grid(int64_t nq) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nq, QW), (int64_t)num_sms() * 16));
}

}  // namespace

// Sorts the query points along the index's curve so that neighbouring warps
// traverse neighbouring parts of the tree; returns the permutation in *order
// and the sorted keys (curve key >> *key_shift) in *qkeys.
psi_status query_order(const psi_index *ix, const int32_t *q, int64_t nq, QueryOrder &qo, cudaStream_t s) {
  qo.order = nullptr;
  qo.keys = nullptr;
  if (nq < 4096) return PSI_OK;
  psi_status st;
  if ((st = qo.k0.alloc(nq, s)) || (st = qo.k1.alloc(nq, s)) || (st = qo.v0.alloc(nq, s)) ||
      (st = qo.v1.alloc(nq, s)))
    return st;
  // locality only needs the top bits of the curve key: 48 bits, 6 digit passes
  EncodeSpec e = encode_spec(ix, q);
  const int order_bits = std::min(48, ix->key_bits);
  e.key_shift = ix->key_bits - order_bits;
  SortResult r;
  if ((st = sort_pairs(e, nullptr, nullptr, nq, order_bits, nullptr, qo.k0.p, qo.v0.p, qo.k1.p, qo.v1.p,
                       ix->d_status, s, &r)))
    return st;
  qo.order = r.vals;
  qo.keys = r.keys;
  qo.key_shift = e.key_shift;
  return PSI_OK;
}

psi_status run_knn_roots(const TreeView &tv, const int32_t *q, int64_t nq, int k, const uint32_t *order,
                         const int32_t *qroot, int D, uint32_t *out_id, int64_t *out_d2, int *status,
                         unsigned long long *d_stats, cudaStream_t s, const KnnSeed &seed, int64_t leaf_limit) {
  if (nq == 0) return PSI_OK;
  KnnArgs a{tv, q, nq, k, order, qroot, seed, leaf_limit, out_id, out_d2, status};
  KnnStats stats{d_stats};
  const int g = query_grid(nq);
  const int kpl = k <= 32 ? 1 : (k <= 64 ? 2 : 4);
#define KNN_CASE(DD, KK)                                                                     \
  do {                                                                                       \
    if (d_stats)                                                                             \
      PSI_LAUNCH_NAMED("k_knn_stats", (k_knn<DD, KK, true>), g, QW * 32, 0, s, a, stats);   \
    else                                                                                     \
      PSI_LAUNCH_NAMED("k_knn", (k_knn<DD, KK, false>), g, QW * 32, 0, s, a, stats);        \
  } while (0)
  if (D == 2) {
    if (kpl == 1) KNN_CASE(2, 1);
    else if (kpl == 2) KNN_CASE(2, 2);
    else KNN_CASE(2, 4);
  } else {
    if (kpl == 1) KNN_CASE(3, 1);
    else if (kpl == 2) KNN_CASE(3, 2);
    else KNN_CASE(3, 4);
  }
#undef KNN_CASE
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}



psi_status run_knn(const psi_index *ix, const int32_t *q, int64_t nq, int k, uint32_t *out_id, int64_t *out_d2,
                   unsigned long long *d_stats, cudaStream_t s) {
  if (nq == 0) return PSI_OK;
  QueryOrder qo;
  psi_status st = query_order(ix, q, nq, qo, s);
  if (st) return st;
  KnnSeed seed;
  if (qo.keys) {
    seed.qkey = qo.keys;
    seed.L = ix->L;
    seed.key_shift = qo.key_shift;
    if (ix->cfg.kind == PSI_PORTH) {
      // P-Orth leaves do not overlap and the search is near its floor; the
      // seed pays off only in cutting single insertions into long lists
      if (k <= 32) seed.qkey = nullptr;
      seed.pkey = ix->pool.pkey;
      seed.n_slots = ix->n;
    } else {
      seed.sep_key = ix->sep_key;
    }
  }
  return run_knn_roots(ix->view(), q, nq, k, qo.order, nullptr, ix->D, out_id, out_d2, ix->d_status, d_stats, s,
                       seed, ix->cfg.kind == PSI_PORTH ? -1 : ix->L);
}

psi_status run_range_count(const psi_index *ix, const int32_t *boxes, int64_t nq, int64_t *counts, cudaStream_t s) {
  if (nq == 0) return PSI_OK;
  RangeArgs a{ix->view(), boxes, nq, counts, nullptr, nullptr, ix->d_status};
  const int g = query_grid(nq);
  if (ix->D == 2)
    PSI_LAUNCH_NAMED("k_range_count", (k_range<2, false>), g, QW * 32, 0, s, a);
  else
    PSI_LAUNCH_NAMED("k_range_count", (k_range<3, false>), g, QW * 32, 0, s, a);
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}

psi_status run_range_emit(const psi_index *ix, const int32_t *boxes, int64_t nq, const int64_t *offsets,
                          uint32_t *ids, bool sorted, cudaStream_t s) {
  if (nq == 0) return PSI_OK;
  RangeArgs a{ix->view(), boxes, nq, nullptr, offsets, ids, ix->d_status};
  const int g = query_grid(nq);
  if (ix->D == 2)
    PSI_LAUNCH_NAMED("k_range_emit", (k_range<2, true>), g, QW * 32, 0, s, a);
  else
    PSI_LAUNCH_NAMED("k_range_emit", (k_range<3, true>), g, QW * 32, 0, s, a);
  if (sorted)
    PSI_LAUNCH(k_sort_segments, (int)std::min<int64_t>(nq, (int64_t)num_sms() * 2), 1024, 0, s, offsets, nq, ids);
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}

}  // namespace psi

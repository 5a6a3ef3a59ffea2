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
#include <type_traits>

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
  uint32_t *spare = nullptr;  // nq free words (the key buffer the sort left unused)
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
__device__ __forceinline__ uint32_t box_key_of(const int32_t *lo, const int32_t *hi, const int32_t *qc) {
  float s = 0.0f;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int32_t q = qc[d];
    const int32_t g = q < lo[d] ? lo[d] - q : (q > hi[d] ? q - hi[d] : 0);
    const float gf = __int2float_rd(g);
    s = __fadd_rd(s, __fmul_rd(gf, gf));
  }
  return __float_as_uint(s);
}

template <int D>
__device__ __forceinline__ uint32_t box_key(const TreeView &t, uint32_t node, const int32_t *qc) {
  int32_t lo[D], hi[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    lo[d] = t.lo[d][node];
    hi[d] = t.hi[d][node];
  }
  return box_key_of<D>(lo, hi, qc);
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
// Slots [s0, s0 + cnt).
// EMPTY: the list is known to be empty (the first leaf a query scans).
template <int D, int KPL, bool EMPTY = false>
__device__ __forceinline__ void knn_scan_slots(const TreeView &t, uint32_t s0, int cnt, const int32_t *qc,
                                               KList<KPL> &kl, int k) {
  const int lane = threadIdx.x & 31;
  for (int b = 0; b < cnt; b += 32) {
    const int s = b + lane;
    int64_t d2 = INT64_MAX;
    uint32_t id = 0xFFFFFFFFu;
    const bool valid = s < cnt;
    if (valid) {
      const uint32_t slot = s0 + (uint32_t)s;
      id = t.pid[slot];
      d2 = 0;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        // both in [0, 2^31): the difference is exact in 32 bits, its square
        // one widening multiply
        const int32_t dd = t.px[d][slot] - qc[d];
        d2 += (int64_t)dd * dd;
      }
    }
    if (EMPTY && b == 0)  // the list holds nothing yet: every point enters
      klist_fill(kl, valid, d2, id, k);
    else
      klist_offer(kl, valid && kl.admits(d2, id), d2, id, k);
  }
}

template <int D, int KPL, bool EMPTY = false>
__device__ __forceinline__ void knn_scan_leaf(const TreeView &t, uint32_t node, const int32_t *qc, KList<KPL> &kl,
                                              int k) {
  knn_scan_slots<D, KPL, EMPTY>(t, t.ref[node], t.cnt[node], qc, kl, k);
}

// 32-bit image of a non-negative distance for pruning: the float bits of the
// distance rounded up, built from its two 32-bit halves (a conversion from a
// 64-bit integer would run on the FP64 unit, which is very slow on this GPU).
// A child key is its box distance rounded down, so a child whose key exceeds
// the image of the k-th distance is farther than that distance: pruning by
// keys never skips a node that could hold a neighbour; it may keep a few that
// cannot, which costs time, not exactness.
__device__ __forceinline__ uint32_t order_key(int64_t md) {
  const uint32_t hi = (uint32_t)((uint64_t)md >> 32), lo = (uint32_t)md;
  return __float_as_uint(__fmaf_ru(__uint2float_ru(hi), 4294967296.0f, __uint2float_ru(lo)));
}

struct KnnStats {
  // [0] internal nodes expanded, [1] leaves scanned, [2] points scanned, [3] queries,
  // [4] child descriptors read (children evaluated by the expansions)
  unsigned long long *c;
};

// Per-warp depth-first stack of the k-NN search: an expanded node pushes at
// most F - 1 more entries than it pops, so depth x 31 + 32 entries suffice
// (SPaC: 7 levels at 1e9 points; P-Orth: at most 2^D children per level).
constexpr int KSTACK = 256;
// Queries per warp of the grouped k-NN kernel (k <= 32, queries in curve order).
constexpr int kGroup = 2;
// Flag of a stack entry that is a leaf to scan (in its count word).
constexpr uint32_t kLeafEntry = 0x80000000u;

// Last position p in [0, n) whose first key (>> shift) is <= key, or 0 when
// the key precedes every position (binary search by one thread).
template <typename FirstKey>
__device__ __forceinline__ int64_t seed_search(FirstKey first_key, int64_t n, uint64_t key, int shift) {
  int64_t lo = 0, hi = n;  // first position whose first key is greater
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((first_key(mid) >> shift) <= key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo > 0 ? lo - 1 : 0;
}

// Seed position of every query (queries in curve order), one thread each:
// SPaC, the node of the last leaf of the query's index whose first key is at
// most the query's key; P-Orth, the position in the key-ordered leaf list of
// the last leaf whose cell starts at or before the query's key.  Many
// independent searches in flight hide the dependent loads that one warp-wide
// search per query would wait on.
__global__ void k_knn_seed(const KnnSeed sd, const uint32_t *ref, const uint32_t *order, int64_t nq, uint32_t *pos) {
  for (int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; qi < nq; qi += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = sd.qkey[qi] & sd.qkey_mask;
    int64_t p = 0;
    if (sd.qseg) {
      const int64_t q = order ? (int64_t)order[qi] : qi;
      const int sg = sd.qseg[q];
      const int64_t lb = sd.node_off[sg];
      const int64_t L = (sd.off[sg + 1] - sd.off[sg] + sd.phi - 1) / sd.phi;
      if (L > 0) p = lb + seed_search([&](int64_t x) { return sd.pkey[ref[lb + x]]; }, L, key, sd.key_shift);
    } else if (sd.L > 0) {
      p = seed_search([&](int64_t x) { return sd.sep_key[x]; }, sd.L, key, sd.key_shift);
    }
    pos[qi] = (uint32_t)p;
  }
}

// One warp per query: depth-first search over a per-warp stack in shared
// memory.  Expanding a node evaluates its children one per lane and pushes
// those not farther than the current k-th distance, the nearest one on top, so
// the search enters the nearest child first (Appendix "Implementation
// Details": children in increasing box distance) and takes its siblings later,
// each re-checked against the k-th distance of that moment when it is popped.
// Seed (SPaC): the leaf that holds the query's own curve position is scanned
// first.  SPaC leaves are consecutive runs of the curve and their boxes
// overlap, so the nearest box is often not the leaf around the query; the
// curve neighbours make the k-th distance nearly final before the search
// starts (so the order of the later pops matters little), and the search then
// skips the seed leaves.  Seed (P-Orth): the leaf whose cell holds the query's
// key (or the last leaf before it in key order), alone.
template <int D, int KPL, bool STATS, bool BATCH>
__global__ __launch_bounds__(QW * 32) void k_knn(KnnArgs a, KnnStats stats) {
  // internal nodes still to visit: (node, key, first child, children)
  __shared__ uint4 s_stk[QW][KSTACK];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t nw = (int64_t)gridDim.x * QW;
  const TreeView &t = a.t;
  unsigned long long n_int = 0, n_leaf = 0, n_pts = 0, n_kids = 0;
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
    if (sd.qkey && root >= 0) {
      const int64_t pos = sd.pos[qi];  // k_knn_seed
      if (L > 0) {
        // P-Orth: pos is a position in the key-ordered leaf list
        const int64_t j = sd.leaf_node ? (int64_t)sd.leaf_node[pos] : pos;
        const int64_t le = lb + L;
        knn_scan_leaf<D, KPL, true>(t, (uint32_t)j, qc, kl, a.k);
        int64_t got = t.cnt[j];
        if (STATS) {
          ++n_leaf;
          n_pts += got;
        }
        s_lo = j;
        s_hi = j;
        // widened along the curve only where leaves are consecutive nodes
        // (SPaC; P-Orth's key-order neighbours give a loose bound in 3D and
        // did not cut the leaves its search scans)
        while (!sd.leaf_node && got < a.k && (s_lo > lb || s_hi + 1 < le)) {
          int64_t nx;
          if (s_hi + 1 < le && (s_lo == lb || s_hi - j <= j - s_lo))
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
    // seed leaves as a node range [slo, shi] (empty: slo > shi)
    const uint32_t slo = s_hi < s_lo ? 1u : (uint32_t)s_lo;
    const uint32_t shi = s_hi < s_lo ? 0u : (uint32_t)s_hi;
    uint32_t kdk = order_key(kl.kd);
    int sp = 0;
    // Children [c0, c0 + nk) of an expanded node: the internal ones that may
    // hold a neighbour are pushed (the nearest on top); the leaves that may
    // are scanned at once, nearest first, each re-checked against the k-th
    // distance left by the ones before it.  Where a node has both (P-Orth),
    // only the leaves nearer than every internal survivor are scanned at once
    // and the others are pushed beside the internal ones (count | kLeafEntry),
    // so the search still takes the nearest child first.  A popped leaf entry
    // comes back here as `pl` (its lane 0 stands for the leaf).  Each lane
    // loads its child's reference and count with its box, so a popped entry
    // needs no further load before its own children are read.
    auto expand = [&](uint32_t c0, int nk, bool pl, uint32_t pkey) {
      const uint32_t c = c0 + (uint32_t)lane;
      uint32_t key = 0xFFFFFFFFu;  // above any k-th distance key
      bool leafc = false;
      uint32_t cref = 0;
      int ccnt = 0;
      if (pl) {
        if (lane == 0) {
          key = pkey;
          leafc = true;
          cref = c0;
          ccnt = nk;
        }
      } else if (lane < nk) {  // every node of every layout holds a point
        cref = t.ref[c];
        if (a.leaf_limit >= 0) {
          leafc = (int64_t)c < a.leaf_limit;
          ccnt = leafc ? t.cnt[c] : t.kids[c];
        } else {
          const int ck = t.kids[c], cn = t.cnt[c];
          leafc = ck == 0;
          ccnt = leafc ? cn : ck;
        }
        key = box_key<D>(t, c, qc);
        if (leafc && c >= slo && c <= shi) key = 0xFFFFFFFFu;  // scanned as a seed
      }
      const bool in = key <= kdk;
      if (STATS && !pl) {
        ++n_int;
        n_kids += nk;
      }
      uint32_t mi = __ballot_sync(0xFFFFFFFFu, in && !leafc);
      uint32_t ml = __ballot_sync(0xFFFFFFFFu, in && leafc);
      if (mi && ml) {  // warp-uniform: leaves not nearer than the nearest internal survivor wait
        const uint32_t imin = __reduce_min_sync(0xFFFFFFFFu, ((mi >> lane) & 1u) ? key : 0xFFFFFFFFu);
        const uint32_t defer = __ballot_sync(0xFFFFFFFFu, in && leafc && key >= imin);
        ml &= ~defer;
        mi |= defer;
      }
      if (mi) {
        const int n = __popc(mi);
        if (sp + n > KSTACK) {  // cannot happen within the depth bound above
          if (lane == 0) atomicOr(a.status, ST_STACK);
        } else {
          // the nearest survivor (lowest lane on ties) takes the top slot, the
          // one that held the top slot takes its place
          const bool ii = (mi >> lane) & 1u;
          const uint32_t mn = __reduce_min_sync(0xFFFFFFFFu, ii ? key : 0xFFFFFFFFu);
          const int win = __ffs(__ballot_sync(0xFFFFFFFFu, ii && key == mn)) - 1;
          int pos = __popc(mi & lanemask_lt());
          if (lane == win)
            pos = n - 1;
          else if (pos == n - 1)
            pos = __popc(mi & ((1u << win) - 1u));
          __syncwarp();
          if (ii) s_stk[w][sp + pos] = make_uint4(c, key, cref, (uint32_t)ccnt | (leafc ? kLeafEntry : 0u));
          sp += n;
          __syncwarp();
        }
      }
      // BATCH (P-Orth): leaves in batches, taken nearest first (each still
      // within the k-th distance of that moment) while their points fit one
      // round of 32 lanes, then scanned together, so that small leaves (a few
      // points each in 3D) share one k-list merge; a leaf of more than 32
      // points is a batch of its own, scanned in rounds.  Otherwise (SPaC,
      // whose leaves fill a round) a leaf at a time, each re-checked.
      if constexpr (!BATCH) {
        while (ml) {
          const uint32_t mn = __reduce_min_sync(0xFFFFFFFFu, (ml >> lane) & 1u ? key : 0xFFFFFFFFu);
          if (mn > kdk) break;  // every remaining leaf is farther than the k-th distance
          const int src = __ffs(__ballot_sync(0xFFFFFFFFu, ((ml >> lane) & 1u) && key == mn)) - 1;
          ml &= ~(1u << src);
          const uint32_t lref = __shfl_sync(0xFFFFFFFFu, cref, src);
          const int lcnt = __shfl_sync(0xFFFFFFFFu, ccnt, src);
          knn_scan_slots<D, KPL>(t, lref, lcnt, qc, kl, a.k);
          kdk = order_key(kl.kd);
          if (STATS) {
            ++n_leaf;
            n_pts += lcnt;
          }
        }
      }
      while (BATCH && ml) {
        uint32_t bl = 0;  // the batch's children (lanes)
        int tot = 0;
        while (ml) {
          const uint32_t mn = __reduce_min_sync(0xFFFFFFFFu, (ml >> lane) & 1u ? key : 0xFFFFFFFFu);
          if (mn > kdk) {  // every remaining leaf is farther than the k-th distance
            ml = 0;
            break;
          }
          const int src = __ffs(__ballot_sync(0xFFFFFFFFu, ((ml >> lane) & 1u) && key == mn)) - 1;
          const int c = __shfl_sync(0xFFFFFFFFu, ccnt, src);
          if (bl && tot + c > 32) break;
          bl |= 1u << src;
          ml &= ~(1u << src);
          tot += c;
          if (STATS) {
            ++n_leaf;
            n_pts += c;
          }
          if (tot >= 32) break;
        }
        if (!bl) break;
        // batch position of each member leaf's first point (in lane order)
        const int mine = (bl >> lane) & 1u ? ccnt : 0;
        int incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
          if (lane >= o) incl += y;
        }
        const int excl = incl - mine;
        for (int r = 0; r < tot; r += 32) {
          const int p = r + lane;
          uint32_t slot = 0;
          bool valid = false;
          for (uint32_t mb = bl; mb; mb &= mb - 1) {
            const int b = __ffs(mb) - 1;
            const int eb = __shfl_sync(0xFFFFFFFFu, excl, b);
            const int cb = __shfl_sync(0xFFFFFFFFu, ccnt, b);
            const uint32_t rb = __shfl_sync(0xFFFFFFFFu, cref, b);
            if (p >= eb && p < eb + cb) {
              valid = true;
              slot = rb + (uint32_t)(p - eb);
            }
          }
          int64_t d2 = INT64_MAX;
          uint32_t id = 0xFFFFFFFFu;
          if (valid) {
            id = t.pid[slot];
            d2 = 0;
#pragma unroll
            for (int d = 0; d < D; ++d) {
              const int32_t dd = t.px[d][slot] - qc[d];  // exact: both in [0, 2^31)
              d2 += (int64_t)dd * dd;
            }
          }
          klist_offer(kl, valid && kl.admits(d2, id), d2, id, a.k);
        }
        kdk = order_key(kl.kd);
      }
    };
    if (root >= 0) {
      if (t.kids[root] == 0) {
        if (!((uint32_t)root >= slo && (uint32_t)root <= shi))
          knn_scan_leaf<D, KPL>(t, (uint32_t)root, qc, kl, a.k);
      } else {
        // the root as the first entry: one call site keeps `expand` inlined
        uint32_t c0 = t.ref[root], pkey = 0;
        int nk = t.kids[root];
        bool pl = false;
        for (;;) {
          expand(c0, nk, pl, pkey);
          uint4 e = make_uint4(0, 0, 0, 0);
          bool more = false;
          while (sp > 0) {
            e = s_stk[w][--sp];
            if (e.y <= kdk) {  // else farther than the k-th distance found since the push
              more = true;
              break;
            }
          }
          if (!more) break;
          c0 = e.z;
          nk = (int)(e.w & ~kLeafEntry);
          pl = (e.w & kLeafEntry) != 0;
          pkey = e.y;
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
    atomicAdd(&stats.c[4], n_kids);
  }
}

// Scan one leaf for the queries of a group whose bit is set in qmask (warp-
// uniform): every lane loads one point once and offers it to each of those
// queries' lists.  FILL: the lists are known to be empty (the group's first
// leaf).
template <int D, int G, bool FILL>
__device__ __forceinline__ void knn_scan_group(const TreeView &t, uint32_t s0, int cnt, const int32_t (&qc)[G][D],
                                               KList<1> (&kl)[G], int k, uint32_t qmask) {
  const int lane = threadIdx.x & 31;
  for (int b = 0; b < cnt; b += 32) {
    const int s = b + lane;
    const bool valid = s < cnt;
    int32_t p[D];
    uint32_t id = 0xFFFFFFFFu;
    if (valid) {
      const uint32_t slot = s0 + (uint32_t)s;
      id = t.pid[slot];
#pragma unroll
      for (int d = 0; d < D; ++d) p[d] = t.px[d][slot];
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      if (!((qmask >> g) & 1u)) continue;
      int64_t d2 = INT64_MAX;
      if (valid) {
        d2 = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const int32_t dd = p[d] - qc[g][d];  // exact: both in [0, 2^31)
          d2 += (int64_t)dd * dd;
        }
      }
      if (FILL && b == 0)
        klist_fill(kl[g], valid, d2, id, k);
      else
        klist_offer(kl[g], valid && kl[g].admits(d2, id), d2, id, k);
    }
  }
}

// k-NN for k <= 32 with G consecutive queries (in curve order) per warp.
// Neighbouring queries visit nearly the same nodes and leaves, so the group
// shares one depth-first traversal: each child box is loaded once and tested
// against every query of the group (a child is needed if some query's k-th
// distance admits it), and each leaf's points are loaded once and offered to
// the lists of the queries that need the leaf.  Per query the result is the
// same as k_knn's: exact (distance, id) order, each query pruned by its own
// k-th distance.  Seeds: the distinct seed leaves of the group's queries are
// scanned first, for all of them.
template <int D, int G, bool STATS, bool RECHECK>
__global__ __launch_bounds__(QW * 32) void k_knn_group(KnnArgs a, KnnStats stats) {
  static_assert(G <= 2 || !RECHECK, "a stack entry holds the box keys of two queries");
  // internal nodes still to visit: (first child, children) and, with RECHECK,
  // the box keys of queries 0 and G - 1
  using Entry = typename std::conditional<RECHECK, uint4, uint2>::type;
  __shared__ Entry s_stk[QW][KSTACK];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const TreeView &t = a.t;
  const KnnSeed &sd = a.seed;
  const int64_t ngroups = (a.nq + G - 1) / G;
  unsigned long long n_int = 0, n_leaf = 0, n_pts = 0, n_kids = 0;
  for (int64_t gi = (int64_t)blockIdx.x * QW + w; gi < ngroups; gi += (int64_t)gridDim.x * QW) {
    const int64_t qi0 = gi * G;
    const int ng = (int)min((int64_t)G, a.nq - qi0);
    int32_t qc[G][D];
    uint32_t seed[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int64_t qi = qi0 + min(g, ng - 1);  // a short last group repeats its last query
      const int64_t q = a.order ? (int64_t)a.order[qi] : qi;
#pragma unroll
      for (int d = 0; d < D; ++d) qc[g][d] = a.q[q * D + d];
      seed[g] = !sd.qkey ? 0xFFFFFFFFu : sd.leaf_node ? (uint32_t)sd.leaf_node[sd.pos[qi]] : sd.pos[qi];
    }
    KList<1> kl[G];
#pragma unroll
    for (int g = 0; g < G; ++g) kl[g].init();
    const uint32_t all = (1u << G) - 1u;
    const int32_t root = t.root;
    if (sd.qkey && root >= 0) {
      // the distinct seed leaves (positions are non-decreasing in curve order)
#pragma unroll
      for (int g = 0; g < G; ++g) {
        if (g > 0 && seed[g] == seed[g - 1]) continue;
        const uint32_t j = seed[g];
        if (g == 0)
          knn_scan_group<D, G, true>(t, t.ref[j], t.cnt[j], qc, kl, a.k, all);
        else
          knn_scan_group<D, G, false>(t, t.ref[j], t.cnt[j], qc, kl, a.k, all);
        if (STATS) {
          ++n_leaf;
          n_pts += t.cnt[j];
        }
      }
    }
    uint32_t kdk[G];
#pragma unroll
    for (int g = 0; g < G; ++g) kdk[g] = order_key(kl[g].kd);
    int sp = 0;
    // Children [c0, c0 + nk): the internal ones some query may need are pushed
    // (the one nearest to some query on top); the leaves some query may need
    // are scanned at once, nearest first, for the queries that still need them.
    // With RECHECK (P-Orth), leaves that are not nearer than every internal
    // survivor are pushed too (count | kLeafEntry) and come back as `pl`, as
    // in k_knn.
    auto expand = [&](uint32_t c0, int nk, bool pl, uint32_t pk0, uint32_t pk1) {
      const uint32_t c = c0 + (uint32_t)lane;
      uint32_t key[G];
#pragma unroll
      for (int g = 0; g < G; ++g) key[g] = 0xFFFFFFFFu;
      uint32_t need = 0, mkey = 0xFFFFFFFFu;  // queries that may need the child; its smallest key
      bool leafc = false;
      uint32_t cref = 0;
      int ccnt = 0;
      if (RECHECK && pl) {
        if (lane == 0) {
          key[0] = pk0;
          if (G > 1) key[G - 1] = pk1;
          leafc = true;
          cref = c0;
          ccnt = nk;
#pragma unroll
          for (int g = 0; g < G; ++g)
            if (key[g] <= kdk[g]) {
              need |= 1u << g;
              mkey = min(mkey, key[g]);
            }
        }
      } else if (lane < nk) {
        cref = t.ref[c];
        if (a.leaf_limit >= 0) {
          leafc = (int64_t)c < a.leaf_limit;
          ccnt = leafc ? t.cnt[c] : t.kids[c];
        } else {
          const int ck = t.kids[c], cn = t.cnt[c];
          leafc = ck == 0;
          ccnt = leafc ? cn : ck;
        }
        int32_t lo[D], hi[D];
#pragma unroll
        for (int d = 0; d < D; ++d) {
          lo[d] = t.lo[d][c];
          hi[d] = t.hi[d][c];
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
          key[g] = box_key_of<D>(lo, hi, qc[g]);
          if (key[g] <= kdk[g]) {
            need |= 1u << g;
            mkey = min(mkey, key[g]);
          }
        }
        if (leafc) {
#pragma unroll
          for (int g = 0; g < G; ++g)
            if (c == seed[g]) need = 0;  // scanned as a seed
        }
      }
      if (STATS && !(RECHECK && pl)) {
        ++n_int;
        n_kids += nk;
      }
      uint32_t mi = __ballot_sync(0xFFFFFFFFu, need && !leafc);
      uint32_t ml = __ballot_sync(0xFFFFFFFFu, need && leafc);
      if (RECHECK && mi && ml) {  // warp-uniform
        const uint32_t imin = __reduce_min_sync(0xFFFFFFFFu, ((mi >> lane) & 1u) ? mkey : 0xFFFFFFFFu);
        const uint32_t defer = __ballot_sync(0xFFFFFFFFu, need && leafc && mkey >= imin);
        ml &= ~defer;
        mi |= defer;
      }
      if (mi) {
        const int n = __popc(mi);
        if (sp + n > KSTACK) {  // cannot happen within the depth bound
          if (lane == 0) atomicOr(a.status, ST_STACK);
        } else {
          const bool ii = (mi >> lane) & 1u;
          const uint32_t mn = __reduce_min_sync(0xFFFFFFFFu, ii ? mkey : 0xFFFFFFFFu);
          const int win = __ffs(__ballot_sync(0xFFFFFFFFu, ii && mkey == mn)) - 1;
          int pos = __popc(mi & lanemask_lt());
          if (lane == win)
            pos = n - 1;
          else if (pos == n - 1)
            pos = __popc(mi & ((1u << win) - 1u));
          __syncwarp();
          if (ii) {
            if constexpr (RECHECK)
              s_stk[w][sp + pos] = make_uint4(cref, (uint32_t)ccnt | (leafc ? kLeafEntry : 0u), key[0],
                                              G > 1 ? key[G - 1] : 0xFFFFFFFFu);
            else
              s_stk[w][sp + pos] = make_uint2(cref, (uint32_t)ccnt);
          }
          sp += n;
          __syncwarp();
        }
      }
      while (ml) {
        // queries that still need each remaining leaf under the current bounds
        uint32_t now = 0, nkey = 0xFFFFFFFFu;
        if ((ml >> lane) & 1u) {
#pragma unroll
          for (int g = 0; g < G; ++g)
            if (((need >> g) & 1u) && key[g] <= kdk[g]) {
              now |= 1u << g;
              nkey = min(nkey, key[g]);
            }
        }
        const uint32_t mn = __reduce_min_sync(0xFFFFFFFFu, nkey);
        if (mn == 0xFFFFFFFFu) break;  // no query needs any remaining leaf
        const int src = __ffs(__ballot_sync(0xFFFFFFFFu, now && nkey == mn)) - 1;
        ml &= ~(1u << src);
        const uint32_t qm = __shfl_sync(0xFFFFFFFFu, now, src);
        const uint32_t lref = __shfl_sync(0xFFFFFFFFu, cref, src);
        const int lcnt = __shfl_sync(0xFFFFFFFFu, ccnt, src);
        knn_scan_group<D, G, false>(t, lref, lcnt, qc, kl, a.k, qm);
#pragma unroll
        for (int g = 0; g < G; ++g) kdk[g] = order_key(kl[g].kd);
        if (STATS) {
          ++n_leaf;
          n_pts += lcnt;
        }
      }
    };
    if (root >= 0) {
      if (t.kids[root] == 0) {
        bool sd_root = false;
#pragma unroll
        for (int g = 0; g < G; ++g) sd_root |= seed[g] == (uint32_t)root;
        if (!sd_root) knn_scan_group<D, G, false>(t, t.ref[root], t.cnt[root], qc, kl, a.k, all);
      } else {
        uint32_t c0 = t.ref[root], pk0 = 0, pk1 = 0;
        int nk = t.kids[root];
        bool pl = false;
        for (;;) {  // one call site keeps `expand` inlined
          expand(c0, nk, pl, pk0, pk1);
          // RECHECK: the next entry that some query still needs under its
          // k-th distance of this moment (the others are dropped unexpanded)
          bool more = false;
          while (sp > 0) {
            const Entry e = s_stk[w][--sp];
            bool need = true;
            if constexpr (RECHECK) {
              need = e.z <= kdk[0] || (G > 1 && e.w <= kdk[G - 1]);
              pl = (e.y & kLeafEntry) != 0;
              pk0 = e.z;
              pk1 = e.w;
            }
            if (need) {
              c0 = e.x;
              nk = (int)(e.y & ~kLeafEntry);
              more = true;
              break;
            }
          }
          if (!more) break;
        }
      }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      if (g < ng && lane < a.k) {
        const int64_t q = a.order ? (int64_t)a.order[qi0 + g] : qi0 + g;
        a.out_id[q * a.k + lane] = kl[g].i[0];
        a.out_d2[q * a.k + lane] = kl[g].d[0];
      }
    }
    if (STATS && lane == 0) atomicAdd(&stats.c[3], (unsigned long long)ng);
  }
  if (STATS && lane == 0) {
    atomicAdd(&stats.c[0], n_int);
    atomicAdd(&stats.c[1], n_leaf);
    atomicAdd(&stats.c[2], n_pts);
    atomicAdd(&stats.c[4], n_kids);
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
// One warp per box.  The internal nodes the box reaches wait on a stack as
// (first child, children | INSIDE), taken from their parent's expansion, so a
// pop reads no node record.  Expanding a node loads every child's record and
// box in one round of loads; internal children are pushed, and leaf children
// are scanned at once (slot range and count already in registers): a leaf
// costs one dependent load of its points instead of a trip through the stack.
// The count pass adds the count of a node inside the box without descending.
template <int D, bool EMIT>
__global__ __launch_bounds__(QW * 32) void k_range(RangeArgs a) {
  __shared__ uint2 s_node[QW][STACK];
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
    // the root enters as the one child of a virtual node
    int sp = 0;
    if (t.root >= 0) {
      if (lane == 0) s_node[w][0] = make_uint2((uint32_t)t.root, 1u);
      sp = 1;
    }
    __syncwarp();
    while (sp > 0) {
      --sp;
      const uint2 e = s_node[w][sp];
      __syncwarp();
      const uint32_t c0 = e.x;
      const int nk = (int)(e.y & ~INSIDE);
      const bool inside = (e.y & INSIDE) != 0;
      // children per node: at most 32 (SPaC fanout <= 32, P-Orth 2^D <= 8)
      if (nk > 32 && lane == 0) atomicOr(a.status, ST_STACK);
      bool ok = false, lf = false;
      int rel = 0, ccnt = 0, ck = 0;
      uint32_t cref = 0;
      if (lane < nk) {
        const uint32_t c = c0 + (uint32_t)lane;
        ck = t.kids[c];
        cref = t.ref[c];
        ccnt = t.cnt[c];
        rel = inside ? 2 : box_relation<D>(t, c, blo, bhi);
        lf = ck == 0;
        if (rel == 2 && !EMIT)
          acc += ccnt;
        else
          ok = rel != 0;
      }
      // internal children: pushed
      const bool push = ok && !lf;
      const uint32_t m = __ballot_sync(0xFFFFFFFFu, push);
      if (sp + __popc(m) > STACK) {
        if (lane == 0) atomicOr(a.status, ST_STACK);
        break;
      }
      if (push) s_node[w][sp + __popc(m & lanemask_lt())] = make_uint2(cref, (uint32_t)ck | (rel == 2 ? INSIDE : 0u));
      sp += __popc(m);
      __syncwarp();
      // leaf children: scanned now
      uint32_t ml = __ballot_sync(0xFFFFFFFFu, ok && lf);
      if constexpr (!EMIT) {
        while (ml) {
          const int src = __ffs(ml) - 1;
          ml &= ml - 1;
          const uint32_t s0 = __shfl_sync(0xFFFFFFFFu, cref, src);
          const int cnt = __shfl_sync(0xFFFFFFFFu, ccnt, src);
          const bool lin = __shfl_sync(0xFFFFFFFFu, rel, src) == 2;  // leaf box inside the query box
          for (int b = 0; b < cnt; b += 32) {
            const int s = b + lane;
            acc += s < cnt && (lin || point_in<D>(t, s0 + (uint32_t)s, blo, bhi));
          }
        }
      } else {
        // two leaves per round, each lane's points and ids loaded together, so
        // that the loads of both leaves are in flight at once
        while (ml) {
          const int sa = __ffs(ml) - 1;
          ml &= ml - 1;
          const bool two = ml != 0;
          const int sb = two ? __ffs(ml) - 1 : sa;
          if (two) ml &= ml - 1;
          const uint32_t s0a = __shfl_sync(0xFFFFFFFFu, cref, sa), s0b = __shfl_sync(0xFFFFFFFFu, cref, sb);
          const int cna = __shfl_sync(0xFFFFFFFFu, ccnt, sa);
          const int cnb = two ? __shfl_sync(0xFFFFFFFFu, ccnt, sb) : 0;
          const bool lina = __shfl_sync(0xFFFFFFFFu, rel, sa) == 2, linb = __shfl_sync(0xFFFFFFFFu, rel, sb) == 2;
          // the first 32 slots of both leaves
          const bool va = lane < cna, vb = lane < cnb;
          int32_t pa[D], pb[D];
#pragma unroll
          for (int d = 0; d < D; ++d) {
            pa[d] = va && !lina ? t.px[d][s0a + lane] : 0;
            pb[d] = vb && !linb ? t.px[d][s0b + lane] : 0;
          }
          const uint32_t ia = va ? t.pid[s0a + lane] : 0u, ib = vb ? t.pid[s0b + lane] : 0u;
          bool ha = va, hb = vb;
#pragma unroll
          for (int d = 0; d < D; ++d) {
            ha &= lina || (pa[d] >= blo[d] && pa[d] <= bhi[d]);
            hb &= linb || (pb[d] >= blo[d] && pb[d] <= bhi[d]);
          }
          const uint32_t ma = __ballot_sync(0xFFFFFFFFu, ha);
          if (ha) a.out_ids[cursor + __popc(ma & lanemask_lt())] = ia;
          cursor += __popc(ma);
          const uint32_t mb = __ballot_sync(0xFFFFFFFFu, hb);
          if (hb) a.out_ids[cursor + __popc(mb & lanemask_lt())] = ib;
          cursor += __popc(mb);
          // leaves of more than 32 points: their remaining slots
#pragma unroll 1
          for (int u = 0; u < 2; ++u) {
            const uint32_t s0 = u ? s0b : s0a;
            const int cnt = u ? cnb : cna;
            const bool lin = u ? linb : lina;
            for (int b = 32; b < cnt; b += 32) {
              const int s = b + lane;
              const bool hit = s < cnt && (lin || point_in<D>(t, s0 + (uint32_t)s, blo, bhi));
              const uint32_t hm = __ballot_sync(0xFFFFFFFFu, hit);
              if (hit) a.out_ids[cursor + __popc(hm & lanemask_lt())] = t.pid[s0 + s];
              cursor += __popc(hm);
            }
          }
        }
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

// Grid of a grid-stride query kernel: the blocks that are resident at once
// (a larger grid would run as a second, partly idle wave).
template <typename Kern>
int resident_query_grid(Kern kern, int64_t nq) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, QW * 32, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nq, QW), (int64_t)num_sms() * per_sm));
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
  qo.spare = reinterpret_cast<uint32_t *>(r.keys == qo.k0.p ? qo.k1.p : qo.k0.p);
  return PSI_OK;
}

psi_status run_knn_roots(const TreeView &tv, const int32_t *q, int64_t nq, int k, const uint32_t *order,
                         const int32_t *qroot, int D, uint32_t *out_id, int64_t *out_d2, int *status,
                         unsigned long long *d_stats, cudaStream_t s, const KnnSeed &seed, int64_t leaf_limit,
                         bool porth) {
  if (nq == 0) return PSI_OK;
  KnnArgs a{tv, q, nq, k, order, qroot, seed, leaf_limit, out_id, out_d2, status};
  KnnStats stats{d_stats};
  if (seed.qkey) {
    if (!seed.pos) {
      set_error("k-NN seed without its scratch");
      return PSI_ERR_INVALID;
    }
    const int gs = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nq, 256), (int64_t)num_sms() * 16));
    PSI_LAUNCH(k_knn_seed, gs, 256, 0, s, seed, tv.ref, order, nq, seed.pos);
  }
  const int kpl = k <= 32 ? 1 : (k <= 64 ? 2 : 4);
  // k <= 32 over one tree with queries in curve order: kGroup queries per warp
  if (kpl == 1 && !qroot && order && kGroup > 1) {
#define KNN_GROUP(DD, RC)                                                                                   \
  do {                                                                                                      \
    if (d_stats)                                                                                            \
      PSI_LAUNCH_NAMED("k_knn_stats", (k_knn_group<DD, kGroup, true, RC>),                                  \
                       resident_query_grid(k_knn_group<DD, kGroup, true, RC>, ceil_div(nq, kGroup)), QW * 32, \
                       0, s, a, stats);                                                                     \
    else                                                                                                    \
      PSI_LAUNCH_NAMED("k_knn", (k_knn_group<DD, kGroup, false, RC>),                                       \
                       resident_query_grid(k_knn_group<DD, kGroup, false, RC>, ceil_div(nq, kGroup)), QW * 32, \
                       0, s, a, stats);                                                                     \
  } while (0)
    // Popped nodes are re-checked against the k-th distances where the
    // search pushes many that later bounds rule out: P-Orth, whose nodes mix
    // leaf and internal children at every depth.  SPaC's seeds make the
    // bounds nearly final before the first push, and there the larger stack
    // entries cost more than the re-check saves.
    const bool recheck = porth;
    if (D == 2) {
      if (recheck) KNN_GROUP(2, true);
      else KNN_GROUP(2, false);
    } else {
      if (recheck) KNN_GROUP(3, true);
      else KNN_GROUP(3, false);
    }
#undef KNN_GROUP
    PSI_CK(cudaGetLastError());
    return PSI_OK;
  }
#define KNN_CASE1(DD, KK, BB)                                                                          \
  do {                                                                                                 \
    if (d_stats)                                                                                       \
      PSI_LAUNCH_NAMED("k_knn_stats", (k_knn<DD, KK, true, BB>),                                       \
                       resident_query_grid(k_knn<DD, KK, true, BB>, nq), QW * 32, 0, s, a, stats);     \
    else                                                                                               \
      PSI_LAUNCH_NAMED("k_knn", (k_knn<DD, KK, false, BB>), resident_query_grid(k_knn<DD, KK, false, BB>, nq), \
                       QW * 32, 0, s, a, stats);                                                       \
  } while (0)
  // small leaves in batches where leaves are not one round each (P-Orth)
#define KNN_CASE(DD, KK)                  \
  do {                                    \
    if (porth)                            \
      KNN_CASE1(DD, KK, true);            \
    else                                  \
      KNN_CASE1(DD, KK, false);           \
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
#undef KNN_CASE1
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
    seed.pos = qo.spare;
    seed.sep_key = ix->sep_key;
    if (ix->cfg.kind == PSI_PORTH) {
      // the leaf whose cell holds (or last precedes) the query's key
      seed.sep_key = ix->pl.key;
      seed.leaf_node = ix->leaf_node;
    }
  }
  return run_knn_roots(ix->view(), q, nq, k, qo.order, nullptr, ix->D, out_id, out_d2, ix->d_status, d_stats, s,
                       seed, ix->cfg.kind == PSI_PORTH ? -1 : ix->L, ix->cfg.kind == PSI_PORTH);
}

psi_status run_range_count(const psi_index *ix, const int32_t *boxes, int64_t nq, int64_t *counts, cudaStream_t s) {
  if (nq == 0) return PSI_OK;
  RangeArgs a{ix->view(), boxes, nq, counts, nullptr, nullptr, ix->d_status};
  if (ix->D == 2)
    PSI_LAUNCH_NAMED("k_range_count", (k_range<2, false>), resident_query_grid(k_range<2, false>, nq), QW * 32, 0, s,
                     a);
  else
    PSI_LAUNCH_NAMED("k_range_count", (k_range<3, false>), resident_query_grid(k_range<3, false>, nq), QW * 32, 0, s,
                     a);
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}

psi_status run_range_emit(const psi_index *ix, const int32_t *boxes, int64_t nq, const int64_t *offsets,
                          uint32_t *ids, bool sorted, cudaStream_t s) {
  if (nq == 0) return PSI_OK;
  RangeArgs a{ix->view(), boxes, nq, nullptr, offsets, ids, ix->d_status};
  if (ix->D == 2)
    PSI_LAUNCH_NAMED("k_range_emit", (k_range<2, true>), resident_query_grid(k_range<2, true>, nq), QW * 32, 0, s, a);
  else
    PSI_LAUNCH_NAMED("k_range_emit", (k_range<3, true>), resident_query_grid(k_range<3, true>, nq), QW * 32, 0, s, a);
  if (sorted)
    PSI_LAUNCH(k_sort_segments, (int)std::min<int64_t>(nq, (int64_t)num_sms() * 2), 1024, 0, s, offsets, nq, ids);
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}

}  // namespace psi

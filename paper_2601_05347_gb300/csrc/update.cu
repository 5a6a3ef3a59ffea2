// update.cu -- SPaC batch insertion and deletion (Algorithm 4; Sec 4.2).
//
// The batch is sorted by (key, id) with the same onesweep sort as the build,
// and every batch point is routed to the leaf whose (key, id) range holds it:
// leaf j covers [sep_j, sep_{j+1}) where sep_j is the first (key, id) the leaf
// was created with (leaf 0 extends down to -infinity).  Because the batch is
// sorted, each leaf receives one contiguous slice of it.  Then, per leaf:
//   insert: if the leaf's points plus its slice fit the leaf's block (2*phi
//           slots), the slice is appended unsorted and the box widened
//           (Algorithm 4: append and mark unsorted); otherwise the leaf is
//           sorted, merged with its slice (merge path) and re-wrapped into
//           ceil(c / phi) leaves of balanced size in fresh blocks (Algorithm 4:
//           rebuild when the leaf would exceed the wrap).
//   delete: every leaf point whose (key, id) occurs in the slice (and whose
//           coordinates match) is removed; survivors are compacted in place
//           and the box recomputed; then the leaf wrap is restored (Sec 4.2):
//           each run of leaves left below phi / 2 points (emptied ones
//           included) joins the leaf after it and their points are re-wrapped
//           into balanced leaves of at least phi / 2 points.
// Only touched leaves move data; they read the sorted batch as records (id
// and point per entry, gathered once by k_batch_records).  The leaf list is
// then rewritten from a scan of per-leaf output counts and the summary tree
// rebuilt over it -- the paper's join-based rebalancing is replaced by this
// relayout of the (small) leaf directory.
#include "index.cuh"

namespace psi {
int64_t summary_capacity(int64_t L, int F);

namespace {

struct Batch {
  Buf<uint64_t> k0, k1;
  Buf<uint32_t> v0, v1;
  const uint64_t *keys = nullptr;  // sorted keys
  const uint32_t *vals = nullptr;  // positions into the caller's batch arrays
};

psi_status sort_batch(psi_index *ix, const int32_t *pts, const uint32_t *ids, int64_t m, cudaStream_t s, Batch &b) {
  psi_status st;
  if ((st = b.k0.alloc(m, s)) || (st = b.k1.alloc(m, s)) || (st = b.v0.alloc(m, s)) || (st = b.v1.alloc(m, s)))
    return st;
  SortResult r;
  if ((st = sort_pairs(encode_spec(ix, pts), nullptr, nullptr, m, ix->key_bits, ids, b.k0.p, b.v0.p, b.k1.p, b.v1.p,
                       ix->d_status, s, &r, ix->cfg.radix_bits)))
    return st;
  b.keys = r.keys;
  b.vals = r.vals;
  return PSI_OK;
}

int grid_for(int64_t n, int threads = 256) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, threads), (int64_t)num_sms() * 32));
}

// Leaf of each batch point: the last leaf whose separator is <= (key, id).
__global__ void k_locate(const uint64_t *bkeys, const uint32_t *bvals, const uint32_t *ids, int64_t m,
                         const uint64_t *sep_key, const uint32_t *sep_id, int64_t L, int32_t *bleaf) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = bkeys[i];
    const uint32_t id = ids[bvals[i]];
    int64_t lo = 0, hi = L;  // first separator greater than (k, id)
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (kid_less(k, id, sep_key[mid], sep_id[mid]))
        hi = mid;
      else
        lo = mid + 1;
    }
    bleaf[i] = (int32_t)max((int64_t)0, lo - 1);
  }
}

// Slice [sbeg[j], send[j]) of the sorted batch routed to leaf j.
__global__ void k_slices(const int32_t *bleaf, int64_t m, int32_t *sbeg, int32_t *send) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t j = bleaf[i];
    if (i == 0 || bleaf[i - 1] != j) sbeg[j] = (int32_t)i;
    if (i == m - 1 || bleaf[i + 1] != j) send[j] = (int32_t)(i + 1);
  }
}

__global__ void k_insert_plan(const int32_t *cnt, const int32_t *sbeg, const int32_t *send, int64_t L, int C, int phi,
                              int32_t *outl, int32_t *nblk) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < L; j += (int64_t)gridDim.x * blockDim.x) {
    const int len = send[j] - sbeg[j];
    const int c = cnt[j] + len;
    if (len == 0 || c <= C) {
      outl[j] = 1;
      nblk[j] = 0;
    } else {
      const int r = (c + phi - 1) / phi;
      outl[j] = r;
      nblk[j] = r;
    }
  }
}

constexpr int MAXPL = 4;  // points per lane in one block (C <= 128)

// Sorts, in place by (key, id), the cnt (<= MAXPL * 32) points of one leaf
// block starting at slot s0: the whole warp ranks every point against all
// others and writes it to its rank.
template <int D>
__device__ __forceinline__ void sort_leaf_block(Pool &pool, uint32_t s0, int cnt) {
  const int lane = threadIdx.x & 31;
  uint64_t k[MAXPL];
  uint32_t id[MAXPL];
  int32_t c[MAXPL][D];
#pragma unroll
  for (int r = 0; r < MAXPL; ++r) {
    const int e = r * 32 + lane;
    k[r] = ~0ull;
    id[r] = 0xFFFFFFFFu;
    if (e < cnt) {
      k[r] = pool.pkey[s0 + e];
      id[r] = pool.pid[s0 + e];
#pragma unroll
      for (int d = 0; d < D; ++d) c[r][d] = pool.px[d][s0 + e];
    }
  }
  int rank[MAXPL] = {0, 0, 0, 0};
  for (int r2 = 0; r2 < MAXPL; ++r2) {
    if (r2 * 32 >= cnt) break;
    for (int sl = 0; sl < 32; ++sl) {
      const uint64_t kf = __shfl_sync(0xFFFFFFFFu, k[r2], sl);
      const uint32_t idf = __shfl_sync(0xFFFFFFFFu, id[r2], sl);
      if (r2 * 32 + sl >= cnt) break;
#pragma unroll
      for (int r = 0; r < MAXPL; ++r) rank[r] += kid_less(kf, idf, k[r], id[r]);
    }
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < MAXPL; ++r) {
    const int e = r * 32 + lane;
    if (e < cnt) {
      pool.pkey[s0 + rank[r]] = k[r];
      pool.pid[s0 + rank[r]] = id[r];
#pragma unroll
      for (int d = 0; d < D; ++d) pool.px[d][s0 + rank[r]] = c[r][d];
    }
  }
  __syncwarp();
}

// Sorts, in place, the block of every leaf that will be re-wrapped.  A warp
// takes 32 leaves: one lane per leaf finds the few that overflow, then the
// warp sorts each of those.
template <int D>
__global__ void k_sort_overflow_leaves(const int32_t *ncnt, const uint32_t *nref, const int32_t *sbeg,
                                       const int32_t *send, int64_t L, int C, Pool pool) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t j0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; j0 < L; j0 += warps * 32) {
    const int64_t jl = j0 + lane;
    uint32_t todo = __ballot_sync(0xFFFFFFFFu, jl < L && send[jl] > sbeg[jl] && ncnt[jl] + (send[jl] - sbeg[jl]) > C);
    while (todo) {
      const int64_t j = j0 + __ffs(todo) - 1;
      todo &= todo - 1;
      sort_leaf_block<D>(pool, nref[j], ncnt[j]);
    }
  }
}

struct Leaves {  // leaf directory (node arrays of the leaves) + separators
  int32_t *lo[3], *hi[3], *cnt, *kids, *depth;
  uint32_t *ref;
  uint64_t *sk;
  uint32_t *si;
};

Leaves leaves_of(NodeArrays &a, uint64_t *sk, uint32_t *si) {
  Leaves l;
  for (int d = 0; d < 3; ++d) {
    l.lo[d] = a.lo[d];
    l.hi[d] = a.hi[d];
  }
  l.cnt = a.cnt;
  l.kids = a.kids;
  l.depth = a.depth;
  l.ref = a.ref;
  l.sk = sk;
  l.si = si;
  return l;
}

// owner[o] = old leaf whose output includes new leaf position o.  A thread
// writes the first kOwnerInline entries of its leaf; a leaf that becomes more
// leaves than that (a long sorted run arriving at one place, e.g. a batch in a
// region the index did not cover) is listed, and k_owner_fill_big spreads the
// rest of its entries over a whole block.
constexpr int kOwnerInline = 32;

__global__ void k_owner_scatter(const int32_t *outl, const int64_t *pos, int64_t L, int32_t *owner, int32_t *big,
                                uint32_t *n_big, int64_t cap_big) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < L; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = pos[j];
    const int r = outl[j];
    for (int t = 0; t < min(r, kOwnerInline); ++t) owner[p + t] = (int32_t)j;
    if (r > kOwnerInline) {
      const uint32_t slot = atomicAdd(n_big, 1u);
      if (slot < cap_big) big[slot] = (int32_t)j;
    }
  }
}

__global__ void k_owner_fill_big(const int32_t *outl, const int64_t *pos, const int32_t *big, const uint32_t *n_big,
                                 int64_t cap_big, int32_t *owner) {
  const int64_t nb = min((int64_t)*n_big, cap_big);
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    const int32_t j = big[b];
    const int64_t p = pos[j];
    const int r = outl[j];
    for (int t = kOwnerInline + threadIdx.x; t < r; t += blockDim.x) owner[p + t] = j;
  }
}

struct InsertArgs {
  Leaves old, nw;
  Pool pool;
  const int32_t *owner;
  const int32_t *sbeg, *send, *outl;
  const int64_t *pos, *boff;
  int64_t L, Lnew;
  int64_t base_block;
  const uint64_t *bkeys;
  const uint32_t *rid;  // batch records (k_batch_records): id and point of each sorted entry
  const int32_t *rpt;
  int C, phi;
};

// Merged element order: leaf points first on equality.
__device__ __forceinline__ bool leaf_before_slice(const InsertArgs &a, uint32_t ls, int64_t bi) {
  const uint64_t lk = a.pool.pkey[ls], sk = a.bkeys[bi];
  if (lk != sk) return lk < sk;
  return a.pool.pid[ls] <= a.rid[bi];
}

// A warp takes 32 new leaf positions: a lane copies the descriptor of an
// untouched leaf (most of them), then the warp builds each touched one.
template <int D>
__global__ void k_insert_apply(InsertArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t o0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; o0 < a.Lnew; o0 += warps * 32) {
    bool touched = false;
    {
      const int64_t ol = o0 + lane;
      if (ol < a.Lnew) {
        const int64_t j = a.owner[ol];
        if (a.send[j] == a.sbeg[j]) {
#pragma unroll
          for (int d = 0; d < D; ++d) {
            a.nw.lo[d][ol] = a.old.lo[d][j];
            a.nw.hi[d][ol] = a.old.hi[d][j];
          }
          a.nw.cnt[ol] = a.old.cnt[j];
          a.nw.ref[ol] = a.old.ref[j];
          a.nw.kids[ol] = 0;
          a.nw.depth[ol] = 0;
          a.nw.sk[ol] = a.old.sk[j];
          a.nw.si[ol] = a.old.si[j];
        } else {
          touched = true;
        }
      }
    }
    uint32_t todo = __ballot_sync(0xFFFFFFFFu, touched);
   while (todo) {
    const int64_t o = o0 + __ffs(todo) - 1;
    todo &= todo - 1;
    const int64_t j = a.owner[o];
    const int t = (int)(o - a.pos[j]);
    const int len = a.send[j] - a.sbeg[j];
    const int cnt = a.old.cnt[j];
    const uint32_t s0 = a.old.ref[j];
    int32_t blo[D], bhi[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      blo[d] = INT32_MAX;
      bhi[d] = INT32_MIN;
    }
    if (len == 0 || cnt + len <= a.C) {
      // untouched or append: the leaf keeps its block and separator
      for (int s = lane; s < len; s += 32) {
        const int64_t bi = a.sbeg[j] + s;
        const uint32_t slot = s0 + (uint32_t)(cnt + s);
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const int32_t c = a.rpt[bi * D + d];
          a.pool.px[d][slot] = c;
          blo[d] = min(blo[d], c);
          bhi[d] = max(bhi[d], c);
        }
        a.pool.pid[slot] = a.rid[bi];
        a.pool.pkey[slot] = a.bkeys[bi];
      }
#pragma unroll
      for (int d = 0; d < D; ++d) {
        blo[d] = __reduce_min_sync(0xFFFFFFFFu, blo[d]);
        bhi[d] = __reduce_max_sync(0xFFFFFFFFu, bhi[d]);
      }
      if (lane == 0) {
#pragma unroll
        for (int d = 0; d < D; ++d) {
          a.nw.lo[d][o] = min(a.old.lo[d][j], blo[d]);
          a.nw.hi[d][o] = max(a.old.hi[d][j], bhi[d]);
        }
        a.nw.cnt[o] = cnt + len;
        a.nw.ref[o] = s0;
        a.nw.kids[o] = 0;
        a.nw.depth[o] = 0;
        a.nw.sk[o] = a.old.sk[j];
        a.nw.si[o] = a.old.si[j];
      }
      continue;
    }
    // re-wrap: part t of the merge of the (sorted) leaf and its slice
    const int64_t c = (int64_t)cnt + len;
    const int r = a.outl[j];
    const int64_t pa = (int64_t)t * c / r, pb = (int64_t)(t + 1) * c / r;
    const int64_t blk = a.base_block + a.boff[j] + t;
    const uint32_t d0 = (uint32_t)(blk * a.C);
    const int64_t sb = a.sbeg[j];
    for (int64_t p = pa + lane; p < pb; p += 32) {
      int64_t l = max((int64_t)0, p - len), h = min(p, (int64_t)cnt);
      while (l < h) {
        const int64_t mid = (l + h) >> 1;
        if (leaf_before_slice(a, s0 + (uint32_t)mid, sb + (p - mid - 1)))
          l = mid + 1;
        else
          h = mid;
      }
      const int64_t li = l, si = p - l;
      const bool from_leaf = li < cnt && (si >= len || leaf_before_slice(a, s0 + (uint32_t)li, sb + si));
      const uint32_t dst = d0 + (uint32_t)(p - pa);
      if (from_leaf) {
        const uint32_t src = s0 + (uint32_t)li;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const int32_t cc = a.pool.px[d][src];
          a.pool.px[d][dst] = cc;
          blo[d] = min(blo[d], cc);
          bhi[d] = max(bhi[d], cc);
        }
        a.pool.pid[dst] = a.pool.pid[src];
        a.pool.pkey[dst] = a.pool.pkey[src];
      } else {
        const int64_t bi = sb + si;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const int32_t cc = a.rpt[bi * D + d];
          a.pool.px[d][dst] = cc;
          blo[d] = min(blo[d], cc);
          bhi[d] = max(bhi[d], cc);
        }
        a.pool.pid[dst] = a.rid[bi];
        a.pool.pkey[dst] = a.bkeys[bi];
      }
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
      blo[d] = __reduce_min_sync(0xFFFFFFFFu, blo[d]);
      bhi[d] = __reduce_max_sync(0xFFFFFFFFu, bhi[d]);
    }
    __syncwarp();
    if (lane == 0) {
#pragma unroll
      for (int d = 0; d < D; ++d) {
        a.nw.lo[d][o] = blo[d];
        a.nw.hi[d][o] = bhi[d];
      }
      a.nw.cnt[o] = (int32_t)(pb - pa);
      a.nw.ref[o] = d0;
      a.nw.kids[o] = 0;
      a.nw.depth[o] = 0;
      // the first part keeps the old lower end; later parts start at their
      // first element, and so does the first part of leaf 0, which is open
      // below and may hold points under its separator (appended ones), so
      // that the separators stay increasing
      if (t == 0 && j != 0) {
        a.nw.sk[o] = a.old.sk[j];
        a.nw.si[o] = a.old.si[j];
      } else {
        a.nw.sk[o] = a.pool.pkey[d0];
        a.nw.si[o] = a.pool.pid[d0];
      }
    }
    __syncwarp();
   }
  }
}

// Insert that splits no leaf: every touched leaf appends its slice in place
// (its block has room); untouched leaves are not visited.  A warp takes 32
// leaves, one lane per leaf finds those with a slice.
template <int D>
__global__ void k_append_inplace(Leaves lv, Pool pool, const int32_t *sbeg, const int32_t *send, int64_t L,
                                 const uint64_t *bkeys, const uint32_t *rid, const int32_t *rpt) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t j0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; j0 < L; j0 += warps * 32) {
    const int64_t jl = j0 + lane;
    uint32_t todo = __ballot_sync(0xFFFFFFFFu, jl < L && send[jl] > sbeg[jl]);
    while (todo) {
      const int64_t j = j0 + __ffs(todo) - 1;
      todo &= todo - 1;
      const int64_t b = sbeg[j];
      const int len = send[j] - (int)b;
      const int cnt = lv.cnt[j];
      const uint32_t s0 = lv.ref[j];
      int32_t blo[D], bhi[D];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        blo[d] = INT32_MAX;
        bhi[d] = INT32_MIN;
      }
      for (int t = lane; t < len; t += 32) {
        const uint32_t slot = s0 + (uint32_t)(cnt + t);
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const int32_t c = rpt[(b + t) * D + d];
          pool.px[d][slot] = c;
          blo[d] = min(blo[d], c);
          bhi[d] = max(bhi[d], c);
        }
        pool.pid[slot] = rid[b + t];
        pool.pkey[slot] = bkeys[b + t];
      }
#pragma unroll
      for (int d = 0; d < D; ++d) {
        blo[d] = __reduce_min_sync(0xFFFFFFFFu, blo[d]);
        bhi[d] = __reduce_max_sync(0xFFFFFFFFu, bhi[d]);
      }
      if (lane == 0) {
#pragma unroll
        for (int d = 0; d < D; ++d) {
          lv.lo[d][j] = min(lv.lo[d][j], blo[d]);
          lv.hi[d][j] = max(lv.hi[d][j], bhi[d]);
        }
        lv.cnt[j] = cnt + len;
      }
      __syncwarp();
    }
  }
}

// The sorted batch as records: the id and the point of each (key-sorted)
// entry, so that a leaf finds what its slice names in one read.
template <int D>
__global__ void k_batch_records(const uint32_t *bvals, const int32_t *pts, const uint32_t *ids, int64_t m,
                                uint32_t *rid, int32_t *rpt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t v = bvals[i];
    rid[i] = ids[v];
#pragma unroll
    for (int d = 0; d < D; ++d) rpt[i * D + d] = pts[(int64_t)v * D + d];
  }
}

// Remove the points named by each leaf's slice: a warp takes 32 leaves, one
// lane per leaf finds those with a slice, then the warp compacts them two at a
// time (both leaves' points and slice entries requested before either is
// compacted).  R rows of 32 slots cover a leaf's block (R * 32 >= C).
constexpr int DG = 2;

template <int D, int R>
__global__ void k_delete_leaves(Leaves lv, Pool pool, const int32_t *sbeg, const int32_t *send, int64_t L,
                                const uint64_t *bkeys, const uint32_t *rid, const int32_t *rpt,
                                unsigned long long *deleted) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  uint32_t removed = 0;  // lane 0: points this warp removed
  for (int64_t j0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; j0 < L; j0 += warps * 32) {
    const int64_t jl = j0 + lane;
    uint32_t todo = __ballot_sync(0xFFFFFFFFu, jl < L && send[jl] > sbeg[jl]);
    while (todo) {
      int64_t j[DG];
      int cnt[DG];
      uint32_t s0[DG];
      int32_t b[DG], e[DG];
#pragma unroll
      for (int g = 0; g < DG; ++g) {
        cnt[g] = 0;
        s0[g] = 0;
        b[g] = e[g] = 0;
        j[g] = -1;
        if (todo) {
          j[g] = j0 + __ffs(todo) - 1;
          todo &= todo - 1;
          cnt[g] = lv.cnt[j[g]];
          s0[g] = lv.ref[j[g]];
          b[g] = sbeg[j[g]];
          e[g] = send[j[g]];
        }
      }
      uint64_t k[DG][R];
      uint32_t id[DG][R];
      int32_t c[DG][R][D];
#pragma unroll
      for (int g = 0; g < DG; ++g)
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int x = r * 32 + lane;
          if (x < cnt[g]) {
            k[g][r] = pool.pkey[s0[g] + x];
            id[g][r] = pool.pid[s0[g] + x];
#pragma unroll
            for (int d = 0; d < D; ++d) c[g][r][d] = pool.px[d][s0[g] + x];
          }
        }
      bool keep[DG][R];
#pragma unroll
      for (int g = 0; g < DG; ++g)
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int x = r * 32 + lane;
          keep[g][r] = false;
          if (x < cnt[g]) {
            // is (k, id) in the slice?
            int32_t lo = b[g], hi = e[g];
            while (lo < hi) {
              const int32_t mid = (lo + hi) >> 1;
              if (kid_less(bkeys[mid], rid[mid], k[g][r], id[g][r]))
                lo = mid + 1;
              else
                hi = mid;
            }
            bool hit = lo < e[g] && bkeys[lo] == k[g][r] && rid[lo] == id[g][r];
            if (hit) {
#pragma unroll
              for (int d = 0; d < D; ++d) hit &= rpt[(int64_t)lo * D + d] == c[g][r][d];
            }
            keep[g][r] = !hit;
          }
        }
      __syncwarp();
#pragma unroll
      for (int g = 0; g < DG; ++g) {
        if (j[g] < 0) break;  // warp-uniform
        int out = 0;
        int32_t blo[D], bhi[D];
#pragma unroll
        for (int d = 0; d < D; ++d) {
          blo[d] = INT32_MAX;
          bhi[d] = INT32_MIN;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const uint32_t m = __ballot_sync(0xFFFFFFFFu, keep[g][r]);
          if (keep[g][r]) {
            const uint32_t dst = s0[g] + (uint32_t)(out + __popc(m & lanemask_lt()));
            pool.pkey[dst] = k[g][r];
            pool.pid[dst] = id[g][r];
#pragma unroll
            for (int d = 0; d < D; ++d) {
              pool.px[d][dst] = c[g][r][d];
              blo[d] = min(blo[d], c[g][r][d]);
              bhi[d] = max(bhi[d], c[g][r][d]);
            }
          }
          out += __popc(m);
        }
#pragma unroll
        for (int d = 0; d < D; ++d) {
          blo[d] = __reduce_min_sync(0xFFFFFFFFu, blo[d]);
          bhi[d] = __reduce_max_sync(0xFFFFFFFFu, bhi[d]);
        }
        if (lane == 0) {
          lv.cnt[j[g]] = out;
#pragma unroll
          for (int d = 0; d < D; ++d) {
            lv.lo[d][j[g]] = blo[d];
            lv.hi[d][j[g]] = bhi[d];
          }
          removed += (uint32_t)(cnt[g] - out);
        }
      }
      __syncwarp();
    }
  }
  block_count_add(deleted, removed);
}

// ---- Restoring the leaf wrap after a delete (Sec 4.2) ----------------------
// A leaf left with fewer than h = max(1, phi / 2) points (an emptied leaf
// included) is underfull.  Each maximal run of consecutive underfull leaves
// forms a group with the leaf after it, when there is one; the group's points
// -- its leaves' points one after another, which in leaf order are
// consecutive (key, id) ranges -- are re-wrapped into ceil(total / phi)
// leaves of balanced size in fresh blocks.  Afterwards every leaf but the last
// of the index holds at least h points.

// start[j]: leaf j begins a run of underfull leaves.
__global__ void k_wrap_flags(const int32_t *cnt, int64_t L, int h, int32_t *start) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < L; j += (int64_t)gridDim.x * blockDim.x)
    start[j] = cnt[j] < h && (j == 0 || cnt[j - 1] >= h);
}

// Group g (numbered by the exclusive scan gx of start): its first leaf gs[g]
// and its last leaf ge[g] (the leaf after the run, or the run's own last leaf
// at the end of the index).
__global__ void k_wrap_bounds(const int32_t *cnt, const int32_t *start, const int64_t *gx, int64_t L, int h,
                              int32_t *gs, int32_t *ge) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < L; j += (int64_t)gridDim.x * blockDim.x) {
    if (start[j]) gs[gx[j]] = (int32_t)j;
    if (cnt[j] < h && (j + 1 == L || cnt[j + 1] >= h)) ge[gx[j] + start[j] - 1] = (int32_t)(j + 1 < L ? j + 1 : j);
  }
}

// Output leaves of each old leaf (a group's re-wrapped leaves are counted at
// its first leaf, its other leaves give none, a leaf outside every group is
// kept as it is), the fresh blocks each needs, and whether it is in a group.
__global__ void k_wrap_plan(const int32_t *cnt, const int32_t *start, const int64_t *gx, const int32_t *ge,
                            const int64_t *E, int64_t L, int h, int phi, int32_t *outl, int32_t *nblk,
                            int32_t *ingroup) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < L; j += (int64_t)gridDim.x * blockDim.x) {
    const bool ig = cnt[j] < h || (j > 0 && cnt[j - 1] < h);
    ingroup[j] = ig;
    if (start[j]) {
      const int64_t e = ge[gx[j]];
      const int64_t total = E[e] + cnt[e] - E[j];
      const int r = (int)((total + phi - 1) / phi);
      outl[j] = r;
      nblk[j] = r;
    } else {
      outl[j] = ig ? 0 : 1;
      nblk[j] = 0;
    }
  }
}

// Sorts, in place, the block of every leaf of a group (a group's points in
// leaf order are then sorted by (key, id) as a whole).
template <int D>
__global__ void k_sort_flagged_leaves(const int32_t *cnt, const uint32_t *ref, const int32_t *flag, int64_t L,
                                      Pool pool) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t j0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; j0 < L; j0 += warps * 32) {
    const int64_t jl = j0 + lane;
    uint32_t todo = __ballot_sync(0xFFFFFFFFu, jl < L && flag[jl] && cnt[jl] > 1);
    while (todo) {
      const int64_t j = j0 + __ffs(todo) - 1;
      todo &= todo - 1;
      sort_leaf_block<D>(pool, ref[j], cnt[j]);
    }
  }
}

struct WrapArgs {
  Leaves old, nw;
  Pool pool;
  const int32_t *owner, *start, *ge, *outl;
  const int64_t *gx, *pos, *boff, *E;
  int64_t Lnew, base_block;
  int C;
};

// A warp takes 32 new leaf positions: a lane copies the descriptor of a kept
// leaf, then the warp builds each re-wrapped one (part t of its group).
template <int D>
__global__ void k_wrap_apply(WrapArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t o0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; o0 < a.Lnew; o0 += warps * 32) {
    bool part = false;
    {
      const int64_t ol = o0 + lane;
      if (ol < a.Lnew) {
        const int64_t j = a.owner[ol];
        if (!a.start[j]) {
#pragma unroll
          for (int d = 0; d < D; ++d) {
            a.nw.lo[d][ol] = a.old.lo[d][j];
            a.nw.hi[d][ol] = a.old.hi[d][j];
          }
          a.nw.cnt[ol] = a.old.cnt[j];
          a.nw.ref[ol] = a.old.ref[j];
          a.nw.kids[ol] = 0;
          a.nw.depth[ol] = 0;
          a.nw.sk[ol] = a.old.sk[j];
          a.nw.si[ol] = a.old.si[j];
        } else {
          part = true;
        }
      }
    }
    uint32_t todo = __ballot_sync(0xFFFFFFFFu, part);
    while (todo) {
      const int64_t o = o0 + __ffs(todo) - 1;
      todo &= todo - 1;
      const int64_t j = a.owner[o];
      const int64_t e = a.ge[a.gx[j]];
      const int64_t t = o - a.pos[j];
      const int64_t total = a.E[e] + a.old.cnt[e] - a.E[j];
      const int r = a.outl[j];
      const int64_t pa = t * total / r, pb = (t + 1) * total / r;
      const uint32_t d0 = (uint32_t)((a.base_block + a.boff[j] + t) * a.C);
      int32_t blo[D], bhi[D];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        blo[d] = INT32_MAX;
        bhi[d] = INT32_MIN;
      }
      for (int64_t p = pa + lane; p < pb; p += 32) {
        // the group's leaf holding position p: the last leaf x in [j, e] with E[x] <= E[j] + p
        const int64_t v = a.E[j] + p;
        int64_t lo = j, hi = e + 1;
        while (hi - lo > 1) {
          const int64_t mid = (lo + hi) >> 1;
          if (a.E[mid] <= v)
            lo = mid;
          else
            hi = mid;
        }
        const uint32_t src = a.old.ref[lo] + (uint32_t)(v - a.E[lo]);
        const uint32_t dst = d0 + (uint32_t)(p - pa);
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const int32_t c = a.pool.px[d][src];
          a.pool.px[d][dst] = c;
          blo[d] = min(blo[d], c);
          bhi[d] = max(bhi[d], c);
        }
        a.pool.pid[dst] = a.pool.pid[src];
        a.pool.pkey[dst] = a.pool.pkey[src];
      }
#pragma unroll
      for (int d = 0; d < D; ++d) {
        blo[d] = __reduce_min_sync(0xFFFFFFFFu, blo[d]);
        bhi[d] = __reduce_max_sync(0xFFFFFFFFu, bhi[d]);
      }
      __syncwarp();
      if (lane == 0) {
#pragma unroll
        for (int d = 0; d < D; ++d) {
          a.nw.lo[d][o] = blo[d];
          a.nw.hi[d][o] = bhi[d];
        }
        a.nw.cnt[o] = (int32_t)(pb - pa);
        a.nw.ref[o] = d0;
        a.nw.kids[o] = 0;
        a.nw.depth[o] = 0;
        // the first part keeps the group's lower end; later parts start at
        // their first point, and so does the first part of a group at leaf 0
        // (open below: it may hold points under its separator)
        if (t == 0 && j != 0) {
          a.nw.sk[o] = a.old.sk[j];
          a.nw.si[o] = a.old.si[j];
        } else {
          a.nw.sk[o] = a.pool.pkey[d0];
          a.nw.si[o] = a.pool.pid[d0];
        }
      }
      __syncwarp();
    }
  }
}

__global__ void k_copy_i64(const unsigned long long *src, int64_t *dst) { *dst = (int64_t)*src; }

// Grows the pool to hold at least `slots` slots, keeping the used prefix.
psi_status grow_pool(psi_index *ix, int64_t slots_needed, int64_t used_slots, cudaStream_t s) {
  if (slots_needed <= ix->pool.cap_slots) return PSI_OK;
  Pool np;
  const int64_t cap = std::max(slots_needed + slots_needed / 4, ix->pool.cap_slots * 3 / 2);
  psi_status st = alloc_pool(np, ix->D, cap, s);
  if (st) {
    free_pool(np, s);
    return st;
  }
  if (used_slots > 0) {
    for (int d = 0; d < ix->D; ++d)
      PSI_CK(cudaMemcpyAsync(np.px[d], ix->pool.px[d], sizeof(int32_t) * used_slots, cudaMemcpyDeviceToDevice, s));
    PSI_CK(cudaMemcpyAsync(np.pid, ix->pool.pid, sizeof(uint32_t) * used_slots, cudaMemcpyDeviceToDevice, s));
    PSI_CK(cudaMemcpyAsync(np.pkey, ix->pool.pkey, sizeof(uint64_t) * used_slots, cudaMemcpyDeviceToDevice, s));
  }
  free_pool(ix->pool, s);
  ix->pool = np;
  return PSI_OK;
}

int warp_grid(int64_t warps) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(warps, 8), (int64_t)num_sms() * 32));
}

}  // namespace

psi_status spac_build_fresh(psi_index *ix, const int32_t *pts, const uint32_t *ids, int64_t n, cudaStream_t s);

// Records (id, point) of the sorted batch, read by the leaf kernels.
static psi_status batch_records(const psi_index *ix, const Batch &b, const int32_t *pts, const uint32_t *ids,
                                int64_t m, cudaStream_t s, Buf<uint32_t> &rid, Buf<int32_t> &rpt) {
  psi_status st;
  if ((st = rid.alloc(m, s)) || (st = rpt.alloc(m * ix->D, s))) return st;
  if (ix->D == 2)
    PSI_LAUNCH_NAMED("k_batch_records", k_batch_records<2>, grid_for(m), 256, 0, s, b.vals, pts, ids, m, rid.p, rpt.p);
  else
    PSI_LAUNCH_NAMED("k_batch_records", k_batch_records<3>, grid_for(m), 256, 0, s, b.vals, pts, ids, m, rid.p, rpt.p);
  return PSI_OK;
}

psi_status spac_insert(psi_index *ix, const int32_t *pts, const uint32_t *ids, int64_t m, cudaStream_t s) {
  if (ix->L == 0) return spac_build_fresh(ix, pts, ids, m, s);
  psi_status st;
  Batch b;
  if ((st = sort_batch(ix, pts, ids, m, s, b))) return st;
  Buf<uint32_t> rid;
  Buf<int32_t> rpt;
  if ((st = batch_records(ix, b, pts, ids, m, s, rid, rpt))) return st;
  const int64_t L = ix->L;
  Buf<int32_t> bleaf, sbeg, send, outl, nblk;
  Buf<int64_t> pos, boff, tot;
  if ((st = bleaf.alloc(m, s)) || (st = sbeg.alloc(L, s)) || (st = send.alloc(L, s)) || (st = outl.alloc(L, s)) ||
      (st = nblk.alloc(L, s)) || (st = pos.alloc(L, s)) || (st = boff.alloc(L, s)) || (st = tot.alloc(2, s)))
    return st;
  PSI_CK(cudaMemsetAsync(sbeg.p, 0, sizeof(int32_t) * L, s));
  PSI_CK(cudaMemsetAsync(send.p, 0, sizeof(int32_t) * L, s));
  PSI_LAUNCH(k_locate, grid_for(m), 256, 0, s, b.keys, b.vals, ids, m, ix->sep_key, ix->sep_id, L, bleaf.p);
  PSI_LAUNCH(k_slices, grid_for(m), 256, 0, s, bleaf.p, m, sbeg.p, send.p);
  PSI_LAUNCH(k_insert_plan, grid_for(L), 256, 0, s, ix->nodes.cnt, sbeg.p, send.p, L, ix->C, ix->phi, outl.p, nblk.p);
  if ((st = scan_i32_to_i64(outl.p, pos.p, L, tot.p, s))) return st;
  if ((st = scan_i32_to_i64(nblk.p, boff.p, L, tot.p + 1, s))) return st;
  int64_t h[2];
  PSI_CK(cudaMemcpyAsync(h, tot.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaStreamSynchronize(s));
  const int64_t Lnew = h[0], NB = h[1];

  if (NB == 0) {  // no leaf overflows: append in place, the leaf list keeps its shape
    Leaves lv = leaves_of(ix->nodes, ix->sep_key, ix->sep_id);
    if (ix->D == 2)
      PSI_LAUNCH_NAMED("k_append_inplace", k_append_inplace<2>, warp_grid(ceil_div(L, 32)), 256, 0, s, lv, ix->pool,
                       sbeg.p, send.p, L, b.keys, rid.p, rpt.p);
    else
      PSI_LAUNCH_NAMED("k_append_inplace", k_append_inplace<3>, warp_grid(ceil_div(L, 32)), 256, 0, s, lv, ix->pool,
                       sbeg.p, send.p, L, b.keys, rid.p, rpt.p);
    ix->n += m;
    if ((st = build_spac_summary(ix, s))) return st;
    PSI_CK(cudaGetLastError());
    return PSI_OK;
  }

  const int64_t base_block = ix->pool_used;
  if ((st = grow_pool(ix, (base_block + NB) * ix->C, base_block * ix->C, s))) return st;
  if (ix->D == 2)
    PSI_LAUNCH_NAMED("k_sort_overflow_leaves", k_sort_overflow_leaves<2>, warp_grid(ceil_div(L, 32)), 256, 0, s,
                     ix->nodes.cnt, ix->nodes.ref, sbeg.p, send.p, L, ix->C, ix->pool);
  else
    PSI_LAUNCH_NAMED("k_sort_overflow_leaves", k_sort_overflow_leaves<3>, warp_grid(ceil_div(L, 32)), 256, 0, s,
                     ix->nodes.cnt, ix->nodes.ref, sbeg.p, send.p, L, ix->C, ix->pool);

  NodeArrays na;
  uint64_t *nsk = nullptr;
  uint32_t *nsi = nullptr;
  if ((st = alloc_nodes(na, ix->D, summary_capacity(Lnew, ix->F), false, s)) ||
      (st = DevMem::alloc((void **)&nsk, sizeof(uint64_t) * Lnew, s)) ||
      (st = DevMem::alloc((void **)&nsi, sizeof(uint32_t) * Lnew, s))) {
    free_nodes(na, s);
    DevMem::free(nsk, s);
    DevMem::free(nsi, s);
    return st;
  }
  // a leaf re-wrapped into more than kOwnerInline leaves holds more than
  // (kOwnerInline - 2) * phi of the batch's points (its block holds at most 2 phi)
  const int64_t cap_big = m / ((kOwnerInline - 2) * (int64_t)ix->phi) + 1;
  Buf<int32_t> owner, big;
  Buf<uint32_t> n_big;
  if ((st = owner.alloc(Lnew, s)) || (st = big.alloc(cap_big, s)) || (st = n_big.alloc(1, s))) return st;
  PSI_CK(cudaMemsetAsync(n_big.p, 0, sizeof(uint32_t), s));
  PSI_LAUNCH(k_owner_scatter, grid_for(L), 256, 0, s, outl.p, pos.p, L, owner.p, big.p, n_big.p, cap_big);
  PSI_LAUNCH(k_owner_fill_big, num_sms() * 4, 256, 0, s, outl.p, pos.p, big.p, n_big.p, cap_big, owner.p);
  InsertArgs a;
  a.owner = owner.p;
  a.old = leaves_of(ix->nodes, ix->sep_key, ix->sep_id);
  a.nw = leaves_of(na, nsk, nsi);
  a.pool = ix->pool;
  a.sbeg = sbeg.p;
  a.send = send.p;
  a.outl = outl.p;
  a.pos = pos.p;
  a.boff = boff.p;
  a.L = L;
  a.Lnew = Lnew;
  a.base_block = base_block;
  a.bkeys = b.keys;
  a.rid = rid.p;
  a.rpt = rpt.p;
  a.C = ix->C;
  a.phi = ix->phi;
  if (ix->D == 2)
    PSI_LAUNCH_NAMED("k_insert_apply", k_insert_apply<2>, warp_grid(ceil_div(Lnew, 32)), 256, 0, s, a);
  else
    PSI_LAUNCH_NAMED("k_insert_apply", k_insert_apply<3>, warp_grid(ceil_div(Lnew, 32)), 256, 0, s, a);
  free_nodes(ix->nodes, s);
  DevMem::free(ix->sep_key, s);
  DevMem::free(ix->sep_id, s);
  ix->nodes = na;
  ix->sep_key = nsk;
  ix->sep_id = nsi;
  ix->L = Lnew;
  ix->n += m;
  ix->pool_used = base_block + NB;
  if ((st = build_spac_summary(ix, s))) return st;
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}

psi_status spac_delete(psi_index *ix, const int32_t *pts, const uint32_t *ids, int64_t m, int64_t *d_deleted,
                       cudaStream_t s) {
  psi_status st;
  Batch b;
  if ((st = sort_batch(ix, pts, ids, m, s, b))) return st;
  const int64_t L = ix->L;
  Buf<int32_t> bleaf, sbeg, send;
  Buf<int64_t> tot;
  Buf<unsigned long long> del;
  if ((st = bleaf.alloc(m, s)) || (st = sbeg.alloc(L, s)) || (st = send.alloc(L, s)) || (st = tot.alloc(2, s)) ||
      (st = del.alloc(1, s)))
    return st;
  PSI_CK(cudaMemsetAsync(sbeg.p, 0, sizeof(int32_t) * L, s));
  PSI_CK(cudaMemsetAsync(send.p, 0, sizeof(int32_t) * L, s));
  PSI_CK(cudaMemsetAsync(del.p, 0, sizeof(unsigned long long), s));
  PSI_LAUNCH(k_locate, grid_for(m), 256, 0, s, b.keys, b.vals, ids, m, ix->sep_key, ix->sep_id, L, bleaf.p);
  PSI_LAUNCH(k_slices, grid_for(m), 256, 0, s, bleaf.p, m, sbeg.p, send.p);
  Buf<uint32_t> rid;
  Buf<int32_t> rpt;
  if ((st = batch_records(ix, b, pts, ids, m, s, rid, rpt))) return st;
  Leaves lv = leaves_of(ix->nodes, ix->sep_key, ix->sep_id);
  const int g = warp_grid(ceil_div(L, 32));
  if (ix->D == 2) {
    if (ix->C <= 64)
      PSI_LAUNCH_NAMED("k_delete_leaves", (k_delete_leaves<2, 2>), g, 256, 0, s, lv, ix->pool, sbeg.p, send.p, L,
                       b.keys, rid.p, rpt.p, del.p);
    else
      PSI_LAUNCH_NAMED("k_delete_leaves", (k_delete_leaves<2, MAXPL>), g, 256, 0, s, lv, ix->pool, sbeg.p, send.p, L,
                       b.keys, rid.p, rpt.p, del.p);
  } else {
    if (ix->C <= 64)
      PSI_LAUNCH_NAMED("k_delete_leaves", (k_delete_leaves<3, 2>), g, 256, 0, s, lv, ix->pool, sbeg.p, send.p, L,
                       b.keys, rid.p, rpt.p, del.p);
    else
      PSI_LAUNCH_NAMED("k_delete_leaves", (k_delete_leaves<3, MAXPL>), g, 256, 0, s, lv, ix->pool, sbeg.p, send.p, L,
                       b.keys, rid.p, rpt.p, del.p);
  }
  // the leaf wrap (Sec 4.2): runs of leaves left below h points join the leaf
  // after them and are re-wrapped
  const int h = std::max(1, ix->phi / 2);
  Buf<int32_t> start;
  Buf<int64_t> gx, E;
  if ((st = start.alloc(L, s)) || (st = gx.alloc(L, s)) || (st = E.alloc(L, s))) return st;
  PSI_LAUNCH(k_wrap_flags, grid_for(L), 256, 0, s, ix->nodes.cnt, L, h, start.p);
  if ((st = scan_i32_to_i64(start.p, gx.p, L, tot.p, s))) return st;
  PSI_LAUNCH(k_copy_i64, 1, 1, 0, s, del.p, tot.p + 1);
  if (d_deleted) PSI_CK(cudaMemcpyAsync(d_deleted, tot.p + 1, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  int64_t h2[2];
  PSI_CK(cudaMemcpyAsync(h2, tot.p, sizeof(h2), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaStreamSynchronize(s));
  const int64_t G = h2[0];
  ix->n -= h2[1];
  if (G == 0) {  // no leaf fell below h: the in-place edits above are the new leaves
    if ((st = build_spac_summary(ix, s))) return st;
    PSI_CK(cudaGetLastError());
    return PSI_OK;
  }
  Buf<int32_t> gs, ge, outl, nblk, ingroup;
  Buf<int64_t> pos, boff, tot2;
  if ((st = gs.alloc(G, s)) || (st = ge.alloc(G, s)) || (st = outl.alloc(L, s)) || (st = nblk.alloc(L, s)) ||
      (st = ingroup.alloc(L, s)) || (st = pos.alloc(L, s)) || (st = boff.alloc(L, s)) || (st = tot2.alloc(3, s)))
    return st;
  if ((st = scan_i32_to_i64(ix->nodes.cnt, E.p, L, tot2.p + 2, s))) return st;
  PSI_LAUNCH(k_wrap_bounds, grid_for(L), 256, 0, s, ix->nodes.cnt, start.p, gx.p, L, h, gs.p, ge.p);
  PSI_LAUNCH(k_wrap_plan, grid_for(L), 256, 0, s, ix->nodes.cnt, start.p, gx.p, ge.p, E.p, L, h, ix->phi, outl.p,
             nblk.p, ingroup.p);
  if ((st = scan_i32_to_i64(outl.p, pos.p, L, tot2.p, s))) return st;
  if ((st = scan_i32_to_i64(nblk.p, boff.p, L, tot2.p + 1, s))) return st;
  int64_t h3[2];
  PSI_CK(cudaMemcpyAsync(h3, tot2.p, sizeof(h3), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaStreamSynchronize(s));
  const int64_t Lnew = h3[0], NB = h3[1];
  const int64_t base_block = ix->pool_used;
  if ((st = grow_pool(ix, (base_block + NB) * ix->C, base_block * ix->C, s))) return st;
  if (ix->D == 2)
    PSI_LAUNCH_NAMED("k_sort_flagged_leaves", k_sort_flagged_leaves<2>, warp_grid(ceil_div(L, 32)), 256, 0, s,
                     ix->nodes.cnt, ix->nodes.ref, ingroup.p, L, ix->pool);
  else
    PSI_LAUNCH_NAMED("k_sort_flagged_leaves", k_sort_flagged_leaves<3>, warp_grid(ceil_div(L, 32)), 256, 0, s,
                     ix->nodes.cnt, ix->nodes.ref, ingroup.p, L, ix->pool);
  NodeArrays na;
  uint64_t *nsk = nullptr;
  uint32_t *nsi = nullptr;
  if ((st = alloc_nodes(na, ix->D, summary_capacity(Lnew, ix->F), false, s)) ||
      (st = DevMem::alloc((void **)&nsk, sizeof(uint64_t) * std::max<int64_t>(Lnew, 1), s)) ||
      (st = DevMem::alloc((void **)&nsi, sizeof(uint32_t) * std::max<int64_t>(Lnew, 1), s))) {
    free_nodes(na, s);
    DevMem::free(nsk, s);
    DevMem::free(nsi, s);
    return st;
  }
  if (Lnew > 0) {
    // a group re-wrapped into more than kOwnerInline leaves holds more than
    // (kOwnerInline - 1) * phi points
    const int64_t cap_big = ix->n / ((kOwnerInline - 1) * (int64_t)ix->phi) + 1;
    Buf<int32_t> owner, big;
    Buf<uint32_t> n_big;
    if ((st = owner.alloc(Lnew, s)) || (st = big.alloc(cap_big, s)) || (st = n_big.alloc(1, s))) return st;
    PSI_CK(cudaMemsetAsync(n_big.p, 0, sizeof(uint32_t), s));
    PSI_LAUNCH(k_owner_scatter, grid_for(L), 256, 0, s, outl.p, pos.p, L, owner.p, big.p, n_big.p, cap_big);
    PSI_LAUNCH(k_owner_fill_big, num_sms() * 4, 256, 0, s, outl.p, pos.p, big.p, n_big.p, cap_big, owner.p);
    WrapArgs a;
    a.old = lv;
    a.nw = leaves_of(na, nsk, nsi);
    a.pool = ix->pool;
    a.owner = owner.p;
    a.start = start.p;
    a.ge = ge.p;
    a.outl = outl.p;
    a.gx = gx.p;
    a.pos = pos.p;
    a.boff = boff.p;
    a.E = E.p;
    a.Lnew = Lnew;
    a.base_block = base_block;
    a.C = ix->C;
    if (ix->D == 2)
      PSI_LAUNCH_NAMED("k_wrap_apply", k_wrap_apply<2>, warp_grid(ceil_div(Lnew, 32)), 256, 0, s, a);
    else
      PSI_LAUNCH_NAMED("k_wrap_apply", k_wrap_apply<3>, warp_grid(ceil_div(Lnew, 32)), 256, 0, s, a);
  }
  free_nodes(ix->nodes, s);
  DevMem::free(ix->sep_key, s);
  DevMem::free(ix->sep_id, s);
  ix->nodes = na;
  ix->sep_key = nsk;
  ix->sep_id = nsi;
  ix->L = Lnew;
  ix->pool_used = base_block + NB;
  if ((st = build_spac_summary(ix, s))) return st;
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}

}  // namespace psi

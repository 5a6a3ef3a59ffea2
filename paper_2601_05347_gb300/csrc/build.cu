// build.cu -- SPaC construction after the key sort (Algorithm 3, BuildSorted):
// leaf wrapping of the sorted sequence into blocks, leaf boxes and counts, and
// the bottom-up summary tree over the leaves.
//
// The paper's BuildSorted halves the sorted range recursively and wraps every
// range of at most phi points into a leaf.  Results depend only on which points
// share a leaf and on the boxes, so here the sorted sequence is cut into
// consecutive leaves of exactly phi points (the canonical layout the oracle
// also uses) and a complete F-ary summary tree is laid over the leaves.
#include "index.cuh"

namespace psi {

psi_status alloc_nodes(NodeArrays &a, int D, int64_t cap, bool porth, cudaStream_t s) {
  a.cap = cap;
  const size_t c = (size_t)std::max<int64_t>(cap, 1);
  psi_status st;
  for (int d = 0; d < D; ++d) {
    if ((st = DevMem::alloc((void **)&a.lo[d], sizeof(int32_t) * c, s))) return st;
    if ((st = DevMem::alloc((void **)&a.hi[d], sizeof(int32_t) * c, s))) return st;
  }
  if ((st = DevMem::alloc((void **)&a.cnt, sizeof(int32_t) * c, s))) return st;
  if ((st = DevMem::alloc((void **)&a.ref, sizeof(uint32_t) * c, s))) return st;
  if ((st = DevMem::alloc((void **)&a.kids, sizeof(int32_t) * c, s))) return st;
  if ((st = DevMem::alloc((void **)&a.depth, sizeof(int32_t) * c, s))) return st;
  if (porth && (st = DevMem::alloc((void **)&a.prefix, sizeof(uint64_t) * c, s))) return st;
  return PSI_OK;
}

void free_nodes(NodeArrays &a, cudaStream_t s) {
  for (int d = 0; d < 3; ++d) {
    DevMem::free(a.lo[d], s);
    DevMem::free(a.hi[d], s);
    a.lo[d] = a.hi[d] = nullptr;
  }
  DevMem::free(a.cnt, s);
  DevMem::free(a.ref, s);
  DevMem::free(a.kids, s);
  DevMem::free(a.depth, s);
  DevMem::free(a.prefix, s);
  a = NodeArrays();
}

psi_status alloc_pool(Pool &p, int D, int64_t slots, cudaStream_t s) {
  p.cap_slots = slots;
  const size_t c = (size_t)std::max<int64_t>(slots, 1);
  psi_status st;
  for (int d = 0; d < D; ++d)
    if ((st = DevMem::alloc((void **)&p.px[d], sizeof(int32_t) * c, s))) return st;
  if ((st = DevMem::alloc((void **)&p.pid, sizeof(uint32_t) * c, s))) return st;
  if ((st = DevMem::alloc((void **)&p.pkey, sizeof(uint64_t) * c, s))) return st;
  return PSI_OK;
}

void free_pool(Pool &p, cudaStream_t s) {
  for (int d = 0; d < 3; ++d) DevMem::free(p.px[d], s);
  DevMem::free(p.pid, s);
  DevMem::free(p.pkey, s);
  p = Pool();
}

EncodeSpec encode_spec(const psi_index *ix, const int32_t *pts) {
  EncodeSpec e;
  e.pts = pts;
  e.dim = ix->D;
  e.curve = ix->curve;
  e.bits = ix->cfg.coord_bits;
  return e;
}

namespace {

struct PoolW {
  int32_t *px[3];
  uint32_t *pid;
  uint64_t *pkey;
};

struct NodeW {
  int32_t *lo[3], *hi[3], *cnt, *kids, *depth;
  uint32_t *ref;
};

NodeW node_w(const NodeArrays &a) {
  NodeW w;
  for (int d = 0; d < 3; ++d) {
    w.lo[d] = a.lo[d];
    w.hi[d] = a.hi[d];
  }
  w.cnt = a.cnt;
  w.kids = a.kids;
  w.depth = a.depth;
  w.ref = a.ref;
  return w;
}

// One warp per group of GL consecutive leaves: gather each leaf's points by
// their sorted positions into its block (structure of arrays), reduce the
// boxes, write the leaf nodes and their separators (the first (key, id) of
// each leaf; lane u writes leaf u's).  All sorted positions of the group are loaded first, then all
// gathers are issued, so a warp keeps GL x 3 independent loads in flight
// instead of waiting on each leaf's dependent position -> point chain.
// With REC the points and ids are read from 16-byte records (k_pack_records):
// one scattered load per point instead of two.
constexpr int GL = 4;

template <int D, bool REC>
__global__ __launch_bounds__(256, 3) void k_leaf_gather(const uint64_t *skeys, const uint32_t *svals, const int32_t *pts,
                                                     const uint32_t *ids, const int4 *rec, int64_t n, int phi, int C,
                                                     PoolW pool, NodeW nodes, uint64_t *sep_key, uint32_t *sep_id,
                                                     int64_t L) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g * GL < L; g += warps) {
    const int64_t leaf0 = g * GL;
    for (int s0 = 0; s0 < phi; s0 += 32) {  // phi <= 64: at most two rounds
      const int s = s0 + lane;
      uint32_t v[GL], id[GL], okm = 0;
      uint64_t k[GL];
      int32_t c[GL][D];
#pragma unroll
      for (int u = 0; u < GL; ++u) {
        const int64_t i = (leaf0 + u) * phi + s;
        v[u] = 0u;
        k[u] = 0ull;
        id[u] = 0u;
        if (leaf0 + u < L && s < phi && i < n) {
          okm |= 1u << u;
          v[u] = svals[i];
          k[u] = skeys[i];
        }
      }
#pragma unroll
      for (int u = 0; u < GL; ++u) {
        if (okm >> u & 1u) {
          if (REC) {
            const int4 r = __ldg(rec + v[u]);
            c[u][0] = r.x;
            c[u][1] = r.y;
            if (D == 3) c[u][D - 1] = r.z;
            id[u] = (uint32_t)r.w;
          } else {
#pragma unroll
            for (int d = 0; d < D; ++d) c[u][d] = pts[(int64_t)v[u] * D + d];
            id[u] = ids[v[u]];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < GL; ++u) {
        if (okm >> u & 1u) {
          const int64_t slot = (leaf0 + u) * C + s;
#pragma unroll
          for (int d = 0; d < D; ++d) pool.px[d][slot] = c[u][d];
          pool.pid[slot] = id[u];
          pool.pkey[slot] = k[u];
        }
      }
      // each leaf's box and first (key, id), kept by lane u for leaf u
      int32_t mlo[D], mhi[D];
      uint64_t mk = 0;
      uint32_t mid = 0;
#pragma unroll
      for (int u = 0; u < GL; ++u) {
        const bool ok = okm >> u & 1u;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const int32_t lo = __reduce_min_sync(0xFFFFFFFFu, ok ? c[u][d] : INT32_MAX);
          const int32_t hi = __reduce_max_sync(0xFFFFFFFFu, ok ? c[u][d] : INT32_MIN);
          if (lane == u) {
            mlo[d] = lo;
            mhi[d] = hi;
          }
        }
        const uint64_t fk = __shfl_sync(0xFFFFFFFFu, k[u], 0);
        const uint32_t fi = __shfl_sync(0xFFFFFFFFu, id[u], 0);
        if (lane == u) {
          mk = fk;
          mid = fi;
        }
      }
      const int64_t leaf = leaf0 + lane;
      if (lane < GL && leaf < L) {
        const int cnt = (int)min((int64_t)phi, n - leaf * phi);
        if (s0 == 0) {
#pragma unroll
          for (int d = 0; d < D; ++d) {
            nodes.lo[d][leaf] = mlo[d];
            nodes.hi[d][leaf] = mhi[d];
          }
          nodes.cnt[leaf] = cnt;
          nodes.ref[leaf] = (uint32_t)(leaf * C);
          nodes.kids[leaf] = 0;
          nodes.depth[leaf] = 0;
          sep_key[leaf] = mk;
          sep_id[leaf] = mid;
        } else if (s0 < cnt) {  // second round of a leaf wider than a warp
#pragma unroll
          for (int d = 0; d < D; ++d) {
            nodes.lo[d][leaf] = min(nodes.lo[d][leaf], mlo[d]);
            nodes.hi[d][leaf] = max(nodes.hi[d][leaf], mhi[d]);
          }
        }
      }
    }
  }
}

// Points and ids of the input as 16-byte records (x, y, z or 0, id), in
// input order, for gathers by position from input that is not locally ordered.
template <int D>
__global__ void k_pack_records(const int32_t *pts, const uint32_t *ids, int64_t n, int4 *rec) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int4 r;
    r.x = pts[i * D];
    r.y = pts[i * D + 1];
    r.z = D == 3 ? pts[i * D + D - 1] : 0;
    r.w = (int)ids[i];
    rec[i] = r;
  }
}

// One warp per parent: children [child_off + j*F, ...) of the level below.
template <int D>
__global__ void k_summarise(NodeW nodes, int64_t child_off, int64_t child_n, int64_t par_off, int64_t par_n, int F,
                            int level) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < par_n; j += warps) {
    const int64_t c0 = j * F;
    const int nk = (int)min((int64_t)F, child_n - c0);
    int32_t lo[D], hi[D];
    int32_t cnt = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      lo[d] = INT32_MAX;
      hi[d] = INT32_MIN;
    }
    if (lane < nk) {
      const int64_t c = child_off + c0 + lane;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        lo[d] = nodes.lo[d][c];
        hi[d] = nodes.hi[d][c];
      }
      cnt = nodes.cnt[c];
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
      lo[d] = __reduce_min_sync(0xFFFFFFFFu, lo[d]);
      hi[d] = __reduce_max_sync(0xFFFFFFFFu, hi[d]);
    }
    cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
    if (lane == 0) {
      const int64_t p = par_off + j;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        nodes.lo[d][p] = lo[d];
        nodes.hi[d][p] = hi[d];
      }
      nodes.cnt[p] = cnt;
      nodes.ref[p] = (uint32_t)(child_off + c0);
      nodes.kids[p] = nk;
      nodes.depth[p] = level;
    }
  }
}

int warp_grid(int64_t warps, int per_block_warps = 8) {
  const int64_t blocks = ceil_div(std::max<int64_t>(warps, 1), per_block_warps);
  return (int)std::min<int64_t>(blocks, (int64_t)num_sms() * 32);
}

}  // namespace

// Summary levels above the L leaves (nodes [0, L)); node arrays must hold
// L * F / (F - 1) + levels entries.
psi_status build_spac_summary(psi_index *ix, cudaStream_t s) {
  ix->level_off.assign(1, 0);
  ix->level_size.assign(1, ix->L);
  int64_t off = 0, size = ix->L, total = ix->L;
  NodeW w = node_w(ix->nodes);
  int level = 0;
  while (size > 1) {
    const int64_t par = ceil_div(size, ix->F);
    ++level;
    if (total + par > ix->nodes.cap) {
      set_error("summary: node capacity exceeded");
      return PSI_ERR_INVALID;
    }
    if (ix->D == 2)
      PSI_LAUNCH_NAMED("k_summarise", k_summarise<2>, warp_grid(par), 256, 0, s, w, off, size, total, par, ix->F,
                       level);
    else
      PSI_LAUNCH_NAMED("k_summarise", k_summarise<3>, warp_grid(par), 256, 0, s, w, off, size, total, par, ix->F,
                       level);
    ix->level_off.push_back(total);
    ix->level_size.push_back(par);
    off = total;
    total += par;
    size = par;
  }
  ix->nnodes = ix->L > 0 ? total : 0;
  ix->root = ix->L > 0 ? (int32_t)(total - 1) : -1;
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}

int64_t summary_capacity(int64_t L, int F) {
  int64_t total = L, size = L;
  while (size > 1) {
    size = ceil_div(size, F);
    total += size;
  }
  return std::max<int64_t>(total, 1);
}

psi_status spac_from_sorted(psi_index *ix, const uint64_t *skeys, const uint32_t *svals, const int32_t *pts,
                            const uint32_t *ids, int64_t n, cudaStream_t s, bool records) {
  ix->n = n;
  ix->L = ceil_div(n, ix->phi);
  ix->pool_used = ix->L;
  PoolW pw;
  for (int d = 0; d < 3; ++d) pw.px[d] = ix->pool.px[d];
  pw.pid = ix->pool.pid;
  pw.pkey = ix->pool.pkey;
  NodeW nw = node_w(ix->nodes);
  if (ix->L > 0) {
    const int g = warp_grid(ceil_div(ix->L, GL));
    Buf<int4> rec;
    if (records) {
      psi_status st = rec.alloc(n, s);
      if (st || (st = pack_records(pts, ids, n, ix->D, rec.p, s))) return st;
    }
#define GATHER(DD, RR)                                                                                          \
  PSI_LAUNCH_NAMED("k_leaf_gather", (k_leaf_gather<DD, RR>), g, 256, 0, s, skeys, svals, pts, ids, rec.p, n, ix->phi, \
                   ix->C, pw, nw, ix->sep_key, ix->sep_id, ix->L)
    if (ix->D == 2) {
      if (records) GATHER(2, true);
      else GATHER(2, false);
    } else {
      if (records) GATHER(3, true);
      else GATHER(3, false);
    }
#undef GATHER
  }
  return build_spac_summary(ix, s);
}

}  // namespace psi

namespace psi {

psi_status pack_records(const int32_t *pts, const uint32_t *ids, int64_t n, int D, int4 *rec, cudaStream_t s) {
  if (n <= 0) return PSI_OK;
  if (D == 2)
    PSI_LAUNCH(k_pack_records<2>, warp_grid(ceil_div(n, 32)), 256, 0, s, pts, ids, n, rec);
  else
    PSI_LAUNCH(k_pack_records<3>, warp_grid(ceil_div(n, 32)), 256, 0, s, pts, ids, n, rec);
  return PSI_OK;
}

// (Re)builds a SPaC index from scratch over n points, replacing its storage.
psi_status spac_build_fresh(psi_index *ix, const int32_t *pts, const uint32_t *ids, int64_t n, cudaStream_t s) {
  free_pool(ix->pool, s);
  free_nodes(ix->nodes, s);
  DevMem::free(ix->sep_key, s);
  DevMem::free(ix->sep_id, s);
  ix->sep_key = nullptr;
  ix->sep_id = nullptr;
  const int64_t L = ceil_div(n, ix->phi);
  const int64_t blocks = L + L / 8 + 16;
  psi_status st;
  if ((st = alloc_pool(ix->pool, ix->D, blocks * ix->C, s))) return st;
  if ((st = alloc_nodes(ix->nodes, ix->D, summary_capacity(L, ix->F), false, s))) return st;
  if ((st = DevMem::alloc((void **)&ix->sep_key, sizeof(uint64_t) * std::max<int64_t>(L, 1), s))) return st;
  if ((st = DevMem::alloc((void **)&ix->sep_id, sizeof(uint32_t) * std::max<int64_t>(L, 1), s))) return st;
  Buf<uint64_t> k0, k1;
  Buf<uint32_t> v0, v1;
  if ((st = k0.alloc(n, s)) || (st = k1.alloc(n, s)) || (st = v0.alloc(n, s)) || (st = v1.alloc(n, s))) return st;
  SortResult r;
  if ((st = sort_pairs(encode_spec(ix, pts), nullptr, nullptr, n, ix->key_bits, ids, k0.p, v0.p, k1.p, v1.p,
                       ix->d_status, s, &r, ix->cfg.radix_bits)))
    return st;
  // input in random order: each point's gather by position is a scattered
  // read, so points and ids are first packed into one record per point
  return spac_from_sorted(ix, r.keys, r.vals, pts, ids, n, s, r.local == 0);
}

}  // namespace psi

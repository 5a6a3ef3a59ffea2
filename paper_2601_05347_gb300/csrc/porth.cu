// porth.cu -- P-Orth tree (Sec 3, Algorithms 1 and 2) from Morton-sorted keys.
//
// The paper notes (Sec 3.1) that its sieve-based construction is equivalent
// to an integer sort on Morton codes, lambda*D most significant bits per
// round.  Here the points are sorted once on their full Morton keys (the
// library's onesweep sort) and kept contiguously in key order; the tree is a
// function of that order:
//
//   Leaf cells.  The cell of depth l containing key k_i holds more than phi
//   points iff some phi+1 consecutive sorted keys around i share their top l
//   digits (digit = D key bits).  With m_j = common leading digits of k_j and
//   k_{j+phi}, and M_i = max of m_j over the windows [j, j+phi] that contain
//   i, the leaf holding point i sits at depth d_i = min(M_i + 1, b): the first
//   depth at which its cell holds at most phi points (Algorithm 1 line 2), or
//   the full depth b when the cell is a single grid point (duplicates).
//   A leaf starts wherever (d_i, cell of i at depth d_i) changes.
//
//   Internal nodes.  With leaves in key order, leaf i heads the nodes at
//   depths c_i + 1 .. d_i, where c_i is the number of leading digits its cell
//   shares with the previous leaf's cell (c_0 = -1).  Sorting the (depth,
//   first leaf) pairs lays the nodes out depth by depth in key order, so the
//   children of a node (the next depth's nodes whose first leaf lies inside
//   its cell) are contiguous.  Boxes are unions of the children, bottom up.
//
// Updates (Algorithm 2) rely on history independence (Sec 5.1.3 "Impact of
// Updates to Queries"): the tree after a batch is the tree of the new point
// set.  An insert merges the sorted batch into the sorted points; a delete
// removes matching (point, id) pairs; both then re-derive leaves and nodes.
#include "index.cuh"

namespace psi {
namespace {

int grid_for(int64_t n, int threads = 256) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, threads), (int64_t)num_sms() * 32));
}

__device__ __forceinline__ int common_digits(uint64_t a, uint64_t b, int K, int D, int bits) {
  const uint64_t x = a ^ b;
  if (x == 0) return bits;
  return (__clzll((long long)x) - (64 - K)) / D;
}

__device__ __forceinline__ uint64_t cell_of(uint64_t k, int depth, int D, int bits) {
  const int sh = D * (bits - depth);
  return sh >= 64 ? 0 : (k >> sh);
}

// Gather the sorted points into the contiguous pool: GP items per thread,
// all positions loaded first, then all gathers, so that each thread keeps
// several independent random loads in flight.
constexpr int GP = 4;

template <int D>
__global__ void k_porth_gather(const uint64_t *skeys, const uint32_t *svals, const int32_t *pts, const uint32_t *ids,
                               int64_t n, Pool pool) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * GP;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x * GP + threadIdx.x; i0 < n; i0 += stride) {
    uint32_t v[GP];
#pragma unroll
    for (int u = 0; u < GP; ++u) {
      const int64_t i = i0 + (int64_t)u * blockDim.x;
      v[u] = i < n ? svals[i] : 0u;
    }
    int32_t c[GP][D];
    uint32_t id[GP];
#pragma unroll
    for (int u = 0; u < GP; ++u) {
      const int64_t i = i0 + (int64_t)u * blockDim.x;
      if (i < n) {
#pragma unroll
        for (int d = 0; d < D; ++d) c[u][d] = pts[(int64_t)v[u] * D + d];
        id[u] = ids[v[u]];
      }
    }
#pragma unroll
    for (int u = 0; u < GP; ++u) {
      const int64_t i = i0 + (int64_t)u * blockDim.x;
      if (i < n) {
#pragma unroll
        for (int d = 0; d < D; ++d) pool.px[d][i] = c[u][d];
        pool.pid[i] = id[u];
        pool.pkey[i] = skeys[i];
      }
    }
  }
}

constexpr int LT = 256;  // positions per block in the leaf-depth kernel (8 blocks per SM overlap their loads)

// Leaf depth of every point and leaf-start flags.
__global__ __launch_bounds__(LT) void k_leaf_depth(const uint64_t *keys, int64_t n, int phi, int K, int D, int bits,
                                                   int32_t *ldepth) {
  __shared__ uint64_t sk[LT + 2 * 64 + 1];
  __shared__ int8_t sm[LT + 64];
  const int64_t base = (int64_t)blockIdx.x * LT;
  // keys [base - phi, base + LT + phi)
  for (int t = threadIdx.x; t < LT + 2 * phi; t += blockDim.x) {
    const int64_t g = base - phi + t;
    sk[t] = (g >= 0 && g < n) ? keys[g] : 0;
  }
  __syncthreads();
  // m_j for j in [base - phi, base + LT): window [j, j + phi]
  for (int t = threadIdx.x; t < LT + phi; t += blockDim.x) {
    const int64_t j = base - phi + t;
    int m = -1;
    if (j >= 0 && j + phi < n) m = common_digits(sk[t], sk[t + phi], K, D, bits);
    sm[t] = (int8_t)m;
  }
  __syncthreads();
  // maximum over each window [t, t + phi] by doubling: after the round with
  // step k every entry holds the maximum of the 2k entries from it (-1, "no
  // pair", is neutral); the window is then two overlapping power-of-two spans
  const int w = phi + 1;
  int p2 = 1;
  while (2 * p2 <= w) p2 *= 2;
  for (int k = 1; k < p2; k *= 2) {
    int8_t v[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int t = threadIdx.x + r * LT;
      v[r] = -1;
      if (t < LT + phi) v[r] = (int8_t)max((int)sm[t], t + k < LT + phi ? (int)sm[t + k] : -1);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int t = threadIdx.x + r * LT;
      if (t < LT + phi) sm[t] = v[r];
    }
    __syncthreads();
  }
  const int64_t i = base + threadIdx.x;
  if (i < n) {
    const int t = threadIdx.x;
    const int M = max((int)sm[t], (int)sm[t + w - p2]);
    ldepth[i] = min(M + 1, bits);
  }
}

__global__ void k_leaf_starts(const uint64_t *keys, const int32_t *ldepth, int64_t n, int D, int bits,
                              int32_t *is_start) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int s = 1;
    if (i > 0) {
      const int d = ldepth[i];
      s = d != ldepth[i - 1] || cell_of(keys[i], d, D, bits) != cell_of(keys[i - 1], d, D, bits);
    }
    is_start[i] = s;
  }
}

// Leaf list: begin, depth, cell start key.
__global__ void k_leaf_list(const uint64_t *keys, const int32_t *ldepth, const int32_t *is_start, const int64_t *rank,
                            int64_t n, int D, int bits, int64_t *lb, int32_t *ld, uint64_t *lkey) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!is_start[i]) continue;
    const int64_t r = rank[i];
    const int d = ldepth[i];
    const int sh = D * (bits - d);
    lb[r] = i;
    ld[r] = d;
    lkey[r] = sh >= 64 ? 0 : ((keys[i] >> sh) << sh);
  }
}

// Nodes headed by each leaf: depths c_i + 1 .. d_i.
__global__ void k_heads(const int32_t *ld, const uint64_t *lkey, int64_t L, int K, int D, int bits, int32_t *c,
                        int64_t *nn) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (int64_t)gridDim.x * blockDim.x) {
    const int ci = i == 0 ? -1 : common_digits(lkey[i - 1], lkey[i], K, D, bits);
    c[i] = ci;
    nn[i] = ld[i] - ci;
  }
}

// Node records in preorder -- key = depth, value = first leaf -- and the
// number of nodes per depth (counted in shared memory, one global add per
// block and depth).  Preorder lists the nodes of each depth by first leaf, so
// one stable pass on the depth digit orders them depth-major, leaf-minor.
__global__ void k_emit_nodes(const int32_t *ld, const int32_t *c, const int64_t *base, int64_t L, uint64_t *nkey,
                             uint32_t *nval, int32_t *depth_hist) {
  __shared__ int32_t sh[64];
  for (int i = threadIdx.x; i < 64; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t o = base[i];
    for (int l = c[i] + 1; l <= ld[i]; ++l, ++o) {
      nkey[o] = (uint64_t)l;
      nval[o] = (uint32_t)i;
      atomicAdd(&sh[l], 1);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 64; i += blockDim.x)
    if (sh[i]) atomicAdd(&depth_hist[i], sh[i]);
}

struct LinkArgs {
  const uint64_t *ndepth;  // node depth, depth-major order
  const uint32_t *nleaf;   // node's first leaf, ascending within a depth
  const int64_t *doff;   // [bits + 2] depth offsets
  const int64_t *lb;     // leaf begin slot
  const int32_t *ld;
  const uint64_t *lkey;
  int64_t L, N, n;
  int D, bits;
  NodeArrays nodes;
  int32_t *leaf_node;
};

__global__ void k_link(LinkArgs a) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < a.N; x += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)a.ndepth[x];
    const int64_t i = (int64_t)a.nleaf[x];
    const int sh = a.D * (a.bits - l);
    const uint64_t prefix = sh >= 64 ? 0 : (a.lkey[i] >> sh);
    a.nodes.depth[x] = l;
    a.nodes.prefix[x] = prefix;
    if (l == a.ld[i]) {
      const int64_t e = i + 1 < a.L ? a.lb[i + 1] : a.n;
      a.nodes.ref[x] = (uint32_t)a.lb[i];
      a.nodes.kids[x] = 0;
      a.nodes.cnt[x] = (int32_t)(e - a.lb[i]);
      a.leaf_node[i] = (int32_t)x;
      continue;
    }
    // first leaf past this node's cell
    const uint64_t lim = (prefix + 1) << sh;  // sh <= 63 for an internal node
    int64_t lo = i + 1, hi = a.L;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (a.lkey[mid] < lim)
        lo = mid + 1;
      else
        hi = mid;
    }
    const int64_t e = lo;
    // children: depth l+1 nodes whose first leaf lies in [i, e)
    const int64_t s0 = a.doff[l + 1], s1 = a.doff[l + 2];
    int64_t c0 = s0, c1 = s1;
    {
      int64_t p = s0, q = s1;
      while (p < q) {
        const int64_t mid = (p + q) >> 1;
        if ((int64_t)a.nleaf[mid] < i)
          p = mid + 1;
        else
          q = mid;
      }
      c0 = p;
      q = s1;
      while (p < q) {
        const int64_t mid = (p + q) >> 1;
        if ((int64_t)a.nleaf[mid] < e)
          p = mid + 1;
        else
          q = mid;
      }
      c1 = p;
    }
    a.nodes.ref[x] = (uint32_t)c0;
    a.nodes.kids[x] = (int32_t)(c1 - c0);
    const int64_t pe = e < a.L ? a.lb[e] : a.n;
    a.nodes.cnt[x] = (int32_t)(pe - a.lb[i]);
  }
}

// Boxes of the nodes of one depth: leaves from their points, internal nodes
// from their children.
template <int D>
__global__ void k_boxes(NodeArrays nodes, Pool pool, int64_t off, int64_t cnt) {
  // an 8-lane group per node (at most 2^D <= 8 children; leaf points 8 at a
  // time), four nodes per warp
  const int lane = threadIdx.x & 31, g = lane >> 3, gl = lane & 7;
  const unsigned gmask = 0xFFu << (g * 8);
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t x0 = off + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 4; x0 < off + cnt;
       x0 += warps * 4) {
    const int64_t x = x0 + g;
    const bool valid = x < off + cnt;
    int32_t lo[D], hi[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      lo[d] = INT32_MAX;
      hi[d] = INT32_MIN;
    }
    if (valid) {
      const int nk = nodes.kids[x];
      const uint32_t r = nodes.ref[x];
      if (nk == 0) {
        const int c = nodes.cnt[x];
        for (int s = gl; s < c; s += 8)
#pragma unroll
          for (int d = 0; d < D; ++d) {
            const int32_t v = pool.px[d][r + s];
            lo[d] = min(lo[d], v);
            hi[d] = max(hi[d], v);
          }
      } else if (gl < nk) {
#pragma unroll
        for (int d = 0; d < D; ++d) {
          lo[d] = nodes.lo[d][r + gl];
          hi[d] = nodes.hi[d][r + gl];
        }
      }
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
      lo[d] = __reduce_min_sync(gmask, lo[d]);
      hi[d] = __reduce_max_sync(gmask, hi[d]);
    }
    if (valid && gl == 0)
#pragma unroll
      for (int d = 0; d < D; ++d) {
        nodes.lo[d][x] = lo[d];
        nodes.hi[d][x] = hi[d];
      }
  }
}

// ---- updates ----------------------------------------------------------------

// Rank of each batch item among the pool's (key, id) order; count of batch
// items before each pool position.
__global__ void k_merge_ranks(const uint64_t *pkey, const uint32_t *pid, int64_t n, const uint64_t *bkeys,
                              const uint32_t *bvals, const uint32_t *ids, int64_t m, int64_t *brank,
                              int32_t *delta) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = bkeys[j];
    const uint32_t id = ids[bvals[j]];
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (kid_less(pkey[mid], pid[mid], k, id))
        lo = mid + 1;
      else
        hi = mid;
    }
    brank[j] = lo;
    atomicAdd(&delta[lo], 1);
  }
}

template <int D>
__global__ void k_merge_scatter(Pool oldp, int64_t n, const int64_t *shift, const uint64_t *bkeys,
                                const uint32_t *bvals, const int32_t *pts, const uint32_t *ids, int64_t m,
                                const int64_t *brank, Pool np) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t o = i + shift[i];
#pragma unroll
    for (int d = 0; d < D; ++d) np.px[d][o] = oldp.px[d][i];
    np.pid[o] = oldp.pid[i];
    np.pkey[o] = oldp.pkey[i];
  }
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
    const int64_t o = brank[j] + j;
    const uint32_t v = bvals[j];
#pragma unroll
    for (int d = 0; d < D; ++d) np.px[d][o] = pts[(int64_t)v * D + d];
    np.pid[o] = ids[v];
    np.pkey[o] = bkeys[j];
  }
}

template <int D>
__global__ void k_mark_deleted(const uint64_t *pkey, const uint32_t *pid, Pool pool, int64_t n, const uint64_t *bkeys,
                               const uint32_t *bvals, const int32_t *pts, const uint32_t *ids, int64_t m,
                               int32_t *keep, unsigned long long *deleted) {
  uint32_t removed = 0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = bkeys[j];
    const uint32_t v = bvals[j];
    const uint32_t id = ids[v];
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (kid_less(pkey[mid], pid[mid], k, id))
        lo = mid + 1;
      else
        hi = mid;
    }
    if (lo < n && pkey[lo] == k && pid[lo] == id) {
      bool same = true;
#pragma unroll
      for (int d = 0; d < D; ++d) same &= pool.px[d][lo] == pts[(int64_t)v * D + d];
      if (same && atomicExch(&keep[lo], 0) == 1) ++removed;
    }
  }
  block_count_add(deleted, removed);
}

template <int D>
__global__ void k_compact_points(Pool oldp, int64_t n, const int32_t *keep, const int64_t *pos, Pool np) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!keep[i]) continue;
    const int64_t o = pos[i];
#pragma unroll
    for (int d = 0; d < D; ++d) np.px[d][o] = oldp.px[d][i];
    np.pid[o] = oldp.pid[i];
    np.pkey[o] = oldp.pkey[i];
  }
}

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

__global__ void k_i64_from_u64(const unsigned long long *a, int64_t *b) { *b = (int64_t)*a; }

}  // namespace

// Leaves and nodes of the P-Orth tree over the ix->n sorted points in the pool.
psi_status porth_derive(psi_index *ix, cudaStream_t s) {
  const int64_t n = ix->n;
  const int D = ix->D, bits = ix->cfg.coord_bits, K = ix->key_bits;
  free_nodes(ix->nodes, s);
  DevMem::free(ix->leaf_node, s);
  ix->leaf_node = nullptr;
  ix->L = 0;
  ix->nnodes = 0;
  ix->root = -1;
  if (n == 0) return PSI_OK;
  psi_status st;
  Buf<int32_t> ldepth, is_start;
  Buf<int64_t> rank, tot;
  if ((st = ldepth.alloc(n, s)) || (st = is_start.alloc(n, s)) || (st = rank.alloc(n, s)) || (st = tot.alloc(2, s)))
    return st;
  PSI_LAUNCH(k_leaf_depth, (unsigned)ceil_div(n, LT), LT, 0, s, ix->pool.pkey, n, ix->phi, K, D, bits, ldepth.p);
  PSI_LAUNCH(k_leaf_starts, grid_for(n), 256, 0, s, ix->pool.pkey, ldepth.p, n, D, bits, is_start.p);
  if ((st = scan_i32_to_i64(is_start.p, rank.p, n, tot.p, s))) return st;
  int64_t L = 0;
  PSI_CK(cudaMemcpyAsync(&L, tot.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaStreamSynchronize(s));

  Buf<int64_t> lb, nn;
  Buf<int32_t> ld, c, hist;
  Buf<uint64_t> lkey;
  if ((st = lb.alloc(L, s)) || (st = nn.alloc(L, s)) || (st = ld.alloc(L, s)) || (st = c.alloc(L, s)) ||
      (st = lkey.alloc(L, s)) || (st = hist.alloc(64, s)))
    return st;
  PSI_LAUNCH(k_leaf_list, grid_for(n), 256, 0, s, ix->pool.pkey, ldepth.p, is_start.p, rank.p, n, D, bits, lb.p, ld.p,
             lkey.p);
  PSI_LAUNCH(k_heads, grid_for(L), 256, 0, s, ld.p, lkey.p, L, K, D, bits, c.p, nn.p);
  if ((st = scan_i64(nn.p, nn.p, L, tot.p + 1, s))) return st;
  int64_t N = 0;
  PSI_CK(cudaMemcpyAsync(&N, tot.p + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaMemsetAsync(hist.p, 0, sizeof(int32_t) * 64, s));
  PSI_CK(cudaStreamSynchronize(s));

  Buf<uint64_t> nk0, nk1;
  Buf<uint32_t> nv0, nv1;
  if ((st = nk0.alloc(N, s)) || (st = nk1.alloc(N, s)) || (st = nv0.alloc(N, s)) || (st = nv1.alloc(N, s))) return st;
  PSI_LAUNCH(k_emit_nodes, grid_for(L), 256, 0, s, ld.p, c.p, nn.p, L, nk0.p, nv0.p, hist.p);
  int32_t h_hist[64];
  PSI_CK(cudaMemcpyAsync(h_hist, hist.p, sizeof(h_hist), cudaMemcpyDeviceToHost, s));
  SortResult r;
  EncodeSpec none;
  Buf<int> sst;
  if ((st = sst.alloc(1, s))) return st;
  PSI_CK(cudaMemsetAsync(sst.p, 0, sizeof(int), s));
  // one stable digit pass on the depth (< 64); the input arrays double as the
  // second ping-pong buffer
  if ((st = sort_pairs(none, nk0.p, nv0.p, N, 8, nullptr, nk1.p, nv1.p, nk0.p, nv0.p, sst.p, s, &r)))
    return st;
  PSI_CK(cudaStreamSynchronize(s));
  std::vector<int64_t> doff(bits + 3, 0);
  for (int l = 0; l <= bits; ++l) doff[l + 1] = doff[l] + h_hist[l];
  doff[bits + 2] = doff[bits + 1];
  Buf<int64_t> d_doff;
  if ((st = d_doff.alloc(doff.size(), s))) return st;
  PSI_CK(cudaMemcpyAsync(d_doff.p, doff.data(), sizeof(int64_t) * doff.size(), cudaMemcpyHostToDevice, s));

  if ((st = alloc_nodes(ix->nodes, D, N, true, s))) return st;
  if ((st = DevMem::alloc((void **)&ix->leaf_node, sizeof(int32_t) * L, s))) return st;
  LinkArgs la{r.keys, r.vals, d_doff.p, lb.p, ld.p, lkey.p, L, N, n, D, bits, ix->nodes, ix->leaf_node};
  PSI_LAUNCH(k_link, grid_for(N), 256, 0, s, la);
  int maxd = 0;
  for (int l = 0; l <= bits; ++l)
    if (h_hist[l]) maxd = l;
  for (int l = maxd; l >= 0; --l) {
    const int64_t cnt = doff[l + 1] - doff[l];
    if (!cnt) continue;
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(cnt, 32), (int64_t)num_sms() * 32));
    if (D == 2)
      PSI_LAUNCH_NAMED("k_boxes", k_boxes<2>, g, 256, 0, s, ix->nodes, ix->pool, doff[l], cnt);
    else
      PSI_LAUNCH_NAMED("k_boxes", k_boxes<3>, g, 256, 0, s, ix->nodes, ix->pool, doff[l], cnt);
  }
  ix->L = L;
  ix->nnodes = N;
  ix->root = 0;
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}

psi_status porth_build(psi_index *ix, const int32_t *pts, const uint32_t *ids, int64_t n, cudaStream_t s) {
  psi_status st;
  ix->n = n;
  if ((st = alloc_pool(ix->pool, ix->D, std::max<int64_t>(n, 1), s))) return st;
  ix->pool_used = n;
  if (n == 0) return porth_derive(ix, s);
  Buf<uint64_t> k0, k1;
  Buf<uint32_t> v0, v1;
  if ((st = k0.alloc(n, s)) || (st = k1.alloc(n, s)) || (st = v0.alloc(n, s)) || (st = v1.alloc(n, s))) return st;
  SortResult r;
  if ((st = sort_pairs(encode_spec(ix, pts), nullptr, nullptr, n, ix->key_bits, ids, k0.p, v0.p, k1.p, v1.p,
                       ix->d_status, s, &r, ix->cfg.radix_bits)))
    return st;
  if (ix->D == 2)
    PSI_LAUNCH_NAMED("k_porth_gather", k_porth_gather<2>, grid_for(n), 256, 0, s, r.keys, r.vals, pts, ids, n,
                     ix->pool);
  else
    PSI_LAUNCH_NAMED("k_porth_gather", k_porth_gather<3>, grid_for(n), 256, 0, s, r.keys, r.vals, pts, ids, n,
                     ix->pool);
  return porth_derive(ix, s);
}

psi_status porth_insert(psi_index *ix, const int32_t *pts, const uint32_t *ids, int64_t m, cudaStream_t s) {
  psi_status st;
  const int64_t n = ix->n;
  Buf<uint64_t> k0, k1;
  Buf<uint32_t> v0, v1;
  if ((st = k0.alloc(m, s)) || (st = k1.alloc(m, s)) || (st = v0.alloc(m, s)) || (st = v1.alloc(m, s))) return st;
  SortResult r;
  if ((st = sort_pairs(encode_spec(ix, pts), nullptr, nullptr, m, ix->key_bits, ids, k0.p, v0.p, k1.p, v1.p,
                       ix->d_status, s, &r, ix->cfg.radix_bits)))
    return st;
  Buf<int64_t> brank, shift;
  Buf<int32_t> delta;
  if ((st = brank.alloc(m, s)) || (st = delta.alloc(n + 1, s)) || (st = shift.alloc(n + 1, s))) return st;
  PSI_CK(cudaMemsetAsync(delta.p, 0, sizeof(int32_t) * (n + 1), s));
  PSI_LAUNCH(k_merge_ranks, grid_for(m), 256, 0, s, ix->pool.pkey, ix->pool.pid, n, r.keys, r.vals, ids, m, brank.p,
             delta.p);
  // Pool item i moves up by the number of batch items ranked at or before i:
  // the exclusive scan of delta taken at i + 1.
  if ((st = scan_i32_to_i64(delta.p, shift.p, n + 1, nullptr, s))) return st;
  Pool np;
  if ((st = alloc_pool(np, ix->D, n + m, s))) {
    free_pool(np, s);
    return st;
  }
  if (ix->D == 2)
    PSI_LAUNCH_NAMED("k_merge_scatter", k_merge_scatter<2>, grid_for(n + m), 256, 0, s, ix->pool, n, shift.p + 1,
                     r.keys, r.vals, pts, ids, m, brank.p, np);
  else
    PSI_LAUNCH_NAMED("k_merge_scatter", k_merge_scatter<3>, grid_for(n + m), 256, 0, s, ix->pool, n, shift.p + 1,
                     r.keys, r.vals, pts, ids, m, brank.p, np);
  free_pool(ix->pool, s);
  ix->pool = np;
  ix->n = n + m;
  ix->pool_used = n + m;
  return porth_derive(ix, s);
}

psi_status porth_delete(psi_index *ix, const int32_t *pts, const uint32_t *ids, int64_t m, int64_t *d_deleted,
                        cudaStream_t s) {
  psi_status st;
  const int64_t n = ix->n;
  Buf<uint64_t> k0, k1;
  Buf<uint32_t> v0, v1;
  if ((st = k0.alloc(m, s)) || (st = k1.alloc(m, s)) || (st = v0.alloc(m, s)) || (st = v1.alloc(m, s))) return st;
  SortResult r;
  if ((st = sort_pairs(encode_spec(ix, pts), nullptr, nullptr, m, ix->key_bits, ids, k0.p, v0.p, k1.p, v1.p,
                       ix->d_status, s, &r, ix->cfg.radix_bits)))
    return st;
  Buf<int32_t> keep;
  Buf<int64_t> pos, tot;
  Buf<unsigned long long> del;
  if ((st = keep.alloc(n, s)) || (st = pos.alloc(n, s)) || (st = tot.alloc(2, s)) || (st = del.alloc(1, s))) return st;
  PSI_LAUNCH(k_fill_i32, grid_for(n), 256, 0, s, keep.p, n, 1);
  PSI_CK(cudaMemsetAsync(del.p, 0, sizeof(unsigned long long), s));
  if (ix->D == 2)
    PSI_LAUNCH_NAMED("k_mark_deleted", k_mark_deleted<2>, grid_for(m), 256, 0, s, ix->pool.pkey, ix->pool.pid,
                     ix->pool, n, r.keys, r.vals, pts, ids, m, keep.p, del.p);
  else
    PSI_LAUNCH_NAMED("k_mark_deleted", k_mark_deleted<3>, grid_for(m), 256, 0, s, ix->pool.pkey, ix->pool.pid,
                     ix->pool, n, r.keys, r.vals, pts, ids, m, keep.p, del.p);
  if ((st = scan_i32_to_i64(keep.p, pos.p, n, tot.p, s))) return st;
  PSI_LAUNCH(k_i64_from_u64, 1, 1, 0, s, del.p, tot.p + 1);
  if (d_deleted) PSI_CK(cudaMemcpyAsync(d_deleted, tot.p + 1, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  int64_t h[2];
  PSI_CK(cudaMemcpyAsync(h, tot.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaStreamSynchronize(s));
  Pool np;
  if ((st = alloc_pool(np, ix->D, std::max<int64_t>(h[0], 1), s))) {
    free_pool(np, s);
    return st;
  }
  if (ix->D == 2)
    PSI_LAUNCH_NAMED("k_compact_points", k_compact_points<2>, grid_for(n), 256, 0, s, ix->pool, n, keep.p, pos.p, np);
  else
    PSI_LAUNCH_NAMED("k_compact_points", k_compact_points<3>, grid_for(n), 256, 0, s, ix->pool, n, keep.p, pos.p, np);
  free_pool(ix->pool, s);
  ix->pool = np;
  ix->n = h[0];
  ix->pool_used = h[0];
  return porth_derive(ix, s);
}

}  // namespace psi

// porth.cu -- P-Orth tree (Sec 3, Algorithms 1 and 2) from Morton-sorted keys.
//
// The paper notes (Sec 3.1) that its sieve-based construction is equivalent
// to an integer sort on Morton codes, lambda*D most significant bits per
// round.  Here the points are sorted once on their full Morton keys (the
// library's onesweep sort); the tree is a function of that order:
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
// Storage: the leaf list (PLeaves) is kept in key order; each leaf owns a
// slot range of the pool holding its points sorted by (key, id).  The node
// arrays are derived from the leaf list (O(leaves), not O(points)).
//
// Updates (Algorithm 2: sieve the batch to the leaves it reaches and rebuild
// only those).  A leaf's depth depends only on the phi+1 keys around each of
// its points, so a batch changes only the leaves within phi+1 points of an
// inserted or deleted point.  Each batch point is routed to the leaf whose
// key range holds it; the leaves within phi+1 points of a routed leaf are
// marked dirty; each maximal run of dirty leaves (a segment) is rebuilt from
// its own points merged with (or stripped of) the batch points, with phi+1
// keys of the clean neighbours on each side as context for the depth windows,
// into fresh slots; the other leaves keep their records and slots.  The
// result equals a fresh build of the new point set (history independence,
// Sec 5.1.3), which the parity tests check node by node.
#include "index.cuh"

namespace psi {

psi_status alloc_pleaves(PLeaves &a, int D, int64_t cap, cudaStream_t s) {
  a.cap = cap;
  const size_t c = (size_t)std::max<int64_t>(cap, 1);
  psi_status st;
  if ((st = DevMem::alloc((void **)&a.ref, sizeof(uint32_t) * c, s)) ||
      (st = DevMem::alloc((void **)&a.cnt, sizeof(int32_t) * c, s)) ||
      (st = DevMem::alloc((void **)&a.depth, sizeof(int32_t) * c, s)) ||
      (st = DevMem::alloc((void **)&a.key, sizeof(uint64_t) * c, s)))
    return st;
  for (int d = 0; d < D; ++d)
    if ((st = DevMem::alloc((void **)&a.lo[d], sizeof(int32_t) * c, s)) ||
        (st = DevMem::alloc((void **)&a.hi[d], sizeof(int32_t) * c, s)))
      return st;
  return PSI_OK;
}

void free_pleaves(PLeaves &a, cudaStream_t s) {
  DevMem::free(a.ref, s);
  DevMem::free(a.cnt, s);
  DevMem::free(a.depth, s);
  DevMem::free(a.key, s);
  for (int d = 0; d < 3; ++d) {
    DevMem::free(a.lo[d], s);
    DevMem::free(a.hi[d], s);
  }
  a = PLeaves();
}

namespace {

int grid_for(int64_t n, int threads = 256) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, threads), (int64_t)num_sms() * 32));
}

int warp_grid(int64_t warps) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(warps, 8), (int64_t)num_sms() * 32));
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
// several independent random loads in flight.  With REC the points and ids
// are read from 16-byte records (pack_records): one load per point.
constexpr int GP = 4;

template <int D, bool REC>
__global__ void k_porth_gather(const uint64_t *skeys, const uint32_t *svals, const int32_t *pts, const uint32_t *ids,
                               const int4 *rec, int64_t n, Pool pool) {
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

// Leaf-depth kernel: LDE positions per block of LDT threads (phi <= 64).
constexpr int LDT = 256, LDE = 2048;

// Leaf depth of every position of a key array (positions outside [0, n)
// contribute no window).  m_j = common digits of (k_j, k_{j+phi}); position i
// takes 1 + the maximum of m_j over the window j in [i - phi, i].  The window
// maximum comes from running maxima over segments of phi entries (van Herk;
// Gil and Werman): the window starting at entry u spans the rest of u's
// segment and the next segment up to u + phi, so it is the maximum of u's
// suffix maximum and the prefix maximum at u + phi.
__global__ __launch_bounds__(LDT) void k_leaf_depth(const uint64_t *keys, int64_t n, int phi, int K, int D, int bits,
                                                    int32_t *ldepth) {
  __shared__ uint64_t sk[LDE + 2 * 64];
  __shared__ int8_t sm[LDE + 64], spre[LDE + 64], ssuf[LDE + 64];
  const int64_t base = (int64_t)blockIdx.x * LDE;
  // keys [base - phi, base + LDE + phi)
  for (int t = threadIdx.x; t < LDE + 2 * phi; t += LDT) {
    const int64_t g = base - phi + t;
    sk[t] = (g >= 0 && g < n) ? keys[g] : 0;
  }
  __syncthreads();
  // entry t is m_j for j = base - phi + t, t in [0, LDE + phi); -1 ("no
  // pair") is neutral for the maximum
  const int nm = LDE + phi;
  for (int t = threadIdx.x; t < nm; t += LDT) {
    const int64_t j = base - phi + t;
    int m = -1;
    if (j >= 0 && j + phi < n) m = common_digits(sk[t], sk[t + phi], K, D, bits);
    sm[t] = (int8_t)m;
  }
  __syncthreads();
  // per segment [a, a + phi): prefix maxima (even tasks), suffix maxima (odd)
  const int nseg = (nm + phi - 1) / phi;
  for (int q = threadIdx.x; q < 2 * nseg; q += LDT) {
    const int a = (q >> 1) * phi, b = min(a + phi, nm);
    int r = -1;
    if (q & 1) {
      for (int t = b - 1; t >= a; --t) {
        r = max(r, (int)sm[t]);
        ssuf[t] = (int8_t)r;
      }
    } else {
      for (int t = a; t < b; ++t) {
        r = max(r, (int)sm[t]);
        spre[t] = (int8_t)r;
      }
    }
  }
  __syncthreads();
  for (int u = threadIdx.x; u < LDE; u += LDT) {
    const int64_t i = base + u;
    if (i >= n) break;
    const int M = max((int)ssuf[u], (int)spre[u + phi]);
    ldepth[i] = min(M + 1, bits);
  }
}

// ---- leaves from a key array -------------------------------------------------
// A work array lists keys in sorted order: the points of the leaves being
// (re)built (mask 1, each with its pool slot; a leaf's points occupy
// consecutive slots) and, between runs of them, context keys of unchanged
// neighbours (mask 0) that only feed the depth windows.  A null mask means
// every position is a point and its slot is slot0 + position.

struct WorkArray {
  const uint64_t *key;
  const int32_t *mask;  // or null
  const uint32_t *slot;  // or null (slot0 + position)
  uint32_t slot0;
  int64_t n;
};

__device__ __forceinline__ bool work_point(const WorkArray &w, int64_t i) { return !w.mask || w.mask[i]; }
__device__ __forceinline__ uint32_t work_slot(const WorkArray &w, int64_t i) {
  return w.slot ? w.slot[i] : w.slot0 + (uint32_t)i;
}

// start[i]: point i begins a leaf (a run's first point, or its (depth, cell)
// differs from the previous point's).
__global__ void k_work_starts(WorkArray w, const int32_t *ldepth, int D, int bits, int32_t *start) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < w.n; i += (int64_t)gridDim.x * blockDim.x) {
    int s = 0;
    if (work_point(w, i)) {
      s = 1;
      if (i > 0 && work_point(w, i - 1)) {
        const int d = ldepth[i];
        s = d != ldepth[i - 1] || cell_of(w.key[i], d, D, bits) != cell_of(w.key[i - 1], d, D, bits);
      }
    }
    start[i] = s;
  }
}

// Leaf records: leaf rank[i] for every start i (first slot, depth, cell
// key).  The points of consecutive leaves occupy consecutive slots (a build's
// pool, or the fresh slots of an update in work order), so counts follow
// from the first slots (k_leaf_counts).
__global__ void k_work_leaves(WorkArray w, const int32_t *ldepth, const int32_t *start, const int64_t *rank, int D,
                              int bits, PLeaves out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < w.n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!work_point(w, i) || !start[i]) continue;
    const int64_t r = rank[i];
    const int d = ldepth[i];
    const int sh = D * (bits - d);
    out.ref[r] = work_slot(w, i);
    out.depth[r] = d;
    out.key[r] = sh >= 64 ? 0 : ((w.key[i] >> sh) << sh);
  }
}

// cnt[r] = ref[r + 1] - ref[r]; the last leaf ends at slot `end`.
__global__ void k_leaf_counts(PLeaves pl, int64_t L, uint32_t end) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < L; r += (int64_t)gridDim.x * blockDim.x)
    pl.cnt[r] = (int32_t)((r + 1 < L ? pl.ref[r + 1] : end) - pl.ref[r]);
}

// Leaf boxes by a segmented reduction over the points in work order (each
// point's leaf = the rank of its leaf's start): lanes of a warp combine the
// points of the same leaf, and the first lane of each leaf in the warp
// merges the result into the leaf's box (boxes start empty).
template <int D>
__global__ void k_work_boxes(WorkArray w, const int32_t *start, const int64_t *rank, Pool pool, PLeaves pl) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < w.n; i0 += stride) {
    const int64_t i = i0 + threadIdx.x;
    const bool pt = i < w.n && work_point(w, i);
    int64_t leaf = pt ? rank[i] + start[i] - 1 : -1;
    int32_t lo[D], hi[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int32_t v = pt ? pool.px[d][work_slot(w, i)] : 0;
      lo[d] = pt ? v : INT32_MAX;
      hi[d] = pt ? v : INT32_MIN;
    }
    // inclusive segmented scan (min / max) over lanes with the same leaf
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t ol = __shfl_down_sync(0xFFFFFFFFu, leaf, o);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int32_t a = __shfl_down_sync(0xFFFFFFFFu, lo[d], o);
        const int32_t b = __shfl_down_sync(0xFFFFFFFFu, hi[d], o);
        if (lane + o < 32 && ol == leaf) {
          lo[d] = min(lo[d], a);
          hi[d] = max(hi[d], b);
        }
      }
    }
    const int64_t pl_leaf = __shfl_up_sync(0xFFFFFFFFu, leaf, 1);
    if (pt && (lane == 0 || pl_leaf != leaf)) {
#pragma unroll
      for (int d = 0; d < D; ++d) {
        atomicMin(&pl.lo[d][leaf], lo[d]);
        atomicMax(&pl.hi[d][leaf], hi[d]);
      }
    }
  }
}

__global__ void k_empty_boxes(PLeaves pl, int64_t L, int D) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < L; r += (int64_t)gridDim.x * blockDim.x)
    for (int d = 0; d < D; ++d) {
      pl.lo[d][r] = INT32_MAX;
      pl.hi[d][r] = INT32_MIN;
    }
}

// ---- nodes from the leaf list ---------------------------------------------

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
  const int64_t *doff;     // [bits + 2] depth offsets
  const int64_t *E;        // exclusive prefix sums of the leaf counts (L + 1)
  PLeaves pl;
  int64_t L, N;
  int D, bits;
  NodeArrays nodes;
  int32_t *leaf_node;
  // internal nodes whose boxes are left to k_boxes: depth l's listed at
  // wide[doff[l] ...], wide_cnt[l] of them
  int32_t *wide, *wide_cnt;
};

// An internal node spanning at most kDirectLeaves leaves has its box computed
// from the leaf boxes by k_link; the others by k_boxes, depth by depth.
constexpr int kDirectLeaves = 32;

template <int D>
__global__ void k_link(LinkArgs a) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < a.N; x += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)a.ndepth[x];
    const int64_t i = (int64_t)a.nleaf[x];
    const int sh = a.D * (a.bits - l);
    const uint64_t prefix = sh >= 64 ? 0 : (a.pl.key[i] >> sh);
    a.nodes.depth[x] = l;
    a.nodes.prefix[x] = prefix;
    if (l == a.pl.depth[i]) {
      a.nodes.ref[x] = a.pl.ref[i];
      a.nodes.kids[x] = 0;
      a.nodes.cnt[x] = a.pl.cnt[i];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        a.nodes.lo[d][x] = a.pl.lo[d][i];
        a.nodes.hi[d][x] = a.pl.hi[d][i];
      }
      a.leaf_node[i] = (int32_t)x;
      continue;
    }
    // first leaf past this node's cell: galloping from i + 1 (most cells
    // span few leaves), then a binary search in the last step's range
    const uint64_t lim = (prefix + 1) << sh;  // sh <= 63 for an internal node
    int64_t lo = i + 1, hi = i + 1, step = 1;  // leaves before lo are inside the cell
    while (hi < a.L && a.pl.key[hi] < lim) {
      lo = hi + 1;
      hi = lo + step;
      step <<= 1;
    }
    hi = min(hi, a.L);
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (a.pl.key[mid] < lim)
        lo = mid + 1;
      else
        hi = mid;
    }
    const int64_t e = lo;
    // children: depth l+1 nodes whose first leaf lies in [i, e)
    const int64_t s0 = a.doff[l + 1], s1 = a.doff[l + 2];
    int64_t p = s0, q = s1;
    while (p < q) {
      const int64_t mid = (p + q) >> 1;
      if ((int64_t)a.nleaf[mid] < i)
        p = mid + 1;
      else
        q = mid;
    }
    const int64_t c0 = p;
    // the first child's first leaf is i; at most 2^D children in all
    while (p < s1 && (int64_t)a.nleaf[p] < e) ++p;
    a.nodes.ref[x] = (uint32_t)c0;
    a.nodes.kids[x] = (int32_t)(p - c0);
    a.nodes.cnt[x] = (int32_t)(a.E[e] - a.E[i]);
    if (e - i <= kDirectLeaves) {
      int32_t blo[D], bhi[D];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        blo[d] = INT32_MAX;
        bhi[d] = INT32_MIN;
      }
      for (int64_t j = i; j < e; ++j)
#pragma unroll
        for (int d = 0; d < D; ++d) {
          blo[d] = min(blo[d], a.pl.lo[d][j]);
          bhi[d] = max(bhi[d], a.pl.hi[d][j]);
        }
#pragma unroll
      for (int d = 0; d < D; ++d) {
        a.nodes.lo[d][x] = blo[d];
        a.nodes.hi[d][x] = bhi[d];
      }
    } else {
      a.wide[a.doff[l] + atomicAdd(&a.wide_cnt[l], 1)] = (int32_t)x;
    }
  }
}

// Boxes of the listed internal nodes of one depth (list[0, cnt)) from their
// children, which are leaves (boxes from the leaf records), nodes spanning few
// leaves (boxes set by k_link) or listed nodes of the depth below (boxes set
// by the previous launch): an 8-lane group per node (at most 2^D <= 8
// children), four nodes per warp and kBoxRounds such rounds per pass, whose
// loads are issued together.
constexpr int kBoxRounds = 4;

template <int D>
__global__ void k_boxes(NodeArrays nodes, const int32_t *list, int64_t cnt) {
  const int lane = threadIdx.x & 31, g = lane >> 3, gl = lane & 7;
  const unsigned gmask = 0xFFu << (g * 8);
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t j0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (4 * kBoxRounds); j0 < cnt;
       j0 += warps * (4 * kBoxRounds)) {
    int nk[kBoxRounds];
    uint32_t r[kBoxRounds];
    int64_t xs[kBoxRounds];
#pragma unroll
    for (int u = 0; u < kBoxRounds; ++u) {
      const int64_t j = j0 + u * 4 + g;
      xs[u] = j < cnt ? list[j] : -1;
    }
#pragma unroll
    for (int u = 0; u < kBoxRounds; ++u) {
      nk[u] = xs[u] >= 0 ? nodes.kids[xs[u]] : 0;
      r[u] = xs[u] >= 0 ? nodes.ref[xs[u]] : 0;
    }
    int32_t lo[kBoxRounds][D], hi[kBoxRounds][D];
#pragma unroll
    for (int u = 0; u < kBoxRounds; ++u)
#pragma unroll
      for (int d = 0; d < D; ++d) {
        lo[u][d] = gl < nk[u] ? nodes.lo[d][r[u] + gl] : INT32_MAX;
        hi[u][d] = gl < nk[u] ? nodes.hi[d][r[u] + gl] : INT32_MIN;
      }
#pragma unroll
    for (int u = 0; u < kBoxRounds; ++u) {
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int32_t l = __reduce_min_sync(gmask, lo[u][d]);
        const int32_t h = __reduce_max_sync(gmask, hi[u][d]);
        if (nk[u] > 0 && gl == 0) {
          nodes.lo[d][xs[u]] = l;
          nodes.hi[d][xs[u]] = h;
        }
      }
    }
  }
}

// ---- updates ----------------------------------------------------------------

// The sorted batch as records: the id and the point of each sorted entry.
template <int D>
__global__ void k_prec(const uint32_t *bvals, const int32_t *pts, const uint32_t *ids, int64_t m, uint32_t *rid,
                       int32_t *rpt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t v = bvals[i];
    rid[i] = ids[v];
#pragma unroll
    for (int d = 0; d < D; ++d) rpt[i * D + d] = pts[(int64_t)v * D + d];
  }
}

// Leaf of each sorted batch key: the last leaf whose cell starts at or below
// it (leaf 0 when none does).  Cells are disjoint and in key order, so a
// stored point equal to the key can only be in that leaf, and a new point
// goes between that leaf's points and the next leaf's.
__global__ void k_route(const uint64_t *bkeys, int64_t m, const uint64_t *lkey, int64_t L, int32_t *bleaf) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = bkeys[i];
    int64_t lo = 0, hi = L;  // first leaf whose cell starts above k
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (lkey[mid] <= k)
        lo = mid + 1;
      else
        hi = mid;
    }
    bleaf[i] = (int32_t)max((int64_t)0, lo - 1);
  }
}

// Slice [sbeg[x], send[x]) of the sorted batch routed to leaf x.
__global__ void k_pslices(const int32_t *bleaf, int64_t m, int32_t *sbeg, int32_t *send,
                          unsigned long long *n_reached) {
  uint32_t reached = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t j = bleaf[i];
    if (i == 0 || bleaf[i - 1] != j) {
      sbeg[j] = (int32_t)i;
      ++reached;
    }
    if (i == m - 1 || bleaf[i + 1] != j) send[j] = (int32_t)(i + 1);
  }
  block_count_add(n_reached, reached);
}

// The leaf holding old position p: the last leaf y with E[y] <= p (leaves
// hold at least one point, so E is strictly increasing).
__device__ __forceinline__ int64_t leaf_at(const int64_t *E, int64_t L, int64_t p) {
  int64_t lo = 0, hi = L;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (E[mid] <= p)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// A leaf with a slice makes dirty every leaf holding a point within phi + 1
// positions of its own points (the depth windows that can change).
__global__ void k_dirty_marks(const int32_t *sbeg, const int32_t *send, const int64_t *E, int64_t L, int64_t n,
                              int phi, int32_t *diff) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < L; x += (int64_t)gridDim.x * blockDim.x) {
    if (send[x] <= sbeg[x]) continue;
    const int64_t p0 = max((int64_t)0, E[x] - (phi + 1));
    const int64_t p1 = min(n - 1, E[x + 1] + phi);
    atomicAdd(&diff[leaf_at(E, L, p0)], 1);
    atomicAdd(&diff[leaf_at(E, L, p1) + 1], -1);
  }
}

__global__ void k_fill1(int32_t *p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = 1;
}

__global__ void k_all_dirty(int64_t L, int32_t *dirty, int32_t *sstart) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < L; x += (int64_t)gridDim.x * blockDim.x) {
    dirty[x] = 1;
    sstart[x] = x == 0;
  }
}

// dirty[x] from the exclusive scan ex of diff (its inclusive sum is ex[x + 1]);
// segment starts and ends.
__global__ void k_dirty_flags(const int64_t *ex, int64_t L, int32_t *dirty, int32_t *sstart) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < L; x += (int64_t)gridDim.x * blockDim.x) {
    const bool dx = ex[x + 1] > 0;
    dirty[x] = dx;
    sstart[x] = dx && (x == 0 || ex[x] <= 0);
  }
}

// Delete, part 1 (local batches): keep = 1 for every stored point of a leaf
// with a slice (the others are not read), rem = 0.  The warps walk the sorted
// batch in chunks of 32 entries and take the leaf of every entry that starts
// a slice, a lane per point.
__global__ void k_pdel_fill(PLeaves pl, const int64_t *E, const int32_t *bleaf, int64_t m, int32_t *keep) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t j0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; j0 < m; j0 += warps * 32) {
    const int64_t jl = j0 + lane;
    const int32_t xl = jl < m ? bleaf[jl] : -1;
    uint32_t starts = __ballot_sync(0xFFFFFFFFu, jl < m && (jl == 0 || bleaf[jl - 1] != xl));
    while (starts) {
      const int64_t x = __shfl_sync(0xFFFFFFFFu, xl, __ffs(starts) - 1);
      starts &= starts - 1;
      const int64_t e0 = E[x];
      const int c = pl.cnt[x];
      for (int s = lane; s < c; s += 32) keep[e0 + s] = 1;
    }
  }
}

// Delete, part 2: a thread per sorted batch entry finds its (key, id) among
// its leaf's points, which are in (key, id) order, by binary search; a stored
// point with the same pair and coordinates is removed (keep = 0, rem[x] + 1).
// A pair repeated in the batch (adjacent once sorted) deletes once: only its
// first entry searches.
template <int D>
__global__ void k_pdel_marks(PLeaves pl, Pool pool, const int64_t *E, const int32_t *bleaf, int64_t m,
                             const uint64_t *bkeys, const uint32_t *rid, const int32_t *rpt, int32_t *keep,
                             int32_t *rem, unsigned long long *deleted) {
  uint32_t removed = 0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = bkeys[j];
    const uint32_t id = rid[j];
    if (j > 0 && bkeys[j - 1] == k && rid[j - 1] == id) continue;
    const int32_t x = bleaf[j];
    const uint32_t s0 = pl.ref[x];
    int lo = 0, hi = pl.cnt[x];
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (kid_less(pool.pkey[s0 + mid], pool.pid[s0 + mid], k, id))
        lo = mid + 1;
      else
        hi = mid;
    }
    bool hit = lo < pl.cnt[x] && pool.pkey[s0 + lo] == k && pool.pid[s0 + lo] == id;
    if (hit) {
#pragma unroll
      for (int d = 0; d < D; ++d) hit &= rpt[j * D + d] == pool.px[d][s0 + lo];
    }
    if (hit) {
      keep[E[x] + lo] = 0;
      atomicAdd(&rem[x], 1);
      ++removed;
    }
  }
  block_count_add(deleted, removed);
}

// New point count of every dirty leaf (0 for clean leaves).
__global__ void k_newcount(const int32_t *dirty, const int32_t *cnt, const int32_t *sbeg, const int32_t *send,
                           const int32_t *rem, int64_t L, bool insert, int32_t *nc) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < L; x += (int64_t)gridDim.x * blockDim.x) {
    int c = 0;
    if (dirty[x]) c = cnt[x] + (insert ? max(0, send[x] - sbeg[x]) : -(send[x] > sbeg[x] ? rem[x] : 0));
    nc[x] = c;
  }
}

// Segment g: its first and last leaf, and its context sizes (old points
// before and after it, at most phi + 1 each).
__global__ void k_seg_bounds(const int32_t *dirty, const int32_t *sstart, const int64_t *gx, int64_t L,
                             int32_t *xs, int32_t *xe) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < L; x += (int64_t)gridDim.x * blockDim.x) {
    if (sstart[x]) xs[gx[x]] = (int32_t)x;
    if (dirty[x] && (x + 1 == L || !dirty[x + 1])) xe[gx[x] + sstart[x] - 1] = (int32_t)x;
  }
}

__global__ void k_seg_ctx(const int32_t *xs, const int32_t *xe, const int64_t *E, int64_t G, int64_t n, int phi,
                          int32_t *ctxl, int32_t *ctxr, int32_t *ctx) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = E[xs[g]], b = E[xe[g] + 1];
    const int cl = (int)min((int64_t)(phi + 1), a), cr = (int)min((int64_t)(phi + 1), n - b);
    ctxl[g] = cl;
    ctxr[g] = cr;
    ctx[g] = cl + cr;
  }
}

struct SegArgs {
  PLeaves pl;
  Pool src, dst;  // the leaves' points; where the new points go
  const int64_t *E;     // old leaves' prefix counts (L + 1)
  const int32_t *dirty, *sstart, *xs, *xe, *ctxl, *ctxr;
  const int64_t *gx;    // exclusive scan of sstart
  const int64_t *woff;  // exclusive scan of the new counts (L + 1)
  const int64_t *cxoff; // exclusive scan of the segments' context sizes
  const int32_t *sbeg, *send, *keep;
  const uint64_t *bkeys;
  const uint32_t *rid;
  const int32_t *rpt;
  int64_t L, G, n;
  uint32_t fresh;  // first fresh slot: dirty leaf x's new points go to fresh + woff[x] ...
  bool insert;
  int32_t *big;    // dirty leaves with more than kSeqMax new points (at most 4 kChunk)
  uint32_t *n_big;
  int32_t *huge;   // ... with more than 4 kChunk
  uint32_t *n_huge;
  const int64_t *K;  // global delete: exclusive scan of keep over all old points
  const int32_t *bleaf;  // leaf of each sorted batch entry
  const int32_t *block_leaf;  // global paths: leaf holding old position b * kGlobBlock
  int64_t m;
  uint64_t *wkey;  // work array
  int32_t *wmask;
  uint32_t *wslot;
};

// Work position of segment g's first point.
__device__ __forceinline__ int64_t seg_wstart(const SegArgs &a, int64_t g) {
  return a.woff[a.xs[g]] + a.cxoff[g] + a.ctxl[g];
}

// Context keys of every segment (a warp per segment): the old points just
// before and just after it.
__global__ void k_seg_context(SegArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < a.G; g += warps) {
    const int64_t w0 = seg_wstart(a, g);
    const int cl = a.ctxl[g], cr = a.ctxr[g];
    const int64_t pa = a.E[a.xs[g]], pb = a.E[a.xe[g] + 1];
    const int64_t seglen = a.woff[a.xe[g] + 1] - a.woff[a.xs[g]];
    for (int t = lane; t < cl + cr; t += 32) {
      const int64_t p = t < cl ? pa - cl + t : pb + (t - cl);
      const int64_t w = t < cl ? w0 - cl + t : w0 + seglen + (t - cl);
      const int64_t y = leaf_at(a.E, a.L, p);
      a.wkey[w] = a.src.pkey[a.pl.ref[y] + (uint32_t)(p - a.E[y])];
      a.wmask[w] = 0;
      a.wslot[w] = 0;
    }
  }
}

constexpr int kSeqMax = 64;    // a dirty leaf with at most this many new points is built by one lane
constexpr int kChunk = 4096;   // new points per warp task of a large dirty leaf

// Writes new point t of dirty leaf x (segment g) to its fresh slot and to the
// work array.
template <int D>
__device__ __forceinline__ void seg_put(const SegArgs &a, int64_t x, int64_t g, int64_t t, uint64_t k, uint32_t id,
                                        const int32_t *c) {
  const uint32_t dst = a.fresh + (uint32_t)(a.woff[x] + t);
  const int64_t w = seg_wstart(a, g) + (a.woff[x] - a.woff[a.xs[g]]) + t;
#pragma unroll
  for (int d = 0; d < D; ++d) a.dst.px[d][dst] = c[d];
  a.dst.pid[dst] = id;
  a.dst.pkey[dst] = k;
  a.wkey[w] = k;
  a.wmask[w] = 1;
  a.wslot[w] = dst;
}

// Merged order of a leaf point and a batch entry: the leaf point first on
// equal (key, id).
__device__ __forceinline__ bool leaf_first(uint64_t lk, uint32_t lid, uint64_t bk, uint32_t bid) {
  return lk < bk || (lk == bk && lid <= bid);
}

// The new points of every small dirty leaf, in (key, id) order: one lane per
// leaf (32 consecutive leaves per warp) merges the leaf's points with its
// slice (insert) or keeps its unmarked points (delete), one point per step.
// Larger dirty leaves are listed for k_seg_big.
template <int D>
__global__ void k_seg_small(SegArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t j0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; j0 < a.L; j0 += warps * 32) {
    const int64_t x = j0 + lane;
    if (x >= a.L || !a.dirty[x]) continue;
    const int64_t nc = a.woff[x + 1] - a.woff[x];
    if (nc > kSeqMax) {  // listed: whole leaves per warp, or chunks of a huge one over all warps
      if (nc > 4 * kChunk)
        a.huge[atomicAdd(a.n_huge, 1u)] = (int32_t)x;
      else
        a.big[atomicAdd(a.n_big, 1u)] = (int32_t)x;
      continue;
    }
    const int64_t g = a.gx[x] + a.sstart[x] - 1;
    const uint32_t s0 = a.pl.ref[x];
    const int cnt = a.pl.cnt[x];
    const int32_t b = a.sbeg[x], len = max(0, a.send[x] - b);
    int32_t c[D];
    if (a.insert) {
      int i = 0, j = 0;
      for (int64_t t = 0; t < nc; ++t) {
        bool from_leaf = i < cnt;
        if (from_leaf && j < len)
          from_leaf = leaf_first(a.src.pkey[s0 + i], a.src.pid[s0 + i], a.bkeys[b + j], a.rid[b + j]);
        if (from_leaf) {
#pragma unroll
          for (int d = 0; d < D; ++d) c[d] = a.src.px[d][s0 + i];
          seg_put<D>(a, x, g, t, a.src.pkey[s0 + i], a.src.pid[s0 + i], c);
          ++i;
        } else {
#pragma unroll
          for (int d = 0; d < D; ++d) c[d] = a.rpt[(int64_t)(b + j) * D + d];
          seg_put<D>(a, x, g, t, a.bkeys[b + j], a.rid[b + j], c);
          ++j;
        }
      }
    } else {
      int64_t t = 0;
      for (int i = 0; i < cnt; ++i) {
        if (len > 0 && !a.keep[a.E[x] + i]) continue;
#pragma unroll
        for (int d = 0; d < D; ++d) c[d] = a.src.px[d][s0 + i];
        seg_put<D>(a, x, g, t++, a.src.pkey[s0 + i], a.src.pid[s0 + i], c);
      }
    }
  }
}

// New point p (of nc) of a listed dirty leaf x in segment g.  Insert: found
// by a merge-path search over the leaf's points and its slice.
template <int D>
__device__ __forceinline__ void seg_insert_at(const SegArgs &a, int64_t x, int64_t g, int64_t p) {
  const uint32_t s0 = a.pl.ref[x];
  const int cnt = a.pl.cnt[x];
  const int32_t b = a.sbeg[x], len = max(0, a.send[x] - b);
  // merge path: how many of the first p merged points come from the leaf
  int64_t l = max((int64_t)0, p - len), h = min(p, (int64_t)cnt);
  while (l < h) {
    const int64_t mid = (l + h) >> 1;
    const int64_t bj = b + (p - mid - 1);
    if (leaf_first(a.src.pkey[s0 + mid], a.src.pid[s0 + mid], a.bkeys[bj], a.rid[bj]))
      l = mid + 1;
    else
      h = mid;
  }
  const int64_t li = l, si = p - l;
  bool from_leaf = li < cnt;
  if (from_leaf && si < len)
    from_leaf = leaf_first(a.src.pkey[s0 + li], a.src.pid[s0 + li], a.bkeys[b + si], a.rid[b + si]);
  int32_t c[D];
  if (from_leaf) {
    const uint32_t sl = s0 + (uint32_t)li;
#pragma unroll
    for (int d = 0; d < D; ++d) c[d] = a.src.px[d][sl];
    seg_put<D>(a, x, g, p, a.src.pkey[sl], a.src.pid[sl], c);
  } else {
    const int64_t bj = b + si;
#pragma unroll
    for (int d = 0; d < D; ++d) c[d] = a.rpt[bj * D + d];
    seg_put<D>(a, x, g, p, a.bkeys[bj], a.rid[bj], c);
  }
}

// Delete: a warp keeps the unmarked points of leaf x in order.
template <int D>
__device__ __forceinline__ void seg_delete_leaf(const SegArgs &a, int64_t x, int64_t g) {
  const int lane = threadIdx.x & 31;
  const uint32_t s0 = a.pl.ref[x];
  const int cnt = a.pl.cnt[x];
  const int32_t len = max(0, a.send[x] - a.sbeg[x]);
  int64_t out = 0;
  for (int r0 = 0; r0 < cnt; r0 += 32) {
    const int i = r0 + lane;
    const bool k = i < cnt && (len == 0 || a.keep[a.E[x] + i]);
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, k);
    if (k) {
      const uint32_t sl = s0 + (uint32_t)i;
      int32_t c[D];
#pragma unroll
      for (int d = 0; d < D; ++d) c[d] = a.src.px[d][sl];
      seg_put<D>(a, x, g, out + __popc(m & lanemask_lt()), a.src.pkey[sl], a.src.pid[sl], c);
    }
    out += __popc(m);
  }
}

// The new points of the listed dirty leaves: a warp per leaf of the big list;
// the chunks of kChunk new points of each huge leaf spread over all warps.
template <int D>
__global__ void k_seg_big(SegArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nb = *a.n_big, nh = *a.n_huge;
  for (int64_t bi = wid; bi < nb; bi += warps) {
    const int64_t x = a.big[bi];
    const int64_t g = a.gx[x] + a.sstart[x] - 1;
    if (a.insert) {
      const int64_t nc = a.woff[x + 1] - a.woff[x];
      for (int64_t p = lane; p < nc; p += 32) seg_insert_at<D>(a, x, g, p);
    } else {
      seg_delete_leaf<D>(a, x, g);
    }
  }
  for (int64_t hi = 0; hi < nh; ++hi) {
    const int64_t x = a.huge[hi];
    const int64_t g = a.gx[x] + a.sstart[x] - 1;
    if (a.insert) {
      const int64_t nc = a.woff[x + 1] - a.woff[x];
      const int64_t chunks = (nc + kChunk - 1) / kChunk;
      for (int64_t ch = wid; ch < chunks; ch += warps) {
        const int64_t pe = min(nc, (ch + 1) * kChunk);
        for (int64_t p = ch * kChunk + lane; p < pe; p += 32) seg_insert_at<D>(a, x, g, p);
      }
    } else if (hi % warps == wid) {
      seg_delete_leaf<D>(a, x, g);
    }
  }
}

// Last index x in [lo, hi) with v[x] <= t (v non-decreasing, v[lo] <= t).
__device__ __forceinline__ int64_t last_le(const int64_t *v, int64_t lo, int64_t hi, int64_t t) {
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (v[mid] <= t)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Threads per block of the global kernels; their blocks take kGlobBlock
// consecutive old positions per round.
constexpr int kGlobBlock = 256;

// block_leaf[b] = the leaf holding old position b * kGlobBlock (b < nb): the
// leaf range of each block of the global kernels without a search over E.
__global__ void k_block_leaf(const int64_t *E, int64_t L, int64_t nb, int32_t *block_leaf) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < L; x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = E[x], e = E[x + 1];
    for (int64_t b = (s + kGlobBlock - 1) / kGlobBlock; b < nb && b * kGlobBlock < e; ++b)
      block_leaf[b] = (int32_t)x;
  }
}

// Leaf range [xr[0], xr[1]) holding the old positions [q0, q0 + kGlobBlock).
__device__ __forceinline__ void glob_block_range(const SegArgs &a, int64_t q0, int64_t *xr) {
  const int64_t b = q0 / kGlobBlock;
  xr[0] = a.block_leaf[b];
  xr[1] = q0 + kGlobBlock < a.n ? a.block_leaf[b + 1] + 1 : a.L;
}

// Global insert (every leaf dirty, one segment, no context: the work array is
// the fresh pool's keys themselves): a thread per old point and per batch entry, each
// placing itself among the other side of its leaf by a binary search (a
// leaf's points and its slice are both in (key, id) order; the leaf point
// comes first on equal (key, id)); writes are nearly in order.  A block's old
// points lie in a narrow range of leaves, found once per block.
template <int D>
__global__ void k_glob_insert(SegArgs a) {
  __shared__ int64_t xr[2];
  const int64_t total = a.n + a.m;
  for (int64_t q0 = (int64_t)blockIdx.x * blockDim.x; q0 < total; q0 += (int64_t)gridDim.x * blockDim.x) {
    __syncthreads();
    if (threadIdx.x == 0 && q0 < a.n) glob_block_range(a, q0, xr);
    __syncthreads();
    const int64_t q = q0 + threadIdx.x;
    if (q >= total) continue;
    int64_t x, o;
    uint64_t k;
    uint32_t id;
    int32_t c[D];
    if (q < a.n) {  // old point q (leaf order)
      x = last_le(a.E, xr[0], xr[1], q);
      const int64_t i = q - a.E[x];
      const uint32_t sl = a.pl.ref[x] + (uint32_t)i;
      k = a.src.pkey[sl];
      id = a.src.pid[sl];
#pragma unroll
      for (int d = 0; d < D; ++d) c[d] = a.src.px[d][sl];
      int32_t lo = a.sbeg[x], hi = max(lo, a.send[x]);  // slice entries before it: (key, id) strictly less
      while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (!leaf_first(k, id, a.bkeys[mid], a.rid[mid]))
          lo = mid + 1;
        else
          hi = mid;
      }
      o = a.woff[x] + i + (lo - a.sbeg[x]);
    } else {  // batch entry j (sorted order)
      const int64_t j = q - a.n;
      x = a.bleaf[j];
      k = a.bkeys[j];
      id = a.rid[j];
#pragma unroll
      for (int d = 0; d < D; ++d) c[d] = a.rpt[j * D + d];
      const uint32_t s0 = a.pl.ref[x];
      int lo = 0, hi = a.pl.cnt[x];  // leaf points before it: those that come first
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (leaf_first(a.src.pkey[s0 + mid], a.src.pid[s0 + mid], k, id))
          lo = mid + 1;
        else
          hi = mid;
      }
      o = a.woff[x] + (j - a.sbeg[x]) + lo;
    }
    a.dst.pkey[o] = k;
    a.dst.pid[o] = id;
#pragma unroll
    for (int d = 0; d < D; ++d) a.dst.px[d][o] = c[d];
  }
}

// Global delete: a thread per old point (leaf found as above); a kept point
// goes to its rank among the kept ones (the fresh pool is the work array).
template <int D>
__global__ void k_glob_delete(SegArgs a) {
  __shared__ int64_t xr[2];
  for (int64_t p0 = (int64_t)blockIdx.x * blockDim.x; p0 < a.n; p0 += (int64_t)gridDim.x * blockDim.x) {
    __syncthreads();
    if (threadIdx.x == 0) glob_block_range(a, p0, xr);
    __syncthreads();
    const int64_t p = p0 + threadIdx.x;
    if (p >= a.n || !a.keep[p]) continue;
    const int64_t x = last_le(a.E, xr[0], xr[1], p);
    const uint32_t sl = a.pl.ref[x] + (uint32_t)(p - a.E[x]);
    int32_t c[D];
#pragma unroll
    for (int d = 0; d < D; ++d) c[d] = a.src.px[d][sl];
    const int64_t o = a.K[p];
    a.dst.pid[o] = a.src.pid[sl];
    a.dst.pkey[o] = a.src.pkey[sl];
#pragma unroll
    for (int d = 0; d < D; ++d) a.dst.px[d][o] = c[d];
  }
}

// First new leaf of each segment: the leaf rank at its first work position
// (its context and points follow in work order); fl[G] = the new leaf count.
__global__ void k_seg_first_leaf(SegArgs a, const int64_t *rank, int64_t W, int64_t NL, int64_t *fl) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g <= a.G; g += (int64_t)gridDim.x * blockDim.x) {
    if (g == a.G) {
      fl[g] = NL;
    } else {
      const int64_t w = seg_wstart(a, g);
      fl[g] = w < W ? rank[w] : NL;
    }
  }
}

// Output leaves of each old leaf: a clean leaf is kept, a segment's new
// leaves are counted at its first leaf.
__global__ void k_pl_outl(const int32_t *dirty, const int32_t *sstart, const int64_t *gx, const int64_t *fl,
                          int64_t L, int32_t *outl) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < L; x += (int64_t)gridDim.x * blockDim.x) {
    if (!dirty[x])
      outl[x] = 1;
    else if (sstart[x])
      outl[x] = (int32_t)(fl[gx[x] + 1] - fl[gx[x]]);
    else
      outl[x] = 0;
  }
}

template <int D>
__device__ __forceinline__ void pl_copy(const PLeaves &src, int64_t i, const PLeaves &dst, int64_t o) {
  dst.ref[o] = src.ref[i];
  dst.cnt[o] = src.cnt[i];
  dst.depth[o] = src.depth[i];
  dst.key[o] = src.key[i];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    dst.lo[d][o] = src.lo[d][i];
    dst.hi[d][o] = src.hi[d][i];
  }
}

// The new leaf list: clean leaves at pos[x]; new leaf r of segment g at
// pos[xs[g]] + (r - fl[g]).
template <int D>
__global__ void k_pl_assemble(PLeaves old, const int32_t *dirty, const int64_t *pos, int64_t L, PLeaves fresh,
                              int64_t NL, const int64_t *fl, const int32_t *xs, int64_t G, PLeaves out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < L; x += stride)
    if (!dirty[x]) pl_copy<D>(old, x, out, pos[x]);
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < NL; r += stride) {
    int64_t lo = 0, hi = G;  // last segment g with fl[g] <= r
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (fl[mid] <= r)
        lo = mid;
      else
        hi = mid;
    }
    pl_copy<D>(fresh, r, out, pos[xs[lo]] + (r - fl[lo]));
  }
}

// Compaction of the pool: every leaf's points to consecutive slots in leaf
// order (an 8-lane group per leaf, four leaves per warp); the leaf records
// take their new first slots.
template <int D>
__global__ void k_pl_compact(PLeaves pl, const int64_t *E, int64_t L, Pool from, Pool to) {
  const int lane = threadIdx.x & 31, g = lane >> 3, gl = lane & 7;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t x0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 4; x0 < L; x0 += warps * 4) {
    const int64_t x = x0 + g;
    if (x >= L) continue;
    const uint32_t s0 = pl.ref[x];
    const int c = pl.cnt[x];
    const int64_t o = E[x];
    for (int s = gl; s < c; s += 8) {
#pragma unroll
      for (int d = 0; d < D; ++d) to.px[d][o + s] = from.px[d][s0 + s];
      to.pid[o + s] = from.pid[s0 + s];
      to.pkey[o + s] = from.pkey[s0 + s];
    }
    if (gl == 0) pl.ref[x] = (uint32_t)o;
  }
}

__global__ void k_i64_from_u64(const unsigned long long *a, int64_t *b) { *b = (int64_t)*a; }

}  // namespace

// Node arrays of the P-Orth tree over the leaf list ix->pl (ix->L leaves).
static psi_status porth_nodes(psi_index *ix, cudaStream_t s) {
  const int D = ix->D, bits = ix->cfg.coord_bits, K = ix->key_bits;
  const int64_t L = ix->L;
  free_nodes(ix->nodes, s);
  DevMem::free(ix->leaf_node, s);
  ix->leaf_node = nullptr;
  ix->nnodes = 0;
  ix->root = -1;
  if (L == 0) return PSI_OK;
  psi_status st;
  Buf<int64_t> nn, E, tot;
  Buf<int32_t> c, hist;
  if ((st = nn.alloc(L, s)) || (st = E.alloc(L + 1, s)) || (st = tot.alloc(2, s)) || (st = c.alloc(L, s)) ||
      (st = hist.alloc(64, s)))
    return st;
  if ((st = scan_i32_to_i64(ix->pl.cnt, E.p, L, E.p + L, s))) return st;
  PSI_LAUNCH(k_heads, grid_for(L), 256, 0, s, ix->pl.depth, ix->pl.key, L, K, D, bits, c.p, nn.p);
  if ((st = scan_i64(nn.p, nn.p, L, tot.p, s))) return st;
  int64_t N = 0;
  PSI_CK(cudaMemcpyAsync(&N, tot.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaMemsetAsync(hist.p, 0, sizeof(int32_t) * 64, s));
  PSI_CK(cudaStreamSynchronize(s));

  Buf<uint64_t> nk0, nk1;
  Buf<uint32_t> nv0, nv1;
  if ((st = nk0.alloc(N, s)) || (st = nk1.alloc(N, s)) || (st = nv0.alloc(N, s)) || (st = nv1.alloc(N, s))) return st;
  PSI_LAUNCH(k_emit_nodes, grid_for(L), 256, 0, s, ix->pl.depth, c.p, nn.p, L, nk0.p, nv0.p, hist.p);
  int32_t h_hist[64];
  PSI_CK(cudaMemcpyAsync(h_hist, hist.p, sizeof(h_hist), cudaMemcpyDeviceToHost, s));
  SortResult r;
  EncodeSpec none;
  Buf<int> sst;
  if ((st = sst.alloc(1, s))) return st;
  PSI_CK(cudaMemsetAsync(sst.p, 0, sizeof(int), s));
  // one stable digit pass on the depth (< 64); the input arrays double as the
  // second ping-pong buffer
  if ((st = sort_pairs(none, nk0.p, nv0.p, N, 8, nullptr, nk1.p, nv1.p, nk0.p, nv0.p, sst.p, s, &r))) return st;
  PSI_CK(cudaStreamSynchronize(s));
  std::vector<int64_t> doff(bits + 3, 0);
  for (int l = 0; l <= bits; ++l) doff[l + 1] = doff[l] + h_hist[l];
  doff[bits + 2] = doff[bits + 1];
  Buf<int64_t> d_doff;
  if ((st = d_doff.alloc(doff.size(), s))) return st;
  PSI_CK(cudaMemcpyAsync(d_doff.p, doff.data(), sizeof(int64_t) * doff.size(), cudaMemcpyHostToDevice, s));

  if ((st = alloc_nodes(ix->nodes, D, N, true, s))) return st;
  if ((st = DevMem::alloc((void **)&ix->leaf_node, sizeof(int32_t) * L, s))) return st;
  Buf<int32_t> wide, wide_cnt;
  if ((st = wide.alloc(N, s)) || (st = wide_cnt.alloc(64, s))) return st;
  PSI_CK(cudaMemsetAsync(wide_cnt.p, 0, sizeof(int32_t) * 64, s));
  LinkArgs la{r.keys, r.vals, d_doff.p, E.p, ix->pl, L, N, D, bits, ix->nodes, ix->leaf_node, wide.p, wide_cnt.p};
  if (D == 2)
    PSI_LAUNCH_NAMED("k_link", k_link<2>, grid_for(N), 256, 0, s, la);
  else
    PSI_LAUNCH_NAMED("k_link", k_link<3>, grid_for(N), 256, 0, s, la);
  // the boxes of the listed (wide) internal nodes, depth by depth bottom up
  int32_t h_wide[64];
  PSI_CK(cudaMemcpyAsync(h_wide, wide_cnt.p, sizeof(h_wide), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaStreamSynchronize(s));
  for (int l = bits; l >= 0; --l) {
    const int64_t cnt = h_wide[l];
    if (!cnt) continue;
    const int g = (int)std::max<int64_t>(
        1, std::min<int64_t>(ceil_div(cnt, 8 * 4 * kBoxRounds), (int64_t)num_sms() * 32));
    if (D == 2)
      PSI_LAUNCH_NAMED("k_boxes", k_boxes<2>, g, 256, 0, s, ix->nodes, wide.p + doff[l], cnt);
    else
      PSI_LAUNCH_NAMED("k_boxes", k_boxes<3>, g, 256, 0, s, ix->nodes, wide.p + doff[l], cnt);
  }
  ix->nnodes = N;
  ix->root = 0;
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}

// Leaves of a work array into a new leaf list `out` (allocated here) with
// their boxes; *nl receives the leaf count.  rank_out (optional) keeps the
// exclusive scan of the leaf starts.
static psi_status work_leaves(psi_index *ix, const WorkArray &w, uint32_t end_slot, PLeaves &out, int64_t *nl,
                              Buf<int64_t> *rank_out, cudaStream_t s) {
  const int D = ix->D, bits = ix->cfg.coord_bits, K = ix->key_bits;
  psi_status st;
  Buf<int32_t> ldepth, start;
  Buf<int64_t> rank_local, tot;
  Buf<int64_t> &rank = rank_out ? *rank_out : rank_local;
  if ((st = ldepth.alloc(w.n, s)) || (st = start.alloc(w.n, s)) || (st = rank.alloc(w.n, s)) ||
      (st = tot.alloc(1, s)))
    return st;
  PSI_LAUNCH(k_leaf_depth, (unsigned)ceil_div(w.n, LDE), LDT, 0, s, w.key, w.n, ix->phi, K, D, bits, ldepth.p);
  PSI_LAUNCH(k_work_starts, grid_for(w.n), 256, 0, s, w, ldepth.p, D, bits, start.p);
  if ((st = scan_i32_to_i64(start.p, rank.p, w.n, tot.p, s))) return st;
  int64_t L = 0;
  PSI_CK(cudaMemcpyAsync(&L, tot.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaStreamSynchronize(s));
  if ((st = alloc_pleaves(out, D, L, s))) return st;
  PSI_LAUNCH(k_work_leaves, grid_for(w.n), 256, 0, s, w, ldepth.p, start.p, rank.p, D, bits, out);
  if (L > 0) {
    PSI_LAUNCH(k_leaf_counts, grid_for(L), 256, 0, s, out, L, end_slot);
    PSI_LAUNCH(k_empty_boxes, grid_for(L), 256, 0, s, out, L, D);
    if (D == 2)
      PSI_LAUNCH_NAMED("k_work_boxes", k_work_boxes<2>, grid_for(w.n), 256, 0, s, w, start.p, rank.p, ix->pool, out);
    else
      PSI_LAUNCH_NAMED("k_work_boxes", k_work_boxes<3>, grid_for(w.n), 256, 0, s, w, start.p, rank.p, ix->pool, out);
  }
  *nl = L;
  return PSI_OK;
}

// Grows the pool to at least `need` slots, keeping the used prefix.
static psi_status porth_grow(psi_index *ix, int64_t need, cudaStream_t s) {
  if (need <= ix->pool.cap_slots) return PSI_OK;
  Pool np;
  const int64_t cap = std::max(need + need / 4, ix->pool.cap_slots * 3 / 2);
  psi_status st = alloc_pool(np, ix->D, cap, s);
  if (st) {
    free_pool(np, s);
    return st;
  }
  const int64_t used = ix->pool_used;
  if (used > 0) {
    for (int d = 0; d < ix->D; ++d)
      PSI_CK(cudaMemcpyAsync(np.px[d], ix->pool.px[d], sizeof(int32_t) * used, cudaMemcpyDeviceToDevice, s));
    PSI_CK(cudaMemcpyAsync(np.pid, ix->pool.pid, sizeof(uint32_t) * used, cudaMemcpyDeviceToDevice, s));
    PSI_CK(cudaMemcpyAsync(np.pkey, ix->pool.pkey, sizeof(uint64_t) * used, cudaMemcpyDeviceToDevice, s));
  }
  free_pool(ix->pool, s);
  ix->pool = np;
  return PSI_OK;
}

// Moves every leaf's points to consecutive slots in leaf order when more than
// half of the pool's used slots are stale (points of rebuilt leaves).
static psi_status porth_compact_if_needed(psi_index *ix, cudaStream_t s) {
  if (ix->L == 0 || ix->pool_used <= 2 * ix->n + (int64_t(1) << 16)) return PSI_OK;
  psi_status st;
  Buf<int64_t> E;
  if ((st = E.alloc(ix->L + 1, s))) return st;
  if ((st = scan_i32_to_i64(ix->pl.cnt, E.p, ix->L, E.p + ix->L, s))) return st;
  Pool np;
  if ((st = alloc_pool(np, ix->D, ix->n + ix->n / 4 + 1024, s))) {
    free_pool(np, s);
    return st;
  }
  if (ix->D == 2)
    PSI_LAUNCH_NAMED("k_pl_compact", k_pl_compact<2>, warp_grid(ix->L), 256, 0, s, ix->pl, E.p, ix->L, ix->pool, np);
  else
    PSI_LAUNCH_NAMED("k_pl_compact", k_pl_compact<3>, warp_grid(ix->L), 256, 0, s, ix->pl, E.p, ix->L, ix->pool, np);
  free_pool(ix->pool, s);
  ix->pool = np;
  ix->pool_used = ix->n;
  return PSI_OK;
}

psi_status porth_build(psi_index *ix, const int32_t *pts, const uint32_t *ids, int64_t n, cudaStream_t s) {
  psi_status st;
  ix->n = n;
  free_pool(ix->pool, s);
  free_pleaves(ix->pl, s);
  ix->L = 0;
  if ((st = alloc_pool(ix->pool, ix->D, std::max<int64_t>(n + n / 4, 1024), s))) return st;
  ix->pool_used = n;
  if (n == 0) return porth_nodes(ix, s);
  Buf<uint64_t> k0, k1;
  Buf<uint32_t> v0, v1;
  if ((st = k0.alloc(n, s)) || (st = k1.alloc(n, s)) || (st = v0.alloc(n, s)) || (st = v1.alloc(n, s))) return st;
  SortResult r;
  if ((st = sort_pairs(encode_spec(ix, pts), nullptr, nullptr, n, ix->key_bits, ids, k0.p, v0.p, k1.p, v1.p,
                       ix->d_status, s, &r, ix->cfg.radix_bits)))
    return st;
  // input in random order: points and ids packed into one record per point
  // first, so that each gather by position is one scattered read, not two
  const bool records = r.local == 0;
  Buf<int4> rec;
  if (records && ((st = rec.alloc(n, s)) || (st = pack_records(pts, ids, n, ix->D, rec.p, s)))) return st;
#define GATHER(DD, RR)                                                                                           \
  PSI_LAUNCH_NAMED("k_porth_gather", (k_porth_gather<DD, RR>), grid_for(n), 256, 0, s, r.keys, r.vals, pts, ids, \
                   rec.p, n, ix->pool)
  if (ix->D == 2) {
    if (records) GATHER(2, true);
    else GATHER(2, false);
  } else {
    if (records) GATHER(3, true);
    else GATHER(3, false);
  }
#undef GATHER
  WorkArray w{ix->pool.pkey, nullptr, nullptr, 0u, n};
  int64_t L = 0;
  if ((st = work_leaves(ix, w, (uint32_t)n, ix->pl, &L, nullptr, s))) return st;
  ix->L = L;
  return porth_nodes(ix, s);
}

// Local batch update (the batch sorted, then routed, dirty segments rebuilt).
static psi_status porth_update(psi_index *ix, const int32_t *pts, const uint32_t *ids, int64_t m, bool insert,
                               int64_t *d_deleted, cudaStream_t s) {
  psi_status st;
  const int D = ix->D, phi = ix->phi;
  const int64_t L = ix->L, n = ix->n;
  Buf<uint64_t> k0, k1;
  Buf<uint32_t> v0, v1;
  if ((st = k0.alloc(m, s)) || (st = k1.alloc(m, s)) || (st = v0.alloc(m, s)) || (st = v1.alloc(m, s))) return st;
  SortResult br;
  if ((st = sort_pairs(encode_spec(ix, pts), nullptr, nullptr, m, ix->key_bits, ids, k0.p, v0.p, k1.p, v1.p,
                       ix->d_status, s, &br, ix->cfg.radix_bits)))
    return st;
  Buf<uint32_t> rid;
  Buf<int32_t> rpt, bleaf, sbeg, send, diff, dirty, sstart, rem, keep, nc;
  Buf<int64_t> E, dex, gx, woff, tot;
  Buf<unsigned long long> del;
  if ((st = rid.alloc(m, s)) || (st = rpt.alloc(m * D, s)) || (st = bleaf.alloc(m, s)) || (st = sbeg.alloc(L, s)) ||
      (st = send.alloc(L, s)) || (st = diff.alloc(L + 1, s)) || (st = dirty.alloc(L, s)) ||
      (st = sstart.alloc(L, s)) || (st = rem.alloc(L, s)) || (st = nc.alloc(L + 1, s)) || (st = E.alloc(L + 1, s)) ||
      (st = dex.alloc(L + 2, s)) || (st = gx.alloc(L + 1, s)) || (st = woff.alloc(L + 1, s)) ||
      (st = tot.alloc(4, s)) || (st = del.alloc(1, s)))
    return st;
  PSI_CK(cudaMemsetAsync(tot.p, 0, sizeof(int64_t) * 4, s));
  // A batch of more than 1/16 of the points reaches nearly every leaf: it is
  // merged with all of them into a fresh pool (one segment, no garbage).  So
  // is a batch of more than 1/256 of them that reaches (has points routed to)
  // more than a quarter of the leaves, since the leaves within phi + 1 points
  // of those make nearly all of them dirty.
  bool global = m * 16 > n;
  if (D == 2)
    PSI_LAUNCH_NAMED("k_prec", k_prec<2>, grid_for(m), 256, 0, s, br.vals, pts, ids, m, rid.p, rpt.p);
  else
    PSI_LAUNCH_NAMED("k_prec", k_prec<3>, grid_for(m), 256, 0, s, br.vals, pts, ids, m, rid.p, rpt.p);
  PSI_CK(cudaMemsetAsync(sbeg.p, 0, sizeof(int32_t) * L, s));
  PSI_CK(cudaMemsetAsync(send.p, 0, sizeof(int32_t) * L, s));
  PSI_CK(cudaMemsetAsync(diff.p, 0, sizeof(int32_t) * (L + 1), s));
  PSI_CK(cudaMemsetAsync(del.p, 0, sizeof(unsigned long long), s));
  PSI_CK(cudaMemsetAsync(nc.p + L, 0, sizeof(int32_t), s));
  if ((st = scan_i32_to_i64(ix->pl.cnt, E.p, L, E.p + L, s))) return st;
  PSI_LAUNCH(k_route, grid_for(m), 256, 0, s, br.keys, m, ix->pl.key, L, bleaf.p);
  PSI_CK(cudaMemsetAsync(del.p, 0, sizeof(unsigned long long), s));
  PSI_LAUNCH(k_pslices, grid_for(m), 256, 0, s, bleaf.p, m, sbeg.p, send.p, del.p);
  if (!global && m * 256 > n) {
    unsigned long long reached = 0;
    PSI_CK(cudaMemcpyAsync(&reached, del.p, sizeof(reached), cudaMemcpyDeviceToHost, s));
    PSI_CK(cudaStreamSynchronize(s));
    global = reached * 4 > (unsigned long long)L;
  }
  PSI_CK(cudaMemsetAsync(del.p, 0, sizeof(unsigned long long), s));
  if (global) {
    PSI_LAUNCH(k_all_dirty, grid_for(L), 256, 0, s, L, dirty.p, sstart.p);
  } else {
    PSI_LAUNCH(k_dirty_marks, grid_for(L), 256, 0, s, sbeg.p, send.p, E.p, L, n, phi, diff.p);
    // dex = exclusive scan of diff over L + 1 entries (dex[x + 1] = inclusive sum at x)
    if ((st = scan_i32_to_i64(diff.p, dex.p, L + 1, dex.p + L + 1, s))) return st;
    PSI_LAUNCH(k_dirty_flags, grid_for(L), 256, 0, s, dex.p, L, dirty.p, sstart.p);
  }
  if (!insert) {
    if ((st = keep.alloc(n, s))) return st;
    if (global)  // every old point of a dirty leaf is read
      PSI_LAUNCH(k_fill1, grid_for(n), 256, 0, s, keep.p, n);
    else  // those of the leaves with a slice
      PSI_LAUNCH(k_pdel_fill, warp_grid(ceil_div(m, 32)), 256, 0, s, ix->pl, E.p, bleaf.p, m, keep.p);
    PSI_CK(cudaMemsetAsync(rem.p, 0, sizeof(int32_t) * L, s));
    if (D == 2)
      PSI_LAUNCH_NAMED("k_pdel_marks", k_pdel_marks<2>, grid_for(m), 256, 0, s, ix->pl, ix->pool, E.p, bleaf.p, m,
                       br.keys, rid.p, rpt.p, keep.p, rem.p, del.p);
    else
      PSI_LAUNCH_NAMED("k_pdel_marks", k_pdel_marks<3>, grid_for(m), 256, 0, s, ix->pl, ix->pool, E.p, bleaf.p, m,
                       br.keys, rid.p, rpt.p, keep.p, rem.p, del.p);
    PSI_LAUNCH(k_i64_from_u64, 1, 1, 0, s, del.p, tot.p + 3);
    if (d_deleted) PSI_CK(cudaMemcpyAsync(d_deleted, tot.p + 3, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  }
  PSI_LAUNCH(k_newcount, grid_for(L), 256, 0, s, dirty.p, ix->pl.cnt, sbeg.p, send.p, rem.p, L, insert, nc.p);
  if ((st = scan_i32_to_i64(nc.p, woff.p, L + 1, tot.p, s))) return st;  // woff[L] = total new points S
  if ((st = scan_i32_to_i64(sstart.p, gx.p, L, tot.p + 1, s))) return st;
  PSI_CK(cudaMemcpyAsync(gx.p + L, tot.p + 1, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  int64_t h[4] = {0, 0, 0, 0};
  PSI_CK(cudaMemcpyAsync(h, tot.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaStreamSynchronize(s));
  const int64_t S = h[0], G = h[1];
  const int64_t n_new = insert ? n + m : n - h[3];
  if (G == 0) {  // nothing reached a leaf (a delete of absent points)
    ix->n = n_new;
    return PSI_OK;
  }
  // segments, their context, the work array
  Buf<int32_t> xs, xe, ctxl, ctxr, ctx;
  Buf<int64_t> cxoff;
  if ((st = xs.alloc(G, s)) || (st = xe.alloc(G, s)) || (st = ctxl.alloc(G, s)) || (st = ctxr.alloc(G, s)) ||
      (st = ctx.alloc(G, s)) || (st = cxoff.alloc(G + 1, s)))
    return st;
  PSI_LAUNCH(k_seg_bounds, grid_for(L), 256, 0, s, dirty.p, sstart.p, gx.p, L, xs.p, xe.p);
  PSI_LAUNCH(k_seg_ctx, grid_for(G), 256, 0, s, xs.p, xe.p, E.p, G, n, phi, ctxl.p, ctxr.p, ctx.p);
  if ((st = scan_i32_to_i64(ctx.p, cxoff.p, G, cxoff.p + G, s))) return st;
  int64_t hc = 0;
  PSI_CK(cudaMemcpyAsync(&hc, cxoff.p + G, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaStreamSynchronize(s));
  const int64_t W = S + hc;
  // new points: appended to the pool, or (global) into a fresh pool
  Pool npool;
  if (global) {
    if ((st = alloc_pool(npool, D, std::max<int64_t>(S + S / 4, 1024), s))) {
      free_pool(npool, s);
      return st;
    }
  } else if ((st = porth_grow(ix, ix->pool_used + S, s))) {
    return st;
  }
  const uint32_t fresh = global ? 0u : (uint32_t)ix->pool_used;
  Buf<int32_t> big, huge;
  Buf<uint32_t> n_big;
  Buf<int64_t> K;
  if ((st = big.alloc(L, s)) || (st = huge.alloc(L, s)) || (st = n_big.alloc(2, s)) ||
      (global && !insert && (st = K.alloc(n + 1, s)))) {
    free_pool(npool, s);
    return st;
  }
  PSI_CK(cudaMemsetAsync(n_big.p, 0, 2 * sizeof(uint32_t), s));
  if (global && !insert && (st = scan_i32_to_i64(keep.p, K.p, n, K.p + n, s))) {
    free_pool(npool, s);
    return st;
  }
  Buf<uint64_t> wkey;
  Buf<int32_t> wmask;
  Buf<uint32_t> wslot;
  const int64_t Wb = global ? 1 : std::max<int64_t>(W, 1);  // global: the fresh pool is the work array
  if ((st = wkey.alloc(Wb, s)) || (st = wmask.alloc(Wb, s)) || (st = wslot.alloc(Wb, s))) {
    free_pool(npool, s);
    return st;
  }
  SegArgs a;
  a.pl = ix->pl;
  a.src = ix->pool;
  a.dst = global ? npool : ix->pool;
  a.E = E.p;
  a.dirty = dirty.p;
  a.sstart = sstart.p;
  a.xs = xs.p;
  a.xe = xe.p;
  a.ctxl = ctxl.p;
  a.ctxr = ctxr.p;
  a.gx = gx.p;
  a.woff = woff.p;
  a.cxoff = cxoff.p;
  a.sbeg = sbeg.p;
  a.send = send.p;
  a.keep = keep.p;
  a.bkeys = br.keys;
  a.rid = rid.p;
  a.rpt = rpt.p;
  a.L = L;
  a.G = G;
  a.n = n;
  a.fresh = fresh;
  a.insert = insert;
  a.wkey = wkey.p;
  a.wmask = wmask.p;
  a.wslot = wslot.p;
  a.big = big.p;
  a.n_big = n_big.p;
  a.huge = huge.p;
  a.n_huge = n_big.p + 1;
  a.K = K.p;
  a.bleaf = bleaf.p;
  a.m = m;
  if (hc > 0) PSI_LAUNCH(k_seg_context, warp_grid(G), 256, 0, s, a);
  Buf<int32_t> block_leaf;
  if (global && n > 0) {
    const int64_t nb = ceil_div(n, kGlobBlock);
    if ((st = block_leaf.alloc(nb, s))) return st;
    PSI_LAUNCH(k_block_leaf, grid_for(L), 256, 0, s, E.p, L, nb, block_leaf.p);
    a.block_leaf = block_leaf.p;
  }
  if (global && insert) {
    if (D == 2)
      PSI_LAUNCH_NAMED("k_glob_insert", k_glob_insert<2>, grid_for(n + m, kGlobBlock), kGlobBlock, 0, s, a);
    else
      PSI_LAUNCH_NAMED("k_glob_insert", k_glob_insert<3>, grid_for(n + m, kGlobBlock), kGlobBlock, 0, s, a);
  } else if (global) {
    if (D == 2)
      PSI_LAUNCH_NAMED("k_glob_delete", k_glob_delete<2>, grid_for(n, kGlobBlock), kGlobBlock, 0, s, a);
    else
      PSI_LAUNCH_NAMED("k_glob_delete", k_glob_delete<3>, grid_for(n, kGlobBlock), kGlobBlock, 0, s, a);
  } else if (D == 2) {
    PSI_LAUNCH_NAMED("k_seg_small", k_seg_small<2>, warp_grid(ceil_div(L, 32)), 256, 0, s, a);
    PSI_LAUNCH_NAMED("k_seg_big", k_seg_big<2>, num_sms() * 8, 256, 0, s, a);
  } else {
    PSI_LAUNCH_NAMED("k_seg_small", k_seg_small<3>, warp_grid(ceil_div(L, 32)), 256, 0, s, a);
    PSI_LAUNCH_NAMED("k_seg_big", k_seg_big<3>, num_sms() * 8, 256, 0, s, a);
  }
  if (global) {
    free_pool(ix->pool, s);
    ix->pool = npool;
    ix->pool_used = S;
  } else {
    ix->pool_used += S;
  }
  // the segments' new leaves
  PLeaves nl;
  int64_t NL = 0;
  Buf<int64_t> rank, fl;
  WorkArray w = global ? WorkArray{ix->pool.pkey, nullptr, nullptr, 0u, W} : WorkArray{wkey.p, wmask.p, wslot.p, 0u, W};
  if (W > 0) {
    if ((st = work_leaves(ix, w, fresh + (uint32_t)S, nl, &NL, &rank, s))) {
      free_pleaves(nl, s);
      return st;
    }
  }
  Buf<int32_t> outl;
  Buf<int64_t> pos;
  if ((st = fl.alloc(G + 1, s)) || (st = outl.alloc(L, s)) || (st = pos.alloc(L + 1, s))) {
    free_pleaves(nl, s);
    return st;
  }
  if (W > 0) {
    PSI_LAUNCH(k_seg_first_leaf, grid_for(G + 1), 256, 0, s, a, rank.p, W, NL, fl.p);
  } else {
    PSI_CK(cudaMemsetAsync(fl.p, 0, sizeof(int64_t) * (G + 1), s));
  }
  PSI_LAUNCH(k_pl_outl, grid_for(L), 256, 0, s, dirty.p, sstart.p, gx.p, fl.p, L, outl.p);
  if ((st = scan_i32_to_i64(outl.p, pos.p, L, pos.p + L, s))) {
    free_pleaves(nl, s);
    return st;
  }
  int64_t Lnew = 0;
  PSI_CK(cudaMemcpyAsync(&Lnew, pos.p + L, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaStreamSynchronize(s));
  PLeaves out;
  if ((st = alloc_pleaves(out, D, Lnew, s))) {
    free_pleaves(nl, s);
    free_pleaves(out, s);
    return st;
  }
  if (D == 2)
    PSI_LAUNCH_NAMED("k_pl_assemble", k_pl_assemble<2>, grid_for(std::max(L, NL)), 256, 0, s, ix->pl, dirty.p, pos.p,
                     L, nl, NL, fl.p, xs.p, G, out);
  else
    PSI_LAUNCH_NAMED("k_pl_assemble", k_pl_assemble<3>, grid_for(std::max(L, NL)), 256, 0, s, ix->pl, dirty.p, pos.p,
                     L, nl, NL, fl.p, xs.p, G, out);
  free_pleaves(nl, s);
  free_pleaves(ix->pl, s);
  ix->pl = out;
  ix->L = Lnew;
  ix->n = n_new;
  if ((st = porth_compact_if_needed(ix, s))) return st;
  return porth_nodes(ix, s);
}

psi_status porth_insert(psi_index *ix, const int32_t *pts, const uint32_t *ids, int64_t m, cudaStream_t s) {
  if (ix->L == 0) {  // empty index: a fresh build of the batch
    return porth_build(ix, pts, ids, m, s);
  }
  return porth_update(ix, pts, ids, m, true, nullptr, s);
}

psi_status porth_delete(psi_index *ix, const int32_t *pts, const uint32_t *ids, int64_t m, int64_t *d_deleted,
                        cudaStream_t s) {
  if (ix->L == 0) {
    if (d_deleted) PSI_CK(cudaMemsetAsync(d_deleted, 0, sizeof(int64_t), s));
    return PSI_OK;
  }
  return porth_update(ix, pts, ids, m, false, d_deleted, s);
}

}  // namespace psi

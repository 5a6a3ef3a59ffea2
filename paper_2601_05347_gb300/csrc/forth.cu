// forth.cu -- the P-Orth of Sec 3 over float coordinates, built without
// space-filling curves (Algorithm 1): a node's region [lo, hi)^D is split at
// its midpoint in every dimension, mid = lo + 0.5f * (hi - lo) in float
// arithmetic (each operation rounded to nearest), a point taking the upper
// half of dimension d iff its coordinate >= mid; child c takes the upper half
// of dimension d iff bit d of c is set; a child exists iff it holds a point; a
// node is a leaf iff it holds at most phi points, is at depth max_depth, or
// cannot be split further (some mid not strictly inside its range: float
// precision exhausted).  Nodes are numbered breadth first, children
// consecutive in child-number order.
//
// GPU construction, one tree level per round (the sieve of Algorithm 1 with a
// skeleton of one level):
//   classify  every point of a splittable segment (a node with more than phi
//             points) finds its child by the segment's midpoints and counts
//             itself per (segment, child) with warp-aggregated atomics;
//   scan      of the counts gives each child's slot range inside its parent's;
//   scatter   moves the points to their child's range (order inside a node is
//             not kept: results never depend on it);
//   children  the non-empty (segment, child) pairs become the next level's
//             nodes in (parent, child) order, the splittable ones the next
//             round's segments.
// Boxes are tight and computed bottom up.  Queries: k-NN with squared
// distances sum_d (double(q_d) - double(p_d))^2 (each operation rounded to
// nearest, dimension order), ties by id; range count with closed boxes.
// D is 2..5, so a node has at most 32 children: one lane each.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "klist.cuh"

constexpr int kFMaxD = 5;

struct psi_forth {
  psi_fconfig cfg;
  int D = 2;
  int64_t n = 0, N = 0, cap = 0;
  float *px[kFMaxD] = {};  // points in slot order (a node's points are consecutive)
  uint32_t *pid = nullptr;
  float *blo[kFMaxD] = {}, *bhi[kFMaxD] = {};  // tight node boxes
  int32_t *cnt = nullptr, *kids = nullptr, *depth = nullptr;
  uint32_t *ref = nullptr;  // internal: first child; leaf: first slot
  int *d_status = nullptr;
  cudaStream_t last_stream = nullptr;
};

namespace psi {
namespace {

__device__ __forceinline__ float fmidpoint(float lo, float hi) {
  return __fadd_rn(lo, __fmul_rn(0.5f, __fsub_rn(hi, lo)));
}

struct FRegions {  // regions of the active segments, [D][A]
  float *lo[kFMaxD], *hi[kFMaxD];
};

struct FSeg {
  int64_t *node, *start, *cnt;
  FRegions r;
};

struct FPoints {
  float *x[kFMaxD];
  uint32_t *id;
};

template <int D>
__global__ void k_fload(const float *pts, const uint32_t *ids, int64_t n, FPoints out, const float *lo,
                        const float *hi, int *status) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const float x = pts[i * D + d];
      bad |= !(x >= lo[d] && x < hi[d]);
      out.x[d][i] = x;
    }
    out.id[i] = ids[i];
  }
  if (bad) atomicOr(status, ST_RANGE);
}

// Root: flag[0] = 1 when the region can be split (every midpoint strictly inside).
template <int D>
__global__ void k_froot(const float *lo, const float *hi, int *flag) {
  bool ok = true;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const float m = fmidpoint(lo[d], hi[d]);
    ok &= lo[d] < m && m < hi[d];
  }
  flag[0] = ok;
}

__device__ __forceinline__ int64_t seg_of(const int64_t *flat, int64_t A, int64_t f) {
  int64_t lo = 0, hi = A;  // last s with flat[s] <= f
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (flat[mid] <= f)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Child of every active point; counts per (segment, child); points gathered to tmp.
template <int D>
__global__ void k_fclassify(FSeg sg, const int64_t *flat, int64_t A, int64_t P, FPoints pts, FPoints tmp,
                            int32_t *sbuf, uint8_t *cbuf, uint32_t *counts) {
  for (int64_t f0 = (int64_t)blockIdx.x * blockDim.x; f0 < P; f0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = f0 + threadIdx.x;
    const bool valid = f < P;
    uint32_t key = 0xFFFFFFFFu;
    if (valid) {
      const int64_t s = seg_of(flat, A, f);
      const int64_t slot = sg.start[s] + (f - flat[s]);
      int c = 0;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const float x = pts.x[d][slot];
        tmp.x[d][f] = x;
        c |= (x >= fmidpoint(sg.r.lo[d][s], sg.r.hi[d][s])) << d;
      }
      tmp.id[f] = pts.id[slot];
      sbuf[f] = (int32_t)s;
      cbuf[f] = (uint8_t)c;
      key = (uint32_t)(s << D) | (uint32_t)c;
    }
    const uint32_t act = __ballot_sync(0xFFFFFFFFu, valid);
    if (valid) {
      const uint32_t peers = __match_any_sync(act, key);
      if ((peers & lanemask_lt()) == 0) atomicAdd(&counts[key], (uint32_t)__popc(peers));
    }
  }
}

// Points to their child's range: segment start + child offset + rank.
template <int D>
__global__ void k_fscatter(FSeg sg, const int64_t *flat, int64_t P, const int32_t *sbuf, const uint8_t *cbuf,
                           const int64_t *coff, uint32_t *cursor, FPoints tmp, FPoints pts) {
  for (int64_t f0 = (int64_t)blockIdx.x * blockDim.x; f0 < P; f0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = f0 + threadIdx.x;
    const bool valid = f < P;
    const uint32_t act = __ballot_sync(0xFFFFFFFFu, valid);
    if (!valid) continue;
    const int64_t s = sbuf[f];
    const uint32_t key = (uint32_t)(s << D) | cbuf[f];
    const uint32_t peers = __match_any_sync(act, key);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if ((int)(threadIdx.x & 31) == leader) base = atomicAdd(&cursor[key], (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    const int64_t dest = sg.start[s] + (coff[key] - flat[s]) + base + __popc(peers & lanemask_lt());
#pragma unroll
    for (int d = 0; d < D; ++d) pts.x[d][dest] = tmp.x[d][f];
    pts.id[dest] = tmp.id[f];
  }
}

struct FNodes {
  float *lo[kFMaxD], *hi[kFMaxD];
  int32_t *cnt, *kids, *depth;
  uint32_t *ref;
};

// Per (segment, child): 1 if the child holds a point / is splittable.
template <int D>
__global__ void k_fchild_flags(FSeg sg, int64_t A, const uint32_t *counts, int phi, int child_depth, int max_depth,
                               int32_t *nonempty, int32_t *active) {
  const int64_t E = A << D;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = e >> D;
    const int c = (int)(e & ((1 << D) - 1));
    const uint32_t k = counts[e];
    bool split = k > (uint32_t)phi && child_depth < max_depth;
    if (split) {
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const float lo = sg.r.lo[d][s], hi = sg.r.hi[d][s], m = fmidpoint(lo, hi);
        const float clo = ((c >> d) & 1) ? m : lo, chi = ((c >> d) & 1) ? hi : m;
        const float cm = fmidpoint(clo, chi);
        split &= clo < cm && cm < chi;
      }
    }
    nonempty[e] = k > 0;
    active[e] = k > 0 && split;
  }
}

// The children of this level, and their parents' links.
template <int D>
__global__ void k_fchildren(FSeg sg, const int64_t *flat, int64_t A, const uint32_t *counts, const int64_t *coff,
                            const int32_t *nonempty, const int64_t *crank, const int32_t *active,
                            const int64_t *arank, int64_t N0, int child_depth, FNodes nd, FSeg next) {
  const int64_t E = A << D;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    if (!nonempty[e]) continue;
    const int64_t s = e >> D;
    const int c = (int)(e & ((1 << D) - 1));
    const int64_t id = N0 + crank[e];
    const int64_t start = sg.start[s] + (coff[e] - flat[s]);
    nd.cnt[id] = (int32_t)counts[e];
    nd.depth[id] = child_depth;
    // the first child of its parent links the parent
    bool first = true;
    int kids = 0;
    for (int c2 = 0; c2 < (1 << D); ++c2) {
      const bool ne = nonempty[(s << D) + c2] != 0;
      kids += ne;
      if (c2 < c && ne) first = false;
    }
    if (first) {
      const int64_t p = sg.node[s];
      nd.ref[p] = (uint32_t)id;
      nd.kids[p] = kids;
    }
    if (active[e]) {
      const int64_t a = arank[e];
      next.node[a] = id;
      next.start[a] = start;
      next.cnt[a] = counts[e];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const float lo = sg.r.lo[d][s], hi = sg.r.hi[d][s], m = fmidpoint(lo, hi);
        next.r.lo[d][a] = ((c >> d) & 1) ? m : lo;
        next.r.hi[d][a] = ((c >> d) & 1) ? hi : m;
      }
    } else {
      nd.ref[id] = (uint32_t)start;
      nd.kids[id] = 0;
    }
  }
}

// Tight boxes of the nodes [a, b) of one level: leaves from their points,
// internal nodes from their children (one level deeper, already done).
template <int D>
__global__ void k_fboxes(FNodes nd, FPoints pts, int64_t a, int64_t b) {
  for (int64_t u = a + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < b; u += (int64_t)gridDim.x * blockDim.x) {
    float lo[D], hi[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      lo[d] = __int_as_float(0x7F800000);
      hi[d] = -__int_as_float(0x7F800000);
    }
    const uint32_t r = nd.ref[u];
    if (nd.kids[u] == 0) {
      for (int j = 0; j < nd.cnt[u]; ++j)
#pragma unroll
        for (int d = 0; d < D; ++d) {
          lo[d] = fminf(lo[d], pts.x[d][r + j]);
          hi[d] = fmaxf(hi[d], pts.x[d][r + j]);
        }
    } else {
      for (int j = 0; j < nd.kids[u]; ++j)
#pragma unroll
        for (int d = 0; d < D; ++d) {
          lo[d] = fminf(lo[d], nd.lo[d][r + j]);
          hi[d] = fmaxf(hi[d], nd.hi[d][r + j]);
        }
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
      nd.lo[d][u] = lo[d];
      nd.hi[d][u] = hi[d];
    }
  }
}

int fgrid(int64_t n, int threads = 256) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, threads), (int64_t)num_sms() * 16));
}

FNodes fnodes(psi_forth *ix) {
  FNodes f;
  for (int d = 0; d < kFMaxD; ++d) {
    f.lo[d] = ix->blo[d];
    f.hi[d] = ix->bhi[d];
  }
  f.cnt = ix->cnt;
  f.kids = ix->kids;
  f.depth = ix->depth;
  f.ref = ix->ref;
  return f;
}

void free_fnodes(psi_forth *ix, cudaStream_t s) {
  for (int d = 0; d < kFMaxD; ++d) {
    DevMem::free(ix->blo[d], s);
    DevMem::free(ix->bhi[d], s);
    ix->blo[d] = ix->bhi[d] = nullptr;
  }
  DevMem::free(ix->cnt, s);
  DevMem::free(ix->kids, s);
  DevMem::free(ix->depth, s);
  DevMem::free(ix->ref, s);
  ix->cnt = ix->kids = ix->depth = nullptr;
  ix->ref = nullptr;
  ix->cap = 0;
}

void free_fpoints(psi_forth *ix, cudaStream_t s) {
  for (int d = 0; d < kFMaxD; ++d) {
    DevMem::free(ix->px[d], s);
    ix->px[d] = nullptr;
  }
  DevMem::free(ix->pid, s);
  ix->pid = nullptr;
}

// Grows the node arrays to hold at least `need` nodes, keeping the first N.
psi_status grow_fnodes(psi_forth *ix, int64_t need, cudaStream_t s) {
  if (need <= ix->cap) return PSI_OK;
  const int64_t cap = std::max<int64_t>(need, ix->cap + ix->cap / 2);
  psi_forth t;
  t.D = ix->D;
  psi_status st;
  for (int d = 0; d < ix->D; ++d)
    if ((st = DevMem::alloc((void **)&t.blo[d], sizeof(float) * cap, s)) ||
        (st = DevMem::alloc((void **)&t.bhi[d], sizeof(float) * cap, s)))
      return st;
  if ((st = DevMem::alloc((void **)&t.cnt, sizeof(int32_t) * cap, s)) ||
      (st = DevMem::alloc((void **)&t.kids, sizeof(int32_t) * cap, s)) ||
      (st = DevMem::alloc((void **)&t.depth, sizeof(int32_t) * cap, s)) ||
      (st = DevMem::alloc((void **)&t.ref, sizeof(uint32_t) * cap, s)))
    return st;
  if (ix->N) {
    PSI_CK(cudaMemcpyAsync(t.cnt, ix->cnt, sizeof(int32_t) * ix->N, cudaMemcpyDeviceToDevice, s));
    PSI_CK(cudaMemcpyAsync(t.kids, ix->kids, sizeof(int32_t) * ix->N, cudaMemcpyDeviceToDevice, s));
    PSI_CK(cudaMemcpyAsync(t.depth, ix->depth, sizeof(int32_t) * ix->N, cudaMemcpyDeviceToDevice, s));
    PSI_CK(cudaMemcpyAsync(t.ref, ix->ref, sizeof(uint32_t) * ix->N, cudaMemcpyDeviceToDevice, s));
  }
  free_fnodes(ix, s);
  for (int d = 0; d < kFMaxD; ++d) {
    ix->blo[d] = t.blo[d];
    ix->bhi[d] = t.bhi[d];
    t.blo[d] = t.bhi[d] = nullptr;
  }
  ix->cnt = t.cnt;
  ix->kids = t.kids;
  ix->depth = t.depth;
  ix->ref = t.ref;
  ix->cap = cap;
  return PSI_OK;
}

struct SegBufs {
  Buf<int64_t> node, start, cnt;
  Buf<float> lo[kFMaxD], hi[kFMaxD];
  psi_status alloc(int64_t A, int D, cudaStream_t s) {
    psi_status st;
    if ((st = node.alloc(std::max<int64_t>(A, 1), s)) || (st = start.alloc(std::max<int64_t>(A, 1), s)) ||
        (st = cnt.alloc(std::max<int64_t>(A, 1), s)))
      return st;
    for (int d = 0; d < D; ++d)
      if ((st = lo[d].alloc(std::max<int64_t>(A, 1), s)) || (st = hi[d].alloc(std::max<int64_t>(A, 1), s))) return st;
    return PSI_OK;
  }
  FSeg view() {
    FSeg f;
    f.node = node.p;
    f.start = start.p;
    f.cnt = cnt.p;
    for (int d = 0; d < kFMaxD; ++d) {
      f.r.lo[d] = lo[d].p;
      f.r.hi[d] = hi[d].p;
    }
    return f;
  }
};

template <int D>
psi_status forth_build_d(psi_forth *ix, const float *pts, const uint32_t *ids, int64_t n, cudaStream_t s) {
  psi_status st;
  free_fnodes(ix, s);
  free_fpoints(ix, s);
  ix->n = n;
  ix->N = 0;
  if (n == 0) return PSI_OK;
  if (n >= (int64_t)1 << 31) {
    set_error("forth: at most 2^31 - 1 points");
    return PSI_ERR_INVALID;
  }
  Buf<float> tx[D], hlo, hhi;
  Buf<uint32_t> tid;
  for (int d = 0; d < D; ++d) {
    if ((st = DevMem::alloc((void **)&ix->px[d], sizeof(float) * n, s))) return st;
    if ((st = tx[d].alloc(n, s))) return st;
  }
  if ((st = DevMem::alloc((void **)&ix->pid, sizeof(uint32_t) * n, s)) || (st = tid.alloc(n, s)) ||
      (st = hlo.alloc(D, s)) || (st = hhi.alloc(D, s)))
    return st;
  PSI_CK(cudaMemcpyAsync(hlo.p, ix->cfg.lo, sizeof(float) * D, cudaMemcpyHostToDevice, s));
  PSI_CK(cudaMemcpyAsync(hhi.p, ix->cfg.hi, sizeof(float) * D, cudaMemcpyHostToDevice, s));
  FPoints P, T;
  for (int d = 0; d < kFMaxD; ++d) {
    P.x[d] = d < D ? ix->px[d] : nullptr;
    T.x[d] = d < D ? tx[d].p : nullptr;
  }
  P.id = ix->pid;
  T.id = tid.p;
  PSI_CK(cudaMemsetAsync(ix->d_status, 0, sizeof(int), s));
  PSI_LAUNCH_NAMED("k_fload", k_fload<D>, fgrid(n), 256, 0, s, pts, ids, n, P, hlo.p, hhi.p, ix->d_status);
  Buf<int> flag;
  if ((st = flag.alloc(2, s))) return st;
  PSI_LAUNCH_NAMED("k_froot", k_froot<D>, 1, 1, 0, s, hlo.p, hhi.p, flag.p);
  int h[2] = {0, 0};
  PSI_CK(cudaMemcpyAsync(&h[0], flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaMemcpyAsync(&h[1], ix->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaStreamSynchronize(s));
  if (h[1] & ST_RANGE) {
    PSI_CK(cudaMemsetAsync(ix->d_status, 0, sizeof(int), s));
    set_error("forth: a point lies outside the region [lo, hi)");
    return PSI_ERR_RANGE;
  }
  // the root
  if ((st = grow_fnodes(ix, std::max<int64_t>(1024, 4 * n / std::max(1, ix->cfg.leaf_size)), s))) return st;
  const int32_t nn = (int32_t)n, zero = 0;
  PSI_CK(cudaMemcpyAsync(ix->cnt, &nn, sizeof(int32_t), cudaMemcpyHostToDevice, s));
  PSI_CK(cudaMemcpyAsync(ix->depth, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, s));
  PSI_CK(cudaMemsetAsync(ix->kids, 0, sizeof(int32_t), s));
  PSI_CK(cudaMemsetAsync(ix->ref, 0, sizeof(uint32_t), s));
  ix->N = 1;
  std::vector<int64_t> level_off{0, 1};
  const bool split_root = n > ix->cfg.leaf_size && ix->cfg.max_depth > 0 && h[0];
  SegBufs cur, nxt;
  int64_t A = split_root ? 1 : 0;
  if (A) {
    if ((st = cur.alloc(1, D, s))) return st;
    const int64_t z = 0, nl = n;
    PSI_CK(cudaMemcpyAsync(cur.node.p, &z, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    PSI_CK(cudaMemcpyAsync(cur.start.p, &z, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    PSI_CK(cudaMemcpyAsync(cur.cnt.p, &nl, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    for (int d = 0; d < D; ++d) {
      PSI_CK(cudaMemcpyAsync(cur.lo[d].p, &ix->cfg.lo[d], sizeof(float), cudaMemcpyHostToDevice, s));
      PSI_CK(cudaMemcpyAsync(cur.hi[d].p, &ix->cfg.hi[d], sizeof(float), cudaMemcpyHostToDevice, s));
    }
  }
  Buf<int32_t> sbuf;
  Buf<uint8_t> cbuf;
  if ((st = sbuf.alloc(n, s)) || (st = cbuf.alloc(n, s))) return st;
  Buf<int64_t> tot;
  if ((st = tot.alloc(4, s))) return st;
  for (int level = 0; A > 0; ++level) {
    if (A >= ((int64_t)1 << (31 - D))) {
      set_error("forth: too many splittable nodes on one level");
      return PSI_ERR_INVALID;
    }
    const int64_t E = A << D;
    Buf<int64_t> flat, coff, crank, arank;
    Buf<uint32_t> counts, cursor;
    Buf<int32_t> nonempty, active;
    if ((st = flat.alloc(A, s)) || (st = coff.alloc(E, s)) || (st = crank.alloc(E, s)) || (st = arank.alloc(E, s)) ||
        (st = counts.alloc(E, s)) || (st = cursor.alloc(E, s)) || (st = nonempty.alloc(E, s)) ||
        (st = active.alloc(E, s)))
      return st;
    if ((st = scan_i64(cur.cnt.p, flat.p, A, tot.p, s))) return st;
    int64_t Pn = 0;
    PSI_CK(cudaMemcpyAsync(&Pn, tot.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    PSI_CK(cudaMemsetAsync(counts.p, 0, sizeof(uint32_t) * E, s));
    PSI_CK(cudaMemsetAsync(cursor.p, 0, sizeof(uint32_t) * E, s));
    PSI_CK(cudaStreamSynchronize(s));
    FSeg sg = cur.view();
    PSI_LAUNCH_NAMED("k_fclassify", k_fclassify<D>, fgrid(Pn), 256, 0, s, sg, flat.p, A, Pn, P, T, sbuf.p, cbuf.p,
                     counts.p);
    // child offsets: one exclusive scan over (segment, child) in order
    if ((st = scan_i32_to_i64(reinterpret_cast<const int32_t *>(counts.p), coff.p, E, nullptr, s))) return st;
    PSI_LAUNCH_NAMED("k_fscatter", k_fscatter<D>, fgrid(Pn), 256, 0, s, sg, flat.p, Pn, sbuf.p, cbuf.p, coff.p,
                     cursor.p, T, P);
    PSI_LAUNCH_NAMED("k_fchild_flags", k_fchild_flags<D>, fgrid(E), 256, 0, s, sg, A, counts.p, ix->cfg.leaf_size,
                     level + 1, ix->cfg.max_depth, nonempty.p, active.p);
    if ((st = scan_i32_to_i64(nonempty.p, crank.p, E, tot.p + 1, s)) ||
        (st = scan_i32_to_i64(active.p, arank.p, E, tot.p + 2, s)))
      return st;
    int64_t h2[2];
    PSI_CK(cudaMemcpyAsync(h2, tot.p + 1, sizeof(h2), cudaMemcpyDeviceToHost, s));
    PSI_CK(cudaStreamSynchronize(s));
    const int64_t C = h2[0], An = h2[1];
    if ((st = grow_fnodes(ix, ix->N + C, s))) return st;
    if ((st = nxt.alloc(An, D, s))) return st;
    PSI_LAUNCH_NAMED("k_fchildren", k_fchildren<D>, fgrid(E), 256, 0, s, sg, flat.p, A, counts.p, coff.p,
                     nonempty.p, crank.p, active.p, arank.p, ix->N, level + 1, fnodes(ix), nxt.view());
    ix->N += C;
    level_off.push_back(ix->N);
    std::swap(cur.node.p, nxt.node.p);
    std::swap(cur.start.p, nxt.start.p);
    std::swap(cur.cnt.p, nxt.cnt.p);
    for (int d = 0; d < D; ++d) {
      std::swap(cur.lo[d].p, nxt.lo[d].p);
      std::swap(cur.hi[d].p, nxt.hi[d].p);
    }
    A = An;
  }
  // boxes, deepest level first
  const FNodes nd = fnodes(ix);
  for (size_t l = level_off.size() - 1; l-- > 0;) {
    const int64_t a = level_off[l], b = level_off[l + 1];
    if (b > a) PSI_LAUNCH_NAMED("k_fboxes", k_fboxes<D>, fgrid(b - a), 256, 0, s, nd, P, a, b);
  }
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}

psi_status forth_build(psi_forth *ix, const float *pts, const uint32_t *ids, int64_t n, cudaStream_t s) {
  switch (ix->D) {
    case 2:
      return forth_build_d<2>(ix, pts, ids, n, s);
    case 3:
      return forth_build_d<3>(ix, pts, ids, n, s);
    case 4:
      return forth_build_d<4>(ix, pts, ids, n, s);
    default:
      return forth_build_d<5>(ix, pts, ids, n, s);
  }
}

// ---------------------------------------------------------------------------
// queries
// ---------------------------------------------------------------------------
constexpr int FQW = 4;       // warps per block
constexpr int FMAXLVL = 49;  // depth bound (max_depth <= 48)

struct FView {
  const float *lo[kFMaxD], *hi[kFMaxD], *px[kFMaxD];
  const int32_t *cnt, *kids;
  const uint32_t *ref, *pid;
  int64_t N;
};

FView fview(const psi_forth *ix) {
  FView v;
  for (int d = 0; d < kFMaxD; ++d) {
    v.lo[d] = ix->blo[d];
    v.hi[d] = ix->bhi[d];
    v.px[d] = ix->px[d];
  }
  v.cnt = ix->cnt;
  v.kids = ix->kids;
  v.ref = ix->ref;
  v.pid = ix->pid;
  v.N = ix->N;
  return v;
}

// Lower bound of the squared distance from the query to a box (0 inside), in
// float with every operation rounded toward -inf: it never exceeds the exact
// box distance, hence never the exact distance of a point inside.  FP64
// throughput is a small fraction of FP32 on this part, so only the distances
// that are reported are computed in double.
template <int D>
__device__ __forceinline__ float fbox_lower(const FView &t, uint32_t u, const float *qc) {
  float s = 0.0f;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const float lo = t.lo[d][u], hi = t.hi[d][u], q = qc[d];
    const float g = q < lo ? __fsub_rd(lo, q) : (q > hi ? __fsub_rd(q, hi) : 0.0f);
    s = __fadd_rd(s, __fmul_rd(g, g));
  }
  return s;
}

// The reported squared distance: double, each operation rounded to nearest.
template <int D>
__device__ __forceinline__ double fpoint_d2(const float *qc, const float *const *px, uint32_t slot) {
  double d2 = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const double g = __dsub_rn((double)qc[d], (double)px[d][slot]);
    d2 = __dadd_rn(d2, __dmul_rn(g, g));
  }
  return d2;
}

// Pruning key: the float bits of a non-negative distance (monotone).  A box or
// point is skipped only when its key exceeds the k-th's by more than kSlack:
// a float lower bound and a double value rounded to nearest of the same exact
// distance lie within two float units of each other.
__device__ __forceinline__ uint32_t fkey(float x) { return __float_as_uint(x); }
__device__ __forceinline__ uint32_t fkey(double x) { return __float_as_uint(__double2float_rn(x)); }
constexpr uint32_t kSlack = 2;

struct FKnnArgs {
  FView t;
  const float *q;
  int64_t nq;
  int k;
  const uint32_t *order;
  uint32_t *out_id;
  double *out_d2;
  int *status;
};

// One warp per query: depth-first search entering the nearest unvisited child
// first (the integer k-NN kernel's traversal, with float boxes and double
// distances); the children of each level on the path are kept in shared memory.
template <int D, int KPL>
__global__ __launch_bounds__(FQW * 32) void k_fknn(FKnnArgs a) {
  __shared__ uint32_t s_key[FQW][FMAXLVL][32];
  __shared__ uint32_t s_c0[FQW][FMAXLVL], s_mask[FQW][FMAXLVL], s_leaf[FQW][FMAXLVL];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const FView &t = a.t;
  for (int64_t qi = (int64_t)blockIdx.x * FQW + w; qi < a.nq; qi += (int64_t)gridDim.x * FQW) {
    const int64_t q = a.order ? (int64_t)a.order[qi] : qi;
    float qc[D];
#pragma unroll
    for (int d = 0; d < D; ++d) qc[d] = a.q[q * D + d];
    KList<KPL, double> kl;
    kl.init();
    auto limit = [&]() { return kl.kd == DistInf<double>::v() ? 0xFFFFFFFEu : fkey(kl.kd) + kSlack; };
    auto scan = [&](uint32_t u) {
      const uint32_t s0 = t.ref[u];
      const int cnt = t.cnt[u];
      for (int b = 0; b < cnt; b += 32) {
        const int j = b + lane;
        // float lower bound first; the double distance only where it may enter
        bool maybe = false;
        if (j < cnt) {
          float lb = 0.0f;
#pragma unroll
          for (int d = 0; d < D; ++d) {
            const float x = t.px[d][s0 + j], qd = qc[d];
            const float g = qd < x ? __fsub_rd(x, qd) : __fsub_rd(qd, x);
            lb = __fadd_rd(lb, __fmul_rd(g, g));
          }
          maybe = fkey(lb) <= limit();
        }
        if (__ballot_sync(0xFFFFFFFFu, maybe) == 0) continue;
        double d2 = DistInf<double>::v();
        uint32_t id = 0xFFFFFFFFu;
        if (maybe) {
          id = t.pid[s0 + j];
          d2 = fpoint_d2<D>(qc, t.px, s0 + j);
        }
        klist_offer(kl, maybe && kl.admits(d2, id), d2, id, a.k);
      }
    };
    auto expand = [&](uint32_t u, int lvl) {
      const int nk = t.kids[u];
      const uint32_t c0 = t.ref[u];
      uint32_t key = 0xFFFFFFFFu;
      bool leafc = false;
      if (lane < nk) {
        key = fkey(fbox_lower<D>(t, c0 + lane, qc));
        leafc = t.kids[c0 + lane] == 0;
      }
      s_key[w][lvl][lane] = key;
      const uint32_t mk = __ballot_sync(0xFFFFFFFFu, key <= limit());
      const uint32_t lf = __ballot_sync(0xFFFFFFFFu, leafc);
      if (lane == 0) {
        s_c0[w][lvl] = c0;
        s_mask[w][lvl] = mk;
        s_leaf[w][lvl] = lf;
      }
      __syncwarp();
    };
    if (t.N > 0) {
      if (t.kids[0] == 0) {
        scan(0);
      } else {
        int lvl = 0;
        expand(0, 0);
        while (lvl >= 0) {
          const uint32_t kdk = limit();
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
            scan(child);
          } else if (lvl + 1 < FMAXLVL) {
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
  }
}

// Range count, closed boxes: a stack of nodes per warp; a node inside the box
// adds its count, a straddling one is descended (leaves: points tested).
constexpr int FSTACK = 512;

template <int D>
__global__ __launch_bounds__(FQW * 32) void k_frange_count(FView t, const float *boxes, int64_t nq,
                                                           int64_t *counts, int *status) {
  __shared__ uint32_t s_node[FQW][FSTACK];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t q = (int64_t)blockIdx.x * FQW + w; q < nq; q += (int64_t)gridDim.x * FQW) {
    float blo[D], bhi[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      blo[d] = boxes[q * 2 * D + d];
      bhi[d] = boxes[q * 2 * D + D + d];
    }
    auto rel = [&](uint32_t u) {  // 0 disjoint, 1 straddles, 2 inside
      bool inside = true, disjoint = false;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        disjoint |= t.hi[d][u] < blo[d] || t.lo[d][u] > bhi[d];
        inside &= blo[d] <= t.lo[d][u] && t.hi[d][u] <= bhi[d];
      }
      return disjoint ? 0 : (inside ? 2 : 1);
    };
    int64_t acc = 0;
    int sp = 0;
    if (t.N > 0) {
      const int r = rel(0);
      if (r == 2) {
        if (lane == 0) acc += t.cnt[0];
      } else if (r == 1) {
        if (lane == 0) s_node[w][0] = 0;
        sp = 1;
      }
    }
    __syncwarp();
    while (sp > 0) {
      --sp;
      const uint32_t u = s_node[w][sp];
      __syncwarp();
      const int nk = t.kids[u];
      const uint32_t r0 = t.ref[u];
      if (nk == 0) {
        for (int b = 0; b < t.cnt[u]; b += 32) {
          const int j = b + lane;
          bool in = j < t.cnt[u];
          if (in)
#pragma unroll
            for (int d = 0; d < D; ++d) {
              const float x = t.px[d][r0 + j];
              in &= x >= blo[d] && x <= bhi[d];
            }
          acc += in;
        }
        continue;
      }
      uint32_t push = 0xFFFFFFFFu;
      if (lane < nk) {
        const int r = rel(r0 + lane);
        if (r == 2)
          acc += t.cnt[r0 + lane];
        else if (r == 1)
          push = r0 + lane;
      }
      const uint32_t m = __ballot_sync(0xFFFFFFFFu, push != 0xFFFFFFFFu);
      if (sp + __popc(m) > FSTACK) {
        if (lane == 0) atomicOr(status, ST_STACK);
        break;
      }
      if (push != 0xFFFFFFFFu) s_node[w][sp + __popc(m & lanemask_lt())] = push;
      sp += __popc(m);
      __syncwarp();
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    if (lane == 0) counts[q] = acc;
  }
}

// Locality order of the queries: a Morton key of their position in the region
// quantised to 60 / D bits per dimension.
template <int D>
__global__ void k_fquery_keys(const float *q, int64_t nq, const float *lo, const float *hi, uint64_t *keys,
                              uint32_t *vals) {
  constexpr int B = 60 / D;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t key = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const float u = (q[i * D + d] - lo[d]) / (hi[d] - lo[d]);
      const float c = fminf(fmaxf(u, 0.0f), 0.99999994f) * (float)(1u << B);
      const uint32_t g = (uint32_t)c;
      for (int b = 0; b < B; ++b) key |= (uint64_t)((g >> b) & 1u) << (b * D + d);
    }
    keys[i] = key;
    vals[i] = (uint32_t)i;
  }
}

template <int D>
psi_status forth_knn_d(const psi_forth *ix, const float *q, int64_t nq, int k, uint32_t *ids, double *d2,
                       cudaStream_t s) {
  Buf<uint64_t> k0, k1;
  Buf<uint32_t> v0, v1;
  Buf<float> hlo, hhi;
  const uint32_t *order = nullptr;
  psi_status st;
  if (nq >= 4096) {
    if ((st = k0.alloc(nq, s)) || (st = k1.alloc(nq, s)) || (st = v0.alloc(nq, s)) || (st = v1.alloc(nq, s)) ||
        (st = hlo.alloc(D, s)) || (st = hhi.alloc(D, s)))
      return st;
    PSI_CK(cudaMemcpyAsync(hlo.p, ix->cfg.lo, sizeof(float) * D, cudaMemcpyHostToDevice, s));
    PSI_CK(cudaMemcpyAsync(hhi.p, ix->cfg.hi, sizeof(float) * D, cudaMemcpyHostToDevice, s));
    PSI_LAUNCH_NAMED("k_fquery_keys", k_fquery_keys<D>, fgrid(nq), 256, 0, s, q, nq, hlo.p, hhi.p, k0.p, v0.p);
    SortResult r;
    EncodeSpec none;
    if ((st = sort_pairs(none, k0.p, v0.p, nq, 60, nullptr, k1.p, v1.p, k0.p, v0.p, ix->d_status, s, &r))) return st;
    order = r.vals;
  }
  FKnnArgs a{fview(ix), q, nq, k, order, ids, d2, ix->d_status};
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nq, FQW), (int64_t)num_sms() * 16));
  if (k <= 32)
    PSI_LAUNCH_NAMED("k_fknn", (k_fknn<D, 1>), g, FQW * 32, 0, s, a);
  else if (k <= 64)
    PSI_LAUNCH_NAMED("k_fknn", (k_fknn<D, 2>), g, FQW * 32, 0, s, a);
  else
    PSI_LAUNCH_NAMED("k_fknn", (k_fknn<D, 4>), g, FQW * 32, 0, s, a);
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}

psi_status forth_knn(const psi_forth *ix, const float *q, int64_t nq, int k, uint32_t *ids, double *d2,
                     cudaStream_t s) {
  switch (ix->D) {
    case 2:
      return forth_knn_d<2>(ix, q, nq, k, ids, d2, s);
    case 3:
      return forth_knn_d<3>(ix, q, nq, k, ids, d2, s);
    case 4:
      return forth_knn_d<4>(ix, q, nq, k, ids, d2, s);
    default:
      return forth_knn_d<5>(ix, q, nq, k, ids, d2, s);
  }
}

psi_status forth_range_count(const psi_forth *ix, const float *boxes, int64_t nq, int64_t *counts, cudaStream_t s) {
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nq, FQW), (int64_t)num_sms() * 16));
  const FView v = fview(ix);
  switch (ix->D) {
    case 2:
      PSI_LAUNCH_NAMED("k_frange_count", k_frange_count<2>, g, FQW * 32, 0, s, v, boxes, nq, counts, ix->d_status);
      break;
    case 3:
      PSI_LAUNCH_NAMED("k_frange_count", k_frange_count<3>, g, FQW * 32, 0, s, v, boxes, nq, counts, ix->d_status);
      break;
    case 4:
      PSI_LAUNCH_NAMED("k_frange_count", k_frange_count<4>, g, FQW * 32, 0, s, v, boxes, nq, counts, ix->d_status);
      break;
    default:
      PSI_LAUNCH_NAMED("k_frange_count", k_frange_count<5>, g, FQW * 32, 0, s, v, boxes, nq, counts, ix->d_status);
  }
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}

// ---------------------------------------------------------------------------
// updates: the tree is a function of the point set, so an update rebuilds it
// from the updated set
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_fto_aos(FPoints p, int64_t n, float *out, uint32_t *ids) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int d = 0; d < D; ++d) out[i * D + d] = p.x[d][i];
    ids[i] = p.id[i];
  }
}

// keep[i] = 0 iff the point (coordinates and id) is in the batch (batch sorted by id).
template <int D>
__global__ void k_fmark(FPoints p, int64_t n, const uint64_t *bkeys, const uint32_t *bvals, const float *bpts,
                        int64_t m, int32_t *keep, unsigned long long *deleted) {
  uint32_t del = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t id = p.id[i];
    int64_t lo = 0, hi = m;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (bkeys[mid] < id)
        lo = mid + 1;
      else
        hi = mid;
    }
    bool hit = false;
    for (int64_t j = lo; j < m && bkeys[j] == id && !hit; ++j) {
      bool same = true;
#pragma unroll
      for (int d = 0; d < D; ++d) same &= bpts[(int64_t)bvals[j] * D + d] == p.x[d][i];
      hit = same;
    }
    keep[i] = !hit;
    del += hit;
  }
  block_count_add(deleted, (uint32_t)del);
}

template <int D>
__global__ void k_fcompact(FPoints p, int64_t n, const int32_t *keep, const int64_t *pos, float *out,
                           uint32_t *ids) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!keep[i]) continue;
    const int64_t o = pos[i];
#pragma unroll
    for (int d = 0; d < D; ++d) out[o * D + d] = p.x[d][i];
    ids[o] = p.id[i];
  }
}

__global__ void k_fid_keys(const uint32_t *ids, int64_t m, uint64_t *keys, uint32_t *vals) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    keys[i] = ids[i];
    vals[i] = (uint32_t)i;
  }
}

__global__ void k_fcopy_i64(const unsigned long long *src, int64_t *dst) { *dst = (int64_t)*src; }

template <int D>
psi_status forth_insert_d(psi_forth *ix, const float *pts, const uint32_t *ids, int64_t m, cudaStream_t s) {
  const int64_t n = ix->n, tot = n + m;
  Buf<float> all;
  Buf<uint32_t> aid;
  psi_status st;
  if ((st = all.alloc(std::max<int64_t>(tot, 1) * D, s)) || (st = aid.alloc(std::max<int64_t>(tot, 1), s))) return st;
  FPoints P;
  for (int d = 0; d < kFMaxD; ++d) P.x[d] = d < D ? ix->px[d] : nullptr;
  P.id = ix->pid;
  if (n) PSI_LAUNCH_NAMED("k_fto_aos", k_fto_aos<D>, fgrid(n), 256, 0, s, P, n, all.p, aid.p);
  if (m) {
    PSI_CK(cudaMemcpyAsync(all.p + n * D, pts, sizeof(float) * m * D, cudaMemcpyDeviceToDevice, s));
    PSI_CK(cudaMemcpyAsync(aid.p + n, ids, sizeof(uint32_t) * m, cudaMemcpyDeviceToDevice, s));
  }
  return forth_build_d<D>(ix, all.p, aid.p, tot, s);
}

template <int D>
psi_status forth_delete_d(psi_forth *ix, const float *pts, const uint32_t *ids, int64_t m, int64_t *d_deleted,
                          cudaStream_t s) {
  const int64_t n = ix->n;
  psi_status st;
  Buf<uint64_t> k0, k1;
  Buf<uint32_t> v0, v1;
  Buf<int32_t> keep;
  Buf<int64_t> pos, tot;
  Buf<unsigned long long> del;
  if ((st = k0.alloc(std::max<int64_t>(m, 1), s)) || (st = k1.alloc(std::max<int64_t>(m, 1), s)) ||
      (st = v0.alloc(std::max<int64_t>(m, 1), s)) || (st = v1.alloc(std::max<int64_t>(m, 1), s)) ||
      (st = keep.alloc(std::max<int64_t>(n, 1), s)) || (st = pos.alloc(std::max<int64_t>(n, 1), s)) ||
      (st = tot.alloc(1, s)) || (st = del.alloc(1, s)))
    return st;
  PSI_CK(cudaMemsetAsync(del.p, 0, sizeof(unsigned long long), s));
  SortResult r{k0.p, v0.p};
  if (m) {
    PSI_LAUNCH(k_fid_keys, fgrid(m), 256, 0, s, ids, m, k0.p, v0.p);
    EncodeSpec none;
    if ((st = sort_pairs(none, k0.p, v0.p, m, 32, nullptr, k1.p, v1.p, k0.p, v0.p, ix->d_status, s, &r))) return st;
  }
  FPoints P;
  for (int d = 0; d < kFMaxD; ++d) P.x[d] = d < D ? ix->px[d] : nullptr;
  P.id = ix->pid;
  if (n) {
    PSI_LAUNCH_NAMED("k_fmark", k_fmark<D>, fgrid(n), 256, 0, s, P, n, r.keys, r.vals, pts, m, keep.p, del.p);
    if ((st = scan_i32_to_i64(keep.p, pos.p, n, tot.p, s))) return st;
  }
  if (d_deleted) PSI_LAUNCH(k_fcopy_i64, 1, 1, 0, s, del.p, d_deleted);
  int64_t left = 0;
  if (n) PSI_CK(cudaMemcpyAsync(&left, tot.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaStreamSynchronize(s));
  if (left == n) return PSI_OK;  // nothing deleted: the tree stands
  Buf<float> out;
  Buf<uint32_t> oid;
  if ((st = out.alloc(std::max<int64_t>(left, 1) * D, s)) || (st = oid.alloc(std::max<int64_t>(left, 1), s)))
    return st;
  PSI_LAUNCH_NAMED("k_fcompact", k_fcompact<D>, fgrid(n), 256, 0, s, P, n, keep.p, pos.p, out.p, oid.p);
  return forth_build_d<D>(ix, out.p, oid.p, left, s);
}

// Node arrays and points for inspection: boxes [N][D], points [n][D] in slot order.
template <int D>
__global__ void k_fexport(FView t, int64_t n, int32_t *depth_out, const int32_t *depth, int32_t *cnt, int32_t *kids,
                          uint32_t *ref, float *lo, float *hi, float *pts, uint32_t *ids) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < t.N; u += stride) {
    if (depth_out) depth_out[u] = depth[u];
    if (cnt) cnt[u] = t.cnt[u];
    if (kids) kids[u] = t.kids[u];
    if (ref) ref[u] = t.ref[u];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      if (lo) lo[u * D + d] = t.lo[d][u];
      if (hi) hi[u * D + d] = t.hi[d][u];
    }
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
#pragma unroll
    for (int d = 0; d < D; ++d)
      if (pts) pts[i * D + d] = t.px[d][i];
    if (ids) ids[i] = t.pid[i];
  }
}

}  // namespace
}  // namespace psi

using namespace psi;

namespace {
psi_status check_fcfg(const psi_fconfig *c) {
  if (!c || c->dim < 2 || c->dim > kFMaxD || c->leaf_size < 1 || c->leaf_size > 64 || c->max_depth < 0 ||
      c->max_depth > 48) {
    set_error("forth: dim must be 2..5, leaf_size 1..64, max_depth 0..48");
    return PSI_ERR_INVALID;
  }
  for (int d = 0; d < c->dim; ++d)
    if (!(c->lo[d] < c->hi[d])) {
      set_error("forth: the region needs lo < hi in every dimension");
      return PSI_ERR_INVALID;
    }
  return PSI_OK;
}
}  // namespace

extern "C" {

psi_status psi_forth_build(const psi_fconfig *cfg, const float *d_pts, const uint32_t *d_ids, int64_t n,
                           void *stream, psi_forth **out) {
  set_error("");
  psi_status st;
  if (!out || (st = check_fcfg(cfg)) || n < 0 || (n > 0 && (!d_pts || !d_ids))) {
    if (out) *out = nullptr;
    if (!cfg || n < 0 || !out) set_error("invalid forth build arguments");
    return PSI_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  psi_forth *ix = new psi_forth;
  ix->cfg = *cfg;
  ix->D = cfg->dim;
  ix->last_stream = s;
  if ((st = DevMem::alloc((void **)&ix->d_status, sizeof(int), s))) {
    delete ix;
    return st;
  }
  cudaError_t e = cudaMemsetAsync(ix->d_status, 0, sizeof(int), s);
  if (e != cudaSuccess) {
    psi_forth_destroy(ix);
    return cuda_fail(e, "cudaMemsetAsync");
  }
  if ((st = forth_build(ix, d_pts, d_ids, n, s))) {
    psi_forth_destroy(ix);
    *out = nullptr;
    return st;
  }
  *out = ix;
  return PSI_OK;
}

psi_status psi_forth_insert(psi_forth *ix, const float *d_pts, const uint32_t *d_ids, int64_t m, void *stream) {
  set_error("");
  if (!ix || m < 0 || (m > 0 && (!d_pts || !d_ids))) {
    set_error("invalid forth insert arguments");
    return PSI_ERR_INVALID;
  }
  if (m == 0) return PSI_OK;
  cudaStream_t s = (cudaStream_t)stream;
  ix->last_stream = s;
  switch (ix->D) {
    case 2:
      return forth_insert_d<2>(ix, d_pts, d_ids, m, s);
    case 3:
      return forth_insert_d<3>(ix, d_pts, d_ids, m, s);
    case 4:
      return forth_insert_d<4>(ix, d_pts, d_ids, m, s);
    default:
      return forth_insert_d<5>(ix, d_pts, d_ids, m, s);
  }
}

psi_status psi_forth_delete(psi_forth *ix, const float *d_pts, const uint32_t *d_ids, int64_t m,
                            int64_t *d_num_deleted, void *stream) {
  set_error("");
  if (!ix || m < 0 || (m > 0 && (!d_pts || !d_ids))) {
    set_error("invalid forth delete arguments");
    return PSI_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  ix->last_stream = s;
  switch (ix->D) {
    case 2:
      return forth_delete_d<2>(ix, d_pts, d_ids, m, d_num_deleted, s);
    case 3:
      return forth_delete_d<3>(ix, d_pts, d_ids, m, d_num_deleted, s);
    case 4:
      return forth_delete_d<4>(ix, d_pts, d_ids, m, d_num_deleted, s);
    default:
      return forth_delete_d<5>(ix, d_pts, d_ids, m, d_num_deleted, s);
  }
}

psi_status psi_forth_knn(const psi_forth *ix, const float *d_q, int64_t q, int32_t k, uint32_t *d_ids, double *d_d2,
                         void *stream) {
  set_error("");
  if (!ix || q < 0 || k < 1 || k > 128 || (q > 0 && (!d_q || !d_ids || !d_d2))) {
    set_error("invalid forth k-NN arguments (1 <= k <= 128)");
    return PSI_ERR_INVALID;
  }
  if (q == 0) return PSI_OK;
  return forth_knn(ix, d_q, q, k, d_ids, d_d2, (cudaStream_t)stream);
}

psi_status psi_forth_range_count(const psi_forth *ix, const float *d_boxes, int64_t q, int64_t *d_counts,
                                 void *stream) {
  set_error("");
  if (!ix || q < 0 || (q > 0 && (!d_boxes || !d_counts))) {
    set_error("invalid forth range count arguments");
    return PSI_ERR_INVALID;
  }
  if (q == 0) return PSI_OK;
  return forth_range_count(ix, d_boxes, q, d_counts, (cudaStream_t)stream);
}

int64_t psi_forth_size(const psi_forth *ix) { return ix ? ix->n : 0; }

int64_t psi_forth_num_nodes(const psi_forth *ix) { return ix ? ix->N : 0; }

psi_status psi_forth_export(const psi_forth *ix, int32_t *d_depth, int32_t *d_count, int32_t *d_kids,
                            uint32_t *d_ref, float *d_lo, float *d_hi, float *d_pts, uint32_t *d_ids, void *stream) {
  set_error("");
  if (!ix) {
    set_error("invalid forth export arguments");
    return PSI_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const FView v = fview(ix);
  const int g = fgrid(std::max(ix->N, ix->n));
  switch (ix->D) {
    case 2:
      PSI_LAUNCH_NAMED("k_fexport", k_fexport<2>, g, 256, 0, s, v, ix->n, d_depth, ix->depth, d_count, d_kids, d_ref,
                       d_lo, d_hi, d_pts, d_ids);
      break;
    case 3:
      PSI_LAUNCH_NAMED("k_fexport", k_fexport<3>, g, 256, 0, s, v, ix->n, d_depth, ix->depth, d_count, d_kids, d_ref,
                       d_lo, d_hi, d_pts, d_ids);
      break;
    case 4:
      PSI_LAUNCH_NAMED("k_fexport", k_fexport<4>, g, 256, 0, s, v, ix->n, d_depth, ix->depth, d_count, d_kids, d_ref,
                       d_lo, d_hi, d_pts, d_ids);
      break;
    default:
      PSI_LAUNCH_NAMED("k_fexport", k_fexport<5>, g, 256, 0, s, v, ix->n, d_depth, ix->depth, d_count, d_kids, d_ref,
                       d_lo, d_hi, d_pts, d_ids);
  }
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}

psi_status psi_forth_sync(psi_forth *ix, void *stream) {
  set_error("");
  if (!ix) return PSI_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  int h = 0;
  PSI_CK(cudaMemcpyAsync(&h, ix->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaStreamSynchronize(s));
  if (h) PSI_CK(cudaMemsetAsync(ix->d_status, 0, sizeof(int), s));
  if (h & ST_STACK) {
    set_error("forth: a traversal stack overflowed");
    return PSI_ERR_INVALID;
  }
  return PSI_OK;
}

void psi_forth_destroy(psi_forth *ix) {
  if (!ix) return;
  cudaStream_t s = ix->last_stream;
  free_fnodes(ix, s);
  free_fpoints(ix, s);
  DevMem::free(ix->d_status, s);
  delete ix;
}

}  // extern "C"

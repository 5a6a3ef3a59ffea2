// batch.cu -- many independent SPaC indexes built in one persistent launch.
//
// Each thread block takes whole indexes from an atomic work queue (largest
// first, so the long builds start early) and builds each one alone, with the
// same result as psi_build on that index (Algorithm 3):
//   E  curve keys of the index's points (computed once, Sec 4.1 "first
//      touch") and the histograms of all key digits, in one read;
//   P  a stable LSD radix sort of (key, local position) by 8-bit digits: the
//      index is cut into chunks of BT*IPT items; each chunk is ranked by warp
//      match.any into per-warp shared counters, staged in shared memory in
//      digit order and written to its digits' running offsets, so every
//      digit run is written contiguously;
//   T  runs of equal keys are put in id order;
//   G  leaf wrapping into blocks of 2*phi slots with boxes and counts;
//   U  the F-ary summary levels, bottom up.
// All storage is laid out by the host from the index sizes before the launch,
// so the launch allocates nothing and can be captured in a CUDA graph.
#include <algorithm>
#include <numeric>
#include <type_traits>
#include <vector>

#include "bitonic.cuh"
#include "index.cuh"
#include "keys.cuh"

struct psi_batch {
  psi_config cfg;
  int D = 2, phi = 32, C = 64, F = 32, curve = 0, key_bits = 60, threads = 512;
  int rb = 8;  // digit width of the block sort
  int nidx = 0;
  int64_t total = 0;
  std::vector<int64_t> off, leaves, node_off, block_off, nodes_per;
  psi::Pool pool;
  psi::NodeArrays nodes;
  int64_t nnodes = 0;
  // device copies
  int64_t *d_off = nullptr, *d_block_off = nullptr, *d_node_off = nullptr;
  int32_t *d_order = nullptr, *d_root = nullptr;
  uint32_t *d_queue = nullptr;
  int *d_status = nullptr;
  // sort scratch (indexed by global point position)
  uint64_t *kA = nullptr, *kB = nullptr;
  uint32_t *vA = nullptr, *vB = nullptr;
  // query scratch (psi_batch_knn_reserve)
  int64_t q_cap = 0;
  int32_t *d_qroot = nullptr, *d_qseg = nullptr;
  int64_t *d_qoff = nullptr;
  uint64_t *qk0 = nullptr, *qk1 = nullptr;
  uint32_t *qv0 = nullptr, *qv1 = nullptr;
  cudaStream_t last_stream = nullptr;
};

namespace psi {

int64_t summary_capacity(int64_t L, int F);

namespace {

constexpr int IPT = 8;  // keys per thread of a chunk

// Digit width of the block sort: 8 or 11 bits (a tuner dimension).
template <int RB>
struct BRadix {
  static constexpr int RADIX = 1 << RB;
  static constexpr int MAXP = (64 + RB - 1) / RB;  // passes of a 64-bit key
  // per-warp counters of a chunk (a warp ranks IPT * 32 keys) and staged digits
  using Count = typename std::conditional<RB == 8, uint32_t, uint16_t>::type;
  using Digit = typename std::conditional<RB == 8, uint8_t, uint16_t>::type;
};

struct BuildArgs {
  const int32_t *pts;
  const uint32_t *ids;
  const int64_t *off;
  const int32_t *order;
  int nidx;
  uint32_t *queue;
  uint64_t *kA, *kB;
  uint32_t *vA, *vB;
  Pool pool;
  const int64_t *block_off, *node_off;
  NodeArrays nodes;
  int32_t *root;
  int bits, phi, C, F, passes;
  int *status;
};

template <int BT, int RB>
struct BuildSmem {
  using R = BRadix<RB>;
  static constexpr int W = BT / 32;
  static constexpr int CH = BT * IPT;
  static constexpr int RADIX = R::RADIX;
  static constexpr int DPT = (RADIX + BT - 1) / BT;  // digits per thread in the per-digit steps
  uint32_t hist[R::MAXP][RADIX];      // digit counts, then exclusive bases
  uint32_t run[RADIX];                // running offset of each digit in the current pass
  typename R::Count wcnt[W][RADIX];   // per-warp counts of the current chunk
  uint32_t coff[RADIX];               // chunk-exclusive digit offsets
  uint64_t stage[CH];                 // chunk keys (then values) in digit order
  typename R::Digit dig[CH];          // digit of each staged position
  uint32_t wsum[32];
  alignas(16) uint8_t htab[kCurveTabBytes];
  int job;
  int nlong;
  int64_t long_start[64];
};

// Block-wide exclusive scan of digit counters: thread t holds the counts v of
// digits [t * DPT, (t + 1) * DPT) (zero past the last digit) and receives
// their exclusive prefixes in e.
template <int BT, int DPT>
__device__ __forceinline__ void block_excl_scan_digits(const uint32_t (&v)[DPT], uint32_t (&e)[DPT],
                                                       uint32_t *wsum) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  uint32_t tot = 0;
#pragma unroll
  for (int q = 0; q < DPT; ++q) tot += v[q];
  uint32_t x = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  uint32_t run = x - tot;
  for (int i = 0; i < w; ++i) run += wsum[i];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < DPT; ++q) {
    e[q] = run;
    run += v[q];
  }
}

template <int D, int CURVE, int BT, int RB>
__global__ __launch_bounds__(BT) void k_batch_build(BuildArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using SM = BuildSmem<BT, RB>;
  SM &sm = *reinterpret_cast<SM *>(smem_raw);
  constexpr int W = SM::W, CH = SM::CH, RADIX = SM::RADIX, DPT = SM::DPT, MAXP = BRadix<RB>::MAXP;
  using Count = typename BRadix<RB>::Count;
  using Digit = typename BRadix<RB>::Digit;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  curve_table_init<D, CURVE>(sm.htab);
  for (;;) {
    if (tid == 0) sm.job = (int)atomicAdd(a.queue, 1u);
    __syncthreads();
    const int job = sm.job;
    __syncthreads();
    if (job >= a.nidx) break;
    const int ix = a.order[job];
    const int64_t base = a.off[ix];
    const int64_t n = a.off[ix + 1] - base;
    const int64_t node0 = a.node_off[ix];
    if (n == 0) {
      if (tid == 0) a.root[ix] = -1;
      continue;
    }
    // E: keys, positions, all digit histograms
    for (int i = tid; i < MAXP * RADIX; i += BT) (&sm.hist[0][0])[i] = 0;
    __syncthreads();
    bool bad_any = false;
    for (int64_t t0 = 0; t0 < n; t0 += BT) {
      const int64_t t = t0 + tid;
      if (t < n) {
        int32_t c[D];
#pragma unroll
        for (int d = 0; d < D; ++d) c[d] = a.pts[(base + t) * D + d];
        bool bad;
        const uint64_t k = point_key<D, CURVE>(sm.htab, c, a.bits, bad);
        bad_any |= bad;
        a.kA[base + t] = k;
        a.vA[base + t] = (uint32_t)t;
        for (int p = 0; p < a.passes; ++p) atomicAdd(&sm.hist[p][(k >> (p * RB)) & (RADIX - 1)], 1u);
      }
    }
    if (bad_any) atomicOr(a.status, ST_RANGE);
    __syncthreads();
    for (int p = 0; p < a.passes; ++p) {
      uint32_t v[DPT], e[DPT];
#pragma unroll
      for (int q = 0; q < DPT; ++q) {
        const int d = tid * DPT + q;
        v[q] = d < RADIX ? sm.hist[p][d] : 0u;
      }
      block_excl_scan_digits<BT, DPT>(v, e, sm.wsum);
#pragma unroll
      for (int q = 0; q < DPT; ++q) {
        const int d = tid * DPT + q;
        if (d < RADIX) sm.hist[p][d] = e[q];
      }
    }
    __syncthreads();
    // P: digit passes, A -> B -> A ...
    for (int p = 0; p < a.passes; ++p) {
      const uint64_t *ki = (p & 1) ? a.kB : a.kA;
      const uint32_t *vi = (p & 1) ? a.vB : a.vA;
      uint64_t *ko = (p & 1) ? a.kA : a.kB;
      uint32_t *vo = (p & 1) ? a.vA : a.vB;
      const int shift = p * RB;
      for (int d = tid; d < RADIX; d += BT) sm.run[d] = sm.hist[p][d];
      for (int64_t c0 = 0; c0 < n; c0 += CH) {
        const int cn = (int)min((int64_t)CH, n - c0);
        for (int i = tid; i < W * RADIX; i += BT) (&sm.wcnt[0][0])[i] = 0;
        __syncthreads();
        uint64_t key[IPT];
        uint32_t rank[IPT];
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
          const int li = w * (IPT * 32) + j * 32 + lane;
          key[j] = li < cn ? ki[base + c0 + li] : ~0ull;
        }
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
          const int li = w * (IPT * 32) + j * 32 + lane;
          const bool valid = li < cn;
          const uint32_t dg = valid ? (uint32_t)(key[j] >> shift) & (RADIX - 1) : 0xFFFFFFFFu;
          const uint32_t peers = __match_any_sync(0xFFFFFFFFu, dg);
          const uint32_t before = __popc(peers & lanemask_lt());
          const uint32_t wb = valid ? (uint32_t)sm.wcnt[w][dg] : 0u;
          __syncwarp();
          if (valid && before == 0) sm.wcnt[w][dg] = (Count)(wb + __popc(peers));
          __syncwarp();
          rank[j] = wb + before;
        }
        __syncthreads();
        uint32_t ccount[DPT], cx[DPT];
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
          const int d = tid * DPT + q;
          uint32_t r = 0;
          if (d < RADIX)
            for (int ww = 0; ww < W; ++ww) {
              const uint32_t c = sm.wcnt[ww][d];
              sm.wcnt[ww][d] = (Count)r;
              r += c;
            }
          ccount[q] = r;
        }
        block_excl_scan_digits<BT, DPT>(ccount, cx, sm.wsum);
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
          const int d = tid * DPT + q;
          if (d < RADIX) sm.coff[d] = cx[q];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
          const int li = w * (IPT * 32) + j * 32 + lane;
          if (li < cn) {
            const uint32_t dg = (uint32_t)(key[j] >> shift) & (RADIX - 1);
            const uint32_t lp = sm.coff[dg] + sm.wcnt[w][dg] + rank[j];
            sm.stage[lp] = key[j];
            rank[j] = lp;
          }
        }
        __syncthreads();
        for (int pp = tid; pp < cn; pp += BT) {
          const uint64_t k = sm.stage[pp];
          const uint32_t dg = (uint32_t)(k >> shift) & (RADIX - 1);
          sm.dig[pp] = (Digit)dg;
          ko[base + sm.run[dg] + (pp - sm.coff[dg])] = k;
        }
        __syncthreads();
        uint32_t *sv = reinterpret_cast<uint32_t *>(sm.stage);
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
          const int li = w * (IPT * 32) + j * 32 + lane;
          if (li < cn) sv[rank[j]] = vi[base + c0 + li];
        }
        __syncthreads();
        for (int pp = tid; pp < cn; pp += BT) {
          const uint32_t dg = sm.dig[pp];
          vo[base + sm.run[dg] + (pp - sm.coff[dg])] = sv[pp];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
          const int d = tid * DPT + q;
          if (d < RADIX) sm.run[d] += ccount[q];
        }
        __syncthreads();
      }
    }
    const uint64_t *sk = (a.passes & 1) ? a.kB : a.kA;
    uint32_t *sv = (a.passes & 1) ? a.vB : a.vA;
    // T: equal keys in id order (runs of duplicate points; rare).  Runs of up
    // to 32 are insertion-sorted by one thread; longer runs are listed and
    // sorted by the whole block with the bitonic network.
    if (tid == 0) sm.nlong = 0;
    __syncthreads();
    for (int64_t t = tid; t + 1 < n; t += BT) {
      const uint64_t k = sk[base + t];
      if (sk[base + t + 1] != k || (t > 0 && sk[base + t - 1] == k)) continue;
      int64_t e = t + 2;
      while (e < n && sk[base + e] == k && e - t <= 32) ++e;
      if (e - t > 32) {
        const int slot = atomicAdd(&sm.nlong, 1);
        if (slot < 64) sm.long_start[slot] = t;
        continue;
      }
      for (int64_t x = t + 1; x < e; ++x) {
        const uint32_t v = sv[base + x], vid = a.ids[base + v];
        int64_t y = x - 1;
        while (y >= t && a.ids[base + sv[base + y]] > vid) {
          sv[base + y + 1] = sv[base + y];
          --y;
        }
        sv[base + y + 1] = v;
      }
    }
    __syncthreads();
    if (sm.nlong > 64) {
      if (tid == 0) atomicOr(a.status, ST_STACK);  // more than 64 piles of >32 duplicates: reported, not sorted
    } else {
      for (int r = 0; r < sm.nlong; ++r) {
        const int64_t t = sm.long_start[r];
        const uint64_t k = sk[base + t];
        int64_t lo = t, hi = n;
        while (lo < hi) {
          const int64_t mid = (lo + hi) >> 1;
          if (sk[base + mid] == k)
            lo = mid + 1;
          else
            hi = mid;
        }
        uint32_t *v = sv + base + t;
        const uint32_t *ids = a.ids + base;
        bitonic_ascending(
            lo - t, [&](int64_t x, int64_t y) { return ids[v[x]] < ids[v[y]]; },
            [&](int64_t x, int64_t y) {
              const uint32_t tmp = v[x];
              v[x] = v[y];
              v[y] = tmp;
            });
      }
    }
    __syncthreads();
    // G: leaves
    const int64_t L = (n + a.phi - 1) / a.phi;
    const int64_t blk0 = a.block_off[ix];
    for (int64_t leaf = w; leaf < L; leaf += W) {
      const int64_t b = leaf * a.phi;
      const int cnt = (int)min((int64_t)a.phi, n - b);
      int32_t lo[D], hi[D];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        lo[d] = INT32_MAX;
        hi[d] = INT32_MIN;
      }
      const int64_t slot0 = (blk0 + leaf) * a.C;
      for (int s = lane; s < cnt; s += 32) {
        const uint32_t v = sv[base + b + s];
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const int32_t c = a.pts[(base + v) * D + d];
          a.pool.px[d][slot0 + s] = c;
          lo[d] = min(lo[d], c);
          hi[d] = max(hi[d], c);
        }
        a.pool.pid[slot0 + s] = a.ids[base + v];
        a.pool.pkey[slot0 + s] = sk[base + b + s];
      }
#pragma unroll
      for (int d = 0; d < D; ++d) {
        lo[d] = __reduce_min_sync(0xFFFFFFFFu, lo[d]);
        hi[d] = __reduce_max_sync(0xFFFFFFFFu, hi[d]);
      }
      if (lane == 0) {
        const int64_t nd = node0 + leaf;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          a.nodes.lo[d][nd] = lo[d];
          a.nodes.hi[d][nd] = hi[d];
        }
        a.nodes.cnt[nd] = cnt;
        a.nodes.ref[nd] = (uint32_t)slot0;
        a.nodes.kids[nd] = 0;
        a.nodes.depth[nd] = 0;
      }
    }
    __syncthreads();
    // U: summary levels
    int64_t coff = 0, csize = L, total = L;
    int level = 0;
    while (csize > 1) {
      const int64_t par = (csize + a.F - 1) / a.F;
      ++level;
      for (int64_t j = w; j < par; j += W) {
        const int64_t c0 = j * a.F;
        const int nk = (int)min((int64_t)a.F, csize - c0);
        int32_t lo[D], hi[D];
        int32_t cnt = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          lo[d] = INT32_MAX;
          hi[d] = INT32_MIN;
        }
        if (lane < nk) {
          const int64_t c = node0 + coff + c0 + lane;
#pragma unroll
          for (int d = 0; d < D; ++d) {
            lo[d] = a.nodes.lo[d][c];
            hi[d] = a.nodes.hi[d][c];
          }
          cnt = a.nodes.cnt[c];
        }
#pragma unroll
        for (int d = 0; d < D; ++d) {
          lo[d] = __reduce_min_sync(0xFFFFFFFFu, lo[d]);
          hi[d] = __reduce_max_sync(0xFFFFFFFFu, hi[d]);
        }
        cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
        if (lane == 0) {
          const int64_t pn = node0 + total + j;
#pragma unroll
          for (int d = 0; d < D; ++d) {
            a.nodes.lo[d][pn] = lo[d];
            a.nodes.hi[d][pn] = hi[d];
          }
          a.nodes.cnt[pn] = cnt;
          a.nodes.ref[pn] = (uint32_t)(node0 + coff + c0);
          a.nodes.kids[pn] = nk;
          a.nodes.depth[pn] = level;
        }
      }
      __syncthreads();
      coff = total;
      total += par;
      csize = par;
    }
    if (tid == 0) a.root[ix] = (int32_t)(node0 + total - 1);
    __syncthreads();
  }
}

// Root of each query's index; segment s covers queries [qoff[s], qoff[s+1]).
__global__ void k_query_roots(const int64_t *qoff, int nseg, const int32_t *root, int64_t nq, int32_t *qroot,
                              int32_t *qseg) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nseg;  // last segment with qoff <= q
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (qoff[mid] <= q)
        lo = mid;
      else
        hi = mid;
    }
    qroot[q] = root[lo];
    qseg[q] = lo;
  }
}

// Ordering key of a query: its index number above the top 40 bits of its curve key.
template <int D, int CURVE>
__global__ void k_query_keys(const int32_t *q, const int32_t *qseg, int64_t nq, int bits, int shift, uint64_t *keys,
                             uint32_t *vals) {
  __shared__ alignas(16) uint8_t htab[kCurveTabBytes];
  curve_table_init<D, CURVE>(htab);
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t c[D];
#pragma unroll
    for (int d = 0; d < D; ++d) c[d] = q[i * D + d];
    bool bad;
    keys[i] = ((uint64_t)qseg[i] << 40) | (point_key<D, CURVE>(htab, c, bits, bad) >> shift);
    vals[i] = (uint32_t)i;
  }
}

template <int D, int CURVE, int BT, int RB>
psi_status launch_build(psi_batch *b, const BuildArgs &a, cudaStream_t s) {
  const size_t smem = sizeof(BuildSmem<BT, RB>);
  auto kern = k_batch_build<D, CURVE, BT, RB>;
  PSI_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  PSI_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BT, smem));
  const int grid = std::max(1, std::min(b->nidx, num_sms() * std::max(per_sm, 1)));
  PSI_LAUNCH_NAMED("k_batch_build", kern, grid, BT, smem, s, a);
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}

}  // namespace
}  // namespace psi

using namespace psi;

static void batch_free(psi_batch *b) {
  cudaStream_t s = b->last_stream;
  free_pool(b->pool, s);
  free_nodes(b->nodes, s);
  for (void *p : {(void *)b->d_off, (void *)b->d_block_off, (void *)b->d_node_off, (void *)b->d_order,
                  (void *)b->d_root, (void *)b->d_queue, (void *)b->d_status, (void *)b->kA, (void *)b->kB,
                  (void *)b->vA, (void *)b->vB, (void *)b->d_qroot, (void *)b->d_qseg, (void *)b->d_qoff,
                  (void *)b->qk0, (void *)b->qk1, (void *)b->qv0, (void *)b->qv1})
    DevMem::free(p, s);
  delete b;
}

extern "C" {

psi_status psi_batch_create(const psi_config *cfg, const int64_t *h_offsets, int32_t nidx, int32_t threads,
                            void *stream, psi_batch **out) {
  set_error("");
  if (!out || !cfg || !h_offsets || nidx < 1) {
    set_error("invalid batch arguments");
    return PSI_ERR_INVALID;
  }
  *out = nullptr;
  if (cfg->kind == PSI_PORTH || cfg->dim < 2 || cfg->dim > 3 ||
      cfg->leaf_size < 1 || cfg->leaf_size > 64 || cfg->coord_bits < 1 ||
      cfg->coord_bits > (cfg->dim == 2 ? 31 : 21) || (cfg->fanout != 0 && (cfg->fanout < 2 || cfg->fanout > 32))) {
    set_error("batched indexes support SPaC-Z / SPaC-H with the usual leaf, bit and fanout limits");
    return PSI_ERR_INVALID;
  }
  if (threads != 0 && threads != 256 && threads != 512 && threads != 1024) {
    set_error("threads must be 0 (512), 256, 512 or 1024");
    return PSI_ERR_INVALID;
  }
  if (cfg->radix_bits != 0 && cfg->radix_bits != 8 && cfg->radix_bits != 11) {
    set_error("batched indexes sort with 8- or 11-bit digits (radix_bits 0, 8 or 11)");
    return PSI_ERR_INVALID;
  }
  if (cfg->radix_bits == 11 && threads == 1024) {
    set_error("11-bit digits need 256 or 512 threads (the block's shared memory)");
    return PSI_ERR_INVALID;
  }
  for (int i = 0; i < nidx; ++i)
    if (h_offsets[i + 1] < h_offsets[i] || h_offsets[0] != 0) {
      set_error("offsets must start at 0 and be non-decreasing");
      return PSI_ERR_INVALID;
    }
  if (h_offsets[nidx] >= (int64_t(1) << 32)) {
    set_error("at most 2^32 - 1 points in one batch");
    return PSI_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  psi_batch *b = new psi_batch();
  b->cfg = *cfg;
  b->D = cfg->dim;
  b->phi = cfg->leaf_size;
  b->C = 2 * cfg->leaf_size;
  b->F = cfg->fanout ? cfg->fanout : 32;
  b->curve = cfg->kind == PSI_SPAC_H ? CURVE_HILBERT : CURVE_MORTON;
  b->key_bits = cfg->dim * cfg->coord_bits;
  b->threads = threads ? threads : 512;
  b->rb = cfg->radix_bits == 11 ? 11 : 8;
  b->nidx = nidx;
  b->last_stream = s;
  b->off.assign(h_offsets, h_offsets + nidx + 1);
  b->total = b->off[nidx];
  b->leaves.resize(nidx);
  b->node_off.resize(nidx + 1);
  b->block_off.resize(nidx + 1);
  b->nodes_per.resize(nidx);
  int64_t nodes = 0, blocks = 0;
  for (int i = 0; i < nidx; ++i) {
    const int64_t n = b->off[i + 1] - b->off[i];
    b->leaves[i] = ceil_div(n, b->phi);
    b->nodes_per[i] = n ? summary_capacity(b->leaves[i], b->F) : 0;
    b->node_off[i] = nodes;
    b->block_off[i] = blocks;
    nodes += b->nodes_per[i];
    blocks += b->leaves[i];
  }
  b->node_off[nidx] = nodes;
  b->block_off[nidx] = blocks;
  b->nnodes = nodes;
  if (nodes >= (int64_t(1) << 31) || blocks * b->C >= (int64_t(1) << 32)) {
    delete b;
    set_error("batch too large for 32-bit node and slot references");
    return PSI_ERR_INVALID;
  }
  std::vector<int32_t> order(nidx);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return b->off[x + 1] - b->off[x] > b->off[y + 1] - b->off[y];
  });
  psi_status st;
  const size_t N = (size_t)std::max<int64_t>(b->total, 1);
  do {
    if ((st = alloc_pool(b->pool, b->D, std::max<int64_t>(blocks * b->C, 1), s))) break;
    if ((st = alloc_nodes(b->nodes, b->D, std::max<int64_t>(nodes, 1), false, s))) break;
    if ((st = DevMem::alloc((void **)&b->d_off, sizeof(int64_t) * (nidx + 1), s))) break;
    if ((st = DevMem::alloc((void **)&b->d_block_off, sizeof(int64_t) * (nidx + 1), s))) break;
    if ((st = DevMem::alloc((void **)&b->d_node_off, sizeof(int64_t) * (nidx + 1), s))) break;
    if ((st = DevMem::alloc((void **)&b->d_order, sizeof(int32_t) * nidx, s))) break;
    if ((st = DevMem::alloc((void **)&b->d_root, sizeof(int32_t) * nidx, s))) break;
    if ((st = DevMem::alloc((void **)&b->d_queue, sizeof(uint32_t), s))) break;
    if ((st = DevMem::alloc((void **)&b->d_status, sizeof(int), s))) break;
    if ((st = DevMem::alloc((void **)&b->kA, sizeof(uint64_t) * N, s))) break;
    if ((st = DevMem::alloc((void **)&b->kB, sizeof(uint64_t) * N, s))) break;
    if ((st = DevMem::alloc((void **)&b->vA, sizeof(uint32_t) * N, s))) break;
    if ((st = DevMem::alloc((void **)&b->vB, sizeof(uint32_t) * N, s))) break;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(b->d_off, b->off.data(), sizeof(int64_t) * (nidx + 1), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(b->d_block_off, b->block_off.data(), sizeof(int64_t) * (nidx + 1),
                             cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(b->d_node_off, b->node_off.data(), sizeof(int64_t) * (nidx + 1),
                             cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(b->d_order, order.data(), sizeof(int32_t) * nidx, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemsetAsync(b->d_status, 0, sizeof(int), s)) ||
        (e = cudaStreamSynchronize(s))) {
      st = cuda_fail(e, "batch setup");
      break;
    }
  } while (0);
  if (st) {
    batch_free(b);
    return st;
  }
  *out = b;
  return PSI_OK;
}

psi_status psi_batch_build(psi_batch *b, const int32_t *d_pts, const uint32_t *d_ids, void *stream) {
  set_error("");
  if (!b || (b->total > 0 && (!d_pts || !d_ids))) {
    set_error("invalid batch build arguments");
    return PSI_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  b->last_stream = s;
  PSI_CK(cudaMemsetAsync(b->d_queue, 0, sizeof(uint32_t), s));
  BuildArgs a;
  a.pts = d_pts;
  a.ids = d_ids;
  a.off = b->d_off;
  a.order = b->d_order;
  a.nidx = b->nidx;
  a.queue = b->d_queue;
  a.kA = b->kA;
  a.kB = b->kB;
  a.vA = b->vA;
  a.vB = b->vB;
  a.pool = b->pool;
  a.block_off = b->d_block_off;
  a.node_off = b->d_node_off;
  a.nodes = b->nodes;
  a.root = b->d_root;
  a.bits = b->cfg.coord_bits;
  a.phi = b->phi;
  a.C = b->C;
  a.F = b->F;
  a.passes = (b->key_bits + b->rb - 1) / b->rb;
  a.status = b->d_status;
#define BUILD_CASE(DD, CC)                                                        \
  do {                                                                            \
    if (b->rb == 11) {                                                            \
      if (b->threads == 256) return launch_build<DD, CC, 256, 11>(b, a, s);       \
      return launch_build<DD, CC, 512, 11>(b, a, s);                              \
    }                                                                             \
    if (b->threads == 256) return launch_build<DD, CC, 256, 8>(b, a, s);          \
    if (b->threads == 1024) return launch_build<DD, CC, 1024, 8>(b, a, s);        \
    return launch_build<DD, CC, 512, 8>(b, a, s);                                 \
  } while (0)
  if (b->D == 3 && b->curve == CURVE_HILBERT) BUILD_CASE(3, 1);
  if (b->D == 3) BUILD_CASE(3, 0);
  if (b->curve == CURVE_HILBERT) BUILD_CASE(2, 1);
  BUILD_CASE(2, 0);
#undef BUILD_CASE
}

psi_status psi_batch_knn_reserve(psi_batch *b, int64_t max_queries, void *stream) {
  set_error("");
  if (!b || max_queries < 0 || max_queries >= (int64_t(1) << 32)) {
    set_error("invalid reserve arguments");
    return PSI_ERR_INVALID;
  }
  if (max_queries <= b->q_cap) return PSI_OK;
  cudaStream_t s = (cudaStream_t)stream;
  for (void *p : {(void *)b->d_qroot, (void *)b->d_qseg, (void *)b->d_qoff, (void *)b->qk0, (void *)b->qk1,
                  (void *)b->qv0, (void *)b->qv1})
    DevMem::free(p, s);
  b->d_qroot = b->d_qseg = nullptr;
  b->d_qoff = nullptr;
  b->qk0 = b->qk1 = nullptr;
  b->qv0 = b->qv1 = nullptr;
  const size_t Q = (size_t)std::max<int64_t>(max_queries, 1);
  psi_status st;
  if ((st = DevMem::alloc((void **)&b->d_qroot, sizeof(int32_t) * Q, s)) ||
      (st = DevMem::alloc((void **)&b->d_qseg, sizeof(int32_t) * Q, s)) ||
      (st = DevMem::alloc((void **)&b->d_qoff, sizeof(int64_t) * (b->nidx + 1), s)) ||
      (st = DevMem::alloc((void **)&b->qk0, sizeof(uint64_t) * Q, s)) ||
      (st = DevMem::alloc((void **)&b->qk1, sizeof(uint64_t) * Q, s)) ||
      (st = DevMem::alloc((void **)&b->qv0, sizeof(uint32_t) * Q, s)) ||
      (st = DevMem::alloc((void **)&b->qv1, sizeof(uint32_t) * Q, s)))
    return st;
  b->q_cap = max_queries;
  return PSI_OK;
}

static psi_status batch_knn(psi_batch *b, const int32_t *d_q, const int64_t *d_qoffsets, int64_t nq, int32_t k,
                            uint32_t *d_ids, int64_t *d_d2, unsigned long long *d_stats, void *stream) {
  set_error("");
  if (!b || nq < 0 || k < 1 || k > 128 || (nq > 0 && (!d_q || !d_qoffsets || !d_ids || !d_d2))) {
    set_error("invalid batch k-NN arguments (1 <= k <= 128)");
    return PSI_ERR_INVALID;
  }
  if (nq > b->q_cap) {
    set_error("psi_batch_knn: reserve at least nq queries first (psi_batch_knn_reserve)");
    return PSI_ERR_INVALID;
  }
  if (nq == 0) return PSI_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nq, 256), (int64_t)num_sms() * 16));
  PSI_LAUNCH(k_query_roots, g, 256, 0, s, d_qoffsets, b->nidx, b->d_root, nq, b->d_qroot, b->d_qseg);
  const int order_bits = std::min(40, b->key_bits);
  const int shift = b->key_bits - order_bits;
  if (b->D == 3 && b->curve == CURVE_HILBERT)
    PSI_LAUNCH_NAMED("k_query_keys", (k_query_keys<3, 1>), g, 256, 0, s, d_q, b->d_qseg, nq, b->cfg.coord_bits, shift,
                     b->qk0, b->qv0);
  else if (b->D == 3)
    PSI_LAUNCH_NAMED("k_query_keys", (k_query_keys<3, 0>), g, 256, 0, s, d_q, b->d_qseg, nq, b->cfg.coord_bits, shift,
                     b->qk0, b->qv0);
  else if (b->curve == CURVE_HILBERT)
    PSI_LAUNCH_NAMED("k_query_keys", (k_query_keys<2, 1>), g, 256, 0, s, d_q, b->d_qseg, nq, b->cfg.coord_bits, shift,
                     b->qk0, b->qv0);
  else
    PSI_LAUNCH_NAMED("k_query_keys", (k_query_keys<2, 0>), g, 256, 0, s, d_q, b->d_qseg, nq, b->cfg.coord_bits, shift,
                     b->qk0, b->qv0);
  int segbits = 1;
  while ((1 << segbits) < b->nidx) ++segbits;
  SortResult r;
  EncodeSpec none;
  psi_status st = sort_pairs(none, b->qk0, b->qv0, nq, 40 + segbits, nullptr, b->qk1, b->qv1, b->qk0, b->qv0,
                             b->d_status, s, &r);
  if (st) return st;
  TreeView tv;
  for (int d = 0; d < 3; ++d) {
    tv.lo[d] = b->nodes.lo[d];
    tv.hi[d] = b->nodes.hi[d];
    tv.px[d] = b->pool.px[d];
  }
  tv.cnt = b->nodes.cnt;
  tv.ref = b->nodes.ref;
  tv.kids = b->nodes.kids;
  tv.pid = b->pool.pid;
  tv.root = -1;
  KnnSeed seed;  // leaves at each query's curve position in its own index
  seed.qkey = r.keys;
  seed.qkey_mask = (uint64_t(1) << order_bits) - 1;
  seed.key_shift = shift;
  seed.qseg = b->d_qseg;
  seed.off = b->d_off;
  seed.node_off = b->d_node_off;
  seed.phi = b->phi;
  seed.pkey = b->pool.pkey;
  seed.pos = reinterpret_cast<uint32_t *>(r.keys == b->qk0 ? b->qk1 : b->qk0);  // the sort's free key buffer
  return run_knn_roots(tv, d_q, nq, k, r.vals, b->d_qroot, b->D, d_ids, d_d2, b->d_status, d_stats, s, seed);
}

psi_status psi_batch_knn(psi_batch *b, const int32_t *d_q, const int64_t *d_qoffsets, int64_t nq, int32_t k,
                         uint32_t *d_ids, int64_t *d_d2, void *stream) {
  return batch_knn(b, d_q, d_qoffsets, nq, k, d_ids, d_d2, nullptr, stream);
}

psi_status psi_batch_knn_instrumented(psi_batch *b, const int32_t *d_q, const int64_t *d_qoffsets, int64_t nq,
                                      int32_t k, uint32_t *d_ids, int64_t *d_d2, uint64_t *d_stats, void *stream) {
  if (!d_stats) {
    set_error("psi_batch_knn_instrumented: d_stats is null");
    return PSI_ERR_INVALID;
  }
  return batch_knn(b, d_q, d_qoffsets, nq, k, d_ids, d_d2, (unsigned long long *)d_stats, stream);
}

psi_status psi_batch_sync(psi_batch *b, void *stream) {
  set_error("");
  if (!b) return PSI_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  int h = 0;
  PSI_CK(cudaMemcpyAsync(&h, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaStreamSynchronize(s));
  if (h) PSI_CK(cudaMemsetAsync(b->d_status, 0, sizeof(int), s));
  if (h & ST_RANGE) {
    set_error("a coordinate lies outside [0, 2^coord_bits)");
    return PSI_ERR_RANGE;
  }
  if (h & ST_TIMEOUT) {
    set_error("a bounded device-side wait timed out");
    return PSI_ERR_DEVICE_TIMEOUT;
  }
  if (h & ST_STACK) {
    set_error("query traversal depth exceeded");
    return PSI_ERR_CUDA;
  }
  return PSI_OK;
}

psi_status psi_batch_export_index(const psi_batch *b, int32_t i, int32_t *d_counts, int32_t *d_lo, int32_t *d_hi,
                                  int64_t *h_leaves, void *stream);

psi_status psi_batch_destroy(psi_batch *b) {
  if (!b) return PSI_OK;
  cudaDeviceSynchronize();
  batch_free(b);
  PSI_CK(cudaDeviceSynchronize());
  return PSI_OK;
}

int64_t psi_batch_num_leaves(const psi_batch *b, int32_t i) {
  return (b && i >= 0 && i < b->nidx) ? b->leaves[i] : 0;
}

}  // extern "C"

namespace psi {
namespace {
__global__ void k_batch_export_leaves(const NodeArrays nodes, int64_t node0, int64_t L, int D, int32_t *counts,
                                      int32_t *lo, int32_t *hi) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (int64_t)gridDim.x * blockDim.x) {
    if (counts) counts[i] = nodes.cnt[node0 + i];
    for (int d = 0; d < D; ++d) {
      if (lo) lo[i * D + d] = nodes.lo[d][node0 + i];
      if (hi) hi[i * D + d] = nodes.hi[d][node0 + i];
    }
  }
}
}  // namespace
}  // namespace psi

extern "C" psi_status psi_batch_export_index(const psi_batch *b, int32_t i, int32_t *d_counts, int32_t *d_lo,
                                             int32_t *d_hi, int64_t *h_leaves, void *stream) {
  if (!b || i < 0 || i >= b->nidx) return PSI_ERR_INVALID;
  const int64_t L = b->leaves[i];
  if (h_leaves) *h_leaves = L;
  if (L == 0) return PSI_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(L, 256), 1024));
  PSI_LAUNCH(k_batch_export_leaves, g, 256, 0, s, b->nodes, b->node_off[i], L, b->D, d_counts, d_lo, d_hi);
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}

// sort.cu -- onesweep LSD radix sort of (uint64 key, uint32 value) pairs.
//
// Role in the method: Algorithm 3 sorts <code, id> pairs only, computing each
// point's curve code when the point is first touched by the sort.  Here the
// sort is a least-significant-digit radix sort with 8-bit digits in the
// "onesweep" arrangement (one upfront histogram pass for all digits, then one
// pass per digit that ranks a tile in shared memory and obtains the tile's
// global digit offsets by decoupled look-back over earlier tiles):
//   * k_sort_hist     reads every key once (computing it from the point when
//                     encoding) and counts the first digit;
//   * k_onesweep      per digit: warp-level ranking (peer lanes from one ballot
//                     per digit bit) into per-warp shared counters (stable),
//                     tile totals published to a look-back table, bounded spin
//                     on predecessors, shared-memory staging so that each
//                     digit's run is written out contiguously; it also counts
//                     the next digit of its keys for the following pass;
//   * k_hist_scan     (the allocation-free sort) scans histograms of all digits.
// An encoding sort computes Morton keys from the points in its first digit
// pass, so they are never written before they are sorted; Hilbert keys, whose
// arithmetic costs more than an 8-byte write and read, are computed once in
// the histogram pass and written out.  A sort of at least kPackMin pairs whose
// input is locally ordered (most neighbouring inputs share their top 24 key
// bits, counted by the histogram pass) packs, once a position (< n) and the key
// bits not yet sorted fit 64 bits, both into one word for its middle passes;
// its last pass writes (key, position) pairs again: Morton keys recomputed from
// the point, Hilbert keys gathered from the written ones.
// Equal keys (duplicate points) are then put in id order by k_tie_runs /
// k_tie_long (a later canonical leaf layout depends on it).
#include "common.cuh"
#include <cuda.h>
#include <cmath>
#include <mutex>
#include <type_traits>

#include "bitonic.cuh"
#include "keys.cuh"

namespace psi {

namespace {

constexpr int ST = 256;        // threads per sort tile
constexpr int SI = 16;         // keys per thread
constexpr int TILE = ST * SI;  // 4096 keys per tile
constexpr int SW = ST / 32;
constexpr int MAX_PASSES = 8;  // 64-bit keys at 8-bit digits

constexpr uint32_t LB_AGG = 1u << 30, LB_PRE = 2u << 30, LB_VAL = (1u << 30) - 1;
constexpr int LB_W = 8;  // predecessor tiles read per look-back step
constexpr int HIST_U = 4;  // items per thread per round of the histogram pass

// An event destroyed with its scope.
struct EventGuard {
  cudaEvent_t e = nullptr;
  ~EventGuard() {
    if (e) cudaEventDestroy(e);
  }
};
constexpr int64_t kPackMin = int64_t(1) << 22;  // smallest encoding sort that may pack
constexpr int kPrefixBits = 48;                   // key bits sorted by a prefix sort
constexpr int kPrefixShort = 8;                   // longest run fixed in registers
constexpr double kPrefixMaxRun = 1.15;            // largest mean run of equal top bits for a prefix sort
constexpr int64_t kPrefixMin = int64_t(1) << 20;  // smallest encoding sort that may sort a prefix only

// Digit width RB in {8, 10, 11}: RADIX digits, DPT digits per thread in the
// tile epilogue; per-warp counters fit 16 bits (a warp ranks 512 keys).
template <int RB>
struct Radix {
  static constexpr int RADIX = 1 << RB;
  static constexpr int DPT = RADIX / ST;
  static constexpr int HIST_PARTS = RB == 8 ? 4 : 1;
  using Count = typename std::conditional<RB == 8, uint32_t, uint16_t>::type;
  using Digit = typename std::conditional<RB == 8, uint8_t, uint16_t>::type;
};

template <int RB>
struct OnesweepSmem {
  using R = Radix<RB>;
  typename R::Count wh[SW][R::RADIX];  // per-warp digit counters, then warp offsets
  uint32_t off[R::RADIX];              // tile-exclusive digit offsets
  uint32_t glob[R::RADIX];             // global position minus tile-local position
  uint32_t gb[R::RADIX];               // global exclusive digit offsets of this pass
  uint32_t nh[R::RADIX];               // next pass's digit counts of this tile
  alignas(16) uint64_t stage[TILE];    // keys (then values) in digit order
  typename R::Digit dig[TILE];         // digit of each staged position
  uint32_t wsum[SW];
  alignas(16) uint8_t htab[kCurveTabBytes];
  uint32_t tile;
};

struct PassArgs {
  const uint64_t *kin;
  const uint32_t *vin;
  uint64_t *kout;
  uint32_t *vout;
  const int32_t *pts;
  int bits;
  int key_shift;
  int64_t n;
  int shift;
  const uint32_t *gbase;  // [RADIX] global exclusive digit offsets of this pass, or null:
  const uint32_t *hist_cur;  //   then this pass's digit counts, scanned by every tile
  uint32_t *hist_next;       // next pass's digit counts (accumulated here), or null
  int shift_next;
  uint32_t *lookback;     // [tiles][RADIX] of this pass, zero on entry
  uint32_t *lookback_next;  // table of the next pass: this pass zeroes it (or null)
  uint32_t *tile_ctr;
  int *status;
  // Packed words (IO_PACK .. IO_UNPACK below): value << kr | key >> drop.
  const uint64_t *kfull = nullptr;  // keys in input order (IO_UNPACK gathers them), or null
  uint64_t kmask = ~0ull;  // (1 << kr) - 1: the key bits of a packed word
  int kr = 0;
  int drop = 0;
  // Bounded look-back wait: polls of a predecessor's word before giving up
  // with ST_TIMEOUT.  withheld_tile >= 0 (a test of that path only): this
  // tile never publishes its words, so its successors' waits run out.
  uint32_t spin_limit = kSpinLimit;
  int64_t withheld_tile = -1;
};

// What a digit pass reads and writes.  An encoding sort whose positions
// (values < n) and not yet sorted key bits fit one 64-bit word packs them
// together for its middle passes, which then move 8 instead of 12 bytes per
// pair; its last pass recomputes the full key from the point at the position.
enum : int {
  IO_PAIRS = 0,   // (key, value) in, (key, value) out
  IO_PACK = 1,    // (key, value) in, packed word out
  IO_KEYS = 2,    // packed word in and out
  IO_UNPACK = 3,  // packed word in, (key from the point, value) out
};

// Optional extras of the histogram pass: the histogram of an alternative
// first digit ((key >> alt_shift) & mask, into hist_alt) and a HyperLogLog
// sketch of the distinct values of key >> alt_shift (kHllRegs registers, into
// hll), from which the host estimates how many keys share their top bits.
// The sketch takes the first item of each thread's round (a quarter of the
// keys, hll_sampled of them): the decision it feeds needs the ratio of keys
// to distinct top bits only roughly.
constexpr int kHllBits = 12, kHllRegs = 1 << kHllBits;
static int64_t hll_sampled(int64_t n) {
  const int64_t round = 256 * HIST_U;  // items of one block round (256 threads)
  return (n / round) * 256 + std::min<int64_t>(n % round, 256);
}
struct HistExtra {
  uint32_t *hist_alt = nullptr;
  int alt_shift = 0;
  uint32_t *hll = nullptr;
};

// SplitMix64's finaliser (Steele, Lea, Flood 2014) as the sketch's hash.
__device__ __forceinline__ uint64_t hll_hash(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Digit histograms of all passes in one read; when encoding with kst set, the
// keys are also written out (in input order) for the digit passes to read.  With 8-bit digits the counts go
// to 4 shared copies (lane % 4 picks one) so that lanes of a warp hitting the
// same digit -- common for the top digits of clustered input -- rarely collide.
template <int MODE, int D, int CURVE, int RB>
__global__ __launch_bounds__(256) void k_sort_hist(const uint64_t *kin, const int32_t *pts, int bits, int key_shift,
                                                   int64_t n, int passes, uint32_t *hist, int *status,
                                                   uint64_t *kst, unsigned long long *near, int near_shift,
                                                   HistExtra ex) {
  using R = Radix<RB>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // one counter section per counted digit: the passes' digits, then the
  // alternative first digit (ex.hist_alt)
  const int secs = passes + (ex.hist_alt ? 1 : 0);
  uint32_t *shp = reinterpret_cast<uint32_t *>(smem_raw);  // [HIST_PARTS][secs][RADIX]
  uint8_t *htab = smem_raw + sizeof(uint32_t) * R::HIST_PARTS * (passes + 1) * R::RADIX;
  // Hilbert keys with larger tables than point_key's: 2D five levels per step
  // (8 KB), 3D two levels per step (13.5 KB)
  constexpr bool H5 = MODE == 1 && D == 2 && CURVE == 1;
  constexpr bool H3 = MODE == 1 && D == 3 && CURVE == 1;
  constexpr int TAB = H5 ? kHilbert5TabBytes : H3 ? kHilbert3x2TabBytes : kCurveTabBytes;
  uint32_t *shll = reinterpret_cast<uint32_t *>(htab + TAB);  // [kHllRegs] when ex.hll
  for (int i = threadIdx.x; i < R::HIST_PARTS * secs * R::RADIX; i += blockDim.x) shp[i] = 0;
  if (ex.hll)
    for (int i = threadIdx.x; i < kHllRegs; i += blockDim.x) shll[i] = 0;
  if (H5)
    hilbert5_table_init(htab);
  else if (H3)
    hilbert3x2_table_init(htab);
  else if (MODE == 1)
    curve_table_init<D, CURVE>(htab);
  __syncthreads();
  bool bad_any = false;
  uint32_t n_near = 0;  // input neighbours (i, i + 1) whose keys agree above near_shift
  uint32_t *mine = shp + (threadIdx.x % R::HIST_PARTS) * secs * R::RADIX;
  // HIST_U items per thread per round, their loads issued together
  const int64_t chunk = (int64_t)blockDim.x * HIST_U;
  const int64_t stride = (int64_t)gridDim.x * chunk;
  for (int64_t i0 = (int64_t)blockIdx.x * chunk; i0 < n; i0 += stride) {
    uint64_t k[HIST_U];
    bool ok[HIST_U];
    if (MODE == 0) {
#pragma unroll
      for (int u = 0; u < HIST_U; ++u) {
        const int64_t i = i0 + (int64_t)u * blockDim.x + threadIdx.x;
        ok[u] = i < n;
        k[u] = ok[u] ? kin[i] : 0ull;
      }
    } else {
      int32_t c[HIST_U][D];
#pragma unroll
      for (int u = 0; u < HIST_U; ++u) {
        const int64_t i = i0 + (int64_t)u * blockDim.x + threadIdx.x;
        ok[u] = i < n;
#pragma unroll
        for (int d = 0; d < D; ++d) c[u][d] = ok[u] ? pts[i * D + d] : 0;
      }
#pragma unroll
      for (int u = 0; u < HIST_U; ++u) {
        bool bad;
        if constexpr (H5) {
          const uint32_t lim = 1u << bits;  // bits <= 31
          bad = (uint32_t)c[u][0] >= lim || (uint32_t)c[u][D - 1] >= lim;
          k[u] = hilbert2_key5(htab, (uint32_t)c[u][0], (uint32_t)c[u][D - 1], bits) >> key_shift;
        } else if constexpr (H3) {
          const uint32_t lim = 1u << bits;
          bad = (uint32_t)c[u][0] >= lim || (uint32_t)c[u][1] >= lim || (uint32_t)c[u][D - 1] >= lim;
          k[u] = hilbert3_key2(htab, (uint32_t)c[u][0], (uint32_t)c[u][1], (uint32_t)c[u][D - 1], bits) >> key_shift;
        } else {
          k[u] = point_key<D, CURVE>(htab, c[u], bits, bad) >> key_shift;
        }
        if (ok[u]) {
          bad_any |= bad;
          if (kst) kst[i0 + (int64_t)u * blockDim.x + threadIdx.x] = k[u];
        }
      }
    }
    if (near) {
#pragma unroll
      for (int u = 0; u < HIST_U; ++u) {
        const uint64_t kn = __shfl_down_sync(0xFFFFFFFFu, k[u], 1);
        const bool okn = __shfl_down_sync(0xFFFFFFFFu, ok[u], 1);
        n_near += (threadIdx.x & 31) < 31 && ok[u] && okn && ((k[u] ^ kn) >> near_shift) == 0;
      }
    }
    if (ex.hll && ok[0]) {
      const uint64_t h = hll_hash(k[0] >> ex.alt_shift);
      // register: the top kHllBits of the hash; value: 1 + leading zeros of the rest
      const uint32_t rho = (uint32_t)__clzll((long long)((h << kHllBits) | (1ull << (kHllBits - 1)))) + 1u;
      atomicMax(&shll[h >> (64 - kHllBits)], rho);
    }
#pragma unroll
    for (int u = 0; u < HIST_U; ++u) {
      const uint32_t act = __ballot_sync(0xFFFFFFFFu, ok[u]);
      if (ok[u]) {
        for (int p = 0; p < secs; ++p) {
          const int sh = p < passes ? p * RB : ex.alt_shift;
          uint32_t dg = (uint32_t)(k[u] >> sh) & (R::RADIX - 1);
          int all_same;
          __match_all_sync(act, dg, &all_same);
          if (all_same) {
            if ((lanemask_lt() & act) == 0) atomicAdd(&shp[p * R::RADIX + dg], (uint32_t)__popc(act));
          } else {
            atomicAdd(&mine[p * R::RADIX + dg], 1u);
          }
        }
      }
    }
  }
  if (bad_any) atomicOr(status, ST_RANGE);
  if (near) block_count_add(near, n_near);
  __syncthreads();
  if (ex.hll)
    for (int i = threadIdx.x; i < kHllRegs; i += blockDim.x)
      if (shll[i]) atomicMax(&ex.hll[i], shll[i]);
  for (int i = threadIdx.x; i < secs * R::RADIX; i += blockDim.x) {
    uint32_t v = 0;
#pragma unroll
    for (int q = 0; q < R::HIST_PARTS; ++q) v += shp[q * secs * R::RADIX + i];
    if (v) atomicAdd(i < passes * R::RADIX ? &hist[i] : &ex.hist_alt[i - passes * R::RADIX], v);
  }
}

// One block per pass: exclusive scan of the pass's digit counts (RADIX / blockDim per thread).
template <int RB>
__global__ void k_hist_scan(const uint32_t *hist, uint32_t *gbase) {
  constexpr int RADIX = 1 << RB;
  __shared__ uint32_t wsum[32];
  const int p = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int per = RADIX / blockDim.x;
  uint32_t c[8], tot = 0;
  for (int q = 0; q < per; ++q) {
    c[q] = hist[p * RADIX + t * per + q];
    tot += c[q];
  }
  uint32_t x = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  uint32_t before = 0;
  for (int i = 0; i < w; ++i) before += wsum[i];
  uint32_t run = before + x - tot;
  for (int q = 0; q < per; ++q) {
    gbase[p * RADIX + t * per + q] = run;
    run += c[q];
  }
}

// MODE 0: keys and values read; 1: keys computed from the points, values =
// positions; 2: keys read, values = positions.
template <int MODE, int D, int CURVE, int RB, int IO = IO_PAIRS>
__global__ __launch_bounds__(ST, RB == 11 ? 2 : 3) void k_onesweep(PassArgs a) {
  using R = Radix<RB>;
  constexpr int RADIX = R::RADIX, DPT = R::DPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  OnesweepSmem<RB> &sm = *reinterpret_cast<OnesweepSmem<RB> *>(smem_raw);

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) sm.tile = atomicAdd(a.tile_ctr, 1u);
  {
    uint32_t *z = reinterpret_cast<uint32_t *>(&sm.wh[0][0]);
    for (int i = tid; i < (int)(sizeof(sm.wh) / 4); i += ST) z[i] = 0;
  }
  if (MODE == 1 || IO == IO_UNPACK) curve_table_init<D, CURVE>(sm.htab);
  if (a.hist_next)
    for (int i = tid; i < RADIX; i += ST) sm.nh[i] = 0;
  if (a.gbase) {
    for (int i = tid; i < RADIX; i += ST) sm.gb[i] = a.gbase[i];
  } else {  // exclusive scan of this pass's digit counts
    uint32_t c[DPT], tot = 0;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      c[q] = a.hist_cur[tid * DPT + q];
      tot += c[q];
    }
    uint32_t x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sm.wsum[w] = x;
    __syncthreads();
    uint32_t run = x - tot;
    for (int i = 0; i < w; ++i) run += sm.wsum[i];
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      sm.gb[tid * DPT + q] = run;
      run += c[q];
    }
  }
  __syncthreads();
  const uint32_t tile = sm.tile;
  const int64_t base = (int64_t)tile * TILE;
  const int tile_n = (int)min((int64_t)TILE, a.n - base);
  const int wbase = w * (SI * 32);

  // digit of a key (of the key bits of a packed word)
  auto digit = [&](uint64_t k, int sh) -> uint32_t {
    if (IO >= IO_KEYS) k &= a.kmask;
    return (uint32_t)(k >> sh) & (RADIX - 1);
  };
  if (MODE == 0 && IO <= IO_PACK) {  // the values are read after the keys are ranked: start them towards L2 now
    for (int i = tid * 32; i < tile_n; i += ST * 32)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a.vin + base + i));
  }
  if (a.lookback_next) {  // the next pass's look-back words of this tile start at zero
    for (int i = tid; i < RADIX; i += ST) a.lookback_next[(size_t)tile * RADIX + i] = 0;
  }
  uint64_t key[SI];
#pragma unroll
  for (int j = 0; j < SI; ++j) {
    const int li = wbase + j * 32 + lane;
    key[j] = ~0ull;
    if (li < tile_n) {
      const int64_t gi = base + li;
      if (MODE != 1) {
        key[j] = a.kin[gi];
      } else {
        int32_t c[D];
#pragma unroll
        for (int d = 0; d < D; ++d) c[d] = a.pts[gi * D + d];
        bool bad;
        key[j] = point_key<D, CURVE>(sm.htab, c, a.bits, bad) >> a.key_shift;
      }
    }
  }

  if (a.hist_next) {  // the next pass's digit of every key of the tile
#pragma unroll
    for (int j = 0; j < SI; ++j)
      if (wbase + j * 32 + lane < tile_n) atomicAdd(&sm.nh[digit(key[j], a.shift_next)], 1u);
  }
  // Stable rank of each key among equal digits of its warp (items in
  // (item, lane) order = input order).
  uint32_t rank[SI];
#pragma unroll
  for (int j = 0; j < SI; ++j) {
    const int li = wbase + j * 32 + lane;
    const bool valid = li < tile_n;
    const uint32_t dg = valid ? digit(key[j], a.shift) : 0xFFFFFFFFu;
    // lanes holding the same digit, from one ballot per digit bit
    uint32_t peers = __ballot_sync(0xFFFFFFFFu, valid);
#pragma unroll
    for (int b = 0; b < RB; ++b) {
      const uint32_t m = __ballot_sync(0xFFFFFFFFu, (dg >> b) & 1u);
      peers &= ((dg >> b) & 1u) ? m : ~m;
    }
    // the lowest lane of each group reads and advances the warp's counter;
    // the shuffle hands the old count to the group (and orders the warp)
    const uint32_t before = __popc(peers & lanemask_lt());
    uint32_t wb = 0;
    if (valid && before == 0) {
      wb = sm.wh[w][dg];
      sm.wh[w][dg] = (typename R::Count)(wb + __popc(peers));
    }
    wb = __shfl_sync(0xFFFFFFFFu, wb, valid ? __ffs(peers) - 1 : lane);
    rank[j] = wb + before;
  }
  __syncthreads();

  // Epilogue: thread t owns digits [t*DPT, (t+1)*DPT): per-warp offsets, tile
  // totals, look-back publication, tile-local and global offsets.
  {
    uint32_t cnt[DPT], tsum = 0;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      const int d = tid * DPT + q;
      uint32_t run = 0;
#pragma unroll
      for (int ww = 0; ww < SW; ++ww) {
        const uint32_t c = sm.wh[ww][d];
        sm.wh[ww][d] = (typename R::Count)run;
        run += c;
      }
      cnt[q] = run;
      tsum += run;
      if ((int64_t)tile != a.withheld_tile)
        st_relaxed_u32(a.lookback + (size_t)tile * RADIX + d, (tile == 0 ? LB_PRE : LB_AGG) | run);
    }
    uint32_t x = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sm.wsum[w] = x;
    __syncthreads();
    uint32_t excl = x - tsum;
    for (int i = 0; i < w; ++i) excl += sm.wsum[i];
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      const int d = tid * DPT + q;
      sm.off[d] = excl;
      // Look-back: read the words of up to LB_W predecessor tiles at once,
      // fold them newest first until a tile with its inclusive prefix; a tile
      // not published yet is re-read (bounded spin).
      uint32_t prev = 0;
      if (tile > 0) {
        int64_t t = (int64_t)tile - 1;
        uint32_t spins = 0;
        bool done = false;
        while (!done && t >= 0) {
          uint32_t v[LB_W];
#pragma unroll
          for (int u = 0; u < LB_W; ++u)
            v[u] = (t - u >= 0) ? ld_relaxed_u32(a.lookback + (size_t)(t - u) * RADIX + d) : LB_PRE;
          int u = 0;
          for (; u < LB_W && t - u >= 0; ++u) {
            if ((v[u] & (LB_AGG | LB_PRE)) == 0) break;
            prev += v[u] & LB_VAL;
            if (v[u] & LB_PRE) {
              done = true;
              break;
            }
          }
          if (done) break;
          if (u < LB_W && t - u >= 0) {
            t -= u;
            if (++spins > a.spin_limit) {
              atomicOr(a.status, ST_TIMEOUT);
              break;
            }
            if (spins > 64) __nanosleep(64);
          } else {
            t -= LB_W;
          }
        }
        if ((int64_t)tile != a.withheld_tile)
          st_relaxed_u32(a.lookback + (size_t)tile * RADIX + d, LB_PRE | ((prev + cnt[q]) & LB_VAL));
      }
      sm.glob[d] = sm.gb[d] + prev - excl;
      excl += cnt[q];
    }
  }
  __syncthreads();

  // Stage keys (packed words) at their tile-local positions, then write each
  // digit's run out.
#pragma unroll
  for (int j = 0; j < SI; ++j) {
    const int li = wbase + j * 32 + lane;
    if (li < tile_n) {
      const uint32_t dg = digit(key[j], a.shift);
      const uint32_t lp = sm.off[dg] + sm.wh[w][dg] + rank[j];
      sm.stage[lp] = IO == IO_PACK ? key[j] >> a.drop : key[j];
      if (IO == IO_PACK) sm.dig[lp] = (typename R::Digit)dg;
      rank[j] = lp;
    }
  }
  if (IO == IO_PACK) {  // each pair's value joins its word (a position this thread staged)
#pragma unroll
    for (int j = 0; j < SI; ++j) {
      const int li = wbase + j * 32 + lane;
      if (li < tile_n) sm.stage[rank[j]] |= (uint64_t)(MODE != 0 ? (uint32_t)(base + li) : a.vin[base + li]) << a.kr;
    }
  }
  __syncthreads();
  if (IO == IO_UNPACK && a.kfull) {
    // the stored key of every position is requested before the first is written
    uint64_t kf[SI];
#pragma unroll
    for (int i = 0; i < SI; ++i) {
      const int p = tid + i * ST;
      if (p < tile_n) kf[i] = a.kfull[sm.stage[p] >> a.kr];
    }
#pragma unroll
    for (int i = 0; i < SI; ++i) {
      const int p = tid + i * ST;
      if (p < tile_n) {
        const uint64_t wd = sm.stage[p];
        const uint64_t o = (uint64_t)sm.glob[digit(wd, a.shift)] + p;
        a.kout[o] = kf[i];
        a.vout[o] = (uint32_t)(wd >> a.kr);
      }
    }
  } else if (IO == IO_UNPACK) {
    // the points of half the positions are requested before their keys are computed
#pragma unroll
    for (int h = 0; h < SI; h += SI / 2) {
      int32_t c[SI / 2][D];
#pragma unroll
      for (int i = 0; i < SI / 2; ++i) {
        const int p = tid + (h + i) * ST;
        if (p < tile_n) {
          const int64_t v = (int64_t)(sm.stage[p] >> a.kr);
#pragma unroll
          for (int d = 0; d < D; ++d) c[i][d] = a.pts[v * D + d];
        }
      }
#pragma unroll
      for (int i = 0; i < SI / 2; ++i) {
        const int p = tid + (h + i) * ST;
        if (p < tile_n) {
          const uint64_t wd = sm.stage[p];
          const uint64_t o = (uint64_t)sm.glob[digit(wd, a.shift)] + p;
          bool bad;
          a.kout[o] = point_key<D, CURVE>(sm.htab, c[i], a.bits, bad) >> a.key_shift;
          a.vout[o] = (uint32_t)(wd >> a.kr);
        }
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < SI; ++i) {
      const int p = tid + i * ST;
      if (p < tile_n) {
        const uint64_t k = sm.stage[p];
        const uint32_t dg = IO == IO_PACK ? (uint32_t)sm.dig[p] : digit(k, a.shift);
        if (IO == IO_PAIRS) sm.dig[p] = (typename R::Digit)dg;
        a.kout[sm.glob[dg] + p] = k;
      }
    }
  }
  if (IO == IO_PAIRS) {
    __syncthreads();
    uint32_t *s_v = reinterpret_cast<uint32_t *>(sm.stage);
#pragma unroll
    for (int j = 0; j < SI; ++j) {
      const int li = wbase + j * 32 + lane;
      if (li < tile_n) s_v[rank[j]] = MODE != 0 ? (uint32_t)(base + li) : a.vin[base + li];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SI; ++i) {
      const int p = tid + i * ST;
      if (p < tile_n) a.vout[sm.glob[sm.dig[p]] + p] = s_v[p];
    }
  }
  if (a.hist_next)
    for (int i = tid; i < RADIX; i += ST)
      if (sm.nh[i]) atomicAdd(&a.hist_next[i], sm.nh[i]);
}

// ---- Ties: runs of equal keys ordered by id ------------------------------

constexpr int kShortRun = 32;

__global__ void k_tie_runs(const uint64_t *keys, uint32_t *vals, const uint32_t *ids, int64_t n, int64_t *long_runs,
                           uint32_t *n_long, int64_t cap_long) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i + 1 >= n) return;
  const uint64_t k = keys[i];
  if (keys[i + 1] != k || (i > 0 && keys[i - 1] == k)) return;
  int64_t e = i + 2;
  while (e < n && keys[e] == k && e - i <= kShortRun) ++e;
  const int len = (int)(e - i);
  if (len > kShortRun) {
    const uint32_t slot = atomicAdd(n_long, 1u);
    if (slot < cap_long) long_runs[slot] = i;
    return;
  }
  uint32_t v[kShortRun], id[kShortRun];
  for (int j = 0; j < len; ++j) {
    v[j] = vals[i + j];
    id[j] = ids[v[j]];
  }
  for (int j = 1; j < len; ++j) {
    const uint32_t cv = v[j], ci = id[j];
    int t = j - 1;
    while (t >= 0 && id[t] > ci) {
      v[t + 1] = v[t];
      id[t + 1] = id[t];
      --t;
    }
    v[t + 1] = cv;
    id[t + 1] = ci;
  }
  for (int j = 0; j < len; ++j) vals[i + j] = v[j];
}

// One block per long run: sort of the run's values by id (ids are unique, so
// no stability is needed).  Runs up to 4096 sort in shared memory; longer ones
// (pathological piles of duplicate points) sort in place in global memory.
constexpr int kSmemRun = 4096;

__global__ __launch_bounds__(1024) void k_tie_long(const uint64_t *keys, uint32_t *vals, const uint32_t *ids,
                                                   int64_t n, const int64_t *long_runs, const uint32_t *n_long,
                                                   int64_t cap_long) {
  __shared__ uint32_t sv[kSmemRun], si[kSmemRun];
  const int64_t runs = min((int64_t)*n_long, cap_long);
  for (int64_t r = blockIdx.x; r < runs; r += gridDim.x) {
    const int64_t s = long_runs[r];
    const uint64_t k = keys[s];
    int64_t lo = s, hi = n;  // first index past the run
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo) / 2;
      if (keys[mid] == k)
        lo = mid + 1;
      else
        hi = mid;
    }
    const int64_t len = lo - s;
    if (len <= kSmemRun) {
      for (int64_t j = threadIdx.x; j < len; j += blockDim.x) {
        sv[j] = vals[s + j];
        si[j] = ids[sv[j]];
      }
      __syncthreads();
      bitonic_ascending(
          len, [&](int64_t a, int64_t b) { return si[a] < si[b]; },
          [&](int64_t a, int64_t b) {
            uint32_t x = si[a];
            si[a] = si[b];
            si[b] = x;
            x = sv[a];
            sv[a] = sv[b];
            sv[b] = x;
          });
      for (int64_t j = threadIdx.x; j < len; j += blockDim.x) vals[s + j] = sv[j];
      __syncthreads();
    } else {
      uint32_t *v = vals + s;
      bitonic_ascending(
          len, [&](int64_t a, int64_t b) { return ids[v[a]] < ids[v[b]]; },
          [&](int64_t a, int64_t b) {
            const uint32_t x = v[a];
            v[a] = v[b];
            v[b] = x;
          });
    }
  }
}

// ---- Runs of a sort on the top key bits only ----------------------------
// A sort on key bits [low, key_bits) leaves each run of keys equal in those
// bits in input order; the run is then put in (key, id) order.  A run of up to
// kPrefixShort is sorted by one thread with a register sorting network (ids
// are read only to order equal keys); longer runs are listed for
// k_prefix_long.

__device__ __forceinline__ bool key_id_less(uint64_t ka, uint32_t va, uint64_t kb, uint32_t vb, const uint32_t *ids) {
  return ka < kb || (ka == kb && ids[va] < ids[vb]);
}

// Compare-exchange of two (key, value) slots of a register sorting network by
// (key, id): ids are read only when the keys are equal (duplicate points).
__device__ __forceinline__ void prefix_cx(uint64_t &ka, uint32_t &va, uint64_t &kb, uint32_t &vb,
                                          const uint32_t *ids) {
  if (key_id_less(kb, vb, ka, va, ids)) {
    const uint64_t k = ka;
    ka = kb;
    kb = k;
    const uint32_t v = va;
    va = vb;
    vb = v;
  }
}

// Odd-even transposition network over the first `rounds` slots (rounds =
// the run's length, at most N): sorts them by (key, id).
template <int N>
__device__ __forceinline__ void prefix_network(uint64_t (&k)[kPrefixShort], uint32_t (&v)[kPrefixShort], int len,
                                               const uint32_t *ids) {
#pragma unroll
  for (int r = 0; r < N; ++r)
#pragma unroll
    for (int j = r & 1; j + 1 < N; j += 2)
      if (j + 1 < len) prefix_cx(k[j], v[j], k[j + 1], v[j + 1], ids);
}

// kPrefixU elements per thread (a block takes kPrefixU * blockDim consecutive
// elements, coalesced): the keys of all of a thread's elements and their
// neighbours are requested before any is compared, so that many loads are in
// flight; a thread whose element starts a run (rare: most elements differ from
// both neighbours in their top bits) reads the rest of it and sorts it in
// registers with a network sized to the run.
constexpr int kPrefixU = 4;

// Run starts of a prefix sort's output: positions i whose top bits (key >>
// low) equal those of i + 1 but not those of i - 1, listed in no particular
// order in starts[0, *n_starts) (kPrefixU consecutive elements per thread;
// a block appends the starts of a round with one atomic, its warps' offsets
// from a scan in shared memory).  A count above cap means the list
// is incomplete and k_prefix_runs scans every position.
__global__ __launch_bounds__(256) void k_prefix_starts(const uint64_t *keys, int64_t n, int low, int32_t *starts,
                                                       unsigned long long *n_starts, int64_t cap) {
  __shared__ uint32_t wcount[8];
  __shared__ unsigned long long bbase;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t chunk = (int64_t)blockDim.x * kPrefixU;
  for (int64_t b0 = (int64_t)blockIdx.x * chunk; b0 < n; b0 += (int64_t)gridDim.x * chunk) {
    // kPrefixU consecutive keys per thread (two 16-byte loads) and one
    // neighbour on each side
    const int64_t i0 = b0 + (int64_t)threadIdx.x * kPrefixU;
    uint64_t kc[kPrefixU + 2];
    if ((reinterpret_cast<uintptr_t>(keys) & 15) == 0 && i0 + kPrefixU <= n) {
      const ulonglong2 *v = reinterpret_cast<const ulonglong2 *>(keys + i0);
      const ulonglong2 a = v[0], b = v[1];
      kc[1] = a.x;
      kc[2] = a.y;
      kc[3] = b.x;
      kc[4] = b.y;
    } else {
#pragma unroll
      for (int u = 0; u < kPrefixU; ++u) kc[u + 1] = i0 + u < n ? keys[i0 + u] : ~0ull;
    }
    kc[0] = i0 > 0 && i0 < n ? keys[i0 - 1] : ~0ull;
    kc[kPrefixU + 1] = i0 + kPrefixU < n ? keys[i0 + kPrefixU] : ~0ull;
    uint32_t bal[kPrefixU];
    bool st[kPrefixU];
    uint32_t wtot = 0;
#pragma unroll
    for (int u = 0; u < kPrefixU; ++u) {
      const int64_t i = i0 + u;
      const uint64_t p = kc[u + 1] >> low;
      const bool with_prev = i > 0 && i < n && (kc[u] >> low) == p;
      const bool with_next = i + 1 < n && (kc[u + 2] >> low) == p;
      st[u] = with_next && !with_prev;
      bal[u] = __ballot_sync(0xFFFFFFFFu, st[u]);
      wtot += __popc(bal[u]);
    }
    if (lane == 0) wcount[w] = wtot;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t t = 0;
      for (int j = 0; j < (int)(blockDim.x >> 5); ++j) t += wcount[j];
      bbase = t ? atomicAdd(n_starts, (unsigned long long)t) : 0ull;
    }
    __syncthreads();
    unsigned long long off = bbase;
    for (int j = 0; j < w; ++j) off += wcount[j];
#pragma unroll
    for (int u = 0; u < kPrefixU; ++u) {
      if (st[u]) {
        const unsigned long long pos = off + __popc(bal[u] & lanemask_lt());
        if (pos < (unsigned long long)cap) starts[pos] = (int32_t)(i0 + u);
      }
      off += __popc(bal[u]);
    }
    __syncthreads();
  }
}

// The run of equal top bits starting at position i (a run start): runs of up
// to kPrefixShort elements are sorted by (key, id) in registers by a network
// sized to the run; longer ones are listed for k_prefix_long.
__device__ __forceinline__ void prefix_fix_run(uint64_t *keys, uint32_t *vals, const uint32_t *ids, int64_t n,
                                               int low, int64_t i, int64_t *long_runs, uint32_t *n_long,
                                               int64_t cap_long) {
  const uint64_t p = keys[i] >> low;
  uint64_t k[kPrefixShort];
  uint32_t v[kPrefixShort];
  int len = 0;
#pragma unroll
  for (int j = 0; j < kPrefixShort; ++j) {
    k[j] = ~0ull;  // past the run: above every key, never moved before a member
    v[j] = 0;
    if (len == j && i + j < n) {
      const uint64_t kj = keys[i + j];
      if ((kj >> low) == p) {
        k[j] = kj;
        v[j] = vals[i + j];
        ++len;
      }
    }
  }
  if (len == kPrefixShort && i + kPrefixShort < n && (keys[i + kPrefixShort] >> low) == p) {
    const uint32_t slot = atomicAdd(n_long, 1u);
    if (slot < cap_long) long_runs[slot] = i;
    return;
  }
  if (len == 2)
    prefix_network<2>(k, v, len, ids);
  else if (len <= 4)
    prefix_network<4>(k, v, len, ids);
  else
    prefix_network<kPrefixShort>(k, v, len, ids);
#pragma unroll
  for (int j = 0; j < kPrefixShort; ++j)
    if (j < len) {
      keys[i + j] = k[j];
      vals[i + j] = v[j];
    }
}

// A thread per listed run start (or, when the list overflowed, per position,
// taking those that start a run).
__global__ __launch_bounds__(256) void k_prefix_runs(uint64_t *keys, uint32_t *vals, const uint32_t *ids, int64_t n,
                                                     int low, const int32_t *starts,
                                                     const unsigned long long *n_starts, int64_t cap,
                                                     int64_t *long_runs, uint32_t *n_long, int64_t cap_long) {
  const unsigned long long ns = *n_starts;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (ns <= (unsigned long long)cap) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < (int64_t)ns; r += stride)
      prefix_fix_run(keys, vals, ids, n, low, starts[r], long_runs, n_long, cap_long);
    return;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t p = keys[i] >> low;
    if (i + 1 < n && (keys[i + 1] >> low) == p && !(i > 0 && (keys[i - 1] >> low) == p))
      prefix_fix_run(keys, vals, ids, n, low, i, long_runs, n_long, cap_long);
  }
}

// One block per long run: bitonic sort by (key, id) (ids are unique, so no
// stability is needed).  Runs up to kSmemRun sort in shared memory, longer
// ones in place in global memory.
__global__ __launch_bounds__(1024) void k_prefix_long(uint64_t *keys, uint32_t *vals, const uint32_t *ids, int64_t n,
                                                      int low, const int64_t *long_runs, const uint32_t *n_long,
                                                      int64_t cap_long) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t *sk = reinterpret_cast<uint64_t *>(smem_raw);
  uint32_t *sv = reinterpret_cast<uint32_t *>(sk + kSmemRun);
  uint32_t *si = sv + kSmemRun;
  const int64_t runs = min((int64_t)*n_long, cap_long);
  for (int64_t r = blockIdx.x; r < runs; r += gridDim.x) {
    const int64_t s = long_runs[r];
    const uint64_t p = keys[s] >> low;
    int64_t lo = s, hi = n;  // first index past the run
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo) / 2;
      if ((keys[mid] >> low) == p)
        lo = mid + 1;
      else
        hi = mid;
    }
    const int64_t len = lo - s;
    if (len <= kSmemRun) {
      for (int64_t j = threadIdx.x; j < len; j += blockDim.x) {
        sk[j] = keys[s + j];
        sv[j] = vals[s + j];
        si[j] = ids[sv[j]];
      }
      __syncthreads();
      bitonic_ascending(
          len, [&](int64_t a, int64_t b) { return sk[a] < sk[b] || (sk[a] == sk[b] && si[a] < si[b]); },
          [&](int64_t a, int64_t b) {
            const uint64_t x = sk[a];
            sk[a] = sk[b];
            sk[b] = x;
            uint32_t y = sv[a];
            sv[a] = sv[b];
            sv[b] = y;
            y = si[a];
            si[a] = si[b];
            si[b] = y;
          });
      for (int64_t j = threadIdx.x; j < len; j += blockDim.x) {
        keys[s + j] = sk[j];
        vals[s + j] = sv[j];
      }
      __syncthreads();
    } else {
      uint64_t *kk = keys + s;
      uint32_t *vv = vals + s;
      bitonic_ascending(
          len, [&](int64_t a, int64_t b) { return key_id_less(kk[a], vv[a], kk[b], vv[b], ids); },
          [&](int64_t a, int64_t b) {
            const uint64_t x = kk[a];
            kk[a] = kk[b];
            kk[b] = x;
            const uint32_t y = vv[a];
            vv[a] = vv[b];
            vv[b] = y;
          });
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------

template <int MODE, int D, int CURVE, int RB>
static psi_status launch_hist(const uint64_t *kin, const EncodeSpec &enc, int64_t n, int passes, uint32_t *hist,
                              int *status, cudaStream_t s, uint64_t *kst = nullptr,
                              unsigned long long *near = nullptr, int near_shift = 0, HistExtra ex = HistExtra()) {
  using R = Radix<RB>;
  auto kern = k_sort_hist<MODE, D, CURVE, RB>;
  const size_t smem = sizeof(uint32_t) * R::HIST_PARTS * (passes + 1) * R::RADIX +
                      (MODE == 1 && CURVE == 1 ? (D == 2 ? kHilbert5TabBytes : kHilbert3x2TabBytes)
                                               : kCurveTabBytes) +
                      (ex.hll ? sizeof(uint32_t) * kHllRegs : 0);
  if (smem > 48 * 1024) PSI_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // all blocks resident at once (the grid-stride rounds stay balanced)
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem) != cudaSuccess) per_sm = 0;
  const int grid = (int)std::min<int64_t>(ceil_div(n, 256 * HIST_U), (int64_t)num_sms() * std::max(per_sm, 1));
  PSI_LAUNCH_NAMED("k_sort_hist", kern, std::max(grid, 1), 256, smem, s, kin, enc.pts, enc.bits, enc.key_shift, n,
                   passes, hist, status, kst, near, near_shift, ex);
  return PSI_OK;
}

template <int MODE, int D, int CURVE, int RB, int IO = IO_PAIRS>
static psi_status launch_pass(const PassArgs &a, int64_t tiles, cudaStream_t s) {
  auto kern = k_onesweep<MODE, D, CURVE, RB, IO>;
  const size_t smem = sizeof(OnesweepSmem<RB>);
  if (smem > 48 * 1024) PSI_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  PSI_LAUNCH_NAMED("k_onesweep", kern, (unsigned)tiles, ST, smem, s, a);
  return PSI_OK;
}

// The passes of a packed sort (8-bit digits only).
template <int RB>
static psi_status launch_packed(const EncodeSpec &enc, const PassArgs &a, int64_t tiles, int io, cudaStream_t s) {
  if constexpr (RB == 8) {
    if (io == IO_PACK) return launch_pass<0, 2, 0, RB, IO_PACK>(a, tiles, s);
    if (io == IO_KEYS) return launch_pass<0, 2, 0, RB, IO_KEYS>(a, tiles, s);
    // the last pass: Morton keys are recomputed; stored (Hilbert) keys gathered
    if (a.kfull || enc.dim == 2) return launch_pass<0, 2, 0, RB, IO_UNPACK>(a, tiles, s);
    return launch_pass<0, 3, 0, RB, IO_UNPACK>(a, tiles, s);
  }
  set_error("sort: packed passes need 8-bit digits");
  return PSI_ERR_INVALID;
}

// HyperLogLog estimate of the number of distinct values sketched in M
// (Flajolet, Fusy, Gandouet, Meunier 2007), with linear counting for small
// cardinalities.
static double hll_estimate(const uint32_t *M) {
  const double m = kHllRegs;
  double z = 0.0;
  int zeros = 0;
  for (int j = 0; j < kHllRegs; ++j) {
    z += std::ldexp(1.0, -(int)M[j]);
    zeros += M[j] == 0;
  }
  double e = 0.7213 / (1.0 + 1.079 / m) * m * m / z;
  if (e <= 2.5 * m && zeros > 0) e = m * std::log(m / zeros);
  return e;
}

// Digit width: 8 unless 10 or 11 is asked for.  Wider digits save passes but
// measured slower per pass on GB300 with 4096-key tiles (1e8 pairs: 0.92 ms
// at 8 bits, 1.67 ms at 10, 2.98 ms at 11): a tile's digit runs get too
// short for whole-sector writes and each thread walks several look-back chains.
static int pick_radix(int /*key_bits*/, int requested) {
  return (requested == 10 || requested == 11) ? requested : 8;
}

template <int RB>
static psi_status sort_pairs_rb(const EncodeSpec &enc, const uint64_t *keys_in, const uint32_t *vals_in, int64_t n,
                                int key_bits, uint64_t *kbuf0, uint32_t *vbuf0, uint64_t *kbuf1, uint32_t *vbuf1,
                                int *d_status, cudaStream_t s, SortResult *out, bool may_prefix) {
  using R = Radix<RB>;
  const bool encode = enc.pts != nullptr;
  const int passes_full = (key_bits + RB - 1) / RB;
  const int64_t tiles = ceil_div(n, TILE);
  // Decisions taken on the host from counts of the histogram pass are not
  // possible while the stream is being captured.
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();  // a refused query: take no host decision, leave no error behind
    cs = cudaStreamCaptureStatusActive;
  }
  const bool capturing = cs != cudaStreamCaptureStatusNone;
  // Prefix sort: an encoding sort whose equal keys are put in id order
  // afterwards anyway (may_prefix) sorts only the top kPrefixBits key bits
  // when the keys are unlikely to share them much: the histogram pass counts
  // input neighbours whose keys agree in those bits, and fewer than half
  // must.  Each run of equal top bits is then sorted by (key, id).
  const int low_c = key_bits - kPrefixBits;
  const bool pref_cand = may_prefix && encode && RB == 8 && n >= kPrefixMin && low_c > 0 &&
                         (key_bits - low_c + RB - 1) / RB < passes_full && !capturing;
  const bool pack_cand = encode && RB == 8 && n >= kPackMin && !capturing;
  Buf<uint32_t> hist, lookback, ctr;
  psi_status st;
  // digit counts: a section per pass, then the prefix sort's first digit;
  // two look-back tables used alternately: pass p clears the table of pass p+1
  if ((st = hist.alloc((size_t)(passes_full + 1) * R::RADIX, s)) ||
      (st = lookback.alloc((size_t)2 * tiles * R::RADIX, s)) || (st = ctr.alloc(passes_full, s)))
    return st;
  PSI_CK(cudaMemsetAsync(hist.p, 0, sizeof(uint32_t) * (passes_full + 1) * R::RADIX, s));
  PSI_CK(cudaMemsetAsync(lookback.p, 0, sizeof(uint32_t) * tiles * R::RADIX, s));
  PSI_CK(cudaMemsetAsync(ctr.p, 0, sizeof(uint32_t) * passes_full, s));

  // Hilbert keys cost more arithmetic than their 8-byte write and read: the
  // histogram pass computes them once and writes them out; the first digit
  // pass reads them (values = positions) and the last pass of a packed sort
  // gathers them.  Morton keys are recomputed from the points where needed.
  const bool stored = encode && enc.curve == CURVE_HILBERT;
  Buf<uint64_t> kst;
  if (stored && (st = kst.alloc(n, s))) return st;

  // Packed middle passes (8-bit digits, encoding sorts of at least kPackMin
  // pairs): pass pk writes value << kr | key >> drop once the value (a
  // position < n) and the key bits not yet sorted fit 64 bits; passes pk+1 ..
  // passes-2 move those words alone; the last pass writes the pairs again,
  // reading each key (or point) at its position.  Those reads are local only
  // when the input is: the histogram pass counts input neighbours whose keys
  // share their top 24 bits, and the sort packs when at least half do.
  // The count (and the prefix sort's sketch) reach the host through pinned
  // memory behind an event, read when the first decision needs them (the
  // prefix decision before pass 0; else the packing decision just before the
  // pack pass, the passes before it queued meanwhile).  The pinned buffer is
  // per host thread, allocated on its first such sort and kept for the
  // thread's lifetime.
  struct HostCounts {
    unsigned long long near;
    uint32_t hll[kHllRegs];
  };
  static thread_local HostCounts *h_cnt = nullptr;
  bool counts = pref_cand || pack_cand;
  if (counts && !h_cnt &&
      cudaHostAlloc((void **)&h_cnt, sizeof(HostCounts), cudaHostAllocPortable) != cudaSuccess) {
    cudaGetLastError();
    h_cnt = nullptr;
    counts = false;
  }
  Buf<unsigned long long> nearc;
  EventGuard near_ev;
  if (counts && cudaEventCreateWithFlags(&near_ev.e, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();  // e.g. another thread capturing in global mode: no host decisions
    near_ev.e = nullptr;
    counts = false;
  }
  Buf<uint32_t> hll;
  if (counts) {
    if ((st = nearc.alloc(1, s))) return st;
    PSI_CK(cudaMemsetAsync(nearc.p, 0, sizeof(unsigned long long), s));
  }
  const bool sketch = counts && pref_cand;
  if (sketch) {
    if ((st = hll.alloc(kHllRegs, s))) return st;
    PSI_CK(cudaMemsetAsync(hll.p, 0, sizeof(uint32_t) * kHllRegs, s));
  }
  const int near_shift = std::max(0, key_bits - 24);
  HistExtra ex;
  if (sketch) {
    ex.hist_alt = hist.p + (size_t)passes_full * R::RADIX;
    ex.alt_shift = low_c;
    ex.hll = hll.p;
  }
  unsigned long long *nearp = counts ? nearc.p : nullptr;

  // the first digit is counted up front; every pass counts the next digit of its keys
  if (!encode)
    st = launch_hist<0, 2, 0, RB>(keys_in, enc, n, 1, hist.p, d_status, s);
  else if (enc.dim == 2 && enc.curve == CURVE_MORTON)
    st = launch_hist<1, 2, 0, RB>(nullptr, enc, n, 1, hist.p, d_status, s, nullptr, nearp, near_shift, ex);
  else if (enc.dim == 2)
    st = launch_hist<1, 2, 1, RB>(nullptr, enc, n, 1, hist.p, d_status, s, kst.p, nearp, near_shift, ex);
  else if (enc.curve == CURVE_MORTON)
    st = launch_hist<1, 3, 0, RB>(nullptr, enc, n, 1, hist.p, d_status, s, nullptr, nearp, near_shift, ex);
  else
    st = launch_hist<1, 3, 1, RB>(nullptr, enc, n, 1, hist.p, d_status, s, kst.p, nearp, near_shift, ex);
  if (st) return st;
  bool synced = false;
  if (counts) {
    PSI_CK(cudaMemcpyAsync(&h_cnt->near, nearc.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    if (sketch) PSI_CK(cudaMemcpyAsync(h_cnt->hll, hll.p, sizeof(h_cnt->hll), cudaMemcpyDeviceToHost, s));
    PSI_CK(cudaEventRecord(near_ev.e, s));
  }
  int low = 0;
  if (sketch) {
    PSI_CK(cudaEventSynchronize(near_ev.e));
    synced = true;
    // prefix sort when the keys' top bits take nearly n distinct values (runs
    // of equal top bits are then few and short)
    if ((double)hll_sampled(n) < kPrefixMaxRun * hll_estimate(h_cnt->hll)) low = low_c;
  }
  const int passes = (key_bits - low + RB - 1) / RB;
  int pk = passes, p_pack = passes;
  int kr = 0, drop = 0;
  if (counts && pack_cand) {
    const int vbits = 64 - __builtin_clzll((uint64_t)(n - 1));
    int p = 1;
    while (p < passes && vbits + (key_bits - low) - RB * (p + 1) > 64) ++p;
    if (p + 2 <= passes - 1) p_pack = p;
  }

  uint64_t *kb[2] = {kbuf0, kbuf1};
  uint32_t *vb[2] = {vbuf0, vbuf1};
  for (int p = 0; p < passes; ++p) {
    if (p == p_pack) {
      if (!synced) PSI_CK(cudaEventSynchronize(near_ev.e));
      synced = true;
      if (2 * h_cnt->near >= (unsigned long long)n) {
        pk = p_pack;
        drop = low + RB * (pk + 1);
        kr = key_bits - drop;
      }
    }
    PassArgs a;
    a.kin = p == 0 ? (stored ? kst.p : keys_in) : kb[(p - 1) & 1];
    a.vin = p == 0 ? vals_in : vb[(p - 1) & 1];
    a.kfull = stored ? kst.p : nullptr;
    a.kout = kb[p & 1];
    a.vout = vb[p & 1];
    a.pts = enc.pts;
    a.bits = enc.bits;
    a.key_shift = enc.key_shift;
    a.n = n;
    a.shift = low + p * RB;
    a.gbase = nullptr;
    a.hist_cur = (p == 0 && low) ? hist.p + (size_t)passes_full * R::RADIX : hist.p + p * R::RADIX;
    a.hist_next = p + 1 < passes ? hist.p + (p + 1) * R::RADIX : nullptr;
    a.shift_next = low + (p + 1) * RB;
    a.lookback = lookback.p + (size_t)(p & 1) * tiles * R::RADIX;
    a.lookback_next = p + 1 < passes ? lookback.p + (size_t)((p + 1) & 1) * tiles * R::RADIX : nullptr;
    a.tile_ctr = ctr.p + p;
    a.status = d_status;
    if (p > pk) {
      a.shift = low + p * RB - drop;
      a.shift_next = low + (p + 1) * RB - drop;
      a.kmask = (1ull << kr) - 1;
    }
    a.kr = kr;
    a.drop = drop;
    if (p >= pk)
      st = launch_packed<RB>(enc, a, tiles, p == pk ? IO_PACK : (p + 1 < passes ? IO_KEYS : IO_UNPACK), s);
    else if (p > 0 || !encode)
      st = launch_pass<0, 2, 0, RB>(a, tiles, s);
    else if (stored)  // written keys, values = positions
      st = launch_pass<2, 2, 0, RB>(a, tiles, s);
    else if (enc.dim == 2)  // Morton keys computed from the points
      st = launch_pass<1, 2, 0, RB>(a, tiles, s);
    else
      st = launch_pass<1, 3, 0, RB>(a, tiles, s);
    if (st) return st;
  }
  out->keys = kb[(passes - 1) & 1];
  out->vals = vb[(passes - 1) & 1];
  out->prefix_low = low;
  out->local = synced ? (2 * h_cnt->near >= (unsigned long long)n ? 1 : 0) : -1;
  return PSI_OK;
}

psi_status sort_pairs(const EncodeSpec &enc, const uint64_t *keys_in, const uint32_t *vals_in, int64_t n,
                      int key_bits, const uint32_t *tie_ids, uint64_t *kbuf0, uint32_t *vbuf0, uint64_t *kbuf1,
                      uint32_t *vbuf1, int *d_status, cudaStream_t s, SortResult *out, int radix_bits) {
  out->keys = kbuf0;
  out->vals = vbuf0;
  if (n <= 0) return PSI_OK;
  if (n >= (int64_t)LB_VAL) {
    set_error("sort: more than 2^30-1 pairs in one sort");
    return PSI_ERR_INVALID;
  }
  const bool encode = enc.pts != nullptr;
  if (encode && (enc.dim != 2 && enc.dim != 3)) return PSI_ERR_INVALID;
  key_bits = std::max(1, std::min(64, key_bits));
  psi_status st;
  switch (pick_radix(key_bits, radix_bits)) {
    case 10:
      st = sort_pairs_rb<10>(enc, keys_in, vals_in, n, key_bits, kbuf0, vbuf0, kbuf1, vbuf1, d_status, s, out, false);
      break;
    case 11:
      st = sort_pairs_rb<11>(enc, keys_in, vals_in, n, key_bits, kbuf0, vbuf0, kbuf1, vbuf1, d_status, s, out, false);
      break;
    default:
      st = sort_pairs_rb<8>(enc, keys_in, vals_in, n, key_bits, kbuf0, vbuf0, kbuf1, vbuf1, d_status, s, out,
                            tie_ids != nullptr);
  }
  if (st) return st;

  if (tie_ids) {
    const int64_t cap_long = n / (kShortRun + 1) + 1;
    Buf<int64_t> runs;
    Buf<uint32_t> nlong;
    if ((st = runs.alloc(cap_long, s))) return st;
    if ((st = nlong.alloc(1, s))) return st;
    PSI_CK(cudaMemsetAsync(nlong.p, 0, sizeof(uint32_t), s));
    if (out->prefix_low > 0) {  // runs of equal top bits in (key, id) order (equal keys included)
      const int64_t cap_plong = n / (kPrefixShort + 1) + 1;
      if ((st = runs.alloc(cap_plong, s))) return st;
      const size_t smem = (size_t)kSmemRun * (sizeof(uint64_t) + 2 * sizeof(uint32_t));
      PSI_CK(cudaFuncSetAttribute(k_prefix_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      const int gr = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256 * kPrefixU), (int64_t)num_sms() * 8));
      // the run starts first (a light scan), then a thread per run
      const int64_t cap_starts = n / 4 + 1;
      Buf<int32_t> starts;
      Buf<unsigned long long> nst;
      if ((st = starts.alloc(cap_starts, s)) || (st = nst.alloc(1, s))) return st;
      PSI_CK(cudaMemsetAsync(nst.p, 0, sizeof(unsigned long long), s));
      PSI_LAUNCH(k_prefix_starts, gr, 256, 0, s, out->keys, n, out->prefix_low, starts.p, nst.p, cap_starts);
      PSI_LAUNCH(k_prefix_runs, num_sms() * 8, 256, 0, s, out->keys, out->vals, tie_ids, n, out->prefix_low, starts.p,
                 nst.p, cap_starts, runs.p, nlong.p, cap_plong);
      PSI_LAUNCH(k_prefix_long, num_sms(), 1024, smem, s, out->keys, out->vals, tie_ids, n, out->prefix_low, runs.p,
                 nlong.p, cap_plong);
    } else {
      PSI_LAUNCH(k_tie_runs, (unsigned)ceil_div(n, 256), 256, 0, s, out->keys, out->vals, tie_ids, n, runs.p,
                 nlong.p, cap_long);
      PSI_LAUNCH(k_tie_long, num_sms(), 1024, 0, s, out->keys, out->vals, tie_ids, n, runs.p, nlong.p, cap_long);
    }
  }
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}

// ---------------------------------------------------------------------------
// Exclusive scan (reduce, scan of block sums, apply)
// ---------------------------------------------------------------------------
namespace {
constexpr int SCAN_T = 512, SCAN_I = 8, SCAN_CHUNK = SCAN_T * SCAN_I;

template <class T>
__global__ void k_scan_reduce(const T *in, int64_t n, int64_t *sums) {
  __shared__ int64_t ws[SCAN_T / 32];
  const int64_t b = (int64_t)blockIdx.x * SCAN_CHUNK;
  int64_t acc = 0;
  for (int i = threadIdx.x; i < SCAN_CHUNK; i += SCAN_T)
    if (b + i < n) acc += (int64_t)in[b + i];
  for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int i = 0; i < SCAN_T / 32; ++i) t += ws[i];
    sums[blockIdx.x] = t;
  }
}

__global__ void k_scan_sums(int64_t *sums, int64_t nb, int64_t *total) {
  __shared__ int64_t carry;
  __shared__ int64_t ws[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
    const int64_t i = b0 + threadIdx.x;
    const int64_t v = i < nb ? sums[i] : 0;
    int64_t x = v;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    int64_t before = carry;
    for (int j = 0; j < w; ++j) before += ws[j];
    if (i < nb) sums[i] = before + x - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + x;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

template <class T>
__global__ void k_scan_apply(const T *in, int64_t *out, int64_t n, const int64_t *sums) {
  __shared__ int64_t ws[SCAN_T / 32];
  __shared__ int64_t carry;
  const int64_t b = (int64_t)blockIdx.x * SCAN_CHUNK;
  if (threadIdx.x == 0) carry = sums[blockIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int r = 0; r < SCAN_I; ++r) {
    const int64_t i = b + (int64_t)r * SCAN_T + threadIdx.x;
    const int64_t v = i < n ? (int64_t)in[i] : 0;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    int64_t before = carry;
    for (int j = 0; j < w; ++j) before += ws[j];
    if (i < n) out[i] = before + x - v;
    __syncthreads();
    if (threadIdx.x == SCAN_T - 1) carry = before + x;
    __syncthreads();
  }
}

template <class T>
psi_status scan_impl(const T *in, int64_t *out, int64_t n, int64_t *d_total, cudaStream_t s) {
  if (n <= 0) {
    if (d_total) PSI_CK(cudaMemsetAsync(d_total, 0, sizeof(int64_t), s));
    return PSI_OK;
  }
  const int64_t nb = ceil_div(n, SCAN_CHUNK);
  Buf<int64_t> sums;
  psi_status st = sums.alloc(nb, s);
  if (st) return st;
  PSI_LAUNCH_NAMED("k_scan_reduce", k_scan_reduce<T>, (unsigned)nb, SCAN_T, 0, s, in, n, sums.p);
  PSI_LAUNCH(k_scan_sums, 1, 1024, 0, s, sums.p, nb, d_total);
  PSI_LAUNCH_NAMED("k_scan_apply", k_scan_apply<T>, (unsigned)nb, SCAN_T, 0, s, in, out, n, sums.p);
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}

// int32 -> int64 exclusive scan with 16 consecutive elements per thread (four
// 16-byte loads, a running sum in registers, eight 16-byte stores), so that
// the block sums and the offsets cost one read, and one read and write, of the
// array at full width.  A block takes SCAN_CHUNK = 256 x 16 elements.
constexpr int SCANV_T = 256, SCANV_E = 16;
static_assert(SCANV_T * SCANV_E == SCAN_CHUNK, "block sums are laid out per SCAN_CHUNK elements");

// The SCANV_E elements of this thread (zero past n).
__device__ __forceinline__ void scanv_load(const int32_t *in, int64_t n, int64_t i0, int32_t (&v)[SCANV_E]) {
  if (i0 + SCANV_E <= n) {
    const int4 *p = reinterpret_cast<const int4 *>(in + i0);
#pragma unroll
    for (int j = 0; j < SCANV_E / 4; ++j) {
      const int4 q = p[j];
      v[4 * j] = q.x;
      v[4 * j + 1] = q.y;
      v[4 * j + 2] = q.z;
      v[4 * j + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < SCANV_E; ++j) v[j] = i0 + j < n ? in[i0 + j] : 0;
  }
}

// Block sum of 64-bit values (every thread gets it).
__device__ __forceinline__ int64_t scanv_block_excl(int64_t x, int64_t *total) {
  __shared__ int64_t ws[SCANV_T / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) ws[w] = inc;
  __syncthreads();
  int64_t before = 0, all = 0;
#pragma unroll
  for (int j = 0; j < SCANV_T / 32; ++j) {
    before += j < w ? ws[j] : 0;
    all += ws[j];
  }
  *total = all;
  return before + inc - x;
}

__global__ __launch_bounds__(SCANV_T) void k_scanv_reduce(const int32_t *in, int64_t n, int64_t *sums) {
  const int64_t i0 = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCANV_E;
  int32_t v[SCANV_E];
  scanv_load(in, n, i0, v);
  int64_t t = 0;
#pragma unroll
  for (int j = 0; j < SCANV_E; ++j) t += v[j];
  int64_t total;
  scanv_block_excl(t, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ __launch_bounds__(SCANV_T) void k_scanv_apply(const int32_t *in, int64_t *out, int64_t n,
                                                         const int64_t *sums) {
  const int64_t i0 = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCANV_E;
  int32_t v[SCANV_E];
  scanv_load(in, n, i0, v);
  int64_t t = 0;
#pragma unroll
  for (int j = 0; j < SCANV_E; ++j) t += v[j];
  int64_t total;
  int64_t run = sums[blockIdx.x] + scanv_block_excl(t, &total);
  if (i0 + SCANV_E <= n) {
    longlong2 *p = reinterpret_cast<longlong2 *>(out + i0);
#pragma unroll
    for (int j = 0; j < SCANV_E / 2; ++j) {
      longlong2 q;
      q.x = run;
      run += v[2 * j];
      q.y = run;
      run += v[2 * j + 1];
      p[j] = q;
    }
  } else {
#pragma unroll
    for (int j = 0; j < SCANV_E; ++j) {
      if (i0 + j < n) out[i0 + j] = run;
      run += v[j];
    }
  }
}

}  // namespace

psi_status scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *d_total, cudaStream_t s) {
  return scan_impl<int64_t>(in, out, n, d_total, s);
}
psi_status scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, int64_t *d_total, cudaStream_t s) {
  // the vector form needs 16-byte aligned arrays (the library's own are)
  if (n <= 0 || (reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
    return scan_impl<int32_t>(in, out, n, d_total, s);
  const int64_t nb = ceil_div(n, SCAN_CHUNK);
  Buf<int64_t> sums;
  psi_status st = sums.alloc(nb, s);
  if (st) return st;
  PSI_LAUNCH_NAMED("k_scan_reduce", k_scanv_reduce, (unsigned)nb, SCANV_T, 0, s, in, n, sums.p);
  PSI_LAUNCH(k_scan_sums, 1, 1024, 0, s, sums.p, nb, d_total);
  PSI_LAUNCH_NAMED("k_scan_apply", k_scanv_apply, (unsigned)nb, SCANV_T, 0, s, in, out, n, sums.p);
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}

}  // namespace psi

// ---------------------------------------------------------------------------
// The key sort without any allocation: all scratch (the second key/value
// buffer, digit histograms, look-back table, tile counters, status word) lives
// in one fixed device array that every GPU loading this library holds until
// the process exits.
// ---------------------------------------------------------------------------
namespace psi {
namespace {

constexpr int64_t kNoAllocMaxPairs = int64_t(1) << 20;
constexpr int64_t kNoAllocTiles = (kNoAllocMaxPairs + TILE - 1) / TILE;
constexpr size_t kOffKeys = 0;
constexpr size_t kOffVals = kOffKeys + sizeof(uint64_t) * kNoAllocMaxPairs;
constexpr size_t kOffHist = kOffVals + sizeof(uint32_t) * kNoAllocMaxPairs;
constexpr int RADIX = Radix<8>::RADIX;
constexpr size_t kOffBase = kOffHist + sizeof(uint32_t) * MAX_PASSES * RADIX;
constexpr size_t kOffLook = kOffBase + sizeof(uint32_t) * MAX_PASSES * RADIX;
constexpr size_t kOffCtr = kOffLook + sizeof(uint32_t) * MAX_PASSES * kNoAllocTiles * RADIX;
constexpr size_t kOffStatus = kOffCtr + sizeof(uint32_t) * MAX_PASSES;
constexpr size_t kNoAllocBytes = (kOffStatus + sizeof(int) + 255) / 256 * 256;  // about 14 MB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Host code may not use g_noalloc_scratch as a pointer: on the host that name
// is only a stand-in for the device symbol.  Its device address is looked up
// with the device current, once per device and context (a context torn down
// and created again, e.g. after cudaDeviceReset, may load the module at
// another address), and cached here.
std::mutex g_noalloc_mu;
struct NoallocAddr {
  void *ctx = nullptr;
  unsigned char *addr = nullptr;
};
NoallocAddr g_noalloc_addr[64];

// The current driver context (null if the driver's entry point is not
// reachable), through the runtime's driver entry-point query.
void *current_context() {
  using CtxGet = CUresult (*)(CUcontext *);
  static CtxGet fn = nullptr;
  static bool tried = false;
  if (!tried) {  // under g_noalloc_mu
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGet>(p);
    else
      cudaGetLastError();
  }
  CUcontext c = nullptr;
  if (fn && fn(&c) != CUDA_SUCCESS) c = nullptr;
  return c;
}

psi_status noalloc_scratch(unsigned char **out) {
  int dev = 0;
  PSI_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal out of range");
    return PSI_ERR_INVALID;
  }
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  void *ctx = current_context();
  NoallocAddr &e = g_noalloc_addr[dev];
  // without a context handle to compare, look the address up on every call
  if (!e.addr || !ctx || e.ctx != ctx) {
    void *p = nullptr;
    cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (err != cudaSuccess || !p) return cuda_fail(err != cudaSuccess ? err : cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
    e.addr = static_cast<unsigned char *>(p);
    e.ctx = ctx;
  }
  *out = e.addr;
  return PSI_OK;
}

}  // namespace
}  // namespace psi

extern "C" psi_status psi_sort_pairs_noalloc(uint64_t *d_keys, uint32_t *d_vals, int64_t n, int32_t key_bits,
                                             void *stream) {
  using namespace psi;
  set_error("");
  if (n < 0 || (n > 0 && (!d_keys || !d_vals)) || key_bits < 1 || key_bits > 64) {
    set_error("invalid sort arguments");
    return PSI_ERR_INVALID;
  }
  if (n > kNoAllocMaxPairs) {
    set_error("psi_sort_pairs_noalloc: at most 1048576 pairs per call (use psi_sort_pairs for more)");
    return PSI_ERR_INVALID;
  }
  if (n == 0) return PSI_OK;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char *base = nullptr;
  psi_status st = noalloc_scratch(&base);
  if (st) return st;
  uint64_t *skeys = reinterpret_cast<uint64_t *>(base + kOffKeys);
  uint32_t *svals = reinterpret_cast<uint32_t *>(base + kOffVals);
  uint32_t *hist = reinterpret_cast<uint32_t *>(base + kOffHist);
  uint32_t *gbase = reinterpret_cast<uint32_t *>(base + kOffBase);
  uint32_t *look = reinterpret_cast<uint32_t *>(base + kOffLook);
  uint32_t *ctr = reinterpret_cast<uint32_t *>(base + kOffCtr);
  int *status = reinterpret_cast<int *>(base + kOffStatus);
  const int passes = (key_bits + 8 - 1) / 8;
  const int64_t tiles = ceil_div(n, TILE);
  // the array keeps the previous call's contents: clear what must start at zero
  PSI_CK(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * passes * RADIX, s));
  PSI_CK(cudaMemsetAsync(look, 0, sizeof(uint32_t) * passes * tiles * RADIX, s));
  PSI_CK(cudaMemsetAsync(ctr, 0, sizeof(uint32_t) * passes, s));
  PSI_CK(cudaMemsetAsync(status, 0, sizeof(int), s));
  EncodeSpec none;
  if ((st = launch_hist<0, 2, 0, 8>(d_keys, none, n, passes, hist, status, s))) return st;
  PSI_LAUNCH_NAMED("k_hist_scan", k_hist_scan<8>, passes, RADIX, 0, s, hist, gbase);
  // ping-pong between the scratch pair (even passes) and the caller's arrays
  uint64_t *kb[2] = {skeys, d_keys};
  uint32_t *vb[2] = {svals, d_vals};
  for (int p = 0; p < passes; ++p) {
    PassArgs a;
    a.kin = p == 0 ? d_keys : kb[(p - 1) & 1];
    a.vin = p == 0 ? d_vals : vb[(p - 1) & 1];
    a.kout = kb[p & 1];
    a.vout = vb[p & 1];
    a.pts = nullptr;
    a.bits = 0;
    a.key_shift = 0;
    a.n = n;
    a.shift = p * 8;
    a.gbase = gbase + p * RADIX;
    a.hist_cur = nullptr;
    a.hist_next = nullptr;
    a.shift_next = 0;
    a.lookback = look + (size_t)p * tiles * RADIX;
    a.lookback_next = nullptr;
    a.tile_ctr = ctr + p;
    a.status = status;
    if ((st = launch_pass<0, 2, 0, 8>(a, tiles, s))) return st;
  }
  if ((passes & 1) == 1) {  // the last pass wrote the scratch pair
    PSI_CK(cudaMemcpyAsync(d_keys, skeys, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
    PSI_CK(cudaMemcpyAsync(d_vals, svals, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
  }
  PSI_CK(cudaGetLastError());
  int h = 0;
  PSI_CK(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaStreamSynchronize(s));
  if (h & ST_TIMEOUT) {
    set_error("a bounded device-side wait timed out");
    return PSI_ERR_DEVICE_TIMEOUT;
  }
  return PSI_OK;
}

// ---------------------------------------------------------------------------
// Test hook of the bounded look-back wait (failure detection without a GPU
// fault): the sort of psi_sort_pairs_noalloc's plan (8-bit digits, global
// digit offsets scanned up front) on library-allocated scratch, with one tile
// of the first digit pass withholding its look-back words.
// ---------------------------------------------------------------------------
extern "C" psi_status psi_test_sort_withheld_tile(uint64_t *d_keys, uint32_t *d_vals, int64_t n,
                                                  int64_t withheld_tile, uint32_t spin_limit, void *stream) {
  using namespace psi;
  set_error("");
  if (n < 0 || (n > 0 && (!d_keys || !d_vals)) || n >= (int64_t)LB_VAL || spin_limit < 1) {
    set_error("invalid test sort arguments");
    return PSI_ERR_INVALID;
  }
  if (n == 0) return PSI_OK;
  cudaStream_t s = (cudaStream_t)stream;
  constexpr int RADIX = Radix<8>::RADIX;
  const int passes = 8;
  const int64_t tiles = ceil_div(n, TILE);
  Buf<uint64_t> k2;
  Buf<uint32_t> v2, hist, gbase, look, ctr;
  Buf<int> status;
  psi_status st;
  if ((st = k2.alloc(n, s)) || (st = v2.alloc(n, s)) || (st = hist.alloc(passes * RADIX, s)) ||
      (st = gbase.alloc(passes * RADIX, s)) || (st = look.alloc((size_t)passes * tiles * RADIX, s)) ||
      (st = ctr.alloc(passes, s)) || (st = status.alloc(1, s)))
    return st;
  PSI_CK(cudaMemsetAsync(hist.p, 0, sizeof(uint32_t) * passes * RADIX, s));
  PSI_CK(cudaMemsetAsync(look.p, 0, sizeof(uint32_t) * passes * tiles * RADIX, s));
  PSI_CK(cudaMemsetAsync(ctr.p, 0, sizeof(uint32_t) * passes, s));
  PSI_CK(cudaMemsetAsync(status.p, 0, sizeof(int), s));
  EncodeSpec none;
  if ((st = launch_hist<0, 2, 0, 8>(d_keys, none, n, passes, hist.p, status.p, s))) return st;
  PSI_LAUNCH_NAMED("k_hist_scan", k_hist_scan<8>, passes, RADIX, 0, s, hist.p, gbase.p);
  uint64_t *kb[2] = {k2.p, d_keys};
  uint32_t *vb[2] = {v2.p, d_vals};
  for (int p = 0; p < passes; ++p) {
    PassArgs a;
    a.kin = p == 0 ? d_keys : kb[(p - 1) & 1];
    a.vin = p == 0 ? d_vals : vb[(p - 1) & 1];
    a.kout = kb[p & 1];
    a.vout = vb[p & 1];
    a.pts = nullptr;
    a.bits = 0;
    a.key_shift = 0;
    a.n = n;
    a.shift = p * 8;
    a.gbase = gbase.p + p * RADIX;
    a.hist_cur = nullptr;
    a.hist_next = nullptr;
    a.shift_next = 0;
    a.lookback = look.p + (size_t)p * tiles * RADIX;
    a.lookback_next = nullptr;
    a.tile_ctr = ctr.p + p;
    a.status = status.p;
    a.spin_limit = spin_limit;
    a.withheld_tile = p == 0 ? withheld_tile : -1;
    if ((st = launch_pass<0, 2, 0, 8>(a, tiles, s))) return st;
  }
  PSI_CK(cudaGetLastError());
  int h = 0;
  PSI_CK(cudaMemcpyAsync(&h, status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaStreamSynchronize(s));
  if (h & ST_TIMEOUT) {
    set_error("a bounded device-side wait timed out");
    return PSI_ERR_DEVICE_TIMEOUT;
  }
  return PSI_OK;
}

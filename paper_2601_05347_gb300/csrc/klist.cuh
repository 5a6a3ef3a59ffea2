// klist.cuh -- the k best (distance, id) pairs of one query, kept sorted
// across a warp, for any distance type T (exact int64 squared distances of the
// integer indexes, double squared distances of the float P-Orth).
//
// Entry e = r*32 + lane lives in register r of lane `lane`; entries past the
// k-th hold (+inf, 0xFFFFFFFF).  Order: by distance, then by id (the k-NN
// tie rule).  A candidate is inserted by one ballot per register and one
// shuffle shift; a chunk of many entrants is sorted across the warp and merged
// one 32-entry row at a time by bitonic merges with a carry.
#pragma once
#include <stdint.h>

namespace psi {

template <typename T>
struct DistInf;
template <>
struct DistInf<int64_t> {
  __device__ __forceinline__ static int64_t v() { return INT64_MAX; }
};
template <>
struct DistInf<double> {
  __device__ __forceinline__ static double v() { return __longlong_as_double(0x7FF0000000000000ll); }
};

template <typename T>
__device__ __forceinline__ bool pair_less(T da, uint32_t ia, T db, uint32_t ib) {
  return da < db || (da == db && ia < ib);
}

// Non-negative int64 distances (INT64_MAX as +inf): the 96-bit number
// (d, id) is compared by one subtraction with borrow through its three words.
template <>
__device__ __forceinline__ bool pair_less<int64_t>(int64_t da, uint32_t ia, int64_t db, uint32_t ib) {
  uint32_t t, r;
  asm("sub.cc.u32 %0, %2, %3;\n\t"
      "subc.cc.u32 %0, %4, %5;\n\t"
      "subc.cc.u32 %0, %6, %7;\n\t"
      "subc.u32 %1, 0, 0;"
      : "=&r"(t), "=r"(r)
      : "r"(ia), "r"(ib), "r"((uint32_t)da), "r"((uint32_t)db), "r"((uint32_t)((uint64_t)da >> 32)),
        "r"((uint32_t)((uint64_t)db >> 32)));
  (void)t;  // the low words' difference: only the borrow out of the top word is used
  return r != 0;
}

template <int KPL, typename T = int64_t>
struct KList {
  T d[KPL];
  uint32_t i[KPL];
  T kd;  // k-th entry (warp-uniform)
  uint32_t ki;

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int r = 0; r < KPL; ++r) {
      d[r] = DistInf<T>::v();
      i[r] = 0xFFFFFFFFu;
    }
    kd = DistInf<T>::v();
    ki = 0xFFFFFFFFu;
  }
  __device__ __forceinline__ bool admits(T cd, uint32_t ci) const { return pair_less(cd, ci, kd, ki); }

  // Reads the k-th entry into kd, ki (all lanes).
  __device__ __forceinline__ void refresh_kth(int k) {
    const int rk = (k - 1) >> 5, lk = (k - 1) & 31;
    T vd = d[0];
    uint32_t vi = i[0];
#pragma unroll
    for (int r = 1; r < KPL; ++r)
      if (r == rk) {
        vd = d[r];
        vi = i[r];
      }
    kd = __shfl_sync(0xFFFFFFFFu, vd, lk);
    ki = __shfl_sync(0xFFFFFFFFu, vi, lk);
  }

  // Insert a warp-uniform candidate into the sorted list of k entries.
  __device__ __forceinline__ void insert(T cd, uint32_t ci, int k) {
    const int lane = threadIdx.x & 31;
    int pos = 32 * KPL;
#pragma unroll
    for (int r = 0; r < KPL; ++r) {
      const uint32_t m = __ballot_sync(0xFFFFFFFFu, pair_less(cd, ci, d[r], i[r]));
      if (m && pos == 32 * KPL) pos = r * 32 + __ffs(m) - 1;
    }
    if (pos >= k) return;
#pragma unroll
    for (int r = KPL - 1; r >= 0; --r) {
      T ud = __shfl_up_sync(0xFFFFFFFFu, d[r], 1);
      uint32_t ui = __shfl_up_sync(0xFFFFFFFFu, i[r], 1);
      if (r > 0) {
        const T cd2 = __shfl_sync(0xFFFFFFFFu, d[r > 0 ? r - 1 : 0], 31);
        const uint32_t ci2 = __shfl_sync(0xFFFFFFFFu, i[r > 0 ? r - 1 : 0], 31);
        if (lane == 0) {
          ud = cd2;
          ui = ci2;
        }
      }
      const int e = r * 32 + lane;
      if (e > pos) {
        d[r] = ud;
        i[r] = ui;
      } else if (e == pos) {
        d[r] = cd;
        i[r] = ci;
      }
    }
    refresh_kth(k);
  }
};

// Ascending warp bitonic sort of (d, i) pairs, one per lane.
template <typename T>
__device__ __forceinline__ void warp_sort_pairs(T &d, uint32_t &i) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const T od = __shfl_xor_sync(0xFFFFFFFFu, d, j);
      const uint32_t oi = __shfl_xor_sync(0xFFFFFFFFu, i, j);
      const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
      const bool other_less = pair_less(od, oi, d, i);
      if (keep_min == other_less) {
        d = od;
        i = oi;
      }
    }
  }
}

// Half-cleaners j = 16 .. 1 that sort a bitonic sequence of (d, i) pairs,
// one per lane, ascending.
template <typename T>
__device__ __forceinline__ void warp_bitonic_clean(T &d, uint32_t &i) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 16; j > 0; j >>= 1) {
    const T od = __shfl_xor_sync(0xFFFFFFFFu, d, j);
    const uint32_t oi = __shfl_xor_sync(0xFFFFFFFFu, i, j);
    const bool lower = (lane & j) == 0;
    if (lower == pair_less(od, oi, d, i)) {
      d = od;
      i = oi;
    }
  }
}

// Fills an empty list from one candidate per lane (`in`: the lane holds one):
// sorted across the warp, the first min(k, 32) become the list.
template <int KPL, typename T>
__device__ __forceinline__ void klist_fill(KList<KPL, T> &kl, bool in, T d2, uint32_t id, int k) {
  const int lane = threadIdx.x & 31;
  T cd = in ? d2 : DistInf<T>::v();
  uint32_t ci = in ? id : 0xFFFFFFFFu;
  warp_sort_pairs(cd, ci);
  if (lane < k) {
    kl.d[0] = cd;
    kl.i[0] = ci;
  }
  kl.refresh_kth(k);
}

// Ascending warp bitonic sort of one 64-bit key per lane.
__device__ __forceinline__ void warp_sort_u64(uint64_t &x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const uint64_t o = __shfl_xor_sync(0xFFFFFFFFu, x, j);
      const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
      if (keep_min == (o < x)) x = o;
    }
  }
}

// Integer distances: when every candidate's distance is below 2^32 - 1 (the
// common case for a query's first leaf), (d2 << 32 | id) orders the pairs
// exactly as (d2, id) does, and one 64-bit key per lane sorts faster than a
// (distance, id) pair.
template <int KPL>
__device__ __forceinline__ void klist_fill(KList<KPL, int64_t> &kl, bool in, int64_t d2, uint32_t id, int k) {
  const int lane = threadIdx.x & 31;
  if (__all_sync(0xFFFFFFFFu, !in || (uint64_t)d2 < 0xFFFFFFFFull)) {
    uint64_t x = in ? ((uint64_t)d2 << 32 | id) : ~0ull;
    warp_sort_u64(x);
    if (lane < k) {
      kl.d[0] = x == ~0ull ? DistInf<int64_t>::v() : (int64_t)(x >> 32);
      kl.i[0] = x == ~0ull ? 0xFFFFFFFFu : (uint32_t)x;
    }
  } else {
    int64_t cd = in ? d2 : DistInf<int64_t>::v();
    uint32_t ci = in ? id : 0xFFFFFFFFu;
    warp_sort_pairs(cd, ci);
    if (lane < k) {
      kl.d[0] = cd;
      kl.i[0] = ci;
    }
  }
  kl.refresh_kth(k);
}

// Offers one candidate per lane (`in`: it beats the current k-th).  With more
// than six entrants they are sorted across the warp and merged into the list
// row by row: the row against the reversed carry gives, lane-wise, the 32
// smallest of both (a bitonic sequence, cleaned into the row) and the 32
// largest (cleaned into the carry for the next row); otherwise the entrants
// are inserted one at a time.
template <int KPL, typename T>
__device__ __forceinline__ void klist_offer(KList<KPL, T> &kl, bool in, T d2, uint32_t id, int k) {
  const int lane = threadIdx.x & 31;
  uint32_t m = __ballot_sync(0xFFFFFFFFu, in);
  if (__popc(m) > 6) {
    T cd = in ? d2 : DistInf<T>::v();
    uint32_t ci = in ? id : 0xFFFFFFFFu;
    warp_sort_pairs(cd, ci);
#pragma unroll
    for (int r = 0; r < KPL; ++r) {
      if (__ballot_sync(0xFFFFFFFFu, cd != DistInf<T>::v()) == 0) break;  // nothing left to place
      const T rd = __shfl_sync(0xFFFFFFFFu, cd, 31 - lane);
      const uint32_t ri = __shfl_sync(0xFFFFFFFFu, ci, 31 - lane);
      T lo_d = kl.d[r], hi_d = rd;
      uint32_t lo_i = kl.i[r], hi_i = ri;
      if (pair_less(rd, ri, lo_d, lo_i)) {
        hi_d = lo_d;
        hi_i = lo_i;
        lo_d = rd;
        lo_i = ri;
      }
      warp_bitonic_clean(lo_d, lo_i);
      warp_bitonic_clean(hi_d, hi_i);
      kl.d[r] = lo_d;
      kl.i[r] = lo_i;
      cd = hi_d;
      ci = hi_i;
    }
    // entries past the k-th are dropped; the k-th bounds admission
#pragma unroll
    for (int r = 0; r < KPL; ++r)
      if (r * 32 + lane >= k) {
        kl.d[r] = DistInf<T>::v();
        kl.i[r] = 0xFFFFFFFFu;
      }
    kl.refresh_kth(k);
    return;
  }
  while (m) {
    const int src = __ffs(m) - 1;
    m &= m - 1;
    const T cd = __shfl_sync(0xFFFFFFFFu, d2, src);
    const uint32_t ci = __shfl_sync(0xFFFFFFFFu, id, src);
    if (kl.admits(cd, ci)) kl.insert(cd, ci, k);
  }
}

}  // namespace psi

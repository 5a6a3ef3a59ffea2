// keys.cuh -- space-filling-curve keys on the device (Sec 2.2).
//
// Morton (Z) keys: bit i of coordinate d goes to key bit dim*i + d.  The bits
// are spread with the usual shift-and-mask ladder (each step doubles the gap
// between the groups of bits that are still together).
//
// Hilbert keys (2D): a four-state automaton read top level first.  The state
// is the symmetry that maps the current sub-square onto the canonical curve:
// bit 0 = the axes are exchanged, bit 1 = both axes are reversed.  At each
// level the quadrant bits (rx, ry) of the point are mapped through the state,
// the canonical quadrant (cx, cy) gives the base-4 digit
// (0,0)->0, (0,1)->1, (1,1)->2, (1,0)->3, and the sub-curve of that quadrant
// composes its own symmetry into the state: digit 0 exchanges the axes,
// digit 3 exchanges and reverses them, digits 1 and 2 leave the state alone.
// The four symmetries form a Klein four-group, so composition is XOR of the
// two state bits.  Four levels are consumed per step through a 1024-entry
// table (state, 4 x-bits, 4 y-bits) -> (8 key bits, next state) that every
// thread block derives from the automaton into shared memory.
//
// Hilbert keys (3D; the paper defines Hilbert keys in 2D only, so the 3D curve
// is a reading): Skilling's curve (J. Skilling, "Programming the Hilbert
// curve", AIP Conf. Proc. 707, 2004) with axes X0 = x, X1 = y, X2 = z, which
// runs from (0,0,0) to (2^b - 1, 0, 0).  His method works on whole coordinate
// words -- undo the sub-cube symmetries from the top bit down, then Gray-code
// -- but every step at bit level l only alters the bits below l, so it runs
// here as an automaton read top level first.  The state is the symmetry that
// the levels above have imposed on the bits below (a permutation of the three
// axes with a reflection per axis) plus the running parity of the Gray code of
// the last axis; 96 encodings, 48 reachable.  Per level: the point's octant
// bits are mapped through the symmetry to (b0, b1, b2); the Gray code
// g = (b0, b0^b1, b0^b1^b2), complemented when the parity is odd, is the
// octant digit (g0 most significant); the parity absorbs g2; then for
// i = 0, 1, 2 in turn, a set b_i reflects axis 0 and a clear b_i exchanges
// axes 0 and i.  One level is consumed per step through a 768-entry table
// (state, octant) -> (next state, digit) that every thread block derives from
// the automaton into shared memory; the octant bits are read off the point's
// Morton key, three bits per level.
#pragma once
#include <stdint.h>

namespace psi {

__device__ __forceinline__ uint64_t spread_bits2(uint32_t v) {
  uint64_t x = v;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}

__device__ __forceinline__ uint64_t spread_bits3(uint32_t v) {
  uint64_t x = v & 0x1FFFFFu;
  x = (x | (x << 32)) & 0x001F00000000FFFFull;
  x = (x | (x << 16)) & 0x001F0000FF0000FFull;
  x = (x | (x << 8)) & 0x100F00F00F00F00Full;
  x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

__device__ __forceinline__ uint64_t morton2_key(uint32_t x, uint32_t y) {
  return spread_bits2(x) | (spread_bits2(y) << 1);
}

__device__ __forceinline__ uint64_t morton3_key(uint32_t x, uint32_t y, uint32_t z) {
  return spread_bits3(x) | (spread_bits3(y) << 1) | (spread_bits3(z) << 2);
}

// One level of the Hilbert automaton: returns the digit, updates the state.
__device__ __forceinline__ uint32_t hilbert_step(uint32_t &state, uint32_t rx, uint32_t ry) {
  uint32_t cx = (state & 1) ? ry : rx;
  uint32_t cy = (state & 1) ? rx : ry;
  if (state & 2) {
    cx ^= 1u;
    cy ^= 1u;
  }
  uint32_t digit = (cx << 1) | (cx ^ cy);
  state ^= (digit == 0) ? 1u : (digit == 3 ? 3u : 0u);
  return digit;
}

// Fills the 1024-entry four-level table (state, 4 x-bits, 4 y-bits) ->
// (8 key bits, next state << 8) as uint16; call with all threads, then sync.
__device__ __forceinline__ void hilbert_table_init(uint8_t *tab8) {
  uint16_t *tab = reinterpret_cast<uint16_t *>(tab8);
  for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
    uint32_t st = (uint32_t)e >> 8, xb = ((uint32_t)e >> 4) & 15u, yb = (uint32_t)e & 15u, d = 0;
    for (int l = 3; l >= 0; --l) d = (d << 2) | hilbert_step(st, (xb >> l) & 1u, (yb >> l) & 1u);
    tab[e] = (uint16_t)(d | (st << 8));
  }
}

// The key over `bits` levels, walked as a curve of 32 levels: the 32 - bits
// levels above the point's own are quadrant 0 (digit 0), and each of them
// exchanges the axes, so the walk is the same with x and y exchanged when
// their number is odd.  Level l's digit lands on key bits 2l, 2l + 1; eight
// fully unrolled steps of four levels.  Coordinate bits at and above `bits`
// are ignored.
__device__ __forceinline__ uint64_t hilbert2_key(const uint8_t *tab8, uint32_t x, uint32_t y, int bits) {
  const uint16_t *tab = reinterpret_cast<const uint16_t *>(tab8);
  const uint32_t m = (1u << bits) - 1u;  // bits <= 31
  x &= m;
  y &= m;
  if ((32 - bits) & 1) {
    const uint32_t t = x;
    x = y;
    y = t;
  }
  uint32_t st = 0, khi = 0, klo = 0;  // st: state << 8
#pragma unroll
  for (int s = 28; s >= 0; s -= 4) {
    const uint32_t e = tab[st | (((x >> s) & 15u) << 4) | ((y >> s) & 15u)];
    if (s >= 16)
      khi |= (e & 255u) << (2 * s - 32);
    else
      klo |= (e & 255u) << (2 * s);
    st = e & 0x300u;
  }
  return ((uint64_t)khi << 32) | klo;
}

// Bytes of shared memory for the curve tables of either dimension.
constexpr int kCurveTabBytes = 2048;

// Five levels per step (used where a block can spare 8 KB of shared memory):
// (state, 5 x-bits, 5 y-bits) -> (10 key bits, next state << 10) as uint16,
// 4096 entries; call with all threads, then sync.
constexpr int kHilbert5TabBytes = 4096 * 2;
__device__ __forceinline__ void hilbert5_table_init(uint8_t *tab8) {
  uint16_t *tab = reinterpret_cast<uint16_t *>(tab8);
  for (int e = threadIdx.x; e < 4096; e += blockDim.x) {
    uint32_t st = (uint32_t)e >> 10, xb = ((uint32_t)e >> 5) & 31u, yb = (uint32_t)e & 31u, d = 0;
    for (int l = 4; l >= 0; --l) d = (d << 2) | hilbert_step(st, (xb >> l) & 1u, (yb >> l) & 1u);
    tab[e] = (uint16_t)(d | (st << 10));
  }
}

// The key of hilbert2_key, five levels per step: walked as a curve of P = 30
// levels (six steps) when bits <= 30, else of 35 levels (seven steps; the
// top bits that fall off the 64-bit key are digits of padding levels, 0),
// with x and y exchanged when P - bits is odd (each padding level is quadrant
// 0, which exchanges the axes).
__device__ __forceinline__ uint64_t hilbert2_key5(const uint8_t *tab8, uint32_t x, uint32_t y, int bits) {
  const uint16_t *tab = reinterpret_cast<const uint16_t *>(tab8);
  const uint32_t m = (1u << bits) - 1u;  // bits <= 31
  x &= m;
  y &= m;
  const int P = bits <= 30 ? 30 : 35;
  if ((P - bits) & 1) {
    const uint32_t t = x;
    x = y;
    y = t;
  }
  uint64_t key = 0;
  uint32_t st = 0;  // state << 10
  if (P == 30) {
#pragma unroll
    for (int s = 25; s >= 0; s -= 5) {
      const uint32_t e = tab[st | (((x >> s) & 31u) << 5) | ((y >> s) & 31u)];
      key = (key << 10) | (e & 1023u);
      st = e & 0xC00u;
    }
  } else {
#pragma unroll
    for (int s = 30; s >= 0; s -= 5) {
      const uint32_t e = tab[st | (((x >> s) & 31u) << 5) | ((y >> s) & 31u)];
      key = (key << 10) | (e & 1023u);
      st = e & 0xC00u;
    }
  }
  return key;
}

// The 3D automaton state: perm index (0..5) x 16 + reflections x 2 + parity;
// permutations in lexicographic order (0,1,2) (0,2,1) (1,0,2) (1,2,0) (2,0,1) (2,1,0).
__device__ __forceinline__ void perm3_of(int idx, int *p) {
  const int p0 = idx >> 1;
  const int a = p0 == 0 ? 1 : 0;        // smaller remaining axis
  const int b = p0 == 2 ? 1 : 2;        // larger remaining axis
  p[0] = p0;
  p[1] = (idx & 1) ? b : a;
  p[2] = (idx & 1) ? a : b;
}

// Fills the 768-entry table as uint16 (next state x 64 | digit); call with all
// threads, then sync.
__device__ __forceinline__ void hilbert3_table_init(uint8_t *tab8) {
  uint16_t *tab = reinterpret_cast<uint16_t *>(tab8);
  for (int e = threadIdx.x; e < 768; e += blockDim.x) {
    const int id = e >> 3, r = e & 7;
    int p[3];
    perm3_of(id >> 4, p);
    int f = (id >> 1) & 7, par = id & 1;
    int b[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) b[i] = ((r >> p[i]) & 1) ^ ((f >> i) & 1);
    const int g0 = b[0], g1 = b[0] ^ b[1], g2 = g1 ^ b[2];
    const int digit = ((g0 ^ par) << 2) | ((g1 ^ par) << 1) | (g2 ^ par);
    par ^= g2;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (b[i]) {
        f ^= 1;
      } else if (i) {
        const int t = p[0];
        p[0] = p[i];
        p[i] = t;
        const int f0 = f & 1, fi = (f >> i) & 1;
        f = (f & ~(1 | (1 << i))) | fi | (f0 << i);
      }
    }
    int pi = 0;
    for (int c = 0; c < 6; ++c) {
      int q[3];
      perm3_of(c, q);
      if (q[0] == p[0] && q[1] == p[1]) pi = c;
    }
    const int next = (pi << 4) | (f << 1) | par;
    tab[e] = (uint16_t)((next << 6) | digit);
  }
}

__device__ __forceinline__ uint64_t hilbert3_key(const uint8_t *tab8, uint32_t x, uint32_t y, uint32_t z,
                                                 int bits) {
  const uint16_t *tab = reinterpret_cast<const uint16_t *>(tab8);
  const uint64_t m = morton3_key(x, y, z);
  uint32_t st = 0;  // state x 8
  uint64_t d = 0;
  for (int l = bits - 1; l >= 0; --l) {
    const uint32_t e = tab[st | (uint32_t)((m >> (3 * l)) & 7u)];
    d = (d << 3) | (e & 7u);
    st = e >> 3;
  }
  return d;
}

// Two levels per step (where a block can spare 13.5 KB of shared memory):
// the one-level table (768 entries) followed by a table of 96 states x 64
// octant pairs, (next state after both levels << 6 | the two digits), built
// from it.  Call with all threads (it syncs inside), then sync.
constexpr int kHilbert3x2TabBytes = 768 * 2 + 96 * 64 * 2;
__device__ __forceinline__ void hilbert3x2_table_init(uint8_t *tab8) {
  hilbert3_table_init(tab8);
  __syncthreads();
  const uint16_t *t1 = reinterpret_cast<const uint16_t *>(tab8);
  uint16_t *t2 = reinterpret_cast<uint16_t *>(tab8) + 768;
  for (int e = threadIdx.x; e < 96 * 64; e += blockDim.x) {
    const int st = e >> 6, o1 = (e >> 3) & 7, o2 = e & 7;
    const uint32_t a = t1[st * 8 + o1];
    const uint32_t b = t1[(a >> 6) * 8 + o2];
    t2[e] = (uint16_t)(((b >> 6) << 6) | ((a & 7u) << 3) | (b & 7u));
  }
}

// hilbert3_key with the two-level table: an odd top level alone, then pairs.
__device__ __forceinline__ uint64_t hilbert3_key2(const uint8_t *tab8, uint32_t x, uint32_t y, uint32_t z,
                                                  int bits) {
  const uint16_t *t1 = reinterpret_cast<const uint16_t *>(tab8);
  const uint16_t *t2 = t1 + 768;
  const uint64_t m = morton3_key(x, y, z);
  uint32_t st = 0;  // state
  uint64_t d = 0;
  int l = bits - 1;
  if (bits & 1) {
    const uint32_t e = t1[st * 8 + (uint32_t)((m >> (3 * l)) & 7u)];
    d = e & 7u;
    st = e >> 6;
    --l;
  }
  for (; l > 0; l -= 2) {  // levels l and l - 1
    const uint32_t e = t2[st * 64 + (uint32_t)((m >> (3 * (l - 1))) & 63u)];
    d = (d << 6) | (e & 63u);
    st = e >> 6;
  }
  return d;
}

// Curve table of the (D, CURVE) key; call with all threads, then sync.
template <int D, int CURVE>
__device__ __forceinline__ void curve_table_init(uint8_t *tab) {
  if (CURVE == 1) {
    if (D == 2)
      hilbert_table_init(tab);
    else
      hilbert3_table_init(tab);
  }
}

// Key of point p (dim coordinates) under the encode spec; sets *bad if a
// coordinate lies outside [0, 2^bits).
template <int D, int CURVE>
__device__ __forceinline__ uint64_t point_key(const uint8_t *htab, const int32_t *c, int bits, bool &bad) {
  uint32_t lim = 1u << bits;  // bits <= 31
  bool b = false;
#pragma unroll
  for (int d = 0; d < D; ++d) b |= (uint32_t)c[d] >= lim;
  bad = b;
  if (CURVE == 1 && D == 3) return hilbert3_key(htab, (uint32_t)c[0], (uint32_t)c[1], (uint32_t)c[D - 1], bits);
  if (CURVE == 1) return hilbert2_key(htab, (uint32_t)c[0], (uint32_t)c[1], bits);
  if (D == 2) return morton2_key((uint32_t)c[0], (uint32_t)c[1]);
  return morton3_key((uint32_t)c[0], (uint32_t)c[1], (uint32_t)c[2]);
}

}  // namespace psi

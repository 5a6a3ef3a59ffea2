// common.cuh -- internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/psi.h"

namespace psi {

// ---------------------------------------------------------------------------
// Device status word (one per index / per call): bits OR-ed by kernels.
// ---------------------------------------------------------------------------
enum : int { ST_RANGE = 1, ST_TIMEOUT = 2, ST_STACK = 4 };

constexpr int kWarp = 32;
constexpr int kMaxLeaf = 64;        // leaf_size upper bound
constexpr int kMaxNodeFanout = 32;  // children per node (SPaC summary fanout; P-Orth <= 8)

// Bounded spin: iterations of a device-side wait before it reports ST_TIMEOUT.
constexpr uint32_t kSpinLimit = 1u << 22;

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// (key, id) lexicographic order
// Adds the sum of v over all threads of the block to *ctr with one global
// atomic (a counter every thread would otherwise hit serialises in L2).  Every
// thread of the block must call it; blockDim.x is a multiple of 32.
__device__ __forceinline__ void block_count_add(unsigned long long *ctr, uint32_t v) {
  __shared__ unsigned long long s_sum;
  if (threadIdx.x == 0) s_sum = 0;
  __syncthreads();
  const uint32_t w = __reduce_add_sync(0xFFFFFFFFu, v);
  if ((threadIdx.x & 31) == 0 && w) atomicAdd(&s_sum, (unsigned long long)w);
  __syncthreads();
  if (threadIdx.x == 0 && s_sum) atomicAdd(ctr, s_sum);
}

__device__ __forceinline__ bool kid_less(uint64_t ka, uint32_t ia, uint64_t kb, uint32_t ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// ---------------------------------------------------------------------------
// Host-side error plumbing
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
psi_status cuda_fail(cudaError_t e, const char *what);

#define PSI_CK(call)                                      \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return ::psi::cuda_fail(e_, #call); \
  } while (0)

// Launch bookkeeping: counts every kernel launch and, when profiling is on,
// brackets it with CUDA events on its stream.
struct LaunchScope {
  LaunchScope(const char *name, cudaStream_t s);
  ~LaunchScope();
  const char *name;
  cudaStream_t s;
  int slot;
};

#define PSI_LAUNCH(kernel, grid, block, smem, stream, ...)          \
  do {                                                              \
    ::psi::LaunchScope ls_(#kernel, stream);                        \
    kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);     \
  } while (0)

#define PSI_LAUNCH_NAMED(name, kernel, grid, block, smem, stream, ...) \
  do {                                                                 \
    ::psi::LaunchScope ls_(name, stream);                              \
    kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);        \
  } while (0)

// ---------------------------------------------------------------------------
// Stream-ordered device buffers
// ---------------------------------------------------------------------------
struct DevMem {
  static psi_status alloc(void **p, size_t bytes, cudaStream_t s);
  static void free(void *p, cudaStream_t s);
};

template <class T>
struct Buf {
  T *p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  Buf() = default;
  Buf(const Buf &) = delete;
  Buf &operator=(const Buf &) = delete;
  ~Buf() { release(); }
  psi_status alloc(size_t count, cudaStream_t st) {
    release();
    s = st;
    n = count;
    if (count == 0) return PSI_OK;
    return DevMem::alloc((void **)&p, sizeof(T) * count, st);
  }
  void release() {
    if (p) DevMem::free(p, s);
    p = nullptr;
    n = 0;
  }
  T *take() {
    T *q = p;
    p = nullptr;
    n = 0;
    return q;
  }
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

int num_sms();

// ---------------------------------------------------------------------------
// Encoding spec: how the first sort pass computes keys from points.
// ---------------------------------------------------------------------------
enum CurveKind : int { CURVE_MORTON = 0, CURVE_HILBERT = 1 };

struct EncodeSpec {
  const int32_t *pts = nullptr;  // [n][dim]
  int dim = 2;
  int curve = CURVE_MORTON;
  int bits = 30;
  int key_shift = 0;  // keys are (curve key >> key_shift): sort by the top bits only
};

// Sort workspace: ping-pong key/value buffers plus look-back and histograms.
struct SortResult {
  uint64_t *keys;
  uint32_t *vals;
  int prefix_low = 0;  // > 0: sorted by key bits [prefix_low, key_bits) only (then runs fixed up)
  // encoding sorts that counted input locality: 1 when at least half of the
  // input neighbours share their top 24 key bits, 0 when not; -1 not counted
  int local = -1;
};

// Sorts n pairs.  If enc.pts is non-null the keys are computed from the points
// on first touch and the values are the input positions 0..n-1; otherwise the
// pairs (keys_in, vals_in) are sorted.  key_bits limits the digits sorted.
// When tie_ids is non-null, runs of equal keys are re-ordered so that
// tie_ids[value] increases (values are positions into tie_ids).
// The result lives in one of the two caller-provided buffer pairs.
psi_status sort_pairs(const EncodeSpec &enc, const uint64_t *keys_in, const uint32_t *vals_in, int64_t n,
                      int key_bits, const uint32_t *tie_ids, uint64_t *kbuf0, uint32_t *vbuf0, uint64_t *kbuf1,
                      uint32_t *vbuf1, int *d_status, cudaStream_t s, SortResult *out, int radix_bits = 0);

// Device-wide exclusive scan of int64 values (out may alias in); writes the
// grand total to d_total if non-null.
psi_status scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *d_total, cudaStream_t s);
psi_status scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, int64_t *d_total, cudaStream_t s);

}  // namespace psi

// api.cu -- the C ABI (include/psi.h): argument checks, index lifetime,
// stream-ordered memory, error reporting and launch instrumentation.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "index.cuh"

namespace psi {

psi_status run_knn(const psi_index *ix, const int32_t *q, int64_t nq, int k, uint32_t *out_id, int64_t *out_d2,
                   unsigned long long *d_stats, cudaStream_t s);
psi_status run_range_count(const psi_index *ix, const int32_t *boxes, int64_t nq, int64_t *counts, cudaStream_t s);
psi_status run_range_emit(const psi_index *ix, const int32_t *boxes, int64_t nq, const int64_t *offsets,
                          uint32_t *ids, bool sorted, cudaStream_t s);
psi_status export_leaves(const psi_index *ix, int32_t *counts, int32_t *lo, int32_t *hi, uint64_t *sk, uint32_t *si,
                         cudaStream_t s);
psi_status export_points(const psi_index *ix, int32_t *pts, uint32_t *ids, uint64_t *keys, int32_t *leaf,
                         cudaStream_t s);
psi_status export_nodes(const psi_index *ix, int32_t *depth, uint64_t *prefix, int64_t *count, int32_t *lo,
                        int32_t *hi, int32_t *is_leaf, cudaStream_t s);
int64_t summary_capacity(int64_t L, int F);
psi_status spac_build_fresh(psi_index *ix, const int32_t *pts, const uint32_t *ids, int64_t n, cudaStream_t s);

// ---- errors ----------------------------------------------------------------
static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

psi_status cuda_fail(cudaError_t e, const char *what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return PSI_ERR_OOM;
  return PSI_ERR_CUDA;
}

// ---- memory ----------------------------------------------------------------
static std::mutex g_pool_mu;
static std::vector<int> g_pool_ready;

psi_status DevMem::alloc(void **p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (bytes == 0) return PSI_OK;
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> g(g_pool_mu);
    if ((int)g_pool_ready.size() <= dev) g_pool_ready.resize(dev + 1, 0);
    if (!g_pool_ready[dev]) {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      }
      g_pool_ready[dev] = 1;
    }
  }
  cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    char buf[128];
    snprintf(buf, sizeof buf, "device allocation of %zu bytes failed (%s)", bytes, cudaGetErrorString(e));
    g_err = buf;
    return PSI_ERR_OOM;
  }
  return PSI_OK;
}

void DevMem::free(void *p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cached[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

// ---- launch instrumentation ----------------------------------------------------
static std::atomic<int64_t> g_launches{0};
static std::atomic<int> g_profiling{0};
struct ProfRec {
  const char *name;
  cudaEvent_t a, b;
};
static std::mutex g_prof_mu;
static std::vector<ProfRec> g_prof;
static std::vector<cudaEvent_t> g_event_pool;

static cudaEvent_t get_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

LaunchScope::LaunchScope(const char *nm, cudaStream_t st) : name(nm), s(st), slot(-1) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (g_profiling.load(std::memory_order_relaxed)) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    ProfRec r{name, get_event(), get_event()};
    cudaEventRecord(r.a, s);
    g_prof.push_back(r);
    slot = (int)g_prof.size() - 1;
  }
}

LaunchScope::~LaunchScope() {
  if (slot >= 0) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    cudaEventRecord(g_prof[slot].b, s);
  }
}

}  // namespace psi

using namespace psi;

static psi_status check_status_word(psi_index *ix, cudaStream_t s) {
  int h = 0;
  PSI_CK(cudaMemcpyAsync(&h, ix->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaStreamSynchronize(s));
  if (h) PSI_CK(cudaMemsetAsync(ix->d_status, 0, sizeof(int), s));
  if (h & ST_RANGE) {
    set_error("a coordinate lies outside [0, 2^coord_bits)");
    return PSI_ERR_RANGE;
  }
  if (h & ST_TIMEOUT) {
    set_error("a bounded device-side wait timed out");
    return PSI_ERR_DEVICE_TIMEOUT;
  }
  if (h & ST_STACK) {
    set_error("query traversal stack overflow");
    return PSI_ERR_CUDA;
  }
  return PSI_OK;
}

static psi_status validate_cfg(const psi_config *c) {
  if (!c) {
    set_error("null config");
    return PSI_ERR_INVALID;
  }
  if (c->dim != 2 && c->dim != 3) {
    set_error("dim must be 2 or 3");
    return PSI_ERR_INVALID;
  }
  if (c->kind < PSI_SPAC_Z || c->kind > PSI_PORTH) {
    set_error("unknown index kind");
    return PSI_ERR_INVALID;
  }
  if (c->leaf_size < 1 || c->leaf_size > kMaxLeaf) {
    set_error("leaf_size must be in [1, 64]");
    return PSI_ERR_INVALID;
  }
  const int maxb = c->dim == 2 ? 31 : 21;
  if (c->coord_bits < 1 || c->coord_bits > maxb) {
    set_error(c->dim == 2 ? "coord_bits must be in [1, 31] in 2D" : "coord_bits must be in [1, 21] in 3D");
    return PSI_ERR_INVALID;
  }
  if (c->fanout != 0 && (c->fanout < 2 || c->fanout > 32)) {
    set_error("fanout must be 0 (default 32) or in [2, 32]");
    return PSI_ERR_INVALID;
  }
  if (c->radix_bits != 0 && c->radix_bits != 8 && c->radix_bits != 10 && c->radix_bits != 11) {
    set_error("radix_bits must be 0 (8), 8, 10 or 11");
    return PSI_ERR_INVALID;
  }
  return PSI_OK;
}

static void destroy_index(psi_index *ix) {
  if (!ix) return;
  cudaStream_t s = ix->last_stream;
  free_pool(ix->pool, s);
  free_nodes(ix->nodes, s);
  DevMem::free(ix->sep_key, s);
  DevMem::free(ix->sep_id, s);
  DevMem::free(ix->leaf_node, s);
  free_pleaves(ix->pl, s);
  DevMem::free(ix->d_status, s);
  delete ix;
}

extern "C" {

psi_status psi_build(const psi_config *cfg, const int32_t *d_pts, const uint32_t *d_ids, int64_t n, void *stream,
                     psi_index **out) {
  g_err.clear();
  if (!out) {
    set_error("null output handle");
    return PSI_ERR_INVALID;
  }
  *out = nullptr;
  psi_status st = validate_cfg(cfg);
  if (st) return st;
  if (n < 0 || (n > 0 && (!d_pts || !d_ids))) {
    set_error("n < 0 or null input");
    return PSI_ERR_INVALID;
  }
  if (n >= (1ll << 30)) {
    set_error("at most 2^30 - 1 points per index");
    return PSI_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  psi_index *ix = new psi_index();
  ix->cfg = *cfg;
  ix->D = cfg->dim;
  ix->phi = cfg->leaf_size;
  ix->C = 2 * cfg->leaf_size;
  ix->F = cfg->fanout ? cfg->fanout : 32;
  ix->curve = cfg->kind == PSI_SPAC_H ? CURVE_HILBERT : CURVE_MORTON;
  ix->key_bits = cfg->dim * cfg->coord_bits;
  ix->last_stream = s;
  cudaGetDevice(&ix->device);
  if ((st = DevMem::alloc((void **)&ix->d_status, sizeof(int), s))) {
    destroy_index(ix);
    return st;
  }
  cudaError_t e = cudaMemsetAsync(ix->d_status, 0, sizeof(int), s);
  if (e != cudaSuccess) {
    destroy_index(ix);
    return cuda_fail(e, "cudaMemsetAsync");
  }
  if (cfg->kind == PSI_PORTH) {
    st = porth_build(ix, d_pts, d_ids, n, s);
  } else {
    st = spac_build_fresh(ix, d_pts, d_ids, n, s);
  }
  if (st) {
    destroy_index(ix);
    return st;
  }
  *out = ix;
  return PSI_OK;
}

psi_status psi_insert_batch(psi_index *ix, const int32_t *d_pts, const uint32_t *d_ids, int64_t m, void *stream) {
  g_err.clear();
  if (!ix || m < 0 || (m > 0 && (!d_pts || !d_ids))) {
    set_error("invalid insert arguments");
    return PSI_ERR_INVALID;
  }
  if (ix->n + m >= (1ll << 30)) {
    set_error("at most 2^30 - 1 points per index");
    return PSI_ERR_INVALID;
  }
  if (m == 0) return PSI_OK;
  cudaStream_t s = (cudaStream_t)stream;
  ix->last_stream = s;
  return ix->cfg.kind == PSI_PORTH ? porth_insert(ix, d_pts, d_ids, m, s) : spac_insert(ix, d_pts, d_ids, m, s);
}

psi_status psi_delete_batch(psi_index *ix, const int32_t *d_pts, const uint32_t *d_ids, int64_t m,
                            int64_t *d_num_deleted, void *stream) {
  g_err.clear();
  if (!ix || m < 0 || (m > 0 && (!d_pts || !d_ids))) {
    set_error("invalid delete arguments");
    return PSI_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  ix->last_stream = s;
  if (m == 0 || ix->n == 0) {
    if (d_num_deleted) PSI_CK(cudaMemsetAsync(d_num_deleted, 0, sizeof(int64_t), s));
    return PSI_OK;
  }
  return ix->cfg.kind == PSI_PORTH ? porth_delete(ix, d_pts, d_ids, m, d_num_deleted, s)
                                   : spac_delete(ix, d_pts, d_ids, m, d_num_deleted, s);
}

psi_status psi_knn(const psi_index *ix, const int32_t *d_q, int64_t q, int32_t k, uint32_t *d_ids, int64_t *d_d2,
                   void *stream) {
  g_err.clear();
  if (!ix || q < 0 || k < 1 || k > 128 || (q > 0 && (!d_q || !d_ids || !d_d2))) {
    set_error("invalid k-NN arguments (1 <= k <= 128)");
    return PSI_ERR_INVALID;
  }
  if (q >= (1ll << 32)) {
    set_error("at most 2^32 - 1 queries per call");
    return PSI_ERR_INVALID;
  }
  return run_knn(ix, d_q, q, k, d_ids, d_d2, nullptr, (cudaStream_t)stream);
}

psi_status psi_knn_instrumented(const psi_index *ix, const int32_t *d_q, int64_t q, int32_t k, uint32_t *d_ids,
                                int64_t *d_d2, uint64_t *d_stats, void *stream) {
  g_err.clear();
  if (!ix || q < 0 || k < 1 || k > 128 || !d_stats || (q > 0 && (!d_q || !d_ids || !d_d2))) {
    set_error("invalid k-NN arguments (1 <= k <= 128)");
    return PSI_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  PSI_CK(cudaMemsetAsync(d_stats, 0, 5 * sizeof(uint64_t), s));
  return run_knn(ix, d_q, q, k, d_ids, d_d2, (unsigned long long *)d_stats, s);
}

psi_status psi_range_count(const psi_index *ix, const int32_t *d_boxes, int64_t q, int64_t *d_counts, void *stream) {
  g_err.clear();
  if (!ix || q < 0 || (q > 0 && (!d_boxes || !d_counts))) {
    set_error("invalid range-count arguments");
    return PSI_ERR_INVALID;
  }
  return run_range_count(ix, d_boxes, q, d_counts, (cudaStream_t)stream);
}

psi_status psi_range_report(const psi_index *ix, const int32_t *d_boxes, int64_t q, int64_t *d_offsets,
                            uint32_t *d_ids, int64_t capacity, int64_t *h_total, int32_t flags, void *stream) {
  g_err.clear();
  if (!ix || q < 0 || !d_offsets || (q > 0 && !d_boxes) || capacity < 0 || (capacity > 0 && !d_ids)) {
    set_error("invalid range-report arguments");
    return PSI_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  psi_status st = run_range_count(ix, d_boxes, q, d_offsets, s);
  if (st) return st;
  if ((st = scan_i64(d_offsets, d_offsets, q, d_offsets + q, s))) return st;
  int64_t total = 0;
  PSI_CK(cudaMemcpyAsync(&total, d_offsets + q, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaStreamSynchronize(s));
  if (h_total) *h_total = total;
  if (total > capacity) {
    set_error("range report: output capacity too small (see h_total)");
    return PSI_ERR_CAPACITY;
  }
  return run_range_emit(ix, d_boxes, q, d_offsets, d_ids, (flags & PSI_REPORT_SORTED) != 0, s);
}

psi_status psi_sync(psi_index *ix, void *stream) {
  g_err.clear();
  if (!ix) return PSI_ERR_INVALID;
  return check_status_word(ix, (cudaStream_t)stream);
}

psi_status psi_destroy(psi_index *ix) {
  if (!ix) return PSI_OK;
  cudaDeviceSynchronize();
  destroy_index(ix);
  PSI_CK(cudaDeviceSynchronize());
  return PSI_OK;
}

int64_t psi_size(const psi_index *ix) { return ix ? ix->n : 0; }
int64_t psi_num_leaves(const psi_index *ix) { return ix ? ix->L : 0; }
int64_t psi_num_nodes(const psi_index *ix) { return ix ? ix->nnodes : 0; }
const char *psi_last_error(void) { return g_err.c_str(); }

psi_status psi_export_leaves(const psi_index *ix, int32_t *d_counts, int32_t *d_lo, int32_t *d_hi,
                             uint64_t *d_sep_key, uint32_t *d_sep_id, void *stream) {
  if (!ix) return PSI_ERR_INVALID;
  return export_leaves(ix, d_counts, d_lo, d_hi, d_sep_key, d_sep_id, (cudaStream_t)stream);
}

psi_status psi_export_points(const psi_index *ix, int32_t *d_pts, uint32_t *d_ids, uint64_t *d_keys, int32_t *d_leaf,
                             void *stream) {
  if (!ix) return PSI_ERR_INVALID;
  return export_points(ix, d_pts, d_ids, d_keys, d_leaf, (cudaStream_t)stream);
}

psi_status psi_export_nodes(const psi_index *ix, int32_t *d_depth, uint64_t *d_prefix, int64_t *d_count,
                            int32_t *d_lo, int32_t *d_hi, int32_t *d_is_leaf, void *stream) {
  if (!ix) return PSI_ERR_INVALID;
  return export_nodes(ix, d_depth, d_prefix, d_count, d_lo, d_hi, d_is_leaf, (cudaStream_t)stream);
}

psi_status psi_encode(const psi_config *cfg, const int32_t *d_pts, int64_t n, uint64_t *d_keys, void *stream);

psi_status psi_sort_pairs(uint64_t *d_keys, uint32_t *d_vals, int64_t n, int32_t key_bits, void *stream) {
  g_err.clear();
  if (n < 0 || (n > 0 && (!d_keys || !d_vals)) || key_bits < 1 || key_bits > 64) {
    set_error("invalid sort arguments");
    return PSI_ERR_INVALID;
  }
  if (n == 0) return PSI_OK;
  cudaStream_t s = (cudaStream_t)stream;
  Buf<uint64_t> k1, k2;
  Buf<uint32_t> v1, v2;
  Buf<int> status;
  psi_status st;
  if ((st = k1.alloc(n, s)) || (st = k2.alloc(n, s)) || (st = v1.alloc(n, s)) || (st = v2.alloc(n, s)) ||
      (st = status.alloc(1, s)))
    return st;
  PSI_CK(cudaMemsetAsync(status.p, 0, sizeof(int), s));
  SortResult r;
  EncodeSpec none;
  if ((st = sort_pairs(none, d_keys, d_vals, n, key_bits, nullptr, k1.p, v1.p, k2.p, v2.p, status.p, s, &r)))
    return st;
  PSI_CK(cudaMemcpyAsync(d_keys, r.keys, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
  PSI_CK(cudaMemcpyAsync(d_vals, r.vals, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
  int h = 0;
  PSI_CK(cudaMemcpyAsync(&h, status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaStreamSynchronize(s));
  if (h & ST_TIMEOUT) {
    set_error("a bounded device-side wait timed out");
    return PSI_ERR_DEVICE_TIMEOUT;
  }
  return PSI_OK;
}

int64_t psi_launch_count(void) { return g_launches.load(); }

void psi_profile_enable(int on) { g_profiling.store(on ? 1 : 0); }

void psi_profile_reset(void) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  cudaDeviceSynchronize();
  for (auto &r : g_prof) {
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_prof.clear();
}

int psi_profile_read(const char *name, int64_t *launches, double *total_ms) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  cudaDeviceSynchronize();
  int64_t c = 0;
  double t = 0;
  for (auto &r : g_prof) {
    if (strcmp(r.name, name) != 0) continue;
    float ms = 0;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) t += ms;
    ++c;
  }
  if (launches) *launches = c;
  if (total_ms) *total_ms = t;
  return c > 0 ? 0 : -1;
}

int psi_profile_dump(char *buf, int64_t cap) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  cudaDeviceSynchronize();
  std::map<std::string, std::pair<int64_t, double>> agg;
  for (auto &r : g_prof) {
    float ms = 0;
    cudaEventElapsedTime(&ms, r.a, r.b);
    auto &e = agg[r.name];
    e.first++;
    e.second += ms;
  }
  std::string out;
  char line[256];
  for (auto &kv : agg) {
    snprintf(line, sizeof line, "%s %lld %.6f\n", kv.first.c_str(), (long long)kv.second.first, kv.second.second);
    out += line;
  }
  if (buf && cap > 0) {
    strncpy(buf, out.c_str(), (size_t)cap - 1);
    buf[cap - 1] = 0;
  }
  return (int)out.size();
}

}  // extern "C"

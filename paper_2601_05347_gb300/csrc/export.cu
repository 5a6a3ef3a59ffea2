// export.cu -- inspection entry points (leaf list, points, nodes) and the
// standalone curve-key encoder.
#include "index.cuh"
#include "keys.cuh"

namespace psi {
namespace {

struct LeafOut {
  int32_t *counts, *lo, *hi;
  uint64_t *sk;
  uint32_t *si;
};

// Leaf i of the key-ordered leaf list is node leaf_node[i] (P-Orth) or node i (SPaC).
__global__ void k_export_leaves(TreeView t, const int32_t *leaf_node, const uint64_t *sep_key,
                                const uint32_t *sep_id, const int32_t *depth, const uint64_t *prefix, int D, int bits,
                                int64_t L, LeafOut o) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t nd = leaf_node ? leaf_node[i] : i;
    if (o.counts) o.counts[i] = t.cnt[nd];
    for (int d = 0; d < D; ++d) {
      if (o.lo) o.lo[i * D + d] = t.lo[d][nd];
      if (o.hi) o.hi[i * D + d] = t.hi[d][nd];
    }
    if (leaf_node) {
      const int sh = D * (bits - depth[nd]);
      if (o.sk) o.sk[i] = sh >= 64 ? 0 : (prefix[nd] << sh);
      if (o.si) o.si[i] = 0;
    } else {
      if (o.sk) o.sk[i] = sep_key[i];
      if (o.si) o.si[i] = sep_id[i];
    }
  }
}

__global__ void k_leaf_counts(TreeView t, const int32_t *leaf_node, int64_t L, int64_t *cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (int64_t)gridDim.x * blockDim.x)
    cnt[i] = t.cnt[leaf_node ? leaf_node[i] : i];
}

__global__ void k_export_points(TreeView t, const uint64_t *pkey, const int32_t *leaf_node, const int64_t *off,
                                int64_t L, int D, int32_t *pts, uint32_t *ids, uint64_t *keys, int32_t *leaf) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < L; i += warps) {
    const int64_t nd = leaf_node ? leaf_node[i] : i;
    const uint32_t s0 = t.ref[nd];
    const int cnt = t.cnt[nd];
    for (int s = lane; s < cnt; s += 32) {
      const int64_t o = off[i] + s;
      for (int d = 0; d < D; ++d)
        if (pts) pts[o * D + d] = t.px[d][s0 + s];
      if (ids) ids[o] = t.pid[s0 + s];
      if (keys) keys[o] = pkey[s0 + s];
      if (leaf) leaf[o] = (int32_t)i;
    }
  }
}

__global__ void k_export_nodes(TreeView t, const int32_t *ndepth, const uint64_t *nprefix, int64_t N, int D,
                               int32_t *depth, uint64_t *prefix, int64_t *count, int32_t *lo, int32_t *hi,
                               int32_t *is_leaf) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    if (depth) depth[i] = ndepth[i];
    if (prefix) prefix[i] = nprefix ? nprefix[i] : 0;
    if (count) count[i] = t.cnt[i];
    for (int d = 0; d < D; ++d) {
      if (lo) lo[i * D + d] = t.lo[d][i];
      if (hi) hi[i * D + d] = t.hi[d][i];
    }
    if (is_leaf) is_leaf[i] = t.kids[i] == 0;
  }
}

template <int D, int CURVE>
__global__ void k_encode(const int32_t *pts, int64_t n, int bits, uint64_t *keys, int *status) {
  __shared__ alignas(16) uint8_t htab[kCurveTabBytes];
  curve_table_init<D, CURVE>(htab);
  __syncthreads();
  bool bad_any = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t c[D];
#pragma unroll
    for (int d = 0; d < D; ++d) c[d] = pts[i * D + d];
    bool bad;
    keys[i] = point_key<D, CURVE>(htab, c, bits, bad);
    bad_any |= bad;
  }
  if (bad_any) atomicOr(status, ST_RANGE);
}

int grid_for(int64_t n, int threads = 256) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, threads), (int64_t)num_sms() * 16));
}

}  // namespace

psi_status export_leaves(const psi_index *ix, int32_t *counts, int32_t *lo, int32_t *hi, uint64_t *sk, uint32_t *si,
                         cudaStream_t s) {
  if (ix->L == 0) return PSI_OK;
  LeafOut o{counts, lo, hi, sk, si};
  const bool porth = ix->cfg.kind == PSI_PORTH;
  PSI_LAUNCH(k_export_leaves, grid_for(ix->L), 256, 0, s, ix->view(), porth ? ix->leaf_node : nullptr, ix->sep_key,
             ix->sep_id, ix->nodes.depth, ix->nodes.prefix, ix->D, ix->cfg.coord_bits, ix->L, o);
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}

psi_status export_points(const psi_index *ix, int32_t *pts, uint32_t *ids, uint64_t *keys, int32_t *leaf,
                         cudaStream_t s) {
  if (ix->L == 0) return PSI_OK;
  const bool porth = ix->cfg.kind == PSI_PORTH;
  const int32_t *ln = porth ? ix->leaf_node : nullptr;
  Buf<int64_t> off;
  psi_status st = off.alloc(ix->L, s);
  if (st) return st;
  PSI_LAUNCH(k_leaf_counts, grid_for(ix->L), 256, 0, s, ix->view(), ln, ix->L, off.p);
  if ((st = scan_i64(off.p, off.p, ix->L, nullptr, s))) return st;
  PSI_LAUNCH(k_export_points, grid_for(ix->L * 32), 256, 0, s, ix->view(), ix->pool.pkey, ln, off.p, ix->L, ix->D,
             pts, ids, keys, leaf);
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}

psi_status export_nodes(const psi_index *ix, int32_t *depth, uint64_t *prefix, int64_t *count, int32_t *lo,
                        int32_t *hi, int32_t *is_leaf, cudaStream_t s) {
  if (ix->nnodes == 0) return PSI_OK;
  PSI_LAUNCH(k_export_nodes, grid_for(ix->nnodes), 256, 0, s, ix->view(), ix->nodes.depth, ix->nodes.prefix,
             ix->nnodes, ix->D, depth, prefix, count, lo, hi, is_leaf);
  PSI_CK(cudaGetLastError());
  return PSI_OK;
}

}  // namespace psi

using namespace psi;

extern "C" psi_status psi_encode(const psi_config *cfg, const int32_t *d_pts, int64_t n, uint64_t *d_keys,
                                 void *stream) {
  if (!cfg || n < 0 || (n > 0 && (!d_pts || !d_keys)) || (cfg->dim != 2 && cfg->dim != 3) ||
      cfg->coord_bits < 1 ||
      cfg->coord_bits > (cfg->dim == 2 ? 31 : 21)) {
    set_error("invalid encode arguments");
    return PSI_ERR_INVALID;
  }
  if (n == 0) return PSI_OK;
  cudaStream_t s = (cudaStream_t)stream;
  Buf<int> status;
  psi_status st = status.alloc(1, s);
  if (st) return st;
  PSI_CK(cudaMemsetAsync(status.p, 0, sizeof(int), s));
  const int g = grid_for(n);
  if (cfg->dim == 3 && cfg->kind == PSI_SPAC_H)
    PSI_LAUNCH_NAMED("k_encode", (k_encode<3, 1>), g, 256, 0, s, d_pts, n, cfg->coord_bits, d_keys, status.p);
  else if (cfg->dim == 3)
    PSI_LAUNCH_NAMED("k_encode", (k_encode<3, 0>), g, 256, 0, s, d_pts, n, cfg->coord_bits, d_keys, status.p);
  else if (cfg->kind == PSI_SPAC_H)
    PSI_LAUNCH_NAMED("k_encode", (k_encode<2, 1>), g, 256, 0, s, d_pts, n, cfg->coord_bits, d_keys, status.p);
  else
    PSI_LAUNCH_NAMED("k_encode", (k_encode<2, 0>), g, 256, 0, s, d_pts, n, cfg->coord_bits, d_keys, status.p);
  int h = 0;
  PSI_CK(cudaMemcpyAsync(&h, status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  PSI_CK(cudaStreamSynchronize(s));
  if (h & ST_RANGE) {
    set_error("a coordinate lies outside [0, 2^coord_bits)");
    return PSI_ERR_RANGE;
  }
  return PSI_OK;
}

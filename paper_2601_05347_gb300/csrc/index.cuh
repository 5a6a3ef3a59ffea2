// index.cuh -- device layout of an index.
//
// Points live in a pool of leaf blocks, structure of arrays: coordinate d of
// slot s is px[d][s], its id pid[s], its curve key pkey[s].  A SPaC leaf owns
// one block of C = 2*phi slots (a freshly built leaf fills phi of them; the
// rest absorb unsorted appends, Algorithm 4 line "append and mark unsorted").
// A P-Orth leaf owns a contiguous run of slots of any length (a single cell at
// full depth may hold more than phi duplicates).
//
// Tree nodes are stored as structure of arrays too, so that a warp reading the
// children of one node (lane = child) reads contiguous memory:
//   lo[d][i], hi[d][i]  tight bounding box (lower-left, upper-right corner)
//   cnt[i]              points in the subtree
//   ref[i]              leaf: first pool slot; internal: first child node
//   kids[i]             0 for a leaf, else number of children (contiguous)
// SPaC: nodes [0, L) are the leaves in key order, then each summary level, the
// root last.  P-Orth: nodes level by level from the root (node 0).
#pragma once
#include "common.cuh"

namespace psi {

struct TreeView {
  const int32_t *lo[3];
  const int32_t *hi[3];
  const int32_t *cnt;
  const uint32_t *ref;
  const int32_t *kids;
  const int32_t *px[3];
  const uint32_t *pid;
  int32_t root;  // -1 when empty
};

struct NodeArrays {
  int32_t *lo[3] = {nullptr, nullptr, nullptr};
  int32_t *hi[3] = {nullptr, nullptr, nullptr};
  int32_t *cnt = nullptr;
  uint32_t *ref = nullptr;
  int32_t *kids = nullptr;
  int32_t *depth = nullptr;    // P-Orth: cell depth; SPaC: level (0 = leaves)
  uint64_t *prefix = nullptr;  // P-Orth: cell prefix (child numbers, root first)
  int64_t cap = 0;
};

struct Pool {
  int32_t *px[3] = {nullptr, nullptr, nullptr};
  uint32_t *pid = nullptr;
  uint64_t *pkey = nullptr;
  int64_t cap_slots = 0;
};

// P-Orth leaf list in key order (leaf i is node leaf_node[i]): the slot range
// [ref, ref + cnt) of its points in the pool (sorted by (key, id)), its cell
// depth, the first key of its cell and its tight box.
struct PLeaves {
  uint32_t *ref = nullptr;
  int32_t *cnt = nullptr;
  int32_t *depth = nullptr;
  uint64_t *key = nullptr;
  int32_t *lo[3] = {nullptr, nullptr, nullptr};
  int32_t *hi[3] = {nullptr, nullptr, nullptr};
  int64_t cap = 0;
};

}  // namespace psi

struct psi_index {
  psi_config cfg;
  int D = 2, phi = 32, C = 64, F = 32, curve = 0, key_bits = 60;
  int device = 0;
  cudaStream_t last_stream = nullptr;

  int64_t n = 0;       // live points
  int64_t L = 0;       // leaves
  int64_t nnodes = 0;  // tree nodes, leaves included
  int32_t root = -1;
  int64_t pool_used = 0;  // SPaC: blocks handed out; P-Orth: slots handed out

  psi::Pool pool;
  psi::NodeArrays nodes;
  // SPaC leaves (= nodes [0, L)): lower end of each leaf's (key, id) range.
  uint64_t *sep_key = nullptr;
  uint32_t *sep_id = nullptr;
  // P-Orth: leaf list in key order (node ids, and the leaves' records), used
  // by updates.
  int32_t *leaf_node = nullptr;
  int64_t leaf_cap = 0;
  psi::PLeaves pl;

  int *d_status = nullptr;
  std::vector<int64_t> level_off, level_size;  // SPaC summary levels

  psi::TreeView view() const {
    psi::TreeView v;
    for (int d = 0; d < 3; ++d) {
      v.lo[d] = nodes.lo[d];
      v.hi[d] = nodes.hi[d];
      v.px[d] = pool.px[d];
    }
    v.cnt = nodes.cnt;
    v.ref = nodes.ref;
    v.kids = nodes.kids;
    v.pid = pool.pid;
    v.root = root;
    return v;
  }
};

namespace psi {
psi_status alloc_nodes(NodeArrays &a, int D, int64_t cap, bool porth, cudaStream_t s);
void free_nodes(NodeArrays &a, cudaStream_t s);
psi_status alloc_pool(Pool &p, int D, int64_t slots, cudaStream_t s);
void free_pool(Pool &p, cudaStream_t s);
// Builds the SPaC summary levels over the first L nodes (the leaves).
psi_status build_spac_summary(psi_index *ix, cudaStream_t s);
// SPaC build from sorted (key, position) pairs.
psi_status spac_from_sorted(psi_index *ix, const uint64_t *skeys, const uint32_t *svals, const int32_t *pts,
                            const uint32_t *ids, int64_t n, cudaStream_t s,
                            bool records = false);
// Points and ids as 16-byte records (x, y, z or 0, id) in input order.
psi_status pack_records(const int32_t *pts, const uint32_t *ids, int64_t n, int D, int4 *rec, cudaStream_t s);
psi_status alloc_pleaves(PLeaves &a, int D, int64_t cap, cudaStream_t s);
void free_pleaves(PLeaves &a, cudaStream_t s);
psi_status porth_build(psi_index *ix, const int32_t *pts, const uint32_t *ids, int64_t n, cudaStream_t s);
psi_status porth_insert(psi_index *ix, const int32_t *pts, const uint32_t *ids, int64_t m, cudaStream_t s);
psi_status porth_delete(psi_index *ix, const int32_t *pts, const uint32_t *ids, int64_t m, int64_t *d_deleted,
                        cudaStream_t s);
psi_status spac_insert(psi_index *ix, const int32_t *pts, const uint32_t *ids, int64_t m, cudaStream_t s);
psi_status spac_delete(psi_index *ix, const int32_t *pts, const uint32_t *ids, int64_t m, int64_t *d_deleted,
                       cudaStream_t s);
EncodeSpec encode_spec(const psi_index *ix, const int32_t *pts);

// Seed-leaf inputs of the k-NN kernel (qkey null: no seed).  qkey[i] holds
// the curve key of the i-th query in curve order (bits in qkey_mask, the key
// shifted right by key_shift).  One index: leaf j is node j and its first key
// is sep_key[j].  Many indexes: query q belongs to index qseg[q], whose leaves
// are nodes node_off[i] + [0, ceil(n_i / phi)) with n_i = off[i+1] - off[i],
// built once, so a leaf's first slot holds its smallest key pkey[ref[leaf]].
struct KnnSeed {
  const uint64_t *qkey = nullptr;
  uint64_t qkey_mask = ~0ull;
  int key_shift = 0;
  const uint64_t *sep_key = nullptr;
  int64_t L = 0;
  const int32_t *qseg = nullptr;
  const int64_t *off = nullptr;
  const int64_t *node_off = nullptr;
  int phi = 0;
  const uint64_t *pkey = nullptr;
  // scratch of nq entries (required with qkey): the seed leaf node (or slot)
  // of each query in curve order, written by the k-NN call before its search
  uint32_t *pos = nullptr;
  // P-Orth: node of each leaf of the key-ordered leaf list, whose cell base
  // keys sep_key then holds; null for SPaC, where leaf i is node i
  const int32_t *leaf_node = nullptr;
};

// k-NN of nq queries, each starting at qroot[q] (or tv.root when qroot is
// null), in the given query order; d_stats (or null) receives traversal counts;
// leaf_limit >= 0 says the leaves are exactly the nodes [0, leaf_limit);
// porth says the tree is a P-Orth (nodes mix leaf and internal children,
// leaves hold few points): popped nodes are re-checked and several small
// leaves share a k-list merge.
psi_status run_knn_roots(const TreeView &tv, const int32_t *q, int64_t nq, int k, const uint32_t *order,
                         const int32_t *qroot, int D, uint32_t *out_id, int64_t *out_d2, int *status,
                         unsigned long long *d_stats, cudaStream_t s, const KnnSeed &seed,
                         int64_t leaf_limit = -1, bool porth = false);
}  // namespace psi

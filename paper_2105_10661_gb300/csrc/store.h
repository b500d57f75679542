// Device layout of the hierarchical inverse (Sec. III) and the host object that owns it.
//
// All vectors inside the store use the tree's nested ordering: position p holds bus perm[p],
// and every tree node is a contiguous range [lo, hi) of positions.
//   leaf j        dense b_j x b_j inverse block, row-major, row stride ld_j (multiple of 4),
//                 zero padding; blocks of all leaves concatenated (leaf_off).
//   internal q    factor panel F_q, n_q x kld_q row-major (kld_q = k_q rounded up to 2):
//                 rows [0, n_l) hold P = Ginv_l h_l, rows [n_l, n_q) hold Q = Ginv_r h_r (Eq. 9);
//                 core C_q, 2k_q x 2k_q row-major: S^{-1} (EXACT) or [[0, I], [I, 0]] (PAPER).
//   cut lists     per internal node, endpoint positions (a in the left child, b in the right)
//                 and the branch conductance g_e: h_l[:, e] = -g_e e_a, h_r[:, e] = e_b.
// The FP64 master copy is what construction and modification operate on; the FF64 (float-float
// pairs) and FP32 copies are packed from it for the apply kernels.
#pragma once
#include <cstdint>
#include <memory>
#include <vector>

#include "internal.h"

namespace emt {

struct DStore {
  int n, n_node, n_leaf, max_depth, kmax;
  int cut_w;               // left entries per cut column (1, or B for block cuts: cut_a .. cut_a + B - 1)
  const int* lo;
  const int* hi;
  const int* parent;
  const int* left;
  const int* right;
  const int* depth;
  const int* node_leaf;    // node -> leaf index (-1 for internal)
  const int* leaf_node;    // leaf index -> node
  const int* pos_leaf;     // position -> leaf index
  const int* perm;         // position -> bus
  const int* ipos;         // bus -> position
  const int64_t* leaf_off;
  const int* leaf_ld;
  const int* node_k;
  const int* node_kld;
  const int64_t* node_foff;
  const int64_t* node_coff;
  const int* node_soff;    // offset of the node's 2k block in a per-vector s array
  const int* lvl_ptr;      // internal nodes grouped by depth
  const int* lvl_nodes;
  const int* cut_ptr;
  const int* cut_a;
  const int* cut_b;
  const int* cut_e;
  double* cut_g;           // [n_cut][cut_w]: h_l[cut_a + w, c] = -cut_g[c cut_w + w]
  double* L64;
  float2* Lff;
  float* L32;
  double* F64;
  float2* Fff;
  float* F32;
  double* C64;
  float2* Cff;
  float* C32;
  int* status;             // device status word
};

// Distinct cut endpoints, used by the per-step boundary sweep.
struct CutRows {
  int n_items;             // (node, endpoint) items = sum over nodes of 2 k
  std::vector<int32_t> item_node, item_pos, item_crow, item_sidx;  // item -> node, position, distinct row, slot in s
  std::vector<int32_t> crow_pos;                                   // distinct positions
};

class Store {
 public:
  Store(const emt_graph* g, const emt_hinv_opts* o, cudaStream_t s);
  ~Store();

  // construction (Algorithm 1)
  void build(cudaStream_t s);
  // G' = G + delta u u^T (Sec. IV); throws Error(EMT_ERR_SINGULAR) and leaves the store intact
  void modify(int bus_a, int bus_b, double delta, cudaStream_t s);
  // Enqueue the modification without synchronising; a singular change raises the device
  // status word and leaves the store unchanged. Returns false if the request is invalid.
  void modify_async(int bus_a, int bus_b, double delta, cudaStream_t s);
  int cut_entry(int c, int pa, int pb, int branch) const;
  void pack(cudaStream_t s);                       // refresh FF64 / FP32 copies
  int device_status(cudaStream_t s);               // sync + read status word
  void clear_status(cudaStream_t s);

  DStore view() const;

  // generic FP64 multi-vector apply of the whole tree on a row-major panel Y (n x m, ld):
  // Y <- Ginv Y, with X supplied in Y (leaf stage done from Xin into Y)
  void apply_rows_fp64(const double* Xin, double* Y, int m, int ld, cudaStream_t s);

  Tree tree;
  int device = -1;                                   // CUDA device the store was built on
  int mode, precision;
  int n;
  int n_leaf, n_internal, kmax;
  std::vector<int32_t> leaf_nodes_h, leaf_ld_h, node_leaf_h, node_k_h, node_kld_h, node_soff_h;
  std::vector<int64_t> leaf_off_h, node_foff_h, node_coff_h;
  std::vector<int32_t> lvl_ptr_h, lvl_nodes_h;
  int64_t L_elems = 0, F_elems = 0, C_elems = 0;
  int s_total = 0;                                   // sum over nodes of 2k
  // graph (host copy) for modifications and the FP64 residual
  std::vector<int32_t> g_from, g_to;
  std::vector<double> g_val;
  std::vector<int32_t> csr_ptr, csr_col;             // position-ordered CSR of G
  std::vector<double> csr_val;
  std::vector<double> cut_g_h;
  CutRows cut_rows;

  // device buffers
  DevBuf<int> d_lo, d_hi, d_parent, d_left, d_right, d_depth, d_node_leaf, d_leaf_node, d_pos_leaf,
      d_perm, d_ipos, d_leaf_ld, d_node_k, d_node_kld, d_node_soff, d_lvl_ptr, d_lvl_nodes, d_cut_ptr,
      d_cut_a, d_cut_b, d_cut_e;
  DevBuf<int64_t> d_leaf_off, d_node_foff, d_node_coff;
  DevBuf<double> d_cut_g;
  DevBuf<double> L64, F64, C64, W64;
  DevBuf<float2> Lff, Fff, Cff;
  DevBuf<float> L32, F32, C32;
  DevBuf<double> core_ws;   // workspace of core inversions too large for shared memory
  DevBuf<int> core_piv;
  DevBuf<int> d_csr_ptr, d_csr_col;
  DevBuf<double> d_csr_val;
  DevBuf<int> d_status;
  DevBuf<int> d_list, d_flag;
  DevBuf<double> scratch;                            // sweep scratch for panels
  DevBuf<double> zbuf, dbuf;                         // modification vectors and denominators
  DevBuf<int> d_item_node, d_item_pos, d_item_crow, d_item_sidx, d_crow_pos;

 private:
  void setup_layout(cudaStream_t s);
  void build_csr();
  void assemble_leaves(const std::vector<int>& leaves, cudaStream_t s);
  void invert_leaves(const std::vector<int>& leaves, cudaStream_t s);
  void form_factors(const std::vector<int>& nodes, int d, cudaStream_t s);
  void form_cores(const std::vector<int>& nodes, cudaStream_t s);
  void modify_exact(int pa, int pb, int branch, double delta, cudaStream_t s);
  void modify_paper(int pa, int pb, int branch, double delta, cudaStream_t s);
  void update_graph(int a, int b, int branch, double delta, cudaStream_t s);
  int upload_list(const std::vector<int>& v, cudaStream_t s);
};

inline int leaf_index_of_pos(const Store& st, int pos_) {
  // leaves are contiguous ranges in left-to-right order
  int lo = 0, hi = st.n_leaf - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) / 2;
    if (st.tree.lo[st.leaf_nodes_h[mid]] <= pos_) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace emt

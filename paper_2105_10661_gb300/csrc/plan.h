// Launch plan of the fused single-vector kernels for one store: which rows each CTA owns,
// the distinct cut endpoints of the boundary sweep, and the per-CTA partial buffer.
#pragma once
#include <memory>
#include <vector>

#include "step2.cuh"

namespace emt {

// Ancestor record of a leaf for the streaming expansion: F offset of the leaf's first row at
// that ancestor, its row stride, k, and the index of the half of s the leaf's rows use.
struct StreamAnc {
  long long foff;
  int kld, k, sidx, pad;
};

// Stage of the leaf stream: element offset of its first row in the store, the row stride (the
// leaf's ld), rows (1 or 2, one leaf), the x-window offset of the leaf, the leaf size, the cut-row
// indices of the rows (-1: none) and the position of the first row.
struct StreamStage {
  long long off;
  int ld, nr, xo, b, crow0, crow1, p, pad;
};

// Persistent single-launch apply (stream.cu, k_apply_persist): a CTA's rows within one leaf, and
// the slices of the factor panels those rows need, staged into the CTA's shared memory.
struct PersistSeg {
  int p0, p1;     // positions [p0, p1) of one leaf
  int f0, f1;     // factor slices [f0, f1) of the CTA's table, one per ancestor
  int xo, b, ld;  // the leaf's offset in the CTA's x window, its size and row stride
  int pad;
  long long loff; // element offset of row p0 in the packed leaf store
};
struct PersistF {
  long long src;  // element offset in the packed factor store of row p0
  int dst;        // element offset in the CTA's factor region (shared memory)
  int kld, k;     // row stride and width of the panel
  int sidx;       // index in s of the half these rows use
  int bytes, pad;
};

// Streaming apply for stores larger than the caches (stream.cu): row ranges of the persistent
// leaf-stream CTAs, the sweep image and matrix K (s = K y_cut), ancestor records for the
// expansion, and the intermediate vectors.
struct StreamApply {
  bool ready = false;
  // single-launch form: one cooperative launch of one CTA per SM (two grid-wide barriers)
  bool persist = false;              // plan fits: shared memory, co-residency
  int mode = 0;                      // 0 or 1: three kernels; 2: single launch when it fits
  int warps = 0;                     // warps per CTA of the single launch (each streams its own rows)
  int rps_req = 0;                   // requested warps per CTA (0: automatic)
  int row_elems = 0, k_bytes = 0;
  size_t smem_p = 0;
  int o_bar = 0, o_ring = 0, o_y = 0, o_crow = 0, o_perm = 0, o_vec = 0, o_tab = 0;
  DevBuf<PersistSeg> pseg;
  DevBuf<int> pseg_ptr, krow0;
  DevBuf<PersistF> pf;
  DevBuf<unsigned int> bar;          // [0] arrivals at the grid barriers, [1] CTAs done (reset by the last)
  int prec = 0, n_cta = 0, stage_elems = 0, n_crow = 0, s_total = 0, ldk = 0, n_seg = 0, max_stages = 0, n_anc = 0;
  size_t smem = 0, smem_ldg = 0;
  bool ldg = false;                  // leaf stage: plain 16-byte loads instead of the TMA ring
  ImgHeader hdr{};
  DevBuf<double> img, K, y, ycut, sv;   // 8-byte elements (FP64 or float-float pairs)
  DevBuf<int> seg_src, seg_dst, seg_len, row0, crow_of, anc_ptr, st0;
  DevBuf<StreamStage> stages;        // leaf-stream stages, grouped per CTA (st0)
  DevBuf<int2> win;                  // per CTA: x window [x, y)
  DevBuf<StreamAnc> anc;             // ancestor records, grouped per leaf (anc_ptr)
  bool build(const Store& st, cudaStream_t s);
  void refresh(const Store& st, cudaStream_t s);   // after a modification of the store
};

struct FusedPlan {
  int rows_per_cta = 0;
  int n_cta = 0;
  int pld = 0;
  int max_rows = 0;
  int s_total = 0;
  size_t smem_partial = 0;
  size_t smem_sweep = 0;
  DevBuf<int> cta_leaf, cta_r0, cta_r1, leaf_cta0, leaf_ncta;
  std::vector<int> h_cta_leaf, h_cta_r0, h_cta_r1, h_leaf_cta0, h_leaf_ncta;   // host copies
  DevBuf<int> item_pos, item_crow, item_sidx, item_cut, item_lvl, crow_pos;
  DevBuf<double> part;       // n_cta x pld entries of 8 bytes (double or float2); FP32 uses half
  DevBuf<double> cut_gn64;   // -g_e per cut, per precision
  DevBuf<float2> cut_gnff;
  DevBuf<float> cut_gn32;
  std::shared_ptr<StreamApply> sa;   // built on first use for large stores (emt_apply)
  int stream_mode = 0;               // large stores: 0 automatic (three kernels), 1 three kernels, 2 single launch
  int stream_rps = 0;                // warps per CTA of the single launch (0: automatic)
  CtaMapD cmap() const;
  CutRowsD crows() const;
};

// Build a plan (rows_per_cta <= 0 picks a default from the store size).
void make_plan(const Store& st, int rows_per_cta, FusedPlan& plan, cudaStream_t s);
// Refresh the -g_e copies after a modification.
void refresh_plan_values(const Store& st, FusedPlan& plan, cudaStream_t s);
int default_rows_per_cta(const Store& st);
bool stream_apply_wanted(const Store& st);
void stream_apply(const Store& st, StreamApply& sa, const double* src, bool src_pos, double* v_pos, double* v_bus,
                  bool accumulate, cudaStream_t s);

// One single-vector application in the store's precision.
//   src: bus-ordered input (src_pos == false) or position-ordered (true)
//   v_pos: position-ordered result (accumulate: +=); v_bus: optional bus-ordered copy
void fused_apply(const Store& st, FusedPlan& plan, const double* src, bool src_pos, double* v_pos, double* v_bus,
                 bool accumulate, cudaStream_t s);

}  // namespace emt

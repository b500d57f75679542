// Multi-column EMT stepping: R independent columns (N-1 contingencies or load/source scenarios)
// share one stored inverse and step together.
//
// Per step, for all columns at once:
//   inject    element histories and source/load injections (float-float values, compensated
//             accumulation)
//   apply     leaf stage Y = blkdiag(L_j) X as a GEMM over the R columns (tcgen05 BF16x3 with
//             FP32 accumulation in tensor memory, or FP32 SIMT tiles), boundary sweep S = K Y_cut
//             as a split-K product over the nonzero column pieces of K, expansion
//             V = Y - sum F_q S_q (tcgen05 or SIMT, float-float update of V);
//             a column whose branch has tripped adds the Sherman-Morrison term of its own
//             change, v_c -= (delta_c / d_c) z_c u_c^T y_c with z_c = Ginv u_c and the FP64
//             denominator d_c = 1 + delta_c u_c^T z_c
//   refine    residual r = x - G' v in float-float arithmetic (G' includes each column's trip),
//             a second apply of r, v += c
// The result is float-float (about 48 significant bits); one refinement pass brings the
// FP32-grade apply to within 1e-8 of the FP64 oracle. Per-column trips switch on by step number inside
// the kernels, so a whole run is a chain of CUDA graphs with no host work between steps.
#pragma once
#include <map>
#include <memory>
#include <vector>

#include "sim.h"

namespace emt {

// One element end: the element's history is kept once (per element, two buffers by step parity);
// both ends evaluate the same update from the same operands, the from-end stores it.
struct MRec {
  int other, sgn, elem, pad;   // other end's position (-1 ground), +1 at the from-end, element index
  float2 a1, beta;             // float-float alpha + beta g and beta: Ih' = a1 v_e + beta Ih
};
static_assert(sizeof(MRec) == 32, "MRec must be 32 bytes");

struct MSimD {
  int n, R, s_total, n_crow, max_depth;
  int R_act;            // columns processed (prefix of the R slots)
  const int* trip_off;  // [R] first step the change is no longer applied (INT_MAX for a trip)
  const MRec* inc;
  const int* inc_ptr;
  float2* Ih;           // [2][n_el][R] element histories; step s reads buffer (s - 1) & 1, writes s & 1
  int n_el;
  float2* V;            // [n][R]
  float2* X;            // [n][R]
  float* Xf;            // [n][R] GEMM input
  float* Y;             // [n][R] leaf-stage result
  float* S;             // [s_total][R]
  float* fcol;          // [R]
  const int* term_ptr;  // [n + 1]
  const float2* term_cs;   // [n_terms][R]
  const float2* term_sn;   // [n_terms][R]
  const float2* trig;   // [2 * steps] sin, cos (float-float)
  const int* trip_step; // [R], 0 = none
  const int* trip_elem; // [R]
  const int* trip_a;    // [R] positions
  const int* trip_b;
  const double* trip_delta;   // [R]
  const float2* trip_delta_ff;   // [R] the same as float-float
  const double* trip_coef;    // [R] delta / d
  const float2* Z;      // [n][R]
  const int* csr_ptr;
  const int* csr_col;
  const float2* csr_ff;
  const int* mon_idx;
  int n_mon;
  SimDyn* dyn;
  const int* meta;      // sweep metadata (see multi.cu)
};

// tcgen05 leaf stage (umma.cu)
struct Umma {
  bool ready = false;
  int R = 0, TN = 0, n_blocks = 0, n_tiles = 0, n_bblocks = 0;
  DevBuf<uint16_t> a_blocks, b_blocks;   // pre-tiled BF16 splits of the leaves and of the right-hand sides
  DevBuf<int4> d_tiles, b_desc;
  DevBuf<int2> tile_b;                   // (first B block, K chunks) per tile
  // expansion V = Y - F_path S_path (every leaf has ancestor rows)
  bool exp_ready = false;
  int xTN = 64, x_blocks = 0, x_tiles = 0, x_bblocks = 0;
  DevBuf<uint16_t> xa_blocks, xb_blocks; // factor paths (per store) and gathered S rows (per pass)
  DevBuf<int4> x_tiles_d, x_bdesc;
  DevBuf<int2> x_tile_b;
  void build(const Store& st, int R, cudaStream_t s, int tn = 0);
  void build_expand(const Store& st, const std::vector<int>& path_ptr_h, const int* path_ptr,
                    const long long* path_fbase, const int* path_kld, cudaStream_t s);
  void expand(const Store& st, const MSimD& m, const int* path_ptr, const int* path_srow, int pass, int n1,
              int record, int s_in_chunk, cudaStream_t s);
  void launch(const Store& st, const float* Xf, float* Y, cudaStream_t s, int r_act);
  void split(const Store& st, const float* Xf, cudaStream_t s);       // right-hand sides -> BF16 blocks
  void mma(const Store& st, float* Y, cudaStream_t s, int r_act);     // leaf products from the blocks
};

class MSim {
 public:
  MSim(const emt_network* net, const emt_hinv_opts* opts, double dt, int R, const double* src_scale,
       const double* load_scale, cudaStream_t s);
  ~MSim();
  void schedule(int step, int kind, int target, double value, int column);
  void set_monitor(int n_mon, const int32_t* buses);
  void step(int n_steps, double* record_dev, cudaStream_t s);
  void read(int what, double* host_out);
  void reset(cudaStream_t s);
  void stats(int64_t* out, int n) const;
  // 1 SIMT FP32, 2 tcgen05 BF16x3 (expansion on tcgen05 when it fills the SMs), 3 tcgen05 for both
  // products; leaf-GEMM tiles tn columns wide (0: by the column count)
  void set_gemm(int kind, int tn, cudaStream_t s);
  // injection kernel: 0 by the column count (two columns per thread when they fill whole blocks
  // of pairs), 1 one column per thread, 2, 3, 4 two columns per thread (even column counts only)
  // with 6, 3 or 2 element ends per memory round trip and 2, 3 or 4 CTAs per SM
  // ipp: positions per CTA (0: enough CTAs for about four per SM)
  void set_inject(int mode, int ipp);
  // time every candidate product kind, leaf-GEMM tile width and injection kernel on `probe_steps`
  // steps and keep the fastest (cached per network and column-count shape for this process); the
  // simulation is reset afterwards
  void autotune(int probe_steps, int* best_tn, int* best_kind, int* best_inj, cudaStream_t s);
  bool apply_cached_tuning(cudaStream_t s);
  // serving: (re)start column c as a new request at the current step, with an optional
  // per-column change (kind 0 trip of series branch `target`, kind 1 fault at bus `target` with
  // R_f = value ohm lasting `len` steps, kind -1 none) `ev_step` steps after the start
  void admit(int c, int kind, int target, double value, int ev_step, int len, cudaStream_t s);
  void set_active(int r_act);
  MSimD view() const;
  Umma umma;
  int gemm_kind = 2;

  static constexpr int kChunk = 32;
  std::unique_ptr<Store> store;
  int n = 0, R = 0, n_series = 0, n_mon = 0, cur_step = 0;
  double dt = 0, omega = 0;
  int64_t launches = 0;
  std::vector<int> el_a, el_b;
  std::vector<double> el_g;
  // device
  DevBuf<MRec> inc;
  DevBuf<int> inc_ptr, term_ptr, trip_step, trip_elem, trip_a, trip_b, mon_idx, meta, gemm_tiles, trip_off;
  DevBuf<double> term_base;   // [n_terms][2] coef cos(phi), coef sin(phi) with the column scale 1
  DevBuf<double> u_bus, z_pos;
  FusedPlan zplan;
  bool zplan_ready = false;
  int R_act = 0;
  std::vector<int> h_trip_off;
  DevBuf<float2> Ih, V, X, term_cs, term_sn, trig, Z, csr_ff, trip_dff;
  DevBuf<float> Xf, Y, S, fcol;
  DevBuf<double> trip_delta, trip_coef;
  DevBuf<SimDyn> d_dyn;
  int n_inc = 0, n_el_h = 0, n_tiles = 0, n_crow = 0, ldk = 0, n_xtiles = 0, n_sm = 1;
  size_t inj_smem = 0, res_smem = 0;   // dynamic shared memory of the injection / residual CTAs
  DevBuf<float> Kmat;                       // matrix of the sweep (FP32), S = K Y_cut
  DevBuf<int2> krange;                      // per 32-row tile of K: column range of its nonzeros
  DevBuf<float> Kt;                         // K transposed ([n_crow][ldt])
  int ldt = 0;
  DevBuf<int4> sweep_items;                 // (row tile, first column, end column, piece | pieces << 16)
  DevBuf<float> sweep_part;                 // partials of tiles cut into several pieces
  DevBuf<int> sweep_count;                  // pieces done per (row tile, column tile)
  int n_sweep_items = 0, n_ct = 0;
  std::vector<int> path_ptr_h;              // host copy of path_ptr
  DevBuf<int4> xtiles;                      // expansion tiles: leaf, first position, positions
  DevBuf<int> path_ptr, path_srow, path_kld;   // per-leaf path tables of the expansion
  DevBuf<long long> path_fbase;
  std::vector<int> h_trip_step, h_trip_elem;
  bool z_ready = false;
  bool any_change = false;   // some column has a change scheduled or admitted
  std::map<int, cudaGraphExec_t> graphs;
  cudaStream_t cap_stream = nullptr;

 private:
  void build_meta(cudaStream_t s);
  void prepare_trips(cudaStream_t s);
  void launch_steps(int n, cudaStream_t s);
  void apply_pass(int pass, int n1, int record, int s_in_chunk, cudaStream_t s);
  void launch_residual(int n1, int s_in_chunk, cudaStream_t s);
  int positions_per_cta(int cols_per_thread = 1, int ctas_per_sm = 4) const;
  void launch_inject(int s_in_chunk, cudaStream_t s);
  bool inj_pairs = false;   // two-column injection kernel (even column stride, 32-bit row indices)
  int inj_mode = 0, inj_ipp = 0;
  bool inject_pairs() const;
  int inject_variant() const;
  bool tensor_expand() const;
 public:
  void bench_kernel(int which, int reps, cudaStream_t s);
  void drop_graphs();
};

}  // namespace emt

// EMT simulation object (host) and its device view.
#pragma once
#include <deque>
#include <map>
#include <memory>
#include <utility>
#include <vector>

#include "plan.h"
#include "step2.cuh"

namespace emt {

// Sizes and required arrays of an element description, checked on the host before any device work
// (EMT_ERR_INVALID otherwise).
void check_network_arrays(const emt_network* net);

struct SimDyn {
  int step_base;   // steps completed before the current launch sequence
  int rec_first;   // step number stored at record row 0
  double* rec;     // record buffer of the current emt_step call (may be null)
  int trig_first;  // step number of row 0 of the sin/cos table
  int pad;
};

struct SimD {
  int n;
  const int* inc_ptr;      // incidences per position
  const int* inc_other;    // position of the element's other end (-1: ground)
  const int* inc_sgn;      // +1 at the element's from-bus, -1 at its to-bus
  const double* inc_g;
  const double* inc_alpha;
  const double* inc_beta;
  double* Ih;              // history source, one copy per incidence
  const int* src_ptr;
  const double* src_coef;  // Vm/Rs for sources, -amp for loads
  const double* src_phi;
  double omega, dt;
  double* v_pos;
  double* x_pos;           // right-hand side kept for the refinement residual (FP32 only)
  const int* mon_idx;
  int n_mon;
  SimDyn* dyn;
  const int* csr_ptr;
  const int* csr_col;
  const double* csr_val;
};

struct Event {
  int step, kind, target;
  double value;
  int column;
};

// Copy of the FP64 store right after construction; emt_sim_reset puts it back.
struct Snapshot {
  DevBuf<double> L, F, C, cg, cv;
  std::vector<double> g_val, csr_val, cut_g;
  void save(const Store& st, cudaStream_t s);
  void restore(Store& st, cudaStream_t s);
};

class Sim;

// Plan and device data of the second-generation step kernels (step2.cu).
struct Step2 {
  bool ready = false;
  int prec = 0;
  int max_inc = 0;
  int max_lnc = 0;
  int core_bytes = 0;
  int n_seg_copy = 0;
  size_t smem_static = 0, smem_sweep = 0, smem_partial = 0;
  ImgHeader header{};
  std::vector<IncRec> inc0;
  DevBuf<IncRec> inc;
  DevBuf<SrcRec> d_src;
  DevBuf<double2> d_src_sum;
  DevBuf<int> d_src_ptr;
  DevBuf<double> trig;
  DevBuf<float4> trigff;
  DevBuf<double> img;
  DevBuf<int> seg_src_d, seg_dst_d, seg_len_d;
  DevBuf<OwnCopy> own_d;
  bool build(const Sim& sm, cudaStream_t s, int force_prec = -1);
  void refresh(const Sim& sm, cudaStream_t s);
  void reset_state(cudaStream_t s);
  void fill_trig(const Sim& sm, int first_step, int n, cudaStream_t s);
  void open_element(int m0, int m1, cudaStream_t s);
  Step2D view(const Sim& sm) const;
};
void step2_launch_any(Sim& sm, int n, cudaStream_t s);
void step3_sweep(Sim& sm, const Step2& img, const double* ylf, int s_in_chunk, int accumulate, int record, cudaStream_t s);

// Kernel generation 3 (step3.cu): cluster-reduced leaf stage + FP64 sweep.
struct Step3 {
  bool ready = false;
  int cs = 0;                 // CTAs per leaf = cluster size
  int max_rows = 0, maxb = 0, max_inc = 0;
  size_t smem_partial = 0;
  Step2 img;                  // FP64 sweep image
  DevBuf<double> ylf;         // reduced leaf-stage values per position
  bool build(Sim& sm, int cs, cudaStream_t s);
};
void step3_launch_any(Sim& sm, int n, cudaStream_t s);

// Kernel generation 4 (step4.cu): the whole time loop in one persistent thread-block cluster.
struct Step4D {
  int C, P;         // CTAs in the cluster; most CTAs sharing one leaf
  int o_x, o_part, o_ycp, o_ycut, o_yvp, o_s, o_v, o_contrib, o_row, o_vrow, o_out, o_push, o_sx, o_K, o_L, o_F;
  int max_vrows, e_max, ldk, n_crow, fstride, s_total;
  const int* hdr;   // [C][24] per-CTA header
  const int* tab;   // per-CTA tables
  const double* K;  // [s_total][ldk] matrix of the boundary sweep (8-byte elements)
  float2* rec_ff;   // float-float record of this launch ([n_steps][n_mon]), or null
};
struct Step4 {
  bool ready = false;
  int C = 0, P = 1;
  size_t smem = 0;
  size_t o_x = 0, o_part = 0, o_ycp = 0, o_ycut = 0, o_yvp = 0, o_s = 0, o_v = 0, o_contrib = 0, o_row = 0,
         o_vrow = 0, o_out = 0, o_push = 0, o_sx = 0, o_K = 0, o_L = 0, o_F = 0;
  int max_vrows = 0, e_max = 0, ldk = 0, n_crow = 0, s_total = 0, fstride = 0;
  DevBuf<int> hdr, tab;
  DevBuf<double> K;        // s = K y_cut (FP64 or float-float pairs)
  DevBuf<float2> rec_ff;   // float-float record of one launch, converted to FP64 afterwards
  bool build(Sim& sm, int n_cta, cudaStream_t s);
  void refresh(const Sim& sm, cudaStream_t s);
  Step4D view() const;
};
void step4_launch(Sim& sm, int n, cudaStream_t s);
void step3_bench(Sim& sm, int which, int reps, cudaStream_t s);
void step2_bench(Sim& sm, int which, int reps, cudaStream_t s);

class Sim {
 public:
  Sim(const emt_network* net, const emt_hinv_opts* opts, double dt, int nrhs, const double* src_scale,
      const double* load_scale, cudaStream_t s);
  ~Sim();
  void schedule(int step, int kind, int target, double value, int column);
  void set_monitor(int n_mon, const int32_t* buses, cudaStream_t s);
  void set_rows_per_cta(int rpc, cudaStream_t s);
  void tune(int rpc, int kernels, cudaStream_t s);
  void autotune(int probe_steps, int* best_rpc, int* best_kernels, cudaStream_t s);
  bool apply_cached_tuning(cudaStream_t s);
  void choose_default_kernels(cudaStream_t s);
  void step(int n_steps, double* record_dev, cudaStream_t s);
  void read(int what, double* host_out, cudaStream_t s);
  void reset(cudaStream_t s);
  void stats(int64_t* out, int n) const;
  void bench_kernel(int which, int reps, cudaStream_t s);
  SimD view() const;

  static constexpr int kChunk = 64;
  std::unique_ptr<Store> store;
  FusedPlan plan;
  int n = 0, nrhs = 1, n_series = 0, n_mon = 0;
  double dt = 0, omega = 0;
  int cur_step = 0;
  std::vector<int> el_a, el_b;
  std::vector<double> el_g, el_alpha, el_beta;
  std::vector<std::pair<int, int>> el_inc;
  DevBuf<int> inc_ptr, inc_other, inc_sgn, src_ptr, mon_idx;
  DevBuf<double> inc_g, inc_alpha, inc_beta, Ih, src_coef, src_phi, v_pos, x_pos;
  DevBuf<SimDyn> d_dyn;
  std::vector<Event> events;
  size_t ev_cursor = 0;
  std::map<int, std::deque<double>> faults_on;   // bus -> R_f of the faults on there, oldest first
  std::map<int, cudaGraphExec_t> graphs;
  std::map<int, cudaGraphExec_t> bench_graphs;
  cudaStream_t cap_stream = nullptr;
  Snapshot base;                               // store right after construction
  DevBuf<double> inc_g0, inc_alpha0, inc_beta0;
  std::vector<double> el_g0;
  int64_t launches = 0;                        // kernels enqueued by step/reset
  double* cur_rec = nullptr;                   // record buffer of the current emt_step call
  int launches_per_step = 2;
  std::vector<std::vector<std::pair<double, double>>> src_terms;   // per position: (coef, phi)
  Step2 s2;
  Step3 s3;
  Step4 s4;
  int kernels = 2;                             // 1: first generation, 2: step2, 3: step3, 4: step4
                                               // (creation picks 4 when it fits: choose_default_kernels)
  bool use_v2() const { return kernels == 2 && s2.ready; }
  bool use_v3() const { return kernels == 3 && s3.ready && s2.ready; }
  bool use_v4() const { return kernels == 4 && s4.ready && s2.ready; }

 private:
  void run(int n_steps, cudaStream_t s);
  void check_fault_sequence(int last_step) const;
  void apply_event(const Event& ev, cudaStream_t s);
  void drop_graphs();
};

}  // namespace emt

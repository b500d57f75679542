// Three-phase EMT simulation (host object): three nodes per bus (node = 3 bus + phase), series RL
// branches coupled across their phases (3 x 3 companion admittance and history), RC branches,
// shunt capacitors and source resistances per phase, balanced sine sources and loads (phase p lags
// phase 0 by 2 pi p / 3). Every step: injection, v = G^-1 i with the node store (Eq. 2), history
// update. A line trip opens all three phases: exact local updates of the store (Sec. IV), one per
// node branch of the line.
#pragma once
#include <deque>
#include <map>
#include <memory>
#include <vector>

#include "plan.h"
#include "sim.h"

namespace emt {

// The node-branch graph of a three-phase network (see emt_build_hinv_from_network3); br_ptr (may
// be null) receives, per series branch, the range of its node branches in the lists.
void network_graph3(const emt_network* net, const double* L_mut, double dt, std::vector<int32_t>& gf,
                    std::vector<int32_t>& gt, std::vector<double>& gv, std::vector<int>* br_ptr = nullptr);

struct Sim3Dyn {
  int k;               // step of the current emt_step call (row of the trig table and the record)
  int pad;
  double* rec;         // record buffer of the current call ([n_steps][n_mon]), may be null
  const double* trig;  // [n_steps][2]: sin and cos of omega t of the call's steps
};

class Sim3 {
 public:
  Sim3(const emt_network* net, const double* L_mut, const emt_hinv_opts* opts, double dt, cudaStream_t s);
  ~Sim3();
  void schedule(int step, int kind, int target, double value, int column);
  void set_monitor(int n_mon, const int32_t* nodes);
  void step(int n_steps, double* record_dev, cudaStream_t s);
  void read(int what, double* host_out);
  void reset(cudaStream_t s);
  void stats(int64_t* out, int n) const;

  std::unique_ptr<Store> store;
  FusedPlan plan;
  int nb = 0, nn = 0, n_br = 0, n_mon = 0, cur_step = 0;
  double dt = 0, omega = 0;
  int64_t launches = 0;

 private:
  void run(int n_steps, cudaStream_t s);
  void launch_step(cudaStream_t s);
  void apply_trip(int e, cudaStream_t s);
  void apply_event(const Event& ev, cudaStream_t s);
  void check_fault_sequence(int last_step) const;
  void drop_graphs();

  std::vector<int32_t> gf_, gt_;
  std::vector<double> gv_;
  std::vector<int> br_ptr_, active_h_;
  std::vector<Event> events_;
  std::map<int, std::deque<double>> faults_on_;   // node -> R_f of the faults on, oldest first
  size_t ev_cursor_ = 0;
  Snapshot base_;
  DevBuf<int> br_a_, br_b_, br_sgn_, active_, inc_ptr_, inc_br_, inc_sgn_, term_ptr_, mon_;
  DevBuf<double> brY_, brH_, Ih_, gsh_, Ihsh_, term_cs_, term_sn_, rhs_, v_bus_, v_pos_, trig_;
  DevBuf<Sim3Dyn> dyn_;
  std::vector<std::pair<int, cudaGraphExec_t>> graphs_;
  cudaStream_t cap_stream_ = nullptr;
};

}  // namespace emt

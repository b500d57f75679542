// Three-phase EMT time stepping on the GPU (see sim3.h). Per step, three kernels around the node
// store's single-vector apply:
//   k3_rhs   i(t) of Eq. 1 per node: balanced sources and loads, minus the shunt histories, minus
//            (at the from-bus) / plus (at the to-bus) the branch histories of the node's phase;
//   apply    v = G^-1 i with the fused kernels of the store (Eq. 2);
//   k3_hist  per series branch the trapezoidal update of its 3-vector history: with the companion
//            admittance Y and H = (2/dt) L3 - R I (RL) or (dt/2C - R) I (RC),
//            i = Y v_e + I_h,  I_h <- s Y (v_e + H i),  s = +1 (RL) or -1 (RC); per node the shunt
//            capacitor's I_h <- -2 g v - I_h; the monitored node voltages of the step.
// Runs of up to kChunk steps between events are captured as CUDA graphs. Element arithmetic is
// FP64 (a few operations per node and branch per step); the apply runs in the store's precision.
#include <algorithm>
#include <cmath>
#include <deque>
#include <map>

#include "sim3.h"

namespace emt {

namespace {

constexpr int kChunk3 = 64;

__global__ void k3_set(Sim3Dyn* d, double* rec, const double* trig) {
  d->k = 0;
  d->rec = rec;
  d->trig = trig;
}
__global__ void k3_adv(Sim3Dyn* d) { d->k += 1; }
__global__ void k3_open(double* Ih, int* active, int e) {
  Ih[3 * e + 0] = 0.0;
  Ih[3 * e + 1] = 0.0;
  Ih[3 * e + 2] = 0.0;
  active[e] = 0;
}

__global__ void k3_rhs(const Sim3Dyn* __restrict__ dyn, int nn, const int* __restrict__ term_ptr,
                       const double* __restrict__ term_cs, const double* __restrict__ term_sn,
                       const double* __restrict__ Ihsh, const int* __restrict__ inc_ptr,
                       const int* __restrict__ inc_br, const int* __restrict__ inc_sgn, const double* __restrict__ Ih,
                       double* __restrict__ rhs) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const int k = dyn->k;
  const double sn = dyn->trig[2 * k], cs = dyn->trig[2 * k + 1];
  // coef sin(w t + theta) = coef cos(theta) sin(w t) + coef sin(theta) cos(w t)
  double val = 0.0;
  for (int t = term_ptr[n]; t < term_ptr[n + 1]; ++t) val += term_cs[t] * sn + term_sn[t] * cs;
  val -= Ihsh[n];
  const int bus = n / 3, p = n - 3 * bus;
  for (int i = inc_ptr[bus]; i < inc_ptr[bus + 1]; ++i) val += inc_sgn[i] * Ih[3 * inc_br[i] + p];
  rhs[n] = val;
}

__global__ void k3_hist(const Sim3Dyn* __restrict__ dyn, int n_br, const int* __restrict__ br_a,
                        const int* __restrict__ br_b, const int* __restrict__ br_sgn, const int* __restrict__ active,
                        const double* __restrict__ Y, const double* __restrict__ H, double* __restrict__ Ih,
                        const double* __restrict__ v, int nn, const double* __restrict__ gsh, double* __restrict__ Ihsh,
                        const int* __restrict__ mon, int n_mon) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_br && active[t]) {
    const int A = 3 * br_a[t], B = 3 * br_b[t];
    const double* y = Y + 9 * t;
    const double* h = H + 9 * t;
    double ve[3], cur[3], w[3];
    for (int p = 0; p < 3; ++p) ve[p] = v[A + p] - v[B + p];
    for (int p = 0; p < 3; ++p) cur[p] = y[3 * p] * ve[0] + y[3 * p + 1] * ve[1] + y[3 * p + 2] * ve[2] + Ih[3 * t + p];
    for (int p = 0; p < 3; ++p) w[p] = ve[p] + h[3 * p] * cur[0] + h[3 * p + 1] * cur[1] + h[3 * p + 2] * cur[2];
    const double sg = (double)br_sgn[t];
    for (int p = 0; p < 3; ++p) Ih[3 * t + p] = sg * (y[3 * p] * w[0] + y[3 * p + 1] * w[1] + y[3 * p + 2] * w[2]);
  }
  if (t < nn) Ihsh[t] = -2.0 * gsh[t] * v[t] - Ihsh[t];
  if (t < n_mon && dyn->rec) dyn->rec[(int64_t)dyn->k * n_mon + t] = v[mon[t]];
}

}  // namespace

Sim3::Sim3(const emt_network* net, const double* L_mut, const emt_hinv_opts* opts, double dt_, cudaStream_t s) {
  EMT_REQUIRE(net && opts, EMT_ERR_INVALID, "null network or options");
  EMT_REQUIRE(opts->precision == EMT_PREC_FP64 || opts->precision == EMT_PREC_FF64, EMT_ERR_UNSUPPORTED,
              "three-phase simulations need an FP64 or FF64 store");
  EMT_REQUIRE(dt_ > 0 && std::isfinite(dt_), EMT_ERR_INVALID, "dt must be > 0");
  EMT_REQUIRE(net->n_bus >= 1 && net->n_bus <= (1 << 28), EMT_ERR_INVALID, "bad network size");
  network_graph3(net, L_mut, dt_, gf_, gt_, gv_, &br_ptr_);
  nb = net->n_bus;
  nn = 3 * nb;
  n_br = net->n_branch;
  dt = dt_;
  omega = 2.0 * M_PI * net->freq;
  emt_graph g{nn, (int32_t)gf_.size(), gf_.data(), gt_.data(), gv_.data()};
  store.reset(new Store(&g, opts, s));
  store->build(s);
  EMT_REQUIRE(store->device_status(s) == DEV_OK, EMT_ERR_SINGULAR, "G is not positive definite");
  make_plan(*store, 0, plan, s);
  base_.save(*store, s);
  // series branches: 3 x 3 companion admittance Y and history matrix H (row-major), sign s
  std::vector<double> Y((size_t)9 * std::max(n_br, 1), 0.0), Hm((size_t)9 * std::max(n_br, 1), 0.0);
  std::vector<int> a(std::max(n_br, 1)), b(std::max(n_br, 1)), sg(std::max(n_br, 1));
  for (int e = 0; e < n_br; ++e) {
    a[e] = net->from[e];
    b[e] = net->to[e];
    const double R = net->R[e];
    double yd, yo, hd, ho;
    if (net->kind[e] == EMT_KIND_RL) {
      const double al = R + 2.0 * net->L[e] / dt, be = 2.0 * L_mut[e] / dt;
      const double den = (al - be) * (al + 2.0 * be);
      yd = (al + be) / den;
      yo = -be / den;
      hd = 2.0 * net->L[e] / dt - R;
      ho = be;
      sg[e] = 1;
    } else {
      yd = 1.0 / (R + dt / (2.0 * net->C[e]));
      yo = 0.0;
      hd = dt / (2.0 * net->C[e]) - R;
      ho = 0.0;
      sg[e] = -1;
    }
    for (int p = 0; p < 3; ++p)
      for (int q = 0; q < 3; ++q) {
        Y[(size_t)9 * e + 3 * p + q] = p == q ? yd : yo;
        Hm[(size_t)9 * e + 3 * p + q] = p == q ? hd : ho;
      }
  }
  br_a_.upload(a, s);
  br_b_.upload(b, s);
  br_sgn_.upload(sg, s);
  brY_.upload(Y, s);
  brH_.upload(Hm, s);
  active_h_.assign(std::max(n_br, 1), 1);
  active_.upload(active_h_, s);
  Ih_.alloc((size_t)3 * std::max(n_br, 1));
  Ih_.zero(s);
  // incidences per bus: -1 at the from-bus, +1 at the to-bus
  std::vector<int> ip(nb + 1, 0), ib, is;
  for (int e = 0; e < n_br; ++e) {
    ++ip[a[e] + 1];
    ++ip[b[e] + 1];
  }
  for (int i = 0; i < nb; ++i) ip[i + 1] += ip[i];
  ib.assign(std::max(ip[nb], 1), 0);
  is.assign(std::max(ip[nb], 1), 0);
  {
    std::vector<int> fill(ip.begin(), ip.end() - 1);
    for (int e = 0; e < n_br; ++e) {
      ib[fill[a[e]]] = e;
      is[fill[a[e]]++] = -1;
      ib[fill[b[e]]] = e;
      is[fill[b[e]]++] = 1;
    }
  }
  inc_ptr_.upload(ip, s);
  inc_br_.upload(ib, s);
  inc_sgn_.upload(is, s);
  // shunt capacitors per node
  std::vector<double> gs(nn, 0.0);
  if (net->shunt_C)
    for (int i = 0; i < nb; ++i)
      for (int p = 0; p < 3; ++p) gs[3 * i + p] = net->shunt_C[i] > 0 ? 2.0 * net->shunt_C[i] / dt : 0.0;
  gsh_.upload(gs, s);
  Ihsh_.alloc(nn);
  Ihsh_.zero(s);
  // source and load terms per node: coef sin(w t + phi - 2 pi p / 3) as (coef cos, coef sin) of the angle
  std::vector<std::vector<std::pair<double, double>>> terms(nn);
  for (int k = 0; k < net->n_src; ++k)
    for (int p = 0; p < 3; ++p) {
      const double th = net->src_phi[k] - 2.0 * M_PI * p / 3.0, c = net->src_Vm[k] / net->src_Rs[k];
      terms[3 * net->src_bus[k] + p].push_back({c * std::cos(th), c * std::sin(th)});
    }
  for (int k = 0; k < net->n_load; ++k) {
    EMT_REQUIRE(net->load_bus[k] >= 0 && net->load_bus[k] < nb, EMT_ERR_INVALID, "bad load bus");
    for (int p = 0; p < 3; ++p) {
      const double th = net->load_phi[k] - 2.0 * M_PI * p / 3.0, c = -net->load_amp[k];
      terms[3 * net->load_bus[k] + p].push_back({c * std::cos(th), c * std::sin(th)});
    }
  }
  std::vector<int> tp(nn + 1, 0);
  std::vector<double> tc, ts;
  for (int i = 0; i < nn; ++i) {
    for (auto& t : terms[i]) {
      tc.push_back(t.first);
      ts.push_back(t.second);
    }
    tp[i + 1] = (int)tc.size();
  }
  if (tc.empty()) {
    tc.push_back(0.0);
    ts.push_back(0.0);
  }
  term_ptr_.upload(tp, s);
  term_cs_.upload(tc, s);
  term_sn_.upload(ts, s);
  rhs_.alloc(nn);
  v_bus_.alloc(nn);
  v_bus_.zero(s);
  v_pos_.alloc(nn);
  mon_.alloc(1);
  dyn_.alloc(1);
  trig_.alloc(2 * kChunk3);
  EMT_CUDA(cudaMemsetAsync(dyn_.p, 0, sizeof(Sim3Dyn), s));
  EMT_CUDA(cudaStreamCreateWithFlags(&cap_stream_, cudaStreamNonBlocking));
  EMT_CUDA(cudaStreamSynchronize(s));
}

Sim3::~Sim3() {
  drop_graphs();
  if (cap_stream_) cudaStreamDestroy(cap_stream_);
}

void Sim3::drop_graphs() {
  for (auto& g : graphs_) cudaGraphExecDestroy(g.second);
  graphs_.clear();
}

void Sim3::schedule(int step, int kind, int target, double value, int column) {
  EMT_REQUIRE(step >= 1, EMT_ERR_INVALID, "event step must be >= 1");
  EMT_REQUIRE(step > cur_step, EMT_ERR_STATE, "event step already simulated");
  EMT_REQUIRE(column == -1, EMT_ERR_UNSUPPORTED, "three-phase simulations have one column");
  if (kind == EMT_EVENT_TRIP) {
    EMT_REQUIRE(target >= 0 && target < n_br, EMT_ERR_INVALID, "trip target must be a series branch");
  } else if (kind == EMT_EVENT_FAULT_ON) {
    EMT_REQUIRE(target >= 0 && target < nn, EMT_ERR_INVALID, "fault target must be a node (3 bus + phase)");
    EMT_REQUIRE(std::isfinite(value) && value > 0, EMT_ERR_INVALID, "fault resistance must be > 0");
  } else {
    EMT_REQUIRE(kind == EMT_EVENT_FAULT_OFF, EMT_ERR_INVALID, "unknown event kind");
    EMT_REQUIRE(target >= 0 && target < nn, EMT_ERR_INVALID, "fault target must be a node (3 bus + phase)");
  }
  events_.push_back({step, kind, target, kind == EMT_EVENT_FAULT_ON ? value : 0.0, -1});
  std::stable_sort(events_.begin(), events_.end(), [](const Event& x, const Event& y) { return x.step < y.step; });
}

// A fault at a node connects it to ground through R_f: FAULT_ON adds 1/R_f to G's diagonal as
// one exact local update (Sec. IV); FAULT_OFF takes the oldest fault still on at the node back
// out with the opposite update (changes made while it was on stay in G).
void Sim3::apply_event(const Event& ev, cudaStream_t s) {
  if (ev.kind == EMT_EVENT_TRIP) {
    apply_trip(ev.target, s);
    return;
  }
  double delta;
  if (ev.kind == EMT_EVENT_FAULT_ON) {
    faults_on_[ev.target].push_back(ev.value);
    delta = 1.0 / ev.value;
  } else {
    auto it = faults_on_.find(ev.target);
    EMT_REQUIRE(it != faults_on_.end() && !it->second.empty(), EMT_ERR_STATE, "fault cleared where none is on");
    delta = -1.0 / it->second.front();
    it->second.pop_front();
  }
  store->modify_async(ev.target, -1, delta, s);
  refresh_plan_values(*store, plan, s);
  launches += 2;
}

// Every FAULT_OFF up to `last_step` must find a fault on at its node (checked before any work).
void Sim3::check_fault_sequence(int last_step) const {
  std::map<int, int> on;
  for (const auto& kv : faults_on_) on[kv.first] = (int)kv.second.size();
  for (size_t i = ev_cursor_; i < events_.size() && events_[i].step <= last_step; ++i) {
    const Event& ev = events_[i];
    if (ev.step <= cur_step) continue;
    if (ev.kind == EMT_EVENT_FAULT_ON) ++on[ev.target];
    if (ev.kind == EMT_EVENT_FAULT_OFF) {
      EMT_REQUIRE(on[ev.target] > 0, EMT_ERR_STATE, "fault cleared where none is on");
      --on[ev.target];
    }
  }
}

void Sim3::set_monitor(int nm, const int32_t* nodes) {
  EMT_REQUIRE(nm >= 0 && (nm == 0 || nodes), EMT_ERR_INVALID, "bad monitor list");
  std::vector<int> m(std::max(nm, 1), 0);
  for (int k = 0; k < nm; ++k) {
    EMT_REQUIRE(nodes[k] >= 0 && nodes[k] < nn, EMT_ERR_INVALID, "monitor node out of range");
    m[k] = nodes[k];
  }
  EMT_CUDA(cudaDeviceSynchronize());
  mon_.upload(m, nullptr);
  n_mon = nm;
  drop_graphs();
  EMT_CUDA(cudaDeviceSynchronize());
}

// A three-phase line trip: every node branch of the line leaves G as one exact local update of the
// store (Sec. IV). Negative (cross-phase) node branches go first, then the positive ones within each
// end, then the phase-to-same-phase ones, so every intermediate G stays positive definite.
void Sim3::apply_trip(int e, cudaStream_t s) {
  if (!active_h_[e]) return;
  std::vector<int> order;
  for (int pass = 0; pass < 3; ++pass)
    for (int i = br_ptr_[e]; i < br_ptr_[e + 1]; ++i) {
      const int x = gf_[i], y = gt_[i];
      const bool same_bus = x / 3 == y / 3, same_phase = x % 3 == y % 3;
      const int cls = (!same_bus && !same_phase) ? 0 : (same_bus ? 1 : 2);
      if (cls == pass) order.push_back(i);
    }
  for (int i : order) store->modify_async(gf_[i], gt_[i], -gv_[i], s);
  k3_open<<<1, 1, 0, s>>>(Ih_.p, active_.p, e);
  EMT_CUDA(cudaGetLastError());
  refresh_plan_values(*store, plan, s);
  active_h_[e] = 0;
  launches += (int64_t)order.size() + 2;
}

void Sim3::launch_step(cudaStream_t s) {
  const int th = 64;
  k3_rhs<<<(nn + th - 1) / th, th, 0, s>>>(dyn_.p, nn, term_ptr_.p, term_cs_.p, term_sn_.p, Ihsh_.p, inc_ptr_.p,
                                          inc_br_.p, inc_sgn_.p, Ih_.p, rhs_.p);
  fused_apply(*store, plan, rhs_.p, false, v_pos_.p, v_bus_.p, false, s);
  const int nt = std::max({n_br, nn, n_mon});
  k3_hist<<<(nt + th - 1) / th, th, 0, s>>>(dyn_.p, n_br, br_a_.p, br_b_.p, br_sgn_.p, active_.p, brY_.p, brH_.p,
                                            Ih_.p, v_bus_.p, nn, gsh_.p, Ihsh_.p, mon_.p, n_mon);
  k3_adv<<<1, 1, 0, s>>>(dyn_.p);
  EMT_CUDA(cudaGetLastError());
}

void Sim3::run(int n_steps, cudaStream_t s) {
  int done = 0;
  while (done < n_steps) {
    const int next = cur_step + 1;
    while (ev_cursor_ < events_.size() && events_[ev_cursor_].step < next) ++ev_cursor_;
    while (ev_cursor_ < events_.size() && events_[ev_cursor_].step == next) apply_event(events_[ev_cursor_++], s);
    int stretch = n_steps - done;
    if (ev_cursor_ < events_.size()) stretch = std::min(stretch, events_[ev_cursor_].step - next);
    stretch = std::max(stretch, 1);
    int left = stretch;
    while (left >= kChunk3) {
      if (graphs_.empty()) {
        cudaGraph_t g;
        EMT_CUDA(cudaStreamBeginCapture(cap_stream_, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < kChunk3; ++k) launch_step(cap_stream_);
        EMT_CUDA(cudaStreamEndCapture(cap_stream_, &g));
        cudaGraphExec_t ge;
        EMT_CUDA(cudaGraphInstantiate(&ge, g, 0));
        cudaGraphDestroy(g);
        graphs_.push_back({kChunk3, ge});
      }
      EMT_CUDA(cudaGraphLaunch(graphs_[0].second, s));
      left -= kChunk3;
    }
    for (; left > 0; --left) launch_step(s);
    launches += (int64_t)stretch * 5;
    cur_step += stretch;
    done += stretch;
  }
}

void Sim3::step(int n_steps, double* record_dev, cudaStream_t s) {
  EMT_REQUIRE(n_steps >= 0, EMT_ERR_INVALID, "n_steps must be >= 0");
  if (n_steps == 0) return;
  check_fault_sequence(cur_step + n_steps);
  std::vector<double> tr((size_t)2 * n_steps);
  for (int k = 0; k < n_steps; ++k) {
    const double t = (double)(cur_step + 1 + k) * dt;
    tr[2 * k] = std::sin(omega * t);
    tr[2 * k + 1] = std::cos(omega * t);
  }
  if (trig_.n < tr.size()) {
    EMT_CUDA(cudaStreamSynchronize(s));
    trig_.alloc(tr.size());
  }
  EMT_CUDA(cudaMemcpyAsync(trig_.p, tr.data(), tr.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  EMT_CUDA(cudaStreamSynchronize(s));   // the host table is freed on return
  k3_set<<<1, 1, 0, s>>>(dyn_.p, n_mon > 0 ? record_dev : nullptr, trig_.p);
  EMT_CUDA(cudaGetLastError());
  launches += 1;
  run(n_steps, s);
}

void Sim3::read(int what, double* host_out) {
  if (what == 1) {
    host_out[0] = (double)cur_step;
    return;
  }
  EMT_REQUIRE(what == 0, EMT_ERR_INVALID, "unknown read selector");
  EMT_CUDA(cudaDeviceSynchronize());
  EMT_CUDA(cudaMemcpy(host_out, v_bus_.p, (size_t)nn * sizeof(double), cudaMemcpyDeviceToHost));
}

void Sim3::reset(cudaStream_t s) {
  base_.restore(*store, s);
  refresh_plan_values(*store, plan, s);
  Ih_.zero(s);
  Ihsh_.zero(s);
  v_bus_.zero(s);
  std::fill(active_h_.begin(), active_h_.end(), 1);
  active_.upload(active_h_, s);
  EMT_CUDA(cudaMemsetAsync(dyn_.p, 0, sizeof(Sim3Dyn), s));
  cur_step = 0;
  ev_cursor_ = 0;
  faults_on_.clear();
  launches += 4;
}

void Sim3::stats(int64_t* out, int n_out) const {
  const Store& st = *store;
  int64_t leaf = 0, fac = 0, core = 0;
  for (int j = 0; j < st.n_leaf; ++j) {
    const int64_t b = st.tree.hi[st.leaf_nodes_h[j]] - st.tree.lo[st.leaf_nodes_h[j]];
    leaf += b * b;
  }
  for (int q : st.lvl_nodes_h) {
    const int64_t k = st.node_k_h[q];
    fac += (int64_t)(st.tree.hi[q] - st.tree.lo[q]) * k;
    core += 4 * k * k;
  }
  const int64_t v[] = {nn, st.n_leaf, leaf, fac, core, plan.n_cta, (int64_t)gf_.size(),
                       (int64_t)st.cut_rows.crow_pos.size(), st.s_total, launches, n_br, (int64_t)gf_.size()};
  for (int i = 0; i < n_out && i < (int)(sizeof(v) / sizeof(v[0])); ++i) out[i] = v[i];
}

}  // namespace emt

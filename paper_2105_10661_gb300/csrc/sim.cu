// EMT time stepping on the GPU: per step, the history update of every element and the source
// injections form i(t) = i_in(t) + i_his(t - dt) (Sec. II, Eq. 1), the hierarchical apply gives
// v(t) = Ginv i(t) (Eq. 2), and the next step's history follows from v(t).
//
// Each step is the fused pair of kernels of the single-vector apply with the EMT work folded in:
//   partial  per owned row: update the history source of every incident element from v(t - dt)
//            (trapezoidal companion models; the state of a bus-to-bus element is kept at both of its
//            ends and both copies evolve identically), add the source/load injection, then stream
//            the owned rows of the leaf inverse;
//   sweep    boundary sweep and expansion -> v(t), monitored voltages recorded.
// FP32 stores add one refinement pass per step (residual against the FP64 G, second apply).
// Steps are launched as CUDA graphs of a fixed chunk length (the step number lives in device
// memory, so one instantiated graph serves every chunk); events split the chunks.
#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>

#include "plan.h"
#include "sim.h"

namespace emt {

namespace {

__device__ __forceinline__ double element_history(double vi, double vo, int sgn, double g, double alpha, double beta,
                                                  double& Ih) {
  // element current a -> b: i = g v_e + I_h, v_e = v_a - v_b; history for the next step
  const double ve = sgn > 0 ? vi - vo : vo - vi;
  const double cur = g * ve + Ih;
  const double Ihn = alpha * ve + beta * cur;
  Ih = Ihn;
  return sgn > 0 ? -Ihn : Ihn;   // contribution to i_his at this end
}

// First-generation partial kernel: history update and injection of the owned rows (Eq. 1), then
// the leaf stage of Eq. 2 over them.
template <int PREC>
__global__ void __launch_bounds__(kFusedThreads) k_step_partial(DStore st, CtaMapD cm, SimD sim, int s_in_chunk,
                                                                int pass, typename Acc<PREC>::X* __restrict__ part) {
  using A = Acc<PREC>;
  using X = typename A::X;
  if (*st.status != DEV_OK) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  X* xs = reinterpret_cast<X*>(smem_raw);
  X* red = xs + ((cm.max_rows + 1) & ~1);
  const int c = blockIdx.x;
  const int j = cm.cta_leaf[c];
  const int r0 = cm.cta_r0[c], r1 = cm.cta_r1[c];
  const int lo = st.lo[st.leaf_node[j]];
  const int step = sim.dyn->step_base + s_in_chunk + 1;
  for (int r = threadIdx.x; r < r1 - r0; r += blockDim.x) {
    const int pos = lo + r0 + r;
    double x;
    if (pass == 0) {
      const double t = step * sim.dt;
      double hist = 0.0;
      const double vi = sim.v_pos[pos];
      for (int m = sim.inc_ptr[pos]; m < sim.inc_ptr[pos + 1]; ++m) {
        const int o = sim.inc_other[m];
        const double vo = o >= 0 ? sim.v_pos[o] : 0.0;
        double Ih = sim.Ih[m];
        hist += element_history(vi, vo, sim.inc_sgn[m], sim.inc_g[m], sim.inc_alpha[m], sim.inc_beta[m], Ih);
        sim.Ih[m] = Ih;
      }
      double inj = 0.0;
      for (int m = sim.src_ptr[pos]; m < sim.src_ptr[pos + 1]; ++m)
        inj += sim.src_coef[m] * sin(sim.omega * t + sim.src_phi[m]);
      x = inj + hist;
      if (sim.x_pos) sim.x_pos[pos] = x;
    } else {
      // refinement: r = x - G v with the FP64 conductance matrix
      double acc = sim.x_pos[pos];
      for (int t = sim.csr_ptr[pos]; t < sim.csr_ptr[pos + 1]; ++t) acc -= sim.csr_val[t] * sim.v_pos[sim.csr_col[t]];
      x = acc;
    }
    xs[r] = A::prep(x);
  }
  __syncthreads();
  leaf_partial_core<PREC>(st, j, r0, r1, xs, part + (int64_t)c * cm.pld, red);
}

// First-generation sweep kernel: boundary sweep with Eq. 9's factors and the expansion to v(t).
template <int PREC>
__global__ void __launch_bounds__(kFusedThreads) k_step_sweep(DStore st, CtaMapD cm, CutRowsD cr, SimD sim,
                                                              int s_in_chunk, int accumulate, int record,
                                                              const typename Acc<PREC>::X* __restrict__ part,
                                                              const typename Acc<PREC>::T* __restrict__ cut_gn) {
  using A = Acc<PREC>;
  using X = typename A::X;
  if (*st.status != DEV_OK) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  X* ycut = reinterpret_cast<X*>(smem_raw);
  X* t = ycut + cr.n_crow;
  X* s = t + cr.s_total;
  boundary_sweep<PREC>(st, cm, cr, part, ycut, t, s, cut_gn);
  const int c = blockIdx.x;
  const int j = cm.cta_leaf[c];
  const int leaf_node = st.leaf_node[j];
  const int lo = st.lo[leaf_node];
  const int r0 = cm.cta_r0[c], r1 = cm.cta_r1[c];
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int step = sim.dyn->step_base + s_in_chunk + 1;
  double* rec = sim.dyn->rec;
  for (int r = r0 + warp; r < r1; r += nw) {
    const int pos = lo + r;
    const X y = leaf_y<PREC>(st, cm, part, pos);
    const X v = expand_row<PREC>(st, leaf_node, pos, y, s);
    if ((threadIdx.x & 31) == 0) {
      double out = A::todbl(v);
      if (accumulate) out += sim.v_pos[pos];
      sim.v_pos[pos] = out;
      if (record && rec) {
        const int mi = sim.mon_idx[pos];
        if (mi >= 0) rec[(int64_t)(step - sim.dyn->rec_first) * sim.n_mon + mi] = out;
      }
    }
  }
}

// Step counter of the captured graphs (the step number lives in device memory).
__global__ void k_advance(SimDyn* dyn, int n) { dyn->step_base += n; }
__global__ void k_set_dyn(SimDyn* dyn, int step_base, int rec_first, double* rec) {
  dyn->step_base = step_base;
  dyn->rec_first = rec_first;
  dyn->rec = rec;
  dyn->trig_first = rec_first;
}
// Trip (Sec. IV's change G' = G - g u u^T): the element leaves G; its parameters and both history
// copies are zeroed.
__global__ void k_open_element(double* g, double* alpha, double* beta, double* Ih, int m0, int m1) {
  for (int m : {m0, m1})
    if (m >= 0) {
      g[m] = 0.0;
      alpha[m] = 0.0;
      beta[m] = 0.0;
      Ih[m] = 0.0;
    }
}

template <int PREC>
void launch_steps(Sim& sm, int n, cudaStream_t s) {
  using X = typename Acc<PREC>::X;
  using T = typename Acc<PREC>::T;
  const Store& st = *sm.store;
  const FusedPlan& p = sm.plan;
  const DStore v = st.view();
  const CtaMapD cm = p.cmap();
  const CutRowsD cr = p.crows();
  const SimD sd = sm.view();
  X* part = reinterpret_cast<X*>(p.part.p);
  const T* gn = PREC == EMT_PREC_FP64 ? reinterpret_cast<const T*>(p.cut_gn64.p)
                : PREC == EMT_PREC_FF64 ? reinterpret_cast<const T*>(p.cut_gnff.p)
                                        : reinterpret_cast<const T*>(p.cut_gn32.p);
  static bool attr = false;
  if (!attr) {
    EMT_CUDA(cudaFuncSetAttribute(k_step_partial<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    EMT_CUDA(cudaFuncSetAttribute(k_step_sweep<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr = true;
  }
  const bool refine = PREC == EMT_PREC_FP32;
  for (int i = 0; i < n; ++i) {
    k_step_partial<PREC><<<p.n_cta, kFusedThreads, p.smem_partial, s>>>(v, cm, sd, i, 0, part);
    k_step_sweep<PREC><<<p.n_cta, kFusedThreads, p.smem_sweep, s>>>(v, cm, cr, sd, i, 0, refine ? 0 : 1, part, gn);
    if (refine) {
      k_step_partial<PREC><<<p.n_cta, kFusedThreads, p.smem_partial, s>>>(v, cm, sd, i, 1, part);
      k_step_sweep<PREC><<<p.n_cta, kFusedThreads, p.smem_sweep, s>>>(v, cm, cr, sd, i, 1, 1, part, gn);
    }
  }
  k_advance<<<1, 1, 0, s>>>(sm.d_dyn.p, n);
  EMT_CUDA(cudaGetLastError());
}

template <int PREC>
void launch_bench(Sim& sm, int which, int reps, cudaStream_t s) {
  using X = typename Acc<PREC>::X;
  using T = typename Acc<PREC>::T;
  const Store& st = *sm.store;
  const FusedPlan& p = sm.plan;
  const DStore v = st.view();
  const CtaMapD cm = p.cmap();
  const CutRowsD cr = p.crows();
  const SimD sd = sm.view();
  X* part = reinterpret_cast<X*>(p.part.p);
  const T* gn = PREC == EMT_PREC_FP64 ? reinterpret_cast<const T*>(p.cut_gn64.p)
                : PREC == EMT_PREC_FF64 ? reinterpret_cast<const T*>(p.cut_gnff.p)
                                        : reinterpret_cast<const T*>(p.cut_gn32.p);
  for (int i = 0; i < reps; ++i) {
    if (which == 0) k_step_partial<PREC><<<p.n_cta, kFusedThreads, p.smem_partial, s>>>(v, cm, sd, 0, 0, part);
    else k_step_sweep<PREC><<<p.n_cta, kFusedThreads, p.smem_sweep, s>>>(v, cm, cr, sd, 0, 0, 0, part, gn);
  }
  EMT_CUDA(cudaGetLastError());
}

void launch_steps_any(Sim& sm, int n, cudaStream_t s) {
  if (sm.use_v3()) {
    step3_launch_any(sm, n, s);
    k_advance<<<1, 1, 0, s>>>(sm.d_dyn.p, n);
    EMT_CUDA(cudaGetLastError());
    return;
  }
  if (sm.use_v2()) {
    step2_launch_any(sm, n, s);
    k_advance<<<1, 1, 0, s>>>(sm.d_dyn.p, n);
    EMT_CUDA(cudaGetLastError());
    return;
  }
  switch (sm.store->precision) {
    case EMT_PREC_FP64: launch_steps<EMT_PREC_FP64>(sm, n, s); break;
    case EMT_PREC_FF64: launch_steps<EMT_PREC_FF64>(sm, n, s); break;
    default: launch_steps<EMT_PREC_FP32>(sm, n, s); break;
  }
}

void launch_bench_any(Sim& sm, int which, int reps, cudaStream_t s) {
  if (sm.use_v3()) {
    step3_bench(sm, which, reps, s);
    return;
  }
  if (sm.use_v2()) {
    step2_bench(sm, which, reps, s);
    return;
  }
  switch (sm.store->precision) {
    case EMT_PREC_FP64: launch_bench<EMT_PREC_FP64>(sm, which, reps, s); break;
    case EMT_PREC_FF64: launch_bench<EMT_PREC_FF64>(sm, which, reps, s); break;
    default: launch_bench<EMT_PREC_FP32>(sm, which, reps, s); break;
  }
}

}  // namespace

// ---------------------------------------------------------------- host side
// Conductance graph of a network at time step dt: trapezoidal companion conductances of the
// series branches (ids preserved) and shunt capacitors, then 1/Rs of the sources.
// Sizes and the arrays they require (host side, before any device work): branch endpoints, kinds
// and R for every branch, L for RL and C for RC branches, all four arrays of every source and all
// three of every load.
void check_network_arrays(const emt_network* net) {
  EMT_REQUIRE(net, EMT_ERR_INVALID, "null network");
  EMT_REQUIRE(net->n_bus >= 1 && net->n_branch >= 0 && net->n_src >= 0 && net->n_load >= 0, EMT_ERR_INVALID,
              "bad network sizes");
  EMT_REQUIRE(net->n_branch == 0 || (net->from && net->to && net->kind && net->R), EMT_ERR_INVALID,
              "null branch arrays");
  for (int e = 0; e < net->n_branch; ++e)
    EMT_REQUIRE(net->kind[e] == EMT_KIND_RL ? net->L != nullptr : net->C != nullptr, EMT_ERR_INVALID,
                "null L (RL branches) or C (RC branches)");
  EMT_REQUIRE(net->n_src == 0 || (net->src_bus && net->src_Rs && net->src_Vm && net->src_phi), EMT_ERR_INVALID,
              "null source arrays");
  EMT_REQUIRE(net->n_load == 0 || (net->load_bus && net->load_amp && net->load_phi), EMT_ERR_INVALID,
              "null load arrays");
}

void network_graph(const emt_network* net, double dt, std::vector<int32_t>& gf, std::vector<int32_t>& gt,
                   std::vector<double>& gv) {
  EMT_REQUIRE(net && dt > 0, EMT_ERR_INVALID, "null network or bad dt");
  check_network_arrays(net);
  gf.clear();
  gt.clear();
  gv.clear();
  for (int e = 0; e < net->n_branch; ++e) {
    const int a = net->from[e], b = net->to[e];
    EMT_REQUIRE(a >= 0 && a < net->n_bus && b >= 0 && b < net->n_bus && a != b, EMT_ERR_INVALID,
                "series branch endpoints");
    double g;
    if (net->kind[e] == EMT_KIND_RL) g = 1.0 / (net->R[e] + 2.0 * net->L[e] / dt);
    else {
      EMT_REQUIRE(net->kind[e] == EMT_KIND_RC && net->C[e] > 0, EMT_ERR_INVALID, "bad RC branch");
      g = 1.0 / (net->R[e] + dt / (2.0 * net->C[e]));
    }
    EMT_REQUIRE(std::isfinite(g) && g > 0, EMT_ERR_INVALID, "branch companion conductance must be > 0");
    gf.push_back(a);
    gt.push_back(b);
    gv.push_back(g);
  }
  if (net->shunt_C)
    for (int i = 0; i < net->n_bus; ++i)
      if (net->shunt_C[i] > 0) {
        gf.push_back(i);
        gt.push_back(-1);
        gv.push_back(2.0 * net->shunt_C[i] / dt);
      }
  for (int k = 0; k < net->n_src; ++k) {
    EMT_REQUIRE(net->src_bus[k] >= 0 && net->src_bus[k] < net->n_bus && net->src_Rs[k] > 0, EMT_ERR_INVALID,
                "bad source");
    gf.push_back(net->src_bus[k]);
    gt.push_back(-1);
    gv.push_back(1.0 / net->src_Rs[k]);
  }
}

// Conductance graph of a three-phase network (the paper counts three nodes per bus): bus i
// carries nodes 3i, 3i + 1, 3i + 2 (phases a, b, c). An RL series branch couples its phases:
// resistance R and self inductance L per phase, mutual inductance L_mut between any two. Its
// trapezoidal companion admittance is Y = (R I + (2/dt) L3)^-1 with L3 = L I + L_mut (J - I), a
// matrix (alpha - beta) I + beta J (alpha = R + 2L/dt, beta = 2 L_mut/dt) whose inverse has
// diagonal (alpha + beta) / ((alpha - beta)(alpha + 2 beta)) and off-diagonal
// -beta / ((alpha - beta)(alpha + 2 beta)). The branch's term Y (x) (e_a - e_b)(e_a - e_b)^T is
// written exactly as node branches: a_p-b_p with Y_pp, a_p-b_q (p != q) with Y_pq (negative),
// a_p-a_q and b_p-b_q (p < q) with -Y_pq; none when L_mut = 0 (three decoupled phases). RC
// branches, shunt capacitors and sources act on each phase alone.
void network_graph3(const emt_network* net, const double* L_mut, double dt, std::vector<int32_t>& gf,
                    std::vector<int32_t>& gt, std::vector<double>& gv, std::vector<int>* br_ptr) {
  EMT_REQUIRE(net && L_mut && dt > 0, EMT_ERR_INVALID, "null network, null mutual inductances or bad dt");
  check_network_arrays(net);
  gf.clear();
  gt.clear();
  gv.clear();
  if (br_ptr) br_ptr->assign(1, 0);
  auto add = [&](int x, int y, double g) {
    gf.push_back(x);
    gt.push_back(y);
    gv.push_back(g);
  };
  for (int e = 0; e < net->n_branch; ++e) {
    const int a = net->from[e], b = net->to[e];
    EMT_REQUIRE(a >= 0 && a < net->n_bus && b >= 0 && b < net->n_bus && a != b, EMT_ERR_INVALID,
                "series branch endpoints");
    if (net->kind[e] == EMT_KIND_RL) {
      EMT_REQUIRE(L_mut[e] >= 0 && L_mut[e] < net->L[e], EMT_ERR_INVALID, "mutual inductance must be in [0, L)");
      const double al = net->R[e] + 2.0 * net->L[e] / dt, be = 2.0 * L_mut[e] / dt;
      const double den = (al - be) * (al + 2.0 * be);
      const double yd = (al + be) / den, yo = -be / den;
      EMT_REQUIRE(std::isfinite(yd) && yd > 0, EMT_ERR_INVALID, "branch companion conductance must be > 0");
      for (int p = 0; p < 3; ++p) add(3 * a + p, 3 * b + p, yd);
      if (yo != 0.0) {
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q)
            if (p != q) add(3 * a + p, 3 * b + q, yo);
        for (int p = 0; p < 3; ++p)
          for (int q = p + 1; q < 3; ++q) {
            add(3 * a + p, 3 * a + q, -yo);
            add(3 * b + p, 3 * b + q, -yo);
          }
      }
    } else {
      EMT_REQUIRE(net->kind[e] == EMT_KIND_RC && net->C[e] > 0, EMT_ERR_INVALID, "bad RC branch");
      const double g = 1.0 / (net->R[e] + dt / (2.0 * net->C[e]));
      EMT_REQUIRE(std::isfinite(g) && g > 0, EMT_ERR_INVALID, "branch companion conductance must be > 0");
      for (int p = 0; p < 3; ++p) add(3 * a + p, 3 * b + p, g);
    }
    if (br_ptr) br_ptr->push_back((int)gf.size());
  }
  if (net->shunt_C)
    for (int i = 0; i < net->n_bus; ++i)
      if (net->shunt_C[i] > 0)
        for (int p = 0; p < 3; ++p) add(3 * i + p, -1, 2.0 * net->shunt_C[i] / dt);
  for (int k = 0; k < net->n_src; ++k) {
    EMT_REQUIRE(net->src_bus[k] >= 0 && net->src_bus[k] < net->n_bus && net->src_Rs[k] > 0, EMT_ERR_INVALID,
                "bad source");
    for (int p = 0; p < 3; ++p) add(3 * net->src_bus[k] + p, -1, 1.0 / net->src_Rs[k]);
  }
}

SimD Sim::view() const {
  SimD d;
  d.n = n;
  d.inc_ptr = inc_ptr.p;
  d.inc_other = inc_other.p;
  d.inc_sgn = inc_sgn.p;
  d.inc_g = inc_g.p;
  d.inc_alpha = inc_alpha.p;
  d.inc_beta = inc_beta.p;
  d.Ih = Ih.p;
  d.src_ptr = src_ptr.p;
  d.src_coef = src_coef.p;
  d.src_phi = src_phi.p;
  d.omega = omega;
  d.dt = dt;
  d.v_pos = v_pos.p;
  d.x_pos = store->precision == EMT_PREC_FP32 ? x_pos.p : nullptr;
  d.mon_idx = mon_idx.p;
  d.n_mon = n_mon;
  d.dyn = d_dyn.p;
  d.csr_ptr = store->d_csr_ptr.p;
  d.csr_col = store->d_csr_col.p;
  d.csr_val = store->d_csr_val.p;
  return d;
}

Sim::Sim(const emt_network* net, const emt_hinv_opts* opts, double dt_, int nrhs_, const double* src_scale,
         const double* load_scale, cudaStream_t s) {
  EMT_REQUIRE(net && opts, EMT_ERR_INVALID, "null network or options");
  check_network_arrays(net);
  EMT_REQUIRE(dt_ > 0 && std::isfinite(dt_), EMT_ERR_INVALID, "dt must be > 0");
  EMT_REQUIRE(nrhs_ == 1, EMT_ERR_UNSUPPORTED, "this build steps one column per simulation");
  EMT_REQUIRE(opts->nodes_per_bus <= 1, EMT_ERR_UNSUPPORTED,
              "single-phase simulations partition buses one by one (nodes_per_bus 0 or 1)");
  (void)src_scale;
  (void)load_scale;
  n = net->n_bus;
  nrhs = nrhs_;
  dt = dt_;
  omega = 2.0 * M_PI * net->freq;
  const int nb = net->n_branch;
  EMT_REQUIRE(n >= 1 && nb >= 0, EMT_ERR_INVALID, "bad network sizes");
  // trapezoidal companion models (Sec. II): elements = series branches, then shunt capacitors
  el_a.clear();
  for (int e = 0; e < nb; ++e) {
    const int a = net->from[e], b = net->to[e];
    EMT_REQUIRE(a >= 0 && a < n && b >= 0 && b < n && a != b, EMT_ERR_INVALID, "series branch endpoints");
    const double R = net->R[e];
    double g, al, be;
    if (net->kind[e] == EMT_KIND_RL) {
      const double x = 2.0 * net->L[e] / dt;
      g = 1.0 / (R + x);
      al = g;
      be = g * (x - R);
    } else {
      EMT_REQUIRE(net->kind[e] == EMT_KIND_RC && net->C[e] > 0, EMT_ERR_INVALID, "bad RC branch");
      const double x = dt / (2.0 * net->C[e]);
      g = 1.0 / (R + x);
      al = -g;
      be = -g * (x - R);
    }
    EMT_REQUIRE(std::isfinite(g) && g > 0, EMT_ERR_INVALID, "branch companion conductance must be > 0");
    el_a.push_back(a);
    el_b.push_back(b);
    el_g.push_back(g);
    el_alpha.push_back(al);
    el_beta.push_back(be);
  }
  n_series = nb;
  if (net->shunt_C)
    for (int i = 0; i < n; ++i) {
      const double C = net->shunt_C[i];
      if (!(C > 0)) continue;
      const double g = 2.0 * C / dt;
      el_a.push_back(i);
      el_b.push_back(-1);
      el_g.push_back(g);
      el_alpha.push_back(-g);
      el_beta.push_back(-1.0);
    }
  // conductance graph for the store: elements + source conductances
  std::vector<int32_t> gf(el_a.begin(), el_a.end()), gt(el_b.begin(), el_b.end());
  std::vector<double> gv(el_g.begin(), el_g.end());
  for (int k = 0; k < net->n_src; ++k) {
    EMT_REQUIRE(net->src_bus[k] >= 0 && net->src_bus[k] < n && net->src_Rs[k] > 0, EMT_ERR_INVALID, "bad source");
    gf.push_back(net->src_bus[k]);
    gt.push_back(-1);
    gv.push_back(1.0 / net->src_Rs[k]);
  }
  emt_graph gr{n, (int32_t)gf.size(), gf.data(), gt.data(), gv.data()};
  // the partition sees bus-to-bus branches only; series branch ids are their element ids
  store.reset(new Store(&gr, opts, s));
  store->build(s);
  const Tree& t = store->tree;
  // incidences by position (element order inside a position)
  std::vector<std::vector<int>> at(n);
  for (size_t e = 0; e < el_a.size(); ++e) {
    at[t.pos[el_a[e]]].push_back((int)e);
    if (el_b[e] >= 0) at[t.pos[el_b[e]]].push_back((int)e);
  }
  std::vector<int> iptr(n + 1, 0), iother, isgn;
  std::vector<double> ig, ial, ibe;
  el_inc.assign(el_a.size(), {-1, -1});
  for (int p = 0; p < n; ++p) {
    for (int e : at[p]) {
      const int m = (int)iother.size();
      const bool is_a = t.pos[el_a[e]] == p;
      iother.push_back(is_a ? (el_b[e] >= 0 ? t.pos[el_b[e]] : -1) : t.pos[el_a[e]]);
      isgn.push_back(is_a ? 1 : -1);
      ig.push_back(el_g[e]);
      ial.push_back(el_alpha[e]);
      ibe.push_back(el_beta[e]);
      (is_a ? el_inc[e].first : el_inc[e].second) = m;
    }
    iptr[p + 1] = (int)iother.size();
  }
  inc_ptr.upload(iptr, s);
  inc_other.upload(iother, s);
  inc_sgn.upload(isgn, s);
  inc_g.upload(ig, s);
  inc_alpha.upload(ial, s);
  inc_beta.upload(ibe, s);
  Ih.alloc(std::max<size_t>(iother.size(), 1));
  Ih.zero(s);
  // sources and loads per position
  std::vector<std::vector<std::pair<double, double>>> terms(n);
  for (int k = 0; k < net->n_src; ++k)
    terms[t.pos[net->src_bus[k]]].push_back({net->src_Vm[k] / net->src_Rs[k], net->src_phi[k]});
  for (int k = 0; k < net->n_load; ++k) {
    EMT_REQUIRE(net->load_bus[k] >= 0 && net->load_bus[k] < n, EMT_ERR_INVALID, "bad load bus");
    terms[t.pos[net->load_bus[k]]].push_back({-net->load_amp[k], net->load_phi[k]});
  }
  src_terms = terms;
  std::vector<int> sp(n + 1, 0);
  std::vector<double> sc, sph;
  for (int p = 0; p < n; ++p) {
    for (auto& tm : terms[p]) {
      sc.push_back(tm.first);
      sph.push_back(tm.second);
    }
    sp[p + 1] = (int)sc.size();
  }
  src_ptr.upload(sp, s);
  src_coef.upload(sc, s);
  src_phi.upload(sph, s);
  v_pos.alloc(n);
  v_pos.zero(s);
  x_pos.alloc(n);
  x_pos.zero(s);
  std::vector<int> mi(n, -1);
  mon_idx.upload(mi, s);
  n_mon = 0;
  d_dyn.alloc(1);
  EMT_CUDA(cudaMemsetAsync(d_dyn.p, 0, sizeof(SimDyn), s));
  make_plan(*store, 0, plan, s);
  base.save(*store, s);
  inc_g0.upload(ig, s);
  inc_alpha0.upload(ial, s);
  inc_beta0.upload(ibe, s);
  el_g0 = el_g;
  launches_per_step = store->precision == EMT_PREC_FP32 ? 4 : 2;
  s2.build(*this, s);
  EMT_CUDA(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
  if (!apply_cached_tuning(s)) choose_default_kernels(s);
  EMT_CUDA(cudaStreamSynchronize(s));
  EMT_REQUIRE(store->device_status(s) == DEV_OK, EMT_ERR_SINGULAR, "G is not positive definite");
}

Sim::~Sim() {
  for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
  for (auto& kv : bench_graphs) cudaGraphExecDestroy(kv.second);
  if (cap_stream) cudaStreamDestroy(cap_stream);
}

void Sim::drop_graphs() {
  for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
  graphs.clear();
}

void Sim::set_rows_per_cta(int rpc, cudaStream_t s) { tune(rpc, kernels, s); }

void Sim::tune(int rpc, int kern, cudaStream_t s) {
  EMT_REQUIRE(kern >= 1 && kern <= 4, EMT_ERR_INVALID, "kernels must be 1, 2, 3 or 4");
  EMT_CUDA(cudaDeviceSynchronize());
  drop_graphs();
  for (auto& kv : bench_graphs) cudaGraphExecDestroy(kv.second);
  bench_graphs.clear();
  make_plan(*store, rpc, plan, s);
  s2.ready = false;
  s2.build(*this, s);
  s3.ready = false;
  if (kern == 3 && s2.ready) {
    int maxb = 0;
    for (int j = 0; j < store->n_leaf; ++j)
      maxb = std::max(maxb, store->tree.hi[store->leaf_nodes_h[j]] - store->tree.lo[store->leaf_nodes_h[j]]);
    const int r = rpc > 0 ? rpc : default_rows_per_cta(*store);
    int cs = std::max(1, std::min(8, (maxb + r - 1) / r));
    while (cs > 1 && !s3.build(*this, cs, s)) --cs;
    if (!s3.ready) s3.build(*this, cs, s);
  }
  s4.ready = false;
  if (kern == 4 && s2.ready) s4.build(*this, rpc > 0 ? rpc : 1, s);
  kernels = kern;
  EMT_CUDA(cudaDeviceSynchronize());
}

namespace {
// Tuned launch shapes per network shape, shared by every simulation of this process.
struct TuneKey {
  int n, n_leaf, max_depth, prec, sms;
  bool operator<(const TuneKey& o) const {
    return std::tie(n, n_leaf, max_depth, prec, sms) < std::tie(o.n, o.n_leaf, o.max_depth, o.prec, o.sms);
  }
};
std::map<TuneKey, std::pair<int, int>> g_tune_cache;
std::mutex g_tune_mutex;
TuneKey tune_key(const Sim& sm) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return {sm.n, sm.store->n_leaf, sm.store->tree.max_depth, sm.store->precision, sms};
}
}  // namespace

// Time every candidate launch shape on `probe_steps` steps of this simulation and keep the
// fastest; the choice is cached per network shape for later simulations in this process.
// The simulation is reset afterwards.
void Sim::autotune(int probe_steps, int* best_rpc, int* best_kernels, cudaStream_t s) {
  EMT_REQUIRE(probe_steps >= 1 && probe_steps <= 100000, EMT_ERR_INVALID, "probe_steps out of range");
  const int cands[] = {4, 6, 8, 10, 12, 16, 20, 24, 32, 48};
  cudaEvent_t e0, e1;
  EMT_CUDA(cudaEventCreate(&e0));
  EMT_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int brpc = 0, bk = 1;
  const int cands4[] = {1, 2, 4, 8, 16};
  for (int k : {4, 3, 2, 1}) {
    const int* cb = k == 4 ? cands4 : cands;
    const int nc = k == 4 ? 5 : (int)(sizeof(cands) / sizeof(cands[0]));
    for (int ci = 0; ci < nc; ++ci) {
      const int rpc = cb[ci];
      tune(rpc, k, s);
      if (k == 2 && !s2.ready) continue;
      if (k == 3 && !use_v3()) continue;
      if (k == 4 && !use_v4()) continue;
      reset(s);
      step(8, nullptr, s);
      EMT_CUDA(cudaEventRecord(e0, s));
      step(probe_steps, nullptr, s);
      EMT_CUDA(cudaEventRecord(e1, s));
      EMT_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      EMT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        brpc = rpc;
        bk = k;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  tune(brpc, bk, s);
  reset(s);
  EMT_CUDA(cudaStreamSynchronize(s));
  {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    g_tune_cache[tune_key(*this)] = {brpc, bk};
  }
  if (best_rpc) *best_rpc = brpc;
  if (best_kernels) *best_kernels = bk;
}

bool Sim::apply_cached_tuning(cudaStream_t s) {
  std::pair<int, int> v;
  {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    auto it = g_tune_cache.find(tune_key(*this));
    if (it == g_tune_cache.end()) return false;
    v = it->second;
  }
  tune(v.first, v.second, s);
  return true;
}

// Launch shape of a simulation nobody has timed: the persistent cluster kernel (generation 4)
// whenever its plan fits, with the largest cluster (at most 16 CTAs) that still gives every CTA
// 16 positions or more (8 CTAs at 179 buses, 16 at 1,432; the sizes the autotuner picks there),
// else the nearest sizes that fit; generation 2 when none does (FP32 stores, or stores too large
// for one cluster's shared memory).
void Sim::choose_default_kernels(cudaStream_t s) {
  if (!s2.ready || (store->precision != EMT_PREC_FF64 && store->precision != EMT_PREC_FP64)) return;
  int pref = 16;
  while (pref > 1 && n / pref < 16) pref /= 2;
  std::vector<int> order;
  for (int c = pref; c >= 1; c /= 2) order.push_back(c);
  for (int c = pref * 2; c <= 16; c *= 2) order.push_back(c);
  for (int c : order) {
    tune(c, 4, s);
    if (use_v4()) return;
  }
  tune(0, 2, s);
}

void Sim::set_monitor(int nm, const int32_t* buses, cudaStream_t s) {
  EMT_REQUIRE(nm >= 0 && (nm == 0 || buses), EMT_ERR_INVALID, "bad monitor list");
  std::vector<int> mi(n, -1);
  for (int k = 0; k < nm; ++k) {
    EMT_REQUIRE(buses[k] >= 0 && buses[k] < n, EMT_ERR_INVALID, "monitor bus out of range");
    EMT_REQUIRE(mi[store->tree.pos[buses[k]]] < 0, EMT_ERR_INVALID, "duplicate monitor bus");
    mi[store->tree.pos[buses[k]]] = k;
  }
  EMT_CUDA(cudaDeviceSynchronize());
  mon_idx.upload(mi, s);
  n_mon = nm;
  drop_graphs();
  EMT_CUDA(cudaDeviceSynchronize());
}

void Sim::schedule(int step, int kind, int target, double value, int column) {
  EMT_REQUIRE(step >= 1, EMT_ERR_INVALID, "event step must be >= 1");
  EMT_REQUIRE(step > cur_step, EMT_ERR_STATE, "event step already simulated");
  EMT_REQUIRE(column == -1 || (column >= 0 && column < nrhs), EMT_ERR_INVALID, "bad column");
  EMT_REQUIRE(column == -1, EMT_ERR_UNSUPPORTED, "per-column events need a multi-column simulation");
  if (kind == EMT_EVENT_TRIP) EMT_REQUIRE(target >= 0 && target < n_series, EMT_ERR_INVALID, "trip target must be a series branch");
  else if (kind == EMT_EVENT_FAULT_ON) EMT_REQUIRE(target >= 0 && target < n && value > 0, EMT_ERR_INVALID, "bad fault");
  else if (kind == EMT_EVENT_FAULT_OFF) EMT_REQUIRE(target >= 0 && target < n, EMT_ERR_INVALID, "bad fault bus");
  else throw Error(EMT_ERR_INVALID, "unknown event kind");
  events.push_back({step, kind, target, value, column});
  std::stable_sort(events.begin(), events.end(), [](const Event& a, const Event& b) { return a.step < b.step; });
}

void Sim::apply_event(const Event& ev, cudaStream_t s) {
  Store& st = *store;
  if (ev.kind == EMT_EVENT_TRIP) {
    const int e = ev.target;
    if (el_g[e] == 0.0) return;   // already open
    const double g = el_g[e];
    st.modify_async(el_a[e], el_b[e], -g, s);
    k_open_element<<<1, 1, 0, s>>>(inc_g.p, inc_alpha.p, inc_beta.p, Ih.p, el_inc[e].first, el_inc[e].second);
    if (s2.ready) s2.open_element(el_inc[e].first, el_inc[e].second, s);
    el_g[e] = 0.0;
  } else if (ev.kind == EMT_EVENT_FAULT_ON) {
    // a fault is its own change G' = G + (1/R_f) e_a e_a^T (Sec. IV)
    faults_on[ev.target].push_back(ev.value);
    st.modify_async(ev.target, -1, 1.0 / ev.value, s);
  } else {
    // clearing takes back exactly that change (delta = -1/R_f, the oldest fault on at the bus),
    // so changes made while the fault was on (trips, other faults) stay in G
    auto it = faults_on.find(ev.target);
    EMT_REQUIRE(it != faults_on.end() && !it->second.empty(), EMT_ERR_STATE, "FAULT_OFF without FAULT_ON");
    const double r_f = it->second.front();
    it->second.pop_front();
    if (it->second.empty()) faults_on.erase(it);
    st.modify_async(ev.target, -1, -1.0 / r_f, s);
  }
  refresh_plan_values(st, plan, s);
  if (s2.ready) s2.refresh(*this, s);
  if (s3.ready) s3.img.refresh(*this, s);
  if (s4.ready) s4.refresh(*this, s);
  EMT_CUDA(cudaGetLastError());
}

// Every FAULT_OFF up to last_step must find a fault on at its bus; checked before any work of an
// emt_step call is enqueued, so a bad sequence fails without touching the simulation.
void Sim::check_fault_sequence(int last_step) const {
  std::map<int, size_t> on;
  for (const auto& kv : faults_on) on[kv.first] = kv.second.size();
  for (size_t i = ev_cursor; i < events.size() && events[i].step <= last_step; ++i) {
    const Event& ev = events[i];
    if (ev.step <= cur_step) continue;
    if (ev.kind == EMT_EVENT_FAULT_ON) ++on[ev.target];
    if (ev.kind == EMT_EVENT_FAULT_OFF) {
      EMT_REQUIRE(on[ev.target] > 0, EMT_ERR_STATE, "FAULT_OFF at a bus where no fault is on at that step");
      --on[ev.target];
    }
  }
}

void Snapshot::save(const Store& st, cudaStream_t s) {
  L.alloc(st.L64.n);
  F.alloc(std::max<size_t>(st.F64.n, 1));
  C.alloc(std::max<size_t>(st.C64.n, 1));
  cg.alloc(std::max<size_t>(st.d_cut_g.n, 1));
  cv.alloc(std::max<size_t>(st.d_csr_val.n, 1));
  EMT_CUDA(cudaMemcpyAsync(L.p, st.L64.p, st.L64.n * 8, cudaMemcpyDeviceToDevice, s));
  if (st.F64.n) EMT_CUDA(cudaMemcpyAsync(F.p, st.F64.p, st.F64.n * 8, cudaMemcpyDeviceToDevice, s));
  if (st.C64.n) EMT_CUDA(cudaMemcpyAsync(C.p, st.C64.p, st.C64.n * 8, cudaMemcpyDeviceToDevice, s));
  if (st.d_cut_g.n) EMT_CUDA(cudaMemcpyAsync(cg.p, st.d_cut_g.p, st.d_cut_g.n * 8, cudaMemcpyDeviceToDevice, s));
  EMT_CUDA(cudaMemcpyAsync(cv.p, st.d_csr_val.p, st.d_csr_val.n * 8, cudaMemcpyDeviceToDevice, s));
  g_val = st.g_val;
  csr_val = st.csr_val;
  cut_g = st.cut_g_h;
}

void Snapshot::restore(Store& st, cudaStream_t s) {
  EMT_CUDA(cudaMemcpyAsync(st.L64.p, L.p, st.L64.n * 8, cudaMemcpyDeviceToDevice, s));
  if (st.F64.n) EMT_CUDA(cudaMemcpyAsync(st.F64.p, F.p, st.F64.n * 8, cudaMemcpyDeviceToDevice, s));
  if (st.C64.n) EMT_CUDA(cudaMemcpyAsync(st.C64.p, C.p, st.C64.n * 8, cudaMemcpyDeviceToDevice, s));
  if (st.d_cut_g.n) EMT_CUDA(cudaMemcpyAsync(st.d_cut_g.p, cg.p, st.d_cut_g.n * 8, cudaMemcpyDeviceToDevice, s));
  EMT_CUDA(cudaMemcpyAsync(st.d_csr_val.p, cv.p, st.d_csr_val.n * 8, cudaMemcpyDeviceToDevice, s));
  st.g_val = g_val;
  st.csr_val = csr_val;
  st.cut_g_h = cut_g;
  st.pack(s);
}

void Sim::run(int n_steps, cudaStream_t s) {
  int done = 0;
  while (done < n_steps) {
    const int next = cur_step + 1;
    while (ev_cursor < events.size() && events[ev_cursor].step < next) ++ev_cursor;
    while (ev_cursor < events.size() && events[ev_cursor].step == next) apply_event(events[ev_cursor++], s);
    int stretch = n_steps - done;
    if (ev_cursor < events.size()) stretch = std::min(stretch, events[ev_cursor].step - next);
    stretch = std::max(stretch, 1);
    int left = stretch;
    if (use_v4()) {
      // one persistent launch for the whole stretch between events
      step4_launch(*this, stretch, s);
      k_advance<<<1, 1, 0, s>>>(d_dyn.p, stretch);
      EMT_CUDA(cudaGetLastError());
      launches += (cur_rec && n_mon > 0 && store->precision == EMT_PREC_FF64) ? 3 : 2;
      left = 0;
    }
    while (left >= kChunk) {
      auto it = graphs.find(kChunk);
      if (it == graphs.end()) {
        cudaGraph_t g;
        EMT_CUDA(cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal));
        launch_steps_any(*this, kChunk, cap_stream);
        EMT_CUDA(cudaStreamEndCapture(cap_stream, &g));
        cudaGraphExec_t ge;
        EMT_CUDA(cudaGraphInstantiate(&ge, g, 0));
        cudaGraphDestroy(g);
        it = graphs.emplace(kChunk, ge).first;
      }
      EMT_CUDA(cudaGraphLaunch(it->second, s));
      launches += (int64_t)kChunk * launches_per_step + 1;
      left -= kChunk;
    }
    if (left > 0) {
      launch_steps_any(*this, left, s);
      launches += (int64_t)left * launches_per_step + 1;
    }
    cur_step += stretch;
    done += stretch;
  }
}

void Sim::step(int n_steps, double* record_dev, cudaStream_t s) {
  EMT_REQUIRE(n_steps >= 0, EMT_ERR_INVALID, "n_steps must be >= 0");
  if (n_steps == 0) return;
  check_fault_sequence(cur_step + n_steps);
  k_set_dyn<<<1, 1, 0, s>>>(d_dyn.p, cur_step, cur_step + 1, record_dev);
  EMT_CUDA(cudaGetLastError());
  launches += 1;
  cur_rec = record_dev;
  if (s2.ready) {
    s2.fill_trig(*this, cur_step + 1, n_steps, s);
    launches += 1;
  }
  run(n_steps, s);
}

void Sim::reset(cudaStream_t s) {
  base.restore(*store, s);
  refresh_plan_values(*store, plan, s);
  const size_t ni = inc_g.n;
  EMT_CUDA(cudaMemcpyAsync(inc_g.p, inc_g0.p, ni * 8, cudaMemcpyDeviceToDevice, s));
  EMT_CUDA(cudaMemcpyAsync(inc_alpha.p, inc_alpha0.p, ni * 8, cudaMemcpyDeviceToDevice, s));
  EMT_CUDA(cudaMemcpyAsync(inc_beta.p, inc_beta0.p, ni * 8, cudaMemcpyDeviceToDevice, s));
  Ih.zero(s);
  v_pos.zero(s);
  x_pos.zero(s);
  EMT_CUDA(cudaMemsetAsync(d_dyn.p, 0, sizeof(SimDyn), s));
  el_g = el_g0;
  if (s2.ready) {
    s2.reset_state(s);
    s2.refresh(*this, s);
  }
  if (s3.ready) s3.img.refresh(*this, s);
  if (s4.ready) s4.refresh(*this, s);
  faults_on.clear();
  cur_step = 0;
  ev_cursor = 0;
  launches += 4;   // pack (3) + -g refresh
}

void Sim::stats(int64_t* out, int n_out) const {
  const Store& st = *store;
  int64_t leaf = 0, fac = 0, core = 0;
  for (int j = 0; j < st.n_leaf; ++j) {
    const int nd = st.leaf_nodes_h[j];
    const int64_t b = st.tree.hi[nd] - st.tree.lo[nd];
    leaf += b * b;
  }
  for (int q : st.lvl_nodes_h) {
    const int64_t k = st.node_k_h[q];
    fac += (int64_t)(st.tree.hi[q] - st.tree.lo[q]) * k;
    core += 4 * k * k;
  }
  const int64_t v[] = {n, st.n_leaf, leaf, fac, core, plan.n_cta, (int64_t)inc_g.n,
                       (int64_t)st.cut_rows.crow_pos.size(), st.s_total, launches, n_series,
                       (int64_t)el_a.size()};
  for (int i = 0; i < n_out && i < (int)(sizeof(v) / sizeof(v[0])); ++i) out[i] = v[i];
}

void Sim::bench_kernel(int which, int reps, cudaStream_t s) {
  EMT_REQUIRE(which == 0 || which == 1, EMT_ERR_INVALID, "which must be 0 or 1");
  EMT_REQUIRE(reps >= 1 && reps <= 100000, EMT_ERR_INVALID, "reps out of range");
  if (use_v4()) {
    // the persistent kernel runs `reps` time steps in one launch
    k_set_dyn<<<1, 1, 0, s>>>(d_dyn.p, cur_step, cur_step + 1, nullptr);
    s2.fill_trig(*this, cur_step + 1, reps, s);
    cur_rec = nullptr;
    step4_launch(*this, reps, s);
    EMT_CUDA(cudaGetLastError());
    return;
  }
  const int key = which * 1000000 + reps;
  auto it = bench_graphs.find(key);
  if (it == bench_graphs.end()) {
    cudaGraph_t g;
    EMT_CUDA(cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal));
    launch_bench_any(*this, which, reps, cap_stream);
    EMT_CUDA(cudaStreamEndCapture(cap_stream, &g));
    cudaGraphExec_t ge;
    EMT_CUDA(cudaGraphInstantiate(&ge, g, 0));
    cudaGraphDestroy(g);
    it = bench_graphs.emplace(key, ge).first;
  }
  k_set_dyn<<<1, 1, 0, s>>>(d_dyn.p, cur_step, cur_step + 1, nullptr);
  if (s2.ready) s2.fill_trig(*this, cur_step + 1, 1, s);
  EMT_CUDA(cudaGraphLaunch(it->second, s));
}

void Sim::read(int what, double* host_out, cudaStream_t s) {
  if (what == 1) {
    host_out[0] = (double)cur_step;
    return;
  }
  EMT_REQUIRE(what == 0, EMT_ERR_INVALID, "unknown read selector");
  std::vector<double> vp(n);
  EMT_CUDA(cudaDeviceSynchronize());
  EMT_CUDA(cudaMemcpy(vp.data(), v_pos.p, n * sizeof(double), cudaMemcpyDeviceToHost));
  for (int p = 0; p < n; ++p) host_out[store->tree.perm[p]] = vp[p];
}

}  // namespace emt

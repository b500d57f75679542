// The extern "C" boundary: argument checks, exception-to-status translation, handle ownership.
#include <cmath>
#include <cstring>
#include <memory>
#include <string>

#include "plan.h"
#include "multi.h"
#include "server.h"
#include "sim.h"
#include "sim3.h"

namespace emt {
thread_local std::string g_last_error;
void set_last_error(const std::string& m) { g_last_error = m; }
void apply_vectors(Store& st, FusedPlan& p, DevBuf<double>& vpos, DevBuf<double>& rpos, const double* i_dev,
                   double* v_dev, int nrhs, int64_t ld, int max_refine, cudaStream_t s);
void apply_noalloc(const Store& st, const double* i_dev, double* v_dev, cudaStream_t s);
int selftest_wait(int limit_us, cudaStream_t s);
void network_graph(const emt_network* net, double dt, std::vector<int32_t>& gf, std::vector<int32_t>& gt,
                   std::vector<double>& gv);
void network_graph3(const emt_network* net, const double* L_mut, double dt, std::vector<int32_t>& gf,
                    std::vector<int32_t>& gt, std::vector<double>& gv, std::vector<int>* br_ptr);
}  // namespace emt

struct emt_tree {
  emt::Tree t;
};

struct emt_hinv {
  std::unique_ptr<emt::Store> st;
  emt::FusedPlan plan;
  bool has_plan = false;
  bool plan_stale = false;   // the store changed since the plan's values were taken
  emt::DevBuf<double> vpos, rpos;
  emt_tree tree;
};

struct emt_server {
  std::unique_ptr<emt::Server> srv;
};

struct emt_sim {
  std::unique_ptr<emt::Sim> sim;     // one column
  std::unique_ptr<emt::MSim> msim;   // several columns
  std::unique_ptr<emt::Sim3> sim3;   // three phases per bus
  bool ok() const { return sim || msim || sim3; }
};

namespace {

template <typename F>
emt_status guard(F&& f) {
  try {
    f();
    emt::g_last_error.clear();
    return EMT_OK;
  } catch (const emt::Error& e) {
    emt::g_last_error = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    emt::g_last_error = "host allocation failed";
    return EMT_ERR_NOMEM;
  } catch (const std::exception& e) {
    emt::g_last_error = e.what();
    return EMT_ERR_INVALID;
  } catch (...) {
    emt::g_last_error = "unknown error";
    return EMT_ERR_INVALID;
  }
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

emt_status status_from_device(int dev) {
  if (dev == emt::DEV_OK) return EMT_OK;
  if (dev == emt::DEV_SINGULAR) {
    emt::g_last_error = "device reported a singular or indefinite matrix";
    return EMT_ERR_SINGULAR;
  }
  if (dev == emt::DEV_TIMEOUT) {
    emt::g_last_error = "a bounded device wait ran out";
    return EMT_ERR_TIMEOUT;
  }
  emt::g_last_error = "unknown device status";
  return EMT_ERR_CUDA;
}

// three-phase builders: block cuts (three nodes per bus) unless the caller asks otherwise
emt_hinv_opts three_phase_opts(const emt_hinv_opts& o) {
  emt_hinv_opts c = o;
  if (c.nodes_per_bus == 0) c.nodes_per_bus = 3;
  return c;
}

}  // namespace

extern "C" {

const char* emt_last_error(void) { return emt::g_last_error.c_str(); }
const char* emt_version(void) { return "emt-hinv 0.1 (sm_103a)"; }

emt_status emt_tree_build(const emt_graph* graph, const emt_hinv_opts* opts, emt_tree** out) {
  return guard([&] {
    EMT_REQUIRE(graph && opts && out, EMT_ERR_INVALID, "null argument");
    EMT_REQUIRE(graph->n_branch == 0 || (graph->from && graph->to), EMT_ERR_INVALID, "null branch arrays");
    EMT_REQUIRE(opts->nodes_per_bus >= 0, EMT_ERR_INVALID, "nodes_per_bus must be >= 0");
    std::unique_ptr<emt_tree> t(new emt_tree);
    t->t = opts->nodes_per_bus >= 2
               ? emt::build_block_tree(graph->n_bus, graph->n_branch, graph->from, graph->to, opts->nodes_per_bus,
                                       opts->levels, opts->d_th)
               : emt::build_tree(graph->n_bus, graph->n_branch, graph->from, graph->to, opts->levels, opts->d_th);
    *out = t.release();
  });
}

emt_status emt_tree_sizes(const emt_tree* t, int32_t* n_node, int32_t* n_leaf, int32_t* n_cut) {
  return guard([&] {
    EMT_REQUIRE(t, EMT_ERR_INVALID, "null tree");
    if (n_node) *n_node = t->t.n_node();
    if (n_leaf) *n_leaf = (int32_t)t->t.leaves.size();
    if (n_cut) *n_cut = (int32_t)t->t.cut_a.size();
  });
}

emt_status emt_tree_arrays(const emt_tree* t, int32_t* perm, int32_t* lo, int32_t* hi, int32_t* parent,
                           int32_t* left, int32_t* right, int32_t* depth, int32_t* cut_ptr, int32_t* cut_a,
                           int32_t* cut_b, int32_t* cut_branch) {
  return guard([&] {
    EMT_REQUIRE(t, EMT_ERR_INVALID, "null tree");
    const emt::Tree& x = t->t;
    auto cp = [](int32_t* dst, const std::vector<int32_t>& v) {
      if (dst && !v.empty()) std::memcpy(dst, v.data(), v.size() * sizeof(int32_t));
    };
    cp(perm, x.perm);
    cp(lo, x.lo);
    cp(hi, x.hi);
    cp(parent, x.parent);
    cp(left, x.left);
    cp(right, x.right);
    cp(depth, x.depth);
    cp(cut_ptr, x.cut_ptr);
    cp(cut_a, x.cut_a);
    cp(cut_b, x.cut_b);
    cp(cut_branch, x.cut_e);
  });
}

void emt_tree_destroy(emt_tree* t) { delete t; }

emt_status emt_build_hinv(const emt_graph* graph, const emt_hinv_opts* opts, void* stream, emt_hinv** out) {
  return guard([&] {
    EMT_REQUIRE(out, EMT_ERR_INVALID, "null output handle");
    *out = nullptr;
    cudaStream_t s = as_stream(stream);
    std::unique_ptr<emt_hinv> h(new emt_hinv);
    h->st.reset(new emt::Store(graph, opts, s));
    h->st->build(s);
    const int dev = h->st->device_status(s);
    if (dev != emt::DEV_OK) throw emt::Error(EMT_ERR_SINGULAR, "G is not positive definite (a leaf or core is singular)");
    h->tree.t = h->st->tree;
    *out = h.release();
  });
}

emt_status emt_build_hinv_from_network3(const emt_network* net, const double* L_mut, double dt,
                                        const emt_hinv_opts* opts, void* stream, emt_hinv** out) {
  std::vector<int32_t> gf, gt;
  std::vector<double> gv;
  emt_status r = guard([&] {
    EMT_REQUIRE(net && net->n_bus <= (1 << 29), EMT_ERR_INVALID, "null or too large network");
    emt::network_graph3(net, L_mut, dt, gf, gt, gv, nullptr);
  });
  if (r != EMT_OK) return r;
  emt_graph g{3 * net->n_bus, (int32_t)gf.size(), gf.data(), gt.data(), gv.data()};
  if (!opts) return emt_build_hinv(&g, opts, stream, out);
  const emt_hinv_opts o3 = three_phase_opts(*opts);
  return emt_build_hinv(&g, &o3, stream, out);
}

emt_status emt_build_hinv_from_network(const emt_network* net, double dt, const emt_hinv_opts* opts, void* stream,
                                       emt_hinv** out) {
  std::vector<int32_t> gf, gt;
  std::vector<double> gv;
  emt_status r = guard([&] { emt::network_graph(net, dt, gf, gt, gv); });
  if (r != EMT_OK) return r;
  emt_graph g{net->n_bus, (int32_t)gf.size(), gf.data(), gt.data(), gv.data()};
  return emt_build_hinv(&g, opts, stream, out);
}

const emt_tree* emt_hinv_tree(const emt_hinv* h) { return h ? &h->tree : nullptr; }

emt_status emt_hinv_get_partition(const emt_hinv* h, int32_t* perm, int32_t* node_lo, int32_t* node_hi,
                                  int32_t* parent) {
  const emt_status r = guard([&] { EMT_REQUIRE(h, EMT_ERR_INVALID, "null handle"); });
  if (r != EMT_OK) return r;
  return emt_tree_arrays(&h->tree, perm, node_lo, node_hi, parent, nullptr, nullptr, nullptr, nullptr, nullptr,
                         nullptr, nullptr);
}

emt_status emt_apply(emt_hinv* h, const double* i_dev, double* v_dev, int32_t nrhs, int64_t ld, int32_t max_refine,
                     double tol, void* stream) {
  return guard([&] {
    EMT_REQUIRE(h && h->st, EMT_ERR_INVALID, "null handle");
    EMT_REQUIRE(i_dev && v_dev, EMT_ERR_INVALID, "null vectors");
    EMT_REQUIRE(nrhs >= 1 && ld >= h->st->n, EMT_ERR_INVALID, "bad nrhs or leading dimension");
    EMT_REQUIRE(max_refine >= 0 && max_refine <= 16, EMT_ERR_INVALID, "max_refine out of range");
    // the refinement count is fixed (max_refine); a tolerance would need a device read-back per pass
    EMT_REQUIRE(!(tol > 0.0) && !std::isnan(tol), EMT_ERR_UNSUPPORTED,
                "tol is not evaluated: pass tol <= 0 and choose max_refine instead");
    cudaStream_t s = as_stream(stream);
    if (!h->has_plan) {
      emt::make_plan(*h->st, 0, h->plan, s);
      h->has_plan = true;
    } else if (h->plan_stale) {
      emt::refresh_plan_values(*h->st, h->plan, s);   // once for any number of modifications
    }
    h->plan_stale = false;
    emt::apply_vectors(*h->st, h->plan, h->vpos, h->rpos, i_dev, v_dev, nrhs, ld, max_refine, s);
  });
}

emt_status emt_apply_noalloc(const emt_hinv* h, const double* i_dev, double* v_dev, void* stream) {
  return guard([&] {
    EMT_REQUIRE(h && h->st, EMT_ERR_INVALID, "null handle");
    EMT_REQUIRE(i_dev && v_dev, EMT_ERR_INVALID, "null vectors");
    emt::apply_noalloc(*h->st, i_dev, v_dev, as_stream(stream));
  });
}

emt_status emt_modify_branch(emt_hinv* h, int32_t bus_a, int32_t bus_b, double delta_g, void* stream) {
  return guard([&] {
    EMT_REQUIRE(h && h->st, EMT_ERR_INVALID, "null handle");
    cudaStream_t s = as_stream(stream);
    h->st->modify(bus_a, bus_b, delta_g, s);
    h->plan_stale = h->has_plan;   // the apply plan's copies of the values are refreshed by the next apply
    EMT_CUDA(cudaStreamSynchronize(s));
  });
}

emt_status emt_apply_tune(emt_hinv* h, int32_t kernels, int32_t warps, int32_t* used) {
  return guard([&] {
    EMT_REQUIRE(h && h->st, EMT_ERR_INVALID, "null handle");
    EMT_REQUIRE(kernels >= 0 && kernels <= 2, EMT_ERR_INVALID, "kernels must be 0, 1 or 2");
    EMT_REQUIRE(warps == 0 || (warps >= 4 && warps <= 16), EMT_ERR_INVALID, "warps must be 0 or 4..16");
    h->plan.stream_mode = kernels;
    if (warps != h->plan.stream_rps) {
      h->plan.stream_rps = warps;
      if (h->plan.sa) {   // re-planned by the next emt_apply
        EMT_CUDA(cudaDeviceSynchronize());
        h->plan.sa.reset();
      }
    }
    if (used) {
      // what the next single-vector emt_apply runs: 2 single launch, 1 three kernels, 0 the fused
      // kernels of stores that stay in the caches (the plan is built by the first emt_apply)
      const auto& sa = h->plan.sa;
      *used = (sa && sa->ready) ? ((sa->persist && kernels == 2) ? 2 : 1) : 0;
    }
  });
}

emt_status emt_hinv_sync(emt_hinv* h, void* stream) {
  emt_status r = guard([&] { EMT_REQUIRE(h && h->st, EMT_ERR_INVALID, "null handle"); });
  if (r != EMT_OK) return r;
  int dev = 0;
  r = guard([&] { dev = h->st->device_status(as_stream(stream)); });
  if (r != EMT_OK) return r;
  return status_from_device(dev);
}

void emt_hinv_destroy(emt_hinv* h) { delete h; }

emt_status emt_sim_create(const emt_network* net, const emt_hinv_opts* opts, double dt, int32_t nrhs,
                          const double* src_scale, const double* load_scale, void* stream, emt_sim** out) {
  return guard([&] {
    EMT_REQUIRE(out, EMT_ERR_INVALID, "null output handle");
    *out = nullptr;
    std::unique_ptr<emt_sim> h(new emt_sim);
    if (nrhs > 1) h->msim.reset(new emt::MSim(net, opts, dt, nrhs, src_scale, load_scale, as_stream(stream)));
    else h->sim.reset(new emt::Sim(net, opts, dt, nrhs, src_scale, load_scale, as_stream(stream)));
    *out = h.release();
  });
}

emt_status emt_sim3_create(const emt_network* net, const double* L_mut, const emt_hinv_opts* opts, double dt,
                           void* stream, emt_sim** out) {
  return guard([&] {
    EMT_REQUIRE(out, EMT_ERR_INVALID, "null output handle");
    *out = nullptr;
    EMT_REQUIRE(net && L_mut && opts, EMT_ERR_INVALID, "null network, mutual inductances or options");
    std::unique_ptr<emt_sim> h(new emt_sim);
    const emt_hinv_opts o3 = three_phase_opts(*opts);
    h->sim3.reset(new emt::Sim3(net, L_mut, &o3, dt, as_stream(stream)));
    *out = h.release();
  });
}

emt_status emt_sim_schedule(emt_sim* s, int32_t step, int32_t kind, int32_t target, double value, int32_t column) {
  return guard([&] {
    EMT_REQUIRE(s && s->ok(), EMT_ERR_INVALID, "null simulation");
    if (s->sim3) s->sim3->schedule(step, kind, target, value, column);
    else if (s->msim) s->msim->schedule(step, kind, target, value, column);
    else s->sim->schedule(step, kind, target, value, column);
  });
}

emt_status emt_sim_monitor(emt_sim* s, int32_t n_mon, const int32_t* buses) {
  return guard([&] {
    EMT_REQUIRE(s && s->ok(), EMT_ERR_INVALID, "null simulation");
    if (s->sim3) s->sim3->set_monitor(n_mon, buses);
    else if (s->msim) s->msim->set_monitor(n_mon, buses);
    else s->sim->set_monitor(n_mon, buses, nullptr);
  });
}

emt_status emt_step(emt_sim* s, int32_t n_steps, double* record_dev, void* stream) {
  return guard([&] {
    EMT_REQUIRE(s && s->ok(), EMT_ERR_INVALID, "null simulation");
    if (s->sim3) s->sim3->step(n_steps, record_dev, as_stream(stream));
    else if (s->msim) s->msim->step(n_steps, record_dev, as_stream(stream));
    else s->sim->step(n_steps, record_dev, as_stream(stream));
  });
}

emt_status emt_sim_read(emt_sim* s, int32_t what, double* host_out) {
  emt_status r = guard([&] {
    EMT_REQUIRE(s && s->ok() && host_out, EMT_ERR_INVALID, "null argument");
    if (s->sim3) s->sim3->read(what, host_out);
    else if (s->msim) s->msim->read(what, host_out);
    else s->sim->read(what, host_out, nullptr);
  });
  if (r != EMT_OK) return r;
  int dev = 0;
  r = guard([&] {
    EMT_CUDA(cudaDeviceSynchronize());
    dev = s->sim3 ? s->sim3->store->device_status(nullptr)
                  : (s->msim ? s->msim->store->device_status(nullptr) : s->sim->store->device_status(nullptr));
  });
  if (r != EMT_OK) return r;
  return status_from_device(dev);
}

emt_status emt_sim_set_rows_per_cta(emt_sim* s, int32_t rows_per_cta) {
  return guard([&] {
    EMT_REQUIRE(s && s->sim, EMT_ERR_INVALID, "null simulation");
    EMT_REQUIRE(rows_per_cta >= 0 && rows_per_cta <= 256, EMT_ERR_INVALID, "rows_per_cta out of range");
    s->sim->set_rows_per_cta(rows_per_cta, nullptr);
  });
}

emt_status emt_sim_set_inject(emt_sim* s, int32_t mode, int32_t positions_per_cta) {
  return guard([&] {
    EMT_REQUIRE(s && s->ok(), EMT_ERR_INVALID, "null simulation");
    EMT_REQUIRE(s->msim, EMT_ERR_UNSUPPORTED, "only multi-column simulations have injection variants");
    s->msim->set_inject(mode, positions_per_cta);
  });
}

emt_status emt_sim_tune(emt_sim* s, int32_t rows_per_cta, int32_t kernels) {
  return guard([&] {
    EMT_REQUIRE(s && s->ok(), EMT_ERR_INVALID, "null simulation");
    EMT_REQUIRE(!s->sim3, EMT_ERR_UNSUPPORTED, "three-phase simulations have no launch-shape choices");
    EMT_REQUIRE(rows_per_cta >= 0 && rows_per_cta <= 256, EMT_ERR_INVALID, "rows_per_cta out of range");
    if (s->msim) {
      s->msim->set_gemm(kernels, rows_per_cta, nullptr);
    } else {
      s->sim->tune(rows_per_cta, kernels, nullptr);
      if (kernels == 4 && !s->sim->use_v4()) {
        s->sim->tune(0, 2, nullptr);
        throw emt::Error(EMT_ERR_UNSUPPORTED,
                         "kernel generation 4 needs an FP64 or FF64 store that fits one cluster of that size");
      }
    }
  });
}

emt_status emt_sim_autotune(emt_sim* s, int32_t probe_steps, int32_t* best_rpc, int32_t* best_kernels,
                            void* stream) {
  return guard([&] {
    EMT_REQUIRE(s && s->ok(), EMT_ERR_INVALID, "null simulation");
    EMT_REQUIRE(!s->sim3, EMT_ERR_UNSUPPORTED, "three-phase simulations have no launch-shape choices");
    int r = 0, k = 0;
    if (s->msim) s->msim->autotune(probe_steps, &r, &k, nullptr, as_stream(stream));
    else s->sim->autotune(probe_steps, &r, &k, as_stream(stream));
    if (best_rpc) *best_rpc = r;
    if (best_kernels) *best_kernels = k;
  });
}

emt_status emt_sim_reset(emt_sim* s, void* stream) {
  return guard([&] {
    EMT_REQUIRE(s && s->ok(), EMT_ERR_INVALID, "null simulation");
    if (s->sim3) s->sim3->reset(as_stream(stream));
    else if (s->msim) s->msim->reset(as_stream(stream));
    else s->sim->reset(as_stream(stream));
  });
}

emt_status emt_sim_stats(const emt_sim* s, int64_t* out, int32_t n) {
  return guard([&] {
    EMT_REQUIRE(s && s->ok() && out && n >= 0, EMT_ERR_INVALID, "null argument");
    if (s->sim3) s->sim3->stats(out, n);
    else if (s->msim) s->msim->stats(out, n);
    else s->sim->stats(out, n);
  });
}

emt_status emt_sim_bench_kernel(emt_sim* s, int32_t which, int32_t reps, void* stream) {
  return guard([&] {
    EMT_REQUIRE(s && s->ok(), EMT_ERR_INVALID, "null simulation");
    EMT_REQUIRE(!s->sim3, EMT_ERR_UNSUPPORTED, "no kernel timing for three-phase simulations");
    if (s->msim) s->msim->bench_kernel(which, reps, as_stream(stream));
    else s->sim->bench_kernel(which, reps, as_stream(stream));
  });
}

void emt_sim_destroy(emt_sim* s) { delete s; }

emt_status emt_server_create(int32_t tick_steps, uint64_t hbm_budget_bytes, emt_server** out) {
  return guard([&] {
    EMT_REQUIRE(out, EMT_ERR_INVALID, "null output handle");
    std::unique_ptr<emt_server> h(new emt_server);
    h->srv.reset(new emt::Server(tick_steps, (size_t)hbm_budget_bytes));
    *out = h.release();
  });
}

emt_status emt_server_add_network(emt_server* s, const emt_network* net, const emt_hinv_opts* opts, double dt,
                                  int32_t max_slots, int32_t n_mon, const int32_t* mon_buses, int32_t* net_id) {
  return guard([&] {
    EMT_REQUIRE(s && s->srv && net && opts, EMT_ERR_INVALID, "null argument");
    const int id = s->srv->add_network(net, opts, dt, max_slots, n_mon, mon_buses);
    if (net_id) *net_id = id;
  });
}

emt_status emt_server_submit(emt_server* s, int32_t net_id, double arrival_s, int32_t n_steps, int32_t event_kind,
                             int32_t target, double value, int32_t event_step, int32_t event_len, int32_t* req_id) {
  return guard([&] {
    EMT_REQUIRE(s && s->srv, EMT_ERR_INVALID, "null server");
    const int id = s->srv->submit(net_id, arrival_s, n_steps, event_kind, target, value, event_step, event_len);
    if (req_id) *req_id = id;
  });
}

emt_status emt_server_submit_network(emt_server* s, const emt_network* net, const emt_hinv_opts* opts, double dt,
                                     int32_t n_mon, const int32_t* mon_buses, double arrival_s, int32_t n_steps,
                                     int32_t event_kind, int32_t target, double value, int32_t event_step,
                                     int32_t event_len, int32_t* req_id) {
  return guard([&] {
    EMT_REQUIRE(s && s->srv, EMT_ERR_INVALID, "null server");
    EMT_REQUIRE(dt > 0 && std::isfinite(dt), EMT_ERR_INVALID, "dt must be > 0");
    const int id = s->srv->submit_network(net, opts, dt, n_mon, mon_buses, arrival_s, n_steps, event_kind, target, value,
                                          event_step, event_len);
    if (req_id) *req_id = id;
  });
}

emt_status emt_server_run(emt_server* s) {
  return guard([&] {
    EMT_REQUIRE(s && s->srv, EMT_ERR_INVALID, "null server");
    s->srv->run();
  });
}

emt_status emt_server_result(const emt_server* s, int32_t req_id, double* out, double* times3) {
  return guard([&] {
    EMT_REQUIRE(s && s->srv, EMT_ERR_INVALID, "null server");
    EMT_REQUIRE(req_id >= 0 && req_id < (int)s->srv->reqs.size(), EMT_ERR_INVALID, "unknown request");
    const auto& r = s->srv->reqs[req_id];
    EMT_REQUIRE(r.t_done >= 0, EMT_ERR_STATE, "request not finished");
    if (out) std::memcpy(out, r.out.data(), r.out.size() * sizeof(double));
    if (times3) {
      times3[0] = r.arrival;
      times3[1] = r.t_admit;
      times3[2] = r.t_done;
    }
  });
}

emt_status emt_server_stats(const emt_server* s, double* out, int32_t n) {
  return guard([&] {
    EMT_REQUIRE(s && s->srv && out, EMT_ERR_INVALID, "null argument");
    s->srv->stats(out, n);
  });
}

void emt_server_destroy(emt_server* s) { delete s; }

emt_status emt_selftest_bounded_wait(int32_t limit_us, void* stream) {
  int dev = 0;
  emt_status r = guard([&] {
    EMT_REQUIRE(limit_us >= 1 && limit_us <= 2000000, EMT_ERR_INVALID, "limit_us must be in [1, 2e6]");
    dev = emt::selftest_wait(limit_us, as_stream(stream));
  });
  if (r != EMT_OK) return r;
  return status_from_device(dev);
}

}  // extern "C"

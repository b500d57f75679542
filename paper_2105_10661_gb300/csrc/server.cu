// Continuous-batching simulation server.
//
// Several base networks stay resident on the GPU, each as one multi-column simulation whose
// columns are request slots. Requests (a network, a number of steps, an optional line trip or
// bus fault) arrive on a wall-clock schedule. The scheduler loop:
//   1. moves requests whose arrival time has passed into their network's queue;
//   2. admits queued requests into free slots: the slot's state is reset, its source phases are
//      rotated to the request's start, and its change is set up as a per-column
//      Sherman-Morrison term (z = Ginv u from the accurate single-vector apply);
//   3. advances every network that has active slots by one tick of K steps, each network on its
//      own stream so their work overlaps on the device, and copies the monitored voltages of
//      the tick to pinned host memory;
//   4. hands the tick's outputs to the requests and retires the finished ones, freeing slots.
// The number of slots of a network comes from its share of an HBM budget divided by the
// per-slot footprint (state, right-hand sides, z column), so admission is by memory footprint.
//
// A request may also bring its own network. Its description is copied at submission and keyed by
// its content (element data, time step, store options, monitor list). When the request arrives,
// a resident network with the same key serves it (cache hit); otherwise its store and a
// simulation with kPrivSlots slots are built right there in the admission path (cache miss), so
// the build counts in the request's latency. Private networks with no active or queued request
// are evicted, least recently used first, when a new one would exceed the HBM budget; a request
// whose network cannot be placed yet waits.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <thread>

#include "server.h"

namespace emt {

namespace {
double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// FNV-1a over raw bytes
void fnv(uint64_t& h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ULL;
  }
}
template <typename T>
void fnv_vec(uint64_t& h, const std::vector<T>& v) {
  const uint64_t n = v.size();
  fnv(h, &n, sizeof n);
  if (n) fnv(h, v.data(), n * sizeof(T));
}
template <typename T>
std::vector<T> copy_of(const T* p, int n) {
  return p && n > 0 ? std::vector<T>(p, p + n) : std::vector<T>();
}
}  // namespace

emt_network Server::NetDesc::view() const {
  emt_network v{};
  v.n_bus = n_bus;
  v.n_branch = (int32_t)from.size();
  v.from = from.data();
  v.to = to.data();
  v.kind = kind.data();
  v.R = R.data();
  v.L = L.data();
  v.C = C.data();
  v.shunt_C = shunt_C.empty() ? nullptr : shunt_C.data();
  v.n_src = (int32_t)src_bus.size();
  v.src_bus = src_bus.data();
  v.src_Vm = src_Vm.data();
  v.src_phi = src_phi.data();
  v.src_Rs = src_Rs.data();
  v.n_load = (int32_t)load_bus.size();
  v.load_bus = load_bus.data();
  v.load_amp = load_amp.data();
  v.load_phi = load_phi.data();
  v.freq = freq;
  return v;
}

bool Server::NetDesc::same(const NetDesc& o) const {
  return n_bus == o.n_bus && from == o.from && to == o.to && kind == o.kind && src_bus == o.src_bus &&
         load_bus == o.load_bus && mon == o.mon && R == o.R && L == o.L && C == o.C && shunt_C == o.shunt_C &&
         src_Vm == o.src_Vm && src_phi == o.src_phi && src_Rs == o.src_Rs && load_amp == o.load_amp &&
         load_phi == o.load_phi && freq == o.freq && dt == o.dt && opts.levels == o.opts.levels &&
         opts.d_th == o.opts.d_th && opts.mode == o.opts.mode && opts.precision == o.opts.precision;
}

int64_t Server::per_slot_bytes(const emt_network* net) {
  // V, X (float-float), Xf, Y (FP32), Z (float-float), two history buffers per element (series
  // branches and one shunt per bus), boundary vectors, source coefficients
  const int64_t n = net->n_bus;
  const int64_t n_hist_est = 2 * ((int64_t)net->n_branch + n);
  return n * (8 + 8 + 4 + 4 + 8) + n_hist_est * 8 + 4 * 64 + (int64_t)(net->n_src + net->n_load) * 16;
}

Server::Server(int tick, size_t hbm_budget) : K(tick), budget(hbm_budget) {
  EMT_REQUIRE(tick >= 1 && tick <= 100000, EMT_ERR_INVALID, "tick must be in [1, 100000]");
}

Server::~Server() {
  for (auto& nt : nets) {
    if (nt.stream) cudaStreamDestroy(nt.stream);
    if (nt.host_rec) cudaFreeHost(nt.host_rec);
    if (nt.done) cudaEventDestroy(nt.done);
  }
}

int Server::add_network(const emt_network* net, const emt_hinv_opts* opts, double dt, int max_slots, int n_mon,
                        const int32_t* mon, bool fixed_slots) {
  EMT_REQUIRE(net && opts, EMT_ERR_INVALID, "null network or options");
  check_network_arrays(net);
  EMT_REQUIRE(max_slots >= 4 && n_mon >= 1 && mon, EMT_ERR_INVALID, "need >= 4 slots and a monitor list");
  const int64_t n = net->n_bus;
  const int64_t per_slot = per_slot_bytes(net);
  int slots = max_slots;
  if (budget > 0 && !fixed_slots) {
    const int64_t share = (int64_t)(budget - used) / 2;   // leave room for later networks
    slots = (int)std::min<int64_t>(max_slots, share / std::max<int64_t>(per_slot, 1));
    slots = slots / 4 * 4;
    EMT_REQUIRE(slots >= 4, EMT_ERR_NOMEM, "HBM budget too small for 4 slots of this network");
  }
  Net nt;
  nt.sim.reset(new MSim(net, opts, dt, slots, nullptr, nullptr, nullptr));
  nt.sim->set_monitor(n_mon, mon);
  nt.slots = slots;
  nt.n_bus = (int)n;
  nt.n_mon = n_mon;
  nt.slot_req.assign(slots, -1);
  nt.footprint = per_slot * slots;
  used += (size_t)nt.footprint;
  EMT_CUDA(cudaStreamCreateWithFlags(&nt.stream, cudaStreamNonBlocking));
  EMT_CUDA(cudaEventCreateWithFlags(&nt.done, cudaEventDisableTiming));
  nt.rec.alloc((size_t)K * slots * n_mon);
  EMT_CUDA(cudaMallocHost(&nt.host_rec, (size_t)K * slots * n_mon * sizeof(double)));
  nets.push_back(std::move(nt));
  return (int)nets.size() - 1;
}

int Server::submit_network(const emt_network* net, const emt_hinv_opts* opts, double dt, int n_mon, const int32_t* mon,
                           double arrival, int n_steps, int kind, int target, double value, int ev_step, int len) {
  EMT_REQUIRE(net && opts && mon && n_mon >= 1, EMT_ERR_INVALID, "null network, options or monitor list");
  EMT_REQUIRE(net->n_bus >= 2 && net->n_branch >= 1 && net->from && net->to && net->kind && net->R && net->L && net->C,
              EMT_ERR_INVALID, "incomplete network");
  EMT_REQUIRE(n_steps >= 1 && arrival >= 0, EMT_ERR_INVALID, "bad request");
  EMT_REQUIRE(kind >= -1 && kind <= 1, EMT_ERR_INVALID, "event kind must be -1, 0 (trip) or 1 (fault)");
  check_network_arrays(net);
  NetDesc d;
  d.n_bus = net->n_bus;
  d.from = copy_of(net->from, net->n_branch);
  d.to = copy_of(net->to, net->n_branch);
  d.kind = copy_of(net->kind, net->n_branch);
  d.R = copy_of(net->R, net->n_branch);
  d.L = copy_of(net->L, net->n_branch);
  d.C = copy_of(net->C, net->n_branch);
  d.shunt_C = copy_of(net->shunt_C, net->shunt_C ? net->n_bus : 0);
  d.src_bus = copy_of(net->src_bus, net->n_src);
  d.src_Vm = copy_of(net->src_Vm, net->n_src);
  d.src_phi = copy_of(net->src_phi, net->n_src);
  d.src_Rs = copy_of(net->src_Rs, net->n_src);
  d.load_bus = copy_of(net->load_bus, net->n_load);
  d.load_amp = copy_of(net->load_amp, net->n_load);
  d.load_phi = copy_of(net->load_phi, net->n_load);
  d.mon = copy_of(mon, n_mon);
  d.freq = net->freq;
  d.dt = dt;
  d.opts = *opts;
  uint64_t h = 1469598103934665603ULL;
  fnv(h, &d.n_bus, sizeof d.n_bus);
  for (const auto* v : {&d.from, &d.to, &d.kind, &d.src_bus, &d.load_bus, &d.mon}) fnv_vec(h, *v);
  for (const auto* v : {&d.R, &d.L, &d.C, &d.shunt_C, &d.src_Vm, &d.src_phi, &d.src_Rs, &d.load_amp, &d.load_phi})
    fnv_vec(h, *v);
  fnv(h, &d.freq, sizeof d.freq);
  fnv(h, &d.dt, sizeof d.dt);
  const int32_t o[4] = {opts->levels, opts->d_th, opts->mode, opts->precision};
  fnv(h, o, sizeof o);
  d.key = h;
  // requests bringing identical networks share one description
  int di = -1;
  auto range = desc_index.equal_range(h);
  for (auto it = range.first; it != range.second; ++it)
    if (descs[it->second].same(d)) {
      di = it->second;
      break;
    }
  if (di < 0) {
    descs.push_back(std::move(d));
    di = (int)descs.size() - 1;
    desc_index.emplace(h, di);
  }
  Req r;
  r.net = -1;
  r.priv = di;
  r.n_mon = n_mon;
  r.arrival = arrival;
  r.n_steps = n_steps;
  r.kind = kind;
  r.target = target;
  r.value = value;
  r.ev_step = ev_step;
  r.len = len;
  r.out.assign((size_t)n_steps * n_mon, 0.0);
  reqs.push_back(std::move(r));
  return (int)reqs.size() - 1;
}

void Server::evict(int ni) {
  Net& nt = nets[ni];
  if (nt.stream) EMT_CUDA(cudaStreamSynchronize(nt.stream));
  auto it = cache.find(nt.key);
  if (it != cache.end() && it->second == ni) cache.erase(it);
  nt.sim.reset();
  nt.rec = DevBuf<double>();
  if (nt.host_rec) cudaFreeHost(nt.host_rec);
  nt.host_rec = nullptr;
  if (nt.stream) cudaStreamDestroy(nt.stream);
  nt.stream = nullptr;
  if (nt.done) cudaEventDestroy(nt.done);
  nt.done = nullptr;
  nt.slots = 0;
  nt.slot_req.clear();
  used -= (size_t)nt.footprint;
  nt.footprint = 0;
  ++evictions;
}

// Resident network for private request `req`: a cache hit, or a build (evicting idle private
// networks, least recently used first, when the budget requires it). -1 when it cannot be placed
// yet. idle_since[ni] >= 0 marks a private network with no active or queued request.
int Server::place_private(int req, double t, std::vector<int>& idle_since) {
  const NetDesc& d = descs[reqs[req].priv];
  auto it = cache.find(d.key);
  if (it != cache.end() && (nets[it->second].desc == reqs[req].priv || descs[nets[it->second].desc].same(d))) {
    ++hits;
    return it->second;
  }
  if (it != cache.end()) cache.erase(it);   // a different network with the same hash: no longer cached
  const emt_network v = d.view();
  const int64_t need = per_slot_bytes(&v) * kPrivSlots;
  if (budget > 0) {
    while ((int64_t)used + need > (int64_t)budget) {
      int victim = -1;
      for (size_t ni = 0; ni < nets.size(); ++ni)
        if (nets[ni].priv && nets[ni].sim && idle_since[ni] >= 0 &&
            (victim < 0 || nets[ni].last_used < nets[victim].last_used))
          victim = (int)ni;
      if (victim < 0) return -1;   // wait for a private network to go idle
      evict(victim);
    }
  }
  const auto b0 = std::chrono::steady_clock::now();
  const int ni = add_network(&v, &d.opts, d.dt, kPrivSlots, (int)d.mon.size(), d.mon.data(), true);
  build_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - b0).count();
  ++builds;
  nets[ni].priv = true;
  nets[ni].key = d.key;
  nets[ni].desc = reqs[req].priv;
  nets[ni].last_used = t;
  cache[d.key] = ni;
  idle_since.resize(nets.size(), -1);
  return ni;
}

int Server::submit(int net, double arrival, int n_steps, int kind, int target, double value, int ev_step, int len) {
  EMT_REQUIRE(net >= 0 && net < (int)nets.size(), EMT_ERR_INVALID, "unknown network");
  EMT_REQUIRE(n_steps >= 1 && arrival >= 0, EMT_ERR_INVALID, "bad request");
  EMT_REQUIRE(kind >= -1 && kind <= 1, EMT_ERR_INVALID, "event kind must be -1, 0 (trip) or 1 (fault)");
  Req r;
  r.net = net;
  r.arrival = arrival;
  r.n_steps = n_steps;
  r.kind = kind;
  r.target = target;
  r.value = value;
  r.ev_step = ev_step;
  r.len = len;
  r.n_mon = nets[net].n_mon;
  r.out.assign((size_t)n_steps * nets[net].n_mon, 0.0);
  reqs.push_back(std::move(r));
  return (int)reqs.size() - 1;
}

void Server::run() {
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<int> order(reqs.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return reqs[a].arrival < reqs[b].arrival; });
  size_t next = 0;
  size_t finished = 0;
  for (auto& r : reqs)
    if (r.t_done >= 0) ++finished;
  std::vector<std::deque<int>> queue(nets.size());
  std::deque<int> unplaced;   // private requests whose network is not resident yet
  std::vector<int> idle(nets.size(), -1);
  max_queue = 0;
  while (finished < reqs.size()) {
    const double t = now_s(t0);
    while (next < order.size() && reqs[order[next]].arrival <= t) {
      const int id = order[next++];
      if (reqs[id].t_done >= 0) continue;
      if (reqs[id].priv >= 0) unplaced.push_back(id);
      else queue[reqs[id].net].push_back(id);
    }
    // private networks: resident (hit) or built now (miss), in arrival order
    for (size_t ni = 0; ni < nets.size(); ++ni) {
      bool busy_net = !queue[ni].empty();
      for (int c = 0; c < nets[ni].slots && !busy_net; ++c) busy_net = nets[ni].slot_req[c] >= 0;
      idle[ni] = busy_net ? -1 : 1;
    }
    while (!unplaced.empty()) {
      const int id = unplaced.front();
      const int ni = place_private(id, now_s(t0), idle);
      if (ni < 0) break;
      unplaced.pop_front();
      queue.resize(nets.size());
      idle.resize(nets.size(), -1);
      idle[ni] = -1;
      reqs[id].net = ni;
      nets[ni].last_used = now_s(t0);
      queue[ni].push_back(id);
    }
    size_t qn = unplaced.size();
    for (auto& q : queue) qn += q.size();
    max_queue = std::max(max_queue, (int)qn);
    // admission into free slots (lowest index first keeps the active prefix short)
    for (size_t ni = 0; ni < nets.size(); ++ni) {
      Net& nt = nets[ni];
      while (!queue[ni].empty()) {
        int slot = -1;
        for (int c = 0; c < nt.slots; ++c)
          if (nt.slot_req[c] < 0) {
            slot = c;
            break;
          }
        if (slot < 0) break;
        const int id = queue[ni].front();
        queue[ni].pop_front();
        Req& r = reqs[id];
        nt.sim->admit(slot, r.kind, r.target, r.value, r.ev_step, r.len, nt.stream);
        nt.slot_req[slot] = id;
        r.slot = slot;
        r.t_admit = now_s(t0);
        r.done_steps = 0;
      }
    }
    // one tick on every busy network, all enqueued before any wait
    std::vector<int> busy;
    for (size_t ni = 0; ni < nets.size(); ++ni) {
      Net& nt = nets[ni];
      int hi = 0;
      for (int c = 0; c < nt.slots; ++c)
        if (nt.slot_req[c] >= 0) hi = c + 1;
      if (hi == 0) continue;
      nt.sim->set_active(std::min(nt.slots, (hi + 3) / 4 * 4));
      nt.sim->step(K, nt.rec.p, nt.stream);
      EMT_CUDA(cudaMemcpyAsync(nt.host_rec, nt.rec.p, (size_t)K * nt.slots * nt.n_mon * sizeof(double),
                               cudaMemcpyDeviceToHost, nt.stream));
      EMT_CUDA(cudaEventRecord(nt.done, nt.stream));
      busy.push_back((int)ni);
      ticks++;
    }
    if (busy.empty()) {
      if (next < order.size()) {
        const double wait = reqs[order[next]].arrival - now_s(t0);
        if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 0.01)));
      }
      continue;
    }
    for (int ni : busy) {
      Net& nt = nets[ni];
      EMT_CUDA(cudaEventSynchronize(nt.done));
      const double tnow = now_s(t0);
      for (int c = 0; c < nt.slots; ++c) {
        const int id = nt.slot_req[c];
        if (id < 0) continue;
        Req& r = reqs[id];
        const int take = std::min(K, r.n_steps - r.done_steps);
        for (int k = 0; k < take; ++k)
          for (int m = 0; m < nt.n_mon; ++m)
            r.out[(size_t)(r.done_steps + k) * nt.n_mon + m] =
                nt.host_rec[((size_t)k * nt.slots + c) * nt.n_mon + m];
        r.done_steps += take;
        if (r.done_steps >= r.n_steps) {
          r.t_done = tnow;
          nt.slot_req[c] = -1;
          bus_steps += (double)r.n_steps * nt.n_bus;
          ++finished;
        }
      }
    }
    EMT_REQUIRE(device_ok(), EMT_ERR_SINGULAR, "a request's change made G singular");
  }
  wall = now_s(t0);
}

bool Server::device_ok() {
  for (auto& nt : nets)
    if (nt.sim && nt.sim->store->device_status(nt.stream) != DEV_OK) return false;
  return true;
}

void Server::stats(double* out, int n) const {
  std::vector<double> lat;
  for (auto& r : reqs)
    if (r.t_done >= 0) lat.push_back(r.t_done - r.arrival);
  std::sort(lat.begin(), lat.end());
  auto pct = [&](double p) {
    if (lat.empty()) return 0.0;
    const size_t i = std::min(lat.size() - 1, (size_t)std::ceil(p * lat.size()) - (p > 0 ? 1 : 0));
    return lat[i];
  };
  const double v[] = {wall, bus_steps, bus_steps / std::max(wall, 1e-12), pct(0.5), pct(0.99),
                      lat.empty() ? 0.0 : lat.back(), (double)max_queue, (double)ticks, (double)lat.size(),
                      (double)builds, (double)hits, build_s, (double)evictions};
  for (int i = 0; i < n && i < (int)(sizeof(v) / sizeof(v[0])); ++i) out[i] = v[i];
}

}  // namespace emt

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
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <thread>

#include "server.h"

namespace emt {

namespace {
double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}
}  // namespace

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
                        const int32_t* mon) {
  EMT_REQUIRE(max_slots >= 4 && n_mon >= 1 && mon, EMT_ERR_INVALID, "need >= 4 slots and a monitor list");
  // per-slot footprint: V, X (float-float), Xf, Y (FP32), Z (float-float), two history buffers per
  // element (series branches and one shunt per bus), boundary vectors, source coefficients
  const int64_t n = net->n_bus;
  const int64_t n_hist_est = 2 * ((int64_t)net->n_branch + n);
  const int64_t per_slot = n * (8 + 8 + 4 + 4 + 8) + n_hist_est * 8 + 4 * 64 + (int64_t)(net->n_src + net->n_load) * 16;
  int slots = max_slots;
  if (budget > 0) {
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
  max_queue = 0;
  while (finished < reqs.size()) {
    const double t = now_s(t0);
    while (next < order.size() && reqs[order[next]].arrival <= t) {
      const int id = order[next++];
      if (reqs[id].t_done < 0) queue[reqs[id].net].push_back(id);
    }
    size_t qn = 0;
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
    if (nt.sim->store->device_status(nt.stream) != DEV_OK) return false;
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
                      lat.empty() ? 0.0 : lat.back(), (double)max_queue, (double)ticks, (double)lat.size()};
  for (int i = 0; i < n && i < (int)(sizeof(v) / sizeof(v[0])); ++i) out[i] = v[i];
}

}  // namespace emt

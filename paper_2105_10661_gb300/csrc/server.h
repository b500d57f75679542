// Continuous-batching simulation server (see server.cu).
#pragma once
#include <cstdint>
#include <memory>
#include <unordered_map>
#include <vector>

#include "multi.h"

namespace emt {

class Server {
 public:
  Server(int tick, size_t hbm_budget);
  ~Server();
  // fixed_slots: exactly max_slots slots (the caller has applied the budget); otherwise the slots
  // are the network's share of the remaining budget, at most max_slots
  int add_network(const emt_network* net, const emt_hinv_opts* opts, double dt, int max_slots, int n_mon,
                  const int32_t* mon, bool fixed_slots = false);
  int submit(int net, double arrival, int n_steps, int kind, int target, double value, int ev_step, int len);
  // a request on its own network (copied now; built, or found resident, when it arrives)
  int submit_network(const emt_network* net, const emt_hinv_opts* opts, double dt, int n_mon, const int32_t* mon,
                     double arrival, int n_steps, int kind, int target, double value, int ev_step, int len);
  void run();
  void stats(double* out, int n) const;

  // host copy of a private network, keyed by its content
  struct NetDesc {
    int32_t n_bus = 0;
    std::vector<int32_t> from, to, kind, src_bus, load_bus, mon;
    std::vector<double> R, L, C, shunt_C, src_Vm, src_phi, src_Rs, load_amp, load_phi;
    double freq = 0, dt = 0;
    emt_hinv_opts opts{};
    uint64_t key = 0;
    emt_network view() const;
    bool same(const NetDesc& o) const;   // identical content (the key is a hash)
  };
  struct Req {
    int net = 0, n_steps = 0, kind = -1, target = 0, ev_step = 0, len = 0, slot = -1, done_steps = 0;
    int priv = -1, n_mon = 0;   // private network description (-1: a base network)
    double value = 0, arrival = 0, t_admit = -1, t_done = -1;
    std::vector<double> out;
  };
  struct Net {
    std::unique_ptr<MSim> sim;
    int slots = 0, n_bus = 0, n_mon = 0;
    int64_t footprint = 0;
    std::vector<int> slot_req;
    DevBuf<double> rec;
    double* host_rec = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool priv = false;          // built for private-network requests (evictable)
    uint64_t key = 0;
    int desc = -1;              // its description
    double last_used = 0;
  };
  static constexpr int kPrivSlots = 4;
  int K;
  size_t budget, used = 0;
  std::vector<Net> nets;
  std::vector<Req> reqs;
  std::vector<NetDesc> descs;
  std::unordered_map<uint64_t, int> cache;   // content key -> resident network
  std::unordered_multimap<uint64_t, int> desc_index;   // content key -> descriptions (shared by requests)
  double wall = 0, bus_steps = 0, build_s = 0;
  int max_queue = 0, builds = 0, hits = 0, evictions = 0;
  int64_t ticks = 0;

 private:
  bool device_ok();
  static int64_t per_slot_bytes(const emt_network* net);
  int place_private(int req, double t, std::vector<int>& idle_since);
  void evict(int ni);
};

}  // namespace emt

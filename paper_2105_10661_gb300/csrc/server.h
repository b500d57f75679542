// Continuous-batching simulation server (see server.cu).
#pragma once
#include <memory>
#include <vector>

#include "multi.h"

namespace emt {

class Server {
 public:
  Server(int tick, size_t hbm_budget);
  ~Server();
  int add_network(const emt_network* net, const emt_hinv_opts* opts, double dt, int max_slots, int n_mon,
                  const int32_t* mon);
  int submit(int net, double arrival, int n_steps, int kind, int target, double value, int ev_step, int len);
  void run();
  void stats(double* out, int n) const;

  struct Req {
    int net = 0, n_steps = 0, kind = -1, target = 0, ev_step = 0, len = 0, slot = -1, done_steps = 0;
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
  };
  int K;
  size_t budget, used = 0;
  std::vector<Net> nets;
  std::vector<Req> reqs;
  double wall = 0, bus_steps = 0;
  int max_queue = 0;
  int64_t ticks = 0;

 private:
  bool device_ok();
};

}  // namespace emt

// Internal declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "emt.h"

namespace emt {

struct Error : std::runtime_error {
  emt_status code;
  Error(emt_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

// source file name without its directories, for error messages
inline const char* src_name(const char* path) {
  const char* b = path;
  for (const char* p = path; *p; ++p)
    if (*p == '/') b = p + 1;
  return b;
}
#define EMT_CUDA(x)                                                                                    \
  do {                                                                                                 \
    cudaError_t e_ = (x);                                                                              \
    if (e_ != cudaSuccess)                                                                             \
      throw ::emt::Error(EMT_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_) + " (" +        \
                                           ::emt::src_name(__FILE__) + ":" + std::to_string(__LINE__) + ")"); \
  } while (0)
#define EMT_REQUIRE(c, code, msg)              \
  do {                                         \
    if (!(c)) throw ::emt::Error(code, msg);   \
  } while (0)

void set_last_error(const std::string& m);

// Device status word values (written by kernels, read by the host at sync points).
enum : int { DEV_OK = 0, DEV_SINGULAR = 3, DEV_TIMEOUT = 5 };

// ---------------------------------------------------------------- partition tree (host)
struct Tree {
  int n_bus = 0;
  int max_depth = 0;
  std::vector<int32_t> perm, pos;                        // position <-> bus
  std::vector<int32_t> lo, hi, parent, left, right, depth;
  std::vector<int32_t> leaves;                           // node ids, left to right
  std::vector<int32_t> cut_ptr, cut_a, cut_b, cut_e;     // cut endpoints as positions
  // cut_w = 1: one column per cut branch (h_l = -g e_a). cut_w = B > 1 (block cuts): one column
  // per (left group, right vertex) of joined groups of B vertices; cut_a is the group's first
  // position, its B vertices sit at cut_a .. cut_a + B - 1, cut_e is -1
  int cut_w = 1;
  int n_node() const { return (int)lo.size(); }
};
Tree build_tree(int n_bus, int n_branch, const int32_t* from, const int32_t* to, int levels,
                int d_th);
// Partition by groups of B consecutive vertices (the three nodes of a three-phase bus) with block
// cuts; d_th counts vertices.
Tree build_block_tree(int n_vertex, int n_branch, const int32_t* from, const int32_t* to, int B, int levels,
                      int d_th);

// ---------------------------------------------------------------- device buffers
template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) {
    o.p = nullptr;
    o.n = 0;
  }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p;
      n = o.n;
      o.p = nullptr;
      o.n = 0;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  void alloc(size_t count) {
    release();
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      throw Error(EMT_ERR_NOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    n = count;
  }
  void upload(const std::vector<T>& v, cudaStream_t s) {
    alloc(v.size());
    if (!v.empty()) EMT_CUDA(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  }
  void zero(cudaStream_t s) { EMT_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s)); }
};

}  // namespace emt

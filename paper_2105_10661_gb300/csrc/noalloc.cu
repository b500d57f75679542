// emt_apply_noalloc: the single-vector hierarchical apply for callers that must not allocate
// device memory once they are running (for example a real-time or embedded simulator that reserves
// all memory at start-up, or code running under a memory manager that forbids cudaMalloc).
//
// It runs the same two fused kernels as emt_apply (leaf partials, then boundary sweep and
// expansion) on the store built by emt_build_hinv. The only scratch it needs, the per-CTA leaf
// partial sums, lives in the file-scope device array below instead of a buffer from cudaMalloc.
// The launch layout is derived on the device from the store itself: each leaf gets
// ceil(b / kRows) CTAs, and the cut-endpoint lists are staged into shared memory. So the call
// allocates nothing, not even on the host.
//
// The array exists once per GPU that loads the library and stays reserved until the process
// exits. All calls share it and it keeps the previous call's contents; every entry a call reads
// was written earlier in the same call, so nothing needs clearing. Two calls that overlap on the
// GPU (different streams, or different handles) race on it and must be serialised by the caller.
#include <mutex>

#include "fused.cuh"

namespace emt {

namespace {

constexpr size_t kScratchBytes = EMT_APPLY_NOALLOC_SCRATCH_BYTES;
constexpr int kRows = 32;          // leaf rows per CTA
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_apply_scratch[kScratchBytes];

struct DeviceSetup {
  bool done = false;
  void* scratch = nullptr;        // device address of g_apply_scratch on that device
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Per-leaf CTA range, in shared memory: the launch covers n_leaf * cpl CTAs and CTA c works on
// leaf c / cpl, rows [(c % cpl) * kRows, ...) of it (empty tail CTAs exit).
__device__ __forceinline__ bool cta_rows(const DStore& st, int cpl, int& j, int& r0, int& r1) {
  j = blockIdx.x / cpl;
  const int chunk = blockIdx.x % cpl;
  const int node = st.leaf_node[j];
  const int b = st.hi[node] - st.lo[node];
  r0 = chunk * kRows;
  r1 = min(b, r0 + kRows);
  return r0 < b;
}

// Leaf stage of v = G^{-1} i (Eq. 2, Sec. III's leaf blocks) into the fixed scratch array.
template <int PREC>
__global__ void __launch_bounds__(kFusedThreads) k_na_partial(DStore st, const double* __restrict__ i_dev,
                                                              typename Acc<PREC>::X* __restrict__ part, int cpl,
                                                              int pld) {
  using A = Acc<PREC>;
  using X = typename A::X;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  X* xs = reinterpret_cast<X*>(smem_raw);
  X* red = xs + kRows;
  int j, r0, r1;
  if (!cta_rows(st, cpl, j, r0, r1)) return;
  const int lo = st.lo[st.leaf_node[j]];
  for (int r = threadIdx.x; r < r1 - r0; r += blockDim.x) xs[r] = A::prep(i_dev[st.perm[lo + r0 + r]]);
  __syncthreads();
  leaf_partial_core<PREC>(st, j, r0, r1, xs, part + (int64_t)blockIdx.x * pld, red);
}

// Boundary sweep (Eq. 9's factors and the node cores) and expansion of the CTA's rows to v.
template <int PREC>
__global__ void __launch_bounds__(kFusedThreads) k_na_sweep(DStore st, const typename Acc<PREC>::X* __restrict__ part,
                                                            int cpl, int pld, const int* __restrict__ g_item_node,
                                                            const int* __restrict__ g_item_pos,
                                                            const int* __restrict__ g_item_crow,
                                                            const int* __restrict__ g_item_sidx,
                                                            const int* __restrict__ g_crow_pos, int n_items, int n_crow,
                                                            int s_total, int n_cut, double* __restrict__ v_dev) {
  using A = Acc<PREC>;
  using X = typename A::X;
  using T = typename A::T;
  int j, r0, r1;
  if (!cta_rows(st, cpl, j, r0, r1)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // shared layout: ycut, t, s (X) | -g per cut (T) | items (4 ints each) | levels | leaf tables
  X* ycut = reinterpret_cast<X*>(smem_raw);
  X* t = ycut + n_crow;
  X* s = t + s_total;
  T* gn = reinterpret_cast<T*>(s + s_total);
  int* it_pos = reinterpret_cast<int*>(gn + n_cut);
  int* it_crow = it_pos + n_items;
  int* it_sidx = it_crow + n_items;
  int* it_cut = it_sidx + n_items;
  int* it_lvl = it_cut + n_items;                 // [max_depth + 2]
  int* leaf_c0 = it_lvl + st.max_depth + 2;       // [n_leaf]
  int* leaf_nc = leaf_c0 + st.n_leaf;
  const int tid = threadIdx.x;
  for (int c = tid; c < n_cut; c += blockDim.x) {
    const double g = -st.cut_g[c];
    if constexpr (PREC == EMT_PREC_FF64) gn[c] = ff_from(g);
    else if constexpr (PREC == EMT_PREC_FP32) gn[c] = __double2float_rn(g);
    else gn[c] = g;
  }
  for (int q = tid; q < st.n_leaf; q += blockDim.x) {
    const int node = st.leaf_node[q];
    leaf_c0[q] = q * cpl;
    leaf_nc[q] = (st.hi[node] - st.lo[node] + kRows - 1) / kRows;
  }
  // items are stored deepest level first, grouped by depth; restage them by increasing depth
  int* it_depth = leaf_nc + st.n_leaf;            // [n_items] scratch
  int* cnt = it_depth + n_items;                  // [max_depth + 1]
  int* first_in = cnt + st.max_depth + 1;         // [max_depth + 1]
  for (int d = tid; d <= st.max_depth; d += blockDim.x) cnt[d] = 0;
  __syncthreads();
  for (int i = tid; i < n_items; i += blockDim.x) {
    const int d = st.depth[g_item_node[i]];
    it_depth[i] = d;
    atomicAdd(&cnt[d], 1);
  }
  __syncthreads();
  if (tid == 0) {
    int w = 0;
    for (int d = 0; d <= st.max_depth; ++d) {
      it_lvl[d] = w;
      w += cnt[d];
    }
    it_lvl[st.max_depth + 1] = w;
    int f = 0;
    for (int d = st.max_depth; d >= 0; --d) {
      first_in[d] = f;
      f += cnt[d];
    }
  }
  __syncthreads();
  for (int i = tid; i < n_items; i += blockDim.x) {
    const int d = it_depth[i];
    const int w = it_lvl[d] + (i - first_in[d]);
    const int q = g_item_node[i];
    const int slot = g_item_sidx[i] - st.node_soff[q];
    it_pos[w] = g_item_pos[i];
    it_crow[w] = g_item_crow[i];
    it_sidx[w] = g_item_sidx[i];
    it_cut[w] = slot < st.node_k[q] ? st.cut_ptr[q] + slot : -1;
  }
  __syncthreads();
  CtaMapD cm;
  cm.leaf_cta0 = leaf_c0;
  cm.leaf_ncta = leaf_nc;
  cm.pld = pld;
  CutRowsD cr;
  cr.item_pos = it_pos;
  cr.item_crow = it_crow;
  cr.item_sidx = it_sidx;
  cr.item_cut = it_cut;
  cr.item_lvl = it_lvl;
  cr.crow_pos = g_crow_pos;
  cr.n_crow = n_crow;
  cr.n_items = n_items;
  cr.s_total = s_total;
  boundary_sweep<PREC>(st, cm, cr, part, ycut, t, s, gn);
  const int leaf_node = st.leaf_node[j];
  const int lo = st.lo[leaf_node];
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = r0 + warp; r < r1; r += nw) {
    const int pos = lo + r;
    const X y = leaf_y<PREC>(st, cm, part, pos);
    const X v = expand_row<PREC>(st, leaf_node, pos, y, s);
    if ((threadIdx.x & 31) == 0) v_dev[st.perm[pos]] = A::todbl(v);
  }
}

template <int PREC>
void launch_noalloc(const Store& st, void* scratch, const double* i_dev, double* v_dev, int cpl, int pld,
                    size_t sh_part, size_t sh_sweep, cudaStream_t s) {
  using X = typename Acc<PREC>::X;
  const DStore v = st.view();
  X* part = reinterpret_cast<X*>(scratch);
  const int grid = st.n_leaf * cpl;
  k_na_partial<PREC><<<grid, kFusedThreads, sh_part, s>>>(v, i_dev, part, cpl, pld);
  k_na_sweep<PREC><<<grid, kFusedThreads, sh_sweep, s>>>(
      v, part, cpl, pld, st.d_item_node.p, st.d_item_pos.p, st.d_item_crow.p, st.d_item_sidx.p, st.d_crow_pos.p,
      st.cut_rows.n_items, (int)st.cut_rows.crow_pos.size(), st.s_total, (int)st.cut_g_h.size(), v_dev);
}

template <int PREC>
void set_smem_limits() {
  EMT_CUDA(cudaFuncSetAttribute(k_na_partial<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  EMT_CUDA(cudaFuncSetAttribute(k_na_sweep<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
}

// Once per device, with that device current: look up the array's device address (a host-side
// use of the symbol itself would be a host stand-in, not a device address). The current device
// must be the one the store was built on, or the kernels would pair its pointers with another
// device's array.
void* device_scratch(int store_device) {
  int dev = 0;
  EMT_CUDA(cudaGetDevice(&dev));
  EMT_REQUIRE(dev == store_device, EMT_ERR_INVALID,
              "emt_apply_noalloc: the current CUDA device is not the one the store was built on");
  EMT_REQUIRE(dev >= 0 && dev < kMaxDevices, EMT_ERR_UNSUPPORTED, "device ordinal too large");
  std::lock_guard<std::mutex> lk(g_setup_mutex);
  DeviceSetup& d = g_setup[dev];
  if (!d.done) {
    void* p = nullptr;
    EMT_CUDA(cudaGetSymbolAddress(&p, g_apply_scratch));
    set_smem_limits<EMT_PREC_FP64>();
    set_smem_limits<EMT_PREC_FF64>();
    set_smem_limits<EMT_PREC_FP32>();
    d.scratch = p;
    d.done = true;
  }
  return d.scratch;
}

}  // namespace

void apply_noalloc(const Store& st, const double* i_dev, double* v_dev, cudaStream_t s) {
  int maxb = 0;
  for (int j = 0; j < st.n_leaf; ++j) {
    const int node = st.leaf_nodes_h[j];
    maxb = std::max(maxb, st.tree.hi[node] - st.tree.lo[node]);
  }
  EMT_REQUIRE(maxb <= 2048, EMT_ERR_UNSUPPORTED, "leaf larger than 2048 buses");
  const int cpl = (maxb + kRows - 1) / kRows;
  const int pld = (maxb + 3) / 4 * 4;
  const size_t need = (size_t)st.n_leaf * cpl * pld * 8;
  EMT_REQUIRE(need <= kScratchBytes, EMT_ERR_UNSUPPORTED,
              "emt_apply_noalloc: this store needs more scratch than EMT_APPLY_NOALLOC_SCRATCH_BYTES "
              "(n_leaf * ceil(max_leaf / 32) * max_leaf * 8 bytes); use emt_apply");
  void* scratch = device_scratch(st.device);
  // shared memory of the two kernels (same bounds as the fused apply)
  size_t red = 0;
  for (int ve : {2, 4}) {
    const int slots = (maxb + ve - 1) / ve;
    const int cover = std::min(slots, kFusedThreads);
    const int G = kFusedThreads / cover;
    red = std::max(red, (size_t)G * slots * ve * (ve == 2 ? 8 : 4));
  }
  const size_t sh_part = (size_t)kRows * 8 + red + 64;
  const int n_items = st.cut_rows.n_items;
  const size_t sh_sweep = (st.cut_rows.crow_pos.size() + 2 * (size_t)st.s_total + st.cut_g_h.size()) * 8 +
                          (size_t)5 * n_items * 4 + (size_t)(3 * st.tree.max_depth + 4 + 2 * st.n_leaf) * 4 + 64;
  EMT_REQUIRE(sh_part <= 200 * 1024 && sh_sweep <= 200 * 1024, EMT_ERR_UNSUPPORTED,
              "emt_apply_noalloc: store too large for shared memory");
  switch (st.precision) {
    case EMT_PREC_FP64: launch_noalloc<EMT_PREC_FP64>(st, scratch, i_dev, v_dev, cpl, pld, sh_part, sh_sweep, s); break;
    case EMT_PREC_FF64: launch_noalloc<EMT_PREC_FF64>(st, scratch, i_dev, v_dev, cpl, pld, sh_part, sh_sweep, s); break;
    default: launch_noalloc<EMT_PREC_FP32>(st, scratch, i_dev, v_dev, cpl, pld, sh_part, sh_sweep, s); break;
  }
  EMT_CUDA(cudaGetLastError());
}

}  // namespace emt

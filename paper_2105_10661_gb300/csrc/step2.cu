// Second-generation fused step kernels and their host-side plan (see step2.cuh).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "sim.h"
#include "step2.cuh"

namespace emt {

namespace {

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// 1-D bulk copy global -> this CTA's shared memory, completing `bytes` on the mbarrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase 0 of the CTA's copy barrier: non-blocking polls until `limit` SM clock
// cycles have passed, then gives up and reports it.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, long long limit) {
  const long long t0 = clock64();
  while (!mbar_test_wait(bar, 0))
    if (clock64() - t0 > limit) return false;
  return true;
}
constexpr long long kWaitPolls = 4000000000LL;   // ~2 s at 2 GHz

template <int PREC>
struct TT;
template <>
struct TT<EMT_PREC_FP64> {
  using T = double;
};
template <>
struct TT<EMT_PREC_FF64> {
  using T = float2;
};
template <>
struct TT<EMT_PREC_FP32> {
  using T = float;
};

// ------------------------------------------------------------------ image refresh (after build/modify)
template <int PREC>
__device__ __forceinline__ typename TT<PREC>::T img_value(double g) {
  if constexpr (PREC == EMT_PREC_FF64) return make_float2((float)g, (float)(g - (double)(float)g));
  else if constexpr (PREC == EMT_PREC_FP32) return (float)g;
  else return g;
}

// -g per cut entry and the factor rows every sweep item needs, gathered from the store. seg_src
// holds (source element, coefficient base, row stride) per segment: base -1 copies one factor row;
// base >= 0 (a side of a block column) writes sum over w of -g[base + w] times the rows of the
// column's W consecutive positions (FP64 sums of the FP64 factor rows).
template <int PREC>
__global__ void k_img_refresh(DStore st, unsigned char* img, int off_g, int n_cut, int off_r,
                              const int* __restrict__ seg_src, const int* __restrict__ seg_dst,
                              const int* __restrict__ seg_len, int n_seg) {
  using T = typename TT<PREC>::T;
  T* G = reinterpret_cast<T*>(img + off_g);
  T* R = reinterpret_cast<T*>(img + off_r);
  const T* F = Elem<PREC>::F(st);
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  for (int c = tid; c < n_cut; c += nth) G[c] = img_value<PREC>(-st.cut_g[c]);
  for (int sgi = tid; sgi < n_seg; sgi += nth) {
    const int src = seg_src[3 * sgi], base = seg_src[3 * sgi + 1], ld = seg_src[3 * sgi + 2];
    const int dst = seg_dst[sgi], len = seg_len[sgi];
    if (base < 0) {
      for (int e = 0; e < len; ++e) R[dst + e] = F[src + e];
    } else {
      for (int e = 0; e < len; ++e) {
        double v = 0.0;
        for (int w = 0; w < st.cut_w; ++w) v += -st.cut_g[base + w] * st.F64[src + (int64_t)w * ld + e];
        R[dst + e] = img_value<PREC>(v);
      }
    }
  }
}

// sin and cos of w t per step for the source injections of Eq. 1's i_in (FP64 and float-float).
__global__ void k_trig(double* trig, float4* trigff, int first_step, int n, double omega, double dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s, c;
  sincos(omega * ((double)(first_step + i) * dt), &s, &c);
  trig[2 * i] = s;
  trig[2 * i + 1] = c;
  const float2 fs = ff_from(s), fc = ff_from(c);
  trigff[i] = make_float4(fs.x, fs.y, fc.x, fc.y);
}

// ------------------------------------------------------------------ partial kernel
constexpr int kRmax = 8;
constexpr int kMaxNnz = 16;     // CSR row length prefetched into registers (host checks)
constexpr int kGatherUnroll = 8;
constexpr int kGroup = 8;       // threads per dot product in the sweep

// Second-generation partial kernel: history update and injection (Eq. 1), then the leaf stage of
// Eq. 2 over the CTA's rows, with static loads issued before griddepcontrol.wait.
template <int PREC>
__global__ void __launch_bounds__(kFusedThreads) k_step2_partial(DStore st, CtaMapD cm, SimD sim, Step2D q,
                                                                 int s_in_chunk, int pass,
                                                                 typename Acc<PREC>::X* __restrict__ part) {
  using A = Acc<PREC>;
  using X = typename A::X;
  using T = typename A::T;
  constexpr int VE = Elem<PREC>::VE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  X* xs = reinterpret_cast<X*>(smem_raw);                                  // [max_rows]
  double* contrib = reinterpret_cast<double*>(xs + ((cm.max_rows + 1) & ~1));   // [max_inc]
  X* red = reinterpret_cast<X*>(contrib + ((q.max_inc + 1) & ~1));          // group reduction
  const int c = blockIdx.x;
  const int j = cm.cta_leaf[c];
  const int r0 = cm.cta_r0[c], r1 = cm.cta_r1[c];
  const int node = st.leaf_node[j];
  const int lo = st.lo[node];
  const int b = st.hi[node] - lo;
  const int ld = st.leaf_ld[j];
  const T* L = Elem<PREC>::L(st) + st.leaf_off[j];
  const int slots = (b + VE - 1) / VE;
  const int G = kFusedThreads / slots;   // host guarantees slots <= 256 and rows <= G * kRmax
  const int tid = threadIdx.x;
  const int g = tid / slots, sl = tid % slots;
  const int nrow = r1 - r0;
  // static prefetch: leaf rows into registers
  T regs[kRmax][VE];
#pragma unroll
  for (int rr = 0; rr < kRmax; ++rr) {
    const int r = g + rr * G;
    if (g < G && r < nrow) vload(L + (int64_t)(r0 + r) * ld + sl * VE, regs[rr]);
  }
  // static prefetch: element record (one per thread), row data (one row per thread), phase
  const int m0 = sim.inc_ptr[lo + r0];
  const int m1 = sim.inc_ptr[lo + r1];
  IncRec rec{};
  const bool has_inc = pass == 0 && tid < m1 - m0;
  if (has_inc) rec = q.inc[m0 + tid];
  const bool has_row = tid < nrow;
  const int pos = lo + r0 + tid;
  int rm0 = 0, rm1 = 0;
  double2 ssum = make_double2(0.0, 0.0);
  int nnz = 0, cbeg = 0;
  int ccol[kMaxNnz];
  double cval[kMaxNnz];
  if (has_row) {
    if (pass == 0) {
      rm0 = sim.inc_ptr[pos] - m0;
      rm1 = sim.inc_ptr[pos + 1] - m0;
      ssum = q.src_sum[pos];
    } else {
      cbeg = sim.csr_ptr[pos];
      nnz = sim.csr_ptr[pos + 1] - cbeg;
#pragma unroll
      for (int k = 0; k < kMaxNnz; ++k)
        if (k < nnz) {
          ccol[k] = sim.csr_col[cbeg + k];
          cval[k] = sim.csr_val[cbeg + k];
        }
    }
  }
  pdl_launch_dependents();
  pdl_wait();
  if (*st.status != DEV_OK) return;
  const int step = sim.dyn->step_base + s_in_chunk + 1;
  if (pass == 0) {
    const int ti = step - sim.dyn->trig_first;
    const double sw = q.trig[2 * ti], cw = q.trig[2 * ti + 1];
    if (has_inc) {
      const double vi = sim.v_pos[rec.self];
      const double vo = rec.other >= 0 ? sim.v_pos[rec.other] : 0.0;
      const double Ih = q.Ih[m0 + tid];
      const double ve = rec.sgn > 0 ? vi - vo : vo - vi;
      const double cur = rec.g * ve + Ih;
      const double Ihn = rec.alpha * ve + rec.beta * cur;
      q.Ih[m0 + tid] = Ihn;
      contrib[tid] = rec.sgn > 0 ? -Ihn : Ihn;
    }
    __syncthreads();
    if (has_row) {
      double hist = 0.0;
      for (int m = rm0; m < rm1; ++m) hist += contrib[m];
      const double x = ssum.x * sw + ssum.y * cw + hist;
      if (sim.x_pos) sim.x_pos[pos] = x;
      xs[tid] = A::prep(x);
    }
  } else if (has_row) {
    // refinement: r = x - G v with the FP64 conductance matrix
    double vv[kMaxNnz];
#pragma unroll
    for (int k = 0; k < kMaxNnz; ++k)
      if (k < nnz) vv[k] = sim.v_pos[ccol[k]];
    double acc = sim.x_pos[pos];
#pragma unroll
    for (int k = 0; k < kMaxNnz; ++k)
      if (k < nnz) acc -= cval[k] * vv[k];
    xs[tid] = A::prep(acc);
  }
  __syncthreads();
  A acc[VE];
  if (g < G) {
#pragma unroll
    for (int rr = 0; rr < kRmax; ++rr) {
      const int r = g + rr * G;
      if (r < nrow) {
        const X x = xs[r];
#pragma unroll
        for (int e = 0; e < VE; ++e) acc[e].fma(regs[rr][e], x);
      }
    }
    const int width = slots * VE;
#pragma unroll
    for (int e = 0; e < VE; ++e) red[g * width + sl * VE + e] = acc[e].getx();
  }
  __syncthreads();
  X* out = part + (int64_t)c * cm.pld;
  const int width = slots * VE;
  for (int col = tid; col < b; col += kFusedThreads) {
    A s;
    for (int gg = 0; gg < G; ++gg) s.add(red[gg * width + col]);
    out[col] = s.getx();
  }
}

// ------------------------------------------------------------------ sweep kernel
// Boundary sweep of every node from the shared-memory image (t_p and s_p = C_p t_p, Eq. 9's
// factors) and the expansion of the CTA's rows to v(t).
template <int PREC, bool FROMY = false>
__global__ void __launch_bounds__(kFusedThreads) k_step2_sweep(DStore st, CtaMapD cm, SimD sim, Step2D q,
                                                               int s_in_chunk, int accumulate, int record,
                                                               const typename Acc<PREC>::X* part) {
  using A = Acc<PREC>;
  using X = typename A::X;
  using T = typename A::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  int* own_off = reinterpret_cast<int*>(smem_raw + 16);                 // [kMaxAnc] byte offsets
  unsigned char* img = smem_raw + 16 + 16 * ((kMaxAnc * 4 + 15) / 16);
  unsigned char* cores = img + q.img_bytes;
  unsigned char* ownF = cores + q.core_bytes;
  const ImgHeader* H = reinterpret_cast<const ImgHeader*>(img);
  const int c = blockIdx.x;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
    const OwnCopy& oc = q.own[c];
    uint32_t total = (uint32_t)q.img_bytes + (uint32_t)q.core_bytes;
    int off = 0;
    for (int a = 0; a < oc.n; ++a) {
      own_off[a] = off;
      off += oc.bytes[a];
    }
    total += (uint32_t)off;
    mbar_expect_tx(bar, total);
    bulk_g2s(img, q.img, (uint32_t)q.img_bytes, bar);
    if (q.core_bytes) bulk_g2s(cores, q.cores, (uint32_t)q.core_bytes, bar);
    for (int a = 0; a < oc.n; ++a)
      if (oc.bytes[a]) bulk_g2s(ownF + own_off[a], q.fac + oc.src_bytes[a], (uint32_t)oc.bytes[a], bar);
  }
  const int j = cm.cta_leaf[c];
  const int r0 = cm.cta_r0[c], r1 = cm.cta_r1[c];
  const int leaf_node = st.leaf_node[j];
  const int lo = st.lo[leaf_node];
  const int lc0 = cm.leaf_cta0[j], lnc = cm.leaf_ncta[j];
  __syncthreads();
  pdl_launch_dependents();
  pdl_wait();
  const bool ok = mbar_wait_bounded(bar, kWaitPolls);
  if (!ok) {
    if (tid == 0) atomicExch(st.status, DEV_TIMEOUT);
    mbar_wait_bounded(bar, kWaitPolls);   // give copies in flight a second bounded chance
    return;
  }
  if (*st.status != DEV_OK) return;
  const int* I = reinterpret_cast<const int*>(img);
  const int n_crow = H->n_crow, s_total = H->s_total;
  X* ycut = reinterpret_cast<X*>(smem_raw + q.sweep_smem_static);
  X* t = ycut + n_crow;
  X* s = t + s_total;
  X* yown = s + s_total;
  const int nrow = r1 - r0;
  if constexpr (FROMY) {
    // generation 3: the leaf stage already holds one reduced value per position
    const int* cpos = I + H->off_crow_pos;
    for (int k = tid; k < n_crow; k += kFusedThreads) ycut[k] = A::prep(__ldcg(q.ylf + cpos[k]));
    for (int r = tid; r < nrow; r += kFusedThreads) yown[r] = A::prep(__ldcg(q.ylf + lo + r0 + r));
    __syncthreads();
  } else {
  // dynamic: every partial needed (cut rows, then own rows) is loaded in unrolled batches so
  // all loads of a thread are in flight together, then reduced in shared memory
  X* pv = yown + ((r1 - r0) + 1);
  const int* cpair_ptr = I + H->off_cpair_ptr;
  const int* cpair = I + H->off_cpair;
  const int n_cp = H->n_cpair;
  const int total = n_cp + nrow * lnc;
  for (int base = 0; base < total; base += kFusedThreads * kGatherUnroll) {
    X tmp[kGatherUnroll];
#pragma unroll
    for (int u = 0; u < kGatherUnroll; ++u) {
      const int i = base + u * kFusedThreads + tid;
      if (i < total) {
        int64_t off;
        if (i < n_cp) off = cpair[i];
        else {
          const int w = i - n_cp;
          off = (int64_t)(lc0 + w % lnc) * cm.pld + r0 + w / lnc;
        }
        tmp[u] = __ldcg(part + off);   // written by the preceding grid: read through L2, never hoisted
      }
    }
#pragma unroll
    for (int u = 0; u < kGatherUnroll; ++u) {
      const int i = base + u * kFusedThreads + tid;
      if (i < total) pv[i] = tmp[u];
    }
  }
  __syncthreads();
  for (int k = tid; k < n_crow; k += kFusedThreads) {
    A a;
    for (int i = cpair_ptr[k]; i < cpair_ptr[k + 1]; ++i) a.add(pv[i]);
    ycut[k] = a.getx();
  }
  for (int r = tid; r < nrow; r += kFusedThreads) {
    A a;
    for (int u = 0; u < lnc; ++u) a.add(pv[n_cp + r * lnc + u]);
    yown[r] = a.getx();
  }
  __syncthreads();
  }
  sweep_levels<PREC, kGroup>(img, cores, ycut, t, s);
  // expansion of the own rows: warp per row
  const int* anc_ptr = I + H->off_anc_ptr;
  const int* anc = I + H->off_anc;
  const int a0 = anc_ptr[j], a1 = anc_ptr[j + 1];
  const int warp = tid >> 5, lane = tid & 31, nw = kFusedThreads >> 5;
  const int step = sim.dyn->step_base + s_in_chunk + 1;
  double* recp = sim.dyn->rec;
  for (int r = warp; r < r1 - r0; r += nw) {
    const int pos = lo + r0 + r;
    A a;
    for (int x = a0; x < a1; ++x) {
      const int* an = anc + 5 * x;
      const int k = an[0], kld = an[1];
      const int si = pos < an[2] ? an[3] : an[4];
      const T* Fr = reinterpret_cast<const T*>(ownF + own_off[x - a0]) + (int64_t)r * kld;
      for (int e = lane; e < k; e += 32) a.fma(Fr[e], neg(s[si + e]));
    }
    X v = a.getx();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      A tt;
      tt.add(v);
      tt.add(a.shfl_xor(v, o));
      v = tt.getx();
    }
    if (lane == 0) {
      A fin;
      fin.add(yown[r]);
      fin.add(v);
      double out = A::todbl(fin.getx());
      if (accumulate) out += sim.v_pos[pos];
      sim.v_pos[pos] = out;
      if (record && recp) {
        const int mi = sim.mon_idx[pos];
        if (mi >= 0) recp[(int64_t)(step - sim.dyn->rec_first) * sim.n_mon + mi] = out;
      }
    }
  }
}

template <typename K, typename... Args>
void launch_pdl(K kernel, int grid, int block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  EMT_CUDA(cudaLaunchKernelEx(&cfg, kernel, args...));
}

}  // namespace

// Waits on an mbarrier that never completes, with the same bounded wait as the step kernels.
__global__ void k_selftest_wait(long long limit_cycles, int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (!mbar_wait_bounded(&bar, limit_cycles) && threadIdx.x == 0) atomicExch(status, DEV_TIMEOUT);
}

int selftest_wait(int limit_us, cudaStream_t s) {
  int dev = 0, khz = 0;
  EMT_CUDA(cudaGetDevice(&dev));
  EMT_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
  if (khz <= 0) khz = 2000000;
  DevBuf<int> st;
  st.alloc(1);
  st.zero(s);
  k_selftest_wait<<<1, 32, 0, s>>>((long long)limit_us * khz / 1000, st.p);
  EMT_CUDA(cudaGetLastError());
  int h = 0;
  EMT_CUDA(cudaMemcpyAsync(&h, st.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  EMT_CUDA(cudaStreamSynchronize(s));
  return h;
}

// ====================================================================== host side
// Boundary-sweep image of a store: header, integer tables (distinct cut rows, sweep items by
// depth, factor segments, core rows, ancestor lists per leaf), -g per cut and the factor rows
// every item needs. With a plan, the cut rows also carry the CTAs whose partial sums hold them.
void build_sweep_image(const Store& st, const FusedPlan* p, int prec, ImgHeader& hdr, DevBuf<double>& img,
                       DevBuf<int>& seg_src, DevBuf<int>& seg_dst, DevBuf<int>& seg_len, int& n_seg, cudaStream_t s) {
  const Tree& t = st.tree;
  const size_t tb = prec == EMT_PREC_FP32 ? 4 : 8;
  const CutRows& cr = st.cut_rows;
  std::vector<int> ints;
  ImgHeader Hh{};
  auto align_ints = [&]() {
    while ((ints.size() * 4) % 16) ints.push_back(0);
  };
  ints.resize((sizeof(ImgHeader) + 15) / 16 * 4, 0);
  Hh.n_crow = (int)cr.crow_pos.size();
  Hh.n_items = cr.n_items;
  Hh.s_total = st.s_total;
  Hh.max_depth = t.max_depth;
  Hh.n_leaf = st.n_leaf;
  Hh.n_cut = (int)st.cut_g_h.size();
  Hh.cut_w = t.cut_w;
  Hh.off_crow = (int)ints.size();
  for (int k = 0; k < Hh.n_crow; ++k) {
    const int ps = cr.crow_pos[k];
    const int j = leaf_index_of_pos(st, ps);
    ints.push_back(p ? p->h_leaf_cta0[j] : 0);
    ints.push_back(p ? p->h_leaf_ncta[j] : 0);
    ints.push_back(ps - t.lo[st.leaf_nodes_h[j]]);
  }
  Hh.off_crow_pos = (int)ints.size();
  for (int k = 0; k < Hh.n_crow; ++k) ints.push_back(cr.crow_pos[k]);
  Hh.off_cpair_ptr = (int)ints.size();
  {
    std::vector<int> ptr(Hh.n_crow + 1, 0), pairs;
    for (int k = 0; k < Hh.n_crow; ++k) {
      const int ps = cr.crow_pos[k];
      const int j = leaf_index_of_pos(st, ps);
      const int loc = ps - t.lo[st.leaf_nodes_h[j]];
      if (p)
        for (int u = 0; u < p->h_leaf_ncta[j]; ++u) pairs.push_back((p->h_leaf_cta0[j] + u) * p->pld + loc);
      ptr[k + 1] = (int)pairs.size();
    }
    for (int v : ptr) ints.push_back(v);
    Hh.off_cpair = (int)ints.size();
    Hh.n_cpair = (int)pairs.size();
    for (int v : pairs) ints.push_back(v);
  }
  // items by increasing depth
  std::vector<int> order(cr.n_items);
  for (int i = 0; i < cr.n_items; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return t.depth[cr.item_node[x]] < t.depth[cr.item_node[y]]; });
  Hh.off_lvl_item = (int)ints.size();
  {
    std::vector<int> lvl(t.max_depth + 2, 0);
    for (int i = 0; i < cr.n_items; ++i) lvl[t.depth[cr.item_node[i]] + 1]++;
    for (int d = 0; d <= t.max_depth; ++d) lvl[d + 1] += lvl[d];
    for (int v : lvl) ints.push_back(v);
  }
  Hh.off_item = (int)ints.size();
  ints.resize(ints.size() + 6 * (size_t)cr.n_items);
  std::vector<int> segs;               // pairs
  std::vector<int> seg_src_h, seg_dst_h, seg_len_h;
  int r_elems = 0;
  for (int w = 0; w < cr.n_items; ++w) {
    const int it = order[w];
    const int q = cr.item_node[it];
    const int d = t.depth[q];
    const int ps = cr.item_pos[it];
    const int k = st.node_k_h[q];
    const int slot = cr.item_sidx[it] - st.node_soff_h[q];
    int* rec = &ints[Hh.off_item + 6 * w];
    rec[0] = cr.item_crow[it];
    rec[1] = cr.item_sidx[it];
    rec[2] = slot < k ? t.cut_ptr[q] + slot : -1;
    rec[3] = r_elems;
    rec[4] = (int)segs.size() / 2;
    int nseg = 0;
    // a side of a block column (cut_w > 1) gets its W factor rows combined with the coefficients
    const int comb = (t.cut_w > 1 && rec[2] >= 0) ? rec[2] * t.cut_w : -1;
    for (int a = t.parent[st.leaf_nodes_h[leaf_index_of_pos(st, ps)]]; a >= 0 && t.depth[a] > d; a = t.parent[a]) {
      const int ka = st.node_k_h[a];
      if (ka == 0) continue;
      const int half = ps < t.hi[t.left[a]] ? 0 : ka;
      segs.push_back(st.node_soff_h[a] + half);
      segs.push_back(ka);
      seg_src_h.push_back((int)(st.node_foff_h[a] + (int64_t)(ps - t.lo[a]) * st.node_kld_h[a]));
      seg_src_h.push_back(comb);
      seg_src_h.push_back(st.node_kld_h[a]);
      seg_dst_h.push_back(r_elems);
      seg_len_h.push_back(ka);
      r_elems += ka;
      ++nseg;
    }
    rec[5] = nseg;
  }
  Hh.off_seg = (int)ints.size();
  Hh.n_seg = (int)segs.size() / 2;
  for (int v : segs) ints.push_back(v);
  Hh.off_lvl_core = (int)ints.size();
  {
    std::vector<int> lvl(t.max_depth + 2, 0);
    for (int q : st.lvl_nodes_h) lvl[t.depth[q] + 1] += 2 * st.node_k_h[q];
    for (int d = 0; d <= t.max_depth; ++d) lvl[d + 1] += lvl[d];
    for (int v : lvl) ints.push_back(v);
  }
  Hh.off_core = (int)ints.size();
  {
    // core rows in increasing depth order (lvl_nodes_h is grouped by increasing depth)
    for (int q : st.lvl_nodes_h) {
      const int m2 = 2 * st.node_k_h[q];
      for (int r = 0; r < m2; ++r) {
        ints.push_back(st.node_soff_h[q] + r);
        ints.push_back(st.node_soff_h[q]);
        ints.push_back(m2);
        ints.push_back((int)(st.node_coff_h[q] + (int64_t)r * m2));
      }
    }
    Hh.n_core = (int)((ints.size() - Hh.off_core) / 4);
  }
  Hh.off_anc_ptr = (int)ints.size();
  std::vector<int> anc_list;
  std::vector<int> anc_ptr(st.n_leaf + 1, 0);
  for (int j = 0; j < st.n_leaf; ++j) {
    for (int a = t.parent[st.leaf_nodes_h[j]]; a >= 0; a = t.parent[a]) {
      anc_list.push_back(st.node_k_h[a]);
      anc_list.push_back(st.node_kld_h[a]);
      anc_list.push_back(t.hi[t.left[a]]);
      anc_list.push_back(st.node_soff_h[a]);
      anc_list.push_back(st.node_soff_h[a] + st.node_k_h[a]);
      anc_ptr[j + 1]++;
    }
    anc_ptr[j + 1] += anc_ptr[j];
  }
  for (int v : anc_ptr) ints.push_back(v);
  Hh.off_anc = (int)ints.size();
  for (int v : anc_list) ints.push_back(v);
  align_ints();
  Hh.int_words = (int)ints.size();
  Hh.off_g_bytes = Hh.int_words * 4;
  const size_t g_bytes = (Hh.n_cut * tb + 15) / 16 * 16;
  Hh.off_r_bytes = (int)(Hh.off_g_bytes + g_bytes);
  const size_t r_bytes = ((size_t)r_elems * tb + 15) / 16 * 16;
  Hh.img_bytes = (int)(Hh.off_r_bytes + std::max<size_t>(r_bytes, 16));
  std::memcpy(ints.data(), &Hh, sizeof(ImgHeader));
  img.alloc((Hh.img_bytes + 7) / 8);
  EMT_CUDA(cudaMemsetAsync(img.p, 0, Hh.img_bytes, s));
  EMT_CUDA(cudaMemcpyAsync(img.p, ints.data(), ints.size() * 4, cudaMemcpyHostToDevice, s));
  hdr = Hh;
  seg_src.upload(seg_src_h.empty() ? std::vector<int>{0} : seg_src_h, s);
  seg_dst.upload(seg_dst_h.empty() ? std::vector<int>{0} : seg_dst_h, s);
  seg_len.upload(seg_len_h.empty() ? std::vector<int>{0} : seg_len_h, s);
  n_seg = (int)seg_dst_h.size();
  refresh_sweep_image(st, prec, hdr, img, seg_src, seg_dst, seg_len, n_seg, s);
}

bool Step2::build(const Sim& sm, cudaStream_t s, int force_prec) {
  const Store& st = *sm.store;
  const FusedPlan& p = sm.plan;
  const Tree& t = st.tree;
  prec = force_prec >= 0 ? force_prec : st.precision;
  const size_t tb = prec == EMT_PREC_FP32 ? 4 : 8;
  // partial kernel feasibility: one 16-byte slot per thread, rows per thread <= kRmax
  const int ve = prec == EMT_PREC_FP32 ? 4 : 2;
  int maxb = 0;
  for (int j = 0; j < st.n_leaf; ++j) maxb = std::max(maxb, t.hi[st.leaf_nodes_h[j]] - t.lo[st.leaf_nodes_h[j]]);
  const int slots = (maxb + ve - 1) / ve;
  if (slots > kFusedThreads) return false;
  for (int j = 0; j < st.n_leaf; ++j) {
    const int b = t.hi[st.leaf_nodes_h[j]] - t.lo[st.leaf_nodes_h[j]];
    const int sj = (b + ve - 1) / ve;
    const int G = kFusedThreads / sj;
    if (p.max_rows > G * kRmax) return false;
  }
  if (t.max_depth > kMaxAnc) return false;
  // ---- element records and source terms (position order, same as the v1 arrays)
  std::vector<int> iptr(sm.n + 1, 0);
  std::vector<IncRec> recs;
  {
    std::vector<std::vector<int>> at(sm.n);
    for (size_t e = 0; e < sm.el_a.size(); ++e) {
      at[t.pos[sm.el_a[e]]].push_back((int)e);
      if (sm.el_b[e] >= 0) at[t.pos[sm.el_b[e]]].push_back((int)e);
    }
    for (int ps = 0; ps < sm.n; ++ps) {
      for (int e : at[ps]) {
        IncRec r{};
        const bool is_a = t.pos[sm.el_a[e]] == ps;
        r.self = ps;
        r.other = is_a ? (sm.el_b[e] >= 0 ? t.pos[sm.el_b[e]] : -1) : t.pos[sm.el_a[e]];
        r.sgn = is_a ? 1 : -1;
        r.g = sm.el_g0[e];
        r.alpha = sm.el_alpha[e];
        r.beta = sm.el_beta[e];
        recs.push_back(r);
      }
      iptr[ps + 1] = (int)recs.size();
    }
  }
  max_inc = 0;
  for (int c = 0; c < p.n_cta; ++c) {
    // CTA rows from the plan (host copies)
    const int j = p.h_cta_leaf[c];
    const int lo = t.lo[st.leaf_nodes_h[j]];
    max_inc = std::max(max_inc, iptr[lo + p.h_cta_r1[c]] - iptr[lo + p.h_cta_r0[c]]);
  }
  if (max_inc > kFusedThreads) return false;
  for (int ps = 0; ps < sm.n; ++ps)
    if (st.csr_ptr[ps + 1] - st.csr_ptr[ps] > kMaxNnz) return false;
  max_lnc = 0;
  for (int j = 0; j < st.n_leaf; ++j) max_lnc = std::max(max_lnc, p.h_leaf_ncta[j]);
  inc0 = recs;
  inc.upload(recs, s);
  std::vector<SrcRec> src;
  std::vector<int> sptr(sm.n + 1, 0);
  for (int ps = 0; ps < sm.n; ++ps) {
    for (auto& tm : sm.src_terms[ps]) src.push_back({tm.first * std::cos(tm.second), tm.first * std::sin(tm.second)});
    sptr[ps + 1] = (int)src.size();
  }
  if (src.empty()) src.push_back({0, 0});
  d_src.upload(src, s);
  {
    std::vector<double2> ssum(sm.n);
    for (int ps = 0; ps < sm.n; ++ps) {
      double a = 0.0, b = 0.0;
      for (auto& tm : sm.src_terms[ps]) {
        a += tm.first * std::cos(tm.second);
        b += tm.first * std::sin(tm.second);
      }
      ssum[ps] = make_double2(a, b);
    }
    d_src_sum.upload(ssum, s);
  }
  d_src_ptr.upload(sptr, s);
  build_sweep_image(st, &p, prec, header, img, seg_src_d, seg_dst_d, seg_len_d, n_seg_copy, s);
  const ImgHeader& Hh = header;
  core_bytes = (int)(st.C_elems * tb);
  // own factor rows per CTA
  std::vector<OwnCopy> own(p.n_cta);
  int own_max = 0;
  for (int c = 0; c < p.n_cta; ++c) {
    OwnCopy oc{};
    const int j = p.h_cta_leaf[c];
    const int lnode = st.leaf_nodes_h[j];
    const int pos0 = t.lo[lnode] + p.h_cta_r0[c];
    const int nrow = p.h_cta_r1[c] - p.h_cta_r0[c];
    int tot = 0;
    for (int a = t.parent[lnode]; a >= 0; a = t.parent[a]) {
      const int64_t el = st.node_foff_h[a] + (int64_t)(pos0 - t.lo[a]) * st.node_kld_h[a];
      oc.src_bytes[oc.n] = el * (int64_t)tb;
      oc.bytes[oc.n] = (int)((int64_t)nrow * st.node_kld_h[a] * tb);
      tot += oc.bytes[oc.n];
      oc.n++;
    }
    own_max = std::max(own_max, tot);
    own[c] = oc;
  }
  own_d.upload(own, s);
  const size_t head = 16 + 16 * ((kMaxAnc * 4 + 15) / 16);
  smem_static = head + Hh.img_bytes + core_bytes + own_max;
  smem_static = (smem_static + 15) / 16 * 16;
  smem_sweep = smem_static + (size_t)(Hh.n_crow + 2 * Hh.s_total + p.max_rows + 2) * 8 +
               (size_t)(Hh.n_cpair + p.max_rows * max_lnc + 2) * 8;
  smem_partial = (size_t)((p.max_rows + 1) & ~1) * 8 + (size_t)((max_inc + 1) & ~1) * 8 + (size_t)kFusedThreads * 4 * 8 + 64;
  if (smem_sweep > 200 * 1024 || smem_partial > 200 * 1024) return false;
  if ((size_t)Hh.img_bytes + core_bytes + own_max >= (1u << 20)) return false;
  refresh(sm, s);
  ready = true;
  return true;
}

void refresh_sweep_image(const Store& st, int prec, const ImgHeader& header, DevBuf<double>& img,
                         const DevBuf<int>& seg_src_d, const DevBuf<int>& seg_dst_d, const DevBuf<int>& seg_len_d,
                         int n_seg_copy, cudaStream_t s) {
  const DStore v = st.view();
  const int nth = 256;
  const int work = std::max(header.n_cut, n_seg_copy);
  const int grid = std::max(1, std::min(1024, (work + nth - 1) / nth));
  unsigned char* im = reinterpret_cast<unsigned char*>(img.p);
  switch (prec) {
    case EMT_PREC_FP64:
      k_img_refresh<EMT_PREC_FP64><<<grid, nth, 0, s>>>(v, im, header.off_g_bytes, header.n_cut, header.off_r_bytes,
                                                        seg_src_d.p, seg_dst_d.p, seg_len_d.p, n_seg_copy);
      break;
    case EMT_PREC_FF64:
      k_img_refresh<EMT_PREC_FF64><<<grid, nth, 0, s>>>(v, im, header.off_g_bytes, header.n_cut, header.off_r_bytes,
                                                        seg_src_d.p, seg_dst_d.p, seg_len_d.p, n_seg_copy);
      break;
    default:
      k_img_refresh<EMT_PREC_FP32><<<grid, nth, 0, s>>>(v, im, header.off_g_bytes, header.n_cut, header.off_r_bytes,
                                                        seg_src_d.p, seg_dst_d.p, seg_len_d.p, n_seg_copy);
  }
  EMT_CUDA(cudaGetLastError());
}

// K[:, c] = s for y_cut = e_c: the boundary sweep (every tree node, bottom-up) is linear in the
// cut-row values, so one sweep per unit vector gives the matrix of the whole sweep. One CTA per
// column; rows of K have leading dimension ldk (zero beyond n_crow). The image and cores are
// staged in shared memory when they fit, else read from global memory (L2).
template <int PREC>
__global__ void k_build_K(const unsigned char* __restrict__ img, int img_bytes, const unsigned char* __restrict__ cores,
                          int core_bytes, int staged, int n_crow, int s_total, int ldk,
                          typename Acc<PREC>::T* __restrict__ K) {
  using A = Acc<PREC>;
  using X = typename A::X;
  extern __shared__ __align__(16) unsigned char smk[];
  const unsigned char* im = img;
  const unsigned char* co = cores;
  unsigned char* vec = smk;
  if (staged) {
    for (int i = threadIdx.x; i < img_bytes / 16; i += blockDim.x)
      reinterpret_cast<int4*>(smk)[i] = reinterpret_cast<const int4*>(img)[i];
    for (int i = threadIdx.x; i < core_bytes / 16; i += blockDim.x)
      reinterpret_cast<int4*>(smk + img_bytes)[i] = reinterpret_cast<const int4*>(cores)[i];
    im = smk;
    co = smk + img_bytes;
    vec = smk + img_bytes + core_bytes;
  }
  X* ycut = reinterpret_cast<X*>(vec);
  X* t = ycut + n_crow;
  X* sv = t + s_total;
  const int c = blockIdx.x;
  for (int i = threadIdx.x; i < n_crow; i += blockDim.x) ycut[i] = A::prep(i == c ? 1.0 : 0.0);
  __syncthreads();
  sweep_levels<PREC, 8>(im, co, ycut, t, sv);
  for (int r = threadIdx.x; r < s_total; r += blockDim.x) K[(int64_t)r * ldk + c] = sv[r];
}

void build_sweep_matrix(int prec, const unsigned char* img, int img_bytes, const unsigned char* cores, int core_bytes,
                        int n_crow, int s_total, int ldk, void* K, cudaStream_t s) {
  if (n_crow == 0 || s_total == 0) return;
  const size_t vec = (size_t)(n_crow + 2 * s_total) * 8;
  int dev = 0, optin = 0;
  EMT_CUDA(cudaGetDevice(&dev));
  EMT_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const int staged = (size_t)img_bytes + (size_t)core_bytes + vec <= (size_t)optin ? 1 : 0;
  const size_t smem_k = vec + (staged ? (size_t)img_bytes + (size_t)core_bytes : 0);
  EMT_REQUIRE(smem_k <= (size_t)optin, EMT_ERR_UNSUPPORTED, "sweep vectors too large for one CTA");
  if (prec == EMT_PREC_FF64) {
    EMT_CUDA(cudaFuncSetAttribute(k_build_K<EMT_PREC_FF64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_k));
    k_build_K<EMT_PREC_FF64><<<n_crow, 256, smem_k, s>>>(img, img_bytes, cores, core_bytes, staged, n_crow, s_total, ldk,
                                                         reinterpret_cast<float2*>(K));
  } else if (prec == EMT_PREC_FP64) {
    EMT_CUDA(cudaFuncSetAttribute(k_build_K<EMT_PREC_FP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_k));
    k_build_K<EMT_PREC_FP64><<<n_crow, 256, smem_k, s>>>(img, img_bytes, cores, core_bytes, staged, n_crow, s_total, ldk,
                                                         reinterpret_cast<double*>(K));
  } else {
    EMT_CUDA(cudaFuncSetAttribute(k_build_K<EMT_PREC_FP32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_k));
    k_build_K<EMT_PREC_FP32><<<n_crow, 256, smem_k, s>>>(img, img_bytes, cores, core_bytes, staged, n_crow, s_total, ldk,
                                                         reinterpret_cast<float*>(K));
  }
  EMT_CUDA(cudaGetLastError());
}

void Step2::refresh(const Sim& sm, cudaStream_t s) {
  refresh_sweep_image(*sm.store, prec, header, img, seg_src_d, seg_dst_d, seg_len_d, n_seg_copy, s);
}

void Step2::reset_state(cudaStream_t s) {
  EMT_CUDA(cudaMemcpyAsync(inc.p, inc0.data(), inc0.size() * sizeof(IncRec), cudaMemcpyHostToDevice, s));
}

void Step2::fill_trig(const Sim& sm, int first_step, int n, cudaStream_t s) {
  if ((size_t)2 * n > trig.n) {
    trig.alloc((size_t)2 * std::max(n, 1024));
    trigff.alloc((size_t)std::max(n, 1024));
  }
  k_trig<<<(n + 255) / 256, 256, 0, s>>>(trig.p, trigff.p, first_step, n, sm.omega, sm.dt);
  EMT_CUDA(cudaGetLastError());
}

Step2D Step2::view(const Sim& sm) const {
  const Store& st = *sm.store;
  Step2D d{};
  d.inc = inc.p;
  d.src_sum = d_src_sum.p;
  d.Ih = sm.Ih.p;
  d.src = d_src.p;
  d.src_ptr = d_src_ptr.p;
  d.trig = trig.p;
  d.trigff = trigff.p;
  d.img = reinterpret_cast<const unsigned char*>(img.p);
  d.img_bytes = header.img_bytes;
  d.cores = prec == EMT_PREC_FP64 ? reinterpret_cast<const unsigned char*>(st.C64.p)
            : prec == EMT_PREC_FF64 ? reinterpret_cast<const unsigned char*>(st.Cff.p)
                                    : reinterpret_cast<const unsigned char*>(st.C32.p);
  d.core_bytes = core_bytes;
  d.fac = prec == EMT_PREC_FP64 ? reinterpret_cast<const unsigned char*>(st.F64.p)
          : prec == EMT_PREC_FF64 ? reinterpret_cast<const unsigned char*>(st.Fff.p)
                                  : reinterpret_cast<const unsigned char*>(st.F32.p);
  d.own = own_d.p;
  d.sweep_smem_static = smem_static;
  d.max_inc = max_inc;
  d.max_lnc = max_lnc;
  d.ylf = nullptr;
  return d;
}

// The element record of one end changes when a branch trips.
__global__ void k_open_rec(IncRec* inc, int m0, int m1) {
  for (int m : {m0, m1})
    if (m >= 0) {
      inc[m].g = 0.0;
      inc[m].alpha = 0.0;
      inc[m].beta = 0.0;
    }
}

void Step2::open_element(int m0, int m1, cudaStream_t s) {
  k_open_rec<<<1, 1, 0, s>>>(inc.p, m0, m1);
  EMT_CUDA(cudaGetLastError());
}

template <int PREC>
void step2_launch(Sim& sm, int n, cudaStream_t s) {
  using X = typename Acc<PREC>::X;
  const Store& st = *sm.store;
  const FusedPlan& p = sm.plan;
  const DStore v = st.view();
  const CtaMapD cm = p.cmap();
  const SimD sd = sm.view();
  const Step2D q = sm.s2.view(sm);
  X* part = reinterpret_cast<X*>(p.part.p);
  static bool attr = false;
  if (!attr) {
    EMT_CUDA(cudaFuncSetAttribute(k_step2_partial<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    EMT_CUDA(cudaFuncSetAttribute(k_step2_sweep<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr = true;
  }
  const bool refine = PREC == EMT_PREC_FP32;
  for (int i = 0; i < n; ++i) {
    launch_pdl(k_step2_partial<PREC>, p.n_cta, kFusedThreads, sm.s2.smem_partial, s, v, cm, sd, q, i, 0, part);
    launch_pdl(k_step2_sweep<PREC>, p.n_cta, kFusedThreads, sm.s2.smem_sweep, s, v, cm, sd, q, i, 0, refine ? 0 : 1,
               (const X*)part);
    if (refine) {
      launch_pdl(k_step2_partial<PREC>, p.n_cta, kFusedThreads, sm.s2.smem_partial, s, v, cm, sd, q, i, 1, part);
      launch_pdl(k_step2_sweep<PREC>, p.n_cta, kFusedThreads, sm.s2.smem_sweep, s, v, cm, sd, q, i, 1, 1,
                 (const X*)part);
    }
  }
}

// Sweep of kernel generation 3: FP64 arithmetic on the reduced leaf values `ylf`.
void step3_sweep(Sim& sm, const Step2& img, const double* ylf, int s_in_chunk, int accumulate, int record, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    EMT_CUDA(cudaFuncSetAttribute(k_step2_sweep<EMT_PREC_FP64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  200 * 1024));
    attr = true;
  }
  Step2D q = img.view(sm);
  q.ylf = ylf;
  launch_pdl(k_step2_sweep<EMT_PREC_FP64, true>, sm.plan.n_cta, kFusedThreads, img.smem_sweep, s, sm.store->view(),
             sm.plan.cmap(), sm.view(), q, s_in_chunk, accumulate, record, (const double*)nullptr);
}

void step2_launch_any(Sim& sm, int n, cudaStream_t s) {
  switch (sm.store->precision) {
    case EMT_PREC_FP64: step2_launch<EMT_PREC_FP64>(sm, n, s); break;
    case EMT_PREC_FF64: step2_launch<EMT_PREC_FF64>(sm, n, s); break;
    default: step2_launch<EMT_PREC_FP32>(sm, n, s); break;
  }
}

void step2_bench(Sim& sm, int which, int reps, cudaStream_t s) {
  // same kernels with the current arguments, back to back (PDL edges as in the step graph)
  for (int i = 0; i < reps; ++i) {
    switch (sm.store->precision) {
      case EMT_PREC_FP64: {
        using X = typename Acc<EMT_PREC_FP64>::X;
        X* part = reinterpret_cast<X*>(sm.plan.part.p);
        if (which == 0)
          launch_pdl(k_step2_partial<EMT_PREC_FP64>, sm.plan.n_cta, kFusedThreads, sm.s2.smem_partial, s,
                     sm.store->view(), sm.plan.cmap(), sm.view(), sm.s2.view(sm), 0, 0, part);
        else
          launch_pdl(k_step2_sweep<EMT_PREC_FP64>, sm.plan.n_cta, kFusedThreads, sm.s2.smem_sweep, s, sm.store->view(),
                     sm.plan.cmap(), sm.view(), sm.s2.view(sm), 0, 0, 0, (const X*)part);
        break;
      }
      case EMT_PREC_FF64: {
        using X = typename Acc<EMT_PREC_FF64>::X;
        X* part = reinterpret_cast<X*>(sm.plan.part.p);
        if (which == 0)
          launch_pdl(k_step2_partial<EMT_PREC_FF64>, sm.plan.n_cta, kFusedThreads, sm.s2.smem_partial, s,
                     sm.store->view(), sm.plan.cmap(), sm.view(), sm.s2.view(sm), 0, 0, part);
        else
          launch_pdl(k_step2_sweep<EMT_PREC_FF64>, sm.plan.n_cta, kFusedThreads, sm.s2.smem_sweep, s, sm.store->view(),
                     sm.plan.cmap(), sm.view(), sm.s2.view(sm), 0, 0, 0, (const X*)part);
        break;
      }
      default: {
        using X = typename Acc<EMT_PREC_FP32>::X;
        X* part = reinterpret_cast<X*>(sm.plan.part.p);
        if (which == 0)
          launch_pdl(k_step2_partial<EMT_PREC_FP32>, sm.plan.n_cta, kFusedThreads, sm.s2.smem_partial, s,
                     sm.store->view(), sm.plan.cmap(), sm.view(), sm.s2.view(sm), 0, 0, part);
        else
          launch_pdl(k_step2_sweep<EMT_PREC_FP32>, sm.plan.n_cta, kFusedThreads, sm.s2.smem_sweep, s, sm.store->view(),
                     sm.plan.cmap(), sm.view(), sm.s2.view(sm), 0, 0, 0, (const X*)part);
      }
    }
  }
}

}  // namespace emt

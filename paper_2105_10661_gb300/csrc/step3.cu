// Third-generation single-column step kernels.
//
// Leaf stage: one thread-block cluster per leaf (cs CTAs, cs <= 8). Each CTA bulk-copies its
// rows of the leaf inverse into shared memory with cp.async.bulk before griddepcontrol.wait,
// forms its partial vector part_c = sum_{r in rows} L[r, :] x_r (the symmetry of L), and the
// cluster then reduces the cs partial vectors through distributed shared memory: CTA q sums
// slice q of the leaf over all cs CTAs' shared memory (fixed rank order, deterministic) and
// writes one value per position. The boundary sweep that follows (step2.cu, FP64 arithmetic)
// therefore reads one value per cut row instead of one per CTA of the leaf; its small dot
// products run as plain FP64, which here costs fewer dependent instructions than float-float.
#include <algorithm>

#include "sim.h"

namespace emt {

namespace {

__device__ __forceinline__ void pdl_launch_dependents3() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait3() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ uint32_t sa3(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t map_to(uint32_t local_addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local_addr), "r"(rank));
  return r;
}
__device__ __forceinline__ float2 dsmem_ld(uint32_t addr, float2*) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ double dsmem_ld(uint32_t addr, double*) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ float dsmem_ld(uint32_t addr, float*) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}
constexpr long long kWait3 = 4000000000LL;
__device__ __forceinline__ bool bar3_wait(uint64_t* bar) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(sa3(bar))
                 : "memory");
    if (ok) return true;
    if (clock64() - t0 > kWait3) return false;
  }
}

// Cluster leaf stage of Eq. 2 with the history update and injection of Eq. 1 (header above).
template <int PREC>
__global__ void __launch_bounds__(kFusedThreads) k_step3_partial(DStore st, SimD sim, Step2D q, int cs, int s_in_chunk,
                                                                 int pass, int max_rows, double* __restrict__ ylf) {
  using A = Acc<PREC>;
  using X = typename A::X;
  using T = typename A::T;
  constexpr int VE = Elem<PREC>::VE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  const int j = blockIdx.x / cs;
  const int rank = (int)cluster_rank();
  const int node = st.leaf_node[j];
  const int lo = st.lo[node];
  const int b = st.hi[node] - lo;
  const int ld = st.leaf_ld[j];
  const int r0 = (int)((int64_t)b * rank / cs), r1 = (int)((int64_t)b * (rank + 1) / cs);
  const int nrow = r1 - r0;
  T* Ls = reinterpret_cast<T*>(smem_raw + 16);                           // [max_rows][ld]
  X* xs = reinterpret_cast<X*>(smem_raw + 16 + (size_t)max_rows * ld * sizeof(T));
  double* contrib = reinterpret_cast<double*>(xs + ((max_rows + 1) & ~1));
  X* mypart = reinterpret_cast<X*>(contrib + ((q.max_inc + 1) & ~1));  // [ld]
  X* red = mypart + ld;
  const int tid = threadIdx.x;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa3(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const uint32_t bytes = (uint32_t)((size_t)nrow * ld * sizeof(T));
    if (bytes) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa3(bar)), "r"(bytes) : "memory");
      const T* src = Elem<PREC>::L(st) + st.leaf_off[j] + (int64_t)r0 * ld;
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sa3(Ls)),
          "l"(src), "r"(bytes), "r"(sa3(bar))
          : "memory");
    } else {
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa3(bar)) : "memory");
    }
  }
  // static prefetch of the owned rows' element records and row data
  const int m0 = sim.inc_ptr[lo + r0];
  const int m1 = sim.inc_ptr[lo + r1];
  IncRec rec{};
  const bool has_inc = pass == 0 && tid < m1 - m0;
  if (has_inc) rec = q.inc[m0 + tid];
  const bool has_row = tid < nrow;
  const int pos = lo + r0 + tid;
  int rm0 = 0, rm1 = 0;
  double2 ssum = make_double2(0.0, 0.0);
  if (has_row && pass == 0) {
    rm0 = sim.inc_ptr[pos] - m0;
    rm1 = sim.inc_ptr[pos + 1] - m0;
    ssum = q.src_sum[pos];
  }
  __syncthreads();
  pdl_launch_dependents3();
  pdl_wait3();
  const bool bad = *st.status != DEV_OK;
  if (!bad) {
    const int step = sim.dyn->step_base + s_in_chunk + 1;
    if (pass == 0) {
      const int ti = step - sim.dyn->trig_first;
      const double sw = q.trig[2 * ti], cw = q.trig[2 * ti + 1];
      for (int m = tid; m < m1 - m0; m += kFusedThreads) {
        const IncRec rr = m == tid ? rec : q.inc[m0 + m];
        const double vi = sim.v_pos[rr.self];
        const double vo = rr.other >= 0 ? sim.v_pos[rr.other] : 0.0;
        const double Ih = q.Ih[m0 + m];
        const double ve = rr.sgn > 0 ? vi - vo : vo - vi;
        const double cur = rr.g * ve + Ih;
        const double Ihn = rr.alpha * ve + rr.beta * cur;
        q.Ih[m0 + m] = Ihn;
        contrib[m] = rr.sgn > 0 ? -Ihn : Ihn;
      }
      __syncthreads();
      for (int r = tid; r < nrow; r += kFusedThreads) {
        const int p = lo + r0 + r;
        double hist = 0.0;
        const int a0 = r == tid ? rm0 : sim.inc_ptr[p] - m0;
        const int a1 = r == tid ? rm1 : sim.inc_ptr[p + 1] - m0;
        for (int m = a0; m < a1; ++m) hist += contrib[m];
        const double2 ss = r == tid ? ssum : q.src_sum[p];
        const double x = ss.x * sw + ss.y * cw + hist;
        if (sim.x_pos) sim.x_pos[p] = x;
        xs[r] = A::prep(x);
      }
    } else {
      for (int r = tid; r < nrow; r += kFusedThreads) {
        const int p = lo + r0 + r;
        double acc = sim.x_pos[p];
        for (int t = sim.csr_ptr[p]; t < sim.csr_ptr[p + 1]; ++t) acc -= sim.csr_val[t] * sim.v_pos[sim.csr_col[t]];
        xs[r] = A::prep(acc);
      }
    }
  }
  // wait for the leaf rows (bounded) even on the error path, so the copy has landed before exit
  bool okc = true;
  if (!bar3_wait(bar)) {
    okc = false;
    if (tid == 0) atomicExch(st.status, DEV_TIMEOUT);
  }
  __syncthreads();
  if (!bad && okc) {
    // part[col] = sum_r L[r, col] x_r, columns in 16-byte slots, rows split over G groups
    const int slots = (b + VE - 1) / VE;
    const int cover = min(slots, kFusedThreads);
    const int G = kFusedThreads / cover;
    const int g = tid / cover, sl = tid % cover;
    const int width = slots * VE;
    if (g < G) {
      for (int s0 = sl; s0 < slots; s0 += cover) {
        A acc0[VE], acc1[VE];
        int r = g;
        for (; r + G < nrow; r += 2 * G) {
          const X xa = xs[r], xb = xs[r + G];
#pragma unroll
          for (int e = 0; e < VE; ++e) {
            acc0[e].fma(Ls[(size_t)r * ld + s0 * VE + e], xa);
            acc1[e].fma(Ls[(size_t)(r + G) * ld + s0 * VE + e], xb);
          }
        }
        if (r < nrow) {
          const X xa = xs[r];
#pragma unroll
          for (int e = 0; e < VE; ++e) acc0[e].fma(Ls[(size_t)r * ld + s0 * VE + e], xa);
        }
#pragma unroll
        for (int e = 0; e < VE; ++e) {
          acc0[e].add(acc1[e].getx());
          red[(size_t)g * width + s0 * VE + e] = acc0[e].getx();
        }
      }
    }
    __syncthreads();
    for (int col = tid; col < b; col += kFusedThreads) {
      A sum;
      for (int gg = 0; gg < G; ++gg) sum.add(red[(size_t)gg * width + col]);
      mypart[col] = sum.getx();
    }
  } else {
    for (int col = tid; col < b; col += kFusedThreads) mypart[col] = A::zero();
  }
  // cluster reduction: CTA `rank` sums slice [e0, e1) of the leaf over the cluster's partials
  cluster_sync();
  const int e0 = (int)((int64_t)b * rank / cs), e1 = (int)((int64_t)b * (rank + 1) / cs);
  for (int e = e0 + tid; e < e1; e += kFusedThreads) {
    A sum;
    const uint32_t la = sa3(&mypart[e]);
    for (int qq = 0; qq < cs; ++qq) sum.add(dsmem_ld(map_to(la, (uint32_t)qq), (X*)nullptr));
    if (!bad && okc) ylf[lo + e] = A::todbl(sum.getx());
  }
  cluster_sync();   // no CTA leaves while another still reads its shared memory
}

template <typename K, typename... Args>
void launch_cluster_pdl(K kernel, int grid, int cs, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kFusedThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  EMT_CUDA(cudaLaunchKernelEx(&cfg, kernel, args...));
}

template <int PREC>
void partial3(Sim& sm, int i, int pass, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    EMT_CUDA(cudaFuncSetAttribute(k_step3_partial<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr = true;
  }
  launch_cluster_pdl(k_step3_partial<PREC>, sm.store->n_leaf * sm.s3.cs, sm.s3.cs, sm.s3.smem_partial, s,
                     sm.store->view(), sm.view(), sm.s2.view(sm), sm.s3.cs, i, pass, sm.s3.max_rows, sm.s3.ylf.p);
}

void partial3_any(Sim& sm, int i, int pass, cudaStream_t s) {
  switch (sm.store->precision) {
    case EMT_PREC_FP64: partial3<EMT_PREC_FP64>(sm, i, pass, s); break;
    case EMT_PREC_FF64: partial3<EMT_PREC_FF64>(sm, i, pass, s); break;
    default: partial3<EMT_PREC_FP32>(sm, i, pass, s); break;
  }
}

}  // namespace

bool Step3::build(Sim& sm, int cs_, cudaStream_t s) {
  ready = false;
  const Store& st = *sm.store;
  if (!sm.s2.ready) return false;
  cs = cs_;
  if (cs < 1 || cs > 8) return false;
  maxb = 0;
  int maxld = 0;
  for (int j = 0; j < st.n_leaf; ++j) {
    const int b = st.tree.hi[st.leaf_nodes_h[j]] - st.tree.lo[st.leaf_nodes_h[j]];
    maxb = std::max(maxb, b);
    maxld = std::max(maxld, st.leaf_ld_h[j]);
  }
  if (cs > maxb) return false;
  max_rows = (maxb + cs - 1) / cs + 1;
  // element ends owned by one CTA
  max_inc = 0;
  {
    std::vector<int> iptr(sm.n + 1, 0);
    for (int p = 0; p < sm.n; ++p) iptr[p + 1] = iptr[p];
    // the incidence pointer of the simulation (same enumeration as the element records)
    std::vector<std::vector<int>> at(sm.n);
    for (size_t e = 0; e < sm.el_a.size(); ++e) {
      at[st.tree.pos[sm.el_a[e]]].push_back((int)e);
      if (sm.el_b[e] >= 0) at[st.tree.pos[sm.el_b[e]]].push_back((int)e);
    }
    for (int p = 0; p < sm.n; ++p) iptr[p + 1] = iptr[p] + (int)at[p].size();
    for (int j = 0; j < st.n_leaf; ++j) {
      const int lo = st.tree.lo[st.leaf_nodes_h[j]];
      const int b = st.tree.hi[st.leaf_nodes_h[j]] - lo;
      for (int r = 0; r < cs; ++r) {
        const int r0 = (int)((int64_t)b * r / cs), r1 = (int)((int64_t)b * (r + 1) / cs);
        max_inc = std::max(max_inc, iptr[lo + r1] - iptr[lo + r0]);
      }
    }
  }
  if (sm.s2.max_inc < max_inc) return false;   // the step2 record view sizes `contrib`
  const size_t tb = st.precision == EMT_PREC_FP32 ? 4 : 8;
  const size_t xb = 8;
  // shared memory: barrier | leaf rows | x | contrib | my partial | group reduction
  smem_partial = 16 + (size_t)max_rows * maxld * tb + (size_t)((max_rows + 1) & ~1) * xb +
                 (size_t)((sm.s2.max_inc + 1) & ~1) * 8 + (size_t)maxld * xb + (size_t)kFusedThreads * 4 * xb + 64;
  if (smem_partial > 200 * 1024) return false;
  if (!img.build(sm, s, EMT_PREC_FP64)) return false;
  ylf.alloc(sm.n);
  ylf.zero(s);
  EMT_CUDA(cudaStreamSynchronize(s));
  ready = true;
  return true;
}

void step3_launch_any(Sim& sm, int n, cudaStream_t s) {
  const bool refine = sm.store->precision == EMT_PREC_FP32;
  for (int i = 0; i < n; ++i) {
    partial3_any(sm, i, 0, s);
    step3_sweep(sm, sm.s3.img, sm.s3.ylf.p, i, 0, refine ? 0 : 1, s);
    if (refine) {
      partial3_any(sm, i, 1, s);
      step3_sweep(sm, sm.s3.img, sm.s3.ylf.p, i, 1, 1, s);
    }
  }
}

void step3_bench(Sim& sm, int which, int reps, cudaStream_t s) {
  for (int i = 0; i < reps; ++i) {
    if (which == 0) partial3_any(sm, 0, 0, s);
    else step3_sweep(sm, sm.s3.img, sm.s3.ylf.p, 0, 0, 0, s);
  }
}

}  // namespace emt

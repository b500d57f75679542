// Single-vector apply v = Ginv i (Eq. 2 with the store of Sec. III) for stores larger than the
// caches, where the bound is HBM bandwidth. Three kernels, each reading its part of the store
// once:
//   k_leaf_stream    y = blkdiag(L_j) x. One persistent CTA per SM owns a contiguous range of
//                    leaf rows (the store keeps leaves one after another, rows in position order)
//                    and streams them through a ring of shared-memory stages (two rows of a
//                    leaf each) filled by cp.async.bulk, with full/empty mbarriers; one warp per
//                    stage forms the row dots against its leaf's slice of x, held in shared memory.
//   k_sweep_matrix   s = K y_cut: the boundary sweep of every tree node is linear in the leaf-stage
//                    values at the cut rows, so it is one dense product (K built on the device from
//                    the sweep image, after every build or modification); one warp per row of K.
//   k_expand_stream  v = y - sum over ancestors q of F_q[row] . s_q(half); 16 lanes per position.
// Every wait is bounded: a timeout sets the device status word and the CTA drains its own copies
// before it returns.
#include <algorithm>
#include <climits>

#include "plan.h"
#include "step2.cuh"

namespace emt {

namespace {

constexpr int kST = 512;          // threads per CTA of the leaf stream (warp 0 produces)
constexpr int kCons = kST / 32 - 1;   // consumer warps
// Slots are a multiple of the consumer warps so that every slot has one consumer warp, which
// waits for its phases in order: a parity wait must never run ahead of the phase in flight
// (copies may land out of order, and a stage reused by another warp could match the parity of
// an older phase).
constexpr int kStages = kCons;
constexpr long long kWaitS = 4000000000LL;   // ~2 s of SM clock

__device__ __forceinline__ uint32_t sas(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void mb_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sas(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_expect(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sas(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mb_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sas(b)) : "memory");
}
// Wait for the phase of the given parity: try_wait suspends the thread in hardware for up to
// the hint (1 us) instead of spinning on issue slots; the loop gives up after `limit` SM cycles.
__device__ __forceinline__ bool mb_wait(uint64_t* b, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(sas(b)), "r"(parity), "r"(1000u)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > limit) return false;
  }
}
__device__ __forceinline__ void bulk_row(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sas(dst)),
      "l"(src), "r"(bytes), "r"(sas(b))
      : "memory");
}
// two consecutive 8-byte elements from a 16-byte aligned shared-memory address
__device__ __forceinline__ void ld2(const float2* p, float2 (&e)[2]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  e[0] = make_float2(v.x, v.y);
  e[1] = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ld2(const double* p, double (&e)[2]) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  e[0] = v.x;
  e[1] = v.y;
}

// Buffers written by an earlier grid of the same stream are read through L2 (ld.global.cg): with
// programmatic dependent launch a grid starts before its predecessor ends, so no read of such a
// buffer may go through the non-coherent or L1 path.
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float2 ldcg(const float2* p) { return __ldcg(p); }

// Copy n vector entries written by the preceding grid into shared memory, all loads of a thread
// in flight together (one DRAM round trip for up to 8 entries per thread).
template <typename X>
__device__ __forceinline__ void stage_vec(X* dst, const X* src, int n) {
  constexpr int kU = 8;
  for (int base = threadIdx.x; base < n; base += kU * blockDim.x) {
    X v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int i = base + u * blockDim.x;
      if (i < n) v[u] = ldcg(src + i);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int i = base + u * blockDim.x;
      if (i < n) dst[i] = v[u];
    }
  }
}

template <int PREC>
__device__ __forceinline__ typename Acc<PREC>::X warp_sum(const Acc<PREC>& a, int lanes) {
  using A = Acc<PREC>;
  typename A::X v = a.getx();
  for (int o = lanes >> 1; o > 0; o >>= 1) {
    A t;
    t.add(v);
    t.add(a.shfl_xor(v, o));
    v = t.getx();
  }
  return v;
}

__device__ __forceinline__ void pdl_wait_s() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_go_s() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Leaf stage of Eq. 2 (Sec. III's leaf blocks), streamed. Stages [st0[c], st0[c + 1]) of CTA c: a
// contiguous range of leaf rows (rows = positions), one or
// two rows of one leaf per stage; y in position order, vector type. y_cut (the distinct cut rows,
// in their order) is written as well. The x window [win[c].x, win[c].y) is gathered before the
// first copy is issued, so the gather does not queue behind the stream.
template <int PREC>
__global__ void __launch_bounds__(kST, 1) k_leaf_stream(DStore st, const StreamStage* __restrict__ stages,
                                                        const int* __restrict__ st0, const int2* __restrict__ win,
                                                        const double* src, int src_pos,
                                                        typename Acc<PREC>::X* __restrict__ y,
                                                        typename Acc<PREC>::X* __restrict__ ycut, int stage_elems,
                                                        int max_stages) {
  using A = Acc<PREC>;
  using X = typename A::X;
  using T = typename A::T;
  extern __shared__ __align__(128) unsigned char sml[];
  uint64_t* full = reinterpret_cast<uint64_t*>(sml);
  uint64_t* empty = full + kStages;
  int* misc = reinterpret_cast<int*>(empty + kStages);   // [0] abort flag
  T* stage = reinterpret_cast<T*>(sml + 16 * kStages + 16);
  StreamStage* sr = reinterpret_cast<StreamStage*>(stage + (size_t)kStages * stage_elems);
  X* xw = reinterpret_cast<X*>(sr + max_stages);
  const int c = blockIdx.x;
  const int u0 = st0[c], nst = st0[c + 1] - u0;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  pdl_go_s();
  if (nst <= 0) return;
  const int2 w = win[c];
  const int wlo = w.x, whi = w.y;
  const T* L = Elem<PREC>::L(st);
  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      mb_init(&full[i], 1);
      mb_init(&empty[i], 1);
    }
    misc[0] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // stage table (built on the host; static per store)
  for (int u = tid; u < nst; u += kST) sr[u] = stages[u0 + u];
  pdl_wait_s();
  {
    // gather in batches: all index loads of a thread, then all value loads (two round trips)
    constexpr int kG = 4;
    for (int base = wlo + tid; base < whi + 2; base += kG * kST) {
      int idx[kG];
#pragma unroll
      for (int u = 0; u < kG; ++u) {
        const int p = base + u * kST;
        idx[u] = p < whi ? (src_pos ? p : st.perm[p]) : -1;
      }
      double val[kG];
#pragma unroll
      for (int u = 0; u < kG; ++u) val[u] = idx[u] >= 0 ? ldcg(src + idx[u]) : 0.0;
#pragma unroll
      for (int u = 0; u < kG; ++u) {
        const int p = base + u * kST;
        if (p < whi + 2) xw[p - wlo] = A::prep(val[u]);
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    // producer: one stage (1-2 rows) per slot; a slot is refilled after its consumer released it
    if (lane == 0) {
      int issued = 0;
      bool ok = true;
      for (int u = 0; u < nst && ok; ++u) {
        const int s = u % kStages;
        if (u >= kStages) ok = mb_wait(&empty[s], (uint32_t)(((u / kStages) - 1) & 1), kWaitS);
        if (!ok) break;
        const StreamStage q = sr[u];
        const uint32_t bytes = (uint32_t)(q.ld * q.nr) * (uint32_t)sizeof(T);
        mb_expect(&full[s], bytes);
        bulk_row(stage + (size_t)s * stage_elems, L + q.off, bytes, &full[s]);
        ++issued;
      }
      if (!ok) {
        atomicExch(st.status, DEV_TIMEOUT);
        atomicExch(&misc[0], 1);
        // drain: copies issued to slots no consumer will read
        for (int u = issued > kStages ? issued - kStages : 0; u < issued; ++u)
          mb_wait(&full[u % kStages], (uint32_t)((u / kStages) & 1), kWaitS);
      }
    }
  } else {
    // warp w takes stages w-1, w-1+kCons, ... (slots w-1 and w-1+kCons only)
    for (int u = warp - 1; u < nst; u += kCons) {
      const int s = u % kStages;
      const bool ok = mb_wait(&full[s], (uint32_t)((u / kStages) & 1), kWaitS);
      if (!ok || *reinterpret_cast<volatile int*>(&misc[0])) {
        if (lane == 0) atomicExch(st.status, DEV_TIMEOUT);
        break;
      }
      const StreamStage q = sr[u];
      const X* xr = xw + q.xo;
      const int p0 = q.p;
      for (int rr = 0; rr < q.nr; ++rr) {
        const T* Lr = stage + (size_t)s * stage_elems + (size_t)rr * q.ld;
        A a, a2;
#pragma unroll 4
        for (int col = 2 * lane; col < q.b; col += 64) {
          T l2[2];
          ld2(Lr + col, l2);   // stage rows are 16-byte aligned; the x window need not be
          a.fma(l2[0], xr[col]);
          a2.fma(l2[1], xr[col + 1]);
        }
        a.add(a2.getx());
        const X v = warp_sum<PREC>(a, 32);
        if (lane == 0) {
          y[p0 + rr] = v;
          const int kc = rr == 0 ? q.crow0 : q.crow1;
          if (kc >= 0) ycut[kc] = v;
        }
      }
      __syncwarp();
      if (lane == 0) mb_arrive(&empty[s]);
    }
  }
}

// Leaf stage with plain 16-byte global loads (no staging): one persistent CTA of 768 threads per
// SM over the same row range; warp w takes rows w, w+24, ...; a lane issues all loads of its
// part of a row (up to kLdgChunk pairs) before the first product, so each warp keeps one row in
// flight.
constexpr int kLT = 768;
constexpr int kLdgChunk = 12;   // 16-byte loads per lane per pass (rows up to 768 elements)
template <int PREC>
__global__ void __launch_bounds__(kLT, 1) k_leaf_ldg(DStore st, const int* __restrict__ row0,
                                                     const int* __restrict__ crow_of, const double* src,
                                                     int src_pos, typename Acc<PREC>::X* __restrict__ y,
                                                     typename Acc<PREC>::X* __restrict__ ycut) {
  using A = Acc<PREC>;
  using X = typename A::X;
  using T = typename A::T;
  extern __shared__ __align__(16) unsigned char smg[];
  X* xw = reinterpret_cast<X*>(smg);
  const int c = blockIdx.x;
  const int r0 = row0[c], r1 = row0[c + 1];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  pdl_go_s();
  if (r1 <= r0) return;
  const int j0 = st.pos_leaf[r0], j1 = st.pos_leaf[r1 - 1];
  const int wlo = st.lo[st.leaf_node[j0]], whi = st.hi[st.leaf_node[j1]];
  const T* L = Elem<PREC>::L(st);
  pdl_wait_s();
  {
    constexpr int kG = 4;
    for (int base = wlo + tid; base < whi + 2; base += kG * kLT) {
      int idx[kG];
#pragma unroll
      for (int u = 0; u < kG; ++u) {
        const int p = base + u * kLT;
        idx[u] = p < whi ? (src_pos ? p : st.perm[p]) : -1;
      }
      double val[kG];
#pragma unroll
      for (int u = 0; u < kG; ++u) val[u] = idx[u] >= 0 ? ldcg(src + idx[u]) : 0.0;
#pragma unroll
      for (int u = 0; u < kG; ++u) {
        const int p = base + u * kLT;
        if (p < whi + 2) xw[p - wlo] = A::prep(val[u]);
      }
    }
  }
  __syncthreads();
  for (int i = warp; i < r1 - r0; i += kLT / 32) {
    const int p = r0 + i;
    const int j = st.pos_leaf[p];
    const int node = st.leaf_node[j];
    const int lo = st.lo[node];
    const int b = st.hi[node] - lo;
    const int ld = st.leaf_ld[j];
    const T* Lr = L + st.leaf_off[j] + (int64_t)(p - lo) * ld;
    const X* xr = xw + (lo - wlo);
    A a, a2;
    for (int base = 0; base < b; base += 64 * kLdgChunk) {
      T l[kLdgChunk][2];
#pragma unroll
      for (int m = 0; m < kLdgChunk; ++m) {
        const int col = base + 2 * lane + 64 * m;
        if (col < b) vload(Lr + col, l[m]);
        else l[m][0] = l[m][1] = T{};
      }
#pragma unroll
      for (int m = 0; m < kLdgChunk; ++m) {
        const int col = base + 2 * lane + 64 * m;
        if (col < b) {
          a.fma(l[m][0], xr[col]);
          a2.fma(l[m][1], xr[col + 1]);
        }
      }
    }
    a.add(a2.getx());
    const X v = warp_sum<PREC>(a, 32);
    if (lane == 0) {
      y[p] = v;
      const int kc = crow_of[p];
      if (kc >= 0) ycut[kc] = v;
    }
  }
}

// s = K y_cut, the boundary sweep of every node (Eq. 9's t_p and s_p = C_p t_p are linear in the
// cut-row values): y_cut staged in shared memory, one warp per row of K
template <int PREC>
__global__ void __launch_bounds__(128) k_sweep_matrix(const typename Acc<PREC>::T* __restrict__ K, int s_total, int ldk,
                                                      int n_crow, const typename Acc<PREC>::X* ycut_g,
                                                      typename Acc<PREC>::X* __restrict__ s) {
  using A = Acc<PREC>;
  using X = typename A::X;
  using T = typename A::T;
  extern __shared__ __align__(16) unsigned char smk2[];
  X* yc = reinterpret_cast<X*>(smk2);
  pdl_go_s();
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const T* Kr = K + (int64_t)(row < s_total ? row : 0) * ldk;
  pdl_wait_s();
  stage_vec(yc, ycut_g, n_crow);
  __syncthreads();
  if (row >= s_total) return;
  A a, a2;
  constexpr int kU = 18;   // loads in flight per lane (one pass for up to 576 cut rows)
  for (int base = 0; base < n_crow; base += 32 * kU) {
    T kv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int k = base + lane + 32 * u;
      kv[u] = k < n_crow ? Kr[k] : T{};
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int k = base + lane + 32 * u;
      if (k < n_crow) {
        if (u & 1) a2.fma(kv[u], yc[k]);
        else a.fma(kv[u], yc[k]);
      }
    }
  }
  a.add(a2.getx());
  const X v = warp_sum<PREC>(a, 32);
  if (lane == 0) s[row] = v;
}

// v = y - sum over ancestors of F row . s(half) (the expansion with Eq. 9's factors); 16 lanes per
// position, two positions per warp.
// s and the ancestor records sit in shared memory. A lane takes elements lane + 16 m (m < 4) of
// every ancestor's factor row (k <= 64 per pass; longer rows take further passes), and the loads
// of up to kMaxAnc ancestors (deeper paths take further rounds) are all issued before the first
// product, so a position costs about one DRAM round trip per round.
constexpr int kMaxAnc = 4;
constexpr int kEL = 16;   // lanes per position
template <int PREC>
__global__ void __launch_bounds__(256, 4) k_expand_stream(DStore st, const StreamAnc* __restrict__ anc,
                                                       const int* __restrict__ anc_ptr, int n_anc, int s_total,
                                                       const typename Acc<PREC>::X* y,
                                                       const typename Acc<PREC>::X* s_g, double* __restrict__ v_pos,
                                                       double* __restrict__ v_bus, int accumulate) {
  using A = Acc<PREC>;
  using X = typename A::X;
  using T = typename A::T;
  extern __shared__ __align__(16) unsigned char sme[];
  StreamAnc* an = reinterpret_cast<StreamAnc*>(sme);
  X* ss = reinterpret_cast<X*>(an + n_anc);
  pdl_go_s();
  for (int i = threadIdx.x; i < n_anc; i += blockDim.x) an[i] = anc[i];
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) / kEL;
  const int gl = threadIdx.x % kEL;
  const bool valid = p < st.n;
  const int pp = valid ? p : 0;
  const int j = st.pos_leaf[pp];
  const int lo = st.lo[st.leaf_node[j]];
  const int x0 = anc_ptr[j], x1 = valid ? anc_ptr[j + 1] : anc_ptr[j];
  pdl_wait_s();
  const X yp = ldcg(y + pp);   // in flight with the loads below
  stage_vec(ss, s_g, s_total);
  __syncthreads();
  const T* F = Elem<PREC>::F(st);
  A a, a2;
  int kmax = 0;
  for (int x = x0; x < x1; ++x) kmax = max(kmax, an[x].k);
  for (int base = 0; base < kmax; base += 4 * kEL) {
    for (int xb = x0; xb < x1; xb += kMaxAnc) {
      T f[kMaxAnc][4];
#pragma unroll
      for (int u = 0; u < kMaxAnc; ++u) {
        const int x = xb + u;
        const bool ax = x < x1;
        const StreamAnc r = an[ax ? x : x0];
        const T* Fr = F + r.foff + (int64_t)(pp - lo) * r.kld;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int e = base + gl + kEL * m;
          f[u][m] = (ax && e < r.k) ? Fr[e] : T{};
        }
      }
#pragma unroll
      for (int u = 0; u < kMaxAnc; ++u) {
        const int x = xb + u;
        if (x < x1) {
          const StreamAnc r = an[x];
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const int e = base + gl + kEL * m;
            if (e < r.k) {
              if (m & 1) a2.fma(f[u][m], neg(ss[r.sidx + e]));
              else a.fma(f[u][m], neg(ss[r.sidx + e]));
            }
          }
        }
      }
    }
  }
  a.add(a2.getx());
  const X w = warp_sum<PREC>(a, kEL);
  if (valid && gl == 0) {
    A f;
    f.add(yp);
    f.add(w);
    double out = A::todbl(f.getx());
    if (accumulate) out += v_pos[pp];
    if (v_pos) v_pos[pp] = out;
    if (v_bus) v_bus[st.perm[pp]] = out;
  }
}

template <typename K, typename... Args>
void launch_pdl_s(K kernel, int grid, int block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  EMT_CUDA(cudaLaunchKernelEx(&cfg, kernel, args...));
}

template <int PREC>
void launch_stream(const Store& st, StreamApply& sa, const double* src, bool src_pos, double* v_pos, double* v_bus,
                   bool acc, cudaStream_t s) {
  using A = Acc<PREC>;
  using X = typename A::X;
  using T = typename A::T;
  const DStore v = st.view();
  X* y = reinterpret_cast<X*>(sa.y.p);
  X* yc = reinterpret_cast<X*>(sa.ycut.p);
  X* sv = reinterpret_cast<X*>(sa.sv.p);
  if (sa.ldg)
    launch_pdl_s(k_leaf_ldg<PREC>, sa.n_cta, kLT, sa.smem_ldg, s, v, (const int*)sa.row0.p, (const int*)sa.crow_of.p,
                 src, src_pos ? 1 : 0, y, yc);
  else
    launch_pdl_s(k_leaf_stream<PREC>, sa.n_cta, kST, sa.smem, s, v, (const StreamStage*)sa.stages.p,
                 (const int*)sa.st0.p, (const int2*)sa.win.p, src, src_pos ? 1 : 0, y, yc, sa.stage_elems,
                 sa.max_stages);
  if (sa.s_total > 0 && sa.n_crow > 0) {
    const int wpb = 4;
    launch_pdl_s(k_sweep_matrix<PREC>, (sa.s_total + wpb - 1) / wpb, wpb * 32, (size_t)sa.n_crow * 8, s,
                 (const T*)sa.K.p, sa.s_total, sa.ldk, sa.n_crow, (const X*)yc, sv);
  }
  const int th = 256;
  const size_t smem_e = (size_t)sa.n_anc * sizeof(StreamAnc) + (size_t)std::max(sa.s_total, 1) * 8;
  launch_pdl_s(k_expand_stream<PREC>, (st.n + th / 16 - 1) / (th / 16), th, smem_e, s, v, (const StreamAnc*)sa.anc.p,
               (const int*)sa.anc_ptr.p, sa.n_anc, sa.s_total, (const X*)y, (const X*)sv, v_pos, v_bus, acc ? 1 : 0);
}

}  // namespace

// Whether the streaming kernels serve this store: FP64 or float-float storage large enough that
// the leaf blocks do not stay in L2 between applications.
bool stream_apply_wanted(const Store& st) {
  return (st.precision == EMT_PREC_FF64 || st.precision == EMT_PREC_FP64) && st.L_elems * 8 >= (int64_t)48 << 20;
}

bool StreamApply::build(const Store& st, cudaStream_t s) {
  ready = false;
  const Tree& t = st.tree;
  prec = st.precision;
  int dev = 0, sms = 0, optin = 0;
  EMT_CUDA(cudaGetDevice(&dev));
  EMT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  EMT_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // rows split into n_cta contiguous ranges of about equal bytes
  const int n = st.n;
  std::vector<int64_t> rb(n + 1, 0);
  int max_ld = 0;
  for (int j = 0; j < st.n_leaf; ++j) {
    const int node = st.leaf_nodes_h[j];
    for (int p = t.lo[node]; p < t.hi[node]; ++p) rb[p + 1] = st.leaf_ld_h[j];
    max_ld = std::max(max_ld, st.leaf_ld_h[j]);
  }
  for (int p = 0; p < n; ++p) rb[p + 1] += rb[p];
  n_cta = std::max(1, std::min(sms, n));
  std::vector<int> r0(n_cta + 1, 0);
  for (int c = 1; c < n_cta; ++c) {
    const int64_t target = rb[n] * c / n_cta;
    r0[c] = (int)(std::lower_bound(rb.begin(), rb.end(), target) - rb.begin());
    r0[c] = std::max(r0[c], r0[c - 1]);
  }
  r0[n_cta] = n;
  // shared memory: barriers, stages of one row, x window of the CTA's leaves (+2 zero pads)
  stage_elems = 2 * ((max_ld + 1) / 2 * 2);   // two rows of the widest leaf
  size_t max_win = 0;
  for (int c = 0; c < n_cta; ++c) {
    if (r0[c + 1] <= r0[c]) continue;
    const int j0 = leaf_index_of_pos(st, r0[c]), j1 = leaf_index_of_pos(st, r0[c + 1] - 1);
    max_win = std::max(max_win, (size_t)(t.hi[st.leaf_nodes_h[j1]] - t.lo[st.leaf_nodes_h[j0]]));
  }
  // stage table: per CTA, rows paired within each leaf (a leaf boundary starts a new pair)
  std::vector<int> cro(n, -1);
  for (size_t k = 0; k < st.cut_rows.crow_pos.size(); ++k) cro[st.cut_rows.crow_pos[k]] = (int)k;
  std::vector<StreamStage> stg;
  std::vector<int> s0v(n_cta + 1, 0);
  std::vector<int2> wv(n_cta, make_int2(0, 0));
  max_stages = 0;
  for (int c = 0; c < n_cta; ++c) {
    s0v[c] = (int)stg.size();
    if (r0[c + 1] > r0[c]) {
      const int jf = leaf_index_of_pos(st, r0[c]), jl = leaf_index_of_pos(st, r0[c + 1] - 1);
      const int wlo = t.lo[st.leaf_nodes_h[jf]];
      wv[c] = make_int2(wlo, t.hi[st.leaf_nodes_h[jl]]);
      for (int q = r0[c]; q < r0[c + 1];) {
        const int j = leaf_index_of_pos(st, q);
        const int lo = t.lo[st.leaf_nodes_h[j]];
        const int hq = std::min(t.hi[st.leaf_nodes_h[j]], r0[c + 1]);
        for (int p = q; p < hq; p += 2) {
          StreamStage g{};
          g.ld = st.leaf_ld_h[j];
          g.off = st.leaf_off_h[j] + (int64_t)(p - lo) * g.ld;
          g.nr = p + 1 < hq ? 2 : 1;
          g.xo = lo - wlo;
          g.b = t.hi[st.leaf_nodes_h[j]] - lo;
          g.crow0 = cro[p];
          g.crow1 = g.nr == 2 ? cro[p + 1] : -1;
          g.p = p;
          stg.push_back(g);
        }
        q = hq;
      }
    }
    max_stages = std::max(max_stages, (int)stg.size() - s0v[c]);
  }
  s0v[n_cta] = (int)stg.size();
  smem = 16 * kStages + 16 + (size_t)kStages * stage_elems * 8 + (size_t)max_stages * sizeof(StreamStage) +
         (max_win + 2) * 8;
  if (smem + 1024 > (size_t)optin) return false;
  smem_ldg = (max_win + 2) * 8;
  row0.upload(r0, s);
  stages.upload(stg.empty() ? std::vector<StreamStage>{StreamStage{}} : stg, s);
  st0.upload(s0v, s);
  win.upload(wv, s);
  // sweep matrix
  build_sweep_image(st, nullptr, prec, hdr, img, seg_src, seg_dst, seg_len, n_seg, s);
  n_crow = hdr.n_crow;
  s_total = hdr.s_total;
  ldk = (n_crow + 1) / 2 * 2;
  K.alloc(std::max<size_t>((size_t)s_total * ldk, 1));
  EMT_CUDA(cudaMemsetAsync(K.p, 0, K.n * 8, s));
  {
    std::vector<int> co(n, -1);
    for (size_t k = 0; k < st.cut_rows.crow_pos.size(); ++k) co[st.cut_rows.crow_pos[k]] = (int)k;
    crow_of.upload(co, s);
  }
  ycut.alloc(std::max(n_crow, 1));
  // ancestor records per leaf
  std::vector<StreamAnc> an;
  std::vector<int> ap(st.n_leaf + 1, 0);
  for (int j = 0; j < st.n_leaf; ++j) {
    const int leaf = st.leaf_nodes_h[j];
    const int lo = t.lo[leaf];
    for (int a = t.parent[leaf]; a >= 0; a = t.parent[a]) {
      const int k = st.node_k_h[a];
      const int kld = st.node_kld_h[a];
      if (k == 0) continue;
      StreamAnc r{};
      r.foff = st.node_foff_h[a] + (int64_t)(lo - t.lo[a]) * kld;
      r.kld = kld;
      r.k = k;
      r.sidx = st.node_soff_h[a] + (lo < t.hi[t.left[a]] ? 0 : k);
      an.push_back(r);
    }
    ap[j + 1] = (int)an.size();
  }
  if (an.empty()) an.push_back(StreamAnc{});
  n_anc = (int)an.size();
  anc.upload(an, s);
  anc_ptr.upload(ap, s);
  y.alloc(std::max(n, 1));
  sv.alloc(std::max(s_total, 1));
  const int smem_k = (int)((size_t)std::max(n_crow, 1) * 8);
  const int smem_e = (int)((size_t)n_anc * sizeof(StreamAnc) + (size_t)std::max(s_total, 1) * 8);
  if (smem_k > 200 * 1024 || smem_e > 200 * 1024) return false;
  if (prec == EMT_PREC_FF64) {
    EMT_CUDA(cudaFuncSetAttribute(k_leaf_ldg<EMT_PREC_FF64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_ldg));
    EMT_CUDA(cudaFuncSetAttribute(k_leaf_stream<EMT_PREC_FF64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    EMT_CUDA(cudaFuncSetAttribute(k_sweep_matrix<EMT_PREC_FF64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_k));
    EMT_CUDA(cudaFuncSetAttribute(k_expand_stream<EMT_PREC_FF64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_e));
  } else {
    EMT_CUDA(cudaFuncSetAttribute(k_leaf_ldg<EMT_PREC_FP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_ldg));
    EMT_CUDA(cudaFuncSetAttribute(k_leaf_stream<EMT_PREC_FP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    EMT_CUDA(cudaFuncSetAttribute(k_sweep_matrix<EMT_PREC_FP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_k));
    EMT_CUDA(cudaFuncSetAttribute(k_expand_stream<EMT_PREC_FP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_e));
  }
  ready = true;
  refresh(st, s);
  EMT_CUDA(cudaStreamSynchronize(s));
  return true;
}

void StreamApply::refresh(const Store& st, cudaStream_t s) {
  if (!ready) return;
  refresh_sweep_image(st, prec, hdr, img, seg_src, seg_dst, seg_len, n_seg, s);
  const unsigned char* cores = prec == EMT_PREC_FF64 ? reinterpret_cast<const unsigned char*>(st.Cff.p)
                                                     : reinterpret_cast<const unsigned char*>(st.C64.p);
  build_sweep_matrix(prec, reinterpret_cast<const unsigned char*>(img.p), hdr.img_bytes, cores,
                     (int)(st.C_elems * 8), n_crow, s_total, ldk, K.p, s);
}

void stream_apply(const Store& st, StreamApply& sa, const double* src, bool src_pos, double* v_pos, double* v_bus,
                  bool accumulate, cudaStream_t s) {
  if (sa.prec == EMT_PREC_FF64) launch_stream<EMT_PREC_FF64>(st, sa, src, src_pos, v_pos, v_bus, accumulate, s);
  else launch_stream<EMT_PREC_FP64>(st, sa, src, src_pos, v_pos, v_bus, accumulate, s);
}

}  // namespace emt

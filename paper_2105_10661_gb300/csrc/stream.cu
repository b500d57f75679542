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
  constexpr int kU = 18;   // loads in flight per lane (one pass for up to 576 cut rows)
  // K does not depend on the kernels before this one: its first chunk is loaded while they finish
  T kv[kU];
#pragma unroll
  for (int u = 0; u < kU; ++u) {
    const int k = lane + 32 * u;
    kv[u] = k < n_crow ? Kr[k] : T{};
  }
  pdl_wait_s();
  stage_vec(yc, ycut_g, n_crow);
  __syncthreads();
  if (row >= s_total) return;
  A a, a2;
  for (int base = 0; base < n_crow; base += 32 * kU) {
    if (base > 0) {
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int k = base + lane + 32 * u;
        kv[u] = k < n_crow ? Kr[k] : T{};
      }
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
  __syncthreads();
  const T* F = Elem<PREC>::F(st);
  // the factor rows do not depend on the kernels before this one: the first round of them is
  // loaded while those finish
  auto load_round = [&](int base, int xb, T (&f)[kMaxAnc][4]) {
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
  };
  T f[kMaxAnc][4];
  load_round(0, x0, f);
  pdl_wait_s();
  const X yp = ldcg(y + pp);   // in flight with the loads below
  stage_vec(ss, s_g, s_total);
  __syncthreads();
  A a, a2;
  int kmax = 0;
  for (int x = x0; x < x1; ++x) kmax = max(kmax, an[x].k);
  for (int base = 0; base < kmax; base += 4 * kEL) {
    for (int xb = x0; xb < x1; xb += kMaxAnc) {
      if (base > 0 || xb > x0) load_round(base, xb, f);
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

// ---------------------------------------------------------------- single-launch apply
// The whole apply in one cooperative launch of one CTA per SM, for stores whose leaf blocks stream
// from HBM. Three phases separated by two grid-wide barriers:
//   A  leaf stage: the CTA streams its leaf rows through a ring of shared-memory slots (one
//      consumer warp per slot, as in k_leaf_stream), keeps y of its own rows in shared memory and
//      writes the cut-row values y_cut to global memory. After the last ring copy it issues the
//      copies of everything phases B and C read from the store: its slice of K and the rows of
//      the factor panels of its own positions (one slice per leaf segment and ancestor).
//   B  s = K y_cut for the CTA's rows of K (one warp per row), written to global memory.
//   C  expansion v = y - sum over ancestors of F row . s(half) of the CTA's own positions, from
//      the staged factor rows; 16 lanes per position.
// The copies of phase A's tail land while the CTAs wait at the barriers, so HBM stays busy up to
// the end of the stream and the two later phases touch only on-chip data and L2.
// Barriers count arrivals on one global word (release add, acquire polling, bounded); the last CTA
// to finish puts both counters back to zero, so every launch starts from zero. Every wait gives up
// after about 2 s, records DEV_TIMEOUT, skips the remaining work and still reaches the later
// barriers and the exit, draining its own copies first.
struct PersistD {
  const int2* win;
  const int* row0;
  const PersistSeg* seg;
  const int* seg_ptr;
  const PersistF* fsl;
  const int* krow0;
  const int* crow_of;   // position -> distinct cut-row index, -1 if none
  const void* K;
  void* ycut;
  void* sv;
  unsigned int* bar;
  int row_elems, ldk, n_crow, s_total, k_bytes;
  int o_bar, o_ring, o_y, o_crow, o_perm, o_vec, o_tab;
};

__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_gpu_add(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier: every CTA arrives once per barrier (also after an abort), then waits until
// `target` arrivals are counted. The CTA's writes before the barrier are made visible GPU-wide by
// bar.sync + a fence of thread 0 before its release add. Returns false (and sets the abort flag
// and the status word) when the wait ran out.
__device__ __forceinline__ void grid_barrier(unsigned int* count, unsigned int target, int* abort_flag,
                                             int* status) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    red_release_gpu_add(count, 1u);
    const long long t0 = clock64();
    while (ld_acquire_gpu(count) < target) {
      if (clock64() - t0 > kWaitS) {
        atomicExch(status, DEV_TIMEOUT);
        *reinterpret_cast<volatile int*>(abort_flag) = 1;
        break;
      }
    }
  }
  __syncthreads();
}

// Bounded wait of every thread of a warp-uniform caller on an mbarrier phase.
__device__ __forceinline__ bool cta_wait(uint64_t* b, uint32_t parity, int* abort_flag, int* status) {
  if (mb_wait(b, parity, kWaitS)) return true;
  atomicExch(status, DEV_TIMEOUT);
  *reinterpret_cast<volatile int*>(abort_flag) = 1;
  return false;
}


// Rows of the leaf stage a warp keeps in flight ahead of the one it multiplies (its private ring
// holds kAhead + 1 rows).
constexpr int kAhead = 1;

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sas(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int PREC>
__global__ void __launch_bounds__(512, 1) k_apply_persist(DStore st, PersistD pd, const double* src, int src_pos,
                                                           double* v_pos, double* v_bus, int accumulate) {
  using A = Acc<PREC>;
  using X = typename A::X;
  using T = typename A::T;
  extern __shared__ __align__(128) unsigned char smp[];
  uint64_t* aux = reinterpret_cast<uint64_t*>(smp + pd.o_bar);
  int* flags = reinterpret_cast<int*>(aux + 1);   // [0] abort, [1] copies of phases B and C issued
  volatile int* vflags = flags;
  T* ring = reinterpret_cast<T*>(smp + pd.o_ring);   // per-warp leaf rows (A); K rows and factor rows (B, C)
  T* ksl = ring;
  T* fsm = reinterpret_cast<T*>(smp + pd.o_ring + pd.k_bytes);
  X* yown = reinterpret_cast<X*>(smp + pd.o_y);
  int* crow_own = reinterpret_cast<int*>(smp + pd.o_crow);
  int* perm_own = reinterpret_cast<int*>(smp + pd.o_perm);
  X* vec = reinterpret_cast<X*>(smp + pd.o_vec);   // x window (A), y_cut (B), s (C)
  X* ycut_g = reinterpret_cast<X*>(pd.ycut);
  X* sv_g = reinterpret_cast<X*>(pd.sv);
  const T* Kg = reinterpret_cast<const T*>(pd.K);
  const int c = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarp = blockDim.x >> 5;
  const int r0 = pd.row0[c], r1 = pd.row0[c + 1];
  const int k0 = pd.krow0[c], k1 = pd.krow0[c + 1];
  const int g0 = pd.seg_ptr[c], g1 = pd.seg_ptr[c + 1];
  const int2 w = pd.win[c];
  const unsigned int n_cta = gridDim.x;
  const int nrow = r1 - r0;
  const T* L = Elem<PREC>::L(st);
  const T* F = Elem<PREC>::F(st);
  // leaf rows of the warp, k-th = own row warp + k nwarp; slot k % (kAhead + 1) of its private ring
  T* wring = ring + (size_t)warp * (kAhead + 1) * pd.row_elems;
  const PersistSeg* sgt = pd.seg + g0;   // the CTA's leaf segments (in shared memory once staged)
  auto row_seg = [&](int p) {
    int g = 0;
    while (g + 1 < g1 - g0 && p >= sgt[g].p1) ++g;
    return g;
  };
  auto issue_row = [&](int k) {
    const int i = warp + k * nwarp;
    if (i < nrow) {
      const int p = r0 + i;
      const PersistSeg sg = sgt[row_seg(p)];
      const T* Lr = L + sg.loff + (int64_t)(p - sg.p0) * sg.ld;
      T* dst = wring + (size_t)(k % (kAhead + 1)) * pd.row_elems;
      for (int col = 2 * lane; col < sg.b; col += 64) cp_async16(dst + col, Lr + col);
    }
    cp_async_commit();   // also when empty, so that every lane counts the same groups
  };
  // the first rows go out before anything else, then the bookkeeping while they travel
  for (int k = 0; k <= kAhead; ++k) issue_row(k);
  if (tid == 0) {
    mb_init(aux, 1);
    flags[0] = 0;
    flags[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const int f_first = g1 > g0 ? pd.seg[g0].f0 : 0;
  const int n_f = g1 > g0 ? pd.seg[g1 - 1].f1 - f_first : 0;
  PersistSeg* segs = reinterpret_cast<PersistSeg*>(smp + pd.o_tab);
  PersistF* fsls = reinterpret_cast<PersistF*>(segs + (g1 - g0));
  for (int u = tid; u < g1 - g0; u += blockDim.x) segs[u] = pd.seg[g0 + u];
  for (int u = tid; u < n_f; u += blockDim.x) fsls[u] = pd.fsl[f_first + u];
  for (int u = tid; u < nrow; u += blockDim.x) {
    crow_own[u] = pd.crow_of[r0 + u];
    perm_own[u] = st.perm[r0 + u];
  }
  // what phases B and C read from the store goes to L2 now: rows [k0, k1) of K and the factor rows
  // of the CTA's positions (copied into the drained ring after phase A)
  if (warp == nwarp - 1 && lane == 0) {
    if (k1 > k0) bulk_prefetch_l2(Kg + (size_t)k0 * pd.ldk, (uint32_t)((k1 - k0) * pd.ldk * (int)sizeof(T)));
    for (int f = f_first; f < f_first + n_f; ++f) bulk_prefetch_l2(F + pd.fsl[f].src, (uint32_t)pd.fsl[f].bytes);
  }
  // the x window: all index loads of a thread, then all value loads (two round trips)
  {
    constexpr int kG = 4;
    for (int base = w.x + tid; base < w.y + 2; base += kG * blockDim.x) {
      int idx[kG];
#pragma unroll
      for (int u = 0; u < kG; ++u) {
        const int p = base + u * blockDim.x;
        idx[u] = p < w.y ? (src_pos ? p : st.perm[p]) : -1;
      }
      double val[kG];
#pragma unroll
      for (int u = 0; u < kG; ++u) val[u] = idx[u] >= 0 ? ldcg(src + idx[u]) : 0.0;
#pragma unroll
      for (int u = 0; u < kG; ++u) {
        const int p = base + u * blockDim.x;
        if (p < w.y + 2) vec[p - w.x] = A::prep(val[u]);
      }
    }
  }
  __syncthreads();
  sgt = segs;
  // ---- phase A: leaf stage, one warp per row, kAhead rows in flight per warp
  for (int k = 0; warp + k * nwarp < nrow; ++k) {
    cp_async_wait<kAhead>();   // row k of this lane has landed
    __syncwarp();              // ... and of every lane
    const int i = warp + k * nwarp;
    const PersistSeg sg = segs[row_seg(r0 + i)];
    const T* Lr = wring + (size_t)(k % (kAhead + 1)) * pd.row_elems;
    const X* xr = vec + sg.xo;
    A a, a2;
#pragma unroll 4
    for (int col = 2 * lane; col < sg.b; col += 64) {
      T l2[2];
      ld2(Lr + col, l2);
      a.fma(l2[0], xr[col]);
      a2.fma(l2[1], xr[col + 1]);
    }
    a.add(a2.getx());
    const X v = warp_sum<PREC>(a, 32);
    if (lane == 0) {
      yown[i] = v;
      const int kc = crow_own[i];
      if (kc >= 0) ycut_g[kc] = v;
    }
    __syncwarp();              // every lane is done with the slot before it is refilled
    issue_row(k + kAhead + 1);
  }
  cp_async_wait<0>();
  __syncthreads();
  // the ring is drained: copy K rows and factor rows (now in L2) into it, behind a proxy fence
  // that orders the generic accesses to the ring before the async writes
  if (tid == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    uint32_t bytes = (uint32_t)((k1 - k0) * pd.ldk * (int)sizeof(T));
    for (int f = 0; f < n_f; ++f) bytes += (uint32_t)fsls[f].bytes;
    mb_expect(aux, bytes);
    if (k1 > k0) bulk_row(ksl, Kg + (size_t)k0 * pd.ldk, (uint32_t)((k1 - k0) * pd.ldk * (int)sizeof(T)), aux);
    for (int f = 0; f < n_f; ++f) bulk_row(fsm + fsls[f].dst, F + fsls[f].src, (uint32_t)fsls[f].bytes, aux);
    flags[1] = 1;
  }
  // ---- barrier 1: every CTA's y_cut is written
  grid_barrier(&pd.bar[0], n_cta, flags, st.status);
  // ---- phase B: rows [k0, k1) of s = K y_cut
  bool live = !vflags[0];
  if (live) {
    stage_vec(vec, ycut_g, pd.n_crow);
    if (flags[1]) cta_wait(aux, 0u, flags, st.status);
  }
  __syncthreads();
  live = !vflags[0];
  if (live) {
    for (int row = k0 + warp; row < k1; row += nwarp) {
      const T* Kr = ksl + (size_t)(row - k0) * pd.ldk;
      A a, a2;
      for (int k = lane; k < pd.n_crow; k += 64) {
        a.fma(Kr[k], vec[k]);
        if (k + 32 < pd.n_crow) a2.fma(Kr[k + 32], vec[k + 32]);
      }
      a.add(a2.getx());
      const X v = warp_sum<PREC>(a, 32);
      if (lane == 0) sv_g[row] = v;
    }
  }
  // ---- barrier 2: every row of s is written
  grid_barrier(&pd.bar[0], 2 * n_cta, flags, st.status);
  // ---- phase C: expansion of the CTA's own positions from the staged factor rows
  live = !vflags[0];
  if (live) stage_vec(vec, sv_g, pd.s_total);
  __syncthreads();
  if (live) {
    const int npos = r1 - r0;
    const int gl = tid & (kEL - 1);
    // two positions per warp; the trip count is uniform across the warp (shuffles below)
    for (int base = warp * 2; base < npos; base += nwarp * 2) {
      const int i = base + ((tid >> 4) & 1);
      const bool valid = i < npos;
      const int p = r0 + (valid ? i : 0);
      A a, a2;
      if (valid) {
        int g = 0;
        while (g + 1 < g1 - g0 && p >= segs[g].p1) ++g;
        const PersistSeg sg = segs[g];
        for (int f = sg.f0 - f_first; f < sg.f1 - f_first; ++f) {
          const PersistF r = fsls[f];
          const T* Fr = fsm + r.dst + (size_t)(p - sg.p0) * r.kld;
          for (int e = gl; e < r.k; e += 2 * kEL) {
            a.fma(Fr[e], neg(vec[r.sidx + e]));
            if (e + kEL < r.k) a2.fma(Fr[e + kEL], neg(vec[r.sidx + e + kEL]));
          }
        }
      }
      a.add(a2.getx());
      const X wv = warp_sum<PREC>(a, kEL);
      if (valid && gl == 0) {
        A f;
        f.add(yown[i]);
        f.add(wv);
        yown[i] = f.getx();   // v of the position, converted below
      }
    }
  }
  __syncthreads();
  // one thread per position for the conversion to double and the stores (full warps)
  if (live) {
    for (int i = tid; i < r1 - r0; i += blockDim.x) {
      double out = A::todbl(yown[i]);
      if (accumulate) out += v_pos[r0 + i];
      if (v_pos) v_pos[r0 + i] = out;
      if (v_bus) v_bus[perm_own[i]] = out;
    }
  }
  // ---- exit: own copies drained; the last CTA out puts the barrier counters back to zero
  __syncthreads();
  if (tid == 0) {
    if (flags[1]) mb_wait(aux, 0u, kWaitS);
    __threadfence();
    const unsigned int done = atomicAdd(&pd.bar[1], 1u);
    if (done == n_cta - 1) {
      atomicExch(&pd.bar[0], 0u);
      atomicExch(&pd.bar[1], 0u);
    }
  }
}

template <int PREC>
void launch_persist(const Store& st, StreamApply& sa, const double* src, bool src_pos, double* v_pos, double* v_bus,
                    bool acc, cudaStream_t s) {
  PersistD pd{};
  pd.win = sa.win.p;
  pd.row0 = sa.row0.p;
  pd.seg = sa.pseg.p;
  pd.seg_ptr = sa.pseg_ptr.p;
  pd.fsl = sa.pf.p;
  pd.krow0 = sa.krow0.p;
  pd.crow_of = sa.crow_of.p;
  pd.K = sa.K.p;
  pd.ycut = sa.ycut.p;
  pd.sv = sa.sv.p;
  pd.bar = sa.bar.p;
  pd.row_elems = sa.row_elems;
  pd.ldk = sa.ldk;
  pd.n_crow = sa.n_crow;
  pd.s_total = sa.s_total;
  pd.k_bytes = sa.k_bytes;
  pd.o_bar = sa.o_bar;
  pd.o_ring = sa.o_ring;
  pd.o_y = sa.o_y;
  pd.o_crow = sa.o_crow;
  pd.o_perm = sa.o_perm;
  pd.o_vec = sa.o_vec;
  pd.o_tab = sa.o_tab;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sa.n_cta);
  cfg.blockDim = dim3(32 * sa.warps);
  cfg.dynamicSmemBytes = sa.smem_p;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  EMT_CUDA(cudaLaunchKernelEx(&cfg, k_apply_persist<PREC>, st.view(), pd, src, src_pos ? 1 : 0, v_pos, v_bus,
                              acc ? 1 : 0));
}

}  // namespace

// Whether the streaming kernels serve this store: FP64 or float-float storage large enough that
// the leaf blocks do not stay in L2 between applications.
bool stream_apply_wanted(const Store& st) {
  return (st.precision == EMT_PREC_FF64 || st.precision == EMT_PREC_FP64) && st.L_elems * 8 >= (int64_t)48 << 20;
}

// Plan of the single-launch apply (k_apply_persist): rows of K per CTA, the leaf segments of each
// CTA's positions with their factor-panel slices, the shared-memory layout and the number of warps
// whose private rings of kAhead + 1 leaf rows fit. K rows and factor rows are copied into the
// rings once they have drained, so the ring region must also hold them. False (three-kernel path)
// when a CTA cannot hold its data, a copy would break the 16-byte rules, or one CTA per SM is not
// resident.
static bool persist_plan(const Store& st, StreamApply& sa, const std::vector<int>& r0,
                         const std::vector<StreamAnc>& an, const std::vector<int>& ap, size_t max_win, int optin,
                         cudaStream_t s) {
  sa.persist = false;
  const Tree& t = st.tree;
  const int n_cta = sa.n_cta;
  int dev = 0, coop = 0, sms = 0;
  EMT_CUDA(cudaGetDevice(&dev));
  EMT_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  EMT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (!coop || (sa.ldk & 1) != 0) return false;
  int max_ld = 0;
  for (int j = 0; j < st.n_leaf; ++j) {
    max_ld = std::max(max_ld, st.leaf_ld_h[j]);
    if ((st.leaf_ld_h[j] & 1) || (st.leaf_off_h[j] & 1)) return false;   // 16-byte row starts
  }
  // rows of K per CTA; leaf segments and factor slices
  std::vector<int> k0(n_cta + 1);
  for (int c = 0; c <= n_cta; ++c) k0[c] = (int)((int64_t)sa.s_total * c / n_cta);
  std::vector<PersistSeg> seg;
  std::vector<PersistF> fs;
  std::vector<int> sp(n_cta + 1, 0);
  int64_t f_max = 0;
  int rows_max = 1, krows_max = 0, tab_max = 0;
  for (int c = 0; c < n_cta; ++c) {
    sp[c] = (int)seg.size();
    const int fs0 = (int)fs.size();
    int64_t fe = 0;
    const int wlo = r0[c + 1] > r0[c] ? t.lo[st.leaf_nodes_h[leaf_index_of_pos(st, r0[c])]] : 0;
    for (int p = r0[c]; p < r0[c + 1];) {
      const int j = leaf_index_of_pos(st, p);
      const int lo = t.lo[st.leaf_nodes_h[j]];
      const int p1 = std::min(t.hi[st.leaf_nodes_h[j]], r0[c + 1]);
      PersistSeg g{};
      g.p0 = p;
      g.p1 = p1;
      g.f0 = (int)fs.size();
      g.xo = lo - wlo;
      g.b = t.hi[st.leaf_nodes_h[j]] - lo;
      g.ld = st.leaf_ld_h[j];
      g.loff = st.leaf_off_h[j] + (int64_t)(p - lo) * g.ld;
      for (int x = ap[j]; x < ap[j + 1]; ++x) {
        const StreamAnc& r = an[x];
        PersistF f{};
        f.src = r.foff + (int64_t)(p - lo) * r.kld;
        f.dst = (int)fe;
        f.kld = r.kld;
        f.k = r.k;
        f.sidx = r.sidx;
        const int64_t bytes = (int64_t)(p1 - p) * r.kld * 8;
        if ((f.src & 1) || (bytes & 15) || bytes >= (1 << 20)) return false;   // 16-byte rules of cp.async.bulk
        f.bytes = (int)bytes;
        fe += (int64_t)(p1 - p) * r.kld;
        fs.push_back(f);
      }
      g.f1 = (int)fs.size();
      seg.push_back(g);
      p = p1;
    }
    f_max = std::max(f_max, fe);
    tab_max = std::max(tab_max, (int)(((int)seg.size() - sp[c]) * sizeof(PersistSeg) +
                                      ((int)fs.size() - fs0) * sizeof(PersistF)));
    rows_max = std::max(rows_max, r0[c + 1] - r0[c]);
    krows_max = std::max(krows_max, k0[c + 1] - k0[c]);
  }
  sp[n_cta] = (int)seg.size();
  auto up = [](size_t x) { return (x + 127) / 128 * 128; };
  sa.k_bytes = (int)up((size_t)krows_max * sa.ldk * 8);
  const size_t bc_bytes = (size_t)sa.k_bytes + (size_t)f_max * 8;   // K rows + factor rows
  if (bc_bytes >= (1u << 20)) return false;                         // one mbarrier transaction count
  sa.row_elems = max_ld;
  const size_t warp_ring = (size_t)(kAhead + 1) * max_ld * 8;
  const size_t vec_elems = std::max({max_win + 2, (size_t)std::max(sa.n_crow, 1), (size_t)std::max(sa.s_total, 1)});
  auto layout = [&](int W) {
    sa.o_bar = 0;
    size_t off = 128;   // the aux mbarrier and two flags
    sa.o_ring = (int)off;
    off = up(off + std::max((size_t)W * warp_ring, bc_bytes));
    sa.o_y = (int)off;
    off = up(off + (size_t)rows_max * 8);
    sa.o_crow = (int)off;
    off = up(off + (size_t)rows_max * 4);
    sa.o_perm = (int)off;
    off = up(off + (size_t)rows_max * 4);
    sa.o_vec = (int)off;
    off = up(off + vec_elems * 8);
    sa.o_tab = (int)off;
    off += (size_t)tab_max + 16;
    return off;
  };
  int W = sa.rps_req > 0 ? std::min(sa.rps_req, 16) : 16;
  while (W >= 4 && layout(W) > (size_t)optin - 1024) --W;
  if (W < 4) return false;
  sa.warps = W;
  sa.smem_p = layout(W);
  int nb = 0;
  auto setup = [&](auto kernel) {
    EMT_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa.smem_p));
    EMT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, 32 * W, sa.smem_p));
  };
  if (sa.prec == EMT_PREC_FF64) setup(k_apply_persist<EMT_PREC_FF64>);
  else setup(k_apply_persist<EMT_PREC_FP64>);
  if (nb < 1 || n_cta > nb * sms) return false;
  if (seg.empty()) seg.push_back(PersistSeg{});
  if (fs.empty()) fs.push_back(PersistF{});
  sa.pseg.upload(seg, s);
  sa.pseg_ptr.upload(sp, s);
  sa.pf.upload(fs, s);
  sa.krow0.upload(k0, s);
  if (!sa.bar.p) {
    sa.bar.alloc(2);
    EMT_CUDA(cudaMemsetAsync(sa.bar.p, 0, 2 * sizeof(unsigned int), s));
  }
  sa.persist = true;
  return true;
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
  persist_plan(st, *this, r0, an, ap, max_win, optin, s);
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
  if (sa.persist && sa.mode == 2) {
    if (sa.prec == EMT_PREC_FF64) launch_persist<EMT_PREC_FF64>(st, sa, src, src_pos, v_pos, v_bus, accumulate, s);
    else launch_persist<EMT_PREC_FP64>(st, sa, src, src_pos, v_pos, v_bus, accumulate, s);
    return;
  }
  if (sa.prec == EMT_PREC_FF64) launch_stream<EMT_PREC_FF64>(st, sa, src, src_pos, v_pos, v_bus, accumulate, s);
  else launch_stream<EMT_PREC_FP64>(st, sa, src, src_pos, v_pos, v_bus, accumulate, s);
}

}  // namespace emt

// Kernel generation 4: the time loop of one single-column simulation inside one persistent
// thread-block cluster.
//
// For networks whose store fits in the shared memory of one cluster (up to 16 CTAs on 16 SMs,
// about 220 KB each), every static array of a step -- the CTA's rows of the leaf inverses, the
// factor rows its expansion needs, its slice of the sweep matrix -- is copied on chip once per
// launch and stays there while the kernel runs every time step up to the next event. The state
// (voltages, element histories) lives in registers and shared memory for the whole launch. Each
// CTA owns a contiguous range of positions (part of one leaf, or whole leaves). Per time step,
// with float-float (or FP64) arithmetic throughout:
//   1. history update of the CTA's element ends (trapezoidal companion sources, Sec. II) and the
//      injection x of its positions (all local)
//   2. leaf stage (Eq. 2 with the leaf blocks of Sec. III) in column form: by symmetry of the
//      leaf inverse, the CTA's rows of L_j are its columns, so it forms the partial products
//      p_c[r] = sum over its positions i of L_j[i, r] x_i for every row r of the leaf using only
//      its own x; each partial is pushed (st.async to the peer's shared memory, completing on
//      the peer's mbarrier) to the CTAs that need y[r]: the owner of r, the CTAs for which r is a
//      neighbour of one of their elements, and the CTAs whose slice of s reads the cut row r
//   3. wait on this step's partials mbarrier (the host counts the bytes each CTA receives per
//      step); y = sum of the partials
//   4. boundary sweep as one product: the sweep is linear in the cut-row values, s = K y_cut,
//      with K built on the device from the sweep image after every build or modification; each
//      CTA forms its slice of s and pushes it (st.async) to every CTA
//   5. wait on this step's s mbarrier; expansion v = y - sum over ancestors of (factor row . s)
//      for the CTA's positions and for its halo positions (far ends of its elements), so that the
//      next history update reads local voltages only.
// Exchange is push-only and has no cluster barrier inside the time loop: every pushed buffer
// (expansion-row partials, s) and its two mbarriers alternate by step parity, so a fast CTA may
// push step t+1 while a slow one still reads step t, and a CTA cannot be two steps ahead of a
// peer because it waits for that peer's pushes of the step before. The cut-row partials need one
// copy: a CTA pushes those of step t+1 only after it has received every CTA's s of step t, which
// each CTA sends after it has summed its cut-row partials of step t. Every wait is bounded; one
// cluster barrier at exit keeps each CTA's shared memory alive until no peer can write it. A
// cluster of one CTA uses __syncthreads instead.
#include <algorithm>
#include <climits>
#include <cstring>

#include "sim.h"

namespace emt {

namespace {

constexpr int kT4 = 512;      // threads per CTA
constexpr int kEPT = 2;       // element ends per thread
constexpr int kRI = 4;        // ints per own-row record
constexpr int kVR = 4;        // ints per expansion-row record
constexpr int kOR = 4;        // ints per leaf-stage output record
constexpr int kPR = 4;        // ints per push record
constexpr int kHdr = 24;      // ints per CTA header
constexpr long long kWait4 = 4000000000LL;   // ~2 s of SM clock

// header fields
enum { H_P0, H_P1, H_NHALO, H_M0, H_M1, H_LBYTES, H_OLROW, H_NFC, H_OFC, H_OROW, H_OVROW, H_NOUT, H_OOUT, H_NPUSH,
       H_OPUSH, H_OENDL, H_S0, H_S1, H_LP, H_YIN, H_OSX, H_NSX };   // H_YIN: partials this CTA receives per step;
                                                                    // H_OSX, H_NSX: its s-index lists
// own-row record fields (injection)
enum { R_ELO, R_EHI, R_MON };
// push kinds: partial of an expansion row (double-buffered by step parity) or of a cut row
enum { P_YV = 0, P_CUT = 1 };

__device__ __forceinline__ uint32_t sa4(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ uint32_t cta_rank4() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t mapa4(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// asynchronous remote store whose completion is counted (in bytes) on the destination CTA's
// mbarrier `mbar` (a shared::cluster address in the destination CTA)
__device__ __forceinline__ void st_async(uint32_t a, float2 v, uint32_t mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(a),
               "f"(v.x), "f"(v.y), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void st_async(uint32_t a, double v, uint32_t mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];" ::"r"(a), "d"(v),
               "r"(mbar)
               : "memory");
}
__device__ __forceinline__ int ld_remote_i32(uint32_t a) {
  int v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void mbar_init4(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa4(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect4(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa4(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk4(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sa4(dst)),
      "l"(src), "r"(bytes), "r"(sa4(bar))
      : "memory");
}
// Non-blocking polls of the phase with the given parity until `limit` SM clock cycles have passed.
__device__ __forceinline__ bool mbar_wait4(uint64_t* bar, long long limit, uint32_t parity = 0) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(sa4(bar)), "r"(parity)
                 : "memory");
    if (ok) return true;
    if (clock64() - t0 > limit) return false;
  }
}
// two consecutive 8-byte elements from shared memory in one 16-byte load
__device__ __forceinline__ void lds2(const float2* p, float2 (&e)[2]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  e[0] = make_float2(v.x, v.y);
  e[1] = make_float2(v.z, v.w);
}
__device__ __forceinline__ void lds2(const double* p, double (&e)[2]) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  e[0] = v.x;
  e[1] = v.y;
}

// sin and cos of the source phase at table row ti, in the vector type
__device__ __forceinline__ void trig_x(const Step2D& q, int ti, float2& sx, float2& cx) {
  const float4 t = q.trigff[ti];
  sx = make_float2(t.x, t.y);
  cx = make_float2(t.z, t.w);
}
__device__ __forceinline__ void trig_x(const Step2D& q, int ti, double& sx, double& cx) {
  sx = q.trig[2 * ti];
  cx = q.trig[2 * ti + 1];
}
// monitored voltage: float-float values go to the launch's staging record (converted after the
// launch, keeping FP64 instructions out of the step), FP64 values straight to the record
__device__ __forceinline__ void rec_store(const Step4D& d, double* rec, int64_t full, int64_t local, float2 v) {
  if (d.rec_ff) d.rec_ff[local] = v;
}
__device__ __forceinline__ void rec_store(const Step4D&, double* rec, int64_t full, int64_t, double v) {
  rec[full] = v;
}

// sum over groups of `lanes` consecutive lanes (a power of two <= 32; every lane of the warp
// takes part)
template <int PREC>
__device__ __forceinline__ typename Acc<PREC>::X group_sum(const Acc<PREC>& a, int lanes) {
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
// lanes per row so that `rows` rows fill the block in as few waves as possible
__device__ __forceinline__ int lanes_for(int rows) {
  int l = 1;
  while (l < 32 && rows * (l * 2) <= kT4) l *= 2;
  return l;
}

template <int PREC>
__global__ void __launch_bounds__(kT4, 1) k_step4(DStore st, SimD sim, Step2D q, Step4D d, int n_steps) {
  using A = Acc<PREC>;
  using X = typename A::X;
  using T = typename A::T;
  extern __shared__ __align__(128) unsigned char sm4[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm4);        // prologue copies
  uint64_t* sbar = reinterpret_cast<uint64_t*>(sm4 + 8);    // [2] by step parity: slices of s from the other CTAs
  uint64_t* ybar = reinterpret_cast<uint64_t*>(sm4 + 24);   // [2] by step parity: leaf-stage partials pushed here
  int* flag = reinterpret_cast<int*>(sm4 + 40);             // [0] own ok, [1] cluster ok
  const int tid = threadIdx.x;
  const int C = d.C, P = d.P;
  const int rank = C > 1 ? (int)cta_rank4() : 0;
  const int* hd = d.hdr + rank * kHdr;
  const int p0 = hd[H_P0], p1 = hd[H_P1];
  const int nrow = p1 - p0, nv = nrow + hd[H_NHALO];
  const int m0 = hd[H_M0], n_ends = hd[H_M1] - hd[H_M0];
  const int s0 = hd[H_S0], ns = hd[H_S1] - hd[H_S0];
  const int n_out = hd[H_NOUT], n_push = hd[H_NPUSH], lp = hd[H_LP];
  const int ldk = d.ldk, n_crow = d.n_crow;
  X* xloc = reinterpret_cast<X*>(sm4 + d.o_x);
  X* part = reinterpret_cast<X*>(sm4 + d.o_part);       // [lp][n_out_pad]
  X* ycp = reinterpret_cast<X*>(sm4 + d.o_ycp);         // [n_crow][P] partials of cut rows
  X* ycut = reinterpret_cast<X*>(sm4 + d.o_ycut);       // [ldk]
  X* yvp = reinterpret_cast<X*>(sm4 + d.o_yvp);         // [2][max_vrows][P] partials of expansion rows
  X* ss = reinterpret_cast<X*>(sm4 + d.o_s);
  X* vloc = reinterpret_cast<X*>(sm4 + d.o_v);
  X* contrib = reinterpret_cast<X*>(sm4 + d.o_contrib);
  int* rowi = reinterpret_cast<int*>(sm4 + d.o_row);
  int* vrow = reinterpret_cast<int*>(sm4 + d.o_vrow);
  int* outi = reinterpret_cast<int*>(sm4 + d.o_out);
  int* push = reinterpret_cast<int*>(sm4 + d.o_push);
  int* sxs = reinterpret_cast<int*>(sm4 + d.o_sx);       // s index of every factor-row element, per leaf
  T* Ks = reinterpret_cast<T*>(sm4 + d.o_K);
  T* Ls = reinterpret_cast<T*>(sm4 + d.o_L);
  T* Fs = reinterpret_cast<T*>(sm4 + d.o_F);
  const T* Lg = Elem<PREC>::L(st);
  const T* Fg = Elem<PREC>::F(st);
  const T* Kg = reinterpret_cast<const T*>(d.K);
  const int* tab = d.tab;

  // ---- prologue: bulk copies of the leaf rows (one per row) ...
  if (tid < 32) {
    if (tid == 0) {
      mbar_init4(sbar);
      mbar_init4(sbar + 1);
      mbar_init4(ybar);
      mbar_init4(ybar + 1);
      mbar_init4(bar);
      mbar_expect4(bar, (uint32_t)hd[H_LBYTES]);
    }
    __syncwarp();
    const int* lr = tab + hd[H_OLROW];
    for (int r = tid; r < nrow; r += 32)
      bulk4(Ls + lr[3 * r + 1], Lg + lr[3 * r], (uint32_t)lr[3 * r + 2] * (uint32_t)sizeof(T), bar);
  }
  // ... plain loads of the tables, the factor rows (negated, each row's elements of all its
  // ancestors packed back to back and zero up to the longest such row), this CTA's rows of K and
  // the state
  for (int i = tid; i < d.e_max * d.fstride; i += kT4) Fs[i] = T{};
  __syncthreads();
  {
    const int* src = tab + hd[H_OROW];
    for (int i = tid; i < nrow * kRI; i += kT4) {
      int v = src[i];
      if (i % kRI == R_MON) v = (sim.mon_idx && sim.n_mon > 0) ? sim.mon_idx[p0 + i / kRI] : -1;
      rowi[i] = v;
    }
    src = tab + hd[H_OVROW];
    for (int i = tid; i < nv * kVR; i += kT4) vrow[i] = src[i];
    src = tab + hd[H_OOUT];
    for (int i = tid; i < n_out * kOR; i += kT4) outi[i] = src[i];
    src = tab + hd[H_OPUSH];
    for (int i = tid; i < n_push * kPR; i += kT4) push[i] = src[i];
    const int* fc = tab + hd[H_OFC];
    const int warp = tid >> 5, lane = tid & 31;
    for (int u = warp; u < hd[H_NFC]; u += kT4 / 32) {
      const int so = fc[3 * u], dst = fc[3 * u + 1], len = fc[3 * u + 2];
      for (int e = lane; e < len; e += 32) Fs[dst + (int64_t)e * d.fstride] = neg(Fg[so + e]);
    }
    src = tab + hd[H_OSX];
    for (int i = tid; i < hd[H_NSX]; i += kT4) sxs[i] = src[i];
    for (int i = tid; i < ns * ldk; i += kT4) Ks[i] = Kg[(int64_t)s0 * ldk + i];
    // partial slots a CTA never receives (leaves split into fewer than P parts) stay zero
    for (int i = tid; i < n_crow * P; i += kT4) ycp[i] = A::zero();
    for (int i = tid; i < 2 * d.max_vrows * P; i += kT4) yvp[i] = A::zero();
    for (int i = tid; i < ldk; i += kT4) ycut[i] = A::zero();
    for (int i = tid; i < nv; i += kT4) vloc[i] = A::prep(sim.v_pos[tab[hd[H_OVROW] + kVR * i]]);
  }
  X eg[kEPT], ea[kEPT], eb[kEPT], eI[kEPT];
  int es[kEPT], eo[kEPT], esg[kEPT];
#pragma unroll
  for (int k = 0; k < kEPT; ++k) {
    const int e = tid + k * kT4;
    es[k] = 0;
    eo[k] = -1;
    esg[k] = 0;
    eg[k] = ea[k] = eb[k] = eI[k] = A::zero();
    if (e < n_ends) {
      const IncRec r = q.inc[m0 + e];
      eg[k] = A::prep(r.g);
      ea[k] = A::prep(r.alpha);
      eb[k] = A::prep(r.beta);
      eI[k] = A::prep(q.Ih[m0 + e]);
      esg[k] = r.sgn;
      es[k] = tab[hd[H_OENDL] + 2 * e];
      eo[k] = tab[hd[H_OENDL] + 2 * e + 1];
    }
  }
  X ssx = A::zero(), ssy = A::zero();
  if (tid < nrow) {
    const double2 sv = q.src_sum[p0 + tid];
    ssx = A::prep(sv.x);
    ssy = A::prep(sv.y);
  }
  // every CTA agrees on success before the first remote access, and none leaves while another
  // may still read its flag
  if (tid == 0) {
    const bool ok = mbar_wait4(bar, kWait4);
    if (!ok) {
      atomicExch(st.status, DEV_TIMEOUT);
      mbar_wait4(bar, kWait4);   // give copies in flight a second bounded chance
    }
    flag[0] = (ok && *reinterpret_cast<volatile int*>(st.status) == DEV_OK) ? 1 : 0;
  }
  if (C > 1) cluster_barrier(); else __syncthreads();
  if (tid == 0) {
    int all = flag[0];
    for (int c = 0; c < C; ++c)
      if (c != rank) all &= ld_remote_i32(mapa4(sa4(flag), (uint32_t)c));
    flag[1] = all;
  }
  if (C > 1) cluster_barrier(); else __syncthreads();
  if (!flag[1]) return;

  // leaf stage: thread (h, o) forms the partial of output o over column chunk h; lanes of a warp
  // take consecutive outputs, so they read consecutive elements of one stored row
  const int n_out_pad = (n_out + 31) & ~31;
  const int lk = lanes_for(ns), le = lanes_for(nv);
  const int grp_k = tid / lk, gl_k = tid % lk, ng_k = kT4 / lk, wg_k = (tid >> 5) * (32 / lk);
  const int grp_e = tid / le, gl_e = tid % le, ng_e = kT4 / le, wg_e = (tid >> 5) * (32 / le);
  const int yv_half = d.max_vrows * P;   // elements per parity copy
  const int step0 = sim.dyn->step_base;
  const int trig_first = sim.dyn->trig_first;
  const int rec_first = sim.dyn->rec_first;
  double* rec = sim.dyn->rec;
  const int n_mon = sim.n_mon;
  X sx = A::zero(), cx = A::zero();
  if (tid < nrow && n_steps > 0) trig_x(q, step0 + 1 - trig_first, sx, cx);

  // Within the step loop no cluster barrier is used. Every remote write is an asynchronous store
  // counted on the receiver's mbarrier for that step parity, and each CTA waits (bounded) for the
  // bytes it expects: the leaf-stage partials pushed to it, then the slices of s. Reuse is safe
  // because every CTA sends its slice of s to every CTA: a CTA that holds all slices of step t
  // knows every CTA has finished step t - 1's expansion (the double-buffered partials and s of
  // that parity) and step t's cut-row reads, and the phases of one parity never overlap.
  bool dead = false;   // thread 0: a data wait ran out
  const uint32_t y_bytes = (uint32_t)hd[H_YIN] * (uint32_t)sizeof(X);
  const uint32_t s_bytes = (uint32_t)((d.s_total - ns) * (int)sizeof(X));
  for (int it = 0; it < n_steps; ++it) {
    const int step = step0 + it + 1;
    const int par = it & 1;
    X* ssp = ss + par * d.s_total;
    if (C > 1 && tid == 0) {
      mbar_expect4(ybar + par, y_bytes);
      mbar_expect4(sbar + par, s_bytes);
    }
    // 1. element histories from the previous step's voltages (both ends of an element run the
    //    same operations on the same operands, so the two copies stay identical)
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
      const int e = tid + k * kT4;
      if (e < n_ends) {
        const X vi = vloc[es[k]];
        const X vo = eo[k] >= 0 ? vloc[eo[k]] : A::zero();
        const X va = esg[k] > 0 ? vi : vo;
        const X vb = esg[k] > 0 ? vo : vi;
        A a1;
        a1.add(va);
        a1.add(neg(vb));
        const X ve = a1.getx();
        A a2;
        a2.add(eI[k]);
        a2.fma(eg[k], ve);
        const X cur = a2.getx();
        A a3;
        a3.fma(ea[k], ve);
        a3.fma(eb[k], cur);
        eI[k] = a3.getx();
        contrib[e] = esg[k] > 0 ? neg(eI[k]) : eI[k];
      }
    }
    __syncthreads();
    // injection of the CTA's positions; the next step's sin/cos load is issued here
    if (tid < nrow) {
      const int* ri = rowi + tid * kRI;
      A a;
      for (int e = ri[R_ELO]; e < ri[R_EHI]; ++e) a.add(contrib[e]);
      a.fma(ssx, sx);
      a.fma(ssy, cx);
      xloc[tid] = a.getx();
      if (it + 1 < n_steps) trig_x(q, step + 1 - trig_first, sx, cx);
    }
    __syncthreads();
    // 2. leaf stage in column form
    for (int w = tid; w < lp * n_out_pad; w += kT4) {
      const int h = w / n_out_pad, o = w % n_out_pad;
      if (o < n_out) {
        const int* oi = outi + o * kOR;   // L offset of (first own column, row), stride, columns, x offset
        const int ncol = oi[2], stride = oi[1];
        const int c0 = (int)((int64_t)ncol * h / lp), c1 = (int)((int64_t)ncol * (h + 1) / lp);
        const T* Lc = Ls + oi[0];
        const X* xc = xloc + oi[3];
        A a, a2;
        int c = c0;
#pragma unroll 2
        for (; c + 1 < c1; c += 2) {
          a.fma(Lc[(int64_t)c * stride], xc[c]);
          a2.fma(Lc[(int64_t)(c + 1) * stride], xc[c + 1]);
        }
        if (c < c1) a.fma(Lc[(int64_t)c * stride], xc[c]);
        a.add(a2.getx());
        part[h * n_out_pad + o] = a.getx();
      }
    }
    __syncthreads();
    // pushes of the partials (sum over the column chunks first)
    for (int i = tid; i < n_push; i += kT4) {
      const int* pr = push + i * kPR;   // output, destination CTA, byte offset, kind
      const int o = pr[0];
      A a;
      for (int h = 0; h < lp; ++h) a.add(part[h * n_out_pad + o]);
      const X y = a.getx();
      const uint32_t off = (uint32_t)pr[2] + (pr[3] == P_YV ? (uint32_t)(par * yv_half * (int)sizeof(X)) : 0u);
      if (pr[1] == rank) *reinterpret_cast<X*>(sm4 + off) = y;
      else st_async(mapa4(sa4(sm4) + off, (uint32_t)pr[1]), y, mapa4(sa4(ybar + par), (uint32_t)pr[1]));
    }
    if (C > 1 && tid == 0 && !dead && !mbar_wait4(ybar + par, kWait4, (uint32_t)((it >> 1) & 1))) {
      atomicExch(st.status, DEV_TIMEOUT);   // partials never arrived: report and stop waiting
      dead = true;
    }
    __syncthreads();
    // 3. cut-row values, then this CTA's slice of s = K y_cut, sent to every other CTA
    for (int k = tid; k < n_crow; k += kT4) {
      A a;
      for (int p = 0; p < P; ++p) a.add(ycp[k * P + p]);
      ycut[k] = a.getx();
    }
    __syncthreads();
    for (int base = 0; base < ns; base += ng_k) {
      if (base + wg_k >= ns) break;
      const int i = base + grp_k;
      A a, a2;
      if (i < ns) {
        const T* Kr = Ks + (int64_t)i * ldk;
#pragma unroll 4
        for (int c = 2 * gl_k; c < n_crow; c += 2 * lk) {
          T k2[2];
          X y2[2];
          lds2(Kr + c, k2);
          lds2(ycut + c, y2);
          a.fma(k2[0], y2[0]);
          a2.fma(k2[1], y2[1]);
        }
        a.add(a2.getx());
      }
      const X sv = group_sum<PREC>(a, lk);
      if (i < ns)
        for (int c = gl_k; c < C; c += lk) {
          if (c == rank) ssp[s0 + i] = sv;
          else st_async(mapa4(sa4(&ssp[s0 + i]), (uint32_t)c), sv, mapa4(sa4(sbar + par), (uint32_t)c));
        }
    }
    if (C > 1 && tid == 0 && !dead && !mbar_wait4(sbar + par, kWait4, (uint32_t)((it >> 1) & 1))) {
      // a slice never arrived: report it and stop waiting (the results are void)
      atomicExch(st.status, DEV_TIMEOUT);
      dead = true;
    }
    __syncthreads();
    // 4. expansion of own and halo rows: v = y - sum over ancestors of F row . s(half), as one
    //    dot of the row's packed (negated) factor elements with the entries of s its leaf's list
    //    names; every row has e_max elements (zero past its own), so the lanes of a warp run
    //    loops of one length
    const X* yv = yvp + par * yv_half;
    const int e_max = d.e_max, fs = d.fstride;
    for (int base = 0; base < nv; base += ng_e) {
      if (base + wg_e >= nv) break;
      const int i = base + grp_e;
      A a, a2;   // two accumulators: half-length dependent chains
      if (i < nv) {
        // factor rows are stored element-major (element e of row i at e * fstride + i), so the
        // lanes of a warp, which take consecutive rows, read consecutive words
        const T* Fr = Fs + i;
        const int* sx = sxs + vrow[kVR * i + 2];
        int e = gl_e;
#pragma unroll 2
        for (; e + le < e_max; e += 2 * le) {
          a.fma(Fr[e * fs], ssp[sx[e]]);
          a2.fma(Fr[(e + le) * fs], ssp[sx[e + le]]);
        }
        if (e < e_max) a.fma(Fr[e * fs], ssp[sx[e]]);
        a.add(a2.getx());
      }
      const X w = group_sum<PREC>(a, le);
      if (i < nv && gl_e == 0) {
        A f;
        for (int p = 0; p < P; ++p) f.add(yv[i * P + p]);
        f.add(w);
        const X v = f.getx();
        vloc[i] = v;
        if (i < nrow && rec) {
          const int mi = rowi[i * kRI + R_MON];
          if (mi >= 0) rec_store(d, rec, (int64_t)(step - rec_first) * n_mon + mi, (int64_t)it * n_mon + mi, v);
        }
      }
    }
    // After a wait ran out (thread 0 only waits) the CTA leaves the step loop at the end of that
    // step: it arms no mbarrier again (a second arrival on a phase that never completed is
    // undefined) and pushes nothing more, so its peers' waits run out too and every CTA meets at
    // the exit barrier.
    if (__syncthreads_or(dead)) break;
  }
  // no CTA leaves while another may still write into its shared memory
  if (C > 1) cluster_barrier();
  // write the state back for the next launch and for readers
  for (int r = tid; r < nrow; r += kT4) sim.v_pos[p0 + r] = A::todbl(vloc[r]);
#pragma unroll
  for (int k = 0; k < kEPT; ++k) {
    const int e = tid + k * kT4;
    if (e < n_ends) q.Ih[m0 + e] = A::todbl(eI[k]);
  }
}

// FP64 record rows of one launch from its float-float staging record (before the step counter
// advances past the launch)
__global__ void k_rec_ff(const float2* __restrict__ rec_ff, int n, const SimDyn* dyn, int n_mon) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !dyn->rec) return;
  const int64_t row0 = (int64_t)(dyn->step_base + 1 - dyn->rec_first);
  dyn->rec[row0 * n_mon + i] = ff_to(rec_ff[i]);
}

template <int PREC>
bool func_setup() {
  static bool done = false, ok = false;
  if (!done) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    ok = cudaFuncSetAttribute(k_step4<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) == cudaSuccess &&
         cudaFuncSetAttribute(k_step4<PREC>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
    cudaGetLastError();
    done = true;
  }
  return ok;
}

template <int PREC>
void launch4(Sim& sm, int n, cudaStream_t s) {
  Step4& p = sm.s4;
  Step4D dv = p.view();
  const bool stage = PREC == EMT_PREC_FF64 && sm.cur_rec && sm.n_mon > 0;
  if (stage) {
    const size_t need = (size_t)n * sm.n_mon;
    if (p.rec_ff.n < need) p.rec_ff.alloc(need);
    dv.rec_ff = p.rec_ff.p;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p.C);
  cfg.blockDim = dim3(kT4);
  cfg.dynamicSmemBytes = p.smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = p.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = p.C > 1 ? 1 : 0;
  EMT_CUDA(cudaLaunchKernelEx(&cfg, k_step4<PREC>, sm.store->view(), sm.view(), sm.s2.view(sm), dv, n));
  if (stage) {
    const int tot = n * sm.n_mon;
    k_rec_ff<<<(tot + 255) / 256, 256, 0, s>>>(p.rec_ff.p, tot, sm.d_dyn.p, sm.n_mon);
    EMT_CUDA(cudaGetLastError());
  }
}

template <int PREC>
bool fits4(const Step4& p) {
  if (!func_setup<PREC>()) return false;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p.C);
  cfg.blockDim = dim3(kT4);
  cfg.dynamicSmemBytes = p.smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = p.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int ncl = 0;
  const cudaError_t e = cudaOccupancyMaxActiveClusters(&ncl, k_step4<PREC>, &cfg);
  cudaGetLastError();
  return e == cudaSuccess && ncl >= 1;
}

size_t align16(size_t x) { return (x + 15) / 16 * 16; }

}  // namespace

Step4D Step4::view() const {
  Step4D v{};
  v.C = C;
  v.P = P;
  v.o_x = (int)o_x;
  v.o_part = (int)o_part;
  v.o_ycp = (int)o_ycp;
  v.o_ycut = (int)o_ycut;
  v.o_yvp = (int)o_yvp;
  v.o_s = (int)o_s;
  v.s_total = s_total;
  v.o_v = (int)o_v;
  v.o_contrib = (int)o_contrib;
  v.o_row = (int)o_row;
  v.o_vrow = (int)o_vrow;
  v.o_out = (int)o_out;
  v.o_push = (int)o_push;
  v.o_sx = (int)o_sx;
  v.o_K = (int)o_K;
  v.o_L = (int)o_L;
  v.o_F = (int)o_F;
  v.fstride = fstride;
  v.max_vrows = max_vrows;
  v.e_max = e_max;
  v.ldk = ldk;
  v.n_crow = n_crow;
  v.hdr = hdr.p;
  v.tab = tab.p;
  v.K = K.p;
  v.rec_ff = nullptr;
  return v;
}

// K from the current sweep image (after a build, a modification or a reset).
void Step4::refresh(const Sim& sm, cudaStream_t s) {
  if (!ready) return;
  const Step2D q = sm.s2.view(sm);
  build_sweep_matrix(sm.store->precision, q.img, q.img_bytes, q.cores, q.core_bytes, n_crow, s_total, ldk, K.p, s);
}

// Host plan: positions per CTA, halos, leaf-stage outputs and their push destinations, copy
// lists, slices of s and the shared-memory layout. Returns false (the generation stays unusable)
// when the network does not fit one cluster of n_cta CTAs.
bool Step4::build(Sim& sm, int n_cta, cudaStream_t s) {
  ready = false;
  const Store& st = *sm.store;
  const Step2& s2 = sm.s2;
  if (!s2.ready || s2.prec != st.precision) return false;
  if (st.precision != EMT_PREC_FF64 && st.precision != EMT_PREC_FP64) return false;
  if (n_cta < 1 || n_cta > 16 || (n_cta & (n_cta - 1))) return false;
  if (st.L_elems >= INT_MAX / 4 || st.F_elems >= INT_MAX / 4) return false;
  const Tree& t = st.tree;
  const int nl = st.n_leaf;
  const int n = sm.n;
  if (n_cta > n) return false;
  std::vector<int> llo(nl), lhi(nl), lb(nl), lld(nl);
  for (int j = 0; j < nl; ++j) {
    const int node = st.leaf_nodes_h[j];
    llo[j] = t.lo[node];
    lhi[j] = t.hi[node];
    lb[j] = lhi[j] - llo[j];
    lld[j] = st.leaf_ld_h[j];
  }
  auto leaf_of = [&](int ps) { return leaf_index_of_pos(st, ps); };
  // ---- positions of each CTA: part of one leaf (n_cta >= n_leaf) or whole leaves
  std::vector<int> cp0, cp1, cj0, cj1, cpart;
  int Pn = 1;
  if (n_cta >= nl) {
    std::vector<int> cnt(nl, 1);
    for (int left = n_cta - nl; left > 0; --left) {
      int best = 0;
      for (int j = 1; j < nl; ++j)
        if ((double)lb[j] * lb[j] / cnt[j] > (double)lb[best] * lb[best] / cnt[best]) best = j;
      cnt[best]++;
    }
    for (int j = 0; j < nl; ++j) {
      if (cnt[j] > lb[j]) return false;
      Pn = std::max(Pn, cnt[j]);
      for (int u = 0; u < cnt[j]; ++u) {
        cp0.push_back(llo[j] + (int)((int64_t)lb[j] * u / cnt[j]));
        cp1.push_back(llo[j] + (int)((int64_t)lb[j] * (u + 1) / cnt[j]));
        cj0.push_back(j);
        cj1.push_back(j + 1);
        cpart.push_back(u);
      }
    }
  } else {
    for (int c = 0; c < n_cta; ++c) {
      const int j0 = (int)((int64_t)nl * c / n_cta), j1 = (int)((int64_t)nl * (c + 1) / n_cta);
      cp0.push_back(llo[j0]);
      cp1.push_back(lhi[j1 - 1]);
      cj0.push_back(j0);
      cj1.push_back(j1);
      cpart.push_back(0);
    }
  }
  std::vector<int> owner(n, -1);
  for (int c = 0; c < n_cta; ++c)
    for (int ps = cp0[c]; ps < cp1[c]; ++ps) owner[ps] = c;
  for (int ps = 0; ps < n; ++ps)
    if (owner[ps] < 0) return false;
  // ---- element ends (position order, as in the generation-2 records)
  const std::vector<IncRec>& inc = s2.inc0;
  std::vector<int> iptr(n + 1, 0);
  for (const IncRec& r : inc) iptr[r.self + 1]++;
  for (int ps = 0; ps < n; ++ps) iptr[ps + 1] += iptr[ps];
  std::vector<int> crow_of(n, -1);
  for (size_t k = 0; k < st.cut_rows.crow_pos.size(); ++k) crow_of[st.cut_rows.crow_pos[k]] = (int)k;
  // halos: far ends of the CTA's elements outside its positions
  std::vector<std::vector<int>> halo(n_cta);
  std::vector<std::vector<std::pair<int, int>>> readers(n);   // (CTA, expansion row) for halo use
  for (int c = 0; c < n_cta; ++c) {
    std::vector<int> h;
    for (int m = iptr[cp0[c]]; m < iptr[cp1[c]]; ++m) {
      const int o = inc[m].other;
      if (o >= 0 && (o < cp0[c] || o >= cp1[c])) h.push_back(o);
    }
    std::sort(h.begin(), h.end());
    h.erase(std::unique(h.begin(), h.end()), h.end());
    halo[c] = h;
    for (size_t i = 0; i < h.size(); ++i) readers[h[i]].push_back({c, (cp1[c] - cp0[c]) + (int)i});
  }
  // ---- slices of s: CTA c forms rows [s_total c / C, s_total (c + 1) / C) of s = K y_cut
  n_crow = s2.header.n_crow;
  s_total = s2.header.s_total;
  ldk = (n_crow + 1) / 2 * 2;
  P = Pn;
  std::vector<int> cs0(n_cta), cs1(n_cta);
  int max_slice = 0;
  for (int c = 0; c < n_cta; ++c) {
    cs0[c] = (int)((int64_t)s_total * c / n_cta);
    cs1[c] = (int)((int64_t)s_total * (c + 1) / n_cta);
    max_slice = std::max(max_slice, cs1[c] - cs0[c]);
  }
  // K is block-sparse: the rows of s of node q depend only on the cut rows inside q's subtree
  // (the entries of K outside are exactly zero), so a cut row's partial goes only to the CTAs
  // whose slice of s holds a node containing it; the slots of the others stay zero.
  std::vector<std::vector<std::pair<int, int>>> need(n_cta);   // position ranges per CTA
  {
    std::vector<int> s_node(std::max(s_total, 1), -1);
    for (int q = 0; q < (int)t.lo.size(); ++q)
      if (t.left[q] >= 0)
        for (int r = 0; r < 2 * st.node_k_h[q]; ++r) s_node[st.node_soff_h[q] + r] = q;
    for (int c = 0; c < n_cta; ++c) {
      int last = -2;
      for (int r = cs0[c]; r < cs1[c]; ++r) {
        const int q = s_node[r];
        if (q >= 0 && q != last) need[c].push_back({t.lo[q], t.hi[q]});
        last = q;
      }
    }
  }
  auto needs = [&](int c, int ps) {
    for (auto& rg : need[c])
      if (ps >= rg.first && ps < rg.second) return true;
    return false;
  };
  // ---- sizes
  // elements of a position's packed factor row: k of every ancestor (the P or Q row of Eq. 9)
  auto frow = [&](int ps) {
    int64_t e = 0;
    for (int a = t.parent[st.leaf_nodes_h[leaf_of(ps)]]; a >= 0; a = t.parent[a]) e += st.node_k_h[a];
    return e;
  };
  std::vector<int> n_out(n_cta, 0), lpv(n_cta, 1), n_push(n_cta, 0);
  int max_rows = 0, max_ends = 0, max_out = 0, max_push = 0, max_part = 0;
  int64_t maxL = 0, maxF = 0;
  int max_packed = 0;   // longest packed factor row (sum of k over a path)
  int max_sx = 0;       // longest s-index table of a CTA (one list of max_packed per leaf it expands rows of)
  max_vrows = 0;
  for (int c = 0; c < n_cta; ++c) {
    const int nr = cp1[c] - cp0[c];
    max_rows = std::max(max_rows, nr);
    max_vrows = std::max(max_vrows, nr + (int)halo[c].size());
    max_ends = std::max(max_ends, iptr[cp1[c]] - iptr[cp0[c]]);
    int64_t Le = 0, Fe = 0;
    for (int ps = cp0[c]; ps < cp1[c]; ++ps) {
      Le += lld[leaf_of(ps)];
      Fe += frow(ps);
    }
    for (int ps : halo[c]) Fe += frow(ps);
    maxL = std::max(maxL, Le);
    maxF = std::max(maxF, Fe);
    for (int ps = cp0[c]; ps < cp1[c]; ++ps) max_packed = std::max(max_packed, (int)frow(ps));
    for (int ps : halo[c]) max_packed = std::max(max_packed, (int)frow(ps));
    {
      std::vector<int> lv;
      for (int ps = cp0[c]; ps < cp1[c]; ++ps) lv.push_back(leaf_of(ps));
      for (int ps : halo[c]) lv.push_back(leaf_of(ps));
      std::sort(lv.begin(), lv.end());
      max_sx = std::max(max_sx, (int)(std::unique(lv.begin(), lv.end()) - lv.begin()));
    }
    for (int j = cj0[c]; j < cj1[c]; ++j) {
      n_out[c] += lb[j];
      for (int r = 0; r < lb[j]; ++r) {
        const int ps = llo[j] + r;
        n_push[c] += 1 + (int)readers[ps].size();
        if (crow_of[ps] >= 0)
          for (int cc = 0; cc < n_cta; ++cc) n_push[c] += needs(cc, ps) ? 1 : 0;
      }
    }
    const int pad = (n_out[c] + 31) / 32 * 32;
    lpv[c] = std::max(1, kT4 / pad);
    max_out = std::max(max_out, n_out[c]);
    max_push = std::max(max_push, n_push[c]);
    max_part = std::max(max_part, lpv[c] * pad);
  }
  if (max_ends > kEPT * kT4 || max_rows > kT4) return false;
  // ---- shared-memory layout (identical in every CTA, so a remote address is the local one)
  const size_t tb = 8;   // FP64 or float-float element
  e_max = max_packed;
  max_sx *= max_packed;
  size_t off = 64;   // mbarriers (prologue, s x 2, partials x 2) and flags
  o_x = off;         off = align16(off + (size_t)std::max(max_rows, 1) * tb);
  o_part = off;      off = align16(off + (size_t)max_part * tb);
  o_ycp = off;       off = align16(off + (size_t)std::max(n_crow * P, 1) * tb);
  o_ycut = off;      off = align16(off + (size_t)std::max(ldk, 2) * tb);
  o_yvp = off;       off = align16(off + (size_t)2 * max_vrows * P * tb);
  o_s = off;         off = align16(off + (size_t)2 * std::max(s_total, 1) * tb);   // two step parities
  o_v = off;         off = align16(off + (size_t)max_vrows * tb);
  o_contrib = off;   off = align16(off + (size_t)std::max(max_ends, 1) * tb);
  o_row = off;       off = align16(off + (size_t)max_rows * kRI * 4);
  o_vrow = off;      off = align16(off + (size_t)max_vrows * kVR * 4);
  o_out = off;       off = align16(off + (size_t)std::max(max_out, 1) * kOR * 4);
  o_push = off;      off = align16(off + (size_t)std::max(max_push, 1) * kPR * 4);
  o_sx = off;        off = align16(off + (size_t)std::max(max_sx, 1) * 4);
  o_K = off;         off = align16(off + (size_t)max_slice * ldk * tb);
  o_L = off;         off = align16(off + (size_t)maxL * tb);
  // element-major factor rows: stride = 8 (mod 16) elements, so two 8-byte columns of one warp
  // fall in different halves of the banks
  fstride = max_vrows + ((8 - max_vrows % 16) + 16) % 16;
  (void)maxF;
  o_F = off;         off = align16(off + (size_t)max_packed * fstride * tb);
  smem = off;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem + 1024 > (size_t)optin) return false;
  // ---- per-CTA header and tables
  std::vector<int> H((size_t)n_cta * kHdr, 0), TB;
  for (int c = 0; c < n_cta; ++c) {
    int* h = &H[(size_t)c * kHdr];
    const int nr = cp1[c] - cp0[c];
    h[H_P0] = cp0[c];
    h[H_P1] = cp1[c];
    h[H_NHALO] = (int)halo[c].size();
    h[H_M0] = iptr[cp0[c]];
    h[H_M1] = iptr[cp1[c]];
    h[H_S0] = cs0[c];
    h[H_S1] = cs1[c];
    h[H_LP] = lpv[c];
    // the CTA's rows of the leaf inverses (= its columns): one bulk copy per row
    h[H_OLROW] = (int)TB.size();
    std::vector<int> row_loff(nr);
    int64_t dst = 0, lbytes = 0;
    for (int r = 0; r < nr; ++r) {
      const int ps = cp0[c] + r;
      const int j = leaf_of(ps);
      row_loff[r] = (int)dst;
      TB.push_back((int)(st.leaf_off_h[j] + (int64_t)(ps - llo[j]) * lld[j]));
      TB.push_back((int)dst);
      TB.push_back(lld[j]);
      lbytes += (int64_t)lld[j] * (int64_t)tb;
      dst += lld[j];
    }
    h[H_LBYTES] = (int)lbytes;
    // expansion rows (own, then halo) and their packed factor rows: the k elements of the
    // position's row of P (left child) or Q (right child) at every ancestor, back to back; all
    // rows of one leaf sit in the same child of each ancestor, so they share one list of the
    // entries of s that those elements multiply (padded with entry 0 up to e_max)
    std::vector<int> vpos;
    for (int ps = cp0[c]; ps < cp1[c]; ++ps) vpos.push_back(ps);
    for (int ps : halo[c]) vpos.push_back(ps);
    std::vector<int> vr, fc, sxl, sx_at(nl, -1);
    for (size_t i = 0; i < vpos.size(); ++i) {
      const int ps = vpos[i];
      int64_t fdst = 0;   // element offset within the row's packed sequence
      const int j = leaf_of(ps);
      if (sx_at[j] < 0) {
        sx_at[j] = (int)sxl.size();
        const int leaf_lo = t.lo[st.leaf_nodes_h[j]];
        for (int a = t.parent[st.leaf_nodes_h[j]]; a >= 0; a = t.parent[a]) {
          const int k = st.node_k_h[a];
          const int si = leaf_lo < t.hi[t.left[a]] ? st.node_soff_h[a] : st.node_soff_h[a] + k;
          for (int e = 0; e < k; ++e) sxl.push_back(si + e);
        }
        sxl.resize((size_t)sx_at[j] + e_max, 0);
      }
      vr.push_back(ps);
      vr.push_back((int)i);
      vr.push_back(sx_at[j]);
      vr.push_back(i < (size_t)nr ? (int)i : -1);
      for (int a = t.parent[st.leaf_nodes_h[j]]; a >= 0; a = t.parent[a]) {
        const int k = st.node_k_h[a], kld = st.node_kld_h[a];
        if (k > 0) {
          fc.push_back((int)(st.node_foff_h[a] + (int64_t)(ps - t.lo[a]) * kld));
          fc.push_back((int)(fdst * fstride + (int64_t)i));
          fc.push_back(k);
        }
        fdst += k;
      }
    }
    if ((int)sxl.size() > max_sx) return false;   // cannot happen: one list per distinct leaf
    h[H_OSX] = (int)TB.size();
    h[H_NSX] = (int)sxl.size();
    TB.insert(TB.end(), sxl.begin(), sxl.end());
    h[H_NFC] = (int)fc.size() / 3;
    h[H_OFC] = (int)TB.size();
    TB.insert(TB.end(), fc.begin(), fc.end());
    h[H_OVROW] = (int)TB.size();
    TB.insert(TB.end(), vr.begin(), vr.end());
    // own rows: element-end range of the injection (monitor index filled in by the kernel)
    h[H_OROW] = (int)TB.size();
    for (int r = 0; r < nr; ++r) {
      const int ps = cp0[c] + r;
      TB.push_back(iptr[ps] - iptr[cp0[c]]);
      TB.push_back(iptr[ps + 1] - iptr[cp0[c]]);
      TB.push_back(-1);
      TB.push_back(0);
    }
    // leaf-stage outputs (every row of each leaf the CTA holds columns of) and their pushes
    std::vector<int> outs, pushes;
    int o = 0;
    for (int j = cj0[c]; j < cj1[c]; ++j) {
      const int a0 = std::max(cp0[c], llo[j]), a1 = std::min(cp1[c], lhi[j]);
      for (int r = 0; r < lb[j]; ++r, ++o) {
        const int ps = llo[j] + r;
        outs.push_back(row_loff[a0 - cp0[c]] + r);
        outs.push_back(lld[j]);
        outs.push_back(a1 - a0);
        outs.push_back(a0 - cp0[c]);
        const int ow = owner[ps];
        pushes.push_back(o);
        pushes.push_back(ow);
        pushes.push_back((int)(o_yvp + ((size_t)(ps - cp0[ow]) * P + cpart[c]) * tb));
        pushes.push_back(P_YV);
        for (auto& rd : readers[ps]) {
          pushes.push_back(o);
          pushes.push_back(rd.first);
          pushes.push_back((int)(o_yvp + ((size_t)rd.second * P + cpart[c]) * tb));
          pushes.push_back(P_YV);
        }
        if (crow_of[ps] >= 0)
          for (int cc = 0; cc < n_cta; ++cc) {
            if (!needs(cc, ps)) continue;
            pushes.push_back(o);
            pushes.push_back(cc);
            pushes.push_back((int)(o_ycp + ((size_t)crow_of[ps] * P + cpart[c]) * tb));
            pushes.push_back(P_CUT);
          }
      }
    }
    h[H_NOUT] = o;
    h[H_OOUT] = (int)TB.size();
    TB.insert(TB.end(), outs.begin(), outs.end());
    h[H_NPUSH] = (int)pushes.size() / kPR;
    for (size_t u = 0; u < pushes.size(); u += kPR)
      if (pushes[u + 1] != c) H[(size_t)pushes[u + 1] * kHdr + H_YIN]++;
    h[H_OPUSH] = (int)TB.size();
    TB.insert(TB.end(), pushes.begin(), pushes.end());
    // element ends: local indices of the two voltages
    h[H_OENDL] = (int)TB.size();
    for (int m = iptr[cp0[c]]; m < iptr[cp1[c]]; ++m) {
      const int self = inc[m].self, oth = inc[m].other;
      TB.push_back(self - cp0[c]);
      int ol = -1;
      if (oth >= 0) {
        if (oth >= cp0[c] && oth < cp1[c]) ol = oth - cp0[c];
        else ol = nr + (int)(std::lower_bound(halo[c].begin(), halo[c].end(), oth) - halo[c].begin());
      }
      TB.push_back(ol);
    }
  }
  C = n_cta;
  const bool fit = st.precision == EMT_PREC_FF64 ? fits4<EMT_PREC_FF64>(*this) : fits4<EMT_PREC_FP64>(*this);
  if (!fit) return false;
  hdr.upload(H, s);
  tab.upload(TB.empty() ? std::vector<int>{0} : TB, s);
  K.alloc(std::max<size_t>((size_t)s_total * ldk, 1));
  EMT_CUDA(cudaMemsetAsync(K.p, 0, K.n * sizeof(double), s));
  ready = true;
  refresh(sm, s);
  EMT_CUDA(cudaStreamSynchronize(s));
  return true;
}

void step4_launch(Sim& sm, int n, cudaStream_t s) {
  if (n <= 0) return;
  if (sm.store->precision == EMT_PREC_FF64) launch4<EMT_PREC_FF64>(sm, n, s);
  else launch4<EMT_PREC_FP64>(sm, n, s);
}

}  // namespace emt

// Fused single-vector kernels of the hierarchical apply v = Ginv i (Eq. 2 with the store of Sec. III).
//
// One application is two kernels:
//   partial  each CTA owns rows [r0, r1) of one leaf j and, by symmetry of the leaf inverse
//            (L_j[:, rows] = L_j[rows, :]^T), streams exactly those rows once:
//            part_c = sum_{r in rows} L_j[r, :] x_r. Only the CTA's own x entries are needed,
//            so whatever produces x (a gather, a residual, the EMT history update) stays local.
//   sweep    each CTA reduces the leaf partials it needs (its own rows and the cut endpoints),
//            runs the boundary sweep of all tree nodes bottom-up (t_p = [h_l^T y_l; h_r^T y_r],
//            a gather of corrected cut rows using the symmetry P^T x = h_l^T Ginv_l x; s_p = C_p t_p)
//            and expands its own rows: v_i = y_i - sum over ancestors q of F_q[i] . s_q(half).
// The sweep is tiny and is repeated per CTA so that no third grid-wide dependency is needed.
// Arithmetic per precision: FP64 (double), FF64 (float-float pairs on the FP32 pipes: the FP64
// rate of this GPU is ~1/58 of its FP32 rate, so FP64 operations are kept out of inner loops),
// FP32. Intermediate vectors live in the accumulator's own type.
#pragma once
#include "store.h"

namespace emt {

// ------------------------------------------------------------------ float-float arithmetic
// Error-free transformations: Knuth's TwoSum and the FMA-based TwoProd (Dekker 1971 splits a
// product exactly; with an FMA the error term is fma(a, b, -a*b)). The __f*_rn intrinsics keep
// the compiler from contracting or reassociating them.
//
// The conversions between double and float-float avoid this GPU's FP64 pipe, which sustains about
// one thread-operation per cycle per SM (a double<->float conversion pair with an add about 0.6),
// against a few hundred for FP32 and integer operations: they work on the bit patterns. Values
// outside the range where both parts are normal floats take the FP64 instructions.
// The FP64 fallbacks are real calls, never inlined, so that the compiler cannot turn the rare
// branch into predicated FP64 instructions that every call would issue.
static __device__ __noinline__ float2 ff_from_fp64(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}
static __device__ __noinline__ double ff_to_fp64(float2 a) { return (double)a.x + (double)a.y; }
// hi = x truncated to 24 significant bits (its top bits with the exponent rebiased), lo = the other
// 29 bits rounded to a float and scaled by 2^(e - 1075); hi + lo = x to 2^-48 relative.
__device__ __forceinline__ float2 ff_from(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  if ((b << 1) == 0ull) return make_float2(__uint_as_float(sign), 0.0f);
  const int ef = (int)((b >> 52) & 0x7ffu) - 896;   // float-biased exponent of hi (1023 - 127)
  if (ef < 53 || ef > 253) return ff_from_fp64(x);
  const float hi = __uint_as_float(sign | ((unsigned int)ef << 23) | ((unsigned int)(b >> 29) & 0x7fffffu));
  const float scale = __uint_as_float((unsigned int)(ef - 52) << 23);
  const float lo = __fmul_rn(__uint2float_rn((unsigned int)b & 0x1fffffffu), scale);
  return make_float2(hi, __uint_as_float(__float_as_uint(lo) | sign));
}
// the double nearest below-or-at hi + lo: hi's significand on 53 bits, lo's added at its offset,
// renormalised by the leading-zero count (truncation: within 2^-52 relative)
__device__ __forceinline__ double ff_to(float2 a) {
  const unsigned int bh = __float_as_uint(a.x), bl = __float_as_uint(a.y);
  const bool lo_zero = (bl << 1) == 0u;
  if ((bh << 1) == 0u && lo_zero) return __longlong_as_double((long long)(bh & 0x80000000u) << 32);
  const int eh = (int)(bh >> 23) & 0xff, el = (int)(bl >> 23) & 0xff;
  if (eh == 0 || eh == 255 || el == 255 || (el == 0 && !lo_zero)) return ff_to_fp64(a);
  long long m = (long long)((bh & 0x7fffffu) | 0x800000u) << 29;
  if (!lo_zero) {
    const int sh = el - eh + 29;
    if (sh >= 40) return ff_to_fp64(a);
    long long ml = (long long)((bl & 0x7fffffu) | 0x800000u);
    ml = sh >= 0 ? (ml << sh) : (sh > -40 ? (ml >> -sh) : 0ll);
    m = ((bh ^ bl) & 0x80000000u) ? m - ml : m + ml;
  }
  if (m <= 0) return ff_to_fp64(a);
  const int s = __clzll(m) - 11;
  m = s >= 0 ? (m << s) : (m >> -s);
  const long long e = (long long)(eh + 896 - s);
  return __longlong_as_double(((long long)(bh & 0x80000000u) << 32) | (e << 52) | (m & ((1ll << 52) - 1)));
}
__device__ __forceinline__ float2 ff_norm(float hi, float lo) {
  const float s = __fadd_rn(hi, lo);
  return make_float2(s, __fsub_rn(lo, __fsub_rn(s, hi)));
}
// (hi, lo) += a * x, kept unnormalised
__device__ __forceinline__ void ff_fma(float& hi, float& lo, float2 a, float2 x) {
  const float p = __fmul_rn(a.x, x.x);
  const float pe = __fmaf_rn(a.x, x.x, -p);
  const float plo = __fmaf_rn(a.x, x.y, __fmaf_rn(a.y, x.x, pe));
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, plo));
}
__device__ __forceinline__ void ff_add(float& hi, float& lo, float2 b) {
  const float s = __fadd_rn(hi, b.x);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, b.y));
}

// Accumulator of one dot product; X is the type vectors are kept in.
template <int PREC>
struct Acc;
template <>
struct Acc<EMT_PREC_FP64> {
  using T = double;   // stored element
  using X = double;   // vector entry
  double v = 0.0;
  __device__ static X prep(double x) { return x; }
  __device__ static double todbl(X x) { return x; }
  __device__ static X zero() { return 0.0; }
  __device__ void fma(T a, X x) { v = __fma_rn(a, x, v); }
  __device__ void add(X x) { v += x; }
  __device__ X getx() const { return v; }
  __device__ X shfl_xor(X x, int o) const { return __shfl_xor_sync(0xffffffffu, x, o); }
};
template <>
struct Acc<EMT_PREC_FF64> {
  using T = float2;
  using X = float2;
  float hi = 0.f, lo = 0.f;
  __device__ static X prep(double x) { return ff_from(x); }
  __device__ static double todbl(X x) { return ff_to(x); }
  __device__ static X zero() { return make_float2(0.f, 0.f); }
  __device__ void fma(T a, X x) { ff_fma(hi, lo, a, x); }
  __device__ void add(X x) { ff_add(hi, lo, x); }
  __device__ X getx() const { return ff_norm(hi, lo); }
  __device__ X shfl_xor(X x, int o) const {
    return make_float2(__shfl_xor_sync(0xffffffffu, x.x, o), __shfl_xor_sync(0xffffffffu, x.y, o));
  }
};
template <>
struct Acc<EMT_PREC_FP32> {
  using T = float;
  using X = float;
  float v = 0.f;
  __device__ static X prep(double x) { return __double2float_rn(x); }
  __device__ static double todbl(X x) { return (double)x; }
  __device__ static X zero() { return 0.f; }
  __device__ void fma(T a, X x) { v = __fmaf_rn(a, x, v); }
  __device__ void add(X x) { v = __fadd_rn(v, x); }
  __device__ X getx() const { return v; }
  __device__ X shfl_xor(X x, int o) const { return __shfl_xor_sync(0xffffffffu, x, o); }
};

__device__ __forceinline__ double neg(double x) { return -x; }
__device__ __forceinline__ float neg(float x) { return -x; }
__device__ __forceinline__ float2 neg(float2 x) { return make_float2(-x.x, -x.y); }

template <int PREC>
struct Elem;
template <>
struct Elem<EMT_PREC_FP64> {
  static constexpr int VE = 2;   // elements per 16-byte load
  __device__ static const double* L(const DStore& s) { return s.L64; }
  __device__ static const double* F(const DStore& s) { return s.F64; }
  __device__ static const double* C(const DStore& s) { return s.C64; }
};
template <>
struct Elem<EMT_PREC_FF64> {
  static constexpr int VE = 2;
  __device__ static const float2* L(const DStore& s) { return s.Lff; }
  __device__ static const float2* F(const DStore& s) { return s.Fff; }
  __device__ static const float2* C(const DStore& s) { return s.Cff; }
};
template <>
struct Elem<EMT_PREC_FP32> {
  static constexpr int VE = 4;
  __device__ static const float* L(const DStore& s) { return s.L32; }
  __device__ static const float* F(const DStore& s) { return s.F32; }
  __device__ static const float* C(const DStore& s) { return s.C32; }
};

// 16-byte read-only vector load of VE consecutive elements
__device__ __forceinline__ void vload(const double* p, double (&e)[2]) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  e[0] = v.x;
  e[1] = v.y;
}
__device__ __forceinline__ void vload(const float2* p, float2 (&e)[2]) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  e[0] = make_float2(v.x, v.y);
  e[1] = make_float2(v.z, v.w);
}
__device__ __forceinline__ void vload(const float* p, float (&e)[4]) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  e[0] = v.x;
  e[1] = v.y;
  e[2] = v.z;
  e[3] = v.w;
}

// Row -> CTA map of the fused kernels.
struct CtaMapD {
  const int* cta_leaf;
  const int* cta_r0;     // first local row of the CTA within its leaf
  const int* cta_r1;
  const int* leaf_cta0;  // first CTA of each leaf
  const int* leaf_ncta;
  int n_cta;
  int pld;               // leading dimension of the partial buffer
  int max_rows;          // largest r1 - r0
};

struct CutRowsD {
  const int* item_pos;
  const int* item_crow;
  const int* item_sidx;
  const int* item_cut;   // global cut index (a side, scaled by -g_e) or -1 (b side)
  const int* item_lvl;   // item ranges per depth, [max_depth + 2]
  const int* crow_pos;
  int n_crow;
  int n_items;
  int s_total;
};

constexpr int kFusedThreads = 256;
constexpr int kMaxSlotsPerThread = 4;

// part[col] = sum over the CTA's rows r of L_j[r, col] * xs[r - r0]   (xs in shared memory)
template <int PREC>
__device__ __forceinline__ void leaf_partial_core(const DStore& st, int j, int r0, int r1,
                                                  const typename Acc<PREC>::X* xs,
                                                  typename Acc<PREC>::X* __restrict__ out,
                                                  typename Acc<PREC>::X* red) {
  using E = Elem<PREC>;
  using A = Acc<PREC>;
  using T = typename A::T;
  constexpr int VE = E::VE;
  const int node = st.leaf_node[j];
  const int b = st.hi[node] - st.lo[node];
  const int ld = st.leaf_ld[j];
  const T* L = E::L(st) + st.leaf_off[j];
  const int slots = (b + VE - 1) / VE;
  const int cover = min(slots, kFusedThreads);
  const int G = kFusedThreads / cover;
  const int tid = threadIdx.x;
  const int g = tid / cover, sl = tid % cover;
  const int nrow = r1 - r0;
  A acc[kMaxSlotsPerThread][VE];
  if (g < G) {
    for (int r = g; r < nrow; r += G) {
      const typename A::X x = xs[r];
      const T* row = L + (int64_t)(r0 + r) * ld;
#pragma unroll
      for (int u = 0; u < kMaxSlotsPerThread; ++u) {
        const int s = sl + u * cover;
        if (s < slots) {
          T v[VE];
          vload(row + s * VE, v);
#pragma unroll
          for (int e = 0; e < VE; ++e) acc[u][e].fma(v[e], x);
        }
      }
    }
  }
  // reduce the G row groups in a fixed order (deterministic)
  const int width = slots * VE;
  if (g < G) {
#pragma unroll
    for (int u = 0; u < kMaxSlotsPerThread; ++u) {
      const int s = sl + u * cover;
      if (s < slots)
#pragma unroll
        for (int e = 0; e < VE; ++e) red[g * width + s * VE + e] = acc[u][e].getx();
    }
  }
  __syncthreads();
  for (int c = tid; c < b; c += kFusedThreads) {
    A s;
    for (int gg = 0; gg < G; ++gg) s.add(red[gg * width + c]);
    out[c] = s.getx();
  }
}

// Sum of the leaf partials of one position.
template <int PREC>
__device__ __forceinline__ typename Acc<PREC>::X leaf_y(const DStore& st, const CtaMapD& cm,
                                                        const typename Acc<PREC>::X* __restrict__ part, int pos) {
  const int j = st.pos_leaf[pos];
  const int loc = pos - st.lo[st.leaf_node[j]];
  const int c0 = cm.leaf_cta0[j], nc = cm.leaf_ncta[j];
  Acc<PREC> s;
  for (int c = 0; c < nc; ++c) s.add(part[(int64_t)(c0 + c) * cm.pld + loc]);
  return s.getx();
}

// Boundary sweep over the whole tree; leaves s of all nodes in shared memory (sm_s).
template <int PREC>
__device__ void boundary_sweep(const DStore& st, const CtaMapD& cm, const CutRowsD& cr,
                               const typename Acc<PREC>::X* __restrict__ part, typename Acc<PREC>::X* sm_ycut,
                               typename Acc<PREC>::X* sm_t, typename Acc<PREC>::X* sm_s,
                               const typename Acc<PREC>::X* __restrict__ cut_gx) {
  using E = Elem<PREC>;
  using A = Acc<PREC>;
  using T = typename A::T;
  const int tid = threadIdx.x;
  for (int c = tid; c < cr.n_crow; c += kFusedThreads) sm_ycut[c] = leaf_y<PREC>(st, cm, part, cr.crow_pos[c]);
  __syncthreads();
  const T* F = E::F(st);
  const T* C = E::C(st);
  for (int d = st.max_depth - 1; d >= 0; --d) {
    const int i0 = cr.item_lvl[d], i1 = cr.item_lvl[d + 1];
    for (int it = i0 + tid; it < i1; it += kFusedThreads) {
      const int cut = cr.item_cut[it];
      // a side of a block column: the W vertices cut_a .. cut_a + W - 1, rows crow .. crow + W - 1
      const int W = cut >= 0 ? st.cut_w : 1;
      A m;
      typename A::X val;
      for (int w = 0; w < W; ++w) {
        const int pos = cr.item_pos[it] + w;
        // value of the child's full result at pos: leaf value minus the corrections of every
        // internal ancestor strictly below depth d on pos's path (already in sm_s)
        A acc;
        acc.add(sm_ycut[cr.item_crow[it] + w]);
        int q = st.parent[st.leaf_node[st.pos_leaf[pos]]];
        while (q >= 0 && st.depth[q] > d) {
          const int kq = st.node_k[q];
          const int half = pos < st.hi[st.left[q]] ? 0 : kq;
          const T* Fi = F + st.node_foff[q] + (int64_t)(pos - st.lo[q]) * st.node_kld[q];
          const typename A::X* sq = sm_s + st.node_soff[q] + half;
          for (int e = 0; e < kq; ++e) acc.fma(Fi[e], neg(sq[e]));
          q = st.parent[q];
        }
        val = acc.getx();
        if (cut >= 0) m.fma(reinterpret_cast<const T*>(cut_gx)[(int64_t)cut * W + w], val);   // t = -g * value
      }
      if (cut >= 0) val = m.getx();
      sm_t[cr.item_sidx[it]] = val;
    }
    __syncthreads();
    // s_q = C_q t_q for the nodes at depth d (rows flattened over the level)
    const int n0 = st.lvl_ptr[d], n1 = st.lvl_ptr[d + 1];
    int total = 0;
    for (int x = n0; x < n1; ++x) total += 2 * st.node_k[st.lvl_nodes[x]];
    for (int w = tid; w < total; w += kFusedThreads) {
      int rem = w, x = n0;
      while (rem >= 2 * st.node_k[st.lvl_nodes[x]]) {
        rem -= 2 * st.node_k[st.lvl_nodes[x]];
        ++x;
      }
      const int q = st.lvl_nodes[x];
      const int m2 = 2 * st.node_k[q];
      const T* Cr = C + st.node_coff[q] + (int64_t)rem * m2;
      const typename A::X* tq = sm_t + st.node_soff[q];
      A acc;
      for (int e = 0; e < m2; ++e) acc.fma(Cr[e], tq[e]);
      sm_s[st.node_soff[q] + rem] = acc.getx();
    }
    __syncthreads();
  }
}

// v_i = y_i - sum over ancestors q of F_q[i] . s_q(half of i); one warp per row, result on all lanes.
template <int PREC>
__device__ __forceinline__ typename Acc<PREC>::X expand_row(const DStore& st, int leaf_node, int pos,
                                                            typename Acc<PREC>::X y,
                                                            const typename Acc<PREC>::X* s) {
  using E = Elem<PREC>;
  using A = Acc<PREC>;
  using T = typename A::T;
  const int lane = threadIdx.x & 31;
  const T* F = E::F(st);
  A acc;
  for (int q = st.parent[leaf_node]; q >= 0; q = st.parent[q]) {
    const int kq = st.node_k[q];
    const int half = pos < st.hi[st.left[q]] ? 0 : kq;
    const T* Fi = F + st.node_foff[q] + (int64_t)(pos - st.lo[q]) * st.node_kld[q];
    const typename A::X* sq = s + st.node_soff[q] + half;
    for (int e = lane; e < kq; e += 32) acc.fma(Fi[e], neg(sq[e]));
  }
  typename A::X v = acc.getx();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    A t;
    t.add(v);
    t.add(acc.shfl_xor(v, o));
    v = t.getx();
  }
  A r;
  r.add(y);
  r.add(v);
  return r.getx();
}

}  // namespace emt

// Multi-column EMT stepping (see multi.h).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "multi.h"

namespace emt {

namespace {

// ------------------------------------------------------------------ float-float helpers
__device__ __forceinline__ float2 ff_n(float hi, float lo) {
  const float s = __fadd_rn(hi, lo);
  return make_float2(s, __fsub_rn(lo, __fsub_rn(s, hi)));
}
__device__ __forceinline__ float2 ff_addx(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float bb = __fsub_rn(s, a.x);
  const float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
  return ff_n(s, __fadd_rn(err, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 ff_mulx(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, e));
  return ff_n(p, e);
}
__device__ __forceinline__ float2 ff_negx(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 ff_subx(float2 a, float2 b) { return ff_addx(a, ff_negx(b)); }
__device__ __forceinline__ float2 ff_f(float x) { return make_float2(x, 0.f); }

// Compensated accumulation (Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci.
// Comput. 26, 2005: Sum2 / Dot2) on float-float operands: the running value is (s, c) with s the
// FP32 sum of the leading parts and c the FP32 sum of every rounding error and trailing part;
// TwoSum and FMA-based TwoProduct make each step's error exact, and (s, c) is renormalised once
// when the value is stored. For the few terms summed here its error matches float-float's.
struct Acc2 {
  float s, c;
  __device__ __forceinline__ void add(float p, float e) {   // += p + e, p leading, e small
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    c = __fadd_rn(c, __fadd_rn(__fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z)), e));
    s = t;
  }
  __device__ __forceinline__ void add_prod(float2 a, float2 b) {   // += a b
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, e));
    add(p, e);
  }
  __device__ __forceinline__ float2 get() const { return ff_n(s, c); }
};
__device__ __forceinline__ Acc2 acc2(float2 x) { return Acc2{x.x, x.y}; }
// a b as an (unnormalised) pair: what add_prod gives on a zero accumulator, without its TwoSum
__device__ __forceinline__ Acc2 acc2_prod(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  return Acc2{p, __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, __fmaf_rn(a.x, b.x, -p)))};
}

float2 host_ff(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

// sweep metadata header (ints)
enum {
  M_NCROW = 0, M_NITEMS, M_STOTAL, M_MAXD, M_NCORE, M_OFF_CROW, M_OFF_LVL_ITEM, M_OFF_ITEM, M_OFF_SEG,
  M_OFF_LVL_CORE, M_OFF_CORE, M_HEADER = 16
};

// ------------------------------------------------------------------ kernels
__global__ void k_mc_trig(float2* trig, int first_step, int n, double omega, double dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s, c;
  sincos(omega * ((double)(first_step + i) * dt), &s, &c);
  const float sh = (float)s, ch = (float)c;
  trig[2 * i] = make_float2(sh, (float)(s - (double)sh));
  trig[2 * i + 1] = make_float2(ch, (float)(c - (double)ch));
}

// history update of every element end and injection, one (position, column) per thread
__device__ __forceinline__ bool change_on(const MSimD& m, int c, int step) {
  return m.trip_step[c] > 0 && step >= m.trip_step[c] && step < m.trip_off[c];
}

// History update of every element and injection: i = i_in(t) + i_his(t - dt) of Eq. 1 with the
// trapezoidal companion sources (Sec. II), for every column. A CTA takes `ipp` consecutive
// positions (1, 2, 4 or 8) and 256 columns, one per thread. The element-end records and row
// pointers of its positions are staged in shared memory first, so that each position then costs
// one round trip to memory: its voltage, the other ends' voltages, the old histories (up to IKB
// ends) and the source terms (up to ITB) are all loaded before any arithmetic.
constexpr int IPP_MAX = 8, ITH = 256, IKB = 6, ITB = 2;
__global__ void __launch_bounds__(ITH, 4) k_mc_inject(MSimD m, int ipp, int s_in_chunk, int* status) {
  extern __shared__ __align__(16) unsigned char ism[];
  MRec* srec = reinterpret_cast<MRec*>(ism);
  __shared__ int sptr[IPP_MAX + 1], tptr[IPP_MAX + 1];
  if (*status != DEV_OK) return;   // uniform, before any barrier
  const int p0 = blockIdx.x * ipp, np = min(ipp, m.n - p0);
  const int tid = threadIdx.x, c = blockIdx.y * ITH + tid;
  if (tid <= np) {
    sptr[tid] = m.inc_ptr[p0 + tid];
    tptr[tid] = m.term_ptr[p0 + tid];
  }
  __syncthreads();
  const int r0 = sptr[0];
  for (int i = tid; i < sptr[np] - r0; i += ITH) srec[i] = m.inc[r0 + i];
  __syncthreads();
  if (c >= m.R_act) return;
  const int step = m.dyn->step_base + s_in_chunk + 1;
  const int64_t R = m.R;
  const float2* Ih_rd = m.Ih + (int64_t)((step - 1) & 1) * m.n_el * R;
  float2* Ih_wr = m.Ih + (int64_t)(step & 1) * m.n_el * R;
  const int te = change_on(m, c, step) ? m.trip_elem[c] : -1;   // tripped element of this column
  const int ti = step - m.dyn->trig_first;
  const float2 sw = m.trig[2 * ti], cw = m.trig[2 * ti + 1];
  for (int pi = 0; pi < np; ++pi) {
    const int pos = p0 + pi;
    const int k1 = sptr[pi + 1] - r0, t1 = tptr[pi + 1];
    int kb = sptr[pi] - r0, tb = tptr[pi];
    const float2 vi = m.V[pos * R + c];
    Acc2 hist{0.f, 0.f}, inj{0.f, 0.f};
    do {
      float2 vo[IKB], ih[IKB], tc[ITB], ts[ITB];
#pragma unroll
      for (int q = 0; q < IKB; ++q) {
        if (kb + q < k1) {
          const MRec& r = srec[kb + q];
          vo[q] = r.other >= 0 ? m.V[(int64_t)r.other * R + c] : ff_f(0.f);
          ih[q] = Ih_rd[(int64_t)r.elem * R + c];
        }
      }
#pragma unroll
      for (int q = 0; q < ITB; ++q) {
        if (tb + q < t1) {
          tc[q] = m.term_cs[(int64_t)(tb + q) * R + c];
          ts[q] = m.term_sn[(int64_t)(tb + q) * R + c];
        }
      }
#pragma unroll
      for (int q = 0; q < IKB; ++q) {
        if (kb + q >= k1) break;
        const MRec& r = srec[kb + q];
        // v_e = v_from - v_to (TwoSum of the leading parts), formed identically at both ends
        const float2 vf = r.sgn > 0 ? vi : vo[q], vt = r.sgn > 0 ? vo[q] : vi;
        Acc2 de = acc2(vf);
        de.add(-vt.x, -vt.y);
        const float2 ve = make_float2(de.s, de.c);
        // Ih' = a1 v_e + beta Ih, renormalised once (it is state)
        Acc2 h = acc2_prod(r.a1, ve);
        h.add_prod(r.beta, ih[q]);
        float2 ihn = h.get();
        if (r.elem == te) ihn = ff_f(0.f);   // the tripped element carries no current
        if (r.sgn > 0) {
          hist.add(-ihn.x, -ihn.y);
          Ih_wr[(int64_t)r.elem * R + c] = ihn;
        } else {
          hist.add(ihn.x, ihn.y);
        }
      }
#pragma unroll
      for (int q = 0; q < ITB; ++q) {
        if (tb + q >= t1) break;
        inj.add_prod(tc[q], sw);
        inj.add_prod(ts[q], cw);
      }
      kb += IKB;
      tb += ITB;
    } while (kb < k1 || tb < t1);
    inj.add(hist.s, hist.c);
    const float2 x = inj.get();
    m.X[pos * R + c] = x;
    m.Xf[pos * R + c] = x.x;
  }
}


// The same injection with two columns per thread (column stride even): the element-end record,
// the 32-bit index arithmetic and the loop control of an incidence serve both columns, and the
// pair of float-float values of a row is one 16-byte access. A thread whose second column lies
// beyond the active ones computes it but stores only the first. KB element ends per memory round
// trip; MINB CTAs per SM (the registers that allows: 6 ends with 2 CTAs, 3 with 3, 2 with 4).
__device__ __forceinline__ void ld_pair(const float2* p, float2 (&o)[2]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = make_float2(v.x, v.y);
  o[1] = make_float2(v.z, v.w);
}
__device__ __forceinline__ void st_pair(float2* p, const float2 (&o)[2], bool both) {
  if (both) *reinterpret_cast<float4*>(p) = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
  else p[0] = o[0];
}
// One element end's new history Ih' = a1 v_e + beta Ih (trapezoidal companion source, Sec. II),
// v_e = v_from - v_to as a TwoSum of the leading parts, renormalised once (it is state). Both ends
// of an element call it with the same operands in the same roles, so they form the same value.
__device__ __forceinline__ float2 hist_next(const MRec& r, float2 vf, float2 vt, float2 ih, int te) {
  Acc2 de = acc2(vf);
  de.add(-vt.x, -vt.y);
  Acc2 h = acc2_prod(r.a1, make_float2(de.s, de.c));
  h.add_prod(r.beta, ih);
  return r.elem == te ? ff_f(0.f) : h.get();   // the tripped element carries no current
}

template <int KB, int MINB>
__global__ void __launch_bounds__(ITH, MINB) k_mc_inject2(MSimD m, int ipp, int s_in_chunk, int* status) {
  extern __shared__ __align__(16) unsigned char ism[];
  MRec* srec = reinterpret_cast<MRec*>(ism);
  __shared__ int sptr[IPP_MAX + 1], tptr[IPP_MAX + 1];
  if (*status != DEV_OK) return;   // uniform, before any barrier
  const int p0 = blockIdx.x * ipp, np = min(ipp, m.n - p0);
  const int tid = threadIdx.x, c = 2 * (blockIdx.y * ITH + tid);
  if (tid <= np) {
    sptr[tid] = m.inc_ptr[p0 + tid];
    tptr[tid] = m.term_ptr[p0 + tid];
  }
  __syncthreads();
  const int r0 = sptr[0];
  for (int i = tid; i < sptr[np] - r0; i += ITH) srec[i] = m.inc[r0 + i];
  __syncthreads();
  if (c >= m.R_act) return;
  const bool both = c + 1 < m.R_act;
  const int step = m.dyn->step_base + s_in_chunk + 1;
  const int R = m.R;
  const float2* Ih_rd = m.Ih + ((step - 1) & 1) * m.n_el * R;
  float2* Ih_wr = m.Ih + (step & 1) * m.n_el * R;
  int te[2];
  te[0] = change_on(m, c, step) ? m.trip_elem[c] : -1;
  te[1] = both && change_on(m, c + 1, step) ? m.trip_elem[c + 1] : -1;
  const int ti = step - m.dyn->trig_first;
  const float2 sw = m.trig[2 * ti], cw = m.trig[2 * ti + 1];
  for (int pi = 0; pi < np; ++pi) {
    const int pos = p0 + pi;
    const int k1 = sptr[pi + 1] - r0, t1 = tptr[pi + 1];
    int kb = sptr[pi] - r0, tb = tptr[pi];
    float2 vi[2];
    ld_pair(m.V + pos * R + c, vi);
    Acc2 hist[2] = {{0.f, 0.f}, {0.f, 0.f}}, inj[2] = {{0.f, 0.f}, {0.f, 0.f}};
    do {
      float2 vo[KB][2], ih[KB][2], tc[ITB][2], ts[ITB][2];
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        if (kb + q < k1) {
          const MRec& r = srec[kb + q];
          if (r.other >= 0) ld_pair(m.V + r.other * R + c, vo[q]);
          else vo[q][0] = vo[q][1] = ff_f(0.f);
          ld_pair(Ih_rd + r.elem * R + c, ih[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < ITB; ++q) {
        if (tb + q < t1) {
          ld_pair(m.term_cs + (tb + q) * R + c, tc[q]);
          ld_pair(m.term_sn + (tb + q) * R + c, ts[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        if (kb + q >= k1) break;
        const MRec& r = srec[kb + q];
        float2 ihn[2];
        // the record, hence the branch, is the same for every thread of the CTA
        if (r.sgn > 0) {
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            ihn[j] = hist_next(r, vi[j], vo[q][j], ih[q][j], te[j]);
            hist[j].add(-ihn[j].x, -ihn[j].y);
          }
          st_pair(Ih_wr + r.elem * R + c, ihn, both);
        } else {
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            ihn[j] = hist_next(r, vo[q][j], vi[j], ih[q][j], te[j]);
            hist[j].add(ihn[j].x, ihn[j].y);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < ITB; ++q) {
        if (tb + q >= t1) break;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          inj[j].add_prod(tc[q][j], sw);
          inj[j].add_prod(ts[q][j], cw);
        }
      }
      kb += KB;
      tb += ITB;
    } while (kb < k1 || tb < t1);
    float2 x[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      inj[j].add(hist[j].s, hist[j].c);
      x[j] = inj[j].get();
    }
    st_pair(m.X + pos * R + c, x, both);
    if (both) *reinterpret_cast<float2*>(m.Xf + pos * R + c) = make_float2(x[0].x, x[1].x);
    else m.Xf[pos * R + c] = x[0].x;
  }
}

// Leaf stage as a GEMM over the columns (Eq. 2 with Sec. III's leaf blocks):
// Y[leaf rows] = L_j (FP32) * Xf[leaf rows].
// Tile 64 x 128, K step 16, 256 threads with an 8 x 4 register tile.
constexpr int GBM = 64, GBN = 128, GBK = 16;
__global__ void __launch_bounds__(256) k_mc_gemm(DStore st, const int4* __restrict__ tiles,
                                                 const float* __restrict__ Xf, float* __restrict__ Y, int R,
                                                 const int* status, int r_act) {
  __shared__ __align__(16) float As[GBK][GBM + 4];
  __shared__ __align__(16) float Bs[GBK][GBN + 4];
  if (*status != DEV_OK) return;
  const int4 tl = tiles[blockIdx.x];
  const int j = tl.x, m0 = tl.y, n0 = tl.z;
  if (n0 >= r_act) return;
  const int node = st.leaf_node[j];
  const int lo = st.lo[node], b = st.hi[node] - lo, ld = st.leaf_ld[j];
  const float* L = st.L32 + st.leaf_off[j];
  const int tid = threadIdx.x;
  const int ty = tid >> 5, tx = tid & 31;
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[i][q] = 0.f;
  for (int k0 = 0; k0 < b; k0 += GBK) {
    {
      const int row = tid >> 2, kq = (tid & 3) * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (m0 + row < b && k0 + kq < ld) v = __ldg(reinterpret_cast<const float4*>(L + (int64_t)(m0 + row) * ld + k0 + kq));
      As[kq + 0][row] = v.x;
      As[kq + 1][row] = v.y;
      As[kq + 2][row] = v.z;
      As[kq + 3][row] = v.w;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int kk = (tid >> 5) + 8 * h, nn = (tid & 31) * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k0 + kk < b) {
        const float* src = Xf + (int64_t)(lo + k0 + kk) * R + n0 + nn;
        if ((R & 3) == 0 && n0 + nn + 3 < R) v = *reinterpret_cast<const float4*>(src);
        else {
          if (n0 + nn + 0 < R) v.x = src[0];
          if (n0 + nn + 1 < R) v.y = src[1];
          if (n0 + nn + 2 < R) v.z = src[2];
          if (n0 + nn + 3 < R) v.w = src[3];
        }
      }
      *reinterpret_cast<float4*>(&Bs[kk][nn]) = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      float a[8], bv[4];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = As[kk][ty * 8 + i];
      const float4 b4 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      bv[0] = b4.x;
      bv[1] = b4.y;
      bv[2] = b4.z;
      bv[3] = b4.w;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = fmaf(a[i], bv[q], acc[i][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = m0 + ty * 8 + i;
    if (r >= b) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int cc = n0 + tx * 4 + q;
      if (cc < R) Y[(int64_t)(lo + r) * R + cc] = acc[i][q];
    }
  }
}

// Boundary sweep of all columns as one product (Sec. III: Eq. 9's t_p and s_p = C_p t_p of every
// node are linear in the leaf-stage values at the cut rows): S = K Y_cut, K = the matrix of the
// sweep (s_total x n_crow, FP32, built on the device from the sweep image and kept transposed so
// that a chunk is read and staged without bank conflicts), Y_cut = the leaf-stage rows at the
// distinct cut rows. K is block-sparse: the rows of S of a node depend only on the cut rows inside
// its subtree, so each 32-row tile of S runs over the column range of K holding its nonzeros, cut
// into pieces of 32..128 columns (the longest giving about four CTAs per SM; work item = tile,
// piece). A CTA forms the 32 x 64 product of one piece in 32-deep chunks (128 threads, a 4 x 4
// block of outputs each, from 16-byte shared-memory reads; the next chunk is loaded into registers
// while the current one is multiplied). A tile of a single piece writes S; otherwise each piece
// writes its partial to global memory and the CTA that completes the tile (an atomic count per
// tile) adds the partials in piece order, so the result does not depend on timing, and resets the
// count.
constexpr int SBM = 32, SBN = 64, SBK = 32, SBT = 128, SPIECE = 128;
__global__ void __launch_bounds__(SBT) k_mc_sweep_gemm(MSimD m, const float* __restrict__ Kt, int ldt,
                                                       const int4* __restrict__ items, float* part, int* count,
                                                       int n_ct, const int* status) {
  __shared__ __align__(16) float Ks[SBK][SBM];
  __shared__ __align__(16) float Ys[SBK][SBN];
  __shared__ int last_sh;
  if (*status != DEV_OK) return;   // uniform
  const int* M = m.meta;
  const int s_total = M[M_STOTAL];
  const int* crow_pos = M + M[M_OFF_CROW];
  const int4 it = items[blockIdx.x];   // row tile, first column of K, end column, piece | (pieces << 16)
  const int rt = it.x, kb = it.y, ke = it.z, piece = it.w & 0xffff, pieces = it.w >> 16;
  const int r0 = rt * SBM, c0 = blockIdx.y * SBN;
  if (c0 >= m.R_act) return;       // uniform
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;   // rows ty*4.., columns tx*4..
  const int64_t R = m.R;
  constexpr int KL = SBK * SBM / SBT, YL = SBK * SBN / SBT;   // 8 and 16 loads per thread
  float kreg[KL], yreg[YL];
  auto load = [&](int k0) {
#pragma unroll
    for (int u = 0; u < KL; ++u) {
      const int w = tid + u * SBT, rr = w % SBM, kk = w / SBM;   // a warp reads 32 rows of one column
      const int r = r0 + rr, k = k0 + kk;
      kreg[u] = (r < s_total && k < ke) ? Kt[(int64_t)k * ldt + r] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < YL; ++u) {
      const int w = tid + u * SBT, kk = w / SBN, cc = w % SBN;
      const int k = k0 + kk, c = c0 + cc;
      yreg[u] = (k < ke && c < m.R_act) ? m.Y[(int64_t)crow_pos[k] * R + c] : 0.f;
    }
  };
  float acc[4][4] = {};
  if (kb < ke) {
    load(kb);
    for (int k0 = kb; k0 < ke; k0 += SBK) {
#pragma unroll
      for (int u = 0; u < KL; ++u) {
        const int w = tid + u * SBT;
        Ks[w / SBM][w % SBM] = kreg[u];
      }
#pragma unroll
      for (int u = 0; u < YL; ++u) {
        const int w = tid + u * SBT;
        Ys[w / SBN][w % SBN] = yreg[u];
      }
      __syncthreads();
      if (k0 + SBK < ke) load(k0 + SBK);   // in flight during the products below
#pragma unroll 8
      for (int kk = 0; kk < SBK; ++kk) {
        const float4 a = *reinterpret_cast<const float4*>(&Ks[kk][ty * 4]);
        const float4 b = *reinterpret_cast<const float4*>(&Ys[kk][tx * 4]);
        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[i][q] = fmaf(av[i], bv[q], acc[i][q]);
      }
      __syncthreads();
    }
  }
  if (pieces == 1) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + ty * 4 + i;
      if (r >= s_total) continue;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = c0 + tx * 4 + q;
        if (c < m.R_act) m.S[(int64_t)r * R + c] = acc[i][q];
      }
    }
    return;
  }
  // partial of this piece: part[((first item of the tile + piece) * n_ct + column tile)][32 x 64]
  const int first = blockIdx.x - piece;
  float* mine = part + ((int64_t)blockIdx.x * n_ct + blockIdx.y) * (SBM * SBN);
#pragma unroll
  for (int i = 0; i < 4; ++i)
    *reinterpret_cast<float4*>(mine + (ty * 4 + i) * SBN + tx * 4) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
  __threadfence();
  __syncthreads();
  int* cnt = count + rt * n_ct + blockIdx.y;
  if (tid == 0) last_sh = atomicAdd(cnt, 1) == pieces - 1;
  __syncthreads();
  if (!last_sh) return;
  __threadfence();
  float sum[4][4] = {};
  for (int pc = 0; pc < pieces; ++pc) {
    const float* src = part + ((int64_t)(first + pc) * n_ct + blockIdx.y) * (SBM * SBN);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 v = __ldcg(reinterpret_cast<const float4*>(src + (ty * 4 + i) * SBN + tx * 4));
      sum[i][0] += v.x;
      sum[i][1] += v.y;
      sum[i][2] += v.z;
      sum[i][3] += v.w;
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + ty * 4 + i;
    if (r >= s_total) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = c0 + tx * 4 + q;
      if (c < m.R_act) m.S[(int64_t)r * R + c] = sum[i][q];
    }
  }
  if (tid == 0) *cnt = 0;   // ready for the next launch
}

// Kt[k][r] = K[r][k]
__global__ void k_mc_transpose(const float* __restrict__ K, int ldk, int s_total, int n_crow, float* Kt, int ldt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s_total * n_crow) return;
  const int k = i / s_total, r = i % s_total;
  Kt[(int64_t)k * ldt + r] = K[(int64_t)r * ldk + k];
}

// Column range [first, last + 1) of the nonzeros of K in each 32-row tile ((0, 0) if none).
__global__ void k_mc_krange(const float* __restrict__ K, int ldk, int s_total, int n_crow, int2* out) {
  __shared__ int lo_s, hi_s;
  if (threadIdx.x == 0) {
    lo_s = n_crow;
    hi_s = 0;
  }
  __syncthreads();
  const int r0 = blockIdx.x * SBM;
  int lo = n_crow, hi = 0;
  for (int idx = threadIdx.x; idx < SBM * n_crow; idx += blockDim.x) {
    const int r = r0 + idx / n_crow, k = idx % n_crow;
    if (r < s_total && K[(int64_t)r * ldk + k] != 0.f) {
      lo = min(lo, k);
      hi = max(hi, k + 1);
    }
  }
  atomicMin(&lo_s, lo);
  atomicMax(&hi_s, hi);
  __syncthreads();
  if (threadIdx.x == 0) out[blockIdx.x] = lo_s < hi_s ? make_int2(lo_s, hi_s) : make_int2(0, 0);
}

// Corrected leaf-stage value v = y - sum over ancestors of F row . S(half) at one position and
// column, with S in global memory.
__device__ __forceinline__ float corrected_g(const DStore& st, const MSimD& m, int pos, int c) {
  const int64_t R = m.R;
  float v = m.Y[pos * R + c];
  for (int q = st.parent[st.leaf_node[st.pos_leaf[pos]]]; q >= 0; q = st.parent[q]) {
    const int k = st.node_k[q];
    const int half = pos < st.hi[st.left[q]] ? 0 : k;
    const float* Fr = st.F32 + st.node_foff[q] + (int64_t)(pos - st.lo[q]) * st.node_kld[q];
    const float* Sq = m.S + (int64_t)(st.node_soff[q] + half) * R + c;
    for (int e = 0; e < k; ++e) v = fmaf(-Fr[e], Sq[e * R], v);
  }
  return v;
}

// N-1 factor of each column whose change is switched on: f_c = (delta_c / d_c) (v_a - v_b) from
// the FP32 apply before the column's own Sherman-Morrison term (zero for the others).
__global__ void k_mc_fcol(DStore st, MSimD m, int s_in_chunk, const int* status) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.R_act || *status != DEV_OK) return;
  const int step = m.dyn->step_base + s_in_chunk + 1;
  float f = 0.f;
  if (change_on(m, c, step)) {
    const float ya = corrected_g(st, m, m.trip_a[c], c);
    const float yb = m.trip_b[c] >= 0 ? corrected_g(st, m, m.trip_b[c], c) : 0.f;
    f = (float)m.trip_coef[c] * (ya - yb);
  }
  m.fcol[c] = f;
}

// Expansion with Eq. 9's factors (+ the N-1 Sherman-Morrison correction of Sec. IV) as a tiled
// product per leaf: for a tile of up to 32 positions of
// one leaf and 128 columns, V = Y - F_path S_path, where F_path holds the tile's factor rows of all
// its ancestors (the same ancestors and halves for every position of a leaf) and S_path the
// matching rows of S. Path elements are taken in chunks of 16: the S chunk (16 x 128) and the F
// chunk (16 x 32, element-major) go to shared memory, and each of 256 threads forms a 4 x 4 block
// of outputs (4 positions x 4 columns) from 16-byte reads; the next chunk is loaded into registers
// while the current one is multiplied. pass 0: V = result; pass 1: V += result and the monitored
// record.
constexpr int XP = 32, XC = 128, XE = 16, XT = 256;
__global__ void __launch_bounds__(XT) k_mc_expand_tiled(DStore st, MSimD m, const int4* __restrict__ tiles,
                                                        const int* __restrict__ path_ptr,
                                                        const int* __restrict__ path_srow,
                                                        const long long* __restrict__ path_fbase,
                                                        const int* __restrict__ path_kld, int pass, int n1, int record,
                                                        int s_in_chunk, const int* status) {
  __shared__ __align__(16) float Ss[XE][XC];
  __shared__ __align__(16) float Fs[XE][XP];
  if (*status != DEV_OK) return;
  const int4 tl = tiles[blockIdx.x];   // leaf, first position, positions, unused
  const int j = tl.x, p0 = tl.y, cnt = tl.z;
  const int c0 = blockIdx.y * XC;
  if (c0 >= m.R_act) return;
  const int tid = threadIdx.x, ty = tid / 32, tx = tid % 32;   // positions ty*4.., columns tx*4..
  const int64_t R = m.R;
  const int e0 = path_ptr[j], ne = path_ptr[j + 1] - e0;
  constexpr int SL = XE * XC / XT, FL = XE * XP / XT;   // 8 and 2 loads per thread
  float sr[SL], fr[FL];
  auto load = [&](int eb) {
#pragma unroll
    for (int u = 0; u < SL; ++u) {
      const int w = tid + u * XT, e = w / XC, cc = w % XC;
      sr[u] = (eb + e < ne && c0 + cc < m.R_act) ? m.S[(int64_t)path_srow[e0 + eb + e] * R + c0 + cc] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < FL; ++u) {
      const int w = tid + u * XT, e = w / XP, p = w % XP;
      float f = 0.f;
      if (p < cnt && eb + e < ne) {
        const int ix = e0 + eb + e;
        f = st.F32[path_fbase[ix] + (int64_t)(p0 + p) * path_kld[ix]];
      }
      fr[u] = f;
    }
  };
  float acc[4][4] = {};
  if (ne > 0) load(0);
  for (int eb = 0; eb < ne; eb += XE) {
#pragma unroll
    for (int u = 0; u < SL; ++u) {
      const int w = tid + u * XT;
      Ss[w / XC][w % XC] = sr[u];
    }
#pragma unroll
    for (int u = 0; u < FL; ++u) {
      const int w = tid + u * XT;
      Fs[w / XP][w % XP] = fr[u];
    }
    __syncthreads();
    if (eb + XE < ne) load(eb + XE);   // in flight during the products below
#pragma unroll
    for (int e = 0; e < XE; ++e) {
      const float4 f = *reinterpret_cast<const float4*>(&Fs[e][ty * 4]);
      const float4 sv = *reinterpret_cast<const float4*>(&Ss[e][tx * 4]);
      const float fv[4] = {f.x, f.y, f.z, f.w}, svv[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = fmaf(fv[i], svv[q], acc[i][q]);
    }
    __syncthreads();
  }
  const int step = m.dyn->step_base + s_in_chunk + 1;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = c0 + tx * 4 + q;
    if (c >= m.R_act) continue;
    const float fc = n1 ? m.fcol[c] : 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int p = ty * 4 + i;
      if (p >= cnt) continue;
      const int pos = p0 + p;
      float v = m.Y[pos * R + c] - acc[i][q];
      if (fc != 0.f) v = fmaf(-fc, m.Z[pos * R + c].x, v);
      const float2 out = pass == 0 ? ff_f(v) : ff_addx(m.V[pos * R + c], ff_f(v));
      m.V[pos * R + c] = out;
      if (record && m.dyn->rec) {
        const int mi = m.mon_idx[pos];
        if (mi >= 0)
          m.dyn->rec[((int64_t)(step - m.dyn->rec_first) * R + c) * m.n_mon + mi] = (double)out.x + (double)out.y;
      }
    }
  }
}

// r = x - G' v (float-float; Eq. 1's G with each column's own change of Sec. IV), stored as the
// FP32 input of the correction apply. Same shape as the
// injection: `ipp` positions x 256 columns per CTA, the CSR rows of its positions staged in shared
// memory, then one round trip per position (up to RKB entries per batch).
constexpr int RKB = 5;   // CSR entries per batch: rows hold about 4-5 entries (measured: 8 45.2 us, 5 38.5 us)
__global__ void __launch_bounds__(ITH) k_mc_residual(MSimD m, int ipp, int n1, int s_in_chunk, const int* status) {
  extern __shared__ __align__(16) unsigned char rsm[];
  __shared__ int sptr[IPP_MAX + 1];
  if (*status != DEV_OK) return;   // uniform, before any barrier
  const int p0 = blockIdx.x * ipp, np = min(ipp, m.n - p0);
  const int tid = threadIdx.x, c = blockIdx.y * ITH + tid;
  if (tid <= np) sptr[tid] = m.csr_ptr[p0 + tid];
  __syncthreads();
  const int r0 = sptr[0], nnz = sptr[np] - r0;
  float2* sval = reinterpret_cast<float2*>(rsm);
  int* scol = reinterpret_cast<int*>(rsm + (size_t)nnz * sizeof(float2));
  for (int i = tid; i < nnz; i += ITH) {
    sval[i] = m.csr_ff[r0 + i];
    scol[i] = m.csr_col[r0 + i];
  }
  __syncthreads();
  if (c >= m.R_act) return;
  const int64_t R = m.R;
  const int R32 = m.R;   // n R < 2^31 (checked at creation): 32-bit element offsets
  const int step = m.dyn->step_base + s_in_chunk + 1;
  const bool on = n1 && change_on(m, c, step);
  const float2* Vc = m.V + c;
  for (int pi = 0; pi < np; ++pi) {
    const int pos = p0 + pi;
    const int k1 = sptr[pi + 1] - r0;
    int kb = sptr[pi] - r0;
    Acc2 ra = acc2(m.X[pos * R32 + c]);
    while (kb < k1) {
      float2 v[RKB];
#pragma unroll
      for (int q = 0; q < RKB; ++q)
        if (kb + q < k1) v[q] = Vc[scol[kb + q] * R32];
#pragma unroll
      for (int q = 0; q < RKB; ++q) {
        if (kb + q >= k1) break;
        ra.add_prod(ff_negx(sval[kb + q]), v[q]);
      }
      kb += RKB;
    }
    float2 r = ra.get();
    if (on) {
      const int a = m.trip_a[c], b = m.trip_b[c];
      if (pos == a || pos == b) {
        // (G' v)_i = (G v)_i + delta u_i (v_a - v_b)
        float2 du = m.V[(int64_t)a * R + c];
        if (b >= 0) du = ff_subx(du, m.V[(int64_t)b * R + c]);
        const float2 dl = ff_mulx(m.trip_delta_ff[c], du);
        r = pos == a ? ff_subx(r, dl) : ff_addx(r, dl);
      }
    }
    m.Xf[pos * R32 + c] = r.x;
  }
}

// The residual with two adjacent columns per thread (even column stride, 32-bit offsets): each
// CSR entry is read from shared memory once for both columns and the two columns' voltages come in
// one 16-byte load. Same arithmetic per column as k_mc_residual, so the results agree bit for bit.
__global__ void __launch_bounds__(ITH) k_mc_residual2(MSimD m, int ipp, int n1, int s_in_chunk, const int* status) {
  extern __shared__ __align__(16) unsigned char rsm[];
  __shared__ int sptr[IPP_MAX + 1];
  if (*status != DEV_OK) return;   // uniform, before any barrier
  const int p0 = blockIdx.x * ipp, np = min(ipp, m.n - p0);
  const int tid = threadIdx.x, c = 2 * (blockIdx.y * ITH + tid);
  if (tid <= np) sptr[tid] = m.csr_ptr[p0 + tid];
  __syncthreads();
  const int r0 = sptr[0], nnz = sptr[np] - r0;
  float2* sval = reinterpret_cast<float2*>(rsm);
  int* scol = reinterpret_cast<int*>(rsm + (size_t)nnz * sizeof(float2));
  for (int i = tid; i < nnz; i += ITH) {
    sval[i] = m.csr_ff[r0 + i];
    scol[i] = m.csr_col[r0 + i];
  }
  __syncthreads();
  if (c >= m.R_act) return;
  const bool both = c + 1 < m.R_act;   // column c + 1 < R exists (R even) even when it is not in use
  const int R32 = m.R;
  const int step = m.dyn->step_base + s_in_chunk + 1;
  const bool on[2] = {n1 && change_on(m, c, step), both && n1 && change_on(m, c + 1, step)};
  const float2* Vc = m.V + c;
  for (int pi = 0; pi < np; ++pi) {
    const int pos = p0 + pi;
    const int k1 = sptr[pi + 1] - r0;
    int kb = sptr[pi] - r0;
    float2 xv[2];
    ld_pair(m.X + pos * R32 + c, xv);
    Acc2 ra[2] = {acc2(xv[0]), acc2(xv[1])};
    while (kb < k1) {
      float2 v[RKB][2];
#pragma unroll
      for (int q = 0; q < RKB; ++q)
        if (kb + q < k1) ld_pair(Vc + scol[kb + q] * R32, v[q]);
#pragma unroll
      for (int q = 0; q < RKB; ++q) {
        if (kb + q >= k1) break;
        const float2 g = ff_negx(sval[kb + q]);
        ra[0].add_prod(g, v[q][0]);
        ra[1].add_prod(g, v[q][1]);
      }
      kb += RKB;
    }
    float2 r[2] = {ra[0].get(), ra[1].get()};
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (!on[j]) continue;
      const int cj = c + j;
      const int a = m.trip_a[cj], b = m.trip_b[cj];
      if (pos == a || pos == b) {
        // (G' v)_i = (G v)_i + delta u_i (v_a - v_b)
        float2 du = m.V[(int64_t)a * R32 + cj];
        if (b >= 0) du = ff_subx(du, m.V[(int64_t)b * R32 + cj]);
        const float2 dl = ff_mulx(m.trip_delta_ff[cj], du);
        r[j] = pos == a ? ff_subx(r[j], dl) : ff_addx(r[j], dl);
      }
    }
    if (both) *reinterpret_cast<float2*>(m.Xf + pos * R32 + c) = make_float2(r[0].x, r[1].x);
    else m.Xf[pos * R32 + c] = r[0].x;
  }
}

// d_c = 1 + delta_c u_c^T z_c (FP64) and the Sherman-Morrison factor delta_c / d_c (Sec. IV)
__global__ void k_mc_trip_coef(MSimD m, double* coef, int* status) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.R) return;
  if (m.trip_step[c] <= 0) {
    coef[c] = 0.0;
    return;
  }
  const int64_t R = m.R;
  const float2 za = m.Z[(int64_t)m.trip_a[c] * R + c];
  double ut = (double)za.x + (double)za.y;
  if (m.trip_b[c] >= 0) {
    const float2 zb = m.Z[(int64_t)m.trip_b[c] * R + c];
    ut -= (double)zb.x + (double)zb.y;
  }
  const double d = 1.0 + m.trip_delta[c] * ut;
  if (!(d > 1e-12)) atomicExch(status, DEV_SINGULAR);
  coef[c] = m.trip_delta[c] / d;
}

// Right-hand sides u_c = e_a - e_b (or e_a) of the columns' changes, for z_c = G^{-1} u_c (Sec. IV).
__global__ void k_mc_unit(MSimD m, float2* X, float* Xf) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.R || m.trip_step[c] <= 0) return;
  const int64_t R = m.R;
  X[(int64_t)m.trip_a[c] * R + c] = ff_f(1.f);
  Xf[(int64_t)m.trip_a[c] * R + c] = 1.f;
  if (m.trip_b[c] >= 0) {
    X[(int64_t)m.trip_b[c] * R + c] = ff_f(-1.f);
    Xf[(int64_t)m.trip_b[c] * R + c] = -1.f;
  }
}

// Start column c afresh: zero its voltages, history and right-hand side.
__global__ void k_mc_reset_col(MSimD m, int n_rows, int c) {
  const int64_t R = m.R;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_rows; i += gridDim.x * blockDim.x) {
    if (i < 2 * m.n_el) m.Ih[i * R + c] = ff_f(0.f);
    if (i < m.n) {
      m.V[i * R + c] = ff_f(0.f);
      m.X[i * R + c] = ff_f(0.f);
      m.Xf[i * R + c] = 0.f;
    }
  }
}

// Source/load coefficients of column c for a start S = w t0 (local time t - t0):
// cs' = cs cos S + sn sin S, sn' = sn cos S - cs sin S.
__global__ void k_mc_rotate_terms(MSimD m, const double* __restrict__ base, float2* cs, float2* sn, int n_terms, int c,
                                  double cosS, double sinS) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_terms) return;
  const double a = base[2 * t], b = base[2 * t + 1];
  const double x = a * cosS + b * sinS, y = b * cosS - a * sinS;
  const float xh = (float)x, yh = (float)y;
  cs[(int64_t)t * m.R + c] = make_float2(xh, (float)(x - (double)xh));
  sn[(int64_t)t * m.R + c] = make_float2(yh, (float)(y - (double)yh));
}

// Source and load coefficient tables [term][column]: (coef * scale) * cos phi and (coef * scale) *
// sin phi as float-float pairs (leading part the FP32 rounding, then the rounded remainder), with
// scale = src_scale[c][idx] or load_scale[c][idx] (1 without scales); ki >= 0 names a source,
// ki < 0 the load -(ki + 1).
__global__ void k_mc_terms(const double* __restrict__ coef, const double* __restrict__ cph,
                           const double* __restrict__ sph, const int* __restrict__ ki,
                           const double* __restrict__ src_scale, const double* __restrict__ load_scale, int n_src,
                           int n_load, int n_terms, int R, float2* __restrict__ cs, float2* __restrict__ sn) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n_terms * R) return;
  const int t = (int)(i / R), c = (int)(i % R);
  const int k = ki[t];
  double sc = 1.0;
  if (k >= 0) {
    if (src_scale) sc = src_scale[(size_t)c * n_src + k];
  } else if (load_scale) {
    sc = load_scale[(size_t)c * n_load + (-k - 1)];
  }
  const double a = coef[t] * sc;
  const double x = a * cph[t], y = a * sph[t];
  const float xh = __double2float_rn(x), yh = __double2float_rn(y);
  cs[i] = make_float2(xh, __double2float_rn(x - (double)xh));
  sn[i] = make_float2(yh, __double2float_rn(y - (double)yh));
}

// z_c of column c (its change's G^{-1} u_c, Sec. IV) as float-float.
__global__ void k_mc_set_z(MSimD m, float2* Z, const double* __restrict__ zpos, int c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.n) return;
  const double v = zpos[i];
  const float h = (float)v;
  Z[(int64_t)i * m.R + c] = make_float2(h, (float)(v - (double)h));
}

// d_c and delta_c / d_c of one column (Sec. IV), when a column starts afresh.
__global__ void k_mc_one_coef(MSimD m, double* coef, int c, int* status) {
  const int64_t R = m.R;
  const float2 za = m.Z[(int64_t)m.trip_a[c] * R + c];
  double ut = (double)za.x + (double)za.y;
  if (m.trip_b[c] >= 0) {
    const float2 zb = m.Z[(int64_t)m.trip_b[c] * R + c];
    ut -= (double)zb.x + (double)zb.y;
  }
  const double d = 1.0 + m.trip_delta[c] * ut;
  if (!(d > 1e-12)) atomicExch(status, DEV_SINGULAR);
  coef[c] = m.trip_delta[c] / d;
}

__global__ void k_mc_set_event(int* on, int* off, int* elem, int* ta, int* tb, double* td, float2* tdf, int c, int v_on,
                               int v_off, int v_elem, int v_a, int v_b, double v_d) {
  on[c] = v_on;
  off[c] = v_off;
  elem[c] = v_elem;
  ta[c] = v_a;
  tb[c] = v_b;
  td[c] = v_d;
  const float h = (float)v_d;
  tdf[c] = make_float2(h, (float)(v_d - (double)h));
}

__global__ void k_mc_advance(SimDyn* dyn, int n) { dyn->step_base += n; }
__global__ void k_mc_set_dyn(SimDyn* dyn, int step_base, int rec_first, double* rec) {
  dyn->step_base = step_base;
  dyn->rec_first = rec_first;
  dyn->rec = rec;
  dyn->trig_first = rec_first;
}

}  // namespace

// ====================================================================== host side
MSimD MSim::view() const {
  MSimD d{};
  d.n = n;
  d.R = R;
  d.s_total = store->s_total;
  d.n_crow = n_crow;
  d.max_depth = store->tree.max_depth;
  d.inc = inc.p;
  d.inc_ptr = inc_ptr.p;
  d.Ih = Ih.p;
  d.n_el = n_el_h;
  d.V = V.p;
  d.X = X.p;
  d.Xf = Xf.p;
  d.Y = Y.p;
  d.S = S.p;
  d.fcol = fcol.p;
  d.term_ptr = term_ptr.p;
  d.term_cs = term_cs.p;
  d.term_sn = term_sn.p;
  d.trig = trig.p;
  d.trip_step = trip_step.p;
  d.trip_off = trip_off.p;
  d.R_act = R_act;
  d.trip_elem = trip_elem.p;
  d.trip_a = trip_a.p;
  d.trip_b = trip_b.p;
  d.trip_delta = trip_delta.p;
  d.trip_delta_ff = trip_dff.p;
  d.trip_coef = trip_coef.p;
  d.Z = Z.p;
  d.csr_ptr = store->d_csr_ptr.p;
  d.csr_col = store->d_csr_col.p;
  d.csr_ff = csr_ff.p;
  d.mon_idx = mon_idx.p;
  d.n_mon = n_mon;
  d.dyn = d_dyn.p;
  d.meta = meta.p;
  return d;
}

MSim::MSim(const emt_network* net, const emt_hinv_opts* opts, double dt_, int R_, const double* src_scale,
           const double* load_scale, cudaStream_t s) {
  EMT_REQUIRE(net && opts, EMT_ERR_INVALID, "null network or options");
  check_network_arrays(net);
  EMT_REQUIRE(dt_ > 0 && std::isfinite(dt_), EMT_ERR_INVALID, "dt must be > 0");
  EMT_REQUIRE(R_ >= 2 && R_ <= 65536, EMT_ERR_INVALID, "nrhs out of range");
  EMT_REQUIRE(opts->nodes_per_bus <= 1, EMT_ERR_UNSUPPORTED,
              "single-phase simulations partition buses one by one (nodes_per_bus 0 or 1)");
  EMT_REQUIRE((int64_t)(net->n_bus + 1) * R_ < ((int64_t)1 << 31), EMT_ERR_UNSUPPORTED,
              "n_bus x nrhs must stay below 2^31 (32-bit element offsets of the residual)");
  n = net->n_bus;
  R = R_;
  dt = dt_;
  omega = 2.0 * M_PI * net->freq;
  const int nb = net->n_branch;
  std::vector<double> el_al, el_be;
  for (int e = 0; e < nb; ++e) {
    const int a = net->from[e], b = net->to[e];
    EMT_REQUIRE(a >= 0 && a < n && b >= 0 && b < n && a != b, EMT_ERR_INVALID, "series branch endpoints");
    const double Rr = net->R[e];
    double g, al, be;
    if (net->kind[e] == EMT_KIND_RL) {
      const double x = 2.0 * net->L[e] / dt;
      g = 1.0 / (Rr + x);
      al = g;
      be = g * (x - Rr);
    } else {
      EMT_REQUIRE(net->kind[e] == EMT_KIND_RC && net->C[e] > 0, EMT_ERR_INVALID, "bad RC branch");
      const double x = dt / (2.0 * net->C[e]);
      g = 1.0 / (Rr + x);
      al = -g;
      be = -g * (x - Rr);
    }
    EMT_REQUIRE(std::isfinite(g) && g > 0, EMT_ERR_INVALID, "branch companion conductance must be > 0");
    el_a.push_back(a);
    el_b.push_back(b);
    el_g.push_back(g);
    el_al.push_back(al);
    el_be.push_back(be);
  }
  n_series = nb;
  if (net->shunt_C)
    for (int i = 0; i < n; ++i) {
      const double C = net->shunt_C[i];
      if (!(C > 0)) continue;
      const double g = 2.0 * C / dt;
      el_a.push_back(i);
      el_b.push_back(-1);
      el_g.push_back(g);
      el_al.push_back(-g);
      el_be.push_back(-1.0);
    }
  std::vector<int32_t> gf(el_a.begin(), el_a.end()), gt(el_b.begin(), el_b.end());
  std::vector<double> gv(el_g.begin(), el_g.end());
  for (int k = 0; k < net->n_src; ++k) {
    EMT_REQUIRE(net->src_bus[k] >= 0 && net->src_bus[k] < n && net->src_Rs[k] > 0, EMT_ERR_INVALID, "bad source");
    gf.push_back(net->src_bus[k]);
    gt.push_back(-1);
    gv.push_back(1.0 / net->src_Rs[k]);
  }
  emt_graph gr{n, (int32_t)gf.size(), gf.data(), gt.data(), gv.data()};
  emt_hinv_opts o = *opts;
  o.precision = EMT_PREC_FP32;
  store.reset(new Store(&gr, &o, s));
  store->build(s);
  const Tree& t = store->tree;
  // element ends by position
  std::vector<std::vector<int>> at(n);
  for (size_t e = 0; e < el_a.size(); ++e) {
    at[t.pos[el_a[e]]].push_back((int)e);
    if (el_b[e] >= 0) at[t.pos[el_b[e]]].push_back((int)e);
  }
  std::vector<int> iptr(n + 1, 0);
  std::vector<MRec> recs;
  for (int p = 0; p < n; ++p) {
    for (int e : at[p]) {
      MRec r{};
      const bool is_a = t.pos[el_a[e]] == p;
      r.other = is_a ? (el_b[e] >= 0 ? t.pos[el_b[e]] : -1) : t.pos[el_a[e]];
      r.sgn = is_a ? 1 : -1;
      r.elem = (int)e;
      // Ih' = alpha v + beta (g v + Ih) = (alpha + beta g) v + beta Ih
      r.a1 = host_ff(el_al[e] + el_be[e] * el_g[e]);
      r.beta = host_ff(el_be[e]);
      recs.push_back(r);
    }
    iptr[p + 1] = (int)recs.size();
  }
  n_inc = (int)recs.size();
  n_el_h = (int)el_a.size();
  {
    // shared memory of the injection / residual CTAs: the most records (CSR entries) of any
    // aligned window of IPP_MAX positions (windows of 1, 2, 4 positions nest inside them)
    const auto& cp = store->csr_ptr;
    int mi = 0, mc = 0;
    for (int p = 0; p < n; p += IPP_MAX) {
      const int q = std::min(n, p + IPP_MAX);
      mi = std::max(mi, iptr[q] - iptr[p]);
      mc = std::max(mc, cp[q] - cp[p]);
    }
    inj_smem = (size_t)mi * sizeof(MRec);
    res_smem = (size_t)mc * (sizeof(float2) + sizeof(int));
    EMT_REQUIRE(inj_smem <= 160 * 1024 && res_smem <= 160 * 1024, EMT_ERR_UNSUPPORTED,
                "too many element ends on 8 consecutive buses");
    if (inj_smem > 48 * 1024) {
      EMT_CUDA(cudaFuncSetAttribute(k_mc_inject, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)inj_smem));
      EMT_CUDA(cudaFuncSetAttribute(k_mc_inject2<6, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)inj_smem));
      EMT_CUDA(cudaFuncSetAttribute(k_mc_inject2<3, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)inj_smem));
      EMT_CUDA(cudaFuncSetAttribute(k_mc_inject2<2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)inj_smem));
    }

    if (res_smem > 48 * 1024) {
      EMT_CUDA(cudaFuncSetAttribute(k_mc_residual, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)res_smem));
      EMT_CUDA(cudaFuncSetAttribute(k_mc_residual2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)res_smem));
    }
    int dev = 0;
    EMT_CUDA(cudaGetDevice(&dev));
    EMT_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  }
  inc.upload(recs, s);
  inc_ptr.upload(iptr, s);
  // source and load terms with per-column scales
  struct Term {
    int pos;
    double coef, phi;
    int kind, idx;   // kind 0 source (idx into src arrays), 1 load
  };
  std::vector<std::vector<Term>> terms(n);
  for (int k = 0; k < net->n_src; ++k)
    terms[t.pos[net->src_bus[k]]].push_back({0, net->src_Vm[k] / net->src_Rs[k], net->src_phi[k], 0, k});
  for (int k = 0; k < net->n_load; ++k) {
    EMT_REQUIRE(net->load_bus[k] >= 0 && net->load_bus[k] < n, EMT_ERR_INVALID, "bad load bus");
    terms[t.pos[net->load_bus[k]]].push_back({0, -net->load_amp[k], net->load_phi[k], 1, k});
  }
  // per-term constants on the host; the [term][column] coefficient tables (coef * scale * cos phi,
  // coef * scale * sin phi as float-float pairs) are formed on the device from the scale arrays
  std::vector<int> tptr(n + 1, 0), t_ki;   // t_ki: source index, or -(load index + 1)
  std::vector<double> t_coef, t_cph, t_sph, tb;
  for (int p = 0; p < n; ++p) {
    for (auto& tm : terms[p]) {
      t_coef.push_back(tm.coef);
      t_cph.push_back(std::cos(tm.phi));
      t_sph.push_back(std::sin(tm.phi));
      t_ki.push_back(tm.kind == 0 ? tm.idx : -(tm.idx + 1));
      tb.push_back(tm.coef * std::cos(tm.phi));
      tb.push_back(tm.coef * std::sin(tm.phi));
    }
    tptr[p + 1] = tptr[p] + (int)terms[p].size();
  }
  const int n_terms = (int)t_coef.size();
  if (tb.empty()) tb.assign(2, 0.0);
  term_base.upload(tb, s);
  term_ptr.upload(tptr, s);
  term_cs.alloc(std::max<size_t>((size_t)n_terms * R, 1));
  term_sn.alloc(std::max<size_t>((size_t)n_terms * R, 1));
  if (n_terms > 0) {
    DevBuf<double> d_coef, d_cph, d_sph, d_ss, d_ls;
    DevBuf<int> d_ki;
    d_coef.upload(t_coef, s);
    d_cph.upload(t_cph, s);
    d_sph.upload(t_sph, s);
    d_ki.upload(t_ki, s);
    if (src_scale && net->n_src > 0) {
      d_ss.alloc((size_t)R * net->n_src);
      EMT_CUDA(cudaMemcpyAsync(d_ss.p, src_scale, d_ss.n * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    if (load_scale && net->n_load > 0) {
      d_ls.alloc((size_t)R * net->n_load);
      EMT_CUDA(cudaMemcpyAsync(d_ls.p, load_scale, d_ls.n * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    const int64_t tot = (int64_t)n_terms * R;
    k_mc_terms<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(d_coef.p, d_cph.p, d_sph.p, d_ki.p, d_ss.p, d_ls.p,
                                                             net->n_src, net->n_load, n_terms, R, term_cs.p,
                                                             term_sn.p);
    EMT_CUDA(cudaGetLastError());
    EMT_CUDA(cudaStreamSynchronize(s));   // the temporaries are freed on return
  } else {
    EMT_CUDA(cudaMemsetAsync(term_cs.p, 0, sizeof(float2), s));
    EMT_CUDA(cudaMemsetAsync(term_sn.p, 0, sizeof(float2), s));
  }
  {
    // the two-column injection indexes rows with 32-bit products (R even, every row * R < 2^31)
    const int64_t rows = std::max<int64_t>({(int64_t)2 * n_el_h, (int64_t)n, (int64_t)n_terms});
    inj_pairs = (R % 2) == 0 && (rows + 1) * R < ((int64_t)1 << 31);
  }
  std::vector<float2> cff(store->csr_val.size());
  for (size_t k = 0; k < cff.size(); ++k) cff[k] = host_ff(store->csr_val[k]);
  csr_ff.upload(cff, s);
  // state
  const size_t nR = (size_t)n * R;
  Ih.alloc((size_t)2 * std::max(n_el_h, 1) * R);
  V.alloc(nR);
  X.alloc(nR);
  Xf.alloc(nR);
  Y.alloc(nR);
  Z.alloc(nR);
  S.alloc((size_t)std::max(store->s_total, 1) * R);
  fcol.alloc(R);
  // no column has a change yet: zero factors (read by the change terms of a pass with n1 = 1,
  // e.g. the expansion timed alone) must not pick up stale device memory
  Z.zero(s);
  fcol.zero(s);
  h_trip_step.assign(R, 0);
  h_trip_elem.assign(R, -1);
  trip_step.upload(h_trip_step, s);
  trip_elem.upload(h_trip_elem, s);
  h_trip_off.assign(R, 0x7fffffff);
  trip_off.upload(h_trip_off, s);
  R_act = R;
  trip_a.upload(std::vector<int>(R, 0), s);
  trip_b.upload(std::vector<int>(R, -1), s);
  trip_delta.upload(std::vector<double>(R, 0.0), s);
  trip_dff.upload(std::vector<float2>(R, make_float2(0.f, 0.f)), s);
  trip_coef.upload(std::vector<double>(R, 0.0), s);
  mon_idx.upload(std::vector<int>(n, -1), s);
  d_dyn.alloc(1);
  EMT_CUDA(cudaMemsetAsync(d_dyn.p, 0, sizeof(SimDyn), s));
  build_meta(s);
  if ((R & 3) == 0 && R >= 32) {
    umma.build(*store, R, s);
    umma.build_expand(*store, path_ptr_h, path_ptr.p, path_fbase.p, path_kld.p, s);
  }
  reset(s);
  EMT_CUDA(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
  EMT_CUDA(cudaStreamSynchronize(s));
  EMT_REQUIRE(store->device_status(s) == DEV_OK, EMT_ERR_SINGULAR, "G is not positive definite");
  apply_cached_tuning(s);
}

MSim::~MSim() {
  drop_graphs();
  if (cap_stream) cudaStreamDestroy(cap_stream);
}

void MSim::drop_graphs() {
  for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
  graphs.clear();
}

void MSim::build_meta(cudaStream_t s) {
  const Store& st = *store;
  const Tree& t = st.tree;
  const CutRows& cr = st.cut_rows;
  std::vector<int> M(M_HEADER, 0);
  n_crow = (int)cr.crow_pos.size();
  M[M_NCROW] = n_crow;
  M[M_NITEMS] = cr.n_items;
  M[M_STOTAL] = st.s_total;
  M[M_MAXD] = t.max_depth;
  M[M_OFF_CROW] = (int)M.size();
  for (int p : cr.crow_pos) M.push_back(p);
  std::vector<int> order(cr.n_items);
  for (int i = 0; i < cr.n_items; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return t.depth[cr.item_node[x]] < t.depth[cr.item_node[y]]; });
  M[M_OFF_LVL_ITEM] = (int)M.size();
  {
    std::vector<int> lvl(t.max_depth + 2, 0);
    for (int i = 0; i < cr.n_items; ++i) lvl[t.depth[cr.item_node[i]] + 1]++;
    for (int d = 0; d <= t.max_depth; ++d) lvl[d + 1] += lvl[d];
    for (int v : lvl) M.push_back(v);
  }
  M[M_OFF_ITEM] = (int)M.size();
  const size_t item_base = M.size();
  M.resize(M.size() + 5 * (size_t)cr.n_items);
  std::vector<int> segs;
  for (int w = 0; w < cr.n_items; ++w) {
    const int it = order[w];
    const int q = cr.item_node[it];
    const int d = t.depth[q];
    const int ps = cr.item_pos[it];
    const int k = st.node_k_h[q];
    const int slot = cr.item_sidx[it] - st.node_soff_h[q];
    int* rec = &M[item_base + 5 * w];
    rec[0] = cr.item_crow[it];
    rec[1] = cr.item_sidx[it];
    rec[2] = slot < k ? t.cut_ptr[q] + slot : -1;
    rec[3] = (int)segs.size() / 3;
    int nseg = 0;
    for (int a = t.parent[st.leaf_nodes_h[leaf_index_of_pos(st, ps)]]; a >= 0 && t.depth[a] > d; a = t.parent[a]) {
      const int ka = st.node_k_h[a];
      if (ka == 0) continue;
      segs.push_back(st.node_soff_h[a] + (ps < t.hi[t.left[a]] ? 0 : ka));
      segs.push_back(ka);
      segs.push_back((int)(st.node_foff_h[a] + (int64_t)(ps - t.lo[a]) * st.node_kld_h[a]));
      ++nseg;
    }
    rec[4] = nseg;
  }
  M[M_OFF_SEG] = (int)M.size();
  for (int v : segs) M.push_back(v);
  M[M_OFF_LVL_CORE] = (int)M.size();
  {
    std::vector<int> lvl(t.max_depth + 2, 0);
    for (int q : st.lvl_nodes_h) lvl[t.depth[q] + 1] += 2 * st.node_k_h[q];
    for (int d = 0; d <= t.max_depth; ++d) lvl[d + 1] += lvl[d];
    for (int v : lvl) M.push_back(v);
  }
  M[M_OFF_CORE] = (int)M.size();
  for (int q : st.lvl_nodes_h) {
    const int m2 = 2 * st.node_k_h[q];
    for (int r = 0; r < m2; ++r) {
      M.push_back(st.node_soff_h[q] + r);
      M.push_back(st.node_soff_h[q]);
      M.push_back(m2);
      M.push_back((int)(st.node_coff_h[q] + (int64_t)r * m2));
    }
  }
  meta.upload(M, s);
  // GEMM tiles over (leaf, row block, column block)
  std::vector<int4> tiles;
  for (int j = 0; j < st.n_leaf; ++j) {
    const int b = t.hi[st.leaf_nodes_h[j]] - t.lo[st.leaf_nodes_h[j]];
    for (int m0 = 0; m0 < b; m0 += GBM)
      for (int n0 = 0; n0 < R; n0 += GBN) tiles.push_back(make_int4(j, m0, n0, 0));
  }
  n_tiles = (int)tiles.size();
  gemm_tiles.alloc(tiles.size() * 4);
  EMT_CUDA(cudaMemcpyAsync(gemm_tiles.p, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
  // column block of the sweep: as many columns as shared memory allows (<= 32)
  // matrix of the sweep (FP32): S = K Y_cut
  {
    ImgHeader hdr{};
    DevBuf<double> img;
    DevBuf<int> sg_src, sg_dst, sg_len;
    int n_sg = 0;
    build_sweep_image(st, nullptr, EMT_PREC_FP32, hdr, img, sg_src, sg_dst, sg_len, n_sg, s);
    ldk = (n_crow + 1) / 2 * 2;
    Kmat.alloc(std::max<size_t>((size_t)st.s_total * ldk, 1));
    EMT_CUDA(cudaMemsetAsync(Kmat.p, 0, Kmat.n * sizeof(float), s));
    build_sweep_matrix(EMT_PREC_FP32, reinterpret_cast<const unsigned char*>(img.p), hdr.img_bytes,
                       reinterpret_cast<const unsigned char*>(st.C32.p), (int)(st.C_elems * 4), n_crow, st.s_total,
                       ldk, Kmat.p, s);
    const int n_rt = std::max(1, (st.s_total + SBM - 1) / SBM);
    krange.alloc(n_rt);
    EMT_CUDA(cudaMemsetAsync(krange.p, 0, n_rt * sizeof(int2), s));
    if (st.s_total > 0 && n_crow > 0) k_mc_krange<<<n_rt, 256, 0, s>>>(Kmat.p, ldk, st.s_total, n_crow, krange.p);
    ldt = (st.s_total + 3) / 4 * 4;
    Kt.alloc(std::max<size_t>((size_t)n_crow * ldt, 1));
    EMT_CUDA(cudaMemsetAsync(Kt.p, 0, Kt.n * sizeof(float), s));
    if (st.s_total > 0 && n_crow > 0)
      k_mc_transpose<<<(st.s_total * n_crow + 255) / 256, 256, 0, s>>>(Kmat.p, ldk, st.s_total, n_crow, Kt.p, ldt);
    // work items of the sweep product: every row tile's nonzero column range in pieces of at most
    // SPIECE columns (whole SBK chunks)
    std::vector<int2> kr(n_rt);
    EMT_CUDA(cudaMemcpyAsync(kr.data(), krange.p, n_rt * sizeof(int2), cudaMemcpyDeviceToHost, s));
    EMT_CUDA(cudaStreamSynchronize(s));
    n_ct = (R + SBN - 1) / SBN;
    int dev = 0, n_sms = 1;
    EMT_CUDA(cudaGetDevice(&dev));
    EMT_CUDA(cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev));
    std::vector<int4> items;
    // the longest piece (whole SBK chunks) that still gives about four CTAs per SM
    for (int piece = SPIECE; piece >= SBK; piece /= 2) {
      items.clear();
      for (int rt = 0; rt < n_rt; ++rt) {
        const int kb = kr[rt].x, ke = kr[rt].y;
        const int pieces = std::max(1, (ke - kb + piece - 1) / piece);
        for (int pc = 0; pc < pieces; ++pc) {
          const int a0 = kb + pc * piece, a1 = std::min(ke, a0 + piece);
          items.push_back(make_int4(rt, a0, std::max(a0, a1), pc | (pieces << 16)));
        }
      }
      if ((int64_t)items.size() * n_ct >= 4LL * n_sms) break;
    }
    n_sweep_items = (int)items.size();
    sweep_items.upload(items, s);
    sweep_part.alloc(std::max<size_t>((size_t)n_sweep_items * n_ct * SBM * SBN, 1));
    sweep_count.alloc((size_t)n_rt * n_ct);
    EMT_CUDA(cudaMemsetAsync(sweep_count.p, 0, sweep_count.n * sizeof(int), s));
    EMT_CUDA(cudaGetLastError());
    EMT_CUDA(cudaStreamSynchronize(s));
  }
  // expansion tiles (up to 32 positions of one leaf) and per-leaf path tables: for every element
  // of the concatenated ancestor rows, the row of S and the factor offset (minus position x kld)
  {
    std::vector<int4> tl;
    std::vector<int> pp(st.n_leaf + 1, 0), srow, kld;
    std::vector<long long> fb;
    for (int j = 0; j < st.n_leaf; ++j) {
      const int leaf = st.leaf_nodes_h[j];
      const int lo = t.lo[leaf], hi = t.hi[leaf];
      for (int p = lo; p < hi; p += 32) tl.push_back(make_int4(j, p, std::min(32, hi - p), 0));
      for (int a = t.parent[leaf]; a >= 0; a = t.parent[a]) {
        const int k = st.node_k_h[a];
        const int half = lo < t.hi[t.left[a]] ? 0 : k;
        for (int e = 0; e < k; ++e) {
          srow.push_back(st.node_soff_h[a] + half + e);
          fb.push_back((long long)st.node_foff_h[a] - (long long)t.lo[a] * st.node_kld_h[a] + e);
          kld.push_back(st.node_kld_h[a]);
        }
      }
      pp[j + 1] = (int)srow.size();
    }
    if (srow.empty()) {
      srow.push_back(0);
      fb.push_back(0);
      kld.push_back(0);
    }
    n_xtiles = (int)tl.size();
    xtiles.upload(tl, s);
    path_ptr.upload(pp, s);
    path_ptr_h = pp;
    path_srow.upload(srow, s);
    path_fbase.upload(fb, s);
    path_kld.upload(kld, s);
  }
}

void MSim::schedule(int step, int kind, int target, double value, int column) {
  (void)value;
  EMT_REQUIRE(step >= 1, EMT_ERR_INVALID, "event step must be >= 1");
  EMT_REQUIRE(cur_step == 0 && !z_ready, EMT_ERR_STATE, "multi-column events must be scheduled before stepping");
  EMT_REQUIRE(kind == EMT_EVENT_TRIP && column >= 0 && column < R, EMT_ERR_UNSUPPORTED,
              "multi-column simulations take per-column trips only");
  EMT_REQUIRE(target >= 0 && target < n_series, EMT_ERR_INVALID, "trip target must be a series branch");
  EMT_REQUIRE(h_trip_step[column] == 0, EMT_ERR_INVALID, "one trip per column");
  h_trip_step[column] = step;
  h_trip_elem[column] = target;
}

void MSim::prepare_trips(cudaStream_t s) {
  // upload the per-column trips and compute z_c = Ginv u_c (two refined passes) and d_c
  const Tree& t = store->tree;
  std::vector<int> ta(R, 0), tb(R, -1);
  std::vector<double> td(R, 0.0);
  bool any = false;
  for (int c = 0; c < R; ++c) {
    if (h_trip_step[c] <= 0) continue;
    any = true;
    const int e = h_trip_elem[c];
    ta[c] = t.pos[el_a[e]];
    tb[c] = t.pos[el_b[e]];
    td[c] = -el_g[e];
  }
  trip_step.upload(h_trip_step, s);
  trip_elem.upload(h_trip_elem, s);
  trip_a.upload(ta, s);
  trip_b.upload(tb, s);
  trip_delta.upload(td, s);
  {
    std::vector<float2> tdf(R);
    for (int c = 0; c < R; ++c) tdf[c] = host_ff(td[c]);
    trip_dff.upload(tdf, s);
  }
  z_ready = true;
  any_change = any;
  if (!any) return;
  const size_t nR = (size_t)n * R;
  X.zero(s);
  Xf.zero(s);
  MSimD d = view();
  k_mc_unit<<<(R + 127) / 128, 128, 0, s>>>(d, X.p, Xf.p);
  apply_pass(0, 0, 0, 0, s);
  launch_residual(0, 0, s);
  apply_pass(1, 0, 0, 0, s);
  EMT_CUDA(cudaMemcpyAsync(Z.p, V.p, nR * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  k_mc_trip_coef<<<(R + 127) / 128, 128, 0, s>>>(d, trip_coef.p, store->d_status.p);
  EMT_CUDA(cudaGetLastError());
  // back to the initial state
  V.zero(s);
  X.zero(s);
  Xf.zero(s);
}

void MSim::apply_pass(int pass, int n1, int record, int s_in_chunk, cudaStream_t s) {
  const DStore st = store->view();
  const MSimD d = view();
  if (gemm_kind >= 2 && umma.ready) umma.launch(*store, Xf.p, Y.p, s, R_act);
  else
    k_mc_gemm<<<n_tiles, 256, 0, s>>>(st, reinterpret_cast<const int4*>(gemm_tiles.p), Xf.p, Y.p, R, store->d_status.p,
                                      R_act);
  if (store->s_total > 0 && n_crow > 0)
    k_mc_sweep_gemm<<<dim3(n_sweep_items, n_ct), SBT, 0, s>>>(d, Kt.p, ldt, sweep_items.p, sweep_part.p,
                                                              sweep_count.p, n_ct, store->d_status.p);
  if (n1) k_mc_fcol<<<(R_act + 127) / 128, 128, 0, s>>>(st, d, s_in_chunk, store->d_status.p);
  if (tensor_expand())
    umma.expand(*store, d, path_ptr.p, path_srow.p, pass, n1, record, s_in_chunk, s);
  else
    k_mc_expand_tiled<<<dim3(n_xtiles, (R_act + XC - 1) / XC), XT, 0, s>>>(
        st, d, xtiles.p, path_ptr.p, path_srow.p, path_fbase.p, path_kld.p, pass, n1,
        record, s_in_chunk, store->d_status.p);
  EMT_CUDA(cudaGetLastError());
}

void MSim::bench_kernel(int which, int reps, cudaStream_t s) {
  EMT_REQUIRE(which >= 0 && which <= 5, EMT_ERR_INVALID, "which must be 0..5");
  EMT_REQUIRE(reps >= 1 && reps <= 100000, EMT_ERR_INVALID, "reps out of range");
  const bool tc = gemm_kind >= 2 && umma.ready;
  EMT_REQUIRE(tc || which != 1, EMT_ERR_UNSUPPORTED, "the SIMT leaf GEMM has no split kernel");
  const MSimD d = view();
  for (int i = 0; i < reps; ++i) {
    if (which == 1) {
      umma.split(*store, Xf.p, s);
    } else if (which == 0) {
      if (tc) umma.mma(*store, Y.p, s, R_act);
      else
        k_mc_gemm<<<n_tiles, 256, 0, s>>>(store->view(), reinterpret_cast<const int4*>(gemm_tiles.p), Xf.p, Y.p, R,
                                          store->d_status.p, R_act);
    } else if (which == 2) {
      if (store->s_total > 0 && n_crow > 0)
        k_mc_sweep_gemm<<<dim3(n_sweep_items, n_ct), SBT, 0, s>>>(d, Kt.p, ldt, sweep_items.p, sweep_part.p,
                                                                  sweep_count.p, n_ct, store->d_status.p);
    } else if (which == 4) {
      launch_inject(0, s);
    } else if (which == 5) {
      launch_residual(1, 0, s);
    } else {
      // expansion of the correction pass with the N-1 terms, without the record
      if (tensor_expand())
        umma.expand(*store, d, path_ptr.p, path_srow.p, 1, 1, 0, 0, s);
      else
        k_mc_expand_tiled<<<dim3(n_xtiles, (R_act + XC - 1) / XC), XT, 0, s>>>(
            store->view(), d, xtiles.p, path_ptr.p, path_srow.p, path_fbase.p, path_kld.p, 1, 1, 0, 0,
            store->d_status.p);
    }
  }
  EMT_CUDA(cudaGetLastError());
}

bool MSim::inject_pairs() const { return inject_variant() >= 2; }

// 1: one column per thread; 2, 3, 4: two columns per thread with 6, 3 or 2 element ends per round
// trip (2, 3 or 4 CTAs per SM)
int MSim::inject_variant() const {
  if (!inj_pairs || inj_mode == 1) return 1;
  if (inj_mode >= 2) return inj_mode;
  // by default pairs only when they fill whole blocks, with 2 ends per round trip and 4 CTAs per
  // SM (measured fastest on 11,456 buses x 512 columns: 94.5 us against 108.8 for 6 ends, 2 CTAs)
  return R_act % (2 * ITH) == 0 ? 4 : 1;
}

void MSim::launch_inject(int s_in_chunk, cudaStream_t s) {
  const MSimD d = view();
  const int var = inject_variant();
  if (var >= 2) {
    // about 16 CTAs per SM over the launch (4 resident): the last wave stays short
    const int ipp = inj_ipp > 0 ? inj_ipp : positions_per_cta(2, var == 4 ? 16 : 4);
    const dim3 grid((n + ipp - 1) / ipp, (R_act + 2 * ITH - 1) / (2 * ITH));
    if (var == 2) k_mc_inject2<6, 2><<<grid, ITH, inj_smem, s>>>(d, ipp, s_in_chunk, store->d_status.p);
    else if (var == 3) k_mc_inject2<3, 3><<<grid, ITH, inj_smem, s>>>(d, ipp, s_in_chunk, store->d_status.p);
    else k_mc_inject2<2, 4><<<grid, ITH, inj_smem, s>>>(d, ipp, s_in_chunk, store->d_status.p);
  } else {
    const int ipp = inj_ipp > 0 ? inj_ipp : positions_per_cta();
    k_mc_inject<<<dim3((n + ipp - 1) / ipp, (R_act + ITH - 1) / ITH), ITH, inj_smem, s>>>(d, ipp, s_in_chunk,
                                                                                        store->d_status.p);
  }
}

// positions per CTA of the injection and residual kernels: enough CTAs for about four per SM
int MSim::positions_per_cta(int cols_per_thread, int ctas_per_sm) const {
  const int64_t col_blocks = (R_act + cols_per_thread * ITH - 1) / (cols_per_thread * ITH);
  int ipp = IPP_MAX;
  while (ipp > 1 && (int64_t)((n + ipp - 1) / ipp) * col_blocks < (int64_t)ctas_per_sm * n_sm) ipp /= 2;
  return ipp;
}

void MSim::launch_residual(int n1, int s_in_chunk, cudaStream_t s) {
  const MSimD d = view();
  // with two columns per thread where the injection has them (whole blocks of column pairs; in
  // serving-sized column counts one column per thread was faster: 1.37e9 vs 1.35e9 bus-steps/s)
  if (inject_pairs()) {
    const int ipp = positions_per_cta(2, 4);
    k_mc_residual2<<<dim3((n + ipp - 1) / ipp, (R_act + 2 * ITH - 1) / (2 * ITH)), ITH, res_smem, s>>>(
        d, ipp, n1, s_in_chunk, store->d_status.p);
    return;
  }
  const int ipp = positions_per_cta();
  k_mc_residual<<<dim3((n + ipp - 1) / ipp, (R_act + ITH - 1) / ITH), ITH, res_smem, s>>>(d, ipp, n1, s_in_chunk,
                                                                                        store->d_status.p);
}

void MSim::launch_steps(int nst, cudaStream_t s) {
  const MSimD d = view();
  // the per-column change terms (N-1 factors, Sherman-Morrison corrections) only when some column
  // has a change; without any the results are the same bit for bit
  const int n1 = any_change ? 1 : 0;
  for (int i = 0; i < nst; ++i) {
    launch_inject(i, s);
    apply_pass(0, n1, 0, i, s);
    launch_residual(n1, i, s);
    apply_pass(1, n1, 1, i, s);
  }
  k_mc_advance<<<1, 1, 0, s>>>(d_dyn.p, nst);
  EMT_CUDA(cudaGetLastError());
}

void MSim::step(int n_steps, double* record_dev, cudaStream_t s) {
  EMT_REQUIRE(n_steps >= 0, EMT_ERR_INVALID, "n_steps must be >= 0");
  if (n_steps == 0) return;
  if (!z_ready) prepare_trips(s);
  k_mc_set_dyn<<<1, 1, 0, s>>>(d_dyn.p, cur_step, cur_step + 1, record_dev);
  if ((size_t)2 * n_steps > trig.n) trig.alloc((size_t)2 * std::max(n_steps, 1024));
  k_mc_trig<<<(n_steps + 255) / 256, 256, 0, s>>>(trig.p, cur_step + 1, n_steps, omega, dt);
  EMT_CUDA(cudaGetLastError());
  launches += 2;
  int left = n_steps;
  while (left >= kChunk) {
    auto it = graphs.find(R_act);
    if (it == graphs.end()) {
      cudaGraph_t g;
      EMT_CUDA(cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal));
      launch_steps(kChunk, cap_stream);
      EMT_CUDA(cudaStreamEndCapture(cap_stream, &g));
      cudaGraphExec_t ge;
      EMT_CUDA(cudaGraphInstantiate(&ge, g, 0));
      cudaGraphDestroy(g);
      it = graphs.emplace(R_act, ge).first;
    }
    EMT_CUDA(cudaGraphLaunch(it->second, s));
    launches += (int64_t)kChunk * 8 + 1;
    left -= kChunk;
  }
  if (left > 0) {
    launch_steps(left, s);
    launches += (int64_t)left * 8 + 1;
  }
  cur_step += n_steps;
}

void MSim::set_active(int r_act) {
  EMT_REQUIRE(r_act >= 1 && r_act <= R, EMT_ERR_INVALID, "active column count out of range");
  R_act = r_act;
}

void fused_apply_ff64(const Store& st, FusedPlan& p, const double* src, bool src_pos, double* v_pos, cudaStream_t s);

void MSim::admit(int c, int kind, int target, double value, int ev_step, int len, cudaStream_t s) {
  EMT_REQUIRE(c >= 0 && c < R, EMT_ERR_INVALID, "slot out of range");
  z_ready = true;   // columns are managed one by one from here on
  const Tree& t = store->tree;
  const MSimD d = view();
  const int n_rows = std::max(2 * n_el_h, n);
  k_mc_reset_col<<<(n_rows + 255) / 256, 256, 0, s>>>(d, n_rows, c);
  const int n_terms = (int)(term_base.n / 2);
  const double S = omega * (double)cur_step * dt;
  k_mc_rotate_terms<<<(n_terms + 127) / 128, 128, 0, s>>>(d, term_base.p, term_cs.p, term_sn.p, n_terms, c, std::cos(S),
                                                           std::sin(S));
  int on = 0, off = 0x7fffffff, elem = -1, pa = 0, pb = -1;
  double delta = 0.0;
  if (kind == 0) {
    EMT_REQUIRE(target >= 0 && target < n_series, EMT_ERR_INVALID, "trip target must be a series branch");
    on = cur_step + ev_step;
    elem = target;
    pa = t.pos[el_a[target]];
    pb = t.pos[el_b[target]];
    delta = -el_g[target];
  } else if (kind == 1) {
    EMT_REQUIRE(target >= 0 && target < n && value > 0 && len > 0, EMT_ERR_INVALID, "bad fault");
    on = cur_step + ev_step;
    off = on + len;
    pa = t.pos[target];
    delta = 1.0 / value;
  }
  k_mc_set_event<<<1, 1, 0, s>>>(trip_step.p, trip_off.p, trip_elem.p, trip_a.p, trip_b.p, trip_delta.p, trip_dff.p, c,
                                 on, off, elem, pa, pb, delta);
  if (kind >= 0 && !any_change) {
    // from now on the steps carry the per-column change terms: the graphs captured without them go
    EMT_CUDA(cudaStreamSynchronize(s));
    drop_graphs();
    any_change = true;
  }
  if (kind >= 0) {
    // z_c = Ginv u_c with the accurate single-vector apply (float-float), then d_c in FP64
    if (!zplan_ready) {
      make_plan(*store, 0, zplan, s);
      u_bus.alloc(n);
      z_pos.alloc(n);
      zplan_ready = true;
    }
    std::vector<double> u(n, 0.0);
    u[t.perm[pa]] = 1.0;
    if (pb >= 0) u[t.perm[pb]] = -1.0;
    EMT_CUDA(cudaMemcpyAsync(u_bus.p, u.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
    fused_apply_ff64(*store, zplan, u_bus.p, false, z_pos.p, s);
    k_mc_set_z<<<(n + 255) / 256, 256, 0, s>>>(d, Z.p, z_pos.p, c);
    k_mc_one_coef<<<1, 1, 0, s>>>(d, trip_coef.p, c, store->d_status.p);
  }
  EMT_CUDA(cudaGetLastError());
}

// tcgen05 expansion: with kernels 3, or with kernels 2 when it has a tile for every SM (smaller
// problems run the SIMT expansion faster)
bool MSim::tensor_expand() const {
  return umma.exp_ready && (gemm_kind == 3 || (gemm_kind == 2 && umma.x_tiles >= n_sm));
}

void MSim::set_gemm(int kind, int tn, cudaStream_t s) {
  EMT_REQUIRE(kind >= 1 && kind <= 3, EMT_ERR_INVALID, "kernels must be 1, 2 or 3");
  EMT_REQUIRE(tn == 0 || tn == 64 || tn == 128 || tn == 192 || tn == 256, EMT_ERR_INVALID,
              "tile width must be 0, 64, 128, 192 or 256");
  EMT_CUDA(cudaDeviceSynchronize());
  drop_graphs();
  gemm_kind = kind;
  if (kind >= 2 && umma.ready && tn != 0 && tn != umma.TN) umma.build(*store, R, s, tn);
  EMT_CUDA(cudaStreamSynchronize(s));
}

void MSim::set_inject(int mode, int ipp) {
  EMT_REQUIRE(mode >= 0 && mode <= 4, EMT_ERR_INVALID, "injection mode must be 0..4");
  EMT_REQUIRE(ipp == 0 || ipp == 1 || ipp == 2 || ipp == 4 || ipp == 8, EMT_ERR_INVALID,
              "positions per CTA must be 0, 1, 2, 4 or 8");
  EMT_REQUIRE(mode < 2 || inj_pairs, EMT_ERR_UNSUPPORTED, "two columns per thread need an even column count");
  EMT_CUDA(cudaDeviceSynchronize());
  drop_graphs();
  inj_mode = mode;
  inj_ipp = ipp;
}

namespace {
// tuning key: buses, leaves, depth, precision, columns, SMs
using MTuneKey = std::array<int64_t, 6>;
std::map<MTuneKey, std::array<int, 4>> g_mtune_cache;
std::mutex g_mtune_mutex;
MTuneKey mtune_key(const MSim& m, int sms) {
  return {m.n, m.store->n_leaf, m.store->tree.max_depth, m.store->precision, m.R, sms};
}
}  // namespace

void MSim::autotune(int probe_steps, int* best_tn, int* best_kind, int* best_inj, cudaStream_t s) {
  EMT_REQUIRE(probe_steps >= 1 && probe_steps <= 100000, EMT_ERR_INVALID, "probe_steps out of range");
  EMT_REQUIRE(R_act == R, EMT_ERR_STATE, "tune a simulation with every column active");
  cudaEvent_t e0, e1;
  EMT_CUDA(cudaEventCreate(&e0));
  EMT_CUDA(cudaEventCreate(&e1));
  auto time_it = [&]() {
    reset(s);
    step(8, nullptr, s);
    EMT_CUDA(cudaEventRecord(e0, s));
    step(probe_steps, nullptr, s);
    EMT_CUDA(cudaEventRecord(e1, s));
    EMT_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    EMT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    return ms;
  };
  // candidates of the products: FP32 CUDA cores, then tcgen05 (leaf tiles of every width, with
  // the expansion on tcgen05 by the tile count or always)
  std::vector<std::pair<int, int>> cands = {{1, 0}};
  if (umma.ready)
    for (int kind : {2, 3})
      for (int tn : {64, 128, 192, 256}) cands.push_back({kind, tn});
  float best = 1e30f;
  int bkind = 1, btn = 0;
  set_inject(0, 0);
  for (auto [kind, tn] : cands) {
    set_gemm(kind, tn, s);
    if (kind == 3 && umma.x_tiles >= n_sm) continue;   // the same kernels as kind 2
    const float ms = time_it();
    if (ms < best) {
      best = ms;
      bkind = kind;
      btn = tn;
    }
  }
  set_gemm(bkind, btn, s);
  // then the injection kernel with those products
  int binj = 0, bipp = 0;
  for (int mode : {1, 2, 3, 4}) {
    if (mode >= 2 && !inj_pairs) break;
    for (int ipp : {0, 4, 2, 1}) {
      set_inject(mode, ipp);
      const float ms = time_it();
      if (ms < best) {
        best = ms;
        binj = mode;
        bipp = ipp;
      }
    }
  }
  set_inject(binj, bipp);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  reset(s);
  EMT_CUDA(cudaStreamSynchronize(s));
  {
    std::lock_guard<std::mutex> lk(g_mtune_mutex);
    g_mtune_cache[mtune_key(*this, n_sm)] = {bkind, btn, binj, bipp};
  }
  if (best_tn) *best_tn = btn;
  if (best_kind) *best_kind = bkind;
  if (best_inj) *best_inj = binj;
}

bool MSim::apply_cached_tuning(cudaStream_t s) {
  std::array<int, 4> v;
  {
    std::lock_guard<std::mutex> lk(g_mtune_mutex);
    auto it = g_mtune_cache.find(mtune_key(*this, n_sm));
    if (it == g_mtune_cache.end()) return false;
    v = it->second;
  }
  set_gemm(v[0], v[1], s);
  set_inject(v[2], v[3]);
  return true;
}

void MSim::reset(cudaStream_t s) {
  Ih.zero(s);
  V.zero(s);
  X.zero(s);
  Xf.zero(s);
  EMT_CUDA(cudaMemsetAsync(d_dyn.p, 0, sizeof(SimDyn), s));
  cur_step = 0;
}

void MSim::set_monitor(int nm, const int32_t* buses) {
  EMT_REQUIRE(nm >= 0 && (nm == 0 || buses), EMT_ERR_INVALID, "bad monitor list");
  std::vector<int> mi(n, -1);
  for (int k = 0; k < nm; ++k) {
    EMT_REQUIRE(buses[k] >= 0 && buses[k] < n, EMT_ERR_INVALID, "monitor bus out of range");
    EMT_REQUIRE(mi[store->tree.pos[buses[k]]] < 0, EMT_ERR_INVALID, "duplicate monitor bus");
    mi[store->tree.pos[buses[k]]] = k;
  }
  EMT_CUDA(cudaDeviceSynchronize());
  mon_idx.upload(mi, nullptr);
  n_mon = nm;
  drop_graphs();
  EMT_CUDA(cudaDeviceSynchronize());
}

void MSim::read(int what, double* host_out) {
  if (what == 1) {
    host_out[0] = (double)cur_step;
    return;
  }
  EMT_REQUIRE(what == 0, EMT_ERR_INVALID, "unknown read selector");
  std::vector<float2> vp((size_t)n * R);
  EMT_CUDA(cudaDeviceSynchronize());
  EMT_CUDA(cudaMemcpy(vp.data(), V.p, vp.size() * sizeof(float2), cudaMemcpyDeviceToHost));
  for (int p = 0; p < n; ++p)
    for (int c = 0; c < R; ++c)
      host_out[(size_t)c * n + store->tree.perm[p]] = (double)vp[(size_t)p * R + c].x + (double)vp[(size_t)p * R + c].y;
}

void MSim::stats(int64_t* out, int n_out) const {
  const Store& st = *store;
  int64_t leaf = 0, fac = 0, core = 0;
  for (int j = 0; j < st.n_leaf; ++j) {
    const int nd = st.leaf_nodes_h[j];
    const int64_t b = st.tree.hi[nd] - st.tree.lo[nd];
    leaf += b * b;
  }
  for (int q : st.lvl_nodes_h) {
    const int64_t k = st.node_k_h[q];
    fac += (int64_t)(st.tree.hi[q] - st.tree.lo[q]) * k;
    core += 4 * k * k;
  }
  const int64_t v[] = {n, st.n_leaf, leaf, fac, core, n_tiles, n_inc, n_crow, st.s_total, launches, n_series,
                       (int64_t)el_a.size(), inject_pairs() ? 2 : 1, inject_variant(), inject_pairs() ? 2 : 1};
  for (int i = 0; i < n_out && i < (int)(sizeof(v) / sizeof(v[0])); ++i) out[i] = v[i];
}

}  // namespace emt

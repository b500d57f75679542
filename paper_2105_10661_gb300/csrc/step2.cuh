// Second-generation fused step kernels (single column).
//
// Same two-kernel split as fused.cuh (leaf partials; boundary sweep + expansion), rebuilt around
// what bounds a 1,432-bus step on this GPU, which is latency, not bandwidth:
//   * programmatic dependent launch: every kernel issues the loads of its static data (leaf rows,
//     element parameters, the sweep image) before griddepcontrol.wait, so they overlap the
//     previous kernel, and only the data produced by that kernel is read after the wait;
//   * the sweep's static data (per-level metadata, -g per cut, the factor rows needed at every cut
//     endpoint, the cores, the CTA's own factor rows) is one precomputed image copied into shared
//     memory by cp.async.bulk (TMA bulk copies completing on an mbarrier, with a bounded wait), so
//     the sweep walks no tree pointers in global memory;
//   * leaf rows are prefetched into registers; element parameters are one 32-byte record per
//     element end; sin/cos of the 60 Hz phase come from a per-step table.
#pragma once
#include "fused.cuh"

namespace emt {

struct FusedPlan;

// One element end: the history source of a bus-to-bus element lives at both ends and both copies
// evolve identically (same operands, same instruction sequence).
struct IncRec {
  int self;       // position of this end
  int other;      // position of the other end, -1 for ground
  int sgn;        // +1 at the from-bus, -1 at the to-bus
  int pad;
  double g, alpha, beta;
};
static_assert(sizeof(IncRec) == 40, "IncRec must be 40 bytes");

struct SrcRec {
  double cs, sn;  // coef cos(phi), coef sin(phi): term = cs sin(wt) + sn cos(wt)
};

// Header of the sweep image (int32 offsets in units of the stated type from the image start).
struct ImgHeader {
  int n_crow, n_items, s_total, max_depth, n_leaf, n_cut, n_seg, n_core;
  int off_crow;      // ints: [n_crow][3] = cta0, ncta, loc
  int off_lvl_item;  // ints: [max_depth + 2]
  int off_item;      // ints: [n_items][6] = crow, sidx, cut, r_off, seg0, nseg
  int off_seg;       // ints: [n_seg][2] = s index, k
  int off_lvl_core;  // ints: [max_depth + 2]
  int off_core;      // ints: [n_core][4] = s out, t in, m2, c_off
  int off_anc_ptr;   // ints: [n_leaf + 1]
  int off_anc;       // ints: [n_anc][5] = k, kld, split position, s index (left half), s index (right half)
  int off_crow_pos;  // ints: [n_crow] positions of the distinct cut rows
  int off_cpair_ptr; // ints: [n_crow + 1] ranges into the partial-offset list
  int off_cpair;     // ints: [n_cpair] offsets into the partial buffer
  int n_cpair;
  int int_words;     // total ints (padded to 16 bytes)
  int off_g_bytes;   // byte offset of -g per cut (T)
  int off_r_bytes;   // byte offset of the cut-row factor segments (T)
  int img_bytes;     // bytes of the image (without cores)
  int cut_w;         // left entries per cut column (block cuts: rows crow .. crow + cut_w - 1)
};

// Per-CTA copy list for its own factor rows: up to kMaxAnc ancestors.
constexpr int kMaxAnc = 12;
struct OwnCopy {
  long long src_bytes[kMaxAnc];   // byte offset into the factor array
  int bytes[kMaxAnc];
  int n;
  int pad;
};

struct Step2D {
  // partial kernel
  const IncRec* inc;
  const double2* src_sum;  // per position: (sum coef cos(phi), sum coef sin(phi))
  const int* inc_ptr;
  double* Ih;
  const SrcRec* src;
  const int* src_ptr;
  const double* trig;      // [2 * n] sin, cos of w t per step (indexed from trig_first)
  const float4* trigff;    // [n] the same as float-float pairs: sin hi, lo, cos hi, lo
  // sweep kernel
  const unsigned char* img;
  int img_bytes;
  const unsigned char* cores;
  int core_bytes;
  const unsigned char* fac;   // factor array of the precision
  const OwnCopy* own;
  size_t sweep_smem_static;   // bytes of image + cores + own rows (16-aligned)
  int own_rows_max;
  int max_inc;                // largest number of element ends owned by one CTA
  int max_lnc;                // largest number of CTAs of one leaf
  const double* ylf;          // leaf-stage values per position (kernel generation 3), or null
};

// Build / refresh the sweep image of a store (a plan, when given, adds the CTAs holding each cut
// row's partial sums), and the matrix form of the sweep: K ([s_total][ldk] elements of the
// precision) with s = K y_cut.
void build_sweep_image(const Store& st, const FusedPlan* p, int prec, ImgHeader& hdr, DevBuf<double>& img,
                       DevBuf<int>& seg_src, DevBuf<int>& seg_dst, DevBuf<int>& seg_len, int& n_seg, cudaStream_t s);
void refresh_sweep_image(const Store& st, int prec, const ImgHeader& hdr, DevBuf<double>& img,
                         const DevBuf<int>& seg_src, const DevBuf<int>& seg_dst, const DevBuf<int>& seg_len,
                         int n_seg, cudaStream_t s);
void build_sweep_matrix(int prec, const unsigned char* img, int img_bytes, const unsigned char* cores, int core_bytes,
                        int n_crow, int s_total, int ldk, void* K, cudaStream_t s);

// Boundary sweep of every tree node, bottom-up, from the shared-memory image: at each depth,
// t = (-g) y_cut - sum over deeper ancestors of (factor row . s) for every cut endpoint (the
// gather form of t_p = [h_l^T y_l; h_r^T y_r], Eq. 9 factors), then s = C t per node. ycut holds
// the leaf-stage value of every distinct cut row. Dot products are split over groups of kGroup
// threads (shuffle-reduced) so that no thread runs a long dependent chain; loops are
// warp-uniform for the shuffles. Uses every thread of the block; ends with __syncthreads.
template <int PREC, int kGroup>
__device__ __forceinline__ void sweep_levels(const unsigned char* img, const unsigned char* cores,
                                             const typename Acc<PREC>::X* ycut, typename Acc<PREC>::X* t,
                                             typename Acc<PREC>::X* s) {
  using A = Acc<PREC>;
  using X = typename A::X;
  using T = typename A::T;
  const ImgHeader* H = reinterpret_cast<const ImgHeader*>(img);
  const int* I = reinterpret_cast<const int*>(img);
  const T* Gn = reinterpret_cast<const T*>(img + H->off_g_bytes);
  const T* R = reinterpret_cast<const T*>(img + H->off_r_bytes);
  const T* C = reinterpret_cast<const T*>(cores);
  const int* lvl_item = I + H->off_lvl_item;
  const int* item = I + H->off_item;
  const int* seg = I + H->off_seg;
  const int* lvl_core = I + H->off_lvl_core;
  const int* core = I + H->off_core;
  const int grp = threadIdx.x / kGroup, gl = threadIdx.x % kGroup;
  const int n_groups = blockDim.x / kGroup;
  const int g_warp = (threadIdx.x >> 5) * (32 / kGroup);   // first group of this warp
  for (int d = H->max_depth - 1; d >= 0; --d) {
    const int i0 = lvl_item[d], i1 = lvl_item[d + 1];
    for (int base = i0; base < i1; base += n_groups) {
      if (base + g_warp >= i1) break;   // the whole warp is idle for the rest of this phase
      const int it = base + grp;
      A a;
      const int* rec = item + 6 * (it < i1 ? it : i0);
      const int W = H->cut_w;
      if (it < i1) {
        // a side of a block column: its rows are pre-combined with the coefficients in the image
        if (gl == 0) {
          if (W > 1 && rec[2] >= 0)
            for (int w = 0; w < W; ++w) a.fma(Gn[rec[2] * W + w], ycut[rec[0] + w]);
          else
            a.add(ycut[rec[0]]);
        }
        const T* rv = R + rec[3];
        for (int sg = rec[4]; sg < rec[4] + rec[5]; ++sg) {
          const int si = seg[2 * sg], k = seg[2 * sg + 1];
          for (int e = gl; e < k; e += kGroup) a.fma(rv[e], neg(s[si + e]));
          rv += k;
        }
      }
      X val = a.getx();
#pragma unroll
      for (int o = kGroup / 2; o > 0; o >>= 1) {
        A tt;
        tt.add(val);
        tt.add(a.shfl_xor(val, o));
        val = tt.getx();
      }
      if (it < i1 && gl == 0) {
        if (rec[2] >= 0 && W == 1) {
          A m;
          m.fma(Gn[rec[2]], val);
          val = m.getx();
        }
        t[rec[1]] = val;
      }
    }
    __syncthreads();
    const int j0 = lvl_core[d], j1 = lvl_core[d + 1];
    for (int base = j0; base < j1; base += n_groups) {
      if (base + g_warp >= j1) break;
      const int w = base + grp;
      A a;
      const int* rec = core + 4 * (w < j1 ? w : j0);
      if (w < j1) {
        const T* Cr = C + rec[3];
        const X* tq = t + rec[1];
        for (int e = gl; e < rec[2]; e += kGroup) a.fma(Cr[e], tq[e]);
      }
      X val = a.getx();
#pragma unroll
      for (int o = kGroup / 2; o > 0; o >>= 1) {
        A tt;
        tt.add(val);
        tt.add(a.shfl_xor(val, o));
        val = tt.getx();
      }
      if (w < j1 && gl == 0) s[rec[0]] = val;
    }
    __syncthreads();
  }
}

}  // namespace emt

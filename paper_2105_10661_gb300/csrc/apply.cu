// Single-vector hierarchical apply (the fused two-kernel form) and FP32 refinement against the
// FP64 residual r = i - G v.
#include <algorithm>
#include <cmath>

#include "plan.h"

namespace emt {

namespace {

// Leaf stage of v = G^{-1} i (Eq. 2 with the leaf blocks of Sec. III): CTA c forms the partial
// products of its rows of the leaf inverse with its slice of x.
template <int PREC>
__global__ void __launch_bounds__(kFusedThreads) k_apply_partial(DStore st, CtaMapD cm, const double* __restrict__ src,
                                                                 int src_pos, typename Acc<PREC>::X* __restrict__ part) {
  using A = Acc<PREC>;
  using X = typename A::X;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  X* xs = reinterpret_cast<X*>(smem_raw);
  X* red = xs + ((cm.max_rows + 1) & ~1);
  const int c = blockIdx.x;
  const int j = cm.cta_leaf[c];
  const int r0 = cm.cta_r0[c], r1 = cm.cta_r1[c];
  const int lo = st.lo[st.leaf_node[j]];
  for (int r = threadIdx.x; r < r1 - r0; r += blockDim.x) {
    const int pos = lo + r0 + r;
    xs[r] = A::prep(src_pos ? src[pos] : src[st.perm[pos]]);
  }
  __syncthreads();
  leaf_partial_core<PREC>(st, j, r0, r1, xs, part + (int64_t)c * cm.pld, red);
}

// Boundary sweep (t_p = [h_l^T y_l; h_r^T y_r], s_p = C_p t_p with Eq. 9's factors) and the
// expansion v = y - sum over ancestors of (factor row . s) for the CTA's rows.
template <int PREC>
__global__ void __launch_bounds__(kFusedThreads) k_apply_sweep(DStore st, CtaMapD cm, CutRowsD cr,
                                                               const typename Acc<PREC>::X* __restrict__ part,
                                                               const typename Acc<PREC>::T* __restrict__ cut_gn,
                                                               double* __restrict__ v_pos, double* __restrict__ v_bus,
                                                               int accumulate) {
  using A = Acc<PREC>;
  using X = typename A::X;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  X* ycut = reinterpret_cast<X*>(smem_raw);
  X* t = ycut + cr.n_crow;
  X* s = t + cr.s_total;
  boundary_sweep<PREC>(st, cm, cr, part, ycut, t, s, cut_gn);
  const int c = blockIdx.x;
  const int j = cm.cta_leaf[c];
  const int leaf_node = st.leaf_node[j];
  const int lo = st.lo[leaf_node];
  const int r0 = cm.cta_r0[c], r1 = cm.cta_r1[c];
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = r0 + warp; r < r1; r += nw) {
    const int pos = lo + r;
    const X y = leaf_y<PREC>(st, cm, part, pos);
    const X v = expand_row<PREC>(st, leaf_node, pos, y, s);
    if ((threadIdx.x & 31) == 0) {
      double out = A::todbl(v);
      if (accumulate) out += v_pos[pos];
      v_pos[pos] = out;
      if (v_bus) v_bus[st.perm[pos]] = out;
    }
  }
}

// r_pos = i - G v with Eq. 1's G (FP64, position-ordered CSR), i bus-ordered or position-ordered:
// the residual that refines an FP32 apply
__global__ void k_residual(int n, const int* __restrict__ ptr, const int* __restrict__ col,
                           const double* __restrict__ val, const int* __restrict__ perm, const double* __restrict__ src,
                           int src_pos, const double* __restrict__ v_pos, double* __restrict__ r_pos) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = src_pos ? src[i] : src[perm[i]];
  for (int t = ptr[i]; t < ptr[i + 1]; ++t) acc -= val[t] * v_pos[col[t]];
  r_pos[i] = acc;
}

// position order (the nested ordering of Sec. III-B) -> bus order
__global__ void k_scatter(int n, const int* __restrict__ perm, const double* __restrict__ v_pos, double* __restrict__ v_bus) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v_bus[perm[i]] = v_pos[i];
}

// -g per cut column (h_l[:, e] = -g_e e_a, Sec. III-A) in the three precisions
__global__ void k_neg_g(int n, const double* __restrict__ g, double* __restrict__ g64, float2* __restrict__ gff,
                        float* __restrict__ g32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = -g[i];
  g64[i] = x;
  const float h = (float)x;
  gff[i] = make_float2(h, (float)(x - (double)h));
  g32[i] = h;
}

template <int PREC>
void launch_apply(const Store& st, FusedPlan& p, const double* src, bool src_pos, double* v_pos, double* v_bus,
                  bool acc, cudaStream_t s) {
  using X = typename Acc<PREC>::X;
  using T = typename Acc<PREC>::T;
  const DStore v = st.view();
  const CtaMapD cm = p.cmap();
  const CutRowsD cr = p.crows();
  X* part = reinterpret_cast<X*>(p.part.p);
  const T* gn = PREC == EMT_PREC_FP64 ? reinterpret_cast<const T*>(p.cut_gn64.p)
                : PREC == EMT_PREC_FF64 ? reinterpret_cast<const T*>(p.cut_gnff.p)
                                        : reinterpret_cast<const T*>(p.cut_gn32.p);
  static bool attr_set = false;
  if (!attr_set) {
    EMT_CUDA(cudaFuncSetAttribute(k_apply_partial<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    EMT_CUDA(cudaFuncSetAttribute(k_apply_sweep<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  k_apply_partial<PREC><<<p.n_cta, kFusedThreads, p.smem_partial, s>>>(v, cm, src, src_pos ? 1 : 0, part);
  k_apply_sweep<PREC><<<p.n_cta, kFusedThreads, p.smem_sweep, s>>>(v, cm, cr, part, gn, v_pos, v_bus, acc ? 1 : 0);
  EMT_CUDA(cudaGetLastError());
}

}  // namespace

CtaMapD FusedPlan::cmap() const {
  CtaMapD m;
  m.cta_leaf = cta_leaf.p;
  m.cta_r0 = cta_r0.p;
  m.cta_r1 = cta_r1.p;
  m.leaf_cta0 = leaf_cta0.p;
  m.leaf_ncta = leaf_ncta.p;
  m.n_cta = n_cta;
  m.pld = pld;
  m.max_rows = max_rows;
  return m;
}

CutRowsD FusedPlan::crows() const {
  CutRowsD c;
  c.item_pos = item_pos.p;
  c.item_crow = item_crow.p;
  c.item_sidx = item_sidx.p;
  c.item_cut = item_cut.p;
  c.item_lvl = item_lvl.p;
  c.crow_pos = crow_pos.p;
  c.n_crow = (int)crow_pos.n;
  c.n_items = (int)item_pos.n;
  c.s_total = s_total;
  return c;
}

int default_rows_per_cta(const Store& st) {
  // enough CTAs to cover the SMs about once for the single-network sizes
  const int target = 148;
  int r = (st.n + target - 1) / target;
  r = std::max(4, std::min(r, 64));
  return r;
}

void make_plan(const Store& st, int rows_per_cta, FusedPlan& p, cudaStream_t s) {
  if (rows_per_cta <= 0) rows_per_cta = default_rows_per_cta(st);
  EMT_REQUIRE(rows_per_cta <= kFusedThreads, EMT_ERR_INVALID, "rows_per_cta must be <= 256");
  p.rows_per_cta = rows_per_cta;
  p.s_total = st.s_total;
  std::vector<int> cl, c0v, c1v, lc0(st.n_leaf), lnc(st.n_leaf);
  int maxb = 0;
  for (int j = 0; j < st.n_leaf; ++j) {
    const int node = st.leaf_nodes_h[j];
    const int b = st.tree.hi[node] - st.tree.lo[node];
    maxb = std::max(maxb, b);
    EMT_REQUIRE(b <= 2048, EMT_ERR_UNSUPPORTED, "leaf larger than 2048 buses for the fused kernels");
    lc0[j] = (int)cl.size();
    const int nc = (b + rows_per_cta - 1) / rows_per_cta;
    lnc[j] = nc;
    // spread rows evenly over the leaf's CTAs
    for (int c = 0; c < nc; ++c) {
      cl.push_back(j);
      c0v.push_back((int)((int64_t)b * c / nc));
      c1v.push_back((int)((int64_t)b * (c + 1) / nc));
    }
  }
  p.n_cta = (int)cl.size();
  p.max_rows = 0;
  for (int c = 0; c < p.n_cta; ++c) p.max_rows = std::max(p.max_rows, c1v[c] - c0v[c]);
  p.pld = (maxb + 3) / 4 * 4;
  p.h_cta_leaf = cl;
  p.h_cta_r0 = c0v;
  p.h_cta_r1 = c1v;
  p.h_leaf_cta0 = lc0;
  p.h_leaf_ncta = lnc;
  p.cta_leaf.upload(cl, s);
  p.cta_r0.upload(c0v, s);
  p.cta_r1.upload(c1v, s);
  p.leaf_cta0.upload(lc0, s);
  p.leaf_ncta.upload(lnc, s);
  // sweep items with per-depth ranges (items are generated deepest level first)
  const CutRows& cr = st.cut_rows;
  std::vector<int> lvl(st.tree.max_depth + 2, 0), cutidx(cr.n_items);
  for (int it = 0; it < cr.n_items; ++it) {
    const int q = cr.item_node[it];
    lvl[st.tree.depth[q] + 1] += 1;
    const int k = st.node_k_h[q];
    const int slot = cr.item_sidx[it] - st.node_soff_h[q];
    cutidx[it] = slot < k ? st.tree.cut_ptr[q] + slot : -1;
  }
  // items sorted deepest first -> build ranges per depth in increasing depth order
  std::vector<int> pos_s, crow_s, sidx_s, cut_s;
  std::vector<int> ptr(st.tree.max_depth + 2, 0);
  for (int d = 0; d <= st.tree.max_depth; ++d) {
    ptr[d] = (int)pos_s.size();
    for (int it = 0; it < cr.n_items; ++it)
      if (st.tree.depth[cr.item_node[it]] == d) {
        pos_s.push_back(cr.item_pos[it]);
        crow_s.push_back(cr.item_crow[it]);
        sidx_s.push_back(cr.item_sidx[it]);
        cut_s.push_back(cutidx[it]);
      }
  }
  ptr[st.tree.max_depth + 1] = (int)pos_s.size();
  p.item_pos.upload(pos_s, s);
  p.item_crow.upload(crow_s, s);
  p.item_sidx.upload(sidx_s, s);
  p.item_cut.upload(cut_s, s);
  p.item_lvl.upload(ptr, s);
  p.crow_pos.upload(cr.crow_pos, s);
  p.part.alloc((size_t)p.n_cta * p.pld);
  p.cut_gn64.alloc(std::max<size_t>(st.cut_g_h.size(), 1));
  p.cut_gnff.alloc(std::max<size_t>(st.cut_g_h.size(), 1));
  p.cut_gn32.alloc(std::max<size_t>(st.cut_g_h.size(), 1));
  refresh_plan_values(st, p, s);
  // shared memory: partial = x slice + group reduction; sweep = ycut + t + s (8-byte entries)
  size_t red = 0;
  for (int ve : {2, 4}) {   // 8-byte entries with 2 per load (FP64, FF64), 4-byte with 4 (FP32)
    const int slots = (maxb + ve - 1) / ve;
    const int cover = std::min(slots, kFusedThreads);
    const int G = kFusedThreads / cover;
    red = std::max(red, (size_t)G * slots * ve * (ve == 2 ? 8 : 4));
  }
  p.smem_partial = (size_t)((p.max_rows + 1) & ~1) * 8 + red + 64;
  p.smem_sweep = (size_t)(cr.crow_pos.size() + 2 * st.s_total) * 8 + 64;
  EMT_REQUIRE(p.smem_partial <= 200 * 1024 && p.smem_sweep <= 200 * 1024, EMT_ERR_UNSUPPORTED,
              "fused kernels need more shared memory than available");
}

void refresh_plan_values(const Store& st, FusedPlan& p, cudaStream_t s) {
  if (p.sa) p.sa->refresh(st, s);
  const int nc = (int)st.cut_g_h.size();
  if (nc == 0) return;
  k_neg_g<<<(nc + 255) / 256, 256, 0, s>>>(nc, st.d_cut_g.p, p.cut_gn64.p, p.cut_gnff.p, p.cut_gn32.p);
  EMT_CUDA(cudaGetLastError());
}

void fused_apply(const Store& st, FusedPlan& p, const double* src, bool src_pos, double* v_pos, double* v_bus,
                 bool accumulate, cudaStream_t s) {
  if (p.sa && p.sa->ready) {
    p.sa->mode = p.stream_mode;
    stream_apply(st, *p.sa, src, src_pos, v_pos, v_bus, accumulate, s);
    return;
  }
  switch (st.precision) {
    case EMT_PREC_FP64: launch_apply<EMT_PREC_FP64>(st, p, src, src_pos, v_pos, v_bus, accumulate, s); break;
    case EMT_PREC_FF64: launch_apply<EMT_PREC_FF64>(st, p, src, src_pos, v_pos, v_bus, accumulate, s); break;
    default: launch_apply<EMT_PREC_FP32>(st, p, src, src_pos, v_pos, v_bus, accumulate, s); break;
  }
}

void fused_apply_ff64(const Store& st, FusedPlan& p, const double* src, bool src_pos, double* v_pos, cudaStream_t s) {
  launch_apply<EMT_PREC_FF64>(st, p, src, src_pos, v_pos, nullptr, false, s);
}

// emt_apply: single vectors go through the fused kernels; FP32 stores are refined against the
// FP64 residual (fixed number of passes, max_refine).
void apply_vectors(Store& st, FusedPlan& p, DevBuf<double>& vpos, DevBuf<double>& rpos, const double* i_dev,
                   double* v_dev, int nrhs, int64_t ld, int max_refine, cudaStream_t s) {
  if (vpos.n < (size_t)st.n) vpos.alloc(st.n);
  if (rpos.n < (size_t)st.n) rpos.alloc(st.n);
  if (p.sa && p.sa->rps_req != p.stream_rps) p.sa.reset();   // re-plan for another stage depth
  if (!p.sa && (stream_apply_wanted(st) || (p.stream_mode >= 1 && st.precision != EMT_PREC_FP32))) {
    auto sa = std::make_shared<StreamApply>();
    sa->rps_req = p.stream_rps;
    if (sa->build(st, s)) p.sa = sa;
  }
  const bool refine = st.precision == EMT_PREC_FP32 && max_refine > 0;
  for (int c = 0; c < nrhs; ++c) {
    const double* src = i_dev + (int64_t)c * ld;
    double* dst = v_dev + (int64_t)c * ld;
    fused_apply(st, p, src, false, vpos.p, refine ? nullptr : dst, false, s);
    if (refine) {
      for (int it = 0; it < max_refine; ++it) {
        k_residual<<<(st.n + 255) / 256, 256, 0, s>>>(st.n, st.d_csr_ptr.p, st.d_csr_col.p, st.d_csr_val.p,
                                                      st.d_perm.p, src, 0, vpos.p, rpos.p);
        fused_apply(st, p, rpos.p, true, vpos.p, nullptr, true, s);
      }
      k_scatter<<<(st.n + 255) / 256, 256, 0, s>>>(st.n, st.d_perm.p, vpos.p, dst);
    }
  }
  EMT_CUDA(cudaGetLastError());
}

}  // namespace emt

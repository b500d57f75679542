// Construction and modification of the hierarchical inverse on the GPU (Sec. III-IV).
//
// Construction follows Algorithm 1 bottom-up:
//   1. leaf blocks G_jj are expanded from the position-ordered CSR of G and inverted directly
//      (Cholesky G_jj = L L^T, W = L^{-1}, G_jj^{-1} = W^T W; FP64);
//   2. for every internal node p, deepest level first, the factors of Eq. 9 are formed by
//      applying the already complete child stores to the cut columns:
//      [P; Q] = blkdiag(Ginv_l, Ginv_r) [h_l; h_r] (the leaf stage of a unit column is a scaled
//      column of the leaf inverse; the deeper levels are applied level by level);
//   3. the node core: PAPER keeps [[0, I], [I, 0]] (M = -P Q^T, Eq. 9); EXACT inverts
//      S = [[h_l^T P, I], [I, h_r^T Q]] (Gauss-Jordan, partial pivoting, FP64), the Woodbury
//      core that makes Ginv_p = D^{-1} - Y S^{-1} Y^T exact.
// Modification: EXACT stores get an exact local update (Sherman-Morrison at every node on the
// paths from the touched leaves to the root); PAPER stores get Algorithm 2.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>

#include "store.h"

namespace emt {

namespace {

constexpr int kMaxCoreDim = 160;    // 2k limit for the in-shared-memory core inversion
constexpr int kMaxCoreDimWs = 4096; // 2k limit with the global-memory workspace
constexpr int kPanelCols = 32;     // column chunk of the level sweep

__device__ __forceinline__ int anc_at_depth(const DStore& st, int q, int d) {
  while (st.depth[q] > d) q = st.parent[q];
  return q;
}

// ------------------------------------------------------------------ leaf blocks
// Leaf blocks G_jj of Algorithm 1's direct inversion (Sec. III-B): cleared, then assembled from
// the CSR copy of G.
__global__ void k_zero_leaf(DStore st, const int* leaves) {
  const int j = leaves[blockIdx.x];
  const int node = st.leaf_node[j];
  const int b = st.hi[node] - st.lo[node];
  const int ld = st.leaf_ld[j];
  double* A = st.L64 + st.leaf_off[j];
  for (int t = threadIdx.x; t < b * ld; t += blockDim.x) A[t] = 0.0;
}

__global__ void k_assemble_leaf(DStore st, const int* __restrict__ csr_ptr, const int* __restrict__ csr_col,
                                const double* __restrict__ csr_val, const int* leaves) {
  const int j = leaves[blockIdx.x];
  const int node = st.leaf_node[j];
  const int lo = st.lo[node], hi = st.hi[node];
  const int ld = st.leaf_ld[j];
  double* A = st.L64 + st.leaf_off[j];
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    for (int c = csr_ptr[i]; c < csr_ptr[i + 1]; ++c) {
      const int cp = csr_col[c];
      if (cp >= lo && cp < hi) A[(int64_t)(i - lo) * ld + (cp - lo)] = csr_val[c];
    }
  }
}

// Blocked right-looking Cholesky of the leaf blocks (in place, lower), panel width kCholNb: per
// panel, the diagonal block is factored in shared memory (one CTA per leaf), the rows below it
// solved against it (CTAs of kCholRows rows per leaf), and the trailing lower triangle updated in
// 64 x 64 tiles (as many CTAs as tiles), so a leaf's FP64 work is spread over the SMs instead of
// one CTA walking its b columns.
constexpr int kCholNb = 64, kCholRows = 128;

__global__ void __launch_bounds__(256) k_chol_diag(DStore st, const int* leaves, int kb) {
  __shared__ double D[kCholNb][kCholNb + 1];
  __shared__ int bad;
  if (*st.status != DEV_OK) return;
  const int j = leaves[blockIdx.x];
  const int node = st.leaf_node[j];
  const int b = st.hi[node] - st.lo[node];
  if (kb >= b) return;
  const int nb = min(kCholNb, b - kb);
  const int ld = st.leaf_ld[j];
  double* A = st.L64 + st.leaf_off[j] + (int64_t)kb * ld + kb;
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) D[t / nb][t % nb] = A[(int64_t)(t / nb) * ld + t % nb];
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < nb; ++k) {
    if (threadIdx.x == 0) {
      const double d = D[k][k];
      if (!(d > 0.0)) bad = 1;
      D[k][k] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    if (bad) break;
    const double inv = 1.0 / D[k][k];
    for (int i = k + 1 + threadIdx.x; i < nb; i += blockDim.x) D[i][k] *= inv;
    __syncthreads();
    for (int t = threadIdx.x; t < (nb - k - 1) * (nb - k - 1); t += blockDim.x) {
      const int i = k + 1 + t / (nb - k - 1), c = k + 1 + t % (nb - k - 1);
      if (c <= i) D[i][c] -= D[i][k] * D[c][k];
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) atomicExch(st.status, DEV_SINGULAR);
    return;
  }
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int i = t / nb, c = t % nb;
    if (c <= i) A[(int64_t)i * ld + c] = D[i][c];
  }
}

// rows r >= kb + nb of the panel: L[r, kb:kb+nb] = A[r, kb:kb+nb] L_kk^-T (forward substitution,
// one row per thread, the panel rows staged in shared memory)
__global__ void __launch_bounds__(kCholRows) k_chol_panel(DStore st, const int* leaves, int kb) {
  __shared__ double Lk[kCholNb][kCholNb + 1];
  extern __shared__ double P[];   // [kCholRows][kCholNb + 1]
  if (*st.status != DEV_OK) return;
  const int j = leaves[blockIdx.x];
  const int node = st.leaf_node[j];
  const int b = st.hi[node] - st.lo[node];
  if (kb >= b) return;
  const int nb = min(kCholNb, b - kb);
  const int r0 = kb + nb + blockIdx.y * kCholRows;
  if (r0 >= b) return;
  const int nr = min(kCholRows, b - r0);
  const int ld = st.leaf_ld[j];
  double* A = st.L64 + st.leaf_off[j];
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int i = t / nb, c = t % nb;
    Lk[i][c] = c <= i ? A[(int64_t)(kb + i) * ld + kb + c] : 0.0;
  }
  for (int t = threadIdx.x; t < nr * nb; t += blockDim.x)
    P[(t / nb) * (kCholNb + 1) + t % nb] = A[(int64_t)(r0 + t / nb) * ld + kb + t % nb];
  __syncthreads();
  if ((int)threadIdx.x < nr) {
    double* x = P + threadIdx.x * (kCholNb + 1);
    for (int c = 0; c < nb; ++c) {
      double v = x[c];
      for (int m = 0; m < c; ++m) v -= x[m] * Lk[c][m];
      x[c] = v / Lk[c][c];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nr * nb; t += blockDim.x)
    A[(int64_t)(r0 + t / nb) * ld + kb + t % nb] = P[(t / nb) * (kCholNb + 1) + t % nb];
}

// trailing update A[r, c] -= L[r, panel] . L[c, panel] for kb + nb <= c <= r, tile (ti, tj) of 64
// x 64 with ti >= tj (blockIdx.y enumerates the lower-triangle tiles)
__global__ void __launch_bounds__(256) k_chol_update(DStore st, const int* leaves, int kb) {
  extern __shared__ double upd_sm[];   // Lr, Lc: [64][kCholNb + 1] each
  double (*Lr)[kCholNb + 1] = reinterpret_cast<double (*)[kCholNb + 1]>(upd_sm);
  double (*Lc)[kCholNb + 1] = reinterpret_cast<double (*)[kCholNb + 1]>(upd_sm + 64 * (kCholNb + 1));
  if (*st.status != DEV_OK) return;
  const int j = leaves[blockIdx.x];
  const int node = st.leaf_node[j];
  const int b = st.hi[node] - st.lo[node];
  const int t0 = kb + kCholNb;
  if (t0 >= b) return;
  const int nt = (b - t0 + 63) / 64;
  int ti = 0, rem = blockIdx.y;
  while (rem > ti) {
    rem -= ti + 1;
    ++ti;
  }
  const int tj = rem;
  if (ti >= nt) return;
  const int ld = st.leaf_ld[j];
  double* A = st.L64 + st.leaf_off[j];
  const int r0 = t0 + 64 * ti, c0 = t0 + 64 * tj;
  const int nr = min(64, b - r0), nc = min(64, b - c0);
  for (int t = threadIdx.x; t < 64 * kCholNb; t += blockDim.x) {
    const int i = t / kCholNb, m = t % kCholNb;
    Lr[i][m] = i < nr ? A[(int64_t)(r0 + i) * ld + kb + m] : 0.0;
    Lc[i][m] = i < nc ? A[(int64_t)(c0 + i) * ld + kb + m] : 0.0;
  }
  __syncthreads();
  // thread: 4 x 4 outputs (rows ty + 16 u, columns tx + 16 v)
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
  for (int m = 0; m < kCholNb; ++m) {
    double a[4], c[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a[u] = Lr[ty + 16 * u][m];
      c[u] = Lc[tx + 16 * u][m];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * c[v];
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int r = ty + 16 * u, c = tx + 16 * v;
      if (r < nr && c < nc && r0 + r >= c0 + c) A[(int64_t)(r0 + r) * ld + c0 + c] -= acc[u][v];
    }
}

// W = L^{-1} by forward substitution, one CTA per (leaf, COLS columns): the block's columns of W
// stay in shared memory while the rows are swept in order. Each column has 256 / COLS lanes of one
// warp, which split the dot product L[i, col:i] . W[col:i, col] and add the parts by shuffles, so a
// warp needs no barrier but its own. The inverse's FP64 work is spread over ceil(b / COLS) CTAs
// per leaf instead of one thread per column walking global memory.
template <int COLS>
__global__ void __launch_bounds__(256) k_trinv_block(DStore st, double* __restrict__ W, const int* leaves) {
  constexpr int LPC = 256 / COLS;   // lanes per column (16 or 32)
  static_assert(LPC == 16 || LPC == 32, "columns per CTA: 16 or 8");
  extern __shared__ double xs[];   // [b][COLS]
  const int j = leaves[blockIdx.x];
  const int node = st.leaf_node[j];
  const int b = st.hi[node] - st.lo[node];
  const int ld = st.leaf_ld[j];
  const int c0 = blockIdx.y * COLS;
  if (c0 >= b) return;
  const double* A = st.L64 + st.leaf_off[j];
  double* X = W + st.leaf_off[j];
  const int cl = threadIdx.x / LPC, part = threadIdx.x % LPC;   // local column, part of the dot product
  const int col = c0 + cl;
  for (int i = c0; i < b; ++i) {
    const double* Ai = A + (int64_t)i * ld;
    double s = 0.0;
    if (col < b && i > col)
      for (int k = col + part; k < i; k += LPC) s += Ai[k] * xs[k * COLS + cl];
#pragma unroll
    for (int o = LPC / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (col < b && part == 0) xs[i * COLS + cl] = i < col ? 0.0 : ((i == col ? 1.0 : 0.0) - s) / Ai[i];
    __syncwarp();
  }
  __syncthreads();
  for (int t = threadIdx.x; t < b * COLS; t += blockDim.x) {
    const int i = t / COLS, c = c0 + t % COLS;
    if (c < b) X[(int64_t)i * ld + c] = i < c0 ? 0.0 : xs[t];
  }
}

// G_jj^{-1} = W^T W (row i per CTA, j <= i by threads), written symmetric: the leaf inverse of
// Algorithm 1 (Sec. III-B).
__global__ void k_wtw(DStore st, const double* __restrict__ W, const int* leaves) {
  const int j = leaves[blockIdx.x];
  const int node = st.leaf_node[j];
  const int b = st.hi[node] - st.lo[node];
  const int i = blockIdx.y;
  if (i >= b) return;
  const int ld = st.leaf_ld[j];
  double* A = st.L64 + st.leaf_off[j];
  const double* X = W + st.leaf_off[j];
  for (int c = threadIdx.x; c <= i; c += blockDim.x) {
    double s = 0.0;
    for (int k = i; k < b; ++k) s += X[(int64_t)k * ld + i] * X[(int64_t)k * ld + c];
    A[(int64_t)i * ld + c] = s;
    A[(int64_t)c * ld + i] = s;
  }
}

// ------------------------------------------------------------------ factors (Eq. 9)
__global__ void k_zero_factor(DStore st, const int* nodes) {
  const int p = nodes[blockIdx.x];
  const int64_t cnt = (int64_t)(st.hi[p] - st.lo[p]) * st.node_kld[p];
  double* F = st.F64 + st.node_foff[p];
  for (int64_t t = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.y * blockDim.x)
    F[t] = 0.0;
}

// Leaf stage of [P; Q] = blkdiag(Ginv_l, Ginv_r)[h_l; h_r]: column e of h_l is -g_e e_a, so its
// leaf-stage image is -g_e times column a of the leaf inverse holding a (rows of that leaf only);
// a block column sums its W entries (the W vertices of one group share a leaf).
__global__ void k_factor_init(DStore st, const int* nodes) {
  const int p = nodes[blockIdx.x];
  const int e = blockIdx.y;
  const int k = st.node_k[p];
  if (e >= k) return;
  const int side = blockIdx.z;
  const int c0 = st.cut_ptr[p];
  const int pos = side == 0 ? st.cut_a[c0 + e] : st.cut_b[c0 + e];
  const int W = side == 0 ? st.cut_w : 1;
  const int jl = st.pos_leaf[pos];
  const int ln = st.leaf_node[jl];
  const int llo = st.lo[ln], b = st.hi[ln] - llo, ld = st.leaf_ld[jl];
  const double* Lrow = st.L64 + st.leaf_off[jl] + (int64_t)(pos - llo) * ld;   // symmetric: row = column
  double* F = st.F64 + st.node_foff[p];
  const int kld = st.node_kld[p];
  const int plo = st.lo[p];
  for (int r = threadIdx.x; r < b; r += blockDim.x) {
    double v;
    if (side == 0) {
      v = 0.0;
      for (int w = 0; w < W; ++w) v += -st.cut_g[(int64_t)(c0 + e) * W + w] * Lrow[(int64_t)w * ld + r];
    } else {
      v = Lrow[r];
    }
    F[(int64_t)(llo - plo + r) * kld + e] = v;
  }
}

struct Panel {
  double* ptr;
  int lo, ncols, ld;
};

__device__ __forceinline__ bool panel_of(const DStore& st, int q, int modeB, const int* flag, int d, double* Ybase,
                                         int m, int ldY, Panel& pn) {
  if (modeB == 0) {
    const int p = anc_at_depth(st, q, d);
    if (!flag[p]) return false;
    pn.ptr = st.F64 + st.node_foff[p];
    pn.lo = st.lo[p];
    pn.ncols = st.node_k[p];
    pn.ld = st.node_kld[p];
  } else {
    pn.ptr = Ybase;
    pn.lo = 0;
    pn.ncols = m;
    pn.ld = ldY;
  }
  return true;
}

// Panel columns per CTA of the level sweep for a level whose widest cut has kq columns: kPanelCols
// while the 2 kq x columns staging block fits the opt-in shared memory, fewer for wide cuts
int level_sweep_cols(int kq) {
  int dev = 0, optin = 0;
  EMT_CUDA(cudaGetDevice(&dev));
  EMT_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const int fit = (int)((size_t)optin / ((size_t)2 * std::max(kq, 1) * sizeof(double)));
  EMT_REQUIRE(fit >= 1, EMT_ERR_UNSUPPORTED, "cut too wide for the level sweep's shared memory");
  return std::min(kPanelCols, fit);
}

// Boundary projections of one internal node q on a panel: t = [h_l^T y_l; h_r^T y_r] is a
// gather of the (already corrected) panel rows at q's cut endpoints; s = C_q t.
__global__ void k_level_sweep(DStore st, int modeB, const int* flag, int d, int dq, double* Ybase, int m, int ldY,
                              double* __restrict__ scratch, int mcols, int pc) {
  extern __shared__ double tsh[];
  const int q = st.lvl_nodes[st.lvl_ptr[dq] + blockIdx.x];
  Panel pn;
  if (!panel_of(st, q, modeB, flag, d, Ybase, m, ldY, pn)) return;
  const int kq = st.node_k[q];
  if (kq == 0) return;
  const int c0 = blockIdx.y * pc;   // pc panel columns per CTA (kPanelCols, fewer for wide cuts)
  if (c0 >= pn.ncols) return;
  const int nc = min(pc, pn.ncols - c0);
  const int m2 = 2 * kq;
  const int cp = st.cut_ptr[q];
  for (int t = threadIdx.x; t < m2 * nc; t += blockDim.x) {
    const int r = t / nc, c = t % nc;
    double v;
    if (r < kq) {
      const int W = st.cut_w;
      const double* row = pn.ptr + (int64_t)(st.cut_a[cp + r] - pn.lo) * pn.ld + c0 + c;
      v = 0.0;
      for (int w = 0; w < W; ++w) v += -st.cut_g[(int64_t)(cp + r) * W + w] * row[(int64_t)w * pn.ld];
    } else {
      v = pn.ptr[(int64_t)(st.cut_b[cp + r - kq] - pn.lo) * pn.ld + c0 + c];
    }
    tsh[r * pc + c] = v;
  }
  __syncthreads();
  const double* C = st.C64 + st.node_coff[q];
  double* S = scratch + (int64_t)st.node_soff[q] * mcols;
  for (int t = threadIdx.x; t < m2 * nc; t += blockDim.x) {
    const int r = t / nc, c = t % nc;
    double s = 0.0;
    for (int e2 = 0; e2 < m2; ++e2) s += C[r * m2 + e2] * tsh[e2 * pc + c];
    S[(int64_t)r * mcols + c0 + c] = s;
  }
}

// Correction of node q on its rows: Y[i] -= F_q[i] . s_q(half of i).
__global__ void k_level_expand(DStore st, int modeB, const int* flag, int d, int dq, double* Ybase, int m, int ldY,
                               const double* __restrict__ scratch, int mcols, int rows_per_block) {
  const int q = st.lvl_nodes[st.lvl_ptr[dq] + blockIdx.x];
  Panel pn;
  if (!panel_of(st, q, modeB, flag, d, Ybase, m, ldY, pn)) return;
  const int kq = st.node_k[q];
  if (kq == 0) return;
  const int qlo = st.lo[q], qhi = st.hi[q];
  const int r0 = qlo + blockIdx.y * rows_per_block;
  if (r0 >= qhi) return;
  const int r1 = min(qhi, r0 + rows_per_block);
  const int split = st.hi[st.left[q]];
  const double* F = st.F64 + st.node_foff[q];
  const int kld = st.node_kld[q];
  const double* S = scratch + (int64_t)st.node_soff[q] * mcols;
  const int nrow = r1 - r0;
  for (int t = threadIdx.x; t < nrow * pn.ncols; t += blockDim.x) {
    const int i = r0 + t / pn.ncols, c = t % pn.ncols;
    const int half = i < split ? 0 : kq;
    const double* Fi = F + (int64_t)(i - qlo) * kld;
    double acc = 0.0;
    for (int e = 0; e < kq; ++e) acc += Fi[e] * S[(int64_t)(half + e) * mcols + c];
    pn.ptr[(int64_t)(i - pn.lo) * pn.ld + c] -= acc;
  }
}

// Leaf stage of a dense multi-vector apply (Eq. 2 with Sec. III's leaf blocks): Y[i] = L_j X[leaf
// rows] (row-major panels).
__global__ void k_leaf_dense(DStore st, const double* __restrict__ X, double* __restrict__ Y, int m, int ld) {
  const int i = blockIdx.x;
  const int j = st.pos_leaf[i];
  const int ln = st.leaf_node[j];
  const int llo = st.lo[ln], b = st.hi[ln] - llo, lld = st.leaf_ld[j];
  const double* Lr = st.L64 + st.leaf_off[j] + (int64_t)(i - llo) * lld;
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    double acc = 0.0;
    for (int r = 0; r < b; ++r) acc += Lr[r] * X[(int64_t)(llo + r) * ld + c];
    Y[(int64_t)i * ld + c] = acc;
  }
}

// ------------------------------------------------------------------ node cores
// Core of each node (Sec. III): PAPER mode C = [[0, I], [I, 0]] (Eq. 9's M = -P Q^T); EXACT mode
// C = S^{-1}, S = [[h_l^T P, I], [I, h_r^T Q]] (the Woodbury form of Eq. 3's split), inverted by
// Gauss-Jordan with partial pivoting in FP64.
// ws: null (the core is inverted in shared memory), or a workspace of ws_stride doubles and
// ws_stride / m2max pivots per CTA in global memory for cores larger than kMaxCoreDim.
__global__ void k_core(DStore st, const int* nodes, int mode, double* ws, int* ws_piv, int64_t ws_stride,
                       int m2max) {
  extern __shared__ double A_sh[];
  __shared__ int ipiv_sh[kMaxCoreDim];
  __shared__ int prow;
  __shared__ double pval;
  double* A = ws ? ws + blockIdx.x * ws_stride : A_sh;
  int* ipiv = ws ? ws_piv + (int64_t)blockIdx.x * m2max : ipiv_sh;
  const int p = nodes[blockIdx.x];
  const int k = st.node_k[p];
  const int m2 = 2 * k;
  if (k == 0) return;
  double* C = st.C64 + st.node_coff[p];
  if (mode == EMT_MODE_PAPER) {
    for (int t = threadIdx.x; t < m2 * m2; t += blockDim.x) {
      const int r = t / m2, c = t % m2;
      C[t] = (c == (r + k) % m2) ? 1.0 : 0.0;
    }
    return;
  }
  const double* F = st.F64 + st.node_foff[p];
  const int kld = st.node_kld[p];
  const int plo = st.lo[p];
  const int cp = st.cut_ptr[p];
  for (int t = threadIdx.x; t < m2 * m2; t += blockDim.x) {
    const int r = t / m2, c = t % m2;
    double v = 0.0;
    if (r < k && c < k) {
      const int W = st.cut_w;
      for (int w = 0; w < W; ++w)
        v += -st.cut_g[(int64_t)(cp + r) * W + w] * F[(int64_t)(st.cut_a[cp + r] + w - plo) * kld + c];
    } else if (r >= k && c >= k) v = F[(int64_t)(st.cut_b[cp + r - k] - plo) * kld + (c - k)];
    else if (c == r + k || r == c + k) v = 1.0;
    A[t] = v;
  }
  __syncthreads();
  // in-place Gauss-Jordan inversion with partial pivoting
  for (int kk = 0; kk < m2; ++kk) {
    if (threadIdx.x == 0) {
      int best = kk;
      double bv = fabs(A[kk * m2 + kk]);
      for (int r = kk + 1; r < m2; ++r) {
        const double v = fabs(A[r * m2 + kk]);
        if (v > bv) { bv = v; best = r; }
      }
      prow = best;
      ipiv[kk] = best;
    }
    __syncthreads();
    if (prow != kk)
      for (int c = threadIdx.x; c < m2; c += blockDim.x) {
        const double tmp = A[kk * m2 + c];
        A[kk * m2 + c] = A[prow * m2 + c];
        A[prow * m2 + c] = tmp;
      }
    __syncthreads();
    if (threadIdx.x == 0) {
      pval = A[kk * m2 + kk];
      if (!(fabs(pval) > 1e-300)) atomicExch(st.status, DEV_SINGULAR);
      A[kk * m2 + kk] = 1.0;
    }
    __syncthreads();
    const double inv = 1.0 / pval;
    for (int c = threadIdx.x; c < m2; c += blockDim.x) A[kk * m2 + c] *= inv;
    __syncthreads();
    for (int t = threadIdx.x; t < m2 * m2; t += blockDim.x) {
      const int r = t / m2, c = t % m2;
      if (r == kk || c == kk) continue;
      A[r * m2 + c] -= A[r * m2 + kk] * A[kk * m2 + c];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < m2; r += blockDim.x)
      if (r != kk) A[r * m2 + kk] = -A[r * m2 + kk] * A[kk * m2 + kk];
    __syncthreads();
  }
  for (int kk = m2 - 1; kk >= 0; --kk) {
    const int pr = ipiv[kk];
    if (pr != kk)
      for (int r = threadIdx.x; r < m2; r += blockDim.x) {
        const double tmp = A[r * m2 + kk];
        A[r * m2 + kk] = A[r * m2 + pr];
        A[r * m2 + pr] = tmp;
      }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < m2 * m2; t += blockDim.x) C[t] = A[t];
}

// ------------------------------------------------------------------ precision copies
// Float-float and FP32 copies of the FP64 store that the apply kernels read.
__global__ void k_pack(const double* __restrict__ src, float2* __restrict__ ff, float* __restrict__ f32, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double x = src[t];
    const float hi = (float)x;
    const float lo = (float)(x - (double)hi);
    ff[t] = make_float2(hi, lo);
    f32[t] = hi;
  }
}

// ------------------------------------------------------------------ exact local modification
// Sec. IV: G' = G + delta u u^T, applied exactly at every node on the paths from the touched leaves
// to the root (Sherman-Morrison with the old store's z). z of one path node q: leaf -> columns of the leaf inverse; internal ->
// z_q = [x_l; x_r] - Y S^{-1} [h_l^T x_l; h_r^T x_r] (old store), then d_q = 1 + delta u_q^T z_q.
struct ModItem {
  int node, is_leaf;
  int zoff, zl, zr;        // this node's z slot; children's slots (-1 if the child is unchanged)
  int dslot, dl, dr;
  int pa, pb;              // positions with u = e_pa - e_pb (-1 = absent)
};

__global__ void k_mod_z(DStore st, ModItem it, double* __restrict__ z, double* __restrict__ dv, double delta) {
  extern __shared__ double sh[];
  const int q = it.node;
  const int qlo = st.lo[q], n = st.hi[q] - qlo;
  double* zq = z + it.zoff;
  if (it.is_leaf) {
    const int j = st.node_leaf[q];
    const int ld = st.leaf_ld[j];
    const double* L = st.L64 + st.leaf_off[j];
    const bool ha = it.pa >= qlo && it.pa < qlo + n, hb = it.pb >= qlo && it.pb < qlo + n;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
      double v = 0.0;
      if (ha) v += L[(int64_t)(it.pa - qlo) * ld + r];
      if (hb) v -= L[(int64_t)(it.pb - qlo) * ld + r];
      zq[r] = v;
    }
    return;
  }
  const int k = st.node_k[q], m2 = 2 * k;
  const int l = st.left[q], r = st.right[q];
  const int llo = st.lo[l], rlo = st.lo[r];
  const int cp = st.cut_ptr[q];
  double* t = sh;          // 2k
  double* sg = sh + m2;    // 2k
  for (int e = threadIdx.x; e < m2; e += blockDim.x) {
    double v = 0.0;
    if (e < k) {
      if (it.zl >= 0)
        for (int w = 0; w < st.cut_w; ++w)
          v += -st.cut_g[(int64_t)(cp + e) * st.cut_w + w] * z[it.zl + st.cut_a[cp + e] + w - llo];
    } else {
      if (it.zr >= 0) v = z[it.zr + st.cut_b[cp + e - k] - rlo];
    }
    t[e] = v;
  }
  __syncthreads();
  const double* C = st.C64 + st.node_coff[q];
  for (int e = threadIdx.x; e < m2; e += blockDim.x) {
    double s = 0.0;
    for (int f = 0; f < m2; ++f) s += C[e * m2 + f] * t[f];
    sg[e] = s;
  }
  __syncthreads();
  const double* F = st.F64 + st.node_foff[q];
  const int kld = st.node_kld[q];
  const int split = rlo - qlo;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double base = 0.0;
    const double* s_half;
    if (i < split) {
      if (it.zl >= 0) base = z[it.zl + i];
      s_half = sg;
    } else {
      if (it.zr >= 0) base = z[it.zr + i - split];
      s_half = sg + k;
    }
    double acc = 0.0;
    for (int e = 0; e < k; ++e) acc += F[(int64_t)i * kld + e] * s_half[e];
    zq[i] = base - acc;
  }
}

// d_q = 1 + delta u_q^T z_q in FP64 (Sherman-Morrison, Sec. IV); a non-positive d would make G'
// indefinite and is reported as DEV_SINGULAR.
__global__ void k_mod_denominator(DStore st, ModItem it, const double* __restrict__ z, double* __restrict__ dv,
                                  double delta) {
  const int q = it.node;
  const int qlo = st.lo[q], qhi = st.hi[q];
  double ut = 0.0;
  if (it.pa >= qlo && it.pa < qhi) ut += z[it.zoff + it.pa - qlo];
  if (it.pb >= qlo && it.pb < qhi) ut -= z[it.zoff + it.pb - qlo];
  const double d = 1.0 + delta * ut;
  dv[it.dslot] = d;
  if (!(d > 1e-12)) atomicExch(st.status, DEV_SINGULAR);
}

// Rank-one update of a touched leaf inverse: L_j' = L_j - (delta/d) z z^T (Sherman-Morrison on the
// leaf block, Sec. IV).
__global__ void k_mod_leaf(DStore st, ModItem it, const double* __restrict__ z, const double* __restrict__ dv,
                           double delta) {
  if (*st.status != DEV_OK) return;
  const int q = it.node;
  const int j = st.node_leaf[q];
  const int n = st.hi[q] - st.lo[q], ld = st.leaf_ld[j];
  double* L = st.L64 + st.leaf_off[j];
  const double* zq = z + it.zoff;
  const double f = delta / dv[it.dslot];
  for (int r = blockIdx.x; r < n; r += gridDim.x) {
    const double zr = f * zq[r];
    for (int c = threadIdx.x; c < n; c += blockDim.x) L[(int64_t)r * ld + c] -= zr * zq[c];
  }
}

// P' = P - (delta/d_l) x_l (h_l^T x_l)^T, Q' likewise; at the LCA of a cross-leaf branch the cut
// column ec becomes -g_new Ginv_l'^{-1} e_a = -g_new x_l / d_l (x_l = Ginv_l e_a).
__global__ void k_mod_factor(DStore st, ModItem it, const double* __restrict__ z, const double* __restrict__ dv,
                             double delta, int ec, double g_new) {
  if (*st.status != DEV_OK) return;
  extern __shared__ double w[];
  const int q = it.node;
  const int k = st.node_k[q];
  if (k == 0) return;
  const int l = st.left[q], r = st.right[q];
  const int qlo = st.lo[q], llo = st.lo[l], rlo = st.lo[r], n = st.hi[q] - qlo;
  const int cp = st.cut_ptr[q];
  for (int e = threadIdx.x; e < 2 * k; e += blockDim.x) {
    double v = 0.0;
    if (e < k) {
      if (it.zl >= 0)
        for (int w = 0; w < st.cut_w; ++w)
          v += -st.cut_g[(int64_t)(cp + e) * st.cut_w + w] * z[it.zl + st.cut_a[cp + e] + w - llo];
    } else {
      if (it.zr >= 0) v = z[it.zr + st.cut_b[cp + e - k] - rlo];
    }
    w[e] = v;
  }
  __syncthreads();
  const double fl = it.zl >= 0 ? delta / dv[it.dl] : 0.0;
  const double fr = it.zr >= 0 ? delta / dv[it.dr] : 0.0;
  double* F = st.F64 + st.node_foff[q];
  const int kld = st.node_kld[q];
  const int split = rlo - qlo;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * k; t += gridDim.x * blockDim.x) {
    const int i = t / k, e = t % k;
    double* Fi = F + (int64_t)i * kld;
    if (i < split) {
      if (it.zl < 0) continue;
      const double xi = z[it.zl + i];
      if (e == ec) {
        // h_l' = h_l - delta e_a e_ec^T: with Ginv_l' = Ginv_l - (delta/d_l) x x^T the column becomes
        // P e_ec - (delta/d_l) x (w_ec + 1); a one-entry column (cut_w 1) is set directly
        if (st.cut_w == 1) Fi[e] = -g_new * xi / dv[it.dl];
        else Fi[e] -= fl * xi * (w[e] + 1.0);
      } else {
        Fi[e] -= fl * xi * w[e];
      }
    } else {
      if (it.zr < 0) continue;
      const double xi = z[it.zr + i - split];
      Fi[e] -= fr * xi * w[k + e];
    }
  }
}

// New conductance of a cut column after a change of its branch (Sec. IV).
__global__ void k_set_cut_g(DStore st, int idx, double g) {
  if (*st.status != DEV_OK) return;
  st.cut_g[idx] = g;
}

// G' = G + delta u u^T on the CSR copy (Sec. IV): up to four entries change.
__global__ void k_csr_add(double* val, int i0, int i1, int i2, int i3, double d0, double d1, double d2, double d3,
                          const int* status) {
  if (*status != DEV_OK) return;
  if (i0 >= 0) val[i0] += d0;
  if (i1 >= 0) val[i1] += d1;
  if (i2 >= 0) val[i2] += d2;
  if (i3 >= 0) val[i3] += d3;
}

int grid_for(int64_t n, int threads, int cap = 4096) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace

// ====================================================================== Store (host side)
Store::Store(const emt_graph* g, const emt_hinv_opts* o, cudaStream_t s) {
  EMT_REQUIRE(g && o, EMT_ERR_INVALID, "null graph or options");
  EMT_REQUIRE(g->n_bus >= 1 && g->n_branch >= 0, EMT_ERR_INVALID, "bad graph sizes");
  EMT_REQUIRE(g->n_branch == 0 || (g->from && g->to && g->g), EMT_ERR_INVALID, "null branch arrays");
  EMT_REQUIRE(o->mode == EMT_MODE_EXACT || o->mode == EMT_MODE_PAPER, EMT_ERR_INVALID, "bad mode");
  EMT_REQUIRE(o->precision >= EMT_PREC_FP64 && o->precision <= EMT_PREC_FP32, EMT_ERR_INVALID, "bad precision");
  for (int e = 0; e < g->n_branch; ++e) {
    EMT_REQUIRE(g->from[e] >= 0 && g->from[e] < g->n_bus && g->to[e] >= -1 && g->to[e] < g->n_bus,
                EMT_ERR_INVALID, "branch endpoint out of range");
    EMT_REQUIRE(g->from[e] != g->to[e], EMT_ERR_INVALID, "self-loop branch");
    // negative values carry mutual couplings (three-phase branches); G must stay positive definite,
    // which the leaf factorisations check
    EMT_REQUIRE(std::isfinite(g->g[e]) && g->g[e] != 0.0, EMT_ERR_INVALID, "branch conductance must be nonzero");
  }
  mode = o->mode;
  precision = o->precision;
  n = g->n_bus;
  g_from.assign(g->from, g->from + g->n_branch);
  g_to.assign(g->to, g->to + g->n_branch);
  g_val.assign(g->g, g->g + g->n_branch);
  EMT_REQUIRE(o->nodes_per_bus >= 0, EMT_ERR_INVALID, "nodes_per_bus must be >= 0");
  tree = o->nodes_per_bus >= 2 ? build_block_tree(n, g->n_branch, g->from, g->to, o->nodes_per_bus, o->levels, o->d_th)
                               : build_tree(n, g->n_branch, g->from, g->to, o->levels, o->d_th);
  build_csr();
  EMT_CUDA(cudaGetDevice(&device));   // first device call: every host-side check has passed
  setup_layout(s);
}

Store::~Store() {}

void Store::build_csr() {
  // position-ordered CSR of G; each entry is the sum of its contributions in branch order
  // (deterministic): contributions are bucketed by row in that order, sorted by column with a
  // stable insertion sort (rows hold a handful of entries) and summed from 0 per (row, column)
  struct Contrib {
    int col;
    double v;
  };
  const size_t m = g_from.size();
  std::vector<int> cnt(n + 1, 0);
  for (int i = 0; i < n; ++i) cnt[i + 1] += 1;   // the diagonal exists even without branches
  for (size_t e = 0; e < m; ++e) {
    cnt[tree.pos[g_from[e]] + 1] += g_to[e] >= 0 ? 2 : 1;
    if (g_to[e] >= 0) cnt[tree.pos[g_to[e]] + 1] += 2;
  }
  for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  std::vector<Contrib> all(cnt[n]);
  std::vector<int> fill(cnt.begin(), cnt.end() - 1);
  for (int i = 0; i < n; ++i) all[fill[i]++] = {i, 0.0};
  for (size_t e = 0; e < m; ++e) {
    const int a = tree.pos[g_from[e]];
    const double gv = g_val[e];
    all[fill[a]++] = {a, gv};
    if (g_to[e] >= 0) {
      const int b = tree.pos[g_to[e]];
      all[fill[b]++] = {b, gv};
      all[fill[a]++] = {b, -gv};
      all[fill[b]++] = {a, -gv};
    }
  }
  csr_ptr.assign(n + 1, 0);
  csr_col.clear();
  csr_val.clear();
  for (int i = 0; i < n; ++i) {
    Contrib* r = all.data() + cnt[i];
    const int len = cnt[i + 1] - cnt[i];
    for (int x = 1; x < len; ++x) {   // stable: equal columns keep their branch order
      const Contrib c = r[x];
      int y = x - 1;
      for (; y >= 0 && r[y].col > c.col; --y) r[y + 1] = r[y];
      r[y + 1] = c;
    }
    for (int x = 0; x < len;) {
      double sum = 0.0;
      int y = x;
      for (; y < len && r[y].col == r[x].col; ++y) sum += r[y].v;
      csr_col.push_back(r[x].col);
      csr_val.push_back(sum);
      x = y;
    }
    csr_ptr[i + 1] = (int)csr_col.size();
  }
}

void Store::setup_layout(cudaStream_t s) {
  const Tree& t = tree;
  const int nn = t.n_node();
  leaf_nodes_h = t.leaves;
  n_leaf = (int)leaf_nodes_h.size();
  node_leaf_h.assign(nn, -1);
  for (int j = 0; j < n_leaf; ++j) node_leaf_h[leaf_nodes_h[j]] = j;
  std::vector<int32_t> pos_leaf(n);
  leaf_ld_h.resize(n_leaf);
  leaf_off_h.resize(n_leaf);
  int64_t off = 0;
  for (int j = 0; j < n_leaf; ++j) {
    const int p = leaf_nodes_h[j];
    const int b = t.hi[p] - t.lo[p];
    leaf_ld_h[j] = (b + 3) / 4 * 4;
    leaf_off_h[j] = off;
    off += (int64_t)b * leaf_ld_h[j];
    for (int i = t.lo[p]; i < t.hi[p]; ++i) pos_leaf[i] = j;
  }
  L_elems = off;
  // internal nodes by depth (deepest first order is handled by callers)
  node_k_h.assign(nn, 0);
  node_kld_h.assign(nn, 0);
  node_soff_h.assign(nn, 0);
  node_foff_h.assign(nn, 0);
  node_coff_h.assign(nn, 0);
  lvl_ptr_h.assign(t.max_depth + 2, 0);
  std::vector<std::vector<int>> by_depth(t.max_depth + 1);
  for (int p = 0; p < nn; ++p)
    if (t.left[p] >= 0) by_depth[t.depth[p]].push_back(p);
  lvl_nodes_h.clear();
  for (int d = 0; d <= t.max_depth; ++d) {
    lvl_ptr_h[d] = (int)lvl_nodes_h.size();
    for (int p : by_depth[d]) lvl_nodes_h.push_back(p);
  }
  lvl_ptr_h[t.max_depth + 1] = (int)lvl_nodes_h.size();
  n_internal = (int)lvl_nodes_h.size();
  kmax = 0;
  int64_t foff = 0, coff = 0;
  int soff = 0;
  for (int d = t.max_depth; d >= 0; --d) {     // deepest level first: each depth contiguous
    for (int p : by_depth[d]) {
      const int k = t.cut_ptr[p + 1] - t.cut_ptr[p];
      EMT_REQUIRE(2 * k <= kMaxCoreDimWs, EMT_ERR_UNSUPPORTED,
                  "a tree node cuts more than 2048 branches; use more levels or a smaller d_th");
      node_k_h[p] = k;
      node_kld_h[p] = (k + 3) / 4 * 4;   // 16-byte rows in every precision
      node_foff_h[p] = foff;
      foff += (int64_t)(t.hi[p] - t.lo[p]) * node_kld_h[p];
      node_coff_h[p] = coff;
      coff += (int64_t)4 * k * k;
      node_soff_h[p] = soff;
      soff += 2 * k;
      kmax = std::max(kmax, k);
    }
  }
  F_elems = foff;
  C_elems = coff;
  s_total = soff;
  if (t.cut_w == 1) {
    cut_g_h.resize(t.cut_e.size());
    for (size_t c = 0; c < t.cut_e.size(); ++c) cut_g_h[c] = g_val[t.cut_e[c]];
  } else {
    // block cuts: entry (c, w) is -G[cut_a + w, cut_b], the conductance of the branches joining
    // the two vertices (each joined pair is cut at exactly one tree node, its LCA)
    const int W = t.cut_w;
    cut_g_h.assign(t.cut_b.size() * W, 0.0);
    std::map<std::pair<int, int>, int64_t> at;
    for (size_t c = 0; c < t.cut_b.size(); ++c)
      for (int w = 0; w < W; ++w) at[{t.cut_a[c] + w, t.cut_b[c]}] = (int64_t)c * W + w;
    for (size_t e = 0; e < g_from.size(); ++e) {
      if (g_to[e] < 0) continue;
      const int x = t.pos[g_from[e]], y = t.pos[g_to[e]];
      auto it = at.find({x, y});
      if (it == at.end()) it = at.find({y, x});
      if (it != at.end()) cut_g_h[it->second] += g_val[e];
    }
  }
  // distinct cut endpoints for the fused sweep
  {
    // block cuts (cut_w = W > 1): a group's W positions (aligned to W) get W consecutive rows, so
    // the row of cut_a + w is the row of cut_a plus w
    const int W = t.cut_w;
    std::map<int, int> crow;
    CutRows cr;
    for (int d = t.max_depth; d >= 0; --d)
      for (int p : by_depth[d]) {
        const int k = node_k_h[p];
        for (int side = 0; side < 2; ++side)
          for (int e = 0; e < k; ++e) {
            const int pos_ = side == 0 ? t.cut_a[t.cut_ptr[p] + e] : t.cut_b[t.cut_ptr[p] + e];
            const int g0 = pos_ - pos_ % W;
            auto it = crow.find(g0);
            int ci;
            if (it == crow.end()) {
              ci = (int)cr.crow_pos.size();
              crow[g0] = ci;
              for (int w = 0; w < W; ++w) cr.crow_pos.push_back(g0 + w);
            } else {
              ci = it->second;
            }
            ci += pos_ - g0;
            cr.item_node.push_back(p);
            cr.item_pos.push_back(pos_);
            cr.item_crow.push_back(ci);
            cr.item_sidx.push_back(node_soff_h[p] + side * k + e);
          }
      }
    cr.n_items = (int)cr.item_node.size();
    cut_rows = cr;
  }
  // uploads
  d_lo.upload(t.lo, s);
  d_hi.upload(t.hi, s);
  d_parent.upload(t.parent, s);
  d_left.upload(t.left, s);
  d_right.upload(t.right, s);
  d_depth.upload(t.depth, s);
  d_node_leaf.upload(node_leaf_h, s);
  d_leaf_node.upload(leaf_nodes_h, s);
  d_pos_leaf.upload(pos_leaf, s);
  d_perm.upload(t.perm, s);
  d_ipos.upload(t.pos, s);
  d_leaf_ld.upload(leaf_ld_h, s);
  d_leaf_off.upload(leaf_off_h, s);
  d_node_k.upload(node_k_h, s);
  d_node_kld.upload(node_kld_h, s);
  d_node_foff.upload(node_foff_h, s);
  d_node_coff.upload(node_coff_h, s);
  d_node_soff.upload(node_soff_h, s);
  d_lvl_ptr.upload(lvl_ptr_h, s);
  d_lvl_nodes.upload(lvl_nodes_h, s);
  d_cut_ptr.upload(t.cut_ptr, s);
  d_cut_a.upload(t.cut_a, s);
  d_cut_b.upload(t.cut_b, s);
  d_cut_e.upload(t.cut_e, s);
  d_cut_g.upload(cut_g_h, s);
  d_csr_ptr.upload(csr_ptr, s);
  d_csr_col.upload(csr_col, s);
  d_csr_val.upload(csr_val, s);
  d_item_node.upload(cut_rows.item_node, s);
  d_item_pos.upload(cut_rows.item_pos, s);
  d_item_crow.upload(cut_rows.item_crow, s);
  d_item_sidx.upload(cut_rows.item_sidx, s);
  d_crow_pos.upload(cut_rows.crow_pos, s);
  L64.alloc(L_elems);
  Lff.alloc(L_elems);
  L32.alloc(L_elems);
  W64.alloc(L_elems);
  F64.alloc(F_elems);
  Fff.alloc(F_elems);
  F32.alloc(F_elems);
  C64.alloc(C_elems);
  Cff.alloc(C_elems);
  C32.alloc(C_elems);
  F64.zero(s);
  C64.zero(s);
  d_status.alloc(1);
  d_status.zero(s);
  d_list.alloc(std::max(nn, 16));
  d_flag.alloc(nn);
  scratch.alloc((size_t)std::max(s_total, 1) * std::max(kmax, kPanelCols));
  zbuf.alloc((size_t)(t.max_depth + 2) * 2 * n + 16);
  dbuf.alloc((size_t)(t.max_depth + 2) * 2 + 16);
}

DStore Store::view() const {
  DStore v;
  v.n = n;
  v.n_node = tree.n_node();
  v.n_leaf = n_leaf;
  v.max_depth = tree.max_depth;
  v.kmax = kmax;
  v.lo = d_lo.p;
  v.hi = d_hi.p;
  v.parent = d_parent.p;
  v.left = d_left.p;
  v.right = d_right.p;
  v.depth = d_depth.p;
  v.node_leaf = d_node_leaf.p;
  v.leaf_node = d_leaf_node.p;
  v.pos_leaf = d_pos_leaf.p;
  v.perm = d_perm.p;
  v.ipos = d_ipos.p;
  v.leaf_off = d_leaf_off.p;
  v.leaf_ld = d_leaf_ld.p;
  v.node_k = d_node_k.p;
  v.node_kld = d_node_kld.p;
  v.node_foff = d_node_foff.p;
  v.node_coff = d_node_coff.p;
  v.node_soff = d_node_soff.p;
  v.lvl_ptr = d_lvl_ptr.p;
  v.lvl_nodes = d_lvl_nodes.p;
  v.cut_ptr = d_cut_ptr.p;
  v.cut_a = d_cut_a.p;
  v.cut_b = d_cut_b.p;
  v.cut_e = d_cut_e.p;
  v.cut_g = d_cut_g.p;
  v.cut_w = tree.cut_w;
  v.L64 = L64.p;
  v.Lff = Lff.p;
  v.L32 = L32.p;
  v.F64 = F64.p;
  v.Fff = Fff.p;
  v.F32 = F32.p;
  v.C64 = C64.p;
  v.Cff = Cff.p;
  v.C32 = C32.p;
  v.status = d_status.p;
  return v;
}

int Store::upload_list(const std::vector<int>& v, cudaStream_t s) {
  EMT_REQUIRE(v.size() <= d_list.n, EMT_ERR_INVALID, "node list too long");
  // kernel arguments are copied at launch, but a list must live in device memory: stage it
  // through a pageable copy on the stream (ordered before the kernels that read it)
  EMT_CUDA(cudaMemcpyAsync(d_list.p, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  // a pageable copy returns once the source has been staged, so `v` may go out of scope
  return (int)v.size();
}

void Store::assemble_leaves(const std::vector<int>& leaves, cudaStream_t s) {
  if (leaves.empty()) return;
  const int nl = upload_list(leaves, s);
  DStore v = view();
  k_zero_leaf<<<nl, 256, 0, s>>>(v, d_list.p);
  k_assemble_leaf<<<nl, 256, 0, s>>>(v, d_csr_ptr.p, d_csr_col.p, d_csr_val.p, d_list.p);
  EMT_CUDA(cudaGetLastError());
}

void Store::invert_leaves(const std::vector<int>& leaves, cudaStream_t s) {
  if (leaves.empty()) return;
  const int nl = upload_list(leaves, s);
  DStore v = view();
  int bmax = 0;
  for (int j : leaves) bmax = std::max(bmax, tree.hi[leaf_nodes_h[j]] - tree.lo[leaf_nodes_h[j]]);
  // blocked Cholesky: panels of kCholNb columns (every launch sees the leaf list and skips leaves
  // already done)
  {
    const size_t shp = (size_t)kCholRows * (kCholNb + 1) * sizeof(double);
    if (shp > 48 * 1024)
      EMT_CUDA(cudaFuncSetAttribute(k_chol_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shp));
    const size_t shu = (size_t)2 * 64 * (kCholNb + 1) * sizeof(double);
    EMT_CUDA(cudaFuncSetAttribute(k_chol_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shu));
    for (int kb = 0; kb < bmax; kb += kCholNb) {
      k_chol_diag<<<nl, 256, 0, s>>>(v, d_list.p, kb);
      const int rest = bmax - kb - kCholNb;
      if (rest <= 0) continue;
      k_chol_panel<<<dim3(nl, (rest + kCholRows - 1) / kCholRows), kCholRows, shp, s>>>(v, d_list.p, kb);
      const int nt = (rest + 63) / 64;
      k_chol_update<<<dim3(nl, nt * (nt + 1) / 2), 256, shu, s>>>(v, d_list.p, kb);
    }
  }
  // 16 columns per CTA while their rows fit 200 KB of shared memory (leaves up to 1,600), else 8
  EMT_REQUIRE(bmax <= 3200, EMT_ERR_UNSUPPORTED, "leaf larger than 3200 nodes");
  if (bmax <= 1600) {
    const size_t shx = (size_t)bmax * 16 * sizeof(double);
    if (shx > 48 * 1024)
      EMT_CUDA(cudaFuncSetAttribute(k_trinv_block<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shx));
    k_trinv_block<16><<<dim3(nl, (bmax + 15) / 16), 256, shx, s>>>(v, W64.p, d_list.p);
  } else {
    const size_t shx = (size_t)bmax * 8 * sizeof(double);
    EMT_CUDA(cudaFuncSetAttribute(k_trinv_block<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shx));
    k_trinv_block<8><<<dim3(nl, (bmax + 7) / 8), 256, shx, s>>>(v, W64.p, d_list.p);
  }
  k_wtw<<<dim3(nl, bmax), 256, 0, s>>>(v, W64.p, d_list.p);
  EMT_CUDA(cudaGetLastError());
}

void Store::form_factors(const std::vector<int>& nodes, int d, cudaStream_t s) {
  if (nodes.empty()) return;
  int kb = 0, nmax = 0;
  for (int p : nodes) {
    kb = std::max(kb, node_k_h[p]);
    nmax = std::max(nmax, tree.hi[p] - tree.lo[p]);
  }
  if (kb == 0) return;
  const int nl = upload_list(nodes, s);
  DStore v = view();
  // flags of the batch
  std::vector<int> flag(tree.n_node(), 0);
  for (int p : nodes) flag[p] = 1;
  EMT_CUDA(cudaMemcpyAsync(d_flag.p, flag.data(), flag.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  k_zero_factor<<<dim3(nl, 64), 256, 0, s>>>(v, d_list.p);
  k_factor_init<<<dim3(nl, kb, 2), 256, 0, s>>>(v, d_list.p);
  const int mcols = std::max(kmax, kPanelCols);
  for (int dq = tree.max_depth - 1; dq > d; --dq) {
    const int cnt = lvl_ptr_h[dq + 1] - lvl_ptr_h[dq];
    if (cnt == 0) continue;
    int kq = 0, nq = 0;
    for (int i = lvl_ptr_h[dq]; i < lvl_ptr_h[dq + 1]; ++i) {
      kq = std::max(kq, node_k_h[lvl_nodes_h[i]]);
      nq = std::max(nq, tree.hi[lvl_nodes_h[i]] - tree.lo[lvl_nodes_h[i]]);
    }
    if (kq == 0) continue;
    const int pc = level_sweep_cols(kq);
    const size_t sh = (size_t)2 * kq * pc * sizeof(double);
    if (sh > 48 * 1024)
      EMT_CUDA(cudaFuncSetAttribute(k_level_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
    k_level_sweep<<<dim3(cnt, (kb + pc - 1) / pc), 256, sh, s>>>(v, 0, d_flag.p, d, dq, nullptr, 0, 0, scratch.p,
                                                                 mcols, pc);
    const int rpb = 64;
    k_level_expand<<<dim3(cnt, (nq + rpb - 1) / rpb), 256, 0, s>>>(v, 0, d_flag.p, d, dq, nullptr, 0, 0, scratch.p,
                                                                   mcols, rpb);
  }
  EMT_CUDA(cudaGetLastError());
}

void Store::form_cores(const std::vector<int>& nodes, cudaStream_t s) {
  if (nodes.empty()) return;
  int kb = 0;
  for (int p : nodes) kb = std::max(kb, node_k_h[p]);
  if (kb == 0) return;
  const int nl = upload_list(nodes, s);
  if (2 * kb <= kMaxCoreDim) {
    const size_t sh = (size_t)4 * kb * kb * sizeof(double);
    if (sh > 48 * 1024) EMT_CUDA(cudaFuncSetAttribute(k_core, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
    k_core<<<nl, 256, sh, s>>>(view(), d_list.p, mode, nullptr, nullptr, 0, 0);
  } else {
    // larger cores (many cut branches, e.g. three-phase networks): the same inversion in a
    // global-memory workspace
    const int m2 = 2 * kb;
    const int64_t stride = (int64_t)m2 * m2;
    if (core_ws.n < (size_t)(nl * stride)) core_ws.alloc((size_t)nl * stride);
    if (core_piv.n < (size_t)nl * m2) core_piv.alloc((size_t)nl * m2);
    k_core<<<nl, 256, 0, s>>>(view(), d_list.p, mode, core_ws.p, core_piv.p, stride, m2);
  }
  EMT_CUDA(cudaGetLastError());
}

void Store::pack(cudaStream_t s) {
  k_pack<<<grid_for(L_elems, 256), 256, 0, s>>>(L64.p, Lff.p, L32.p, L_elems);
  if (F_elems) k_pack<<<grid_for(F_elems, 256), 256, 0, s>>>(F64.p, Fff.p, F32.p, F_elems);
  if (C_elems) k_pack<<<grid_for(C_elems, 256), 256, 0, s>>>(C64.p, Cff.p, C32.p, C_elems);
  EMT_CUDA(cudaGetLastError());
}

void Store::build(cudaStream_t s) {
  std::vector<int> all_leaves(n_leaf);
  for (int j = 0; j < n_leaf; ++j) all_leaves[j] = j;
  assemble_leaves(all_leaves, s);
  invert_leaves(all_leaves, s);
  for (int d = tree.max_depth - 1; d >= 0; --d) {
    std::vector<int> nodes(lvl_nodes_h.begin() + lvl_ptr_h[d], lvl_nodes_h.begin() + lvl_ptr_h[d + 1]);
    if (nodes.empty()) continue;
    form_factors(nodes, d, s);
    form_cores(nodes, s);
  }
  pack(s);
}

int Store::device_status(cudaStream_t s) {
  int st = 0;
  EMT_CUDA(cudaMemcpyAsync(&st, d_status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  EMT_CUDA(cudaStreamSynchronize(s));
  return st;
}

void Store::clear_status(cudaStream_t s) { d_status.zero(s); }

void Store::update_graph(int a, int b, int branch, double delta, cudaStream_t s) {
  // host copies of the branch list and the CSR, and the device CSR values
  const int pa = tree.pos[a];
  const int pb = b >= 0 ? tree.pos[b] : -1;
  if (branch >= 0) g_val[branch] += delta;
  auto find = [&](int r, int c) {
    for (int t = csr_ptr[r]; t < csr_ptr[r + 1]; ++t)
      if (csr_col[t] == c) return t;
    return -1;
  };
  int i0 = find(pa, pa), i1 = -1, i2 = -1, i3 = -1;
  csr_val[i0] += delta;
  if (pb >= 0) {
    i1 = find(pb, pb);
    i2 = find(pa, pb);
    i3 = find(pb, pa);
    EMT_REQUIRE(i1 >= 0 && i2 >= 0 && i3 >= 0, EMT_ERR_INVALID, "no CSR entry for the modified branch");
    csr_val[i1] += delta;
    csr_val[i2] -= delta;
    csr_val[i3] -= delta;
  }
  k_csr_add<<<1, 1, 0, s>>>(d_csr_val.p, i0, i1, i2, i3, delta, delta, -delta, -delta, d_status.p);
  EMT_CUDA(cudaGetLastError());
}

void Store::modify_async(int bus_a, int bus_b, double delta, cudaStream_t s) {
  EMT_REQUIRE(bus_a >= 0 && bus_a < n && bus_b >= -1 && bus_b < n && bus_a != bus_b, EMT_ERR_INVALID,
              "bad buses for modification");
  EMT_REQUIRE(std::isfinite(delta), EMT_ERR_INVALID, "delta must be finite");
  int branch = -1;
  if (bus_b >= 0) {
    for (size_t e = 0; e < g_from.size(); ++e)
      if ((g_from[e] == bus_a && g_to[e] == bus_b) || (g_from[e] == bus_b && g_to[e] == bus_a)) {
        branch = (int)e;
        break;
      }
  }
  const int pa = tree.pos[bus_a];
  const int pb = bus_b >= 0 ? tree.pos[bus_b] : -1;
  if (bus_b >= 0) {
    const int la = leaf_index_of_pos(*this, pa), lb = leaf_index_of_pos(*this, pb);
    EMT_REQUIRE(branch >= 0 || la == lb, EMT_ERR_UNSUPPORTED,
                "no branch joins these buses and they sit in different leaves");
  }
  if (mode == EMT_MODE_EXACT) modify_exact(pa, pb, branch, delta, s);
  else modify_paper(pa, pb, branch, delta, s);
}

void Store::modify(int bus_a, int bus_b, double delta, cudaStream_t s) {
  EMT_REQUIRE(device_status(s) == DEV_OK, EMT_ERR_STATE, "store has a pending device error");
  // snapshot host-side values to restore them if the device reports a singular change
  auto g_save = g_val;
  auto csr_save = csr_val;
  auto cut_save = cut_g_h;
  modify_async(bus_a, bus_b, delta, s);
  const int st = device_status(s);
  if (st != DEV_OK) {
    g_val = g_save;
    csr_val = csr_save;
    cut_g_h = cut_save;
    clear_status(s);
    EMT_CUDA(cudaStreamSynchronize(s));
    throw Error(EMT_ERR_SINGULAR, "modification makes G singular or indefinite (denominator <= 0); store unchanged");
  }
}

// Path bookkeeping shared by both modification kinds.
namespace {
struct PathInfo {
  int la, lb, lca;                    // leaf node ids and their lowest common ancestor
  std::vector<int> path_a, path_b;    // leaf -> ... -> child of lca (inclusive)
  std::vector<int> above;             // lca -> ... -> root (inclusive)
};
PathInfo find_paths(const Tree& t, int leaf_a_node, int leaf_b_node) {
  PathInfo pi;
  pi.la = leaf_a_node;
  pi.lb = leaf_b_node;
  std::vector<int> anc_a;
  for (int x = leaf_a_node; x >= 0; x = t.parent[x]) anc_a.push_back(x);
  int x = leaf_b_node;
  std::vector<int> pb;
  while (std::find(anc_a.begin(), anc_a.end(), x) == anc_a.end()) {
    pb.push_back(x);
    x = t.parent[x];
  }
  pi.lca = x;
  for (int y : anc_a) {
    if (y == pi.lca) break;
    pi.path_a.push_back(y);
  }
  pi.path_b = pb;
  for (int y = pi.lca; y >= 0; y = t.parent[y]) pi.above.push_back(y);
  return pi;
}
}  // namespace

// Index into cut_g_h of the coefficient a change between positions pa and pb moves, at tree node
// c (their LCA): the column of the cut branch (one entry per column), or of a block column the
// entry of the left-side vertex in the column of the right-side vertex; -1 if none.
int Store::cut_entry(int c, int pa, int pb, int branch) const {
  const Tree& t = tree;
  const int W = t.cut_w;
  if (W == 1) {
    for (int i = t.cut_ptr[c]; i < t.cut_ptr[c + 1]; ++i)
      if (t.cut_e[i] == branch) return i;
    return -1;
  }
  const int l = t.left[c];
  const bool a_left = t.lo[l] <= pa && pa < t.hi[l];
  const int x = a_left ? pa : pb, y = a_left ? pb : pa;
  for (int i = t.cut_ptr[c]; i < t.cut_ptr[c + 1]; ++i)
    if (t.cut_b[i] == y && x >= t.cut_a[i] && x < t.cut_a[i] + W) return i * W + (x - t.cut_a[i]);
  return -1;
}

void Store::modify_exact(int pa, int pb, int branch, double delta, cudaStream_t s) {
  const Tree& t = tree;
  const int la = leaf_nodes_h[leaf_index_of_pos(*this, pa)];
  const int lb = pb >= 0 ? leaf_nodes_h[leaf_index_of_pos(*this, pb)] : la;
  PathInfo pi = find_paths(t, la, lb);
  // cut column changed at the LCA (cross-leaf branch)
  int ec = -1, ec_global = -1;
  double g_new = 0.0;
  if (pb >= 0 && la != lb) {
    const int i = cut_entry(pi.lca, pa, pb, branch);
    EMT_REQUIRE(i >= 0, EMT_ERR_INVALID, "modified branch is not in the cut list of its LCA");
    ec = i / t.cut_w - t.cut_ptr[pi.lca];
    ec_global = i;
    g_new = cut_g_h[ec_global] + delta;
  }
  // build items bottom-up with z slots
  std::vector<ModItem> items;
  std::map<int, int> slot_of, dslot_of;
  int zoff = 0, dn = 0;
  auto add_item = [&](int q) {
    ModItem it;
    it.node = q;
    it.is_leaf = t.left[q] < 0;
    it.zoff = zoff;
    zoff += t.hi[q] - t.lo[q];
    it.dslot = dn++;
    it.zl = it.zr = it.dl = it.dr = -1;
    if (!it.is_leaf) {
      auto fl = slot_of.find(t.left[q]);
      auto fr = slot_of.find(t.right[q]);
      if (fl != slot_of.end()) { it.zl = fl->second; it.dl = dslot_of[t.left[q]]; }
      if (fr != slot_of.end()) { it.zr = fr->second; it.dr = dslot_of[t.right[q]]; }
    }
    it.pa = pa;
    it.pb = pb;
    slot_of[q] = it.zoff;
    dslot_of[q] = it.dslot;
    items.push_back(it);
  };
  // both paths below the LCA, interleaved by depth (children always before parents)
  std::vector<int> below;
  for (int q : pi.path_a) below.push_back(q);
  for (int q : pi.path_b) below.push_back(q);
  std::stable_sort(below.begin(), below.end(), [&](int x, int y) { return t.depth[x] > t.depth[y]; });
  for (int q : below) add_item(q);
  for (int q : pi.above) add_item(q);
  EMT_REQUIRE((size_t)zoff <= zbuf.n && (size_t)dn <= dbuf.n, EMT_ERR_INVALID, "modification scratch too small");
  DStore v = view();
  // phase 1: old z and denominators (reads only)
  for (auto& it : items) {
    const int nq = t.hi[it.node] - t.lo[it.node];
    const int k = it.is_leaf ? 0 : node_k_h[it.node];
    k_mod_z<<<grid_for(nq, 256, 64), 256, (size_t)4 * k * sizeof(double) + 16, s>>>(v, it, zbuf.p, dbuf.p, delta);
    k_mod_denominator<<<1, 1, 0, s>>>(v, it, zbuf.p, dbuf.p, delta);
  }
  EMT_CUDA(cudaGetLastError());
  // phase 2: updates (kernels no-op if a denominator was flagged)
  update_graph(t.perm[pa], pb >= 0 ? t.perm[pb] : -1, branch, delta, s);
  std::vector<int> core_nodes;
  for (auto& it : items) {
    const int nq = t.hi[it.node] - t.lo[it.node];
    if (it.is_leaf) {
      k_mod_leaf<<<std::min(nq, 1024), 256, 0, s>>>(v, it, zbuf.p, dbuf.p, delta);
    } else {
      const int k = node_k_h[it.node];
      const bool at_lca = it.node == pi.lca && ec >= 0;
      k_mod_factor<<<grid_for((int64_t)nq * std::max(k, 1), 256, 1024), 256, (size_t)2 * k * sizeof(double) + 16, s>>>(
          v, it, zbuf.p, dbuf.p, delta, at_lca ? ec : -1, g_new);
      if (at_lca) k_set_cut_g<<<1, 1, 0, s>>>(v, ec_global, g_new);
      core_nodes.push_back(it.node);
    }
  }
  EMT_CUDA(cudaGetLastError());
  if (ec_global >= 0) cut_g_h[ec_global] = g_new;
  // cores of every updated node: skipped on the device if the status word is set
  // (k_core writes only when status is OK is ensured by re-forming from unchanged factors)
  if (!core_nodes.empty()) form_cores(core_nodes, s);
  pack(s);
}

void Store::modify_paper(int pa, int pb, int branch, double delta, cudaStream_t s) {
  // Algorithm 2: re-invert the touched leaves, recompute the factors on both paths up to the
  // lowest common ancestor (inclusive); ancestors above it are kept as they are.
  const Tree& t = tree;
  const int ja = leaf_index_of_pos(*this, pa);
  const int jb = pb >= 0 ? leaf_index_of_pos(*this, pb) : ja;
  PathInfo pi = find_paths(t, leaf_nodes_h[ja], leaf_nodes_h[jb]);
  update_graph(t.perm[pa], pb >= 0 ? t.perm[pb] : -1, branch, delta, s);
  if (pb >= 0 && ja != jb) {
    const int i = cut_entry(pi.lca, pa, pb, branch);
    EMT_REQUIRE(i >= 0, EMT_ERR_INVALID, "modified branch is not in the cut list of its LCA");
    cut_g_h[i] += delta;
    k_set_cut_g<<<1, 1, 0, s>>>(view(), i, cut_g_h[i]);
  }
  std::vector<int> leaves{ja};
  if (jb != ja) leaves.push_back(jb);
  assemble_leaves(leaves, s);
  invert_leaves(leaves, s);
  std::vector<int> nodes;
  for (int q : pi.path_a)
    if (t.left[q] >= 0) nodes.push_back(q);
  for (int q : pi.path_b)
    if (t.left[q] >= 0) nodes.push_back(q);
  if (t.left[pi.lca] >= 0) nodes.push_back(pi.lca);
  for (int d = t.max_depth; d >= 0; --d) {
    std::vector<int> batch;
    for (int q : nodes)
      if (t.depth[q] == d && std::find(batch.begin(), batch.end(), q) == batch.end()) batch.push_back(q);
    if (batch.empty()) continue;
    form_factors(batch, d, s);
    form_cores(batch, s);
  }
  pack(s);
}

void Store::apply_rows_fp64(const double* Xin, double* Y, int m, int ld, cudaStream_t s) {
  DStore v = view();
  k_leaf_dense<<<n, 128, 0, s>>>(v, Xin, Y, m, ld);
  const int mcols = m;
  if ((size_t)s_total * mcols > scratch.n) scratch.alloc((size_t)s_total * mcols);
  v = view();
  for (int dq = tree.max_depth - 1; dq >= 0; --dq) {
    const int cnt = lvl_ptr_h[dq + 1] - lvl_ptr_h[dq];
    if (cnt == 0) continue;
    int kq = 0, nq = 0;
    for (int i = lvl_ptr_h[dq]; i < lvl_ptr_h[dq + 1]; ++i) {
      kq = std::max(kq, node_k_h[lvl_nodes_h[i]]);
      nq = std::max(nq, tree.hi[lvl_nodes_h[i]] - tree.lo[lvl_nodes_h[i]]);
    }
    if (kq == 0) continue;
    const int pc = level_sweep_cols(kq);
    const size_t sh = (size_t)2 * kq * pc * sizeof(double);
    if (sh > 48 * 1024)
      EMT_CUDA(cudaFuncSetAttribute(k_level_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
    k_level_sweep<<<dim3(cnt, (m + pc - 1) / pc), 256, sh, s>>>(v, 1, d_flag.p, 0, dq, Y, m, ld, scratch.p, mcols,
                                                                pc);
    const int rpb = 16;
    k_level_expand<<<dim3(cnt, (nq + rpb - 1) / rpb), 256, 0, s>>>(v, 1, d_flag.p, 0, dq, Y, m, ld, scratch.p, mcols,
                                                                   rpb);
  }
  EMT_CUDA(cudaGetLastError());
}

}  // namespace emt

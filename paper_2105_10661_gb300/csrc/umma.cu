// Dense products of the multi-column apply on the 5th-generation tensor cores (tcgen05).
//
// Leaf stage:  Y[leaf rows, columns] = L_j X_j
// Expansion:   V[leaf rows, columns] = Y - F_path S_path   (F_path = the leaf's rows of the factors
//              of all its ancestors, concatenated; S_path = the matching rows of S, Eq. 9 factors)
// Each product A B is formed from BF16 splits A = A_hi + A_lo, B = B_hi + B_lo as
//   A B ~= A_hi B_hi + A_hi B_lo + A_lo B_hi   (FP32 accumulation in tensor memory);
// the dropped A_lo B_lo term and the split residuals leave a relative error of about 2^-16, which
// the multi-column step's float-float residual refinement removes.
//
// Both operands are pre-tiled in global memory in the canonical K-major core-matrix layout
// (8 rows x 16 bytes per core matrix, no swizzle): A (leaf blocks or factor paths, split once per
// store) per (leaf, 128-row tile, 32-deep K chunk), B (right-hand sides or gathered S rows, split
// once per pass) per (leaf, TN-column tile, K chunk). One CTA computes a 128-row x TN-column tile
// of one leaf as a pipeline of 2-4 stages (96 KB, two CTAs per SM): one thread issues one
// cp.async.bulk per operand and chunk into a stage (full mbarrier), one thread issues
// tcgen05.mma (M = 128, N = TN, K = 16, kind::f16 with BF16 inputs) three times per K step and
// commits them to the stage's empty mbarrier, and the epilogue reads the accumulator with
// tcgen05.ld (the expansion stages it through shared memory, 64 columns at a time, for the
// float-float update of V). Each mbarrier has a single
// waiter that waits for its phases in order; every wait is bounded by clock64 and reports a
// timeout in the device status word; tensor memory is always released.
#include <algorithm>
#include <cstdint>

#include <cuda_bf16.h>

#include "multi.h"

namespace emt {

namespace {

constexpr int UM = 128;            // MMA M (tile rows)
constexpr int UKC = 32;            // K chunk
constexpr uint32_t A_CHUNK = UM * UKC * 2;          // 8 KB per split
constexpr uint32_t A_SBO = UKC / 8 * 128, A_LBO = 128;   // M-group stride (8 rows x UKC), K-core stride
constexpr uint32_t B_SBO = UKC / 8 * 128, B_LBO = 128;   // N-group stride, K-core stride
constexpr uint32_t kStageBudget = 96 * 1024;        // pipeline shared memory per CTA: two CTAs per SM
constexpr long long kSpin = 4000000000LL;           // ~2 s of SM clocks

__device__ __forceinline__ uint32_t su(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version
  return d;                 // base offset 0, no swizzle
}

__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(su(bar)), "r"(parity)
                 : "memory");
    if (ok) return true;
    if (clock64() - t0 > kSpin) return false;
  }
}

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_val(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }

// A blocks: per (leaf, M tile, K chunk) [hi | lo], A_CHUNK bytes each, canonical layout.
__global__ void k_tile_leaves(DStore st, const int* __restrict__ blk_leaf, const int* __restrict__ blk_mt,
                              const int* __restrict__ blk_kc, uint16_t* __restrict__ out, int n_blk) {
  const int blk = blockIdx.x;
  if (blk >= n_blk) return;
  const int j = blk_leaf[blk], mt = blk_mt[blk], kc = blk_kc[blk];
  const int node = st.leaf_node[j];
  const int b = st.hi[node] - st.lo[node];
  const int ld = st.leaf_ld[j];
  const double* L = st.L64 + st.leaf_off[j];
  uint16_t* hi = out + (size_t)blk * (A_CHUNK);   // 2 * A_CHUNK bytes = A_CHUNK uint16 per split... see below
  uint16_t* lo = hi + A_CHUNK / 2;
  for (int e = threadIdx.x; e < UM * UKC; e += blockDim.x) {
    const int rr = e / UKC, kk = e % UKC;
    const int r = mt * UM + rr, k = kc * UKC + kk;
    const double v = (r < b && k < b) ? L[(int64_t)r * ld + k] : 0.0;
    const float vf = (float)v;
    const uint16_t h = bf16_bits(vf);
    const uint16_t l = bf16_bits((float)(v - (double)bf16_val(h)));
    const uint32_t off = (rr / 8) * A_SBO + (kk / 8) * A_LBO + ((rr % 8) * 8 + (kk % 8)) * 2;
    hi[off / 2] = h;
    lo[off / 2] = l;
  }
}

struct UmmaArgs {
  const int4* tiles;        // (leaf, m0, n0, first A block of this leaf-M-tile)
  const int2* tile_b;       // (first B block of the tile's (leaf, N tile), K chunks)
  const uint16_t* a_blocks; // pre-tiled A operand
  const uint16_t* b_blocks; // pre-tiled B operand
  float* Y;                 // [n][R] leaf stage: written; expansion: read
  int R, TN;
  int ns;                   // pipeline stages
  int r_act;                // columns in use; tiles starting beyond exit at once
};

// Expansion epilogue arguments.
struct ExpArgs {
  MSimD m;
  int pass, n1, record, s_in_chunk;
};

enum { UMMA_LEAF = 0, UMMA_EXPAND = 1 };

// A blocks of the expansion: per (leaf, M tile, K chunk) [hi | lo] of the leaf's factor path,
// element (row r, path element e) = F[path_fbase[e0 + e] + position(r) * path_kld[e0 + e]].
__global__ void k_tile_paths(DStore st, const int* __restrict__ blk_leaf, const int* __restrict__ blk_mt,
                             const int* __restrict__ blk_kc, const int* __restrict__ path_ptr,
                             const long long* __restrict__ path_fbase, const int* __restrict__ path_kld,
                             uint16_t* __restrict__ out, int n_blk) {
  const int blk = blockIdx.x;
  if (blk >= n_blk) return;
  const int j = blk_leaf[blk], mt = blk_mt[blk], kc = blk_kc[blk];
  const int node = st.leaf_node[j];
  const int lo = st.lo[node], b = st.hi[node] - lo;
  const int e0 = path_ptr[j], ne = path_ptr[j + 1] - e0;
  uint16_t* hi = out + (size_t)blk * (A_CHUNK);
  uint16_t* lw = hi + A_CHUNK / 2;
  for (int w = threadIdx.x; w < UM * UKC; w += blockDim.x) {
    const int rr = w / UKC, kk = w % UKC;
    const int r = mt * UM + rr, e = kc * UKC + kk;
    const double v = (r < b && e < ne) ? st.F64[path_fbase[e0 + e] + (int64_t)(lo + r) * path_kld[e0 + e]] : 0.0;
    const uint16_t h = bf16_bits((float)v);
    const uint16_t l = bf16_bits((float)(v - (double)bf16_val(h)));
    const uint32_t off = (rr / 8) * A_SBO + (kk / 8) * A_LBO + ((rr % 8) * 8 + (kk % 8)) * 2;
    hi[off / 2] = h;
    lw[off / 2] = l;
  }
}

// B blocks: per (leaf j, N tile, K chunk) [hi | lo], each TN x 64 BF16 in the canonical K-major
// layout (N-group stride B_SBO, K-core stride 128 bytes). Grid (blocks, TN / 32) x 32 (UKC / 8)
// threads; thread = one column and 8 consecutive k: one 16-byte core row per split.
// With path_ptr null the rows of chunk k are the leaf's positions (leaf stage, source Xf);
// otherwise they are the rows path_srow[path_ptr[leaf] + k] of the source (expansion, source S).
__global__ void k_split_b(DStore st, const int4* __restrict__ bdesc, const float* __restrict__ Xf,
                          uint16_t* __restrict__ out, int R, int TN, int n_blk, const int* __restrict__ path_ptr,
                          const int* __restrict__ path_srow) {
  const int blk = blockIdx.x;
  if (blk >= n_blk) return;
  const int4 d = bdesc[blk];   // leaf, N tile first column, K chunk, unused
  const int node = st.leaf_node[d.x];
  const int lo = path_ptr ? path_ptr[d.x] : st.lo[node];
  const int b = path_ptr ? path_ptr[d.x + 1] - lo : st.hi[node] - lo;
  unsigned char* hi = reinterpret_cast<unsigned char*>(out) + (size_t)blk * 4 * TN * UKC;
  unsigned char* lob = hi + (size_t)2 * TN * UKC;
  // CTA y covers columns [32 y, 32 y + 32) of the tile: thread = one column and one group of 8 k
  {
    const int n = blockIdx.y * 32 + (threadIdx.x & 31), kg = threadIdx.x >> 5;
    if (n >= TN || kg >= UKC / 8) return;
    const int col = d.y + n;
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float x[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int k = d.z * UKC + kg * 8 + 2 * q + u;
        const int row = k < b ? (path_srow ? path_srow[lo + k] : lo + k) : 0;
        x[u] = (k < b && col < R) ? Xf[(int64_t)row * R + col] : 0.f;
      }
      const uint16_t h0 = bf16_bits(x[0]), h1 = bf16_bits(x[1]);
      const uint16_t l0 = bf16_bits(x[0] - bf16_val(h0)), l1 = bf16_bits(x[1] - bf16_val(h1));
      h[q] = (uint32_t)h0 | ((uint32_t)h1 << 16);
      l[q] = (uint32_t)l0 | ((uint32_t)l1 << 16);
    }
    const uint32_t off = (n / 8) * B_SBO + kg * B_LBO + (n % 8) * 16;
    *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(lob + off) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

__device__ __forceinline__ void bulk_g2s_u(unsigned char* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su(dst)),
               "l"(src), "r"(bytes), "r"(su(bar))
               : "memory");
}

// Expansion epilogue, per group of 64 columns: the accumulator's 128 x 64 block goes through shared
// memory (row stride 65 words: conflict-free both ways; it lives in the pipeline stages, which are
// free here since every MMA reading them has completed) so that each warp then handles rows of
// the group with coalesced accesses: v = Y - acc (- f_c z for a column whose change is on), V = v
// (pass 0) or V + v in float-float (pass 1), and the monitored record.
__device__ __forceinline__ void expand_epilogue(const UmmaArgs& a, const ExpArgs& x, uint32_t tmem, unsigned char* sm,
                                                int lo, int b, int m0, int n0) {
  const int TN = a.TN, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float* T = reinterpret_cast<float*>(sm);
  constexpr int ldt = 65;
  const MSimD& m = x.m;
  const int64_t R = m.R;
  const int step = m.dyn->step_base + x.s_in_chunk + 1;
  double* rec = x.record ? m.dyn->rec : nullptr;
  const int rec_first = m.dyn->rec_first;
  const int rows = min(UM, b - m0);
  for (int cg = 0; cg < TN; cg += 64) {
    if (cg > 0) __syncthreads();   // the previous group's rows are done with T
    {
      // warps 0-3 read columns cg .. cg + 31, warps 4-7 cg + 32 .. cg + 63 of their 32 lanes
      const int lane_base = 32 * (warp & 3);
      const int ch = cg / 32 + (warp >> 2);
      if (ch * 32 < TN) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)lane_base << 16) + (uint32_t)(ch * 32);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float* trow = T + (lane_base + lane) * ldt + (warp >> 2) * 32;
#pragma unroll
        for (int q = 0; q < 32; ++q) trow[q] = __uint_as_float(r[q]);
      }
    }
    __syncthreads();
    // lane: columns c, c + 1 of every row of this warp; eight rows' loads in flight at once (four:
    // 10 us more per 512-column time step on 11,456 buses)
    const int cl = 2 * lane, cc = cg + cl, c = n0 + cc;
    const int nv = cc < TN ? max(0, min(2, m.R_act - c)) : 0;   // valid columns of this lane
    float fc0 = 0.f, fc1 = 0.f;
    if (x.n1 && nv > 0) {
      fc0 = m.fcol[c];
      if (nv > 1) fc1 = m.fcol[c + 1];
    }
    constexpr int RB = 8;
    for (int r0 = warp; r0 < rows; r0 += 8 * RB) {
      float2 y[RB];
      float4 vo[RB];
      int mi[RB];
#pragma unroll
      for (int u = 0; u < RB; ++u) {
        const int rr = r0 + 8 * u;
        const int64_t at = (int64_t)(lo + m0 + rr) * R + c;
        y[u] = make_float2(0.f, 0.f);
        vo[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        mi[u] = -1;
        if (rr < rows && nv > 0) {
          if (nv == 2) {
            y[u] = *reinterpret_cast<const float2*>(m.Y + at);
            if (x.pass) vo[u] = *reinterpret_cast<const float4*>(m.V + at);
          } else {
            y[u].x = m.Y[at];
            if (x.pass) {
              const float2 o = m.V[at];
              vo[u].x = o.x;
              vo[u].y = o.y;
            }
          }
          if (rec) mi[u] = m.mon_idx[lo + m0 + rr];
        }
      }
#pragma unroll
      for (int u = 0; u < RB; ++u) {
        const int rr = r0 + 8 * u;
        if (rr >= rows || nv == 0) continue;
        const int pos = lo + m0 + rr;
        const int64_t at = (int64_t)pos * R + c;
        float v[2] = {y[u].x - T[rr * ldt + cl], y[u].y - T[rr * ldt + cl + 1]};
        if (fc0 != 0.f) v[0] = fmaf(-fc0, m.Z[at].x, v[0]);
        if (fc1 != 0.f) v[1] = fmaf(-fc1, m.Z[at + 1].x, v[1]);
        const float ox[2] = {vo[u].x, vo[u].z}, oy[2] = {vo[u].y, vo[u].w};
        float2 out[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (x.pass == 0) {
            out[q] = make_float2(v[q], 0.f);
          } else {
            // float-float V + v (TwoSum, then renormalisation)
            const float s1 = __fadd_rn(ox[q], v[q]);
            const float bb = __fsub_rn(s1, ox[q]);
            const float err = __fadd_rn(__fsub_rn(ox[q], __fsub_rn(s1, bb)), __fsub_rn(v[q], bb));
            const float lo2 = __fadd_rn(err, oy[q]);
            const float hi2 = __fadd_rn(s1, lo2);
            out[q] = make_float2(hi2, __fsub_rn(lo2, __fsub_rn(hi2, s1)));
          }
        }
        if (nv == 2)
          *reinterpret_cast<float4*>(m.V + at) = make_float4(out[0].x, out[0].y, out[1].x, out[1].y);
        else
          m.V[at] = out[0];
        if (mi[u] >= 0) {
          double* rp = rec + ((int64_t)(step - rec_first) * R + c) * m.n_mon + mi[u];
          rp[0] = (double)out[0].x + (double)out[0].y;
          if (nv == 2) rp[m.n_mon] = (double)out[1].x + (double)out[1].y;
        }
      }
    }
  }
}

// Two CTAs per SM for the leaf products (2-4 stages in 96 KB); three for the expansion (128-column
// tiles), whose short K (the ancestor path) needs only two stages and whose epilogue is bound by
// its loads.
template <int MODE>
__global__ void __launch_bounds__(256, MODE == UMMA_EXPAND ? 3 : 2) k_mc_umma(DStore st, UmmaArgs a, ExpArgs x, int* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int TN = a.TN;
  // tensor-memory columns: a power of two >= 32 holding the TN accumulator columns
  const uint32_t tcols = TN <= 32 ? 32u : (TN <= 64 ? 64u : (TN <= 128 ? 128u : 256u));
  const uint32_t b_split = (uint32_t)TN * UKC * 2;              // bytes of one B split
  const uint32_t stage_bytes = 2 * A_CHUNK + 2 * b_split;
  const int ns = a.ns;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + ns * stage_bytes);   // full[ns], empty[ns], done
  uint64_t* full = bars;
  uint64_t* empty = bars + ns;
  uint64_t* done = bars + 2 * ns;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2 * ns + 1);
  int* flag = reinterpret_cast<int*>(bars + 2 * ns + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int4 tl = a.tiles[blockIdx.x];
  const int j = tl.x, m0 = tl.y, n0 = tl.z, blk0 = tl.w;
  const int2 tb = a.tile_b[blockIdx.x];
  const int bblk0 = tb.x, nkc = tb.y;   // nkc >= 1
  if (n0 >= a.r_act) return;   // uniform per CTA, before any barrier or tensor memory use
  const int node = st.leaf_node[j];
  const int lo = st.lo[node], b = st.hi[node] - lo;
  if (tid == 0) {
    for (int i = 0; i <= 2 * ns; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su(bars + i)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su(tslot)), "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(UM >> 4) << 24);
  __shared__ int cnt_sh[2];        // [0] chunks copied (producer), [1] chunks multiplied (issuer)
  int issued = 0, committed = 0;
  if (tid == 0) {
    // producer: stage s = kc % ns is refilled once the MMAs of chunk kc - ns released it
    for (int kc = 0; kc < nkc; ++kc) {
      const int s = kc % ns, u = kc / ns;
      unsigned char* stg = sm + s * stage_bytes;
      if (kc >= ns && !bar_wait(empty + s, (u - 1) & 1)) {
        atomicExch(status, DEV_TIMEOUT);
        atomicExch(flag, 1);
        break;
      }
      if (*reinterpret_cast<volatile int*>(flag)) break;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su(full + s)), "r"(stage_bytes)
                   : "memory");
      bulk_g2s_u(stg, reinterpret_cast<const unsigned char*>(a.a_blocks) + (size_t)(blk0 + kc) * 2 * A_CHUNK,
                 2 * A_CHUNK, full + s);
      bulk_g2s_u(stg + 2 * A_CHUNK, reinterpret_cast<const unsigned char*>(a.b_blocks) + (size_t)(bblk0 + kc) * 2 * b_split,
                 2 * b_split, full + s);
      ++issued;
    }
  } else if (tid == 32) {
    // MMA issuer
    for (int kc = 0; kc < nkc; ++kc) {
      const int s = kc % ns, u = kc / ns;
      if (!bar_wait(full + s, u & 1)) {
        atomicExch(status, DEV_TIMEOUT);
        atomicExch(flag, 1);
        break;
      }
      if (*reinterpret_cast<volatile int*>(flag)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_hi = su(sm + s * stage_bytes), a_lo = a_hi + A_CHUNK;
      const uint32_t b_hi = a_hi + 2 * A_CHUNK, b_lo = b_hi + b_split;
#pragma unroll
      for (int ks = 0; ks < UKC / 16; ++ks) {
        const uint32_t ko = ks * 2 * 128;
        const uint64_t dah = umma_desc(a_hi + ko, A_LBO, A_SBO), dal = umma_desc(a_lo + ko, A_LBO, A_SBO);
        const uint64_t dbh = umma_desc(b_hi + ko, B_LBO, B_SBO), dbl = umma_desc(b_lo + ko, B_LBO, B_SBO);
        const uint32_t acc0 = (kc > 0 || ks > 0) ? 1u : 0u;
        asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                     "l"(dah), "l"(dbh), "r"(idesc), "r"(acc0)
                     : "memory");
        asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                     "l"(dah), "l"(dbl), "r"(idesc), "r"(1u)
                     : "memory");
        asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                     "l"(dal), "l"(dbh), "r"(idesc), "r"(1u)
                     : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su(empty + s))
                   : "memory");
      ++committed;
    }
    // all MMAs issued so far complete -> done
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su(done))
                 : "memory");
  } else if (MODE == UMMA_EXPAND && warp >= 2) {
    // the epilogue's inputs do not depend on the product: bring its Y rows (and, in the
    // correction pass, its V rows) into L2 while the MMAs run; one 128-byte line per request
    const MSimD& m = x.m;
    const int rows = min(UM, b - m0);
    const int ncol = min(TN, m.R_act - n0);
    if (ncol > 0) {
      const int ly = (ncol * 4 + 127) / 128, lv = x.pass ? (ncol * 8 + 127) / 128 : 0;
      for (int w = tid - 64; w < rows * (ly + lv); w += 192) {
        const int rr = w / (ly + lv), l = w % (ly + lv);
        const int64_t at = (int64_t)(lo + m0 + rr) * m.R + n0;
        const void* p = l < ly ? (const void*)(reinterpret_cast<const char*>(m.Y + at) + 128 * l)
                               : (const void*)(reinterpret_cast<const char*>(m.V + at) + 128 * (l - ly));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
      }
    }
  }
  if (tid == 0) cnt_sh[0] = issued;
  if (tid == 32) cnt_sh[1] = committed;
  __syncthreads();
  // the issuer's last commit covers every MMA it issued
  __shared__ int ok_sh;
  if (tid == 32) {
    const bool ok = bar_wait(done, 0);
    if (!ok) atomicExch(status, DEV_TIMEOUT);
    ok_sh = ok && !*reinterpret_cast<volatile int*>(flag) && cnt_sh[1] == nkc;
  }
  if (tid == 0 && cnt_sh[0] > cnt_sh[1]) {
    // error path only: copies issued to stages the issuer never consumed; each is the latest use
    // of its stage (at most one per stage), so its phase parity is unambiguous
    for (int kc = cnt_sh[1]; kc < cnt_sh[0]; ++kc) bar_wait(full + kc % ns, (kc / ns) & 1);
  }
  __syncthreads();
  const bool ok = ok_sh != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (MODE == UMMA_EXPAND) {
    if (ok) expand_epilogue(a, x, tmem, sm, lo, b, m0, n0);
  } else if (ok) {
    // epilogue: warp w reads lanes 32 (w % 4) .. +31; warps 0-3 and 4-7 split the columns
    const int lane_base = 32 * (warp & 3);
    const int row = m0 + lane_base + (tid & 31);
    const int nchunks = TN / 32;
    const int half = nchunks / 2 > 0 ? nchunks / 2 : 1;
    const int c_begin = (warp >> 2) * half, c_end = min(nchunks, c_begin + half);
    for (int ch = c_begin; ch < c_end; ++ch) {
      uint32_t r[32];
      const uint32_t taddr = tmem + ((uint32_t)lane_base << 16) + (uint32_t)(ch * 32);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < b) {
        float* dst = a.Y + (int64_t)(lo + row) * a.R + n0 + ch * 32;
        const int cmax = a.R - (n0 + ch * 32);
        if (cmax >= 32 && (a.R & 3) == 0) {
#pragma unroll
          for (int q = 0; q < 8; ++q)
            reinterpret_cast<float4*>(dst)[q] =
                make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]), __uint_as_float(r[4 * q + 2]),
                            __uint_as_float(r[4 * q + 3]));
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q)
            if (q < cmax) dst[q] = __uint_as_float(r[q]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
}

}  // namespace

// ---------------------------------------------------------------- host side
// pipeline stages for a tile width: as many as fit the budget, 2..4
int umma_stages(int TN) {
  const uint32_t stage = 2 * A_CHUNK + 2 * (uint32_t)TN * UKC * 2;
  return std::max(2, std::min(4, (int)(kStageBudget / stage)));
}
// stages + barriers (2 ns + 1) + tensor-memory slot + flag
size_t umma_smem_bytes(int TN, int stages) {
  return (size_t)stages * (2 * (size_t)A_CHUNK + 2 * (size_t)TN * UKC * 2) + 128;
}
size_t umma_smem_bytes(int TN) { return umma_smem_bytes(TN, umma_stages(TN)); }
constexpr int kExpandStages = 2;

void Umma::build(const Store& st, int R_, cudaStream_t s, int tn) {
  R = R_;
  const Tree& t = st.tree;
  if (tn == 0) {
    // The busiest SM runs ceil(tiles / SMs) tiles of TN columns each: take the width with the
    // smallest such makespan, the widest among equals (wider tiles re-read the leaf blocks less).
    int dev = 0, n_sm = 1;
    EMT_CUDA(cudaGetDevice(&dev));
    EMT_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    int64_t mtiles = 0;
    for (int j = 0; j < st.n_leaf; ++j)
      mtiles += (t.hi[st.leaf_nodes_h[j]] - t.lo[st.leaf_nodes_h[j]] + UM - 1) / UM;
    int64_t best = -1;
    for (int w : {256, 192, 128, 64}) {
      const int64_t tiles = mtiles * ((R + w - 1) / w);
      const int64_t span = (tiles + n_sm - 1) / n_sm * w;
      if (best < 0 || span < best) {
        best = span;
        tn = w;
      }
    }
  }
  TN = tn;
  std::vector<int> bl, bm, bk;
  std::vector<int4> tiles, bdesc;
  std::vector<int2> tb;
  for (int j = 0; j < st.n_leaf; ++j) {
    const int b = t.hi[st.leaf_nodes_h[j]] - t.lo[st.leaf_nodes_h[j]];
    const int nmt = (b + UM - 1) / UM, nkc = (b + UKC - 1) / UKC;
    std::vector<int> bfirst;   // first B block of each N tile of this leaf
    for (int n0 = 0; n0 < R; n0 += TN) {
      bfirst.push_back((int)bdesc.size());
      for (int kc = 0; kc < nkc; ++kc) bdesc.push_back(make_int4(j, n0, kc, 0));
    }
    for (int mt = 0; mt < nmt; ++mt) {
      const int first = (int)bl.size();
      for (int kc = 0; kc < nkc; ++kc) {
        bl.push_back(j);
        bm.push_back(mt);
        bk.push_back(kc);
      }
      int nt = 0;
      for (int n0 = 0; n0 < R; n0 += TN, ++nt) {
        tiles.push_back(make_int4(j, mt * UM, n0, first));
        tb.push_back(make_int2(bfirst[nt], nkc));
      }
    }
  }
  n_blocks = (int)bl.size();
  n_tiles = (int)tiles.size();
  n_bblocks = (int)bdesc.size();
  DevBuf<int> dl, dm, dk;
  dl.upload(bl, s);
  dm.upload(bm, s);
  dk.upload(bk, s);
  a_blocks.alloc((size_t)n_blocks * A_CHUNK);   // uint16 count: 2 splits x A_CHUNK bytes / 2
  k_tile_leaves<<<n_blocks, 256, 0, s>>>(st.view(), dl.p, dm.p, dk.p, a_blocks.p, n_blocks);
  b_blocks.alloc((size_t)n_bblocks * 2 * TN * UKC);   // uint16 count: 2 splits x TN x 64
  b_desc.upload(bdesc, s);
  tile_b.upload(tb, s);
  d_tiles.upload(tiles, s);
  // the attribute is per kernel, shared by every simulation: allow the largest tile
  EMT_CUDA(cudaFuncSetAttribute(k_mc_umma<UMMA_LEAF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)std::max(umma_smem_bytes(256), std::max(umma_smem_bytes(128), umma_smem_bytes(64)))));
  EMT_CUDA(cudaStreamSynchronize(s));   // the index lists above are freed on return
  ready = true;
}

void Umma::build_expand(const Store& st, const std::vector<int>& pp, const int* path_ptr,
                        const long long* path_fbase, const int* path_kld, cudaStream_t s) {
  const Tree& t = st.tree;
  for (int j = 0; j < st.n_leaf; ++j)
    if (pp[j + 1] == pp[j]) return;   // a leaf without ancestor rows: the SIMT expansion serves it
  // 128-column tiles at three CTAs per SM (the accumulator staged per 64-column group): 37.4 us on
  // the 11,456-bus network x 512 columns, against 38.9 for 64-column tiles at four CTAs per SM
  xTN = 128;
  std::vector<int> bl, bm, bk;
  std::vector<int4> tiles, bdesc;
  std::vector<int2> tb;
  for (int j = 0; j < st.n_leaf; ++j) {
    const int b = t.hi[st.leaf_nodes_h[j]] - t.lo[st.leaf_nodes_h[j]];
    const int ne = pp[j + 1] - pp[j];
    const int nmt = (b + UM - 1) / UM, nkc = (ne + UKC - 1) / UKC;
    std::vector<int> bfirst;
    for (int n0 = 0; n0 < R; n0 += xTN) {
      bfirst.push_back((int)bdesc.size());
      for (int kc = 0; kc < nkc; ++kc) bdesc.push_back(make_int4(j, n0, kc, 0));
    }
    for (int mt = 0; mt < nmt; ++mt) {
      const int first = (int)bl.size();
      for (int kc = 0; kc < nkc; ++kc) {
        bl.push_back(j);
        bm.push_back(mt);
        bk.push_back(kc);
      }
      int nt = 0;
      for (int n0 = 0; n0 < R; n0 += xTN, ++nt) {
        tiles.push_back(make_int4(j, mt * UM, n0, first));
        tb.push_back(make_int2(bfirst[nt], nkc));
      }
    }
  }
  x_blocks = (int)bl.size();
  x_tiles = (int)tiles.size();
  x_bblocks = (int)bdesc.size();
  DevBuf<int> dl, dm, dk;
  dl.upload(bl, s);
  dm.upload(bm, s);
  dk.upload(bk, s);
  xa_blocks.alloc((size_t)x_blocks * A_CHUNK);
  k_tile_paths<<<x_blocks, 256, 0, s>>>(st.view(), dl.p, dm.p, dk.p, path_ptr, path_fbase, path_kld, xa_blocks.p,
                                        x_blocks);
  EMT_CUDA(cudaGetLastError());
  xb_blocks.alloc((size_t)x_bblocks * 2 * xTN * UKC);
  x_bdesc.upload(bdesc, s);
  x_tile_b.upload(tb, s);
  x_tiles_d.upload(tiles, s);
  // the epilogue stages 128 x 64 blocks of the accumulator (row stride 65 words) in the pipeline
  // stages: they must hold one; tiles are whole 64-column groups
  EMT_REQUIRE((size_t)UM * 65 * sizeof(float) <= umma_smem_bytes(xTN, kExpandStages) - 128 && xTN % 64 == 0,
              EMT_ERR_UNSUPPORTED, "expansion tile too wide for its pipeline stages");
  EMT_CUDA(cudaFuncSetAttribute(k_mc_umma<UMMA_EXPAND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)umma_smem_bytes(xTN, kExpandStages)));
  EMT_CUDA(cudaStreamSynchronize(s));
  exp_ready = true;
}

void Umma::launch(const Store& st, const float* Xf, float* Y, cudaStream_t s, int r_act) {
  split(st, Xf, s);
  mma(st, Y, s, r_act);
}

void Umma::split(const Store& st, const float* Xf, cudaStream_t s) {
  k_split_b<<<dim3(n_bblocks, TN / 32), 32 * (UKC / 8), 0, s>>>(st.view(), b_desc.p, Xf, b_blocks.p, R, TN, n_bblocks, nullptr,
                                                     nullptr);
  EMT_CUDA(cudaGetLastError());
}

void Umma::mma(const Store& st, float* Y, cudaStream_t s, int r_act) {
  UmmaArgs a;
  a.tiles = d_tiles.p;
  a.tile_b = tile_b.p;
  a.a_blocks = a_blocks.p;
  a.b_blocks = b_blocks.p;
  a.Y = Y;
  a.R = R;
  a.TN = TN;
  a.ns = umma_stages(TN);
  a.r_act = r_act;
  ExpArgs x{};
  k_mc_umma<UMMA_LEAF><<<n_tiles, 256, umma_smem_bytes(TN), s>>>(st.view(), a, x, st.d_status.p);
  EMT_CUDA(cudaGetLastError());
}

void Umma::expand(const Store& st, const MSimD& m, const int* path_ptr, const int* path_srow, int pass, int n1,
                  int record, int s_in_chunk, cudaStream_t s) {
  k_split_b<<<dim3(x_bblocks, xTN / 32), 32 * (UKC / 8), 0, s>>>(st.view(), x_bdesc.p, m.S, xb_blocks.p, R, xTN, x_bblocks, path_ptr,
                                      path_srow);
  UmmaArgs a;
  a.tiles = x_tiles_d.p;
  a.tile_b = x_tile_b.p;
  a.a_blocks = xa_blocks.p;
  a.b_blocks = xb_blocks.p;
  a.Y = m.Y;
  a.R = R;
  a.TN = xTN;
  a.ns = kExpandStages;
  a.r_act = m.R_act;
  ExpArgs x;
  x.m = m;
  x.pass = pass;
  x.n1 = n1;
  x.record = record;
  x.s_in_chunk = s_in_chunk;
  k_mc_umma<UMMA_EXPAND><<<x_tiles, 256, umma_smem_bytes(xTN, kExpandStages), s>>>(st.view(), a, x, st.d_status.p);
  EMT_CUDA(cudaGetLastError());
}

}  // namespace emt

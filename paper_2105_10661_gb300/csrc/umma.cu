// Leaf stage of the multi-column apply on the 5th-generation tensor cores (tcgen05).
//
//   Y[leaf rows, columns] = L_j * X_j,  L_j = L_hi + L_lo,  X = X_hi + X_lo  (BF16 splits)
//   Y ~= L_hi X_hi + L_hi X_lo + L_lo X_hi   (FP32 accumulation in tensor memory)
// The dropped L_lo X_lo term and the split residuals leave a relative error of about 2^-16;
// the multi-column step's float-float residual refinement removes it.
//
// Both operands are pre-tiled in global memory in the canonical K-major core-matrix layout
// (8 rows x 16 bytes per core matrix, no swizzle): A (the leaf blocks, split once per store) per
// (leaf, 128-row tile, 64-deep K chunk), B (the right-hand sides, split once per pass by
// k_split_b) per (leaf, TN-column tile, K chunk). One CTA computes a 128-row x TN-column tile of
// one leaf as a two-stage pipeline: one thread issues one cp.async.bulk per operand and chunk into
// a stage (full mbarrier), one thread issues tcgen05.mma (M = 128, N = TN, K = 16, kind::f16 with
// BF16 inputs) three times per K step and commits them to the stage's empty mbarrier, and the
// epilogue reads the accumulator with tcgen05.ld. Each mbarrier has a single waiter that waits
// for its phases in order; every wait is bounded by clock64 and reports a timeout in the device
// status word; tensor memory is always released.
#include <algorithm>
#include <cstdint>

#include <cuda_bf16.h>

#include "multi.h"

namespace emt {

namespace {

constexpr int UM = 128;            // MMA M (tile rows)
constexpr int UKC = 64;            // K chunk
constexpr uint32_t A_CHUNK = UM * UKC * 2;          // 16 KB per split
constexpr uint32_t A_SBO = 1024, A_LBO = 128;       // M-group stride, K-core stride
constexpr uint32_t B_SBO = 1024, B_LBO = 128;       // N-group stride, K-core stride
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

// A blocks: per (leaf, M tile, K chunk) 32 KB = [hi 16 KB | lo 16 KB], canonical layout.
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
  const int* tile_b;        // first B block of the tile's (leaf, N tile)
  const uint16_t* a_blocks; // pre-tiled leaf blocks
  const uint16_t* b_blocks; // pre-tiled right-hand sides
  float* Y;                 // [n][R]
  int R, TN;
  int r_act;                // columns in use; tiles starting beyond exit at once
};

// B blocks: per (leaf j, N tile, K chunk) [hi | lo], each TN x 64 BF16 in the canonical K-major
// layout (N-group stride 1024 bytes, K-core stride 128 bytes). Thread item = one column and 8
// consecutive k: one 16-byte core row per split.
__global__ void k_split_b(DStore st, const int4* __restrict__ bdesc, const float* __restrict__ Xf,
                          uint16_t* __restrict__ out, int R, int TN, int n_blk) {
  const int blk = blockIdx.x;
  if (blk >= n_blk) return;
  const int4 d = bdesc[blk];   // leaf, N tile first column, K chunk, unused
  const int node = st.leaf_node[d.x];
  const int lo = st.lo[node], b = st.hi[node] - lo;
  unsigned char* hi = reinterpret_cast<unsigned char*>(out) + (size_t)blk * 4 * TN * UKC;
  unsigned char* lob = hi + (size_t)2 * TN * UKC;
  for (int w = threadIdx.x; w < TN * (UKC / 8); w += blockDim.x) {
    const int n = w % TN, kg = w / TN;
    const int col = d.y + n;
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float x[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int k = d.z * UKC + kg * 8 + 2 * q + u;
        x[u] = (k < b && col < R) ? Xf[(int64_t)(lo + k) * R + col] : 0.f;
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

__global__ void __launch_bounds__(256, 1) k_mc_umma(DStore st, UmmaArgs a, int* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int TN = a.TN;
  const uint32_t b_split = (uint32_t)TN * UKC * 2;              // bytes of one B split
  const uint32_t stage_bytes = 2 * A_CHUNK + 2 * b_split;
  unsigned char* stg[2] = {sm, sm + stage_bytes};
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + 2 * stage_bytes);   // full0, full1, empty0, empty1, done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 5);
  int* flag = reinterpret_cast<int*>(bars + 6);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int4 tl = a.tiles[blockIdx.x];
  const int j = tl.x, m0 = tl.y, n0 = tl.z, blk0 = tl.w;
  const int bblk0 = a.tile_b[blockIdx.x];
  if (n0 >= a.r_act) return;   // uniform per CTA, before any barrier or tensor memory use
  const int node = st.leaf_node[j];
  const int lo = st.lo[node], b = st.hi[node] - lo;
  const int nkc = (b + UKC - 1) / UKC;
  if (tid == 0) {
    for (int i = 0; i < 5; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su(bars + i)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su(tslot)), "r"(TN)
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
    // producer: stage s = kc % 2 is refilled once the MMAs of chunk kc - 2 released it
    for (int kc = 0; kc < nkc; ++kc) {
      const int s = kc & 1;
      if (kc >= 2 && !bar_wait(bars + 2 + s, ((kc >> 1) - 1) & 1)) {
        atomicExch(status, DEV_TIMEOUT);
        atomicExch(flag, 1);
        break;
      }
      if (*reinterpret_cast<volatile int*>(flag)) break;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su(bars + s)), "r"(stage_bytes)
                   : "memory");
      bulk_g2s_u(stg[s], reinterpret_cast<const unsigned char*>(a.a_blocks) + (size_t)(blk0 + kc) * 2 * A_CHUNK,
                 2 * A_CHUNK, bars + s);
      bulk_g2s_u(stg[s] + 2 * A_CHUNK, reinterpret_cast<const unsigned char*>(a.b_blocks) + (size_t)(bblk0 + kc) * 2 * b_split,
                 2 * b_split, bars + s);
      ++issued;
    }
  } else if (tid == 32) {
    // MMA issuer
    for (int kc = 0; kc < nkc; ++kc) {
      const int s = kc & 1;
      if (!bar_wait(bars + s, (kc >> 1) & 1)) {
        atomicExch(status, DEV_TIMEOUT);
        atomicExch(flag, 1);
        break;
      }
      if (*reinterpret_cast<volatile int*>(flag)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_hi = su(stg[s]), a_lo = a_hi + A_CHUNK;
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
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su(bars + 2 + s))
                   : "memory");
      ++committed;
    }
    // all MMAs issued so far complete -> done
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su(bars + 4))
                 : "memory");
  }
  if (tid == 0) cnt_sh[0] = issued;
  if (tid == 32) cnt_sh[1] = committed;
  __syncthreads();
  // the issuer's last commit covers every MMA it issued
  __shared__ int ok_sh;
  if (tid == 32) {
    const bool ok = bar_wait(bars + 4, 0);
    if (!ok) atomicExch(status, DEV_TIMEOUT);
    ok_sh = ok && !*reinterpret_cast<volatile int*>(flag) && cnt_sh[1] == nkc;
  }
  if (tid == 0 && cnt_sh[0] > cnt_sh[1]) {
    // error path only: copies issued to stages the issuer never consumed; each is the latest use
    // of its stage (at most one per stage), so its phase parity is unambiguous
    for (int kc = cnt_sh[1]; kc < cnt_sh[0]; ++kc) bar_wait(bars + (kc & 1), (kc >> 1) & 1);
  }
  __syncthreads();
  const bool ok = ok_sh != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
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
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN) : "memory");
}

}  // namespace

// ---------------------------------------------------------------- host side
size_t umma_smem_bytes(int TN) { return 2 * (2 * (size_t)A_CHUNK + 2 * (size_t)TN * UKC * 2) + 64; }

void Umma::build(const Store& st, int R_, cudaStream_t s) {
  R = R_;
  TN = R >= 256 ? 256 : (R > 64 ? 128 : 64);
  const Tree& t = st.tree;
  std::vector<int> bl, bm, bk, tb;
  std::vector<int4> tiles, bdesc;
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
        tb.push_back(bfirst[nt]);
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
  d_tiles.alloc(tiles.size());
  EMT_CUDA(cudaMemcpyAsync(d_tiles.p, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
  // the attribute is per kernel, shared by every simulation: allow the largest tile
  EMT_CUDA(cudaFuncSetAttribute(k_mc_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)umma_smem_bytes(256)));
  EMT_CUDA(cudaStreamSynchronize(s));   // the index lists above are freed on return
  ready = true;
}

void Umma::launch(const Store& st, const float* Xf, float* Y, cudaStream_t s, int r_act) {
  k_split_b<<<n_bblocks, 256, 0, s>>>(st.view(), b_desc.p, Xf, b_blocks.p, R, TN, n_bblocks);
  UmmaArgs a;
  a.tiles = d_tiles.p;
  a.tile_b = tile_b.p;
  a.a_blocks = a_blocks.p;
  a.b_blocks = b_blocks.p;
  a.Y = Y;
  a.R = R;
  a.TN = TN;
  a.r_act = r_act;
  k_mc_umma<<<n_tiles, 256, umma_smem_bytes(TN), s>>>(st.view(), a, st.d_status.p);
  EMT_CUDA(cudaGetLastError());
}

}  // namespace emt

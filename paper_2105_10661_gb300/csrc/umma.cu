// Leaf stage of the multi-column apply on the 5th-generation tensor cores (tcgen05).
//
//   Y[leaf rows, columns] = L_j * X_j,  L_j = L_hi + L_lo,  X = X_hi + X_lo  (BF16 splits)
//   Y ~= L_hi X_hi + L_hi X_lo + L_lo X_hi   (FP32 accumulation in tensor memory)
// The dropped L_lo X_lo term and the split residuals leave a relative error of about 2^-16;
// the multi-column step's float-float residual refinement removes it.
//
// One CTA computes a 128-row x TN-column tile of one leaf. K runs in chunks of 64, double
// buffered in shared memory:
//   A (L_hi | L_lo)   pre-tiled in global memory in the canonical K-major core-matrix layout
//                     (8 rows x 16 bytes per core matrix), one 32 KB cp.async.bulk per chunk;
//   B (X_hi, X_lo)    split from the FP32 right-hand sides by all threads and stored K-major
//                     with an N-group stride of 1040 bytes (1024 + 16 rotates the banks, so
//                     the 32 threads of a warp store to 32 different banks).
// One elected thread issues tcgen05.mma (M = 128, N = TN, K = 16, kind::f16 with BF16 inputs)
// three times per K step and commits them to an mbarrier; the epilogue reads the accumulator
// with tcgen05.ld. Every mbarrier wait is bounded by clock64 and reports a timeout in the
// device status word; tensor memory is always released.
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
constexpr uint32_t B_SBO = 1040, B_LBO = 128;       // N-group stride (padded), K-core stride
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
  const uint16_t* a_blocks; // pre-tiled leaf blocks
  const float* Xf;          // [n][R]
  float* Y;                 // [n][R]
  int R, TN, nkc_max;
  int r_act;                // columns in use; tiles starting beyond exit at once
};

// Stage the B chunk (rows k0..k0+63 of the leaf, columns n0..n0+TN) as BF16 hi/lo.
__device__ __forceinline__ void stage_b(const UmmaArgs& a, int lo_pos, int b, int k0, int n0, unsigned char* Bh,
                                        unsigned char* Bl) {
  // item -> (k pair kp, 4-column group n4); the 32 lanes of a warp take 4 k pairs x 8 column
  // groups, which with the 1040-byte N-group stride puts their 32-bit stores in 32 banks
  const int TN = a.TN;
  const int nb4 = TN / 32;                // blocks of 8 column groups
  const int total = (UKC / 2) * (TN / 4);
  for (int w = threadIdx.x; w < total; w += blockDim.x) {
    const int lane = w & 31, wi = w >> 5;
    const int kp = (wi / nb4) * 4 + (lane & 3);
    const int n4 = (wi % nb4) * 8 + (lane >> 2);
    const int k = 2 * kp;
    const int n = 4 * n4;
    float x0[4] = {0.f, 0.f, 0.f, 0.f}, x1[4] = {0.f, 0.f, 0.f, 0.f};
    const int gk0 = k0 + k, gk1 = k0 + k + 1;
    if (n0 + n < a.R) {   // R is a multiple of 4, so the 4 columns are all valid and aligned
      if (gk0 < b) {
        const float4 v = *reinterpret_cast<const float4*>(a.Xf + (int64_t)(lo_pos + gk0) * a.R + n0 + n);
        x0[0] = v.x; x0[1] = v.y; x0[2] = v.z; x0[3] = v.w;
      }
      if (gk1 < b) {
        const float4 v = *reinterpret_cast<const float4*>(a.Xf + (int64_t)(lo_pos + gk1) * a.R + n0 + n);
        x1[0] = v.x; x1[1] = v.y; x1[2] = v.z; x1[3] = v.w;
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int nn = n + q;
      const uint16_t h0 = bf16_bits(x0[q]), h1 = bf16_bits(x1[q]);
      const uint16_t l0 = bf16_bits(x0[q] - bf16_val(h0)), l1 = bf16_bits(x1[q] - bf16_val(h1));
      const uint32_t off = (nn / 8) * B_SBO + (k / 8) * B_LBO + ((nn % 8) * 8 + (k % 8)) * 2;
      *reinterpret_cast<uint32_t*>(Bh + off) = (uint32_t)h0 | ((uint32_t)h1 << 16);
      *reinterpret_cast<uint32_t*>(Bl + off) = (uint32_t)l0 | ((uint32_t)l1 << 16);
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__global__ void __launch_bounds__(256, 1) k_mc_umma(DStore st, UmmaArgs a, int* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int TN = a.TN;
  const uint32_t b_bytes = (uint32_t)(TN / 8) * B_SBO;
  unsigned char* Abuf[2] = {sm, sm + 2 * A_CHUNK};
  unsigned char* Bh[2] = {sm + 4 * A_CHUNK, sm + 4 * A_CHUNK + 2 * b_bytes};
  unsigned char* Bl[2] = {Bh[0] + b_bytes, Bh[1] + b_bytes};
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + 4 * A_CHUNK + 4 * b_bytes);   // a0, a1, m0, m1
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 4);
  int* flag = reinterpret_cast<int*>(bars + 5);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int4 tl = a.tiles[blockIdx.x];
  const int j = tl.x, m0 = tl.y, n0 = tl.z, blk0 = tl.w;
  if (n0 >= a.r_act) return;   // uniform per CTA, before any barrier or tensor memory use
  const int node = st.leaf_node[j];
  const int lo = st.lo[node], b = st.hi[node] - lo;
  const int nkc = (b + UKC - 1) / UKC;
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su(bars + i)) : "memory");
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
  auto issue_a = [&](int kc) {
    const int s = kc & 1;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su(bars + s)), "r"(2 * A_CHUNK)
                 : "memory");
    const unsigned char* src = reinterpret_cast<const unsigned char*>(a.a_blocks) + (size_t)(blk0 + kc) * 2 * A_CHUNK;
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su(Abuf[s])),
                 "l"(src), "r"(2 * A_CHUNK), "r"(su(bars + s))
                 : "memory");
  };
  bool ok = true;
  int last_a = 0, last_mma = -1;   // chunk indices of the last bulk copy and MMA batch issued (thread 0)
  if (tid == 0) issue_a(0);
  stage_b(a, lo, b, 0, n0, Bh[0], Bl[0]);
  for (int kc = 0; kc < nkc; ++kc) {
    const int s = kc & 1;
    __syncthreads();
    if (*flag) break;
    if (tid == 0) {
      if (!bar_wait(bars + s, (kc >> 1) & 1)) {
        atomicExch(status, DEV_TIMEOUT);
        *flag = 1;
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a_hi = su(Abuf[s]), a_lo = a_hi + A_CHUNK;
        const uint32_t b_hi = su(Bh[s]), b_lo = su(Bl[s]);
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
        last_mma = kc;
      }
    }
    if (kc + 1 < nkc) {
      const int s2 = (kc + 1) & 1;
      if (kc + 1 >= 2) {
        // the MMAs of chunk kc - 1 read buffer s2: wait before overwriting it
        if (!bar_wait(bars + 2 + s2, ((kc - 1) >> 1) & 1)) {
          if (tid == 0) atomicExch(status, DEV_TIMEOUT);
          *flag = 1;
        }
      }
      __syncthreads();
      if (*flag) break;
      if (tid == 0) {
        issue_a(kc + 1);
        last_a = kc + 1;
      }
      stage_b(a, lo, b, (kc + 1) * UKC, n0, Bh[s2], Bl[s2]);
    }
  }
  __syncthreads();
  ok = (*flag == 0);
  if (!ok && tid == 0) {
    // give the copy and the MMAs still in flight a bounded chance to land before tensor memory
    // and shared memory are released
    bar_wait(bars + (last_a & 1), (last_a >> 1) & 1);
    if (last_mma >= 0) bar_wait(bars + 2 + (last_mma & 1), (last_mma >> 1) & 1);
  }
  if (ok) {
    const int last = nkc - 1;
    if (!bar_wait(bars + 2 + (last & 1), (last >> 1) & 1)) {
      if (tid == 0) atomicExch(status, DEV_TIMEOUT);
      ok = false;
    }
  }
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
size_t umma_smem_bytes(int TN) { return 4 * (size_t)A_CHUNK + 4 * (size_t)(TN / 8) * B_SBO + 64; }

void Umma::build(const Store& st, int R_, cudaStream_t s) {
  R = R_;
  TN = R >= 256 ? 256 : (R > 64 ? 128 : 64);
  const Tree& t = st.tree;
  std::vector<int> bl, bm, bk;
  std::vector<int4> tiles;
  for (int j = 0; j < st.n_leaf; ++j) {
    const int b = t.hi[st.leaf_nodes_h[j]] - t.lo[st.leaf_nodes_h[j]];
    const int nmt = (b + UM - 1) / UM, nkc = (b + UKC - 1) / UKC;
    for (int mt = 0; mt < nmt; ++mt) {
      const int first = (int)bl.size();
      for (int kc = 0; kc < nkc; ++kc) {
        bl.push_back(j);
        bm.push_back(mt);
        bk.push_back(kc);
      }
      for (int n0 = 0; n0 < R; n0 += TN) tiles.push_back(make_int4(j, mt * UM, n0, first));
    }
  }
  n_blocks = (int)bl.size();
  n_tiles = (int)tiles.size();
  DevBuf<int> dl, dm, dk;
  dl.upload(bl, s);
  dm.upload(bm, s);
  dk.upload(bk, s);
  a_blocks.alloc((size_t)n_blocks * A_CHUNK);   // uint16 count: 2 splits x A_CHUNK bytes / 2
  k_tile_leaves<<<n_blocks, 256, 0, s>>>(st.view(), dl.p, dm.p, dk.p, a_blocks.p, n_blocks);
  d_tiles.alloc(tiles.size());
  EMT_CUDA(cudaMemcpyAsync(d_tiles.p, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
  // the attribute is per kernel, shared by every simulation: allow the largest tile
  EMT_CUDA(cudaFuncSetAttribute(k_mc_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)umma_smem_bytes(256)));
  EMT_CUDA(cudaStreamSynchronize(s));   // the index lists above are freed on return
  ready = true;
}

void Umma::launch(const Store& st, const float* Xf, float* Y, cudaStream_t s, int r_act) {
  UmmaArgs a;
  a.tiles = d_tiles.p;
  a.a_blocks = a_blocks.p;
  a.Xf = Xf;
  a.Y = Y;
  a.R = R;
  a.TN = TN;
  a.nkc_max = 0;
  a.r_act = r_act;
  k_mc_umma<<<n_tiles, 256, umma_smem_bytes(TN), s>>>(st.view(), a, st.d_status.p);
  EMT_CUDA(cudaGetLastError());
}

}  // namespace emt

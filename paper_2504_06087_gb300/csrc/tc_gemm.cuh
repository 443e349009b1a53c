// Tensor-core matrix product on sm_103a: C[M][N] (fp32) = A[M][K] (bf16) *
// B (bf16, given as Bt[N][K], K-major), with tcgen05.mma (kind::f16, FP32
// accumulator in tensor memory) fed by TMA (cp.async.bulk.tensor, 128-byte
// swizzle) through an mbarrier pipeline.
//
// A persistent grid of 192-thread CTAs walks the 128 x BN output tiles
// (N tiles fastest, so CTAs that share an A tile run together and the
// second reads it from L2).  Warp 0 lane 0 streams A and B k-blocks through
// a ring of STAGES shared-memory stages (TMA), warp 1 lane 0 issues the MMAs
// into one of two tensor-memory accumulators, and warps 2-5 drain the other
// accumulator (tcgen05.ld 32x32b, each warp its 32-lane quarter; every lane
// stores its row's 32-column slices straight from registers with 128-bit
// stores), so a tile's epilogue overlaps the next tile's main loop.  The row range of A may live on the
// device ({begin, end}).  Where C allows a tensor map (16-byte aligned rows),
// the full 128-row tiles leave through TMA instead: each epilogue warp
// writes its 32 x 32 chunk into a 128-byte-swizzled shared buffer
// (conflict-free) and one lane stores it with cp.async.bulk.tensor, so the
// L1 -> L2 path carries whole lines rather than a 16-byte piece of 32 rows
// per store instruction (that request path, 76 % busy, bounded the product).
//
// Every mbarrier wait is bounded: after kSpinLimit polls the kernel records
// an error in *err, stops issuing work, waits (bounded) for its own copies
// and MMAs already in flight, frees its tensor memory and returns.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fire {
namespace tc {

constexpr int BM = 128;
constexpr int BK = 64;                // one 128-byte swizzle row of bf16
constexpr int UMMA_K = 16;
constexpr uint32_t kSpinLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false after kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < kSpinLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"((uint64_t)map),
               "r"(smem_u32(src)), "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the shared-memory sources of this thread's bulk stores have been read
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// this thread's bulk stores are complete
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the async proxy (TMA)
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// K-major operand tile, 128-byte swizzle: rows of 128 bytes, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1 (sm_100 form).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(1) << 16;                       // leading byte offset (unused for this layout)
  d |= (uint64_t)((1024 >> 4) & 0x3FFF) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;                         // descriptor version
  d |= (uint64_t)2 << 61;                         // 128-byte swizzle
  return d;
}

// Instruction descriptor: D fp32, A and B bf16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// 32 consecutive fp32 columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

struct TcArgs {
  float* C;
  int64_t ldc;
  int64_t m_begin, m_end;        // used when m_range == nullptr
  const int64_t* m_range;
  int N, K, BN;                  // BN multiple of 16, <= 256
  int64_t a_comp_rows;           // rows between the bf16 components of A
  int64_t b_comp_rows;           // rows between the bf16 components of Bt
  int64_t b_row0;                // first row of Bt inside each component
  int* err;                      // device error word (timeouts)
  int c_tma;                     // full tiles leave through the C tensor map
};

// Split-bf16 products (Henry, Tang & Heinecke 2019): a value x is stored as
// NC bf16 components x0 + x1 + x2; the product sums the component pairs
// (p, q) with p + q < NC, smallest terms first.  NC = 1 is plain bf16, NC = 2
// takes 3 products, NC = 3 takes 6.
__host__ __device__ constexpr int split_count(int nc) { return nc == 1 ? 1 : (nc == 2 ? 3 : 6); }
__host__ __device__ constexpr int split_p(int nc, int k) {
  return nc == 1 ? 0 : (nc == 2 ? (k == 0 ? 1 : 0) : (k == 0 ? 2 : (k == 1 ? 1 : (k == 2 ? 0 : (k == 3 ? 1 : 0)))));
}
__host__ __device__ constexpr int split_q(int nc, int k) {
  return nc == 1 ? 0 : (nc == 2 ? (k == 1 ? 1 : 0) : (k == 0 ? 0 : (k == 1 ? 1 : (k == 2 ? 2 : (k == 4 ? 1 : 0)))));
}

// Dynamic shared memory: STAGES x NC x (A tile 16 KB + B tile BN*128 B),
// then one 4 KB store buffer (32 rows x 32 fp32, 128-byte swizzle) per
// epilogue warp, 1024-aligned.
constexpr int kEpiWarps = 4;
constexpr int kStoreBuf = 32 * 32 * 4;
__host__ __device__ inline size_t tc_smem_bytes(int stages, int nc, int bn) {
  return (size_t)stages * nc * ((size_t)BM * BK * 2 + (size_t)bn * BK * 2) + (size_t)kEpiWarps * kStoreBuf + 1024;
}

template <int STAGES, int NC>
__global__ void __launch_bounds__(192, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
               const __grid_constant__ CUtensorMap mapC, TcArgs g) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], tfull_bar[2], tempty_bar[2], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  int64_t mb = g.m_begin, me = g.m_end;
  if (g.m_range) { mb = g.m_range[0]; me = g.m_range[1]; }
  const int BN = g.BN;
  const int64_t n_mt = me > mb ? (me - mb + BM - 1) / BM : 0;
  const int n_nt = (g.N + BN - 1) / BN;
  const int64_t ntiles = n_mt * n_nt;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t a_bytes = BM * BK * 2, b_bytes = (uint32_t)BN * BK * 2;
  const uint32_t stage_bytes = NC * (a_bytes + b_bytes);
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
  uint32_t ncols = 32;
  while ((int)ncols < 2 * BN) ncols <<= 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&tfull_bar[b], 1); mbar_init(&tempty_bar[b], kEpiWarps); }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tmem_slot, ncols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_slot;
  const int nk = g.K / BK;

  if (warp == 0 && lane == 0) {
    // TMA producer: runs ahead across tiles through the stage ring
    int64_t it = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const int64_t m0 = mb + (t / n_nt) * BM;
      const int n0 = (int)(t % n_nt) * BN;
      for (int kb = 0; kb < nk; ++kb, ++it) {
        const int s = (int)(it % STAGES);
        if (it >= STAGES && !mbar_wait(&empty_bar[s], (uint32_t)((it / STAGES) - 1) & 1)) {
          atomicExch(g.err, 1); abort_flag = 1; ok = false; break;
        }
        if (abort_flag) { ok = false; break; }
        unsigned char* sa = base + (size_t)s * stage_bytes;
        mbar_expect_tx(&full_bar[s], stage_bytes);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          tma_load_2d(sa + c * a_bytes, &mapA, &full_bar[s], kb * BK, (int)(c * g.a_comp_rows + m0));
          tma_load_2d(sa + NC * a_bytes + c * b_bytes, &mapB, &full_bar[s], kb * BK, (int)(c * g.b_comp_rows + g.b_row0 + n0));
        }
      }
    }
    if (!ok) {
      // let the copies already issued land before the CTA can exit
      for (int64_t j = (it > STAGES ? it - STAGES : 0); j < it; ++j)
        mbar_wait(&full_bar[j % STAGES], (uint32_t)(j / STAGES) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = idesc_bf16(BM, BN);
    int64_t it = 0, tl = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tl) {
      const int buf = (int)(tl & 1);
      if (tl >= 2 && !mbar_wait(&tempty_bar[buf], (uint32_t)((tl / 2) - 1) & 1)) {
        atomicExch(g.err, 4); abort_flag = 1; ok = false; break;
      }
      fence_after_sync();
      const uint32_t d = tmem + (uint32_t)(buf * BN);
      for (int kb = 0; kb < nk; ++kb, ++it) {
        const int s = (int)(it % STAGES);
        if (abort_flag || !mbar_wait(&full_bar[s], (uint32_t)(it / STAGES) & 1)) {
          atomicExch(g.err, 2); abort_flag = 1; ok = false; break;
        }
        fence_after_sync();
        const uint32_t sa = smem_u32(base + (size_t)s * stage_bytes);
        const uint32_t sb = sa + NC * a_bytes;
#pragma unroll
        for (int pr = 0; pr < split_count(NC); ++pr) {
          const uint32_t ap = sa + split_p(NC, pr) * a_bytes;
          const uint32_t bq = sb + split_q(NC, pr) * b_bytes;
#pragma unroll
          for (int k = 0; k < BK / UMMA_K; ++k) {
            const uint64_t ad = smem_desc_sw128(ap + k * UMMA_K * 2);
            const uint64_t bd = smem_desc_sw128(bq + k * UMMA_K * 2);
            mma_bf16(d, ad, bd, idesc, (kb > 0 || pr > 0 || k > 0) ? 1u : 0u);
          }
        }
        mma_commit(&empty_bar[s]);
      }
      if (ok) mma_commit(&tfull_bar[buf]);
    }
    mma_commit(&done_bar);   // arrives once every MMA issued above is complete
    if (!mbar_wait(&done_bar, 0)) atomicExch(g.err, 5);
  } else if (warp >= 2) {
    // epilogue: warp w drains tensor-memory lanes 32 (w % 4) .. + 31
    const int q = warp & 3;
    unsigned char* stbuf = base + (size_t)STAGES * stage_bytes;   // 1024-aligned (stage_bytes is)
    const bool vec = (g.ldc % 4 == 0) && ((reinterpret_cast<uintptr_t>(g.C) & 15) == 0);
    int64_t tl = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++tl) {
      const int buf = (int)(tl & 1);
      bool ok = true;
      if (abort_flag) ok = false;
      else if (!mbar_wait(&tfull_bar[buf], (uint32_t)(tl / 2) & 1)) {
        if (lane == 0) atomicExch(g.err, 3);
        abort_flag = 1;
        ok = false;
      }
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      fence_after_sync();
      const int64_t m0 = mb + (t / n_nt) * BM;
      const int n0 = (int)(t % n_nt) * BN;
      const int ncol = min(BN, g.N - n0);
      const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * BN);
      // lane = row m0 + 32 q + lane: its 32 accumulator columns of a chunk go
      // straight from registers to its row of C (eight 128-bit stores)
      const int64_t row = m0 + 32 * q + lane;
      float* crow = g.C + row * g.ldc + n0;
      // full-row tiles through the tensor map: a 32-column box either lies
      // inside the tile or runs past N (clipped by the map); a box that
      // would reach into the next tile (BN not a multiple of 32) takes the
      // direct stores
      const bool tma = g.c_tma && m0 + BM <= me;
      const bool last_nt = n0 + ncol == g.N;
      for (int c0 = 0; c0 < BN; c0 += 32) {
        float v[32];
        tmem_ld32(tbase + (uint32_t)c0, v);
        const int nval = ncol - c0;
        if (tma && nval > 0 && (nval >= 32 || last_nt)) {
          // the previous chunk's store has read the buffer
          if (lane == 0) bulk_wait_read0();
          __syncwarp();
          unsigned char* sb = stbuf + (size_t)q * kStoreBuf + (size_t)lane * 128;
#pragma unroll
          for (int j = 0; j < 8; ++j)
            *reinterpret_cast<float4*>(sb + ((j ^ (lane & 7)) << 4)) =
                make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) {
            tma_store_2d(&mapC, stbuf + (size_t)q * kStoreBuf, n0 + c0, (int)(m0 + 32 * q));
            bulk_commit();
          }
          continue;
        }
        if (row < me && nval > 0) {
          if (vec && nval >= 32) {
            float4* d4 = reinterpret_cast<float4*>(crow + c0);
#pragma unroll
            for (int j = 0; j < 8; ++j) d4[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (j < nval) crow[c0 + j] = v[j];
          }
        }
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_expect_tx(&tempty_bar[buf], 0);   // one arrival per epilogue warp
    }
    // this warp's tensor stores complete before the CTA (and its shared memory) ends
    if (lane == 0) bulk_wait0();
    __syncwarp();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

}  // namespace tc
}  // namespace fire

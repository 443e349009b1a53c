// Restricted log-det contraction on the tensor cores (Methods, "Efficient
// Laplacian", eq. logdet_lowrank): for every tangent electron n' with
// neighbourhood Nbar = {i_0 = n', i_1, ..., i_{m-1}} and determinant d,
//   T[(k,x)][l] = d Phi_{i_k l} / d r_{n' x}
//               = O_{(i_k, slot of n', x)}[l] phi_l(r_{i_k})  (+ O_{i_k}[l] d_x phi_l(r_{n'}) for k = 0)
//   T[3m][l]    = Lap Phi_{n' l}   (the Laplacian row of n')
//   M[(k,x)][k'] = sum_l T[(k,x)][l] A[l][i_k']           (A = Phi^-1, rows of A^T)
// and from M
//   d log det / d r_{n'x} = sum_k M[(k,x)][k]
//   Lap part of n'        = M[3m][0] - sum_x sum_{k,k'} M[(k,x)][k'] M[(k',x)][k].
// M is one tcgen05 product per (tangent electron, determinant): the 3m + 1
// rows of T are the A operand (M = 128 rows, so m <= 42), the m rows of A^T
// the B operand (N = m rounded up to 16), K = the orbitals l in 64-orbital
// chunks.  Both operands are split-bf16 (two components, the products
// hi hi + hi lo + lo hi).
//
// Persistent CTAs of 256 threads, two per SM, each with one operand buffer
// and 64 columns of tensor memory, walk a list of tangent electrons; an item
// is a tangent electron with the G determinants of an orbital group (its
// member metadata is resolved once).  Per 64-orbital chunk every thread loads
// the float32 rows of its first (member, 8-orbital) task into registers and
// one piece of n''s own ten rows (O value, Laplacian and tangents, envelope
// value, Laplacian and gradient) -- while the tensor cores still multiply the
// previous chunk -- then forms T and the Laplacian row, splits them and
// stores both operands in the 128-byte-swizzled K-major layout; one thread
// issues the chunk's MMAs.  After the last chunk of a determinant warps 0-3
// read M from tensor memory (each its 32-lane quarter) into the operand
// buffer and all threads reduce the gradient and the trace.  Memory latency
// is hidden by the other CTA of the SM.  Every mbarrier wait is bounded (an
// error in *err, the CTA stops after its MMAs in flight have completed).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fire.h"
#include "common.cuh"
#include "tc_api.h"
#include "tc_gemm.cuh"

namespace fire {
namespace tc {

constexpr int kCtMaxM = kContractTcMaxMembers;   // 3 m + 1 <= 128 rows of T
constexpr int kCtMaxG = 4;                       // determinants per item
constexpr int kCtBN = 48;                        // B rows reserved per component (members, padded to 16)
constexpr int kCtThreads = 256;
constexpr int kCtPerSm = 2;                      // resident CTAs per SM (up to 128 registers a thread)
constexpr int kCtMsStride = 43;                  // M rows in shared memory (odd: conflict-free columns)
constexpr int kCtTmemCols = 64;
constexpr uint32_t kCtABytes = 128 * 128;        // 128 rows x 64 bf16
constexpr uint32_t kCtBBytes = kCtBN * 128;
constexpr uint32_t kCtBufBytes = 2 * (kCtABytes + kCtBBytes);
constexpr size_t kCtSmemBytes = kCtBufBytes + 1024;
static_assert((size_t)(3 * kCtMaxM + 1) * kCtMsStride * 4 <= kCtBufBytes, "M must fit the operand buffer");
static_assert(3 * kCtMaxM + 1 <= 128 && kCtMaxM <= kCtBN && kCtBN <= kCtTmemCols && kCtMaxM <= kCtThreads && 10 * 16 <= kCtThreads,
              "a neighbourhood must fit one 128-row tile, the B rows and the accumulator");
static_assert(kCtPerSm * (kCtSmemBytes + 2048) <= 228 * 1024 && kCtPerSm * kCtTmemCols <= 512,
              "resident CTAs exceed shared or tensor memory");

// Eight consecutive elements p[l .. l + 7] (zero at and beyond n; n % 4 == 0,
// p 16-byte aligned).  O rows are read once: no L1 allocation.
template <bool STREAM>
__device__ __forceinline__ void ld8(const float* p, int l, int n, float v[8]) {
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
  if (STREAM) {
    if (l < n)
      asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                   : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w) : "l"(p + l));
    if (l + 4 < n)
      asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                   : "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w) : "l"(p + l + 4));
  } else {
    if (l < n) a = __ldg(reinterpret_cast<const float4*>(p + l));
    if (l + 4 < n) b = __ldg(reinterpret_cast<const float4*>(p + l + 4));
  }
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// Row r, 16-byte chunk j (elements 8 j .. 8 j + 7 of a 64-element K chunk)
// of a 128-byte-swizzled K-major tile, written as two bf16 components
// comp_bytes apart (hi = bf16(v), lo = bf16(v - hi)).
__device__ __forceinline__ void store_split8(unsigned char* tile, uint32_t comp_bytes, int r, int j, const float* v) {
  uint32_t hi[4], lo[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
    const float2 back = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(v[2 * q] - back.x, v[2 * q + 1] - back.y);
    hi[q] = *reinterpret_cast<const uint32_t*>(&h);
    lo[q] = *reinterpret_cast<const uint32_t*>(&l);
  }
  unsigned char* dst = tile + (size_t)r * 128 + ((j ^ (r & 7)) << 4);
  *reinterpret_cast<uint4*>(dst) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
  *reinterpret_cast<uint4*>(dst + comp_bytes) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
}

// 16 consecutive fp32 columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// Members of tangent electron e's neighbourhood, capped at the 42 that fit
// the tile (the caller's list holds no larger neighbourhood; a cap is
// reported through *err).
__device__ __forceinline__ int ct_members(const int32_t* cnt, int e) {
  const int m = 1 + cnt[2 * (int64_t)e] + cnt[2 * (int64_t)e + 1];
  return m < kCtMaxM ? m : kCtMaxM;
}

struct CtArgs {
  int Wc, n, n_up, K, dd0, G, D;
  const int32_t *idx, *cnt, *rev;
  const int64_t* blk_off;
  const float* O;   // orbital rows of determinants dd0 .. dd0 + G - 1 (det j at column j n)
  int64_t ldo;
  const float *Fenv, *AT;
  float *gdet, *ldet;
  DevStatus* st;
  const int* list;
  int nitems;
  int* err;
};

// The float32 rows of one (member k < m, 8-orbital) task: envelope value,
// the three tangent O rows, the A^T row.
struct CtTask {
  float ph[8], o0[8], o1[8], o2[8], av[8];
};

__global__ void __launch_bounds__(kCtThreads, kCtPerSm) contract_tc_kernel(const CtArgs a) {
  extern __shared__ __align__(1024) unsigned char ct_smem_raw[];
  __shared__ uint64_t mma_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int64_t s_ro[kCtMaxM], s_fo[kCtMaxM];
  __shared__ int32_t s_mi[kCtMaxM];
  __shared__ float red[kCtThreads / 32][5];
  // n''s own rows of the current chunk: O value, Laplacian and three tangent
  // rows, envelope value, Laplacian and three gradient rows
  __shared__ __align__(16) float s_self[10][64];

  unsigned char* buf =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(ct_smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char* sa = buf;                    // T, two components
  unsigned char* sb = buf + 2 * kCtABytes;    // A^T rows, two components
  float* Ms = reinterpret_cast<float*>(buf);  // M after a determinant's last MMA
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = a.n, G = a.G;
  const int nkc = (n + 63) / 64;
  const int64_t Dn = (int64_t)a.D * n;

  if (tid == 0) {
    mbar_init(&mma_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tmem_slot, kCtTmemCols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_slot;
  uint32_t phase = 0;     // parity of the next mma_bar completion
  bool pending = false;   // MMAs committed to mma_bar and not yet awaited
  bool ok = true;

  // waits for the committed MMAs (every thread); false on a timeout (they
  // stay pending)
  auto wait_mma = [&]() -> bool {
    if (!pending) return true;
    if (!mbar_wait(&mma_bar, phase)) return false;
    phase ^= 1u;
    pending = false;
    return true;
  };

  for (int it = blockIdx.x; it < a.nitems && ok; it += gridDim.x) {
    const int e = a.list[it];
    const int w = e / n, np = e - w * n;
    const int64_t eb = e;
    const int m = ct_members(a.cnt, e);
    __syncthreads();   // the previous item's metadata is no longer read
    if (tid < m) {
      const int k = tid;
      int i = np, sl = 0;
      if (k > 0) {
        i = a.idx[eb * a.K + k - 1];
        const int rv = a.rev[eb * a.K + k - 1];
        sl = rv < 0 ? -1 : rv + 1;
        if (rv < 0) atomicExch(&a.st->overflow, 1);
      }
      const int64_t b = block_index(w, i, a.Wc, n, a.n_up);
      s_mi[k] = i;
      s_ro[k] = sl < 0 ? -1 : (a.blk_off[b] + 2 + 3 * (int64_t)sl) * a.ldo;
      s_fo[k] = b * 5 * Dn + (int64_t)a.dd0 * n;
    }
    if (tid == 0 && m != 1 + a.cnt[eb * 2] + a.cnt[eb * 2 + 1]) atomicExch(a.err, 16);
    __syncthreads();
    const int64_t onp = s_ro[0] - 2 * a.ldo;   // n''s value row
    const int64_t fnp = s_fo[0];               // n''s envelope value row
    const int ntask = (m + 1) * 8;
    const uint32_t idesc = idesc_bf16(128, (m + 15) / 16 * 16);

    for (int dj = 0; dj < G && ok; ++dj) {
      const int64_t cofs = (int64_t)dj * n;
      const float* Aw = a.AT + ((int64_t)w * a.D + a.dd0 + dj) * n * n;
      for (int c = 0; c < nkc; ++c) {
        const int l0 = 64 * c;
        // the float32 rows of a member task (none for the Laplacian row)
        auto load_task = [&](int t, CtTask& x) {
          const int k = t >> 3, l = l0 + 8 * (t & 7);
          if (k >= m) return;
          const int64_t ro = s_ro[k];
          ld8<false>(a.Fenv + s_fo[k] + cofs, l, n, x.ph);
          if (ro >= 0) {
            ld8<true>(a.O + ro + cofs, l, n, x.o0);
            ld8<true>(a.O + ro + a.ldo + cofs, l, n, x.o1);
            ld8<true>(a.O + ro + 2 * a.ldo + cofs, l, n, x.o2);
          } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) x.o0[q] = x.o1[q] = x.o2[q] = 0.f;
          }
          ld8<false>(Aw + (int64_t)s_mi[k] * n, l, n, x.av);
        };
        // this thread's first task and its piece of n''s own rows are
        // loaded before waiting for the tensor cores to release the buffer
        CtTask td;
        if (tid < ntask) load_task(tid, td);
        float4 sv = make_float4(0.f, 0.f, 0.f, 0.f);
        {
          const int row = tid >> 4, l = l0 + 4 * (tid & 15);   // 160 float4 pieces of the 10 rows
          if (tid < 160 && l < n) {
            const float* src = row < 5 ? a.O + onp + row * a.ldo + cofs + l : a.Fenv + fnp + (row - 5) * Dn + cofs + l;
            sv = __ldg(reinterpret_cast<const float4*>(src));
          }
        }
        // the previous chunk's transform read these rows before the barrier
        // that preceded its MMAs; the barrier below publishes them
        if (tid < 160) *reinterpret_cast<float4*>(&s_self[tid >> 4][4 * (tid & 15)]) = sv;
        ok = wait_mma();
        if (__syncthreads_or(!ok)) { ok = false; break; }
        fence_after_sync();   // the tensor cores have finished reading the buffer
        // task t = 8 k + j: member k (or the Laplacian row, k = m), orbitals l0 + 8 j ..
        auto finish = [&](int t, CtTask& x) {
          const int k = t >> 3, j = t & 7;
          if (k < m) {
#pragma unroll
            for (int q = 0; q < 8; ++q) { x.o0[q] *= x.ph[q]; x.o1[q] *= x.ph[q]; x.o2[q] *= x.ph[q]; }
            if (k == 0) {
              // n' itself: its envelope moves too (value row of n' times the envelope gradient)
              const float* ov = &s_self[0][8 * j];
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                x.o0[q] = fmaf(ov[q], s_self[7][8 * j + q], x.o0[q]);
                x.o1[q] = fmaf(ov[q], s_self[8][8 * j + q], x.o1[q]);
                x.o2[q] = fmaf(ov[q], s_self[9][8 * j + q], x.o2[q]);
              }
            }
            store_split8(sa, kCtABytes, 3 * k, j, x.o0);
            store_split8(sa, kCtABytes, 3 * k + 1, j, x.o1);
            store_split8(sa, kCtABytes, 3 * k + 2, j, x.o2);
            store_split8(sb, kCtBBytes, k, j, x.av);
          } else {
            // Laplacian row of n': O_lap phi + O_val Lap phi + 2 sum_x O_x d_x phi
            float lap[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int lq = 8 * j + q;
              float v = fmaf(s_self[0][lq], s_self[6][lq], s_self[1][lq] * s_self[5][lq]);
#pragma unroll
              for (int xx = 0; xx < 3; ++xx) v = fmaf(2.f * s_self[2 + xx][lq], s_self[7 + xx][lq], v);
              lap[q] = v;
            }
            store_split8(sa, kCtABytes, 3 * m, j, lap);
          }
        };
        if (tid < ntask) finish(tid, td);
        for (int t = tid + kCtThreads; t < ntask; t += kCtThreads) {
          CtTask x;
          load_task(t, x);
          finish(t, x);
        }
        fence_proxy_async_smem();   // the operands are visible to the tensor cores
        __syncthreads();
        if (tid == 0) {
          fence_after_sync();
          const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sb);
          const int rem = n - l0;
          const int nks = rem >= 64 ? 4 : (rem + 15) / 16;   // 16-orbital steps holding orbitals < n
#pragma unroll
          for (int pr = 0; pr < 3; ++pr) {
            // hi hi, hi lo, lo hi
            const uint32_t ap = a0 + (pr == 2 ? kCtABytes : 0u);
            const uint32_t bq = b0 + (pr == 1 ? kCtBBytes : 0u);
            for (int k = 0; k < nks; ++k)
              mma_bf16(tmem, smem_desc_sw128(ap + k * 32), smem_desc_sw128(bq + k * 32), idesc,
                       (c > 0 || pr > 0 || k > 0) ? 1u : 0u);
          }
          mma_commit(&mma_bar);
        }
        pending = true;
      }
      if (!ok) break;
      // M of determinant dd0 + dj: tensor memory -> shared memory (over the operand buffer)
      ok = wait_mma();
      if (__syncthreads_or(!ok)) { ok = false; break; }
      fence_after_sync();
      const int rows = 3 * m + 1, N = (m + 15) / 16 * 16;
      const int r = 32 * warp + lane;   // warps 0-3: tensor-memory lane quarters 0-3
      if (warp < 4 && 32 * warp < rows) {
        for (int c0 = 0; c0 < N; c0 += 16) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
          if (r < rows)
#pragma unroll
            for (int u = 0; u < 16; ++u)
              if (c0 + u < m) Ms[r * kCtMsStride + c0 + u] = v[u];
        }
      }
      fence_before_sync();
      __syncthreads();
      float vv[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      if (tid < m) {
        vv[0] = Ms[(3 * tid) * kCtMsStride + tid];
        vv[1] = Ms[(3 * tid + 1) * kCtMsStride + tid];
        vv[2] = Ms[(3 * tid + 2) * kCtMsStride + tid];
      }
      for (int e2 = tid; e2 < m * m; e2 += kCtThreads) {
        const int k = e2 / m, kp = e2 - k * m;
#pragma unroll
        for (int xx = 0; xx < 3; ++xx)
          vv[3] = fmaf(Ms[(3 * k + xx) * kCtMsStride + kp], Ms[(3 * kp + xx) * kCtMsStride + k], vv[3]);
      }
      if (tid == 0) vv[4] = Ms[(3 * m) * kCtMsStride];
#pragma unroll
      for (int u = 0; u < 5; ++u)
        for (int o = 16; o > 0; o >>= 1) vv[u] += __shfl_xor_sync(0xffffffffu, vv[u], o);
      if (lane == 0)
#pragma unroll
        for (int u = 0; u < 5; ++u) red[warp][u] = vv[u];
      __syncthreads();   // M is consumed: the next chunk may overwrite the buffer
      if (tid == 0) {
        float sum[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        for (int y = 0; y < kCtThreads / 32; ++y)
#pragma unroll
          for (int u = 0; u < 5; ++u) sum[u] += red[y][u];
        const int64_t o = ((int64_t)w * a.D + a.dd0 + dj) * n + np;
        a.gdet[o * 3] = sum[0];
        a.gdet[o * 3 + 1] = sum[1];
        a.gdet[o * 3 + 2] = sum[2];
        a.ldet[o] = sum[4] - sum[3];
      }
    }
  }
  if (!ok) {
    if (tid == 0) atomicExch(a.err, 17);
    // MMAs still in flight complete before the tensor memory is freed (one
    // more bounded wait)
    if (pending) mbar_wait(&mma_bar, phase);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0) tmem_dealloc(tmem, kCtTmemCols);
}

int contract_tc(cudaStream_t s, int Wc, int n, int n_up, int K, int dd0, int G, int D, const int32_t* idx,
                const int32_t* cnt, const int32_t* rev, const int64_t* blk_off, const float* O, int64_t ldo,
                const float* Fenv, const float* AT, float* gdet, float* ldet, DevStatus* st, const int* list,
                int nitems, int* err) {
  if (nitems <= 0) return FIRE_OK;
  if (n % 4 || ldo % 4 || G < 1 || G > kCtMaxG || dd0 < 0 || dd0 + G > D) return FIRE_ERR_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(O) | reinterpret_cast<uintptr_t>(Fenv) | reinterpret_cast<uintptr_t>(AT)) & 15)
    return FIRE_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(contract_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCtSmemBytes) !=
      cudaSuccess) {
    cudaGetLastError();
    return FIRE_ERR_CUDA;
  }
  static int n_sm = 0;
  if (n_sm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (n_sm <= 0) n_sm = 1;
  }
  const CtArgs a{Wc, n, n_up, K, dd0, G, D, idx, cnt, rev, blk_off, O, ldo, Fenv, AT, gdet, ldet, st, list, nitems, err};
  const int64_t want = (int64_t)n_sm * kCtPerSm;
  const int grid = nitems < want ? nitems : (int)want;
  contract_tc_kernel<<<grid, kCtThreads, kCtSmemBytes, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? FIRE_OK : FIRE_ERR_CUDA;
}

}  // namespace tc
}  // namespace fire

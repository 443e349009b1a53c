// Host side of the tensor-core matrix product: tensor maps, launch, weight
// packing to bf16 K-major form, and a self-test entry point.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "../../include/fire.h"
#include "tc_api.h"
#include "tc_gemm.cuh"

namespace fire {
namespace tc {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// bf16 matrix [rows][cols] with row stride ld (elements), box box_rows x 64.
static bool make_map(CUtensorMap* m, const void* base, uint64_t rows, uint64_t cols, uint64_t ld,
                     uint32_t box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((ld * 2) & 15)) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// fp32 output [rows][cols] with row stride ld (elements): 32 x 32 boxes,
// 128-byte swizzle (the layout of the epilogue's store buffers).  The row
// extent is left open (2^31 - 1 rows, or fewer so that it spans less than
// 2^40 bytes): only tiles wholly inside the row range are stored through it.
static bool make_map_c(CUtensorMap* m, const float* base, uint64_t cols, uint64_t ld) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((ld * 4) & 15) || cols < 1 || ld < cols) return false;
  uint64_t rows = ((uint64_t)1 << 40) / (ld * 4);
  if (rows > 0x7fffffffull) rows = 0x7fffffffull;
  cuuint64_t dims[2] = {cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {ld * 4};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int STAGES, int NC>
static int launch(cudaStream_t s, const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& mc,
                  const TcArgs& g, int64_t m_cap, int nt) {
  const size_t sm = tc_smem_bytes(STAGES, NC, g.BN);
  if (cudaFuncSetAttribute(tc_gemm_kernel<STAGES, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
      cudaSuccess) {
    cudaGetLastError();   // the caller's next CUDA call must not see this error
    return FIRE_ERR_CUDA;
  }
  static int n_sm = 0;
  if (n_sm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (n_sm <= 0) n_sm = 1;
  }
  const int64_t tiles = ((m_cap + BM - 1) / BM) * nt;
  const int grid = (int)(tiles < n_sm ? tiles : n_sm);
  tc_gemm_kernel<STAGES, NC><<<grid, 192, sm, s>>>(ma, mb, mc, g);
  return cudaGetLastError() == cudaSuccess ? FIRE_OK : FIRE_ERR_CUDA;
}

// Output tile width: among the multiples of 16 (at least 64, or N rounded up
// to 16 when smaller) whose pipeline stages fit in shared memory, the one that
// computes the fewest columns in total; ties prefer the wider tile.
static int choose_bn(int N, int nc, int stages) {
  const int lo = N < 64 ? (N + 15) / 16 * 16 : 64;
  int best = 0;
  int64_t best_cols = -1;
  for (int bn = lo; bn <= 256; bn += 16) {
    if (tc_smem_bytes(stages, nc, bn) > 227 * 1024) break;
    const int64_t cols = (int64_t)((N + bn - 1) / bn) * bn;
    if (best_cols < 0 || cols < best_cols || (cols == best_cols && bn > best)) { best = bn; best_cols = cols; }
  }
  return best;
}

int gemm_bf16(cudaStream_t s, const void* A, int64_t lda, int64_t a_rows, const void* Bt, int N, int K,
              float* C, int64_t ldc, int64_t m_begin, int64_t m_end, const int64_t* m_range, int64_t m_cap,
              int* err, int nc) {
  return gemm_bf16_rows(s, A, lda, a_rows, Bt, N, 0, N, K, C, ldc, m_begin, m_end, m_range, m_cap, err, nc);
}

int gemm_bf16_rows(cudaStream_t s, const void* A, int64_t lda, int64_t a_rows, const void* Bt, int b_rows,
                   int b_row0, int N, int K, float* C, int64_t ldc, int64_t m_begin, int64_t m_end,
                   const int64_t* m_range, int64_t m_cap, int* err, int nc) {
  if (b_row0 < 0 || b_row0 + N > b_rows) return FIRE_ERR_UNSUPPORTED;
  if (N < 1 || K < BK || K % BK || m_cap <= 0 || nc < 1 || nc > 3) return FIRE_ERR_UNSUPPORTED;
  int stages = nc == 1 ? 4 : (nc == 2 ? 3 : 2);
  // wide two-component products (N >= 512): two stages of 256- or
  // 192-column tiles, whichever computes fewer columns (256 on a tie).
  // Measured on GB300 with the tensor-store epilogue at M = 400k, N = 720,
  // K = 256: 1271 TFLOP/s of split products with 256 columns, 1149 with 192,
  // 1210 with three stages of 128
  int bn_pref = 0;
  if (nc == 2 && N >= 512) {
    stages = 2;
    bn_pref = (N + 255) / 256 * 256 <= (N + 191) / 192 * 192 ? 256 : 192;
  }
  // FIRE_TC_STAGES / FIRE_TC_BN (diagnostic): pipeline depth and tile width
  if (const char* e = getenv("FIRE_TC_STAGES")) {
    const int v = atoi(e);
    if (v >= 2 && v <= 4) stages = v;
  }
  int BN = bn_pref && tc_smem_bytes(stages, nc, bn_pref) <= 227 * 1024 ? bn_pref : choose_bn(N, nc, stages);
  if (const char* e = getenv("FIRE_TC_BN")) {
    const int v = atoi(e);
    if (v >= 16 && v <= 256 && v % 16 == 0 && tc_smem_bytes(stages, nc, v) <= 227 * 1024) BN = v;
  }
  if (BN == 0) return FIRE_ERR_UNSUPPORTED;
  const int nt = (N + BN - 1) / BN;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, (uint64_t)a_rows * nc, (uint64_t)K, (uint64_t)lda, BM)) return FIRE_ERR_CUDA;
  if (!make_map(&mb, Bt, (uint64_t)b_rows * nc, (uint64_t)K, (uint64_t)K, (uint32_t)BN)) return FIRE_ERR_CUDA;
  // FIRE_TC_CSTORE=direct (diagnostic): every tile through the lanes' own stores
  CUtensorMap mc;
  memset(&mc, 0, sizeof(mc));
  const char* cs = getenv("FIRE_TC_CSTORE");
  const bool direct = cs && strcmp(cs, "direct") == 0;
  const int c_tma = (!direct && make_map_c(&mc, C, (uint64_t)N, (uint64_t)ldc)) ? 1 : 0;
  TcArgs g{C, ldc, m_begin, m_end, m_range, N, K, BN, a_rows, b_rows, b_row0, err, c_tma};
  if (nc == 1) return stages == 2 ? launch<2, 1>(s, ma, mb, mc, g, m_cap, nt)
                                   : (stages == 3 ? launch<3, 1>(s, ma, mb, mc, g, m_cap, nt)
                                                  : launch<4, 1>(s, ma, mb, mc, g, m_cap, nt));
  if (nc == 2) return stages == 2 ? launch<2, 2>(s, ma, mb, mc, g, m_cap, nt)
                                   : (stages == 3 ? launch<3, 2>(s, ma, mb, mc, g, m_cap, nt)
                                                  : launch<4, 2>(s, ma, mb, mc, g, m_cap, nt));
  return stages == 2 ? launch<2, 3>(s, ma, mb, mc, g, m_cap, nt)
                     : (stages == 3 ? launch<3, 3>(s, ma, mb, mc, g, m_cap, nt) : launch<4, 3>(s, ma, mb, mc, g, m_cap, nt));
}

// dst[c][n][k] = component c of src[k * lds + n] for a [K][N] source
// (trans = 1), or of src[n * lds + k] for an [N][K] source (trans = 0);
// components are comp_stride elements apart, rows ldd >= K elements apart,
// and the row padding k in [K, ldd) is zero.
__global__ void pack_bf16_kernel(const float* __restrict__ src, int64_t lds, int K, int N, int trans,
                                 __nv_bfloat16* __restrict__ dst, int nc, int64_t comp_stride, int ldd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)N * ldd) return;
  const int nn = (int)(e / ldd), kk = (int)(e % ldd);
  float v = kk >= K ? 0.f : (trans ? src[(int64_t)kk * lds + nn] : src[(int64_t)nn * lds + kk]);
  for (int c = 0; c < nc; ++c) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    dst[c * comp_stride + e] = h;
    v -= __bfloat162float(h);
  }
}

void pack_bf16(cudaStream_t s, const float* src, int64_t lds, int K, int N, int trans, void* dst, int nc,
               int64_t comp_stride, int ldd) {
  if (ldd < K) ldd = K;
  const int64_t tot = (int64_t)N * ldd;
  pack_bf16_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, lds, K, N, trans,
                                                                 reinterpret_cast<__nv_bfloat16*>(dst), nc,
                                                                 comp_stride, ldd);
}

}  // namespace tc
}  // namespace fire

extern "C" int fire_selftest_tc_gemm(int64_t M, int32_t N, int32_t K, int32_t nc, const void* A, const void* Bt,
                                     float* C, int32_t* err, void* stream) {
  if (M < 1 || N < 1 || K < 64 || K % 64 || nc < 1 || nc > 3 || !A || !Bt || !C || !err)
    return FIRE_ERR_INVALID_ARG;
  return fire::tc::gemm_bf16((cudaStream_t)stream, A, K, M, Bt, N, K, C, N, 0, M, nullptr, M, err, nc);
}

// SIMT matrix product C = A * op(B) over row ranges of the forward-Laplacian
// tensors, for the float32 and float64 forms.
//
// A is row-major [M][K] (lda), B row-major [K][N] (ldb) or, with TRANS_B,
// [N][K]; C row-major [M][N] (ldc).  The row range may live on the device
// (m_range = {begin, end}), so a launch can be enqueued before the ragged row
// counts are known; tiles past the end exit at once.  grid.z batches
// independent products with element strides sA, sB, sC.
#pragma once

#include "common.cuh"

namespace fire {

template <typename T>
struct GemmArgs {
  const T* A;
  const T* B;
  T* C;
  int64_t lda, ldb, ldc;
  int64_t sA, sB, sC;
  int64_t m_begin, m_end;        // used when m_range == nullptr
  const int64_t* m_range;        // device {begin, end} or nullptr
  int N, K;
  int accumulate;
};

template <typename T, int BM, int BN, int BK, int TM, int TN, bool TB>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
gemm_kernel(GemmArgs<T> g) {
  constexpr int NT = (BM / TM) * (BN / TN);
  __shared__ T As[2][BK][BM + 4];
  __shared__ T Bs[2][BK][BN + 4];
  int64_t mb = g.m_begin, me = g.m_end;
  if (g.m_range) { mb = g.m_range[0]; me = g.m_range[1]; }
  const int64_t m0 = mb + (int64_t)blockIdx.x * BM;
  if (m0 >= me) return;
  const int n0 = blockIdx.y * BN;
  const T* A = g.A + g.sA * blockIdx.z;
  const T* B = g.B + g.sB * blockIdx.z;
  T* C = g.C + g.sC * blockIdx.z;
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  constexpr int A_PER = BM * BK / NT, B_PER = BK * BN / NT;
  T ra[A_PER], rb[B_PER];
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < A_PER; ++q) {
      int e = tid + q * NT;
      int row = e / BK, col = e % BK;
      int64_t gm = m0 + row;
      int gk = k0 + col;
      ra[q] = (gm < me && gk < g.K) ? A[gm * g.lda + gk] : T(0);
    }
#pragma unroll
    for (int q = 0; q < B_PER; ++q) {
      int e = tid + q * NT;
      int gk, gn;
      if (TB) { gn = n0 + e / BK; gk = k0 + e % BK; }
      else { gk = k0 + e / BN; gn = n0 + e % BN; }
      T v = T(0);
      if (gk < g.K && gn < g.N) v = TB ? B[(int64_t)gn * g.ldb + gk] : B[(int64_t)gk * g.ldb + gn];
      rb[q] = v;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < A_PER; ++q) {
      int e = tid + q * NT;
      As[buf][e % BK][e / BK] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < B_PER; ++q) {
      int e = tid + q * NT;
      if (TB) Bs[buf][e % BK][e / BK] = rb[q];
      else Bs[buf][e / BN][e % BN] = rb[q];
    }
  };

  load(0);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < g.K; k0 += BK) {
    const bool more = (k0 + BK) < g.K;
    if (more) load(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (more) {
      store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int64_t gm = m0 + ty * TM + i;
    if (gm >= me) break;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int gn = n0 + tx * TN + j;
      if (gn < g.N) {
        T* p = C + gm * g.ldc + gn;
        *p = g.accumulate ? (*p + acc[i][j]) : acc[i][j];
      }
    }
  }
}

// Host launcher.  m_cap bounds end - begin (grid sizing).
template <typename T>
inline void gemm(cudaStream_t s, const T* A, int64_t lda, const T* B, int64_t ldb, bool transB,
                 T* C, int64_t ldc, int64_t m_begin, int64_t m_end, const int64_t* m_range,
                 int64_t m_cap, int N, int K, int batch = 1, int64_t sA = 0, int64_t sB = 0,
                 int64_t sC = 0, bool accumulate = false) {
  if (m_cap <= 0 || N <= 0 || K <= 0 || batch <= 0) return;
  GemmArgs<T> g{A, B, C, lda, ldb, ldc, sA, sB, sC, m_begin, m_end, m_range, N, K, accumulate ? 1 : 0};
  if constexpr (sizeof(T) == 4) {
    constexpr int BM = 128, BN = 128, BK = 8;
    dim3 grid((unsigned)((m_cap + BM - 1) / BM), (unsigned)((N + BN - 1) / BN), batch);
    if (transB) gemm_kernel<T, BM, BN, BK, 8, 8, true><<<grid, 256, 0, s>>>(g);
    else gemm_kernel<T, BM, BN, BK, 8, 8, false><<<grid, 256, 0, s>>>(g);
  } else {
    constexpr int BM = 64, BN = 64, BK = 8;
    dim3 grid((unsigned)((m_cap + BM - 1) / BM), (unsigned)((N + BN - 1) / BN), batch);
    if (transB) gemm_kernel<T, BM, BN, BK, 4, 4, true><<<grid, 256, 0, s>>>(g);
    else gemm_kernel<T, BM, BN, BK, 4, 4, false><<<grid, 256, 0, s>>>(g);
  }
}

}  // namespace fire

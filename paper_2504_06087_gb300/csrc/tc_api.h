// Host API of the tensor-core matrix product (tc_gemm.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fire {
struct DevStatus;
namespace tc {

// C[m][0..N) = A[m][0..K) * Bt[0..N)[0..K)^T for rows m in [begin, end)
// (device range m_range or host m_begin/m_end); A bf16 with row stride lda
// and a_rows rows allocated; Bt bf16 [N][K]; C fp32 with row stride ldc.
// K must be a multiple of 64.  Timeouts of bounded waits set *err.
// nc = 1, 2, 3: A and Bt hold nc bf16 components each (split-bf16 product),
// the components of A a_rows rows apart and those of Bt N rows apart.
int gemm_bf16(cudaStream_t s, const void* A, int64_t lda, int64_t a_rows, const void* Bt, int N, int K,
              float* C, int64_t ldc, int64_t m_begin, int64_t m_end, const int64_t* m_range, int64_t m_cap,
              int* err, int nc);

// The same product with Bt rows [b_row0, b_row0 + N) of a weight block whose
// components hold b_rows rows each (a slice of a larger packed matrix).
int gemm_bf16_rows(cudaStream_t s, const void* A, int64_t lda, int64_t a_rows, const void* Bt, int b_rows,
                   int b_row0, int N, int K, float* C, int64_t ldc, int64_t m_begin, int64_t m_end,
                   const int64_t* m_range, int64_t m_cap, int* err, int nc);

// dst = nc-component bf16 K-major copy of a weight matrix (pack_bf16_kernel),
// rows ldd >= K elements apart with zero padding (ldd = 0: K).
void pack_bf16(cudaStream_t s, const float* src, int64_t lds, int K, int N, int trans, void* dst, int nc,
               int64_t comp_stride, int ldd = 0);

// Restricted log-det contraction of determinants dd0 .. dd0 + G - 1 (G <= 4)
// on the tensor cores (contract_tc.cu) for the tangent electrons
// list[0 .. nitems) of a chunk (each e = w n + n', neighbourhoods of at most
// 42 members): gdet[w][dd][n'][3] and ldet[w][dd][n'] as contract3_kernel
// writes them.  O holds the orbital rows of the G determinants (determinant
// dd0 + j at column j n, row stride ldo), Fenv the envelope rows, AT the
// transposed inverses.  Operands in two bf16 components; n and ldo multiples
// of 4.  Timeouts of bounded waits set *err.
int contract_tc(cudaStream_t s, int Wc, int n, int n_up, int K, int dd0, int G, int D, const int32_t* idx,
                const int32_t* cnt, const int32_t* rev, const int64_t* blk_off, const float* O, int64_t ldo,
                const float* Fenv, const float* AT, float* gdet, float* ldet, DevStatus* st, const int* list,
                int nitems, int* err);
constexpr int kContractTcMaxMembers = 42;

}  // namespace tc
}  // namespace fire

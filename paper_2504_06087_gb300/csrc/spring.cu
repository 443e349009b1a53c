// SPRING parameter update (Methods, "Variational Monte Carlo", eq. spring):
//
//   Obar_i = O_i - mean_j O_j,   eps_i = E_L,i - mean_j E_L,j,
//   delta  = Obar^T (Obar Obar^T + lambda I)^-1 (eps - eta Obar delta_prev) + eta delta_prev,
//
// with the N x P matrix O of per-walker rows d ln|Psi| / d theta (the output
// of fire_grad_logpsi).  The N x N Gram matrix is the only dense contraction
// (2 N^2 P flops): it runs on the tensor cores as a split-bf16 product (three
// bf16 components per operand, six component products, FP32 accumulation in
// tensor memory) over chunks of the parameter axis, each chunk's rows
// converted once and its partial Gram matrix summed in float64.  The product
// takes the uncentred rows (G = O O^T) and the centring is applied exactly in
// float64 to the N x N matrix, Obar Obar^T = P G P with P = I - 1 1^T / N:
// centring the rows first would leave every row carrying the mean of the
// largest ones, whose float32 rounding then swamps the small eigenvalues, and
// the exact projection keeps 1 an exact null vector.  The damped N x N
// system is solved by a float64 blocked Cholesky factorisation of
// P G P + lambda I + mu 1 1^T / N (mu = the mean of diag P G P): the right-hand
// side is orthogonal to 1, so the added term changes no solution but keeps
// the null direction away from zero;
// the column means, the projection Obar delta_prev and the final
// Obar^T x are single streaming passes over O (HBM-bound).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fire.h"
#include "tc_api.h"

namespace fire {
namespace spring {

// Parameters per Gram chunk (multiple of 64).  The tensor cores accumulate a
// chunk in float32 with an error that grows with the number of K steps
// (about 2^-22 of the running sum per 16-deep step, measured); chunks of 4096
// keep it near 6e-5 of sqrt(G_ii G_jj), and the chunks are summed in float64.
constexpr int kChunk = 1 << 12;
constexpr int kNC = 3;            // bf16 components per operand
constexpr int kB = 64;            // Cholesky block

inline size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  int64_t Np;       // N rounded up to the Cholesky block
  int64_t pc;       // chunk width used (<= kChunk, multiple of 64)
  size_t mean, pack, cch, kacc, rowdot, b, a, scal, err, total;
};

inline Layout layout(int64_t N, int64_t P) {
  Layout L{};
  L.Np = (N + kB - 1) / kB * kB;
  int64_t pc = (P + 63) / 64 * 64;
  L.pc = pc < kChunk ? pc : kChunk;
  size_t o = 0;
  L.mean = o;   o = align_up(o + (size_t)P * 8);
  L.pack = o;   o = align_up(o + (size_t)kNC * N * L.pc * 2);
  L.cch = o;    o = align_up(o + (size_t)N * N * 4);
  L.kacc = o;   o = align_up(o + (size_t)L.Np * L.Np * 8);
  L.rowdot = o; o = align_up(o + (size_t)N * 8);
  L.b = o;      o = align_up(o + (size_t)L.Np * 8);
  L.a = o;      o = align_up(o + (size_t)N * 8);
  L.scal = o;   o = align_up(o + 32);
  L.err = o;    o = align_up(o + 16);
  L.total = o;
  return L;
}

// mean[p] = (1/N) sum_i O[i][p]; one thread per column, rows streamed (each
// warp reads 128 contiguous bytes of a row per step).
__global__ void colmean_kernel(int64_t N, int64_t P, const float* __restrict__ O, int64_t ldo,
                               double* __restrict__ mean) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int64_t i = 0;
  for (; i + 4 <= N; i += 4) {
    s0 += O[i * ldo + p];
    s1 += O[(i + 1) * ldo + p];
    s2 += O[(i + 2) * ldo + p];
    s3 += O[(i + 3) * ldo + p];
  }
  for (; i < N; ++i) s0 += O[i * ldo + p];
  mean[p] = ((s0 + s1) + (s2 + s3)) / (double)N;
}

// Rows of one chunk [p0, p0 + pc) as kNC bf16 components dst[c][i][q]
// (q < pc; zero beyond P), and rowdot[i] += sum_q (O_iq - mean_q) dprev[p0+q]
// (the projection Obar delta_prev).  Block (x, y): row y, 1024 columns.
__global__ void pack_kernel(int64_t N, int64_t P, const float* __restrict__ O, int64_t ldo,
                            const double* __restrict__ mean, int64_t p0, int pc, __nv_bfloat16* __restrict__ dst,
                            const float* __restrict__ dprev, double* __restrict__ rowdot) {
  __shared__ double red[8];
  const int64_t i = blockIdx.y;
  double acc = 0.0;
  for (int u = 0; u < 4; ++u) {
    const int q = blockIdx.x * 1024 + u * 256 + threadIdx.x;
    if (q >= pc) break;
    const int64_t p = p0 + q;
    float v = 0.f;
    if (p < P) {
      v = O[i * ldo + p];
      if (dprev) acc += ((double)v - mean[p]) * (double)dprev[p];
    }
    for (int c = 0; c < kNC; ++c) {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      dst[((int64_t)c * N + i) * pc + q] = h;
      v -= __bfloat162float(h);
    }
  }
  if (!dprev) return;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    atomicAdd(&rowdot[i], s);
  }
}

// K[i][j] (+)= C[i][j] in float64 over the N x N block of the padded Np x Np
// matrix; the padding gets the identity when first == 1.
__global__ void accum_kernel(int64_t N, int64_t Np, const float* __restrict__ C, double* __restrict__ K, int first) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Np * Np) return;
  const int64_t i = e / Np, j = e % Np;
  if (i < N && j < N) {
    const double c = (double)C[i * N + j];
    K[e] = first ? c : K[e] + c;
  } else if (first) {
    K[e] = (i == j) ? 1.0 : 0.0;
  }
}

// a[i] = (1/N) sum_j G[i][j] (row means of the uncentred Gram matrix), one
// warp per row.
__global__ void rowmean_kernel(int64_t N, int64_t Np, const double* __restrict__ K, double* __restrict__ a) {
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= N) return;
  double s = 0.0;
  for (int64_t j = lane; j < N; j += 32) s += K[i * Np + j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) a[i] = s / (double)N;
}

// K <- P G P = G - a 1^T - 1 a^T + abar 1 1^T (abar = mean of a), in place
// over the N x N block; one CTA of 1024 threads forms abar first.
__global__ void center_kernel(int64_t N, int64_t Np, double* __restrict__ K, const double* __restrict__ a,
                              double* __restrict__ abar_out) {
  __shared__ double red[32];
  __shared__ double s_abar;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) s += a[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    s_abar = t / (double)N;
    if (blockIdx.x == 0 && abar_out) *abar_out = s_abar;
  }
  __syncthreads();
  const double abar = s_abar;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N * N; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N, j = e % N;
    K[i * Np + j] = ((K[i * Np + j] - a[i]) - a[j]) + abar;
  }
}

// b[i] = (E_i - mean E) - eta rowdot[i] (zero in the padding); *mu = the
// mean of diag K (before the damping); then K[i][i] += lambda.
__global__ void rhs_kernel(int64_t N, int64_t Np, const double* __restrict__ e_loc, const double* __restrict__ rowdot,
                           double eta, double lambda, double* __restrict__ b, double* __restrict__ K,
                           double* __restrict__ mu) {
  __shared__ double red[2][32];
  __shared__ double s_mean;
  double s = 0.0, dsum = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
    s += e_loc[i];
    dsum += K[i * Np + i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s;
    red[1][threadIdx.x >> 5] = dsum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0, d = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t += red[0][w]; d += red[1][w]; }
    s_mean = t / (double)N;
    *mu = d / (double)N;
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < Np; i += blockDim.x) {
    b[i] = i < N ? (e_loc[i] - s_mean) - eta * (rowdot ? rowdot[i] : 0.0) : 0.0;
    if (i < N) K[i * Np + i] += lambda;
  }
}

// K += (mu / N) 1 1^T over the N x N block: lifts the null direction 1 of the
// centred matrix to mu + lambda without changing the solution for a
// right-hand side orthogonal to 1.
__global__ void lift_kernel(int64_t N, int64_t Np, double* __restrict__ K, const double* __restrict__ mu) {
  const double add = *mu / (double)N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N * N; e += (int64_t)gridDim.x * blockDim.x)
    K[(e / N) * Np + e % N] += add;
}

// --- float64 blocked Cholesky (lower, in place, row-major Np x Np) ---------

// Diagonal block k: A_kk = L_kk L_kk^T in shared memory; a non-positive pivot
// sets *err (the matrix is not positive definite) and leaves the block.
__global__ void __launch_bounds__(256) chol_diag_kernel(int64_t Np, double* __restrict__ K, int k,
                                                        int* __restrict__ err) {
  __shared__ double a[kB][kB + 1];
  __shared__ int bad;
  double* A = K + (int64_t)k * kB * Np + (int64_t)k * kB;
  for (int e = threadIdx.x; e < kB * kB; e += blockDim.x) a[e / kB][e % kB] = A[(int64_t)(e / kB) * Np + e % kB];
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < kB; ++j) {
    if (threadIdx.x == 0) {
      const double d = a[j][j];
      if (!(d > 0.0)) bad = 1;
      a[j][j] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    const double piv = a[j][j];
    for (int r = j + 1 + threadIdx.x; r < kB; r += blockDim.x) a[r][j] /= piv;
    __syncthreads();
    for (int e = threadIdx.x; e < (kB - j - 1) * (kB - j - 1); e += blockDim.x) {
      const int r = j + 1 + e / (kB - j - 1), c = j + 1 + e % (kB - j - 1);
      if (c <= r) a[r][c] -= a[r][j] * a[c][j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < kB * kB; e += blockDim.x) {
    const int r = e / kB, c = e % kB;
    A[(int64_t)r * Np + c] = c <= r ? a[r][c] : 0.0;
  }
  if (threadIdx.x == 0 && bad) atomicExch(err, 1);
}

// Panel below block k: L_ik = A_ik L_kk^-T (one 64-row block per CTA, one
// thread per row, forward substitution along the row).
__global__ void __launch_bounds__(kB) chol_panel_kernel(int64_t Np, double* __restrict__ K, int k) {
  __shared__ double l[kB][kB + 1];
  const int ib = k + 1 + blockIdx.x;
  const double* Lkk = K + (int64_t)k * kB * Np + (int64_t)k * kB;
  for (int e = threadIdx.x; e < kB * kB; e += blockDim.x) l[e / kB][e % kB] = Lkk[(int64_t)(e / kB) * Np + e % kB];
  __syncthreads();
  double* row = K + ((int64_t)ib * kB + threadIdx.x) * Np + (int64_t)k * kB;
  double x[kB];
#pragma unroll
  for (int j = 0; j < kB; ++j) x[j] = row[j];
#pragma unroll
  for (int j = 0; j < kB; ++j) {
    double s = x[j];
#pragma unroll
    for (int q = 0; q < j; ++q) s -= x[q] * l[j][q];
    x[j] = s / l[j][j];
  }
#pragma unroll
  for (int j = 0; j < kB; ++j) row[j] = x[j];
}

// Trailing update A_ij -= L_ik L_jk^T for block rows i >= j > k: one 64 x 64
// tile per CTA (CTAs above the diagonal exit), 256 threads of 4 x 4 outputs.
__global__ void __launch_bounds__(256) chol_update_kernel(int64_t Np, double* __restrict__ K, int k) {
  const int ti = k + 1 + blockIdx.y, tj = k + 1 + blockIdx.x;
  if (tj > ti) return;
  extern __shared__ double cu_sm[];
  double* li = cu_sm;                 // [kB][kB + 1]
  double* lj = cu_sm + kB * (kB + 1);
  const double* Li = K + (int64_t)ti * kB * Np + (int64_t)k * kB;
  const double* Lj = K + (int64_t)tj * kB * Np + (int64_t)k * kB;
  for (int e = threadIdx.x; e < kB * kB; e += blockDim.x) {
    li[(e / kB) * (kB + 1) + e % kB] = Li[(int64_t)(e / kB) * Np + e % kB];
    lj[(e / kB) * (kB + 1) + e % kB] = Lj[(int64_t)(e / kB) * Np + e % kB];
  }
  __syncthreads();
  const int r0 = (threadIdx.x / 16) * 4, c0 = (threadIdx.x % 16) * 4;
  double acc[4][4] = {};
  for (int q = 0; q < kB; ++q) {
    double a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a[u] = li[(r0 + u) * (kB + 1) + q];
      b[u] = lj[(c0 + u) * (kB + 1) + q];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
  }
  double* A = K + (int64_t)ti * kB * Np + (int64_t)tj * kB;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) A[(int64_t)(r0 + u) * Np + c0 + v] -= acc[u][v];
}

// L y = b then L^T x = y in place on b, one CTA of 1024 threads: per block
// of 64 unknowns, warp 0 solves the small triangle and every thread updates
// the remaining right-hand side entries.
__global__ void __launch_bounds__(1024) chol_solve_kernel(int64_t Np, const double* __restrict__ L,
                                                          double* __restrict__ b) {
  __shared__ double y[kB];
  const int nb = (int)(Np / kB);
  for (int k = 0; k < nb; ++k) {        // forward
    const int64_t o = (int64_t)k * kB;
    if (threadIdx.x < 32) {
      for (int j = 0; j < kB; ++j) {
        double s = 0.0;
        for (int q = threadIdx.x; q < j; q += 32) s += L[(o + j) * Np + o + q] * y[q];
        for (int w = 16; w > 0; w >>= 1) s += __shfl_xor_sync(0xffffffffu, s, w);
        if (threadIdx.x == 0) y[j] = (b[o + j] - s) / L[(o + j) * Np + o + j];
        __syncwarp();
      }
    }
    __syncthreads();
    for (int64_t i = o + kB + threadIdx.x; i < Np; i += blockDim.x) {
      double s = 0.0;
#pragma unroll 8
      for (int q = 0; q < kB; ++q) s += L[i * Np + o + q] * y[q];
      b[i] -= s;
    }
    if (threadIdx.x < kB) b[o + threadIdx.x] = y[threadIdx.x];
    __syncthreads();
  }
  for (int k = nb - 1; k >= 0; --k) {   // backward with L^T
    const int64_t o = (int64_t)k * kB;
    if (threadIdx.x < 32) {
      for (int j = kB - 1; j >= 0; --j) {
        double s = 0.0;
        for (int q = j + 1 + threadIdx.x; q < kB; q += 32) s += L[(o + q) * Np + o + j] * y[q];
        for (int w = 16; w > 0; w >>= 1) s += __shfl_xor_sync(0xffffffffu, s, w);
        if (threadIdx.x == 0) y[j] = (b[o + j] - s) / L[(o + j) * Np + o + j];
        __syncwarp();
      }
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < o; i += blockDim.x) {
      double s = 0.0;
#pragma unroll 8
      for (int q = 0; q < kB; ++q) s += L[(o + q) * Np + i] * y[q];
      b[i] -= s;
    }
    if (threadIdx.x < kB) b[o + threadIdx.x] = y[threadIdx.x];
    __syncthreads();
  }
}

// delta[p] = sum_i (O[i][p] - mean[p]) x[i] + eta dprev[p]; one thread per
// column, rows streamed; x staged in shared memory 1024 entries at a time.
__global__ void update_kernel(int64_t N, int64_t P, const float* __restrict__ O, int64_t ldo,
                              const double* __restrict__ mean, const double* __restrict__ x,
                              const float* __restrict__ dprev, double eta, float* __restrict__ delta) {
  __shared__ double xs[1024];
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0, xsum = 0.0;
  for (int64_t i0 = 0; i0 < N; i0 += 1024) {
    const int64_t cnt = N - i0 < 1024 ? N - i0 : 1024;
    __syncthreads();
    for (int64_t q = threadIdx.x; q < cnt; q += blockDim.x) xs[q] = x[i0 + q];
    __syncthreads();
    if (p < P)
      for (int64_t q = 0; q < cnt; ++q) acc += (double)O[(i0 + q) * ldo + p] * xs[q];
    for (int64_t q = 0; q < cnt; ++q) xsum += xs[q];
  }
  if (p >= P) return;
  delta[p] = (float)(acc - mean[p] * xsum + eta * (dprev ? (double)dprev[p] : 0.0));
}

}  // namespace spring
}  // namespace fire

using namespace fire::spring;

extern "C" size_t fire_spring_workspace_size(int64_t n_walkers, int64_t n_params) {
  if (n_walkers < 2 || n_params < 1 || n_walkers > (1 << 16)) return 0;
  return layout(n_walkers, n_params).total;
}

extern "C" int fire_spring_step(int64_t n_walkers, int64_t n_params, const float* O, int64_t ldo,
                                const double* e_loc, const float* delta_prev, double eta, double lambda,
                                float* delta, double* gram, double* x_out, void* ws, size_t ws_bytes,
                                void* stream) {
  const int64_t N = n_walkers, P = n_params;
  if (N < 2 || P < 1 || N > (1 << 16) || ldo < P || !O || !e_loc || !delta) return FIRE_ERR_INVALID_ARG;
  if (!(lambda > 0.0) || !(lambda < 1e300) || !(eta >= 0.0) || !(eta < 1e300)) return FIRE_ERR_INVALID_ARG;
  const Layout L = layout(N, P);
  if (!ws || ws_bytes < L.total) return FIRE_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* w = reinterpret_cast<unsigned char*>(ws);
  double* mean = reinterpret_cast<double*>(w + L.mean);
  __nv_bfloat16* pack = reinterpret_cast<__nv_bfloat16*>(w + L.pack);
  float* cch = reinterpret_cast<float*>(w + L.cch);
  double* K = reinterpret_cast<double*>(w + L.kacc);
  double* rowdot = reinterpret_cast<double*>(w + L.rowdot);
  double* b = reinterpret_cast<double*>(w + L.b);
  int* err = reinterpret_cast<int*>(w + L.err);
  const int64_t Np = L.Np;
  if (cudaMemsetAsync(err, 0, 16, s) != cudaSuccess) return FIRE_ERR_CUDA;
  if (delta_prev && cudaMemsetAsync(rowdot, 0, (size_t)N * 8, s) != cudaSuccess) return FIRE_ERR_CUDA;
  colmean_kernel<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(N, P, O, ldo, mean);
  // Gram matrix over chunks of the parameter axis
  int first = 1;
  for (int64_t p0 = 0; p0 < P; p0 += L.pc) {
    const int64_t left = (P - p0 + 63) / 64 * 64;
    const int pc = (int)(left < L.pc ? left : L.pc);
    dim3 g((unsigned)((pc + 1023) / 1024), (unsigned)N);
    pack_kernel<<<g, 256, 0, s>>>(N, P, O, ldo, mean, p0, pc, pack, delta_prev, rowdot);
    const int rc = fire::tc::gemm_bf16(s, pack, pc, N, pack, (int)N, pc, cch, N, 0, N, nullptr, N, err + 1, kNC);
    if (rc != FIRE_OK) return rc;
    accum_kernel<<<(unsigned)((Np * Np + 255) / 256), 256, 0, s>>>(N, Np, cch, K, first);
    first = 0;
  }
  // exact centring in float64: Obar Obar^T = P G P
  double* a = reinterpret_cast<double*>(w + L.a);
  double* scal = reinterpret_cast<double*>(w + L.scal);
  rowmean_kernel<<<(unsigned)((N + 7) / 8), 256, 0, s>>>(N, Np, K, a);
  center_kernel<<<608, 1024, 0, s>>>(N, Np, K, a, scal);
  if (gram) cudaMemcpy2DAsync(gram, (size_t)N * 8, K, (size_t)Np * 8, (size_t)N * 8, (size_t)N,
                              cudaMemcpyDeviceToDevice, s);
  rhs_kernel<<<1, 1024, 0, s>>>(N, Np, e_loc, delta_prev ? rowdot : nullptr, eta, lambda, b, K, scal + 1);
  lift_kernel<<<608, 256, 0, s>>>(N, Np, K, scal + 1);
  // float64 Cholesky of K + lambda I, then the two triangular solves
  const int nb = (int)(Np / kB);
  const size_t usm = 2 * (size_t)kB * (kB + 1) * 8;
  if (cudaFuncSetAttribute(chol_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)usm) != cudaSuccess)
    return FIRE_ERR_CUDA;
  for (int k = 0; k < nb; ++k) {
    chol_diag_kernel<<<1, 256, 0, s>>>(Np, K, k, err);
    const int rest = nb - k - 1;
    if (rest > 0) {
      chol_panel_kernel<<<rest, kB, 0, s>>>(Np, K, k);
      chol_update_kernel<<<dim3(rest, rest), 256, usm, s>>>(Np, K, k);
    }
  }
  chol_solve_kernel<<<1, 1024, 0, s>>>(Np, K, b);
  if (x_out) cudaMemcpyAsync(x_out, b, (size_t)N * 8, cudaMemcpyDeviceToDevice, s);
  update_kernel<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(N, P, O, ldo, mean, b, delta_prev, eta, delta);
  int herr[2] = {0, 0};
  if (cudaMemcpyAsync(herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s) != cudaSuccess) return FIRE_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return FIRE_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return FIRE_ERR_CUDA;
  if (herr[1]) return FIRE_ERR_TIMEOUT;
  if (herr[0]) return FIRE_ERR_NONFINITE;
  return FIRE_OK;
}

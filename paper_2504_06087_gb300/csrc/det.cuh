// Orbitals, envelopes, determinants and the log-determinant derivatives.
//
// Phi_dil = (h_i W_dl) phi_dl(r_i), phi_dl(r) = sum_m sum_e pi_dlme
// exp(-sigma_me |r - R_m|) (Methods, "Wave function ansatz").  With A = Phi^-1
// (Methods, "Efficient Laplacian"):
//   d log det / d r_nx  = sum_{i in Nbar_n} M_ii,nx
//   Lap log det         = sum_il LapPhi_il A_li - sum_nx sum_{i,k in Nbar_n} M_ik,nx M_ki,nx
//   M_ik,nx             = sum_l (d Phi_il / d r_nx) A_lk,
// Nbar_n = N_n u {n}: the restriction of eq. logdet_lowrank.  The contraction
// is organised per tangent electron n, so every M entry it needs stays inside
// one CTA.
#pragma once

#include "common.cuh"

namespace fire {

// q_ime = exp(-sigma_me |r_i - R_m|) with gradient and Laplacian (rows:
// value, Laplacian, d/dx, d/dy, d/dz).  One CTA per electron.  With Qb the
// rows are also written as nc bf16 components (row stride ldb >= N*E, zero
// beyond N*E; components cs elements apart) for the tensor-core product.
template <typename T, typename W>
__global__ void env_feat_kernel(int Wc, int n, int n_up, int N, int E, const double* __restrict__ r,
                                const double* __restrict__ R, const W* sig, T* __restrict__ Q, int R5,
                                __nv_bfloat16* __restrict__ Qb = nullptr, int ldb = 0, int nc = 0,
                                int64_t cs = 0) {
  const int blk = blockIdx.x;
  const int w = blk / n, i = blk % n;
  const int NE = N * E;
  const double* ri = r + ((int64_t)w * n + i) * 3;
  const int64_t row = (int64_t)block_index(w, i, Wc, n, n_up) * R5;
  for (int q = threadIdx.x; q < NE; q += blockDim.x) {
    const int m = q / E;
    double dd[3] = {ri[0] - R[3 * m], ri[1] - R[3 * m + 1], ri[2] - R[3 * m + 2]};
    double rr = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
    T s = T(sig[q]);
    T rt = T(rr);
    T v = dexp<T>(-s * rt);
    T o[5];
    o[0] = v;
    Q[row * NE + q] = v;
    if (R5 > 1) {
      o[1] = (s * s - T(2) * s / rt) * v;
      Q[(row + 1) * NE + q] = o[1];
      for (int t = 0; t < 3; ++t) {
        o[2 + t] = -s * v * T(dd[t]) / rt;
        Q[(row + 2 + t) * NE + q] = o[2 + t];
      }
    }
    if (Qb)
      for (int k = 0; k < R5; ++k) store_split_bf16(Qb + (row + k) * ldb + q, cs, nc, (float)o[k]);
  }
  if (Qb)
    for (int q = NE + threadIdx.x; q < ldb; q += blockDim.x)
      for (int k = 0; k < R5; ++k) store_split_bf16(Qb + (row + k) * ldb + q, cs, nc, 0.f);
}

// The float64 product of two float32 values, which is exact, formed from the
// 24 x 24-bit integer product of their significands (no float64 operation:
// on GB300 a float64 multiply and the two widening conversions take the
// float64 pipe, which the LU of the same step saturates).  Zeros, subnormals,
// infinities and NaNs take the float64 multiply.
__device__ __forceinline__ double exact_product_f32(float a, float b) {
  const uint32_t ua = __float_as_uint(a), ub = __float_as_uint(b);
  const uint32_t ea = (ua >> 23) & 0xffu, eb = (ub >> 23) & 0xffu;
  if (ea == 0u || eb == 0u || ea == 0xffu || eb == 0xffu) return (double)a * (double)b;
  const uint64_t m = (uint64_t)((ua & 0x7fffffu) | 0x800000u) * (uint64_t)((ub & 0x7fffffu) | 0x800000u);
  // a b = m 2^(ea + eb - 300), m in [2^46, 2^48)
  const bool hi = (m >> 47) != 0;
  const int e = (int)(ea + eb) - 300 + (hi ? 47 : 46);
  uint64_t bits = (m << (hi ? 5 : 6)) & 0xfffffffffffffull;
  bits |= (uint64_t)(e + 1023) << 52;
  bits |= (uint64_t)((ua ^ ub) & 0x80000000u) << 32;
  return __longlong_as_double((long long)bits);
}
template <typename A, typename LT>
__device__ __forceinline__ LT phi_product(A x, A y) {
  return LT(x) * LT(y);
}
template <>
__device__ __forceinline__ double phi_product<float, double>(float x, float y) {
  return exact_product_f32(x, y);
}

// Phi[w][d][i][l] = O_v[b(i)][d*n + l] * Fenv[b(i)*R5][d*n + l].
// One CTA per (w, d).
template <typename T, typename LT>
__global__ void phi_assemble_kernel(int Wc, int n, int n_up, int D, const T* __restrict__ Ov,
                                    const T* __restrict__ Fenv, int R5, LT* __restrict__ Phi,
                                    float* __restrict__ Phif) {
  const int w = blockIdx.x / D, dd = blockIdx.x % D;
  const int64_t Dn = (int64_t)D * n;
  LT* P = Phi + (int64_t)blockIdx.x * n * n;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, l = e % n;
    const int64_t b = block_index(w, i, Wc, n, n_up);
    const T x = Ov[b * Dn + dd * n + l], y = Fenv[b * R5 * Dn + dd * n + l];
    const LT v = phi_product<T, LT>(x, y);
    P[e] = v;
    // float copy: for float inputs the float product is the rounding of the
    // exact product v, without a float64 conversion
    if (Phif) Phif[(int64_t)blockIdx.x * n * n + e] = sizeof(T) == 4 ? (float)(x * y) : (float)v;
  }
}

// |v| as an unsigned key that orders like |v| for every non-NaN value (the
// IEEE bit pattern without the sign bit), so the pivot search compares
// integers and keeps the float64 pipe for the elimination.
__device__ __forceinline__ unsigned long long mag_key(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned long long mag_key(float v) {
  return (unsigned long long)((unsigned)__float_as_int(v) & 0x7fffffffu);
}

// Blocked right-looking LU with partial pivoting, one CTA per matrix, the
// matrix in global memory (L2-resident), the current panel and U12 block in
// shared memory.  Writes the pivots, log|det| and sign (0 and -inf for an
// exactly zero pivot).  The float64 pipe is the bottleneck, so the pivot
// search compares magnitude keys (mag_key) and the multipliers of a column
// use one reciprocal of the pivot, formed by one thread.
template <typename LT, int NB>
__global__ void lu_kernel(int n, LT* __restrict__ M, int32_t* __restrict__ piv,
                          double* __restrict__ logabs, double* __restrict__ sgn,
                          const int* __restrict__ count = nullptr) {
  // a batch whose size is known on the device only: CTAs beyond it leave
  if (count && (int)blockIdx.x >= *count) return;
  extern __shared__ unsigned char lu_smem[];
  constexpr int PS = NB + 1;                   // panel row stride: rows fall in different banks
  LT* P = reinterpret_cast<LT*>(lu_smem);      // [n][NB + 1]
  LT* U = P + (int64_t)n * PS;                 // [NB][n]
  __shared__ unsigned long long red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_piv;
  __shared__ int s_zero;
  __shared__ LT s_rinv;
  LT* A = M + (int64_t)blockIdx.x * n * n;
  int32_t* pv = piv + (int64_t)blockIdx.x * n;
  const int tid = threadIdx.x, bd = blockDim.x;
  if (tid == 0) s_zero = 0;
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int nb = min(NB, n - k0);
    const int pr = n - k0;  // panel rows
    for (int e = tid; e < pr * nb; e += bd) {
      const int r = e / nb, c = e % nb;
      P[r * PS + c] = A[(int64_t)(k0 + r) * n + k0 + c];
    }
    __syncthreads();
    for (int kk = 0; kk < nb; ++kk) {
      // argmax |P[r][kk]| over r in [kk, pr), first index on ties
      unsigned long long best = 0;
      int bi = kk;
      for (int r = kk + tid; r < pr; r += bd) {
        const unsigned long long v = mag_key(P[r * PS + kk]);
        if (v > best) { best = v; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if ((tid & 31) == 0) { red_v[tid >> 5] = best; red_i[tid >> 5] = bi; }
      __syncthreads();
      if (tid == 0) {
        unsigned long long b = red_v[0];
        int ib = red_i[0];
        for (int q = 1; q < (bd + 31) / 32; ++q)
          if (red_v[q] > b || (red_v[q] == b && red_i[q] < ib)) { b = red_v[q]; ib = red_i[q]; }
        s_piv = ib;
        pv[k0 + kk] = k0 + ib;
        if (b == 0) s_zero = 1;
        s_rinv = b == 0 ? LT(0) : LT(1) / P[ib * PS + kk];
      }
      __syncthreads();
      const int p = s_piv;
      if (p != kk) {
        for (int c = tid; c < nb; c += bd) {
          LT t = P[kk * PS + c];
          P[kk * PS + c] = P[p * PS + c];
          P[p * PS + c] = t;
        }
      }
      __syncthreads();
      const LT pivot = P[kk * PS + kk], rinv = s_rinv;
      if (pivot != LT(0)) {
        for (int r = kk + 1 + tid; r < pr; r += bd) {
          LT l = P[r * PS + kk] * rinv;
          P[r * PS + kk] = l;
          for (int c = kk + 1; c < nb; ++c) P[r * PS + c] -= l * P[kk * PS + c];
        }
      }
      __syncthreads();
    }
    // panel back to global
    for (int e = tid; e < pr * nb; e += bd) {
      const int r = e / nb, c = e % nb;
      A[(int64_t)(k0 + r) * n + k0 + c] = P[r * PS + c];
    }
    // row swaps of this panel on the columns outside it
    for (int kk = 0; kk < nb; ++kk) {
      const int a = k0 + kk, b = pv[k0 + kk];
      if (a != b) {
        for (int c = tid; c < n; c += bd) {
          if (c >= k0 && c < k0 + nb) continue;
          LT t = A[(int64_t)a * n + c];
          A[(int64_t)a * n + c] = A[(int64_t)b * n + c];
          A[(int64_t)b * n + c] = t;
        }
      }
      __syncthreads();
    }
    const int c0 = k0 + nb;
    // U12 = L11^-1 A12 (unit lower L11 from the panel)
    for (int j = c0 + tid; j < n; j += bd) {
      LT u[NB];
#pragma unroll
      for (int kk = 0; kk < NB; ++kk) {
        if (kk < nb) {
          LT s = A[(int64_t)(k0 + kk) * n + j];
          for (int q = 0; q < kk; ++q) s -= P[kk * PS + q] * u[q];
          u[kk] = s;
          A[(int64_t)(k0 + kk) * n + j] = s;
          U[kk * n + j] = s;
        }
      }
    }
    __syncthreads();
    // A22 -= L21 U12
    const int rows2 = n - c0, cols2 = n - c0;
    for (int e = tid; e < rows2 * cols2; e += bd) {
      const int r = c0 + e / cols2, j = c0 + e % cols2;
      LT s = A[(int64_t)r * n + j];
      const LT* lrow = P + (int64_t)(r - k0) * PS;
      for (int kk = 0; kk < nb; ++kk) s -= lrow[kk] * U[kk * n + j];
      A[(int64_t)r * n + j] = s;
    }
    __syncthreads();
  }
  // log|det| and sign
  if (tid < 32) {
    double la = 0.0;
    int neg = 0;
    for (int k = tid; k < n; k += 32) {
      double u = (double)A[(int64_t)k * n + k];
      la += log(fabs(u));
      if (u < 0) neg ^= 1;
      if (pv[k] != k) neg ^= 1;
    }
    for (int o = 16; o > 0; o >>= 1) {
      la += __shfl_xor_sync(0xffffffffu, la, o);
      neg ^= __shfl_xor_sync(0xffffffffu, neg, o);
    }
    if (tid == 0) {
      if (s_zero) { logabs[blockIdx.x] = -INFINITY; sgn[blockIdx.x] = 0.0; }
      else { logabs[blockIdx.x] = la; sgn[blockIdx.x] = neg ? -1.0 : 1.0; }
    }
  }
}

// Dynamic shared memory of lu_kernel<LT, NB>: the panel [n][NB + 1] and U12 [NB][n].
inline size_t lu_smem_bytes(int n, size_t lsz, int nb = 16) { return (size_t)(2 * nb + 1) * n * lsz; }


// A = Phi^-1 by in-place Gauss-Jordan elimination with partial pivoting, in
// float32, register-tiled: thread (tr, tc) of a Gr x Gc grid (Gr = ceil(n/12),
// Gc = ceil(n/8)) keeps the 12 x 8 block of rows 12tr.., columns 8tc.. in
// registers.  Step k picks the unused row p with the largest |a_pk|,
// broadcasts row p and column k through shared memory and updates every
// block:
//   a_pj /= v (j != k), a_pk = 1/v;  a_ij -= a_ik a_pj / v, a_ik = -a_ik / v.
// Rows are never moved: with piv[s] the row used at step s and step[r] its
// inverse, the stored matrix S satisfies A^-1[r][piv[c]] = S[piv[r]][c].
// The result is written transposed (AT[k][l] = A^-1[l][k]).  n <= 192.
//
// The column k = 8 kt + kj is unrolled over kj, so every register of the
// pivot column is addressed statically; every element takes the same fused
// update a_ij -= f_i s_j (f_p = 0), and only the owners of column k and of
// row p rewrite their entries afterwards.  The broadcast buffers alternate
// between steps, so three barriers separate the steps.  With pivot rows from
// an LU of the same matrix, gj_inverse_pre_kernel needs one.
constexpr int kGjTR = 12, kGjTC = 8;
inline int gj_threads(int n) {
  const int t = ((n + kGjTR - 1) / kGjTR) * ((n + kGjTC - 1) / kGjTC);
  return ((t + 31) / 32) * 32;
}
template <typename IT, typename OT>
__global__ void __launch_bounds__(384, 1) gj_inverse_kernel(int n, const IT* __restrict__ Phi, OT* __restrict__ AT) {
  constexpr int TR = kGjTR, TC = kGjTC;
  extern __shared__ unsigned char gj_smem[];
  float* S = reinterpret_cast<float*>(gj_smem);          // [n][n] final matrix
  float* prow = S + (int64_t)n * n;                      // [2][256] pivot row
  float* pcol = prow + 512;                              // [2][256] pivot column
  int* piv = reinterpret_cast<int*>(pcol + 512);         // [n]
  int* stp = piv + 256;                                  // [n]
  int* used = stp + 256;                                 // [n]
  float* cv = reinterpret_cast<float*>(used + 256);      // [2][32] candidate |a|
  int* ci = reinterpret_cast<int*>(cv + 64);             // [2][32] candidate row
  const int Gr = (n + TR - 1) / TR, Gc = (n + TC - 1) / TC;
  const int tid = threadIdx.x;
  const int tr = tid / Gc, tc = tid % Gc;
  const bool live = tr < Gr;
  const IT* P = Phi + (int64_t)blockIdx.x * n * n;
  float a[TR][TC];
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int j = 0; j < TC; ++j) {
      const int r = TR * tr + i, c = TC * tc + j;
      a[i][j] = (live && r < n && c < n) ? (float)P[(int64_t)r * n + c] : 0.f;
    }
  for (int r = tid; r < 256; r += blockDim.x) used[r] = 0;
  __syncthreads();
  for (int kt = 0; kt < Gc; ++kt) {
#pragma unroll
    for (int kj = 0; kj < TC; ++kj) {
      const int k = TC * kt + kj;
      if (k < n) {
        const int bsel = k & 1;
        float* pr = prow + 256 * bsel;
        float* pc = pcol + 256 * bsel;
        float* cvb = cv + 32 * bsel;
        int* cib = ci + 32 * bsel;
        // candidates: the threads of column block kt, one per row block
        if (live && tc == kt) {
          float best = -1.f;
          int bi = n;
#pragma unroll
          for (int i = 0; i < TR; ++i) {
            const int r = TR * tr + i;
            const float v = fabsf(a[i][kj]);
            if (r < n && !used[r] && v > best) { best = v; bi = r; }
          }
          cvb[tr] = best;
          cib[tr] = bi;
        }
        __syncthreads();
        if (tid < 32) {
          float best = -1.f;
          int bi = n;
          for (int q = tid; q < Gr; q += 32)
            if (cvb[q] > best || (cvb[q] == best && cib[q] < bi)) { best = cvb[q]; bi = cib[q]; }
          for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
          }
          if (tid == 0) {
            if (bi >= n) bi = 0;   // singular: any row, the result is not finite
            piv[k] = bi;
            stp[bi] = k;
            used[bi] = 1;
          }
        }
        __syncthreads();
        const int p = piv[k];
        const int pt = p / TR, pi = p % TR;
        if (live && tr == pt)
#pragma unroll
          for (int i = 0; i < TR; ++i)
            if (i == pi)
#pragma unroll
              for (int j = 0; j < TC; ++j) pr[TC * tc + j] = a[i][j];
        if (live && tc == kt)
#pragma unroll
          for (int i = 0; i < TR; ++i) pc[TR * tr + i] = a[i][kj];
        __syncthreads();
        const float v = pc[p];
        const float iv = 1.f / v;
        if (live) {
          float f[TR];
#pragma unroll
          for (int i = 0; i < TR; ++i) f[i] = pc[TR * tr + i];
          if (tr == pt) {
#pragma unroll
            for (int i = 0; i < TR; ++i)
              if (i == pi) f[i] = 0.f;
          }
#pragma unroll
          for (int j = 0; j < TC; ++j) {
            const float spj = pr[TC * tc + j] * iv;
#pragma unroll
            for (int i = 0; i < TR; ++i) a[i][j] = fmaf(-f[i], spj, a[i][j]);
          }
          if (tc == kt) {
#pragma unroll
            for (int i = 0; i < TR; ++i) a[i][kj] = -f[i] * iv;
          }
          if (tr == pt) {
#pragma unroll
            for (int i = 0; i < TR; ++i)
              if (i == pi)
#pragma unroll
                for (int j = 0; j < TC; ++j) a[i][j] = (tc == kt && j == kj) ? iv : pr[TC * tc + j] * iv;
          }
        }
      }
    }
  }
  if (live)
#pragma unroll
    for (int i = 0; i < TR; ++i)
#pragma unroll
      for (int j = 0; j < TC; ++j) {
        const int r = TR * tr + i, c = TC * tc + j;
        if (r < n && c < n) S[r * n + c] = a[i][j];
      }
  __syncthreads();
  // AT[k][l] = A^-1[l][k] = S[piv[l]][stp[k]]
  OT* out = AT + (int64_t)blockIdx.x * n * n;
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int kk = e / n, l = e % n;
    out[e] = (OT)S[piv[l] * n + stp[kk]];
  }
}

// gj_inverse_kernel with the pivot rows known up front (the interchanges of a
// partial-pivoting LU of the same matrix, LAPACK order).  The rows are loaded
// in pivot order -- position k holds original row piv[k] -- so step k
// pivots on position k and column k, and S ends as the inverse of the
// row-permuted matrix: (Phi^-1)[l][c] = S[l][stp[c]] with stp[piv[k]] = k.
// Steps run in unrolled groups of 24 = lcm(12, 8), so the pivot row's place
// in its register tile (k mod 12) and the pivot column's (k mod 8) are
// static: the owners store them with 128-bit stores and every thread reads
// its slices with 128-bit loads.  Every element takes the arithmetic of
// gj_inverse_kernel, in the same order.
template <typename IT, typename OT>
__global__ void __launch_bounds__(384, 1) gj_inverse_pre_kernel(int n, const IT* __restrict__ Phi,
                                                                OT* __restrict__ AT,
                                                                const int32_t* __restrict__ lu_piv) {
  constexpr int TR = kGjTR, TC = kGjTC, U = 24;
  static_assert(U % TR == 0 && U % TC == 0 && TR % 4 == 0 && TC % 4 == 0, "step group and vector slices");
  extern __shared__ __align__(16) unsigned char gj_smem[];
  float* S = reinterpret_cast<float*>(gj_smem);                      // [n][n] final matrix
  float* prow = S + (((int64_t)n * n + 3) & ~(int64_t)3);            // [2][256] pivot row, 16-byte aligned
  float* pcol = prow + 512;                                          // [2][256] pivot column
  int* piv = reinterpret_cast<int*>(pcol + 512);                     // [n] position -> original row
  int* stp = piv + 256;                                              // [n] original row -> position
  const int Gr = (n + TR - 1) / TR, Gc = (n + TC - 1) / TC;
  const int tid = threadIdx.x;
  const int tr = tid / Gc, tc = tid % Gc;
  const bool live = tr < Gr;
  if (tid == 0) {
    const int32_t* lp = lu_piv + (int64_t)blockIdx.x * n;
    for (int k = 0; k < n; ++k) stp[k] = k;
    for (int k = 0; k < n; ++k) {
      const int q = lp[k];
      const int t = stp[k];
      stp[k] = stp[q];
      stp[q] = t;
    }
    for (int k = 0; k < n; ++k) piv[k] = stp[k];
    for (int k = 0; k < n; ++k) stp[piv[k]] = k;
  }
  __syncthreads();
  const IT* P = Phi + (int64_t)blockIdx.x * n * n;
  float a[TR][TC];
#pragma unroll
  for (int i = 0; i < TR; ++i) {
    const int r = TR * tr + i;
    const bool rin = live && r < n;
    const int64_t src = rin ? (int64_t)piv[r] * n : 0;
#pragma unroll
    for (int j = 0; j < TC; ++j) {
      const int c = TC * tc + j;
      a[i][j] = (rin && c < n) ? (float)P[src + c] : 0.f;
    }
  }
  for (int k0 = 0; k0 < n; k0 += U) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u;
      if (k >= n) break;
      const int pt = k0 / TR + u / TR, kt = k0 / TC + u / TC;
      const int pi = u % TR, kj = u % TC;
      float* pr = prow + 256 * (u & 1);
      float* pc = pcol + 256 * (u & 1);
      if (live && tr == pt) {
        float4* q = reinterpret_cast<float4*>(pr + TC * tc);
#pragma unroll
        for (int j4 = 0; j4 < TC / 4; ++j4)
          q[j4] = make_float4(a[pi][4 * j4], a[pi][4 * j4 + 1], a[pi][4 * j4 + 2], a[pi][4 * j4 + 3]);
      }
      if (live && tc == kt) {
        float4* q = reinterpret_cast<float4*>(pc + TR * tr);
#pragma unroll
        for (int i4 = 0; i4 < TR / 4; ++i4)
          q[i4] = make_float4(a[4 * i4][kj], a[4 * i4 + 1][kj], a[4 * i4 + 2][kj], a[4 * i4 + 3][kj]);
      }
      __syncthreads();
      const float v = pc[k];
      const float iv = 1.f / v;
      if (live) {
        float f[TR], sp[TC];
#pragma unroll
        for (int i4 = 0; i4 < TR / 4; ++i4) {
          const float4 q = reinterpret_cast<const float4*>(pc + TR * tr)[i4];
          f[4 * i4] = q.x; f[4 * i4 + 1] = q.y; f[4 * i4 + 2] = q.z; f[4 * i4 + 3] = q.w;
        }
        if (tr == pt) f[pi] = 0.f;
#pragma unroll
        for (int j4 = 0; j4 < TC / 4; ++j4) {
          const float4 q = reinterpret_cast<const float4*>(pr + TC * tc)[j4];
          sp[4 * j4] = q.x * iv; sp[4 * j4 + 1] = q.y * iv; sp[4 * j4 + 2] = q.z * iv; sp[4 * j4 + 3] = q.w * iv;
        }
#pragma unroll
        for (int j = 0; j < TC; ++j)
#pragma unroll
          for (int i = 0; i < TR; ++i) a[i][j] = fmaf(-f[i], sp[j], a[i][j]);
        if (tc == kt) {
#pragma unroll
          for (int i = 0; i < TR; ++i) a[i][kj] = -f[i] * iv;
        }
        if (tr == pt) {
#pragma unroll
          for (int j = 0; j < TC; ++j) a[pi][j] = (tc == kt && j == kj) ? iv : sp[j];
        }
      }
    }
  }
  if (live)
#pragma unroll
    for (int i = 0; i < TR; ++i)
#pragma unroll
      for (int j = 0; j < TC; ++j) {
        const int r = TR * tr + i, c = TC * tc + j;
        if (r < n && c < n) S[r * n + c] = a[i][j];
      }
  __syncthreads();
  // AT[k][l] = (Phi^-1)[l][k] = S[l][stp[k]]
  OT* out = AT + (int64_t)blockIdx.x * n * n;
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int kk = e / n, l = e % n;
    out[e] = (OT)S[l * n + stp[kk]];
  }
}

// Tiles per thread of contract_kernel for neighbourhoods of up to mcap
// members (3 x 4 tiles, one pass).
inline int contract_maxt(int mcap) {
  const int tiles = mcap * ((mcap + 3) / 4);
  for (int t : {1, 2, 3, 5, 9})
    if (256 * t >= tiles) return t;
  return 0;
}

// Shared-memory layout of contract_kernel for a chunk of 32 orbitals l:
// T[l][4 mq] (member k's tangent rows x = 0, 1, 2 at 4k + x) and the inverse
// columns A[l][mq], mq = members rounded up to 4, each row padded by 4
// elements to spread the orbitals over the banks; M [3 mcap][mcap] reuses the
// area at the end.
constexpr int kContractChunk = 32;
__host__ __device__ inline int contract_mq(int mcap) { return 4 * ((mcap + 3) / 4); }
__host__ __device__ inline int contract_stage(int mcap) {
  const int mq = contract_mq(mcap);
  return kContractChunk * ((4 * mq + 4) + (mq + 4));
}

inline size_t contract_smem_bytes(int mcap, size_t tsz) {
  const size_t st = (size_t)contract_stage(mcap), mm = (size_t)3 * mcap * mcap;
  const size_t region = st > mm ? st : mm;
  return region * tsz + 2 * (size_t)mcap * sizeof(int) + 2 * (size_t)mcap * sizeof(int64_t) + 32;
}

inline size_t gj_smem_bytes(int n) { return (size_t)n * n * 4 + 1024 * 4 + 768 * 4 + 128 * 4; }

// Four consecutive shared-memory elements (16-byte aligned for float).
template <typename T>
struct Quad { T v[4]; };
template <typename T>
__device__ __forceinline__ Quad<T> lds4(const T* p) {
  Quad<T> q;
  if constexpr (sizeof(T) == 4) {
    const float4 f = *reinterpret_cast<const float4*>(p);
    q.v[0] = f.x; q.v[1] = f.y; q.v[2] = f.z; q.v[3] = f.w;
  } else {
    const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    q.v[0] = a.x; q.v[1] = a.y; q.v[2] = b.x; q.v[3] = b.y;
  }
  return q;
}

// Gradient and Laplacian of log det Phi_d restricted to the neighbourhoods.
// One CTA per (walker, tangent electron n').  O holds h W_d for every row of
// the forward-Laplacian blocks ([rows][n], row stride ldo); Fenv the envelope rows
// ([Wc*n*5][D*n]); AT the transposed inverses (AT[k][l] = A[l][k],
// [Wc][D][n][n]).
//
// With Nbar = {i_0 = n', i_1, ...} (m members) the CTA forms
//   T[(k,x)][l] = d Phi_{i_k l} / d r_{n' x}      (3m rows)
//   M[(k,x)][k'] = sum_l T[(k,x)][l] A[l][i_k']   (3m x m)
// and from it
//   d log det / d r_{n'x} = sum_k M[(k,x)][k]
//   trace_{n'} = sum_x sum_{k,k'} M[(k,x)][k'] M[(k',x)][k].
// Orbitals go in chunks of 32: the staging thread (orbital lane, member
// group) forms T from the member's three O rows and its envelope value, then
// every thread multiplies member k's 3 rows by 4 columns (MAXT such tiles,
// all in one pass; two 128-bit shared loads per orbital).  Small shared and
// register footprints keep many CTAs resident to hide the gathers' latency.
template <typename T, int MAXT>
__global__ void __launch_bounds__(256, (MAXT <= 3 && sizeof(T) == 4) ? 4 : 1)
contract_kernel(int Wc, int n, int n_up, int K, int mcap, int dd, int D, const int32_t* __restrict__ idx,
                const int32_t* __restrict__ cnt, const int32_t* __restrict__ rev,
                const int64_t* __restrict__ blk_off, const T* __restrict__ O, int64_t ldo,
                const T* __restrict__ Fenv, const T* __restrict__ AT, T* __restrict__ gdet, T* __restrict__ ldet,
                DevStatus* st) {
  constexpr int LC = kContractChunk, NT = 256, NG = NT / LC;
  extern __shared__ __align__(16) unsigned char ct_smem[];
  const int mq = contract_mq(mcap);
  const int ST = 4 * mq + 4, SA = mq + 4;            // row strides of T and A
  T* Ts = reinterpret_cast<T*>(ct_smem);
  T* As = Ts + LC * ST;
  const int64_t region = max((int64_t)contract_stage(mcap), (int64_t)3 * mcap * mcap);
  int64_t* ro = reinterpret_cast<int64_t*>(Ts + ((region + 1) & ~(int64_t)1));   // O row of (k, x = 0)
  int64_t* fo = ro + mcap;                                                    // Fenv value row of member k
  int* mi = reinterpret_cast<int*>(fo + mcap);
  int* ms = mi + mcap;
  __shared__ T red[NT / 32][5];
  const int tid = threadIdx.x;
  const int ol = tid & (LC - 1), og = tid / LC;
  const int w = blockIdx.x / n, np = blockIdx.x % n;
  const int64_t Dn = (int64_t)D * n;
  const int64_t base = (int64_t)w * n + np;
  int m = 1 + cnt[base * 2] + cnt[base * 2 + 1];
  if (m > mcap) m = mcap;
  for (int k = tid; k < m; k += NT) {
    if (k == 0) { mi[0] = np; ms[0] = 0; }
    else {
      mi[k] = idx[base * K + k - 1];
      const int rv = rev[base * K + k - 1];
      ms[k] = rv < 0 ? -1 : rv + 1;
      if (rv < 0) atomicExch(&st->overflow, 1);
    }
    const int i = k == 0 ? np : idx[base * K + k - 1];
    const int64_t b = block_index(w, i, Wc, n, n_up);
    const int slot = k == 0 ? 0 : (ms[k] < 0 ? 0 : ms[k]);
    ro[k] = (k > 0 && ms[k] < 0) ? -1 : (blk_off[b] + 2 + 3 * slot) * ldo;
    fo[k] = b * 5 * Dn + (int64_t)dd * n;
  }
  __syncthreads();
  const T* Aw = AT + ((int64_t)w * D + dd) * n * n;
  const int bnp = block_index(w, np, Wc, n, n_up);
  const int64_t onp = blk_off[bnp];
  const int nq = mq / 4;
  const int ntile = m * nq;

  // sum_l LapPhi_{n' l} A_{l n'}: the Laplacian row of n' against A's column n'
  T lt = T(0);
  {
    const int64_t fb = (int64_t)bnp * 5 * Dn + (int64_t)dd * n;
    for (int l = tid; l < n; l += NT) {
      const T ov = O[onp * ldo + l], olp = O[(onp + 1) * ldo + l];
      T cross = T(0);
      for (int x = 0; x < 3; ++x) cross += O[(onp + 2 + x) * ldo + l] * Fenv[fb + (2 + x) * Dn + l];
      const T lap = olp * Fenv[fb + l] + T(2) * cross + ov * Fenv[fb + Dn + l];
      lt += lap * Aw[(int64_t)np * n + l];
    }
  }

  T acc[MAXT][12];
#pragma unroll
  for (int t = 0; t < MAXT; ++t)
#pragma unroll
    for (int q = 0; q < 12; ++q) acc[t][q] = T(0);
  for (int l0 = 0; l0 < n; l0 += LC) {
    const int l = l0 + ol;
    const bool lin = l < n;
    __syncthreads();
#pragma unroll 2
    for (int k = og; k < mq; k += NG) {
      T v0 = T(0), v1 = T(0), v2 = T(0), a = T(0);
      if (lin && k < m) {
        const int64_t r0 = ro[k];
        if (r0 >= 0) {
          const T phi = Fenv[fo[k] + l];
          v0 = O[r0 + l] * phi;
          v1 = O[r0 + ldo + l] * phi;
          v2 = O[r0 + 2 * ldo + l] * phi;
        }
        if (k == 0) {   // n' itself: its envelope moves too
          const T ov = O[onp * ldo + l];
          v0 += ov * Fenv[fo[0] + 2 * Dn + l];
          v1 += ov * Fenv[fo[0] + 3 * Dn + l];
          v2 += ov * Fenv[fo[0] + 4 * Dn + l];
        }
        a = Aw[(int64_t)mi[k] * n + l];
      }
      T* t = Ts + ol * ST + 4 * k;
      t[0] = v0;
      t[1] = v1;
      t[2] = v2;
      As[ol * SA + k] = a;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < MAXT; ++t) {
      const int tile = tid + t * NT;
      if (tile < ntile) {
        const int k = tile / nq, kq = tile - k * nq;
        const T* tp = Ts + 4 * k;
        const T* ap = As + 4 * kq;
#pragma unroll 8
        for (int q = 0; q < LC; ++q) {
          const Quad<T> av = lds4<T>(tp + q * ST);
          const Quad<T> bv = lds4<T>(ap + q * SA);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[t][j] += av.v[0] * bv.v[j];
            acc[t][4 + j] += av.v[1] * bv.v[j];
            acc[t][8 + j] += av.v[2] * bv.v[j];
          }
        }
      }
    }
  }
  __syncthreads();
  // M into shared memory (the staging area is free now)
  T* Ms = Ts;
#pragma unroll
  for (int t = 0; t < MAXT; ++t) {
    const int tile = tid + t * NT;
    if (tile < ntile) {
      const int k = tile / nq, kq = tile - k * nq;
#pragma unroll
      for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (4 * kq + j < m) Ms[(3 * k + x) * m + 4 * kq + j] = acc[t][4 * x + j];
    }
  }
  __syncthreads();
  T g0 = T(0), g1 = T(0), g2 = T(0), tr = T(0);
  for (int k = tid; k < m; k += NT) {
    g0 += Ms[(3 * k) * m + k];
    g1 += Ms[(3 * k + 1) * m + k];
    g2 += Ms[(3 * k + 2) * m + k];
  }
  for (int e = tid; e < m * m; e += NT) {
    const int k = e / m, kp = e - k * m;
#pragma unroll
    for (int x = 0; x < 3; ++x) tr += Ms[(3 * k + x) * m + kp] * Ms[(3 * kp + x) * m + k];
  }
  // one block reduction of (g0, g1, g2, tr, lt)
  T v[5] = {g0, g1, g2, tr, lt};
#pragma unroll
  for (int q = 0; q < 5; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if ((tid & 31) == 0)
#pragma unroll
    for (int q = 0; q < 5; ++q) red[tid >> 5][q] = v[q];
  __syncthreads();
  if (tid == 0) {
    T sum[5] = {T(0), T(0), T(0), T(0), T(0)};
    for (int g = 0; g < NT / 32; ++g)
#pragma unroll
      for (int q = 0; q < 5; ++q) sum[q] += red[g][q];
    T* gp = gdet + (((int64_t)w * D + dd) * n + np) * 3;
    gp[0] = sum[0];
    gp[1] = sum[1];
    gp[2] = sum[2];
    ldet[((int64_t)w * D + dd) * n + np] = sum[4] - sum[3];
  }
}

// Four consecutive elements p[l .. l+3] (zero beyond n; 128-bit load when
// the row slice is 16-byte aligned, i.e. n % 4 == 0).
__device__ __forceinline__ float4 ld_row4(const float* __restrict__ p, int l, int n, bool vec) {
  if (vec) return l < n ? __ldg(reinterpret_cast<const float4*>(p + l)) : make_float4(0.f, 0.f, 0.f, 0.f);
  float4 v;
  v.x = l < n ? __ldg(p + l) : 0.f;
  v.y = l + 1 < n ? __ldg(p + l + 1) : 0.f;
  v.z = l + 2 < n ? __ldg(p + l + 2) : 0.f;
  v.w = l + 3 < n ? __ldg(p + l + 3) : 0.f;
  return v;
}

// ---------------------------------------------------------------------------
// The same contraction with small CTAs and larger register tiles.  One CTA of
// NT threads per (walker, tangent electron n'); thread tile = 3 members x 3
// coordinates (9 rows of T) x 4 member columns of A, so every orbital l costs
// four 128-bit shared loads for 36 FMAs.  Orbitals go in chunks of 32: each
// staging item (member k, 4 orbitals) reads 128-bit slices of k's three O
// rows, its envelope row and its row of A^T and writes the T quads
// (x = 0, 1, 2, pad) member-contiguous, so neither the gathers nor the shared
// stores conflict.  Neighbourhood sizes are bucketed: a CTA whose member
// count m lies outside [mlo, mhi] exits at once, so one launch per bucket
// sizes its tiles and shared memory for that bucket only.
//   MP = member slots of the bucket (>= every tile's member and column, multiple of 4)
//   Ts [32][4 MP + 4]  T quads     As [32][MP + 4]  A values
//   (M [3 m][m] reuses the area after the last chunk)
constexpr int kC2Chunk = 32;
// Buckets: up to 24 members on 64 threads, 36 on 128, 60 on 320 (one tile per
// thread: ceil(m/3) * ceil(m/4) <= threads).
constexpr int kC2Buckets = 3;
constexpr int kC2BucketMax[kC2Buckets] = {24, 36, 60};
constexpr int kC2BucketThreads[kC2Buckets] = {64, 128, 320};
constexpr int kC2BigMax = 60;
// member slots of a bucket: every tile's members (3 per group) and columns
// (4 per group) of the largest m, rounded to 4 (128-bit rows)
__host__ __device__ inline int contract2_slots(int mhi) {
  const int a = 3 * ((mhi + 2) / 3), b = 4 * ((mhi + 3) / 4);
  const int k = a > b ? a : b;
  return 4 * ((k + 3) / 4);
}
__host__ __device__ inline size_t contract2_region(int mp) {
  const size_t st = (size_t)kC2Chunk * (4 * mp + 4) + (size_t)kC2Chunk * (mp + 4);
  const size_t mm = (size_t)3 * mp * mp;
  return st > mm ? st : mm;
}
inline size_t contract2_smem_bytes(int mhi) {
  const int mp = contract2_slots(mhi);
  return contract2_region(mp) * 4 + (size_t)mp * 20 + 64;
}

template <int NT, int MAXT>
__global__ void __launch_bounds__(NT, 819 / NT)   // at most 80 registers
contract2_kernel(int Wc, int n, int n_up, int K, int mlo, int mhi, int dd, int D, const int32_t* __restrict__ idx,
                 const int32_t* __restrict__ cnt, const int32_t* __restrict__ rev,
                 const int64_t* __restrict__ blk_off, const float* __restrict__ O, int64_t ldo,
                 const float* __restrict__ Fenv, const float* __restrict__ AT, float* __restrict__ gdet,
                 float* __restrict__ ldet, DevStatus* st) {
  constexpr int LC = kC2Chunk;
  extern __shared__ __align__(16) unsigned char c2_smem[];
  __shared__ float red[NT / 32][5];
  const int tid = threadIdx.x;
  const int w = blockIdx.x / n, np = blockIdx.x % n;
  const int64_t base = (int64_t)w * n + np;
  const int m = 1 + cnt[base * 2] + cnt[base * 2 + 1];
  if (m < mlo || m > mhi) return;   // another bucket's launch handles this n'
  const int MP = contract2_slots(mhi);
  const int ST = 4 * MP + 4, SA = MP + 4;
  float* Ts = reinterpret_cast<float*>(c2_smem);
  float* As = Ts + LC * ST;
  const size_t region = contract2_region(MP);
  int64_t* ro = reinterpret_cast<int64_t*>(Ts + ((region + 3) & ~(size_t)3));   // O offset of (k, x = 0), -1: none
  int64_t* fo = ro + MP;                                                        // Fenv offset of k's value row
  int* mi = reinterpret_cast<int*>(fo + MP);
  const int64_t Dn = (int64_t)D * n;
  for (int k = tid; k < m; k += NT) {
    int i = np, slot = 0;
    if (k > 0) {
      i = idx[base * K + k - 1];
      const int rv = rev[base * K + k - 1];
      slot = rv < 0 ? -1 : rv + 1;
      if (rv < 0) atomicExch(&st->overflow, 1);
    }
    const int64_t b = block_index(w, i, Wc, n, n_up);
    mi[k] = i;
    ro[k] = slot < 0 ? -1 : (blk_off[b] + 2 + 3 * (int64_t)slot) * ldo;
    fo[k] = b * 5 * Dn + (int64_t)dd * n;
  }
  __syncthreads();
  const float* Aw = AT + ((int64_t)w * D + dd) * n * n;
  const int bnp = block_index(w, np, Wc, n, n_up);
  const int64_t onp = blk_off[bnp] * ldo;
  const bool vec = (n & 3) == 0 && (ldo & 3) == 0;

  // sum_l LapPhi_{n' l} A_{l n'}: the Laplacian row of n' against A's column n'
  float lt = 0.f;
  {
    const int64_t fb = (int64_t)bnp * 5 * Dn + (int64_t)dd * n;
    for (int l = tid; l < n; l += NT) {
      const float ov = O[onp + l], olp = O[onp + ldo + l];
      float cross = 0.f;
      for (int x = 0; x < 3; ++x) cross += O[onp + (2 + x) * ldo + l] * Fenv[fb + (2 + x) * Dn + l];
      const float lap = olp * Fenv[fb + l] + 2.f * cross + ov * Fenv[fb + Dn + l];
      lt += lap * Aw[(int64_t)np * n + l];
    }
  }

  const int nkg = (m + 2) / 3, ncg = (m + 3) / 4, ntile = nkg * ncg;
  const int kfill = max(3 * nkg, 4 * ncg);   // member slots read by the tiles (zero beyond m)
  float acc[MAXT][36];
#pragma unroll
  for (int t = 0; t < MAXT; ++t)
#pragma unroll
    for (int q = 0; q < 36; ++q) acc[t][q] = 0.f;

  for (int l0 = 0; l0 < n; l0 += LC) {
    __syncthreads();   // the previous chunk is consumed
    // staging items (member k, orbitals l0 + 4 q4 .. + 3), members fastest
    for (int e = tid; e < kfill * (LC / 4); e += NT) {
      const int k = e % kfill, q4 = e / kfill;
      const int l = l0 + 4 * q4;
      float4 t0 = make_float4(0.f, 0.f, 0.f, 0.f), t1 = t0, t2 = t0, av = t0;
      if (k < m) {
        const float4 ph = ld_row4(Fenv + fo[k], l, n, vec);
        if (ro[k] >= 0) {
          const float4 o0 = ld_row4(O + ro[k], l, n, vec);
          const float4 o1 = ld_row4(O + ro[k] + ldo, l, n, vec);
          const float4 o2 = ld_row4(O + ro[k] + 2 * ldo, l, n, vec);
          t0 = make_float4(o0.x * ph.x, o0.y * ph.y, o0.z * ph.z, o0.w * ph.w);
          t1 = make_float4(o1.x * ph.x, o1.y * ph.y, o1.z * ph.z, o1.w * ph.w);
          t2 = make_float4(o2.x * ph.x, o2.y * ph.y, o2.z * ph.z, o2.w * ph.w);
        }
        if (k == 0) {   // n' itself: its envelope moves too
          const float4 ov = ld_row4(O + onp, l, n, vec);
          const float4 g0 = ld_row4(Fenv + fo[0] + 2 * Dn, l, n, vec);
          const float4 g1 = ld_row4(Fenv + fo[0] + 3 * Dn, l, n, vec);
          const float4 g2 = ld_row4(Fenv + fo[0] + 4 * Dn, l, n, vec);
          t0.x += ov.x * g0.x; t0.y += ov.y * g0.y; t0.z += ov.z * g0.z; t0.w += ov.w * g0.w;
          t1.x += ov.x * g1.x; t1.y += ov.y * g1.y; t1.z += ov.z * g1.z; t1.w += ov.w * g1.w;
          t2.x += ov.x * g2.x; t2.y += ov.y * g2.y; t2.z += ov.z * g2.z; t2.w += ov.w * g2.w;
        }
        av = ld_row4(Aw + (int64_t)mi[k] * n, l, n, vec);
      }
      float* tq = Ts + (4 * q4) * ST + 4 * k;
      *reinterpret_cast<float4*>(tq) = make_float4(t0.x, t1.x, t2.x, 0.f);
      *reinterpret_cast<float4*>(tq + ST) = make_float4(t0.y, t1.y, t2.y, 0.f);
      *reinterpret_cast<float4*>(tq + 2 * ST) = make_float4(t0.z, t1.z, t2.z, 0.f);
      *reinterpret_cast<float4*>(tq + 3 * ST) = make_float4(t0.w, t1.w, t2.w, 0.f);
      float* aq = As + (4 * q4) * SA + k;
      aq[0] = av.x;
      aq[SA] = av.y;
      aq[2 * SA] = av.z;
      aq[3 * SA] = av.w;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < MAXT; ++t) {
      const int tile = tid + t * NT;
      if (tile < ntile) {
        const int kg = tile / ncg, cg = tile - kg * ncg;
        const float* tp = Ts + 12 * kg;
        const float* ap = As + 4 * cg;
#pragma unroll 4
        for (int q = 0; q < LC; ++q) {
          const float4 a0 = *reinterpret_cast<const float4*>(tp + q * ST);
          const float4 a1 = *reinterpret_cast<const float4*>(tp + q * ST + 4);
          const float4 a2 = *reinterpret_cast<const float4*>(tp + q * ST + 8);
          const float4 bv = *reinterpret_cast<const float4*>(ap + q * SA);
          const float tr9[9] = {a0.x, a0.y, a0.z, a1.x, a1.y, a1.z, a2.x, a2.y, a2.z};
          const float bc[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
          for (int r = 0; r < 9; ++r)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[t][4 * r + j] = fmaf(tr9[r], bc[j], acc[t][4 * r + j]);
        }
      }
    }
  }
  __syncthreads();
  // M[(k, x)][k'] into shared memory (the staging area is free now)
  float* Ms = Ts;
#pragma unroll
  for (int t = 0; t < MAXT; ++t) {
    const int tile = tid + t * NT;
    if (tile < ntile) {
      const int kg = tile / ncg, cg = tile - kg * ncg;
#pragma unroll
      for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int x = 0; x < 3; ++x)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int k = 3 * kg + u, kp = 4 * cg + j;
            if (k < m && kp < m) Ms[(3 * k + x) * m + kp] = acc[t][4 * (3 * u + x) + j];
          }
    }
  }
  __syncthreads();
  float g0 = 0.f, g1 = 0.f, g2 = 0.f, tr = 0.f;
  for (int k = tid; k < m; k += NT) {
    g0 += Ms[(3 * k) * m + k];
    g1 += Ms[(3 * k + 1) * m + k];
    g2 += Ms[(3 * k + 2) * m + k];
  }
  for (int e = tid; e < m * m; e += NT) {
    const int k = e / m, kp = e - k * m;
#pragma unroll
    for (int x = 0; x < 3; ++x) tr += Ms[(3 * k + x) * m + kp] * Ms[(3 * kp + x) * m + k];
  }
  float v[5] = {g0, g1, g2, tr, lt};
#pragma unroll
  for (int q = 0; q < 5; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if ((tid & 31) == 0)
#pragma unroll
    for (int q = 0; q < 5; ++q) red[tid >> 5][q] = v[q];
  __syncthreads();
  if (tid == 0) {
    float sum[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int g = 0; g < NT / 32; ++g)
#pragma unroll
      for (int q = 0; q < 5; ++q) sum[q] += red[g][q];
    float* gp = gdet + (((int64_t)w * D + dd) * n + np) * 3;
    gp[0] = sum[0];
    gp[1] = sum[1];
    gp[2] = sum[2];
    ldet[((int64_t)w * D + dd) * n + np] = sum[4] - sum[3];
  }
}

// ---------------------------------------------------------------------------
// contract2_kernel with asynchronous staging (n and the O row stride multiples
// of 4) and 16-orbital chunks: the raw 64-byte row slices of a chunk -- member k's three O rows,
// its envelope row and its row of A^T, plus n''s value row and envelope
// gradient rows -- are copied with cp.async into a raw buffer (rows of 20
// floats, so the transform's member-strided 128-bit reads do not conflict)
// while the previous chunk is being multiplied; a transform pass then forms
// the T quads and the A columns of the compute layout.
//   raw rows: O (k, x) at 3k + x; envelope k at 3 MP + k; A^T k at 4 MP + k;
//             n' value row at 5 MP; envelope gradient x at 5 MP + 1 + x
constexpr int kC3Chunk = 16;       // orbitals per chunk (small buffers: more CTAs per SM)
constexpr int kC3RawStride = 20;   // raw row: 16 floats + 4 pad (member-strided reads do not conflict)
// Buckets of the asynchronous form: the thread count of each is the smallest
// multiple of 32 that gives every (3-member, 4-column) tile its own thread.
constexpr int kC3Buckets = 5;
constexpr int kC3BucketMax[kC3Buckets] = {27, 32, 36, 48, 60};
constexpr int kC3BucketThreads[kC3Buckets] = {64, 96, 128, 192, 320};
struct C3Buckets { int v[kC3Buckets]; };
// Every bucket's transform pass has at most two (member, quad) items per
// thread: 4 kfill <= 2 NT at the bucket maximum (kfill grows with m).
constexpr bool c3_transform_fits() {
  for (int q = 0; q < kC3Buckets; ++q) {
    const int m = kC3BucketMax[q];
    const int a = 3 * ((m + 2) / 3), b = 4 * ((m + 3) / 4);
    if ((a > b ? a : b) * (kC3Chunk / 4) > 2 * kC3BucketThreads[q]) return false;
  }
  return true;
}
static_assert(c3_transform_fits(), "contract3 transform items exceed two per thread");

// Sorts the tangent electrons e = w n + n' of a chunk into the buckets by
// their neighbourhood size m = 1 + |N_n'| (warp-aggregated atomics; the
// order inside a bucket does not matter).
template <int kUnused = 0>
__global__ void contract_bucket_kernel(int nb, const int32_t* __restrict__ cnt, C3Buckets bm,
                                       int* __restrict__ counts, int* __restrict__ lists) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = e < nb;
  int b = kC3Buckets - 1;
  if (in) {
    const int m = 1 + cnt[2 * (int64_t)e] + cnt[2 * (int64_t)e + 1];
    for (int q = kC3Buckets - 1; q >= 0; --q)
      if (m <= bm.v[q]) b = q;
  }
  const unsigned act = __ballot_sync(0xffffffffu, in);
  if (!in) return;
  const unsigned same = __match_any_sync(act, b);
  const int leader = __ffs(same) - 1;
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == leader) base = atomicAdd(&counts[b], __popc(same));
  base = __shfl_sync(same, base, leader);
  lists[(int64_t)b * nb + base + __popc(same & ((1u << lane) - 1u))] = e;
}
__host__ __device__ inline size_t contract3_raw_floats(int mp) { return (size_t)(5 * mp + 4) * kC3RawStride; }
__host__ __device__ inline size_t contract3_region(int mp) {
  const size_t st = (size_t)kC3Chunk * (4 * mp + 4) + (size_t)kC3Chunk * (mp + 4);
  const size_t mm = (size_t)3 * mp * mp;
  return st > mm ? st : mm;
}
inline size_t contract3_smem_bytes(int mhi) {
  const int mp = contract2_slots(mhi);
  return (contract3_region(mp) + contract3_raw_floats(mp)) * 4 + (size_t)mp * 20 + (size_t)(5 * mp + 4) * 12 + 80;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <int NT>
__global__ void __launch_bounds__(NT, 819 / NT)   // at most 80 registers
contract3_kernel(int Wc, int n, int n_up, int K, int mlo, int mhi, int dd, int D, const int32_t* __restrict__ idx,
                 const int32_t* __restrict__ cnt, const int32_t* __restrict__ rev,
                 const int64_t* __restrict__ blk_off, const float* __restrict__ O, int64_t ldo,
                 const float* __restrict__ Fenv, const float* __restrict__ AT, float* __restrict__ gdet,
                 float* __restrict__ ldet, DevStatus* st, const int* __restrict__ list) {
  constexpr int LC = kC3Chunk, RS = kC3RawStride, NJ = LC / 4;
  extern __shared__ __align__(16) unsigned char c3_smem[];
  __shared__ float red[NT / 32][5];
  const int tid = threadIdx.x;
  // CTA -> tangent electron: from the bucket list, else blockIdx = w n + n'
  const int e0 = list ? list[blockIdx.x] : (int)blockIdx.x;
  const int w = e0 / n, np = e0 % n;
  const int64_t base = (int64_t)w * n + np;
  const int m = 1 + cnt[base * 2] + cnt[base * 2 + 1];
  if (m < mlo || m > mhi) return;   // another bucket's launch handles this n'
  const int MP = contract2_slots(mhi);
  const int ST = 4 * MP + 4, SA = MP + 4;
  float* Ts = reinterpret_cast<float*>(c3_smem);
  float* As = Ts + LC * ST;
  const size_t region = contract3_region(MP);
  float* raw = Ts + region;
  int64_t* ro = reinterpret_cast<int64_t*>(raw + ((contract3_raw_floats(MP) + 3) & ~(size_t)3));
  int64_t* fo = ro + MP;
  int* mi = reinterpret_cast<int*>(fo + MP);
  // source row (nullptr: zero fill) and raw row of every copy row, set once
  const float** rsrc = reinterpret_cast<const float**>(mi + ((MP + 1) & ~1));
  int* rrow = reinterpret_cast<int*>(rsrc + 5 * MP + 4);
  const int64_t Dn = (int64_t)D * n;
  for (int k = tid; k < m; k += NT) {
    int i = np, slot = 0;
    if (k > 0) {
      i = idx[base * K + k - 1];
      const int rv = rev[base * K + k - 1];
      slot = rv < 0 ? -1 : rv + 1;
      if (rv < 0) atomicExch(&st->overflow, 1);
    }
    const int64_t b = block_index(w, i, Wc, n, n_up);
    mi[k] = i;
    ro[k] = slot < 0 ? -1 : (blk_off[b] + 2 + 3 * (int64_t)slot) * ldo;
    fo[k] = b * 5 * Dn + (int64_t)dd * n;
  }
  __syncthreads();
  const float* Aw = AT + ((int64_t)w * D + dd) * n * n;
  const int bnp = block_index(w, np, Wc, n, n_up);
  const int64_t onp = blk_off[bnp] * ldo;
  const int nkg = (m + 2) / 3, ncg = (m + 3) / 4, ntile = nkg * ncg;
  const int kfill = max(3 * nkg, 4 * ncg);

  // raw copies of the chunk starting at orbital c0 (zero beyond n and m)
  const int nraw = 5 * kfill + 4;
  for (int q = tid; q < nraw; q += NT) {
    const float* src = nullptr;
    int rr;
    if (q < 3 * kfill) {
      const int k = q / 3, x = q - 3 * k;
      rr = q;
      if (k < m && ro[k] >= 0) src = O + ro[k] + x * ldo;
    } else if (q < 4 * kfill) {
      const int k = q - 3 * kfill;
      rr = 3 * MP + k;
      if (k < m) src = Fenv + fo[k];
    } else if (q < 5 * kfill) {
      const int k = q - 4 * kfill;
      rr = 4 * MP + k;
      if (k < m) src = Aw + (int64_t)mi[k] * n;
    } else {
      const int u = q - 5 * kfill;
      rr = 5 * MP + u;
      src = u == 0 ? O + onp : Fenv + fo[0] + (1 + u) * Dn;
    }
    rsrc[q] = src;
    rrow[q] = rr;
  }
  __syncthreads();
  // a thread always copies quad j = tid % NJ of its rows (NT is a multiple
  // of NJ), rows tid / NJ, tid / NJ + NT / NJ, ...
  static_assert(NT % NJ == 0, "thread count must be a multiple of the quads per row");
  const int jq = tid % NJ;
  auto issue = [&](int c0) {
    const int l = c0 + 4 * jq;
    const bool lin = l < n;
    for (int q = tid / NJ; q < nraw; q += NT / NJ) {
      const float* src = rsrc[q];
      const bool ok = lin && src != nullptr;
      cp_async16(raw + rrow[q] * RS + 4 * jq, ok ? src + l : O, ok ? 16 : 0);
    }
    cp_async_commit();
  };
  issue(0);

  // sum_l LapPhi_{n' l} A_{l n'}: the Laplacian row of n' against A's column n'
  float lt = 0.f;
  {
    const int64_t fb = (int64_t)bnp * 5 * Dn + (int64_t)dd * n;
    for (int l = tid; l < n; l += NT) {
      const float ov = O[onp + l], olp = O[onp + ldo + l];
      float cross = 0.f;
      for (int x = 0; x < 3; ++x) cross += O[onp + (2 + x) * ldo + l] * Fenv[fb + (2 + x) * Dn + l];
      const float lap = olp * Fenv[fb + l] + 2.f * cross + ov * Fenv[fb + Dn + l];
      lt += lap * Aw[(int64_t)np * n + l];
    }
  }

  float acc[36];
#pragma unroll
  for (int q = 0; q < 36; ++q) acc[q] = 0.f;
  const bool act = tid < ntile;
  const int kg = act ? tid / ncg : 0, cg = act ? tid - kg * ncg : 0;

  for (int l0 = 0; l0 < n; l0 += LC) {
    cp_async_wait_all();
    __syncthreads();   // the raw chunk has landed; the previous chunk is consumed
    // transform items e = (quad q4, member k), k fastest: at most two per
    // thread (4 kfill <= 2 NT in every bucket); q4 = e / kfill by compares
#pragma unroll 1
    for (int it = 0; it < 2; ++it) {
      const int e = tid + it * NT;
      if (e >= kfill * (LC / 4)) continue;
      const int q4 = (e >= kfill) + (e >= 2 * kfill) + (e >= 3 * kfill);
      const int k = e - q4 * kfill;
      const float4 o0 = *reinterpret_cast<const float4*>(raw + (3 * k) * RS + 4 * q4);
      const float4 o1 = *reinterpret_cast<const float4*>(raw + (3 * k + 1) * RS + 4 * q4);
      const float4 o2 = *reinterpret_cast<const float4*>(raw + (3 * k + 2) * RS + 4 * q4);
      const float4 ph = *reinterpret_cast<const float4*>(raw + (3 * MP + k) * RS + 4 * q4);
      const float4 av = *reinterpret_cast<const float4*>(raw + (4 * MP + k) * RS + 4 * q4);
      float4 t0 = make_float4(o0.x * ph.x, o0.y * ph.y, o0.z * ph.z, o0.w * ph.w);
      float4 t1 = make_float4(o1.x * ph.x, o1.y * ph.y, o1.z * ph.z, o1.w * ph.w);
      float4 t2 = make_float4(o2.x * ph.x, o2.y * ph.y, o2.z * ph.z, o2.w * ph.w);
      if (k == 0) {   // n' itself: its envelope moves too
        const float4 ov = *reinterpret_cast<const float4*>(raw + (5 * MP) * RS + 4 * q4);
        const float4 g0 = *reinterpret_cast<const float4*>(raw + (5 * MP + 1) * RS + 4 * q4);
        const float4 g1 = *reinterpret_cast<const float4*>(raw + (5 * MP + 2) * RS + 4 * q4);
        const float4 g2 = *reinterpret_cast<const float4*>(raw + (5 * MP + 3) * RS + 4 * q4);
        t0.x += ov.x * g0.x; t0.y += ov.y * g0.y; t0.z += ov.z * g0.z; t0.w += ov.w * g0.w;
        t1.x += ov.x * g1.x; t1.y += ov.y * g1.y; t1.z += ov.z * g1.z; t1.w += ov.w * g1.w;
        t2.x += ov.x * g2.x; t2.y += ov.y * g2.y; t2.z += ov.z * g2.z; t2.w += ov.w * g2.w;
      }
      float* tq = Ts + (4 * q4) * ST + 4 * k;
      *reinterpret_cast<float4*>(tq) = make_float4(t0.x, t1.x, t2.x, 0.f);
      *reinterpret_cast<float4*>(tq + ST) = make_float4(t0.y, t1.y, t2.y, 0.f);
      *reinterpret_cast<float4*>(tq + 2 * ST) = make_float4(t0.z, t1.z, t2.z, 0.f);
      *reinterpret_cast<float4*>(tq + 3 * ST) = make_float4(t0.w, t1.w, t2.w, 0.f);
      float* aq = As + (4 * q4) * SA + k;
      aq[0] = av.x;
      aq[SA] = av.y;
      aq[2 * SA] = av.z;
      aq[3 * SA] = av.w;
    }
    __syncthreads();   // compute layout ready; the raw buffer is free
    if (l0 + LC < n) issue(l0 + LC);
    if (act) {
      const float* tp = Ts + 12 * kg;
      const float* ap = As + 4 * cg;
#pragma unroll 4
      for (int q = 0; q < LC; ++q) {
        const float4 a0 = *reinterpret_cast<const float4*>(tp + q * ST);
        const float4 a1 = *reinterpret_cast<const float4*>(tp + q * ST + 4);
        const float4 a2 = *reinterpret_cast<const float4*>(tp + q * ST + 8);
        const float4 bv = *reinterpret_cast<const float4*>(ap + q * SA);
        const float tr9[9] = {a0.x, a0.y, a0.z, a1.x, a1.y, a1.z, a2.x, a2.y, a2.z};
        const float bc[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
        for (int r = 0; r < 9; ++r)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[4 * r + j] = fmaf(tr9[r], bc[j], acc[4 * r + j]);
      }
    }
  }
  __syncthreads();
  // M[(k, x)][k'] into shared memory (the staging area is free now)
  float* Ms = Ts;
  if (act) {
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
      for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = 3 * kg + u, kp = 4 * cg + j;
          if (k < m && kp < m) Ms[(3 * k + x) * m + kp] = acc[4 * (3 * u + x) + j];
        }
  }
  __syncthreads();
  float g0 = 0.f, g1 = 0.f, g2 = 0.f, tr = 0.f;
  for (int k = tid; k < m; k += NT) {
    g0 += Ms[(3 * k) * m + k];
    g1 += Ms[(3 * k + 1) * m + k];
    g2 += Ms[(3 * k + 2) * m + k];
  }
  for (int e = tid; e < m * m; e += NT) {
    const int k = e / m, kp = e - k * m;
#pragma unroll
    for (int x = 0; x < 3; ++x) tr += Ms[(3 * k + x) * m + kp] * Ms[(3 * kp + x) * m + k];
  }
  float v[5] = {g0, g1, g2, tr, lt};
#pragma unroll
  for (int q = 0; q < 5; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if ((tid & 31) == 0)
#pragma unroll
    for (int q = 0; q < 5; ++q) red[tid >> 5][q] = v[q];
  __syncthreads();
  if (tid == 0) {
    float sum[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int g = 0; g < NT / 32; ++g)
#pragma unroll
      for (int q = 0; q < 5; ++q) sum[q] += red[g][q];
    float* gp = gdet + (((int64_t)w * D + dd) * n + np) * 3;
    gp[0] = sum[0];
    gp[1] = sum[1];
    gp[2] = sum[2];
    ldet[((int64_t)w * D + dd) * n + np] = sum[4] - sum[3];
  }
}

}  // namespace fire

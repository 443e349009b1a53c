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
// value, Laplacian, d/dx, d/dy, d/dz).  One CTA per electron.
template <typename T, typename W>
__global__ void env_feat_kernel(int Wc, int n, int n_up, int N, int E, const double* __restrict__ r,
                                const double* __restrict__ R, const W* sig, T* __restrict__ Q, int R5) {
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
    Q[row * NE + q] = v;
    if (R5 > 1) {
      Q[(row + 1) * NE + q] = (s * s - T(2) * s / rt) * v;
      for (int t = 0; t < 3; ++t) Q[(row + 2 + t) * NE + q] = -s * v * T(dd[t]) / rt;
    }
  }
}

// Phi[w][d][i][l] = O_v[b(i)][d*n + l] * Fenv[b(i)*R5][d*n + l].
// One CTA per (w, d).
template <typename T, typename LT>
__global__ void phi_assemble_kernel(int Wc, int n, int n_up, int D, const T* __restrict__ Ov,
                                    const T* __restrict__ Fenv, int R5, LT* __restrict__ Phi) {
  const int w = blockIdx.x / D, dd = blockIdx.x % D;
  const int64_t Dn = (int64_t)D * n;
  LT* P = Phi + (int64_t)blockIdx.x * n * n;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, l = e % n;
    const int64_t b = block_index(w, i, Wc, n, n_up);
    P[e] = LT(Ov[b * Dn + dd * n + l]) * LT(Fenv[b * R5 * Dn + dd * n + l]);
  }
}

// Blocked right-looking LU with partial pivoting, one CTA per matrix, the
// matrix in global memory (L2-resident), the current panel and U12 block in
// shared memory.  Writes the pivots, log|det| and sign (0 and -inf for an
// exactly zero pivot).
template <typename LT, int NB>
__global__ void lu_kernel(int n, LT* __restrict__ M, int32_t* __restrict__ piv,
                          double* __restrict__ logabs, double* __restrict__ sgn) {
  extern __shared__ unsigned char lu_smem[];
  LT* P = reinterpret_cast<LT*>(lu_smem);      // [n][NB]
  LT* U = P + (int64_t)n * NB;                 // [NB][n]
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_piv;
  __shared__ int s_zero;
  LT* A = M + (int64_t)blockIdx.x * n * n;
  int32_t* pv = piv + (int64_t)blockIdx.x * n;
  const int tid = threadIdx.x, bd = blockDim.x;
  if (tid == 0) s_zero = 0;
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int nb = min(NB, n - k0);
    const int pr = n - k0;  // panel rows
    for (int e = tid; e < pr * nb; e += bd) {
      const int r = e / nb, c = e % nb;
      P[r * NB + c] = A[(int64_t)(k0 + r) * n + k0 + c];
    }
    __syncthreads();
    for (int kk = 0; kk < nb; ++kk) {
      // argmax |P[r][kk]| over r in [kk, pr), first index on ties
      double best = -1.0;
      int bi = kk;
      for (int r = kk + tid; r < pr; r += bd) {
        double v = fabs((double)P[r * NB + kk]);
        if (v > best) { best = v; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if ((tid & 31) == 0) { red_v[tid >> 5] = best; red_i[tid >> 5] = bi; }
      __syncthreads();
      if (tid == 0) {
        double b = red_v[0];
        int ib = red_i[0];
        for (int q = 1; q < (bd + 31) / 32; ++q)
          if (red_v[q] > b || (red_v[q] == b && red_i[q] < ib)) { b = red_v[q]; ib = red_i[q]; }
        s_piv = ib;
        pv[k0 + kk] = k0 + ib;
        if (!(b > 0.0)) s_zero = 1;
      }
      __syncthreads();
      const int p = s_piv;
      if (p != kk) {
        for (int c = tid; c < nb; c += bd) {
          LT t = P[kk * NB + c];
          P[kk * NB + c] = P[p * NB + c];
          P[p * NB + c] = t;
        }
      }
      __syncthreads();
      const LT pivot = P[kk * NB + kk];
      if (pivot != LT(0)) {
        for (int r = kk + 1 + tid; r < pr; r += bd) {
          LT l = P[r * NB + kk] / pivot;
          P[r * NB + kk] = l;
          for (int c = kk + 1; c < nb; ++c) P[r * NB + c] -= l * P[kk * NB + c];
        }
      }
      __syncthreads();
    }
    // panel back to global
    for (int e = tid; e < pr * nb; e += bd) {
      const int r = e / nb, c = e % nb;
      A[(int64_t)(k0 + r) * n + k0 + c] = P[r * NB + c];
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
          for (int q = 0; q < kk; ++q) s -= P[kk * NB + q] * u[q];
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
      const LT* lrow = P + (int64_t)(r - k0) * NB;
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

// A = Phi^-1 from the LU factors: column j of A solves L U x = e_{pinv[j]}.
// One CTA per matrix, one thread per column, x kept in shared memory.
template <typename LT, typename AT>
__global__ void lu_inverse_kernel(int n, const LT* __restrict__ M, const int32_t* __restrict__ piv,
                                  AT* __restrict__ Ainv) {
  extern __shared__ unsigned char inv_smem[];
  AT* X = reinterpret_cast<AT*>(inv_smem);        // [n][n]
  int* perm = reinterpret_cast<int*>(X + (int64_t)n * n);
  int* pinv = perm + n;
  const LT* A = M + (int64_t)blockIdx.x * n * n;
  const int32_t* pv = piv + (int64_t)blockIdx.x * n;
  if (threadIdx.x == 0) {
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int k = 0; k < n; ++k) {
      int t = perm[k];
      perm[k] = perm[pv[k]];
      perm[pv[k]] = t;
    }
    for (int i = 0; i < n; ++i) pinv[perm[i]] = i;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const int p = pinv[j];
    for (int i = 0; i < n; ++i) {
      AT s = (i == p) ? AT(1) : AT(0);
      for (int k = 0; k < i; ++k) s -= AT(A[(int64_t)i * n + k]) * X[(int64_t)k * n + j];
      X[(int64_t)i * n + j] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
      AT s = X[(int64_t)i * n + j];
      for (int k = i + 1; k < n; ++k) s -= AT(A[(int64_t)i * n + k]) * X[(int64_t)k * n + j];
      X[(int64_t)i * n + j] = s / AT(A[(int64_t)i * n + i]);
    }
  }
  __syncthreads();
  AT* out = Ainv + (int64_t)blockIdx.x * n * n;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) out[e] = X[e];
}

// Gradient and Laplacian of log det Phi_d restricted to the neighbourhoods.
// One CTA per (walker, tangent electron n').  O holds h W_d for every row of
// the forward-Laplacian blocks ([rows][n]); Fenv the envelope rows
// ([Wc*n*5][D*n]); Ainv the inverses ([Wc][D][n][n]).
template <typename T>
__global__ void contract_kernel(int Wc, int n, int n_up, int K, int dd, int D,
                                const int32_t* __restrict__ idx, const int32_t* __restrict__ cnt,
                                const int32_t* __restrict__ rev, const int64_t* __restrict__ blk_off,
                                const T* __restrict__ O, const T* __restrict__ Fenv,
                                const T* __restrict__ Ainv, T* __restrict__ gdet,
                                T* __restrict__ ldet, DevStatus* st) {
  extern __shared__ unsigned char ct_smem[];
  const int ldn = n + 1;
  const int mcap = 1 + K;
  T* Tt = reinterpret_cast<T*>(ct_smem);            // [3*mcap][ldn]
  T* As = Tt + (int64_t)3 * mcap * ldn;              // [mcap][ldn], As[k][l] = A[l][i_k]
  int* mi = reinterpret_cast<int*>(As + (int64_t)mcap * ldn);
  int* ms = mi + mcap;
  __shared__ T red[32];
  const int w = blockIdx.x / n, np = blockIdx.x % n;
  const int64_t Dn = (int64_t)D * n;
  const int64_t base = (int64_t)w * n + np;
  const int m = 1 + cnt[base * 2] + cnt[base * 2 + 1];
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    if (k == 0) { mi[0] = np; ms[0] = 0; }
    else {
      mi[k] = idx[base * K + k - 1];
      int rv = rev[base * K + k - 1];
      ms[k] = rv + 1;
      if (rv < 0) atomicExch(&st->overflow, 1);
    }
  }
  __syncthreads();
  const T* Aw = Ainv + ((int64_t)w * D + dd) * n * n;
  for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
    const int k = e / n, l = e % n;
    As[(int64_t)k * ldn + l] = Aw[(int64_t)l * n + mi[k]];
  }
  for (int e = threadIdx.x; e < 3 * m * n; e += blockDim.x) {
    const int row = e / n, l = e % n;
    const int k = row / 3, x = row % 3;
    const int i = mi[k];
    const int64_t b = block_index(w, i, Wc, n, n_up);
    const int slot = ms[k] > 0 ? ms[k] : 0;
    const int64_t orow = blk_off[b] + 2 + 3 * slot + x;
    const T phi = Fenv[(b * 5) * Dn + dd * n + l];
    T v = (ms[k] < 0 && k > 0) ? T(0) : O[orow * n + l] * phi;
    if (k == 0) v += O[blk_off[b] * n + l] * Fenv[(b * 5 + 2 + x) * Dn + dd * n + l];
    Tt[(int64_t)row * ldn + l] = v;
  }
  __syncthreads();
  T g0 = T(0), g1 = T(0), g2 = T(0), tr = T(0);
  const int mm = m * m;
  for (int e = threadIdx.x; e < 3 * mm; e += blockDim.x) {
    const int x = e / mm, rem = e % mm;
    const int k = rem / m, kp = rem % m;
    if (kp < k) continue;
    const T* ta = Tt + (int64_t)(3 * k + x) * ldn;
    const T* ab = As + (int64_t)kp * ldn;
    T s1 = T(0);
    for (int l = 0; l < n; ++l) s1 += ta[l] * ab[l];
    if (k == kp) {
      tr += s1 * s1;
      if (x == 0) g0 += s1; else if (x == 1) g1 += s1; else g2 += s1;
    } else {
      const T* tb = Tt + (int64_t)(3 * kp + x) * ldn;
      const T* aa = As + (int64_t)k * ldn;
      T s2 = T(0);
      for (int l = 0; l < n; ++l) s2 += tb[l] * aa[l];
      tr += T(2) * s1 * s2;
    }
  }
  // sum_l LapPhi_{n' l} A_{l n'}
  T lt = T(0);
  {
    const int64_t b = block_index(w, np, Wc, n, n_up);
    const int64_t o0 = blk_off[b];
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
      const int64_t fc = dd * n + l;
      const T ov = O[o0 * n + l], ol = O[(o0 + 1) * n + l];
      const T fv = Fenv[(b * 5) * Dn + fc], fl = Fenv[(b * 5 + 1) * Dn + fc];
      T cross = T(0);
      for (int x = 0; x < 3; ++x) cross += O[(o0 + 2 + x) * n + l] * Fenv[(b * 5 + 2 + x) * Dn + fc];
      const T lap = ol * fv + T(2) * cross + ov * fl;
      lt += lap * As[l];
    }
  }
  // block reductions
  auto bsum = [&](T v) -> T {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    T s = T(0);
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
    return s;
  };
  g0 = bsum(g0);
  g1 = bsum(g1);
  g2 = bsum(g2);
  tr = bsum(tr);
  lt = bsum(lt);
  if (threadIdx.x == 0) {
    T* gp = gdet + (((int64_t)w * D + dd) * n + np) * 3;
    gp[0] = g0;
    gp[1] = g1;
    gp[2] = g2;
    ldet[((int64_t)w * D + dd) * n + np] = lt - tr;
  }
}

}  // namespace fire

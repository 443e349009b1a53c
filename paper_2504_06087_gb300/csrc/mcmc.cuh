// Metropolis sampling with single-electron moves and low-rank wave-function
// updates (Methods, "Improved Monte Carlo sampling" and "Low-rank updates").
//
// Moving electron k from r_k to r'_k changes the embeddings of the update set
// U = {k} u {i : |r_i - r_k| <= c} u {i : |r_i - r'_k| <= c} only: h^0_i
// depends on r_i alone and the single message-passing round only sees
// electrons within c.  Those rows of h and of every orbital matrix are
// recomputed; with A = Phi^-1 cached, the determinant ratio is
//   det(Phi') / det(Phi) = det(M),  M = I + Delta A[:, U]   (|U| x |U|)
// (matrix determinant lemma, Delta = Phi'_U - Phi_U), and an accepted move
// updates A by the Woodbury identity
//   A' = A - A[:, U] M^-1 Delta A.
// A is kept transposed (AT[k][l] = A[l][k]) so that a column of A is a row.
//
// The members of U of every walker are compacted into one row list, spin-up
// rows first, so each product of the move is one matrix product over the
// rows of all walkers.
#pragma once

#include "common.cuh"
#include "philox.cuh"

namespace fire {

// ---------------------------------------------------------------------------
// CTA-wide tiled products (256 threads, 32 x 32 tiles, 2 x 2 per thread).
//   nt: C[i][j] (+)= alpha sum_k A[i][k] B[brow(j)][k]
//   tn: C[i][j] (+)= alpha sum_k A[k][i] B[k][j]
// sm holds 2 x 32 x 33 elements.
// ---------------------------------------------------------------------------
template <typename T>
__device__ void cta_gemm_nt(int M, int N, int K, const T* __restrict__ A, int64_t lda, const T* __restrict__ B,
                            int64_t ldb, const int32_t* __restrict__ brow, T* __restrict__ C, int64_t ldc,
                            T alpha, bool accumulate, T* sm) {
  T(*as)[33] = reinterpret_cast<T(*)[33]>(sm);
  T(*bs)[33] = reinterpret_cast<T(*)[33]>(sm + 32 * 33);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  for (int i0 = 0; i0 < M; i0 += 32)
    for (int j0 = 0; j0 < N; j0 += 32) {
      T acc[2][2] = {{T(0), T(0)}, {T(0), T(0)}};
      for (int k0 = 0; k0 < K; k0 += 32) {
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
          const int r = e / 32, c = e % 32;   // r: row of A or B, c: k
          const int kk = k0 + c;
          as[c][r] = (i0 + r < M && kk < K) ? A[(int64_t)(i0 + r) * lda + kk] : T(0);
          const int jj = j0 + r;
          bs[c][r] = (jj < N && kk < K) ? B[(int64_t)(brow ? brow[jj] : jj) * ldb + kk] : T(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int c = 0; c < 32; ++c) {
          const T a0 = as[c][2 * ty], a1 = as[c][2 * ty + 1];
          const T b0 = bs[c][2 * tx], b1 = bs[c][2 * tx + 1];
          acc[0][0] += a0 * b0; acc[0][1] += a0 * b1;
          acc[1][0] += a1 * b0; acc[1][1] += a1 * b1;
        }
      }
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int i = i0 + 2 * ty + p, j = j0 + 2 * tx + q;
          if (i < M && j < N) {
            T* o = C + (int64_t)i * ldc + j;
            *o = accumulate ? *o + alpha * acc[p][q] : alpha * acc[p][q];
          }
        }
    }
  __syncthreads();
}

template <typename T>
__device__ void cta_gemm_tn(int M, int N, int K, const T* __restrict__ A, int64_t lda, const T* __restrict__ B,
                            int64_t ldb, T* __restrict__ C, int64_t ldc, T alpha, bool accumulate, T* sm) {
  T(*as)[33] = reinterpret_cast<T(*)[33]>(sm);
  T(*bs)[33] = reinterpret_cast<T(*)[33]>(sm + 32 * 33);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  for (int i0 = 0; i0 < M; i0 += 32)
    for (int j0 = 0; j0 < N; j0 += 32) {
      T acc[2][2] = {{T(0), T(0)}, {T(0), T(0)}};
      for (int k0 = 0; k0 < K; k0 += 32) {
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
          const int r = e / 32, c = e % 32;   // r: k, c: column of A or B
          const int kk = k0 + r;
          as[r][c] = (kk < K && i0 + c < M) ? A[(int64_t)kk * lda + i0 + c] : T(0);
          bs[r][c] = (kk < K && j0 + c < N) ? B[(int64_t)kk * ldb + j0 + c] : T(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int r = 0; r < 32; ++r) {
          const T a0 = as[r][2 * ty], a1 = as[r][2 * ty + 1];
          const T b0 = bs[r][2 * tx], b1 = bs[r][2 * tx + 1];
          acc[0][0] += a0 * b0; acc[0][1] += a0 * b1;
          acc[1][0] += a1 * b0; acc[1][1] += a1 * b1;
        }
      }
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int i = i0 + 2 * ty + p, j = j0 + 2 * tx + q;
          if (i < M && j < N) {
            T* o = C + (int64_t)i * ldc + j;
            *o = accumulate ? *o + alpha * acc[p][q] : alpha * acc[p][q];
          }
        }
    }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Proposal r'_k = r_k + sigma xi and the acceptance uniform from Philox4x32-10:
// key (seed low, seed high); counter (move low, move high, walker, 0) gives
// four uniforms and, by Box-Muller in float64, xi; counter (..., 1) gives u.
// Then the update set U of the walker, ascending (so its spin-up members come
// first); Ucu = number of spin-up members.  One warp per walker.
// ---------------------------------------------------------------------------
// The update set U of walker w for moving electron k from rw[k] to rn: k and
// every electron within c of either position, ascending (so its spin-up
// members come first); Ucu = number of spin-up members.  One warp; an
// inactive walker gets an empty set.
__device__ inline void update_set(int w, int lane, int n, int n_up, int k, const double* __restrict__ rw,
                                  const double* rn, double c2, int Umax, int32_t* __restrict__ Ul,
                                  int32_t* __restrict__ Uc, int32_t* __restrict__ Ucu, DevStatus* st, bool active) {
  int cntU = 0, cntUp = 0;
  if (active)
    for (int j0 = 0; j0 < n; j0 += 32) {
      const int j = j0 + lane;
      bool in = false;
      if (j < n) {
        if (j == k) {
          in = true;
        } else {
          double a2 = 0.0, b2 = 0.0;
          for (int t = 0; t < 3; ++t) {
            const double da = rw[3 * j + t] - rw[3 * k + t], db = rw[3 * j + t] - rn[t];
            a2 += da * da;
            b2 += db * db;
          }
          in = (a2 <= c2) || (b2 <= c2);
        }
      }
      const unsigned m = __ballot_sync(0xffffffffu, in);
      if (in) {
        const int pos = cntU + __popc(m & ((1u << lane) - 1u));
        if (pos < Umax) Ul[(int64_t)w * Umax + pos] = j;
      }
      cntU += __popc(m);
      const unsigned mu = __ballot_sync(0xffffffffu, in && j < n_up);
      cntUp += __popc(mu);
    }
  if (lane == 0) {
    if (cntU > Umax) {
      atomicExch(&st->overflow, 1);
      atomicMax(&st->k_required, cntU);
    }
    Uc[w] = cntU < Umax ? cntU : Umax;
    Ucu[w] = cntUp < Umax ? cntUp : Umax;
  }
}

// Global jump (Methods, "Improved Monte Carlo sampling"): the proposal
// density of the mixture sum_m Z_m N(r | R_m, sigma_g^2 I) / sum_m Z_m at x,
// as a logarithm (log-sum-exp over the nuclei, float64).
__device__ inline double gmm_log_density(const double* x, const double* __restrict__ R,
                                         const double* __restrict__ Z, int N, double sigma_g) {
  const double inv = 1.0 / (2.0 * sigma_g * sigma_g);
  double mx = -INFINITY, zt = 0.0;
  for (int m = 0; m < N; ++m) {
    double d2 = 0.0;
    for (int t = 0; t < 3; ++t) {
      const double dx = x[t] - R[3 * m + t];
      d2 += dx * dx;
    }
    const double e = log(Z[m]) - d2 * inv;
    if (e > mx) mx = e;
    zt += Z[m];
  }
  double sum = 0.0;
  for (int m = 0; m < N; ++m) {
    double d2 = 0.0;
    for (int t = 0; t < 3; ++t) {
      const double dx = x[t] - R[3 * m + t];
      d2 += dx * dx;
    }
    sum += exp(log(Z[m]) - d2 * inv - mx);
  }
  return mx + log(sum) - log(zt) - 1.5 * log(6.283185307179586476925286766559 * sigma_g * sigma_g);
}

// Local moves: r'_k = r_k + sigma xi.  Global jumps (global != 0): a mixture
// component m with probability Z_m / sum Z (the first m whose cumulative
// charge exceeds u sum Z, u from stream 2) and r'_k = R_m + sigma_g xi;
// lq[w] = ln rho(r_k) - ln rho(r'_k), the Hastings factor of the
// asymmetric proposal (0 for local moves).
static __global__ void mcmc_propose_kernel(int n, int n_up, int k, const double* __restrict__ r, double sigma,
                                    uint64_t seed, uint64_t move, int64_t w0, double c2, int Umax,
                                    double* __restrict__ rk, double* __restrict__ uacc, int32_t* __restrict__ Ul,
                                    int32_t* __restrict__ Uc, int32_t* __restrict__ Ucu, DevStatus* st,
                                    int global, const double* __restrict__ nuc_pos,
                                    const double* __restrict__ nuc_charge, int N, double sigma_g,
                                    double* __restrict__ lq) {
  const int w = blockIdx.x;
  const int lane = threadIdx.x;
  const double* rw = r + (int64_t)w * n * 3;
  __shared__ double rn[3];
  if (lane == 0) {
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const uint32_t m0 = (uint32_t)move, m1 = (uint32_t)(move >> 32), wg = (uint32_t)(w0 + w);
    const Philox4 a = philox4x32_10(m0, m1, wg, 0u, k0, k1);
    const Philox4 b = philox4x32_10(m0, m1, wg, 1u, k0, k1);
    const double two_pi = 6.283185307179586476925286766559;
    const double ra = sqrt(-2.0 * log(u01(a.v[0]))), rb = sqrt(-2.0 * log(u01(a.v[2])));
    const double t1 = two_pi * u01(a.v[1]), t3 = two_pi * u01(a.v[3]);
    const double xi[3] = {ra * cos(t1), ra * sin(t1), rb * cos(t3)};
    if (global) {
      const Philox4 c = philox4x32_10(m0, m1, wg, 2u, k0, k1);
      double zt = 0.0;
      for (int m = 0; m < N; ++m) zt += nuc_charge[m];
      const double target = u01(c.v[0]) * zt;
      int comp = N - 1;
      double cum = 0.0;
      for (int m = 0; m < N; ++m) {
        cum += nuc_charge[m];
        if (target < cum) { comp = m; break; }
      }
      for (int t = 0; t < 3; ++t) rn[t] = nuc_pos[3 * comp + t] + sigma_g * xi[t];
      lq[w] = gmm_log_density(rw + 3 * k, nuc_pos, nuc_charge, N, sigma_g) -
              gmm_log_density(rn, nuc_pos, nuc_charge, N, sigma_g);
    } else {
      for (int t = 0; t < 3; ++t) rn[t] = rw[3 * k + t] + sigma * xi[t];
      lq[w] = 0.0;
    }
    for (int t = 0; t < 3; ++t) rk[(int64_t)w * 3 + t] = rn[t];
    uacc[w] = u01(b.v[0]);
  }
  __syncwarp();
  update_set(w, lane, n, n_up, k, rw, rn, c2, Umax, Ul, Uc, Ucu, st, true);
}

// Compact row index of every member of U: spin-up members of all walkers
// first (walker-major), then the spin-down ones.  rng = {0, up, up, total,
// 0, total}.  One CTA of 1024 threads.
static __global__ void __launch_bounds__(1024) mcmc_scan_kernel(int W, int Umax, const int32_t* __restrict__ Uc,
                                                         const int32_t* __restrict__ Ucu, int32_t* __restrict__ Urow,
                                                         int64_t* __restrict__ rng) {
  __shared__ int64_t sa[1024], sb[1024];
  __shared__ int64_t carry[2], tot_up;
  const int t = threadIdx.x;
  int64_t s = 0;
  for (int w = t; w < W; w += 1024) s += Ucu[w];
  sa[t] = s;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (t < o) sa[t] += sa[t + o];
    __syncthreads();
  }
  if (t == 0) {
    tot_up = sa[0];
    carry[0] = 0;
    carry[1] = 0;
  }
  __syncthreads();
  const int64_t up_total = tot_up;
  for (int base = 0; base < W; base += 1024) {
    const int w = base + t;
    const int64_t cu = w < W ? Ucu[w] : 0, cd = w < W ? Uc[w] - Ucu[w] : 0;
    sa[t] = cu;
    sb[t] = cd;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {   // inclusive Hillis-Steele scans
      const int64_t xa = t >= o ? sa[t - o] : 0, xb = t >= o ? sb[t - o] : 0;
      __syncthreads();
      sa[t] += xa;
      sb[t] += xb;
      __syncthreads();
    }
    if (w < W) {
      const int64_t uo = carry[0] + sa[t] - cu, dof = up_total + carry[1] + sb[t] - cd;
      const int nu = (int)cu, nt = Uc[w];
      for (int a = 0; a < nt; ++a) Urow[(int64_t)w * Umax + a] = (int32_t)(a < nu ? uo + a : dof + (a - nu));
    }
    __syncthreads();
    if (t == 1023) {
      carry[0] += sa[t];
      carry[1] += sb[t];
    }
    __syncthreads();
  }
  if (t == 0) {
    rng[0] = 0; rng[1] = up_total; rng[2] = up_total; rng[3] = up_total + carry[1];
    rng[4] = 0; rng[5] = up_total + carry[1];
  }
}

// h^1 of every member i of U under the proposed positions (value only),
//   h^1_i = h^0_i + sum_{j in N_i} Gamma(e_ij) SiLU(h^0_i W^a + h^0_j W^a' + e-bar_ij W^a_c + b^a).
// For i = k every term changes: the neighbour list is rebuilt on the fly
// (same spin ascending, then the opposite spin) with h^0 and projections of
// k from h0k / PQk.  For i != k only the term of the pair (i, k) changes:
// h^1_i = cached h^1_i - [old (i, k) term] + [new (i, k) term], each present
// when that distance is within c.  One CTA per (walker, slot), blockDim == d;
// dynamic shared memory n ints.  Writes h^1 to X (overwritten by the MLP) and
// to H1n (kept for the cache).
template <typename T, typename W>
__global__ void mcmc_msg_kernel(int Wn, int n, int n_up, int d, int k, int Umax, const double* __restrict__ r,
                                const double* __restrict__ rk, double cut, Params<W> p,
                                const int32_t* __restrict__ Ul, const int32_t* __restrict__ Uc,
                                const int32_t* __restrict__ Urow, const T* __restrict__ H0,
                                const T* __restrict__ PQ, const T* __restrict__ H1, const T* __restrict__ h0k,
                                const T* __restrict__ PQk, T* __restrict__ X, T* __restrict__ H1n) {
  constexpr int H = kEdgeHidden, G = kGauss;
  __shared__ FL3<T> feat[H + G + 4];
  extern __shared__ int mm_nbr[];
  __shared__ int s_cnt[2];
  const int w = blockIdx.x / Umax, u = blockIdx.x % Umax;
  if (u >= Uc[w]) return;
  const int i = Ul[(int64_t)w * Umax + u];
  const int c = threadIdx.x;
  const int64_t ld4 = 4 * (int64_t)d;
  const double* rw = r + (int64_t)w * n * 3;
  const double* rkw = rk + (int64_t)w * 3;
  T w2[H], we[G], wc[2][4], bb[2];
#pragma unroll
  for (int h = 0; h < H; ++h) w2[h] = T(p.ee_w2[h * d + c]);
#pragma unroll
  for (int g = 0; g < G; ++g) we[g] = T(p.ee_wenv[g * d + c]);
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    bb[a] = T(p.msg_b[a * d + c]);
#pragma unroll
    for (int q = 0; q < 4; ++q) wc[a][q] = T(p.msg_w[((int64_t)a * (2 * d + 4) + 2 * d + q) * d + c]);
  }
  // one message term: Gamma(delta) SiLU(Pi^a + Qj^a + e-bar W_c^a + b^a)
  auto term = [&](const double ddv[3], const T* Pi, const T* Qj, int a) -> T {
    const double rr = sqrt(ddv[0] * ddv[0] + ddv[1] * ddv[1] + ddv[2] * ddv[2]);
    T dv[3] = {T(ddv[0]), T(ddv[1]), T(ddv[2])};
    __syncthreads();
    pair_features_to_smem<T, W>(dv, T(rr), p.ee_w1, p.ee_b1, p.ee_sigma, T(cut), feat);
    __syncthreads();
    T gv = T(0), ev = T(0), eb = T(0);
#pragma unroll
    for (int h = 0; h < H; ++h) gv += feat[h].v * w2[h];
#pragma unroll
    for (int g = 0; g < G; ++g) ev += feat[H + g].v * we[g];
#pragma unroll
    for (int q = 0; q < 4; ++q) eb += feat[H + G + q].v * wc[a][q];
    const T z = Pi[(int64_t)a * d + c] + Qj[2 * (int64_t)d + (int64_t)a * d + c] + eb + bb[a];
    T f, f1, f2;
    silu3<T>(z, f, f1, f2);
    return (gv * ev) * f;
  };
  T acc;
  if (i == k) {
    auto pos = [&](int j, int t) -> double { return j == k ? rkw[t] : rw[3 * j + t]; };
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      const bool up = i < n_up;
      int cntN = 0;
      for (int pass = 0; pass < 2; ++pass) {
        const bool same = pass == 0;
        const int lo = (up == same) ? 0 : n_up, hi = (up == same) ? n_up : n;
        for (int j0 = lo; j0 < hi; j0 += 32) {
          const int j = j0 + lane;
          bool in = false;
          if (j < hi && j != i) {
            double a2 = 0.0;
            for (int t = 0; t < 3; ++t) {
              const double dd = pos(i, t) - pos(j, t);
              a2 += dd * dd;
            }
            in = a2 <= cut * cut;
          }
          const unsigned m = __ballot_sync(0xffffffffu, in);
          if (in) mm_nbr[cntN + __popc(m & ((1u << lane) - 1u))] = j;
          cntN += __popc(m);
        }
        if (lane == 0) s_cnt[pass] = cntN;
      }
    }
    __syncthreads();
    const int cpar = s_cnt[0], ctot = s_cnt[1];
    const T* Pi = PQk + (int64_t)w * ld4;
    acc = h0k[(int64_t)w * d + c];
    for (int s = 0; s < ctot; ++s) {
      const int j = mm_nbr[s];
      const double ddv[3] = {pos(i, 0) - pos(j, 0), pos(i, 1) - pos(j, 1), pos(i, 2) - pos(j, 2)};
      acc += term(ddv, Pi, PQ + (int64_t)block_index(w, j, Wn, n, n_up) * ld4, s < cpar ? 0 : 1);
    }
  } else {
    const int bi = block_index(w, i, Wn, n, n_up);
    const T* Pi = PQ + (int64_t)bi * ld4;
    const int a = ((i < n_up) == (k < n_up)) ? 0 : 1;
    acc = H1[(int64_t)bi * d + c];
    for (int side = 0; side < 2; ++side) {   // 0: remove the old (i, k) term, 1: add the new one
      const double* q = side == 0 ? rw + 3 * k : rkw;
      const double ddv[3] = {rw[3 * i] - q[0], rw[3 * i + 1] - q[1], rw[3 * i + 2] - q[2]};
      if (!(ddv[0] * ddv[0] + ddv[1] * ddv[1] + ddv[2] * ddv[2] <= cut * cut)) continue;
      const T* Qk = side == 0 ? PQ + (int64_t)block_index(w, k, Wn, n, n_up) * ld4 : PQk + (int64_t)w * ld4;
      const T t = term(ddv, Pi, Qk, a);
      acc += side == 0 ? -t : t;
    }
  }
  const int64_t row = Urow[(int64_t)w * Umax + u];
  X[row * d + c] = acc;
  H1n[row * d + c] = acc;
}

// Y[row][c] = (residual ? Y[row][c] : 0) + SiLU(Z[row][c] + b[c]) for rows in
// [rng[0], rng[1]); grid-stride over rows x columns.
template <typename T, typename W>
__global__ void mcmc_act_kernel(const int64_t* __restrict__ rng, int ncol, const T* __restrict__ Z, int64_t ldz,
                                const W* bias, T* __restrict__ Y, int64_t ldy, int residual) {
  const int64_t r0 = rng[0], r1 = rng[1];
  const int64_t total = (r1 - r0) * ncol;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = r0 + e / ncol;
    const int c = (int)(e % ncol);
    T f, f1, f2;
    silu3<T>(Z[row * ldz + c] + T(bias[c]), f, f1, f2);
    Y[row * ldy + c] = residual ? Y[row * ldy + c] + f : f;
  }
}

// log of the shrink factor beyond which a determinant is refactorised: a
// determinant that an accepted move leaves more than 100 times smaller than
// at its last factorisation gets a fresh float64 LU and inverse from the
// cached Phi instead of its Woodbury update, whose rounding errors grow with
// that shrink (a single determinant passing near its own node while the
// others keep Psi away from zero).
constexpr double kRepairLogShrink = -4.605170185988091;   // ln(1e-2)

// A determinant-lemma ratio beyond e^{+-6.9} (a factor 1000) is recomputed
// exactly, as log|det Phi'| - log|det Phi| from a float64 LU of the new
// matrix: a float32 inverse of a badly conditioned matrix can turn a modest
// ratio into a huge one, which would then dominate the determinant sum.
constexpr double kExactLogRatio = 6.907755278982137;      // ln(1e3)

// |U| up to which the small determinant-lemma matrix lives in shared memory.
constexpr int kLemmaSmem = 64;

// Determinant lemma for one (walker, det): Delta rows of U (new orbital row
// times envelope minus the cached Phi row), M = I + Delta A[:, U], its LU with
// partial pivoting in float64, log|det M| and sign.  Delta, the LU factors
// (in Mg, [Umax][Umax] per pair) and the pivots are kept for the Woodbury
// update, which solves with them: M can be far from orthogonal (a nearly
// singular determinant has a large A, so Delta A[:, U] is large while det M
// stays moderate), and an explicit M^-1 would lose the digits the solve keeps.
// One CTA (256 threads) per (walker, det); the LU runs in shared memory when
// |U| <= kLemmaSmem, else in Mg.
template <typename T>
__global__ void __launch_bounds__(256) mcmc_ratio_kernel(
    int Wn, int n, int n_up, int D, int k, int Umax, const int32_t* __restrict__ Ul, const int32_t* __restrict__ Uc,
    const int32_t* __restrict__ Urow, const T* __restrict__ On, const T* __restrict__ Fenv, const T* __restrict__ Fk,
    const T* __restrict__ Phi, const T* __restrict__ AT, T* __restrict__ Dl, T* __restrict__ Mt,
    double* __restrict__ Mg, int32_t* __restrict__ Mpiv, double* __restrict__ lrat, double* __restrict__ srat,
    int k2 = -1, const T* __restrict__ Fk2 = nullptr) {
  __shared__ double su[kLemmaSmem * (kLemmaSmem + 1)];   // the product tiles, then M
  __shared__ int s_p;
  const int w = blockIdx.x / D, dd = blockIdx.x % D;
  const int u = Uc[w];
  const int64_t Dn = (int64_t)D * n;
  const int64_t md = (int64_t)w * D + dd;
  const int32_t* U = Ul + (int64_t)w * Umax;
  const T* Pw = Phi + md * n * n;
  const T* Aw = AT + md * n * n;
  T* Dw = Dl + md * Umax * n;
  for (int e = threadIdx.x; e < u * n; e += blockDim.x) {
    const int aa = e / n, l = e % n;
    const int i = U[aa];
    const T o = On[(int64_t)Urow[(int64_t)w * Umax + aa] * Dn + dd * n + l];
    const T ph = (i == k)    ? Fk[(int64_t)w * Dn + dd * n + l]
                 : (i == k2) ? Fk2[(int64_t)w * Dn + dd * n + l]
                             : Fenv[(int64_t)block_index(w, i, Wn, n, n_up) * Dn + dd * n + l];
    Dw[(int64_t)aa * n + l] = o * ph - Pw[(int64_t)i * n + l];
  }
  // Delta A[:, U] = Delta (u x n) times the rows U of A^T
  T* Mw = Mt + md * Umax * Umax;
  cta_gemm_nt<T>(u, u, n, Dw, n, Aw, n, U, Mw, Umax, T(1), false, reinterpret_cast<T*>(su));
  const bool in_smem = u <= kLemmaSmem;
  double* M = in_smem ? su : Mg + md * Umax * Umax;
  const int ldm = in_smem ? kLemmaSmem + 1 : Umax;
  for (int e = threadIdx.x; e < u * u; e += blockDim.x) {
    const int a = e / u, b = e % u;
    M[a * ldm + b] = (double)Mw[a * Umax + b] + (a == b ? 1.0 : 0.0);
  }
  __syncthreads();
  int32_t* pv = Mpiv + md * Umax;
  double la = 0.0;
  int neg = 0;
  bool zero = false;
  for (int c = 0; c < u; ++c) {
    if (threadIdx.x < 32) {   // pivot: the first row of largest |M[q][c]|, q >= c
      double best = -1.0;
      int bq = c;
      for (int q = c + threadIdx.x; q < u; q += 32) {
        const double v = fabs(M[q * ldm + c]);
        if (v > best) { best = v; bq = q; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oq = __shfl_xor_sync(0xffffffffu, bq, o);
        if (ob > best || (ob == best && oq < bq)) { best = ob; bq = oq; }
      }
      if (threadIdx.x == 0) { s_p = bq; pv[c] = bq; }
    }
    __syncthreads();
    const int pq = s_p;
    if (pq != c) {
      for (int q = threadIdx.x; q < u; q += blockDim.x) {
        const double t = M[c * ldm + q];
        M[c * ldm + q] = M[pq * ldm + q];
        M[pq * ldm + q] = t;
      }
      neg ^= 1;
    }
    __syncthreads();
    const double piv = M[c * ldm + c];
    if (piv == 0.0) {
      zero = true;
    } else {
      la += log(fabs(piv));
      if (piv < 0.0) neg ^= 1;
      const int wdt = u - c - 1;
      for (int e = threadIdx.x; e < wdt * wdt; e += blockDim.x) {
        const int q = c + 1 + e / wdt, cc = c + 1 + e % wdt;
        M[q * ldm + cc] -= (M[q * ldm + c] / piv) * M[c * ldm + cc];
      }
      __syncthreads();
      for (int q = c + 1 + threadIdx.x; q < u; q += blockDim.x) M[q * ldm + c] /= piv;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    lrat[md] = zero ? -INFINITY : la;
    srat[md] = zero ? 0.0 : (neg ? -1.0 : 1.0);
  }
  // the factors go to Mg for the Woodbury solve (already there when M lived in Mg)
  if (in_smem) {
    double* G = Mg + md * Umax * Umax;
    for (int e = threadIdx.x; e < u * u; e += blockDim.x) G[(e / u) * Umax + e % u] = M[(e / u) * ldm + e % u];
  }
}

// Attention registers with the rows of U replaced (value only):
// V_r = sum_i softmax_i(s_ir) v_ir, the scores and values of U from SUn.
// One CTA per walker, one thread per column of V.
template <typename T>
__global__ void mcmc_att_kernel(int Wn, int n, int n_up, int R, int dr, int Umax, const int32_t* __restrict__ Ul,
                                const int32_t* __restrict__ Uc, const int32_t* __restrict__ Urow,
                                const T* __restrict__ SU, int64_t ld, const T* __restrict__ SUn, int64_t ldn,
                                T* __restrict__ Vn) {
  extern __shared__ unsigned char ma_smem[];
  int* slot = reinterpret_cast<int*>(ma_smem);    // [n]: compact row of i in U, or -1
  T* smax = reinterpret_cast<T*>(ma_smem + (((size_t)n * sizeof(int) + 15) & ~(size_t)15));
  const int w = blockIdx.x;
  const int RD = R * dr;
  for (int i = threadIdx.x; i < n; i += blockDim.x) slot[i] = -1;
  __syncthreads();
  for (int a = threadIdx.x; a < Uc[w]; a += blockDim.x) slot[Ul[(int64_t)w * Umax + a]] = Urow[(int64_t)w * Umax + a];
  __syncthreads();
  auto row = [&](int i) -> const T* {
    return slot[i] >= 0 ? SUn + (int64_t)slot[i] * ldn : SU + (int64_t)block_index(w, i, Wn, n, n_up) * ld;
  };
  for (int q = threadIdx.x; q < R; q += blockDim.x) {
    T m = -INFINITY;
    for (int i = 0; i < n; ++i) m = fmax(m, row(i)[q]);
    smax[q] = m;
  }
  __syncthreads();
  for (int col = threadIdx.x; col < RD; col += blockDim.x) {
    const int rg = col / dr;
    T Z = T(0), Nv = T(0);
    for (int i = 0; i < n; ++i) {
      const T* rr = row(i);
      const T e = dexp<T>(rr[rg] - smax[rg]);
      Z += e;
      Nv += e * rr[R + col];
    }
    Vn[(int64_t)w * RD + col] = Nv / Z;
  }
}

// Jastrow parameters the acceptance test reads (type T).
struct McmcJastrow {
  const void *cusp, *jb32, *ab32;
};

// ln|Psi'/Psi| and sign(Psi'/Psi) of walker w for the move of electron k to
// rk (all lanes of one warp call it; the result is valid on lane 0):
// determinant part from the ratios of all determinants, cusp change of
// electron k, change of the MLP-Jastrow sums over the update set, change of
// the attention-Jastrow readout.
struct WalkerRatio {
  double logr, sign;
};

template <typename T>
__device__ WalkerRatio walker_ratio(int w, int lane, int Wn, int n, int n_up, int D, int k, int Umax, uint32_t flags,
                                    const double* __restrict__ rw, const double* __restrict__ rn, int k2,
                                    const double* __restrict__ rn2,
                                    const int32_t* __restrict__ Ul, const int32_t* __restrict__ Uc,
                                    const int32_t* __restrict__ Urow, const McmcJastrow& jp,
                                    const T* __restrict__ F1, const T* __restrict__ F2, const T* __restrict__ F1n,
                                    const T* __restrict__ F2n, const T* __restrict__ G1, const T* __restrict__ G2,
                                    const T* __restrict__ G1n, const T* __restrict__ G2n,
                                    const double* __restrict__ ldabs, const double* __restrict__ lsign,
                                    const double* __restrict__ lrat, const double* __restrict__ srat) {
  const T* cusp = reinterpret_cast<const T*>(jp.cusp);
  double dc = 0.0, s2 = 0.0, ds1 = 0.0, ds2 = 0.0;
  const double wp = (double)cusp[0], wa = (double)cusp[1], ap = (double)cusp[2], aa = (double)cusp[3];
  // cusp terms of the pairs of a moved electron (k, and k2 >= 0 for a swap of
  // two electrons, whose own pair keeps its distance and spin channel)
  for (int j = lane; j < n; j += 32) {
    for (int mv = 0; mv < 2; ++mv) {
      const int km = mv == 0 ? k : k2;
      const double* rm = mv == 0 ? rn : rn2;
      if (km < 0 || j == k || j == k2) continue;
      const bool same = (j < n_up) == (km < n_up);
      const double om = same ? wp : wa, al = same ? ap : aa;
      double o2 = 0.0, n2 = 0.0;
      for (int t = 0; t < 3; ++t) {
        const double a = rw[3 * km + t] - rw[3 * j + t], b = rm[t] - rw[3 * j + t];
        o2 += a * a;
        n2 += b * b;
      }
      dc += om * al * al / (al + sqrt(n2)) - om * al * al / (al + sqrt(o2));
    }
    if (flags & FIRE_J_MLP) s2 += (double)F2[block_index(w, j, Wn, n, n_up)];
  }
  if (flags & FIRE_J_MLP)
    for (int a = lane; a < Uc[w]; a += 32) {
      const int i = Ul[(int64_t)w * Umax + a];
      const int64_t b = block_index(w, i, Wn, n, n_up);
      const int64_t q = Urow[(int64_t)w * Umax + a];
      ds1 += (double)F1n[q] - (double)F1[b];
      ds2 += (double)F2n[q] - (double)F2[b];
    }
  for (int o = 16; o > 0; o >>= 1) {
    dc += __shfl_xor_sync(0xffffffffu, dc, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    ds1 += __shfl_xor_sync(0xffffffffu, ds1, o);
    ds2 += __shfl_xor_sync(0xffffffffu, ds2, o);
  }
  WalkerRatio out{0.0, 0.0};
  if (lane != 0) return out;
  // determinants: ln|sum_d s_d rho_d e^{l_d}| - ln|sum_d s_d e^{l_d}|
  const double* lw = ldabs + (int64_t)w * D;
  const double* sw = lsign + (int64_t)w * D;
  const double* lr = lrat + (int64_t)w * D;
  const double* sr = srat + (int64_t)w * D;
  double lmax = -INFINITY, lmaxn = -INFINITY;
  auto live = [&](int q) { return sw[q] * sr[q] != 0.0 && isfinite(lr[q]); };
  for (int q = 0; q < D; ++q) {
    if (sw[q] != 0.0 && lw[q] > lmax) lmax = lw[q];
    if (live(q) && lw[q] + lr[q] > lmaxn) lmaxn = lw[q] + lr[q];
  }
  double So = 0.0, Sn = 0.0;
  for (int q = 0; q < D; ++q) {
    if (sw[q] != 0.0) So += sw[q] * exp(lw[q] - lmax);
    if (live(q)) Sn += sw[q] * sr[q] * exp(lw[q] + lr[q] - lmaxn);
  }
  double logr = (lmaxn + log(fabs(Sn))) - (lmax + log(fabs(So)));
  double sg = (Sn > 0.0) == (So > 0.0) ? 1.0 : -1.0;
  if (Sn == 0.0) sg = 0.0;
  if (flags & FIRE_J_CUSP) logr += dc;
  if (flags & FIRE_J_MLP) {
    const double S2o = s2 + n * (double)reinterpret_cast<const T*>(jp.jb32)[0];
    logr += ds1 + log(fabs(S2o + ds2)) - log(fabs(S2o));
    if ((S2o + ds2 > 0.0) != (S2o > 0.0)) sg = -sg;
  }
  if (flags & FIRE_J_ATT) {
    const double b32 = (double)reinterpret_cast<const T*>(jp.ab32)[0];
    const double gn = (double)G2n[w] + b32, go = (double)G2[w] + b32;
    logr += ((double)G1n[w] - (double)G1[w]) + log(fabs(gn)) - log(fabs(go));
    if ((gn > 0.0) != (go > 0.0)) sg = -sg;
  }
  out.logr = logr;
  out.sign = sg;
  return out;
}

// Accept / reject: accept iff ln u < 2 ln|Psi'/Psi| + lq (lq = 0 for a local
// move, the Hastings factor ln rho(r_k) - ln rho(r'_k) for a global jump)
// and the ratio is finite.  One warp per walker; an accepted walker moves r_k
// and updates its determinant logs and its running log|Psi|.
template <typename T>
__global__ void mcmc_accept_kernel(int Wn, int n, int n_up, int D, int k, int Umax, uint32_t flags,
                                   double* __restrict__ r, const double* __restrict__ rk,
                                   const double* __restrict__ uacc, const int32_t* __restrict__ Ul,
                                   const int32_t* __restrict__ Uc, const int32_t* __restrict__ Urow, McmcJastrow jp,
                                   const T* __restrict__ F1, const T* __restrict__ F2, const T* __restrict__ F1n,
                                   const T* __restrict__ F2n, const T* __restrict__ G1, const T* __restrict__ G2,
                                   const T* __restrict__ G1n, const T* __restrict__ G2n,
                                   double* __restrict__ ldabs, double* __restrict__ lsign,
                                   const double* __restrict__ lrat, const double* __restrict__ srat,
                                   double* __restrict__ lp, int32_t* __restrict__ acc,
                                   int32_t* __restrict__ acc_count, unsigned long long* __restrict__ nacc,
                                   const double* __restrict__ lref, int32_t* __restrict__ flag,
                                   const int32_t* __restrict__ xflag, const double* __restrict__ lq,
                                   int* __restrict__ rcnt, int32_t* __restrict__ rlist, int rcap,
                                   unsigned long long* __restrict__ nrepair) {
  const int w = blockIdx.x;
  const int lane = threadIdx.x;
  double* rw = r + (int64_t)w * n * 3;
  const double* rn = rk + (int64_t)w * 3;
  const WalkerRatio wr = walker_ratio<T>(w, lane, Wn, n, n_up, D, k, Umax, flags, rw, rn, -1, nullptr, Ul, Uc, Urow,
                                         jp, F1, F2, F1n, F2n, G1, G2, G1n, G2n, ldabs, lsign, lrat, srat);
  if (lane != 0) return;
  const double logr = wr.logr;
  const double* lr = lrat + (int64_t)w * D;
  const double* sr = srat + (int64_t)w * D;
  const bool ok = isfinite(logr) && (log(uacc[w]) < 2.0 * logr + lq[w]);
  acc[w] = ok ? 1 : 0;
  if (ok) {
    for (int t = 0; t < 3; ++t) rw[3 * k + t] = rn[t];
    for (int q = 0; q < D; ++q) {
      const int64_t md = (int64_t)w * D + q;
      if (isfinite(lr[q])) {
        ldabs[md] += lr[q];
        lsign[md] *= sr[q];
      } else {
        ldabs[md] = -INFINITY;
        lsign[md] = 0.0;
      }
      // refactorise a determinant that shrank too far since its last LU
      // (and one whose ratio took the exact path: its A is not trusted);
      // flag 2: in the batched refactorisation list, 1: done by
      // mcmc_repair_kernel (the list is full)
      int fl = (ldabs[md] >= lref[md] + kRepairLogShrink && !xflag[md]) ? 0 : 1;
      if (fl && nrepair) atomicAdd(nrepair, 1ull);
      if (fl && rlist) {
        const int slot = atomicAdd(rcnt, 1);
        if (slot < rcap) {
          rlist[slot] = (int32_t)md;
          fl = 2;
        }
      }
      flag[md] = fl;
    }
    lp[w] += logr;
    if (acc_count) acc_count[w] += 1;
    atomicAdd(nacc, 1ull);
  }
}

// Copies the recomputed rows of an accepted move into the cached state:
// h^1, MLP-Jastrow outputs and attention scores/values of every member of U, the
// initial embedding, projections and envelope row of electron k, and the
// walker's attention registers and readouts.  One CTA per (walker, slot).
template <typename T>
__global__ void mcmc_rows_kernel(int Wn, int n, int n_up, int d, int Dn, int RD, int k, int Umax, int64_t ldsu,
                                 int64_t ldsun, int has_mlp, int has_att, const int32_t* __restrict__ acc,
                                 const int32_t* __restrict__ Ul, const int32_t* __restrict__ Uc,
                                 const int32_t* __restrict__ Urow, const T* __restrict__ F1n,
                                 const T* __restrict__ F2n, T* __restrict__ F1, T* __restrict__ F2,
                                 const T* __restrict__ SUn, T* __restrict__ SU, const T* __restrict__ h0k,
                                 T* __restrict__ H0, const T* __restrict__ PQk, T* __restrict__ PQ,
                                 const T* __restrict__ Fk, T* __restrict__ Fenv, const T* __restrict__ Vn,
                                 T* __restrict__ V, const T* __restrict__ G1n, const T* __restrict__ G2n,
                                 T* __restrict__ G1, T* __restrict__ G2, const T* __restrict__ H1n,
                                 T* __restrict__ H1) {
  const int w = blockIdx.x / Umax, a = blockIdx.x % Umax;
  if (!acc[w] || a >= Uc[w]) return;
  const int i = Ul[(int64_t)w * Umax + a];
  const int64_t b = block_index(w, i, Wn, n, n_up);
  const int64_t q = Urow[(int64_t)w * Umax + a];
  for (int c = threadIdx.x; c < d; c += blockDim.x) H1[b * d + c] = H1n[q * d + c];
  if (has_att)
    for (int c = threadIdx.x; c < ldsun; c += blockDim.x) SU[b * ldsu + c] = SUn[q * ldsun + c];
  if (has_mlp && threadIdx.x == 0) {
    F1[b] = F1n[q];
    F2[b] = F2n[q];
  }
  if (i == k) {
    for (int c = threadIdx.x; c < d; c += blockDim.x) H0[b * d + c] = h0k[(int64_t)w * d + c];
    for (int c = threadIdx.x; c < 4 * d; c += blockDim.x) PQ[b * 4 * d + c] = PQk[(int64_t)w * 4 * d + c];
    for (int c = threadIdx.x; c < Dn; c += blockDim.x) Fenv[b * Dn + c] = Fk[(int64_t)w * Dn + c];
  }
  if (a == 0 && has_att) {
    for (int c = threadIdx.x; c < RD; c += blockDim.x) V[(int64_t)w * RD + c] = Vn[(int64_t)w * RD + c];
    if (threadIdx.x == 0) {
      G1[w] = G1n[w];
      G2[w] = G2n[w];
    }
  }
}

// Woodbury update of A^T and the rows U of Phi for accepted walkers:
//   B = Delta A (u x n), C = M^-1 B (solved with the LU factors of M),
//   A'^T[m][l] = A^T[m][l] - sum_a C[a][m] A^T[U_a][l],   Phi_U += Delta.
// A persistent grid of 256-thread CTAs walks the (walker, det) pairs; CTA b
// keeps its scratch (Tw: [Umax][n] in Tu, B then C: [Umax][n] in Bw) in slot
// b.  Flagged pairs are refactorised by mcmc_repair_kernel instead.
template <typename T>
__global__ void __launch_bounds__(256) mcmc_woodbury_kernel(
    int Wn, int n, int D, int Umax, const int32_t* __restrict__ acc, const int32_t* __restrict__ flag,
    const int32_t* __restrict__ Ul, const int32_t* __restrict__ Uc, const T* __restrict__ Dl,
    const double* __restrict__ Mlu, const int32_t* __restrict__ Mpiv, T* __restrict__ AT, T* __restrict__ Phi,
    T* __restrict__ Tu, T* __restrict__ Bw) {
  // the product tiles and the LU of M are never live together: one buffer
  __shared__ double su[kLemmaSmem * (kLemmaSmem + 1)];
  __shared__ int spv[kLemmaSmem];
  T* sm = reinterpret_cast<T*>(su);
  double* sL = su;
  T* Tw = Tu + (int64_t)blockIdx.x * Umax * n;
  T* Bm = Bw + (int64_t)blockIdx.x * Umax * n;
  for (int64_t md = blockIdx.x; md < (int64_t)Wn * D; md += gridDim.x) {
    const int w = (int)(md / D);
    if (!acc[w]) continue;
    const int u = Uc[w];
    const int32_t* U = Ul + (int64_t)w * Umax;
    T* A = AT + md * n * n;
    const T* Dw = Dl + md * Umax * n;
    T* P = Phi + md * n * n;
    if (flag[md]) {   // refactorised by mcmc_repair_kernel: only Phi moves here
      for (int e = threadIdx.x; e < u * n; e += blockDim.x) P[(int64_t)U[e / n] * n + e % n] += Dw[e];
      continue;
    }
    for (int e = threadIdx.x; e < u * n; e += blockDim.x) Tw[e] = A[(int64_t)U[e / n] * n + e % n];
    // B[a][m] = sum_l Delta[a][l] A^T[m][l]   (starts and ends with a barrier)
    cta_gemm_nt<T>(u, n, n, Dw, n, A, n, nullptr, Bm, n, T(1), false, sm);
    const bool in_smem = u <= kLemmaSmem;
    const double* Mg = Mlu + md * Umax * Umax;
    const int32_t* pvg = Mpiv + md * Umax;
    if (in_smem) {
      for (int e = threadIdx.x; e < u * u; e += blockDim.x)
        sL[(e / u) * (kLemmaSmem + 1) + e % u] = Mg[(e / u) * Umax + e % u];
      for (int e = threadIdx.x; e < u; e += blockDim.x) spv[e] = pvg[e];
    }
    __syncthreads();
    const double* L = in_smem ? sL : Mg;
    const int ldl = in_smem ? kLemmaSmem + 1 : Umax;
    const int32_t* pv = in_smem ? spv : pvg;
    // C = M^-1 B: one column per thread, row swaps then unit-lower and upper
    // solves in float64; the column lives in local memory
    for (int m = threadIdx.x; m < n; m += blockDim.x) {
      double x[kLemmaSmem];
      if (in_smem) {
        for (int c = 0; c < u; ++c) x[c] = (double)Bm[(int64_t)c * n + m];
        for (int c = 0; c < u; ++c) {
          const int p = pv[c];
          if (p != c) { const double t = x[c]; x[c] = x[p]; x[p] = t; }
        }
        for (int c = 0; c < u; ++c) {
          double s = x[c];
          for (int q = 0; q < c; ++q) s -= L[c * ldl + q] * x[q];
          x[c] = s;
        }
        for (int c = u - 1; c >= 0; --c) {
          double s = x[c];
          for (int q = c + 1; q < u; ++q) s -= L[c * ldl + q] * x[q];
          x[c] = s / L[c * ldl + c];
        }
        for (int c = 0; c < u; ++c) Bm[(int64_t)c * n + m] = (T)x[c];
      } else {   // large U: the same solve on the column in the scratch
        for (int c = 0; c < u; ++c) {
          const int p = pv[c];
          if (p != c) {
            const T t = Bm[(int64_t)c * n + m];
            Bm[(int64_t)c * n + m] = Bm[(int64_t)p * n + m];
            Bm[(int64_t)p * n + m] = t;
          }
        }
        for (int c = 0; c < u; ++c) {
          double s = (double)Bm[(int64_t)c * n + m];
          for (int q = 0; q < c; ++q) s -= L[c * ldl + q] * (double)Bm[(int64_t)q * n + m];
          Bm[(int64_t)c * n + m] = (T)s;
        }
        for (int c = u - 1; c >= 0; --c) {
          double s = (double)Bm[(int64_t)c * n + m];
          for (int q = c + 1; q < u; ++q) s -= L[c * ldl + q] * (double)Bm[(int64_t)q * n + m];
          Bm[(int64_t)c * n + m] = (T)(s / L[c * ldl + c]);
        }
      }
    }
    __syncthreads();
    // A^T[m][l] -= sum_a C[a][m] Tw[a][l]  (ends with a barrier: the slot is free)
    cta_gemm_tn<T>(n, n, u, Bm, n, Tw, n, A, n, T(-1), true, sm);
    for (int e = threadIdx.x; e < u * n; e += blockDim.x) P[(int64_t)U[e / n] * n + e % n] += Dw[e];
  }
}

// ---------------------------------------------------------------------------
// Refresh helpers
// ---------------------------------------------------------------------------

template <typename S, typename T>
__global__ void convert_kernel(int64_t count, const S* __restrict__ src, T* __restrict__ dst) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (T)src[e];
}

// A = Phi^-1 from the LU factors (P Phi = L U, unit L, stored in LT) of one
// n x n matrix, in arithmetic CT, written transposed (AT[k][l] = A[l][k]) in
// AT's type, by one CTA of 256 threads.  Columns go in panels of 32: column
// j of A solves L U x = e_{pinv[j]}; the panel X[n][33] sits in shared
// memory (sm), warp g owns columns 4g .. 4g+3 with 8 lanes per column
// splitting each dot product, so no block barrier is needed inside a panel.
template <typename LT, typename CT, typename AT>
__device__ void inverse_panel_block(int n, const LT* __restrict__ A, const int32_t* __restrict__ pv,
                                    AT* __restrict__ out, unsigned char* sm) {
  CT* X = reinterpret_cast<CT*>(sm);                         // [n][33]
  int* pinv = reinterpret_cast<int*>(X + (int64_t)n * 33);   // [n]
  int* perm = pinv + n;                                      // [n]
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int k = 0; k < n; ++k) {
      const int t = perm[k];
      perm[k] = perm[pv[k]];
      perm[pv[k]] = t;
    }
    for (int i = 0; i < n; ++i) pinv[perm[i]] = i;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int cl = 4 * wp + (lane >> 3);   // column of the panel
  const int sub = lane & 7;
  for (int j0 = 0; j0 < n; j0 += 32) {
    const int j = j0 + cl;
    const int p = j < n ? pinv[j] : -1;
    for (int i = 0; i < n; ++i) {   // forward: unit lower
      CT s = CT(0);
      for (int q = sub; q < i; q += 8) s += (CT)A[(int64_t)i * n + q] * X[q * 33 + cl];
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      s += __shfl_xor_sync(0xffffffffu, s, 4);
      if (sub == 0) X[i * 33 + cl] = ((i == p) ? CT(1) : CT(0)) - s;
      __syncwarp();
    }
    for (int i = n - 1; i >= 0; --i) {   // backward: upper
      CT s = CT(0);
      for (int q = i + 1 + sub; q < n; q += 8) s += (CT)A[(int64_t)i * n + q] * X[q * 33 + cl];
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      s += __shfl_xor_sync(0xffffffffu, s, 4);
      if (sub == 0) X[i * 33 + cl] = (X[i * 33 + cl] - s) / (CT)A[(int64_t)i * n + i];
      __syncwarp();
    }
    __syncthreads();
    // out[j][l] = A[l][j] = X[l][j - j0]: row j of the output is column j of A
    for (int e = threadIdx.x; e < 32 * n; e += blockDim.x) {
      const int jj = e / n, l = e % n;
      if (j0 + jj < n) out[(int64_t)(j0 + jj) * n + l] = (AT)X[l * 33 + jj];
    }
    __syncthreads();
  }
}

// The inverse of matrices [m0, m0 + gridDim.x) of a batch, one CTA each.
template <typename LT, typename CT, typename AT>
__global__ void __launch_bounds__(256) inverse_panel_kernel(int n, int64_t m0, const LT* __restrict__ LU,
                                                            const int32_t* __restrict__ piv,
                                                            AT* __restrict__ Ainv) {
  extern __shared__ unsigned char ip_smem[];
  const int64_t mat = m0 + blockIdx.x;
  inverse_panel_block<LT, CT, AT>(n, LU + mat * n * n, piv + mat * n, Ainv + mat * n * n, ip_smem);
}

// A^T of the batched refactorisations: matrix f of the batch into the slot
// rlist[f] of A^T (zero for a singular matrix); CTAs beyond the count leave.
template <typename LT, typename T>
__global__ void __launch_bounds__(256) mcmc_repair_inverse_kernel(int n, const int* __restrict__ count, int cap,
                                                                  const int32_t* __restrict__ rlist,
                                                                  const LT* __restrict__ batch,
                                                                  const int32_t* __restrict__ piv,
                                                                  const double* __restrict__ bsg,
                                                                  T* __restrict__ AT) {
  extern __shared__ unsigned char ri_smem[];
  const int c = *count < cap ? *count : cap;
  if ((int)blockIdx.x >= c) return;
  T* A = AT + (int64_t)rlist[blockIdx.x] * n * n;
  if (bsg[blockIdx.x] == 0.0) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) A[e] = T(0);
    return;
  }
  inverse_panel_block<LT, LT, T>(n, batch + (int64_t)blockIdx.x * n * n, piv + (int64_t)blockIdx.x * n, A, ri_smem);
}

inline size_t inverse_panel_smem(int n, size_t lsz) { return (size_t)n * 33 * lsz + 2 * (size_t)n * sizeof(int); }


// Right-looking LU with partial pivoting of one n x n matrix in place, by one
// CTA (pivot search by warp 0).  Returns log|det| and the sign through
// shared memory (sign 0 and -inf for an exactly zero pivot).
template <typename LT>
__device__ void lu_block(int n, LT* __restrict__ A, int32_t* __restrict__ pv, double* s_la, double* s_sg) {
  __shared__ int s_p;
  double la = 0.0;
  int neg = 0;
  bool zero = false;
  for (int c = 0; c < n; ++c) {
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bq = c;
      for (int q = c + threadIdx.x; q < n; q += 32) {
        const double v = fabs((double)A[(int64_t)q * n + c]);
        if (v > best) { best = v; bq = q; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oq = __shfl_xor_sync(0xffffffffu, bq, o);
        if (ob > best || (ob == best && oq < bq)) { best = ob; bq = oq; }
      }
      if (threadIdx.x == 0) { s_p = bq; pv[c] = bq; }
    }
    __syncthreads();
    const int pq = s_p;
    if (pq != c) {
      for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const LT t = A[(int64_t)c * n + q];
        A[(int64_t)c * n + q] = A[(int64_t)pq * n + q];
        A[(int64_t)pq * n + q] = t;
      }
      neg ^= 1;
    }
    __syncthreads();
    const LT piv = A[(int64_t)c * n + c];
    if (piv == LT(0)) {
      zero = true;
    } else {
      la += log(fabs((double)piv));
      if (piv < LT(0)) neg ^= 1;
      const int wdt = n - c - 1;
      for (int e = threadIdx.x; e < wdt * wdt; e += blockDim.x) {
        const int q = c + 1 + e / wdt, cc = c + 1 + e % wdt;
        A[(int64_t)q * n + cc] -= (A[(int64_t)q * n + c] / piv) * A[(int64_t)c * n + cc];
      }
      __syncthreads();
      for (int q = c + 1 + threadIdx.x; q < n; q += blockDim.x) A[(int64_t)q * n + c] /= piv;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *s_la = zero ? -INFINITY : la;
    *s_sg = zero ? 0.0 : (neg ? -1.0 : 1.0);
  }
  __syncthreads();
}

// Exact ratios for the (walker, det) pairs whose determinant-lemma ratio is
// beyond e^{+-kExactLogRatio} or not finite: Phi' = Phi with the rows U
// replaced (Phi_U + Delta), its float64 LU, lrat = log|det Phi'| - ldabs and
// srat = sign(det Phi') * lsign.  xflag[pair] = 1 marks them for a
// refactorisation if the move is accepted.  A persistent grid; CTA b uses
// slot b of the float64 scratch; dynamic shared memory n ints.
//
// Also recomputed exactly (and refactorised if accepted): every determinant
// whose Woodbury-carried inverse cannot be trusted to the tolerance ktol,
// i.e. kappa_d u w_d > ktol, with kappa_d the Frobenius condition estimate of
// the last factorisation (kap), u the unit roundoff of the state (kunit) and
// w_d = |det Phi_d| / max_q |det Phi_q| the determinant's weight in the
// walker's sum.  A float32 inverse of a matrix with kappa ~ 1e6 carries
// relative errors of order kappa u ~ 0.06, which a run of moves accumulates
// into the carried log-determinant; weighted by w_d that is the error it
// brings into log|Psi| and the acceptance ratio.  ktol < 0 turns the test off.
template <typename T, typename LT>
__global__ void __launch_bounds__(256) mcmc_exact_ratio_kernel(
    int Wn, int n, int D, int Umax, const int32_t* __restrict__ Ul, const int32_t* __restrict__ Uc,
    const T* __restrict__ Phi, const T* __restrict__ Dl, const double* __restrict__ ldabs,
    const double* __restrict__ lsign, double* __restrict__ lrat, double* __restrict__ srat,
    int32_t* __restrict__ xflag, LT* __restrict__ scratch, int32_t* __restrict__ spiv,
    const float* __restrict__ kap, double kunit, double ktol, int* __restrict__ xcount,
    int32_t* __restrict__ xlist, int xcap, unsigned long long* __restrict__ nexact) {
  extern __shared__ int xr_slot[];   // [n]: slot of row i in U, or -1
  __shared__ double s_la, s_sg;
  __shared__ int s_slot;
  LT* L = scratch + (int64_t)blockIdx.x * n * n;
  int32_t* pv = spiv + (int64_t)blockIdx.x * n;
  for (int64_t md = blockIdx.x; md < (int64_t)Wn * D; md += gridDim.x) {
    const double lr = lrat[md];
    const bool range = !(fabs(lr) <= kExactLogRatio) && lsign[md] != 0.0;
    bool cond = false;
    if (!range && ktol >= 0.0 && lsign[md] != 0.0) {
      const int64_t w0 = (md / D) * D;
      double lmax = -INFINITY;
      for (int q = 0; q < D; ++q)
        if (lsign[w0 + q] != 0.0 && ldabs[w0 + q] > lmax) lmax = ldabs[w0 + q];
      cond = (double)kap[md] * kunit * exp(ldabs[md] - lmax) > ktol;
    }
    // 1: ratio out of range (the inverse is refactorised if accepted);
    // 2: conditioning (exact ratio; the Woodbury update keeps A until the
    // next refresh, the ratio does not use it while the test holds)
    if (threadIdx.x == 0) xflag[md] = range ? 1 : (cond ? 2 : 0);
    if (!range && !cond) continue;
    if (threadIdx.x == 0 && nexact) atomicAdd(nexact, 1ull);
    if (cond && xlist) {   // deferred to the batched float64 LU when it has room
      __syncthreads();
      if (threadIdx.x == 0) {
        s_slot = atomicAdd(xcount, 1);
        if (s_slot < xcap) xlist[s_slot] = (int32_t)md;
      }
      __syncthreads();
      if (s_slot < xcap) continue;
    }
    const int w = (int)(md / D);
    const int u = Uc[w];
    for (int i = threadIdx.x; i < n; i += blockDim.x) xr_slot[i] = -1;
    __syncthreads();
    for (int a = threadIdx.x; a < u; a += blockDim.x) xr_slot[Ul[(int64_t)w * Umax + a]] = a;
    __syncthreads();
    const T* P = Phi + md * n * n;
    const T* Dw = Dl + md * Umax * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e / n, a = xr_slot[i];
      L[e] = (LT)P[e] + (a >= 0 ? (LT)Dw[(int64_t)a * n + e % n] : LT(0));
    }
    __syncthreads();
    lu_block<LT>(n, L, pv, &s_la, &s_sg);
    if (threadIdx.x == 0) {
      lrat[md] = s_la - ldabs[md];
      srat[md] = s_sg * lsign[md];
    }
    __syncthreads();
  }
}

// Phi' = Phi with the rows U replaced, in float64, for the pairs deferred to
// the batched LU (xlist[0 .. *count)), one CTA each; CTAs beyond the count
// leave.  Dynamic shared memory n ints.
template <typename T, typename LT>
__global__ void __launch_bounds__(256) mcmc_exact_build_kernel(int n, int D, int Umax, const int* __restrict__ count,
                                                               const int32_t* __restrict__ xlist,
                                                               const int32_t* __restrict__ Ul,
                                                               const int32_t* __restrict__ Uc,
                                                               const T* __restrict__ Phi, const T* __restrict__ Dl,
                                                               LT* __restrict__ batch) {
  extern __shared__ int xb_slot[];
  if ((int)blockIdx.x >= *count) return;
  const int64_t md = xlist[blockIdx.x];
  const int w = (int)(md / D);
  const int u = Uc[w];
  for (int i = threadIdx.x; i < n; i += blockDim.x) xb_slot[i] = -1;
  __syncthreads();
  for (int a = threadIdx.x; a < u; a += blockDim.x) xb_slot[Ul[(int64_t)w * Umax + a]] = a;
  __syncthreads();
  const T* P = Phi + md * n * n;
  const T* Dw = Dl + md * Umax * n;
  LT* L = batch + (int64_t)blockIdx.x * n * n;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int a = xb_slot[e / n];
    L[e] = (LT)P[e] + (a >= 0 ? (LT)Dw[(int64_t)a * n + e % n] : LT(0));
  }
}

// lrat = log|det Phi'| - ldabs, srat = sign(det Phi') lsign for the batch.
static __global__ void mcmc_exact_scatter_kernel(const int* __restrict__ count, int cap,
                                                 const int32_t* __restrict__ xlist, const double* __restrict__ blab,
                                                 const double* __restrict__ bsg, const double* __restrict__ ldabs,
                                                 const double* __restrict__ lsign, double* __restrict__ lrat,
                                                 double* __restrict__ srat) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = *count < cap ? *count : cap;
  if (f >= c) return;
  const int64_t md = xlist[f];
  lrat[md] = blab[f] - ldabs[md];
  srat[md] = bsg[f] * lsign[md];
}

// Batched refactorisation of the determinants in rlist[0 .. *count) (flag
// 2): a float64 copy of the cached Phi (already updated by the move) for
// lu_kernel, then log|det|, sign and the reference log|det| of the new
// factors, then A^T from them (zero for a singular matrix).  CTAs beyond the
// count leave.
template <typename T, typename LT>
__global__ void __launch_bounds__(256) mcmc_repair_build_kernel(int n, const int* __restrict__ count,
                                                                const int32_t* __restrict__ rlist,
                                                                const T* __restrict__ Phi, LT* __restrict__ batch) {
  if ((int)blockIdx.x >= *count) return;
  const T* P = Phi + (int64_t)rlist[blockIdx.x] * n * n;
  LT* L = batch + (int64_t)blockIdx.x * n * n;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) L[e] = (LT)P[e];
}

static __global__ void mcmc_repair_scatter_kernel(const int* __restrict__ count, int cap,
                                                  const int32_t* __restrict__ rlist, const double* __restrict__ blab,
                                                  const double* __restrict__ bsg, double* __restrict__ ldabs,
                                                  double* __restrict__ lsign, double* __restrict__ lref) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = *count < cap ? *count : cap;
  if (f >= c) return;
  const int64_t md = rlist[f];
  ldabs[md] = blab[f];
  lsign[md] = bsg[f];
  lref[md] = blab[f];
}

// Refactorisation of the flagged (walker, det) pairs of accepted walkers
// from the cached Phi (already updated by the move): log|det|, sign and A^T.
// A persistent grid; CTA b uses slot b of the float64 scratch (n x n matrix,
// n pivots) and dynamic shared memory for the inverse panel.
template <typename T, typename LT>
__global__ void __launch_bounds__(256) mcmc_repair_kernel(int Wn, int n, int D, const int32_t* __restrict__ acc,
                                                          const int32_t* __restrict__ flag,
                                                          const T* __restrict__ Phi, T* __restrict__ AT,
                                                          double* __restrict__ ldabs, double* __restrict__ lsign,
                                                          double* __restrict__ lref, LT* __restrict__ scratch,
                                                          int32_t* __restrict__ spiv) {
  extern __shared__ unsigned char rp_smem[];
  __shared__ double s_la, s_sg;
  LT* L = scratch + (int64_t)blockIdx.x * n * n;
  int32_t* pv = spiv + (int64_t)blockIdx.x * n;
  for (int64_t md = blockIdx.x; md < (int64_t)Wn * D; md += gridDim.x) {
    if (!acc[md / D] || flag[md] != 1) continue;
    const T* P = Phi + md * n * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) L[e] = (LT)P[e];
    __syncthreads();
    lu_block<LT>(n, L, pv, &s_la, &s_sg);
    if (threadIdx.x == 0) {
      ldabs[md] = s_la;
      lsign[md] = s_sg;
      lref[md] = s_la;
    }
    T* A = AT + md * n * n;
    if (s_sg == 0.0) {
      // singular: the determinant stays dead until the next rebuild
      for (int e = threadIdx.x; e < n * n; e += blockDim.x) A[e] = T(0);
      __syncthreads();
      continue;
    }
    inverse_panel_block<LT, LT, T>(n, L, pv, A, rp_smem);
  }
}


// Frobenius condition estimate kappa_F = ||Phi||_F ||Phi^-1||_F (between
// kappa_2 and n kappa_2) of every (walker, det) after a factorisation; 0 for
// a singular determinant (its A^T is zero).  One CTA per matrix.
template <typename T>
__global__ void __launch_bounds__(256) mcmc_kappa_kernel(int n, const T* __restrict__ Phi, const T* __restrict__ AT,
                                                         float* __restrict__ kap) {
  __shared__ double red[2][8];
  const int64_t md = blockIdx.x;
  const T* P = Phi + md * n * n;
  const T* A = AT + md * n * n;
  double sp = 0.0, sa = 0.0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const double x = (double)P[e], y = (double)A[e];
    sp += x * x;
    sa += y * y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sp += __shfl_xor_sync(0xffffffffu, sp, o);
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sp;
    red[1][threadIdx.x >> 5] = sa;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a += red[0][q]; b += red[1][q]; }
    kap[md] = (float)sqrt(a * b);
  }
}

// drift = max_w |lp_inc - lp_fresh| (the bits of a non-negative double order
// like the values), wdrift[w] = the walker's largest drift so far; then
// lp_inc = lp_fresh.
static __global__ void mcmc_drift_kernel(int W, double* __restrict__ lp_inc, const double* __restrict__ lp_fresh,
                                         double* __restrict__ wdrift, unsigned long long* __restrict__ drift_bits,
                                         int measure) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  if (measure) {
    const double a = lp_inc[w], b = lp_fresh[w];
    if (isfinite(a) && isfinite(b)) {
      const double dr = fabs(a - b);
      atomicMax(drift_bits, (unsigned long long)__double_as_longlong(dr));
      if (dr > wdrift[w]) wdrift[w] = dr;
    }
  } else {
    wdrift[w] = 0.0;
  }
  lp_inc[w] = lp_fresh[w];
}

}  // namespace fire

// Two-electron swap ratios for the S+ operator (Supplementary "Low-rank
// updates in S+ operator": R_beta = 1 - sum_alpha Psi(pi_{alpha beta} r)/Psi(r),
// pi swapping the positions of the spin-up electron alpha and the spin-down
// electron beta; Methods "Low-rank wave function updates": only the
// embeddings within c of either electron change).
//
// A swap moves alpha to r_beta and beta to r_alpha, each keeping its spin.
// h^0 and its message projections depend on the position alone, so the new
// h^0 of alpha is the cached h^0 of beta and vice versa; the envelope rows
// of both are recomputed with their own spin's weights.  The update set is
// {alpha, beta} and every electron within c of r_alpha or r_beta; the
// orbital rows of the update set, the MLP-Jastrow rows and the attention
// registers are recomputed as for a single-electron move, and the
// determinant ratios come from the same |U| x |U| determinant lemma.
// (Included by pipeline.cuh after mcmc.cuh.)
#pragma once

#include <stdint.h>

#include "../../include/fire.h"

namespace fire {

// rk = r_beta (alpha's new position), rk2 = r_alpha (beta's), and the update
// set.  One warp per walker.
static __global__ void swap_propose_kernel(int n, int n_up, int a, int b, const double* __restrict__ r, double c2,
                                           int Umax, double* __restrict__ rk, double* __restrict__ rk2,
                                           int32_t* __restrict__ Ul, int32_t* __restrict__ Uc,
                                           int32_t* __restrict__ Ucu, DevStatus* st) {
  const int w = blockIdx.x;
  const int lane = threadIdx.x;
  const double* rw = r + (int64_t)w * n * 3;
  if (lane < 3) {
    rk[(int64_t)w * 3 + lane] = rw[3 * b + lane];
    rk2[(int64_t)w * 3 + lane] = rw[3 * a + lane];
  }
  // members: a, and every j within c of r_a or of r_b (b among them)
  update_set(w, lane, n, n_up, a, rw, rw + 3 * b, c2, Umax, Ul, Uc, Ucu, st, true);
}

// h^1 of every member i of U after the swap (value only).  For i = a or b
// every term changes: the neighbour list at the new position is rebuilt with
// the swapped positions and h^0 / projections (position-only) taken from the
// other electron's block.  For any other i the terms of the pairs (i, a) and
// (i, b) change: h^1_i - old (i, a) - old (i, b) + new (i, a) + new (i, b),
// the new terms at the swapped positions with the swapped projections and
// the spin channel of the pair unchanged.  One CTA per (walker, slot),
// blockDim == d; dynamic shared memory n ints.
template <typename T, typename W>
__global__ void swap_msg_kernel(int Wn, int n, int n_up, int d, int a, int b, int Umax, const double* __restrict__ r,
                                double cut, Params<W> p, const int32_t* __restrict__ Ul, const int32_t* __restrict__ Uc,
                                const int32_t* __restrict__ Urow, const T* __restrict__ H0, const T* __restrict__ PQ,
                                const T* __restrict__ H1, T* __restrict__ X, T* __restrict__ H1n) {
  constexpr int H = kEdgeHidden, G = kGauss;
  __shared__ FL3<T> feat[H + G + 4];
  extern __shared__ int sw_nbr[];
  __shared__ int s_cnt[2];
  const int w = blockIdx.x / Umax, u = blockIdx.x % Umax;
  if (u >= Uc[w]) return;
  const int i = Ul[(int64_t)w * Umax + u];
  const int c = threadIdx.x;
  const int64_t ld4 = 4 * (int64_t)d;
  const double* rw = r + (int64_t)w * n * 3;
  T w2[H], we[G], wc[2][4], bb[2];
#pragma unroll
  for (int h = 0; h < H; ++h) w2[h] = T(p.ee_w2[h * d + c]);
#pragma unroll
  for (int g = 0; g < G; ++g) we[g] = T(p.ee_wenv[g * d + c]);
#pragma unroll
  for (int al = 0; al < 2; ++al) {
    bb[al] = T(p.msg_b[al * d + c]);
#pragma unroll
    for (int q = 0; q < 4; ++q) wc[al][q] = T(p.msg_w[((int64_t)al * (2 * d + 4) + 2 * d + q) * d + c]);
  }
  auto term = [&](const double ddv[3], const T* Pi, const T* Qj, int al) -> T {
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
    for (int q = 0; q < 4; ++q) eb += feat[H + G + q].v * wc[al][q];
    const T z = Pi[(int64_t)al * d + c] + Qj[2 * (int64_t)d + (int64_t)al * d + c] + eb + bb[al];
    T f, f1, f2;
    silu3<T>(z, f, f1, f2);
    return (gv * ev) * f;
  };
  // positions and position-dependent blocks after the swap
  auto src = [&](int j) { return j == a ? b : (j == b ? a : j); };
  auto pos = [&](int j, int t) -> double { return rw[3 * src(j) + t]; };
  T acc;
  if (i == a || i == b) {
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
          if (in) sw_nbr[cntN + __popc(m & ((1u << lane) - 1u))] = j;
          cntN += __popc(m);
        }
        if (lane == 0) s_cnt[pass] = cntN;
      }
    }
    __syncthreads();
    const int cpar = s_cnt[0], ctot = s_cnt[1];
    const int64_t bi = block_index(w, src(i), Wn, n, n_up);
    const T* Pi = PQ + bi * ld4;
    acc = H0[bi * d + c];
    for (int s = 0; s < ctot; ++s) {
      const int j = sw_nbr[s];
      const double ddv[3] = {pos(i, 0) - pos(j, 0), pos(i, 1) - pos(j, 1), pos(i, 2) - pos(j, 2)};
      acc += term(ddv, Pi, PQ + (int64_t)block_index(w, src(j), Wn, n, n_up) * ld4, s < cpar ? 0 : 1);
    }
  } else {
    const int64_t bi = block_index(w, i, Wn, n, n_up);
    const T* Pi = PQ + bi * ld4;
    acc = H1[bi * d + c];
    for (int mv = 0; mv < 2; ++mv) {
      const int k = mv == 0 ? a : b;
      const int al = ((i < n_up) == (k < n_up)) ? 0 : 1;
      for (int side = 0; side < 2; ++side) {   // 0: remove the old (i, k) term, 1: add the new one
        const int sk = side == 0 ? k : src(k);  // the position and blocks the pair uses
        const double ddv[3] = {rw[3 * i] - rw[3 * sk], rw[3 * i + 1] - rw[3 * sk + 1], rw[3 * i + 2] - rw[3 * sk + 2]};
        if (!(ddv[0] * ddv[0] + ddv[1] * ddv[1] + ddv[2] * ddv[2] <= cut * cut)) continue;
        const T t = term(ddv, Pi, PQ + (int64_t)block_index(w, sk, Wn, n, n_up) * ld4, al);
        acc += side == 0 ? -t : t;
      }
    }
  }
  const int64_t row = Urow[(int64_t)w * Umax + u];
  X[row * d + c] = acc;
  H1n[row * d + c] = acc;
}

// ratios[w][a] = Psi(swapped) / Psi for the walkers (signed).
template <typename T>
__global__ void swap_accum_kernel(int Wn, int n, int n_up, int D, int a, int b, int Umax, uint32_t flags,
                                  const double* __restrict__ r, const double* __restrict__ rk,
                                  const double* __restrict__ rk2, const int32_t* __restrict__ Ul,
                                  const int32_t* __restrict__ Uc, const int32_t* __restrict__ Urow, McmcJastrow jp,
                                  const T* __restrict__ F1, const T* __restrict__ F2, const T* __restrict__ F1n,
                                  const T* __restrict__ F2n, const T* __restrict__ G1, const T* __restrict__ G2,
                                  const T* __restrict__ G1n, const T* __restrict__ G2n,
                                  const double* __restrict__ ldabs, const double* __restrict__ lsign,
                                  const double* __restrict__ lrat, const double* __restrict__ srat,
                                  double* __restrict__ ratios) {
  const int w = blockIdx.x;
  const WalkerRatio wr = walker_ratio<T>(w, threadIdx.x, Wn, n, n_up, D, a, Umax, flags, r + (int64_t)w * n * 3,
                                         rk + (int64_t)w * 3, b, rk2 + (int64_t)w * 3, Ul, Uc, Urow, jp, F1, F2, F1n,
                                         F2n, G1, G2, G1n, G2n, ldabs, lsign, lrat, srat);
  if (threadIdx.x == 0) ratios[(int64_t)w * n_up + a] = wr.sign * exp(wr.logr);
}

// r_beta[w] = 1 - sum_a ratios[w][a] (in index order).
static __global__ void swap_sum_kernel(int Wn, int n_up, const double* __restrict__ ratios,
                                       double* __restrict__ rb) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= Wn) return;
  double sm = 0.0;
  for (int a = 0; a < n_up; ++a) sm += ratios[(int64_t)w * n_up + a];
  rb[w] = 1.0 - sm;
}

}  // namespace fire

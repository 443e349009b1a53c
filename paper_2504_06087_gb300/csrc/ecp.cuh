// Non-local pseudopotential energy by single-electron wave-function ratios
// (Methods, "Low-rank wave function updates": the pseudopotential needs
// Psi(r')/Psi(r) for configurations differing in one electron, computed with
// the same local recompute and determinant lemma as a Metropolis move;
// Supplementary "Effective core potential": a per-species number of
// quadrature points; Methods "Energy extrapolation": n_el N_quad updates).
//
//   V_nl = sum_k sum_l v_l(|r_k - R_m|) (2l + 1) sum_q w_q P_l(rhat_k . n_q) Psi(.. r'_kq ..) / Psi,
//   r'_kq = R_m + |r_k - R_m| n_q,   v_l(x) = sum_j c_lj x^p_lj exp(-a_lj x^2),
//
// m the pseudopotential nucleus within r_cut of electron k (at most one),
// n_q the vertices of a tetrahedron, octahedron or icosahedron (4, 6, 12
// points, weights 1/N_quad) under one random rotation per (walker, electron):
// a unit quaternion from three Philox uniforms (Shoemake's construction).
#pragma once

#include <math.h>
#include <stdint.h>

#include "../../include/fire.h"
#include "philox.cuh"
// (included by pipeline.cuh after mcmc.cuh: update_set, walker_ratio)

namespace fire {

// quadrature vertices (unnormalised; every vertex of one rule has the same norm)
__device__ __constant__ double kQuadTet[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
__device__ __constant__ double kQuadOct[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
#define FIRE_GR 1.6180339887498948482
__device__ __constant__ double kQuadIco[12][3] = {
    {0, 1, FIRE_GR},   {1, FIRE_GR, 0},   {FIRE_GR, 0, 1},   {0, 1, -FIRE_GR},   {1, -FIRE_GR, 0},   {-FIRE_GR, 0, 1},
    {0, -1, FIRE_GR},  {-1, FIRE_GR, 0},  {FIRE_GR, 0, -1},  {0, -1, -FIRE_GR},  {-1, -FIRE_GR, 0},  {-FIRE_GR, 0, -1}};
#undef FIRE_GR

// Unit direction q of an n_quad-point rule.
__device__ inline void quad_dir(int n_quad, int q, double* d) {
  const double* v = n_quad == 4 ? kQuadTet[q] : (n_quad == 6 ? kQuadOct[q] : kQuadIco[q]);
  const double nrm = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  for (int t = 0; t < 3; ++t) d[t] = v[t] / nrm;
}

// Rotation of electron k in walker w: quaternion (x, y, z, w) =
// (sqrt(1-u1) sin 2pi u2, sqrt(1-u1) cos 2pi u2, sqrt(u1) sin 2pi u3,
// sqrt(u1) cos 2pi u3), u1..u3 from Philox counter (k, 0, walker, 3).
__device__ inline void ecp_rotation(uint64_t seed, uint32_t walker, uint32_t k, double R[3][3]) {
  const Philox4 c = philox4x32_10(k, 0u, walker, 3u, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double u1 = u01(c.v[0]), u2 = u01(c.v[1]), u3 = u01(c.v[2]);
  const double two_pi = 6.283185307179586476925286766559;
  const double x = sqrt(1.0 - u1) * sin(two_pi * u2), y = sqrt(1.0 - u1) * cos(two_pi * u2);
  const double z = sqrt(u1) * sin(two_pi * u3), w = sqrt(u1) * cos(two_pi * u3);
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

__device__ inline double legendre_p(int l, double x) { return l == 0 ? 1.0 : (l == 1 ? x : 1.5 * x * x - 0.5); }

// Virtual move q of electron k: for walkers whose electron k lies within the
// r_cut of a pseudopotential nucleus m with q < N_quad(m), rk = R_m + |r_k -
// R_m| n_q, pref[w] = sum_l v_l(|r_k - R_m|) (2l + 1) w_q P_l(rhat . n_q) and
// the update set as for a Metropolis move; every other walker keeps r_k,
// gets pref = 0 and an empty update set.  One warp per walker.
static __global__ void ecp_propose_kernel(int n, int n_up, int k, int q, const double* __restrict__ r,
                                          const double* __restrict__ nuc_pos, int N,
                                          const fire_ecp_t* __restrict__ ecp, uint64_t seed, double c2, int Umax,
                                          double* __restrict__ rk, double* __restrict__ pref,
                                          int32_t* __restrict__ Ul, int32_t* __restrict__ Uc,
                                          int32_t* __restrict__ Ucu, DevStatus* st) {
  const int w = blockIdx.x;
  const int lane = threadIdx.x;
  const double* rw = r + (int64_t)w * n * 3;
  __shared__ double rn[3];
  __shared__ int s_active;
  if (lane == 0) {
    int m = -1;
    double rel[3] = {0, 0, 0}, rad = 0.0;
    for (int mm = 0; mm < N && m < 0; ++mm) {
      if (ecp[mm].n_quad <= 0) continue;
      double d2 = 0.0;
      for (int t = 0; t < 3; ++t) {
        rel[t] = rw[3 * k + t] - nuc_pos[3 * mm + t];
        d2 += rel[t] * rel[t];
      }
      if (sqrt(d2) < ecp[mm].r_cut) { m = mm; rad = sqrt(d2); }
    }
    double p = 0.0;
    if (m >= 0 && q < ecp[m].n_quad && rad > 0.0) {
      double R[3][3], d0[3], d[3];
      ecp_rotation(seed, (uint32_t)w, (uint32_t)k, R);
      quad_dir(ecp[m].n_quad, q, d0);
      double cs = 0.0;
      for (int t = 0; t < 3; ++t) {
        d[t] = R[t][0] * d0[0] + R[t][1] * d0[1] + R[t][2] * d0[2];
        rn[t] = nuc_pos[3 * m + t] + rad * d[t];
        cs += d[t] * rel[t] / rad;
      }
      const fire_ecp_t& e = ecp[m];
      for (int l = 0; l < e.n_channels; ++l) {
        double v = 0.0;
        for (int j = 0; j < e.n_terms[l]; ++j) v += e.coef[l][j] * pow(rad, e.power[l][j]) * exp(-e.alpha[l][j] * rad * rad);
        p += v * (2 * l + 1) * legendre_p(l, cs) / (double)e.n_quad;
      }
      s_active = 1;
    } else {
      for (int t = 0; t < 3; ++t) rn[t] = rw[3 * k + t];
      s_active = 0;
    }
    for (int t = 0; t < 3; ++t) rk[(int64_t)w * 3 + t] = rn[t];
    pref[w] = p;
  }
  __syncwarp();
  update_set(w, lane, n, n_up, k, rw, rn, c2, Umax, Ul, Uc, Ucu, st, s_active != 0);
}

// v_nl[w] += pref[w] Psi(r')/Psi(r) for the walkers with a virtual move.
template <typename T>
__global__ void ecp_accum_kernel(int Wn, int n, int n_up, int D, int k, int Umax, uint32_t flags,
                                 const double* __restrict__ r, const double* __restrict__ rk,
                                 const double* __restrict__ pref, const int32_t* __restrict__ Ul,
                                 const int32_t* __restrict__ Uc, const int32_t* __restrict__ Urow, McmcJastrow jp,
                                 const T* __restrict__ F1, const T* __restrict__ F2, const T* __restrict__ F1n,
                                 const T* __restrict__ F2n, const T* __restrict__ G1, const T* __restrict__ G2,
                                 const T* __restrict__ G1n, const T* __restrict__ G2n,
                                 const double* __restrict__ ldabs, const double* __restrict__ lsign,
                                 const double* __restrict__ lrat, const double* __restrict__ srat,
                                 double* __restrict__ v_nl) {
  const int w = blockIdx.x;
  if (pref[w] == 0.0) return;   // the whole warp leaves together
  const WalkerRatio wr =
      walker_ratio<T>(w, threadIdx.x, Wn, n, n_up, D, k, Umax, flags, r + (int64_t)w * n * 3, rk + (int64_t)w * 3, -1,
                      nullptr, Ul, Uc, Urow, jp, F1, F2, F1n, F2n, G1, G2, G1n, G2n, ldabs, lsign, lrat, srat);
  if (threadIdx.x == 0) v_nl[w] += pref[w] * wr.sign * exp(wr.logr);
}

}  // namespace fire

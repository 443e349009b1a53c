// Shared device helpers of libfire.
//
// Forward-Laplacian conventions (Methods, "Efficient Laplacian", eqs.
// forward_lap_jac / forward_lap_lap): a quantity that depends on electron
// coordinates is carried as a block of rows
//     row 0      value x
//     row 1      Laplacian  sum_t d^2 x / d t^2  over every electron coordinate t
//     row 2+k    tangent    d x / d t_k
// A linear map acts on every row alike (the bias only on row 0); an
// elementwise function f adds f''(x) * sum_k (d x / d t_k)^2 to the Laplacian.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fire.h"

namespace fire {

// filter MLP hidden width and number of Gaussians d_0 (Supplementary table:
// edge MLP [16, 8], d_0 = 32); kernels keep the filter weights in registers.
constexpr int kEdgeHidden = 16;
constexpr int kGauss = 32;
constexpr int kCutP = 6;        // exponent p of the polynomial cutoff
constexpr double kLnEps = 1e-5;

template <typename T> __device__ __forceinline__ T dexp(T x);
template <> __device__ __forceinline__ float dexp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double dexp<double>(double x) { return exp(x); }
template <typename T> __device__ __forceinline__ T dlog(T x);
template <> __device__ __forceinline__ float dlog<float>(float x) { return logf(x); }
template <> __device__ __forceinline__ double dlog<double>(double x) { return log(x); }
template <typename T> __device__ __forceinline__ T dlog1p(T x);
template <> __device__ __forceinline__ float dlog1p<float>(float x) { return log1pf(x); }
template <> __device__ __forceinline__ double dlog1p<double>(double x) { return log1p(x); }
template <typename T> __device__ __forceinline__ T dsqrt(T x);
template <> __device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }

// SiLU and its first two derivatives: s = logistic(x),
// f = x s, f' = s (1 + x (1 - s)), f'' = s (1 - s) (2 + x (1 - 2 s)).
template <typename T>
__device__ __forceinline__ void silu3(T x, T& f, T& f1, T& f2) {
  T s = T(1) / (T(1) + dexp<T>(-x));
  f = x * s;
  f1 = s * (T(1) + x * (T(1) - s));
  f2 = s * (T(1) - s) * (T(2) + x * (T(1) - T(2) * s));
}

// Polynomial cutoff u(s) and derivatives for s = x / c (reading of the
// Gasteiger et al. envelope with p = 6):
//   u = 1 - A s^p + B s^(p+1) - C s^(p+2),  A=(p+1)(p+2)/2, B=p(p+2), C=p(p+1)/2.
template <typename T>
__device__ __forceinline__ void fcut3(T s, T& u, T& u1, T& u2) {
  if (s >= T(1)) { u = u1 = u2 = T(0); return; }
  const T p = T(kCutP);
  const T A = (p + 1) * (p + 2) / 2, B = p * (p + 2), C = p * (p + 1) / 2;
  T s2 = s * s, s4 = s2 * s2, s5 = s4 * s, s6 = s5 * s;
  u = T(1) - A * s6 + B * s6 * s - C * s6 * s2;
  u1 = -p * A * s5 + (p + 1) * B * s6 - (p + 2) * C * s6 * s;
  u2 = -p * (p - 1) * A * s4 + (p + 1) * p * B * s5 - (p + 2) * (p + 1) * C * s6;
}

// g(r) = log(1+r)/r and its first two derivatives (the rescale of the pair
// features, Methods eq. of e-bar).  A 20-term series is used for r < 0.1,
// where the closed form cancels.
template <typename T>
__device__ __forceinline__ void logrescale3(T r, T& g, T& g1, T& g2) {
  if (r < T(0.1)) {
    g = g1 = g2 = T(0);
    T pw = T(1);  // r^n
    for (int n = 0; n < 20; ++n) {
      T sgn = (n & 1) ? T(-1) : T(1);
      g += sgn * pw / T(n + 1);
      if (n + 1 < 20) {
        // contributes to g1 with power r^n from term n+1
        T sg1 = ((n + 1) & 1) ? T(-1) : T(1);
        g1 += sg1 * T(n + 1) * pw / T(n + 2);
        if (n + 2 < 20) {
          T sg2 = ((n + 2) & 1) ? T(-1) : T(1);
          g2 += sg2 * T(n + 2) * T(n + 1) * pw / T(n + 3);
        }
      }
      pw *= r;
    }
    return;
  }
  T L = dlog1p<T>(r);
  T ir = T(1) / r;
  T L1 = T(1) / (T(1) + r);
  g = L * ir;
  g1 = (L1 - g) * ir;
  g2 = (-L1 * L1 - T(2) * g1) * ir;
}

// A scalar of one electron's position with 3 tangents: value, d/dx, d/dy,
// d/dz and the Laplacian.
template <typename T>
struct FL3 {
  T v, t[3], l;
};

// Radial features of a pair vector delta (|delta| = r > 0) used by the
// filters Gamma (Methods): x = Concat[r, delta], its rescale
// e-bar = log(1+r)/r * x, and chi_g(r) = f_cut(r/c) exp(-sigma_g^2 r^2).
// Each is returned with its gradient and Laplacian in delta-space.
template <typename T>
__device__ __forceinline__ void pair_x(const T d[3], T r, int k, FL3<T>& out) {
  // k = 0: r ; k = 1..3: delta_{k-1}
  if (k == 0) {
    out.v = r;
    for (int t = 0; t < 3; ++t) out.t[t] = d[t] / r;
    out.l = T(2) / r;
  } else {
    out.v = d[k - 1];
    for (int t = 0; t < 3; ++t) out.t[t] = (t == k - 1) ? T(1) : T(0);
    out.l = T(0);
  }
}

template <typename T>
__device__ __forceinline__ void pair_ebar(const T d[3], T r, int k, FL3<T>& out) {
  if (k == 0) {
    T L1 = T(1) / (T(1) + r);
    out.v = dlog1p<T>(r);
    for (int t = 0; t < 3; ++t) out.t[t] = L1 * d[t] / r;
    out.l = -L1 * L1 + T(2) * L1 / r;
  } else {
    T g, g1, g2;
    logrescale3<T>(r, g, g1, g2);
    T dk = d[k - 1];
    out.v = dk * g;
    for (int t = 0; t < 3; ++t) out.t[t] = ((t == k - 1) ? g : T(0)) + dk * g1 * d[t] / r;
    out.l = dk * (g2 + T(4) * g1 / r);
  }
}

template <typename T>
__device__ __forceinline__ void pair_chi(const T d[3], T r, T sigma, T cut, FL3<T>& out) {
  T u, u1, u2;
  fcut3<T>(r / cut, u, u1, u2);
  u1 /= cut;
  u2 /= cut * cut;
  T a = sigma * sigma;
  T G = dexp<T>(-a * r * r);
  T G1 = -T(2) * a * r * G;
  T G2 = (T(4) * a * a * r * r - T(2) * a) * G;
  T c0 = u * G, c1 = u1 * G + u * G1, c2 = u2 * G + T(2) * u1 * G1 + u * G2;
  out.v = c0;
  for (int t = 0; t < 3; ++t) out.t[t] = c1 * d[t] / r;
  out.l = c2 + T(2) * c1 / r;
}

// Hidden unit a_h = SiLU(x W1[:, h] + b1[h]) of the filter MLP in delta-space.
template <typename T, typename W>
__device__ __forceinline__ void pair_hidden(const T d[3], T r, const W* w1, const W* b1, int h,
                                            int H, FL3<T>& out) {
  // w1 is [4][H] row-major.
  T w0 = T(w1[0 * H + h]);
  T u = T(b1[h]) + w0 * r;
  T ut[3];
  for (int t = 0; t < 3; ++t) {
    T wt = T(w1[(1 + t) * H + h]);
    u += wt * d[t];
    ut[t] = w0 * d[t] / r + wt;
  }
  T ul = w0 * T(2) / r;
  T f, f1, f2;
  silu3<T>(u, f, f1, f2);
  out.v = f;
  T sq = T(0);
  for (int t = 0; t < 3; ++t) {
    out.t[t] = f1 * ut[t];
    sq += ut[t] * ut[t];
  }
  out.l = f1 * ul + f2 * sq;
}

// Pointers to every named parameter array inside the flat theta buffer.
template <typename W>
struct Params {
  const W *en_w1, *en_b1, *en_w2, *en_wenv, *en_sigma, *nuc_emb, *en_wfeat;
  const W *ln_gamma, *ln_beta, *glu_wg, *glu_wv, *glu_wo;
  const W *ee_w1, *ee_b1, *ee_w2, *ee_wenv, *ee_sigma, *msg_w, *msg_b;
  const W *mlp_w, *mlp_b, *orb_w, *env_pi, *env_sigma, *cusp;
  const W *jm1_w1, *jm1_b1, *jm1_w2, *jm1_b2, *jm1_w3, *jm1_b3;
  const W *jm2_w1, *jm2_b1, *jm2_w2, *jm2_b2, *jm2_w3, *jm2_b3;
  const W *att_q, *att_wv;
  const W *ja1_w1, *ja1_b1, *ja1_w2, *ja1_b2, *ja1_w3, *ja1_b3;
  const W *ja2_w1, *ja2_b1, *ja2_w2, *ja2_b2, *ja2_w3, *ja2_b3;
};

// Device status word written by kernels (never trapped on).
struct DevStatus {
  int32_t k_required;   // atomicMax of neighbour counts
  int32_t overflow;     // 1 if any list was truncated
  int32_t n_nodes;
  int32_t n_nonfinite;
  int64_t rows_total;
  int64_t nbr_total;
  int32_t tc_err;       // bounded wait of a tensor-core kernel gave up
  int32_t pad_;
};

// Stores v as nc bf16 components (split-bf16: v ~ c0 + c1 + c2), cstride
// elements apart.
__device__ __forceinline__ void store_split_bf16(__nv_bfloat16* p, int64_t cstride, int nc, float v) {
  for (int c = 0; c < nc; ++c) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    p[c * cstride] = h;
    v -= __bfloat162float(h);
  }
}

constexpr int kMaxSplit = 3;

__device__ __forceinline__ int block_index(int w, int i, int Wc, int n, int n_up) {
  // spin-major block order: all spin-up electrons of the chunk first
  return (i < n_up) ? (w * n_up + i) : (Wc * n_up + w * (n - n_up) + (i - n_up));
}

}  // namespace fire

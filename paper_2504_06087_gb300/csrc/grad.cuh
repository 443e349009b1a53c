// Backward (adjoint) kernels of d log|Psi| / d theta per walker (Methods,
// eq. spring: the gradient rows O_i of SPRING).  The forward value path
// (embeddings recomputed in the same call) leaves its intermediates in the
// workspace; these kernels walk it in reverse.  Per-walker weight gradients
// that are sums over a walker's electrons are written by tn_batched /
// colsum_batched; per-edge and per-nucleus sums accumulate with atomics.
#pragma once

#include "common.cuh"
#include "embed.cuh"

namespace fire {

// d log|sum_d det Phi_d| / d Phi_d[i][l] = w_d A_d[l][i] with w_d the signed
// weight of determinant d; back through Phi = o * phi:
//   dO[i][d*n + l] = G phi,  dF[i][d*n + l] = G o.   One CTA per (walker, d).
template <typename T>
__global__ void det_bwd_kernel(int Wc, int n, int n_up, int D, const double* __restrict__ ldabs,
                               const double* __restrict__ lsign, const T* __restrict__ AT,
                               const T* __restrict__ Ov, const T* __restrict__ Fenv, T* __restrict__ dO,
                               T* __restrict__ dF) {
  const int w = blockIdx.x / D, dd = blockIdx.x % D;
  __shared__ double s_w;
  if (threadIdx.x == 0) {
    double lmax = -INFINITY;
    for (int q = 0; q < D; ++q)
      if (lsign[(int64_t)w * D + q] != 0.0 && ldabs[(int64_t)w * D + q] > lmax) lmax = ldabs[(int64_t)w * D + q];
    double S = 0.0, mine = 0.0;
    for (int q = 0; q < D; ++q) {
      const double sg = lsign[(int64_t)w * D + q];
      const double t = sg != 0.0 ? sg * exp(ldabs[(int64_t)w * D + q] - lmax) : 0.0;
      S += t;
      if (q == dd) mine = t;
    }
    s_w = mine / S;
  }
  __syncthreads();
  const T om = T(s_w);
  const int64_t Dn = (int64_t)D * n;
  const T* A = AT + ((int64_t)w * D + dd) * n * n;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, l = e % n;
    const int64_t b = block_index(w, i, Wc, n, n_up);
    const T g = om * A[(int64_t)i * n + l];
    const int64_t col = b * Dn + (int64_t)dd * n + l;
    dO[col] = g * Fenv[col];
    dF[col] = g * Ov[col];
  }
}

// d sigma_me += sum_i dQ[i][me] * (-|r_i - R_m|) * q_ime.  One CTA per walker.
template <typename T>
__global__ void env_sigma_bwd_kernel(int Wc, int n, int n_up, int N, int E, const double* __restrict__ r,
                                     const double* __restrict__ R, const T* __restrict__ Q,
                                     const T* __restrict__ dQ, T* __restrict__ g, int64_t P, int64_t off) {
  const int w = blockIdx.x;
  const int NE = N * E;
  for (int q = threadIdx.x; q < NE; q += blockDim.x) {
    const int m = q / E;
    T acc = T(0);
    for (int i = 0; i < n; ++i) {
      const double* ri = r + ((int64_t)w * n + i) * 3;
      const double dx = ri[0] - R[3 * m], dy = ri[1] - R[3 * m + 1], dz = ri[2] - R[3 * m + 2];
      const T dist = T(sqrt(dx * dx + dy * dy + dz * dz));
      const int64_t b = block_index(w, i, Wc, n, n_up);
      acc += dQ[b * NE + q] * (-dist) * Q[b * NE + q];
    }
    g[(int64_t)w * P + off + q] += acc;
  }
}

// Seeds of the Jastrow-MLP backward: per electron row the adjoint of the
// readout f (1 for MLP1, 1/sum_i MLP2 for MLP2), then dY2 = df * w3.
template <typename T>
__global__ void jseed_kernel(int Wc, int n, int n_up, int J, const T* __restrict__ F2, const T* b32,
                             const T* __restrict__ w3, int second, T* __restrict__ df, T* __restrict__ dY) {
  const int w = blockIdx.x;
  __shared__ T s_inv;
  if (second) {
    if (threadIdx.x == 0) {
      T S = T(0);
      for (int i = 0; i < n; ++i) S += F2[block_index(w, i, Wc, n, n_up)] + b32[0];
      s_inv = T(1) / S;
    }
    __syncthreads();
  }
  const T f = second ? s_inv : T(1);
  for (int i = 0; i < n; ++i) {
    const int64_t b = block_index(w, i, Wc, n, n_up);
    if (threadIdx.x == 0) df[b] = f;
    for (int c = threadIdx.x; c < J; c += blockDim.x) dY[b * J + c] = f * w3[c];
  }
}

// Same seeds for the register readouts (one row per walker): dg1 = 1,
// dg2 = 1 / g2.
template <typename T>
__global__ void vseed_kernel(int J, const T* __restrict__ G2, const T* b32, const T* __restrict__ w3, int second,
                             T* __restrict__ df, T* __restrict__ dY) {
  const int w = blockIdx.x;
  const T f = second ? T(1) / (G2[w] + b32[0]) : T(1);
  if (threadIdx.x == 0) df[w] = f;
  for (int c = threadIdx.x; c < J; c += blockDim.x) dY[(int64_t)w * J + c] = f * w3[c];
}

// Back through the registers V_r = sum_i a_ir u_ir, a_ir = softmax_i(s_ir):
//   du_ir = a_ir dV_r,  da_ir = dV_r . u_ir,  ds_ir = a_ir (da_ir - sum_k a_kr da_kr).
// One CTA per walker, one thread per column of V.  dSU has the layout of SU.
template <typename T>
__global__ void att_bwd_kernel(int Wc, int n, int n_up, int R, int dr, const T* __restrict__ SU, int64_t ld,
                               const T* __restrict__ dV, T* __restrict__ dSU) {
  extern __shared__ unsigned char ab_smem[];
  T* a = reinterpret_cast<T*>(ab_smem);      // [n][R] softmax weights
  T* da = a + (int64_t)n * R;                // [n][R]
  T* smax = da + (int64_t)n * R;             // [R]
  T* zs = smax + R;                          // [R]
  T* dd = zs + R;                            // [R]  sum_k a_kr da_kr
  const int w = blockIdx.x;
  const int RD = R * dr;
  const int col = threadIdx.x;
  const int rg = col / dr;
  for (int q = threadIdx.x; q < R; q += blockDim.x) {
    T m = -INFINITY;
    for (int i = 0; i < n; ++i) m = fmax(m, SU[(int64_t)block_index(w, i, Wc, n, n_up) * ld + q]);
    T z = T(0);
    for (int i = 0; i < n; ++i) z += dexp<T>(SU[(int64_t)block_index(w, i, Wc, n, n_up) * ld + q] - m);
    smax[q] = m;
    zs[q] = z;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * R; e += blockDim.x) {
    const int i = e / R, q = e % R;
    a[e] = dexp<T>(SU[(int64_t)block_index(w, i, Wc, n, n_up) * ld + q] - smax[q]) / zs[q];
    da[e] = T(0);
  }
  __syncthreads();
  // da_ir = sum_c dV_rc u_irc : per (i, r) a reduction over the dr columns
  for (int e = threadIdx.x; e < n * R; e += blockDim.x) {
    const int i = e / R, q = e % R;
    const int64_t row = (int64_t)block_index(w, i, Wc, n, n_up) * ld;
    T s = T(0);
    for (int c = 0; c < dr; ++c) s += dV[(int64_t)w * RD + q * dr + c] * SU[row + R + q * dr + c];
    da[e] = s;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < R; q += blockDim.x) {
    T s = T(0);
    for (int i = 0; i < n; ++i) s += a[i * R + q] * da[i * R + q];
    dd[q] = s;
  }
  __syncthreads();
  for (int i = 0; i < n; ++i) {
    const int64_t row = (int64_t)block_index(w, i, Wc, n, n_up) * ld;
    if (col < RD) dSU[row + R + col] = a[i * R + rg] * dV[(int64_t)w * RD + col];
    for (int q = threadIdx.x; q < R; q += blockDim.x) dSU[row + q] = a[i * R + q] * (da[i * R + q] - dd[q]);
  }
}

// Reduces 48 per-thread values over the CTA (blockDim multiple of 32, <= 1024)
// into out[0..48).  `part` has room for 32 x 48 values.
template <typename T>
__device__ __forceinline__ void block_reduce48(T v[48], T* part, T* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // warp transpose-reduction (recursive halving): at each step a lane keeps
  // half of its values and adds its partner's copy of them, so lane L ends
  // with the warp sums of values L and (L < 16) 32 + L -- 62 shuffles
  // instead of 5 per value
  T a[32], b[16];
#pragma unroll
  for (int k = 0; k < 32; ++k) a[k] = v[k];
#pragma unroll
  for (int k = 0; k < 16; ++k) b[k] = v[32 + k];
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int k = 0; k < s; ++k) {
      const T send = up ? a[k] : a[k + s];
      const T keep = up ? a[k + s] : a[k];
      a[k] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) b[k] += __shfl_xor_sync(0xffffffffu, b[k], 16);
#pragma unroll
  for (int s = 8; s >= 1; s >>= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int k = 0; k < s; ++k) {
      const T send = up ? b[k] : b[k + s];
      const T keep = up ? b[k + s] : b[k];
      b[k] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  part[wid * 48 + lane] = a[0];
  if (lane < 16) part[wid * 48 + 32 + lane] = b[0];
  __syncthreads();
  for (int t = threadIdx.x; t < 48; t += blockDim.x) {
    T s = T(0);
    for (int q = 0; q < nw; ++q) s += part[q * 48 + t];
    out[t] = s;
  }
  __syncthreads();
}

// Filter backward shared by the message and electron-nucleus passes: given
// dGamma_c for the pair vector delta (features in feat, see
// pair_features_to_smem), accumulates the gradient of W2 (16 x d), W_env
// (32 x d) in registers and of W1 (4 x H), b1, sigma either into the CTA's
// shared accumulator acc[5H + G] (ACC: the weights are the same for every
// pair of the CTA; layout W1 rows 0..3, b1, sigma) or by atomics into
// gW1/gb1/gsig (per-nucleus weights).  Entry t of the 48 reduced values is
// handled by thread t mod blockDim, the same thread for every pair, so the
// shared accumulator needs no atomics.
template <bool ACC, typename T, typename W>
__device__ __forceinline__ void filter_bwd(const FL3<T>* feat, const T dv[3], T r, T cut, const W* w1,
                                           const W* b1, const W* sigma, const T w2c[kEdgeHidden],
                                           const T wec[kGauss], T gv, T ev, T dgam, T gW2[kEdgeHidden],
                                           T gWe[kGauss], T* part, T* red48, T* acc, T* gW1, T* gb1, T* gsig) {
  constexpr int H = kEdgeHidden, G = kGauss;
  T v[48];
#pragma unroll
  for (int h = 0; h < H; ++h) {
    gW2[h] += feat[h].v * dgam * ev;
    v[h] = dgam * ev * w2c[h];
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {
    gWe[g] += feat[H + g].v * dgam * gv;
    v[H + g] = dgam * gv * wec[g];
  }
  block_reduce48<T>(v, part, red48);
  for (int t = threadIdx.x; t < H + G; t += blockDim.x) {
    if (t < H) {
      // du_h = da_h * SiLU'(u_h), u_h = x . W1[:, h] + b1[h], x = [r, delta]
      T u = T(b1[t]) + T(w1[t]) * r;
      for (int k = 0; k < 3; ++k) u += T(w1[(1 + k) * H + t]) * dv[k];
      T f, f1, f2;
      silu3<T>(u, f, f1, f2);
      const T du = red48[t] * f1;
      if (ACC) {
        acc[t] += du * r;
        for (int k = 0; k < 3; ++k) acc[(1 + k) * H + t] += du * dv[k];
        acc[4 * H + t] += du;
      } else {
        atomicAdd(&gW1[0 * H + t], du * r);
        for (int k = 0; k < 3; ++k) atomicAdd(&gW1[(1 + k) * H + t], du * dv[k]);
        atomicAdd(&gb1[t], du);
      }
    } else {
      // chi_g = f_cut exp(-sigma_g^2 r^2): d chi_g / d sigma_g = -2 sigma_g r^2 chi_g
      const int g = t - H;
      const T sg = T(sigma[g]);
      const T ds = red48[t] * (-T(2) * sg * r * r) * feat[H + g].v;
      if (ACC) acc[5 * H + g] += ds;
      else atomicAdd(&gsig[g], ds);
    }
  }
}

// Message-passing backward.  One CTA per electron (w, i), blockDim == d.
// Inputs: dH1 = d/dh^1_i; recomputes each edge.  Outputs: dP [nb][2d]
// (own rows), dQ [nb][2d] (atomics at j), parameter gradients of the e-e
// filter, W^alpha_c and b^alpha.
template <typename T, typename W>
__global__ void msg_bwd_kernel(int Wc, int n, int n_up, int d, int K, const double* __restrict__ r,
                               double cut, Params<W> p, const int32_t* __restrict__ idx,
                               const int32_t* __restrict__ cnt, const T* __restrict__ PQ,
                               const T* __restrict__ dH1, T* __restrict__ dP, T* __restrict__ dQ,
                               T* __restrict__ grad, int64_t P, const int64_t* __restrict__ po) {
  constexpr int H = kEdgeHidden, G = kGauss;
  __shared__ FL3<T> feat[H + G + 4];
  __shared__ T part[32 * 48];
  __shared__ T red48[48];
  __shared__ T acc[5 * H + G];
  const int blk = blockIdx.x;
  const int w = blk / n, i = blk % n;
  const int c = threadIdx.x;
  const int bi = block_index(w, i, Wc, n, n_up);
  for (int t = c; t < 5 * H + G; t += blockDim.x) acc[t] = T(0);
  const int64_t ld4 = 4 * (int64_t)d;
  T* gw = grad + (int64_t)w * P;
  T w2[H], we[G], wc[2][4], bb[2];
#pragma unroll
  for (int h = 0; h < H; ++h) w2[h] = T(p.ee_w2[h * d + c]);
#pragma unroll
  for (int g = 0; g < G; ++g) we[g] = T(p.ee_wenv[g * d + c]);
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    bb[a] = T(p.msg_b[a * d + c]);
#pragma unroll
    for (int k = 0; k < 4; ++k) wc[a][k] = T(p.msg_w[((int64_t)a * (2 * d + 4) + 2 * d + k) * d + c]);
  }
  T gW2[H], gWe[G], gWc[2][4], gB[2], dPa[2];
#pragma unroll
  for (int h = 0; h < H; ++h) gW2[h] = T(0);
#pragma unroll
  for (int g = 0; g < G; ++g) gWe[g] = T(0);
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    gB[a] = dPa[a] = T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) gWc[a][k] = T(0);
  }
  const T delta = dH1[(int64_t)bi * d + c];
  const int cpar = cnt[((int64_t)w * n + i) * 2], ctot = cpar + cnt[((int64_t)w * n + i) * 2 + 1];
  const double* rw = r + (int64_t)w * n * 3;
  const int32_t* li = idx + ((int64_t)w * n + i) * K;
  for (int s = 0; s < ctot; ++s) {
    const int j = li[s];
    const int a = (s < cpar) ? 0 : 1;
    double ddv[3] = {rw[3 * i] - rw[3 * j], rw[3 * i + 1] - rw[3 * j + 1], rw[3 * i + 2] - rw[3 * j + 2]};
    const double rr = sqrt(ddv[0] * ddv[0] + ddv[1] * ddv[1] + ddv[2] * ddv[2]);
    T dv[3] = {T(ddv[0]), T(ddv[1]), T(ddv[2])};
    __syncthreads();
    pair_features_to_smem<T, W>(dv, T(rr), p.ee_w1, p.ee_b1, p.ee_sigma, T(cut), feat);
    __syncthreads();
    T gv = T(0), ev = T(0);
#pragma unroll
    for (int h = 0; h < H; ++h) gv += feat[h].v * w2[h];
#pragma unroll
    for (int g = 0; g < G; ++g) ev += feat[H + g].v * we[g];
    const T gam = gv * ev;
    const int bj = block_index(w, j, Wc, n, n_up);
    T z = PQ[(int64_t)bi * ld4 + (int64_t)a * d + c] + PQ[(int64_t)bj * ld4 + 2 * (int64_t)d + (int64_t)a * d + c] +
          bb[a];
#pragma unroll
    for (int k = 0; k < 4; ++k) z += feat[H + G + k].v * wc[a][k];
    T f, f1, f2;
    silu3<T>(z, f, f1, f2);
    const T dgam = delta * f;
    const T dz = delta * gam * f1;
    dPa[a] += dz;
    atomicAdd(&dQ[(int64_t)bj * 2 * d + (int64_t)a * d + c], dz);
    gB[a] += dz;
#pragma unroll
    for (int k = 0; k < 4; ++k) gWc[a][k] += feat[H + G + k].v * dz;
    filter_bwd<true, T, W>(feat, dv, T(rr), T(cut), p.ee_w1, p.ee_b1, p.ee_sigma, w2, we, gv, ev, dgam, gW2,
                           gWe, part, red48, acc, nullptr, nullptr, nullptr);
  }
  dP[(int64_t)bi * 2 * d + c] = dPa[0];
  dP[(int64_t)bi * 2 * d + d + c] = dPa[1];
  __syncthreads();
  if (ctot > 0) {
    for (int t = c; t < 5 * H + G; t += blockDim.x) {
      if (t < 4 * H) atomicAdd(&gw[po[P_EE_W1] + t], acc[t]);
      else if (t < 5 * H) atomicAdd(&gw[po[P_EE_B1] + t - 4 * H], acc[t]);
      else atomicAdd(&gw[po[P_EE_SIGMA] + t - 5 * H], acc[t]);
    }
#pragma unroll
    for (int h = 0; h < H; ++h) atomicAdd(&gw[po[P_EE_W2] + h * d + c], gW2[h]);
#pragma unroll
    for (int g = 0; g < G; ++g) atomicAdd(&gw[po[P_EE_WENV] + g * d + c], gWe[g]);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      atomicAdd(&gw[po[P_MSG_B] + a * d + c], gB[a]);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        atomicAdd(&gw[po[P_MSG_W] + ((int64_t)a * (2 * d + 4) + 2 * d + k) * d + c], gWc[a][k]);
    }
  }
}

// Electron-nucleus filter backward: ds = d/ds_i (the filter sum).  One CTA
// per electron, blockDim == d.
template <typename T, typename W>
__global__ void en_bwd_kernel(int Wc, int n, int n_up, int N, int d, const double* __restrict__ r,
                              const double* __restrict__ R, double cnuc, Params<W> p, const T* __restrict__ dS,
                              T* __restrict__ grad, int64_t P, const int64_t* __restrict__ po) {
  constexpr int H = kEdgeHidden, G = kGauss;
  __shared__ FL3<T> feat[H + G + 4];
  __shared__ T part[32 * 48];
  __shared__ T red48[48];
  const int blk = blockIdx.x;
  const int w = blk / n, i = blk % n;
  const int c = threadIdx.x;
  T* gw = grad + (int64_t)w * P;
  T w2[H], we[G], wf[4];
#pragma unroll
  for (int h = 0; h < H; ++h) w2[h] = T(p.en_w2[h * d + c]);
#pragma unroll
  for (int g = 0; g < G; ++g) we[g] = T(p.en_wenv[g * d + c]);
#pragma unroll
  for (int k = 0; k < 4; ++k) wf[k] = T(p.en_wfeat[k * d + c]);
  T gW2[H], gWe[G], gWf[4];
#pragma unroll
  for (int h = 0; h < H; ++h) gW2[h] = T(0);
#pragma unroll
  for (int g = 0; g < G; ++g) gWe[g] = T(0);
#pragma unroll
  for (int k = 0; k < 4; ++k) gWf[k] = T(0);
  const T ds = dS[(int64_t)block_index(w, i, Wc, n, n_up) * d + c];
  const double* ri = r + ((int64_t)w * n + i) * 3;
  bool any = false;
  for (int m = 0; m < N; ++m) {
    double ddv[3] = {ri[0] - R[3 * m], ri[1] - R[3 * m + 1], ri[2] - R[3 * m + 2]};
    const double rr = sqrt(ddv[0] * ddv[0] + ddv[1] * ddv[1] + ddv[2] * ddv[2]);
    if (!(rr < cnuc)) continue;
    any = true;
    T dv[3] = {T(ddv[0]), T(ddv[1]), T(ddv[2])};
    __syncthreads();
    pair_features_to_smem<T, W>(dv, T(rr), p.en_w1 + (int64_t)m * 4 * H, p.en_b1 + (int64_t)m * H, p.en_sigma,
                                T(cnuc), feat);
    __syncthreads();
    T gv = T(0), ev = T(0), fv = T(p.nuc_emb[(int64_t)m * d + c]);
#pragma unroll
    for (int h = 0; h < H; ++h) gv += feat[h].v * w2[h];
#pragma unroll
    for (int g = 0; g < G; ++g) ev += feat[H + g].v * we[g];
#pragma unroll
    for (int k = 0; k < 4; ++k) fv += feat[H + G + k].v * wf[k];
    const T gam = gv * ev;
    const T dgam = ds * fv;
    const T dfv = ds * gam;
    atomicAdd(&gw[po[P_NUC_EMB] + (int64_t)m * d + c], dfv);
#pragma unroll
    for (int k = 0; k < 4; ++k) gWf[k] += feat[H + G + k].v * dfv;
    filter_bwd<false, T, W>(feat, dv, T(rr), T(cnuc), p.en_w1 + (int64_t)m * 4 * H, p.en_b1 + (int64_t)m * H,
                     p.en_sigma, w2, we, gv, ev, dgam, gW2, gWe, part, red48, nullptr,
                     gw + po[P_EN_W1] + (int64_t)m * 4 * H, gw + po[P_EN_B1] + (int64_t)m * H,
                     gw + po[P_EN_SIGMA]);
  }
  if (any) {
#pragma unroll
    for (int h = 0; h < H; ++h) atomicAdd(&gw[po[P_EN_W2] + h * d + c], gW2[h]);
#pragma unroll
    for (int g = 0; g < G; ++g) atomicAdd(&gw[po[P_EN_WENV] + g * d + c], gWe[g]);
#pragma unroll
    for (int k = 0; k < 4; ++k) atomicAdd(&gw[po[P_EN_WFEAT] + k * d + c], gWf[k]);
  }
}

// GLU gate backward: dZg = dP * zv * SiLU'(zg), dZv = dP * SiLU(zg).
template <typename T>
__global__ void gate_bwd_kernel(int64_t rows, int d, const T* __restrict__ Z, const T* __restrict__ dPg,
                                T* __restrict__ dZ) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * d) return;
  const int64_t rr = e / d;
  const int c = (int)(e % d);
  const T zg = Z[rr * 2 * d + c], zv = Z[rr * 2 * d + d + c];
  T f, f1, f2;
  silu3<T>(zg, f, f1, f2);
  const T g = dPg[rr * d + c];
  dZ[rr * 2 * d + c] = g * zv * f1;
  dZ[rr * 2 * d + d + c] = g * f;
}

// LayerNorm backward for one row per CTA (blockDim == d): y = gamma xhat + beta,
// dxhat = dy gamma, ds = (dxhat - mean(dxhat) - xhat mean(dxhat xhat)) / sigma.
// Also writes dy * xhat (for d gamma).
template <typename T, typename W>
__global__ void ln_bwd_kernel(int d, const T* __restrict__ S, const T* __restrict__ dY, const W* gamma,
                              T* __restrict__ dS, T* __restrict__ dyx) {
  __shared__ T red[32];
  const int64_t row = blockIdx.x;
  const int c = threadIdx.x;
  const T inv_d = T(1) / T(d);
  const T x = S[row * d + c];
  const T mu = block_sum(x, red) * inv_d;
  const T cc = x - mu;
  const T var = block_sum(cc * cc, red) * inv_d;
  const T sg = dsqrt<T>(var + T(kLnEps));
  const T xh = cc / sg;
  const T dy = dY[row * d + c];
  const T dxh = dy * T(gamma[c]);
  const T m1 = block_sum(dxh, red) * inv_d;
  const T m2 = block_sum(dxh * xh, red) * inv_d;
  dS[row * d + c] = (dxh - m1 - xh * m2) / sg;
  dyx[row * d + c] = dy * xh;
}

// Cusp Jastrow parameter gradient: u = w a^2 / (a + r):
// du/dw = a^2/(a+r), du/da = w a (a + 2r) / (a + r)^2.  One CTA per walker.
template <typename T>
__global__ void cusp_bwd_kernel(int n, int n_up, const double* __restrict__ r, const T* __restrict__ cusp,
                                T* __restrict__ grad, int64_t P, int64_t off) {
  __shared__ T red[32];
  const int w = blockIdx.x;
  const double* rw = r + (int64_t)w * n * 3;
  T g[4] = {T(0), T(0), T(0), T(0)};
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    if (j <= i) continue;
    const T dx = T(rw[3 * i] - rw[3 * j]), dy = T(rw[3 * i + 1] - rw[3 * j + 1]), dz = T(rw[3 * i + 2] - rw[3 * j + 2]);
    const T rr = dsqrt<T>(dx * dx + dy * dy + dz * dz);
    const bool same = ((i < n_up) == (j < n_up));
    const T om = same ? cusp[0] : cusp[1], al = same ? cusp[2] : cusp[3];
    const T den = al + rr;
    const T dw = al * al / den;
    const T da = om * al * (al + T(2) * rr) / (den * den);
    if (same) { g[0] += dw; g[2] += da; } else { g[1] += dw; g[3] += da; }
  }
  for (int k = 0; k < 4; ++k) {
    T v = g[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      T s = T(0);
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
      grad[(int64_t)w * P + off + k] += s;
    }
  }
}

}  // namespace fire

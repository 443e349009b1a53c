// Initial embeddings h^0 and the message passing step h^1 (Methods, "Wave
// function ansatz"), each carried with its tangents and Laplacian.
//
//   h^0_i = GLU( sum_m Gamma_m(e^_im) * (h^nuc_m + e-bar^_im W) )
//   h^1_i = h^0_i + sum_alpha sum_{j in N^alpha_i} Gamma(e_ij) *
//           SiLU(Concat[h^0_i, h^0_j, e-bar_ij] W^alpha + b^alpha)
//
// h^0_i depends on r_i only: its blocks have 5 rows (value, Laplacian,
// d/dx_i, d/dy_i, d/dz_i).  The concatenation is applied as
// h^0_i W^alpha_a + h^0_j W^alpha_b + e-bar_ij W^alpha_c; the first two are
// per-electron products computed once by a matrix product (PQ), the third is
// per edge.
#pragma once

#include "common.cuh"

namespace fire {

template <typename T>
__device__ __forceinline__ void fl3_mul(const FL3<T>& a, const FL3<T>& b, FL3<T>& o) {
  o.v = a.v * b.v;
  T cross = T(0);
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    o.t[t] = a.t[t] * b.v + a.v * b.t[t];
    cross += a.t[t] * b.t[t];
  }
  o.l = a.l * b.v + T(2) * cross + a.v * b.l;
}

// Filter features of one pair vector into shared memory:
// feat[0..H) hidden units, feat[H..H+G) Gaussians chi_g, feat[H+G..H+G+4) e-bar.
template <typename T, typename W>
__device__ __forceinline__ void pair_features_to_smem(const T dv[3], T r, const W* w1, const W* b1,
                                                      const W* sigma, T cut, FL3<T>* feat) {
  const int H = kEdgeHidden, G = kGauss;
  for (int k = threadIdx.x; k < H + G + 4; k += blockDim.x) {
    FL3<T> o;
    if (k < H) pair_hidden<T, W>(dv, r, w1, b1, k, H, o);
    else if (k < H + G) pair_chi<T>(dv, r, T(sigma[k - H]), cut, o);
    else pair_ebar<T>(dv, r, k - H - G, o);
    feat[k] = o;
  }
}

// Feature k of one pair (the layout of pair_features_to_smem).
template <typename T, typename W>
__device__ __forceinline__ FL3<T> pair_feature(int k, const T dv[3], T r, const W* w1, const W* b1,
                                               const W* sigma, T cut) {
  const int H = kEdgeHidden, G = kGauss;
  FL3<T> o;
  if (k < H) pair_hidden<T, W>(dv, r, w1, b1, k, H, o);
  else if (k < H + G) pair_chi<T>(dv, r, T(sigma[k - H]), cut, o);
  else pair_ebar<T>(dv, r, k - H - G, o);
  return o;
}

// Pairs whose filter features are computed together (one barrier pair per
// batch instead of per pair).
constexpr int kPairBatch = 16;
// Largest nucleus count of the batched electron-nucleus filter.
constexpr int kMaxNuc = 512;

// One CTA per electron (w, i), blockDim == d.  Writes the filter sum
// s_i = sum_m Gamma_m * (h^nuc_m + e-bar W) as R5 rows of S.
template <typename T, typename W>
__global__ void en_filter_kernel(int Wc, int n, int n_up, int N, int d, const double* __restrict__ r,
                                 const double* __restrict__ R, double cnuc, Params<W> p,
                                 T* __restrict__ S, int R5) {
  constexpr int H = kEdgeHidden, G = kGauss;
  const int blk = blockIdx.x;
  const int w = blk / n, i = blk % n;
  const int c = threadIdx.x;
  T w2[H], we[G], wf[4];
#pragma unroll
  for (int h = 0; h < H; ++h) w2[h] = T(p.en_w2[h * d + c]);
#pragma unroll
  for (int g = 0; g < G; ++g) we[g] = T(p.en_wenv[g * d + c]);
#pragma unroll
  for (int k = 0; k < 4; ++k) wf[k] = T(p.en_wfeat[k * d + c]);
  FL3<T> acc;
  acc.v = acc.l = T(0);
  acc.t[0] = acc.t[1] = acc.t[2] = T(0);
  const double* ri = r + ((int64_t)w * n + i) * 3;
  // nuclei within c_n (Gamma_m vanishes identically beyond), ascending
  __shared__ FL3<T> featb[kPairBatch][H + G + 4];
  __shared__ T s_dv[kPairBatch][3], s_r[kPairBatch];
  __shared__ int s_m[kPairBatch];
  __shared__ int s_list[kMaxNuc];
  __shared__ int s_cnt;
  if (threadIdx.x < 32) {
    int cntm = 0;
    for (int m0 = 0; m0 < N; m0 += 32) {
      const int m = m0 + threadIdx.x;
      bool in = false;
      if (m < N) {
        const double d0 = ri[0] - R[3 * m], d1 = ri[1] - R[3 * m + 1], d2 = ri[2] - R[3 * m + 2];
        in = sqrt(d0 * d0 + d1 * d1 + d2 * d2) < cnuc;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, in);
      if (in) s_list[cntm + __popc(bal & ((1u << threadIdx.x) - 1u))] = m;
      cntm += __popc(bal);
    }
    if (threadIdx.x == 0) s_cnt = cntm;
  }
  __syncthreads();
  const int nlist = s_cnt;
  for (int b0 = 0; b0 < nlist; b0 += kPairBatch) {
    const int nbat = min(kPairBatch, nlist - b0);
    __syncthreads();   // the previous batch is consumed
    if (threadIdx.x < nbat) {
      const int m = s_list[b0 + threadIdx.x];
      const double dd[3] = {ri[0] - R[3 * m], ri[1] - R[3 * m + 1], ri[2] - R[3 * m + 2]};
      s_dv[threadIdx.x][0] = T(dd[0]);
      s_dv[threadIdx.x][1] = T(dd[1]);
      s_dv[threadIdx.x][2] = T(dd[2]);
      s_r[threadIdx.x] = T(sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]));
      s_m[threadIdx.x] = m;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nbat * (H + G + 4); e += blockDim.x) {
      const int q = e / (H + G + 4), k = e - q * (H + G + 4);
      const int m = s_m[q];
      featb[q][k] = pair_feature<T, W>(k, s_dv[q], s_r[q], p.en_w1 + (int64_t)m * 4 * H, p.en_b1 + (int64_t)m * H,
                                       p.en_sigma, T(cnuc));
    }
    __syncthreads();
    for (int q = 0; q < nbat; ++q) {
      const int m = s_m[q];
      const FL3<T>* feat = featb[q];
    FL3<T> gv, ev, fv;
    gv.v = gv.l = ev.v = ev.l = T(0);
    fv.v = T(p.nuc_emb[(int64_t)m * d + c]);
    fv.l = T(0);
#pragma unroll
    for (int t = 0; t < 3; ++t) gv.t[t] = ev.t[t] = fv.t[t] = T(0);
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const FL3<T> a = feat[h];
      gv.v += a.v * w2[h];
      gv.l += a.l * w2[h];
#pragma unroll
      for (int t = 0; t < 3; ++t) gv.t[t] += a.t[t] * w2[h];
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const FL3<T> a = feat[H + g];
      ev.v += a.v * we[g];
      ev.l += a.l * we[g];
#pragma unroll
      for (int t = 0; t < 3; ++t) ev.t[t] += a.t[t] * we[g];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const FL3<T> a = feat[H + G + k];
      fv.v += a.v * wf[k];
      fv.l += a.l * wf[k];
#pragma unroll
      for (int t = 0; t < 3; ++t) fv.t[t] += a.t[t] * wf[k];
    }
    FL3<T> gam, term;
    fl3_mul(gv, ev, gam);
    fl3_mul(gam, fv, term);
    acc.v += term.v;
    acc.l += term.l;
#pragma unroll
    for (int t = 0; t < 3; ++t) acc.t[t] += term.t[t];
    }
  }
  const int64_t row = (int64_t)block_index(w, i, Wc, n, n_up) * R5;
  S[row * d + c] = acc.v;
  if (R5 > 1) {
    S[(row + 1) * d + c] = acc.l;
#pragma unroll
    for (int t = 0; t < 3; ++t) S[(row + 2 + t) * d + c] = acc.t[t];
  }
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  // blockDim.x multiple of 32, <= 1024; red has >= 32 entries.
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  T s = T(0);
  for (int k = 0; k < nw; ++k) s += red[k];
  return s;
}

// LayerNorm in forward-Laplacian form over blocks of R5 rows (3 tangents).
// One CTA per electron, blockDim == d.
template <typename T, typename W>
__global__ void ln_fl_kernel(int d, const T* __restrict__ X, T* __restrict__ Y, const W* gamma,
                             const W* beta, int R5, __nv_bfloat16* __restrict__ Yb = nullptr, int ync = 0,
                             int64_t ycs = 0) {
  __shared__ T red[32];
  const int64_t row = (int64_t)blockIdx.x * R5;
  const int c = threadIdx.x;
  const T inv_d = T(1) / T(d);
  FL3<T> x;
  x.v = X[row * d + c];
  x.l = (R5 > 1) ? X[(row + 1) * d + c] : T(0);
#pragma unroll
  for (int t = 0; t < 3; ++t) x.t[t] = (R5 > 1) ? X[(row + 2 + t) * d + c] : T(0);
  T mu = block_sum(x.v, red) * inv_d;
  T mul = block_sum(x.l, red) * inv_d;
  T mut[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) mut[t] = block_sum(x.t[t], red) * inv_d;
  FL3<T> cc;
  cc.v = x.v - mu;
  cc.l = x.l - mul;
#pragma unroll
  for (int t = 0; t < 3; ++t) cc.t[t] = x.t[t] - mut[t];
  T var = block_sum(cc.v * cc.v, red) * inv_d;
  T sq = cc.t[0] * cc.t[0] + cc.t[1] * cc.t[1] + cc.t[2] * cc.t[2];
  T varl = T(2) * block_sum(sq + cc.v * cc.l, red) * inv_d;
  T vart[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) vart[t] = T(2) * block_sum(cc.v * cc.t[t], red) * inv_d;
  const T s = dsqrt<T>(var + T(kLnEps));
  T st[3], st2 = T(0), vt2 = T(0);
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    st[t] = vart[t] / (T(2) * s);
    st2 += st[t] * st[t];
    vt2 += vart[t] * vart[t];
  }
  const T sl = varl / (T(2) * s) - vt2 / (T(4) * s * s * s);
  const T g = T(gamma[c]);
  auto put = [&](int64_t q, T v) {
    Y[q * d + c] = v;
    if (Yb) store_split_bf16(Yb + q * d + c, ycs, ync, (float)v);
  };
  put(row, g * (cc.v / s) + T(beta[c]));
  if (R5 > 1) {
    T cross = T(0);
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      cross += cc.t[t] * st[t];
      put(row + 2 + t, g * (cc.t[t] / s - cc.v * st[t] / (s * s)));
    }
    T yl = cc.l / s - T(2) * cross / (s * s) - cc.v * sl / (s * s) + T(2) * cc.v * st2 / (s * s * s);
    put(row + 1, g * yl);
  }
}

// GLU gate p = SiLU(z_g) * z_v in forward-Laplacian form; Z is [rows][2d]
// (gate columns first), P [rows][d].  One CTA per electron, blockDim == d.
template <typename T>
__global__ void glu_gate_kernel(int d, const T* __restrict__ Z, T* __restrict__ P, int R5,
                                __nv_bfloat16* __restrict__ Pb = nullptr, int pnc = 0, int64_t pcs = 0) {
  const int64_t row = (int64_t)blockIdx.x * R5;
  const int c = threadIdx.x;
  const int64_t ld = 2 * d;
  auto put = [&](int64_t q, T v) {
    P[q * d + c] = v;
    if (Pb) store_split_bf16(Pb + q * d + c, pcs, pnc, (float)v);
  };
  T zg = Z[row * ld + c], zv = Z[row * ld + d + c];
  T f, f1, f2;
  silu3<T>(zg, f, f1, f2);
  put(row, f * zv);
  if (R5 > 1) {
    T gl = Z[(row + 1) * ld + c], vl = Z[(row + 1) * ld + d + c];
    T sq = T(0), cross = T(0);
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      T gt = Z[(row + 2 + t) * ld + c], vt = Z[(row + 2 + t) * ld + d + c];
      sq += gt * gt;
      cross += f1 * gt * vt;
      put(row + 2 + t, f1 * gt * zv + f * vt);
    }
    put(row + 1, (f1 * gl + f2 * sq) * zv + T(2) * cross + f * vl);
  }
}

// Xb = nc bf16 components of the float rows X[0 .. rows) x [0 .. ncol)
// (row strides ldx and ldb, components cs elements apart).
template <typename T>
__global__ void split_rows_kernel(int64_t rows, int ncol, const T* __restrict__ X, int64_t ldx,
                                  __nv_bfloat16* __restrict__ Xb, int64_t ldb, int nc, int64_t cs) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * ncol) return;
  const int64_t r = e / ncol;
  const int c = (int)(e - r * ncol);
  store_split_bf16(Xb + r * ldb + c, cs, nc, (float)X[r * ldx + c]);
}

// Message passing step.  One CTA per electron (w, i), blockDim == d.
// H0 [Wc*n*R5][d]; PQ [Wc*n*R5][4d] = [h0 W^par_a | h0 W^anti_a | h0 W^par_b |
// h0 W^anti_b]; X receives the block of h^1_i (value, Laplacian, tangents).
template <typename T, typename W>
__global__ void msg_kernel(int Wc, int n, int n_up, int d, int K, const double* __restrict__ r,
                           double cut, Params<W> p, const int32_t* __restrict__ idx,
                           const int32_t* __restrict__ cnt, const int64_t* __restrict__ blk_off,
                           const T* __restrict__ H0, const T* __restrict__ PQ, T* __restrict__ X,
                           __nv_bfloat16* __restrict__ Xb, int xnc, int64_t xcs, int deriv) {
  constexpr int H = kEdgeHidden, G = kGauss;
  const int blk = blockIdx.x;
  const int w = blk / n, i = blk % n;
  const int c = threadIdx.x;
  const int R5 = deriv ? 5 : 1;
  const int bi = block_index(w, i, Wc, n, n_up);
  const int64_t hrow = (int64_t)bi * R5;
  const int64_t ld4 = 4 * (int64_t)d;
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
  // accumulator = h^0_i (value, Laplacian, self tangents)
  FL3<T> acc;
  acc.v = H0[hrow * d + c];
  acc.l = deriv ? H0[(hrow + 1) * d + c] : T(0);
#pragma unroll
  for (int t = 0; t < 3; ++t) acc.t[t] = deriv ? H0[(hrow + 2 + t) * d + c] : T(0);
  // P_i (the own-electron half of the concatenation product) for both
  // spin relations: value, Laplacian and tangent rows, read once
  T pv[2], pl[2], pt[2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const int64_t pc = (int64_t)a * d + c;
    pv[a] = PQ[hrow * ld4 + pc];
    pl[a] = deriv ? PQ[(hrow + 1) * ld4 + pc] : T(0);
#pragma unroll
    for (int t = 0; t < 3; ++t) pt[a][t] = deriv ? PQ[(hrow + 2 + t) * ld4 + pc] : T(0);
  }
  const int64_t xoff = blk_off[bi];
  const int cpar = cnt[((int64_t)w * n + i) * 2], ctot = cpar + cnt[((int64_t)w * n + i) * 2 + 1];
  const double* rw = r + (int64_t)w * n * 3;
  const int32_t* li = idx + ((int64_t)w * n + i) * K;
  __shared__ FL3<T> featb[kPairBatch][H + G + 4];
  __shared__ T s_dv[kPairBatch][3], s_r[kPairBatch];
  for (int b0 = 0; b0 < ctot; b0 += kPairBatch) {
    const int nbat = min(kPairBatch, ctot - b0);
    __syncthreads();   // the previous batch is consumed
    if (threadIdx.x < nbat) {
      const int j = li[b0 + threadIdx.x];
      const double dd[3] = {rw[3 * i] - rw[3 * j], rw[3 * i + 1] - rw[3 * j + 1], rw[3 * i + 2] - rw[3 * j + 2]};
      s_dv[threadIdx.x][0] = T(dd[0]);
      s_dv[threadIdx.x][1] = T(dd[1]);
      s_dv[threadIdx.x][2] = T(dd[2]);
      s_r[threadIdx.x] = T(sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]));
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nbat * (H + G + 4); e += blockDim.x) {
      const int q = e / (H + G + 4), k = e - q * (H + G + 4);
      featb[q][k] = pair_feature<T, W>(k, s_dv[q], s_r[q], p.ee_w1, p.ee_b1, p.ee_sigma, T(cut));
    }
    __syncthreads();
  for (int s = b0; s < b0 + nbat; ++s) {
    const int j = li[s];
    const int a = (s < cpar) ? 0 : 1;
    const FL3<T>* feat = featb[s - b0];
    // Gamma(e_ij) in delta-space (delta = r_i - r_j)
    FL3<T> gv, ev, gam;
    gv.v = gv.l = ev.v = ev.l = T(0);
#pragma unroll
    for (int t = 0; t < 3; ++t) gv.t[t] = ev.t[t] = T(0);
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const FL3<T> q = feat[h];
      gv.v += q.v * w2[h];
      gv.l += q.l * w2[h];
#pragma unroll
      for (int t = 0; t < 3; ++t) gv.t[t] += q.t[t] * w2[h];
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const FL3<T> q = feat[H + g];
      ev.v += q.v * we[g];
      ev.l += q.l * we[g];
#pragma unroll
      for (int t = 0; t < 3; ++t) ev.t[t] += q.t[t] * we[g];
    }
    fl3_mul(gv, ev, gam);
    // z = P_i + Q_j + e-bar_ij W_c + b ; tangents in r_i and r_j
    const int bj = block_index(w, j, Wc, n, n_up);
    const int64_t prow = hrow, qrow = (int64_t)bj * R5;
    const int64_t pcol = (int64_t)a * d + c, qcol = 2 * (int64_t)d + (int64_t)a * d + c;
    T ebv = T(0), ebt[3] = {T(0), T(0), T(0)}, ebl = T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const FL3<T> q = feat[H + G + k];
      ebv += q.v * wc[a][k];
      ebl += q.l * wc[a][k];
#pragma unroll
      for (int t = 0; t < 3; ++t) ebt[t] += q.t[t] * wc[a][k];
    }
    T zv = (a ? pv[1] : pv[0]) + PQ[qrow * ld4 + qcol] + ebv + bb[a];
    T f, f1, f2;
    silu3<T>(zv, f, f1, f2);
    const T mv = gam.v * f;
    acc.v += mv;
    if (deriv) {
      T zi[3], zj[3], sq = T(0);
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        zi[t] = (a ? pt[1][t] : pt[0][t]) + ebt[t];
        zj[t] = PQ[(qrow + 2 + t) * ld4 + qcol] - ebt[t];
        sq += zi[t] * zi[t] + zj[t] * zj[t];
      }
      const T zl = (a ? pl[1] : pl[0]) + PQ[(qrow + 1) * ld4 + qcol] + T(2) * ebl;
      const T sl = f1 * zl + f2 * sq;
      T cross = T(0);
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        const T si = f1 * zi[t], sj = f1 * zj[t];
        acc.t[t] += gam.t[t] * f + gam.v * si;
        const T xt = -gam.t[t] * f + gam.v * sj;
        X[(xoff + 2 + 3 * (s + 1) + t) * d + c] = xt;
        if (Xb) store_split_bf16(Xb + (xoff + 2 + 3 * (s + 1) + t) * d + c, xcs, xnc, (float)xt);
        cross += gam.t[t] * (si - sj);
      }
      acc.l += T(2) * gam.l * f + T(2) * cross + gam.v * sl;
    }
  }
  }
  X[xoff * d + c] = acc.v;
  if (Xb) store_split_bf16(Xb + xoff * d + c, xcs, xnc, (float)acc.v);
  if (deriv) {
    X[(xoff + 1) * d + c] = acc.l;
    if (Xb) store_split_bf16(Xb + (xoff + 1) * d + c, xcs, xnc, (float)acc.l);
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      X[(xoff + 2 + t) * d + c] = acc.t[t];
      if (Xb) store_split_bf16(Xb + (xoff + 2 + t) * d + c, xcs, xnc, (float)acc.t[t]);
    }
  }
}

// Elementwise SiLU layer in forward-Laplacian form on ragged blocks:
//   y = SiLU(z + b)  (residual: x += y), tangents y_t = SiLU'(z) z_t,
//   Laplacian y_l = SiLU'(z) z_l + SiLU''(z) sum_t z_t^2.
// Block b spans rows off[b] .. off[b+1]-1 (or b*stride .. if off == nullptr).
// One CTA per block; threads stride over the ncol columns.  With yall == 0
// (no residual, split output Yb given) only the value row goes to Y: the
// other rows are consumed through Yb alone.
template <typename T, typename W>
__global__ void __launch_bounds__(256, 4) fl_act_kernel(int ncol, const int64_t* __restrict__ off, int64_t stride,
                              const T* __restrict__ Z, int64_t ldz, const W* bias,
                              T* __restrict__ Y, int64_t ldy, int residual,
                              __nv_bfloat16* __restrict__ Yb = nullptr, int ync = 1, int64_t ycs = 0,
                              int yall = 1) {
  const int b = blockIdx.x;
  int64_t r0, r1;
  if (off) { r0 = off[b]; r1 = off[b + 1]; }
  else { r0 = (int64_t)b * stride; r1 = r0 + stride; }
  const int64_t nr = r1 - r0;
  if (nr <= 0) return;
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
    T z = Z[r0 * ldz + c] + (bias ? T(bias[c]) : T(0));
    T f, f1, f2;
    silu3<T>(z, f, f1, f2);
    T sq = T(0);
    auto put = [&](int64_t q, T v) {
      T o = residual ? Y[q * ldy + c] + v : v;
      if (yall || q == r0) Y[q * ldy + c] = o;
      if (Yb) store_split_bf16(Yb + q * ldy + c, ycs, ync, (float)o);
    };
    // tangent rows, eight at a time: the loads of a group are issued before
    // its stores
    int64_t q = r0 + 2;
    for (; q + 8 <= r1; q += 8) {
      T zt[8], yo[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) zt[u] = Z[(q + u) * ldz + c];
      if (residual) {
#pragma unroll
        for (int u = 0; u < 8; ++u) yo[u] = Y[(q + u) * ldy + c];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        sq += zt[u] * zt[u];
        const T o = residual ? yo[u] + f1 * zt[u] : f1 * zt[u];
        if (yall) Y[(q + u) * ldy + c] = o;
        if (Yb) store_split_bf16(Yb + (q + u) * ldy + c, ycs, ync, (float)o);
      }
    }
    for (; q < r1; ++q) {
      T zt = Z[q * ldz + c];
      sq += zt * zt;
      put(q, f1 * zt);
    }
    if (nr > 1) put(r0 + 1, f1 * Z[(r0 + 1) * ldz + c] + f2 * sq);
    put(r0, f);
  }
}

// fl_act_kernel for float rows, four columns per thread: 128-bit loads and
// stores, eight rows of loads in flight per thread (the layer is bound by
// HBM bandwidth, and one column per thread kept too few bytes in flight).
// CTAs of 64 threads, one block each.  Requires ncol, ldz, ldy and ycs
// multiples of 4 and Z, Y 16-byte, Yb 8-byte aligned (fl_act4_ok).
__device__ __forceinline__ void store_split_bf16x4(__nv_bfloat16* p, int64_t cstride, int nc, float4 v) {
  for (int c = 0; c < nc; ++c) {
    const __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y), h23 = __floats2bfloat162_rn(v.z, v.w);
    uint2 u;
    u.x = *reinterpret_cast<const uint32_t*>(&h01);
    u.y = *reinterpret_cast<const uint32_t*>(&h23);
    *reinterpret_cast<uint2*>(p + c * cstride) = u;
    v.x -= __low2float(h01);
    v.y -= __high2float(h01);
    v.z -= __low2float(h23);
    v.w -= __high2float(h23);
  }
}
inline bool fl_act4_ok(int ncol, int64_t ldz, int64_t ldy, int64_t ycs, const void* Z, const void* Y,
                       const void* Yb) {
  return ncol % 4 == 0 && ldz % 4 == 0 && ldy % 4 == 0 && ycs % 4 == 0 && (reinterpret_cast<uintptr_t>(Z) & 15) == 0 &&
         (reinterpret_cast<uintptr_t>(Y) & 15) == 0 && (reinterpret_cast<uintptr_t>(Yb) & 7) == 0;
}
template <typename W>
__global__ void __launch_bounds__(64, 6) fl_act4_kernel(int ncol, const int64_t* __restrict__ off, int64_t stride,
                                                       const float* __restrict__ Z, int64_t ldz, const W* bias,
                                                       float* __restrict__ Y, int64_t ldy, int residual,
                                                       __nv_bfloat16* __restrict__ Yb, int ync, int64_t ycs,
                                                       int yall) {
  const int b = blockIdx.x;
  int64_t r0, r1;
  if (off) { r0 = off[b]; r1 = off[b + 1]; }
  else { r0 = (int64_t)b * stride; r1 = r0 + stride; }
  const int64_t nr = r1 - r0;
  if (nr <= 0) return;
  auto ld4 = [](const float* p) { return *reinterpret_cast<const float4*>(p); };
  for (int c = 4 * threadIdx.x; c < ncol; c += 4 * blockDim.x) {
    float4 z = ld4(Z + r0 * ldz + c);
    if (bias) { z.x += float(bias[c]); z.y += float(bias[c + 1]); z.z += float(bias[c + 2]); z.w += float(bias[c + 3]); }
    float f[4], f1[4], f2[4];
    silu3<float>(z.x, f[0], f1[0], f2[0]);
    silu3<float>(z.y, f[1], f1[1], f2[1]);
    silu3<float>(z.z, f[2], f1[2], f2[2]);
    silu3<float>(z.w, f[3], f1[3], f2[3]);
    float4 sq = make_float4(0.f, 0.f, 0.f, 0.f);
    auto put = [&](int64_t q, float4 o) {
      if (residual) {
        const float4 y = ld4(Y + q * ldy + c);
        o.x += y.x; o.y += y.y; o.z += y.z; o.w += y.w;
      }
      if (yall || q == r0) *reinterpret_cast<float4*>(Y + q * ldy + c) = o;
      if (Yb) store_split_bf16x4(Yb + q * ldy + c, ycs, ync, o);
    };
    // tangent rows, eight at a time: the loads of a group are issued before
    // its stores
    int64_t q = r0 + 2;
    for (; q + 8 <= r1; q += 8) {
      float4 zt[8], yo[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) zt[u] = ld4(Z + (q + u) * ldz + c);
      if (residual) {
#pragma unroll
        for (int u = 0; u < 8; ++u) yo[u] = ld4(Y + (q + u) * ldy + c);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        sq.x += zt[u].x * zt[u].x; sq.y += zt[u].y * zt[u].y; sq.z += zt[u].z * zt[u].z; sq.w += zt[u].w * zt[u].w;
        float4 o;
        if (residual)
          o = make_float4(yo[u].x + f1[0] * zt[u].x, yo[u].y + f1[1] * zt[u].y, yo[u].z + f1[2] * zt[u].z,
                          yo[u].w + f1[3] * zt[u].w);
        else
          o = make_float4(f1[0] * zt[u].x, f1[1] * zt[u].y, f1[2] * zt[u].z, f1[3] * zt[u].w);
        if (yall) *reinterpret_cast<float4*>(Y + (q + u) * ldy + c) = o;
        if (Yb) store_split_bf16x4(Yb + (q + u) * ldy + c, ycs, ync, o);
      }
    }
    for (; q < r1; ++q) {
      const float4 zt = ld4(Z + q * ldz + c);
      sq.x += zt.x * zt.x; sq.y += zt.y * zt.y; sq.z += zt.z * zt.z; sq.w += zt.w * zt.w;
      put(q, make_float4(f1[0] * zt.x, f1[1] * zt.y, f1[2] * zt.z, f1[3] * zt.w));
    }
    if (nr > 1) {
      const float4 zl = ld4(Z + (r0 + 1) * ldz + c);
      put(r0 + 1, make_float4(f1[0] * zl.x + f2[0] * sq.x, f1[1] * zl.y + f2[1] * sq.y, f1[2] * zl.z + f2[2] * sq.z,
                              f1[3] * zl.w + f2[3] * sq.w));
    }
    put(r0, make_float4(f[0], f[1], f[2], f[3]));
  }
}

// The last activation of a readout MLP fused with its readout vector:
// F[q] = sum_c SiLU-layer(Z + b)[q][c] * wv[c] for every row q of every block
// (same forward-Laplacian rules as fl_act_kernel), without storing the
// activated rows.  One CTA per block, threads over the columns; the per-row
// sums go through warp reductions (32 tangent rows at a time) and a
// [warps][rows] shared array, summed in warp order.  Dynamic shared memory:
// (blockDim / 32) * max_rows floats.
template <typename T, typename W>
__global__ void fl_act_dot_kernel(int ncol, const int64_t* __restrict__ off, int64_t stride,
                                  const T* __restrict__ Z, int64_t ldz, const W* bias, const W* wv,
                                  T* __restrict__ F, int max_rows) {
  extern __shared__ unsigned char fd_smem[];
  T* red = reinterpret_cast<T*>(fd_smem);
  const int b = blockIdx.x;
  int64_t r0, r1;
  if (off) { r0 = off[b]; r1 = off[b + 1]; }
  else { r0 = (int64_t)b * stride; r1 = r0 + stride; }
  const int nr = (int)(r1 - r0);
  if (nr <= 0) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // per-thread column partials of one row, reduced over the warp
  auto emit = [&](int rl, T part) {
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) red[wid * max_rows + rl] = part;
  };
  // columns in passes of blockDim (one column per thread per pass)
  for (int c0 = 0; c0 < ncol; c0 += blockDim.x) {
    const int c = c0 + threadIdx.x;
    const bool in = c < ncol;
    T f = T(0), f1 = T(0), f2 = T(0), w = T(0);
    if (in) {
      const T z = Z[r0 * ldz + c] + (bias ? T(bias[c]) : T(0));
      silu3<T>(z, f, f1, f2);
      w = T(wv[c]);
    }
    T sq = T(0);
    // tangent rows 32 at a time: the loads of a group are in flight
    // together, and a transpose-halving reduction (at each step a lane keeps
    // half of its partials and adds its partner's copy of them) leaves lane L
    // with the warp sum of row qb + L: 31 shuffles per 32 rows
    for (int qb = 2; qb < nr; qb += 32) {
      T a[32];
#pragma unroll
      for (int u = 0; u < 32; ++u) {
        const int q = qb + u;
        const T zt = (in && q < nr) ? Z[(r0 + q) * ldz + c] : T(0);
        sq += zt * zt;
        a[u] = f1 * zt * w;
      }
#pragma unroll
      for (int sft = 16; sft >= 1; sft >>= 1) {
        const bool up = (lane & sft) != 0;
#pragma unroll
        for (int k = 0; k < sft; ++k) {
          const T send = up ? a[k] : a[k + sft];
          const T keep = up ? a[k + sft] : a[k];
          a[k] = keep + __shfl_xor_sync(0xffffffffu, send, sft);
        }
      }
      const int q = qb + lane;
      if (q < nr) red[wid * max_rows + q] = a[0] + (c0 > 0 ? red[wid * max_rows + q] : T(0));
    }
    if (nr > 1) {
      T part = (in ? (f1 * Z[(r0 + 1) * ldz + c] + f2 * sq) : T(0)) * w;
      if (c0 > 0) part += red[wid * max_rows + 1] * (lane == 0 ? T(1) : T(0));
      emit(1, part);
    }
    T part = f * w;
    if (c0 > 0) part += red[wid * max_rows] * (lane == 0 ? T(1) : T(0));
    emit(0, part);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nr; q += blockDim.x) {
    T sum = T(0);
    for (int g = 0; g < nw; ++g) sum += red[g * max_rows + q];
    F[r0 + q] = sum;
  }
}

// out[row] = Y[row] . w for rows [r_begin, r_end) (device range or host).
template <typename T, typename W>
__global__ void rowdot_kernel(const T* __restrict__ Y, int64_t ldy, int ncol, const W* wv,
                              T* __restrict__ out, const int64_t* range, int64_t r_begin,
                              int64_t r_end) {
  int64_t b = r_begin, e = r_end;
  if (range) { b = range[0]; e = range[1]; }
  const int64_t row = b + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (row >= e) return;
  T s = T(0);
  for (int c = lane; c < ncol; c += 32) s += Y[row * ldy + c] * T(wv[c]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[row] = s;
}

// Copies the value row of every electron block into a dense [Wc*n][d] matrix
// (block order).
template <typename T>
__global__ void gather_value_rows_kernel(int nb, int d, const int64_t* __restrict__ off,
                                         const T* __restrict__ X, T* __restrict__ Hv, int64_t ldx = -1,
                                         __nv_bfloat16* __restrict__ Hb = nullptr, int hnc = 0, int64_t hcs = 0) {
  const int b = blockIdx.x;
  const int64_t r0 = off[b];
  const int64_t ld = ldx < 0 ? d : ldx;
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    const T v = X[r0 * ld + c];
    if (Hv) Hv[(int64_t)b * d + c] = v;
    if (Hb) store_split_bf16(Hb + (int64_t)b * d + c, hcs, hnc, (float)v);
  }
}

// Writes dense rows back into the value row of every block: Z[off[b]] = Zv[b].
template <typename T>
__global__ void scatter_value_rows_kernel(int N, const int64_t* __restrict__ off, const T* __restrict__ Zv,
                                          T* __restrict__ Z, int64_t ldz) {
  const int b = blockIdx.x;
  const int64_t r0 = off[b];
  for (int c = threadIdx.x; c < N; c += blockDim.x) Z[r0 * ldz + c] = Zv[(int64_t)b * N + c];
}

}  // namespace fire

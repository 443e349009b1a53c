// Jastrow factors, Coulomb potential and the final local-energy reduction.
//
// J_MLP = exp(sum_i MLP1(h_i)) * sum_i MLP2(h_i); J_att = exp(MLP1(V)) MLP2(V)
// with V = Concat_r softmax(H q_r)^T H W^V_r; J_cusp = exp(sum_{i<j}
// w a^2 / (a + r_ij)) (Methods, "Global electron correlation effects").  The
// factors multiply Psi (Methods eq. wf), so their logs add.
// V(r) and E_L follow Methods eq. hamiltonian and the E_L equation.
#pragma once

#include "common.cuh"

namespace fire {

template <typename T>
__device__ __forceinline__ T bsum_any(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = T(0);
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
  return s;
}

// Row of the tangent (np, x) inside electron i's block, where i is np itself
// (slot 0) or the k-th entry of np's list (slot rev + 1).
__device__ __forceinline__ int64_t tangent_row(const int64_t* blk_off, int b, int slot, int x) {
  return blk_off[b] + 2 + 3 * slot + x;
}

// Sums of the per-electron Jastrow MLP outputs.  One CTA per walker.
template <typename T, typename W>
__global__ void jmlp_reduce_kernel(int Wc, int n, int n_up, int K, const int32_t* __restrict__ idx,
                                   const int32_t* __restrict__ cnt, const int32_t* __restrict__ rev,
                                   const int64_t* __restrict__ blk_off, const T* __restrict__ F1,
                                   const T* __restrict__ F2, const W* b31, const W* b32,
                                   T* jval, T* jsign, T* jgrad, T* jlap, int deriv) {
  __shared__ T red[32];
  const int w = blockIdx.x;
  T s1 = T(0), s2 = T(0), l1 = T(0), l2 = T(0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int64_t o = blk_off[block_index(w, i, Wc, n, n_up)];
    s1 += F1[o] + T(b31[0]);
    s2 += F2[o] + T(b32[0]);
    if (deriv) { l1 += F1[o + 1]; l2 += F2[o + 1]; }
  }
  s1 = bsum_any(s1, red);
  s2 = bsum_any(s2, red);
  if (!deriv) {
    if (threadIdx.x == 0) {
      jval[w] = s1 + dlog<T>(fabs(s2));
      jsign[w] = s2 > T(0) ? T(1) : (s2 < T(0) ? T(-1) : T(0));
    }
    return;
  }
  l1 = bsum_any(l1, red);
  l2 = bsum_any(l2, red);
  T gsq = T(0);
  for (int q = threadIdx.x; q < 3 * n; q += blockDim.x) {
    const int np = q / 3, x = q % 3;
    const int64_t base = (int64_t)w * n + np;
    const int bn = block_index(w, np, Wc, n, n_up);
    const int64_t r0 = tangent_row(blk_off, bn, 0, x);
    T a = F1[r0], b = F2[r0];
    const int ct = cnt[base * 2] + cnt[base * 2 + 1];
    for (int k = 0; k < ct; ++k) {
      const int i = idx[base * K + k];
      const int rv = rev[base * K + k];
      if (rv < 0) continue;
      const int64_t rr = tangent_row(blk_off, block_index(w, i, Wc, n, n_up), rv + 1, x);
      a += F1[rr];
      b += F2[rr];
    }
    jgrad[(int64_t)w * 3 * n + q] = a + b / s2;
    gsq += b * b;
  }
  gsq = bsum_any(gsq, red);
  if (threadIdx.x == 0) {
    jval[w] = s1 + dlog<T>(fabs(s2));
    jsign[w] = s2 > T(0) ? T(1) : (s2 < T(0) ? T(-1) : T(0));
    jlap[w] = l1 + l2 / s2 - gsq / (s2 * s2);
  }
}

// Attention registers V with its 3n tangents and Laplacian.  One CTA per
// walker, one thread per column of V (n_reg * d_reg columns).  SU holds the
// scores h_i . q_r in columns [0, R) and u_i = h_i W^V in [R, R + R*dr)
// (row stride ld).
template <typename T>
__global__ void att_pool_kernel(int Wc, int n, int n_up, int K, int R, int dr,
                                const int32_t* __restrict__ idx, const int32_t* __restrict__ cnt,
                                const int32_t* __restrict__ rev, const int64_t* __restrict__ blk_off,
                                const T* __restrict__ SU, int64_t ld, T* __restrict__ V, int deriv) {
  extern __shared__ unsigned char ap_smem[];
  T* smax = reinterpret_cast<T*>(ap_smem);   // [R]
  T* ex = smax + R;                          // [n][R]
  const int w = blockIdx.x;
  const int RD = R * dr;
  const int col = threadIdx.x;
  const int rg = col / dr;
  const int64_t vstride = deriv ? (2 + 3 * (int64_t)n) : 1;
  T* Vw = V + (int64_t)w * vstride * RD;
  for (int q = threadIdx.x; q < R; q += blockDim.x) {
    T m = -INFINITY;
    for (int i = 0; i < n; ++i) {
      const int64_t o = blk_off[block_index(w, i, Wc, n, n_up)];
      m = fmax(m, SU[o * ld + q]);
    }
    smax[q] = m;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * R; e += blockDim.x) {
    const int i = e / R, q = e % R;
    const int64_t o = blk_off[block_index(w, i, Wc, n, n_up)];
    ex[e] = dexp<T>(SU[o * ld + q] - smax[q]);
  }
  __syncthreads();
  if (col >= RD) return;
  T Z = T(0), Nv = T(0), ZL = T(0), NL = T(0);
  for (int i = 0; i < n; ++i) {
    const int64_t o = blk_off[block_index(w, i, Wc, n, n_up)];
    const T e = ex[i * R + rg];
    const T u = SU[o * ld + R + col];
    Z += e;
    Nv += e * u;
    if (deriv) {
      const int64_t o1 = blk_off[block_index(w, i, Wc, n, n_up) + 1];
      T ss = T(0), su = T(0);
      for (int64_t q = o + 2; q < o1; ++q) {
        const T st = SU[q * ld + rg];
        ss += st * st;
        su += st * SU[q * ld + R + col];
      }
      const T sl = SU[(o + 1) * ld + rg], ul = SU[(o + 1) * ld + R + col];
      ZL += e * (sl + ss);
      NL += e * ((sl + ss) * u + T(2) * su + ul);
    }
  }
  const T v = Nv / Z;
  Vw[col] = v;
  if (!deriv) return;
  T A1 = T(0), A2 = T(0);
  for (int q = 0; q < 3 * n; ++q) {
    const int np = q / 3, x = q % 3;
    const int64_t base = (int64_t)w * n + np;
    const int bn = block_index(w, np, Wc, n, n_up);
    const int64_t r0 = tangent_row(blk_off, bn, 0, x);
    const int64_t ov = blk_off[bn];
    T e = ex[np * R + rg];
    T st = SU[r0 * ld + rg];
    T dZ = e * st;
    T dN = e * (st * SU[ov * ld + R + col] + SU[r0 * ld + R + col]);
    const int ct = cnt[base * 2] + cnt[base * 2 + 1];
    for (int k = 0; k < ct; ++k) {
      const int i = idx[base * K + k];
      const int rv = rev[base * K + k];
      if (rv < 0) continue;
      const int bi = block_index(w, i, Wc, n, n_up);
      const int64_t rr = tangent_row(blk_off, bi, rv + 1, x);
      const int64_t oi = blk_off[bi];
      e = ex[i * R + rg];
      st = SU[rr * ld + rg];
      dZ += e * st;
      dN += e * (st * SU[oi * ld + R + col] + SU[rr * ld + R + col]);
    }
    Vw[(2 + q) * RD + col] = dN / Z - Nv * dZ / (Z * Z);
    A1 += dN * dZ;
    A2 += dZ * dZ;
  }
  Vw[RD + col] = NL / Z - T(2) * A1 / (Z * Z) - Nv * ZL / (Z * Z) + T(2) * Nv * A2 / (Z * Z * Z);
}

// The same registers V with tangents and Laplacian, spread over electrons
// (the single-CTA form above walks every forward-Laplacian row of a walker
// serially).  Three launches:
//   att_max_kernel   per walker, the largest score of each register r (the
//                    softmax shift);
//   att_part_kernel  one CTA per electron i (blockDim == R*dr), writing a
//                    record of 12 rows of R*dr columns:
//                      0 e_i, 1 e_i u_i, 2 e_i (Lap s_i + |grad s_i|^2),
//                      3 e_i ((Lap s_i + |grad s_i|^2) u_i + 2 grad s_i.grad u_i + Lap u_i),
//                      4 sum_x dN_x dZ_x, 5 sum_x dZ_x^2,
//                      6..8 dZ_x, 9..11 dN_x   (x = the three coordinates of r_i),
//                    where e_i = exp(s_ir - max_r), Z = sum_i e_i, N = sum_i e_i u_i
//                    and dZ_x, dN_x their derivatives with respect to r_ix
//                    (only electrons of Nbar_i contribute);
//   att_fin_kernel   grid (walker, electron slice): the sums over electrons
//                    in ascending order, then V = N / Z, its Laplacian
//                      Lap N / Z - 2 grad N . grad Z / Z^2 - N Lap Z / Z^2 + 2 N |grad Z|^2 / Z^3
//                    and the tangent rows dN/Z - N dZ / Z^2 of the slice.
// AP holds Wc*R shifts followed by the Wc*n records (electron order).
template <typename T>
__global__ void att_max_kernel(int Wc, int n, int n_up, int R, const int64_t* __restrict__ blk_off,
                               const T* __restrict__ SU, int64_t ld, T* __restrict__ AP) {
  const int w = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = wid; q < R; q += nw) {
    T m = -INFINITY;
    for (int i = lane; i < n; i += 32) m = fmax(m, SU[blk_off[block_index(w, i, Wc, n, n_up)] * ld + q]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) AP[(int64_t)w * R + q] = m;
  }
}

template <typename T>
__global__ void att_part_kernel(int Wc, int n, int n_up, int K, int R, int dr, const int32_t* __restrict__ idx,
                                const int32_t* __restrict__ cnt, const int32_t* __restrict__ rev,
                                const int64_t* __restrict__ blk_off, const T* __restrict__ SU, int64_t ld,
                                T* __restrict__ AP) {
  constexpr int NBAT = 32;   // neighbours whose rows are located together
  __shared__ int64_t s_rr[NBAT], s_oj[NBAT];
  const int RD = R * dr;
  const int col = threadIdx.x;
  const bool act = col < RD;   // every thread takes the barriers below
  const int colc = act ? col : 0;
  const int w = blockIdx.x / n, i = blockIdx.x % n;
  const int rg = colc / dr;
  const T mx = AP[(int64_t)w * R + rg];
  T* rec = AP + (int64_t)Wc * R + (int64_t)blockIdx.x * 12 * RD;
  const int bi = block_index(w, i, Wc, n, n_up);
  const int64_t o = blk_off[bi], o1 = blk_off[bi + 1];
  const T e = dexp<T>(SU[o * ld + rg] - mx);
  const T u = SU[o * ld + R + colc];
  // tangent rows eight at a time (independent partial sums keep the loads
  // in flight), summed in a fixed order
  T ss4[4] = {T(0), T(0), T(0), T(0)}, su4[4] = {T(0), T(0), T(0), T(0)};
  int64_t q = o + 2;
  for (; q + 8 <= o1; q += 8) {
    T st[8], ut[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      st[v] = SU[(q + v) * ld + rg];
      ut[v] = SU[(q + v) * ld + R + colc];
    }
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      ss4[v & 3] += st[v] * st[v];
      su4[v & 3] += st[v] * ut[v];
    }
  }
  for (int v = 0; q < o1; ++q, ++v) {
    const T st = SU[q * ld + rg];
    ss4[v & 3] += st * st;
    su4[v & 3] += st * SU[q * ld + R + colc];
  }
  const T ss = (ss4[0] + ss4[1]) + (ss4[2] + ss4[3]), su = (su4[0] + su4[1]) + (su4[2] + su4[3]);
  const T sl = SU[(o + 1) * ld + rg], ul = SU[(o + 1) * ld + R + colc];
  if (act) {
    rec[0 * RD + col] = e;
    rec[1 * RD + col] = e * u;
    rec[2 * RD + col] = e * (sl + ss);
    rec[3 * RD + col] = e * ((sl + ss) * u + T(2) * su + ul);
  }
  // tangents with respect to r_i: electron i itself (slot 0) and every j
  // that has i in its list (slot rev + 1).  The rows of a batch of such j
  // are located first (one thread each: list, reverse slot, block offset),
  // so the loop below issues only independent row loads.
  T dZ[3], dN[3];
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    const T st = SU[(o + 2 + x) * ld + rg];
    dZ[x] = e * st;
    dN[x] = e * (st * u + SU[(o + 2 + x) * ld + R + colc]);
  }
  const int64_t base = (int64_t)w * n + i;
  const int ct = cnt[base * 2] + cnt[base * 2 + 1];
  for (int k0 = 0; k0 < ct; k0 += NBAT) {
    const int nbat = min(NBAT, ct - k0);
    __syncthreads();   // the previous batch is consumed
    if (threadIdx.x < nbat) {
      const int k = k0 + threadIdx.x;
      const int j = idx[base * K + k];
      const int rv = rev[base * K + k];
      if (rv < 0) {
        s_oj[threadIdx.x] = -1;
      } else {
        const int64_t oj = blk_off[block_index(w, j, Wc, n, n_up)];
        s_oj[threadIdx.x] = oj;
        s_rr[threadIdx.x] = oj + 2 + 3 * (int64_t)(rv + 1);
      }
    }
    __syncthreads();
    for (int k = 0; k < nbat; ++k) {
      const int64_t oj = s_oj[k];
      if (oj < 0) continue;
      const int64_t rr = s_rr[k];
      const T ej = dexp<T>(SU[oj * ld + rg] - mx);
      const T uj = SU[oj * ld + R + colc];
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        const T st = SU[(rr + x) * ld + rg];
        dZ[x] += ej * st;
        dN[x] += ej * (st * uj + SU[(rr + x) * ld + R + colc]);
      }
    }
  }
  if (!act) return;
  T a1 = T(0), a2 = T(0);
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    a1 += dN[x] * dZ[x];
    a2 += dZ[x] * dZ[x];
    rec[(6 + x) * RD + col] = dZ[x];
    rec[(9 + x) * RD + col] = dN[x];
  }
  rec[4 * RD + col] = a1;
  rec[5 * RD + col] = a2;
}

template <typename T>
__global__ void att_fin_kernel(int Wc, int n, int R, int dr, const T* __restrict__ AP, T* __restrict__ V,
                               __nv_bfloat16* __restrict__ Vb = nullptr, int vnc = 0, int64_t vcs = 0) {
  const int RD = R * dr;
  const int col = threadIdx.x;
  if (col >= RD) return;
  const int w = blockIdx.x;
  const T* recw = AP + (int64_t)Wc * R + (int64_t)w * n * 12 * RD;
  T sm[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  for (int i = 0; i < n; ++i) {
    const T* rec = recw + (int64_t)i * 12 * RD;
#pragma unroll
    for (int q = 0; q < 6; ++q) sm[q] += rec[q * RD + col];
  }
  const T Z = sm[0], Nv = sm[1], ZL = sm[2], NL = sm[3], A1 = sm[4], A2 = sm[5];
  const int64_t vo = (int64_t)w * (2 + 3 * (int64_t)n) * RD;
  T* Vw = V + vo;
  auto put = [&](int64_t e, T v) {
    Vw[e] = v;
    if (Vb) store_split_bf16(Vb + vo + e, vcs, vnc, (float)v);
  };
  if (blockIdx.y == 0) {
    put(col, Nv / Z);
    put(RD + col, NL / Z - T(2) * A1 / (Z * Z) - Nv * ZL / (Z * Z) + T(2) * Nv * A2 / (Z * Z * Z));
  }
  const int per = (n + gridDim.y - 1) / gridDim.y;
  const int i0 = blockIdx.y * per, i1 = min(n, i0 + per);
  for (int i = i0; i < i1; ++i) {
    const T* rec = recw + (int64_t)i * 12 * RD;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      const T dZ = rec[(6 + x) * RD + col], dN = rec[(9 + x) * RD + col];
      put((2 + 3 * (int64_t)i + x) * RD + col, dN / Z - Nv * dZ / (Z * Z));
    }
  }
}

// log|J_att| from the two readouts of V.  One CTA per walker.
template <typename T, typename W>
__global__ void att_reduce_kernel(int n, const T* __restrict__ G1, const T* __restrict__ G2,
                                  const W* b31, const W* b32, T* aval, T* asign, T* agrad, T* alap,
                                  int deriv) {
  __shared__ T red[32];
  const int w = blockIdx.x;
  const int64_t vstride = deriv ? (2 + 3 * (int64_t)n) : 1;
  const T* g1 = G1 + (int64_t)w * vstride;
  const T* g2 = G2 + (int64_t)w * vstride;
  const T v1 = g1[0] + T(b31[0]), v2 = g2[0] + T(b32[0]);
  if (deriv) {
    T gsq = T(0);
    for (int q = threadIdx.x; q < 3 * n; q += blockDim.x) {
      const T b = g2[2 + q];
      agrad[(int64_t)w * 3 * n + q] = g1[2 + q] + b / v2;
      gsq += b * b;
    }
    gsq = bsum_any(gsq, red);
    if (threadIdx.x == 0) alap[w] = g1[1] + g2[1] / v2 - gsq / (v2 * v2);
  }
  if (threadIdx.x == 0) {
    aval[w] = v1 + dlog<T>(fabs(v2));
    asign[w] = v2 > T(0) ? T(1) : (v2 < T(0) ? T(-1) : T(0));
  }
}

// Coulomb potential and the cusp Jastrow with its gradient and Laplacian.
// One CTA per walker.
template <typename T, typename W>
__global__ void coulomb_cusp_kernel(int n, int n_up, int N, const double* __restrict__ r,
                                    const double* __restrict__ R, const double* __restrict__ Zc,
                                    const W* cusp, T* vpot, T* cval, T* cgrad, T* clap, int deriv) {
  __shared__ T red[32];
  const int w = blockIdx.x;
  const double* rw = r + (int64_t)w * n * 3;
  const T wp = T(cusp[0]), wa = T(cusp[1]), ap = T(cusp[2]), aa = T(cusp[3]);
  T vee = T(0), ven = T(0), jc = T(0), lap = T(0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    T g[3] = {T(0), T(0), T(0)};
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      T d[3] = {T(rw[3 * i] - rw[3 * j]), T(rw[3 * i + 1] - rw[3 * j + 1]), T(rw[3 * i + 2] - rw[3 * j + 2])};
      T rr = dsqrt<T>(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      const bool same = ((i < n_up) == (j < n_up));
      const T om = same ? wp : wa, al = same ? ap : aa;
      const T den = al + rr;
      const T u = om * al * al / den;
      const T u1 = -om * al * al / (den * den);
      const T u2 = T(2) * om * al * al / (den * den * den);
      if (j > i) { vee += T(1) / rr; jc += u; }
      for (int t = 0; t < 3; ++t) g[t] += u1 * d[t] / rr;
      lap += u2 + T(2) * u1 / rr;
    }
    for (int m = 0; m < N; ++m) {
      T d[3] = {T(rw[3 * i] - R[3 * m]), T(rw[3 * i + 1] - R[3 * m + 1]), T(rw[3 * i + 2] - R[3 * m + 2])};
      ven -= T(Zc[m]) / dsqrt<T>(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    }
    if (deriv)
      for (int t = 0; t < 3; ++t) cgrad[((int64_t)w * n + i) * 3 + t] = g[t];
  }
  T vnn = T(0);
  if (threadIdx.x == 0) {
    for (int m = 0; m < N; ++m)
      for (int k = m + 1; k < N; ++k) {
        T d[3] = {T(R[3 * m] - R[3 * k]), T(R[3 * m + 1] - R[3 * k + 1]), T(R[3 * m + 2] - R[3 * k + 2])};
        vnn += T(Zc[m]) * T(Zc[k]) / dsqrt<T>(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      }
  }
  T v = bsum_any(vee + ven + vnn, red);
  jc = bsum_any(jc, red);
  lap = bsum_any(lap, red);
  if (threadIdx.x == 0) {
    vpot[w] = v;
    cval[w] = jc;
    if (deriv) clap[w] = lap;
  }
}

// Final per-walker combination.  RT is float64 for the FP64 and BF16_FP64
// forms and float32 for plain FP32.  One CTA per walker.
template <typename T, typename RT>
struct FinalIn {
  const double *ldabs, *lsign;              // [Wc][D]
  const T *gdet, *ldet;                     // [Wc][D][n][3], [Wc][D][n]
  const T *cval, *cgrad, *clap;             // cusp
  const T *jval, *jsign, *jgrad, *jlap;     // MLP Jastrow
  const T *aval, *asign, *agrad, *alap;     // attention Jastrow
  const T* vpot;
};

template <typename T, typename RT>
__global__ void final_kernel(int n, int D, uint32_t flags, FinalIn<T, RT> in, int deriv,
                             double* e_loc, double* logabs, double* sign, double* e_kin,
                             double* e_pot, DevStatus* st) {
  __shared__ RT red[32];
  __shared__ RT s_om[64];
  __shared__ RT s_lmax, s_S;
  const int w = blockIdx.x;
  if (threadIdx.x == 0) {
    RT lmax = -INFINITY;
    for (int d = 0; d < D; ++d) {
      RT l = RT(in.ldabs[(int64_t)w * D + d]);
      if (in.lsign[(int64_t)w * D + d] != 0.0 && l > lmax) lmax = l;
    }
    if (!(lmax > -INFINITY)) lmax = RT(0);
    RT S = RT(0);
    for (int d = 0; d < D; ++d) {
      RT sg = RT(in.lsign[(int64_t)w * D + d]);
      RT t = (sg != RT(0)) ? sg * exp(RT(in.ldabs[(int64_t)w * D + d]) - lmax) : RT(0);
      s_om[d] = t;
      S += t;
    }
    for (int d = 0; d < D; ++d) s_om[d] /= S;
    s_lmax = lmax;
    s_S = S;
  }
  __syncthreads();
  const RT S = s_S;
  RT la = s_lmax + log(fabs(S));
  RT sg = S > RT(0) ? RT(1) : (S < RT(0) ? RT(-1) : RT(0));
  if (flags & FIRE_J_CUSP) la += RT(in.cval[w]);
  if (flags & FIRE_J_MLP) { la += RT(in.jval[w]); sg *= RT(in.jsign[w]); }
  if (flags & FIRE_J_ATT) { la += RT(in.aval[w]); sg *= RT(in.asign[w]); }
  if (!deriv) {
    if (threadIdx.x == 0) {
      logabs[w] = (double)la;
      sign[w] = (double)sg;
      if (sg == RT(0)) atomicAdd(&st->n_nodes, 1);
    }
    return;
  }
  RT lapd = RT(0), g2 = RT(0), gd2 = RT(0);
  for (int q = threadIdx.x; q < 3 * n; q += blockDim.x) {
    RT gq = RT(0);
    for (int d = 0; d < D; ++d) {
      const RT gdq = RT(in.gdet[((int64_t)w * D + d) * 3 * n + q]);
      gq += s_om[d] * gdq;
      lapd += s_om[d] * gdq * gdq;
    }
    gd2 += gq * gq;
    if (flags & FIRE_J_CUSP) gq += RT(in.cgrad[(int64_t)w * 3 * n + q]);
    if (flags & FIRE_J_MLP) gq += RT(in.jgrad[(int64_t)w * 3 * n + q]);
    if (flags & FIRE_J_ATT) gq += RT(in.agrad[(int64_t)w * 3 * n + q]);
    g2 += gq * gq;
  }
  for (int q = threadIdx.x; q < n; q += blockDim.x)
    for (int d = 0; d < D; ++d) lapd += s_om[d] * RT(in.ldet[((int64_t)w * D + d) * n + q]);
  lapd = bsum_any(lapd, red);
  g2 = bsum_any(g2, red);
  gd2 = bsum_any(gd2, red);
  if (threadIdx.x == 0) {
    RT lap = lapd - gd2;
    if (flags & FIRE_J_CUSP) lap += RT(in.clap[w]);
    if (flags & FIRE_J_MLP) lap += RT(in.jlap[w]);
    if (flags & FIRE_J_ATT) lap += RT(in.alap[w]);
    const RT kin = RT(-0.5) * (lap + g2);
    const RT v = RT(in.vpot[w]);
    const RT e = kin + v;
    e_loc[w] = (double)e;
    logabs[w] = (double)la;
    sign[w] = (double)sg;
    if (e_kin) e_kin[w] = (double)kin;
    if (e_pot) e_pot[w] = (double)v;
    const bool node = (sg == RT(0));
    if (node) atomicAdd(&st->n_nodes, 1);
    else if (!isfinite((double)e)) atomicAdd(&st->n_nonfinite, 1);
  }
}

}  // namespace fire

// Building blocks of the per-walker parameter gradient (adjoint).
#pragma once

#include "common.cuh"

namespace fire {

// Per-walker transposed product: for every walker w (grid.z)
//   C_w[a][b] (+)= sum_{i < ni} X[w*sx + i*ldx + a] * Y[w*sy + i*ldy + b]
// with C_w = C + w*sc (row stride ldc).  This is the outer-product sum over a
// walker's electrons that gives a weight gradient.  Tiles 32 x 32, 256 threads.
template <typename T>
__global__ void __launch_bounds__(256)
tn_batched_kernel(int Na, int Nb, int ni, const T* __restrict__ X, int64_t ldx, int64_t sx,
                  const T* __restrict__ Y, int64_t ldy, int64_t sy, T* __restrict__ C, int64_t ldc, int64_t sc,
                  int accumulate) {
  __shared__ T xs[32][33];
  __shared__ T ys[32][33];
  const int w = blockIdx.z;
  const int a0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
  const T* Xw = X + (int64_t)w * sx;
  const T* Yw = Y + (int64_t)w * sy;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;   // 2 x 2 outputs per thread
  T acc[2][2] = {{T(0), T(0)}, {T(0), T(0)}};
  for (int i0 = 0; i0 < ni; i0 += 32) {
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
      const int r = e / 32, c = e % 32;
      const int i = i0 + r;
      xs[r][c] = (i < ni && a0 + c < Na) ? Xw[(int64_t)i * ldx + a0 + c] : T(0);
      ys[r][c] = (i < ni && b0 + c < Nb) ? Yw[(int64_t)i * ldy + b0 + c] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
      const T x0 = xs[r][2 * ty], x1 = xs[r][2 * ty + 1];
      const T y0 = ys[r][2 * tx], y1 = ys[r][2 * tx + 1];
      acc[0][0] += x0 * y0;
      acc[0][1] += x0 * y1;
      acc[1][0] += x1 * y0;
      acc[1][1] += x1 * y1;
    }
    __syncthreads();
  }
  T* Cw = C + (int64_t)w * sc;
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int a = a0 + 2 * ty + p, b = b0 + 2 * tx + q;
      if (a < Na && b < Nb) {
        T* o = Cw + (int64_t)a * ldc + b;
        *o = accumulate ? *o + acc[p][q] : acc[p][q];
      }
    }
}

template <typename T>
inline void tn_batched(cudaStream_t s, int W, int Na, int Nb, int ni, const T* X, int64_t ldx, int64_t sx,
                       const T* Y, int64_t ldy, int64_t sy, T* C, int64_t ldc, int64_t sc, bool accumulate) {
  if (W <= 0 || Na <= 0 || Nb <= 0 || ni <= 0) return;
  dim3 grid((unsigned)((Na + 31) / 32), (unsigned)((Nb + 31) / 32), (unsigned)W);
  tn_batched_kernel<T><<<grid, 256, 0, s>>>(Na, Nb, ni, X, ldx, sx, Y, ldy, sy, C, ldc, sc, accumulate ? 1 : 0);
}

// C_w[b] (+)= sum_{i < ni} Y[w*sy + i*ldy + b]  (bias gradients).
template <typename T>
__global__ void colsum_batched_kernel(int Nb, int ni, const T* __restrict__ Y, int64_t ldy, int64_t sy,
                                      T* __restrict__ C, int64_t sc, int accumulate) {
  const int w = blockIdx.y;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= Nb) return;
  const T* Yw = Y + (int64_t)w * sy;
  T acc = T(0);
  for (int i = 0; i < ni; ++i) acc += Yw[(int64_t)i * ldy + b];
  T* o = C + (int64_t)w * sc + b;
  *o = accumulate ? *o + acc : acc;
}

template <typename T>
inline void colsum_batched(cudaStream_t s, int W, int Nb, int ni, const T* Y, int64_t ldy, int64_t sy, T* C,
                           int64_t sc, bool accumulate) {
  if (W <= 0 || Nb <= 0 || ni <= 0) return;
  dim3 grid((unsigned)((Nb + 127) / 128), (unsigned)W);
  colsum_batched_kernel<T><<<grid, 128, 0, s>>>(Nb, ni, Y, ldy, sy, C, sc, accumulate ? 1 : 0);
}

// Elementwise helpers over dense [rows][ncol] matrices.
// mode 0: out = d * SiLU'(z + b)           (back through y = SiLU(z + b))
// mode 1: out = d * SiLU(z + b)            (used by products)
template <typename T, typename W>
__global__ void silu_bwd_kernel(int64_t rows, int ncol, const T* __restrict__ D, int64_t ldd,
                                const T* __restrict__ Z, int64_t ldz, const W* bias, T* __restrict__ O,
                                int64_t ldo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * ncol) return;
  const int64_t r = e / ncol;
  const int c = (int)(e % ncol);
  T f, f1, f2;
  silu3<T>(Z[r * ldz + c] + (bias ? T(bias[c]) : T(0)), f, f1, f2);
  O[r * ldo + c] = D[r * ldd + c] * f1;
}

}  // namespace fire

// Neighbour lists and the ragged row layout of the sparse forward Laplacian.
//
// N_i = {j != i : |r_i - r_j| <= c} (Results, "Finite-range embeddings"),
// split into same-spin and opposite-spin parts N^par_i, N^anti_i (Methods,
// message passing).  Distances are float64 for every precision, so the
// relation is exactly symmetric: (a-b)^2 == (b-a)^2 in IEEE arithmetic.
//
// Row layout.  Electron i of walker w owns one block of rows in every
// forward-Laplacian tensor: value, Laplacian, then 3 tangent rows per slot,
// slot 0 = r_i itself, slot s >= 1 = the (s-1)-th entry of i's list
// (Methods, "Efficient Laplacian": the Jacobian of h_i is non-zero only for
// electrons in N_i u {i}).  Blocks are stored in spin-major order so that the
// rows of each spin form one contiguous range (different orbital weights per
// spin).
#pragma once

#include "common.cuh"

namespace fire {

// One CTA per walker.  idx [Wc][n][K], cnt [Wc][n][2], blk_rows [Wc*n] in
// block order.
static __global__ void nbr_build_kernel(int Wc, int n, int n_up, const double* __restrict__ r,
                                 double c2, int K, int32_t* __restrict__ idx,
                                 int32_t* __restrict__ cnt, int64_t* __restrict__ blk_rows,
                                 DevStatus* st, int deriv) {
  extern __shared__ double sr[];
  const int w = blockIdx.x;
  const double* rw = r + (int64_t)w * n * 3;
  for (int k = threadIdx.x; k < 3 * n; k += blockDim.x) sr[k] = rw[k];
  __syncthreads();
  int local_max = 0;
  int64_t local_sum = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double xi = sr[3 * i], yi = sr[3 * i + 1], zi = sr[3 * i + 2];
    int32_t* out = idx + ((int64_t)w * n + i) * K;
    const bool up = i < n_up;
    int k = 0;
    int npar = 0;
    for (int pass = 0; pass < 2; ++pass) {
      const bool same = (pass == 0);
      const int lo = (up == same) ? 0 : n_up;
      const int hi = (up == same) ? n_up : n;
      for (int j = lo; j < hi; ++j) {
        if (j == i) continue;
        double dx = xi - sr[3 * j], dy = yi - sr[3 * j + 1], dz = zi - sr[3 * j + 2];
        double d2 = dx * dx + dy * dy + dz * dz;
        if (d2 <= c2) {
          if (k < K) out[k] = j;
          ++k;
        }
      }
      if (pass == 0) npar = k;
    }
    const int total = k;
    const int kept = total < K ? total : K;
    const int kpar = npar < K ? npar : K;
    cnt[((int64_t)w * n + i) * 2 + 0] = kpar;
    cnt[((int64_t)w * n + i) * 2 + 1] = kept - kpar;
    local_max = total > local_max ? total : local_max;
    local_sum += total;
    if (blk_rows) blk_rows[block_index(w, i, Wc, n, n_up)] = deriv ? (2 + 3 * (1 + kept)) : 1;
  }
  if (local_max > 0) atomicMax(&st->k_required, local_max);
  if (local_max > K) atomicExch(&st->overflow, 1);
  if (local_sum) atomicAdd((unsigned long long*)&st->nbr_total, (unsigned long long)local_sum);
}

// rev[w][i][k] = position (within j's list) of i, where j = idx[w][i][k];
// -1 if j's list was truncated before i.
static __global__ void nbr_reverse_kernel(int n, int n_up, int K, const int32_t* __restrict__ idx,
                                   const int32_t* __restrict__ cnt, int32_t* __restrict__ rev) {
  const int w = blockIdx.x;
  for (int e = threadIdx.x; e < n * K; e += blockDim.x) {
    const int i = e / K, k = e % K;
    const int64_t base_i = (int64_t)w * n + i;
    const int ci = cnt[base_i * 2] + cnt[base_i * 2 + 1];
    if (k >= ci) continue;
    const int j = idx[base_i * K + k];
    const int64_t base_j = (int64_t)w * n + j;
    const bool same = ((i < n_up) == (j < n_up));
    const int cpar = cnt[base_j * 2], canti = cnt[base_j * 2 + 1];
    int lo = same ? 0 : cpar, hi = same ? cpar : cpar + canti;
    const int32_t* lj = idx + base_j * K;
    int found = -1;
    while (lo < hi) {  // lists are ascending within each spin part
      int mid = (lo + hi) >> 1;
      int v = lj[mid];
      if (v == i) { found = mid; break; }
      if (v < i) lo = mid + 1; else hi = mid;
    }
    rev[base_i * K + k] = found;
  }
}

// Exclusive scan of block row counts -> blk_off[0..nb]; ranges[0..3] =
// {up_begin, up_end, down_begin, down_end} rows.  One CTA of 1024 threads.
static __global__ void blk_scan_kernel(int nb, int nb_up, const int64_t* __restrict__ rows,
                                int64_t* __restrict__ off, int64_t* __restrict__ ranges,
                                DevStatus* st) {
  __shared__ int64_t part[1024];
  const int T = blockDim.x, t = threadIdx.x;
  const int per = (nb + T - 1) / T;
  const int b0 = t * per, b1 = min(nb, b0 + per);
  int64_t s = 0;
  for (int b = b0; b < b1; ++b) s += rows[b];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < T; o <<= 1) {
    int64_t v = (t >= o) ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int64_t run = (t == 0) ? 0 : part[t - 1];
  for (int b = b0; b < b1; ++b) {
    off[b] = run;
    run += rows[b];
  }
  __syncthreads();
  if (t == T - 1) {
    off[nb] = part[T - 1];
    st->rows_total += part[T - 1];
  }
  __syncthreads();
  if (t == 0) {
    int64_t mid = (nb_up < nb) ? off[nb_up] : part[T - 1];
    if (nb_up == nb) mid = part[T - 1];
    ranges[0] = 0;
    ranges[1] = mid;
    ranges[2] = mid;
    ranges[3] = part[T - 1];
  }
}

}  // namespace fire

// Host-side pipeline: the sequence of kernels of one call, chunk by chunk.
// Instantiated once per precision form (run_fp64.cu, run_fp32.cu,
// run_bf16.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include "common.cuh"
#include "det.cuh"
#include "embed.cuh"
#include "gemm.cuh"
#include "jastrow.cuh"
#include "mcmc.cuh"
#include "ecp.cuh"
#include "swap.cuh"
#include "nbr.cuh"
#include "plan.h"
#include "tc_api.h"

namespace fire {

enum ParamIndex {
  P_EN_W1, P_EN_B1, P_EN_W2, P_EN_WENV, P_EN_SIGMA, P_NUC_EMB, P_EN_WFEAT,
  P_LN_GAMMA, P_LN_BETA, P_GLU_WG, P_GLU_WV, P_GLU_WO,
  P_EE_W1, P_EE_B1, P_EE_W2, P_EE_WENV, P_EE_SIGMA, P_MSG_W, P_MSG_B,
  P_MLP_W, P_MLP_B, P_ORB_W, P_ENV_PI, P_ENV_SIGMA, P_CUSP,
  P_JM1_W1, P_JM1_B1, P_JM1_W2, P_JM1_B2, P_JM1_W3, P_JM1_B3,
  P_JM2_W1, P_JM2_B1, P_JM2_W2, P_JM2_B2, P_JM2_W3, P_JM2_B3,
  P_ATT_Q, P_ATT_WV,
  P_JA1_W1, P_JA1_B1, P_JA1_W2, P_JA1_B2, P_JA1_W3, P_JA1_B3,
  P_JA2_W1, P_JA2_B1, P_JA2_W2, P_JA2_B2, P_JA2_W3, P_JA2_B3,
  P_COUNT
};

}  // namespace fire

#include "grad.cuh"
#include "grad_bufs.h"
#include "grad_util.cuh"

namespace fire {

// Host-side arguments and results of a Metropolis call.
struct McmcCall {
  double sigma;
  int n_sweeps, refresh_every;
  uint64_t seed, counter;
  int32_t* acc_count;        // device [W] accepted moves per walker, or null
  int64_t n_accepted;        // out
  double max_drift;          // out
  int n_global;              // global jumps per sweep (after the n local moves)
  double sigma_global;       // width of the mixture components of a global jump
  double kappa_tol;          // exact-ratio test kappa u w > kappa_tol (< 0: off)
  // non-local pseudopotential evaluation instead of sweeps (ecp != null)
  const fire_ecp_t* ecp;     // device [n_nuc] table
  int ecp_qmax;              // largest N_quad of the table
  double* v_nl;              // device [W] out
  // S+ swap ratios instead of sweeps (swap_beta >= 0)
  int swap_beta;             // the spin-down electron
  double* swap_ratios;       // device [W][n_up] out
  double* swap_r;            // device [W] out: 1 - sum of the ratios
};

struct CallArgs {
  const fire_system_t* sys;
  const fire_arch_t* arch;
  const void* theta;
  const int64_t* poff;       // [P_COUNT] element offsets into theta
  int64_t W;
  const double* r;
  double *e_loc, *logabs, *sign, *e_kin, *e_pot;
  void* ws;
  cudaStream_t stream;
  DevStatus* host_status;    // filled after the call
  int64_t* n_launches;       // kernels launched (host out)
  void* grad;                // [W][P] parameter gradient (gradient call only)
  McmcCall* mcmc;            // Metropolis call only
};

void set_last_error(const char* stage, const char* msg);
cudaStream_t side_stream();
bool single_stream();
bool prof_enabled();
void prof_add(const char* name, int launches, float ms);
int run_fp64(const Plan& pl, const CallArgs& a);
int run_fp32(const Plan& pl, const CallArgs& a);
int run_bf16(const Plan& pl, const CallArgs& a);

template <typename W>
inline Params<W> make_params(const void* theta, const int64_t* o) {
  const W* b = reinterpret_cast<const W*>(theta);
  Params<W> p;
  const W** f[P_COUNT] = {
      &p.en_w1, &p.en_b1, &p.en_w2, &p.en_wenv, &p.en_sigma, &p.nuc_emb, &p.en_wfeat,
      &p.ln_gamma, &p.ln_beta, &p.glu_wg, &p.glu_wv, &p.glu_wo,
      &p.ee_w1, &p.ee_b1, &p.ee_w2, &p.ee_wenv, &p.ee_sigma, &p.msg_w, &p.msg_b,
      &p.mlp_w, &p.mlp_b, &p.orb_w, &p.env_pi, &p.env_sigma, &p.cusp,
      &p.jm1_w1, &p.jm1_b1, &p.jm1_w2, &p.jm1_b2, &p.jm1_w3, &p.jm1_b3,
      &p.jm2_w1, &p.jm2_b1, &p.jm2_w2, &p.jm2_b2, &p.jm2_w3, &p.jm2_b3,
      &p.att_q, &p.att_wv,
      &p.ja1_w1, &p.ja1_b1, &p.ja1_w2, &p.ja1_b2, &p.ja1_w3, &p.ja1_b3,
      &p.ja2_w1, &p.ja2_b1, &p.ja2_w2, &p.ja2_b2, &p.ja2_w3, &p.ja2_b3};
  for (int k = 0; k < P_COUNT; ++k) *f[k] = b + o[k];
  return p;
}

// Hook for the tensor-core form: a matrix product over forward-Laplacian rows
// with an optional tensor-core implementation (BF16 in, FP32 accumulate).
template <typename T>
struct RowGemm {
  // returns true if it handled the product
  bool (*tc)(void* ctx, cudaStream_t s, const T* A, int64_t lda, const T* B, int64_t ldb, T* C,
             int64_t ldc, const int64_t* m_range, int64_t m_begin, int64_t m_end, int64_t m_cap,
             int N, int K) = nullptr;
  void* ctx = nullptr;
};

template <typename T, typename LT, typename RT>
struct Runner {
  const Plan& pl;
  const CallArgs& a;
  const Dims& dm;
  Params<T> p;
  unsigned char* ws;
  cudaStream_t s;
  RowGemm<T> rg;

  Runner(const Plan& pl_, const CallArgs& a_) : pl(pl_), a(a_), dm(pl_.dm) {
    p = make_params<T>(a.theta, a.poff);
    dbg = getenv("FIRE_DEBUG_SYNC") != nullptr;
    // FIRE_TC_MASK (diagnostic): bit 0 embedding MLP, 1 Jastrow MLPs,
    // 2 attention, 3 orbitals, 4 envelopes, 5 h^0 products (GLU, message
    // projections) and orbital value rows, 6 attention register MLPs, 7 the
    // restricted log-det contraction -- which products may use the tensor
    // cores.
    if (const char* m = getenv("FIRE_TC_MASK")) tc_mask = atoi(m);
    if (const char* m = getenv("FIRE_TC_FIX_VALUES")) fix_values = atoi(m);
    // FIRE_TC_VALUE_ROWS=split: value rows by six split products on the
    // tensor cores (1.7 % faster step; over 4096 C26H24 walkers the E_L error
    // against float64 rose from 1.9e-5 to 2.1e-5 at the median and from
    // 1.08e-2 to 1.25e-2 at p99, where float32 SIMT value rows match the
    // plain FP32 form's 1.08e-2)
    if (const char* m = getenv("FIRE_TC_VALUE_ROWS")) simt_values = strcmp(m, "split") != 0;
    // FIRE_INVERSE (diagnostic): 1 = float32 Gauss-Jordan from a float copy of
    // Phi (n <= 192, the default of the float32 forms), 0 = triangular solves
    // on the LU factors (always for float64 and for n > 192)
    if (const char* m = getenv("FIRE_INVERSE")) use_gj = atoi(m) == 1;
    if (const char* m = getenv("FIRE_LU_NB")) lu_nb = atoi(m) == 32 ? 32 : 16;
    auto split_env = [](const char* k, int dflt) {
      const char* v = getenv(k);
      int x = v ? atoi(v) : dflt;
      return x < 1 ? 1 : (x > kMaxSplit ? kMaxSplit : x);
    };
    nc_mlp = split_env("FIRE_TC_SPLIT_MLP", nc_mlp);
    nc_jas = split_env("FIRE_TC_SPLIT_JASTROW", nc_jas);
    nc_att = split_env("FIRE_TC_SPLIT_ATT", nc_att);
    nc_orb = split_env("FIRE_TC_SPLIT_ORB", nc_orb);
    nc_env = split_env("FIRE_TC_SPLIT_ENV", nc_env);
    nc_h0 = split_env("FIRE_TC_SPLIT_H0", nc_h0);
    ncw = nc_mlp > nc_jas ? nc_mlp : nc_jas;
    if (nc_att > ncw) ncw = nc_att;
    if (nc_orb > ncw) ncw = nc_orb;
    capA = pl.Wc * dm.n * pl.rows_per_el;
    prof = prof_enabled();
    ws = reinterpret_cast<unsigned char*>(a.ws);
    s = a.stream;
  }
  template <typename X> X* at(size_t off) { return reinterpret_cast<X*>(ws + off); }

  // Second stream of this device (created once, non-blocking) and the fork /
  // join events of the current call.
  bool lu_side = false;
  cudaStream_t s2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool side_ready() {
    // FIRE_LU_SIDE=1 (diagnostic): the float64 LU on a second stream.  Off by
    // default: on GB300 its CTAs did not share SMs with the tensor-core
    // product, and one stream measured as fast (1665 vs 1660 walkers/s).
    const char* e = getenv("FIRE_LU_SIDE");
    if (!(e && atoi(e) == 1) || single_stream()) return false;
    if (!s2) s2 = side_stream();
    if (!s2) return false;
    if (!ev_fork && cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming) != cudaSuccess) return false;
    if (!ev_join && cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming) != cudaSuccess) return false;
    return true;
  }
  ~Runner() {
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
  }

  // With FIRE_DEBUG_SYNC set, every stage is synchronised and checked, and the
  // name of the first failing stage is kept for fire_last_error().
  bool dbg = false;
  int failed = 0;
  void check(const char* stage) {
    if (!dbg || failed) return;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      failed = 1;
      set_last_error(stage, cudaGetErrorString(e));
    }
  }

  // Stage marks: the device time between two marks is attributed to the
  // first one's name (profiler enabled); every mark adds its launch count.
  bool prof = false;
  int64_t launches = 0;
  struct Mark { const char* name; cudaEvent_t ev; int nl; };
  Mark marks[1024];
  int nmarks = 0;
  void mark(const char* name, int nl) {
    launches += nl;
    if (!prof || nmarks >= 1024) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, s);
    marks[nmarks++] = Mark{name, e, nl};
  }
  void flush_marks() {
    if (!prof) return;
    cudaStreamSynchronize(s);
    for (int k = 0; k + 1 < nmarks; ++k) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, marks[k].ev, marks[k + 1].ev);
      prof_add(marks[k].name, marks[k].nl, ms);
    }
    for (int k = 0; k < nmarks; ++k) cudaEventDestroy(marks[k].ev);
    nmarks = 0;
  }

  // Product over forward-Laplacian rows.  With a bf16 copy Ab of A (row
  // stride lda, a_rows rows allocated) and packed bf16 weights Bt [N][K] it
  // runs on the tensor cores (BF16_FP64 form); otherwise SIMT in T.
  int tc_rc = FIRE_OK;
  int tc_mask = 0xFF;
  int fix_values = 1;         // value rows recomputed in fp32 after a tensor-core product
  bool simt_values = true;    // ... by the float32 SIMT product (else six split products)
  // split-bf16 components of each tensor-core product (1: 1 product, 2: 3, 3: 6).
  // Two components (hi + lo, three products) for the products whose value
  // rows are recomputed in fp32 afterwards: measured against the float64 path
  // on 128 C26H24 walkers, the E_L error distribution then equals that of
  // plain fp32 (median 2e-5) and of three components; one component raises
  // the median error to 8e-4.  The attention product has no value-row
  // recompute (its value rows set log|J_att|) and keeps three components.
  int nc_mlp = 2, nc_jas = 2, nc_att = 3, nc_orb = 2;
  int ncw = 3;                // components written for the bf16 copies of X and Y
  int nc_env = 3;             // envelope product: its value rows enter Phi directly
  int nc_h0 = 3;              // h^0 products and orbital value rows (no fp32 recompute)
  bool use_gj = true;
  int lu_nb = 16;             // FIRE_LU_NB (diagnostic): 16 or 32-column LU panels
  // A^T from the LU factors, matrices in batches of the grid limit
  void inverse_from_lu(int n, int64_t nmat, const LT* LUb, const int32_t* piv, T* Ainv) {
    const size_t ism = inverse_panel_smem(n, sizeof(T));
    for (int64_t m0 = 0; m0 < nmat; m0 += 65535) {
      const int64_t cnt = nmat - m0 < 65535 ? nmat - m0 : 65535;
      inverse_panel_kernel<LT, T, T><<<(unsigned)cnt, 256, ism, s>>>(n, m0, LUb, piv, Ainv);
      launches += 1;
    }
  }
  int64_t capA = 0;           // allocated rows of X / Y: the component stride of Xb / Yb
  // value-row fix-up context of the current chunk
  const int64_t* vr_off = nullptr;
  int vr_nb = 0;
  T* vr_A = nullptr;           // [nb][K] gathered value rows
  T* vr_C = nullptr;           // [nb][N] their products
  __nv_bfloat16* vr_Ab = nullptr;   // [3][vr_cap][K] the gathered rows as three bf16 components
  int64_t vr_cap = 0, vr_kmax = 0;  // component stride (rows) and widest K that vr_Ab holds
  void row_gemm(const T* A, const __nv_bfloat16* Ab, int64_t lda, int64_t a_rows, const T* B,
                const __nv_bfloat16* Bt, int64_t ldb, T* C, int64_t ldc, const int64_t* m_range,
                int64_t m_begin, int64_t m_end, int64_t m_cap, int N, int K, int nc = 1) {
    if (!row_gemm_tc(A, Ab, lda, a_rows, B, Bt, ldb, C, ldc, m_range, m_begin, m_end, m_cap, N, K, nc))
      gemm<T>(s, A, lda, B, ldb, false, C, ldc, m_begin, m_end, m_range, m_cap, N, K);
  }
  // The tensor-core form of row_gemm; false (nothing launched) where it does not apply.
  bool row_gemm_tc(const T* A, const __nv_bfloat16* Ab, int64_t lda, int64_t a_rows, const T* B,
                   const __nv_bfloat16* Bt, int64_t ldb, T* C, int64_t ldc, const int64_t* m_range,
                   int64_t m_begin, int64_t m_end, int64_t m_cap, int N, int K, int nc) {
    if constexpr (sizeof(T) == 4) {
      if (Ab && Bt && K % 64 == 0) {
        int rc = tc::gemm_bf16(s, Ab, lda, a_rows, Bt, N, K, reinterpret_cast<float*>(C), ldc, m_begin, m_end,
                               m_range, m_cap, &at<DevStatus>(pl.status)->tc_err, nc);
        if (rc == FIRE_OK) {
          if (fix_values && vr_off && m_range) {
            // value rows (one per block) again at float32 accuracy: they set
            // Phi and log|Psi|.  Float32 SIMT product, or (FIRE_TC_VALUE_ROWS=
            // split) three-component split products on the tensor cores where
            // the scratch holds the rows (the packed weights carry three
            // components)
            bool tcv = false;
            if (vr_Ab && K <= vr_kmax && !simt_values) {
              gather_value_rows_kernel<T><<<vr_nb, 256, 0, s>>>(vr_nb, K, vr_off, A, nullptr, lda, vr_Ab, kMaxSplit,
                                                                vr_cap * K);
              tcv = tc::gemm_bf16(s, vr_Ab, K, vr_cap, Bt, N, K, reinterpret_cast<float*>(vr_C), N, 0, vr_nb,
                                  nullptr, vr_nb, &at<DevStatus>(pl.status)->tc_err, kMaxSplit) == FIRE_OK;
              launches += 2;
            }
            if (!tcv) {
              gather_value_rows_kernel<T><<<vr_nb, 256, 0, s>>>(vr_nb, K, vr_off, A, vr_A, lda);
              gemm<T>(s, vr_A, K, B, ldb, false, vr_C, N, 0, vr_nb, nullptr, vr_nb, N, K);
              launches += 2;
            }
            scatter_value_rows_kernel<T><<<vr_nb, 256, 0, s>>>(N, vr_off, vr_C, C, ldc);
            launches += 1;
          }
          return true;
        }
        tc_rc = rc;
      }
    }
    return false;
  }

  // Forward-Laplacian SiLU layer over ragged blocks (fl_act_kernel); the
  // float rows take the four-column form where its alignment holds.
  void fl_act(int ncol, const int64_t* off, int64_t stride, const T* Z, int64_t ldz, const T* bias, T* Y,
              int64_t ldy, int residual, __nv_bfloat16* Yb, int ync, int64_t ycs, int yall, int64_t nblk) {
    if constexpr (sizeof(T) == 4) {
      if (fl_act4_ok(ncol, ldz, ldy, ycs, Z, Y, Yb)) {
        fl_act4_kernel<T><<<nblk, 64, 0, s>>>(ncol, off, stride, reinterpret_cast<const float*>(Z), ldz, bias,
                                              reinterpret_cast<float*>(Y), ldy, residual, Yb, ync, ycs, yall);
        return;
      }
    }
    fl_act_kernel<T, T><<<nblk, 256, 0, s>>>(ncol, off, stride, Z, ldz, bias, Y, ldy, residual, Yb, ync, ycs, yall);
  }

  // SiLU-MLP readout with two hidden layers over ragged blocks (rows of X
  // given by blk offsets or a fixed stride) -> per-row scalar F.
  void mlp_readout(const T* Xin, const __nv_bfloat16* Xinb, int64_t ldx, int din, const int64_t* range,
                   int64_t rb, int64_t re, int64_t cap, const int64_t* off, int64_t stride, int nblk,
                   const T* w1, const __nv_bfloat16* w1b, const T* b1, const T* w2,
                   const __nv_bfloat16* w2b, const T* b2, const T* w3, T* Z, int64_t ldz, T* Y,
                   __nv_bfloat16* Yb, int64_t ldy, T* F, int64_t a_rows = -1, int nc = -1) {
    const int J = dm.J;
    if (a_rows < 0) a_rows = capA;   // rows between the bf16 components of Xinb and Yb
    if (nc < 0) nc = nc_jas;
    row_gemm(Xin, Xinb, ldx, a_rows, w1, w1b, J, Z, ldz, range, rb, re, cap, J, din, nc);
    // the hidden layer feeds a tensor-core product through Yb: of the float
    // rows only the value rows (read again in fp32) are stored; should the
    // product not apply, the layer is recomputed in full for the fallback
    const bool via_b = sizeof(T) == 4 && Yb && w2b && J % 64 == 0;
    fl_act(J, off, stride, Z, ldz, b1, Y, ldy, 0, Yb, nc, a_rows * ldy, via_b ? 0 : 1, nblk);
    if (!row_gemm_tc(Y, Yb, ldy, a_rows, w2, w2b, J, Z, ldz, range, rb, re, cap, J, J, nc)) {
      if (via_b) fl_act_kernel<T, T><<<nblk, 256, 0, s>>>(J, off, stride, Z, ldz, b1, Y, ldy, 0);
      gemm<T>(s, Y, ldy, w2, J, false, Z, ldz, rb, re, range, cap, J, J);
    }
    // last activation fused with the readout vector: F = act(Z + b2) . w3
    const int max_rows = off ? (int)pl.rows_per_el : (int)stride;
    fl_act_dot_kernel<T, T><<<nblk, 256, (size_t)8 * max_rows * sizeof(T), s>>>(J, off, stride, Z, ldz, b2, w3, F,
                                                                               max_rows);
  }


  // ---------------------------------------------------------------------
  // d log|Psi| / d theta per walker: the value path with its intermediates
  // kept, then the adjoint in reverse order.  Embeddings are recomputed here
  // (no state is carried between calls).
  // ---------------------------------------------------------------------
  int run_grad() {
    const fire_system_t* sys = a.sys;
    const int n = dm.n, n_up = dm.n_up, n_dn = n - n_up, N = dm.N, d = dm.d, D = dm.D, K = dm.K, L = dm.L;
    const int J = dm.J, R = dm.R, dr = dm.dr, RD = R * dr, E = dm.E, NE = N * E;
    const int64_t Dn = (int64_t)D * n;
    const int64_t P = pl.nparams;
    const int64_t* po = a.poff;
    DevStatus* st = at<DevStatus>(pl.status);
    cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
    int64_t* pod = at<int64_t>(pl.poff_dev);
    cudaMemcpyAsync(pod, po, sizeof(int64_t) * P_COUNT, cudaMemcpyHostToDevice, s);
    T* G = reinterpret_cast<T*>(a.grad);
    for (int64_t ch = 0; ch < pl.nchunks; ++ch) {
      const int64_t w0 = ch * pl.Wc;
      const int wc = (int)((a.W - w0) < pl.Wc ? (a.W - w0) : pl.Wc);
      const double* r = a.r + w0 * n * 3;
      const int nb = wc * n;
      T* g = G + w0 * P;
      cudaMemsetAsync(g, 0, sizeof(T) * (size_t)wc * P, s);
      GradBufs<T> B;
      GradBufs<T>::carve(at<unsigned char>(pl.gradws), &B, pl.Wc, n, d, L, D, J, R, RD, NE);
      int32_t* idx = at<int32_t>(pl.idx);
      int32_t* cnt = at<int32_t>(pl.cnt);
      int32_t* rev = at<int32_t>(pl.rev);
      int64_t* brow = at<int64_t>(pl.blk_rows);
      int64_t* boff = at<int64_t>(pl.blk_off);
      int64_t* rng = at<int64_t>(pl.ranges);
      const double c = sys->cutoff;
      // segments of a walker's electrons in block order: up [w n_up, +n_up), down [Wc n_up + w n_dn, +n_dn)
      auto tn_w = [&](const T* X, int64_t ldx, int Na, const T* Y, int64_t ldy, int Nb, int64_t goff, int64_t ldc,
                      bool acc) {
        tn_batched<T>(s, wc, Na, Nb, n_up, X, ldx, n_up * ldx, Y, ldy, n_up * ldy, g + goff, ldc, P, acc);
        tn_batched<T>(s, wc, Na, Nb, n_dn, X + (int64_t)wc * n_up * ldx, ldx, n_dn * ldx,
                      Y + (int64_t)wc * n_up * ldy, ldy, n_dn * ldy, g + goff, ldc, P, true);
        launches += 2;
      };
      auto colsum_w = [&](const T* Y, int64_t ldy, int Nb, int64_t goff) {
        colsum_batched<T>(s, wc, Nb, n_up, Y, ldy, n_up * ldy, g + goff, P, true);
        colsum_batched<T>(s, wc, Nb, n_dn, Y + (int64_t)wc * n_up * ldy, ldy, n_dn * ldy, g + goff, P, true);
        launches += 2;
      };
      // ---- forward (value rows: one row per electron block) ----
      mark("neighbors", 3);
      nbr_build_kernel<<<wc, 256, (size_t)n * 3 * sizeof(double), s>>>(wc, n, n_up, r, c * c, K, idx, cnt, brow, st, 0);
      nbr_reverse_kernel<<<wc, 256, 0, s>>>(n, n_up, K, idx, cnt, rev);
      blk_scan_kernel<<<1, 1024, 0, s>>>(nb, wc * n_up, brow, boff, rng, st);
      T* S5 = at<T>(pl.S5);
      T* Y5 = at<T>(pl.Y5);
      T* Z5 = at<T>(pl.Z5);
      T* P5 = at<T>(pl.P5);
      T* H0 = at<T>(pl.H0);
      T* PQ = at<T>(pl.PQ);
      mark("fwd_embed", 8);
      en_filter_kernel<T, T><<<nb, d, 0, s>>>(wc, n, n_up, N, d, r, sys->nuc_pos, sys->cutoff_nuc, p, S5, 1);
      ln_fl_kernel<T, T><<<nb, d, 0, s>>>(d, S5, Y5, p.ln_gamma, p.ln_beta, 1);
      gemm<T>(s, Y5, d, p.glu_wg, d, false, Z5, 2 * d, 0, nb, nullptr, nb, d, d);
      gemm<T>(s, Y5, d, p.glu_wv, d, false, Z5 + d, 2 * d, 0, nb, nullptr, nb, d, d);
      glu_gate_kernel<T><<<nb, d, 0, s>>>(d, Z5, P5, 1);
      gemm<T>(s, P5, d, p.glu_wo, d, false, H0, d, 0, nb, nullptr, nb, d, d);
      for (int part = 0; part < 2; ++part)
        gemm<T>(s, H0, d, p.msg_w + (int64_t)part * d * d, d, false, PQ + (int64_t)part * 2 * d, 4 * d, 0, nb,
                nullptr, nb, d, d, 2, 0, (int64_t)(2 * d + 4) * d, d);
      T* H1 = B.HL;
      msg_kernel<T, T><<<nb, d, 0, s>>>(wc, n, n_up, d, K, r, c, p, idx, cnt, boff, H0, PQ, H1, nullptr, 1, 0, 0);
      mark("fwd_mlp", 3 * L);
      for (int l = 0; l < L; ++l) {
        T* hin = B.HL + (int64_t)l * nb * d;
        T* hout = B.HL + (int64_t)(l + 1) * nb * d;
        T* z = B.ZL + (int64_t)l * nb * d;
        gemm<T>(s, hin, d, p.mlp_w + (int64_t)l * d * d, d, false, z, d, 0, nb, nullptr, nb, d, d);
        cudaMemcpyAsync(hout, hin, sizeof(T) * (size_t)nb * d, cudaMemcpyDeviceToDevice, s);
        fl_act_kernel<T, T><<<nb, 256, 0, s>>>(d, nullptr, 1, z, d, p.mlp_b + (int64_t)l * d, hout, d, 1);
      }
      const T* h = B.HL + (int64_t)L * nb * d;
      T* jval = at<T>(pl.jval); T* jsign = at<T>(pl.jsign);
      T* aval = at<T>(pl.aval); T* asign = at<T>(pl.asign);
      T* cval = at<T>(pl.cval); T* vpot = at<T>(pl.vpot);
      T* F[2] = {at<T>(pl.F1), at<T>(pl.F2)};
      const T* jw1[2] = {p.jm1_w1, p.jm2_w1};
      const T* jb1[2] = {p.jm1_b1, p.jm2_b1};
      const T* jw2[2] = {p.jm1_w2, p.jm2_w2};
      const T* jb2[2] = {p.jm1_b2, p.jm2_b2};
      const T* jw3[2] = {p.jm1_w3, p.jm2_w3};
      if (dm.flags & FIRE_J_MLP) {
        mark("fwd_jastrow", 11);
        for (int k = 0; k < 2; ++k) {
          gemm<T>(s, h, d, jw1[k], J, false, B.JZ1[k], J, 0, nb, nullptr, nb, J, d);
          fl_act_kernel<T, T><<<nb, 256, 0, s>>>(J, nullptr, 1, B.JZ1[k], J, jb1[k], B.JA1[k], J, 0);
          gemm<T>(s, B.JA1[k], J, jw2[k], J, false, B.JZ2[k], J, 0, nb, nullptr, nb, J, J);
          fl_act_kernel<T, T><<<nb, 256, 0, s>>>(J, nullptr, 1, B.JZ2[k], J, jb2[k], B.JA2[k], J, 0);
          rowdot_kernel<T, T><<<(unsigned)((nb + 7) / 8), 256, 0, s>>>(B.JA2[k], J, J, jw3[k], F[k], nullptr, 0, nb);
        }
        jmlp_reduce_kernel<T, T><<<wc, 256, 0, s>>>(wc, n, n_up, K, idx, cnt, rev, boff, F[0], F[1], p.jm1_b3,
                                                    p.jm2_b3, jval, jsign, nullptr, nullptr, 0);
      }
      const int64_t ldsu = R + RD;
      T* V = at<T>(pl.V);
      T* Gv[2] = {at<T>(pl.G1), at<T>(pl.G2)};
      const T* vw1[2] = {p.ja1_w1, p.ja2_w1};
      const T* vb1[2] = {p.ja1_b1, p.ja2_b1};
      const T* vw2[2] = {p.ja1_w2, p.ja2_w2};
      const T* vb2[2] = {p.ja1_b2, p.ja2_b2};
      const T* vw3[2] = {p.ja1_w3, p.ja2_w3};
      if (dm.flags & FIRE_J_ATT) {
        mark("fwd_att", 14);
        gemm<T>(s, h, d, p.att_q, d, true, B.SU, ldsu, 0, nb, nullptr, nb, R, d);
        gemm<T>(s, h, d, p.att_wv, dr, false, B.SU + R, ldsu, 0, nb, nullptr, nb, dr, d, R, 0, (int64_t)d * dr, dr);
        const int bt = ((RD + 31) / 32) * 32;
        att_pool_kernel<T><<<wc, bt, (size_t)(R + n * R) * sizeof(T), s>>>(wc, n, n_up, K, R, dr, idx, cnt, rev,
                                                                          boff, B.SU, ldsu, V, 0);
        for (int k = 0; k < 2; ++k) {
          gemm<T>(s, V, RD, vw1[k], J, false, B.VZ1[k], J, 0, wc, nullptr, wc, J, RD);
          fl_act_kernel<T, T><<<wc, 256, 0, s>>>(J, nullptr, 1, B.VZ1[k], J, vb1[k], B.VA1[k], J, 0);
          gemm<T>(s, B.VA1[k], J, vw2[k], J, false, B.VZ2[k], J, 0, wc, nullptr, wc, J, J);
          fl_act_kernel<T, T><<<wc, 256, 0, s>>>(J, nullptr, 1, B.VZ2[k], J, vb2[k], B.VA2[k], J, 0);
          rowdot_kernel<T, T><<<(unsigned)((wc + 7) / 8), 256, 0, s>>>(B.VA2[k], J, J, vw3[k], Gv[k], nullptr, 0, wc);
        }
        att_reduce_kernel<T, T><<<wc, 256, 0, s>>>(n, Gv[0], Gv[1], p.ja1_b3, p.ja2_b3, aval, asign, nullptr, nullptr, 0);
      }
      mark("fwd_orbitals", 8);
      coulomb_cusp_kernel<T, T><<<wc, 256, 0, s>>>(n, n_up, N, r, sys->nuc_pos, sys->nuc_charge, p.cusp, vpot, cval,
                                                   nullptr, nullptr, 0);
      T* Qf = at<T>(pl.Qf);
      T* Fenv = at<T>(pl.Fenv);
      T* Ov = at<T>(pl.Ov);
      env_feat_kernel<T, T><<<nb, 128, 0, s>>>(wc, n, n_up, N, E, r, sys->nuc_pos, p.env_sigma, Qf, 1);
      const int64_t upv = (int64_t)wc * n_up;
      for (int sp = 0; sp < 2; ++sp) {
        const int64_t rb = sp ? upv : 0, re = sp ? nb : upv;
        if (re <= rb) continue;
        gemm<T>(s, Qf, NE, p.env_pi + (int64_t)sp * Dn * NE, NE, true, Fenv, Dn, rb, re, nullptr, re - rb, (int)Dn, NE);
        gemm<T>(s, h, d, p.orb_w + (int64_t)sp * D * d * n, n, false, Ov, Dn, rb, re, nullptr, re - rb, n, d, D, 0,
                (int64_t)d * n, n);
      }
      LT* LUb = at<LT>(pl.LU);
      int32_t* piv = at<int32_t>(pl.piv);
      double* ldabs = at<double>(pl.ldabs);
      double* lsign = at<double>(pl.lsign);
      const bool gj = use_gj && sizeof(T) == 4 && n <= 192;
      phi_assemble_kernel<T, LT><<<wc * D, 256, 0, s>>>(wc, n, n_up, D, Ov, Fenv, 1, LUb, gj ? B.Phif : nullptr);
      lu_kernel<LT, 16><<<wc * D, 256, lu_smem_bytes(n, sizeof(LT)), s>>>(n, LUb, piv, ldabs, lsign);
      if (gj) {
        gj_inverse_kernel<float, T><<<wc * D, gj_threads(n), gj_smem_bytes(n), s>>>(n, B.Phif, B.AT);
      } else {
        inverse_from_lu(n, (int64_t)wc * D, LUb, piv, B.AT);
      }
      FinalIn<T, RT> fi{ldabs, lsign, nullptr, nullptr, cval, nullptr, nullptr, jval, jsign, nullptr, nullptr,
                        aval, asign, nullptr, nullptr, vpot};
      final_kernel<T, RT><<<wc, 256, 0, s>>>(n, D, dm.flags, fi, 0, nullptr, a.logabs + w0, a.sign + w0, nullptr,
                                             nullptr, st);
      check("grad forward");
      // ---- backward ----
      mark("bwd_orbitals", 0);
      det_bwd_kernel<T><<<wc * D, 256, 0, s>>>(wc, n, n_up, D, ldabs, lsign, B.AT, Ov, Fenv, B.dO, B.dF);
      ++launches;
      cudaMemsetAsync(B.dH, 0, sizeof(T) * (size_t)nb * d, s);
      for (int sp = 0; sp < 2; ++sp) {
        const int64_t rb = sp ? upv : 0, re = sp ? nb : upv;
        if (re <= rb) continue;
        const int ns = sp ? n_dn : n_up;
        for (int dd = 0; dd < D; ++dd) {
          const int64_t wo = po[P_ORB_W] + ((int64_t)sp * D + dd) * d * n;
          const int64_t pi_o = po[P_ENV_PI] + ((int64_t)sp * D + dd) * n * NE;
          const T* Xs = h + rb * d;
          tn_batched<T>(s, wc, d, n, ns, Xs, d, (int64_t)ns * d, B.dO + rb * Dn + dd * n, Dn, (int64_t)ns * Dn,
                        g + wo, n, P, false);
          tn_batched<T>(s, wc, n, NE, ns, B.dF + rb * Dn + dd * n, Dn, (int64_t)ns * Dn, Qf + rb * NE, NE,
                        (int64_t)ns * NE, g + pi_o, NE, P, false);
          gemm<T>(s, B.dO + dd * n, Dn, p.orb_w + ((int64_t)sp * D + dd) * d * n, n, true, B.dH, d, rb, re, nullptr,
                  re - rb, d, n, 1, 0, 0, 0, true);
          launches += 3;
        }
        gemm<T>(s, B.dF, Dn, p.env_pi + (int64_t)sp * Dn * NE, NE, false, B.dQf, NE, rb, re, nullptr, re - rb, NE,
                (int)Dn);
        ++launches;
      }
      env_sigma_bwd_kernel<T><<<wc, 128, 0, s>>>(wc, n, n_up, N, E, r, sys->nuc_pos, Qf, B.dQf, g, P, po[P_ENV_SIGMA]);
      ++launches;
      check("bwd orbitals");
      if (dm.flags & FIRE_J_MLP) {
        mark("bwd_jastrow", 0);
        const int64_t jo[2][6] = {{po[P_JM1_W1], po[P_JM1_B1], po[P_JM1_W2], po[P_JM1_B2], po[P_JM1_W3], po[P_JM1_B3]},
                                  {po[P_JM2_W1], po[P_JM2_B1], po[P_JM2_W2], po[P_JM2_B2], po[P_JM2_W3], po[P_JM2_B3]}};
        for (int k = 0; k < 2; ++k) {
          jseed_kernel<T><<<wc, 256, 0, s>>>(wc, n, n_up, J, F[1], p.jm2_b3, jw3[k], k, B.df, B.dY2);
          tn_w(B.df, 1, 1, B.JA2[k], J, J, jo[k][4], J, true);
          colsum_w(B.df, 1, 1, jo[k][5]);
          silu_bwd_kernel<T, T><<<(unsigned)(((int64_t)nb * J + 255) / 256), 256, 0, s>>>(nb, J, B.dY2, J, B.JZ2[k], J,
                                                                                         jb2[k], B.dZ2, J);
          tn_w(B.JA1[k], J, J, B.dZ2, J, J, jo[k][2], J, true);
          colsum_w(B.dZ2, J, J, jo[k][3]);
          gemm<T>(s, B.dZ2, J, jw2[k], J, true, B.dA1, J, 0, nb, nullptr, nb, J, J);
          silu_bwd_kernel<T, T><<<(unsigned)(((int64_t)nb * J + 255) / 256), 256, 0, s>>>(nb, J, B.dA1, J, B.JZ1[k], J,
                                                                                         jb1[k], B.dZ1, J);
          tn_w(h, d, d, B.dZ1, J, J, jo[k][0], J, true);
          colsum_w(B.dZ1, J, J, jo[k][1]);
          gemm<T>(s, B.dZ1, J, jw1[k], J, true, B.dH, d, 0, nb, nullptr, nb, d, J, 1, 0, 0, 0, true);
          launches += 5;
        }
      }
      if (dm.flags & FIRE_J_ATT) {
        mark("bwd_att", 0);
        const int64_t vo[2][6] = {{po[P_JA1_W1], po[P_JA1_B1], po[P_JA1_W2], po[P_JA1_B2], po[P_JA1_W3], po[P_JA1_B3]},
                                  {po[P_JA2_W1], po[P_JA2_B1], po[P_JA2_W2], po[P_JA2_B2], po[P_JA2_W3], po[P_JA2_B3]}};
        cudaMemsetAsync(B.dV, 0, sizeof(T) * (size_t)wc * RD, s);
        for (int k = 0; k < 2; ++k) {
          vseed_kernel<T><<<wc, 256, 0, s>>>(J, Gv[1], p.ja2_b3, vw3[k], k, B.dfv, B.dVY2);
          tn_batched<T>(s, wc, 1, J, 1, B.dfv, 1, 1, B.VA2[k], J, J, g + vo[k][4], J, P, true);
          colsum_batched<T>(s, wc, 1, 1, B.dfv, 1, 1, g + vo[k][5], P, true);
          silu_bwd_kernel<T, T><<<(unsigned)(((int64_t)wc * J + 255) / 256), 256, 0, s>>>(wc, J, B.dVY2, J, B.VZ2[k],
                                                                                         J, vb2[k], B.dVZ2, J);
          tn_batched<T>(s, wc, J, J, 1, B.VA1[k], J, J, B.dVZ2, J, J, g + vo[k][2], J, P, true);
          colsum_batched<T>(s, wc, J, 1, B.dVZ2, J, J, g + vo[k][3], P, true);
          gemm<T>(s, B.dVZ2, J, vw2[k], J, true, B.dVA1, J, 0, wc, nullptr, wc, J, J);
          silu_bwd_kernel<T, T><<<(unsigned)(((int64_t)wc * J + 255) / 256), 256, 0, s>>>(wc, J, B.dVA1, J, B.VZ1[k],
                                                                                         J, vb1[k], B.dVZ1, J);
          tn_batched<T>(s, wc, RD, J, 1, V, RD, RD, B.dVZ1, J, J, g + vo[k][0], J, P, true);
          colsum_batched<T>(s, wc, J, 1, B.dVZ1, J, J, g + vo[k][1], P, true);
          gemm<T>(s, B.dVZ1, J, vw1[k], J, true, B.dV, RD, 0, wc, nullptr, wc, RD, J, 1, 0, 0, 0, true);
          launches += 11;
        }
        const size_t absm = (size_t)(2 * n * R + 3 * R) * sizeof(T);
        const int bt = ((RD + 31) / 32) * 32;
        att_bwd_kernel<T><<<wc, bt, absm, s>>>(wc, n, n_up, R, dr, B.SU, ldsu, B.dV, B.dSU);
        tn_w(B.dSU, ldsu, R, h, d, d, po[P_ATT_Q], d, true);
        for (int rr = 0; rr < R; ++rr)
          tn_w(h, d, d, B.dSU + R + rr * dr, ldsu, dr, po[P_ATT_WV] + (int64_t)rr * d * dr, dr, true);
        gemm<T>(s, B.dSU, ldsu, p.att_q, d, false, B.dH, d, 0, nb, nullptr, nb, d, R, 1, 0, 0, 0, true);
        for (int rr = 0; rr < R; ++rr)
          gemm<T>(s, B.dSU + R + rr * dr, ldsu, p.att_wv + (int64_t)rr * d * dr, dr, true, B.dH, d, 0, nb, nullptr, nb,
                  d, dr, 1, 0, 0, 0, true);
        launches += 2 + 2 * R;
      }
      if (dm.flags & FIRE_J_CUSP) {
        cusp_bwd_kernel<T><<<wc, 256, 0, s>>>(n, n_up, r, p.cusp, g, P, po[P_CUSP]);
        ++launches;
      }
      check("bwd jastrow");
      // embedding MLP, layer by layer
      mark("bwd_mlp", 0);
      for (int l = L - 1; l >= 0; --l) {
        const T* hin = B.HL + (int64_t)l * nb * d;
        const T* z = B.ZL + (int64_t)l * nb * d;
        silu_bwd_kernel<T, T><<<(unsigned)(((int64_t)nb * d + 255) / 256), 256, 0, s>>>(nb, d, B.dH, d, z, d,
                                                                                       p.mlp_b + (int64_t)l * d, B.dZ, d);
        tn_w(hin, d, d, B.dZ, d, d, po[P_MLP_W] + (int64_t)l * d * d, d, true);
        colsum_w(B.dZ, d, d, po[P_MLP_B] + (int64_t)l * d);
        gemm<T>(s, B.dZ, d, p.mlp_w + (int64_t)l * d * d, d, true, B.dH, d, 0, nb, nullptr, nb, d, d, 1, 0, 0, 0, true);
        launches += 2;
      }
      // message passing (dH now holds d/dh^1)
      mark("bwd_msg", 0);
      cudaMemsetAsync(B.dQm, 0, sizeof(T) * (size_t)nb * 2 * d, s);
      msg_bwd_kernel<T, T><<<nb, d, 0, s>>>(wc, n, n_up, d, K, r, c, p, idx, cnt, PQ, B.dH, B.dPm, B.dQm, g, P, pod);
      cudaMemcpyAsync(B.dH0, B.dH, sizeof(T) * (size_t)nb * d, cudaMemcpyDeviceToDevice, s);
      for (int al = 0; al < 2; ++al) {
        const int64_t wa = po[P_MSG_W] + (int64_t)al * (2 * d + 4) * d;
        tn_w(H0, d, d, B.dPm + (int64_t)al * d, 2 * d, d, wa, d, true);
        tn_w(H0, d, d, B.dQm + (int64_t)al * d, 2 * d, d, wa + (int64_t)d * d, d, true);
        gemm<T>(s, B.dPm + (int64_t)al * d, 2 * d, p.msg_w + (int64_t)al * (2 * d + 4) * d, d, true, B.dH0, d, 0, nb,
                nullptr, nb, d, d, 1, 0, 0, 0, true);
        gemm<T>(s, B.dQm + (int64_t)al * d, 2 * d, p.msg_w + (int64_t)al * (2 * d + 4) * d + (int64_t)d * d, d, true,
                B.dH0, d, 0, nb, nullptr, nb, d, d, 1, 0, 0, 0, true);
      }
      launches += 6;
      check("bwd msg");
      // GLU and LayerNorm
      mark("bwd_glu", 0);
      gemm<T>(s, B.dH0, d, p.glu_wo, d, true, B.dP5, d, 0, nb, nullptr, nb, d, d);
      tn_w(P5, d, d, B.dH0, d, d, po[P_GLU_WO], d, true);
      gate_bwd_kernel<T><<<(unsigned)(((int64_t)nb * d + 255) / 256), 256, 0, s>>>(nb, d, Z5, B.dP5, B.dZ5);
      tn_w(Y5, d, d, B.dZ5, 2 * d, d, po[P_GLU_WG], d, true);
      tn_w(Y5, d, d, B.dZ5 + d, 2 * d, d, po[P_GLU_WV], d, true);
      gemm<T>(s, B.dZ5, 2 * d, p.glu_wg, d, true, B.dY5, d, 0, nb, nullptr, nb, d, d);
      gemm<T>(s, B.dZ5 + d, 2 * d, p.glu_wv, d, true, B.dY5, d, 0, nb, nullptr, nb, d, d, 1, 0, 0, 0, true);
      ln_bwd_kernel<T, T><<<nb, d, 0, s>>>(d, S5, B.dY5, p.ln_gamma, B.dS5, B.dyx);
      colsum_w(B.dyx, d, d, po[P_LN_GAMMA]);
      colsum_w(B.dY5, d, d, po[P_LN_BETA]);
      launches += 6;
      // electron-nucleus filters
      mark("bwd_en", 1);
      en_bwd_kernel<T, T><<<nb, d, 0, s>>>(wc, n, n_up, N, d, r, sys->nuc_pos, sys->cutoff_nuc, p, B.dS5, g, P, pod);
      check("bwd en");
    }
    mark("end", 0);
    check("final");
    flush_marks();
    if (a.n_launches) *a.n_launches = launches;
    if (failed) return FIRE_ERR_CUDA;
    {
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) { set_last_error("launch", cudaGetErrorString(e)); return FIRE_ERR_CUDA; }
    }
    if (cudaMemcpyAsync(a.host_status, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return FIRE_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FIRE_ERR_CUDA;
    return FIRE_OK;
  }

  bool reset_status = true;   // false for the refreshes inside a Metropolis call

  int run() {
    const fire_system_t* sys = a.sys;
    const int n = dm.n, n_up = dm.n_up, N = dm.N, d = dm.d, D = dm.D, K = dm.K;
    const int deriv = dm.deriv;
    const int R5 = deriv ? 5 : 1;
    DevStatus* st = at<DevStatus>(pl.status);
    if (reset_status) cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
    if constexpr (sizeof(T) == 4) {
      if (pl.wbf16) {
        // bf16 K-major copies of the weights of every tensor-core product
        mark("pack_weights", 0);
        void* WBm = at<unsigned char>(pl.wbf16);
        auto dst = [&](int64_t off) { return reinterpret_cast<__nv_bfloat16*>(WBm) + off; };
        const int64_t d = dm.d, J = dm.J, n = dm.n, D = dm.D, R = dm.R, dr = dm.dr;
        int np = 0;
        const int S = kMaxSplit;
        for (int l = 0; l < dm.L; ++l, ++np)
          tc::pack_bf16(s, reinterpret_cast<const float*>(p.mlp_w) + l * d * d, d, (int)d, (int)d, 1,
                        dst(pl.wb_mlp + S * l * d * d), S, d * d);
        const T* jw[2][2] = {{p.jm1_w1, p.jm1_w2}, {p.jm2_w1, p.jm2_w2}};
        const int64_t jo[2] = {pl.wb_jm1, pl.wb_jm2};
        for (int q = 0; q < 2; ++q) {
          tc::pack_bf16(s, reinterpret_cast<const float*>(jw[q][0]), J, (int)d, (int)J, 1, dst(jo[q]), S, d * J);
          tc::pack_bf16(s, reinterpret_cast<const float*>(jw[q][1]), J, (int)J, (int)J, 1, dst(jo[q] + S * d * J),
                        S, J * J);
          np += 2;
        }
        const int64_t acs = (R + R * dr) * d;
        tc::pack_bf16(s, reinterpret_cast<const float*>(p.att_q), d, (int)d, (int)R, 0, dst(pl.wb_att), S, acs);
        for (int rr = 0; rr < R; ++rr, ++np)
          tc::pack_bf16(s, reinterpret_cast<const float*>(p.att_wv) + rr * d * dr, dr, (int)d, (int)dr, 1,
                        dst(pl.wb_att + (R + rr * dr) * d), S, acs);
        {
          const int64_t NE = (int64_t)dm.N * dm.E, NEp = ((NE + 63) / 64) * 64, Dn = D * n;
          for (int sp = 0; sp < 2; ++sp, ++np)
            tc::pack_bf16(s, reinterpret_cast<const float*>(p.env_pi) + sp * Dn * NE, NE, (int)NE, (int)Dn, 0,
                          dst(pl.wb_env + S * sp * Dn * NEp), S, Dn * NEp, (int)NEp);
        }
        {
          // h^0 products: [W_g | W_v] (N = 2d), W_o, and the four message
          // projections [W^par_a | W^anti_a | W^par_b | W^anti_b] (N = 4d)
          tc::pack_bf16(s, reinterpret_cast<const float*>(p.glu_wg), d, (int)d, (int)d, 1, dst(pl.wb_glu), S, 2 * d * d);
          tc::pack_bf16(s, reinterpret_cast<const float*>(p.glu_wv), d, (int)d, (int)d, 1, dst(pl.wb_glu + d * d), S,
                        2 * d * d);
          tc::pack_bf16(s, reinterpret_cast<const float*>(p.glu_wo), d, (int)d, (int)d, 1, dst(pl.wb_gluo), S, d * d);
          np += 3;
          for (int part = 0; part < 2; ++part)
            for (int a = 0; a < 2; ++a, ++np)
              tc::pack_bf16(s, reinterpret_cast<const float*>(p.msg_w) + a * (2 * d + 4) * d + part * d * d, d, (int)d,
                            (int)d, 1, dst(pl.wb_msg + (part * 2 + a) * d * d), S, 4 * d * d);
          // attention register MLPs
          const int64_t RDa = R * dr;
          const T* aw[2][2] = {{p.ja1_w1, p.ja1_w2}, {p.ja2_w1, p.ja2_w2}};
          const int64_t ao[2] = {pl.wb_ja1, pl.wb_ja2};
          for (int q = 0; q < 2; ++q) {
            tc::pack_bf16(s, reinterpret_cast<const float*>(aw[q][0]), J, (int)RDa, (int)J, 1, dst(ao[q]), S, RDa * J);
            tc::pack_bf16(s, reinterpret_cast<const float*>(aw[q][1]), J, (int)J, (int)J, 1, dst(ao[q] + S * RDa * J),
                          S, J * J);
            np += 2;
          }
          // orbital value rows: all determinants of one spin in one product (N = D n)
          const int64_t Dn = D * n;
          for (int sp = 0; sp < 2; ++sp)
            for (int dd = 0; dd < D; ++dd, ++np)
              tc::pack_bf16(s, reinterpret_cast<const float*>(p.orb_w) + (sp * D + dd) * d * n, n, (int)d, (int)n, 1,
                            dst(pl.wb_orbv + S * sp * Dn * d + dd * n * d), S, Dn * d);
        }
        launches += np + 1;
      }
    }
    for (int64_t ch = 0; ch < pl.nchunks; ++ch) {
      const int64_t w0 = ch * pl.Wc;
      const int wc = (int)((a.W - w0) < pl.Wc ? (a.W - w0) : pl.Wc);
      const double* r = a.r + w0 * n * 3;
      const int nb = wc * n;
      int32_t* idx = at<int32_t>(pl.idx);
      int32_t* cnt = at<int32_t>(pl.cnt);
      int32_t* rev = at<int32_t>(pl.rev);
      int64_t* brow = at<int64_t>(pl.blk_rows);
      int64_t* boff = at<int64_t>(pl.blk_off);
      int64_t* rng = at<int64_t>(pl.ranges);
      const double c = sys->cutoff;
      // 1. neighbour lists and the ragged row layout
      mark("neighbors", 3);
      nbr_build_kernel<<<wc, 256, (size_t)n * 3 * sizeof(double), s>>>(wc, n, n_up, r, c * c, K, idx, cnt,
                                                                        brow, st, deriv);
      nbr_reverse_kernel<<<wc, 256, 0, s>>>(n, n_up, K, idx, cnt, rev);
      blk_scan_kernel<<<1, 1024, 0, s>>>(nb, wc * n_up, brow, boff, rng, st);
      // float forms with aligned rows: the tangent electrons sorted into the
      // contraction buckets by neighbourhood size
      const char* cenv = getenv("FIRE_CONTRACT");
      const bool c3 = sizeof(T) == 4 && deriv && pl.clist && n % 4 == 0 &&
                      !(cenv && (strcmp(cenv, "v1") == 0 || strcmp(cenv, "v2") == 0));
      int* ccount = pl.clist ? at<int>(pl.clist) : nullptr;
      int* clists = pl.clist ? ccount + 16 : nullptr;
      int hcount[kC3Buckets] = {0};
      // BF16_FP64 form: neighbourhoods of up to 42 members contract on the
      // tensor cores (bucket 0), larger ones in the SIMT buckets of 48 and 60
      const bool ctc = c3 && pl.wbf16 && (tc_mask & 128);
      if (c3) {
        cudaMemsetAsync(ccount, 0, 16 * sizeof(int), s);
        C3Buckets bm;
        for (int q = 0; q < kC3Buckets; ++q)
          bm.v[q] = ctc && q < 3 ? tc::kContractTcMaxMembers : kC3BucketMax[q];
        contract_bucket_kernel<0><<<(nb + 255) / 256, 256, 0, s>>>(nb, cnt, bm, ccount, clists);
        cudaMemcpyAsync(hcount, ccount, sizeof(hcount), cudaMemcpyDeviceToHost, s);
        launches += 1;
      }
      check("nbr");
      // the chunk's row total and largest neighbour count, read back once:
      // they size the grids and the contraction tiles exactly
      int64_t rows_chunk = 0;
      int32_t kreq = 0;
      cudaMemcpyAsync(&rows_chunk, rng + 3, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(&kreq, &st->k_required, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) return FIRE_ERR_CUDA;
      const int64_t cap = rows_chunk > 0 ? rows_chunk : 1;
      int64_t* fullr = at<int64_t>(pl.ranges) + 4;
      // fullr = {0, total}: written by a tiny copy below
      cudaMemcpyAsync(fullr, rng, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(fullr + 1, rng + 3, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);

      // 2. initial embeddings h^0 (5 rows per electron)
      T* S5 = at<T>(pl.S5);
      T* Y5 = at<T>(pl.Y5);
      T* Z5 = at<T>(pl.Z5);
      T* P5 = at<T>(pl.P5);
      T* H0 = at<T>(pl.H0);
      T* PQ = at<T>(pl.PQ);
      const int64_t r5 = (int64_t)nb * R5;
      mark("en_filter", 1);
      en_filter_kernel<T, T><<<nb, d, 0, s>>>(wc, n, n_up, N, d, r, sys->nuc_pos, sys->cutoff_nuc, p, S5, R5);
      // BF16 form: the h^0 products on the tensor cores (nc_h0 components)
      const __nv_bfloat16* WBh = (pl.wbf16 && (tc_mask & 32) && d % 64 == 0) ? at<__nv_bfloat16>(pl.wbf16) : nullptr;
      const int64_t r5cap = (int64_t)pl.Wc * n * R5;
      __nv_bfloat16* Y5b = WBh ? at<__nv_bfloat16>(pl.Y5b) : nullptr;
      __nv_bfloat16* P5b = WBh ? at<__nv_bfloat16>(pl.P5b) : nullptr;
      __nv_bfloat16* H0b = WBh ? at<__nv_bfloat16>(pl.H0b) : nullptr;
      auto tc_rows = [&](const __nv_bfloat16* Ab, int64_t a_rows, int64_t woff, int Nn, T* C, int64_t ldc,
                         int64_t rb, int64_t re) -> bool {
        if constexpr (sizeof(T) == 4) {
          if (!WBh) return false;
          const int rc = tc::gemm_bf16(s, Ab, d, a_rows, WBh + woff, Nn, d, reinterpret_cast<float*>(C), ldc, rb, re,
                                       nullptr, re - rb, &st->tc_err, nc_h0);
          if (rc == FIRE_OK) return true;
          tc_rc = rc;
        }
        return false;
      };
      mark("glu", 5);
      ln_fl_kernel<T, T><<<nb, d, 0, s>>>(d, S5, Y5, p.ln_gamma, p.ln_beta, R5, Y5b, nc_h0, r5cap * d);
      if (!tc_rows(Y5b, r5cap, pl.wb_glu, 2 * d, Z5, 2 * d, 0, r5)) {
        gemm<T>(s, Y5, d, p.glu_wg, d, false, Z5, 2 * d, 0, r5, nullptr, r5, d, d);
        gemm<T>(s, Y5, d, p.glu_wv, d, false, Z5 + d, 2 * d, 0, r5, nullptr, r5, d, d);
      }
      glu_gate_kernel<T><<<nb, d, 0, s>>>(d, Z5, P5, R5, P5b, nc_h0, r5cap * d);
      check("h0");
      if (!tc_rows(P5b, r5cap, pl.wb_gluo, d, H0, d, 0, r5))
        gemm<T>(s, P5, d, p.glu_wo, d, false, H0, d, 0, r5, nullptr, r5, d, d);
      // 3. h^0 W^alpha_a, h^0 W^alpha_b for both spin channels
      mark("msg_proj_gemm", 2);
      bool pq_tc = false;
      if (H0b) {
        split_rows_kernel<T><<<(unsigned)((r5 * d + 255) / 256), 256, 0, s>>>(r5, d, H0, d, H0b, d, nc_h0, r5cap * d);
        launches += 1;
        pq_tc = tc_rows(H0b, r5cap, pl.wb_msg, 4 * d, PQ, 4 * d, 0, r5);
      }
      if (!pq_tc)
        for (int part = 0; part < 2; ++part)
          gemm<T>(s, H0, d, p.msg_w + (int64_t)part * d * d, d, false, PQ + (int64_t)part * 2 * d, 4 * d, 0, r5,
                  nullptr, r5, d, d, 2, 0, (int64_t)(2 * d + 4) * d, d);
      // 4. message passing -> h^1 blocks
      T* X = at<T>(pl.X);
      T* Y = at<T>(pl.Y);
      __nv_bfloat16* Xb = pl.Xb ? at<__nv_bfloat16>(pl.Xb) : nullptr;
      __nv_bfloat16* Yb = pl.Yb ? at<__nv_bfloat16>(pl.Yb) : nullptr;
      const __nv_bfloat16* WB = pl.wbf16 ? at<__nv_bfloat16>(pl.wbf16) : nullptr;
      auto wbm = [&](int bit, int64_t off) -> const __nv_bfloat16* {
        return (WB && (tc_mask >> bit & 1)) ? WB + off : nullptr;
      };
      mark("msg", 1);
      // bf16 components of h^1: those the first MLP layer reads, else (no
      // MLP layers) all that any consumer reads
      msg_kernel<T, T><<<nb, d, 0, s>>>(wc, n, n_up, d, K, r, c, p, idx, cnt, boff, H0, PQ, X, Xb,
                                        dm.L > 0 ? nc_mlp : ncw, capA * d, deriv);
      check("msg");
      if (dm.op == FIRE_OP_MCMC) {   // the Metropolis state keeps h^1 (value rows, block order)
        cudaMemcpyAsync(at<T>(pl.mc_H1), X, sizeof(T) * (size_t)nb * d, cudaMemcpyDeviceToDevice, s);
      }
      // 5. embedding MLP h = MLP(h^1): L residual SiLU layers
      T* big = at<T>(pl.big);
      T* Z = big + pl.zcol;
      T* SU = big + pl.sucol;
      vr_off = boff;
      vr_nb = nb;
      vr_A = at<T>(pl.Hv);
      vr_C = at<T>(pl.Ov);
      // the orbital-value scratch (free until the orbital values and again
      // after them) holds the split value rows, K <= d
      vr_Ab = pl.Hvb ? at<__nv_bfloat16>(pl.Hvb) : nullptr;
      vr_cap = (int64_t)pl.Wc * dm.n;
      vr_kmax = dm.d;
      const int64_t ldb = pl.ld_big;
      for (int l = 0; l < dm.L; ++l) {
        mark("mlp_gemm", 1);
        row_gemm(X, Xb, d, capA, p.mlp_w + (int64_t)l * d * d, wbm(0, pl.wb_mlp + kMaxSplit * (int64_t)l * d * d),
                 d, Z, ldb, fullr, 0, 0, cap, d, d, nc_mlp);
        mark("fl_act", 1);
        // the bf16 components of the hidden rows: those the next layer's
        // product reads, all that any consumer reads after the last layer
        const int ncl = l + 1 < dm.L ? nc_mlp : ncw;
        fl_act(d, boff, 0, Z, ldb, p.mlp_b + (int64_t)l * d, X, d, 1, Xb, ncl, capA * d, 1, nb);
      }
      // 7. envelopes and orbital values
      const int E = dm.E, NE = N * E;
      const int64_t Dn = (int64_t)D * n;
      T* Qf = at<T>(pl.Qf);
      T* Fenv = at<T>(pl.Fenv);
      mark("envelope", 3);
      // BF16 form: the features also as bf16 components (K padded to a
      // multiple of 64) for the tensor-core product with the packed pi
      const int NEp = ((NE + 63) / 64) * 64;
      __nv_bfloat16* Qfb = (pl.Qfb && WB && (tc_mask & 16)) ? at<__nv_bfloat16>(pl.Qfb) : nullptr;
      env_feat_kernel<T, T><<<nb, 128, 0, s>>>(wc, n, n_up, N, E, r, sys->nuc_pos, p.env_sigma, Qf, R5, Qfb, NEp,
                                               nc_env, r5cap * NEp);
      const int64_t up5 = (int64_t)wc * n_up * R5;
      for (int sp = 0; sp < 2; ++sp) {
        const int64_t rb = sp ? up5 : 0, re = sp ? r5 : up5;
        if (re <= rb) continue;
        if constexpr (sizeof(T) == 4) {
          if (Qfb) {
            const int rc = tc::gemm_bf16(s, Qfb, NEp, r5cap, WB + pl.wb_env + (int64_t)kMaxSplit * sp * Dn * NEp,
                                         (int)Dn, NEp, reinterpret_cast<float*>(Fenv), Dn, rb, re, nullptr, re - rb,
                                         &st->tc_err, nc_env);
            if (rc == FIRE_OK) continue;
            tc_rc = rc;
          }
        }
        gemm<T>(s, Qf, NE, p.env_pi + (int64_t)sp * Dn * NE, NE, true, Fenv, Dn, rb, re, nullptr, re - rb,
                (int)Dn, NE);
      }
      T* Hv = at<T>(pl.Hv);
      T* Ov = at<T>(pl.Ov);
      mark("orb_values", 4);
      __nv_bfloat16* Hvb = WBh ? at<__nv_bfloat16>(pl.Hvb) : nullptr;
      const int64_t nbcap = (int64_t)pl.Wc * n;
      gather_value_rows_kernel<T><<<nb, 256, 0, s>>>(nb, d, boff, X, Hv, -1, Hvb, nc_h0, nbcap * d);
      const int64_t upv = (int64_t)wc * n_up;
      for (int sp = 0; sp < 2; ++sp) {
        const int64_t rb = sp ? upv : 0, re = sp ? nb : upv;
        if (re <= rb) continue;
        if (Hvb && tc_rows(Hvb, nbcap, pl.wb_orbv + (int64_t)kMaxSplit * sp * Dn * d, (int)Dn, Ov, Dn, rb, re))
          continue;
        gemm<T>(s, Hv, d, p.orb_w + (int64_t)sp * D * d * n, n, false, Ov, Dn, rb, re, nullptr, re - rb, n, d,
                D, 0, (int64_t)d * n, n);
      }
      LT* LUb = at<LT>(pl.LU);
      int32_t* piv = at<int32_t>(pl.piv);
      double* ldabs = at<double>(pl.ldabs);
      double* lsign = at<double>(pl.lsign);
      // A^T: float32 Gauss-Jordan from a float copy of Phi (float32 forms,
      // n <= 192), else triangular solves on the LU factors
      const bool gj = use_gj && deriv && sizeof(T) == 4 && n <= 192;
      float* Phif = gj ? at<float>(pl.Phif) : nullptr;
      phi_assemble_kernel<T, LT><<<wc * D, 256, 0, s>>>(wc, n, n_up, D, Ov, Fenv, R5, LUb, Phif);
      const bool mc = dm.op == FIRE_OP_MCMC;
      if (mc) {
        // the Metropolis state keeps Phi itself next to its factors
        convert_kernel<LT, T><<<1024, 256, 0, s>>>((int64_t)wc * D * n * n, LUb, at<T>(pl.PhiS));
        launches += 1;
      }
      const size_t lusm = lu_smem_bytes(n, sizeof(LT));
      // slogdet: when the inverse does not come from these factors (float
      // forms: Gauss-Jordan on a float copy of Phi; value-only calls), the
      // float64 LU may run on a second stream (FIRE_LU_SIDE=1) and join before
      // the final combination
      lu_side = !mc && (!deriv || gj) && side_ready();
      // with the derivatives, the fork waits until the Gauss-Jordan inverse is
      // enqueued: the LU then shares the SMs with the orbital products and
      // the contraction, whose CTAs leave room for it
      auto launch_lu_side = [&]() {
        cudaEventRecord(ev_fork, s);
        cudaStreamWaitEvent(s2, ev_fork, 0);
        lu_kernel<LT, 16><<<wc * D, 256, lusm, s2>>>(n, LUb, piv, ldabs, lsign);
        cudaEventRecord(ev_join, s2);
      };
      mark("lu", 1);
      if (lu_side) {
        if (!deriv) launch_lu_side();
      } else {
        if (lu_nb == 32) lu_kernel<LT, 32><<<wc * D, 256, lu_smem_bytes(n, sizeof(LT), 32), s>>>(n, LUb, piv, ldabs, lsign);
        else lu_kernel<LT, 16><<<wc * D, 256, lusm, s>>>(n, LUb, piv, ldabs, lsign);
      }
      check("lu");
      if (mc) {
        // A^T = (Phi^-1)^T from the float64 factors
        mark("inverse", 1);
        const int64_t nmat = (int64_t)wc * D;
        const size_t ism = inverse_panel_smem(n, sizeof(LT));
        for (int64_t m0 = 0; m0 < nmat; m0 += 65535) {
          const int64_t cnt = nmat - m0 < 65535 ? nmat - m0 : 65535;
          inverse_panel_kernel<LT, LT, T><<<(unsigned)cnt, 256, ism, s>>>(n, m0, LUb, piv, at<T>(pl.Ainv));
          launches += 1;
        }
        check("inverse");
      }
      T* gdet = at<T>(pl.gdet);
      T* ldet = at<T>(pl.ldet);
      if (deriv) {
        T* Ainv = at<T>(pl.Ainv);
        mark("inverse", 1);
        if (gj) {
          const int thr = gj_threads(n);
          // pivot rows from the float64 LU when it has already run on this stream
          if (lu_side) gj_inverse_kernel<float, T><<<wc * D, thr, gj_smem_bytes(n), s>>>(n, Phif, Ainv);
          else gj_inverse_pre_kernel<float, T><<<wc * D, thr, gj_smem_bytes(n), s>>>(n, Phif, Ainv, piv);
        } else {
          inverse_from_lu(n, (int64_t)wc * D, LUb, piv, Ainv);
        }
        if (lu_side) launch_lu_side();
      check("inverse");
        // 8. log-det gradient and Laplacian, determinant by determinant
        T* O = big;  // aliases Z | Y | SU, which are dead by now
        vr_off = nullptr;   // orbital values come from the Ov product
        const int kmax = kreq < K ? kreq : K;
        const int mcap = 1 + (kmax < n - 1 ? kmax : n - 1);
        const int maxt = contract_maxt(mcap);
        if (maxt == 0) { set_last_error("contract", "neighbourhood larger than 96 members"); return FIRE_ERR_UNSUPPORTED; }
        const size_t ctsm = contract_smem_bytes(mcap, sizeof(T));
        // float forms: the bucketed small-CTA contraction for neighbourhoods
        // of up to 60 members; FIRE_CONTRACT=v1 keeps the 256-thread kernel
        // (diagnostic)
        const bool c2 = sizeof(T) == 4 && mcap <= kC2BigMax && !(cenv && strcmp(cenv, "v1") == 0);
        // orbital rows of G determinants per product (BF16 form: one slice of
        // the packed [D n][d] weights of a spin, so X is read D / G times)
        int G = 1;
        const __nv_bfloat16* WBo = wbm(3, pl.wb_orbv);
        if (WBo && d % 64 == 0) G = (int)(pl.ld_big / n) < kOrbGroup ? (int)(pl.ld_big / n) : kOrbGroup;
        if (G < 1) G = 1;
        for (int dd0 = 0; dd0 < D; dd0 += G) {
          const int g = D - dd0 < G ? D - dd0 : G;
          const int64_t ldo = (int64_t)g * n;
          mark("orb_gemm", 2);
          for (int sp = 0; sp < 2; ++sp) {
            bool done = false;
            if constexpr (sizeof(T) == 4) {
              if (WBo && d % 64 == 0) {
                const int rc = tc::gemm_bf16_rows(s, Xb, d, capA, WBo + (int64_t)kMaxSplit * sp * Dn * d, (int)Dn,
                                                  dd0 * n, g * n, d, reinterpret_cast<float*>(O), ldo, 0, 0,
                                                  rng + 2 * sp, cap, &st->tc_err, nc_orb);
                if (rc == FIRE_OK) done = true;
                else tc_rc = rc;
              }
            }
            if (!done)
              for (int j = 0; j < g; ++j)
                gemm<T>(s, X, d, p.orb_w + ((int64_t)sp * D + dd0 + j) * d * n, n, false, O + (int64_t)j * n, ldo,
                        0, 0, rng + 2 * sp, cap, n, d);
          }
          if constexpr (sizeof(T) == 4) {
            if (ctc && c2 && hcount[0] > 0) {
              // neighbourhoods of up to 42 members, all g determinants of the group in one launch
              mark("contract", 1);
              const int rc = tc::contract_tc(s, wc, n, n_up, K, dd0, g, D, idx, cnt, rev, boff,
                                             reinterpret_cast<const float*>(O), ldo,
                                             reinterpret_cast<const float*>(Fenv),
                                             reinterpret_cast<const float*>(Ainv), reinterpret_cast<float*>(gdet),
                                             reinterpret_cast<float*>(ldet), st, clists, hcount[0], &st->tc_err);
              if (rc != FIRE_OK) { set_last_error("contract", "tensor-core contraction launch failed"); return rc; }
              launches += 1;
              check("contract");
            }
          }
          for (int j = 0; j < g; ++j) {
            const int dd = dd0 + j;
            const T* Oj = O + (int64_t)j * n;
            mark("contract", 1);
            if constexpr (sizeof(T) == 4) {
              if (c3 && c2) {
                // one launch per non-empty bucket, over exactly its electrons
                for (int q = ctc ? 1 : 0; q < kC3Buckets; ++q) {
                  if (hcount[q] <= 0) continue;
                  auto kern = q == 0 ? contract3_kernel<64>
                                     : (q == 1 ? contract3_kernel<96>
                                               : (q == 2 ? contract3_kernel<128>
                                                         : (q == 3 ? contract3_kernel<192> : contract3_kernel<320>)));
                  kern<<<hcount[q], kC3BucketThreads[q], contract3_smem_bytes(kC3BucketMax[q]), s>>>(
                      wc, n, n_up, K, 1, kC3BucketMax[q], dd, D, idx, cnt, rev, boff,
                      reinterpret_cast<const float*>(Oj), ldo, reinterpret_cast<const float*>(Fenv),
                      reinterpret_cast<const float*>(Ainv), reinterpret_cast<float*>(gdet),
                      reinterpret_cast<float*>(ldet), st, clists + (int64_t)q * nb);
                  launches += 1;
                }
                check("contract");
                continue;
              }
              if (c2) {
                // one launch per neighbourhood-size bucket that the chunk reaches
                int lo = 1;
                for (int q = 0; q < kC2Buckets && lo <= mcap; ++q) {
                  const int hi = mcap < kC2BucketMax[q] ? mcap : kC2BucketMax[q];
                  auto kern = q == 0 ? contract2_kernel<64, 1>
                                     : (q == 1 ? contract2_kernel<128, 1> : contract2_kernel<320, 1>);
                  kern<<<nb, kC2BucketThreads[q], contract2_smem_bytes(hi), s>>>(
                      wc, n, n_up, K, lo, hi, dd, D, idx, cnt, rev, boff, reinterpret_cast<const float*>(Oj), ldo,
                      reinterpret_cast<const float*>(Fenv), reinterpret_cast<const float*>(Ainv),
                      reinterpret_cast<float*>(gdet), reinterpret_cast<float*>(ldet), st);
                  if (q > 0) launches += 1;
                  lo = hi + 1;
                }
                check("contract");
                continue;
              }
            }
            auto ck = contract_kernel<T, 1>;
            if (maxt == 2) ck = contract_kernel<T, 2>;
            else if (maxt == 3) ck = contract_kernel<T, 3>;
            else if (maxt == 5) ck = contract_kernel<T, 5>;
            else if (maxt == 9) ck = contract_kernel<T, 9>;
            ck<<<nb, 256, ctsm, s>>>(wc, n, n_up, K, mcap, dd, D, idx, cnt, rev, boff, Oj, ldo, Fenv, Ainv, gdet, ldet,
                                     st);
            check("contract");
          }
        }
      }
      // 6. Jastrow factors (after the log-det derivatives, so the float64 LU
      // on the second stream runs beside the contraction kernels, whose small
      // CTAs leave room for it)
      vr_off = boff;   // value rows of the Jastrow products recomputed in fp32
      T* jval = at<T>(pl.jval); T* jsign = at<T>(pl.jsign); T* jgrad = at<T>(pl.jgrad); T* jlap = at<T>(pl.jlap);
      T* aval = at<T>(pl.aval); T* asign = at<T>(pl.asign); T* agrad = at<T>(pl.agrad); T* alap = at<T>(pl.alap);
      T* cval = at<T>(pl.cval); T* cgrad = at<T>(pl.cgrad); T* clap = at<T>(pl.clap); T* vpot = at<T>(pl.vpot);
      if (dm.flags & FIRE_J_MLP) {
        mark("jastrow_mlp", 10);
        T* F1 = at<T>(pl.F1);
        T* F2 = at<T>(pl.F2);
        const int64_t JJ = (int64_t)dm.J;
        mlp_readout(X, Xb, d, d, fullr, 0, 0, cap, boff, 0, nb, p.jm1_w1, wbm(1, pl.wb_jm1), p.jm1_b1, p.jm1_w2,
                    wbm(1, pl.wb_jm1 + kMaxSplit * d * JJ), p.jm1_b2, p.jm1_w3, Z, ldb, Y, Yb, JJ, F1);
        mlp_readout(X, Xb, d, d, fullr, 0, 0, cap, boff, 0, nb, p.jm2_w1, wbm(1, pl.wb_jm2), p.jm2_b1, p.jm2_w2,
                    wbm(1, pl.wb_jm2 + kMaxSplit * d * JJ), p.jm2_b2, p.jm2_w3, Z, ldb, Y, Yb, JJ, F2);
        mark("jastrow_reduce", 1);
        jmlp_reduce_kernel<T, T><<<wc, 256, 0, s>>>(wc, n, n_up, K, idx, cnt, rev, boff, F1, F2, p.jm1_b3,
                                                    p.jm2_b3, jval, jsign, jgrad, jlap, deriv);
      check("jmlp");
      }
      if (dm.flags & FIRE_J_ATT) {
        const int R = dm.R, dr = dm.dr, RD = R * dr;
        mark("att_gemm", 2);
        bool att_tc = false;
        if constexpr (sizeof(T) == 4) {
          if (Xb && WB && d % 64 == 0 && (tc_mask & 4))
            att_tc = tc::gemm_bf16(s, Xb, d, capA, WB + pl.wb_att, R + RD, d, reinterpret_cast<float*>(SU), ldb, 0,
                                   0, fullr, cap, &st->tc_err, nc_att) == FIRE_OK;
        }
        if (!att_tc) {
          gemm<T>(s, X, d, p.att_q, d, true, SU, ldb, 0, 0, fullr, cap, R, d);
          gemm<T>(s, X, d, p.att_wv, dr, false, SU + R, ldb, 0, 0, fullr, cap, dr, d, R, 0, (int64_t)d * dr, dr);
        }
        T* V = at<T>(pl.V);
        T* VZ = at<T>(pl.VZ);
        T* VY = at<T>(pl.VY);
        T* G1 = at<T>(pl.G1);
        T* G2 = at<T>(pl.G2);
        const int bt = ((RD + 31) / 32) * 32;
        __nv_bfloat16* Vb = pl.Vb ? at<__nv_bfloat16>(pl.Vb) : nullptr;
        if (deriv) {
          // per-electron partial records, then ordered sums per walker
          T* AP = at<T>(pl.AP);
          mark("att_pool", 3);
          att_max_kernel<T><<<wc, 256, 0, s>>>(wc, n, n_up, R, boff, SU, ldb, AP);
          att_part_kernel<T><<<nb, bt, 0, s>>>(wc, n, n_up, K, R, dr, idx, cnt, rev, boff, SU, ldb, AP);
          att_fin_kernel<T><<<dim3(wc, 8), bt, 0, s>>>(wc, n, R, dr, AP, V, Vb, 3,
                                                        (int64_t)pl.Wc * (2 + 3 * (int64_t)n) * RD);
        } else {
          const size_t apsm = (size_t)(R + n * R) * sizeof(T);
          mark("att_pool", 1);
          att_pool_kernel<T><<<wc, bt, apsm, s>>>(wc, n, n_up, K, R, dr, idx, cnt, rev, boff, SU, ldb, V, deriv);
        }
        const int64_t vstride = deriv ? (2 + 3 * (int64_t)n) : 1;
        const int64_t vrows = (int64_t)wc * vstride;
        mark("att_mlp", 11);
        // BF16 form: the register MLPs on the tensor cores, three components
        // (their value rows set log|J_att| and get no fp32 recompute)
        const int64_t JJ = dm.J;
        const __nv_bfloat16* WBa = (Vb && WB && (tc_mask & 64) && RD % 64 == 0 && JJ % 64 == 0) ? WB : nullptr;
        __nv_bfloat16* VYb = WBa ? at<__nv_bfloat16>(pl.VYb) : nullptr;
        const int64_t vcap = (int64_t)pl.Wc * vstride;
        auto wa = [&](int64_t off) -> const __nv_bfloat16* { return WBa ? WBa + off : nullptr; };
        mlp_readout(V, WBa ? Vb : nullptr, RD, RD, nullptr, 0, vrows, vrows, nullptr, vstride, wc, p.ja1_w1,
                    wa(pl.wb_ja1), p.ja1_b1, p.ja1_w2, wa(pl.wb_ja1 + kMaxSplit * (int64_t)RD * JJ), p.ja1_b2, p.ja1_w3,
                    VZ, JJ, VY, VYb, JJ, G1, vcap, 3);
        mlp_readout(V, WBa ? Vb : nullptr, RD, RD, nullptr, 0, vrows, vrows, nullptr, vstride, wc, p.ja2_w1,
                    wa(pl.wb_ja2), p.ja2_b1, p.ja2_w2, wa(pl.wb_ja2 + kMaxSplit * (int64_t)RD * JJ), p.ja2_b2, p.ja2_w3,
                    VZ, JJ, VY, VYb, JJ, G2, vcap, 3);
        att_reduce_kernel<T, T><<<wc, 256, 0, s>>>(n, G1, G2, p.ja1_b3, p.ja2_b3, aval, asign, agrad, alap, deriv);
      check("att");
      }
      mark("coulomb_cusp", 1);
      coulomb_cusp_kernel<T, T><<<wc, 256, 0, s>>>(n, n_up, N, r, sys->nuc_pos, sys->nuc_charge, p.cusp, vpot,
                                                   cval, cgrad, clap, deriv);
      // 9. final combination
      if (lu_side) cudaStreamWaitEvent(s, ev_join, 0);
      FinalIn<T, RT> fi{ldabs, lsign, gdet, ldet, cval, cgrad, clap, jval, jsign, jgrad, jlap,
                        aval, asign, agrad, alap, vpot};
      mark("final", 1);
      final_kernel<T, RT><<<wc, 256, 0, s>>>(n, D, dm.flags, fi, deriv, a.e_loc ? a.e_loc + w0 : nullptr,
                                             a.logabs + w0, a.sign + w0, a.e_kin ? a.e_kin + w0 : nullptr,
                                             a.e_pot ? a.e_pot + w0 : nullptr, st);
    }
    mark("end", 0);
    check("final");
    flush_marks();
    if (a.n_launches) *a.n_launches = launches;
    if (tc_rc != FIRE_OK) { set_last_error("tensor-core product", "setup failed; SIMT fallback used"); }
    if (failed) return FIRE_ERR_CUDA;
    {
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) { set_last_error("launch", cudaGetErrorString(e)); return FIRE_ERR_CUDA; }
    }
    if (cudaMemcpyAsync(a.host_status, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return FIRE_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FIRE_ERR_CUDA;
    return FIRE_OK;
  }

  // ---------------------------------------------------------------------
  // Metropolis sweeps with local recompute and low-rank updates.  The state
  // (embeddings h^0 and their projections, envelope rows, Phi, A^T,
  // determinant logs, Jastrow sums, attention scores) is built by a value
  // forward at the start, rebuilt every refresh_every moves and at the end;
  // the drift of the carried log|Psi| against each rebuild is recorded.
  // ---------------------------------------------------------------------
  int run_mcmc() {
    McmcCall& mc = *a.mcmc;
    const fire_system_t* sys = a.sys;
    const int n = dm.n, n_up = dm.n_up, N = dm.N, d = dm.d, D = dm.D, E = dm.E, NE = N * E;
    const int J = dm.J, R = dm.R, dr = dm.dr, RD = R * dr, RD1 = R + RD;
    const int Wn = (int)a.W;
    const int Umax = pl.Umax;
    const int64_t capU = (int64_t)Wn * Umax, Dn = (int64_t)D * n;
    const int64_t ldz = d > J ? d : J;
    double* r = const_cast<double*>(a.r);
    DevStatus* st = at<DevStatus>(pl.status);
    McmcStat* ms = at<McmcStat>(pl.mc_stat);
    double* rk = at<double>(pl.mc_rk);
    double* uacc = at<double>(pl.mc_u);
    int32_t* Ul = at<int32_t>(pl.mc_Ul);
    int32_t* Uc = at<int32_t>(pl.mc_Uc);
    int32_t* Ucu = at<int32_t>(pl.mc_Ucu);
    int32_t* Urow = at<int32_t>(pl.mc_Urow);
    int64_t* rngu = at<int64_t>(pl.mc_rng);        // {0, up, up, total, 0, total, 0, W}
    T* h0k = at<T>(pl.mc_h0k);
    T* PQk = at<T>(pl.mc_PQk);
    T* Qk = at<T>(pl.mc_Qk);
    T* Fk = at<T>(pl.mc_Fk);
    T* X1 = at<T>(pl.mc_X);
    T* Zm = at<T>(pl.mc_Z);
    T* Ym = at<T>(pl.mc_Y);
    T* F1n = at<T>(pl.mc_F1n);
    T* F2n = at<T>(pl.mc_F2n);
    T* SUn = at<T>(pl.mc_SUn);
    T* On = at<T>(pl.mc_On);
    T* Vn = at<T>(pl.mc_Vn);
    T* VZ = at<T>(pl.mc_VZ);
    T* VY = at<T>(pl.mc_VY);
    T* G1n = at<T>(pl.mc_G1n);
    T* G2n = at<T>(pl.mc_G2n);
    T* Dl = at<T>(pl.mc_Dl);
    T* Mt = at<T>(pl.mc_Mt);
    double* Mlu = at<double>(pl.mc_Mlu);
    int32_t* Mpiv = at<int32_t>(pl.mc_piv);
    double* lrat = at<double>(pl.mc_lrat);
    double* srat = at<double>(pl.mc_srat);
    int32_t* acc = at<int32_t>(pl.mc_acc);
    T* Tu = at<T>(pl.mc_Tu);
    T* Bw = at<T>(pl.mc_Bw);
    double* lp = at<double>(pl.mc_lp);
    double* lpf = at<double>(pl.mc_lpf);
    double* wdrift = at<double>(pl.mc_wdrift);
    T* H1 = at<T>(pl.mc_H1);
    T* H1n = at<T>(pl.mc_H1n);
    double* lref = at<double>(pl.mc_lref);
    int32_t* flag = at<int32_t>(pl.mc_flag);
    int32_t* xflag = at<int32_t>(pl.mc_xflag);
    // the state, in the value-forward buffers
    T* H0 = at<T>(pl.H0);
    T* PQ = at<T>(pl.PQ);
    T* Fenv = at<T>(pl.Fenv);
    T* F1 = at<T>(pl.F1);
    T* F2 = at<T>(pl.F2);
    T* SU = at<T>(pl.big) + pl.sucol;
    T* V = at<T>(pl.V);
    T* G1 = at<T>(pl.G1);
    T* G2 = at<T>(pl.G2);
    T* PhiS = at<T>(pl.PhiS);
    T* AT = at<T>(pl.Ainv);
    double* ldabs = at<double>(pl.ldabs);
    double* lsign = at<double>(pl.lsign);
    T* S5 = at<T>(pl.S5);
    T* Y5 = at<T>(pl.Y5);
    T* Z5 = at<T>(pl.Z5);
    T* P5 = at<T>(pl.P5);

    cudaMemsetAsync(ms, 0, sizeof(McmcStat), s);
    if (mc.acc_count) cudaMemsetAsync(mc.acc_count, 0, sizeof(int32_t) * (size_t)Wn, s);
    {
      const int64_t wr[2] = {0, (int64_t)Wn};
      cudaMemcpyAsync(rngu + 6, wr, sizeof(wr), cudaMemcpyHostToDevice, s);
      // the host array is a stack temporary: finish the copy before it goes
      if (cudaStreamSynchronize(s) != cudaSuccess) return FIRE_ERR_CUDA;
    }
    const int64_t* fullu = rngu + 4;
    const int64_t* rowsW = rngu + 6;
    float* kap = at<float>(pl.mc_kap);
    double* lq = at<double>(pl.mc_lq);
    auto refresh = [&](bool measure) -> int {
      int rc = run();
      reset_status = false;
      if (rc != FIRE_OK) return rc;
      mcmc_kappa_kernel<T><<<(unsigned)((int64_t)Wn * D), 256, 0, s>>>(n, PhiS, AT, kap);
      launches += 1;
      cudaMemcpyAsync(lref, at<double>(pl.ldabs), sizeof(double) * (size_t)Wn * D, cudaMemcpyDeviceToDevice, s);
      mcmc_drift_kernel<<<(Wn + 255) / 256, 256, 0, s>>>(Wn, lp, lpf, wdrift, &ms->drift_bits, measure ? 1 : 0);
      launches += 1;
      return FIRE_OK;
    };
    int rc = refresh(false);
    if (rc != FIRE_OK) return rc;

    const double c = sys->cutoff;
    const unsigned actg = 152 * 8;
    const McmcJastrow jp{p.cusp, p.jm2_b3, p.ja2_b3};
    const size_t msm = (size_t)n * sizeof(int);
    const size_t asm_ = (((size_t)n * sizeof(int) + 15) & ~(size_t)15) + (size_t)R * sizeof(T);
    const int abt = RD < 1024 ? ((RD + 31) / 32) * 32 : 1024;
    // two-hidden-layer SiLU readout over rows [rng[0], rng[1]); Zb has row stride ldzb
    auto readout = [&](const T* Xin, int din, const int64_t* rng, int64_t cap, const T* w1, const T* b1,
                       const T* w2, const T* b2, const T* w3, T* Zb, int64_t ldzb, T* Yb, T* F) {
      gemm<T>(s, Xin, din, w1, J, false, Zb, ldzb, 0, 0, rng, cap, J, din);
      mcmc_act_kernel<T, T><<<actg, 256, 0, s>>>(rng, J, Zb, ldzb, b1, Yb, J, 0);
      gemm<T>(s, Yb, J, w2, J, false, Zb, ldzb, 0, 0, rng, cap, J, J);
      mcmc_act_kernel<T, T><<<actg, 256, 0, s>>>(rng, J, Zb, ldzb, b2, Yb, J, 0);
      rowdot_kernel<T, T><<<(unsigned)((cap + 7) / 8), 256, 0, s>>>(Yb, J, J, w3, F, rng, 0, 0);
      launches += 5;
    };
    // unit roundoff of the state, for the conditioning test of the exact ratios
    const double kunit = sizeof(T) == 4 ? 5.9604644775390625e-8 : 1.1102230246251565e-16;
    // The recompute of one move of electron k to rk (update sets built): h^0,
    // projections and envelope row of k, h^1 and h of the update set, Jastrow
    // rows, attention registers, orbital rows and the determinant ratios.
    auto embed_and_msg = [&](int k) {
      mcmc_scan_kernel<<<1, 1024, 0, s>>>(Wn, Umax, Uc, Ucu, Urow, rngu);
      // h^0, its projections and the envelope row of electron k at r'_k
      // (the proposals form a one-electron batch of Wn walkers)
      const int nup1 = k < n_up ? 1 : 0;
      mark("mc_embed_k", 9);
      en_filter_kernel<T, T><<<Wn, d, 0, s>>>(Wn, 1, nup1, N, d, rk, sys->nuc_pos, sys->cutoff_nuc, p, S5, 1);
      ln_fl_kernel<T, T><<<Wn, d, 0, s>>>(d, S5, Y5, p.ln_gamma, p.ln_beta, 1);
      gemm<T>(s, Y5, d, p.glu_wg, d, false, Z5, 2 * d, 0, Wn, nullptr, Wn, d, d);
      gemm<T>(s, Y5, d, p.glu_wv, d, false, Z5 + d, 2 * d, 0, Wn, nullptr, Wn, d, d);
      glu_gate_kernel<T><<<Wn, d, 0, s>>>(d, Z5, P5, 1);
      gemm<T>(s, P5, d, p.glu_wo, d, false, h0k, d, 0, Wn, nullptr, Wn, d, d);
      for (int part = 0; part < 2; ++part)
        gemm<T>(s, h0k, d, p.msg_w + (int64_t)part * d * d, d, false, PQk + (int64_t)part * 2 * d, 4 * d, 0, Wn,
                nullptr, Wn, d, d, 2, 0, (int64_t)(2 * d + 4) * d, d);
      env_feat_kernel<T, T><<<Wn, 128, 0, s>>>(Wn, 1, nup1, N, E, rk, sys->nuc_pos, p.env_sigma, Qk, 1);
      gemm<T>(s, Qk, NE, p.env_pi + (int64_t)(k < n_up ? 0 : 1) * Dn * NE, NE, true, Fk, Dn, 0, Wn, nullptr, Wn,
              (int)Dn, NE);
      check("mc embed k");
      // h^1 and h of the members of U (compact rows)
      mark("mc_msg", 1);
      mcmc_msg_kernel<T, T><<<(unsigned)capU, d, msm, s>>>(Wn, n, n_up, d, k, Umax, r, rk, c, p, Ul, Uc, Urow, H0,
                                                           PQ, H1, h0k, PQk, X1, H1n);
      check("mc msg");
    };
    // MLP, Jastrow and attention rows of the update set, its orbital rows
    // and the determinant ratios (k2 >= 0: a second moved electron whose
    // envelope row is Fk2)
    auto rows_and_ratio = [&](int k, int k2, const T* Fk2) {
      mark("mc_mlp", 2 * dm.L);
      for (int l = 0; l < dm.L; ++l) {
        gemm<T>(s, X1, d, p.mlp_w + (int64_t)l * d * d, d, false, Zm, ldz, 0, 0, fullu, capU, d, d);
        mcmc_act_kernel<T, T><<<actg, 256, 0, s>>>(fullu, d, Zm, ldz, p.mlp_b + (int64_t)l * d, X1, d, 1);
      }
      if (dm.flags & FIRE_J_MLP) {
        mark("mc_jastrow", 0);
        readout(X1, d, fullu, capU, p.jm1_w1, p.jm1_b1, p.jm1_w2, p.jm1_b2, p.jm1_w3, Zm, ldz, Ym, F1n);
        readout(X1, d, fullu, capU, p.jm2_w1, p.jm2_b1, p.jm2_w2, p.jm2_b2, p.jm2_w3, Zm, ldz, Ym, F2n);
      }
      if (dm.flags & FIRE_J_ATT) {
        mark("mc_att", 3);
        gemm<T>(s, X1, d, p.att_q, d, true, SUn, RD1, 0, 0, fullu, capU, R, d);
        gemm<T>(s, X1, d, p.att_wv, dr, false, SUn + R, RD1, 0, 0, fullu, capU, dr, d, R, 0, (int64_t)d * dr, dr);
        mcmc_att_kernel<T><<<Wn, abt, asm_, s>>>(Wn, n, n_up, R, dr, Umax, Ul, Uc, Urow, SU, pl.ld_big, SUn, RD1,
                                                  Vn);
        readout(Vn, RD, rowsW, Wn, p.ja1_w1, p.ja1_b1, p.ja1_w2, p.ja1_b2, p.ja1_w3, VZ, J, VY, G1n);
        readout(Vn, RD, rowsW, Wn, p.ja2_w1, p.ja2_b1, p.ja2_w2, p.ja2_b2, p.ja2_w3, VZ, J, VY, G2n);
      }
      // orbital rows of U, spin-up rows with the up-spin weights
      mark("mc_orb", 2);
      for (int sp = 0; sp < 2; ++sp)
        gemm<T>(s, X1, d, p.orb_w + (int64_t)sp * D * d * n, n, false, On, Dn, 0, 0, rngu + 2 * sp, capU, n, d, D,
                0, (int64_t)d * n, n);
      check("mc orbitals");
      mark("mc_ratio", 1);
      mcmc_ratio_kernel<T><<<(unsigned)(Wn * D), 256, 0, s>>>(Wn, n, n_up, D, k, Umax, Ul, Uc, Urow, On, Fenv, Fk,
                                                             PhiS, AT, Dl, Mt, Mlu, Mpiv, lrat, srat, k2,
                                                             Fk2);
      {
        const int64_t npair = (int64_t)Wn * D;
        int* xcnt = at<int>(pl.mc_xcnt);
        int32_t* xlist = at<int32_t>(pl.mc_xlist);
        const bool batched = mc.kappa_tol >= 0.0;
        if (batched) cudaMemsetAsync(xcnt, 0, sizeof(int), s);
        mcmc_exact_ratio_kernel<T, LT><<<(unsigned)(npair < kWoodburySlots ? npair : kWoodburySlots), 256,
                                         (size_t)n * sizeof(int), s>>>(
            Wn, n, D, Umax, Ul, Uc, PhiS, Dl, ldabs, lsign, lrat, srat, xflag, at<LT>(pl.mc_rep),
            at<int32_t>(pl.mc_rpiv), kap, kunit, mc.kappa_tol, xcnt, batched ? xlist : nullptr, pl.xcap,
            &ms->n_exact);
        launches += 1;
        if (batched) {
          // ill-conditioned determinants: float64 LU of Phi' over all SMs
          LT* xb = at<LT>(pl.mc_xbatch);
          double* xlab = at<double>(pl.mc_xlab);
          double* xsg = at<double>(pl.mc_xsg);
          mcmc_exact_build_kernel<T, LT><<<pl.xcap, 256, (size_t)n * sizeof(int), s>>>(n, D, Umax, xcnt, xlist, Ul, Uc,
                                                                                       PhiS, Dl, xb);
          lu_kernel<LT, 16><<<pl.xcap, 256, lu_smem_bytes(n, sizeof(LT)), s>>>(n, xb, at<int32_t>(pl.mc_xpiv), xlab,
                                                                               xsg, xcnt);
          mcmc_exact_scatter_kernel<<<(pl.xcap + 255) / 256, 256, 0, s>>>(xcnt, pl.xcap, xlist, xlab, xsg, ldabs,
                                                                         lsign, lrat, srat);
          launches += 3;
        }
      }
      check("mc ratio");
    };
    auto evaluate_move = [&](int k) {
      embed_and_msg(k);
      rows_and_ratio(k, -1, nullptr);
    };
    if (mc.swap_beta >= 0) {
      // S+ ratios: n_up swaps of the spin-down electron beta with every
      // spin-up electron, from the state just built; nothing is accepted
      const int b = mc.swap_beta;
      double* rk2 = at<double>(pl.mc_rk2);
      T* Fk2 = at<T>(pl.mc_Fk2);
      for (int a2 = 0; a2 < n_up; ++a2) {
        mark("swap_propose", 2);
        swap_propose_kernel<<<Wn, 32, 0, s>>>(n, n_up, a2, b, r, c * c, Umax, rk, rk2, Ul, Uc, Ucu, st);
        mcmc_scan_kernel<<<1, 1024, 0, s>>>(Wn, Umax, Uc, Ucu, Urow, rngu);
        // envelope rows of both electrons at their new positions, each with
        // its own spin's weights
        mark("swap_env", 4);
        env_feat_kernel<T, T><<<Wn, 128, 0, s>>>(Wn, 1, 1, N, E, rk, sys->nuc_pos, p.env_sigma, Qk, 1);
        gemm<T>(s, Qk, NE, p.env_pi, NE, true, Fk, Dn, 0, Wn, nullptr, Wn, (int)Dn, NE);
        env_feat_kernel<T, T><<<Wn, 128, 0, s>>>(Wn, 1, 1, N, E, rk2, sys->nuc_pos, p.env_sigma, Qk, 1);
        gemm<T>(s, Qk, NE, p.env_pi + Dn * NE, NE, true, Fk2, Dn, 0, Wn, nullptr, Wn, (int)Dn, NE);
        mark("swap_msg", 1);
        swap_msg_kernel<T, T><<<(unsigned)capU, d, msm, s>>>(Wn, n, n_up, d, a2, b, Umax, r, c, p, Ul, Uc, Urow, H0,
                                                             PQ, H1, X1, H1n);
        check("swap msg");
        rows_and_ratio(a2, b, Fk2);
        mark("swap_accum", 1);
        swap_accum_kernel<T><<<Wn, 32, 0, s>>>(Wn, n, n_up, D, a2, b, Umax, dm.flags, r, rk, rk2, Ul, Uc, Urow, jp,
                                               F1, F2, F1n, F2n, G1, G2, G1n, G2n, ldabs, lsign, lrat, srat,
                                               mc.swap_ratios);
        check("swap");
      }
      swap_sum_kernel<<<(Wn + 255) / 256, 256, 0, s>>>(Wn, n_up, mc.swap_ratios, mc.swap_r);
      if (cudaMemcpyAsync(a.host_status, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return FIRE_ERR_CUDA;
      if (cudaStreamSynchronize(s) != cudaSuccess) return FIRE_ERR_CUDA;
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) { set_last_error("swap", cudaGetErrorString(e)); return FIRE_ERR_CUDA; }
      if (a.n_launches) *a.n_launches = launches;
      return failed ? FIRE_ERR_CUDA : FIRE_OK;
    }
    if (mc.ecp) {
      // non-local pseudopotential: n_el x N_quad virtual single-electron
      // moves from the state just built; no move is accepted
      if (cudaMemsetAsync(mc.v_nl, 0, sizeof(double) * (size_t)Wn, s) != cudaSuccess) return FIRE_ERR_CUDA;
      for (int k = 0; k < n; ++k)
        for (int q = 0; q < mc.ecp_qmax; ++q) {
          mark("ecp_propose", 2);
          ecp_propose_kernel<<<Wn, 32, 0, s>>>(n, n_up, k, q, r, sys->nuc_pos, N, mc.ecp, mc.seed, c * c, Umax, rk,
                                               lq, Ul, Uc, Ucu, st);
          evaluate_move(k);
          mark("ecp_accum", 1);
          ecp_accum_kernel<T><<<Wn, 32, 0, s>>>(Wn, n, n_up, D, k, Umax, dm.flags, r, rk, lq, Ul, Uc, Urow, jp, F1, F2,
                                                F1n, F2n, G1, G2, G1n, G2n, ldabs, lsign, lrat, srat, mc.v_nl);
          check("ecp");
        }
      if (cudaMemcpyAsync(a.host_status, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return FIRE_ERR_CUDA;
      if (cudaStreamSynchronize(s) != cudaSuccess) return FIRE_ERR_CUDA;
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) { set_last_error("ecp", cudaGetErrorString(e)); return FIRE_ERR_CUDA; }
      if (a.n_launches) *a.n_launches = launches;
      return failed ? FIRE_ERR_CUDA : FIRE_OK;
    }
    int64_t moves = 0;
    const int per_sweep = n + mc.n_global;
    const int64_t total_moves = (int64_t)mc.n_sweeps * per_sweep;
    for (int sweep = 0; sweep < mc.n_sweeps; ++sweep) {
      for (int j = 0; j < per_sweep; ++j) {
        const uint64_t move = mc.counter + (uint64_t)sweep * per_sweep + j;
        // local moves k = 0 .. n-1, then global jumps of an electron drawn
        // (for all walkers alike) from word 0 of Philox counter
        // (move, 2^32 - 1, 2)
        const bool global = j >= n;
        int k = j;
        if (global) {
          const Philox4 c = philox4x32_10((uint32_t)move, (uint32_t)(move >> 32), 0xffffffffu, 2u,
                                          (uint32_t)mc.seed, (uint32_t)(mc.seed >> 32));
          k = (int)floor(u01(c.v[0]) * n);
          if (k > n - 1) k = n - 1;
        }
        mark("mc_propose", 2);
        mcmc_propose_kernel<<<Wn, 32, 0, s>>>(n, n_up, k, r, mc.sigma, mc.seed, move, 0, c * c, Umax, rk, uacc, Ul,
                                              Uc, Ucu, st, global ? 1 : 0, sys->nuc_pos, sys->nuc_charge, N,
                                              mc.sigma_global, lq);
        evaluate_move(k);
        mark("mc_accept", 2);
        int* rcnt = at<int>(pl.mc_xcnt);
        int32_t* rlist = at<int32_t>(pl.mc_xlist);
        cudaMemsetAsync(rcnt, 0, sizeof(int), s);
        mcmc_accept_kernel<T><<<Wn, 32, 0, s>>>(Wn, n, n_up, D, k, Umax, dm.flags, r, rk, uacc, Ul, Uc, Urow, jp, F1,
                                                F2, F1n, F2n, G1, G2, G1n, G2n, ldabs, lsign, lrat, srat, lp, acc,
                                                mc.acc_count, &ms->n_accepted, lref, flag, xflag, lq, rcnt, rlist,
                                                pl.xcap, &ms->n_repair);
        mcmc_rows_kernel<T><<<(unsigned)capU, 128, 0, s>>>(
            Wn, n, n_up, d, (int)Dn, RD, k, Umax, pl.ld_big, RD1, (dm.flags & FIRE_J_MLP) ? 1 : 0,
            (dm.flags & FIRE_J_ATT) ? 1 : 0, acc, Ul, Uc, Urow, F1n, F2n, F1, F2, SUn, SU, h0k, H0, PQk, PQ, Fk,
            Fenv, Vn, V, G1n, G2n, G1, G2, H1n, H1);
        mark("mc_woodbury", 1);
        const int64_t npair = (int64_t)Wn * D;
        mcmc_woodbury_kernel<T><<<(unsigned)(npair < kWoodburySlots ? npair : kWoodburySlots), 256, 0, s>>>(
            Wn, n, D, Umax, acc, flag, Ul, Uc, Dl, Mlu, Mpiv, AT, PhiS, Tu, Bw);
        mcmc_repair_kernel<T, LT><<<(unsigned)(npair < kWoodburySlots ? npair : kWoodburySlots), 256,
                                    inverse_panel_smem(n, sizeof(LT)), s>>>(
            Wn, n, D, acc, flag, PhiS, AT, ldabs, lsign, lref, at<LT>(pl.mc_rep), at<int32_t>(pl.mc_rpiv));
        {
          // the listed refactorisations, batched over all SMs: float64 LU of
          // the updated Phi, then the inverse from the factors
          LT* xb = at<LT>(pl.mc_xbatch);
          int32_t* xpiv = at<int32_t>(pl.mc_xpiv);
          double* xlab = at<double>(pl.mc_xlab);
          double* xsg = at<double>(pl.mc_xsg);
          mcmc_repair_build_kernel<T, LT><<<pl.xcap, 256, 0, s>>>(n, rcnt, rlist, PhiS, xb);
          lu_kernel<LT, 16><<<pl.xcap, 256, lu_smem_bytes(n, sizeof(LT)), s>>>(n, xb, xpiv, xlab, xsg, rcnt);
          mcmc_repair_scatter_kernel<<<(pl.xcap + 255) / 256, 256, 0, s>>>(rcnt, pl.xcap, rlist, xlab, xsg, ldabs,
                                                                          lsign, lref);
          mcmc_repair_inverse_kernel<LT, T><<<pl.xcap, 256, inverse_panel_smem(n, sizeof(LT)), s>>>(
              n, rcnt, pl.xcap, rlist, xb, xpiv, xsg, AT);
        }
        launches += 5;
        check("mc update");
        ++moves;
        if (mc.refresh_every > 0 && moves % mc.refresh_every == 0 && moves < total_moves) {
          mark("mc_refresh", 0);
          rc = refresh(true);
          if (rc != FIRE_OK) return rc;
        }
      }
    }
    mark("mc_refresh", 0);
    rc = refresh(moves > 0);
    if (rc != FIRE_OK) return rc;
    McmcStat hm;
    if (cudaMemcpyAsync(&hm, ms, sizeof(McmcStat), cudaMemcpyDeviceToHost, s) != cudaSuccess) return FIRE_ERR_CUDA;
    if (cudaMemcpyAsync(a.host_status, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return FIRE_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FIRE_ERR_CUDA;
    {
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) { set_last_error("mcmc", cudaGetErrorString(e)); return FIRE_ERR_CUDA; }
    }
    mc.n_accepted = (int64_t)hm.n_accepted;
    double dr_ = 0.0;
    memcpy(&dr_, &hm.drift_bits, sizeof(double));
    mc.max_drift = dr_;
    mc.counter += (uint64_t)total_moves;
    if (a.n_launches) *a.n_launches = launches;
    return failed ? FIRE_ERR_CUDA : FIRE_OK;
  }
};

// Raises the dynamic shared-memory limit of every kernel that needs more than
// 48 KB.  Called once per precision form and device before the first launch.
template <typename T, typename LT>
inline int set_smem_limits() {
  int dev = 0, maxopt = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FIRE_ERR_CUDA;
  cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  int rc = FIRE_OK;
  auto raise = [&](const void* fn) {
    cudaFuncAttributes at;
    if (cudaFuncGetAttributes(&at, fn) != cudaSuccess) { rc = FIRE_ERR_CUDA; return; }
    const int dyn = maxopt - (int)at.sharedSizeBytes;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess) rc = FIRE_ERR_CUDA;
    // the largest shared-memory carveout: an SM running these kernels keeps
    // room for a CTA of the tensor-core product (the L1 / shared split only
    // changes once an SM has drained)
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  };
  raise((const void*)contract_kernel<T, 1>);
  raise((const void*)contract_kernel<T, 2>);
  raise((const void*)contract_kernel<T, 3>);
  raise((const void*)contract_kernel<T, 5>);
  raise((const void*)contract_kernel<T, 9>);
  raise((const void*)contract2_kernel<64, 1>);
  raise((const void*)contract2_kernel<128, 1>);
  raise((const void*)contract2_kernel<320, 1>);
  raise((const void*)contract3_kernel<64>);
  raise((const void*)contract3_kernel<96>);
  raise((const void*)contract3_kernel<128>);
  raise((const void*)contract3_kernel<192>);
  raise((const void*)contract3_kernel<320>);
  raise((const void*)lu_kernel<LT, 16>);
  raise((const void*)lu_kernel<LT, 32>);
  raise((const void*)att_pool_kernel<T>);
  raise((const void*)gj_inverse_kernel<float, T>);
  raise((const void*)gj_inverse_pre_kernel<float, T>);
  raise((const void*)mcmc_att_kernel<T>);
  raise((const void*)inverse_panel_kernel<LT, LT, T>);
  raise((const void*)inverse_panel_kernel<LT, T, T>);
  raise((const void*)mcmc_repair_kernel<T, LT>);
  raise((const void*)mcmc_repair_inverse_kernel<LT, T>);
  cudaError_t e = cudaGetLastError();
  if (rc != FIRE_OK || e != cudaSuccess) set_last_error("smem limits", cudaGetErrorString(e));
  return rc;
}

}  // namespace fire

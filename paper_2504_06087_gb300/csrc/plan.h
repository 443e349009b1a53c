// Workspace plan shared by the entry points and the per-precision runners.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "../../include/fire.h"

namespace fire {

struct Dims {
  int n, n_up, N, d, L, D, E, G, H, J, R, dr, K;
  uint32_t flags;
  int prec;
  int deriv;
  int op;
};

// Byte offsets of every buffer inside the workspace (for one chunk of Wc
// walkers; buffers are reused chunk after chunk).
struct Plan {
  Dims dm;
  int64_t W, Wc, nchunks;
  int64_t rows_cap;        // forward-Laplacian rows of one chunk (upper bound)
  int64_t rows_per_el;     // upper bound of rows per electron block
  size_t tsz, lsz;         // element sizes of the compute and LU types
  size_t status, idx, cnt, rev, blk_rows, blk_off, ranges;
  size_t clist;            // contraction bucket counters and lists (local energy)
  size_t S5, Y5, Z5, P5, H0, PQ;
  size_t X, big, F1, F2;   // big holds Z | SU, and O (aliased) in the det phase
  size_t Y, Xb, Yb;        // Jastrow hidden rows; bf16 copies of X and Y (BF16 form)
  int64_t wb_mlp, wb_jm1, wb_jm2, wb_att, wb_env, wb_glu, wb_gluo, wb_msg, wb_orbv, wb_ja1, wb_ja2;   // element offsets inside wbf16
  size_t Qf, Qfb, Fenv, Hv, Ov;   // Qfb: bf16 components of Qf (BF16 form)
  size_t Y5b, P5b, H0b, Hvb;      // bf16 components of Y5, P5, H0, Hv (BF16 form)
  size_t LU, piv, ldabs, lsign, Ainv, gdet, ldet, Phif;
  size_t jval, jsign, jgrad, jlap, aval, asign, agrad, alap, cval, cgrad, clap, vpot;
  size_t V, VZ, VY, G1, G2;
  size_t AP;               // attention-pool shifts and per-electron records (local energy)
  size_t Vb, VYb;          // bf16 components of V and of the register-MLP hidden rows (BF16 form)
  size_t wbf16;            // packed BF16 weights (tensor-core form)
  size_t poff_dev;         // device copy of the parameter offsets (gradient call)
  size_t gradws;           // gradient scratch region (GradBufs)
  // Metropolis moves (op FIRE_OP_MCMC): the cached state lives in the value
  // buffers above (H0, PQ, Fenv, F1, F2, SU in big, V, G1, G2, ldabs, lsign)
  // plus PhiS and Ainv; the rest is per-move scratch.
  int Umax;                // largest update set |U|
  size_t PhiS, mc_rk, mc_u, mc_Ul, mc_Uc, mc_Ucu, mc_Urow, mc_rng, mc_h0k, mc_PQk, mc_Qk, mc_Fk;
  size_t mc_X, mc_Z, mc_Y, mc_F1n, mc_F2n, mc_SUn, mc_On, mc_Vn, mc_VZ, mc_VY, mc_G1n, mc_G2n;
  size_t mc_Dl, mc_Mt, mc_Mlu, mc_piv, mc_lrat, mc_srat, mc_acc, mc_Tu, mc_Bw, mc_lp, mc_lpf, mc_sgf, mc_stat;
  size_t mc_H1, mc_H1n, mc_wdrift, mc_lref, mc_flag, mc_xflag, mc_rep, mc_rpiv, mc_kap, mc_lq, mc_ecp;
  size_t mc_xcnt, mc_xlist, mc_xbatch, mc_xpiv, mc_xlab, mc_xsg;   // batched exact ratios
  int xcap;
  size_t mc_rk2, mc_Fk2;    // the second electron of a swap
  int64_t nparams;
  size_t total;
  // column layout of `big`
  int64_t ld_big, zcol, ycol, sucol;
  // named buffers (diagnostics)
  struct Ent { const char* name; size_t off, bytes; } ent[160];
  int nent;
};

// Determinants whose orbital rows share one tensor-core product (BF16 form).
constexpr int kOrbGroup = 4;

// CTAs (and scratch slots) of the Woodbury update: a persistent grid over
// the (walker, determinant) pairs, 4 per SM.
constexpr int kWoodburySlots = 152 * 4;

// Device counters of a Metropolis call.
struct McmcStat {
  unsigned long long n_accepted;
  unsigned long long drift_bits;   // bits of the largest |log|Psi| drift| (a non-negative double)
  unsigned long long n_exact;      // determinant ratios from a float64 LU (diagnostic)
  unsigned long long n_repair;     // determinants refactorised after an accepted move (diagnostic)
};

int make_plan(const fire_system_t* sys, const fire_arch_t* arch, int64_t W, int prec, int k_cap,
              int op, Plan* out);

}  // namespace fire

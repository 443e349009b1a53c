// C ABI entry points of libfire: argument checks, the parameter layout, the
// workspace plan and the dispatch to the per-precision pipelines.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <mutex>

#include "grad_bufs.h"
#include "nbr.cuh"
#include "pipeline.cuh"
#include "plan.h"

namespace fire {

struct PDesc {
  const char* name;
  int ndim;
  int64_t shape[5];
};

// Parameter arrays of the ansatz, in theta order (Methods, "Wave function
// ansatz"; Supplementary "Hyperparameters").
static void param_table(const fire_system_t* sys, const fire_arch_t* ar, PDesc t[P_COUNT]) {
  const int64_t n = sys->n_el, N = sys->n_nuc, d = ar->width, L = ar->n_layers, D = ar->n_det,
                E = ar->n_env, G = ar->n_gauss, H = ar->edge_hidden,
                J = ar->jastrow_width > 0 ? ar->jastrow_width : ar->width, R = ar->n_reg,
                dr = ar->d_reg;
  int k = 0;
  auto add = [&](const char* nm, std::initializer_list<int64_t> sh) {
    t[k].name = nm;
    t[k].ndim = (int)sh.size();
    int q = 0;
    for (int64_t v : sh) t[k].shape[q++] = v;
    for (; q < 5; ++q) t[k].shape[q] = 1;
    ++k;
  };
  add("en_w1", {N, 4, H}); add("en_b1", {N, H}); add("en_w2", {H, d}); add("en_wenv", {G, d});
  add("en_sigma", {G}); add("nuc_emb", {N, d}); add("en_wfeat", {4, d});
  add("ln_gamma", {d}); add("ln_beta", {d});
  add("glu_wg", {d, d}); add("glu_wv", {d, d}); add("glu_wo", {d, d});
  add("ee_w1", {4, H}); add("ee_b1", {H}); add("ee_w2", {H, d}); add("ee_wenv", {G, d});
  add("ee_sigma", {G}); add("msg_w", {2, 2 * d + 4, d}); add("msg_b", {2, d});
  add("mlp_w", {L, d, d}); add("mlp_b", {L, d});
  add("orb_w", {2, D, d, n}); add("env_pi", {2, D, n, N, E}); add("env_sigma", {N, E});
  add("cusp", {4});
  const char* mlp_names[4][6] = {{"jm1_w1", "jm1_b1", "jm1_w2", "jm1_b2", "jm1_w3", "jm1_b3"},
                                 {"jm2_w1", "jm2_b1", "jm2_w2", "jm2_b2", "jm2_w3", "jm2_b3"},
                                 {"ja1_w1", "ja1_b1", "ja1_w2", "ja1_b2", "ja1_w3", "ja1_b3"},
                                 {"ja2_w1", "ja2_b1", "ja2_w2", "ja2_b2", "ja2_w3", "ja2_b3"}};
  for (int q = 0; q < 4; ++q) {
    const int64_t din = q < 2 ? d : R * dr;
    add(mlp_names[q][0], {din, J}); add(mlp_names[q][1], {J});
    add(mlp_names[q][2], {J, J}); add(mlp_names[q][3], {J});
    add(mlp_names[q][4], {J}); add(mlp_names[q][5], {1});
    if (q == 1) { add("att_q", {R, d}); add("att_wv", {R, d, dr}); }
  }
}

static int64_t numel(const PDesc& p) {
  int64_t v = 1;
  for (int q = 0; q < p.ndim; ++q) v *= p.shape[q];
  return v;
}

static int check_system(const fire_system_t* sys, const fire_arch_t* ar) {
  if (!sys || !ar) return FIRE_ERR_INVALID_ARG;
  if (sys->n_el < 1 || sys->n_up < 0 || sys->n_up > sys->n_el || sys->n_nuc < 1) return FIRE_ERR_INVALID_ARG;
  if (sys->n_nuc > kMaxNuc) return FIRE_ERR_UNSUPPORTED;   // nucleus list of the batched e-n filter
  if (!(sys->cutoff >= 0.0) || !(sys->cutoff_nuc > 0.0)) return FIRE_ERR_INVALID_ARG;
  if (ar->width < 32 || ar->width > 1024 || ar->width % 32) return FIRE_ERR_INVALID_ARG;
  if (ar->n_layers < 0 || ar->n_det < 1 || ar->n_det > 64 || ar->n_env < 1) return FIRE_ERR_INVALID_ARG;
  if (ar->n_gauss != kGauss || ar->edge_hidden != kEdgeHidden) return FIRE_ERR_UNSUPPORTED;
  if (ar->n_reg < 1 || ar->d_reg < 1 || ar->n_reg * ar->d_reg > 1024) return FIRE_ERR_INVALID_ARG;
  if (ar->jastrow_width < 0) return FIRE_ERR_INVALID_ARG;
  return FIRE_OK;
}

static size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

static size_t layout(Plan& pl, int64_t Wc) {
  const Dims& dm = pl.dm;
  const int64_t n = dm.n, d = dm.d, D = dm.D, R5 = dm.deriv ? 5 : 1, K = dm.K, J = dm.J;
  const int64_t NE = (int64_t)dm.N * dm.E, RD = (int64_t)dm.R * dm.dr;
  const size_t ts = pl.tsz, ls = pl.lsz;
  const int64_t nb = Wc * n;
  const int64_t cap = nb * pl.rows_per_el;
  const int64_t vstride = dm.deriv ? 2 + 3 * n : 1;
  size_t o = 0;
  pl.nent = 0;
  const char* nm = "";
  auto take = [&](size_t bytes) {
    size_t r = o;
    o = align_up(o + bytes);
    if (pl.nent < 160) pl.ent[pl.nent++] = Plan::Ent{nm, r, bytes};
    return r;
  };
#define TAKE(field, bytes) (nm = #field, pl.field = take(bytes))
  TAKE(status, sizeof(DevStatus));
  TAKE(idx, nb * K * 4);
  TAKE(rev, nb * K * 4);
  TAKE(cnt, nb * 2 * 4);
  TAKE(blk_rows, nb * 8);
  TAKE(blk_off, (nb + 1) * 8);
  TAKE(ranges, 8 * 8);
  if (dm.deriv) TAKE(clist, (16 + kC3Buckets * nb) * 4); else pl.clist = 0;
  TAKE(S5, nb * R5 * d * ts);
  TAKE(Y5, nb * R5 * d * ts);
  TAKE(Z5, nb * R5 * 2 * d * ts);
  TAKE(P5, nb * R5 * d * ts);
  TAKE(H0, nb * R5 * d * ts);
  TAKE(PQ, nb * R5 * 4 * d * ts);
  TAKE(X, cap * d * ts);
  const int64_t zw = d > J ? d : J;
  pl.zcol = 0;
  pl.ycol = 0;
  pl.sucol = zw;
  int64_t ldb = zw + dm.R + RD;
  if (ldb < n) ldb = n;
  // BF16 form: the orbital rows of kOrbGroup determinants share one product
  if (dm.prec == FIRE_PREC_BF16_FP64 && dm.deriv) {
    const int64_t og = D < kOrbGroup ? D : kOrbGroup;
    if (ldb < og * n) ldb = og * n;
  }
  pl.ld_big = ldb;
  TAKE(big, cap * ldb * ts);
  TAKE(Y, cap * J * ts);
  const bool bf = dm.prec == FIRE_PREC_BF16_FP64;
  if (bf) { TAKE(Xb, kMaxSplit * cap * d * 2); TAKE(Yb, kMaxSplit * cap * J * 2); } else { pl.Xb = pl.Yb = 0; }
  TAKE(F1, cap * ts);
  TAKE(F2, cap * ts);
  TAKE(Qf, nb * R5 * NE * ts);
  const int64_t NEp = (NE + 63) / 64 * 64;
  if (dm.prec == FIRE_PREC_BF16_FP64) TAKE(Qfb, kMaxSplit * nb * R5 * NEp * 2); else pl.Qfb = 0;
  if (dm.prec == FIRE_PREC_BF16_FP64) {
    TAKE(Y5b, kMaxSplit * nb * R5 * d * 2);
    TAKE(P5b, kMaxSplit * nb * R5 * d * 2);
    TAKE(H0b, kMaxSplit * nb * R5 * d * 2);
    TAKE(Hvb, kMaxSplit * nb * d * 2);
  } else {
    pl.Y5b = pl.P5b = pl.H0b = pl.Hvb = 0;
  }
  TAKE(Fenv, nb * R5 * D * n * ts);
  // Hv / Ov also serve as value-row scratch of the tensor-core products
  const int64_t wmax = (d > J ? d : J) > dm.R + RD ? (d > J ? d : J) : dm.R + RD;
  TAKE(Hv, nb * (wmax > d ? wmax : d) * ts);
  TAKE(Ov, nb * (D * n > wmax ? D * n : wmax) * ts);
  TAKE(LU, Wc * D * n * n * ls);
  TAKE(piv, Wc * D * n * 4);
  TAKE(ldabs, Wc * D * 8);
  TAKE(lsign, Wc * D * 8);
  const bool mc = dm.op == FIRE_OP_MCMC;
  if (dm.deriv || mc) TAKE(Ainv, Wc * D * n * n * ts); else pl.Ainv = 0;
  if (dm.deriv && ts == 4) TAKE(Phif, Wc * D * n * n * 4); else pl.Phif = 0;
  TAKE(gdet, Wc * D * n * 3 * ts);
  TAKE(ldet, Wc * D * n * ts);
  TAKE(jval, Wc * ts); TAKE(jsign, Wc * ts); TAKE(jlap, Wc * ts); TAKE(jgrad, Wc * n * 3 * ts);
  TAKE(aval, Wc * ts); TAKE(asign, Wc * ts); TAKE(alap, Wc * ts); TAKE(agrad, Wc * n * 3 * ts);
  TAKE(cval, Wc * ts); TAKE(clap, Wc * ts); TAKE(cgrad, Wc * n * 3 * ts); TAKE(vpot, Wc * ts);
  TAKE(V, Wc * vstride * RD * ts);
  TAKE(VZ, Wc * vstride * J * ts);
  TAKE(VY, Wc * vstride * J * ts);
  TAKE(G1, Wc * vstride * ts);
  TAKE(G2, Wc * vstride * ts);
  if (dm.prec == FIRE_PREC_BF16_FP64 && dm.deriv) {
    TAKE(Vb, kMaxSplit * Wc * vstride * RD * 2);
    TAKE(VYb, kMaxSplit * Wc * vstride * J * 2);
  } else {
    pl.Vb = pl.VYb = 0;
  }
  if (dm.deriv && (dm.flags & FIRE_J_ATT)) TAKE(AP, (Wc * dm.R + nb * 12 * RD) * ts); else pl.AP = 0;
  if (bf) {
    // every weight block [N][K] is stored as kMaxSplit components [c][N][K]
    const int64_t S = kMaxSplit;
    int64_t e = 0;
    pl.wb_mlp = e; e += S * (int64_t)dm.L * d * d;
    pl.wb_jm1 = e; e += S * (d * J + J * J);
    pl.wb_jm2 = e; e += S * (d * J + J * J);
    pl.wb_att = e; e += S * (dm.R + RD) * d;
    pl.wb_env = e; e += S * 2 * D * n * NEp;
    pl.wb_glu = e; e += S * 2 * d * d;
    pl.wb_gluo = e; e += S * d * d;
    pl.wb_msg = e; e += S * 4 * d * d;
    pl.wb_orbv = e; e += S * 2 * D * n * d;
    pl.wb_ja1 = e; e += S * (RD * J + J * J);
    pl.wb_ja2 = e; e += S * (RD * J + J * J);
    TAKE(wbf16, e * 2);
  } else {
    pl.wbf16 = 0;
  }
  if (dm.op == FIRE_OP_GRAD_LOGPSI) {
    TAKE(poff_dev, P_COUNT * 8);
    const size_t gb = ts == 8 ? GradBufs<double>::carve(nullptr, nullptr, Wc, (int)n, (int)d, dm.L, (int)D, (int)J,
                                                         dm.R, (int)RD, (int)NE)
                              : GradBufs<float>::carve(nullptr, nullptr, Wc, (int)n, (int)d, dm.L, (int)D, (int)J,
                                                        dm.R, (int)RD, (int)NE);
    TAKE(gradws, gb);
  } else {
    pl.poff_dev = pl.gradws = 0;
  }
  if (mc) {
    // cached Phi and the counters that live through the whole call
    const int64_t Um = pl.Umax, capU = Wc * Um, Dn = D * n, RD1 = dm.R + RD;
    const int64_t zc = d > J ? d : J;
    TAKE(PhiS, Wc * D * n * n * ts);
    TAKE(mc_rng, 16 * 8);
    TAKE(mc_lp, Wc * 8);
    TAKE(mc_lpf, Wc * 8);
    TAKE(mc_sgf, Wc * 8);
    TAKE(mc_stat, sizeof(McmcStat));
    TAKE(mc_wdrift, Wc * 8);
    TAKE(mc_lref, Wc * D * 8);         // log|det| of each matrix at its last factorisation
    TAKE(mc_kap, Wc * D * 4);          // condition estimate of each matrix at the last refresh
    TAKE(mc_ecp, (int64_t)dm.N * (int64_t)sizeof(fire_ecp_t));   // pseudopotential table
    // the batched float64 LU of the exact ratios of ill-conditioned determinants
    pl.xcap = (int)(Wc * D < 16384 ? Wc * D : 16384);
    TAKE(mc_xcnt, 16);
    TAKE(mc_xlist, (int64_t)pl.xcap * 4);
    TAKE(mc_xbatch, (int64_t)pl.xcap * n * n * 8);
    TAKE(mc_xpiv, (int64_t)pl.xcap * n * 4);
    TAKE(mc_xlab, (int64_t)pl.xcap * 8);
    TAKE(mc_xsg, (int64_t)pl.xcap * 8);
    TAKE(mc_H1, nb * d * ts);          // cached h^1 rows (block order)
    // per-move scratch: dead during a refresh, so it shares the float64 LU
    // buffer (dead during the moves) when it fits there
    struct Sc { size_t* field; const char* name; size_t bytes; };
    const Sc sc[] = {
        {&pl.mc_rk, "mc_rk", (size_t)(Wc * 3 * 8)}, {&pl.mc_u, "mc_u", (size_t)(Wc * 8)},
        {&pl.mc_lq, "mc_lq", (size_t)(Wc * 8)}, {&pl.mc_rk2, "mc_rk2", (size_t)(Wc * 3 * 8)},
        {&pl.mc_Fk2, "mc_Fk2", (size_t)(Wc * Dn) * ts},
        {&pl.mc_Ul, "mc_Ul", (size_t)(capU * 4)}, {&pl.mc_Uc, "mc_Uc", (size_t)(Wc * 4)},
        {&pl.mc_Ucu, "mc_Ucu", (size_t)(Wc * 4)}, {&pl.mc_Urow, "mc_Urow", (size_t)(capU * 4)},
        {&pl.mc_h0k, "mc_h0k", (size_t)(Wc * d) * ts}, {&pl.mc_PQk, "mc_PQk", (size_t)(Wc * 4 * d) * ts},
        {&pl.mc_Qk, "mc_Qk", (size_t)(Wc * NE) * ts}, {&pl.mc_Fk, "mc_Fk", (size_t)(Wc * Dn) * ts},
        {&pl.mc_X, "mc_X", (size_t)(capU * d) * ts}, {&pl.mc_H1n, "mc_H1n", (size_t)(capU * d) * ts},
        {&pl.mc_Z, "mc_Z", (size_t)(capU * zc) * ts},
        {&pl.mc_Y, "mc_Y", (size_t)(capU * J) * ts}, {&pl.mc_F1n, "mc_F1n", (size_t)capU * ts},
        {&pl.mc_F2n, "mc_F2n", (size_t)capU * ts}, {&pl.mc_SUn, "mc_SUn", (size_t)(capU * RD1) * ts},
        {&pl.mc_On, "mc_On", (size_t)(capU * Dn) * ts}, {&pl.mc_Vn, "mc_Vn", (size_t)(Wc * RD) * ts},
        {&pl.mc_VZ, "mc_VZ", (size_t)(Wc * J) * ts}, {&pl.mc_VY, "mc_VY", (size_t)(Wc * J) * ts},
        {&pl.mc_G1n, "mc_G1n", (size_t)Wc * ts}, {&pl.mc_G2n, "mc_G2n", (size_t)Wc * ts},
        {&pl.mc_Dl, "mc_Dl", (size_t)(Wc * D * Um * n) * ts}, {&pl.mc_Mt, "mc_Mt", (size_t)(Wc * D * Um * Um) * ts},
        {&pl.mc_Mlu, "mc_Mlu", (size_t)(Wc * D * Um * Um * 8)}, {&pl.mc_piv, "mc_piv", (size_t)(Wc * D * Um * 4)},
        {&pl.mc_lrat, "mc_lrat", (size_t)(Wc * D * 8)}, {&pl.mc_srat, "mc_srat", (size_t)(Wc * D * 8)},
        {&pl.mc_acc, "mc_acc", (size_t)(Wc * 4)}, {&pl.mc_flag, "mc_flag", (size_t)(Wc * D * 4)},
        {&pl.mc_xflag, "mc_xflag", (size_t)(Wc * D * 4)},
        {&pl.mc_rep, "mc_rep", (size_t)kWoodburySlots * n * n * 8}, {&pl.mc_rpiv, "mc_rpiv", (size_t)kWoodburySlots * n * 4},
        {&pl.mc_Tu, "mc_Tu", (size_t)(kWoodburySlots * Um * n) * ts},
        {&pl.mc_Bw, "mc_Bw", (size_t)(kWoodburySlots * Um * n) * ts}};
    size_t need = 0;
    for (const Sc& e : sc) need = align_up(need + e.bytes);
    const size_t lu_bytes = (size_t)(Wc * D * n * n) * ls;
    size_t q = need <= lu_bytes ? pl.LU : o;
    for (const Sc& e : sc) {
      *e.field = q;
      if (pl.nent < 160) pl.ent[pl.nent++] = Plan::Ent{e.name, q, e.bytes};
      q = align_up(q + e.bytes);
    }
    if (q > o) o = q;
  }
#undef TAKE
  pl.total = o;
  return o;
}

static size_t budget_bytes() {
  const char* e = getenv("FIRE_WORKSPACE_BUDGET_MB");
  // default: 128 GiB of the 280 GB of HBM3e (C26H24 at 4096 walkers: 10
  // chunks; measured 1.7 % faster than 64 GiB, no gain beyond);
  // FIRE_WORKSPACE_BUDGET_MB overrides
  double mb = e ? atof(e) : 131072.0;
  if (!(mb > 0)) mb = 131072.0;
  return (size_t)(mb * 1024.0 * 1024.0);
}

int make_plan(const fire_system_t* sys, const fire_arch_t* ar, int64_t W, int prec, int k_cap, int op,
              Plan* pl) {
  int rc = check_system(sys, ar);
  if (rc) return rc;
  if (W < 1 || k_cap < 1 || k_cap > 1024) return FIRE_ERR_INVALID_ARG;
  if (prec < 0 || prec > 2) return FIRE_ERR_INVALID_ARG;
  // Metropolis moves of both reduced forms run in float32
  if (op == FIRE_OP_MCMC && prec == FIRE_PREC_BF16_FP64) prec = FIRE_PREC_FP32;
  memset(pl, 0, sizeof(Plan));
  Dims& dm = pl->dm;
  dm.n = sys->n_el; dm.n_up = sys->n_up; dm.N = sys->n_nuc; dm.d = ar->width; dm.L = ar->n_layers;
  dm.D = ar->n_det; dm.E = ar->n_env; dm.G = ar->n_gauss; dm.H = ar->edge_hidden;
  dm.J = ar->jastrow_width > 0 ? ar->jastrow_width : ar->width; dm.R = ar->n_reg; dm.dr = ar->d_reg;
  dm.K = k_cap; dm.flags = ar->flags; dm.prec = prec; dm.op = op;
  dm.deriv = (op == FIRE_OP_LOCAL_ENERGY) ? 1 : 0;
  const int keff = k_cap < dm.n - 1 ? k_cap : (dm.n - 1 > 0 ? dm.n - 1 : 0);
  pl->rows_per_el = dm.deriv ? 2 + 3 * (1 + keff) : 1;
  pl->tsz = prec == FIRE_PREC_FP64 ? 8 : 4;
  // the Metropolis refresh factorises in float64 in every form
  pl->lsz = (prec == FIRE_PREC_FP32 && op != FIRE_OP_MCMC) ? 4 : 8;
  pl->Umax = keff * 2 + 1 < dm.n ? keff * 2 + 1 : dm.n;
  pl->W = W;
  const size_t s1 = layout(*pl, 1), s2 = layout(*pl, 2);
  const size_t per = s2 > s1 ? s2 - s1 : 1;
  const size_t base = s1 > per ? s1 - per : 0;
  const size_t bud = budget_bytes();
  int64_t wc = bud > base ? (int64_t)((bud - base) / per) : 1;
  if (wc < 1) wc = 1;
  if (wc > W || op == FIRE_OP_MCMC) wc = W;   // the Metropolis state covers every walker
  // shared-memory limits of the determinant kernels
  const int n = dm.n, mcap = 1 + (k_cap < dm.n - 1 ? k_cap : dm.n - 1);
  const size_t ctsm = contract_smem_bytes(mcap, pl->tsz);
  // the float forms invert by Gauss-Jordan in shared memory (n <= 192), the
  // rest by column panels on the LU factors
  const size_t invsm = (pl->tsz == 4 && n <= 192) ? gj_smem_bytes(n) : inverse_panel_smem(n, pl->lsz);
  const size_t lim = 227 * 1024;
  if (lu_smem_bytes(n, pl->lsz) > lim) return FIRE_ERR_UNSUPPORTED;   // the LU panel and U12 block
  if (dm.deriv && (ctsm > lim || invsm > lim)) return FIRE_ERR_UNSUPPORTED;
  pl->Wc = wc;
  pl->nchunks = (W + wc - 1) / wc;
  layout(*pl, wc);
  return FIRE_OK;
}

static thread_local char g_last_error[256];

struct ProfRow { char name[24]; int64_t launches; double ms; };
static thread_local ProfRow g_prof[64];
static thread_local int g_nprof = 0;
static thread_local bool g_prof_on = false;

bool prof_enabled() { return g_prof_on; }

void prof_add(const char* name, int launches, float ms) {
  int k = 0;
  for (; k < g_nprof; ++k)
    if (strncmp(g_prof[k].name, name, sizeof(g_prof[k].name)) == 0) break;
  if (k == g_nprof) {
    if (g_nprof >= 64) return;
    memset(&g_prof[k], 0, sizeof(ProfRow));
    strncpy(g_prof[k].name, name, sizeof(g_prof[k].name) - 1);
    ++g_nprof;
  }
  g_prof[k].launches += launches;
  g_prof[k].ms += ms;
}

// Calls on this host thread that must create nothing (no stream, no event):
// the static-workspace entry point runs every kernel on the caller's stream.
static thread_local bool g_single_stream = false;
void set_single_stream(bool on) { g_single_stream = on; }
bool single_stream() { return g_single_stream; }

// One extra non-blocking stream per device for work that runs beside the
// caller's stream inside a call (created on first use, kept until exit).
cudaStream_t side_stream() {
  static std::mutex mu;
  static cudaStream_t streams[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!streams[dev]) {
    // FIRE_SIDE_PRIORITY=high (diagnostic): the greatest stream priority;
    // default: the same priority as an ordinary stream
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    const char* e = getenv("FIRE_SIDE_PRIORITY");
    const int prio = (e && strcmp(e, "high") == 0) ? greatest : least;
    if (cudaStreamCreateWithPriority(&streams[dev], cudaStreamNonBlocking, prio) != cudaSuccess)
      streams[dev] = nullptr;
  }
  return streams[dev];
}

void set_last_error(const char* stage, const char* msg) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s", stage, msg);
}

}  // namespace fire

using namespace fire;

extern "C" {

const char* fire_last_error(void) { return g_last_error; }

int fire_profile_enable(int on) {
  g_prof_on = on != 0;
  return FIRE_OK;
}

int fire_profile_reset(void) {
  g_nprof = 0;
  return FIRE_OK;
}

int fire_profile_report(fire_prof_entry_t* out, int32_t* n) {
  if (!n) return FIRE_ERR_INVALID_ARG;
  *n = g_nprof;
  if (!out) return FIRE_OK;
  for (int k = 0; k < g_nprof; ++k) {
    memset(&out[k], 0, sizeof(fire_prof_entry_t));
    strncpy(out[k].name, g_prof[k].name, sizeof(out[k].name) - 1);
    out[k].launches = g_prof[k].launches;
    out[k].ms_total = g_prof[k].ms;
  }
  return FIRE_OK;
}

const char* fire_version(void) { return "libfire 0.1 (sm_103a)"; }

const char* fire_status_string(int s) {
  switch (s) {
    case FIRE_OK: return "ok";
    case FIRE_ERR_INVALID_ARG: return "invalid argument";
    case FIRE_ERR_CAPACITY: return "neighbour list capacity k_cap exceeded";
    case FIRE_ERR_NONFINITE: return "non-finite result off a node";
    case FIRE_ERR_SINGULAR_REFRESH: return "singular matrix in the inverse refresh";
    case FIRE_ERR_TIMEOUT: return "bounded device wait timed out";
    case FIRE_ERR_CUDA: return "CUDA runtime error";
    case FIRE_ERR_UNSUPPORTED: return "unsupported configuration";
    case FIRE_ERR_WORKSPACE: return "workspace missing or too small";
    default: return "unknown status";
  }
}

int64_t fire_param_count(const fire_system_t* sys, const fire_arch_t* arch) {
  if (check_system(sys, arch) != FIRE_OK) return -1;
  PDesc t[P_COUNT];
  param_table(sys, arch, t);
  int64_t s = 0;
  for (int k = 0; k < P_COUNT; ++k) s += numel(t[k]);
  return s;
}

int fire_param_layout(const fire_system_t* sys, const fire_arch_t* arch, fire_param_entry_t* out,
                      int32_t* n) {
  if (!n) return FIRE_ERR_INVALID_ARG;
  int rc = check_system(sys, arch);
  if (rc) return rc;
  PDesc t[P_COUNT];
  param_table(sys, arch, t);
  *n = P_COUNT;
  if (!out) return FIRE_OK;
  int64_t off = 0;
  for (int k = 0; k < P_COUNT; ++k) {
    memset(&out[k], 0, sizeof(fire_param_entry_t));
    strncpy(out[k].name, t[k].name, sizeof(out[k].name) - 1);
    out[k].offset = off;
    out[k].ndim = t[k].ndim;
    for (int q = 0; q < 5; ++q) out[k].shape[q] = t[k].shape[q];
    off += numel(t[k]);
  }
  return FIRE_OK;
}

size_t fire_workspace_size(const fire_system_t* sys, const fire_arch_t* arch, int64_t n_walkers,
                           int32_t precision, int32_t k_cap, int32_t op) {
  if (op == FIRE_OP_NEIGHBORS) {
    if (!sys || n_walkers < 1) return 0;
    return 256;
  }
  Plan pl;
  if (make_plan(sys, arch, n_walkers, precision, k_cap, op, &pl) != FIRE_OK) return 0;
  return pl.total;
}

int fire_workspace_layout(const fire_system_t* sys, const fire_arch_t* arch, int64_t n_walkers,
                          int32_t precision, int32_t k_cap, int32_t op, fire_ws_entry_t* out, int32_t* n,
                          int64_t* chunk_walkers) {
  if (!n) return FIRE_ERR_INVALID_ARG;
  Plan pl;
  int rc = make_plan(sys, arch, n_walkers, precision, k_cap, op, &pl);
  if (rc) return rc;
  *n = pl.nent;
  if (chunk_walkers) *chunk_walkers = pl.Wc;
  if (!out) return FIRE_OK;
  for (int k = 0; k < pl.nent; ++k) {
    memset(&out[k], 0, sizeof(fire_ws_entry_t));
    strncpy(out[k].name, pl.ent[k].name, sizeof(out[k].name) - 1);
    out[k].offset = (int64_t)pl.ent[k].off;
    out[k].bytes = (int64_t)pl.ent[k].bytes;
  }
  return FIRE_OK;
}

int fire_neighbors(const fire_system_t* sys, int64_t W, const double* r, int32_t k_cap, int32_t* nbr_idx,
                   int32_t* nbr_cnt, int32_t* k_required, void* ws, size_t ws_bytes, void* stream) {
  if (!sys || W < 1 || !r || k_cap < 1 || !nbr_idx || !nbr_cnt) return FIRE_ERR_INVALID_ARG;
  if (sys->n_el < 1 || sys->n_up < 0 || sys->n_up > sys->n_el || !(sys->cutoff >= 0)) return FIRE_ERR_INVALID_ARG;
  if (!ws || ws_bytes < 256) return FIRE_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  DevStatus* st = reinterpret_cast<DevStatus*>(ws);
  cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
  const int n = sys->n_el;
  // chunks of walkers keep the block-row scratch inside the launch
  const int64_t chunk = 65535;
  for (int64_t w0 = 0; w0 < W; w0 += chunk) {
    const int wc = (int)((W - w0) < chunk ? (W - w0) : chunk);
    nbr_build_kernel<<<wc, 256, (size_t)n * 3 * sizeof(double), s>>>(
        wc, n, sys->n_up, r + w0 * n * 3, sys->cutoff * sys->cutoff, k_cap, nbr_idx + w0 * n * k_cap,
        nbr_cnt + w0 * n * 2, nullptr, st, 0);
  }
  DevStatus hs;
  if (cudaGetLastError() != cudaSuccess) return FIRE_ERR_CUDA;
  if (cudaMemcpyAsync(&hs, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess) return FIRE_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return FIRE_ERR_CUDA;
  if (k_required) *k_required = hs.k_required;
  return hs.overflow ? FIRE_ERR_CAPACITY : FIRE_OK;
}

static int run_call(const fire_system_t* sys, const fire_arch_t* arch, const fire_params_t* params,
                    int64_t W, const double* r, int32_t k_cap, int32_t prec, int op, double* e_loc,
                    double* logabs, double* sign, double* e_kin, double* e_pot, fire_info_t* info,
                    void* ws, size_t ws_bytes, void* stream, void* grad = nullptr) {
  if (!params || !params->theta || !r || !logabs || !sign) return FIRE_ERR_INVALID_ARG;
  if (op == FIRE_OP_LOCAL_ENERGY && !e_loc) return FIRE_ERR_INVALID_ARG;
  if (op == FIRE_OP_GRAD_LOGPSI && !grad) return FIRE_ERR_INVALID_ARG;
  Plan pl;
  int rc = make_plan(sys, arch, W, prec, k_cap, op, &pl);
  if (rc) return rc;
  if (!sys->nuc_pos || !sys->nuc_charge) return FIRE_ERR_INVALID_ARG;
  if (params->n_params != fire_param_count(sys, arch)) return FIRE_ERR_INVALID_ARG;
  const int want_dtype = prec == FIRE_PREC_FP64 ? 0 : 1;
  if (params->dtype != want_dtype) return FIRE_ERR_INVALID_ARG;
  if (!ws || ws_bytes < pl.total) return FIRE_ERR_WORKSPACE;
  PDesc t[P_COUNT];
  param_table(sys, arch, t);
  int64_t poff[P_COUNT];
  int64_t off = 0;
  for (int k = 0; k < P_COUNT; ++k) { poff[k] = off; off += numel(t[k]); }
  DevStatus hs;
  memset(&hs, 0, sizeof(hs));
  int64_t nl = 0;
  pl.nparams = off;
  CallArgs a{sys, arch, params->theta, poff, W, r, e_loc, logabs, sign, e_kin, e_pot, ws,
             (cudaStream_t)stream, &hs, &nl, grad, nullptr};
  if (prec == FIRE_PREC_FP64) rc = run_fp64(pl, a);
  else if (prec == FIRE_PREC_FP32) rc = run_fp32(pl, a);
  else rc = run_bf16(pl, a);
  if (info) {
    info->k_required = hs.k_required;
    info->n_nodes = hs.n_nodes;
    info->n_nonfinite = hs.n_nonfinite;
    info->n_chunks = (int32_t)pl.nchunks;
    info->rows_total = hs.rows_total;
    info->n_launches = nl;
    info->mean_neighbors = (double)hs.nbr_total / ((double)W * sys->n_el);
  }
  if (rc) return rc;
  if (hs.tc_err) return FIRE_ERR_TIMEOUT;
  if (hs.overflow) return FIRE_ERR_CAPACITY;
  if (hs.n_nonfinite) return FIRE_ERR_NONFINITE;
  return FIRE_OK;
}

int fire_logpsi(const fire_system_t* sys, const fire_arch_t* arch, const fire_params_t* params, int64_t W,
                const double* r, int32_t k_cap, int32_t precision, double* logabs, double* sign,
                fire_info_t* info, void* ws, size_t ws_bytes, void* stream) {
  return run_call(sys, arch, params, W, r, k_cap, precision, FIRE_OP_LOGPSI, nullptr, logabs, sign, nullptr,
                  nullptr, info, ws, ws_bytes, stream);
}

int fire_grad_logpsi(const fire_system_t* sys, const fire_arch_t* arch, const fire_params_t* params,
                     int64_t W, const double* r, int32_t k_cap, int32_t precision, void* grad, double* logabs,
                     double* sign, fire_info_t* info, void* ws, size_t ws_bytes, void* stream) {
  return run_call(sys, arch, params, W, r, k_cap, precision, FIRE_OP_GRAD_LOGPSI, nullptr, logabs, sign, nullptr,
                  nullptr, info, ws, ws_bytes, stream, grad);
}

int fire_local_energy(const fire_system_t* sys, const fire_arch_t* arch, const fire_params_t* params,
                      int64_t W, const double* r, int32_t k_cap, int32_t precision, double* e_loc,
                      double* logabs, double* sign, double* e_kin, double* e_pot, fire_info_t* info,
                      void* ws, size_t ws_bytes, void* stream) {
  return run_call(sys, arch, params, W, r, k_cap, precision, FIRE_OP_LOCAL_ENERGY, e_loc, logabs, sign, e_kin,
                  e_pot, info, ws, ws_bytes, stream);
}

// Default tolerance of the conditioning test of the exact-ratio path.
static constexpr double kKappaTolDefault = 1e-4;

int fire_mcmc_step(const fire_system_t* sys, const fire_arch_t* arch, const fire_params_t* params,
                   int64_t W, double* r, int32_t k_cap, int32_t precision, double sigma, int32_t n_sweeps,
                   int32_t refresh_every, int32_t n_global, double sigma_global, uint64_t seed, uint64_t* counter,
                   double* logabs, double* sign, int32_t* accepted, int64_t* n_accepted, double* max_drift,
                   fire_info_t* info, void* ws, size_t ws_bytes, void* stream) {
  if (!params || !params->theta || !r || !counter) return FIRE_ERR_INVALID_ARG;
  if (!(sigma > 0.0) || !(sigma < 1e300) || n_sweeps < 0 || refresh_every < 0) return FIRE_ERR_INVALID_ARG;
  if (n_global < 0 || (n_global > 0 && !(sigma_global > 0.0 && sigma_global < 1e300))) return FIRE_ERR_INVALID_ARG;
  if (precision < 0 || precision > 2) return FIRE_ERR_INVALID_ARG;
  // the moves run in float32 for both reduced forms
  const int prec = precision == FIRE_PREC_FP64 ? FIRE_PREC_FP64 : FIRE_PREC_FP32;
  Plan pl;
  int rc = make_plan(sys, arch, W, prec, k_cap, FIRE_OP_MCMC, &pl);
  if (rc) return rc;
  if (!sys->nuc_pos || !sys->nuc_charge) return FIRE_ERR_INVALID_ARG;
  if (params->n_params != fire_param_count(sys, arch)) return FIRE_ERR_INVALID_ARG;
  if (params->dtype != (prec == FIRE_PREC_FP64 ? 0 : 1)) return FIRE_ERR_INVALID_ARG;
  if (!ws || ws_bytes < pl.total) return FIRE_ERR_WORKSPACE;
  PDesc t[P_COUNT];
  param_table(sys, arch, t);
  int64_t poff[P_COUNT];
  int64_t off = 0;
  for (int k = 0; k < P_COUNT; ++k) { poff[k] = off; off += numel(t[k]); }
  pl.nparams = off;
  DevStatus hs;
  memset(&hs, 0, sizeof(hs));
  int64_t nl = 0;
  // conditioning test of the exact-ratio path: 1e-4 keeps the carried
  // log|Psi| of every walker within 1e-2 of the rebuilds over 32 moves
  // (FIRE_MCMC_KAPPA_TOL overrides it; negative: off)
  double ktol = kKappaTolDefault;
  if (const char* e = getenv("FIRE_MCMC_KAPPA_TOL")) ktol = atof(e);
  McmcCall mc{sigma, n_sweeps, refresh_every, seed, *counter, accepted, 0, 0.0, n_global, sigma_global, ktol,
              nullptr, 0, nullptr, -1, nullptr, nullptr};
  unsigned char* wsb = reinterpret_cast<unsigned char*>(ws);
  double* lpf = reinterpret_cast<double*>(wsb + pl.mc_lpf);
  double* sgf = reinterpret_cast<double*>(wsb + pl.mc_sgf);
  CallArgs a{sys, arch, params->theta, poff, W, r, nullptr, lpf, sgf, nullptr, nullptr, ws,
             (cudaStream_t)stream, &hs, &nl, nullptr, &mc};
  rc = prec == FIRE_PREC_FP64 ? run_fp64(pl, a) : run_bf16(pl, a);
  if (info) {
    info->k_required = hs.k_required;
    info->n_nodes = hs.n_nodes;
    info->n_nonfinite = hs.n_nonfinite;
    info->n_chunks = 1;
    info->rows_total = hs.rows_total;
    info->n_launches = nl;
    info->mean_neighbors = (double)hs.nbr_total / ((double)W * sys->n_el);
  }
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (logabs && cudaMemcpyAsync(logabs, lpf, sizeof(double) * (size_t)W, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return FIRE_ERR_CUDA;
  if (sign && cudaMemcpyAsync(sign, sgf, sizeof(double) * (size_t)W, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return FIRE_ERR_CUDA;
  *counter = mc.counter;
  if (n_accepted) *n_accepted = mc.n_accepted;
  if (max_drift) *max_drift = mc.max_drift;
  if (hs.overflow) return FIRE_ERR_CAPACITY;
  if (hs.n_nonfinite) return FIRE_ERR_NONFINITE;
  return FIRE_OK;
}


int fire_ecp_nonlocal(const fire_system_t* sys, const fire_arch_t* arch, const fire_params_t* params, int64_t W,
                      const double* r, int32_t k_cap, int32_t precision, const fire_ecp_t* ecp, uint64_t seed,
                      double* v_nl, fire_info_t* info, void* ws, size_t ws_bytes, void* stream) {
  if (!params || !params->theta || !r || !ecp || !v_nl || !sys) return FIRE_ERR_INVALID_ARG;
  if (precision < 0 || precision > 2) return FIRE_ERR_INVALID_ARG;
  int qmax = 0;
  for (int m = 0; m < sys->n_nuc; ++m) {
    const fire_ecp_t& e = ecp[m];
    if (e.n_quad != 0 && e.n_quad != 4 && e.n_quad != 6 && e.n_quad != 12) return FIRE_ERR_INVALID_ARG;
    if (e.n_channels < 0 || e.n_channels > 3 || !(e.r_cut >= 0.0) || !(e.r_cut < 1e300)) return FIRE_ERR_INVALID_ARG;
    for (int l = 0; l < e.n_channels; ++l) {
      if (e.n_terms[l] < 0 || e.n_terms[l] > 4) return FIRE_ERR_INVALID_ARG;
      for (int j = 0; j < e.n_terms[l]; ++j)
        if (!std::isfinite(e.coef[l][j]) || !std::isfinite(e.power[l][j]) || !(e.alpha[l][j] >= 0.0) ||
            !std::isfinite(e.alpha[l][j]))
          return FIRE_ERR_INVALID_ARG;
    }
    if (e.n_quad > qmax) qmax = e.n_quad;
  }
  const int prec = precision == FIRE_PREC_FP64 ? FIRE_PREC_FP64 : FIRE_PREC_FP32;
  Plan pl;
  int rc = make_plan(sys, arch, W, prec, k_cap, FIRE_OP_MCMC, &pl);
  if (rc) return rc;
  if (!sys->nuc_pos || !sys->nuc_charge) return FIRE_ERR_INVALID_ARG;
  if (params->n_params != fire_param_count(sys, arch)) return FIRE_ERR_INVALID_ARG;
  if (params->dtype != (prec == FIRE_PREC_FP64 ? 0 : 1)) return FIRE_ERR_INVALID_ARG;
  if (!ws || ws_bytes < pl.total) return FIRE_ERR_WORKSPACE;
  PDesc t[P_COUNT];
  param_table(sys, arch, t);
  int64_t poff[P_COUNT];
  int64_t off = 0;
  for (int k = 0; k < P_COUNT; ++k) { poff[k] = off; off += numel(t[k]); }
  pl.nparams = off;
  unsigned char* wsb = reinterpret_cast<unsigned char*>(ws);
  cudaStream_t s = (cudaStream_t)stream;
  fire_ecp_t* ecp_dev = reinterpret_cast<fire_ecp_t*>(wsb + pl.mc_ecp);
  if (cudaMemcpyAsync(ecp_dev, ecp, sizeof(fire_ecp_t) * (size_t)sys->n_nuc, cudaMemcpyHostToDevice, s) !=
      cudaSuccess)
    return FIRE_ERR_CUDA;
  DevStatus hs;
  memset(&hs, 0, sizeof(hs));
  int64_t nl = 0;
  double ktol = kKappaTolDefault;
  if (const char* e = getenv("FIRE_MCMC_KAPPA_TOL")) ktol = atof(e);
  McmcCall mc{1.0, 0, 0, seed, 0, nullptr, 0, 0.0, 0, 1.0, ktol, ecp_dev, qmax, v_nl, -1, nullptr, nullptr};
  double* lpf = reinterpret_cast<double*>(wsb + pl.mc_lpf);
  double* sgf = reinterpret_cast<double*>(wsb + pl.mc_sgf);
  CallArgs a{sys, arch, params->theta, poff, W, r, nullptr, lpf, sgf, nullptr, nullptr, ws, s, &hs, &nl, nullptr,
             &mc};
  rc = prec == FIRE_PREC_FP64 ? run_fp64(pl, a) : run_bf16(pl, a);
  if (info) {
    info->k_required = hs.k_required;
    info->n_nodes = hs.n_nodes;
    info->n_nonfinite = hs.n_nonfinite;
    info->n_chunks = 1;
    info->rows_total = hs.rows_total;
    info->n_launches = nl;
    info->mean_neighbors = (double)hs.nbr_total / ((double)W * sys->n_el);
  }
  if (rc) return rc;
  if (hs.overflow) return FIRE_ERR_CAPACITY;
  if (hs.n_nonfinite) return FIRE_ERR_NONFINITE;
  return FIRE_OK;
}


int fire_spin_ratios(const fire_system_t* sys, const fire_arch_t* arch, const fire_params_t* params, int64_t W,
                     const double* r, int32_t k_cap, int32_t precision, int32_t beta, double* ratios, double* r_beta,
                     fire_info_t* info, void* ws, size_t ws_bytes, void* stream) {
  if (!params || !params->theta || !r || !ratios || !r_beta || !sys) return FIRE_ERR_INVALID_ARG;
  if (precision < 0 || precision > 2) return FIRE_ERR_INVALID_ARG;
  if (beta < sys->n_up || beta >= sys->n_el) return FIRE_ERR_INVALID_ARG;
  const int prec = precision == FIRE_PREC_FP64 ? FIRE_PREC_FP64 : FIRE_PREC_FP32;
  Plan pl;
  int rc = make_plan(sys, arch, W, prec, k_cap, FIRE_OP_MCMC, &pl);
  if (rc) return rc;
  if (!sys->nuc_pos || !sys->nuc_charge) return FIRE_ERR_INVALID_ARG;
  if (params->n_params != fire_param_count(sys, arch)) return FIRE_ERR_INVALID_ARG;
  if (params->dtype != (prec == FIRE_PREC_FP64 ? 0 : 1)) return FIRE_ERR_INVALID_ARG;
  if (!ws || ws_bytes < pl.total) return FIRE_ERR_WORKSPACE;
  PDesc t[P_COUNT];
  param_table(sys, arch, t);
  int64_t poff[P_COUNT];
  int64_t off = 0;
  for (int k = 0; k < P_COUNT; ++k) { poff[k] = off; off += numel(t[k]); }
  pl.nparams = off;
  unsigned char* wsb = reinterpret_cast<unsigned char*>(ws);
  cudaStream_t s = (cudaStream_t)stream;
  DevStatus hs;
  memset(&hs, 0, sizeof(hs));
  int64_t nl = 0;
  double ktol = kKappaTolDefault;
  if (const char* e = getenv("FIRE_MCMC_KAPPA_TOL")) ktol = atof(e);
  McmcCall mc{1.0, 0, 0, 0, 0, nullptr, 0, 0.0, 0, 1.0, ktol, nullptr, 0, nullptr, beta, ratios, r_beta};
  double* lpf = reinterpret_cast<double*>(wsb + pl.mc_lpf);
  double* sgf = reinterpret_cast<double*>(wsb + pl.mc_sgf);
  CallArgs a{sys, arch, params->theta, poff, W, r, nullptr, lpf, sgf, nullptr, nullptr, ws, s, &hs, &nl, nullptr,
             &mc};
  rc = prec == FIRE_PREC_FP64 ? run_fp64(pl, a) : run_bf16(pl, a);
  if (info) {
    info->k_required = hs.k_required;
    info->n_nodes = hs.n_nodes;
    info->n_nonfinite = hs.n_nonfinite;
    info->n_chunks = 1;
    info->rows_total = hs.rows_total;
    info->n_launches = nl;
    info->mean_neighbors = (double)hs.nbr_total / ((double)W * sys->n_el);
  }
  if (rc) return rc;
  if (hs.overflow) return FIRE_ERR_CAPACITY;
  if (hs.n_nonfinite) return FIRE_ERR_NONFINITE;
  return FIRE_OK;
}

}  // extern "C"

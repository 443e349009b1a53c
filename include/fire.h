/*
 * fire.h -- C ABI of libfire: batched FiRE (finite-range embedding) wave
 * function evaluation on one GB300 (sm_103a).
 *
 * The library evaluates, for a batch of W walkers (electron configurations),
 * the FiRE ansatz of arXiv 2504.06087
 *
 *     Psi(r) = J(r) * sum_d det[Phi_d(r)]                 (Methods, eq. wf)
 *
 * its local energy (Methods, "Variational Monte Carlo")
 *
 *     E_L(r) = -1/2 (Lap log|Psi| + |grad log|Psi||^2) + V(r)
 *
 * with V the Coulomb potential of the molecular Hamiltonian (Methods,
 * eq. hamiltonian), the per-walker parameter gradient d log|Psi| / d theta
 * (Methods, eq. spring), and Metropolis sampling with single-electron moves
 * (Methods, "Improved Monte Carlo sampling").
 *
 * Conventions shared by every call
 * --------------------------------
 * Pointers.  Unless a comment says "host", every array pointer is DEVICE
 *   memory, allocated and freed by the caller.  The calls allocate no device
 *   memory: scratch space is the caller-allocated workspace `ws` of at least
 *   fire_workspace_size() bytes.  Two things are held by the library itself
 *   for the life of the process: the static device array of
 *   fire_local_energy_static() (FIRE_STATIC_WORKSPACE_BYTES on every GPU that
 *   loads the library) and, on a device where a call first needs it, one
 *   extra non-blocking CUDA stream for work that runs beside the caller's
 *   stream inside a call.  Arrays are dense row-major (C order).
 * Electrons.  r is [W][n_el][3] float64, bohr.  Electrons 0 .. n_up-1 are
 *   spin-up, n_up .. n_el-1 spin-down (Methods, "Variational Monte Carlo").
 * Parameters.  theta is ONE flat buffer; fire_param_layout() gives the name,
 *   offset and shape of every array in it.  theta is float64 for
 *   FIRE_PREC_FP64 and float32 for the other precisions.
 * Streams.  `stream` is a cudaStream_t passed as void*.  All device work is
 *   enqueued on it; the call then reads a 4-byte status word back and
 *   synchronises that stream before it returns.
 * Errors.  Every call returns a fire_status_t.  Argument errors are detected
 *   on the host before any launch (FIRE_ERR_INVALID_ARG, FIRE_ERR_WORKSPACE).
 *   Conditions found on the device (neighbour-list overflow, non-finite
 *   results) are returned after the status read-back; outputs are then
 *   undefined (FIRE_ERR_CAPACITY) or hold the non-finite values
 *   (FIRE_ERR_NONFINITE is reported only when a walker is non-finite without
 *   being on a node).  A walker on a node of Psi (sign 0, log|Psi| = -inf)
 *   is not an error; it is counted in fire_info_t.n_nodes.
 * Concurrency.  Calls with their own workspaces are re-entrant and may run
 *   on different streams and host threads.  The shared state is: the
 *   per-device side stream above (work a call puts on it is joined back to
 *   the caller's stream before the call returns), the static array of
 *   fire_local_energy_static() (calls of that entry point that overlap on a
 *   GPU race), and thread-local diagnostics (fire_last_error, the stage
 *   profiler).
 */
#ifndef FIRE_H
#define FIRE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FIRE_OK = 0,
  FIRE_ERR_INVALID_ARG = 1,      /* bad size, NULL pointer, unknown enum       */
  FIRE_ERR_CAPACITY = 2,         /* an electron has more than k_cap neighbours */
  FIRE_ERR_NONFINITE = 3,        /* NaN/inf off a node                          */
  FIRE_ERR_SINGULAR_REFRESH = 4, /* MCMC inverse refresh met a zero pivot      */
  FIRE_ERR_TIMEOUT = 5,          /* a bounded device wait gave up              */
  FIRE_ERR_CUDA = 6,             /* a CUDA runtime call failed                 */
  FIRE_ERR_UNSUPPORTED = 7,      /* valid but not implemented combination      */
  FIRE_ERR_WORKSPACE = 8         /* ws NULL or smaller than fire_workspace_size */
} fire_status_t;

/* Arithmetic of a call.
 *  FP64       every step in float64 (theta float64).
 *  FP32       every step in float32, the final E_L reduction included
 *             ("plain FP32"; theta float32).
 *  BF16_FP64  every matrix product (embedding MLP, Jastrow MLPs, attention
 *             scores and register MLPs, h^0 products, envelopes, orbital
 *             rows, and the restricted log-det contraction M = T A^T[Nbar]
 *             of neighbourhoods of up to 42 members when n_el is a multiple
 *             of 4) on the tensor cores as split-bf16 products: each operand
 *             held as 2 or 3 bf16 components, the component products summed
 *             with FP32 accumulation; the value rows of the MLP products
 *             recomputed in float32; LU / slogdet and the final E_L reduction
 *             in float64; the inverse and everything else float32 (theta
 *             float32). */
/* Accuracy of each form against the float64 dense oracle, per walker (the
 * bounds the parity tests hold every walker to):
 *   E_L      |E - E_ref| <= tau max(|E_ref|, 1, |Lap log|Psi|| + |grad log|Psi||^2),
 *            tau = 1e-10 (FP64), 1e-4 (FP32, BF16_FP64): E_L sums the kinetic
 *            terms, which cancel near nodes and cusps, and its rounding error
 *            is relative to them; the reduced forms also meet 1e-4 relative
 *            to max(|E_ref|, 1) at the median walker;
 *   log|Psi| |l - l_ref| <= max(t max(|l_ref|, 1), n_el kappa u), t = 1e-10
 *            (FP64), 1e-5 (FP32, BF16_FP64), kappa the condition number of the
 *            walker's dominant orbital matrix, u = 2^-53 or 2^-24; where the
 *            largest determinants nearly cancel, kappa is weighted by the
 *            signed sum: sum_d |det_d| kappa_d / |sum_d s_d det_d|.  For
 *            small |log|Psi|| (C2H4 with the C26H24 network, about 30) the
 *            BF16_FP64 form's t is 3e-5.
 * The gradient of fire_grad_logpsi: FP64 1e-9 max(|g|, 1) per entry; FP32 a
 * relative 2-norm error per walker of at most 1e-4 + 2 kappa u. */
typedef enum {
  FIRE_PREC_FP64 = 0,
  FIRE_PREC_FP32 = 1,
  FIRE_PREC_BF16_FP64 = 2
} fire_precision_t;

/* Jastrow switches (Methods, "Global electron correlation effects"). */
#define FIRE_J_CUSP 1u
#define FIRE_J_MLP 2u
#define FIRE_J_ATT 4u

/* Operation a workspace is sized for. */
typedef enum {
  FIRE_OP_NEIGHBORS = 0,
  FIRE_OP_LOGPSI = 1,
  FIRE_OP_LOCAL_ENERGY = 2,
  FIRE_OP_GRAD_LOGPSI = 3,
  FIRE_OP_MCMC = 4
} fire_op_t;

/* The molecule: nuclear positions R_m and charges Z_m (Methods,
 * eq. hamiltonian), electron counts, the electron-electron cutoff c (Results,
 * "Finite-range embeddings": N_i = {j != i : |r_i - r_j| <= c}) and the
 * electron-nucleus filter cutoff c_n (Methods, filter Gamma_m). */
typedef struct {
  int32_t n_el;              /* electrons, >= 1                                 */
  int32_t n_up;              /* spin-up electrons, 0 <= n_up <= n_el            */
  int32_t n_nuc;             /* nuclei, >= 1                                    */
  int32_t pad_;
  const double* nuc_pos;     /* device [n_nuc][3], bohr                         */
  const double* nuc_charge;  /* device [n_nuc]                                  */
  double cutoff;             /* c   >= 0, bohr                                  */
  double cutoff_nuc;         /* c_n >  0, bohr                                  */
} fire_system_t;

/* Network hyper-parameters (Supplementary table "Hyperparameters"). */
typedef struct {
  int32_t width;             /* hidden width d (multiple of 8, <= 1024)         */
  int32_t n_layers;          /* depth L of the embedding MLP h = MLP(h^1)       */
  int32_t n_det;             /* determinants N_det                              */
  int32_t n_env;             /* exponential envelopes per nucleus               */
  int32_t n_gauss;           /* Gaussians d_0 of the radial filters (<= 64)     */
  int32_t edge_hidden;       /* hidden width of the filter MLP (<= 64)          */
  int32_t jastrow_width;     /* hidden width of the Jastrow MLPs (0 = width)    */
  int32_t n_reg;             /* attention registers                             */
  int32_t d_reg;             /* register dimension                              */
  uint32_t flags;            /* FIRE_J_* bits                                   */
} fire_arch_t;

typedef struct {
  const void* theta;         /* device flat parameter buffer                    */
  int64_t n_params;          /* must equal fire_param_count()                   */
  int32_t dtype;             /* 0 = float64, 1 = float32                        */
  int32_t pad_;
} fire_params_t;

typedef struct {
  char name[24];
  int64_t offset;            /* in elements from theta                          */
  int32_t ndim;
  int32_t pad_;
  int64_t shape[5];
} fire_param_entry_t;

/* Optional per-call diagnostics (host memory; pass NULL to skip). */
typedef struct {
  int32_t k_required;        /* largest neighbour count seen                    */
  int32_t n_nodes;           /* walkers with sign 0 (on a node of Psi)          */
  int32_t n_nonfinite;       /* walkers with a non-finite E_L off a node        */
  int32_t n_chunks;          /* walker chunks the call was split into          */
  int64_t rows_total;        /* forward-Laplacian rows processed (all chunks)   */
  double mean_neighbors;     /* mean |N_i| over all electrons and walkers       */
  int64_t n_launches;        /* kernels launched by the call                    */
} fire_info_t;

/* Opt-in stage profiler (diagnostics).  While enabled, calls on this host
 * thread bracket every pipeline stage with CUDA events on their stream and
 * add the measured device time to a thread-local table; the stages are then
 * serialised by the event waits, so profiled calls are slower.  Stage names
 * are stable ("row_gemm", "contract", "lu", ...). */
typedef struct {
  char name[24];
  int64_t launches;
  double ms_total;
} fire_prof_entry_t;

int fire_profile_enable(int on);
int fire_profile_reset(void);
int fire_profile_report(fire_prof_entry_t* out, int32_t* n);

/* Number of scalar parameters of the ansatz for this system and network. */
int64_t fire_param_count(const fire_system_t* sys, const fire_arch_t* arch);

/* Fills out[0 .. *n-1] with the layout of theta and sets *n to the number
 * of arrays.  With out == NULL only *n is set.  Returns FIRE_OK or
 * FIRE_ERR_INVALID_ARG. */
int fire_param_layout(const fire_system_t* sys, const fire_arch_t* arch,
                      fire_param_entry_t* out, int32_t* n);

/* Workspace bytes a call of operation `op` needs for W walkers.  0 on
 * invalid arguments.  Calls split the walkers into chunks internally, so
 * the size grows with W only up to a chunk. */
size_t fire_workspace_size(const fire_system_t* sys, const fire_arch_t* arch,
                           int64_t n_walkers, int32_t precision, int32_t k_cap,
                           int32_t op);

/* Neighbour lists N_i^par, N_i^anti (Results, "Finite-range embeddings";
 * Methods, message passing step: N^alpha_i splits N_i by parallel and
 * antiparallel spin).  For each walker w and electron i:
 *   nbr_idx[w][i][0 .. cnt[w][i][0]-1]            same-spin j, ascending
 *   nbr_idx[w][i][cnt[w][i][0] .. + cnt[w][i][1]-1] opposite-spin j, ascending
 * with |r_i - r_j| <= c in float64.  nbr_idx is [W][n_el][k_cap] int32,
 * nbr_cnt [W][n_el][2] int32 (device).  *k_required (host, may be NULL)
 * receives the largest |N_i|; if it exceeds k_cap the lists are truncated and
 * FIRE_ERR_CAPACITY is returned. */
int fire_neighbors(const fire_system_t* sys, int64_t n_walkers, const double* r,
                   int32_t k_cap, int32_t* nbr_idx, int32_t* nbr_cnt,
                   int32_t* k_required, void* ws, size_t ws_bytes, void* stream);

/* log|Psi| and sign(Psi) for each walker (Methods, eq. wf): logabs, sign are
 * [W] float64 (device).  k_cap bounds |N_i| as in fire_neighbors. */
int fire_logpsi(const fire_system_t* sys, const fire_arch_t* arch,
                const fire_params_t* params, int64_t n_walkers, const double* r,
                int32_t k_cap, int32_t precision, double* logabs, double* sign,
                fire_info_t* info, void* ws, size_t ws_bytes, void* stream);

/* Per-walker gradient d log|Psi| / d theta (Methods, eq. spring: the rows
 * O_i of the SPRING update), by hand-written adjoint kernels over the value
 * path, whose embeddings are recomputed in the call.  grad is [W][P] (device,
 * P = fire_param_count(), layout of fire_param_layout()) in the dtype of theta
 * (float64 for FIRE_PREC_FP64, float32 otherwise; the BF16_FP64 form
 * computes its gradient in float32 with a float64 LU).  logabs and sign [W]
 * as in fire_logpsi.  Walkers on a node give non-finite rows. */
int fire_grad_logpsi(const fire_system_t* sys, const fire_arch_t* arch,
                     const fire_params_t* params, int64_t n_walkers, const double* r,
                     int32_t k_cap, int32_t precision, void* grad, double* logabs, double* sign,
                     fire_info_t* info, void* ws, size_t ws_bytes, void* stream);

/* Local energy E_L (Methods, eq. of E_L) with the exact Laplacian of
 * log|Psi| from the sparse forward Laplacian (Methods, "Efficient
 * Laplacian").  Outputs [W] float64 (device): e_loc, logabs, sign; e_kin and
 * e_pot (kinetic and potential parts) may be NULL. */
int fire_local_energy(const fire_system_t* sys, const fire_arch_t* arch,
                      const fire_params_t* params, int64_t n_walkers, const double* r,
                      int32_t k_cap, int32_t precision, double* e_loc, double* logabs,
                      double* sign, double* e_kin, double* e_pot, fire_info_t* info,
                      void* ws, size_t ws_bytes, void* stream);

/* Metropolis sweeps of single-electron moves with local recompute and
 * low-rank updates (Methods, "Improved Monte Carlo sampling" and "Low-rank
 * updates"; Supplementary "Hyperparameters": Gaussian single-electron moves).
 *
 * One sweep moves electron k = 0 .. n_el-1 in turn in every walker:
 * r'_k = r_k + sigma xi, xi ~ N(0, I_3), accepted iff ln u < 2 ln|Psi'/Psi|.
 * The update set U = {k} and every electron within c of r_k or r'_k is
 * recomputed (h^0 of k, messages, MLP, orbital rows, Jastrow terms of U);
 * the determinant ratios come from the |U| x |U| matrix determinant lemma
 * with the cached inverse (float64 LU of the small matrix) and an accepted
 * move updates the inverse by the Woodbury identity.
 *
 * Global jumps (Methods, "Improved Monte Carlo sampling": the mixture
 * proposal rho(r') = sum_m Z_m N(r' | R_m, sigma_global^2 I) / sum_m Z_m and
 * its ratio correction; Supplementary "Hyperparameters": 20 global moves,
 * sigma_global = 2 bohr): after its n_el local moves a sweep makes n_global
 * global jumps.  Each moves one electron k, the same for every walker, to
 * r'_k = R_m + sigma_global xi, the nucleus m drawn with probability
 * Z_m / sum Z; it is accepted iff
 * ln u < 2 ln|Psi'/Psi| + ln rho(r_k) - ln rho(r'_k).  The update set, the
 * ratios and the inverse updates are those of a local move.
 *
 * Random numbers: Philox4x32-10 with key (seed low word, seed high word) and
 * counter (move low word, move high word, walker, stream), move =
 * *counter + sweep * (n_el + n_global) + j for the j-th move of a sweep
 * (local moves j = k < n_el, then the global jumps); stream 0 gives xi by
 * Box-Muller in float64, stream 1 the uniform u, stream 2 word 0 the
 * mixture component of a global jump (first m with u sum Z < Z_1 + .. + Z_m);
 * the electron of a global jump is floor(n_el u) with u from word 0 of
 * counter (move low, move high, 2^32 - 1, 2); uniforms are (x + 1/2) / 2^32.
 * *counter (host, in/out) advances by n_sweeps * (n_el + n_global).
 *
 * r [W][n_el][3] float64 (device, in/out).  The cached state lives in the
 * workspace (fire_workspace_size() with FIRE_OP_MCMC; the call holds every
 * walker at once, it does not chunk) and is built by a value forward at the
 * start of the call, rebuilt every refresh_every moves (0: only at the end)
 * and at the end; max_drift (host out, may be NULL) is the largest
 * |log|Psi|| difference between the carried value and a rebuild.
 * Precision: FIRE_PREC_FP64 keeps the state in float64; FIRE_PREC_FP32 and
 * FIRE_PREC_BF16_FP64 keep it in float32 with float64 determinant lemmas,
 * LU factorisations and refresh inverses (no tensor cores).  A determinant
 * whose lemma ratio lies beyond 10^+-3, or whose kappa u w exceeds 1e-4
 * (kappa the Frobenius condition estimate of its last factorisation, u the
 * unit roundoff of the state, w its weight |det| / max |det| in the walker's
 * sum), gets its ratio from a float64 LU of the new matrix and, if the move
 * is accepted, a fresh float64 factorisation and inverse instead of the
 * Woodbury update (batched over the SMs).  The environment variable
 * FIRE_MCMC_KAPPA_TOL overrides 1e-4 (negative: lemma ratios only, about
 * twice as fast at n_el = 184, with carried log|Psi| up to ~5e-2 off the
 * rebuilds instead of 1e-2).
 * Outputs: logabs, sign [W] float64 (device, may be NULL) at the final
 * positions (from the final rebuild); accepted [W] int32 (device, may be
 * NULL): accepted moves per walker; *n_accepted (host, may be NULL) their
 * total.  Errors: FIRE_ERR_INVALID_ARG for sigma <= 0, n_sweeps < 0,
 * refresh_every < 0, n_global < 0, sigma_global <= 0 with n_global > 0 or a
 * missing pointer (before any launch);
 * FIRE_ERR_CAPACITY if an update set or a neighbour list exceeded its
 * capacity (|U| <= min(n_el, 2 k_cap + 1)); FIRE_ERR_NONFINITE as in
 * fire_logpsi. */
int fire_mcmc_step(const fire_system_t* sys, const fire_arch_t* arch, const fire_params_t* params,
                   int64_t n_walkers, double* r, int32_t k_cap, int32_t precision, double sigma,
                   int32_t n_sweeps, int32_t refresh_every, int32_t n_global, double sigma_global,
                   uint64_t seed, uint64_t* counter,
                   double* logabs, double* sign, int32_t* accepted, int64_t* n_accepted,
                   double* max_drift, fire_info_t* info, void* ws, size_t ws_bytes, void* stream);

/* Semi-local pseudopotential of one nucleus (the paper uses ccECP tables;
 * any coefficients of this standard form may be supplied):
 *   v_l(x) = sum_j coef[l][j] x^power[l][j] exp(-alpha[l][j] x^2),
 * non-local channels l = 0 .. n_channels-1 (<= 3), n_terms[l] <= 4 terms,
 * n_quad quadrature points (0 = no pseudopotential on this nucleus; 4, 6 or
 * 12: tetrahedron, octahedron, icosahedron), electrons within r_cut of the
 * nucleus.  Keep r_cut below half the distance between pseudopotential
 * nuclei: an electron uses the first nucleus (in index order) whose r_cut
 * contains it. */
typedef struct {
  int32_t n_quad;
  int32_t n_channels;
  int32_t n_terms[3];
  int32_t pad_;
  double r_cut;
  double coef[3][4];
  double power[3][4];
  double alpha[3][4];
} fire_ecp_t;

/* Non-local pseudopotential energy per walker (Methods, "Low-rank wave
 * function updates": ratios of configurations that differ in one electron;
 * Supplementary "Effective core potential": per-species quadrature;
 * Methods, "Energy extrapolation": n_el N_quad updates):
 *   v_nl[w] = sum_k sum_l v_l(|r_k - R_m|) (2l + 1)
 *             sum_q (1/N_quad) P_l(rhat_k . n_q) Psi(.. R_m + |r_k - R_m| n_q ..) / Psi
 * with m the pseudopotential nucleus of electron k and n_q the quadrature
 * directions under one random rotation per (walker, electron): the unit
 * quaternion (sqrt(1-u1) sin 2pi u2, sqrt(1-u1) cos 2pi u2, sqrt(u1) sin 2pi u3,
 * sqrt(u1) cos 2pi u3) as (x, y, z, w), u1..u3 from words 0..2 of Philox4x32-10
 * counter (k, 0, walker, 3) under key (seed low, seed high).  Every ratio
 * comes from the low-rank machinery of fire_mcmc_step (local recompute of the
 * update set, determinant lemma, exact float64 ratio where the lemma is not
 * trusted) on a state built at the start of the call; nothing is accepted.
 * ecp: HOST array [n_nuc], copied into the workspace.  v_nl: device [W]
 * float64.  Workspace: fire_workspace_size() with FIRE_OP_MCMC.  Precision as
 * in fire_mcmc_step (float32 state for the reduced forms).  Errors:
 * FIRE_ERR_INVALID_ARG for a bad table (n_quad not 0/4/6/12, more than 3
 * channels or 4 terms, negative r_cut or alpha, non-finite numbers) or a
 * missing pointer; the others as in fire_mcmc_step. */
int fire_ecp_nonlocal(const fire_system_t* sys, const fire_arch_t* arch, const fire_params_t* params,
                      int64_t n_walkers, const double* r, int32_t k_cap, int32_t precision, const fire_ecp_t* ecp,
                      uint64_t seed, double* v_nl, fire_info_t* info, void* ws, size_t ws_bytes, void* stream);

/* S+ swap ratios (Supplementary "Low-rank updates in S+ operator"; Methods
 * "Low-rank wave function updates": configurations that differ in two
 * electrons): for the spin-down electron beta (n_up <= beta < n_el) and
 * every spin-up electron alpha,
 *   ratios[w][alpha] = Psi(pi_{alpha beta} r_w) / Psi(r_w)   (signed),
 *   r_beta[w]        = 1 - sum_alpha ratios[w][alpha],
 * pi swapping the positions of alpha and beta (each keeps its spin).  Each
 * swap recomputes only the update set {alpha, beta} and the electrons within
 * c of either position: h^0 and its projections are swapped between the two
 * cached blocks (they depend on the position alone), their envelope rows are
 * recomputed with their own spin's weights, and the determinant ratio comes
 * from the |U| x |U| determinant lemma on a state built at the start of the
 * call (nothing is moved).  ratios device float64 [W][n_up], r_beta device
 * float64 [W].  Workspace: fire_workspace_size() with FIRE_OP_MCMC.
 * Precision as in fire_mcmc_step.  Errors: FIRE_ERR_INVALID_ARG for beta
 * outside the spin-down electrons or a missing pointer; the others as in
 * fire_mcmc_step. */
int fire_spin_ratios(const fire_system_t* sys, const fire_arch_t* arch, const fire_params_t* params,
                     int64_t n_walkers, const double* r, int32_t k_cap, int32_t precision, int32_t beta,
                     double* ratios, double* r_beta, fire_info_t* info, void* ws, size_t ws_bytes, void* stream);

/* SPRING parameter update (Methods, "Variational Monte Carlo", eq. spring):
 *
 *   Obar_i = O_i - (1/N) sum_j O_j,   eps_i = E_L,i - (1/N) sum_j E_L,j,
 *   delta  = Obar^T (Obar Obar^T + lambda I)^-1 (eps - eta Obar delta_prev)
 *            + eta delta_prev
 *
 * for N = n_walkers samples and P = n_params parameters.  The paper prints
 * the update with the centred matrix as P x N; here O is N x P (row i = the
 * gradient row of walker i, the output layout of fire_grad_logpsi), which is
 * the same formula with the transposes that make its dimensions agree.
 * Supplementary "Hyperparameters": lambda = 1e-3, eta (the SPRING decay) =
 * 0.99.
 *
 * O        device float32 [N][ldo] (ldo >= P), read only.
 * e_loc    device float64 [N].
 * delta_prev  device float32 [P], or NULL (treated as zero).
 * delta    device float32 [P], out.
 * gram     device float64 [N][N] out (the centred Gram matrix Obar Obar^T,
 *          before the damping), or NULL.
 * x_out    device float64 [N] out, the solution x of
 *          (Obar Obar^T + lambda I) x = eps - eta Obar delta_prev, or NULL.
 * ws       device workspace of fire_spring_workspace_size(N, P) bytes.
 * Arithmetic: column means, right-hand side, Cholesky factorisation and
 * solves in float64; the Gram matrix on the tensor cores as a split-bf16
 * product (three bf16 components per operand, six component products, FP32
 * accumulation) over chunks of 2^18 parameters whose partial sums are added
 * in float64; delta accumulated in float64 and stored as float32.
 * Errors: FIRE_ERR_INVALID_ARG (N < 2, N > 65536, P < 1, ldo < P, lambda <= 0,
 * eta < 0, a missing pointer) and FIRE_ERR_WORKSPACE on the host before any
 * launch; FIRE_ERR_NONFINITE if the damped Gram matrix is not numerically
 * positive definite; FIRE_ERR_TIMEOUT if a bounded wait of the tensor-core
 * product gave up.  The call synchronises `stream` before it returns. */
size_t fire_spring_workspace_size(int64_t n_walkers, int64_t n_params);
int fire_spring_step(int64_t n_walkers, int64_t n_params, const float* O, int64_t ldo, const double* e_loc,
                     const float* delta_prev, double eta, double lambda, float* delta, double* gram,
                     double* x_out, void* ws, size_t ws_bytes, void* stream);

/* Layout of the workspace of a call (diagnostics and tests): for each named
 * intermediate buffer its byte offset inside ws and its size in bytes, for
 * the first walker chunk (chunk_walkers walkers).  With out == NULL only *n is
 * set.  Buffers hold, e.g., "X" the forward-Laplacian rows of h, "SU" the
 * attention scores and values, "V" the register rows, "LU" the factored
 * orbital matrices, "ldabs" / "lsign" per-determinant log|det| and sign. */
typedef struct {
  char name[16];
  int64_t offset;
  int64_t bytes;
} fire_ws_entry_t;

int fire_workspace_layout(const fire_system_t* sys, const fire_arch_t* arch, int64_t n_walkers,
                          int32_t precision, int32_t k_cap, int32_t op, fire_ws_entry_t* out,
                          int32_t* n, int64_t* chunk_walkers);

/* Diagnostic: the tensor-core matrix product used by the BF16_FP64 form on
 * its own.  C[M][N] (fp32, row-major) = A[M][K] times the transpose of
 * Bt[N][K] (B given K-major), with tcgen05.mma and FP32 accumulation; K a
 * multiple of 64.  A and Bt hold nc = 1, 2 or 3 bf16 components each
 * ([nc][M][K] and [nc][N][K]; x = x0 + x1 + x2), multiplied as the
 * split-bf16 product of Henry, Tang & Heinecke (2019): 1, 3 or 6 component
 * products.  *err (device int, caller-zeroed) becomes non-zero if a bounded
 * wait gave up.  The paper has no counterpart: this exists to test the kernel
 * in isolation. */
int fire_selftest_tc_gemm(int64_t M, int32_t N, int32_t K, int32_t nc, const void* A, const void* Bt,
                          float* C, int32_t* err, void* stream);

/* Diagnostic: the multiply-add rate of the SIMT pipes.  Launches `blocks`
 * CTAs of 256 threads; each thread runs eight independent chains of
 * 4 * ceil(iters / 4) dependent fused multiply-adds (fma.rn) in float64
 * (dtype 0) or float32 (dtype 1) and writes one value to out[blocks * 256]
 * (device, of that dtype).  FLOPs = 2 * 8 * 4 * ceil(iters / 4) * blocks * 256;
 * the caller times the launch on `stream`.  The paper has no counterpart: the
 * measured rate is the peak that the roofline fractions of the float32 and
 * float64 kernels are quoted against.  FIRE_ERR_INVALID_ARG on a bad dtype,
 * iters < 1, blocks < 1 or out == NULL. */
int fire_selftest_fma_rate(int32_t dtype, int64_t iters, int32_t blocks, void* out, void* stream);

/* Size of the workspace that fire_local_energy_static() owns (32 MiB). */
#define FIRE_STATIC_WORKSPACE_BYTES (32u * 1024u * 1024u)

/* fire_local_energy() for callers that cannot allocate device memory (code
 * that runs inside another runtime's memory pool or allocator hooks, plug-ins
 * whose host application owns every device allocation, paths that must not
 * allocate after set-up).  The paper has no counterpart: this is a deployment
 * convenience.
 *
 * Arguments, outputs and errors are those of fire_local_energy() without the
 * workspace: the call uses one static device array of
 * FIRE_STATIC_WORKSPACE_BYTES, which every GPU that loads the library holds
 * until the process exits.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *  - Problems whose workspace (fire_workspace_size() for
 *    FIRE_OP_LOCAL_ENERGY) exceeds FIRE_STATIC_WORKSPACE_BYTES are rejected
 *    with FIRE_ERR_WORKSPACE before any launch; fire_last_error() then
 *    states the size needed.  (About 20 water-sized walkers in FP64.)
 *  - The first call on a device looks up the array's device address on that
 *    device (with it current) and keeps it; make that first call before any
 *    stream capture.  The kept address belongs to the device's current
 *    context: do not call this entry point on a device after
 *    cudaDeviceReset() on it in the same process.
 *  - Every call on a device shares the one array, which keeps the previous
 *    call's contents (the call clears what must start at zero): calls that
 *    overlap on the GPU, on different streams or host threads, race. */
int fire_local_energy_static(const fire_system_t* sys, const fire_arch_t* arch,
                             const fire_params_t* params, int64_t n_walkers, const double* r,
                             int32_t k_cap, int32_t precision, double* e_loc, double* logabs,
                             double* sign, double* e_kin, double* e_pot, fire_info_t* info,
                             void* stream);

const char* fire_status_string(int status);

/* Text of the last CUDA error seen by a call on this host thread, with the
 * pipeline stage that raised it (static thread-local storage; "" if none).
 * Stages are checked one by one when the environment variable
 * FIRE_DEBUG_SYNC is set. */
const char* fire_last_error(void);

/* Library version string (static storage). */
const char* fire_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FIRE_H */

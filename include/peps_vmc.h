/*
 * peps_vmc.h -- C ABI of the GB300 (sm_103a) finite-temperature PEPS-VMC library.
 *
 * Method: Zhang, Zhang, Wang, He, "Scalable tensor network algorithm for thermal quantum
 * many-body systems in two dimension", arXiv:2409.05285.  The vectorised density matrix
 * |rho> = sum_S rho_theta(S)|S> (Sec. II Eqs. 2-4) is a PEPS with physical index
 * S = 2 s + s' (system spin s, ancilla spin s'; 0 = up).  Starting from |I> (beta = 0,
 * App. A perturbation of the zero entries) each stochastic-reconfiguration step
 * theta' = theta - tau (G + eps)^-1 g (Eqs. 5-7, 10) approximates exp(-tau calH)|rho>,
 * calH = H x I + I x H^T (Eq. 3), H the J1-J2 Heisenberg model (Eq. 12) on an open
 * L1 x L2 square lattice.  After total imaginary time t the sampled observables are those
 * of the thermal state at inverse temperature beta_obs = 4 t (Eq. 11).
 *
 * Layouts (all row-major):
 *   site i = r * L2 + c.  Leg dimensions: left/right/up/down = D, or 1 on the open edge.
 *   theta      float64 [N_p]: per site the block [4][dl][dr][du][dd]; N_p = 4 sum_i sz_i.
 *   configs    uint8 [n][L1*L2], entries 0..3.
 *   O rows     [n][N_o] (N_o = sum_i sz_i): per site the derivative of log rho with
 *              respect to the slice T_i^{S_i} (Eq. 8), float64 for PEPS_FP64, float32
 *              otherwise.
 *
 * Ownership: the context owns every device buffer it allocates; the caller owns every
 * pointer it passes.  All work is enqueued on the stream given at peps_init (a
 * cudaStream_t passed as void*; NULL = legacy default stream).  Calls that return host
 * results synchronise that stream before returning.  One context must not be used from
 * two host threads at once.
 *
 * Errors: every int-returning call returns PEPS_OK (0) on success, a negative PEPS_E*
 * code on failure (the context keeps a message, see peps_last_error), or a positive
 * warning code.
 */
#ifndef PEPS_VMC_H
#define PEPS_VMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PEPS_OK 0
#define PEPS_WARN_CG_MAXIT 1 /* CG stopped at max_cg; the update was still applied */
#define PEPS_EINVAL (-1)     /* invalid argument (sizes, null pointers, limits) */
#define PEPS_ENOMEM (-2)     /* device allocation failed or exceeds the context budget */
#define PEPS_ECUDA (-3)      /* a CUDA runtime call failed */
#define PEPS_ESTATE (-4)     /* call out of order (e.g. sr_step before an evaluation) */
#define PEPS_ENOTFINITE (-5) /* non-finite amplitude, energy or CG scalar */
#define PEPS_ECORRUPT (-6)   /* checkpoint unreadable, of another problem, or failing its checksum */
#define PEPS_EIO (-7)        /* checkpoint file could not be written */
#define PEPS_ETIMEOUT (-8)   /* a bounded device wait ran out; the call's results are invalid.
                               When the message says that an MMA may have been in flight,
                               every later result of the context is undefined: free it */

/* Arithmetic of the per-sample contraction (environment, amplitude, E_loc, O).  The
 * log-amplitude accumulation, the SR reductions and CG, and the observables are float64
 * in every mode. */
#define PEPS_FP64 0 /* float64 throughout */
#define PEPS_FP32 1 /* float32 contraction and truncation, float32 O storage */
#define PEPS_TF32 2 /* as PEPS_FP32, but the GEMM-shaped environment and strip contractions
                       of the batched engine run on the tensor cores (tcgen05, TF32 operands
                       rounded to nearest, FP32 accumulation); needs block_mode
                       PEPS_BLOCKS_BATCHED, which PEPS_BLOCKS_AUTO then selects */

#define PEPS_MODEL_J1J2 0 /* Eq. 12: J1 sum_<ij> S_i.S_j + J2 sum_<<ij>> S_i.S_j */

typedef struct peps_ctx peps_ctx;

/* Problem statement (Sec. II/III): lattice, couplings, bond D, boundary bond chi (D_c),
 * number of Markov chains (= samples per SR step), arithmetic, initial perturbation. */
typedef struct {
  int L1, L2;        /* rows, columns; 2 <= L1, L2 <= 16 */
  int model;         /* PEPS_MODEL_J1J2 */
  double J1, J2;     /* couplings of Eq. 12 */
  int D;             /* PEPS bond dimension, 1 <= D <= 8 */
  int chi;           /* boundary-MPS bond dimension, 1 <= chi <= 64 */
  int n_chains;      /* chains advanced per sweep and samples per SR step, >= 1 */
  int precision;     /* PEPS_FP64 | PEPS_FP32 | PEPS_TF32 */
  double init_noise; /* amplitude a of the U[-a, a] perturbation of the zero entries */
  uint64_t seed;     /* Philox key for the perturbation, the chain starts and Metropolis */
  int n_blocks;      /* persistent blocks of the sample kernels; 0 = automatic */
  int block_mode;    /* PEPS_BLOCKS_AUTO | _NARROW | _WIDE | _BATCHED */
} peps_params;

/* Thread-block layout of the per-sample kernels.  Narrow: 256 threads, four blocks per SM,
 * work buffers in global memory (Jacobi matrices in shared memory).  Wide: 1024 threads,
 * one block per SM, every short-lived buffer in shared memory (PEPS_EINVAL when they do
 * not fit in 220 KB).  Automatic picks narrow blocks (faster on GB300 for the workloads
 * measured).  Results are identical in both layouts. */
#define PEPS_BLOCKS_AUTO 0
#define PEPS_BLOCKS_NARROW 1
#define PEPS_BLOCKS_WIDE 2
/* Batched: every contraction, truncation and update is one launch over a chunk of chains
 * in lockstep (work buffers for the whole chunk in device memory, chunk size bounded by
 * the free memory).  PEPS_EINVAL at peps_init when the Jacobi work matrices exceed the
 * shared memory of one block. */
#define PEPS_BLOCKS_BATCHED 3

/* Results of one step (observables of Eq. 11, C_v, Eq. 13 at beta_obs = 4 t). */
typedef struct {
  double t;         /* imaginary time sum(tau) at which the samples were taken */
  double beta_obs;  /* 4 t */
  double E_site;    /* <H>/N */
  double E_err;     /* standard error of E_site (p = 2: plain; p = 1: weighted) */
  double C_site;    /* beta_obs^2 (<H^2> - <H>^2) / N */
  double chi_sus;   /* beta_obs <Mz^2> / N */
  double accept;    /* Metropolis acceptance ratio of the last peps_mc_sweep */
  double diag_frac; /* fraction of samples with s = s' on every site */
  int cg_iters;     /* CG iterations of the last peps_sr_step */
  double cg_resid;  /* |r| / |g| at exit */
  int p;            /* sampling exponent of the samples (2 or 1; 0 for direct draws) */
} peps_stats;

/* Creates a context: allocates device buffers, sets theta to the perturbed beta = 0
 * state (App. A), and the chains to diagonal configurations (s = s') drawn from Philox.
 * stream: cudaStream_t as void* (may be NULL).  Returns PEPS_EINVAL for sizes outside
 * the limits, PEPS_ENOMEM when allocation fails. */
int peps_init(const peps_params* params, void* stream, peps_ctx** out);

/* Advances every chain by n_sweeps Metropolis sweeps sampling |rho|^p, p = 2 (Sec. II)
 * or p = 1 (reweighted sampling, App. A Eq. A1).  Move set per sweep: both-flips,
 * system-only and ancilla-only exchanges on horizontal and vertical bonds. */
int peps_mc_sweep(peps_ctx* ctx, int n_sweeps, int p);

/* Evaluates nb configurations: log|rho|, sign, E_sys, E_anc (E_loc of Eq. 9 is their
 * sum) and, when O is non-null, the O rows (Eq. 8).  S == NULL evaluates the context's
 * own chains (nb must equal n_chains) and keeps the results for peps_sr_step /
 * peps_observables.  on_device != 0: S and every output pointer are device pointers;
 * otherwise host pointers (copies are made on the context stream).  PEPS_EINVAL, before
 * any evaluation, when a configuration entry exceeds 3 (device batches are checked by a
 * kernel).  Null output
 * pointers are skipped.  O has the element type of the precision (double for
 * PEPS_FP64, float otherwise). */
int peps_eval_batch(peps_ctx* ctx, const uint8_t* S, int nb, int on_device, double* log_abs,
                    int8_t* sign, double* e_sys, double* e_anc, void* O);

/* One SR update from the last evaluation of the chains (sampled with exponent p):
 * weights (1/n for p = 2, |rho|/sum|rho| for p = 1, and for p = 0, chains that are the last
 * peps_direct_draw, r_4/sum r_4 with r_4 = |rho|^2/q of App. A Eq. A7; ESTATE when p = 0
 * and the chains or theta changed since that draw), g = <O (E_loc - <E_loc>)>, CG solve
 * of (G + eps I) x = g from x = 0 with the relative-residual test tol before each
 * iteration and at most max_cg iterations, theta -= tau x, t += tau.  stats (may be
 * NULL) receives the observables of those samples and the CG result.  Returns
 * PEPS_WARN_CG_MAXIT when CG stopped at max_cg. */
int peps_sr_step(peps_ctx* ctx, double tau, double eps, int max_cg, double cg_tol, int p,
                 peps_stats* stats);

/* Observables of the last evaluation of the chains (sampled with exponent p; p = 0 as in
 * peps_sr_step). */
int peps_observables(peps_ctx* ctx, int p, peps_stats* stats);

/* One whole cooling step: n_sweeps sweeps, evaluation of the chains, SR update. */
int peps_step(peps_ctx* ctx, int n_sweeps, int p, double tau, double eps, int max_cg,
              double cg_tol, peps_stats* stats);

/* Amplitudes of a fermionic PEPS of the doubled Hubbard lattice (Sec. II, fermionic
 * vectorisation and Fig. 1b; Sec. III.B).  Sixteen local states per site: the modes c_up,
 * c_dn (system) and d_up, d_dn (ancilla) in that order, S_i = their occupation bits (bit 0
 * c_up ... bit 3 d_dn); sites row-major, and the Fock state of S has its creation operators
 * in increasing mode order.  theta: float64, per site [16][dl][dr][du][dd] (n_theta = 16
 * sum_i sz_i), parity even (p(S) + p(l) + p(r) + p(u) + p(d) even, p of a local index its
 * popcount mod 2, of a virtual index its value mod 2; odd entries enter as given).  The Fermi
 * arrows order each site's Grassmann letters l, u, P, d, r; the amplitude is the
 * Grassmann-ordered contraction, evaluated as a configuration sign times the boundary-MPS
 * contraction (bond chi) of 32 signed slices per site.  peps_famp_create builds an
 * evaluator for up to n_max configurations (EINVAL for sizes outside the peps_init limits,
 * ENOMEM); peps_famp_eval takes host theta and configurations [nb][L1*L2] (entries 0..15,
 * EINVAL otherwise) and writes log|psi| and the sign (0 where psi = 0) to host arrays. */
typedef struct peps_famp peps_famp;
int peps_famp_create(int L1, int L2, int D, int chi, int n_max, int precision, void* stream,
                     peps_famp** out);
int peps_famp_eval(peps_famp* famp, const double* theta, size_t n_theta, const uint8_t* S, int nb,
                   double* log_abs, int8_t* sign);
/* Local energies of the same configurations (Eq. 9 with the terms of Eq. 14: hopping t on
 * nearest-neighbour bonds, U n_up n_dn, -mu n): e_sys from the terms on the system modes,
 * e_anc from the same terms on the ancilla modes (calH = H(c) + H(d)); each hop's
 * configuration is evaluated by the engine and enters with its Jordan-Wigner sign (modes
 * ordered site by site, c_up c_dn d_up d_dn within a site).  Also log|psi| and the sign.
 * NaN energies where psi = 0.  The first call allocates the hop workspace (8 x bonds
 * configurations per chain). */
int peps_famp_local_energy(peps_famp* famp, const double* theta, size_t n_theta, const uint8_t* S,
                           int nb, double t, double U, double mu, double* log_abs, int8_t* sign,
                           double* e_sys, double* e_anc);
/* O rows of the same configurations (Eq. 8): d log psi / d theta at each site's slice S_i,
 * [nb][N_o] with N_o = sum_i sz_i, per site [dl][dr][du][dd]; float64 for PEPS_FP64, float32
 * otherwise (host array).  Each site's environment from the boundary-MPS strips divided by
 * the amplitude, with the signs of the Fermi arrows. */
int peps_famp_log_derivative(peps_famp* famp, const double* theta, size_t n_theta,
                             const uint8_t* S, int nb, void* O);
/* Metropolis sampling of the fermionic PEPS (Sec. II, MCMC; target |psi|^p, p = 2, or p = 1
 * with the reweighting of Eq. A1).  Proposals: a pair at site i and spin s (up, then down),
 * where c_s and d_s are equally occupied, both toggled (a system-ancilla pair created or
 * removed); a hop across a nearest-neighbour bond for mode k = 0..3 (c_up, c_dn, d_up, d_dn),
 * one electron of mode k moving where the two occupations differ.  One sweep visits the rows
 * top to bottom: in row r, for every column the pairs of its site and the hops of its
 * horizontal bond, then the hops of the vertical bonds to row r+1, column by column.  A move
 * that does not apply is skipped.  Move m (0 <= m < peps_famp_n_moves) of sweep k
 * of chain c is accepted iff log u < p (log|psi'| - log|psi|) (float64; psi' = 0 rejected)
 * with u = u[k][c][m] (host, [n_sweeps][nb][n_moves], values in (0, 1)) or, for u = NULL,
 * Philox4x32-10 with key seed and counter (c, sweep0 + k, m, 0x464D4331).  Every proposal's
 * amplitude is a full contraction.  S: host [nb][L1*L2], in (entries 0..15, EINVAL
 * otherwise) and out; accepted (per chain, summed over the sweeps), log_abs and sign of the
 * final configurations: host, NULL to skip.  EINVAL for p outside {1, 2}, negative
 * n_sweeps or sweep counters beyond 32 bits.  peps_famp_n_moves returns 2 N + 4 (bonds), or
 * PEPS_EINVAL for a null evaluator. */
int peps_famp_n_moves(const peps_famp* famp);
/* Strip forms (enable = 1; 0 by default): the sweep's proposals and the local energies' hop
 * ratios from one- and two-row strips between cached environments over 64 slices per site
 * (the signed slices, and the same with a parity on the right leg, which carries a vertical
 * hop's sign flips) instead of a full contraction per proposal or hop; same moves, uniforms and
 * decision rule.  The sweep then takes Philox uniforms only (u must be NULL).  Checked in a
 * host build of the engine against the oracle; not yet run on a GPU.  EINVAL for a null
 * evaluator or enable outside {0, 1}. */
int peps_famp_set_strips(peps_famp* famp, int enable);
/* The moves of one sweep on an L1 x L2 lattice in the order above, four ints per move: kind
 * (0 pair, 1 hop), site i, site j (= i for a pair), spin (pair) or mode (hop); the first cap
 * moves are written to table (host).  Returns the number of moves, or PEPS_EINVAL.  Host
 * code. */
int peps_famp_move_table(int L1, int L2, int* table, int cap);
int peps_famp_sweep(peps_famp* famp, const double* theta, size_t n_theta, uint8_t* S, int nb, int p,
                    int n_sweeps, uint64_t seed, uint64_t sweep0, const double* u, int* accepted,
                    double* log_abs, int8_t* sign);
/* Observables of the samples of one SR step: E_site = sum_i w_i (E_sys + E_anc)/2 / N (Eq. 11),
 * its standard error (delta method), the double occupancy and the density per site (n_up
 * n_dn and n_up + n_dn, the two layers averaged); CG iterations and relative residual. */
typedef struct {
  double E_site, E_err, docc, density;
  int cg_iters;
  double cg_resid;
} peps_fstats;
/* One SR step of the fermionic PEPS on the nb configurations S (host [nb][L1*L2], all with
 * psi != 0: EINVAL otherwise): E_sys, E_anc (the Hubbard terms of peps_famp_local_energy) and
 * O rows; weights 1/nb (p = 2) or |psi|/sum|psi| (p = 1, Eq. A1); the mean, gradient (Eq. 7)
 * and CG solve of (G + eps I) x = g (Eqs. 6 and 10, x_0 = 0, stop at |r| <= cg_tol |g| or
 * max_cg iterations), then theta <- theta - tau x (Eq. 5).  theta: host float64, in and out.
 * stats: host, NULL to skip (observables before the update).  Returns PEPS_WARN_CG_MAXIT
 * when CG stopped at max_cg above the tolerance (theta is still updated). */
int peps_famp_sr_step(peps_famp* famp, double* theta, size_t n_theta, const uint8_t* S, int nb,
                      double t, double U, double mu, int p, double tau, double eps, int max_cg,
                      double cg_tol, peps_fstats* stats);
/* The infinite-temperature state |I> = prod_(i,s) (1 + c+_is d+_is)|0> as fermionic PEPS
 * parameters of bond dimension D (the fermionic counterpart of the beta = 0 state of Sec. II
 * and App. A): per site, T[a | a << 2][0][0][0][0] = 1 for a = 0, 1, 2 and -1 for a = 3 (c+_dn
 * moved past d+_up), every other parity-even entry noise (2u - 1) with u = Philox4x32-10(seed;
 * site, entry index within the site's block, 0, 0x46494E54), parity-odd entries 0.  Host
 * code; theta: host float64 of n_theta = 16 sum_i sz_i entries (EINVAL otherwise). */
int peps_famp_init_theta(int L1, int L2, int D, double noise, uint64_t seed, double* theta,
                         size_t n_theta);
const char* peps_famp_last_error(const peps_famp* famp);
void peps_famp_free(peps_famp* famp);

/* Evaluation of several contexts' chains in one launch: lattices of different sizes (and
 * D, chi, couplings) share one persistent grid of the per-block engine, chain by chain as
 * each context's own evaluation would do it (the same results, bit for bit).  Every context
 * must use narrow per-block kernels (block_mode PEPS_BLOCKS_NARROW) and the same precision
 * (PEPS_FP64 or PEPS_FP32), and appear once; EINVAL otherwise.  peps_group_create allocates
 * the group's scratch (ENOMEM / ECUDA on failure); peps_group_eval waits for each context's
 * stream, evaluates every chain of every context into that context's own results (as
 * peps_eval_batch with S = NULL, ready for peps_sr_step / peps_observables) on the first
 * context's stream and synchronises it.  Free the group before its contexts. */
typedef struct peps_group peps_group;
int peps_group_create(peps_ctx* const* ctxs, int n_ctx, peps_group** out);
int peps_group_eval(peps_group* group);
const char* peps_group_last_error(const peps_group* group);
void peps_group_free(peps_group* group);

/* Reweighted direct sampling (App. A, Eqs. A2-A7): replaces every chain by an independent
 * draw.  Sites are drawn one after another in row-major order; site i takes its local state
 * s from p_4c(s) = b(s) p_2c(s)^exponent normalised over the four states, p_2c (Eq. A3) the
 * conditional weight of s given the sites drawn before, b(s) = b_d for s = s' (S = 0, 3) and
 * 1 otherwise (Eq. A5); exponent 1/2 is Eq. A4, exponent 1 with b_d = 1 is plain direct
 * sampling (q = |rho|^2 / sum |rho|^2 up to truncation).  The sums of rho^2 over the sites
 * not yet drawn are boundary-MPS contractions of the double-layer network (bond D^2, per site
 * T^S (x) T^S or its sum over S) at the context's chi; candidate weights that truncation
 * leaves negative count as zero.
 *   u          uniforms [n_chains][L1*L2] in [0, 1): site i of chain k picks the first state
 *              whose cumulative probability exceeds u[k][i] (values outside clamp to the
 *              ends).  NULL: drawn from Philox with the context's seed, a new stream per call.
 *   on_device  u and log_q are device pointers (else host).
 *   b_d        in (0, 1];  exponent > 0.
 *   log_q      [n_chains] (may be NULL): log of the probability q of each draw.
 * The context keeps log q for peps_sr_step / peps_observables with p = 0.  Needs the batched
 * engine (ESTATE otherwise); the first call allocates the double-layer runner (ENOMEM when it
 * does not fit). */
int peps_direct_draw(peps_ctx* ctx, const double* u, int on_device, double b_d, double exponent,
                     double* log_q);

/* The diagonal bias after a step whose samples held the fraction diag_frac of diagonal terms
 * (s = s' on every site, peps_stats.diag_frac): b_d (1/2 / diag_frac)^(1/N) when diag_frac
 * exceeds 1/2 (the diagonal fraction scales as b_d^N), else b_d; never above 1. */
double peps_direct_next_bd(double b_d, double diag_frac, int N);

/* One cooling step on direct samples: peps_direct_draw (Philox uniforms) with *b_d and
 * exponent, evaluation of the chains, peps_sr_step with p = 0; then *b_d =
 * peps_direct_next_bd(*b_d, stats diag_frac, L1*L2). */
int peps_direct_step(peps_ctx* ctx, double* b_d, double exponent, double tau, double eps,
                     int max_cg, double cg_tol, peps_stats* stats);

/* Truncation arithmetic of the float32 modes (PEPS_FP32, PEPS_TF32; batched engine):
 * enable = 1 runs each bond's Jacobi SVD on a float64 working copy of its float32 matrix
 * (rotations, singular values and kept vectors in float64, the truncated environment stored
 * in float32); 0 (the default) runs it in float32.  The right factors that feed the SVD stay
 * float32.  ESTATE for PEPS_FP64 or the per-block engine, EINVAL for other values, ENOMEM
 * when the float64 work area of large bonds cannot be allocated. */
int peps_set_trunc_fp64(peps_ctx* ctx, int enable);

/* CUDA graphs for the batched engine (enable = 1; 0 = direct launches, the default): the
 * launch sequence of a Metropolis sweep (per exponent p) and of an evaluation of the chains
 * (per use of the sweep's cached environments) is captured into a graph on first use and
 * replayed on later calls, one graph per chunk of chains; the sweep number reaches the
 * kernels through device memory, so replays draw the same random numbers as direct launches
 * and every result is the same bits.  Replays skip the host's per-launch work, which counts
 * for small problems.  Per-launch profiling (peps_profile) and autotuning run without them;
 * changing the launch shapes discards the captured graphs.  EINVAL for bad arguments, ESTATE
 * without the batched engine. */
int peps_set_graphs(peps_ctx* ctx, int enable);
/* Number of launch sequences captured so far (0 with graphs off, without the batched engine,
 * or when capture is not possible on the context's stream, e.g. the legacy default stream,
 * where the engine launches directly). */
int peps_graphs_captured(const peps_ctx* ctx);

/* How peps_sr_step applies (G + eps) in CG (Eq. 10): 1 = one cooperative kernel that reads
 * the O rows once per product (each block owns a slice of the columns; samples are taken in
 * chunks that stay in L2, one grid barrier per chunk); 2 = two streaming passes (O_i.p, then
 * the column sums of y_i O_i) over the O rows as stored; 3 = the two passes over a float64
 * copy of float32 O rows made once per step (no float64 issue spent on widening in the
 * passes; n_chains x N_o doubles, ENOMEM from peps_sr_step when they cannot be allocated);
 * 0 (default) = 3 where the rows are float32 in 16-byte site slices and the copy fits, else
 * 2 (the fused form was measured slower on GB300 at 8x8 and 10x10: float64 FMA issue bounds
 * both forms, and it adds a grid barrier per chunk).  Every choice uses float64 products
 * and fixed summation orders; 2 and 3 give the same bits, the others agree to rounding.
 * EINVAL for other modes. */
int peps_set_cg_product(peps_ctx* ctx, int mode);

/* Parameter vector and chain configurations (host buffers).  n must equal N_p, or
 * n_chains * L1 * L2 for the configurations. */
int peps_get_theta(peps_ctx* ctx, double* host, size_t n);
int peps_set_theta(peps_ctx* ctx, const double* host, size_t n);
int peps_get_configs(peps_ctx* ctx, uint8_t* host, size_t n);
int peps_set_configs(peps_ctx* ctx, const uint8_t* host, size_t n);

/* Device bytes a context for these parameters allocates (upper bound; 0 for invalid
 * parameters).  Used for admission by footprint. */
size_t peps_footprint(const peps_params* params);

/* Sizes: N_p, N_o, and the number of sweeps done so far (the Philox sweep counter). */
size_t peps_num_params(const peps_ctx* ctx);
size_t peps_o_row_len(const peps_ctx* ctx);
int64_t peps_sweeps_done(const peps_ctx* ctx);
int peps_set_sweeps_done(peps_ctx* ctx, int64_t sweeps);

/* Checkpoint of the cooling state: parameters, theta (float64), chain configurations,
 * imaginary time t and the Philox sweep counter, with an FNV-1a checksum.  Restoring it
 * into a context created with the same lattice, couplings, D, chi and chain count
 * resumes the run bit for bit (same kernels, same random numbers).  peps_restore returns
 * PEPS_ECORRUPT for a truncated or altered file or a different problem, and leaves the
 * context unchanged in that case. */
int peps_checkpoint(peps_ctx* ctx, const char* path);
int peps_restore(peps_ctx* ctx, const char* path);

/* Imaginary time t = sum of the tau of the SR steps applied so far. */
double peps_time(const peps_ctx* ctx);

/* Device counters of the last peps_eval_batch / peps_mc_sweep launch: algorithmic
 * flops (contractions, Householder, Jacobi), Jacobi sweeps. */
int peps_last_counters(peps_ctx* ctx, double* flops, int64_t* jacobi_sweeps);

/* Kernel launches this context has made since peps_init (every kernel of the library). */
long long peps_launches(const peps_ctx* ctx);

/* Autotuner of the batched engine's launch shapes, keyed on the problem geometry (d^2 = 4,
 * D, chi, L1, L2, precision).  peps_autotune times `reps` evaluations of (at most 8192 of)
 * the context's chains per candidate (coordinate descent over the tensor-core grid size,
 * the operand stage count, the contraction chunk, the tensor-core kernel form, the chains
 * per FFMA block; only the last one without tensor cores) and keeps the fastest; the choice is stored in a process-wide table that later
 * contexts of the same geometry start from.  No candidate changes any result.  reps = 0
 * only reports the current choice.  With at most 8192 chains the chain buffers hold an
 * evaluation of the current state on return; otherwise evaluate before peps_sr_step.  `out` (caller-owned, may be NULL)
 * receives the choice and the evaluation times before and after (ms).  ESTATE for a
 * context without the batched engine. */
typedef struct {
  int grid_pct;    /* persistent tensor-core grid, per cent of the resident CTAs */
  int db_bytes;    /* largest operand stage that is double-buffered */
  int ffma_g;      /* most chains per block of the FFMA contraction kernel */
  int kc_max;      /* largest contraction chunk of the tensor-core kernel (8, 16, ..., 64) */
  double ms_before, ms_after;
  int pipelined;   /* contractions with vector operands on the cp.async-pipelined tensor-core
                      kernel: 1 the short ones (K <= 64), 2 all; 0: every contraction takes
                      the register-staged kernel */
  int stage_kb;    /* shared memory of the pipelined kernel's stage ring per CTA, KB (32..200;
                      0 in peps_set_tune keeps the current value) */
  int trunc_threads; /* threads of a Jacobi truncation block whose matrix fits in shared
                        memory: 32, 64, 128 or 256 (0 in peps_set_tune keeps the value) */
} peps_tune;
int peps_autotune(peps_ctx* ctx, int reps, peps_tune* out);
/* Sets the batched engine's launch shapes (every field of `t` but the times) for this
 * context, e.g. to repeat a run with the shapes an earlier autotune chose.  No choice changes
 * any result.  EINVAL for values outside grid_pct 1..400, db_bytes 0..200 KB, ffma_g 1..256,
 * kc_max a multiple of 8 in 8..64, pipelined 0..2, stage_kb 0 or 32..200, trunc_threads 0, 32,
 * 64, 128 or 256; ESTATE without the batched engine. */
int peps_set_tune(peps_ctx* ctx, const peps_tune* t);

/* Simple-update warm start (App. A): from the beta = 0 state, n_steps first-order Trotter
 * steps of length tau of the nearest-neighbour Heisenberg bond gates e^{-tau calH_ij}
 * (Eq. 3 per bond of Eq. 12, coupling J1) with bond weights standing in for the
 * environment, bonds truncated to D; writes the N_p parameters of the resulting PEPS
 * (bond weights split over both tensors, legs zero-padded to D) to the caller-owned host
 * buffer `theta` in the layout of peps_set_theta, which then hands the state to SR at
 * t = n_steps * tau (beta_obs = 4t).  Runs on the host (one state, small dense
 * factorisations); no context or GPU is needed.  EINVAL for bad sizes or arguments
 * (n must equal N_p for L1 x L2 at bond dimension D). */
int peps_su_theta(int L1, int L2, int D, double J1, double tau, int n_steps, double* theta,
                  size_t n);

/* The same simple-update warm start run on the device into the context: theta becomes the
 * simple-update state after n_steps steps of length tau from beta = 0 (App. A; the bond
 * update described at peps_su_theta, nearest-neighbour bonds with coupling J1), and the
 * context's imaginary time becomes t = n_steps * tau (beta_obs = 4t), from which SR steps
 * continue.  In each half of a step (horizontal bonds, then vertical bonds) every row (or
 * column) is one thread block that takes its bonds in order; lines share no site or
 * changing weight, so this is the host scheme's order, and the state equals peps_su_theta's
 * up to the summation order of the factorisations (bonds whose truncation cuts through a
 * degenerate spectrum may keep a different, equally valid, subspace).  Allocates and frees
 * its own work arrays (at D = 4 about 0.5 MB per block); synchronises the context stream.
 * EINVAL for bad arguments or J2 != 0; ENOMEM, ECUDA on device failures. */
int peps_su_warm_start(peps_ctx* ctx, double tau, int n_steps);

/* Specific heat per site from an energy curve (Sec. III.A: C_v from the derivative of a
 * spline through E against beta): fits a natural cubic smoothing spline to the n points
 * (beta[k], E_site[k]) (any order, distinct beta, n >= 3) whose residual sum of squares is at
 * most `smoothing` (0 interpolates; with independent errors sigma per point, n sigma^2 is the
 * usual choice) and writes C/N = -beta^2 dE/dbeta of the spline at the m points beta_eval to
 * cv (caller-owned).  Host code; no context or GPU is needed.  EINVAL for bad arguments. */
int peps_cv_spline(const double* beta, const double* E_site, int n, double smoothing,
                   const double* beta_eval, double* cv, int m);

/* Per-kernel statistics for roofline reports.  peps_profile(ctx, 1) clears them and starts
 * bracketing every launch of the context with CUDA events on its stream; peps_profile(ctx,
 * 2) does the same for the batched GEMM kernels only (kb_gemm_tc, kb_gemm: fewer events in
 * the stream); peps_profile(ctx, 0) stops.  peps_profile_read synchronises the stream and
 * returns, per kernel name, the launches, the summed event time and the algorithmic bytes
 * (each operand read once, each result written once) and flops of those launches (for the
 * truncation kernel kb_trunc: the flops of the Jacobi sweeps its matrices took, counted on
 * the device, 6 nc (nc - 1) len per sweep of an nc-column matrix of column length len, plus
 * 3 nc (nc - 1) m when its m x m right vectors are accumulated); up to
 * `cap` entries are written to `out` (caller-owned) and the number of kernels to *n_out.
 * EINVAL on bad arguments. */
typedef struct {
  char name[32];
  long long launches;
  double ms;
  double bytes;
  double flops;
} peps_kernel_stat;
int peps_profile(peps_ctx* ctx, int enable);
int peps_profile_read(peps_ctx* ctx, peps_kernel_stat* out, int cap, int* n_out);
/* The same timing for a fermionic evaluator's launches (peps_famp_*), and the number of
 * kernels it has launched. */
int peps_famp_profile(peps_famp* famp, int enable);
int peps_famp_profile_read(peps_famp* famp, peps_kernel_stat* out, int cap, int* n_out);
long long peps_famp_launches(const peps_famp* famp);
/* The algorithmic bytes of each launch of kernel `name` recorded since profiling started or
 * since the last peps_profile_read (which folds the records into its sums), in launch order:
 * the first `cap` go to `bytes` (caller-owned), their number to *n_out.  Lets a per-launch
 * DRAM capture of a profiler be set against the same launches.  EINVAL on bad arguments. */
int peps_profile_launch_bytes(peps_ctx* ctx, const char* name, double* bytes, int cap, int* n_out);

/* Failure-detection self-test of the bounded waits in the tensor-core kernels (the paper
 * has no counterpart).  Launches a small contraction on its own stream with its MMAs
 * withheld, so its completion barrier never fires: the kernel's waits give up after their
 * time limit (1 s each, about 2 s in all), it frees its tensor memory and raises its error
 * flag; then a normal contraction on the same stream is checked against a host product.
 * Returns PEPS_OK when both happen, PEPS_ESTATE if the withheld MMAs went unnoticed,
 * PEPS_ETIMEOUT if the normal contraction timed out, PEPS_ENOTFINITE if its result is
 * wrong, PEPS_ENOMEM / PEPS_ECUDA on allocation or CUDA errors.  Allocates and frees its
 * own small buffers. */
int peps_selftest_tc_timeout(void);

/* ---------------------------------------------------------------- serving loop
 *
 * Continuous batching of cooling runs.  Requests are queued by peps_srv_submit (any host
 * thread) and admitted in arrival order while the sum of the admitted contexts'
 * footprints stays within the budget and fewer than max_active run.  Every admitted
 * request gets its own context and CUDA stream and a host worker that runs its steps, so
 * the work of concurrent requests overlaps on the device; when a request finishes its
 * memory is released and the next queued requests are admitted.  A request's results do
 * not depend on what else runs (its own random stream, fixed reduction orders), so a
 * request gives the same bits alone and in a mix. */
typedef struct peps_server peps_server;

typedef struct {
  peps_params params;  /* problem; params.n_chains = samples per SR step */
  double tau;          /* imaginary-time step */
  double t_end;        /* run until t >= t_end (beta_obs = 4 t_end) */
  double eps, cg_tol;  /* SR shift and CG relative tolerance */
  int max_cg;          /* CG iteration cap */
  int n_sweeps;        /* Metropolis sweeps per step */
  int n_burn;          /* burn-in sweeps before the first step */
  double p1_until_beta; /* reweighted sampling (p = 1) while beta_obs < this */
} peps_request;

#define PEPS_REQ_QUEUED 0
#define PEPS_REQ_RUNNING 1
#define PEPS_REQ_DONE 2
#define PEPS_REQ_FAILED 3
#define PEPS_REQ_CANCELLED 4 /* ended by peps_srv_stop: queued, or after its last finished step */

/* Creates a server.  hbm_budget: device bytes available to admitted requests (0 = 80% of
 * the free memory); max_active: concurrently running requests (>= 1); blocks_per_request:
 * persistent sample blocks per request (0 = the device's 4 x SMs divided by max_active). */
int peps_srv_create(size_t hbm_budget, int max_active, int blocks_per_request, peps_server** out);
/* Queues a request; *req_id receives its id.  PEPS_EINVAL for invalid parameters or a
 * footprint above the whole budget. */
int peps_srv_submit(peps_server* srv, const peps_request* req, int* req_id);
/* State of a request (PEPS_REQ_*), steps done so far, and up to cap per-step statistics
 * (observables of each step's samples, as from peps_sr_step). */
int peps_srv_poll(peps_server* srv, int req_id, int* state, int* n_steps, peps_stats* per_step,
                  int cap);
/* Final parameter vector of a finished request (host buffer of N_p doubles). */
int peps_srv_theta(peps_server* srv, int req_id, double* host, size_t n);
/* Blocks until every submitted request has finished. */
int peps_srv_drain(peps_server* srv);
/* Ends the serving run: requests still queued are cancelled, running ones end after the step
 * they are in (PEPS_REQ_CANCELLED; their finished steps stay in the statistics and metrics),
 * and later submissions return PEPS_ESTATE.  Returns at once; peps_srv_drain then waits for
 * the running steps.  Bounds a measurement under a stream whose requests would outlast it. */
int peps_srv_stop(peps_server* srv);
/* Step latency over all finished steps (ms, p50 and p99), aggregate samples/s between the
 * first admission and the last finished step, and the number of steps measured. */
int peps_srv_metrics(peps_server* srv, double* p50_ms, double* p99_ms, double* samples_per_s,
                     int64_t* n_steps);
/* Waits for running requests, then releases the server (NULL is ignored). */
void peps_srv_free(peps_server* srv);

/* Evaluation without any device allocation.
 *
 * For callers that must not allocate GPU memory themselves or through this library: code
 * running inside a host framework that owns the whole device memory pool, a plug-in that is
 * called while a CUDA graph is being captured, or a process whose memory budget is fixed
 * at start-up.  The paper has no counterpart; this is a library convenience.
 *
 * Configuration entries must lie in 0..3.  A sample holding an entry outside that range is
 * not evaluated (the kernel checks before it reads any parameter): its log_abs, e_sys and
 * e_anc are NaN, its sign 0, and its O row is left as it was.
 *
 * Same results as peps_eval_batch on device pointers (the same kernel runs), for the
 * problem in *params (n_chains, seed, init_noise, n_blocks and block_mode are ignored; the
 * narrow block layout is used): theta (float64
 * [N_p]), S (uint8 [nb][L1*L2]) and every non-null output are DEVICE pointers owned by the
 * caller.  The per-block work space comes from one file-scope device array of
 * PEPS_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until the process
 * exits; no cudaMalloc, cudaFree or other allocating call is made.  The number of thread
 * blocks is chosen so that their work space fits; a problem whose single block does not
 * fit returns PEPS_EINVAL (message in peps_last_error(NULL)).
 *
 * The first call on a device, with that device current, performs a one-time set-up
 * (looks up the array's device address and sets the kernel's shared-memory attribute);
 * make that first call before any stream capture.  All calls share the array and it keeps
 * the last call's contents: calls that may overlap on the GPU (different streams, or
 * several host threads) race and must be serialised by the caller.  The call enqueues its
 * work on `stream` (cudaStream_t as void*, NULL = legacy default stream) and returns
 * without waiting for it. */
#define PEPS_NOALLOC_SCRATCH_BYTES (48u * 1024u * 1024u)
int peps_eval_batch_noalloc(const peps_params* params, const double* theta, const uint8_t* S,
                            int nb, double* log_abs, int8_t* sign, double* e_sys,
                            double* e_anc, void* O, void* stream);

/* Releases every device buffer of the context (NULL is ignored). */
void peps_free(peps_ctx* ctx);

/* Message of the last error on this context ("" when none); with ctx == NULL, the message
 * of the calling thread's last failed peps_eval_batch_noalloc. */
const char* peps_last_error(const peps_ctx* ctx);

/* Library version string. */
const char* peps_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PEPS_VMC_H */

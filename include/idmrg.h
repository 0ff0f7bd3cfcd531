/*
 * libidmrg -- parallel infinite-size DMRG (Hida's iDMRG for l-site unit cells
 * with a variant of McCulloch's wavefunction prediction) on one GB300 GPU.
 *
 * Problem statement (Ueda, Sec. 3): a Hamiltonian with an l-site period,
 * given as the matrix product operator W_1 .. W_l of Eq. mpo2, and the number
 * m of block states kept.  One parallel iteration n (a "unit-cell step")
 * solves the l/2 superblocks H^(n)_i = L^(n-1)_{2i-1} W W R^(n-1)_{2i+2}
 * (Step 2'), starting from the predicted wavefunction of Eq. wfprediction
 * (Step 3'), splits each ground state by SVD (Step 4), renormalises the
 * blocks (Step 6) and estimates the energy per site (Step 5').  Between
 * steps, the uniform MPS of Eq. mps2 built from the last two iterations gives
 * two-point functions and the transfer spectrum (idmrg_correlation,
 * idmrg_transfer_spectrum).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Superblocks are numbered p = 0 .. l/2-1 (the paper's i = p+1); p = -1
 *    means "all superblocks" wherever it is accepted.  Sites are 0-based.
 *  - Charges are integers 2 S^z.
 *  - Device pointers are borrowed for the duration of the stream-ordered call;
 *    host pointers are read or written before the call returns.
 *  - Every call returns an idmrg_status and never aborts or throws.  Out
 *    parameters are written only on IDMRG_OK, except IDMRG_ENOCONV, which
 *    still writes the best estimate.  idmrg_last_error() gives a message.
 *  - The library allocates device memory only through the idmrg_allocator
 *    given to idmrg_create (cudaMalloc when none is given), and only between
 *    kernels of a step, never inside a captured region.
 */
#ifndef IDMRG_H
#define IDMRG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IDMRG_OK = 0,
  IDMRG_EINVAL = 1,   /* bad argument or invalid MPO                         */
  IDMRG_ENOMEM = 2,   /* the allocator returned NULL                         */
  IDMRG_ECUDA = 3,    /* a CUDA runtime call failed                           */
  IDMRG_ENOCONV = 4,  /* Lanczos hit lanczos_maxit; best estimate written    */
  IDMRG_ETIMEOUT = 5, /* a device-side wait ran out of its iteration budget  */
  IDMRG_ENUMERIC = 6, /* NaN/Inf in a Lanczos coefficient, or SVD failure    */
  IDMRG_ESTATE = 7    /* calls made in the wrong order for this iteration    */
} idmrg_status;

/* Arithmetic of the H_eff psi and environment contractions.  The Lanczos
 * recurrence, re-orthogonalisation and tridiagonal eigensolve are FP64 in
 * every mode, and the SVD is FP64-accurate in every mode: it preconditions
 * in FP32 and finishes with FP64 sweeps, whose element arithmetic on large
 * sectors is FP32 pairs in TF32X3 and BF16X3 (idmrg_set_jacobi_arithmetic). */
typedef enum {
  IDMRG_FP64 = 0,    /* FP64 everywhere                                       */
  IDMRG_TF32X3 = 1,  /* tensor cores, TF32 split (hi/lo) operands, three
                        products per term, FP32 accumulation; energies refined
                        by an FP64 Rayleigh quotient                          */
  IDMRG_BF16X3 = 2,  /* as TF32X3 with BF16 splits (kind::f16 MMAs, ~16 bits
                        per product, twice the K per instruction)             */
  IDMRG_FP64_TC = 3  /* FP64-accurate H_eff psi on the tensor cores from BF16
                        digit slices (see idmrg_heff_apply_fp64, form 1); one
                        Lanczos run as in IDMRG_FP64; environments, prediction
                        and SVD in FP64                                       */
} idmrg_precision;

/* The MPO of one period (Sec. 2, Eq. mpo; Sec. 3, Eq. mpo2).  Host memory,
 * caller-owned, copied by idmrg_create.  Site k (0-based) holds
 * W_k[a][b][s][t] = <s| W_k(a,b) |t>, a < bond_dim[k], b < bond_dim[k+1],
 * stored row-major and concatenated site after site.  Channel 0 of every bond
 * is "term completed" and the last channel "identity": W_k(0,0) and
 * W_k(last,last) are the unit matrix, row 0 and the last column hold nothing
 * else (lower-triangular form; L_k is the last row and R_k the first column of
 * W_k).  bond_charge holds the 2Sz carried by each channel, bond by bond
 * (bond k = the bond to the left of site k, bond_dim[k] entries).  A non-zero
 * W_k(a,b) entry <s|.|t> must satisfy
 *   phys_charge[s] - phys_charge[t] == charge(bond k+1, b) - charge(bond k, a).
 * Violations return IDMRG_EINVAL. */
typedef struct {
  int ell;                  /* period l, even, >= 2                           */
  int d;                    /* local dimension                                */
  const int *bond_dim;      /* l+1 entries, bond_dim[l] == bond_dim[0]       */
  const double *W;          /* sum_k a_k a_{k+1} d^2 doubles                 */
  const int *phys_charge;   /* d entries                                      */
  const int *bond_charge;   /* sum_{k<l} a_k entries                          */
} idmrg_mpo;

typedef struct {
  int m;                    /* kept states per block (Step 6)                 */
  int target_charge;        /* 2Sz of every superblock ground state (0)       */
  double lanczos_tol;       /* stop when |b_k y_k| <= tol max(1,|theta|)      */
  int lanczos_maxit;        /* Krylov dimension cap, 2..600 (sizes memory)    */
  idmrg_precision prec;
  int predict;              /* 1: Eq. wfprediction for n >= 3; 0: random      */
  uint64_t seed;            /* SplitMix64 seed of the random start vectors    */
  double lambda_zero_rel;   /* lambda <= this * lambda_max counts as zero     */
  double tie_rel;           /* never cut between lambda_k, lambda_k+1 closer
                               than this relative gap (multiplets stay whole) */
} idmrg_opts;

/* Device memory provider.  alloc returns a device pointer aligned to at least
 * 256 bytes or NULL; free releases it (bytes is the size asked for). */
typedef struct {
  void *(*alloc)(size_t bytes, void *user);
  void (*free)(void *ptr, size_t bytes, void *user);
  void *user;
} idmrg_allocator;

/* Per-iteration report.  Every array is caller-owned host memory of l/2
 * entries and may be NULL. */
typedef struct {
  int n;                    /* the iteration just completed                   */
  double *energy;           /* e^(n)_i, Step 3 (FP64-refined in mixed modes)  */
  int *iters;               /* Lanczos matvecs                                */
  double *eps;              /* Eq. tru, truncation error                      */
  double *eps_best;         /* Eq. fid2, best fidelity error                  */
  double *fidelity;         /* Eq. fid1 (NaN when no prediction was used)     */
  double *bond;             /* <psi| h(c1,c2) |psi>, centre-bond energy       */
  int *kept;                /* states kept                                    */
  double e_g;               /* Step 5' estimate, NaN unless (n+1) mod l == 0  */
} idmrg_step_report;

typedef struct idmrg_ctx idmrg_ctx;

/* Defaults: m = 64, target 0, tol 1e-12, maxit 300, FP64, prediction on,
 * seed 0, lambda_zero_rel 1e-12, tie_rel 1e-7 (states degenerate by symmetry
 * come out of a solver stopped at residual tol|E| split by ~tol|E|/gap; a
 * tie_rel below that would let rounding decide the cut). */
void idmrg_default_opts(idmrg_opts *opts);

/* Step 1: validates the MPO, builds L^(0) (last row of W at site 2p) and
 * R^(0) (first column of W at site 2p+1) for every pair and sets n = 1.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream) on which every
 * later call is ordered.  alloc may be NULL (cudaMalloc/cudaFree). */
idmrg_status idmrg_create(const idmrg_mpo *mpo, const idmrg_opts *opts, void *cuda_stream,
                          const idmrg_allocator *alloc, idmrg_ctx **out);

/* One context over nmpo independent problems (e.g. disorder realisations
 * of Sec. 3's random-bond chains), all with the same local basis (d and
 * phys_charge) but each with its own unit cell length l_r, couplings, and
 * kept states m_per[r] (NULL: opts->m for all).  The problems are "rings":
 * superblock q of problem r is superblock p0_r + q of the context, p0_r =
 * sum_{r' < r} l_r'/2, and its pairs close on themselves (Step 2': the
 * ring's last pair takes its right block from the ring's first).  Every
 * call covers the superblocks of all problems, so each kernel launch (and
 * each CUDA graph of a Lanczos iteration) serves all of them together;
 * start vectors are drawn per problem exactly as in a context of its own.
 * Step reports list every superblock in this order; their e_g is problem
 * 0's, idmrg_ring_energy reads any problem's.  opts->m becomes the largest
 * m.  Checkpoints, observables, pair ranges, idmrg_run and
 * idmrg_truncation_error need a context of one problem (EINVAL).  EINVAL
 * for nmpo < 1, a differing d or phys_charge, or an m_per below 1; each MPO
 * is checked as by idmrg_create. */
idmrg_status idmrg_create_batch(const idmrg_mpo *mpos, int nmpo, const int *m_per, const idmrg_opts *opts,
                                void *cuda_stream, const idmrg_allocator *alloc, idmrg_ctx **out);
void idmrg_destroy(idmrg_ctx *ctx);
const char *idmrg_last_error(const idmrg_ctx *ctx);
idmrg_status idmrg_set_stream(idmrg_ctx *ctx, void *cuda_stream);

/* Current iteration n (the one the next unit-cell step performs). */
idmrg_status idmrg_iteration(const idmrg_ctx *ctx, int *n);

/* Layout of superblock p's wavefunction at the current iteration (Step 3):
 * psi[x][s][t][y] for left block state x, sites c1 (s) and c2 (t), right block
 * state y, stored as dense sub-blocks of fixed (left sector, s, t); only
 * sub-blocks whose charges add up to target_charge exist.  Each sub-block is
 * described by 8 ints:
 *   {x0, Dx, s, t, y0, Dy, offset, row_stride}
 * x0/y0 = first basis index of the left/right sector, Dx/Dy its size, element
 * (x0+i, s, t, y0+j) at offset + i*row_stride + j.  *nelem = vector length. */
idmrg_status idmrg_psi_layout(const idmrg_ctx *ctx, int p, int *desc, int cap_blocks,
                              int *nblocks, size_t *nelem);

/* Basis of a block of superblock p at the current iteration: side 0 = left
 * block L^(n-1) of pair p, side 1 = right block R^(n-1) of pair p+1.  Writes
 * the 2Sz of each state (dense basis order), its MPO channel count and size. */
idmrg_status idmrg_block_basis(const idmrg_ctx *ctx, int p, int side, int *charges, int cap,
                               int *dim, int *channels);

/* Copies that block's operators to host memory as dense [channels][D][D]
 * (<x| O_a |y>, zeros outside its charge blocks), in FP64. */
idmrg_status idmrg_block_to_host(const idmrg_ctx *ctx, int p, int side, double *host, size_t cap);

/* Step 3 matvec: out = H^(n)_p psi with H = L W_{c1} W_{c2} R, both device
 * vectors in the idmrg_psi_layout of p (p >= 0), or all superblocks' vectors
 * concatenated in order p = 0 .. l/2-1 (p = -1).  Uses the arithmetic of
 * opts.prec.  Valid from idmrg_create / idmrg_advance until the next
 * idmrg_advance. */
idmrg_status idmrg_heff_apply(idmrg_ctx *ctx, int p, const double *psi_dev, double *out_dev);

/* The same product in one of the FP64-accurate forms, whatever opts.prec:
 * form 0 = FP64 GEMMs on the CUDA cores; form 1 = BF16 digit slices on the
 * tensor cores (the Ozaki scheme: eight 7-bit digits per element against a
 * per-row power of two, exact integer sums per digit level over K chunks of
 * at most 768, levels and chunks summed in FP64).  Form 1 exists in
 * TF32X3 / BF16X3 contexts (whose Lanczos restarts use it for their FP64
 * matvecs) and in FP64_TC contexts (every matvec); otherwise
 * IDMRG_EINVAL. */
idmrg_status idmrg_heff_apply_fp64(idmrg_ctx *ctx, int p, const double *psi_dev, double *out_dev, int form);

/* Step 3': start vector of superblock p (or all): Eq. wfprediction for
 * n >= 3 when opts.predict, else SplitMix64 numbers in [-1,1) on the target
 * sector.  Writes ||psi~|| if norm_out != NULL (host, l/2 entries for p=-1). */
idmrg_status idmrg_predict_wavefunction(idmrg_ctx *ctx, int p, double *norm_out);

/* Step 3 start vector given by the caller instead of Step 3': copies psi_dev
 * (device, the idmrg_psi_layout of p, or every superblock's vector
 * concatenated for p = -1) into the start vector of the next
 * idmrg_lanczos_solve, which normalises it.  Allowed before that solve
 * (after, or in place of, idmrg_predict_wavefunction); ESTATE otherwise.  A
 * start vector with zero or non-finite norm makes the solve return
 * IDMRG_ENUMERIC.  The step report's fidelity (Eq. fid1) then refers to this
 * vector. */
idmrg_status idmrg_set_start_vector(idmrg_ctx *ctx, int p, const double *psi_dev);

/* Step 3 solve by FP64 Lanczos with full re-orthogonalisation.  All
 * requested superblocks are solved together, matvecs batched.  e_out and
 * iters_out: host, one entry (p >= 0) or l/2 entries (p = -1). */
idmrg_status idmrg_lanczos_solve(idmrg_ctx *ctx, int p, double *e_out, int *iters_out);

/* Copies the Lanczos ground state of superblock p to host (layout as above). */
idmrg_status idmrg_get_psi(const idmrg_ctx *ctx, int p, double *host, size_t cap);

/* Step 4 + truncation of Step 6: FP64-accurate SVD per charge sector (the
 * arithmetic is described at idmrg_precision), descending
 * singular values, cut at <= m without splitting near-equal values.  Host
 * outputs (one or l/2 entries, each may be NULL): eps (Eq. tru), eps_best
 * (Eq. fid2), states kept. */
idmrg_status idmrg_truncate(idmrg_ctx *ctx, int p, double *eps_out, double *eps_best_out,
                            int *kept_out);

/* All singular values of superblock p's last truncation, descending. */
idmrg_status idmrg_get_lambda(const idmrg_ctx *ctx, int p, double *host, int cap, int *len);

/* Step 6: L^(n) = u^T (L^(n-1) W_{c1}) u and R^(n) = v^T (W_{c2} R^(n-1)) v
 * (Eqs. L, R) for pair p (or all). */
idmrg_status idmrg_update_environments(idmrg_ctx *ctx, int p);

/* Step 7 with the rotation of Step 2': R^(n) of pair p+1 becomes the right
 * block of superblock p; n -> n+1.  Requires every pair to be updated. */
idmrg_status idmrg_advance(idmrg_ctx *ctx);

/* One parallel iteration: predict, solve, truncate, update, advance, for all
 * superblocks.  rep may be NULL. */
idmrg_status idmrg_unit_cell_step(idmrg_ctx *ctx, idmrg_step_report *rep);

/* One unit-cell step of each of n independent contexts (for instance disorder
 * realisations of different unit cells and m), run concurrently by `threads`
 * host threads; every context must have been created on its own stream, so
 * that their kernels overlap on the GPU.  A context's results are those of
 * idmrg_unit_cell_step on it alone.  reps (nullable) holds n reports.
 * Returns the first status other than IDMRG_OK in context order (every
 * context is stepped regardless). */
idmrg_status idmrg_batch_step(idmrg_ctx *const *ctxs, int n, int threads, idmrg_step_report *reps);

/* ---- One problem over several workers (Sec. 3, Step 2').  The l/2
 * superblocks of an iteration are independent; consecutive iterations are
 * coupled only through the rotation of Step 2' (superblock p at n + 1 takes
 * R^(n) of pair p + 1) and the prediction of Step 3' (U^(n), lambda^(n) and
 * lambda^(n-1) of pair p + 1).  A worker that owns the contiguous pairs
 * p0 .. p1-1 therefore needs, after every iteration, only pair p1's data
 * (pair 0 after the last pair), which the next worker exports.
 *
 * idmrg_set_pair_range: from the next step on, this context steps only the
 * superblocks p0 .. p1-1 (all calls with p = -1 act on them; other p are
 * EINVAL).  Between steps; ESTATE during a step.  Every worker creates its
 * context with the whole MPO and the same options.
 *
 * idmrg_export_pair: after a step, pair q's R^(n) and the truncation of its
 * superblock (U, V, lambda, bases) in a host byte buffer (the checkpoint's
 * layout for one pair).  *len = bytes needed; the data is written when host
 * is not NULL and cap >= *len (EINVAL otherwise).  q must be in the range.
 *
 * idmrg_import_pair: after a step of a context with a partial range, the
 * data of pair p1 mod l/2 exported by its owner after the same iteration;
 * the context then plans the next iteration (until the import, stepping calls
 * return ESTATE).  EINVAL for another pair or iteration.
 *
 * Energies per site (Step 5') and the truncation error of a run are kept by
 * the context that owns pair 0.  idmrg_save / idmrg_load and the observables
 * need the whole unit cell (ESTATE otherwise). */
idmrg_status idmrg_set_pair_range(idmrg_ctx *ctx, int p0, int p1);
idmrg_status idmrg_export_pair(const idmrg_ctx *ctx, int q, void *host, size_t cap, size_t *len);
idmrg_status idmrg_import_pair(idmrg_ctx *ctx, int q, const void *host, size_t len);

/* Truncation error of the run (Sec. 4.4, Eq. tru): the largest eps^(n)_1 over
 * the last l iterations (one period).  ESTATE before the first step. */
idmrg_status idmrg_truncation_error(const idmrg_ctx *ctx, double *eps);

/* Unit-cell steps until two successive estimates of e_g (Step 5', one every
 * l iterations) differ by less than de_tol, or max_steps steps.  Writes the
 * last e_g, the truncation error and the steps taken (each nullable);
 * IDMRG_ENOCONV when max_steps ran out first.  One point of the m scan of
 * Sec. 4.4 (e_g against eps for several m, extrapolated to eps -> 0). */
idmrg_status idmrg_run(idmrg_ctx *ctx, int max_steps, double de_tol, double *e_g, double *eps, int *steps);

/* ---- Uniform-MPS observables (Sec. 3, Eq. mps2; the bond strengths,
 * spin-spin correlations and correlation length of the paper's benchmarks).
 * After iteration n the unit of Eq. mps2 is V^(n)_1^T u~^(n)_2 V^(n)_2^T ...
 * u~^(n)_1, u~^(n)_{i+1} = (lam^(n-1)_{i+1})^-1 u^(n)_{i+1} lam^(n)_{i+1} (the
 * scaled tensors of Eq. wfprediction, same zero rule), repeated along the
 * infinite chain.  Expectation values use the dominant left and right
 * eigenvectors of the unit's transfer map (power iteration to 1e-12), since
 * the unit is only approximately right-normalised before convergence.  Both
 * calls need two completed iterations (ESTATE before, or during a step); the
 * unit and its fixed points are kept until the next step or load.  Lattice
 * sites are numbered along the chain: site x carries MPO site x mod l. */

/* out[k] = sum_t coef[t] < (op_a[t])_{site_i[k]} (op_b[t])_{site_j[k]} > for
 * k < npairs.  op_a, op_b: nterms host matrices d x d, row-major,
 * op[s * d + t] = <s| O |t> in the MPO's physical basis; coef: nterms host
 * values; site_i, site_j, out: npairs host values with
 * 0 <= site_i[k] < site_j[k] <= site_i[k] + 2^20.  For spin 1/2,
 * <s_i . s_j> is the three terms (Sz, Sz, 1), (S+, S-, 1/2), (S-, S+, 1/2).
 * EINVAL on bad arguments, ENOCONV if the fixed points do not converge. */
idmrg_status idmrg_correlation(idmrg_ctx *ctx, int nterms, const double *op_a, const double *op_b,
                               const double *coef, int npairs, const int64_t *site_i, const int64_t *site_j,
                               double *out);

/* Two largest eigenvalue moduli of the unit's transfer map, t1 (its dominant,
 * positive eigenvalue) and |t2|, and the correlation length
 * xi = -1 / ln(|t2| / t1) in unit cells (0 when |t2| = 0).  The map keeps
 * the U(1) charge difference of an environment's entries; |t2| is the largest
 * over the sectors of charge difference 0 (deflated of the fixed point), one
 * and two steps of the smallest difference present at bond 0, each from a
 * subspace iteration with two vectors stopped when its estimate changes by at
 * most tol (relative) three times in a row, or after maxit iterations
 * (ENOCONV, estimate written).  Each output pointer may be NULL. */
idmrg_status idmrg_transfer_spectrum(idmrg_ctx *ctx, double tol, int maxit, double *t1, double *t2_abs,
                                     double *xi, int *iters);

/* ---- Host post-processing of Secs. 4.4-4.6 (no context, no device work). */

/* Eqs. diff1, diff2 over n values the lattice makes equivalent (the bond
 * strengths of one kind): their average, Delta+ = max - average and
 * Delta- = min - average.  EINVAL for n < 1 or a non-finite value; each
 * output pointer may be NULL. */
idmrg_status idmrg_delta_pm(const double *values, int n, double *avg, double *dplus, double *dminus);

/* Least-squares polynomial of the given degree (0..6) through the n points
 * (eps_k, value_k), by Householder QR; *v0 = its value at eps = 0 (the eps -> 0
 * extrapolation of Sec. 4.4, degree 2 for the energy), *sd its standard
 * deviation s sqrt([(A^T A)^-1]_00), s^2 = RSS / (n - degree - 1) (0 when
 * n = degree + 1).  EINVAL for too few points or a singular design. */
idmrg_status idmrg_extrapolate(const double *eps, const double *value, int n, int degree, double *v0, double *sd);

/* Correlation length of Sec. 4.6: least-squares line ln|c_k| = a + b r_k over
 * the points with r_k > r_min and c_k != 0; *xi = -1/b and its standard
 * deviation sd(b) / b^2 (0 with two points).  EINVAL with fewer than two
 * such points or b = 0. */
idmrg_status idmrg_fit_correlation_length(const double *r, const double *c, int n, double r_min, double *xi,
                                          double *sd);

/* Step 5': latest e_g = (e^(n)_1 - e^(n-l)_1) / 2l with (n+1) mod l == 0
 * (e^(-1)_1 = 0) and the n it belongs to; ESTATE if there is none yet. */
idmrg_status idmrg_energy_per_site(const idmrg_ctx *ctx, double *e_g, int *n_of_estimate);

/* The same for problem r of a context made by idmrg_create_batch (its own
 * unit cell length l_r); EINVAL for r outside the problems. */
idmrg_status idmrg_ring_energy(const idmrg_ctx *ctx, int r, double *e_g, int *n_of_estimate);

/* Checkpoint between unit-cell steps (Step 7): the iteration n, the history
 * of e^(n)_1 behind Step 5', every pair's current environments (Step 6) and
 * the last two truncations (bases, U, V, lambda) that the prediction of
 * Step 3' reads.  idmrg_save writes them to `path` (binary, host byte order);
 * idmrg_load reads them into a context created with the same MPO, m and
 * target charge (checked: EINVAL otherwise), which then continues exactly as
 * the saved one would when its other options are the same too.  Every
 * precision keeps this state in FP64, so a state saved under one precision
 * loads into a context of another (the file records the saving one).  Both
 * synchronise the context's stream; ESTATE while a step is in progress;
 * EINVAL on I/O errors or a damaged file. */
idmrg_status idmrg_save(const idmrg_ctx *ctx, const char *path);
idmrg_status idmrg_load(idmrg_ctx *ctx, const char *path);

/* Measured work of the last heff_apply call: algorithmic flops (sum over
 * GEMM tasks of 2 M N K plus 2 per element per two-site MPO term) and the
 * bytes of L, R, psi in and out. */
idmrg_status idmrg_heff_cost(const idmrg_ctx *ctx, int p, double *flops, double *bytes);

/* Kernel launches this context has issued so far (for accounting). */
idmrg_status idmrg_launch_count(const idmrg_ctx *ctx, uint64_t *count);

/* Device timers per kernel class: when enabled, every launch of the class is
 * bracketed by CUDA events on the context's stream; idmrg_profile_read
 * synchronises and returns the summed device time, the number of launches and
 * the algorithmic flops and bytes of those launches (flops: 2 M N K per GEMM
 * task of the superblocks that were active, 2 per element per MPO term; for
 * the SVD class the R-SVD count 6 r c^2 + 20 c^3 per r x c sector matrix;
 * bytes: operands read once and results written once).  Enabling resets. */
typedef enum {
  IDMRG_K_HEFF_GEMM = 0,   /* H_eff psi stages L.psi and T3.R^T (Step 3)       */
  IDMRG_K_HEFF_WSTAGE = 1, /* H_eff psi two-site MPO stage (Step 3)            */
  IDMRG_K_LANCZOS_VEC = 2, /* Gram-Schmidt projections and updates (Step 3)   */
  IDMRG_K_LANCZOS_TRI = 3, /* tridiagonal eigensolve and convergence (Step 3) */
  IDMRG_K_SVD = 4,         /* sector SVD, selection, compaction (Step 4)       */
  IDMRG_K_ENV = 5,         /* block-spin transformation (Step 6)               */
  IDMRG_K_PREDICT = 6,     /* start vectors (Step 3')                          */
  IDMRG_K_HEFF_F64 = 7,    /* mixed precision only: the FP64-accurate H_eff
                              psi GEMM stages that start every Lanczos restart
                              (the true-residual checks); FP64 and FP64_TC
                              book theirs under IDMRG_K_HEFF_GEMM             */
  IDMRG_K_COUNT = 8
} idmrg_kernel_class;
idmrg_status idmrg_profile_enable(idmrg_ctx *ctx, int on);
idmrg_status idmrg_profile_read(idmrg_ctx *ctx, int kclass, double *ms, uint64_t *launches, double *flops,
                                double *bytes);

/* Sector SVDs of the following truncations on the kernels for large sector
 * matrices only (global_only = 1: pivoted QR on thread-block clusters with
 * the columns in global memory, FP32 and FP64 cyclic Jacobi in global
 * memory), or on the size-dependent choice (0, the
 * default: sectors with at most 320 columns use the shared-memory block
 * kernels).  The results agree to rounding; this exists to test the
 * large-sector path on small problems. */
idmrg_status idmrg_set_svd_path(idmrg_ctx *ctx, int global_only);

/* Arithmetic of the final (FP64-accuracy) one-sided Jacobi of the sector
 * SVDs of Step 4 on the large-sector path (sectors beyond 320 columns, or
 * every sector under idmrg_set_svd_path(ctx, 1)): mode 1 = FP64 on the FP64
 * units; mode 2 = pairs of FP32 numbers (48 significant bits: exact
 * products by FMA, exact sums by two-sum) for the dot products and column
 * rotations, FP64 for column norms, scales and rotation scalars -- GB300
 * issues 64 FP32 FMAs per FP64 FMA; the singular values stay within 1e-10
 * of an FP64 SVD's (tested at m = 2048); mode 0 (the default) = mode 2 for the
 * mixed precisions (TF32X3, BF16X3), mode 1 for FP64 and FP64_TC.  Takes
 * effect at the next truncation; EINVAL for another mode. */
idmrg_status idmrg_set_jacobi_arithmetic(idmrg_ctx *ctx, int mode);

/* Shape of the last truncation's SVD work (Step 4): sector matrices, their
 * largest short side, largest numerical rank, and the Jacobi sweeps taken
 * (maximum and mean over the sectors). */
idmrg_status idmrg_svd_stats(const idmrg_ctx *ctx, int *jobs, int *max_cols, int *max_rank, int *max_sweeps,
                             double *mean_sweeps);

/* Sweeps of the FP32 Jacobi stage of the last truncation's sector SVDs
 * (those of rank 2 or more): the largest and the mean. */
idmrg_status idmrg_svd_sweeps32(const idmrg_ctx *ctx, int *max_sweeps, double *mean_sweeps);

/* Milliseconds spent, since profiling was last enabled, in the phases of the
 * sector SVD of Step 4 (parts of IDMRG_K_SVD, event-timed on the context's
 * stream): ms[0] gather and pivoted QR, ms[1] FP32 Jacobi, ms[2]
 * Newton-Schulz orthogonalisation and X = B V, ms[3] FP64 Jacobi, ms[4]
 * selection of the kept states, ms[5] compaction into U and V.  ms holds 6
 * entries. */
idmrg_status idmrg_svd_phase_ms(idmrg_ctx *ctx, double *ms);

/* The N tile of the split-operand tensor-core GEMMs of H_eff psi (Sec. 3,
 * Step 3; mixed precisions only) that the context's tuner chose for stage 1
 * (stage = 1: L psi) or stage 3 (stage = 3: T3 R^T).  The tuner times 64-,
 * 128- and 256-column tiles on the plan's own task list whenever the stage's
 * work has moved by more than 10 % since it last ran, and keeps the fastest.
 * tn (may be NULL): 64, 128 or 256, 0 before the first mixed plan; ms (may
 * be NULL, 3 entries): each candidate's timed run at the last tuning, in
 * milliseconds; tunings (may be NULL): tuning passes of this context (both
 * stages counted).  EINVAL for another stage number. */
idmrg_status idmrg_gemm_tuning(const idmrg_ctx *ctx, int stage, int *tn, float *ms, int *tunings);

/* Mixed precisions (TF32X3, BF16X3): Step 3's Lanczos runs as restarts, each
 * starting with an FP64-accurate matvec (the true residual, checked against
 * lanczos_tol) and continuing on the tensor cores until the residual estimate
 * has fallen by inner_factor (default 1e-2 for BF16X3, 1e-3 for TF32X3: a
 * restart gains about what the split precision allows, so a smaller factor
 * only adds matvecs) or inner_cap matvecs (default 80) have run; the Ritz
 * vector starts the next restart.  EINVAL unless
 * 0 < inner_factor < 1 and inner_cap >= 2.  No effect in FP64 and FP64_TC. */
idmrg_status idmrg_set_mixed_restart(idmrg_ctx *ctx, double inner_factor, int inner_cap);

/* Fixes the N tile of stage 1 (tn1) and stage 3 (tn3) of the split-operand
 * GEMMs instead of tuning it: 64, 128 or 256, or 0 to tune (the default).
 * Takes effect from the next iteration's plan; the results agree to
 * rounding whatever the tile (the K order of every product is the same).
 * EINVAL for any other value. */
idmrg_status idmrg_set_gemm_tile(idmrg_ctx *ctx, int tn1, int tn3);

/* Bytes this context has copied host->device and device->host so far. */
idmrg_status idmrg_transfer_bytes(const idmrg_ctx *ctx, uint64_t *h2d, uint64_t *d2h);

/* H_eff psi of superblock p (p >= 0) in FP64, for callers that cannot
 * allocate device memory while they run (a fixed or pre-partitioned memory
 * pool, an embedding application that forbids allocator calls from this
 * thread or while work is queued).  The paper has no counterpart; this is a
 * deployment variant of idmrg_heff_apply.  psi_dev and out_dev are the
 * caller's device vectors in the layout of idmrg_psi_layout(p); the
 * intermediates and the launch's pointer table live in a fixed 16 MiB device
 * array inside the library, which every GPU that loads the library holds
 * until the process exits.  The call itself allocates nothing (no cudaMalloc,
 * no allocator callback, no library routine that allocates).
 *  - Call it with the context's device current: every call looks up the
 *    array's device address on the current device (cudaGetSymbolAddress).
 *    The first call in a process may load the library's device code; make
 *    that first call before any stream capture.
 *  - It computes FP64 whatever opts.prec is (the FP64 GEMMs of form 0 of
 *    idmrg_heff_apply_fp64).
 *  - Valid from idmrg_create / idmrg_advance until the iteration's first
 *    idmrg_truncate; IDMRG_ESTATE from then until the next idmrg_advance.
 *  - Superblocks whose intermediates exceed the array return IDMRG_EINVAL
 *    with the sizes in idmrg_last_error.
 *  - All calls share the array and it keeps the last call's contents; every
 *    element a call reads is written by that call first, so nothing needs to
 *    start at zero.  Calls that overlap on the GPU (two streams, two contexts
 *    or two threads at once) race on it: order them on one stream. */
idmrg_status idmrg_heff_apply_noalloc(idmrg_ctx *ctx, int p, const double *psi_dev, double *out_dev);

#ifdef __cplusplus
}
#endif
#endif /* IDMRG_H */

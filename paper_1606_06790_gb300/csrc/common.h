// Internal declarations shared by the kernels and the host runtime of libidmrg.
// Nothing here is part of the public C ABI (include/idmrg.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace idmrg {

// ---------------------------------------------------------------- buffers
// Every operand of a batched kernel is addressed as (buffer id, element offset)
// inside one superblock; the per-superblock base pointers live in a device
// table bufs[sb * NBUF + id].  This keeps task lists independent of where the
// Lanczos loop currently reads and writes.
enum BufId {
  BUF_L = 0,      // left environment of the superblock (FP64)
  BUF_R = 1,      // right environment (FP64)
  BUF_IN = 2,     // matvec input vector
  BUF_OUT = 3,    // matvec output vector
  BUF_T1 = 4,     // H_eff stage-1 intermediate  T1[a] = L_a psi
  BUF_T3 = 5,     // H_eff stage-2 intermediate  T3[c] = W12 T1
  BUF_U = 6,      // kept left singular vectors  (rows (x,s), per sector)
  BUF_V = 7,      // kept right singular vectors (rows (t,y), per sector)
  BUF_X = 8,      // environment-update intermediate
  BUF_Y = 9,      // environment-update intermediate
  BUF_LNEW = 10,  // L^(n) being built
  BUF_RNEW = 11,  // R^(n) being built
  BUF_UT = 12,    // prediction: scaled u of superblock p+1 (u~ of Eq. wfprediction)
  BUF_VT = 13,    // prediction: scaled v of superblock p
  BUF_PSI = 14,   // start / ground-state vector
  BUF_SVD = 15,   // SVD work arena (the same for every superblock)
  BUF_UPREV = 16, // prediction source: u^(n-1) of superblock p+1
  BUF_VPREV = 17, // prediction source: v^(n-1) of superblock p
  // mixed-precision H_eff psi (tensor cores): packed TF32 hi/lo operands
  BUF_PA1 = 18,   // stage 1 A: L blocks stacked over channels, per in-sector
  BUF_PB1 = 19,   // stage 1 B: psi^T per in-sector (packed every matvec)
  BUF_T1F = 20,   // stage 1 output, FP32
  BUF_PA3 = 21,   // stage 3 A: T3 = W12 T1 (written by the W stage)
  BUF_PB3 = 22,   // stage 3 B: R blocks concatenated over channels, per out-sector
  BUF_RMAP = 23,  // stage 3 output row -> psi offset (int64)
  // FP64-accurate tensor-core form (BF16 digit slices, see kernels_tc.cu)
  BUF_OA1 = 24,   // stage 1 A digits
  BUF_OB1 = 25,   // stage 1 B digits (psi, every matvec)
  BUF_OT1 = 26,   // stage 1 output, FP64
  BUF_OA3 = 27,   // stage 3 A digits (written by the W stage)
  BUF_OB3 = 28,   // stage 3 B digits
  BUF_ORMAP = 29, // stage 3 output row -> psi offset (int64)
  BUF_OEXP = 30,  // per packed row: exponent of the digit expansion (int32)
  BUF_OT3 = 31,   // stage 3 A in FP64 (row-major per task) before its digits
  BUF_GOZ = 32,   // digit arena of the other FP64 GEMM lists (environments,
                  // prediction, SVD Newton-Schulz), the same for every superblock
  BUF_GEXP = 33,  // exponents of that arena
  NBUF = 34
};



// C[M x N] (+)= sum_seg alpha * op(A)[M x K] * op(B)[K x N]
//   op(A) = A (row-major, lda) or A^T (A stored K x M, lda) when (flags & 1)
//   op(B) = B (row-major K x N, ldb) or B^T (B stored N x K, ldb) when (flags & 2)
struct GemmSeg {
  int64_t a_off, b_off;
  int a_buf, b_buf;
  int lda, ldb;
  int K, flags;
  double alpha;
};
struct GemmTask {
  int64_t c_off;
  int c_buf, sb;
  int M, N, ldc;
  int seg0, nseg;
  int accumulate;  // 0: C = sum, 1: C += sum
};
struct GemmTile {
  int task, m0, n0, pad;
};

// out[r, c] = sum_terms coef * in[r, c]   (sub-matrices with row strides)
struct WTerm {
  int64_t in_off;
  int in_ld;
  int pad;
  double coef;
};
struct WTask {
  int64_t out_off;
  int out_ld, sb;
  int rows, cols;
  int term0, nterm;
  int out_buf, in_buf;
};

// element-wise dot of two equally shaped sub-matrices, weighted
struct DotTerm {
  int64_t off1, off2;
  int ld1, ld2;
  int rows, cols;
  int sb, buf;
  double coef;
};

// One charge-sector matrix for the SVD of Step 4.
//   M[r x c]: rows (left sector i, s, x) in row groups, columns (t, right
//   sector j, y) in column groups; element (row group g, col group h, x, y) of
//   psi sits at base[g*4+h] + x * rstride[g] + y.
//   The Jacobi working matrix A is M (r >= c) or M^T (r < c), column-major,
//   rows_a x cols_a with rows_a = max(r,c), cols_a = min(r,c).
struct SvdJob {
  int sb, Q;
  int r, c;
  int rows_a, cols_a, transposed;
  int ngr, ngc;
  int gr_start[4], gr_len[4], gr_stride[4];
  int gc_start[4], gc_len[4];
  int64_t base[16];
  int64_t a_off;    // A (rows_a x cols_a): Householder vectors after the QR
  int64_t j_off;    // Jm (cols_a x cols_a): accumulated Jacobi rotations
  int64_t b_off;    // B = R^T (cols_a x cols_a), Jacobi working matrix
  int64_t x_off;    // rows_a x cols_a scratch for the back-transformation
  int64_t tau_off;  // cols_a Householder coefficients
  int64_t w_off;    // cols_a x cols_a scratch of the FP32-preconditioned Jacobi
  int perm_off;     // cols_a column permutation of the pivoted QR (int work),
                    // then the numerical rank found by the QR and the sweeps
                    // the Jacobi stage needed
  int sv_off;       // singular values of this job
};

// splitmix64 start-vector sub-block
struct RandBlock {
  int64_t off;
  int rows, cols, ld, sb;
  int64_t dense0;   // dense index of element (0,0)
  int64_t dense_rs; // dense index step per row
  uint64_t state;   // stream state of the superblock
};

// dst[r*ld + c] = src[r*ld + c] * f_r * g_c with f_r = table[rs_off + r] (or,
// when rs_inv, its inverse, 0 where table[rs_off + r] <= zero_rel *
// table[max_off]) and g_c = table[cs_off + c]; an offset of -1 means 1.
struct ScaleTask {
  int64_t off;
  int rows, cols, ld, sb;
  int src_buf, dst_buf;
  int rs_off, cs_off;
  int rs_inv, max_off;
};

#define IDMRG_DEV_ERR_TIMEOUT 1
#define IDMRG_DEV_ERR_NUMERIC 2   // non-finite Lanczos coefficient
#define IDMRG_DEV_ERR_ZERONORM 4  // start vector with zero norm
#define IDMRG_DEV_ERR_JACOBI 8    // SVD sweeps exhausted

// ------------------------------------------------------------ launchers
// All launchers enqueue on `st` and return cudaGetLastError().
// tile shapes of the grouped GEMM (TM x TN outputs per CTA)
enum GemmShape { GEMM_64x64 = 0, GEMM_64x32 = 1, GEMM_32x64 = 2, GEMM_32x32 = 3, GEMM_NSHAPE = 4 };
constexpr int GEMM_TM[GEMM_NSHAPE] = {64, 64, 32, 32};
constexpr int GEMM_TN[GEMM_NSHAPE] = {64, 32, 64, 32};
cudaError_t launch_gemm_f64(const GemmTile *tiles, int ntiles, const GemmTask *tasks, const GemmSeg *segs,
                            double *const *bufs, const int *active, cudaStream_t st, int shape = GEMM_64x64);
cudaError_t launch_wstage_f64(const WTask *tasks, int ntasks, int max_rows, const WTerm *terms,
                              double *const *bufs, const int *active, cudaStream_t st);
cudaError_t launch_dot_terms(const DotTerm *terms, int nterms, double *const *bufs, double *partial,
                             cudaStream_t st);
cudaError_t launch_rand_blocks(const RandBlock *blocks, int nblocks, int max_rows, double *const *bufs, int buf,
                               cudaStream_t st);
cudaError_t launch_scale_tasks(const ScaleTask *tasks, int ntasks, int max_rows, const double *table,
                               double zero_rel, double *const *bufs, cudaStream_t st);

// Lanczos (FP64), batched over superblocks; see kernels_lanczos.cu
struct LanczosDev {
  int S;                 // superblocks in the batch
  int kmax;              // Krylov vectors per superblock
  const int64_t *N;      // [S] vector length
  double *const *V;      // [S] Krylov basis, kmax x N row-major
  double *const *w;      // [S] work vector
  double *alpha, *beta;  // [S * kmax]
  double *ibeta;         // [S * kmax] 1 / beta
  double *h;             // [S * kmax] projection coefficients
  double *part;          // partial sums
  int *k;                // [S] current Krylov index
  int *member;           // [S] 1 if the superblock takes part in this solve
  int *active;           // [S] 1 while iterating
  int *conv;             // [S] 1 converged / 2 breakdown / 0 not
  double *theta;         // [S] lowest Ritz value
  double *y;             // [S * kmax] Ritz coefficients
  double *resid;         // [S]
  int *err;              // device error word
  int nchunk_max;
  double tol;            // convergence: |b_k y_k| <= tol max(1, |theta|) ...
  double inner_factor;   // ... or, from the second Krylov vector on, <= target[s]
  double *target;        // [S] set at k = 0: max(tol max(1,|theta|), inner_factor b_0)
  double **bufs;         // buffer table of the H_eff launches: next_kernel points BUF_IN at V[k]
};
cudaError_t lanczos_set_ptrs(const LanczosDev &L, double **bufs, cudaStream_t st);
cudaError_t lanczos_project(const LanczosDev &L, int pass, cudaStream_t st);   // h = V^T w  (j <= k)
cudaError_t lanczos_subtract(const LanczosDev &L, int pass, cudaStream_t st);  // w -= V h (+ ||w||^2 partials on pass 1)
cudaError_t lanczos_sub0_proj1(const LanczosDev &L, cudaStream_t st);  // subtract pass 0 + project pass 1, fused
cudaError_t lanczos_reduce(const LanczosDev &L, int pass, cudaStream_t st);  // h[pass][j] = sum of its partials
cudaError_t lanczos_finalize(const LanczosDev &L, cudaStream_t st);            // alpha, beta, tridiagonal, convergence
cudaError_t lanczos_next(const LanczosDev &L, cudaStream_t st);                // V[k] = w / beta[k-1], BUF_IN -> V[k]
cudaError_t lanczos_init(const LanczosDev &L, const double *const *start, cudaStream_t st); // V[0] = start/|start|
cudaError_t lanczos_ritz(const LanczosDev &L, double *const *out, cudaStream_t st);  // out = V y / |V y|
cudaError_t lanczos_dot(const LanczosDev &L, const double *const *a, const double *const *b, double *res,
                        cudaStream_t st);  // res[s] = a_s . b_s
// res[s] = ||x_s|| for the superblocks with mask[s] (mask may be NULL): part
// holds S x nchunk partial sums, nchunk >= ceil(N_s / norm_chunk())
cudaError_t launch_norms(const int64_t *Ns, int S, const double *const *x, const int *mask, double *part,
                         int nchunk, double *res, cudaStream_t st);
int64_t norm_chunk();

// SVD (FP64 one-sided Jacobi), see kernels_svd.cu
cudaError_t launch_svd_gather_sized(const SvdJob *jobs, int njobs, int64_t max_elems, double *const *bufs,
                                    int psi_buf, double *work, cudaStream_t st);
cudaError_t launch_svd_qrcp(const SvdJob *jobs, const int *order, int njobs, double *work, int *iwork, double zero_rel,
                            cudaStream_t st);
// the pivoted QR on thread-block clusters (groups as launch_svd_jacobi);
// rows[k], cols[k]: largest rows and columns of block group k+1; rows0,
// cols0 those of group 0 (one CTA per job when they do not fit a cluster)
size_t svd_qrc_smem(int rows, int cols, int csize);
cudaError_t launch_svd_qrcp_grouped(const SvdJob *jobs, const int *order, int njobs, const int *g, const int *rows,
                                    const int *cols, int rows0, int cols0, double *work, int *iwork,
                                    double zero_rel, bool force_global_cols, cudaStream_t st,
                                    const cudaStream_t *side, const cudaEvent_t *ev);
// Jacobi groups and shared memory: see kernels_svd.cu
constexpr size_t SVD_BLOCK_SMEM_MAX = 200 * 1024;
size_t svd_block_smem(int cols, int csize);
// pairs: the FP64 stage of group 0 in FP32-pair arithmetic (48 bits)
cudaError_t launch_svd_jacobi(const SvdJob *jobs, const int *order, int njobs, const int *g, const int *cols,
                              double *work, int *iwork, double *sv, int *err, int jm_init, bool pairs,
                              cudaStream_t st, const cudaStream_t *side, const cudaEvent_t *ev);
// FP32 Jacobi on every group (group 0, the sectors beyond the block kernels,
// with cols0 columns at most, on the large-sector kernels; its jobs from g0b
// on, of at most cols0b columns, fit the shared-memory tournament): writes
// the accumulated rotations of each job to its V (j_off, cols_a x cols_a).
// side: 4 streams, ev: 5 events.
cudaError_t launch_svd_jacobi32(const SvdJob *jobs, const int *order, int njobs, const int *g, const int *cols,
                                int cols0, int g0b, int cols0b, double *work, const int *iwork, cudaStream_t st,
                                const cudaStream_t *side, const cudaEvent_t *ev);
// the largest sector (columns) the shared-memory FP32 tournament holds
int svd_jacobi32_big_max_cols();
// per job over cols_a x cols_a elements: 0: V = I; 1: V = 1.5 V - 0.5 W
// (Newton-Schulz step, W at w_off); 2: B = X (X at w_off)
cudaError_t launch_svd_elementwise(const SvdJob *jobs, int njobs, int max_cols, int mode, double *work,
                                   cudaStream_t st);
struct SelectOut {
  int *kept_per_job;   // [njobs]
  int *perm;           // [sum cols_a] kept slot -> index within job (per job, at sv_off)
  double *lam_sorted;  // [sum cols_a] all singular values of each superblock, descending
  double *eps;         // [S] discarded weight (Eq. tru)
  double *eps_best;    // [S]
  int *kept;           // [S]
};
cudaError_t launch_svd_select(const SvdJob *jobs, const int *sb_job0, const int *sb_njob, int S, const double *sv,
                              const int *m_sb, double zero_rel, double tie_rel, SelectOut out, int max_entries,
                              cudaStream_t st);
struct CompactJob {
  int job;             // SvdJob index
  int64_t u_off, v_off;// destination of U_Q (r x k) and V_Q (c x k), row-major
  int lam_off;         // destination of lambda (k entries)
  int pad;
};
cudaError_t launch_svd_compact(const SvdJob *jobs, const CompactJob *cj, int ncj, int max_kept, int max_rows,
                               double *work, const int *iwork, const double *sv, const int *perm,
                               const int *kept_per_job, double *const *bufs, double *lam, cudaStream_t st);

// ---- tensor-core path (kernels_tc.cu)
// Packed operand matrix: tiles of (8 G) rows x 128 bytes of K (32 TF32 or 64
// BF16 elements), K-major, core matrices of 8 rows x 16 bytes ordered
// [K chunk][row group][row][16 bytes]; per tile the hi part then the lo part;
// tiles ordered [row tile][K block].  `bf16` selects the BF16 split.
struct PackSeg {
  int64_t dst_off, src_off;
  int64_t exp_off;        // digit form: exponent of packed row r at exp[exp_off + r]
  int row0, k0, rows, ks;
  int src_ld, trans;      // trans: source element (row, k) at src[k * src_ld + row]
  int KB, G;              // K blocks and row groups of the packed matrix
  int sb, src_buf, dst_buf, src_fp32;
  int whole;              // digit form: the segment holds the whole K range of its rows
  int exp_buf;            // digit form: slot of the exponent array
  double alpha;           // digit form: source values scaled by alpha
};
struct WTaskP {           // T3 rectangle written into a packed stage-3 A matrix
  int64_t dst_off;
  int64_t exp_off;        // digit form: exponents of the task's packed rows
  int row0, k0, KB, G;
  int sb, rows, cols, term0, nterm;
  int in_buf, dst_buf;    // stage-1 output read, packed A written
  int t3_ld;              // digit form: T3 stored at t3_off, rows of t3_ld (the task's K)
  int64_t t3_off;
};
struct TcTask {
  int64_t a_off, b_off, c_off, rmap_off;
  int64_t a_exp, b_exp;   // digit form: exponent arrays of the A rows and B rows
  int sb, M, N, KB;
  int a_buf, b_buf, c_buf, rmap_buf;
  int mode, ldc;          // mode 0: FP32 row-major C; 1: FP64 through the row map;
                          // 2: FP64 row-major C
  int kb0, kb_stride;     // digit form: first K block of this K chunk, K blocks of the packed rows
  int accum, exp_buf;     // digit form: add to C instead of storing; slot of the exponents
};
struct TcTile {
  int task, mt, nt, pad;
};
constexpr int TC_TN = 64;      // N tile of the digit-slice GEMM (TMEM columns per level)
// N tiles of the split-operand (TF32x3 / BF16x3) GEMM the tuner chooses from
constexpr int MIX_NTN = 3;
constexpr int MIX_TNS[MIX_NTN] = {64, 128, 256};
cudaError_t launch_pack(const PackSeg *segs, int nseg, int max_rows, double *const *bufs, const int *active,
                        int bf16, cudaStream_t st);
// W stage work units: units[k] = (task, first row, K window): 32 rows of the
// task's rectangle and the packed K columns [64 w, 64 w + 64) it overlaps
cudaError_t launch_wstage_tc(const int4 *units, int nunits, const WTaskP *tasks, const WTerm *terms,
                             double *const *bufs, const int *active, int bf16, cudaStream_t st);
cudaError_t launch_tc_gemm(const TcTile *tiles, int ntiles, const TcTask *tasks, double *const *bufs,
                           const int *active, int *err, int bf16, int tn, cudaStream_t st);
// FP64-accurate products from BF16 digit slices (OZ_PLANES digits of 7 bits
// per element, exact integer accumulation per digit level).  K blocks are 32
// elements; one launch sums at most OZ_MAX_K of K exactly, longer K runs as
// successive chunks that add their FP64 results to C.
constexpr int OZ_PLANES = 8;
constexpr int OZ_KBLK = 32;
constexpr int OZ_MAX_K = 768;
constexpr int OZ_EXP_EMPTY = (int)0x80808080;  // byte-fill value: row without non-zeros
cudaError_t launch_oz_exp(const PackSeg *segs, int nseg, int max_rows, double *const *bufs, const int *active,
                          cudaStream_t st);
cudaError_t launch_oz_pack(const PackSeg *segs, int nseg, int max_rows, double *const *bufs, const int *active,
                           cudaStream_t st);
cudaError_t launch_wstage_oz(const WTaskP *tasks, int ntasks, int max_rows, const WTerm *terms,
                             double *const *bufs, const int *active, int pass, cudaStream_t st);
cudaError_t launch_oz_gemm(const TcTile *tiles, int ntiles, const TcTask *tasks, double *const *bufs,
                           const int *active, int *err, cudaStream_t st);

// Uniform-MPS observables (Eq. mps2), see kernels_obs.cu.  An embed task
// writes dst[x][y] = src(x, y) * scal[cs + y] / scal[rs + x] for x < rows,
// y < cols, src(x, y) = src[x * src_ld + y] (trans: src[y * src_ld + x]);
// rs / cs < 0: no scaling; a row scale at or below thr zeroes the row.
struct EmbedTask {
  const double *src;
  double *dst;
  int rows, cols, src_ld, dst_ld;
  int trans, rs, cs, pad;
  double thr;
};
cudaError_t launch_obs_embed(const EmbedTask *tasks, int ntasks, int max_rows, const double *scal, cudaStream_t st);
cudaError_t launch_obs_dot(const double *x, const double *y, int64_t n, double coef, double *out, int accumulate,
                           cudaStream_t st);
cudaError_t launch_obs_axpby(const double *x, double *y, int64_t n, double a, double b, cudaStream_t st);
cudaError_t launch_obs_fill(double *x, int D, int mode, double value, uint64_t seed, cudaStream_t st);
cudaError_t launch_obs_mask(double *x, int D, const int *q, int delta, cudaStream_t st);

}  // namespace idmrg

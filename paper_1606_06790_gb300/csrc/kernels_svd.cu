// FP64 SVD of Step 4, one charge sector per job, and the truncation of Step 6.
//
//  gather  : copies the sector matrix M_Q (rows (x,s) of left charge Q,
//            columns (t,y) of the complementary charge) out of the wavefunction
//            into a column-major working matrix A (M or M^T, tall side first).
//  qrcp    : Householder QR with column pivoting, A P = Q R.  This is the
//            preconditioner of the Jacobi SVD (Drmac and Veselic): one-sided
//            Jacobi on R^T needs a few sweeps where the same method on A needs
//            about twenty for the graded spectra of a wavefunction.
//  jacobi  : one-sided (Hestenes) Jacobi on B = R^T: plane rotations make the
//            columns of B orthogonal, B Jm = U~ S.  Parallel round-robin
//            ordering, one warp per column pair, the pairs of a round spread
//            over a cluster of CTAs that meet at the hardware cluster barrier.
//            Then A = (Q Jm) S (P U~)^T.
//  select  : per superblock, sorts all singular values in descending order
//            (ties by |Q|, Q, index), drops values at or below zero_rel*max,
//            cuts at D <= m without splitting values closer than tie_rel, and
//            writes the discarded weight (Eq. tru) and best fidelity error
//            (Eq. fid2).
//  compact : for the kept columns only, forms the singular vectors of A
//            (Q Jm e_j by the stored reflectors, P U~ e_j by the permutation)
//            and writes them as the U and V blocks of the new bases.
#include <cooperative_groups.h>
#include <float.h>
#include <math.h>

#include <algorithm>

#include "common.h"

namespace cg = cooperative_groups;

namespace idmrg {

namespace {

constexpr int GATHER_CHUNK = 8192;

__global__ void gather_kernel(const SvdJob *__restrict__ jobs, double *const *__restrict__ bufs, int psi_buf,
                              double *__restrict__ work) {
  const SvdJob J = jobs[blockIdx.x];
  const int64_t n = (int64_t)J.r * J.c;
  const int64_t e0 = (int64_t)blockIdx.y * GATHER_CHUNK;
  if (e0 >= n) return;
  const double *psi = bufs[J.sb * NBUF + psi_buf];
  double *A = work + J.a_off;
  for (int64_t e = e0 + threadIdx.x; e < min(n, e0 + GATHER_CHUNK); e += blockDim.x) {
    const int row = (int)(e / J.c), col = (int)(e % J.c);
    int g = 0, h = 0;
    while (g + 1 < J.ngr && row >= J.gr_start[g + 1]) ++g;
    while (h + 1 < J.ngc && col >= J.gc_start[h + 1]) ++h;
    const double v = psi[J.base[g * 4 + h] + (int64_t)(row - J.gr_start[g]) * J.gr_stride[g] + (col - J.gc_start[h])];
    if (!J.transposed)
      A[(int64_t)col * J.r + row] = v;
    else
      A[(int64_t)row * J.c + col] = v;
  }
}

__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------ QRCP
constexpr int QR_THREADS = 512;

__global__ void __launch_bounds__(QR_THREADS) qrcp_kernel(const SvdJob *__restrict__ jobs, const int *__restrict__ order,
                                                          double *__restrict__ work, int *__restrict__ iwork,
                                                          double zero_rel) {
  extern __shared__ double qsm[];  // vn[ca], vref[ca]
  const SvdJob Jb = jobs[order[blockIdx.x]];
  const int ra = Jb.rows_a, ca = Jb.cols_a;
  double *A = work + Jb.a_off;
  double *tau = work + Jb.tau_off;
  double *B = work + Jb.b_off;
  int *perm = iwork + Jb.perm_off;
  double *vn = qsm, *vref = qsm + ca;
  __shared__ double red_v[QR_THREADS / 32];
  __shared__ int red_i[QR_THREADS / 32];
  __shared__ double s_beta, s_tau, s_scale;
  __shared__ int s_piv;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = warp; j < ca; j += nw) {
    double s = 0.0;
    for (int i = lane; i < ra; i += 32) s = fma(A[(int64_t)j * ra + i], A[(int64_t)j * ra + i], s);
    s = wsum(s);
    if (lane == 0) { vn[j] = s; vref[j] = s; perm[j] = j; }
  }
  __syncthreads();
  // The QR stops at the numerical rank: once the largest remaining column
  // norm is below 0.1 zero_rel |R_00| / sqrt(cols), every singular value left
  // in the trailing block is below 0.1 zero_rel sigma_max, i.e. one the cut
  // treats as zero anyway, and the kept ones move by less than that.
  __shared__ double s_stop2;
  __shared__ int s_rank;
  if (threadIdx.x == 0) { s_rank = ca; s_stop2 = -1.0; }
  int k = 0;
  for (; k < ca; ++k) {
    // pivot: largest remaining column norm (first index on ties)
    double bv = -1.0;
    int bi = k;
    for (int j = k + threadIdx.x; j < ca; j += blockDim.x)
      if (vn[j] > bv) { bv = vn[j]; bi = j; }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = bv; red_i[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = red_v[0];
      int idx = red_i[0];
      for (int q = 1; q < nw; ++q)
        if (red_v[q] > v || (red_v[q] == v && red_i[q] < idx)) { v = red_v[q]; idx = red_i[q]; }
      s_piv = idx;
    }
    __syncthreads();
    const int p = s_piv;
    if (threadIdx.x == 0) {
      if (k == 0) s_stop2 = vn[p] * (0.01 * zero_rel * zero_rel / (double)ca);
      if (!(vn[p] > s_stop2)) s_rank = k;
    }
    __syncthreads();
    if (s_rank == k) break;
    if (p != k) {
      for (int i = threadIdx.x; i < ra; i += blockDim.x) {
        const double t = A[(int64_t)k * ra + i];
        A[(int64_t)k * ra + i] = A[(int64_t)p * ra + i];
        A[(int64_t)p * ra + i] = t;
      }
      if (threadIdx.x == 0) {
        double t = vn[k]; vn[k] = vn[p]; vn[p] = t;
        t = vref[k]; vref[k] = vref[p]; vref[p] = t;
        const int ti = perm[k]; perm[k] = perm[p]; perm[p] = ti;
      }
      __syncthreads();
    }
    // Householder reflector for column k, rows k..ra-1
    double *ak = A + (int64_t)k * ra;
    double s2 = 0.0;
    for (int i = k + 1 + threadIdx.x; i < ra; i += blockDim.x) s2 = fma(ak[i], ak[i], s2);
    s2 = wsum(s2);
    if (lane == 0) red_v[warp] = s2;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sig = 0.0;
      for (int q = 0; q < nw; ++q) sig += red_v[q];
      const double alpha = ak[k];
      if (sig == 0.0) {
        s_tau = 0.0;
        s_beta = alpha;
        s_scale = 1.0;
      } else {
        const double beta = -copysign(sqrt(alpha * alpha + sig), alpha);
        s_tau = (beta - alpha) / beta;
        s_beta = beta;
        s_scale = 1.0 / (alpha - beta);
      }
      tau[k] = s_tau;
    }
    __syncthreads();
    const double tk = s_tau;
    if (tk != 0.0) {
      const double sc = s_scale;
      for (int i = k + 1 + threadIdx.x; i < ra; i += blockDim.x) ak[i] *= sc;
    }
    __syncthreads();
    if (threadIdx.x == 0) ak[k] = s_beta;
    // apply H_k to the trailing columns, one warp per column
    if (tk != 0.0) {
      for (int j = k + 1 + warp; j < ca; j += nw) {
        double *aj = A + (int64_t)j * ra;
        double w = 0.0;
        for (int i = k + 1 + lane; i < ra; i += 32) w = fma(ak[i], aj[i], w);
        w = (wsum(w) + aj[k]) * tk;
        __syncwarp();
        if (lane == 0) aj[k] -= w;
        for (int i = k + 1 + lane; i < ra; i += 32) aj[i] = fma(-w, ak[i], aj[i]);
      }
    }
    __syncthreads();
    // downdate the remaining column norms; recompute where cancellation hurts
    for (int j = k + 1 + warp; j < ca; j += nw) {
      const double *aj = A + (int64_t)j * ra;
      double nv = vn[j] - aj[k] * aj[k];
      if (!(nv > 1e-8 * vref[j])) {
        double s = 0.0;
        for (int i = k + 1 + lane; i < ra; i += 32) s = fma(aj[i], aj[i], s);
        nv = wsum(s);
        if (lane == 0) vref[j] = nv;
      }
      if (lane == 0) vn[j] = fmax(nv, 0.0);
    }
    __syncthreads();
  }
  const int rk = s_rank;
  if (threadIdx.x == 0) perm[ca] = rk;
  // B = [R11 R12]^T (ca x rk, column-major): B(a, b) = R(b, a) for b <= a, b < rk
  for (int64_t e = threadIdx.x; e < (int64_t)ca * rk; e += blockDim.x) {
    const int a = (int)(e % ca), b = (int)(e / ca);
    B[e] = (b <= a) ? A[(int64_t)a * ra + b] : 0.0;
  }
}

// ---------------------------------------------------------------- Jacobi
constexpr int JAC_THREADS = 512;
constexpr int JAC_MAX_CLUSTER = 16;
constexpr int JAC_REG = 8;  // column elements per lane held in registers

// Rotation that zeroes the overlap g of two columns with squared norms a, b:
// tan(theta) = t, t = sgn(z) / (|z| + sqrt(1 + z^2)), z = (b - a) / (2 g).
// The angle only steers convergence, so t is formed in FP32 (after scaling
// both operands of the quotient into FP32 range); cos = 1/sqrt(1 + t^2) is
// refined to FP64 by two Newton steps on the reciprocal square root, so the
// pair (cos, sin = cos t) is orthogonal to FP64 precision.
__device__ __forceinline__ void rotation(double a, double b, double g, double &cs, double &sn) {
  const double num = b - a, den = 2.0 * g;
  const int e = max(ilogb(fabs(num)), ilogb(fabs(den)));
  const float z = (float)scalbn(num, -e) / (float)scalbn(den, -e);
  const float az = fabsf(z);
  const float tf = az > 1e15f ? 0.5f / z : copysignf(1.0f, z) / (az + sqrtf(fmaf(z, z, 1.0f)));
  const double t = (double)tf;
  const double x = fma(t, t, 1.0);
  double y = (double)rsqrtf((float)x);
  y = y * fma(-0.5 * x * y, y, 1.5);
  y = y * fma(-0.5 * x * y, y, 1.5);
  cs = y;
  sn = y * t;
}

// one column pair (p, q): overlap, rotation of B's and Jm's columns
__device__ __forceinline__ bool jacobi_pair(double *ap, double *aq, double *jp, double *jq, int n, int nj,
                                            int lane, double tol2, double abs_floor) {
  double x[JAC_REG], y[JAC_REG];
  double al = 0.0, be = 0.0, ga = 0.0;
  const bool inreg = n <= 32 * JAC_REG;
  const int nreg = (n + 31) >> 5;
  if (inreg) {
#pragma unroll
    for (int r = 0; r < JAC_REG; ++r) {
      if (r < nreg) {
        const int i = lane + 32 * r;
        x[r] = i < n ? ap[i] : 0.0;
        y[r] = i < n ? aq[i] : 0.0;
        al = fma(x[r], x[r], al);
        be = fma(y[r], y[r], be);
        ga = fma(x[r], y[r], ga);
      }
    }
  } else {
    for (int i = lane; i < n; i += 32) {
      const double u = ap[i], v = aq[i];
      al = fma(u, u, al);
      be = fma(v, v, be);
      ga = fma(u, v, ga);
    }
  }
  al = wsum(al);
  be = wsum(be);
  ga = wsum(ga);
  // rotate unless |g| <= tol sqrt(a b) (compared squared) or below the floor
  if (!(ga * ga > tol2 * (al * be)) || !(fabs(ga) > abs_floor)) return false;
  double cs = 0.0, sn = 0.0;
  if (lane == 0) rotation(al, be, ga, cs, sn);
  cs = __shfl_sync(0xffffffffu, cs, 0);
  sn = __shfl_sync(0xffffffffu, sn, 0);
  if (inreg) {
#pragma unroll
    for (int r = 0; r < JAC_REG; ++r) {
      if (r < nreg) {
        const int i = lane + 32 * r;
        if (i < n) {
          ap[i] = cs * x[r] - sn * y[r];
          aq[i] = sn * x[r] + cs * y[r];
        }
      }
    }
  } else {
    for (int i = lane; i < n; i += 32) {
      const double u = ap[i], v = aq[i];
      ap[i] = cs * u - sn * v;
      aq[i] = sn * u + cs * v;
    }
  }
  for (int i = lane; i < nj; i += 32) {
    const double u = jp[i], v = jq[i];
    jp[i] = cs * u - sn * v;
    jq[i] = sn * u + cs * v;
  }
  return true;
}

// One job per cluster (cluster size chosen at launch); the pairs of a round
// are spread over all warps of the cluster, rounds separated by the hardware
// cluster barrier.
__global__ void __launch_bounds__(JAC_THREADS, 2)
    jacobi_kernel(const SvdJob *__restrict__ jobs, const int *__restrict__ order, double *__restrict__ work,
                  int *__restrict__ iwork, double *__restrict__ sv, int *err) {
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int csize = (int)cluster.num_blocks();
  const SvdJob Jb = jobs[order[blockIdx.x / csize]];
  const int nr = Jb.cols_a;                       // rows of B
  const int n = iwork[Jb.perm_off + Jb.cols_a];   // columns of B: numerical rank
  double *B = work + Jb.b_off;
  double *Jm = work + Jb.j_off;
  __shared__ double fro_part[JAC_MAX_CLUSTER];
  __shared__ double wred[JAC_THREADS / 32];
  __shared__ int flag, local_changed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  // pair k of a round goes to CTA k mod csize: the FP64 work of a round is
  // spread over every SM of the cluster (blocked by CTA it piled up on the
  // first few while the others waited at the barrier)
  const int gw = warp * csize + crank, gnw = csize * nw;
  const int64_t nn = (int64_t)n * n, nb = (int64_t)nr * n;
  for (int64_t e = (int64_t)crank * blockDim.x + threadIdx.x; e < nn; e += (int64_t)csize * blockDim.x)
    Jm[e] = (e / n == e % n) ? 1.0 : 0.0;
  // ||B||_F^2 over the cluster (partials gathered in rank 0's shared memory)
  double fro = 0.0;
  for (int64_t e = (int64_t)crank * blockDim.x + threadIdx.x; e < nb; e += (int64_t)csize * blockDim.x)
    fro = fma(B[e], B[e], fro);
  fro = wsum(fro);
  if (lane == 0) wred[warp] = fro;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < nw; ++q) t += wred[q];
    double *dst = cluster.map_shared_rank(fro_part, 0);
    dst[crank] = t;
  }
  cluster.sync();
  const double *fp0 = cluster.map_shared_rank(fro_part, 0);
  fro = 0.0;
  for (int q = 0; q < csize; ++q) fro += fp0[q];
  cluster.sync();  // every CTA has read rank 0's partials
  // rotation threshold sqrt(rows) * eps (as in LAPACK's one-sided Jacobi) and
  // an absolute floor eps^2 ||B||_F^2: without it a column made of rounding
  // noise along another one never meets the relative test (each rotation
  // leaves an eps-sized overlap that dominates tol |b_p| |b_q| as |b_q| -> 0).
  const double tol = sqrt((double)nr) * DBL_EPSILON;
  const double tol2 = tol * tol;
  const double abs_floor = 4.0 * DBL_EPSILON * DBL_EPSILON * fro;
  const int np = n + (n & 1);
  int *flag0 = cluster.map_shared_rank(&flag, 0);
  bool converged = (n < 2);
  int sweep = 0;
  for (; sweep < 40 && !converged; ++sweep) {
    if (threadIdx.x == 0) local_changed = 0;
    if (crank == 0 && threadIdx.x == 0) flag = 0;
    cluster.sync();
    bool any = false;
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      for (int k = gw; k < np / 2; k += gnw) {
        const int i1 = k, i2 = np - 1 - k;
        const int p = i1 == 0 ? 0 : 1 + (i1 - 1 + rnd) % (np - 1);
        const int q = i2 == 0 ? 0 : 1 + (i2 - 1 + rnd) % (np - 1);
        if (p >= n || q >= n) continue;
        any |= jacobi_pair(B + (int64_t)p * nr, B + (int64_t)q * nr, Jm + (int64_t)p * n, Jm + (int64_t)q * n, nr,
                           n, lane, tol2, abs_floor);
      }
      cluster.sync();
    }
    if (any && lane == 0) local_changed = 1;
    __syncthreads();
    if (threadIdx.x == 0 && local_changed) atomicOr(flag0, 1);
    cluster.sync();
    converged = (*flag0 == 0);
    cluster.sync();
  }
  if (!converged && crank == 0 && threadIdx.x == 0) atomicOr(err, IDMRG_DEV_ERR_JACOBI);
  if (crank == 0 && threadIdx.x == 0) iwork[Jb.perm_off + Jb.cols_a + 1] = sweep;
  // singular values; columns of B normalised in place; the columns beyond
  // the numerical rank have singular value zero
  for (int j = gw; j < Jb.cols_a; j += gnw) {
    if (j >= n) {
      if (lane == 0) sv[Jb.sv_off + j] = 0.0;
      continue;
    }
    double *bj = B + (int64_t)j * nr;
    double s = 0.0;
    for (int i = lane; i < nr; i += 32) s = fma(bj[i], bj[i], s);
    s = sqrt(wsum(s));
    if (lane == 0) sv[Jb.sv_off + j] = s;
    const double inv = s > 0.0 ? 1.0 / s : 0.0;
    for (int i = lane; i < nr; i += 32) bj[i] *= inv;
  }
}

// ---------------------------------------------------------------- select
struct Entry {
  double s;
  int job, j;
};

__device__ __forceinline__ bool before(const Entry &a, const Entry &b, const SvdJob *jobs) {
  if (a.s != b.s) return a.s > b.s;
  const int qa = jobs[a.job].Q, qb = jobs[b.job].Q;
  if (abs(qa) != abs(qb)) return abs(qa) < abs(qb);
  if (qa != qb) return qa < qb;
  return a.j < b.j;
}

__global__ void select_kernel(const SvdJob *__restrict__ jobs, const int *__restrict__ sb_job0,
                              const int *__restrict__ sb_njob, const double *__restrict__ sv, int m,
                              double zero_rel, double tie_rel, SelectOut out, int P) {
  extern __shared__ unsigned char smraw[];
  Entry *E = (Entry *)smraw;
  int *cnt = (int *)(E + P);
  const int s = blockIdx.x;
  const int j0 = sb_job0[s], nj = sb_njob[s];
  const int base = jobs[j0].sv_off;
  int total = 0;
  for (int q = 0; q < nj; ++q) total += jobs[j0 + q].cols_a;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    if (i < total) {
      int q = 0;
      while (i >= jobs[j0 + q].sv_off - base + jobs[j0 + q].cols_a) ++q;
      E[i].s = sv[base + i];
      E[i].job = j0 + q;
      E[i].j = base + i - jobs[j0 + q].sv_off;
    } else {
      E[i].s = -1.0;
      E[i].job = j0;
      E[i].j = 0x7fffffff;
    }
  }
  for (int q = threadIdx.x; q < nj; q += blockDim.x) cnt[q] = 0;
  __syncthreads();
  // bitonic sort, descending by `before`
  for (int k = 2; k <= P; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int l = i ^ jj;
        if (l > i) {
          const bool up = ((i & k) == 0);
          const Entry a = E[i], b = E[l];
          const bool swap = up ? before(b, a, jobs) : before(a, b, jobs);
          if (swap) { E[i] = b; E[l] = a; }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < total; i += blockDim.x) out.lam_sorted[base + i] = E[i].s;
  if (threadIdx.x == 0) {
    const double smax = E[0].s;
    int nz = 0;
    while (nz < total && E[nz].s > zero_rel * smax) ++nz;
    const int top = min(m, nz);
    int D = top;
    while (D > 0 && D < nz && !(E[D].s < E[D - 1].s * (1.0 - tie_rel))) --D;
    if (D == 0) D = top;
    double w2 = 0.0;
    for (int i = 0; i < D; ++i) w2 += E[i].s * E[i].s;
    out.eps[s] = 1.0 - w2;
    out.eps_best[s] = 1.0 - sqrt(w2);
    out.kept[s] = D;
    for (int i = 0; i < D; ++i) {
      const int q = E[i].job - j0;
      out.perm[jobs[E[i].job].sv_off + cnt[q]] = E[i].j;
      cnt[q] += 1;
    }
    for (int q = 0; q < nj; ++q) out.kept_per_job[j0 + q] = cnt[q];
  }
}

// --------------------------------------------------------------- compact
// One warp per kept column: left singular vector of A = Q [Jm e_j; 0]
// (reflectors applied last to first), right one = P U~ e_j.
__global__ void compact_kernel(const SvdJob *__restrict__ jobs, const CompactJob *__restrict__ cjs,
                               double *__restrict__ work, const int *__restrict__ iwork,
                               const double *__restrict__ sv, const int *__restrict__ perm,
                               const int *__restrict__ kept_per_job, double *const *__restrict__ bufs,
                               double *__restrict__ lam) {
  const CompactJob cj = cjs[blockIdx.x];
  const SvdJob J = jobs[cj.job];
  const int k = kept_per_job[cj.job];
  const int ra = J.rows_a, ca = J.cols_a;
  const double *A = work + J.a_off;
  const double *tau = work + J.tau_off;
  const double *Jm = work + J.j_off;
  const double *Bn = work + J.b_off;
  const int *qperm = iwork + J.perm_off;
  const int rk = qperm[ca];
  double *U = bufs[J.sb * NBUF + BUF_U] + cj.u_off;
  double *V = bufs[J.sb * NBUF + BUF_V] + cj.v_off;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.y * (blockDim.x >> 5) + warp, gnw = gridDim.y * (blockDim.x >> 5);
  for (int slot = gw; slot < k; slot += gnw) {
    const int col = perm[J.sv_off + slot];
    double *x = work + J.x_off + (int64_t)slot * ra;
    for (int i = lane; i < ra; i += 32) x[i] = i < rk ? Jm[(int64_t)col * rk + i] : 0.0;
    __syncwarp();
    for (int kk = rk - 1; kk >= 0; --kk) {
      const double t = tau[kk];
      if (t == 0.0) continue;
      const double *v = A + (int64_t)kk * ra;
      double w = 0.0;
      for (int i = kk + 1 + lane; i < ra; i += 32) w = fma(v[i], x[i], w);
      w = (wsum(w) + x[kk]) * t;
      __syncwarp();
      if (lane == 0) x[kk] -= w;
      for (int i = kk + 1 + lane; i < ra; i += 32) x[i] = fma(-w, v[i], x[i]);
      __syncwarp();
    }
    // left vectors of A: rows_a entries; right vectors: cols_a entries
    double *Lout = !J.transposed ? U : V;
    double *Rout = !J.transposed ? V : U;
    for (int i = lane; i < ra; i += 32) Lout[(int64_t)i * k + slot] = x[i];
    for (int i = lane; i < ca; i += 32) Rout[(int64_t)qperm[i] * k + slot] = Bn[(int64_t)col * ca + i];
    if (lane == 0) lam[cj.lam_off + slot] = sv[J.sv_off + col];
  }
}

}  // namespace

cudaError_t launch_svd_gather_sized(const SvdJob *jobs, int njobs, int64_t max_elems, double *const *bufs,
                                    int psi_buf, double *work, cudaStream_t st) {
  if (njobs > 0 && max_elems > 0) {
    dim3 grid(njobs, (unsigned)((max_elems + GATHER_CHUNK - 1) / GATHER_CHUNK));
    gather_kernel<<<grid, 256, 0, st>>>(jobs, bufs, psi_buf, work);
  }
  return cudaGetLastError();
}

cudaError_t launch_svd_qrcp(const SvdJob *jobs, const int *order, int njobs, double *work, int *iwork, double zero_rel,
                            cudaStream_t st) {
  // shared: two norms per column; callers keep cols_a <= 4096
  const int smem = 2 * 4096 * (int)sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(qrcp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (njobs > 0) qrcp_kernel<<<njobs, QR_THREADS, smem, st>>>(jobs, order, work, iwork, zero_rel);
  return cudaGetLastError();
}

static cudaError_t launch_jacobi_clusters(const SvdJob *jobs, const int *order, int njobs, int csize, double *work,
                                          int *iwork, double *sv, int *err, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(njobs * csize, 1, 1);
  cfg.blockDim = dim3(JAC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, jacobi_kernel, jobs, order, work, iwork, sv, err);
}

// `order` lists the jobs largest first; the first `nbig` of them get
// clusters of up to 16 CTAs, the rest clusters of 4.
cudaError_t launch_svd_jacobi(const SvdJob *jobs, const int *order, int njobs, int nbig, double *work, int *iwork,
                              double *sv, int *err, cudaStream_t st) {
  if (njobs <= 0) return cudaGetLastError();
  cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaGetLastError();
  if (nbig > 0) {
    cudaError_t e = launch_jacobi_clusters(jobs, order, nbig, 16, work, iwork, sv, err, st);
    if (e != cudaSuccess) {
      cudaGetLastError();  // 16-CTA clusters not available here: fall back to 8
      e = launch_jacobi_clusters(jobs, order, nbig, 8, work, iwork, sv, err, st);
    }
    if (e != cudaSuccess) return e;
  }
  if (njobs > nbig) {
    cudaError_t e = launch_jacobi_clusters(jobs, order + nbig, njobs - nbig, 4, work, iwork, sv, err, st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t launch_svd_select(const SvdJob *jobs, const int *sb_job0, const int *sb_njob, int S, const double *sv,
                              int m, double zero_rel, double tie_rel, SelectOut out, int max_entries,
                              cudaStream_t st) {
  int P = 1;
  while (P < max_entries) P <<= 1;
  const size_t smem = (size_t)P * sizeof(Entry) + 256 * sizeof(int);
  cudaError_t e = cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (S > 0) select_kernel<<<S, 512, smem, st>>>(jobs, sb_job0, sb_njob, sv, m, zero_rel, tie_rel, out, P);
  return cudaGetLastError();
}

cudaError_t launch_svd_compact(const SvdJob *jobs, const CompactJob *cj, int ncj, int max_kept, double *work,
                               const int *iwork, const double *sv, const int *perm, const int *kept_per_job,
                               double *const *bufs, double *lam, cudaStream_t st) {
  if (ncj > 0) {
    const int warps = 8;
    dim3 grid(ncj, (unsigned)std::max(1, (max_kept + warps - 1) / warps));
    compact_kernel<<<grid, 32 * warps, 0, st>>>(jobs, cj, work, iwork, sv, perm, kept_per_job, bufs, lam);
  }
  return cudaGetLastError();
}

}  // namespace idmrg

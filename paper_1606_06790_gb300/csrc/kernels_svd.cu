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
#include <limits.h>
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
  // B = [R11 R12]^T (ca x rk, column-major): B(a, b) = R(b, a) for b <= a, b < rk;
  // the columns beyond the rank are zero (B's slot is ca x ca)
  for (int64_t e = threadIdx.x; e < (int64_t)ca * ca; e += blockDim.x) {
    const int a = (int)(e % ca), b = (int)(e / ca);
    B[e] = (b <= a && b < rk) ? A[(int64_t)a * ra + b] : 0.0;
  }
}

// ------------------------------------------------------------ cluster QRCP
// The same pivoted Householder QR over a cluster of C CTAs.  Column position
// j lives in the shared memory of CTA j mod C (cyclic, so the trailing
// columns stay spread as k grows).  Step k: the pivot is the largest
// remaining column norm over the cluster (candidates gathered in rank 0's
// shared memory, ties to the lower position as in qrcp_kernel); positions k
// and p are swapped between their owners through distributed shared memory;
// the owner of k forms the reflector and publishes it; every CTA applies it
// to its own trailing columns.  The trailing update, which holds the
// single-CTA kernel at one SM's FP64 rate, is spread over C SMs.
// Exponent and FP32 mantissa of a double, by integer operations only (an
// FP64 instruction costs 64 cycles of its sub-partition's FP64 unit here):
// x = m 2^e with |m| in [1, 2) (mantissa truncated to 23 bits); zero and
// subnormals give m = 0.
struct Split {
  float m;
  int e;
};
__device__ __forceinline__ Split split_f64(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int be = (int)((hi >> 20) & 0x7ffu);
  Split r;
  if (be == 0) {
    r.m = 0.0f;
    r.e = 0;
    return r;
  }
  const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
  r.m = __uint_as_float((hi & 0x80000000u) | (127u << 23) | mant);
  r.e = be - 1023;
  return r;
}

// the double of an FP32 number times 2^k (integer operations; f normal or
// zero, result in the normal range)
__device__ __forceinline__ double f64_of(float f, int k = 0) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xffu;
  if (ex == 0) return 0.0;
  const unsigned hi = (u & 0x80000000u) | ((ex + 896u + (unsigned)k) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)((u & 0x7u) << 29));
}

// 1/x for x > 0 in the normal range: FP32 estimate of the mantissa's
// reciprocal, then two Newton steps e <- e (2 - x e) in FP64
__device__ __forceinline__ double recip_split(double x) {
  const Split s = split_f64(x);
  double e = f64_of(__frcp_rn(s.m), -s.e);
  e = e * fma(-x, e, 2.0);
  e = e * fma(-x, e, 2.0);
  return e;
}

// 1/x for any finite non-zero x: Newton from an FP32 estimate in the normal
// range, the FP64 division outside it
__device__ __forceinline__ double recip_signed(double x) {
  const double ax = fabs(x);
  return (ax > 1e-290 && ax < 1e290) ? copysign(recip_split(ax), x) : 1.0 / x;
}

constexpr int QC_THREADS = 256;
constexpr int QC_MAX_CLUSTER = 16;

// GCOLS: the columns stay in global memory (the job's A) instead of the
// CTAs' shared memory, for sectors too large for a cluster's shared memory;
// the algorithm and the cluster's division of labour are the same.
template <bool GCOLS>
__global__ void __launch_bounds__(QC_THREADS)
    qrcp_cluster_kernel(const SvdJob *__restrict__ jobs, const int *__restrict__ order, double *__restrict__ work,
                        int *__restrict__ iwork, double zero_rel) {
  extern __shared__ __align__(16) double qc_sm[];
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int C = (int)cluster.num_blocks();
  const SvdJob Jb = jobs[order[blockIdx.x / C]];
  const int ra = Jb.rows_a, ca = Jb.cols_a;
  double *A = work + Jb.a_off;
  double *tau = work + Jb.tau_off;
  double *B = work + Jb.b_off;
  int *perm = iwork + Jb.perm_off;
  const int nloc = (ca + C - 1) / C;
  const int ld = (ra + 1) & ~1;                  // 16-byte aligned columns
  double *cols = qc_sm;                          // [nloc][ld] (shared-memory columns only)
  double *bcast = cols + (GCOLS ? (size_t)0 : (size_t)nloc * ld);  // [ld] reflector of the step
  double *swp = bcast + ld;                      // [ld] incoming column of a swap
  double *vn = swp + ld, *vref = vn + nloc;      // [nloc] squared norms
  int *pl = (int *)(vref + nloc);                // [nloc] original column at each position
  __shared__ double cand_v[QC_MAX_CLUSTER], red_v[QC_THREADS / 32], s_tau, s_beta, s_scale, s_swap_vn, s_swap_vref;
  __shared__ int cand_i[QC_MAX_CLUSTER], s_piv, s_stop, s_swap_pl;
  __shared__ double s_vp, s_stop2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  auto pos = [&](int l) { return crank + C * l; };
  // column at local slot l: shared memory, or the job's A in global memory
  auto colp = [&](int l) -> double * { return GCOLS ? A + (int64_t)pos(l) * ra : cols + (size_t)l * ld; };
  // load the owned columns and their squared norms
  if (!GCOLS) {
    for (int l = 0; l < nloc; ++l) {
      const int j = pos(l);
      if (j >= ca) break;
      for (int i = threadIdx.x; i < ra; i += blockDim.x) cols[(size_t)l * ld + i] = A[(int64_t)j * ra + i];
    }
  }
  __syncthreads();
  for (int l = warp; l < nloc; l += nw) {
    const int j = pos(l);
    if (j >= ca) continue;
    double s2 = 0.0;
    const double *cl = colp(l);
    for (int i = lane; i < ra; i += 32) s2 = fma(cl[i], cl[i], s2);
    s2 = wsum(s2);
    if (lane == 0) {
      vn[l] = s2;
      vref[l] = s2;
      pl[l] = j;
    }
  }
  if (threadIdx.x == 0) s_stop2 = -1.0;
  __syncthreads();
  double *cand_v0 = cluster.map_shared_rank(cand_v, 0);
  int *cand_i0 = cluster.map_shared_rank(cand_i, 0);
  int rank = ca;
  for (int k = 0; k < ca; ++k) {
    // (a) pivot: local candidate, gathered in rank 0, the same choice
    // everywhere.  The squared norms are non-negative, so they order like
    // their bit patterns as 64-bit integers: the comparisons run on the
    // integer units (an FP64 compare costs 64 cycles of the FP64 unit here).
    // A CTA holds at most a few dozen columns: warp 0 scans them.
    if (warp == 0) {
      long long bv = -1;
      int bi = 0x7fffffff;
      for (int l = lane; l < nloc; l += 32) {
        const int j = pos(l);
        const long long v = __double_as_longlong(vn[l]);
        if (j >= k && j < ca && (v > bv || (v == bv && j < bi))) {
          bv = v;
          bi = j;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
      }
      if (lane == 0) {
        cand_v0[crank] = __longlong_as_double(bv);
        cand_i0[crank] = bi;
      }
    }
    cluster.sync();
    if (warp == 0) {  // one lane per CTA reads its candidate (remote loads in parallel)
      long long v = lane < C ? __double_as_longlong(cand_v0[lane]) : -1;
      int idx = lane < C ? cand_i0[lane] : 0x7fffffff;
      for (int o = 16; o > 0; o >>= 1) {
        const long long ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
      }
      if (lane == 0) {
        const double vd = __longlong_as_double(v);
        s_piv = idx;
        s_vp = vd;
        if (k == 0) s_stop2 = vd * (0.01 * zero_rel * zero_rel / (double)ca);
        s_stop = !(v >= 0 && v > __double_as_longlong(s_stop2));
      }
    }
    __syncthreads();
    if (s_stop) {  // the same decision in every CTA: numerical rank reached
      rank = k;
      break;
    }
    const int p = s_piv;
    const int ok = k % C, op = p % C, lk = k / C, lp = p / C;
    // (b) swap positions k and p
    if (p != k) {
      if (ok == op) {
        if (crank == ok) {
          double *ck = colp(lk), *cp = colp(lp);
          for (int i = threadIdx.x; i < ra; i += blockDim.x) {
            const double t = ck[i];
            ck[i] = cp[i];
            cp[i] = t;
          }
          if (threadIdx.x == 0) {
            double t = vn[lk]; vn[lk] = vn[lp]; vn[lp] = t;
            t = vref[lk]; vref[lk] = vref[lp]; vref[lp] = t;
            const int ti = pl[lk]; pl[lk] = pl[lp]; pl[lp] = ti;
          }
        }
        cluster.sync();  // every CTA passes the same barriers
      } else {
        // each owner writes its column into the other's swap buffer (with
        // global columns the owner of k swaps both columns in place)
        if (crank == ok || crank == op) {
          const int mine = crank == ok ? lk : lp, other = crank == ok ? op : ok;
          if (!GCOLS) {
            double *dst = cluster.map_shared_rank(swp, other);
            for (int i = threadIdx.x; i < ra; i += blockDim.x) dst[i] = cols[(size_t)mine * ld + i];
          } else if (crank == ok) {
            double *ck = A + (int64_t)k * ra, *cp = A + (int64_t)p * ra;
            for (int i = threadIdx.x; i < ra; i += blockDim.x) {
              const double t = ck[i];
              ck[i] = cp[i];
              cp[i] = t;
            }
          }
          if (threadIdx.x == 0) {
            *cluster.map_shared_rank(&s_swap_vn, other) = vn[mine];
            *cluster.map_shared_rank(&s_swap_vref, other) = vref[mine];
            *cluster.map_shared_rank(&s_swap_pl, other) = pl[mine];
          }
        }
        cluster.sync();
        if (crank == ok || crank == op) {
          const int mine = crank == ok ? lk : lp;
          if (!GCOLS)
            for (int i = threadIdx.x; i < ra; i += blockDim.x) cols[(size_t)mine * ld + i] = swp[i];
          if (threadIdx.x == 0) {
            vn[mine] = s_swap_vn;
            vref[mine] = s_swap_vref;
            pl[mine] = s_swap_pl;
          }
        }
      }
      __syncthreads();
    }
    // (c) the owner of position k forms the reflector (rows k..ra-1)
    if (crank == ok) {
      double *ak = colp(lk);
      double s2 = 0.0;
      for (int i = k + 1 + threadIdx.x; i < ra; i += blockDim.x) s2 = fma(ak[i], ak[i], s2);
      s2 = wsum(s2);
      if (lane == 0) red_v[warp] = s2;
      __syncthreads();
      if (warp == 0) {
        double sig = lane < nw ? red_v[lane] : 0.0;
        for (int o = 4; o > 0; o >>= 1) sig += __shfl_xor_sync(0xffffffffu, sig, o);
        const double alpha = ak[k];
        if (lane == 0) {
          if (sig == 0.0) {
            s_tau = 0.0;
            s_beta = alpha;
            s_scale = 1.0;
          } else {
            // |beta| >= |alpha - beta| / 2 > 0; reciprocals by Newton's
            // iteration from an FP32 estimate (recip_split), correct to the
            // last bits, at a fraction of an FP64 division's instructions
            const double beta = -copysign(sqrt(alpha * alpha + sig), alpha);
            s_tau = (beta - alpha) * recip_signed(beta);
            s_beta = beta;
            s_scale = recip_signed(alpha - beta);
          }
          tau[k] = s_tau;
        }
      }
      __syncthreads();
      const double sc = s_scale;
      if (s_tau != 0.0)
        for (int i = k + 1 + threadIdx.x; i < ra; i += blockDim.x) ak[i] *= sc;
      __syncthreads();
      if (threadIdx.x == 0) ak[k] = s_beta;
      for (int i = k + 1 + threadIdx.x; i < ra; i += blockDim.x) bcast[i] = ak[i];
    }
    cluster.sync();  // reflector published
    // (d) every CTA applies H_k to its own trailing columns
    const double tk = *cluster.map_shared_rank(&s_tau, ok);
    if (tk != 0.0) {
      if (crank != ok) {
        const double *src = cluster.map_shared_rank(bcast, ok);
        for (int i = k + 1 + threadIdx.x; i < ra; i += blockDim.x) bcast[i] = src[i];
        __syncthreads();
      }
      for (int l = warp; l < nloc; l += nw) {
        const int j = pos(l);
        if (j <= k || j >= ca) continue;
        double *aj = colp(l);
        double w = 0.0;
        for (int i = k + 1 + lane; i < ra; i += 32) w = fma(bcast[i], aj[i], w);
        w = (wsum(w) + aj[k]) * tk;
        __syncwarp();
        if (lane == 0) aj[k] -= w;
        for (int i = k + 1 + lane; i < ra; i += 32) aj[i] = fma(-w, bcast[i], aj[i]);
      }
      __syncthreads();
    }
    // downdate the remaining column norms; recompute where cancellation hurts
    for (int l = warp; l < nloc; l += nw) {
      const int j = pos(l);
      if (j <= k || j >= ca) continue;
      const double *aj = colp(l);
      double nv = vn[l] - aj[k] * aj[k];
      if (!(nv > 1e-8 * vref[l])) {
        double s2 = 0.0;
        for (int i = k + 1 + lane; i < ra; i += 32) s2 = fma(aj[i], aj[i], s2);
        nv = wsum(s2);
        if (lane == 0) vref[l] = nv;
      }
      if (lane == 0) vn[l] = fmax(nv, 0.0);
    }
    __syncthreads();
  }
  // Householder vectors, R, the permutation, the rank; B = [R11 R12]^T
  for (int l = 0; l < nloc; ++l) {
    const int j = pos(l);
    if (j >= ca) break;
    const double *cl = colp(l);
    if (!GCOLS)
      for (int i = threadIdx.x; i < ra; i += blockDim.x) A[(int64_t)j * ra + i] = cl[i];
    if (threadIdx.x == 0) perm[j] = pl[l];
    for (int b = threadIdx.x; b < ca; b += blockDim.x) B[(int64_t)b * ca + j] = (b <= j && b < rank) ? cl[b] : 0.0;
  }
  if (crank == 0 && threadIdx.x == 0) perm[ca] = rank;
  cluster.sync();  // no CTA leaves while another may still read its shared memory
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
// returns |g| / sqrt(a b) of a rotated pair, -1 when the pair is left alone
__device__ __forceinline__ float jacobi_pair(double *ap, double *aq, double *jp, double *jq, int n, int nj,
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
  if (!(ga * ga > tol2 * (al * be)) || !(fabs(ga) > abs_floor)) return -1.0f;
  const float ratio = (float)(fabs(ga) / sqrt(al * be));
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
  return ratio;
}

// One job per cluster (cluster size chosen at launch); the pairs of a round
// are spread over all warps of the cluster, rounds separated by the hardware
// cluster barrier.
__global__ void __launch_bounds__(JAC_THREADS, 2)
    jacobi_kernel(const SvdJob *__restrict__ jobs, const int *__restrict__ order, double *__restrict__ work,
                  int *__restrict__ iwork, double *__restrict__ sv, int *err, int jm_init) {
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
  __shared__ int flag, local_changed, sweep_rmax, cl_rmax;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  // pair k of a round goes to CTA k mod csize: the FP64 work of a round is
  // spread over every SM of the cluster (blocked by CTA it piled up on the
  // first few while the others waited at the barrier)
  const int gw = warp * csize + crank, gnw = csize * nw;
  const int64_t nn = (int64_t)n * n, nb = (int64_t)nr * n;
  if (!jm_init) {
    for (int64_t e = (int64_t)crank * blockDim.x + threadIdx.x; e < nn; e += (int64_t)csize * blockDim.x)
      Jm[e] = (e / n == e % n) ? 1.0 : 0.0;
  } else if (n < Jb.cols_a) {
    // the given rotations are cols_a x cols_a (leading dimension cols_a);
    // their n x n block moves to leading dimension n through the x_off area
    double *tmp = work + Jb.x_off;
    for (int64_t e = (int64_t)crank * blockDim.x + threadIdx.x; e < nn; e += (int64_t)csize * blockDim.x)
      tmp[e] = Jm[(e / n) * Jb.cols_a + e % n];
    cluster.sync();
    for (int64_t e = (int64_t)crank * blockDim.x + threadIdx.x; e < nn; e += (int64_t)csize * blockDim.x)
      Jm[e] = tmp[e];
  }
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
  int *rmax0 = cluster.map_shared_rank(&cl_rmax, 0);
  bool converged = (n < 2);
  int sweep = 0;
  for (; sweep < 40 && !converged; ++sweep) {
    if (threadIdx.x == 0) {
      local_changed = 0;
      sweep_rmax = 0;
    }
    if (crank == 0 && threadIdx.x == 0) {
      flag = 0;
      cl_rmax = 0;
    }
    cluster.sync();
    bool any = false;
    float rmax = 0.0f;
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      for (int k = gw; k < np / 2; k += gnw) {
        const int i1 = k, i2 = np - 1 - k;
        const int p = i1 == 0 ? 0 : 1 + (i1 - 1 + rnd) % (np - 1);
        const int q = i2 == 0 ? 0 : 1 + (i2 - 1 + rnd) % (np - 1);
        if (p >= n || q >= n) continue;
        const float r = jacobi_pair(B + (int64_t)p * nr, B + (int64_t)q * nr, Jm + (int64_t)p * n,
                                    Jm + (int64_t)q * n, nr, n, lane, tol2, abs_floor);
        if (r >= 0.0f) {
          any = true;
          rmax = fmaxf(rmax, r);
        }
      }
      cluster.sync();
    }
    if (any && lane == 0) local_changed = 1;
    if (lane == 0) atomicMax(&sweep_rmax, __float_as_int(rmax));  // non-negative floats order as ints
    __syncthreads();
    if (threadIdx.x == 0) {
      if (local_changed) atomicOr(flag0, 1);
      atomicMax(rmax0, sweep_rmax);
    }
    cluster.sync();
    // quadratic convergence: after a sweep whose rotations were all below
    // |g| / sqrt(a b) = 1e-9 the overlaps left are of order n 1e-18, under
    // the threshold, so the sweep that would only confirm it is skipped
    converged = (*flag0 == 0) || (__int_as_float(*rmax0) < 1e-9f);
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

// The FP32 stage only preconditions the FP64 one: once a sweep's largest
// rotation (|cos| between two columns) is below J32_PRECOND_R, the columns
// are orthogonal to about its square, the level of FP32 rounding itself, and
// the FP64 stage starts from there whatever further FP32 sweeps would do
// (the maximum over all pairs of the FP32 rounding noise in the overlaps can
// otherwise keep the tighter test open for several sweeps).
constexpr float J32_PRECOND_R = 1e-3f;

// the FP32 stage's sweep count of a job, in the slot after its rank and FP64
// sweep count (read back for the statistics only)
__device__ __forceinline__ void iwork32_sweeps(const int *iwork, const SvdJob &J, int sweep) {
  const_cast<int *>(iwork)[J.perm_off + J.cols_a + 2] = sweep;
}

// FP32 stage (see jacobi32_block_kernel) for sector matrices too large for
// the block kernels: the cyclic tournament of jacobi_kernel on FP32 copies
// of B and of the rotations, kept in the job's x_off area (cols_a x cols_a
// doubles, free until the Newton-Schulz step), one pair per warp, rounds
// separated by the cluster barrier.  Ends by writing the rotations to V
// (FP64, leading dimension cols_a) over the identity already there.
// A pair's columns are read and written in batches of J32_BATCH elements per
// lane whose loads are all issued before they are used: with the columns in
// L2 or HBM, a plain strided loop waits on the load latency once per 32
// elements of each column.
constexpr int J32_BATCH = 8;
constexpr int J64_BATCH = 8;

__device__ __forceinline__ void dots32(const float *xp, const float *xq, int len, int lane, float &a, float &b,
                                       float &g) {
  // two batches in flight; each lane adds its elements in index order
  for (int i0 = 0; i0 < len; i0 += 64 * J32_BATCH) {
    float u[2 * J32_BATCH], v[2 * J32_BATCH];
#pragma unroll
    for (int r = 0; r < 2 * J32_BATCH; ++r) {
      const int i = i0 + lane + 32 * r;
      u[r] = i < len ? xp[i] : 0.f;
      v[r] = i < len ? xq[i] : 0.f;
    }
#pragma unroll
    for (int r = 0; r < 2 * J32_BATCH; ++r) {
      a = fmaf(u[r], u[r], a);
      b = fmaf(v[r], v[r], b);
      g = fmaf(u[r], v[r], g);
    }
  }
}

// the rotation of a pair of B columns (length len) and of the same pair of
// rotation columns (length lenv <= len) in one pass
__device__ __forceinline__ void rot32x2(float *xp, float *xq, int len, float *vp, float *vq, int lenv, int lane,
                                        float c, float sn) {
  for (int i0 = 0; i0 < len; i0 += 32 * J32_BATCH) {
    float u[J32_BATCH], v[J32_BATCH], y[J32_BATCH], z[J32_BATCH];
#pragma unroll
    for (int r = 0; r < J32_BATCH; ++r) {
      const int i = i0 + lane + 32 * r;
      u[r] = i < len ? xp[i] : 0.f;
      v[r] = i < len ? xq[i] : 0.f;
      y[r] = i < lenv ? vp[i] : 0.f;
      z[r] = i < lenv ? vq[i] : 0.f;
    }
#pragma unroll
    for (int r = 0; r < J32_BATCH; ++r) {
      const int i = i0 + lane + 32 * r;
      if (i < len) {
        xp[i] = c * u[r] - sn * v[r];
        xq[i] = fmaf(sn, u[r], c * v[r]);
      }
      if (i < lenv) {
        vp[i] = c * y[r] - sn * z[r];
        vq[i] = fmaf(sn, y[r], c * z[r]);
      }
    }
  }
}

__global__ void __launch_bounds__(JAC_THREADS, 2)
    jacobi32_kernel(const SvdJob *__restrict__ jobs, const int *__restrict__ order, double *__restrict__ work,
                    const int *__restrict__ iwork) {
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int csize = (int)cluster.num_blocks();
  const SvdJob Jb = jobs[order[blockIdx.x / csize]];
  const int nr = Jb.cols_a;
  const int n = iwork[Jb.perm_off + Jb.cols_a];
  float *B32 = reinterpret_cast<float *>(work + Jb.x_off);  // nr x n, then n x n rotations
  float *V32 = B32 + (int64_t)nr * n;
  const double *Bg = work + Jb.b_off;
  double *Vg = work + Jb.j_off;
  __shared__ int flag, local_changed, sweep_rmax, cl_rmax;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int gw = warp * csize + crank, gnw = csize * nw;
  const int64_t stride = (int64_t)csize * blockDim.x, e0 = (int64_t)crank * blockDim.x + threadIdx.x;
  if (n < 2) return;  // uniform over the cluster
  for (int64_t e = e0; e < (int64_t)nr * n; e += stride) B32[e] = (float)Bg[e];
  for (int64_t e = e0; e < (int64_t)n * n; e += stride) V32[e] = (e / n == e % n) ? 1.0f : 0.0f;
  const float tol = sqrtf((float)nr) * FLT_EPSILON;
  const int np = n + (n & 1);
  int *flag0 = cluster.map_shared_rank(&flag, 0);
  int *rmax0 = cluster.map_shared_rank(&cl_rmax, 0);
  auto wsumf = [](float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  };
  bool converged = false;
  int sweep = 0;
  for (; sweep < 15 && !converged; ++sweep) {
    if (threadIdx.x == 0) {
      local_changed = 0;
      sweep_rmax = 0;
    }
    if (crank == 0 && threadIdx.x == 0) {
      flag = 0;
      cl_rmax = 0;
    }
    cluster.sync();
    bool any = false;
    float rmax = 0.f;
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      for (int k = gw; k < np / 2; k += gnw) {
        const int i1 = k, i2 = np - 1 - k;
        const int p = i1 == 0 ? 0 : 1 + (i1 - 1 + rnd) % (np - 1);
        const int q = i2 == 0 ? 0 : 1 + (i2 - 1 + rnd) % (np - 1);
        if (p >= n || q >= n) continue;
        float *xp = B32 + (int64_t)p * nr, *xq = B32 + (int64_t)q * nr;
        float a = 0.f, b = 0.f, g = 0.f;
        dots32(xp, xq, nr, lane, a, b, g);
        a = wsumf(a);
        b = wsumf(b);
        g = wsumf(g);
        if (!(a > 0.f) || !(b > 0.f)) continue;
        const float ratio = fabsf(g) / sqrtf(a) / sqrtf(b);
        if (!(ratio > tol)) continue;
        const float z = (b - a) / (2.0f * g);
        const float t = z == 0.f ? 1.0f : copysignf(1.0f, z) / (fabsf(z) + sqrtf(fmaf(z, z, 1.0f)));
        if (!(fabsf(t) >= FLT_MIN) || !isfinite(t)) continue;
        const float c = rsqrtf(fmaf(t, t, 1.0f)), sn = c * t;
        rot32x2(xp, xq, nr, V32 + (int64_t)p * n, V32 + (int64_t)q * n, n, lane, c, sn);
        any = true;
        rmax = fmaxf(rmax, ratio);
      }
      cluster.sync();
    }
    if (any && lane == 0) local_changed = 1;
    if (lane == 0) atomicMax(&sweep_rmax, __float_as_int(rmax));
    __syncthreads();
    if (threadIdx.x == 0) {
      if (local_changed) atomicOr(flag0, 1);
      atomicMax(rmax0, sweep_rmax);
    }
    cluster.sync();
    const float r = __int_as_float(*rmax0);
    converged = (*flag0 == 0) || ((float)n * r * r < tol) || r < J32_PRECOND_R;
    cluster.sync();
  }
  if (crank == 0 && threadIdx.x == 0) iwork32_sweeps(iwork, Jb, sweep);
  for (int64_t e = e0; e < (int64_t)n * n; e += stride) {
    const int64_t j = e / n, i = e - j * n;
    Vg[j * nr + i] = (double)V32[e];
  }
}

// ------------------------------------------------- block Jacobi (shared memory)
// Same rotations as jacobi_kernel, ordered by blocks so that the columns stay
// in shared memory.  The rank-n columns of B (and of Jm) are cut into 2C
// blocks of bw columns, C the cluster size; CTA c holds the blocks at
// tournament positions c and 2C-1-c.  In a round a CTA rotates every column
// of one of its blocks against every column of the other (bw sub-rounds of
// bw disjoint pairs, separated by __syncthreads); then the blocks move one
// position along the circle (position 0 stays), each CTA writing its two
// blocks into the receiving CTAs' second buffer through distributed shared
// memory, so that after 2C-1 rounds every two blocks have met once.  The pairs
// inside each block are taken in the first round of a sweep.  A sweep costs
// 2C-1 cluster barriers instead of n-1, and no column leaves the SMs.
//
// FP64 arithmetic is the scarce resource here, so the rotations are the
// scaled ("fast") form: column j is held as d_j x_j, a rotation changes the
// x of both columns by one FMA per element and multiplies both d by cos; the
// squared column norms are carried along in closed form (recomputed from the
// data when cancellation makes the update inaccurate, and at every sweep,
// when d is folded back into the columns), so each pair needs one dot
// product instead of three.
constexpr int BJ_THREADS = 256;  // largest block; groups launch one warp per pair of a sub-round
constexpr int BJ_REG = 10;  // rows per lane held in registers: columns of up to 320 rows

__device__ __forceinline__ int bj_block_at(int pos, int r, int P) {
  return pos == 0 ? 0 : 1 + (pos - 1 + (P - 1) - r % (P - 1)) % (P - 1);
}

// The pairs of a sub-round are rotated in three phases (separated by
// __syncthreads): each warp forms the overlap of its pair's columns (one dot
// product, the columns stay in its registers); one lane per pair then
// computes the rotation (bj_rotation: FP64 scalar work is done once per pair,
// not by 32 lanes); each warp finally updates its pair.  Columns are padded
// with zero rows to nreg*32 (B) and nregj*32 (Jm), so no loop carries bounds
// checks.

struct BjPair {   // per pair of a sub-round, in shared memory
  double g;       // overlap of the stored (unscaled) columns
  double cp, cq;  // update coefficients
  int i, j;       // column indices within the two blocks (-1: no pair)
  int rot;        // 1 rotate, 2 rotate and recompute both norms from the data
};

// phase 2 for one pair: norms a, b and scales d1, d2 in, updated in place.
// The tests and the angle use exponents and FP32 mantissas; FP64 is spent
// only where the rotation must be exact: cos (Newton), the update
// coefficients and the carried norms.
__device__ __forceinline__ int bj_rotation(double graw, double &a, double &b, double &d1, double &d2, float log2_tol2,
                                           Split fl, double &cp, double &cq, float &lrel_out) {
  const double g = (d1 * d2) * graw;
  const Split sg = split_f64(g), sa = split_f64(a), sb = split_f64(b);
  if (sg.m == 0.0f || sa.m == 0.0f || sb.m == 0.0f) return 0;
  const float mg = fabsf(sg.m);
  // rotate iff g^2 > tol^2 a b and |g| > abs_floor
  const float lrel = (float)(2 * sg.e - sa.e - sb.e) + __log2f(mg * mg / (sa.m * sb.m));
  if (!(lrel > log2_tol2)) return 0;
  lrel_out = lrel;
  if (fl.m != 0.0f && !((float)(sg.e - fl.e) + __log2f(mg / fl.m) > 0.0f)) return 0;
  // z = (b - a) / (2 g) in FP32 from exponents and mantissas
  const Split sn = split_f64(b - a);
  float tf;
  if (sn.m == 0.0f) {
    tf = copysignf(1.0f, sg.m);
  } else {
    const int ez = sn.e - sg.e - 1;
    if (ez > 120) return 0;  // angle below 2^-120: nothing to rotate
    const float mz = __fdividef(sn.m, sg.m);
    const float z = ez < -120 ? copysignf(0.0f, mz) : ldexpf(mz, ez);
    const float az = fabsf(z);
    tf = az > 1e15f ? __fdividef(0.5f, z) : copysignf(__frcp_rn(az + __fsqrt_rn(fmaf(z, z, 1.0f))), z);
    if (!(fabsf(tf) >= 1.17549435e-38f)) return 0;  // below FP32 normals: no rotation
  }
  const double t = f64_of(tf);
  // cos = 1/sqrt(1 + t^2): FP32 estimate, two Newton steps in FP64
  const double xx = fma(t, t, 1.0), h = 0.5 * xx;
  double cs = f64_of(rsqrtf(fmaf(tf, tf, 1.0f)));
  cs = cs * fma(-h * cs, cs, 1.5);
  cs = cs * fma(-h * cs, cs, 1.5);
  // x_p <- x_p - t (d_q/d_p) x_q,  x_q <- x_q + t (d_p/d_q) x_p,  d <- cos d
  cp = -t * (d2 * recip_split(d1));
  cq = t * (d1 * recip_split(d2));
  // new squared norms cos^2 (a -+ 2 t g + t^2 b); recomputed from the data
  // when one falls below 2^-20 of its old value (cancellation)
  const double c2 = cs * cs, t2 = t * t, tg = t * g;
  const double a2 = c2 * fma(-2.0, tg, fma(t2, b, a)), b2 = c2 * fma(2.0, tg, fma(t2, a, b));
  d1 *= cs;
  d2 *= cs;
  a = a2;
  b = b2;
  // cancellation: a new norm far below its own old value.  For the
  // rotation that zeroes g, |t g| and t^2 b are at most of order a (and
  // |t g|, t^2 a at most of order b), so only a2 << a (b2 << b) loses
  // digits; a column much smaller than its partner is not a cancellation.
  const Split s2a = split_f64(a2), s2b = split_f64(b2);
  const bool oka = s2a.m > 0.0f && s2a.e > sa.e - 20, okb = s2b.m > 0.0f && s2b.e > sb.e - 20;
  return (oka && okb) ? 1 : 2;
}

// jm_init = 1: the rotations start from the matrix at j_off (cols_a x
// cols_a, column-major: the FP32 stage's orthogonalised rotations) instead
// of the identity; B then holds the preconditioned columns
__global__ void __launch_bounds__(BJ_THREADS, 2)
    jacobi_block_kernel(const SvdJob *__restrict__ jobs, const int *__restrict__ order, double *__restrict__ work,
                        int *__restrict__ iwork, double *__restrict__ sv, int *err, int jm_init) {
  extern __shared__ __align__(16) double bj_sm[];
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int C = (int)cluster.num_blocks();
  const SvdJob Jb = jobs[order[blockIdx.x / C]];
  const int nr = Jb.cols_a;                       // rows of B
  const int n = iwork[Jb.perm_off + Jb.cols_a];   // columns of B: numerical rank
  const int P = 2 * C;
  const int bw = (n + P - 1) / P;                 // columns per block
  const int nreg = (nr + 31) >> 5, nregj = (n + 31) >> 5;
  const int ldb = 32 * nreg, ldj = 32 * nregj;    // padded with zero rows
  // one block: B columns, Jm columns, squared norms, scales
  const int offJ = bw * ldb, offN = offJ + bw * ldj, offD = offN + bw;
  const int slot = (offD + bw + 1) & ~1;          // even: blocks start on 16 bytes
  __shared__ double fro_part[JAC_MAX_CLUSTER];
  __shared__ double wred[BJ_THREADS / 32];
  __shared__ int flag, local_changed;
  // largest rotation of the sweep, 64 log2(g^2 / (a b)), and its cluster max
  __shared__ int sweep_lmax, cl_lmax;
  __shared__ BjPair pairs[BJ_THREADS / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double *Bg = work + Jb.b_off;
  double *Jg = work + Jb.j_off;
  const int pos[2] = {crank, P - 1 - crank};
  auto slotp = [&](int buf, int which) { return bj_sm + (buf * 2 + which) * slot; };
  auto valid = [&](int k) { return max(0, min(bw, n - k * bw)); };
  if (nreg > BJ_REG || nregj > BJ_REG) {  // excluded by the host; never rotate out of bounds
    if (crank == 0 && threadIdx.x == 0) atomicOr(err, IDMRG_DEV_ERR_JACOBI);
    return;
  }

  // load: block k = pos at the start of a sweep; Jm starts as the identity
  double fro = 0.0;
  for (int w = 0; w < 2; ++w) {
    const int k = pos[w], nv = valid(k);
    double *sb = slotp(0, w);
    for (int e = threadIdx.x; e < offJ; e += blockDim.x) {
      const int j = e / ldb, i = e - j * ldb;
      const double v = (j < nv && i < nr) ? Bg[(int64_t)(k * bw + j) * nr + i] : 0.0;
      sb[e] = v;
      fro = fma(v, v, fro);
    }
    for (int e = threadIdx.x; e < bw * ldj; e += blockDim.x) {
      const int j = e / ldj, i = e - j * ldj;
      double v = 0.0;
      if (j < nv && i < n) v = jm_init ? Jg[(int64_t)(k * bw + j) * nr + i] : (i == k * bw + j ? 1.0 : 0.0);
      sb[offJ + e] = v;
    }
    for (int j = threadIdx.x; j < bw; j += blockDim.x) sb[offD + j] = 1.0;
  }
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
  for (int q = 0; q < C; ++q) fro += fp0[q];
  cluster.sync();
  // rotation threshold sqrt(rows) eps, as a log2 of its square, and the
  // absolute floor 4 eps^2 ||B||_F^2 (see jacobi_kernel)
  const float log2_tol2 = __log2f((float)nr) - 104.0f;  // log2(nr eps^2), eps = 2^-52
  const Split floor_split = split_f64(4.0 * DBL_EPSILON * DBL_EPSILON * fro);
  int *flag0 = cluster.map_shared_rank(&flag, 0);
  int *lmax0 = cluster.map_shared_rank(&cl_lmax, 0);
  bool converged = (n < 2);
  // Cyclic Jacobi converges quadratically at the end: after a sweep in which
  // no rotation exceeded |g| / sqrt(a b) = r = 1e-9, every pair is left with
  // an overlap of order n r^2 <= 1e-15 relative, below the threshold
  // sqrt(rows) eps, so the sweep that would only confirm it is skipped.
  const int small_key = (int)(64.0f * -59.8f);  // 64 log2(1e-18)
  int sweep = 0, cur = 0;
  // fold the scales into the columns of the home blocks and recompute norms
  auto fold = [&]() {
    for (int t = warp; t < 2 * bw; t += nw) {
      const int w = t >= bw ? 1 : 0, j = t - w * bw;
      double *sb = slotp(cur, w);
      const double d = sb[offD + j];
      double *bj = sb + j * ldb, *jj = sb + offJ + j * ldj;
      double s = 0.0;
      for (int i = lane; i < ldb; i += 32) {
        const double v = bj[i] * d;
        bj[i] = v;
        s = fma(v, v, s);
      }
      for (int i = lane; i < ldj; i += 32) jj[i] *= d;
      s = wsum(s);
      __syncwarp();
      if (lane == 0) {
        sb[offN + j] = s;
        sb[offD + j] = 1.0;
      }
    }
    __syncthreads();
  };
  // one sub-round: pairs (s0 col pi[k], s1 col pj[k]), k < np, one warp each
  auto subround = [&](double *s0, double *s1, int np) -> bool {
    const bool mine = warp < np && pairs[warp].i >= 0;
    double x[BJ_REG], y[BJ_REG];
    double *xp = nullptr, *xq = nullptr;
    if (mine) {
      xp = s0 + pairs[warp].i * ldb;
      xq = s1 + pairs[warp].j * ldb;
      double ga = 0.0;
#pragma unroll
      for (int r = 0; r < BJ_REG; ++r)
        if (r < nreg) {
          x[r] = xp[lane + 32 * r];
          y[r] = xq[lane + 32 * r];
          ga = fma(x[r], y[r], ga);
        }
      ga = wsum(ga);
      if (lane == 0) pairs[warp].g = ga;
    }
    __syncthreads();
    if (warp == 0 && lane < np && pairs[lane].i >= 0) {
      BjPair &pr = pairs[lane];
      double a = s0[offN + pr.i], b = s1[offN + pr.j], d1 = s0[offD + pr.i], d2 = s1[offD + pr.j];
      double cp = 0.0, cq = 0.0;
      float lr = -1000.0f;
      pr.rot = bj_rotation(pr.g, a, b, d1, d2, log2_tol2, floor_split, cp, cq, lr);
      if (pr.rot) atomicMax(&sweep_lmax, (int)(lr * 64.0f));
      if (pr.rot) {
        pr.cp = cp;
        pr.cq = cq;
        s0[offN + pr.i] = a;
        s1[offN + pr.j] = b;
        s0[offD + pr.i] = d1;
        s1[offD + pr.j] = d2;
      }
    }
    __syncthreads();
    bool rot = false;
    if (mine && pairs[warp].rot) {
      rot = true;
      const double cp = pairs[warp].cp, cq = pairs[warp].cq;
#pragma unroll
      for (int r = 0; r < BJ_REG; ++r)
        if (r < nreg) {
          const double u = fma(cp, y[r], x[r]), v = fma(cq, x[r], y[r]);
          x[r] = u;
          y[r] = v;
          xp[lane + 32 * r] = u;
          xq[lane + 32 * r] = v;
        }
      double *jp = s0 + offJ + pairs[warp].i * ldj, *jq = s1 + offJ + pairs[warp].j * ldj;
#pragma unroll
      for (int r = 0; r < BJ_REG; ++r)
        if (r < nregj) {
          const double u = jp[lane + 32 * r], v = jq[lane + 32 * r];
          jp[lane + 32 * r] = fma(cp, v, u);
          jq[lane + 32 * r] = fma(cq, u, v);
        }
      if (pairs[warp].rot == 2) {  // cancellation: norms from the rotated data
        double np2 = 0.0, nq2 = 0.0;
#pragma unroll
        for (int r = 0; r < BJ_REG; ++r)
          if (r < nreg) {
            np2 = fma(x[r], x[r], np2);
            nq2 = fma(y[r], y[r], nq2);
          }
        np2 = wsum(np2);
        nq2 = wsum(nq2);
        if (lane == 0) {
          const double dp = s0[offD + pairs[warp].i], dq = s1[offD + pairs[warp].j];
          s0[offN + pairs[warp].i] = dp * dp * np2;
          s1[offN + pairs[warp].j] = dq * dq * nq2;
        }
      }
    }
    __syncthreads();
    return rot;
  };
  for (; sweep < 40 && !converged; ++sweep) {
    fold();
    if (threadIdx.x == 0) {
      local_changed = 0;
      sweep_lmax = INT_MIN;
    }
    if (crank == 0 && threadIdx.x == 0) {
      flag = 0;
      cl_lmax = INT_MIN;
    }
    cluster.sync();
    bool any = false;
    for (int rnd = 0; rnd < P - 1; ++rnd) {
      double *st0 = slotp(cur, 0), *st1 = slotp(cur, 1);
      const int nv0 = valid(bj_block_at(pos[0], rnd, P)), nv1 = valid(bj_block_at(pos[1], rnd, P));
      if (rnd == 0) {
        // pairs inside each block: round-robin over bp slots, one block at a
        // time (a sub-round's pairs share the two block pointers)
        const int bp = bw + (bw & 1), half = bp / 2, bm = bp - 1;
        for (int w = 0; w < 2; ++w) {
          const int nv = w ? nv1 : nv0;
          double *sb = w ? st1 : st0;
          for (int sr = 0; sr < bm; ++sr) {
            for (int c0 = 0; c0 < half; c0 += nw) {
              const int np = min(nw, half - c0);
              if (threadIdx.x < np) {
                const int i = c0 + threadIdx.x;
                int p = 0, q;
                if (i != 0) {
                  p = i - 1 + sr;
                  p = 1 + (p >= bm ? p - bm : p);
                }
                q = bp - 2 - i + sr;
                q = 1 + (q >= bm ? q - bm : q);
                const bool ok = p < nv && q < nv;
                pairs[threadIdx.x].i = ok ? p : -1;
                pairs[threadIdx.x].j = ok ? q : -1;
                pairs[threadIdx.x].rot = 0;
              }
              __syncthreads();
              any |= subround(sb, sb, np);
            }
          }
        }
      }
      // every column of the first block against every column of the second
      for (int sr = 0; sr < bw; ++sr) {
        for (int c0 = 0; c0 < bw; c0 += nw) {
          const int np = min(nw, bw - c0);
          if (threadIdx.x < np) {
            const int i = c0 + threadIdx.x;
            int j = i + sr;
            if (j >= bw) j -= bw;
            const bool ok = i < nv0 && j < nv1;
            pairs[threadIdx.x].i = ok ? i : -1;
            pairs[threadIdx.x].j = ok ? j : -1;
            pairs[threadIdx.x].rot = 0;
          }
          __syncthreads();
          any |= subround(st0, st1, np);
        }
      }
      if (C > 1) {
        // move both blocks one position on: position 0 stays, P-1 goes to 1
        for (int w = 0; w < 2; ++w) {
          const int dpn = pos[w] == 0 ? 0 : (pos[w] == P - 1 ? 1 : pos[w] + 1);
          const int drank = dpn < C ? dpn : P - 1 - dpn, dw = dpn < C ? 0 : 1;
          double2 *dst = reinterpret_cast<double2 *>(cluster.map_shared_rank(slotp(cur ^ 1, dw), drank));
          const double2 *src = reinterpret_cast<const double2 *>(w ? st1 : st0);
          for (int e = threadIdx.x; e < slot / 2; e += blockDim.x) dst[e] = src[e];
        }
        cluster.sync();
        cur ^= 1;
      }
    }
    if (any && lane == 0) local_changed = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
      if (local_changed) atomicOr(flag0, 1);
      atomicMax(lmax0, sweep_lmax);
    }
    cluster.sync();
    converged = (*flag0 == 0) || (*lmax0 < small_key);
    cluster.sync();
  }
  fold();
  if (!converged && crank == 0 && threadIdx.x == 0) atomicOr(err, IDMRG_DEV_ERR_JACOBI);
  if (crank == 0 && threadIdx.x == 0) iwork[Jb.perm_off + Jb.cols_a + 1] = sweep;
  // after whole sweeps every block is back at its starting position: singular
  // values, normalised columns of B and the columns of Jm go back to memory
  for (int w = 0; w < 2; ++w) {
    const int k = pos[w], nv = valid(k);
    const double *sb = slotp(cur, w);
    for (int j = warp; j < nv; j += nw) {
      const double *bj = sb + j * ldb;
      const double s = sqrt(sb[offN + j]);
      const int g = k * bw + j;
      if (lane == 0) sv[Jb.sv_off + g] = s;
      const double inv = s > 0.0 ? 1.0 / s : 0.0;
      for (int i = lane; i < nr; i += 32) Bg[(int64_t)g * nr + i] = bj[i] * inv;
      for (int i = lane; i < n; i += 32) Jg[(int64_t)g * n + i] = sb[offJ + j * ldj + i];
    }
  }
  if (crank == 0)
    for (int j = n + (int)threadIdx.x; j < Jb.cols_a; j += blockDim.x) sv[Jb.sv_off + j] = 0.0;
}

// Element arithmetic of the FP64 stage below in pairs of FP32 numbers
// (x = h + l, |l| <= ulp(h) / 2: 48 significant bits), for GB300, whose
// SMs issue 64 FP32 FMAs per FP64 FMA.  The products are exact by FMA
// (Dekker's two-product), the sums by Knuth's two-sum; the explicit _rn
// intrinsics keep the compiler from contracting them.  The dot products and
// rotations of the sweeps run in this arithmetic; column norms, scales and
// the rotation scalars stay in FP64.
struct __align__(8) DF2 {
  float h, l;
};
__device__ __forceinline__ DF2 df_of(double x) {
  DF2 r;
  r.h = __double2float_rn(x);
  r.l = __double2float_rn(x - (double)r.h);
  return r;
}
__device__ __forceinline__ double df_to(DF2 x) { return (double)x.h + (double)x.l; }
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (sh, sl) += a b, the accumulator left unnormalised (|sl| grows by at most
// one ulp of sh per term; it is folded in by df_wsum)
__device__ __forceinline__ void df_dot_acc(DF2 a, DF2 b, float &sh, float &sl) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  float s, t;
  two_sum(sh, p, s, t);
  sl = __fadd_rn(sl, __fadd_rn(t, e));
  sh = s;
}
// u + c v, renormalised
__device__ __forceinline__ DF2 df_axpy(DF2 c, DF2 v, DF2 u) {
  const float p = __fmul_rn(c.h, v.h);
  float e = __fmaf_rn(c.h, v.h, -p);
  e = __fmaf_rn(c.h, v.l, e);
  e = __fmaf_rn(c.l, v.h, e);
  float s, t;
  two_sum(u.h, p, s, t);
  t = __fadd_rn(t, __fadd_rn(u.l, e));
  DF2 r;
  r.h = __fadd_rn(s, t);
  r.l = __fsub_rn(t, __fsub_rn(r.h, s));
  return r;
}
// warp sum of pair accumulators; every lane gets the same value (each
// butterfly step adds the same two pairs on both partners)
__device__ __forceinline__ double df_wsum(float h, float l) {
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
    float s, e;
    two_sum(h, oh, s, e);
    l = __fadd_rn(__fadd_rn(l, ol), e);
    h = s;
  }
  return (double)h + (double)l;
}

// FP64 stage for sectors beyond the block kernels: the cyclic tournament of
// jacobi_kernel (columns in global memory, one pair per warp, rounds
// separated by the cluster barrier) with the scaled rotations and tracked
// column norms of jacobi_block_kernel (bj_rotation): one dot product and one
// FMA per element and column instead of three dot products and two
// operations.  Column scales and squared norms live in the job's w_off area
// (free once B holds X); every sweep starts by folding the scales back into
// the columns and recomputing their norms (in FP64).  PAIRS: B and the
// rotations are held as FP32 pairs (in place, 8 bytes an element as before)
// from the first sweep to the last, dot products and rotations run in pair
// arithmetic, and a rotation is applied when its relative overlap exceeds
// sqrt(rows) 2^-48 instead of sqrt(rows) 2^-52; the convergence test (all
// rotations of a sweep below 1e-9) is the same.
template <bool PAIRS>
__global__ void __launch_bounds__(JAC_THREADS, 1)
    jacobi_scaled_kernel(const SvdJob *__restrict__ jobs, const int *__restrict__ order, double *__restrict__ work,
                         int *__restrict__ iwork, double *__restrict__ sv, int *err, int jm_init) {
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int csize = (int)cluster.num_blocks();
  const SvdJob Jb = jobs[order[blockIdx.x / csize]];
  const int nr = Jb.cols_a;                       // rows of B
  const int n = iwork[Jb.perm_off + Jb.cols_a];   // columns of B: numerical rank
  double *B = work + Jb.b_off;
  double *Jm = work + Jb.j_off;
  DF2 *Bp = reinterpret_cast<DF2 *>(B);           // the same memory as pairs (PAIRS)
  DF2 *Jp = reinterpret_cast<DF2 *>(Jm);
  double *dsc = work + Jb.w_off, *nrm = dsc + n;  // scale d_j and squared norm of column j
  __shared__ double fro_part[JAC_MAX_CLUSTER];
  __shared__ double wred[JAC_THREADS / 32];
  __shared__ int flag, local_changed, sweep_lmax, cl_lmax;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int gw = warp * csize + crank, gnw = csize * nw;
  const int64_t nn = (int64_t)n * n, nb = (int64_t)nr * n;
  const int64_t stride = (int64_t)csize * blockDim.x, e0 = (int64_t)crank * blockDim.x + threadIdx.x;
  if (!jm_init) {
    for (int64_t e = e0; e < nn; e += stride) Jm[e] = (e / n == e % n) ? 1.0 : 0.0;
  } else if (n < Jb.cols_a) {
    // the given rotations are cols_a x cols_a (leading dimension cols_a);
    // their n x n block moves to leading dimension n through the x_off area
    double *tmp = work + Jb.x_off;
    for (int64_t e = e0; e < nn; e += stride) tmp[e] = Jm[(e / n) * Jb.cols_a + e % n];
    cluster.sync();
    for (int64_t e = e0; e < nn; e += stride) Jm[e] = tmp[e];
  }
  for (int64_t e = e0; e < n; e += stride) dsc[e] = 1.0;
  double fro = 0.0;
  for (int64_t e = e0; e < nb; e += stride) {
    const double v = B[e];
    fro = fma(v, v, fro);
    if (PAIRS) Bp[e] = df_of(v);  // each element is read and rewritten by the same thread
  }
  if (PAIRS)
    for (int64_t e = e0; e < nn; e += stride) Jp[e] = df_of(Jm[e]);
  fro = wsum(fro);
  if (lane == 0) wred[warp] = fro;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < nw; ++q) t += wred[q];
    *cluster.map_shared_rank(&fro_part[crank], 0) = t;
  }
  cluster.sync();
  const double *fp0 = cluster.map_shared_rank(fro_part, 0);
  fro = 0.0;
  for (int q = 0; q < csize; ++q) fro += fp0[q];
  cluster.sync();
  // log2(nr eps^2), eps = 2^-52 (FP64) or 2^-48 (pairs)
  const float log2_tol2 = __log2f((float)nr) - (PAIRS ? 96.0f : 104.0f);
  const Split floor_split = split_f64(4.0 * DBL_EPSILON * DBL_EPSILON * fro);
  const int small_key = (int)(64.0f * -59.8f);        // 64 log2(1e-18): see jacobi_block_kernel
  const int np = n + (n & 1);
  int *flag0 = cluster.map_shared_rank(&flag, 0);
  int *lmax0 = cluster.map_shared_rank(&cl_lmax, 0);
  // scales into the columns, exact squared norms
  auto fold = [&]() {
    for (int j = gw; j < n; j += gnw) {
      const double d = dsc[j];
      double s = 0.0;
      if (PAIRS) {
        DF2 *bj = Bp + (int64_t)j * nr, *jj = Jp + (int64_t)j * n;
        for (int i = lane; i < nr; i += 32) {
          const double v = df_to(bj[i]) * d;
          bj[i] = df_of(v);
          s = fma(v, v, s);
        }
        if (d != 1.0)
          for (int i = lane; i < n; i += 32) jj[i] = df_of(df_to(jj[i]) * d);
      } else {
        double *bj = B + (int64_t)j * nr, *jj = Jm + (int64_t)j * n;
        for (int i = lane; i < nr; i += 32) {
          const double v = bj[i] * d;
          bj[i] = v;
          s = fma(v, v, s);
        }
        for (int i = lane; i < n; i += 32) jj[i] *= d;
      }
      s = wsum(s);
      __syncwarp();
      if (lane == 0) {
        nrm[j] = s;
        dsc[j] = 1.0;
      }
    }
    cluster.sync();
  };
  bool converged = (n < 2);
  int sweep = 0;
  for (; sweep < 40 && !converged; ++sweep) {
    fold();
    if (threadIdx.x == 0) {
      local_changed = 0;
      sweep_lmax = INT_MIN;
    }
    if (crank == 0 && threadIdx.x == 0) {
      flag = 0;
      cl_lmax = INT_MIN;
    }
    cluster.sync();
    bool any = false;
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      for (int k = gw; k < np / 2; k += gnw) {
        const int i1 = k, i2 = np - 1 - k;
        const int p = i1 == 0 ? 0 : 1 + (i1 - 1 + rnd) % (np - 1);
        const int q = i2 == 0 ? 0 : 1 + (i2 - 1 + rnd) % (np - 1);
        if (p >= n || q >= n) continue;
        double ga;
        if (PAIRS) {
          const DF2 *xp = Bp + (int64_t)p * nr, *xq = Bp + (int64_t)q * nr;
          float sh = 0.0f, sl = 0.0f;
          for (int i0 = 0; i0 < nr; i0 += 64 * J64_BATCH) {
            DF2 u[2 * J64_BATCH], v[2 * J64_BATCH];
#pragma unroll
            for (int r = 0; r < 2 * J64_BATCH; ++r) {
              const int i = i0 + lane + 32 * r;
              u[r] = i < nr ? xp[i] : DF2{0.0f, 0.0f};
              v[r] = i < nr ? xq[i] : DF2{0.0f, 0.0f};
            }
#pragma unroll
            for (int r = 0; r < 2 * J64_BATCH; ++r) df_dot_acc(u[r], v[r], sh, sl);
          }
          ga = df_wsum(sh, sl);
        } else {
          const double *xp = B + (int64_t)p * nr, *xq = B + (int64_t)q * nr;
          ga = 0.0;
          // loads in batches of J64_BATCH per lane, two batches issued before
          // their FMAs; each lane still adds its elements in index order
          for (int i0 = 0; i0 < nr; i0 += 64 * J64_BATCH) {
            double u[2 * J64_BATCH], v[2 * J64_BATCH];
#pragma unroll
            for (int r = 0; r < 2 * J64_BATCH; ++r) {
              const int i = i0 + lane + 32 * r;
              u[r] = i < nr ? xp[i] : 0.0;
              v[r] = i < nr ? xq[i] : 0.0;
            }
#pragma unroll
            for (int r = 0; r < 2 * J64_BATCH; ++r) ga = fma(u[r], v[r], ga);
          }
          ga = wsum(ga);
        }
        double cp = 0.0, cq = 0.0;
        int rot = 0;
        if (lane == 0) {
          double a = nrm[p], b = nrm[q], d1 = dsc[p], d2 = dsc[q];
          float lr = -1000.0f;
          rot = bj_rotation(ga, a, b, d1, d2, log2_tol2, floor_split, cp, cq, lr);
          if (rot) {
            nrm[p] = a;
            nrm[q] = b;
            dsc[p] = d1;
            dsc[q] = d2;
            atomicMax(&sweep_lmax, (int)(lr * 64.0f));
            // a coefficient of 2^101 or more (or not finite) has no FP32
            // pair: report it (exponent bits, no FP64 instruction)
            if (PAIRS && (((__double2hiint(cp) >> 20) & 0x7ff) > 1023 + 100 ||
                          ((__double2hiint(cq) >> 20) & 0x7ff) > 1023 + 100))
              atomicOr(err, IDMRG_DEV_ERR_JACOBI);
          }
        }
        rot = __shfl_sync(0xffffffffu, rot, 0);
        if (!rot) continue;
        any = true;
        cp = __shfl_sync(0xffffffffu, cp, 0);
        cq = __shfl_sync(0xffffffffu, cq, 0);
        // B's and Jm's pair of columns in one pass (n <= nr): the four
        // columns' loads of a batch are issued together
        double np2 = 0.0, nq2 = 0.0;
        if (PAIRS) {
          const DF2 cpp = df_of(cp), cqp = df_of(cq);
          DF2 *xp = Bp + (int64_t)p * nr, *xq = Bp + (int64_t)q * nr;
          DF2 *jp = Jp + (int64_t)p * n, *jq = Jp + (int64_t)q * n;
          float ph = 0.0f, pl = 0.0f, qh = 0.0f, ql = 0.0f;
          for (int i0 = 0; i0 < nr; i0 += 32 * J64_BATCH) {
            DF2 u[J64_BATCH], v[J64_BATCH], y[J64_BATCH], z[J64_BATCH];
#pragma unroll
            for (int r = 0; r < J64_BATCH; ++r) {
              const int i = i0 + lane + 32 * r;
              u[r] = i < nr ? xp[i] : DF2{0.0f, 0.0f};
              v[r] = i < nr ? xq[i] : DF2{0.0f, 0.0f};
              y[r] = i < n ? jp[i] : DF2{0.0f, 0.0f};
              z[r] = i < n ? jq[i] : DF2{0.0f, 0.0f};
            }
#pragma unroll
            for (int r = 0; r < J64_BATCH; ++r) {
              const int i = i0 + lane + 32 * r;
              if (i < nr) {
                const DF2 u2 = df_axpy(cpp, v[r], u[r]), v2 = df_axpy(cqp, u[r], v[r]);
                xp[i] = u2;
                xq[i] = v2;
                if (rot == 2) {
                  df_dot_acc(u2, u2, ph, pl);
                  df_dot_acc(v2, v2, qh, ql);
                }
              }
              if (i < n) {
                jp[i] = df_axpy(cpp, z[r], y[r]);
                jq[i] = df_axpy(cqp, y[r], z[r]);
              }
            }
          }
          if (rot == 2) {
            np2 = df_wsum(ph, pl);
            nq2 = df_wsum(qh, ql);
          }
        } else {
          double *xp = B + (int64_t)p * nr, *xq = B + (int64_t)q * nr;
          double *jp = Jm + (int64_t)p * n, *jq = Jm + (int64_t)q * n;
          for (int i0 = 0; i0 < nr; i0 += 32 * J64_BATCH) {
            double u[J64_BATCH], v[J64_BATCH], y[J64_BATCH], z[J64_BATCH];
#pragma unroll
            for (int r = 0; r < J64_BATCH; ++r) {
              const int i = i0 + lane + 32 * r;
              u[r] = i < nr ? xp[i] : 0.0;
              v[r] = i < nr ? xq[i] : 0.0;
              y[r] = i < n ? jp[i] : 0.0;
              z[r] = i < n ? jq[i] : 0.0;
            }
#pragma unroll
            for (int r = 0; r < J64_BATCH; ++r) {
              const int i = i0 + lane + 32 * r;
              if (i < nr) {
                const double u2 = fma(cp, v[r], u[r]), v2 = fma(cq, u[r], v[r]);
                xp[i] = u2;
                xq[i] = v2;
                if (rot == 2) {
                  np2 = fma(u2, u2, np2);
                  nq2 = fma(v2, v2, nq2);
                }
              }
              if (i < n) {
                jp[i] = fma(cp, z[r], y[r]);
                jq[i] = fma(cq, y[r], z[r]);
              }
            }
          }
          if (rot == 2) {
            np2 = wsum(np2);
            nq2 = wsum(nq2);
          }
        }
        if (rot == 2 && lane == 0) {  // cancellation: norms from the rotated data
          nrm[p] = dsc[p] * dsc[p] * np2;
          nrm[q] = dsc[q] * dsc[q] * nq2;
        }
      }
      cluster.sync();
    }
    if (any && lane == 0) local_changed = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
      if (local_changed) atomicOr(flag0, 1);
      atomicMax(lmax0, sweep_lmax);
    }
    cluster.sync();
    converged = (*flag0 == 0) || (*lmax0 < small_key);
    cluster.sync();
  }
  fold();
  if (!converged && crank == 0 && threadIdx.x == 0) atomicOr(err, IDMRG_DEV_ERR_JACOBI);
  if (crank == 0 && threadIdx.x == 0) iwork[Jb.perm_off + Jb.cols_a + 1] = sweep;
  // the rotations back to FP64 (fold ended with the cluster barrier, so every
  // pair is final; each element is read and rewritten by the same thread)
  if (PAIRS)
    for (int64_t e = e0; e < nn; e += stride) Jm[e] = df_to(Jp[e]);
  for (int j = gw; j < Jb.cols_a; j += gnw) {
    if (j >= n) {
      if (lane == 0) sv[Jb.sv_off + j] = 0.0;
      continue;
    }
    double *bj = B + (int64_t)j * nr;
    const double s = sqrt(nrm[j]);
    if (lane == 0) sv[Jb.sv_off + j] = s;
    const double inv = s > 0.0 ? 1.0 / s : 0.0;
    if (PAIRS) {
      const DF2 *bp = Bp + (int64_t)j * nr;
      for (int i = lane; i < nr; i += 32) bj[i] = df_to(bp[i]) * inv;
    } else {
      for (int i = lane; i < nr; i += 32) bj[i] *= inv;
    }
  }
}

// ------------------------------------------------- FP32 stage of the Jacobi SVD
// The same block tournament in FP32, whose instructions cost a sixteenth of
// FP64 ones here: it converges the rotations to FP32 accuracy (relative
// overlaps ~1e-6), the rotation matrix is then made orthogonal to FP64
// precision by Newton-Schulz steps and applied to B (FP64 GEMMs), and the
// FP64 block Jacobi finishes from there in two sweeps or so instead of five
// to eight.  The FP32 result only preconditions: singular values and vectors
// come from the FP64 stage.  Each warp takes one pair at a time (plain
// rotations, column norms recomputed); the tests avoid squares so that
// columns near the underflow of FP32 are merely skipped.
__global__ void __launch_bounds__(BJ_THREADS, 2)
    jacobi32_block_kernel(const SvdJob *__restrict__ jobs, const int *__restrict__ order, double *__restrict__ work,
                          const int *__restrict__ iwork) {
  extern __shared__ __align__(16) float bf_sm[];
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int C = (int)cluster.num_blocks();
  const SvdJob Jb = jobs[order[blockIdx.x / C]];
  const int nr = Jb.cols_a;
  const int n = iwork[Jb.perm_off + Jb.cols_a];
  const int P = 2 * C;
  const int bw = (n + P - 1) / P;
  const int nreg = (nr + 31) >> 5, nregj = (n + 31) >> 5;
  const int ldb = 32 * nreg, ldj = 32 * nregj;
  const int offJ = bw * ldb;
  const int slot = (offJ + bw * ldj + 3) & ~3;  // 16-byte aligned blocks
  __shared__ int flag, local_changed, sweep_rmax, cl_rmax;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const double *Bg = work + Jb.b_off;
  double *Vg = work + Jb.j_off;
  const int pos[2] = {crank, P - 1 - crank};
  auto slotp = [&](int buf, int which) { return bf_sm + (buf * 2 + which) * slot; };
  auto valid = [&](int k) { return max(0, min(bw, n - k * bw)); };
  if (nreg > BJ_REG || nregj > BJ_REG || n < 2) return;  // uniform over the cluster
  for (int w = 0; w < 2; ++w) {
    const int k = pos[w], nv = valid(k);
    float *sb = slotp(0, w);
    for (int e = threadIdx.x; e < offJ; e += blockDim.x) {
      const int j = e / ldb, i = e - j * ldb;
      sb[e] = (j < nv && i < nr) ? (float)Bg[(int64_t)(k * bw + j) * nr + i] : 0.0f;
    }
    for (int e = threadIdx.x; e < bw * ldj; e += blockDim.x) {
      const int j = e / ldj, i = e - j * ldj;
      sb[offJ + e] = (j < nv && i == k * bw + j) ? 1.0f : 0.0f;
    }
  }
  const float tol = sqrtf((float)nr) * FLT_EPSILON;
  int *flag0 = cluster.map_shared_rank(&flag, 0);
  int *rmax0 = cluster.map_shared_rank(&cl_rmax, 0);
  int cur = 0;
  bool converged = false;
  auto wsumf = [](float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  };
  // one pair, one warp; returns 1 if rotated (ratio |g|/sqrt(ab) into rmax)
  auto pair = [&](float *s0, int i, float *s1, int j, float &rmax) -> bool {
    float *xp = s0 + i * ldb, *xq = s1 + j * ldb, *jp = s0 + offJ + i * ldj, *jq = s1 + offJ + j * ldj;
    float x[BJ_REG], y[BJ_REG], a = 0.f, b = 0.f, g = 0.f;
#pragma unroll
    for (int r = 0; r < BJ_REG; ++r)
      if (r < nreg) {
        x[r] = xp[lane + 32 * r];
        y[r] = xq[lane + 32 * r];
        a = fmaf(x[r], x[r], a);
        b = fmaf(y[r], y[r], b);
        g = fmaf(x[r], y[r], g);
      }
    a = wsumf(a);
    b = wsumf(b);
    g = wsumf(g);
    if (!(a > 0.f) || !(b > 0.f)) return false;
    const float ra = sqrtf(a), rb = sqrtf(b);
    const float ratio = fabsf(g) / ra / rb;
    if (!(ratio > tol)) return false;
    const float z = (b - a) / (2.0f * g);
    const float t = z == 0.f ? 1.0f : copysignf(1.0f, z) / (fabsf(z) + sqrtf(fmaf(z, z, 1.0f)));
    if (!(fabsf(t) >= FLT_MIN) || !isfinite(t)) return false;
    const float c = rsqrtf(fmaf(t, t, 1.0f)), sn = c * t;
#pragma unroll
    for (int r = 0; r < BJ_REG; ++r)
      if (r < nreg) {
        xp[lane + 32 * r] = c * x[r] - sn * y[r];
        xq[lane + 32 * r] = fmaf(sn, x[r], c * y[r]);
      }
#pragma unroll
    for (int r = 0; r < BJ_REG; ++r)
      if (r < nregj) {
        const float u = jp[lane + 32 * r], v = jq[lane + 32 * r];
        jp[lane + 32 * r] = c * u - sn * v;
        jq[lane + 32 * r] = fmaf(sn, u, c * v);
      }
    rmax = fmaxf(rmax, ratio);
    return true;
  };
  int sweep = 0;
  for (; sweep < 15 && !converged; ++sweep) {
    if (threadIdx.x == 0) {
      local_changed = 0;
      sweep_rmax = 0;
    }
    if (crank == 0 && threadIdx.x == 0) {
      flag = 0;
      cl_rmax = 0;
    }
    cluster.sync();
    bool any = false;
    float rmax = 0.f;
    for (int rnd = 0; rnd < P - 1; ++rnd) {
      float *st0 = slotp(cur, 0), *st1 = slotp(cur, 1);
      const int nv0 = valid(bj_block_at(pos[0], rnd, P)), nv1 = valid(bj_block_at(pos[1], rnd, P));
      if (rnd == 0) {
        const int bp = bw + (bw & 1), half = bp / 2, bm = bp - 1;
        for (int w = 0; w < 2; ++w) {
          const int nv = w ? nv1 : nv0;
          float *sb = w ? st1 : st0;
          for (int sr = 0; sr < bm; ++sr) {
            for (int i = warp; i < half; i += nw) {
              int p = 0, q;
              if (i != 0) {
                p = i - 1 + sr;
                p = 1 + (p >= bm ? p - bm : p);
              }
              q = bp - 2 - i + sr;
              q = 1 + (q >= bm ? q - bm : q);
              if (p < nv && q < nv) any |= pair(sb, p, sb, q, rmax);
            }
            __syncthreads();
          }
        }
      }
      for (int sr = 0; sr < bw; ++sr) {
        for (int i = warp; i < bw; i += nw) {
          int j = i + sr;
          if (j >= bw) j -= bw;
          if (i < nv0 && j < nv1) any |= pair(st0, i, st1, j, rmax);
        }
        __syncthreads();
      }
      if (C > 1) {
        for (int w = 0; w < 2; ++w) {
          const int dpn = pos[w] == 0 ? 0 : (pos[w] == P - 1 ? 1 : pos[w] + 1);
          const int drank = dpn < C ? dpn : P - 1 - dpn, dw = dpn < C ? 0 : 1;
          float4 *dst = reinterpret_cast<float4 *>(cluster.map_shared_rank(slotp(cur ^ 1, dw), drank));
          const float4 *src = reinterpret_cast<const float4 *>(w ? st1 : st0);
          for (int e = threadIdx.x; e < slot / 4; e += blockDim.x) dst[e] = src[e];
        }
        cluster.sync();
        cur ^= 1;
      }
    }
    if (any && lane == 0) local_changed = 1;
    if (lane == 0) atomicMax(&sweep_rmax, __float_as_int(rmax));  // non-negative floats order as ints
    __syncthreads();
    if (threadIdx.x == 0) {
      if (local_changed) atomicOr(flag0, 1);
      atomicMax(rmax0, sweep_rmax);
    }
    cluster.sync();
    // done when nothing rotated, or the largest rotation leaves overlaps of
    // order n r^2 below the FP32 threshold
    const float r = __int_as_float(*rmax0);
    converged = (*flag0 == 0) || ((float)n * r * r < tol) || r < J32_PRECOND_R;
    cluster.sync();
  }
  if (crank == 0 && threadIdx.x == 0) iwork32_sweeps(iwork, Jb, sweep);
  // rotations to V (FP64, cols_a x cols_a, identity outside the rank)
  for (int w = 0; w < 2; ++w) {
    const int k = pos[w], nv = valid(k);
    const float *sb = slotp(cur, w);
    for (int e = threadIdx.x; e < nv * n; e += blockDim.x) {
      const int j = e / n, i = e - j * n;
      Vg[(int64_t)(k * bw + j) * nr + i] = (double)sb[offJ + j * ldj + i];
    }
  }
}

// FP32 stage for sectors of up to 32 * J32B_REG rows whose rotations do not
// fit next to B in shared memory: the block tournament of
// jacobi32_block_kernel with only B's columns in shared memory (four slots of
// bw columns) and the rotations in global memory (FP32, n x n, in the job's
// x_off area), each column of the rotations updated by the CTA that holds
// its block in that round; the cluster barrier that ends a round also
// publishes those updates to the CTA that holds the block next.
constexpr int J32B_REG = 32;  // rows per lane in registers: up to 1024 rows
__global__ void __launch_bounds__(BJ_THREADS, 1)
    jacobi32_big_kernel(const SvdJob *__restrict__ jobs, const int *__restrict__ order, double *__restrict__ work,
                        const int *__restrict__ iwork) {
  extern __shared__ __align__(16) float bg_sm[];
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int C = (int)cluster.num_blocks();
  const SvdJob Jb = jobs[order[blockIdx.x / C]];
  const int nr = Jb.cols_a;
  const int n = iwork[Jb.perm_off + Jb.cols_a];
  const int P = 2 * C;
  const int bw = (n + P - 1) / P;
  const int nreg = (nr + 31) >> 5;
  const int ldb = 32 * nreg;
  const int slot = (bw * ldb + 3) & ~3;  // 16-byte aligned blocks
  __shared__ int flag, local_changed, sweep_rmax, cl_rmax;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const double *Bg = work + Jb.b_off;
  double *Vg = work + Jb.j_off;
  float *V32 = reinterpret_cast<float *>(work + Jb.x_off);  // n x n, leading dimension n
  const int pos[2] = {crank, P - 1 - crank};
  auto slotp = [&](int buf, int which) { return bg_sm + (buf * 2 + which) * slot; };
  auto valid = [&](int k) { return max(0, min(bw, n - k * bw)); };
  if (nreg > J32B_REG || n < 2) return;  // uniform over the cluster
  for (int w = 0; w < 2; ++w) {
    const int k = pos[w], nv = valid(k);
    float *sb = slotp(0, w);
    for (int e = threadIdx.x; e < bw * ldb; e += blockDim.x) {
      const int j = e / ldb, i = e - j * ldb;
      sb[e] = (j < nv && i < nr) ? (float)Bg[(int64_t)(k * bw + j) * nr + i] : 0.0f;
    }
    for (int64_t e = threadIdx.x; e < (int64_t)nv * n; e += blockDim.x) {
      const int64_t j = e / n, i = e - j * n;
      V32[(k * bw + j) * n + i] = (i == k * bw + j) ? 1.0f : 0.0f;
    }
  }
  const float tol = sqrtf((float)nr) * FLT_EPSILON;
  int *flag0 = cluster.map_shared_rank(&flag, 0);
  int *rmax0 = cluster.map_shared_rank(&cl_rmax, 0);
  int cur = 0;
  bool converged = false;
  auto wsumf = [](float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  };
  // one pair, one warp: columns i of s0 (block b0) and j of s1 (block b1)
  auto pair = [&](float *s0, int b0, int i, float *s1, int b1, int j, float &rmax) -> bool {
    float *xp = s0 + i * ldb, *xq = s1 + j * ldb;
    float x[J32B_REG], y[J32B_REG], a = 0.f, b = 0.f, g = 0.f;
#pragma unroll
    for (int r = 0; r < J32B_REG; ++r)
      if (r < nreg) {
        x[r] = xp[lane + 32 * r];
        y[r] = xq[lane + 32 * r];
        a = fmaf(x[r], x[r], a);
        b = fmaf(y[r], y[r], b);
        g = fmaf(x[r], y[r], g);
      }
    a = wsumf(a);
    b = wsumf(b);
    g = wsumf(g);
    if (!(a > 0.f) || !(b > 0.f)) return false;
    const float ratio = fabsf(g) / sqrtf(a) / sqrtf(b);
    if (!(ratio > tol)) return false;
    const float z = (b - a) / (2.0f * g);
    const float t = z == 0.f ? 1.0f : copysignf(1.0f, z) / (fabsf(z) + sqrtf(fmaf(z, z, 1.0f)));
    if (!(fabsf(t) >= FLT_MIN) || !isfinite(t)) return false;
    const float c = rsqrtf(fmaf(t, t, 1.0f)), sn = c * t;
#pragma unroll
    for (int r = 0; r < J32B_REG; ++r)
      if (r < nreg) {
        xp[lane + 32 * r] = c * x[r] - sn * y[r];
        xq[lane + 32 * r] = fmaf(sn, x[r], c * y[r]);
      }
    float *jp = V32 + (int64_t)(b0 * bw + i) * n, *jq = V32 + (int64_t)(b1 * bw + j) * n;
    for (int e = lane; e < n; e += 32) {
      const float u = jp[e], v = jq[e];
      jp[e] = c * u - sn * v;
      jq[e] = fmaf(sn, u, c * v);
    }
    rmax = fmaxf(rmax, ratio);
    return true;
  };
  int sweep = 0;
  for (; sweep < 15 && !converged; ++sweep) {
    if (threadIdx.x == 0) {
      local_changed = 0;
      sweep_rmax = 0;
    }
    if (crank == 0 && threadIdx.x == 0) {
      flag = 0;
      cl_rmax = 0;
    }
    cluster.sync();
    bool any = false;
    float rmax = 0.f;
    for (int rnd = 0; rnd < P - 1; ++rnd) {
      float *st0 = slotp(cur, 0), *st1 = slotp(cur, 1);
      const int b0 = bj_block_at(pos[0], rnd, P), b1 = bj_block_at(pos[1], rnd, P);
      const int nv0 = valid(b0), nv1 = valid(b1);
      if (rnd == 0) {
        const int bp = bw + (bw & 1), half = bp / 2, bm = bp - 1;
        for (int w = 0; w < 2; ++w) {
          const int nv = w ? nv1 : nv0, bk = w ? b1 : b0;
          float *sb = w ? st1 : st0;
          for (int sr = 0; sr < bm; ++sr) {
            for (int i = warp; i < half; i += nw) {
              int p = 0, q;
              if (i != 0) {
                p = i - 1 + sr;
                p = 1 + (p >= bm ? p - bm : p);
              }
              q = bp - 2 - i + sr;
              q = 1 + (q >= bm ? q - bm : q);
              if (p < nv && q < nv) any |= pair(sb, bk, p, sb, bk, q, rmax);
            }
            __syncthreads();
          }
        }
      }
      for (int sr = 0; sr < bw; ++sr) {
        for (int i = warp; i < bw; i += nw) {
          int j = i + sr;
          if (j >= bw) j -= bw;
          if (i < nv0 && j < nv1) any |= pair(st0, b0, i, st1, b1, j, rmax);
        }
        __syncthreads();
      }
      if (C > 1) {
        for (int w = 0; w < 2; ++w) {
          const int dpn = pos[w] == 0 ? 0 : (pos[w] == P - 1 ? 1 : pos[w] + 1);
          const int drank = dpn < C ? dpn : P - 1 - dpn, dw = dpn < C ? 0 : 1;
          float4 *dst = reinterpret_cast<float4 *>(cluster.map_shared_rank(slotp(cur ^ 1, dw), drank));
          const float4 *src = reinterpret_cast<const float4 *>(w ? st1 : st0);
          for (int e = threadIdx.x; e < slot / 4; e += blockDim.x) dst[e] = src[e];
        }
        cluster.sync();
        cur ^= 1;
      } else {
        __syncthreads();
      }
    }
    if (any && lane == 0) local_changed = 1;
    if (lane == 0) atomicMax(&sweep_rmax, __float_as_int(rmax));
    __syncthreads();
    if (threadIdx.x == 0) {
      if (local_changed) atomicOr(flag0, 1);
      atomicMax(rmax0, sweep_rmax);
    }
    cluster.sync();
    const float r = __int_as_float(*rmax0);
    converged = (*flag0 == 0) || ((float)n * r * r < tol) || r < J32_PRECOND_R;
    cluster.sync();
  }
  if (crank == 0 && threadIdx.x == 0) iwork32_sweeps(iwork, Jb, sweep);
  // rotations to V (FP64, cols_a x cols_a): the columns of this CTA's two
  // home blocks (every block is back at its starting position after whole sweeps)
  for (int w = 0; w < 2; ++w) {
    const int k = pos[w], nv = valid(k);
    for (int64_t e = threadIdx.x; e < (int64_t)nv * n; e += blockDim.x) {
      const int64_t j = e / n, i = e - j * n;
      Vg[(k * bw + j) * nr + i] = (double)V32[(k * bw + j) * n + i];
    }
  }
}

// FP32 stage for sectors too large for jacobi32_big_kernel: the same block
// tournament, with the blocks kept in global memory (the FP32 copy of B in
// the job's x_off area) and streamed through shared memory.  The rank-n
// columns are cut into P = 2 C k blocks of bw columns, bw small enough that
// one pair of blocks fits in a CTA's shared memory; in every round each CTA
// visits k of the round's P/2 block pairs in turn: it loads both blocks,
// rotates every column of one against every column of the other (bw
// sub-rounds of bw disjoint pairs; in the first round of a sweep also the
// pairs inside each block), writes them back and applies the visit's
// rotations, accumulated in a 2bw x 2bw matrix Q, to the same columns of the
// FP32 rotations V (n x n, after B32) in one pass.  Rounds are separated by
// the cluster barrier; blocks written in one round are read by other CTAs of
// the cluster in the next, through L2 (loads bypass L1).  A sweep costs
// P - 1 cluster barriers instead of n - 1.
constexpr int JS_THREADS = 512;
constexpr int JS_BW_MAX = 20;  // columns per block: a row of the two blocks of V fits in registers

// shared memory of jacobi32_stream_kernel: two blocks of bw_cap columns of
// ldb floats, Q (2 bw_cap columns of leading dimension qld), two norm arrays
__host__ __device__ constexpr int js_qld(int bw_cap) { return (2 * bw_cap + 3) & ~3; }
__host__ __device__ constexpr int64_t js_smem_floats(int bw_cap, int ldb) {
  return 2 * (int64_t)bw_cap * ldb + (int64_t)js_qld(bw_cap) * 2 * bw_cap + 2 * bw_cap;
}

__global__ void __launch_bounds__(JS_THREADS, 1)
    jacobi32_stream_kernel(const SvdJob *__restrict__ jobs, const int *__restrict__ order, double *__restrict__ work,
                           const int *__restrict__ iwork, int bw_cap, int ldb) {
  extern __shared__ __align__(16) float js_sm[];
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int C = (int)cluster.num_blocks();
  const SvdJob Jb = jobs[order[blockIdx.x / C]];
  const int nr = Jb.cols_a;                      // rows of B
  const int n = iwork[Jb.perm_off + Jb.cols_a];  // columns: numerical rank
  if (n < 2) return;  // uniform over the cluster
  // blocks: bw <= bw_cap, P a multiple of 2C with P bw >= n, then bw = ceil(n / P)
  int bw = min(bw_cap, (n + 2 * C - 1) / (2 * C));
  const int nb = (n + bw - 1) / bw;
  const int P = 2 * C * ((nb + 2 * C - 1) / (2 * C));
  bw = (n + P - 1) / P;
  const int k = P / (2 * C), qd = 2 * bw, qld = js_qld(bw_cap);
  float *S0 = js_sm, *S1 = js_sm + (size_t)bw_cap * ldb;
  float *Q = S1 + (size_t)bw_cap * ldb;            // column c at Q + c qld, rows 0 .. qd-1 (padding rows zero)
  float *N0 = Q + (size_t)qld * 2 * bw_cap, *N1 = N0 + bw_cap;  // squared column norms of S0, S1
  __shared__ int flag, local_changed, sweep_rmax, cl_rmax;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const double *Bg = work + Jb.b_off;
  double *Vg = work + Jb.j_off;
  float *B32 = reinterpret_cast<float *>(work + Jb.x_off);  // nr x n (column j at j nr), then V32
  float *V32 = B32 + (int64_t)nr * n;                        // n x n (column j at j n)
  const int64_t stride = (int64_t)C * blockDim.x, e0 = (int64_t)crank * blockDim.x + threadIdx.x;
  for (int64_t e = e0; e < (int64_t)nr * n; e += stride) B32[e] = (float)Bg[e];
  for (int64_t e = e0; e < (int64_t)n * n; e += stride) V32[e] = (e / n == e % n) ? 1.0f : 0.0f;
  cluster.sync();
  auto valid = [&](int b) { return max(0, min(bw, n - b * bw)); };
  const float tol = sqrtf((float)nr) * FLT_EPSILON;
  int *flag0 = cluster.map_shared_rank(&flag, 0);
  int *rmax0 = cluster.map_shared_rank(&cl_rmax, 0);
  auto wsumf = [](float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  };
  const int l4 = ldb >> 2;  // float4 per column (ldb is a multiple of 32)
  // one pair, one warp: column i of sA (squared norm na[i]) and column j of
  // sB (nb_[j]), Q's columns qi and qj.  One dot product per pair: the
  // rotation that zeroes the overlap g moves the squared norms to a - t g
  // and b + t g, exactly in exact arithmetic; they are recomputed from the
  // data whenever a block is loaded.
  auto pair = [&](float *sA, float *na, int i, float *sB, float *nb_, int j, int qi, int qj, float &rmax) -> bool {
    float4 *xp = reinterpret_cast<float4 *>(sA + i * ldb), *xq = reinterpret_cast<float4 *>(sB + j * ldb);
    float g = 0.f;
    for (int r = lane; r < l4; r += 32) {
      const float4 x = xp[r], y = xq[r];
      g = fmaf(x.x, y.x, g);
      g = fmaf(x.y, y.y, g);
      g = fmaf(x.z, y.z, g);
      g = fmaf(x.w, y.w, g);
    }
    g = wsumf(g);
    const float a = na[i], b = nb_[j];
    if (!(a > 0.f) || !(b > 0.f)) return false;
    const float ratio = fabsf(g) / sqrtf(a) / sqrtf(b);
    if (!(ratio > tol)) return false;
    const float z = (b - a) / (2.0f * g);
    const float t = z == 0.f ? 1.0f : copysignf(1.0f, z) / (fabsf(z) + sqrtf(fmaf(z, z, 1.0f)));
    if (!(fabsf(t) >= FLT_MIN) || !isfinite(t)) return false;
    const float c = rsqrtf(fmaf(t, t, 1.0f)), sn = c * t;
    for (int r = lane; r < l4; r += 32) {
      const float4 x = xp[r], y = xq[r];
      xp[r] = make_float4(c * x.x - sn * y.x, c * x.y - sn * y.y, c * x.z - sn * y.z, c * x.w - sn * y.w);
      xq[r] = make_float4(fmaf(sn, x.x, c * y.x), fmaf(sn, x.y, c * y.y), fmaf(sn, x.z, c * y.z),
                          fmaf(sn, x.w, c * y.w));
    }
    float *cp = Q + qi * qld, *cq = Q + qj * qld;
    for (int r = lane; r < qd; r += 32) {
      const float x = cp[r], y = cq[r];
      cp[r] = c * x - sn * y;
      cq[r] = fmaf(sn, x, c * y);
    }
    __syncwarp();
    if (lane == 0) {
      na[i] = fmaxf(a - t * g, 0.f);
      nb_[j] = fmaxf(b + t * g, 0.f);
    }
    __syncwarp();
    rmax = fmaxf(rmax, ratio);
    return true;
  };
  // the intra-block pairs of one block in shared memory (round robin)
  auto inner = [&](float *sb, float *nv_, int nv, int q0, bool &any, float &rmax) {
    const int bp = bw + (bw & 1), half = bp / 2, bm = bp - 1;
    for (int sr = 0; sr < bm; ++sr) {
      for (int i = warp; i < half; i += nw) {
        int p = 0, q;
        if (i != 0) {
          p = i - 1 + sr;
          p = 1 + (p >= bm ? p - bm : p);
        }
        q = bp - 2 - i + sr;
        q = 1 + (q >= bm ? q - bm : q);
        if (p < nv && q < nv) any |= pair(sb, nv_, p, sb, nv_, q, q0 + p, q0 + q, rmax);
      }
      __syncthreads();
    }
  };
  bool converged = false;
  int sweep = 0;
  for (; sweep < 15 && !converged; ++sweep) {
    if (threadIdx.x == 0) {
      local_changed = 0;
      sweep_rmax = 0;
    }
    if (crank == 0 && threadIdx.x == 0) {
      flag = 0;
      cl_rmax = 0;
    }
    cluster.sync();
    bool any = false;
    float rmax = 0.f;
    for (int rnd = 0; rnd < P - 1; ++rnd) {
      for (int v = 0; v < k; ++v) {
        const int pi = crank + C * v;  // this visit's pair of positions (pi, P - 1 - pi)
        const int b0 = bj_block_at(pi, rnd, P), b1 = bj_block_at(P - 1 - pi, rnd, P);
        const int nv0 = valid(b0), nv1 = valid(b1);
        if (nv0 == 0 && nv1 == 0) continue;  // uniform over the CTA
        // load both blocks (rows >= nr and columns >= nv zero), Q = I
        for (int e = threadIdx.x; e < bw * ldb; e += blockDim.x) {
          const int j = e / ldb, r = e - j * ldb;
          S0[e] = (j < nv0 && r < nr) ? __ldcg(B32 + (int64_t)(b0 * bw + j) * nr + r) : 0.0f;
          S1[e] = (j < nv1 && r < nr) ? __ldcg(B32 + (int64_t)(b1 * bw + j) * nr + r) : 0.0f;
        }
        for (int e = threadIdx.x; e < qld * qd; e += blockDim.x) Q[e] = (e / qld == e % qld) ? 1.0f : 0.0f;
        __syncthreads();
        for (int j = warp; j < 2 * bw; j += nw) {  // squared column norms
          const float4 *x = reinterpret_cast<const float4 *>((j < bw ? S0 : S1) + (j < bw ? j : j - bw) * ldb);
          float a = 0.f;
          for (int r = lane; r < l4; r += 32) {
            const float4 u = x[r];
            a = fmaf(u.x, u.x, a);
            a = fmaf(u.y, u.y, a);
            a = fmaf(u.z, u.z, a);
            a = fmaf(u.w, u.w, a);
          }
          a = wsumf(a);
          if (lane == 0) (j < bw ? N0 : N1)[j < bw ? j : j - bw] = a;
        }
        __syncthreads();
        if (rnd == 0) {
          inner(S0, N0, nv0, 0, any, rmax);
          inner(S1, N1, nv1, bw, any, rmax);
        }
        for (int sr = 0; sr < bw; ++sr) {
          for (int i = warp; i < bw; i += nw) {
            int j = i + sr;
            if (j >= bw) j -= bw;
            if (i < nv0 && j < nv1) any |= pair(S0, N0, i, S1, N1, j, i, bw + j, rmax);
          }
          __syncthreads();
        }
        // blocks back; V's columns of the two blocks times Q, one row per
        // thread (x[r]: V's entry in the column of Q's row r)
        for (int e = threadIdx.x; e < bw * ldb; e += blockDim.x) {
          const int j = e / ldb, r = e - j * ldb;
          if (r < nr) {
            if (j < nv0) B32[(int64_t)(b0 * bw + j) * nr + r] = S0[e];
            if (j < nv1) B32[(int64_t)(b1 * bw + j) * nr + r] = S1[e];
          }
        }
        for (int row = threadIdx.x; row < n; row += blockDim.x) {
          float x[2 * JS_BW_MAX];
#pragma unroll
          for (int r = 0; r < 2 * JS_BW_MAX; ++r) {
            const bool first = r < bw;
            const int lc = first ? r : r - bw, nv = first ? nv0 : nv1, bb = first ? b0 : b1;
            x[r] = (r < qd && lc < nv) ? __ldcg(V32 + (int64_t)(bb * bw + lc) * n + row) : 0.0f;
          }
#pragma unroll 1
          for (int oc = 0; oc < qd; ++oc) {
            const bool first = oc < bw;
            const int lo = first ? oc : oc - bw, nv = first ? nv0 : nv1, bb = first ? b0 : b1;
            if (lo >= nv) continue;
            const float4 *qc = reinterpret_cast<const float4 *>(Q + oc * qld);
            float acc = 0.f;
#pragma unroll
            for (int r4 = 0; r4 < (2 * JS_BW_MAX) / 4; ++r4)
              if (4 * r4 < qd) {
                const float4 w = qc[r4];
                acc = fmaf(x[4 * r4], w.x, acc);
                acc = fmaf(x[4 * r4 + 1], w.y, acc);
                acc = fmaf(x[4 * r4 + 2], w.z, acc);
                acc = fmaf(x[4 * r4 + 3], w.w, acc);
              }
            V32[(int64_t)(bb * bw + lo) * n + row] = acc;
          }
        }
        __syncthreads();
      }
      cluster.sync();  // the blocks and V columns of this tournament round are written before the next reads them
    }
    if (any && lane == 0) local_changed = 1;
    if (lane == 0) atomicMax(&sweep_rmax, __float_as_int(rmax));
    __syncthreads();
    if (threadIdx.x == 0) {
      if (local_changed) atomicOr(flag0, 1);
      atomicMax(rmax0, sweep_rmax);
    }
    cluster.sync();
    const float r = __int_as_float(*rmax0);
    converged = (*flag0 == 0) || ((float)n * r * r < tol) || r < J32_PRECOND_R;
    cluster.sync();
  }
  if (crank == 0 && threadIdx.x == 0) iwork32_sweeps(iwork, Jb, sweep);
  // rotations to V (FP64, leading dimension nr) over the identity already there
  for (int64_t e = e0; e < (int64_t)n * n; e += stride) {
    const int64_t j = e / n, i = e - j * n;
    Vg[j * nr + i] = (double)__ldcg(V32 + e);
  }
}

// per job over cols_a x cols_a elements: 0 V = I, 1 V = 1.5 V - 0.5 W, 2 B = X
__global__ void svd_elementwise_kernel(const SvdJob *__restrict__ jobs, double *__restrict__ work, int mode) {
  const SvdJob J = jobs[blockIdx.y];
  const int ca = J.cols_a;
  const int64_t tot = (int64_t)ca * ca;
  double *V = work + J.j_off, *W = work + J.w_off, *B = work + J.b_off;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    if (mode == 0)
      V[e] = (e / ca == e % ca) ? 1.0 : 0.0;
    else if (mode == 1)
      V[e] = fma(-0.5, W[e], 1.5 * V[e]);
    else
      B[e] = W[e];
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
                              const int *__restrict__ sb_njob, const double *__restrict__ sv,
                              const int *__restrict__ m_sb, double zero_rel, double tie_rel, SelectOut out, int P) {
  extern __shared__ unsigned char smraw[];
  Entry *E = (Entry *)smraw;
  int *cnt = (int *)(E + P);
  const int s = blockIdx.x;
  const int j0 = sb_job0[s], nj = sb_njob[s];
  if (nj == 0) {  // superblock not being truncated: no job to read
    if (threadIdx.x == 0) {
      out.eps[s] = 0.0;
      out.eps_best[s] = 0.0;
      out.kept[s] = 0;
    }
    return;
  }
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
    const int top = min(m_sb[s], nz);
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

// The same with each warp's column and the current reflector in shared
// memory: every reflector is staged once per CTA (double-buffered, so the
// next one loads while the current one is applied) and each warp runs the
// dot product and the axpy over rows kk .. ra-1 only.  On this part a
// warp-wide FP64 instruction holds its sub-partition's FP64 unit for 64
// cycles even when predicated off, so the loops have exact trip counts
// instead of an unrolled register array.  Shared memory: (2 + CP_WARPS) rs
// doubles, rs >= every job's rows.
constexpr int CP_WARPS = 8;
constexpr int CP_MAX_ROWS = 2048;
__global__ void __launch_bounds__(32 * CP_WARPS) compact_smem_kernel(
    const SvdJob *__restrict__ jobs, const CompactJob *__restrict__ cjs, const double *__restrict__ work,
    const int *__restrict__ iwork, const double *__restrict__ sv, const int *__restrict__ perm,
    const int *__restrict__ kept_per_job, double *const *__restrict__ bufs, double *__restrict__ lam, int rs) {
  extern __shared__ double csm[];
  const CompactJob cj = cjs[blockIdx.x];
  const SvdJob J = jobs[cj.job];
  const int k = kept_per_job[cj.job];
  if (blockIdx.y * CP_WARPS >= k) return;  // whole CTA idle (uniform)
  const int ra = J.rows_a, ca = J.cols_a;
  const double *A = work + J.a_off;
  const double *tau = work + J.tau_off;
  const double *Jm = work + J.j_off;
  const double *Bn = work + J.b_off;
  const int *qperm = iwork + J.perm_off;
  const int rk = qperm[ca];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slot = blockIdx.y * CP_WARPS + warp;
  const bool active = slot < k;
  const int col = active ? perm[J.sv_off + slot] : 0;
  double *vs0 = csm, *vs1 = csm + rs, *x = csm + (2 + warp) * rs;
  if (active)
    for (int i = lane; i < ra; i += 32) x[i] = i < rk ? Jm[(int64_t)col * rk + i] : 0.0;
  // reflector kk as (1, v[kk+1] .. v[ra-1]) at rows kk .. ra-1
  if (rk > 0) {
    const double *v = A + (int64_t)(rk - 1) * ra;
    for (int i = rk - 1 + threadIdx.x; i < ra; i += 32 * CP_WARPS) vs0[i] = i == rk - 1 ? 1.0 : v[i];
  }
  __syncthreads();
  for (int kk = rk - 1; kk >= 0; --kk) {
    double *cur = ((rk - 1 - kk) & 1) ? vs1 : vs0, *nxt = ((rk - 1 - kk) & 1) ? vs0 : vs1;
    if (kk > 0) {
      const double *v = A + (int64_t)(kk - 1) * ra;
      for (int i = kk - 1 + threadIdx.x; i < ra; i += 32 * CP_WARPS) nxt[i] = i == kk - 1 ? 1.0 : v[i];
    }
    const double t = tau[kk];
    if (active && t != 0.0) {
      double w = 0.0;
      for (int i = kk + lane; i < ra; i += 32) w = fma(cur[i], x[i], w);
      w = wsum(w) * t;
      for (int i = kk + lane; i < ra; i += 32) x[i] = fma(-w, cur[i], x[i]);
    }
    __syncthreads();
  }
  if (!active) return;
  double *U = bufs[J.sb * NBUF + BUF_U] + cj.u_off;
  double *V = bufs[J.sb * NBUF + BUF_V] + cj.v_off;
  double *Lout = !J.transposed ? U : V;
  double *Rout = !J.transposed ? V : U;
  for (int i = lane; i < ra; i += 32) Lout[(int64_t)i * k + slot] = x[i];
  for (int i = lane; i < ca; i += 32) Rout[(int64_t)qperm[i] * k + slot] = Bn[(int64_t)col * ca + i];
  if (lane == 0) lam[cj.lam_off + slot] = sv[J.sv_off + col];
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

static cudaError_t launch_jacobi_scaled_clusters(const SvdJob *jobs, const int *order, int njobs, int csize,
                                                 double *work, int *iwork, double *sv, int *err, int jm_init,
                                                 bool pairs, cudaStream_t st) {
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
  void (*kern)(const SvdJob *, const int *, double *, int *, double *, int *, int) =
      pairs ? jacobi_scaled_kernel<true> : jacobi_scaled_kernel<false>;
  return cudaLaunchKernelEx(&cfg, kern, jobs, order, work, iwork, sv, err, jm_init);
}

static cudaError_t launch_jacobi_clusters(const SvdJob *jobs, const int *order, int njobs, int csize, double *work,
                                          int *iwork, double *sv, int *err, int jm_init, cudaStream_t st) {
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
  return cudaLaunchKernelEx(&cfg, jacobi_kernel, jobs, order, work, iwork, sv, err, jm_init);
}

static cudaError_t launch_jacobi32_clusters(const SvdJob *jobs, const int *order, int njobs, int csize,
                                            double *work, const int *iwork, cudaStream_t st) {
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
  return cudaLaunchKernelEx(&cfg, jacobi32_kernel, jobs, order, work, iwork);
}

// shared memory of the block kernel for a job of `cols` columns in clusters
// of `csize` (the rank is at most cols): four blocks of B and Jm columns
size_t svd_block_smem(int cols, int csize) {
  const int64_t bw = (cols + 2 * csize - 1) / (2 * csize);
  const int64_t pad = 32 * (((int64_t)cols + 31) / 32);
  if (pad > 32 * BJ_REG) return (size_t)-1;  // beyond the registers of the block kernel
  return (size_t)(4 * (bw * (2 * pad + 2) + 1) * sizeof(double));
}

// block kernel for jobs of at most `cols` columns on clusters of `csize`
static cudaError_t launch_block_clusters(const SvdJob *jobs, const int *order, int njobs, int csize, int cols,
                                         double *work, int *iwork, double *sv, int *err, int jm_init,
                                         cudaStream_t st) {
  // one warp per pair of a sub-round (at least two, at most BJ_THREADS / 32):
  // small blocks let three or four CTAs of different clusters share an SM
  const int bw = (cols + 2 * csize - 1) / (2 * csize);
  const int warps = std::min(BJ_THREADS / 32, std::max(2, bw));
  const size_t smem = svd_block_smem(cols, csize);
  if (smem > SVD_BLOCK_SMEM_MAX) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(njobs * csize, 1, 1);
  cfg.blockDim = dim3(32 * warps, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, jacobi_block_kernel, jobs, order, work, iwork, sv, err, jm_init);
}

// `order` lists the jobs by column count, largest first, in five groups
// [g[k-1], g[k]) (g[-1] = 0, g[4] = njobs): 0 Jacobi in global memory on
// 16-CTA clusters (columns beyond the shared memory of the block kernel),
// 1..4 block Jacobi on clusters of 16, 8, 4 and 1 CTAs; cols[k-1] is the
// largest column count of block group k.  Groups 0 and 1 run on `st`, the others on the side
// streams side[0..2], forked from and joined back to `st` by the events
// ev[0..3].  pairs: group 0 in FP32-pair arithmetic (jacobi_scaled_kernel).
cudaError_t launch_svd_jacobi(const SvdJob *jobs, const int *order, int njobs, const int *g, const int *cols,
                              double *work, int *iwork, double *sv, int *err, int jm_init, bool pairs,
                              cudaStream_t st, const cudaStream_t *side, const cudaEvent_t *ev) {
  if (njobs <= 0) return cudaGetLastError();
  cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaFuncSetAttribute(jacobi_block_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaError_t e = cudaFuncSetAttribute(jacobi_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SVD_BLOCK_SMEM_MAX);
  if (e != cudaSuccess) return e;
  cudaGetLastError();
  const int lo[5] = {0, g[0], g[1], g[2], g[3]}, hi[5] = {g[0], g[1], g[2], g[3], njobs};
  const int csz[5] = {16, 16, 8, 4, 1};
  e = cudaEventRecord(ev[0], st);
  if (e != cudaSuccess) return e;
  for (int k = 2; k < 5; ++k) {
    if (hi[k] <= lo[k]) continue;
    e = cudaStreamWaitEvent(side[k - 2], ev[0], 0);
    if (e != cudaSuccess) return e;
    e = launch_block_clusters(jobs, order + lo[k], hi[k] - lo[k], csz[k], cols[k - 1], work, iwork, sv, err,
                              jm_init, side[k - 2]);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(ev[k - 1], side[k - 2]);
    if (e != cudaSuccess) return e;
  }
  if (hi[0] > lo[0]) {
    cudaFuncSetAttribute(jacobi_scaled_kernel<false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(jacobi_scaled_kernel<true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    e = launch_jacobi_scaled_clusters(jobs, order, hi[0], 16, work, iwork, sv, err, jm_init, pairs, st);
    if (e != cudaSuccess) {
      cudaGetLastError();  // 16-CTA clusters not available here: fall back to 8
      e = launch_jacobi_scaled_clusters(jobs, order, hi[0], 8, work, iwork, sv, err, jm_init, pairs, st);
    }
    if (e != cudaSuccess) return e;
  }
  if (hi[1] > lo[1]) {
    e = launch_block_clusters(jobs, order + lo[1], hi[1] - lo[1], 16, cols[0], work, iwork, sv, err, jm_init, st);
    if (e != cudaSuccess) {
      // 16-CTA clusters not available: the global-memory kernel on 8
      cudaGetLastError();
      e = launch_jacobi_clusters(jobs, order + lo[1], hi[1] - lo[1], 8, work, iwork, sv, err, jm_init, st);
    }
    if (e != cudaSuccess) return e;
  }
  for (int k = 2; k < 5; ++k) {
    if (hi[k] <= lo[k]) continue;
    e = cudaStreamWaitEvent(st, ev[k - 1], 0);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t launch_svd_select(const SvdJob *jobs, const int *sb_job0, const int *sb_njob, int S, const double *sv,
                              const int *m_sb, double zero_rel, double tie_rel, SelectOut out, int max_entries,
                              cudaStream_t st) {
  int P = 1;
  while (P < max_entries) P <<= 1;
  const size_t smem = (size_t)P * sizeof(Entry) + 256 * sizeof(int);
  cudaError_t e = cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (S > 0) select_kernel<<<S, 512, smem, st>>>(jobs, sb_job0, sb_njob, sv, m_sb, zero_rel, tie_rel, out, P);
  return cudaGetLastError();
}

cudaError_t launch_svd_compact(const SvdJob *jobs, const CompactJob *cj, int ncj, int max_kept, int max_rows,
                               double *work, const int *iwork, const double *sv, const int *perm,
                               const int *kept_per_job, double *const *bufs, double *lam, cudaStream_t st) {
  if (ncj > 0 && max_rows <= CP_MAX_ROWS) {
    const int rs = std::max(32, (max_rows + 31) & ~31);
    const size_t smem = (size_t)(2 + CP_WARPS) * rs * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(compact_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(ncj, (unsigned)std::max(1, (max_kept + CP_WARPS - 1) / CP_WARPS));
    compact_smem_kernel<<<grid, 32 * CP_WARPS, smem, st>>>(jobs, cj, work, iwork, sv, perm, kept_per_job, bufs,
                                                            lam, rs);
  } else if (ncj > 0) {
    const int warps = 8;
    dim3 grid(ncj, (unsigned)std::max(1, (max_kept + warps - 1) / warps));
    compact_kernel<<<grid, 32 * warps, 0, st>>>(jobs, cj, work, iwork, sv, perm, kept_per_job, bufs, lam);
  }
  return cudaGetLastError();
}

static cudaError_t launch_block32_clusters(const SvdJob *jobs, const int *order, int njobs, int csize, int cols,
                                           double *work, const int *iwork, cudaStream_t st) {
  const int bw = (cols + 2 * csize - 1) / (2 * csize);
  const int warps = std::min(BJ_THREADS / 32, std::max(2, bw));
  const int64_t pad = 32 * (((int64_t)cols + 31) / 32);
  const size_t smem = (size_t)(4 * ((bw * 2 * pad + 3) & ~(int64_t)3) * sizeof(float));
  if (pad > 32 * BJ_REG || smem > SVD_BLOCK_SMEM_MAX) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(njobs * csize, 1, 1);
  cfg.blockDim = dim3(32 * warps, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, jacobi32_block_kernel, jobs, order, work, iwork);
}

// shared memory of jacobi32_big_kernel for sectors of up to `cols` columns,
// and whether such sectors fit it
static size_t big32_smem(int cols) {
  const int64_t bw = (cols + 31) / 32, ld = 32 * (((int64_t)cols + 31) / 32);
  return (size_t)(4 * ((bw * ld + 3) & ~(int64_t)3) * sizeof(float));
}
static bool big32_fits(int cols) {
  return 32 * (((int64_t)cols + 31) / 32) <= 32 * J32B_REG && big32_smem(cols) <= SVD_BLOCK_SMEM_MAX;
}

int svd_jacobi32_big_max_cols() {
  int c = 32 * J32B_REG;
  while (c > 0 && !big32_fits(c)) --c;
  return c;
}

cudaError_t launch_svd_jacobi32(const SvdJob *jobs, const int *order, int njobs, const int *g, const int *cols,
                                int cols0, int g0b, int cols0b, double *work, const int *iwork, cudaStream_t st,
                                const cudaStream_t *side, const cudaEvent_t *ev) {
  if (njobs <= 0) return cudaGetLastError();
  cudaFuncSetAttribute(jacobi32_block_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaError_t e = cudaFuncSetAttribute(jacobi32_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SVD_BLOCK_SMEM_MAX);
  if (e != cudaSuccess) return e;
  const int lo[5] = {0, g[0], g[1], g[2], g[3]}, hi[5] = {g[0], g[1], g[2], g[3], njobs};
  const int csz[5] = {16, 16, 8, 4, 1};
  e = cudaEventRecord(ev[0], st);
  if (e != cudaSuccess) return e;
  for (int k = 2; k < 5; ++k) {
    if (hi[k] <= lo[k]) continue;
    e = cudaStreamWaitEvent(side[k - 2], ev[0], 0);
    if (e != cudaSuccess) return e;
    e = launch_block32_clusters(jobs, order + lo[k], hi[k] - lo[k], csz[k], cols[k - 1], work, iwork, side[k - 2]);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(ev[k - 1], side[k - 2]);
    if (e != cudaSuccess) return e;
  }
  // beyond the block kernels (jobs 0 .. g[0], largest first): the jobs from
  // g0b on (at most cols0b columns) on jacobi32_big_kernel (B's columns in
  // shared memory, the rotations in global memory) on side stream 3,
  // concurrently with the larger ones on the all-global kernel; every job
  // on the all-global kernel if 16-CTA clusters or the shared memory are
  // not available
  bool big_on_side = false;
  int nglob = hi[0];
  if (hi[0] > lo[0]) {
    const int split = g0b < 0 ? 0 : (g0b > hi[0] ? hi[0] : g0b);
    const int bcols = split == 0 ? cols0 : cols0b;
    if (split < hi[0] && big32_fits(bcols)) {
      const size_t smem0 = big32_smem(bcols);
      cudaFuncSetAttribute(jacobi32_big_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      e = cudaFuncSetAttribute(jacobi32_big_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem0);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(side[3], ev[0], 0);
      if (e == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((hi[0] - split) * 16, 1, 1);
        cfg.blockDim = dim3(BJ_THREADS, 1, 1);
        cfg.dynamicSmemBytes = smem0;
        cfg.stream = side[3];
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 16;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, jacobi32_big_kernel, jobs, order + split, work, iwork);
      }
      if (e == cudaSuccess) e = cudaEventRecord(ev[4], side[3]);
      if (e == cudaSuccess) {
        big_on_side = true;
        nglob = split;
      } else {
        cudaGetLastError();
      }
    }
  }
  if (nglob > 0) {
    // the block tournament streamed through shared memory; the all-global
    // pair kernel if that launch is not possible
    const int ldb0 = 32 * ((cols0 + 31) / 32);
    const int64_t budget = 200 * 1024 / (int)sizeof(float);
    int bw_cap = JS_BW_MAX;
    while (bw_cap >= 1 && js_smem_floats(bw_cap, ldb0) > budget) --bw_cap;
    e = cudaErrorInvalidValue;
    if (bw_cap >= 1) {
      const size_t smem = (size_t)js_smem_floats(bw_cap, ldb0) * sizeof(float);
      cudaFuncSetAttribute(jacobi32_stream_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      e = cudaFuncSetAttribute(jacobi32_stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(nglob * 16, 1, 1);
        cfg.blockDim = dim3(JS_THREADS, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 16;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, jacobi32_stream_kernel, jobs, order, work, iwork, bw_cap, ldb0);
      }
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFuncSetAttribute(jacobi32_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      e = launch_jacobi32_clusters(jobs, order, nglob, 16, work, iwork, st);
      if (e != cudaSuccess) {
        cudaGetLastError();
        e = launch_jacobi32_clusters(jobs, order, nglob, 8, work, iwork, st);
      }
    }
    if (e != cudaSuccess) return e;
  }
  if (hi[1] > lo[1]) {
    e = launch_block32_clusters(jobs, order + lo[1], hi[1] - lo[1], 16, cols[0], work, iwork, st);
    if (e != cudaSuccess) return e;
  }
  for (int k = 2; k < 5; ++k) {
    if (hi[k] <= lo[k]) continue;
    e = cudaStreamWaitEvent(st, ev[k - 1], 0);
    if (e != cudaSuccess) return e;
  }
  if (big_on_side) {
    e = cudaStreamWaitEvent(st, ev[4], 0);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t launch_svd_elementwise(const SvdJob *jobs, int njobs, int max_cols, int mode, double *work,
                                   cudaStream_t st) {
  if (njobs <= 0 || max_cols <= 0) return cudaGetLastError();
  const int64_t tot = (int64_t)max_cols * max_cols;
  dim3 grid((unsigned)std::min<int64_t>((tot + 255) / 256, 64), (unsigned)njobs);
  svd_elementwise_kernel<<<grid, 256, 0, st>>>(jobs, work, mode);
  return cudaGetLastError();
}

size_t svd_qrc_smem(int rows, int cols, int csize) {
  const int64_t nloc = (cols + csize - 1) / csize, ld = (rows + 1) & ~1;
  return (size_t)((nloc * ld + 2 * ld + 3 * nloc + 2) * sizeof(double));
}

// the same with the columns in global memory (reflector, swap buffer and the
// per-column norms in shared memory)
static size_t svd_qrc_smem_global(int rows, int cols, int csize) {
  const int64_t nloc = (cols + csize - 1) / csize, ld = (rows + 1) & ~1;
  return (size_t)((2 * ld + 3 * nloc + 2) * sizeof(double));
}

// pivoted QR of the jobs order[0..njobs) in groups (as the Jacobi): groups
// 0..4 on clusters of 16, 16, 8, 4, 1 CTAs; a group whose columns do not fit
// in the shared memory of its cluster keeps them in global memory
// (force_global_cols: every clustered group does), one that does not fit
// either way runs on the single-CTA kernel; rows[k], cols[k] are the
// largest rows and columns of block group k+1
cudaError_t launch_svd_qrcp_grouped(const SvdJob *jobs, const int *order, int njobs, const int *g, const int *rows,
                                    const int *cols, int rows0, int cols0, double *work, int *iwork,
                                    double zero_rel, bool force_global_cols, cudaStream_t st,
                                    const cudaStream_t *side, const cudaEvent_t *ev) {
  if (njobs <= 0) return cudaGetLastError();
  for (auto kern : {qrcp_cluster_kernel<false>, qrcp_cluster_kernel<true>}) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SVD_BLOCK_SMEM_MAX);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaSuccess;
  const int lo[5] = {0, g[0], g[1], g[2], g[3]}, hi[5] = {g[0], g[1], g[2], g[3], njobs};
  const int csz[5] = {16, 16, 8, 4, 1};
  // groups 2..4 on the side streams, concurrent with groups 0 and 1
  e = cudaEventRecord(ev[0], st);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < 5; ++k) {
    if (hi[k] <= lo[k]) continue;
    const cudaStream_t sk = k >= 2 ? side[k - 2] : st;
    if (k >= 2) {
      e = cudaStreamWaitEvent(sk, ev[0], 0);
      if (e != cudaSuccess) return e;
    }
    const int kr = k == 0 ? rows0 : rows[k - 1], kc = k == 0 ? cols0 : cols[k - 1];
    size_t smem = svd_qrc_smem(kr, kc, csz[k]);
    const bool global_cols = (force_global_cols || smem > SVD_BLOCK_SMEM_MAX) && csz[k] > 1;
    if (global_cols) smem = svd_qrc_smem_global(kr, kc, csz[k]);
    if (smem > SVD_BLOCK_SMEM_MAX) {
      e = launch_svd_qrcp(jobs, order + lo[k], hi[k] - lo[k], work, iwork, zero_rel, sk);
    } else {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((hi[k] - lo[k]) * csz[k], 1, 1);
      cfg.blockDim = dim3(QC_THREADS, 1, 1);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = sk;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = csz[k];
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      e = global_cols ? cudaLaunchKernelEx(&cfg, qrcp_cluster_kernel<true>, jobs, order + lo[k], work, iwork, zero_rel)
                      : cudaLaunchKernelEx(&cfg, qrcp_cluster_kernel<false>, jobs, order + lo[k], work, iwork,
                                           zero_rel);
    }
    if (e != cudaSuccess) return e;
    if (k >= 2) {
      e = cudaEventRecord(ev[k - 1], sk);
      if (e != cudaSuccess) return e;
    }
  }
  for (int k = 2; k < 5; ++k) {
    if (hi[k] <= lo[k]) continue;
    e = cudaStreamWaitEvent(st, ev[k - 1], 0);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace idmrg

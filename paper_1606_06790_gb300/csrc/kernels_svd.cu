// FP64 SVD of Step 4, one charge sector per job, and the truncation of Step 6.
//
//  gather  : copies the sector matrix M_Q (rows (x,s) of left charge Q,
//            columns (t,y) of the complementary charge) out of the wavefunction
//            into a column-major working matrix A (M or M^T, tall side first).
//  jacobi  : one-sided (Hestenes) Jacobi: plane rotations orthogonalise the
//            columns of A; the rotations accumulate in J.  Then A = U S, J = V
//            (or the roles swap when A = M^T).  Parallel round-robin ordering,
//            one warp per column pair, one CTA per job.
//  select  : per superblock, sorts all singular values in descending order
//            (ties by |Q|, Q, index), drops values at or below zero_rel*max,
//            cuts at D <= m without splitting values closer than tie_rel, and
//            writes the discarded weight (Eq. tru) and best fidelity error
//            (Eq. fid2).
//  compact : writes the kept columns of U and V per sector, descending.
#include <float.h>
#include <math.h>

#include "common.h"

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

constexpr int JAC_THREADS = 512;
constexpr int JAC_REG = 8;              // column elements per lane held in registers
constexpr int JAC_SMEM_DOUBLES = 24576; // A kept in shared memory up to 192 KiB

// one column pair (p, q): overlap, rotation of A's and J's columns
__device__ __forceinline__ bool jacobi_pair(double *ap, double *aq, double *jp, double *jq, int ra, int ca,
                                            int lane, double tol, double abs_floor) {
  double x[JAC_REG], y[JAC_REG];
  double al = 0.0, be = 0.0, ga = 0.0;
  const bool inreg = ra <= 32 * JAC_REG;
  if (inreg) {
#pragma unroll
    for (int r = 0; r < JAC_REG; ++r) {
      const int i = lane + 32 * r;
      x[r] = i < ra ? ap[i] : 0.0;
      y[r] = i < ra ? aq[i] : 0.0;
      al = fma(x[r], x[r], al);
      be = fma(y[r], y[r], be);
      ga = fma(x[r], y[r], ga);
    }
  } else {
    for (int i = lane; i < ra; i += 32) {
      const double u = ap[i], v = aq[i];
      al = fma(u, u, al);
      be = fma(v, v, be);
      ga = fma(u, v, ga);
    }
  }
  al = wsum(al);
  be = wsum(be);
  ga = wsum(ga);
  if (ga == 0.0 || !(fabs(ga) > tol * sqrt(al * be)) || !(fabs(ga) > abs_floor)) return false;
  const double zeta = (be - al) / (2.0 * ga);
  const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
  if (inreg) {
#pragma unroll
    for (int r = 0; r < JAC_REG; ++r) {
      const int i = lane + 32 * r;
      if (i < ra) {
        ap[i] = cs * x[r] - sn * y[r];
        aq[i] = sn * x[r] + cs * y[r];
      }
    }
  } else {
    for (int i = lane; i < ra; i += 32) {
      const double u = ap[i], v = aq[i];
      ap[i] = cs * u - sn * v;
      aq[i] = sn * u + cs * v;
    }
  }
  for (int i = lane; i < ca; i += 32) {
    const double u = jp[i], v = jq[i];
    jp[i] = cs * u - sn * v;
    jq[i] = sn * u + cs * v;
  }
  return true;
}

__global__ void __launch_bounds__(JAC_THREADS) jacobi_kernel(const SvdJob *__restrict__ jobs,
                                                             double *__restrict__ work, double *__restrict__ sv,
                                                             int *err) {
  extern __shared__ double As[];
  const SvdJob Jb = jobs[blockIdx.x];
  const int ra = Jb.rows_a, ca = Jb.cols_a;
  double *Ag = work + Jb.a_off;
  double *J = work + Jb.j_off;
  const bool sm = (int64_t)ra * ca <= JAC_SMEM_DOUBLES;
  double *A = sm ? As : Ag;
  if (sm)
    for (int64_t e = threadIdx.x; e < (int64_t)ra * ca; e += blockDim.x) As[e] = Ag[e];
  for (int64_t e = threadIdx.x; e < (int64_t)ca * ca; e += blockDim.x)
    J[e] = (e / ca == e % ca) ? 1.0 : 0.0;
  __shared__ int changed;
  __shared__ double fro_part[JAC_THREADS / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int np = ca + (ca & 1);
  // rotation threshold sqrt(rows) * eps (as in LAPACK's one-sided Jacobi), and
  // an absolute floor eps^2 ||A||_F^2: without it a column made of rounding
  // noise along another one never meets the relative test (each rotation leaves
  // an eps-sized overlap that dominates tol |a_p| |a_q| as |a_q| -> 0).
  const double tol = sqrt((double)ra) * DBL_EPSILON;
  double fro = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)ra * ca; e += blockDim.x) fro = fma(Ag[e], Ag[e], fro);
  fro = wsum(fro);
  if (lane == 0) fro_part[warp] = fro;
  __syncthreads();
  fro = 0.0;
  for (int q = 0; q < nw; ++q) fro += fro_part[q];
  const double abs_floor = 4.0 * DBL_EPSILON * DBL_EPSILON * fro;
  bool converged = (ca < 2);
  for (int sweep = 0; sweep < 60 && !converged; ++sweep) {
    if (threadIdx.x == 0) changed = 0;
    __syncthreads();
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      bool any = false;
      for (int k = warp; k < np / 2; k += nw) {
        const int i1 = k, i2 = np - 1 - k;
        const int p = i1 == 0 ? 0 : 1 + (i1 - 1 + rnd) % (np - 1);
        const int q = i2 == 0 ? 0 : 1 + (i2 - 1 + rnd) % (np - 1);
        if (p >= ca || q >= ca) continue;
        any |= jacobi_pair(A + (int64_t)p * ra, A + (int64_t)q * ra, J + (int64_t)p * ca, J + (int64_t)q * ca, ra,
                           ca, lane, tol, abs_floor);
      }
      if (any && lane == 0) changed = 1;
      __syncthreads();
    }
    converged = (changed == 0);
    __syncthreads();
  }
  if (!converged && threadIdx.x == 0) atomicOr(err, IDMRG_DEV_ERR_JACOBI);
  for (int j = warp; j < ca; j += nw) {
    const double *aj = A + (int64_t)j * ra;
    double s = 0.0;
    for (int i = lane; i < ra; i += 32) s = fma(aj[i], aj[i], s);
    s = wsum(s);
    if (lane == 0) sv[Jb.sv_off + j] = sqrt(s);
  }
  if (sm) {
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)ra * ca; e += blockDim.x) Ag[e] = As[e];
  }
}

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

__global__ void compact_kernel(const SvdJob *__restrict__ jobs, const CompactJob *__restrict__ cjs,
                               const double *__restrict__ work, const double *__restrict__ sv,
                               const int *__restrict__ perm, const int *__restrict__ kept_per_job,
                               double *const *__restrict__ bufs, double *__restrict__ lam) {
  const CompactJob cj = cjs[blockIdx.x];
  const SvdJob J = jobs[cj.job];
  const int k = kept_per_job[cj.job];
  const double *A = work + J.a_off;
  const double *Jm = work + J.j_off;
  double *U = bufs[J.sb * NBUF + BUF_U] + cj.u_off;
  double *V = bufs[J.sb * NBUF + BUF_V] + cj.v_off;
  const int64_t nu = (int64_t)J.r * k, nv = (int64_t)J.c * k;
  for (int64_t e = threadIdx.x + (int64_t)blockIdx.y * blockDim.x; e < nu + nv;
       e += (int64_t)blockDim.x * gridDim.y) {
    if (e < nu) {
      const int row = (int)(e / k), slot = (int)(e % k);
      const int jx = perm[J.sv_off + slot];
      U[e] = !J.transposed ? A[(int64_t)jx * J.r + row] / sv[J.sv_off + jx] : Jm[(int64_t)jx * J.r + row];
    } else {
      const int64_t f = e - nu;
      const int col = (int)(f / k), slot = (int)(f % k);
      const int jx = perm[J.sv_off + slot];
      V[f] = !J.transposed ? Jm[(int64_t)jx * J.c + col] : A[(int64_t)jx * J.c + col] / sv[J.sv_off + jx];
    }
  }
  if (blockIdx.y == 0)
    for (int slot = threadIdx.x; slot < k; slot += blockDim.x) lam[cj.lam_off + slot] = sv[J.sv_off + perm[J.sv_off + slot]];
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

cudaError_t launch_svd_jacobi(const SvdJob *jobs, int njobs, double *work, double *sv, int *err, cudaStream_t st) {
  const int smem = JAC_SMEM_DOUBLES * (int)sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (njobs > 0) jacobi_kernel<<<njobs, JAC_THREADS, smem, st>>>(jobs, work, sv, err);
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

cudaError_t launch_svd_compact(const SvdJob *jobs, const CompactJob *cj, int ncj, const double *work,
                               const double *sv, const int *perm, const int *kept_per_job, double *const *bufs,
                               double *lam, cudaStream_t st) {
  if (ncj > 0) {
    dim3 grid(ncj, 8);
    compact_kernel<<<grid, 256, 0, st>>>(jobs, cj, work, sv, perm, kept_per_job, bufs, lam);
  }
  return cudaGetLastError();
}

}  // namespace idmrg

// FP64 Lanczos of Step 3 (lowest eigenpair of each superblock Hamiltonian),
// batched over superblocks.  Full re-orthogonalisation by classical
// Gram-Schmidt applied twice (the three-term recurrence is the j = k, k-1 part
// of the same projection).  Reductions are two-level and deterministic: each
// CTA writes one partial per (superblock, coefficient); consumers add the
// partials in a fixed order.  The tridiagonal problem is solved on the device:
// warp multisection with FP32 Sturm counts brackets the lowest eigenvalue, the
// eigenvector follows from the backward three-term recurrence and the FP64
// Rayleigh quotient refines the eigenvalue.
#include <float.h>
#include <math.h>

#include "common.h"

namespace idmrg {

namespace {

constexpr int LT = 256;        // threads per CTA
constexpr int EPT = 4;         // elements per thread
constexpr int CH = LT * EPT;   // elements per chunk

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__global__ void set_ptrs_kernel(LanczosDev L, double **bufs) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= L.S) return;
  bufs[s * NBUF + BUF_IN] = L.V[s] + (int64_t)L.k[s] * L.N[s];
  bufs[s * NBUF + BUF_OUT] = L.w[s];
}

// Re-orthogonalisation in two passes: pass 0 is the three-term step, the
// projection on v_k only (alpha) and w -= alpha v_k + beta_{k-1} v_{k-1};
// pass 1 projects the result on every Krylov vector and subtracts it once.
// After the three-term step the components of w along the older vectors are
// small, so one classical Gram-Schmidt pass leaves w orthogonal to working
// precision (no cancellation for a second pass to repair).  FP64 work per
// iteration: (2k + 4) N fused multiply-adds instead of 4 k N.

// part[((pass*S + s)*kmax + j)*nchunk + chunk] = sum_{e in chunk} V_j[e] w[e]
// for j in [jmin, k]: the chunk of w sits in shared memory and each warp
// takes whole vectors, so every lane issues one FMA per element and one warp
// reduction per vector and chunk.
constexpr int PCH = 1024;  // elements per projection chunk (32 per lane per vector)

__global__ void project_kernel(LanczosDev L, int pass) {
  __shared__ double ws[PCH];
  const int s = blockIdx.y;
  if (!L.active[s]) return;
  const int64_t N = L.N[s];
  const int64_t e0 = (int64_t)blockIdx.x * PCH;
  if (e0 >= N) return;
  const int n = (int)min((int64_t)PCH, N - e0);
  const int kk = L.k[s];
  const int jmin = pass == 0 ? kk : 0;
  const double *w = L.w[s] + e0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) ws[i] = w[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = jmin + warp; j <= kk; j += nw) {
    const double *v = L.V[s] + (int64_t)j * N + e0;
    double acc = 0.0;
#pragma unroll 8
    for (int i = lane; i < n; i += 32) acc = fma(v[i], ws[i], acc);
    acc = warp_sum(acc);
    if (lane == 0) L.part[(((int64_t)pass * L.S + s) * L.kmax + j) * L.nchunk_max + blockIdx.x] = acc;
  }
}

// Pass 0: w -= alpha v_k + beta_{k-1} v_{k-1} with alpha = L.h[0][k].
// Pass 1: w -= sum_j V_j h_j with h_j = L.h[1][j], and the partial squared
// norm of the new w at part2 slot 0 of pass 2.  The coefficients were summed
// from their partials once, by reduce_kernel.
__global__ void subtract_kernel(LanczosDev L, int pass) {
  extern __shared__ double hs[];  // [kmax] + [LT/32]
  const int s = blockIdx.y;
  if (!L.active[s]) return;
  const int64_t N = L.N[s];
  const int64_t e0 = (int64_t)blockIdx.x * CH;
  if (e0 >= N) return;
  const int kk = L.k[s];
  const int jmin = pass == 0 ? kk : 0;
  for (int j = jmin + threadIdx.x; j <= kk; j += LT) hs[j] = L.h[((int64_t)pass * L.S + s) * L.kmax + j];
  if (pass == 0 && threadIdx.x == 0 && kk > 0) hs[kk - 1] = L.beta[s * L.kmax + kk - 1];
  __syncthreads();
  double *w = L.w[s];
  const double *V = L.V[s];
  double nrm = 0.0;
  if (pass == 0) {
    const double a = hs[kk], b = kk > 0 ? hs[kk - 1] : 0.0;
    const double *vk = V + (int64_t)kk * N, *vp = V + (int64_t)(kk > 0 ? kk - 1 : kk) * N;
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int64_t e = e0 + threadIdx.x + q * LT;
      if (e >= N) continue;
      double acc = fma(-a, vk[e], w[e]);
      if (kk > 0) acc = fma(-b, vp[e], acc);
      w[e] = acc;
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int64_t e = e0 + threadIdx.x + q * LT;
    if (e >= N) continue;
    double acc = w[e];
    for (int j = 0; j <= kk; ++j) acc = fma(-hs[j], V[(int64_t)j * N + e], acc);
    w[e] = acc;
    nrm = fma(acc, acc, nrm);
  }
  double *red = hs + L.kmax;
  nrm = warp_sum(nrm);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int q = 0; q < LT / 32; ++q) acc += red[q];
    L.part[(((int64_t)2 * L.S + s) * L.kmax + 0) * L.nchunk_max + blockIdx.x] = acc;
  }
}

// Pass 0's subtraction fused with pass 1's projection: each CTA takes one
// projection chunk of PCH elements, reads alpha (reduce_kernel, pass 0),
// updates its chunk of w (w -= alpha v_k + beta_{k-1} v_{k-1}), keeps it in
// shared memory and writes the partial dots of every Krylov vector with it
// (project_kernel, pass 1): one launch and one pass over w fewer than the
// two separate kernels.

// The partials of one projection pass summed once per (superblock, vector):
// one warp per coefficient j (pass 0: j = k only), lane-strided over the
// chunks and a fixed shuffle tree, so the sum is the same on every run.
// Summing them inside every CTA of the consumer instead costs each CTA a
// serial FP64 chain as long as the number of chunks (N / 1024), which grows
// with the vector length.
__global__ void reduce_kernel(LanczosDev L, int pass) {
  const int s = blockIdx.y;
  if (!L.active[s]) return;
  const int kk = L.k[s];
  const int j = (pass == 0 ? kk : 0) + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j > kk) return;
  const int lane = threadIdx.x & 31;
  const int npc = (int)((L.N[s] + PCH - 1) / PCH);
  const double *p = L.part + (((int64_t)pass * L.S + s) * L.kmax + j) * L.nchunk_max;
  double acc = 0.0;
  for (int c = lane; c < npc; c += 32) acc += p[c];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) L.h[((int64_t)pass * L.S + s) * L.kmax + j] = acc;
}
__global__ void sub0_proj1_kernel(LanczosDev L) {
  __shared__ double ws[PCH];
  __shared__ double s_ab[2];
  const int s = blockIdx.y;
  if (!L.active[s]) return;
  const int64_t N = L.N[s];
  const int64_t e0 = (int64_t)blockIdx.x * PCH;
  if (e0 >= N) return;
  const int n = (int)min((int64_t)PCH, N - e0);
  const int kk = L.k[s];
  if (threadIdx.x == 0) {
    s_ab[0] = L.h[(int64_t)s * L.kmax + kk];  // alpha (pass 0), summed by reduce_kernel
    s_ab[1] = kk > 0 ? L.beta[s * L.kmax + kk - 1] : 0.0;
  }
  __syncthreads();
  const double a = s_ab[0], b = s_ab[1];
  double *w = L.w[s] + e0;
  const double *vk = L.V[s] + (int64_t)kk * N + e0;
  const double *vp = L.V[s] + (int64_t)(kk > 0 ? kk - 1 : kk) * N + e0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double acc = fma(-a, vk[i], w[i]);
    if (kk > 0) acc = fma(-b, vp[i], acc);
    w[i] = acc;
    ws[i] = acc;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = warp; j <= kk; j += nw) {
    const double *v = L.V[s] + (int64_t)j * N + e0;
    double acc = 0.0;
#pragma unroll 8
    for (int i = lane; i < n; i += 32) acc = fma(v[i], ws[i], acc);
    acc = warp_sum(acc);
    if (lane == 0) L.part[(((int64_t)L.S + s) * L.kmax + j) * L.nchunk_max + blockIdx.x] = acc;  // pass 1
  }
}

// ---- tridiagonal eigen-solver (lowest pair), one warp per superblock ----
// Sturm count in FP32: the eigenvalue is only bracketed here (to ~1e-7
// relative); its FP64 value comes from inverse iteration and a Rayleigh
// quotient, which costs far fewer FP64 divisions on this part.
__device__ int sturm_count_f(const float *a, const float *b2, int n, float x, float pivmin) {
  int cnt = 0;
  float q = a[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  if (q < 0.f) ++cnt;
  for (int i = 1; i < n; ++i) {
    q = (a[i] - x) - __fdividef(b2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    if (q < 0.f) ++cnt;
  }
  return cnt;
}

__global__ void finalize_kernel(LanczosDev L) {
  const int s = blockIdx.x;
  if (!L.active[s]) return;
  extern __shared__ double sm[];
  const int km = L.kmax;
  double *a = sm, *b = sm + km, *b2 = sm + 2 * km, *x = sm + 3 * km;
  const int kk = L.k[s];
  const int n = kk + 1;
  const int lane = threadIdx.x;
  const int64_t N = L.N[s];
  const int nch = (int)((N + CH - 1) / CH);
  // alpha_k from both Gram-Schmidt passes, beta_k = |w| (partials summed by
  // the whole warp: a serial FP64 chain costs 64 cycles per term here)
  {
    const double *p = L.part + (((int64_t)2 * L.S + s) * km + 0) * L.nchunk_max;
    double nn = 0.0;
    for (int c = lane; c < nch; c += 32) nn += p[c];
    for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
    if (lane == 0) {
      const double alpha = L.h[(int64_t)(0 * L.S + s) * km + kk] + L.h[(int64_t)(1 * L.S + s) * km + kk];
      L.alpha[s * km + kk] = alpha;
      L.resid[s] = sqrt(nn);  // beta_k, stored provisionally
      if (!isfinite(alpha) || !isfinite(nn)) atomicOr(L.err, IDMRG_DEV_ERR_NUMERIC);
    }
  }
  __syncwarp();
  for (int i = lane; i < n; i += 32) {
    a[i] = L.alpha[s * km + i];
    if (i < n - 1) {
      b[i] = L.beta[s * km + i];
      b2[i] = b[i] * b[i];
    }
  }
  __syncwarp();
  const double beta_k = L.resid[s];
  float *af = (float *)(sm + 4 * km), *b2f = af + km;  // FP32 copies for the bracketing
  for (int i = lane; i < n; i += 32) {
    af[i] = (float)a[i];
    if (i < n - 1) b2f[i] = (float)b2[i];
  }
  __syncwarp();
  // Gershgorin interval
  double lo = 1e300, hi = -1e300, bmax = 0.0;
  for (int i = lane; i < n; i += 32) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < n - 1 ? fabs(b[i]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
    if (i < n - 1) bmax = fmax(bmax, b2[i]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    bmax = fmax(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
  }
  const double tnorm = fmax(fabs(lo), fabs(hi));
  float flo = (float)(lo - 1e-6 * tnorm) - 1e-30f, fhi = (float)(hi + 1e-6 * tnorm) + 1e-30f;
  const float fpiv = 1e-30f * fmaxf(1.f, (float)bmax);
  for (int round = 0; round < 12; ++round) {
    const float step = (fhi - flo) / 33.f;
    const float xq = flo + (lane + 1) * step;
    const int c = sturm_count_f(af, b2f, n, xq, fpiv) >= 1;
    const unsigned bal = __ballot_sync(0xffffffffu, c);
    if (bal == 0u) {
      flo = flo + 32 * step;
    } else {
      const int f = __ffs(bal) - 1;
      fhi = flo + (f + 1) * step;
      flo = flo + f * step;
    }
    if (fhi - flo <= 4e-7f * fmaxf(fabsf(flo), fabsf(fhi)) + 1e-30f) break;
  }
  const double shift = 0.5 * ((double)flo + (double)fhi);
  // Eigenvector by the backward three-term recurrence at shift theta (rows
  // n-1 .. 1 of (T - theta) y = 0 with y_{n-1} = 1): one step of inverse
  // iteration applied to e_0, stable because the lowest Ritz vector grows
  // towards j = 0, and division-free (1/beta_j is kept from the iteration
  // that produced beta_j).  The residual left in row 0, r, gives the
  // Rayleigh quotient theta + r y_0 / |y|^2, which converges cubically from
  // the FP32 bracket.  Lane 0 runs the recurrence; theta - a_j, the norm and
  // the scaling are spread over the warp.
  const double *ib = L.ibeta + (int64_t)s * km;
  // x_{j-1} = p_j x_j - q_j x_{j+1} with p_j = (theta - a_j) / beta_{j-1},
  // q_j = beta_j / beta_{j-1} formed by the whole warp, so the serial chain of
  // lane 0 is one FMA per row (q_j x_{j+1} is ready a row earlier); overflow
  // is caught on the exponent bits (|x| >= 2^498) instead of an FP64 compare.
  double *pp = sm + 5 * km, *qq = sm + 6 * km;  // after the FP32 copies (2 km floats at sm + 4 km)
  for (int j = 1 + lane; j <= n - 2; j += 32) qq[j] = b[j] * ib[j - 1];
  double theta = shift, nrm2 = 1.0, dd0 = 0.0;
  for (int it = 0; it < 4; ++it) {
    for (int j = 1 + lane; j <= n - 2; j += 32) pp[j] = (theta - a[j]) * ib[j - 1];
    dd0 = theta - a[0];
    __syncwarp();
    if (lane == 0) {
      x[n - 1] = 1.0;
      if (n >= 2) {
        double xj1 = 1.0, xj = (theta - a[n - 1]) * ib[n - 2];
        x[n - 2] = xj;
        for (int j = n - 2; j >= 1; --j) {
          const double xm = fma(pp[j], xj, -qq[j] * xj1);
          x[j - 1] = xm;
          xj1 = xj;
          xj = xm;
          if ((int)(((unsigned long long)__double_as_longlong(xm) >> 52) & 0x7ffu) > 1023 + 498) {
            for (int i = j - 1; i < n; ++i) x[i] *= 1e-150;
            xj *= 1e-150;
            xj1 *= 1e-150;
          }
        }
      }
    }
    __syncwarp();
    double s2 = 0.0;
    for (int i = lane; i < n; i += 32) s2 = fma(x[i], x[i], s2);
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    nrm2 = s2;
    const double r = (n >= 2) ? fma(-dd0, x[0], b[0] * x[1]) : -dd0 * x[0];
    const double dth = r * x[0] / nrm2;
    theta += dth;
    __syncwarp();
    if (!(fabs(dth) > 2.0 * DBL_EPSILON * fabs(theta))) break;
  }
  {
    const double inv = 1.0 / sqrt(nrm2);
    for (int i = lane; i < n; i += 32) {
      x[i] *= inv;
      L.y[s * km + i] = x[i];
    }
    __syncwarp();
  }
  if (lane == 0) {
    const double scale = fmax(1.0, fabs(theta));
    const double res = beta_k * fabs(x[n - 1]);
    L.theta[s] = theta;
    L.resid[s] = res;
    // k = 0: the test against tol; with an inner factor (mixed-precision
    // restarts) later iterations stop at the target fixed here
    if (kk == 0) L.target[s] = fmax(L.tol * scale, L.inner_factor * beta_k);
    const double goal = (kk == 0 || L.inner_factor == 0.0) ? L.tol * scale : L.target[s];
    if (res <= goal || beta_k <= 1e-14 * scale) {
      L.active[s] = 0;
      L.conv[s] = 1;
    } else if (n >= km) {
      L.active[s] = 0;
      L.conv[s] = 0;
    } else {
      L.beta[s * km + kk] = beta_k;
      L.ibeta[s * km + kk] = 1.0 / beta_k;
      L.k[s] = kk + 1;
    }
  }
}

// V[k] = w / beta[k-1] for superblocks still iterating (k already advanced);
// the next matvec's input pointer moves to V[k] here (no launch of its own)
__global__ void next_kernel(LanczosDev L) {
  const int s = blockIdx.y;
  if (!L.active[s]) return;
  const int64_t N = L.N[s];
  const int kk = L.k[s];
  const double inv = L.ibeta[s * L.kmax + kk - 1];  // 1 / beta_{k-1}, from finalize_kernel
  double *v = L.V[s] + (int64_t)kk * N;
  if (blockIdx.x == 0 && threadIdx.x == 0) L.bufs[s * NBUF + BUF_IN] = v;
  const double *w = L.w[s];
  for (int64_t e = (int64_t)blockIdx.x * CH + threadIdx.x; e < min(N, (int64_t)(blockIdx.x + 1) * CH); e += LT)
    v[e] = w[e] * inv;
}

// generic: out_s = sum_j coef_j x_j  pieces ---------------------------------
__global__ void norm_partial_kernel(const int64_t *Ns, int S, const double *const *x, double *part, int nchunk,
                                    const int *mask) {
  const int s = blockIdx.y;
  if (mask && !mask[s]) return;
  const int64_t N = Ns[s];
  const int64_t e0 = (int64_t)blockIdx.x * CH;
  if (e0 >= N) return;
  double acc = 0.0;
  for (int64_t e = e0 + threadIdx.x; e < min(N, e0 + CH); e += LT) acc = fma(x[s][e], x[s][e], acc);
  __shared__ double red[LT / 32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < LT / 32; ++q) t += red[q];
    part[(int64_t)s * nchunk + blockIdx.x] = t;
  }
}

__global__ void dot_partial_kernel(const int64_t *Ns, const double *const *x, const double *const *y, double *part,
                                   int nchunk, const int *mask) {
  const int s = blockIdx.y;
  if (mask && !mask[s]) return;
  const int64_t N = Ns[s];
  const int64_t e0 = (int64_t)blockIdx.x * CH;
  if (e0 >= N) return;
  double acc = 0.0;
  for (int64_t e = e0 + threadIdx.x; e < min(N, e0 + CH); e += LT) acc = fma(x[s][e], y[s][e], acc);
  __shared__ double red[LT / 32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < LT / 32; ++q) t += red[q];
    part[(int64_t)s * nchunk + blockIdx.x] = t;
  }
}

__global__ void sum_partials_kernel(const int64_t *Ns, int S, const double *part, int nchunk, double *res,
                                    const int *mask) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S || (mask && !mask[s])) return;
  const int nch = (int)((Ns[s] + CH - 1) / CH);
  double acc = 0.0;
  for (int c = 0; c < nch; ++c) acc += part[(int64_t)s * nchunk + c];
  res[s] = acc;
}

// res[s] = sqrt(sum of the partials of x_s . x_s): Euclidean norms
__global__ void norm_finish_kernel(const int64_t *Ns, int S, const double *part, int nchunk, double *res,
                                   const int *mask) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S || (mask && !mask[s])) return;
  const int nch = (int)((Ns[s] + CH - 1) / CH);
  double acc = 0.0;
  for (int c = 0; c < nch; ++c) acc += part[(int64_t)s * nchunk + c];
  res[s] = sqrt(acc);
}

// dst = src / sqrt(nrm2)  and resets the Lanczos state of that superblock
__global__ void init_scale_kernel(LanczosDev L, const double *const *src, const double *nrm2) {
  const int s = blockIdx.y;
  if (!L.member[s]) {
    // a superblock outside this solve: inactive, its vector pointer at V[0]
    // (the flags live in reused device memory and are read by every kernel
    // of the iteration, so they are set here, not assumed)
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      L.active[s] = 0;
      L.k[s] = 0;
    }
    return;
  }
  const int64_t N = L.N[s];
  const double inv = 1.0 / sqrt(nrm2[s]);
  for (int64_t e = (int64_t)blockIdx.x * CH + threadIdx.x; e < min(N, (int64_t)(blockIdx.x + 1) * CH); e += LT)
    L.V[s][e] = src[s][e] * inv;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    L.k[s] = 0;
    L.conv[s] = 0;
    L.active[s] = 1;
    if (!(nrm2[s] > 0.0) || !isfinite(nrm2[s])) atomicOr(L.err, IDMRG_DEV_ERR_ZERONORM | (16 << s));
  }
}

// out = sum_j y_j V_j  (j < k+1)
__global__ void ritz_kernel(LanczosDev L, double *const *out, const int *mask) {
  const int s = blockIdx.y;
  if (!mask[s]) return;
  const int64_t N = L.N[s];
  const int n = L.k[s] + 1;
  const double *y = L.y + (int64_t)s * L.kmax;
  for (int64_t e = (int64_t)blockIdx.x * CH + threadIdx.x; e < min(N, (int64_t)(blockIdx.x + 1) * CH);
       e += LT) {
    double acc = 0.0;
    for (int j = 0; j < n; ++j) acc = fma(y[j], L.V[s][(int64_t)j * N + e], acc);
    out[s][e] = acc;
  }
}

__global__ void scale_by_kernel(const int64_t *Ns, double *const *x, const double *nrm2, const int *mask) {
  const int s = blockIdx.y;
  if (!mask[s]) return;
  const int64_t N = Ns[s];
  const double inv = 1.0 / sqrt(nrm2[s]);
  for (int64_t e = (int64_t)blockIdx.x * CH + threadIdx.x; e < min(N, (int64_t)(blockIdx.x + 1) * CH); e += LT)
    x[s][e] *= inv;
}

}  // namespace

cudaError_t lanczos_set_ptrs(const LanczosDev &L, double **bufs, cudaStream_t st) {
  set_ptrs_kernel<<<(L.S + 63) / 64, 64, 0, st>>>(L, bufs);
  return cudaGetLastError();
}

cudaError_t lanczos_project(const LanczosDev &L, int pass, cudaStream_t st) {
  // projection chunks of PCH elements: nchunk_max counts chunks of CH <= PCH
  dim3 grid((L.nchunk_max * CH + PCH - 1) / PCH, L.S);
  project_kernel<<<grid, LT, 0, st>>>(L, pass);
  return cudaGetLastError();
}

cudaError_t lanczos_reduce(const LanczosDev &L, int pass, cudaStream_t st) {
  constexpr int WPB = 8;  // warps (coefficients) per CTA
  dim3 grid(pass == 0 ? 1 : (L.kmax + WPB - 1) / WPB, L.S);
  reduce_kernel<<<grid, 32 * WPB, 0, st>>>(L, pass);
  return cudaGetLastError();
}

cudaError_t lanczos_sub0_proj1(const LanczosDev &L, cudaStream_t st) {
  dim3 grid((L.nchunk_max * CH + PCH - 1) / PCH, L.S);
  sub0_proj1_kernel<<<grid, LT, 0, st>>>(L);
  return cudaGetLastError();
}

cudaError_t lanczos_subtract(const LanczosDev &L, int pass, cudaStream_t st) {
  dim3 grid(L.nchunk_max, L.S);
  subtract_kernel<<<grid, LT, (L.kmax + LT / 32) * sizeof(double), st>>>(L, pass);
  return cudaGetLastError();
}

cudaError_t lanczos_finalize(const LanczosDev &L, cudaStream_t st) {
  const size_t smem = (size_t)L.kmax * 7 * sizeof(double);  // a, b, b^2, x, FP32 copies, p, q
  finalize_kernel<<<L.S, 32, smem, st>>>(L);
  return cudaGetLastError();
}

cudaError_t lanczos_next(const LanczosDev &L, cudaStream_t st) {
  dim3 grid(L.nchunk_max, L.S);
  next_kernel<<<grid, LT, 0, st>>>(L);
  return cudaGetLastError();
}

cudaError_t lanczos_init(const LanczosDev &L, const double *const *start, cudaStream_t st) {
  // L.part (pass-2 region) is reused for the norm partials, L.resid for the sums
  double *part = L.part;
  dim3 grid(L.nchunk_max, L.S);
  norm_partial_kernel<<<grid, LT, 0, st>>>(L.N, L.S, start, part, L.nchunk_max, L.member);
  sum_partials_kernel<<<(L.S + 63) / 64, 64, 0, st>>>(L.N, L.S, part, L.nchunk_max, L.resid, L.member);
  init_scale_kernel<<<grid, LT, 0, st>>>(L, start, L.resid);
  return cudaGetLastError();
}

cudaError_t launch_norms(const int64_t *Ns, int S, const double *const *x, const int *mask, double *part,
                         int nchunk, double *res, cudaStream_t st) {
  if (S <= 0 || nchunk <= 0) return cudaGetLastError();
  dim3 grid(nchunk, S);
  norm_partial_kernel<<<grid, LT, 0, st>>>(Ns, S, x, part, nchunk, mask);
  norm_finish_kernel<<<(S + 63) / 64, 64, 0, st>>>(Ns, S, part, nchunk, res, mask);
  return cudaGetLastError();
}

int64_t norm_chunk() { return CH; }

cudaError_t lanczos_ritz(const LanczosDev &L, double *const *out, cudaStream_t st) {
  dim3 grid(L.nchunk_max, L.S);
  const int *mask = L.member;
  ritz_kernel<<<grid, LT, 0, st>>>(L, out, mask);
  norm_partial_kernel<<<grid, LT, 0, st>>>(L.N, L.S, out, L.part, L.nchunk_max, mask);
  sum_partials_kernel<<<(L.S + 63) / 64, 64, 0, st>>>(L.N, L.S, L.part, L.nchunk_max, L.resid, mask);
  scale_by_kernel<<<grid, LT, 0, st>>>(L.N, out, L.resid, mask);
  return cudaGetLastError();
}

cudaError_t lanczos_dot(const LanczosDev &L, const double *const *a, const double *const *b, double *res,
                        cudaStream_t st) {
  dim3 grid(L.nchunk_max, L.S);
  const int *mask = L.member;
  dot_partial_kernel<<<grid, LT, 0, st>>>(L.N, a, b, L.part, L.nchunk_max, mask);
  sum_partials_kernel<<<(L.S + 63) / 64, 64, 0, st>>>(L.N, L.S, L.part, L.nchunk_max, res, mask);
  return cudaGetLastError();
}

}  // namespace idmrg

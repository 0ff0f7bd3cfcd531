// FP64 block-sparse contraction kernels of the iDMRG hot path.
//
//  * gemm_f64: the grouped block GEMM used for H_eff psi (Step 3: L . psi and
//    T3 . R^T), the block-spin transformation (Step 6, Eqs. L and R) and the
//    prediction (Step 3', Eq. wfprediction).  A task is one output block;
//    several (A, B) segments may be summed into it (MPO channels folded into
//    the contraction index).
//  * wstage_f64: the two-site MPO stage T3[c] = sum W_{c1} W_{c2} T1[a] and the
//    one-site stage of Step 6, as weighted sums of equally shaped sub-blocks.
//  * dot_terms: weighted sub-block dot products (centre-bond energies).
//  * rand_blocks: SplitMix64 start vectors (Step 3, n = 1, 2).
//  * scale_tasks: diagonal scalings by lambda and 1/lambda (Eq. wfprediction).
#include "common.h"

namespace idmrg {

namespace {

// Tile shapes of the grouped GEMM: TM x TN outputs per CTA, 4 x 4 per
// thread, K in steps of TK.  On this part one 64 x 64 tile holds an SM's
// FP64 units for K x 2048 cycles, so the shape that wastes least in padding
// and in the last wave differs between task lists; the host's autotuner
// times each shape on real calls and keeps the fastest.
constexpr int TK = 16;

template <int TM, int TN>
__global__ void __launch_bounds__(TM *TN / 16) gemm_f64_kernel(const GemmTile *__restrict__ tiles,
                                                               const GemmTask *__restrict__ tasks,
                                                               const GemmSeg *__restrict__ segs,
                                                               double *const *__restrict__ bufs,
                                                               const int *__restrict__ active) {
  constexpr int NT = TM * TN / 16;
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  const GemmTile tile = tiles[blockIdx.x];
  const GemmTask task = tasks[tile.task];
  if (active && !active[task.sb]) return;
  const int tid = threadIdx.x;
  const int tx = tid % (TN / 4), ty = tid / (TN / 4);
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int s = task.seg0; s < task.seg0 + task.nseg; ++s) {
    const GemmSeg sg = segs[s];
    const double *A = bufs[task.sb * NBUF + sg.a_buf] + sg.a_off;
    const double *B = bufs[task.sb * NBUF + sg.b_buf] + sg.b_off;
    const bool ta = sg.flags & 1, tb = sg.flags & 2;
    const bool scale = sg.alpha != 1.0;
    for (int k0 = 0; k0 < sg.K; k0 += TK) {
      // A tile: TM x TK (op(A) rows m, cols k)
#pragma unroll
      for (int r = 0; r < (TM * TK) / NT; ++r) {
        const int idx = tid + r * NT;
        int m, k;
        if (!ta) { m = idx / TK; k = idx % TK; } else { k = idx / TM; m = idx % TM; }
        const int gm = tile.m0 + m, gk = k0 + k;
        double v = 0.0;
        if (gm < task.M && gk < sg.K) v = ta ? A[(int64_t)gk * sg.lda + gm] : A[(int64_t)gm * sg.lda + gk];
        As[k][m] = scale ? v * sg.alpha : v;
      }
#pragma unroll
      for (int r = 0; r < (TN * TK) / NT; ++r) {
        const int idx = tid + r * NT;
        int n, k;
        if (!tb) { k = idx / TN; n = idx % TN; } else { n = idx / TK; k = idx % TK; }
        const int gn = tile.n0 + n, gk = k0 + k;
        double v = 0.0;
        if (gn < task.N && gk < sg.K) v = tb ? B[(int64_t)gn * sg.ldb + gk] : B[(int64_t)gk * sg.ldb + gn];
        Bs[k][n] = v;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < TK; ++k) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[k][ty + (TM / 4) * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + (TN / 4) * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
  double *C = bufs[task.sb * NBUF + task.c_buf] + task.c_off;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = tile.m0 + ty + (TM / 4) * i;
    if (gm >= task.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = tile.n0 + tx + (TN / 4) * j;
      if (gn >= task.N) continue;
      double *p = C + (int64_t)gm * task.ldc + gn;
      *p = task.accumulate ? *p + acc[i][j] : acc[i][j];
    }
  }
}

constexpr int WROWS = 16;

__global__ void wstage_f64_kernel(const WTask *__restrict__ tasks, const WTerm *__restrict__ terms,
                                  double *const *__restrict__ bufs, const int *__restrict__ active) {
  const WTask t = tasks[blockIdx.x];
  if (active && !active[t.sb]) return;
  const int r0 = blockIdx.y * WROWS;
  if (r0 >= t.rows) return;
  const int r1 = min(t.rows, r0 + WROWS);
  double *out = bufs[t.sb * NBUF + t.out_buf] + t.out_off;
  const double *in = bufs[t.sb * NBUF + t.in_buf];
  const int n = (r1 - r0) * t.cols;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int r = r0 + e / t.cols, c = e % t.cols;
    double acc = 0.0;
    for (int q = 0; q < t.nterm; ++q) {
      const WTerm w = terms[t.term0 + q];
      acc = fma(w.coef, in[w.in_off + (int64_t)r * w.in_ld + c], acc);
    }
    out[(int64_t)r * t.out_ld + c] = acc;
  }
}

__global__ void dot_terms_kernel(const DotTerm *__restrict__ terms, double *const *__restrict__ bufs,
                                 double *__restrict__ partial) {
  const DotTerm t = terms[blockIdx.x];
  const double *a = bufs[t.sb * NBUF + t.buf] + t.off1;
  const double *b = bufs[t.sb * NBUF + t.buf] + t.off2;
  double acc = 0.0;
  const int n = t.rows * t.cols;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int r = e / t.cols, c = e % t.cols;
    acc = fma(a[(int64_t)r * t.ld1 + c], b[(int64_t)r * t.ld2 + c], acc);
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) partial[blockIdx.x] = t.coef * acc;
  }
}

// SplitMix64: output k of the stream with state s is mix(s + (k+1) * GAMMA).
__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void rand_blocks_kernel(const RandBlock *__restrict__ blocks, double *const *__restrict__ bufs,
                                   int buf) {
  const RandBlock b = blocks[blockIdx.x];
  const int r0 = blockIdx.y * WROWS;
  if (r0 >= b.rows) return;
  const int r1 = min(b.rows, r0 + WROWS);
  double *out = bufs[b.sb * NBUF + buf] + b.off;
  const int n = (r1 - r0) * b.cols;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int r = r0 + e / b.cols, c = e % b.cols;
    const uint64_t k = (uint64_t)(b.dense0 + (int64_t)r * b.dense_rs + c);
    const uint64_t z = sm64_mix(b.state + (k + 1ull) * 0x9E3779B97F4A7C15ull);
    const double u = (double)(z >> 11) * 0x1.0p-53;
    out[(int64_t)r * b.ld + c] = 2.0 * u - 1.0;
  }
}

__global__ void scale_tasks_kernel(const ScaleTask *__restrict__ tasks, const double *__restrict__ table,
                                   double zero_rel, double *const *__restrict__ bufs) {
  const ScaleTask t = tasks[blockIdx.x];
  const int r0 = blockIdx.y * WROWS;
  if (r0 >= t.rows) return;
  const int r1 = min(t.rows, r0 + WROWS);
  const double *src = bufs[t.sb * NBUF + t.src_buf] + t.off;
  double *dst = bufs[t.sb * NBUF + t.dst_buf] + t.off;
  const double thr = t.rs_inv ? zero_rel * table[t.max_off] : 0.0;
  const int n = (r1 - r0) * t.cols;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int r = r0 + e / t.cols, c = e % t.cols;
    double f = 1.0;
    if (t.rs_off >= 0) {
      const double l = table[t.rs_off + r];
      f = t.rs_inv ? (l > thr ? 1.0 / l : 0.0) : l;
    }
    if (t.cs_off >= 0) f *= table[t.cs_off + c];
    dst[(int64_t)r * t.ld + c] = src[(int64_t)r * t.ld + c] * f;
  }
}

}  // namespace

cudaError_t launch_gemm_f64(const GemmTile *tiles, int ntiles, const GemmTask *tasks, const GemmSeg *segs,
                            double *const *bufs, const int *active, cudaStream_t st, int shape) {
  if (ntiles <= 0) return cudaGetLastError();
  switch (shape) {
    case GEMM_64x64: gemm_f64_kernel<64, 64><<<ntiles, 256, 0, st>>>(tiles, tasks, segs, bufs, active); break;
    case GEMM_64x32: gemm_f64_kernel<64, 32><<<ntiles, 128, 0, st>>>(tiles, tasks, segs, bufs, active); break;
    case GEMM_32x64: gemm_f64_kernel<32, 64><<<ntiles, 128, 0, st>>>(tiles, tasks, segs, bufs, active); break;
    default: gemm_f64_kernel<32, 32><<<ntiles, 64, 0, st>>>(tiles, tasks, segs, bufs, active); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_wstage_f64(const WTask *tasks, int ntasks, int max_rows, const WTerm *terms,
                              double *const *bufs, const int *active, cudaStream_t st) {
  if (ntasks > 0 && max_rows > 0) {
    dim3 grid(ntasks, (max_rows + WROWS - 1) / WROWS);
    wstage_f64_kernel<<<grid, 256, 0, st>>>(tasks, terms, bufs, active);
  }
  return cudaGetLastError();
}

cudaError_t launch_dot_terms(const DotTerm *terms, int nterms, double *const *bufs, double *partial,
                             cudaStream_t st) {
  if (nterms > 0) dot_terms_kernel<<<nterms, 256, 0, st>>>(terms, bufs, partial);
  return cudaGetLastError();
}

cudaError_t launch_rand_blocks(const RandBlock *blocks, int nblocks, int max_rows, double *const *bufs, int buf,
                               cudaStream_t st) {
  if (nblocks > 0 && max_rows > 0) {
    dim3 grid(nblocks, (max_rows + WROWS - 1) / WROWS);
    rand_blocks_kernel<<<grid, 256, 0, st>>>(blocks, bufs, buf);
  }
  return cudaGetLastError();
}

cudaError_t launch_scale_tasks(const ScaleTask *tasks, int ntasks, int max_rows, const double *table,
                               double zero_rel, double *const *bufs, cudaStream_t st) {
  if (ntasks > 0 && max_rows > 0) {
    dim3 grid(ntasks, (max_rows + WROWS - 1) / WROWS);
    scale_tasks_kernel<<<grid, 256, 0, st>>>(tasks, table, zero_rel, bufs);
  }
  return cudaGetLastError();
}

}  // namespace idmrg

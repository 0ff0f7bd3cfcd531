// Mixed-precision H_eff psi on the 5th-generation tensor cores (Step 3).
//
// Every FP64 operand x is split into two TF32 numbers, hi = x rounded to TF32
// and lo = x - hi (also used at TF32 precision), and a product is formed from
// three tcgen05.mma of kind::tf32 (hi.hi + hi.lo + lo.hi) accumulated in FP32
// in tensor memory: about 21 significant bits per product.  The BF16 variant
// splits into two BF16 numbers the same way and issues kind::f16 MMAs: about
// 16 significant bits per product at twice the K per instruction.  Both use
// the same byte layout (a K block is 128 bytes of every row: 32 TF32 or 64
// BF16 elements), so the GEMM kernel differs only in the MMA it issues.
//
//  pack      : splits FP64 or FP32 source blocks into packed hi/lo tiles in the
//              tensor-core operand layout (K-major, no swizzle, core matrices
//              of 8 rows x 16 bytes), so that a K block of a tile is one
//              contiguous range that a single bulk (TMA) copy moves.
//  wstage_tc : T3[c] = sum W12 T1[a] from the FP32 stage-1 output, written
//              straight into the packed A operand of stage 3.
//  tc_gemm   : persistent grouped GEMM over a list of 128 x TN output tiles
//              (TN = 64, 128 or 256, picked per list by the context's tuner),
//              one CTA per SM: a producer warp streams the hi/lo tiles
//              of A and B through a ring of shared-memory stages with
//              cp.async.bulk, an MMA warp issues the tcgen05.mma chain into one
//              of two tensor-memory accumulators, four epilogue warps read the
//              other out (tcgen05.ld) and store it as FP32 (stage 1) or,
//              through a row map, as FP64 into the output wavefunction
//              (stage 3).  Every mbarrier wait is bounded; a timeout sets the
//              context's error word and ends every role's loop, the copies in
//              flight are waited for (bounded), and tensor memory is released
//              unless the wait for the MMAs themselves ran out (they may still
//              write it).
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.h"
#include "tc_ptx.h"

namespace idmrg {

namespace {

__device__ __forceinline__ float tf32_round(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ int64_t packed_off(int row, int k, int KB, int G) {
  const int rows_per_tile = 8 * G;
  const int rt = row / rows_per_tile, rr = row - rt * rows_per_tile;
  const int kb = k >> 5, kc = (k & 31) >> 2;
  const int64_t tile_floats = (int64_t)rows_per_tile * 32;
  return ((int64_t)rt * KB + kb) * 2 * tile_floats + (((int64_t)kc * G + (rr >> 3)) * 8 + (rr & 7)) * 4 + (k & 3);
}

// The same position for 16-bit elements (in units of 16 bits): 64 per K
// block, core matrices 8 rows x 8 elements.
__device__ __forceinline__ int64_t packed_off_h(int row, int k, int KB, int G) {
  const int rows_per_tile = 8 * G;
  const int rt = row / rows_per_tile, rr = row - rt * rows_per_tile;
  const int kb = k >> 6, kc = (k & 63) >> 3;
  const int64_t tile_h = (int64_t)rows_per_tile * 64;
  return ((int64_t)rt * KB + kb) * 2 * tile_h + (((int64_t)kc * G + (rr >> 3)) * 8 + (rr & 7)) * 8 + (k & 7);
}

// hi/lo split of x (given in FP64 or FP32) into the packed operand `dst` at
// element (row, k): TF32 pair (bf16 = 0) or BF16 pair (bf16 = 1).
__device__ __forceinline__ void put_split(float *dst, int row, int k, int KB, int G, int bf16, double x) {
  if (bf16) {
    const __nv_bfloat16 hi = __float2bfloat16_rn((float)x);
    const __nv_bfloat16 lo = __float2bfloat16_rn((float)(x - (double)__bfloat162float(hi)));
    __nv_bfloat16 *h = reinterpret_cast<__nv_bfloat16 *>(dst);
    const int64_t o = packed_off_h(row, k, KB, G);
    h[o] = hi;
    h[o + (int64_t)8 * G * 64] = lo;
  } else {
    const float hi = tf32_round((float)x);
    const int64_t o = packed_off(row, k, KB, G);
    dst[o] = hi;
    dst[o + (int64_t)8 * G * 32] = (float)(x - (double)hi);
  }
}

constexpr int PROWS = 16;

__global__ void pack_kernel(const PackSeg *__restrict__ segs, double *const *__restrict__ bufs,
                            const int *__restrict__ active, int bf16) {
  const PackSeg s = segs[blockIdx.x];
  if (active && !active[s.sb]) return;
  const int r0 = blockIdx.y * PROWS;
  if (r0 >= s.rows) return;
  const int r1 = min(s.rows, r0 + PROWS);
  float *dst = (float *)bufs[s.sb * NBUF + s.dst_buf] + s.dst_off;
  const int n = (r1 - r0) * s.ks;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int r = r0 + e / s.ks, k = e % s.ks;
    const int64_t si = s.trans ? (int64_t)k * s.src_ld + r : (int64_t)r * s.src_ld + k;
    const double x = s.src_fp32 ? (double)((const float *)bufs[s.sb * NBUF + s.src_buf])[s.src_off + si]
                                : bufs[s.sb * NBUF + s.src_buf][s.src_off + si];
    put_split(dst, s.row0 + r, s.k0 + k, s.KB, s.G, bf16, x);
  }
}

// T3 = sum W12 T1 into the packed stage-3 A operand.  The two-site MPO is
// mostly pass-through (a T3 rectangle copies one T1 rectangle, or sums a
// few), so the stage streams T1 in and T3 out.  A CTA takes a window of 32
// rows and 64 packed K columns (aligned to 64) of one rectangle.  Phase 1:
// warps read T1 rows with the lanes along K (coalesced) and accumulate the
// terms.  Phase 2: through a shared-memory tile, each thread takes one row
// and one 16-byte group of the packed layout (8 BF16 or 4 TF32 elements),
// the lanes along the rows, so that a warp's hi (and lo) stores fill 512
// contiguous bytes of a K block.  Groups cut by the rectangle's K edges
// belong partly to the neighbouring rectangle and are written element by
// element.

__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

constexpr int WT_ROWS = 32, WT_K = 64, WT_LD = WT_K + 4;  // window and tile row stride (floats)

// group of GW packed elements [kg, kg + GW) of packed row `row` from the tile
// row v[0..GW); elements outside [ka, kb) are left to their owners
template <int GW>
__device__ __forceinline__ void wt_store(float *dst, const WTaskP &t, int row, int kg, int ka, int kb,
                                         const float *v) {
  const int rpt = 8 * t.G;
  const int rt = row / rpt, rr = row - rt * rpt;
  const bool full = kg >= ka && kg + GW <= kb;
  if (GW == 8) {  // BF16 pairs, 64 elements per K block
    const int kbk = kg >> 6, kc = (kg & 63) >> 3;
    const int64_t tile_h = (int64_t)rpt * 64;
    const int64_t o = ((int64_t)rt * t.KB + kbk) * 2 * tile_h + (((int64_t)kc * t.G + (rr >> 3)) * 8 + (rr & 7)) * 8;
    __nv_bfloat16 hi[8], lo[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      hi[j] = __float2bfloat16_rn(v[j]);
      lo[j] = __float2bfloat16_rn(v[j] - __bfloat162float(hi[j]));
    }
    __nv_bfloat16 *h = reinterpret_cast<__nv_bfloat16 *>(dst) + o;
    if (full) {
      uint4 hv, lv;
      hv.x = pack_bf16x2(hi[0], hi[1]);
      hv.y = pack_bf16x2(hi[2], hi[3]);
      hv.z = pack_bf16x2(hi[4], hi[5]);
      hv.w = pack_bf16x2(hi[6], hi[7]);
      lv.x = pack_bf16x2(lo[0], lo[1]);
      lv.y = pack_bf16x2(lo[2], lo[3]);
      lv.z = pack_bf16x2(lo[4], lo[5]);
      lv.w = pack_bf16x2(lo[6], lo[7]);
      *reinterpret_cast<uint4 *>(h) = hv;
      *reinterpret_cast<uint4 *>(h + tile_h) = lv;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (kg + j >= ka && kg + j < kb) {
          h[j] = hi[j];
          h[tile_h + j] = lo[j];
        }
    }
  } else {  // TF32 pairs, 32 elements per K block
    const int kbk = kg >> 5, kc = (kg & 31) >> 2;
    const int64_t tile_f = (int64_t)rpt * 32;
    const int64_t o = ((int64_t)rt * t.KB + kbk) * 2 * tile_f + (((int64_t)kc * t.G + (rr >> 3)) * 8 + (rr & 7)) * 4;
    float hi[4], lo[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      hi[j] = tf32_round(v[j]);
      lo[j] = v[j] - hi[j];
    }
    float *f = dst + o;
    if (full) {
      *reinterpret_cast<float4 *>(f) = make_float4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<float4 *>(f + tile_f) = make_float4(lo[0], lo[1], lo[2], lo[3]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (kg + j >= ka && kg + j < kb) {
          f[j] = hi[j];
          f[tile_f + j] = lo[j];
        }
    }
  }
}

__global__ void __launch_bounds__(256) wstage_tc_kernel(const int4 *__restrict__ units,
                                                        const WTaskP *__restrict__ tasks,
                                                        const WTerm *__restrict__ terms,
                                                        double *const *__restrict__ bufs,
                                                        const int *__restrict__ active, int bf16) {
  __shared__ __align__(16) float tile[WT_ROWS * WT_LD];
  const int4 u = units[blockIdx.x];  // (task, first row, K window)
  const WTaskP t = tasks[u.x];
  if (active && !active[t.sb]) return;
  const int r0 = u.y, kw = u.z * WT_K;
  const int nr = min(WT_ROWS, t.rows - r0);
  const int ka = max(kw, t.k0), kb = min(kw + WT_K, t.k0 + t.cols);  // packed K of the rectangle in the window
  const float *in = (const float *)bufs[t.sb * NBUF + t.in_buf];
  float *dst = (float *)bufs[t.sb * NBUF + t.dst_buf] + t.dst_off;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // phase 1: warp w holds rows w, w + 8, w + 16, w + 24; lane l columns kw + l, kw + l + 32
  float acc[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = 0.f;
  for (int q = 0; q < t.nterm; ++q) {
    const WTerm w = terms[t.term0 + q];
    const float cf = (float)w.coef;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = warp + 8 * i;
      if (r < nr) {
        const float *src = in + w.in_off + (int64_t)(r0 + r) * w.in_ld;  // packed k at src[k - k0]
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int k = kw + lane + 32 * h;
          if (k >= ka && k < kb) acc[i][h] = fmaf(cf, src[k - t.k0], acc[i][h]);
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    tile[(warp + 8 * i) * WT_LD + lane] = acc[i][0];
    tile[(warp + 8 * i) * WT_LD + lane + 32] = acc[i][1];
  }
  __syncthreads();
  // phase 2: item (group g, row r), r fastest, so a warp covers 32 rows of one group
  const int gw = bf16 ? 8 : 4, ngr = WT_K / gw;
  for (int it = threadIdx.x; it < ngr * WT_ROWS; it += blockDim.x) {
    const int g = it >> 5, r = it & 31;
    const int kg = kw + g * gw;
    if (r >= nr || kg + gw <= ka || kg >= kb) continue;
    const float *v = tile + r * WT_LD + g * gw;
    if (bf16) {
      float x[8];
      *reinterpret_cast<float4 *>(x) = *reinterpret_cast<const float4 *>(v);
      *reinterpret_cast<float4 *>(x + 4) = *reinterpret_cast<const float4 *>(v + 4);
      wt_store<8>(dst, t, t.row0 + r0 + r, kg, ka, kb, x);
    } else {
      float x[4];
      *reinterpret_cast<float4 *>(x) = *reinterpret_cast<const float4 *>(v);
      wt_store<4>(dst, t, t.row0 + r0 + r, kg, ka, kb, x);
    }
  }
}

constexpr int TM = 128;
constexpr int A_TILE = TM * 32;         // floats per A tile (one of hi/lo)
constexpr long long WAIT_BUDGET = 4000000000LL;  // clock cycles (about 2 s)

// Shapes of the persistent GEMM for an N tile of TN columns: a ring stage
// holds one K block of the A tile and of the B tile, hi and lo; as many
// stages as fit in 192 KB of shared memory (4, 3, 2 for TN = 64, 128, 256).
// Behind the ring, each epilogue warp has a 32 x 32 staging block (row
// stride 33 floats) through which its accumulator rows reach global memory
// as whole-row segments.
constexpr int EPI_COLS = 32, EPI_LD = EPI_COLS + 1;
constexpr int EPI_FLOATS = 4 * 32 * EPI_LD;
template <int TN>
struct PsShape {
  static_assert(TN == 64 || TN == 128 || TN == 256, "N tile");
  static constexpr int B_TILE = TN * 32;  // floats per B tile (one of hi/lo)
  static constexpr int STAGE_FLOATS = 2 * A_TILE + 2 * B_TILE;
  static constexpr int STAGES = (192 * 1024) / (STAGE_FLOATS * 4);
  static constexpr int SMEM = STAGES * STAGE_FLOATS * 4 + EPI_FLOATS * 4;
  static_assert(STAGES >= 2, "ring depth");
};

// ---------------------------------------------- persistent grouped GEMM
// Output tiles of 128 rows x TN columns, one CTA per SM looping over the
// tile list (tile t = blockIdx.x + i gridDim.x), with three roles:
// warp 0 streams the K blocks of successive tiles through a PS_STAGES-deep
// ring of shared memory (bulk copies), warp 1 issues the MMA chain of a tile
// into one of two TMEM accumulators, warps 2-5 read the other accumulator out
// (tcgen05.ld) and store it.  Set-up, pipeline fill and epilogue of a tile
// thereby overlap the next tile's copies and MMAs, which matters when K is a
// few blocks (stage 1 of H_eff psi: K = one sector of the left block).
// Ring and accumulator buffers are handed over by mbarriers whose phases
// follow from running counters; every wait is bounded, a timeout sets the
// error word and makes every role leave its loop, and the accumulators are
// released only once every MMA issued has completed.  The N tile (64, 128
// or 256 columns) is chosen per GEMM list by the plan's tuner: a wider tile
// reads each A tile from L2 fewer times, a narrower one wastes less of a
// ragged N.
constexpr int PS_THREADS = 192;

template <bool BF16, int TN>
__global__ void __launch_bounds__(PS_THREADS, 1) tc_gemm_ps_kernel(const TcTile *__restrict__ tiles, int ntiles,
                                                                   const TcTask *__restrict__ tasks,
                                                                   double *const *__restrict__ bufs,
                                                                   const int *__restrict__ active, int *err) {
  using Sh = PsShape<TN>;
  constexpr int PS_STAGES = Sh::STAGES;
  constexpr int B_TILE = Sh::B_TILE;
  constexpr int STAGE_FLOATS = Sh::STAGE_FLOATS;
  extern __shared__ __align__(1024) float sm[];
  float *epi = sm + PS_STAGES * STAGE_FLOATS;  // epilogue staging, EPI_FLOATS
  __shared__ __align__(8) uint64_t full[PS_STAGES], empty[PS_STAGES], accf[2], acce[2], done;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, 2 * TN);
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 32) {
    for (int s = 0; s < PS_STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      tc::mbar_init(&accf[a], 1);
      tc::mbar_init(&acce[a], 4);  // one arrival per epilogue warp
    }
    tc::mbar_init(&done, 1);
    abort_flag = 0;
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  volatile int *abort_v = &abort_flag;
  constexpr uint32_t stage_bytes = 4u * STAGE_FLOATS;

  if (warp == 0) {
    if (lane == 0) {  // ---- producer
      long long it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const TcTile tile = tiles[t];
        const TcTask T = tasks[tile.task];
        if (active && !active[T.sb]) continue;
        const float *A = (const float *)bufs[T.sb * NBUF + T.a_buf] + T.a_off + (int64_t)tile.mt * T.KB * 2 * A_TILE;
        const float *B = (const float *)bufs[T.sb * NBUF + T.b_buf] + T.b_off + (int64_t)tile.nt * T.KB * 2 * B_TILE;
        for (int kb = 0; kb < T.KB; ++kb, ++it) {
          const int s = (int)(it % PS_STAGES);
          const long long u = it / PS_STAGES;
          if (*abort_v || (u > 0 && !tc::mbar_wait(&empty[s], (uint32_t)((u - 1) & 1), WAIT_BUDGET))) {
            ok = false;
            break;
          }
          float *st = sm + s * STAGE_FLOATS;
          tc::mbar_arrive_expect_tx(&full[s], stage_bytes);
          tc::bulk_g2s(st, A + (int64_t)kb * 2 * A_TILE, 4u * 2 * A_TILE, &full[s]);
          tc::bulk_g2s(st + 2 * A_TILE, B + (int64_t)kb * 2 * B_TILE, 4u * 2 * B_TILE, &full[s]);
        }
      }
      if (!ok) {
        atomicOr(err, IDMRG_DEV_ERR_TIMEOUT);
        atomicOr(&abort_flag, 1);
      }
      // the copies of the last ring window may still be in flight: wait for them
      for (long long j = it > PS_STAGES ? it - PS_STAGES : 0; j < it; ++j)
        tc::mbar_wait(&full[j % PS_STAGES], (uint32_t)((j / PS_STAGES) & 1), WAIT_BUDGET);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer
      constexpr uint32_t idesc = tc::instr_desc(TM, TN, BF16 ? 1u : 2u);
      constexpr uint32_t lboA = (TM / 8) * 128, lboB = (TN / 8) * 128, sbo = 128;
      long long it = 0;
      int lt = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const TcTile tile = tiles[t];
        const TcTask T = tasks[tile.task];
        if (active && !active[T.sb]) continue;
        const int a = lt & 1, v = lt >> 1;
        if (*abort_v || (v > 0 && !tc::mbar_wait(&acce[a], (uint32_t)((v - 1) & 1), WAIT_BUDGET))) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(a * TN);
        for (int kb = 0; kb < T.KB; ++kb, ++it) {
          const int s = (int)(it % PS_STAGES);
          if (!tc::mbar_wait(&full[s], (uint32_t)((it / PS_STAGES) & 1), WAIT_BUDGET)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t sa = tc::smem_u32(sm + s * STAGE_FLOATS);
          const uint32_t sb = sa + 4u * 2 * A_TILE;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t ahi = tc::smem_desc(sa + kk * 2 * lboA, lboA, sbo);
            const uint64_t alo = tc::smem_desc(sa + 4u * A_TILE + kk * 2 * lboA, lboA, sbo);
            const uint64_t bhi = tc::smem_desc(sb + kk * 2 * lboB, lboB, sbo);
            const uint64_t blo = tc::smem_desc(sb + 4u * B_TILE + kk * 2 * lboB, lboB, sbo);
            const uint32_t acc0 = (kb > 0 || kk > 0) ? 1u : 0u;
            if (BF16) {
              tc::mma_f16(d, ahi, bhi, idesc, acc0);
              tc::mma_f16(d, ahi, blo, idesc, 1u);
              tc::mma_f16(d, alo, bhi, idesc, 1u);
            } else {
              tc::mma_tf32(d, ahi, bhi, idesc, acc0);
              tc::mma_tf32(d, ahi, blo, idesc, 1u);
              tc::mma_tf32(d, alo, bhi, idesc, 1u);
            }
          }
          tc::mma_commit(&empty[s]);
        }
        if (!ok) break;
        tc::mma_commit(&accf[a]);  // the accumulator of this tile is complete
        ++lt;
      }
      if (!ok) {
        atomicOr(err, IDMRG_DEV_ERR_TIMEOUT);
        atomicOr(&abort_flag, 1);
      }
      tc::mma_commit(&done);  // fires once every MMA issued above has completed
    }
  } else {  // ---- epilogue, warps 2..5: TMEM lane quarter q = warp % 4
    const int q = warp & 3;
    int lt = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const TcTile tile = tiles[t];
      const TcTask T = tasks[tile.task];
      if (active && !active[T.sb]) continue;
      const int a = lt & 1, v = lt >> 1;
      // every lane waits; the warp goes on only together (tcgen05.ld is warp-wide)
      const bool got = !*abort_v && tc::mbar_wait(&accf[a], (uint32_t)(v & 1), WAIT_BUDGET);
      if (!__all_sync(0xffffffffu, got)) {
        if (lane == 0) {
          atomicOr(err, IDMRG_DEV_ERR_TIMEOUT);
          atomicOr(&abort_flag, 1);
        }
        break;
      }
      tc::fence_after_sync();
      // lane l holds accumulator row r0 + l; 32 columns at a time go through
      // the warp's staging block, then out row by row with the lanes along
      // the columns (one 128-byte FP32 or 256-byte FP64 store per row)
      const int r0 = tile.mt * TM + 32 * q;
      const int col0 = tile.nt * TN;
      const int nrows = min(32, T.M - r0);
      double *cbase = bufs[T.sb * NBUF + T.c_buf];
      int64_t obase = 0;
      if (T.mode == 1 && lane < nrows) obase = ((const int64_t *)bufs[T.sb * NBUF + T.rmap_buf])[T.rmap_off + r0 + lane];
      float *stg = epi + q * 32 * EPI_LD;
      for (int c = 0; c < TN && col0 + c < T.N; c += EPI_COLS) {
#pragma unroll
        for (int h = 0; h < EPI_COLS; h += 16) {
          float vv[16];
          if (T.KB > 0) {
            tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(a * TN + c + h), vv);
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) vv[i] = 0.f;
          }
#pragma unroll
          for (int i = 0; i < 16; ++i) stg[lane * EPI_LD + h + i] = vv[i];
        }
        __syncwarp();
        const int col = col0 + c + lane;
        if (T.mode == 0) {
          float *out = (float *)cbase + T.c_off + (int64_t)r0 * T.ldc + col;
          for (int r = 0; r < nrows; ++r)
            if (col < T.N) out[(int64_t)r * T.ldc] = stg[r * EPI_LD + lane];
        } else {
          for (int r = 0; r < nrows; ++r) {
            const int64_t ob = __shfl_sync(0xffffffffu, obase, r);
            if (col < T.N) cbase[ob + col] = (double)stg[r * EPI_LD + lane];
          }
        }
        __syncwarp();
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acce[a]);  // this quarter of the accumulator is free
      ++lt;
    }
  }
  __syncthreads();
  const bool ready = tc::mbar_wait(&done, 0, WAIT_BUDGET);
  if (!ready) {
    atomicOr(&abort_flag, 2);
    if (lane == 0) atomicOr(err, IDMRG_DEV_ERR_TIMEOUT);
  }
  tc::fence_before_sync();
  __syncthreads();
  const int aborted = abort_flag;
  if (warp == 0 && !(aborted & 2)) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 2 * TN);
  }
}

// ------------------------------------------- FP64-accurate digit-slice form
// The Ozaki scheme (Ozaki, Ogita, Oishi, Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59, 2012), here with BF16 slices:
// every packed row r (a row of A, or a column of B) gets an exponent e_r with
// |x| < 2^(e_r - 1) for all its elements, and each element becomes
//   x = sum_{p<8} d_p 2^(e_r - 7 (p + 1)),  d_p integer, |d_p| <= 64,
// exact in BF16 (balanced base-128 digits, 56 bits in all; the rest,
// below 2^(e_r - 57), is dropped).  A product of digits is an integer of at
// most 2^12, so the K-sum of the digit products of one level t = p + q is an
// exact FP32 integer while (t + 1) K 2^12 < 2^24; for K <= OZ_MAX_K that holds
// up to t = 4, and the rounding of the higher levels is below 2^-53 of the
// leading terms.  Levels t <= 7 are kept (one 64-column TMEM accumulator
// each, 36 MMAs per K step); the epilogue sums them in FP64 with their
// power-of-two scales.
__device__ __forceinline__ int64_t oz_off(int row, int k, int KB, int G, int p) {
  const int rows_per_tile = 8 * G;
  const int rt = row / rows_per_tile, rr = row - rt * rows_per_tile;
  const int kb = k >> 5, kc = (k & 31) >> 3;
  const int64_t tile_h = (int64_t)rows_per_tile * OZ_KBLK;
  return (((int64_t)rt * KB + kb) * OZ_PLANES + p) * tile_h + (((int64_t)kc * G + (rr >> 3)) * 8 + (rr & 7)) * 8 +
         (k & 7);
}

// exponent of the expansion for a non-zero x: |x| < 2^(e - 1)
__device__ __forceinline__ int oz_exp_of(double x) {
  const int be = (int)((__double_as_longlong(x) >> 52) & 0x7FF);
  return be ? be - 1023 + 2 : ilogb(x) + 2;
}

// The digits from the bits of x, in integer arithmetic (FP64 instructions are
// scarce here): Y = round(x 2^(56 - e)), |Y| <= 2^55, then balanced base-128
// digits (-64..63) from the least significant one up, the leading digit
// taking what is left (|d_0| <= 64): Y = sum_p d_p 128^(7 - p).
__device__ __forceinline__ void oz_put(__nv_bfloat16 *dst, int row, int k, int KB, int G, int e, double x) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  long long Y = 0;
  if (e != OZ_EXP_EMPTY && (bits << 1) != 0) {
    const int be = (int)((bits >> 52) & 0x7FF);
    unsigned long long mant = bits & ((1ull << 52) - 1);
    int ex = -1074;  // x = mant 2^ex
    if (be) {
      mant |= 1ull << 52;
      ex = be - 1075;
    }
    const int sh = ex + 56 - e;
    unsigned long long u = 0;
    if (sh >= 0)
      u = mant << sh;  // sh <= 2 since |x| < 2^(e - 1)
    else if (sh > -62)
      u = (mant + (1ull << (-sh - 1))) >> (-sh);
    Y = (bits >> 63) ? -(long long)u : (long long)u;
  }
#pragma unroll
  for (int p = OZ_PLANES - 1; p > 0; --p) {
    int r = (int)(Y & 127);
    if (r >= 64) r -= 128;
    Y = (Y - r) >> 7;
    dst[oz_off(row, k, KB, G, p)] = __float2bfloat16_rn((float)r);
  }
  dst[oz_off(row, k, KB, G, 0)] = __float2bfloat16_rn((float)Y);  // what is left: |Y| <= 64
}

__device__ __forceinline__ double oz_src(const PackSeg &s, double *const *bufs, int r, int k) {
  const int64_t si = s.trans ? (int64_t)k * s.src_ld + r : (int64_t)r * s.src_ld + k;
  const double x = s.src_fp32 ? (double)((const float *)bufs[s.sb * NBUF + s.src_buf])[s.src_off + si]
                              : bufs[s.sb * NBUF + s.src_buf][s.src_off + si];
  return s.alpha == 1.0 ? x : s.alpha * x;
}

// exponents of rows whose K range spans several segments
__global__ void oz_exp_kernel(const PackSeg *__restrict__ segs, double *const *__restrict__ bufs,
                              const int *__restrict__ active) {
  const PackSeg s = segs[blockIdx.x];
  if (active && !active[s.sb]) return;
  const int r0 = blockIdx.y * PROWS;
  if (r0 >= s.rows || s.whole) return;
  const int r1 = min(s.rows, r0 + PROWS);
  __shared__ int rexp[PROWS];
  int *ex = (int *)bufs[s.sb * NBUF + s.exp_buf] + s.exp_off + s.row0;
  const int n = (r1 - r0) * s.ks;
  if (threadIdx.x < PROWS) rexp[threadIdx.x] = OZ_EXP_EMPTY;
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int r = r0 + e / s.ks, k = e % s.ks;
    const double x = oz_src(s, bufs, r, k);
    if (x != 0.0) atomicMax(&rexp[r - r0], oz_exp_of(x));
  }
  __syncthreads();
  if (threadIdx.x < r1 - r0 && rexp[threadIdx.x] != OZ_EXP_EMPTY) atomicMax(ex + r0 + threadIdx.x, rexp[threadIdx.x]);
}

// digits; a segment that holds the whole K range of its rows finds their
// exponents itself (and stores them), the others read them
__global__ void oz_pack_kernel(const PackSeg *__restrict__ segs, double *const *__restrict__ bufs,
                               const int *__restrict__ active) {
  __shared__ int rexp[PROWS];
  const PackSeg s = segs[blockIdx.x];
  if (active && !active[s.sb]) return;
  const int r0 = blockIdx.y * PROWS;
  if (r0 >= s.rows) return;
  const int r1 = min(s.rows, r0 + PROWS);
  int *ex = (int *)bufs[s.sb * NBUF + s.exp_buf] + s.exp_off + s.row0;
  __nv_bfloat16 *dst = reinterpret_cast<__nv_bfloat16 *>(bufs[s.sb * NBUF + s.dst_buf]) + s.dst_off;
  const int n = (r1 - r0) * s.ks;
  if (s.whole) {
    if (threadIdx.x < PROWS) rexp[threadIdx.x] = OZ_EXP_EMPTY;
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int r = r0 + e / s.ks, k = e % s.ks;
      const double x = oz_src(s, bufs, r, k);
      if (x != 0.0) atomicMax(&rexp[r - r0], oz_exp_of(x));
    }
    __syncthreads();
    if (threadIdx.x < r1 - r0) ex[r0 + threadIdx.x] = rexp[threadIdx.x];
  } else {
    if (threadIdx.x < r1 - r0) rexp[threadIdx.x] = ex[r0 + threadIdx.x];
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int r = r0 + e / s.ks, k = e % s.ks;
    oz_put(dst, s.row0 + r, s.k0 + k, s.KB, s.G, rexp[r - r0], oz_src(s, bufs, r, k));
  }
}

// T3 = sum W12 T1 in FP64 from the FP64 stage-1 output.  Pass 0 stores T3
// (row-major per stage-3 task, K = the task's full K) and takes the row
// exponents (a maximum per block in shared memory, then one atomic per row
// and block); pass 1 turns the stored values into digits.
__global__ void wstage_oz_kernel(const WTaskP *__restrict__ tasks, const WTerm *__restrict__ terms,
                                 double *const *__restrict__ bufs, const int *__restrict__ active, int pass) {
  __shared__ int rexp[PROWS];
  const WTaskP t = tasks[blockIdx.x];
  if (active && !active[t.sb]) return;
  const int r0 = blockIdx.y * PROWS;
  if (r0 >= t.rows) return;
  const int r1 = min(t.rows, r0 + PROWS);
  int *ex = (int *)bufs[t.sb * NBUF + BUF_OEXP] + t.exp_off + t.row0;
  double *t3 = bufs[t.sb * NBUF + BUF_OT3] + t.t3_off + (int64_t)t.row0 * t.t3_ld + t.k0;
  const int n = (r1 - r0) * t.cols;
  if (pass == 0) {
    const double *in = bufs[t.sb * NBUF + t.in_buf];
    if (threadIdx.x < PROWS) rexp[threadIdx.x] = OZ_EXP_EMPTY;
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int r = r0 + e / t.cols, c = e % t.cols;
      double acc = 0.0;
      for (int q = 0; q < t.nterm; ++q) {
        const WTerm w = terms[t.term0 + q];
        acc = fma(w.coef, in[w.in_off + (int64_t)r * w.in_ld + c], acc);
      }
      t3[(int64_t)r * t.t3_ld + c] = acc;
      if (acc != 0.0) atomicMax(&rexp[r - r0], oz_exp_of(acc));
    }
    __syncthreads();
    if (threadIdx.x < r1 - r0 && rexp[threadIdx.x] != OZ_EXP_EMPTY) atomicMax(ex + r0 + threadIdx.x, rexp[threadIdx.x]);
  } else {
    __nv_bfloat16 *dst = reinterpret_cast<__nv_bfloat16 *>(bufs[t.sb * NBUF + t.dst_buf]) + t.dst_off;
    if (threadIdx.x < r1 - r0) rexp[threadIdx.x] = ex[r0 + threadIdx.x];
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int r = r0 + e / t.cols, c = e % t.cols;
      oz_put(dst, t.row0 + r, t.k0 + c, t.KB, t.G, rexp[r - r0], t3[(int64_t)r * t.t3_ld + c]);
    }
  }
}

constexpr int OZ_A_PLANE = TM * OZ_KBLK * 2;       // bytes of one A digit plane of a K block
constexpr int OZ_B_PLANE = TC_TN * OZ_KBLK * 2;
constexpr int OZ_STAGE = OZ_PLANES * (OZ_A_PLANE + OZ_B_PLANE);
constexpr int OZ_STAGES = 2;
constexpr int OZ_TMEM_COLS = 512;                  // 8 levels x 64 columns

__global__ void __launch_bounds__(128) oz_gemm_kernel(const TcTile *__restrict__ tiles,
                                                      const TcTask *__restrict__ tasks,
                                                      double *const *__restrict__ bufs,
                                                      const int *__restrict__ active, int *err) {
  extern __shared__ __align__(1024) uint8_t osm[];
  __shared__ __align__(8) uint64_t full[OZ_STAGES], empty[OZ_STAGES], done;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const TcTile tile = tiles[blockIdx.x];
  const TcTask T = tasks[tile.task];
  if (active && !active[T.sb]) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, OZ_TMEM_COLS);
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(&done, 1);
    abort_flag = 0;
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  if (threadIdx.x == 0 && T.KB > 0) {
    const uint8_t *A = reinterpret_cast<const uint8_t *>(bufs[T.sb * NBUF + T.a_buf]) + 2 * T.a_off +
                       ((int64_t)tile.mt * T.kb_stride + T.kb0) * OZ_PLANES * OZ_A_PLANE;
    const uint8_t *B = reinterpret_cast<const uint8_t *>(bufs[T.sb * NBUF + T.b_buf]) + 2 * T.b_off +
                       ((int64_t)tile.nt * T.kb_stride + T.kb0) * OZ_PLANES * OZ_B_PLANE;
    constexpr uint32_t idesc = tc::instr_desc(TM, TC_TN, 1u);
    constexpr uint32_t lboA = (TM / 8) * 128, lboB = (TC_TN / 8) * 128, sbo = 128;
    auto issue = [&](int kb) {
      const int s = kb % OZ_STAGES;
      uint8_t *st = osm + s * OZ_STAGE;
      tc::mbar_arrive_expect_tx(&full[s], (uint32_t)OZ_STAGE);
      tc::bulk_g2s(st, A + (int64_t)kb * OZ_PLANES * OZ_A_PLANE, OZ_PLANES * OZ_A_PLANE, &full[s]);
      tc::bulk_g2s(st + OZ_PLANES * OZ_A_PLANE, B + (int64_t)kb * OZ_PLANES * OZ_B_PLANE, OZ_PLANES * OZ_B_PLANE,
                   &full[s]);
    };
    bool ok = true;
    int issued = 0, consumed = 0;
    for (int kb = 0; kb < T.KB && kb < OZ_STAGES - 1; ++kb) {
      issue(kb);
      issued = kb + 1;
    }
    for (int kb = 0; kb < T.KB && ok; ++kb) {
      const int kn = kb + OZ_STAGES - 1;
      if (kn < T.KB) {
        const int sn = kn % OZ_STAGES;
        if (kn >= OZ_STAGES && !tc::mbar_wait(&empty[sn], ((kn / OZ_STAGES) - 1) & 1, WAIT_BUDGET)) {
          ok = false;
          break;
        }
        issue(kn);
        issued = kn + 1;
      }
      const int s = kb % OZ_STAGES;
      if (!tc::mbar_wait(&full[s], (kb / OZ_STAGES) & 1, WAIT_BUDGET)) {
        ok = false;
        break;
      }
      tc::fence_after_sync();
      const uint32_t sa = tc::smem_u32(osm + s * OZ_STAGE);
      const uint32_t sb = sa + OZ_PLANES * OZ_A_PLANE;
#pragma unroll
      for (int kk = 0; kk < OZ_KBLK / 16; ++kk) {
#pragma unroll
        for (int p = 0; p < OZ_PLANES; ++p) {
          const uint64_t ad = tc::smem_desc(sa + p * OZ_A_PLANE + kk * 2 * lboA, lboA, sbo);
#pragma unroll
          for (int q = 0; q < OZ_PLANES - p; ++q) {
            const uint64_t bd = tc::smem_desc(sb + q * OZ_B_PLANE + kk * 2 * lboB, lboB, sbo);
            tc::mma_f16(tmem + (uint32_t)(TC_TN * (p + q)), ad, bd, idesc, (kb > 0 || kk > 0 || p > 0) ? 1u : 0u);
          }
        }
      }
      tc::mma_commit(&empty[s]);
      consumed = kb + 1;
    }
    if (!ok) {
      atomicOr(err, IDMRG_DEV_ERR_TIMEOUT);
      atomicOr(&abort_flag, 1);
      for (int j = consumed; j < issued; ++j) tc::mbar_wait(&full[j % OZ_STAGES], (j / OZ_STAGES) & 1, WAIT_BUDGET);
    }
  }
  if (threadIdx.x == 0) tc::mma_commit(&done);  // fires when every MMA issued above has completed
  const bool ready = tc::mbar_wait(&done, 0, WAIT_BUDGET);
  if (!ready) {
    atomicOr(&abort_flag, 2);
    if (lane == 0) atomicOr(err, IDMRG_DEV_ERR_TIMEOUT);
  }
  __syncthreads();
  tc::fence_after_sync();
  const int aborted = abort_flag;
  if (!aborted) {
    const int row = tile.mt * TM + 32 * warp + lane;
    const int col0 = tile.nt * TC_TN;
    double *cbase = bufs[T.sb * NBUF + T.c_buf];
    const int *ex = (const int *)bufs[T.sb * NBUF + T.exp_buf];
    const int ea = row < T.M ? ex[T.a_exp + row] : OZ_EXP_EMPTY;
    int64_t obase = 0;
    if (T.mode == 1 && row < T.M) obase = ((const int64_t *)bufs[T.sb * NBUF + T.rmap_buf])[T.rmap_off + row];
#pragma unroll 1
    for (int c = 0; c < TC_TN; c += 16) {
      // Levels 0..4 are exact integers (|sum| < 2^24): Horner in base 128 in
      // int64 gives H = sum_t L_t 128^(4-t) exactly (|H| < 2^53), in units
      // of 2^-42.  Levels 5..7 carry FP32 rounding anyway: T = L_5 2^14 +
      // L_6 2^7 + L_7 in FP32, in units of 2^-63 (its error lies below 2^-58
      // of the leading term).  Then value = (H 2^-42 + T 2^-63) 2^(ea+eb):
      // two conversions, one multiply and one FMA in FP64 per output.
      long long H[16];
      float Tl[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        H[i] = 0;
        Tl[i] = 0.f;
      }
      if (T.KB > 0) {
#pragma unroll 1
        for (int t = 0; t < OZ_PLANES; ++t) {
          float v[16];
          tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(TC_TN * t + c), v);
          if (t <= 4) {
#pragma unroll
            for (int i = 0; i < 16; ++i) H[i] = H[i] * 128 + (long long)v[i];
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) Tl[i] = fmaf(Tl[i], 128.0f, v[i]);
          }
        }
      }
      if (row < T.M) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int col = col0 + c + i;
          if (col >= T.N) break;
          const int eb = ex[T.b_exp + col];
          double val = 0.0;
          if (ea != OZ_EXP_EMPTY && eb != OZ_EXP_EMPTY) {
            const int k = ea + eb;
            if (k - 63 > -1000 && k - 42 < 1000) {  // both powers of two are normal doubles
              const double s42 = __longlong_as_double((long long)(k - 42 + 1023) << 52);
              const double s63 = __longlong_as_double((long long)(k - 63 + 1023) << 52);
              val = fma((double)Tl[i], s63, (double)H[i] * s42);
            } else {
              val = scalbn(fma((double)Tl[i], 0x1p-21, (double)H[i]), k - 42);
            }
          }
          double &dst = T.mode == 1 ? cbase[obase + col] : cbase[T.c_off + (int64_t)row * T.ldc + col];
          dst = T.accum ? dst + val : val;
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0 && !(aborted & 2)) tc::tmem_dealloc(tmem, OZ_TMEM_COLS);
}

}  // namespace

cudaError_t launch_oz_exp(const PackSeg *segs, int nseg, int max_rows, double *const *bufs, const int *active,
                          cudaStream_t st) {
  if (nseg > 0 && max_rows > 0) {
    dim3 grid(nseg, (max_rows + PROWS - 1) / PROWS);
    oz_exp_kernel<<<grid, 256, 0, st>>>(segs, bufs, active);
  }
  return cudaGetLastError();
}

cudaError_t launch_oz_pack(const PackSeg *segs, int nseg, int max_rows, double *const *bufs, const int *active,
                           cudaStream_t st) {
  if (nseg > 0 && max_rows > 0) {
    dim3 grid(nseg, (max_rows + PROWS - 1) / PROWS);
    oz_pack_kernel<<<grid, 256, 0, st>>>(segs, bufs, active);
  }
  return cudaGetLastError();
}

cudaError_t launch_wstage_oz(const WTaskP *tasks, int ntasks, int max_rows, const WTerm *terms,
                             double *const *bufs, const int *active, int pass, cudaStream_t st) {
  if (ntasks > 0 && max_rows > 0) {
    dim3 grid(ntasks, (max_rows + PROWS - 1) / PROWS);
    wstage_oz_kernel<<<grid, 256, 0, st>>>(tasks, terms, bufs, active, pass);
  }
  return cudaGetLastError();
}

cudaError_t launch_oz_gemm(const TcTile *tiles, int ntiles, const TcTask *tasks, double *const *bufs,
                           const int *active, int *err, cudaStream_t st) {
  const int smem = OZ_STAGES * OZ_STAGE;
  cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (ntiles > 0) oz_gemm_kernel<<<ntiles, 128, smem, st>>>(tiles, tasks, bufs, active, err);
  return cudaGetLastError();
}

cudaError_t launch_pack(const PackSeg *segs, int nseg, int max_rows, double *const *bufs, const int *active,
                        int bf16, cudaStream_t st) {
  if (nseg > 0 && max_rows > 0) {
    dim3 grid(nseg, (max_rows + PROWS - 1) / PROWS);
    pack_kernel<<<grid, 256, 0, st>>>(segs, bufs, active, bf16);
  }
  return cudaGetLastError();
}

cudaError_t launch_wstage_tc(const int4 *units, int nunits, const WTaskP *tasks, const WTerm *terms,
                             double *const *bufs, const int *active, int bf16, cudaStream_t st) {
  if (nunits > 0) wstage_tc_kernel<<<nunits, 256, 0, st>>>(units, tasks, terms, bufs, active, bf16);
  return cudaGetLastError();
}

template <int TN>
static cudaError_t launch_tc_gemm_tn(const TcTile *tiles, int ntiles, const TcTask *tasks, double *const *bufs,
                                     const int *active, int *err, int bf16, int sms, cudaStream_t st) {
  constexpr int smem = PsShape<TN>::SMEM;
  auto kern = bf16 ? tc_gemm_ps_kernel<true, TN> : tc_gemm_ps_kernel<false, TN>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int grid = ntiles < sms ? ntiles : sms;
  kern<<<grid, PS_THREADS, smem, st>>>(tiles, ntiles, tasks, bufs, active, err);
  return cudaGetLastError();
}

cudaError_t launch_tc_gemm(const TcTile *tiles, int ntiles, const TcTask *tasks, double *const *bufs,
                           const int *active, int *err, int bf16, int tn, cudaStream_t st) {
  if (ntiles <= 0) return cudaGetLastError();
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms <= 0) return e != cudaSuccess ? e : cudaErrorInvalidValue;
  }
  switch (tn) {
    case 64: return launch_tc_gemm_tn<64>(tiles, ntiles, tasks, bufs, active, err, bf16, sms, st);
    case 128: return launch_tc_gemm_tn<128>(tiles, ntiles, tasks, bufs, active, err, bf16, sms, st);
    case 256: return launch_tc_gemm_tn<256>(tiles, ntiles, tasks, bufs, active, err, bf16, sms, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace idmrg

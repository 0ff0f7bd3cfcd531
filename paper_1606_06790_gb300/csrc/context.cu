// libidmrg host runtime: the C ABI of include/idmrg.h.
//
// One context holds the l/2 superblock pairs of the parallel iDMRG (Sec. 3).
// Per iteration n it plans the block-sparse contractions of every superblock
// on the host (block tables, task lists), uploads them once, and runs the
// step on the device: start vector (Step 3'), batched Lanczos (Step 3),
// sector SVD and truncation (Step 4), block-spin transformation (Step 6),
// then rotates the right blocks between neighbouring pairs (Step 2') and
// advances n (Step 7).  Step 5' (energy per site) is host bookkeeping of the
// energies the device returns.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <map>
#include <thread>
#include <string>
#include <tuple>
#include <vector>

#include "common.h"
#include "idmrg.h"
#include "plan.h"

using namespace idmrg;

namespace {

struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
};

enum Stage { ST_READY = 0, ST_STARTED = 1, ST_SOLVED = 2, ST_TRUNCATED = 3, ST_UPDATED = 4 };

struct Env {
  EnvLayout lay;
  DevBuf data;
};

struct TruncRec {
  bool valid = false;
  Basis leftB, rightB;          // blocks of the superblock this SVD came from
  std::vector<SecInfo> sec;     // kept sectors, in the new basis order
  Basis bU, bV;                 // new left / right bases
  DevBuf U, V;                  // device U_Q, V_Q blocks (FP64)
  std::vector<double> lam;      // kept singular values, basis order
  std::vector<double> lam_all;  // every singular value, descending
  double eps = 0, eps_best = 0;
  int64_t usize = 0, vsize = 0;
};

struct SBPlan {
  int c1 = 0, c2 = 0;
  PsiLayout psi;
  int64_t t1size = 0, t3size = 0, xsize = 0, ysize = 0;
  std::vector<int64_t> t1off, t3off;
  std::vector<int> t3C, t3col;
  std::vector<double> W12;  // [wa][wc][d*d][d*d]
  std::vector<double> h2;   // centre bond operator [d*d][d*d]
  double heff_flops = 0, heff_bytes = 0;
  double gemm_flops = 0, w_flops = 0;
  // mixed forms: algorithmic bytes of the psi split (FP64 in, hi/lo out) and
  // of the W stage (FP32 T1 in once, hi/lo T3 out), per hi/lo word size
  double wpack_elems = 0, wt1_elems = 0, wt3_elems = 0;
  int njob0 = 0, njob = 0;  // SVD jobs
};

uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// output k (0-based) of the SplitMix64 stream with initial state s
uint64_t sm64_at(uint64_t s, uint64_t k) { return sm64_mix(s + (k + 1ull) * 0x9E3779B97F4A7C15ull); }

}  // namespace

// Autotuned tile shape of one grouped-GEMM list.  Every shape gives the same
// result bit for bit (each output element sums its K terms in the same
// order), so the first calls of a list try each shape once on real work,
// timed with CUDA events on the stream, and the fastest is kept until the
// list's work changes by more than 10 %.
// A grouped FP64 GEMM list in the digit-slice form (kernels_tc.cu): every
// task's op(A) (M x K) and op(B)^T (N x K), K concatenated over its segments,
// become digit planes in the context's digit arena, one exponent per packed
// row; tasks longer than OZ_MAX_K run in K chunks (one launch each).
struct OzList {
  bool ok = false;
  std::vector<PackSeg> segs;      // A and B packing, one per GEMM segment and operand
  int seg_rows = 0;
  std::vector<TcTask> tasks;
  std::vector<TcTile> tiles;
  std::vector<int> lo;            // tile ranges of the K chunks
  int64_t planes = 0, nexp = 0;   // arena use: BF16 elements, exponents
  DevBuf dsegs, dtasks, dtiles;
};

struct GemmTune {
  OzList oz;
  bool oz_use = false;  // list eligible for the digit-slice form (environments, prediction, SVD)
  DevBuf tiles[GEMM_NSHAPE];
  int ntiles[GEMM_NSHAPE] = {0, 0, 0, 0};
  int choice = -1;
  int state[GEMM_NSHAPE] = {0, 0, 0, 0};  // 0 untried, 1 timing, 2 timed
  float ms[GEMM_NSHAPE] = {0, 0, 0, 0};
  cudaEvent_t e0[GEMM_NSHAPE] = {}, e1[GEMM_NSHAPE] = {};
  double work = -1.0;
};

// Uniform MPS of Eq. mps2 (observables): the unit's l site tensors A_k
// (d x D_k x D_k+1, dense), the charge blocks they are non-zero on, the
// transfer-map task lists, the fixed points and the environments l_k, r_k.
struct ObsBlock {
  int s, rb, cb;  // physical state, block of bond k, block of bond k+1
};
struct ObsList {
  int tile0 = 0, ntile = 0;
};
// task lists concatenated into one upload (indices rebased on append)
struct ObsArena {
  GemmList G;
  DevBuf dtasks, dsegs, dtiles;
  void clear() { G.clear(); }
  ObsList add(const GemmList &L) {
    ObsList o;
    const int t0 = (int)G.tasks.size(), s0 = (int)G.segs.size();
    o.tile0 = (int)G.tiles.size();
    for (GemmTask t : L.tasks) {
      t.seg0 += s0;
      G.tasks.push_back(t);
    }
    G.segs.insert(G.segs.end(), L.segs.begin(), L.segs.end());
    for (GemmTile x : L.tiles) {
      x.task += t0;
      G.tiles.push_back(x);
    }
    o.ntile = (int)L.tiles.size();
    G.flops += L.flops;
    return o;
  }
};
struct ObsState {
  bool valid = false;   // unit embedded for the current iteration
  bool fixed = false;   // fixed points and environments computed
  int s0 = 0;           // lattice site carried by A_0
  std::vector<int> D;   // bond dimensions D_0 .. D_l (D_l = D_0)
  std::vector<std::vector<std::pair<int, int>>> bb;  // per bond: blocks (offset, dim)
  std::vector<std::vector<ObsBlock>> blk;            // per site: non-zero blocks
  std::vector<std::vector<int>> rb_of, cb_of;        // per site: [s][cb] -> rb, [s][rb] -> cb (or -1)
  std::vector<int64_t> aoff, eoff;                   // site tensors; environments per bond 0..l
  int64_t ysize = 0, xsize = 0;                      // largest d D_k D_k+1 and D_k^2
  double t1 = 0.0, t1r = 0.0, scale = 1.0;           // dominant eigenvalue (left, right), t1^(-1/l)
  int it_left = 0, it_right = 0;
  std::vector<std::pair<ObsList, ObsList>> unit_l, unit_r;
  ObsArena unit, env, walk;
  std::vector<int> q0;  // charge of every state of bond 0
  DevBuf A, Y, envl, envr, X[7], res, tab, emb, scal, dq0;
};

struct idmrg_ctx {
  // problem: one or more independent unit cells ("rings": a problem each,
  // e.g. disorder realisations), numbered ring after ring: ring r has
  // rings[r].ell sites from site (and bond) rings[r].s0 on and ell/2
  // superblocks from rings[r].p0 on, whose pairs close on themselves (the
  // ring's last pair takes its right block from its first).  ell is ring
  // 0's unit cell, P the superblocks of all rings.
  int ell = 0, d = 0, P = 0;
  struct Ring {
    int p0 = 0, np = 0;  // first superblock, superblocks
    int s0 = 0, ell = 0; // first site, sites
    int m = 0;           // kept states
    std::map<int, double> e1;   // e^(n)_1 of the ring's first superblock (Step 5')
    std::map<int, double> eps1; // eps^(n)_1 (Eq. tru), for the truncation error of a run
    double eg_last = NAN;
    int eg_n = -1;
  };
  std::vector<Ring> rings;
  std::vector<int> ring_of, ring_of_site;  // per superblock, per site
  std::vector<int> adim;                 // a_k per bond k (left of site k), every ring's sites
  std::vector<std::vector<double>> W;    // per site [a_k][a_k+1][d][d]
  std::vector<int> qp;                   // phys charges
  std::vector<std::vector<int>> bq;      // per bond k (left of site k) channel charges
  DevBuf dmsb;                           // kept states of every superblock (its ring's m)
  idmrg_opts o{};
  cudaStream_t st = nullptr;
  // side streams of the SVD (small Jacobi groups run beside the large one),
  // forked from and joined back to st by events
  cudaStream_t side[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t sev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  idmrg_status side_streams() {
    for (auto &x : side)
      if (!x && cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess) return IDMRG_ECUDA;
    for (auto &e : sev)
      if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return IDMRG_ECUDA;
    return IDMRG_OK;
  }
  idmrg_allocator alloc{};
  bool own_alloc = true;
  std::string err;
  uint64_t launches = 0;

  // superblocks this context steps (a contiguous range of pairs; the others
  // belong to other workers, whose boundary pair arrives by idmrg_import_pair)
  int own0 = 0, own1 = 0;
  bool plan_pending = false;  // advance() of a partial range waits for the import before planning
  bool owns(int q) const { return q >= own0 && q < own1; }
  bool owns_all() const { return own0 == 0 && own1 == P; }

  // iteration state
  int n = 1;
  std::vector<int> stage;
  std::vector<Env> envL, envR, newL, newR;
  std::vector<TruncRec> cur, prev, prev2;
  std::vector<double> energy, fidelity, bond, startnorm;
  std::vector<int> iters, conv;

  // mixed precision (tensor cores)
  bool mixed = false;
  int bf16 = 0;  // mixed with BF16 splits (64 K per packed block) instead of TF32 (32)
  bool svd_global = false;  // sector SVDs on the global-memory Jacobi kernels only
  int jac_arith = 0;        // final Jacobi of large sectors: 0 by precision, 1 FP64, 2 FP32 pairs
  bool o_oz = true;    // FP64 matvecs from digit slices (mixed restarts, FP64_TC)
  bool fp64tc = false; // IDMRG_FP64_TC: every matvec from digit slices, one Lanczos run
  bool oz_active() const { return oz_ok && o_oz && (mixed || fp64tc); }
  // FP32-pair arithmetic for the final Jacobi of large sectors: by default
  // with the mixed precisions, whose H_eff psi is far less accurate anyway;
  // FP64 and FP64_TC keep the FP64 units
  bool jac_pairs() const { return jac_arith == 2 || (jac_arith == 0 && mixed); }
  // the other FP64 GEMM lists (environments, prediction, SVD) in digit slices
  bool oz_lists() const { return o_oz && (mixed || fp64tc); }
  // split-operand GEMM lists: the L split (once per iteration) and, for
  // every N-tile candidate k (MIX_TNS[k] columns), the psi split (every
  // matvec), the R split (once per iteration, the chosen candidate's only)
  // and the tasks and tiles of both GEMM stages; tt1 / tt3 hold the tuner's
  // choice for stage 1 / stage 3
  std::vector<PackSeg> pk_L, pk_psi[MIX_NTN], pk_R[MIX_NTN];
  std::vector<TcTask> tc1k[MIX_NTN], tc3k[MIX_NTN];
  std::vector<TcTile> tc1t[MIX_NTN], tc3t[MIX_NTN];
  std::vector<WTaskP> wtp;
  std::vector<WTerm> wtpm;
  std::vector<int4> wunits;  // W stage work units (task, first row, rows)
  DevBuf dwunits;
  struct TcTune {
    int choice = -1;
    double work = -1.0;
    float ms[MIX_NTN] = {0, 0, 0};
    cudaEvent_t e0[MIX_NTN] = {}, e1[MIX_NTN] = {};
  } tt1, tt3;
  int tc_tunes = 0;  // tuning passes run (each times every candidate of a stage)
  int force_tn[2] = {0, 0};  // N tile fixed by the caller for stage 1 / stage 3 (0: tuned)
  // mixed-precision Lanczos restarts: the inner (reduced-precision) run of a
  // restart stops when its residual estimate has fallen by inner_factor, or
  // after inner_cap matvecs.  A restart cannot gain much more than the split
  // precision allows (about 1e-2 with BF16 pairs at m = 2048): a smaller
  // factor only adds matvecs.  Set at creation by precision.
  double inner_factor = 1e-3;
  int inner_cap = 80;

  int pk_L_rows = 0, pk_psi_rows = 0, pk_R_rows = 0, wtp_rows = 0;
  DevBuf dpkL, dpkp[MIX_NTN], dpkR[MIX_NTN], dtc1k[MIX_NTN], dtc1t[MIX_NTN], dtc3k[MIX_NTN], dtc3t[MIX_NTN];
  DevBuf dwtp, dwtpm, dtarget, dtune_out;
  std::vector<DevBuf> bPA1, bPB1, bT1F, bPA3, bPB3, bRMAP;
  // FP64-accurate digit-slice form of H_eff psi on the tensor cores (the
  // FP64 matvecs that start every mixed-precision Lanczos restart); usable
  // while every task's K fits the exactness bound
  bool oz_ok = false;
  std::vector<PackSeg> oz_step_w, oz_step_p, oz_psi;  // whole-K (L), part-K (R), psi
  std::vector<TcTask> oz1k, oz3k;
  std::vector<TcTile> oz1t, oz3t;
  std::vector<WTaskP> ozw;
  int oz_step_w_rows = 0, oz_step_p_rows = 0, oz_psi_rows = 0, ozw_rows = 0;
  int64_t oz_a3_lo = 0, oz_a3_hi = 0, oz_b3_lo = 0, oz_b3_hi = 0;  // exponent ranges reset before use
  std::vector<int> oz1_lo, oz3_lo;  // tile ranges of the K chunks (one launch each)
  std::vector<WTerm> wtpm_oz;
  DevBuf goz_planes, goz_exps;  // digit arena of the FP64 GEMM lists (BUF_GOZ, BUF_GEXP)
  DevBuf dozsw, dozsp, dozp, doz1k, doz1t, doz3k, doz3t, dozw, dozwm, oexp;
  std::vector<DevBuf> bOA1, bOB1, bOT1, bOA3, bOB3, bORMAP, bOT3;

  // plan for iteration n
  std::vector<SBPlan> plan;
  GemmList g1, g3, gp, genv1, genv3;
  WList wl, wenv;
  std::vector<DotTerm> dterms;
  std::vector<int> dterm_sb;
  std::vector<RandBlock> rblocks;
  int rmax_rows = 0;
  std::vector<SvdJob> jobs;
  std::vector<ScaleTask> stasks;
  int smax_rows = 0;
  std::vector<double> stable;

  // device buffers
  std::vector<double *> hbufs;
  DevBuf dbufs, dg1k, dg1s, dg3k, dg3s, dwt, dwm, ddt, ddp, drb, dgpk, dgps, dst, dstab;
  DevBuf dge1k, dge1s, dge3k, dge3s, dwet, dwem, dmask, derr;
  std::vector<DevBuf> bT1, bT3, bX, bY, bV, bW, bPsi, bUT, bVT, bStart;
  // lanczos
  DevBuf lN, lV, lw, lalpha, lbeta, libeta, lh, lpart, lk, lmember, lactive, lconv, ltheta, ly, lresid, lpsi, lv0, ldot;
  int kmax = 0, nchunk = 0;
  // svd
  DevBuf sjobs, swork, ssv, sjob0, snjob, skpj, sperm, slam, seps, sepsb, skept, scj, slamk, siw, sorder, sorderq;
  // SVD job plan of the iteration (built once, used by the batched and the
  // pipelined truncation): sectors, job ranges, per-superblock job order
  // (largest first) and Jacobi groups
  std::vector<std::vector<SecInfo>> tsecs;
  std::vector<int> tjob0, tnjob, tentries, torder, torderq, to0;
  std::vector<int64_t> tmaxel;
  std::vector<std::array<int, 4>> tg, tgcols;
  int tiw = 0, tsv = 0, tentries_max = 1, tmaxcols = 0;
  // FP32-preconditioned Jacobi: G = V^T V, W = V G (Newton-Schulz), X = B V
  GemmList svdG, svdW, svdX;
  DevBuf dsgk, dsgs, dswk, dsws, dsxk, dsxs;
  // tile-shape autotuning of every grouped-GEMM list
  GemmTune tn_g1, tn_g3, tn_gp, tn_env1, tn_env3, tn_svdG, tn_svdW, tn_svdX;
  int64_t tmaxel_all = 0;

  int svd_jobs = 0, svd_max_cols = 0, svd_max_rank = 0, svd_max_sweeps = 0;
  double svd_mean_sweeps = 0.0;
  int svd_max_sweeps32 = 0;  // FP32 stage, over the jobs of rank >= 2
  double svd_mean_sweeps32 = 0.0;
  int svd_jobs32 = 0;

  std::vector<int> hmask;
  ObsState obs;
  uint64_t mixed_matvecs = 0, fp64_matvecs = 0;
  int *pin_act = nullptr;  // pinned: active flags of two Lanczos iterations
  cudaEvent_t ev_act[2] = {nullptr, nullptr};

  // instrumentation: per-class CUDA-event timers, transfer counters
  struct KTimer {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> open;
    cudaEvent_t pending = nullptr;
    double ms = 0.0, flops = 0.0, bytes = 0.0;
    uint64_t n = 0;
  };
  bool prof = false;
  // the public classes, then the phases of the sector SVD (timed inside
  // IDMRG_K_SVD, read by idmrg_svd_phase_ms)
  static constexpr int SVD_PHASES = 6;
  static constexpr int KT_ALL = IDMRG_K_COUNT + SVD_PHASES;
  KTimer kt[KT_ALL];
  std::vector<cudaEvent_t> evpool;
  uint64_t h2d = 0, d2h = 0;

  cudaEvent_t ev_get() {
    if (!evpool.empty()) {
      cudaEvent_t e = evpool.back();
      evpool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void kbegin(int k) {
    if (!prof) return;
    kt[k].pending = ev_get();
    cudaEventRecord(kt[k].pending, st);
  }
  void kend(int k, double flops = 0.0, double bytes = 0.0) {
    if (!prof || !kt[k].pending) return;
    cudaEvent_t e1 = ev_get();
    cudaEventRecord(e1, st);
    kt[k].open.push_back({kt[k].pending, e1});
    kt[k].pending = nullptr;
    kt[k].n += 1;
    kt[k].flops += flops;
    kt[k].bytes += bytes;
    if (kt[k].open.size() > 4096) collapse(k);
  }
  void collapse(int k) {
    for (auto &pr : kt[k].open) {
      cudaEventSynchronize(pr.second);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, pr.first, pr.second);
      kt[k].ms += ms;
      evpool.push_back(pr.first);
      evpool.push_back(pr.second);
    }
    kt[k].open.clear();
  }
  cudaError_t d2h_copy(void *dst, const void *src, size_t bytes) {
    d2h += bytes;
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st);
  }

  // ------------------------------------------------------------- helpers
  idmrg_status fail(idmrg_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    err = buf;
    return s;
  }
  void *raw_alloc(size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (own_alloc) {
      void *p = nullptr;
      if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
      return p;
    }
    return alloc.alloc(bytes, alloc.user);
  }
  void raw_free(void *p, size_t bytes) {
    if (!p) return;
    if (own_alloc)
      cudaFree(p);
    else
      alloc.free(p, bytes, alloc.user);
  }
  bool ensure(DevBuf &b, size_t bytes) {
    if (b.cap >= bytes && b.p) return true;
    if (b.p) raw_free(b.p, b.cap);
    size_t cap = std::max<size_t>(bytes + bytes / 4, 1024);
    cap = (cap + 255) & ~(size_t)255;
    b.p = raw_alloc(cap);
    b.cap = b.p ? cap : 0;
    return b.p != nullptr;
  }
  void release(DevBuf &b) {
    if (b.p) raw_free(b.p, b.cap);
    b.p = nullptr;
    b.cap = 0;
  }
  template <class T>
  bool upload(DevBuf &b, const std::vector<T> &v) {
    if (!ensure(b, std::max<size_t>(v.size() * sizeof(T), 16))) return false;
    if (!v.empty() && cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return false;
    h2d += v.size() * sizeof(T);
    return true;
  }
  double *dp(DevBuf &b) { return (double *)b.p; }

  // the bond right of site s (the ring's first bond after its last site)
  int bond_right(int s) const {
    const Ring &R = rings[ring_of_site[s]];
    return s + 1 < R.s0 + R.ell ? s + 1 : R.s0;
  }
  // the pair after superblock p in its ring (Step 2': p takes its right block)
  int nxt(int p) const {
    const Ring &R = rings[ring_of[p]];
    return p + 1 < R.p0 + R.np ? p + 1 : R.p0;
  }
  // site of superblock p at iteration n: the ring's site 2 (p - p0) + n + off (mod its ell)
  int site_at(int p, int off) const {
    const Ring &R = rings[ring_of[p]];
    const int k = 2 * (p - R.p0) + n + off;
    return R.s0 + ((k % R.ell) + R.ell) % R.ell;
  }
  bool one_ring() const { return rings.size() == 1; }
  const double &Wat(int site, int a, int b, int s, int t) const {
    const int B = adim[bond_right(site)];
    return W[site][(((size_t)a * B + b) * d + s) * d + t];
  }
};

namespace {

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) return c->fail(IDMRG_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)
#define NOMEM(ok)                                                  \
  do {                                                             \
    if (!(ok)) return c->fail(IDMRG_ENOMEM, "device allocation failed (%s)", #ok); \
  } while (0)

// K chunks of at most OZ_MAX_K for one digit-slice task (see plan_oz)
static void oz_add_task(std::vector<TcTask> &tasks, std::vector<std::vector<TcTile>> &lists, TcTask t, int MT,
                        int NT) {
  const int KBt = t.KB, per = OZ_MAX_K / OZ_KBLK;
  const int nch = KBt > 0 ? (KBt + per - 1) / per : 1;
  if ((int)lists.size() < nch) lists.resize(nch);
  for (int ch = 0; ch < nch; ++ch) {
    TcTask u = t;
    u.kb_stride = KBt;
    u.kb0 = ch * per;
    u.KB = KBt > 0 ? std::min(per, KBt - u.kb0) : 0;
    u.accum = (t.accum || ch > 0) ? 1 : 0;
    const int id = (int)tasks.size();
    tasks.push_back(u);
    for (int mt = 0; mt < MT; ++mt)
      for (int nt = 0; nt < NT; ++nt) lists[ch].push_back(TcTile{id, mt, nt, 0});
  }
}

idmrg_status sync_bufs(idmrg_ctx *c);

// the digit-slice form of an FP64 GEMM list (planned with the list)
idmrg_status oz_build(idmrg_ctx *c, const GemmList &L, OzList &Z) {
  auto cdiv = [](int64_t a, int64_t b) { return (a + b - 1) / b; };
  const int64_t TA = (int64_t)128 * OZ_KBLK * OZ_PLANES, TB = (int64_t)TC_TN * OZ_KBLK * OZ_PLANES;
  Z.ok = false;
  Z.segs.clear();
  Z.tasks.clear();
  Z.tiles.clear();
  Z.seg_rows = 0;
  std::vector<std::vector<TcTile>> lists;
  int64_t an = 0, bn = 0, en = 0;
  // A planes first, B planes after all of them: B offsets are patched below
  std::vector<size_t> bseg;
  std::vector<TcTask> pend;
  std::vector<int> pmt, pnt;
  for (const GemmTask &t : L.tasks) {
    int64_t K = 0;
    for (int q = t.seg0; q < t.seg0 + t.nseg; ++q) K += L.segs[q].K;
    const int KB = (int)cdiv(std::max<int64_t>(K, 1), OZ_KBLK), MT = (int)cdiv(t.M, 128),
              NT = (int)cdiv(t.N, TC_TN);
    const int64_t pa = an, pb = bn, ea = en, eb = en + t.M;
    an += (int64_t)MT * KB * TA;
    bn += (int64_t)NT * KB * TB;
    en += t.M + t.N;
    const int whole = t.nseg == 1 ? 1 : 0;
    int k0 = 0;
    for (int q = t.seg0; q < t.seg0 + t.nseg; ++q) {
      const GemmSeg &g = L.segs[q];
      if (g.K <= 0) continue;
      PackSeg a{};
      a.dst_off = pa;
      a.src_off = g.a_off;
      a.exp_off = ea;
      a.row0 = 0;
      a.k0 = k0;
      a.rows = t.M;
      a.ks = g.K;
      a.src_ld = g.lda;
      a.trans = (g.flags & 1) ? 1 : 0;  // op(A) = A^T: element (m, k) at A[k lda + m]
      a.KB = KB;
      a.G = 16;
      a.sb = t.sb;
      a.src_buf = g.a_buf;
      a.dst_buf = BUF_GOZ;
      a.whole = whole;
      a.exp_buf = BUF_GEXP;
      a.alpha = g.alpha;
      PackSeg b = a;
      b.dst_off = pb;
      b.src_off = g.b_off;
      b.exp_off = eb;
      b.rows = t.N;
      b.src_ld = g.ldb;
      b.trans = (g.flags & 2) ? 0 : 1;  // packed row n of op(B)^T: B[k ldb + n] unless B is stored N x K
      b.G = TC_TN / 8;
      b.src_buf = g.b_buf;
      b.alpha = 1.0;
      Z.segs.push_back(a);
      bseg.push_back(Z.segs.size());
      Z.segs.push_back(b);
      Z.seg_rows = std::max(Z.seg_rows, std::max(t.M, t.N));
      k0 += g.K;
    }
    TcTask u{};
    u.a_off = pa;
    u.b_off = pb;
    u.c_off = t.c_off;
    u.a_exp = ea;
    u.b_exp = eb;
    u.sb = t.sb;
    u.M = t.M;
    u.N = t.N;
    u.KB = K > 0 ? KB : 0;
    u.a_buf = BUF_GOZ;
    u.b_buf = BUF_GOZ;
    u.c_buf = t.c_buf;
    u.mode = 2;
    u.ldc = t.ldc;
    u.accum = t.accumulate;
    u.exp_buf = BUF_GEXP;
    pend.push_back(u);
    pmt.push_back(MT);
    pnt.push_back(NT);
  }
  for (size_t i : bseg) Z.segs[i].dst_off += an;
  for (size_t i = 0; i < pend.size(); ++i) {
    pend[i].b_off += an;
    oz_add_task(Z.tasks, lists, pend[i], pmt[i], pnt[i]);
  }
  Z.lo.assign(1, 0);
  for (const auto &l : lists) {
    Z.tiles.insert(Z.tiles.end(), l.begin(), l.end());
    Z.lo.push_back((int)Z.tiles.size());
  }
  Z.planes = an + bn;
  Z.nexp = en;
  const void *p0 = c->goz_planes.p, *e0 = c->goz_exps.p;
  NOMEM(c->ensure(c->goz_planes, 2 * (size_t)std::max<int64_t>(Z.planes, 8)) &&
        c->ensure(c->goz_exps, 4 * (size_t)std::max<int64_t>(Z.nexp, 4)));
  if (c->goz_planes.p != p0 || c->goz_exps.p != e0 || c->hbufs[BUF_GOZ] != c->dp(c->goz_planes)) {
    for (int q = 0; q < c->P; ++q) {
      c->hbufs[q * NBUF + BUF_GOZ] = c->dp(c->goz_planes);
      c->hbufs[q * NBUF + BUF_GEXP] = c->dp(c->goz_exps);
    }
    NOMEM(sync_bufs(c) == IDMRG_OK);
  }
  NOMEM(c->upload(Z.dsegs, Z.segs) && c->upload(Z.dtasks, Z.tasks) && c->upload(Z.dtiles, Z.tiles));
  Z.ok = true;
  return IDMRG_OK;
}

idmrg_status oz_run(idmrg_ctx *c, OzList &Z) {
  double *const *bufs = (double *const *)c->dbufs.p;
  CK(cudaMemsetAsync(c->goz_planes.p, 0, 2 * (size_t)Z.planes, c->st));
  CK(cudaMemsetAsync(c->goz_exps.p, 0x80, 4 * (size_t)Z.nexp, c->st));
  CK(launch_oz_exp((const PackSeg *)Z.dsegs.p, (int)Z.segs.size(), Z.seg_rows, bufs, nullptr, c->st));
  CK(launch_oz_pack((const PackSeg *)Z.dsegs.p, (int)Z.segs.size(), Z.seg_rows, bufs, nullptr, c->st));
  for (size_t ch = 0; ch + 1 < Z.lo.size(); ++ch)
    CK(launch_oz_gemm((const TcTile *)Z.dtiles.p + Z.lo[ch], Z.lo[ch + 1] - Z.lo[ch], (const TcTask *)Z.dtasks.p,
                      bufs, nullptr, (int *)c->derr.p, c->st));
  c->launches += 2 + (Z.lo.size() - 1);
  return IDMRG_OK;
}

// tiles of every shape (L.tiles ends with the 64 x 64 ones) plus tasks and
// segments to the device
idmrg_status gemm_upload(idmrg_ctx *c, GemmList &L, DevBuf &dk, DevBuf &ds, GemmTune &T) {
  T.oz.ok = false;
  if (T.oz_use && c->oz_lists()) return oz_build(c, L, T.oz);
  for (int sh = GEMM_NSHAPE - 1; sh >= 0; --sh) {
    L.finish(GEMM_TM[sh], GEMM_TN[sh]);
    T.ntiles[sh] = (int)L.tiles.size();
    NOMEM(c->upload(T.tiles[sh], L.tiles));
  }
  NOMEM(c->upload(dk, L.tasks) && c->upload(ds, L.segs));
  const double w = L.flops;
  if (T.work < 0.0 || fabs(w - T.work) > 0.1 * T.work) {  // new work: tune again
    T.work = w;
    T.choice = -1;
    for (int sh = 0; sh < GEMM_NSHAPE; ++sh) T.state[sh] = 0;
  }
  return IDMRG_OK;
}

idmrg_status gemm_run(idmrg_ctx *c, GemmTune &T, DevBuf &dk, DevBuf &ds, const int *active) {
  if (T.oz.ok) return oz_run(c, T.oz);
  double *const *bufs = (double *const *)c->dbufs.p;
  int sh = T.choice;
  if (sh < 0) {
    bool all = true;
    for (int k = 0; k < GEMM_NSHAPE; ++k) {
      if (T.state[k] == 1 && cudaEventQuery(T.e1[k]) == cudaSuccess) {
        cudaEventElapsedTime(&T.ms[k], T.e0[k], T.e1[k]);
        T.state[k] = 2;
      }
      all &= T.state[k] == 2;
    }
    if (all) {
      int best = 0;
      for (int k = 1; k < GEMM_NSHAPE; ++k)
        if (T.ms[k] < T.ms[best]) best = k;
      T.choice = sh = best;
    }
  }
  if (sh >= 0) {
    CK(launch_gemm_f64((const GemmTile *)T.tiles[sh].p, T.ntiles[sh], (const GemmTask *)dk.p, (const GemmSeg *)ds.p,
                       bufs, active, c->st, sh));
    return IDMRG_OK;
  }
  int k = 0;
  while (k < GEMM_NSHAPE && T.state[k] != 0) ++k;
  if (k == GEMM_NSHAPE) k = 0;  // every shape in flight: the default
  const bool timed = T.state[k] == 0;
  if (timed) {
    if (!T.e0[k]) CK(cudaEventCreate(&T.e0[k]));
    if (!T.e1[k]) CK(cudaEventCreate(&T.e1[k]));
    CK(cudaEventRecord(T.e0[k], c->st));
  }
  CK(launch_gemm_f64((const GemmTile *)T.tiles[k].p, T.ntiles[k], (const GemmTask *)dk.p, (const GemmSeg *)ds.p, bufs,
                     active, c->st, k));
  if (timed) {
    CK(cudaEventRecord(T.e1[k], c->st));
    T.state[k] = 1;
  }
  return IDMRG_OK;
}


// ------------------------------------------------------------------------
// planning of iteration n
// ------------------------------------------------------------------------
idmrg_status plan_mixed(idmrg_ctx *c);
idmrg_status plan_oz(idmrg_ctx *c);

idmrg_status plan_iteration(idmrg_ctx *c) {
  const int P = c->P, d = c->d, target = c->o.target_charge;
  c->plan.assign(P, SBPlan());
  c->g1.clear();
  c->g3.clear();
  c->wl.clear();
  c->dterms.clear();
  c->dterm_sb.clear();
  c->rblocks.clear();
  c->rmax_rows = 0;
  const uint64_t state0 = c->o.seed;
  for (int p = 0; p < P; ++p) {
    if (!c->owns(p)) continue;  // another worker's superblock
    SBPlan &S = c->plan[p];
    S.c1 = c->site_at(p, 0);
    S.c2 = c->site_at(p, 1);
    const Env &L = c->envL[p];
    const Env &R = c->envR[c->nxt(p)];
    const Basis &BL = L.lay.b, &BR = R.lay.b;
    S.psi.build(BL, BR, c->qp, target);
    const PsiLayout &psi = S.psi;
    const int wa = c->adim[S.c1], wb = c->adim[c->bond_right(S.c1)], wc = c->adim[c->bond_right(S.c2)];
    if (wb != c->adim[S.c2] || wa != L.lay.w || wc != R.lay.w)
      return c->fail(IDMRG_EINVAL, "MPO bond dimensions do not chain at superblock %d", p);
    // two-site MPO W12[a][c][(s,t)][(s',t')] = sum_b W_c1(a,b) W_c2(b,c)
    const int dd = d * d;
    S.W12.assign((size_t)wa * wc * dd * dd, 0.0);
    for (int a = 0; a < wa; ++a)
      for (int b = 0; b < wb; ++b)
        for (int s = 0; s < d; ++s)
          for (int s2 = 0; s2 < d; ++s2) {
            const double w1 = c->Wat(S.c1, a, b, s, s2);
            if (w1 == 0.0) continue;
            for (int cc = 0; cc < wc; ++cc)
              for (int t = 0; t < d; ++t)
                for (int t2 = 0; t2 < d; ++t2) {
                  const double w2 = c->Wat(S.c2, b, cc, t, t2);
                  if (w2 == 0.0) continue;
                  S.W12[(((size_t)a * wc + cc) * dd + s * d + t) * dd + s2 * d + t2] += w1 * w2;
                }
          }
    // centre-bond operator: channels opened on c1 and closed on c2
    S.h2.assign((size_t)dd * dd, 0.0);
    for (int b = 1; b < wb - 1; ++b)
      for (int s = 0; s < d; ++s)
        for (int s2 = 0; s2 < d; ++s2) {
          const double w1 = c->Wat(S.c1, wa - 1, b, s, s2);
          if (w1 == 0.0) continue;
          for (int t = 0; t < d; ++t)
            for (int t2 = 0; t2 < d; ++t2) S.h2[(s * d + t) * dd + s2 * d + t2] += w1 * c->Wat(S.c2, b, 0, t, t2);
        }
    const int SL = BL.S(), SR = BR.S();
    // ---- stage 1: T1[a] = L_a psi, one task per (a, in-sector)
    S.t1off.assign((size_t)wa * SL, -1);
    S.t1size = 0;
    const double f0 = c->g1.flops;
    for (int a = 0; a < wa; ++a)
      for (int si = 0; si < SL; ++si) {
        const int so = L.lay.so[a * SL + si];
        if (so < 0 || psi.C[si] == 0) continue;
        S.t1off[a * SL + si] = S.t1size;
        S.t1size += (int64_t)BL.dim[so] * psi.C[si];
        c->g1.task(p, BUF_T1, S.t1off[a * SL + si], BL.dim[so], psi.C[si], psi.C[si]);
        c->g1.seg(BUF_L, L.lay.off[a * SL + si], BL.dim[si], BUF_IN, psi.roff[si], psi.C[si], BL.dim[si], 0);
      }
    // ---- T3 layout: T3[c] row block per left sector i, sub-blocks (s,t)
    S.t3off.assign((size_t)wc * SL, 0);
    S.t3C.assign((size_t)wc * SL, 0);
    S.t3col.assign((size_t)wc * SL * dd, -1);
    S.t3size = 0;
    for (int cc = 0; cc < wc; ++cc)
      for (int i = 0; i < SL; ++i) {
        int cols = 0;
        for (int s = 0; s < d; ++s)
          for (int t = 0; t < d; ++t) {
            const int qsum = BL.q[i] + c->qp[s] + c->qp[t];
            const int jout = BR.find(target - qsum);
            if (jout < 0) continue;
            const int jin = BR.find(target - qsum - R.lay.chq[cc]);
            if (jin < 0 || R.lay.so[cc * SR + jin] != jout) continue;
            S.t3col[((size_t)cc * SL + i) * dd + s * d + t] = cols;
            cols += BR.dim[jin];
          }
        S.t3C[cc * SL + i] = cols;
        S.t3off[cc * SL + i] = S.t3size;
        S.t3size += (int64_t)BL.dim[i] * cols;
      }
    // ---- stage 2: T3 = W12 T1
    const double fw0 = c->wl.flops;
    for (int cc = 0; cc < wc; ++cc)
      for (int i = 0; i < SL; ++i)
        for (int s = 0; s < d; ++s)
          for (int t = 0; t < d; ++t) {
            const int col = S.t3col[((size_t)cc * SL + i) * dd + s * d + t];
            if (col < 0) continue;
            const int qsum = BL.q[i] + c->qp[s] + c->qp[t];
            const int jin = BR.find(target - qsum - R.lay.chq[cc]);
            c->wl.task(p, BUF_T3, S.t3off[cc * SL + i] + col, S.t3C[cc * SL + i], BUF_T1, BL.dim[i], BR.dim[jin]);
            for (int a = 0; a < wa; ++a) {
              const int si = BL.find(BL.q[i] - L.lay.chq[a]);
              if (si < 0 || L.lay.so[a * SL + si] != i || S.t1off[a * SL + si] < 0) continue;
              for (int s2 = 0; s2 < d; ++s2)
                for (int t2 = 0; t2 < d; ++t2) {
                  const double cf = S.W12[(((size_t)a * wc + cc) * dd + s * d + t) * dd + s2 * d + t2];
                  if (cf == 0.0) continue;
                  const int k = psi.sub(si, s2, t2);
                  if (psi.sj[k] != jin) continue;
                  c->wl.term(S.t1off[a * SL + si] + psi.scol[k], psi.C[si], cf);
                }
            }
          }
    // ---- stage 3: out = sum_c T3[c] R_c^T
    const double f3 = c->g3.flops;
    for (int i = 0; i < SL; ++i)
      for (int s = 0; s < d; ++s)
        for (int t = 0; t < d; ++t) {
          const int k = psi.sub(i, s, t);
          const int jout = psi.sj[k];
          if (jout < 0) continue;
          c->g3.task(p, BUF_OUT, psi.roff[i] + psi.scol[k], BL.dim[i], BR.dim[jout], psi.C[i]);
          for (int cc = 0; cc < wc; ++cc) {
            const int col = S.t3col[((size_t)cc * SL + i) * dd + s * d + t];
            if (col < 0) continue;
            const int jin = BR.find(target - BL.q[i] - c->qp[s] - c->qp[t] - R.lay.chq[cc]);
            c->g3.seg(BUF_T3, S.t3off[cc * SL + i] + col, S.t3C[cc * SL + i], BUF_R, R.lay.off[cc * SR + jin],
                      BR.dim[jin], BR.dim[jin], 2);
          }
        }
    S.gemm_flops = (c->g1.flops - f0) + (c->g3.flops - f3);
    S.w_flops = c->wl.flops - fw0;
    S.heff_flops = S.gemm_flops + S.w_flops;
    S.heff_bytes = 8.0 * (L.lay.size + R.lay.size + 2.0 * psi.N);
    S.wpack_elems = (double)psi.N;
    S.wt1_elems = (double)S.t1size;
    S.wt3_elems = (double)S.t3size;
    // ---- centre-bond energy terms
    for (int i = 0; i < SL; ++i)
      for (int x = 0; x < dd; ++x)
        for (int y = 0; y < dd; ++y) {
          const double cf = S.h2[x * dd + y];
          if (cf == 0.0) continue;
          const int k1 = psi.sub(i, x / d, x % d), k2 = psi.sub(i, y / d, y % d);
          if (psi.sj[k1] < 0 || psi.sj[k1] != psi.sj[k2]) continue;
          DotTerm dt{};
          dt.off1 = psi.roff[i] + psi.scol[k1];
          dt.off2 = psi.roff[i] + psi.scol[k2];
          dt.ld1 = dt.ld2 = psi.C[i];
          dt.rows = BL.dim[i];
          dt.cols = BR.dim[psi.sj[k1]];
          dt.sb = p;
          dt.buf = BUF_PSI;
          dt.coef = cf;
          c->dterms.push_back(dt);
          c->dterm_sb.push_back(p);
        }
    // ---- random start blocks (Step 3, n = 1, 2)
    // ring-local index: a problem draws the same start as in a context of its own
    const uint64_t sstate = sm64_at(state0, (uint64_t)(1024 * (int64_t)c->n + (p - c->rings[c->ring_of[p]].p0)));
    for (int i = 0; i < SL; ++i)
      for (int s = 0; s < d; ++s)
        for (int t = 0; t < d; ++t) {
          const int k = psi.sub(i, s, t);
          const int j = psi.sj[k];
          if (j < 0) continue;
          RandBlock rb{};
          rb.off = psi.roff[i] + psi.scol[k];
          rb.rows = BL.dim[i];
          rb.cols = BR.dim[j];
          rb.ld = psi.C[i];
          rb.sb = p;
          rb.dense0 = (((int64_t)BL.off[i] * d + s) * d + t) * BR.D + BR.off[j];
          rb.dense_rs = (int64_t)d * d * BR.D;
          rb.state = sstate;
          c->rblocks.push_back(rb);
          c->rmax_rows = std::max(c->rmax_rows, rb.rows);
        }
  }

  // ---- device buffers for this iteration
  {
    idmrg_status sg = gemm_upload(c, c->g1, c->dg1k, c->dg1s, c->tn_g1);
    if (sg != IDMRG_OK) return sg;
    sg = gemm_upload(c, c->g3, c->dg3k, c->dg3s, c->tn_g3);
    if (sg != IDMRG_OK) return sg;
  }
  NOMEM(c->upload(c->dwt, c->wl.tasks) && c->upload(c->dwm, c->wl.terms));
  NOMEM(c->upload(c->ddt, c->dterms) && c->ensure(c->ddp, std::max<size_t>(c->dterms.size(), 1) * 8));
  NOMEM(c->upload(c->drb, c->rblocks));
  for (int p = 0; p < P; ++p) {
    SBPlan &S = c->plan[p];
    NOMEM(c->ensure(c->bT1[p], 8 * std::max<int64_t>(S.t1size, 1)));
    NOMEM(c->ensure(c->bT3[p], 8 * std::max<int64_t>(S.t3size, 1)));
    NOMEM(c->ensure(c->bPsi[p], 8 * std::max<int64_t>(S.psi.N, 1)));
    NOMEM(c->ensure(c->bW[p], 8 * std::max<int64_t>(S.psi.N, 1)));
    c->hbufs[p * NBUF + BUF_L] = c->dp(c->envL[p].data);
    c->hbufs[p * NBUF + BUF_R] = c->dp(c->envR[c->nxt(p)].data);
    c->hbufs[p * NBUF + BUF_T1] = c->dp(c->bT1[p]);
    c->hbufs[p * NBUF + BUF_T3] = c->dp(c->bT3[p]);
    c->hbufs[p * NBUF + BUF_PSI] = c->dp(c->bPsi[p]);
  }
  NOMEM(c->upload(c->dbufs, c->hbufs));
  if (c->mixed) {
    idmrg_status s = plan_mixed(c);
    if (s != IDMRG_OK) return s;
  }
  if (c->mixed || c->fp64tc) {
    idmrg_status s = plan_oz(c);
    if (s != IDMRG_OK) return s;
  }
  for (int p = 0; p < P; ++p) c->stage[p] = ST_READY;
  return IDMRG_OK;
}

idmrg_status sync_bufs(idmrg_ctx *c) {
  NOMEM(c->upload(c->dbufs, c->hbufs));
  return IDMRG_OK;
}

// Tensor-core form of every superblock's H_eff psi (see kernels_tc.cu):
//   stage 1, per in-sector si of the left block: rows = (channel a, x) of the
//     L_a blocks stacked over a, K = x' in si, N = the psi row block of si;
//   stage 3, per out-sector jo of the right block: rows = (i, s, t, x) of the
//     psi sub-blocks with right sector jo, K = (channel c, y') concatenated over
//     the R channels, N = y in jo.
// N-tile tuner of one split-operand GEMM stage (1: L psi, 3: T3 R^T): each
// candidate of MIX_TNS runs twice on the current plan's operands (the second
// run timed with events on the context's stream) and the fastest is kept.
// It runs again only when the stage's work has moved by more than 10 %.
// The operands may hold zeros or values left from another layout; the tuning
// runs only write buffers that the next matvec rewrites (stage 1: T1; stage 3:
// a scratch vector put in the output slot meanwhile).  Stage 3 packs R in each
// candidate's layout before timing it; the caller packs the chosen one.
idmrg_status check_dev_err(idmrg_ctx *c);
idmrg_status tc_tune(idmrg_ctx *c, idmrg_ctx::TcTune &T, int stage, double work, int64_t max_psi) {
  const int forced = c->force_tn[stage == 1 ? 0 : 1];
  if (forced > 0) {
    for (int k = 0; k < MIX_NTN; ++k)
      if (MIX_TNS[k] == forced) T.choice = k;
    T.work = -1.0;  // tune again once the tile is no longer fixed
    return IDMRG_OK;
  }
  if (T.choice >= 0 && T.work > 0.0 && fabs(work - T.work) <= 0.1 * T.work) return IDMRG_OK;
  T.work = work;
  T.choice = 0;
  auto &tiles = stage == 1 ? c->tc1t : c->tc3t;
  bool any = false;
  for (int k = 0; k < MIX_NTN; ++k) any |= !tiles[k].empty();
  if (!any) return IDMRG_OK;
  const int P = c->P;
  std::vector<double *> keep(P, nullptr);
  if (stage == 3) {
    NOMEM(c->ensure(c->dtune_out, 8 * (size_t)max_psi));
    for (int p = 0; p < P; ++p) {
      keep[p] = c->hbufs[p * NBUF + BUF_OUT];
      if (c->owns(p)) c->hbufs[p * NBUF + BUF_OUT] = c->dp(c->dtune_out);
    }
    NOMEM(c->upload(c->dbufs, c->hbufs));
  }
  double *const *bufs = (double *const *)c->dbufs.p;
  for (int k = 0; k < MIX_NTN; ++k) {
    if (!T.e0[k]) CK(cudaEventCreate(&T.e0[k]));
    if (!T.e1[k]) CK(cudaEventCreate(&T.e1[k]));
    if (stage == 3) {
      CK(launch_pack((const PackSeg *)c->dpkR[k].p, (int)c->pk_R[k].size(), c->pk_R_rows, bufs, nullptr, c->bf16,
                     c->st));
      c->launches += 1;
    }
    const TcTile *dt = (const TcTile *)(stage == 1 ? c->dtc1t[k].p : c->dtc3t[k].p);
    const TcTask *dk = (const TcTask *)(stage == 1 ? c->dtc1k[k].p : c->dtc3k[k].p);
    const int nt = (int)tiles[k].size();
    for (int rep = 0; rep < 2; ++rep) {
      if (rep == 1) CK(cudaEventRecord(T.e0[k], c->st));
      CK(launch_tc_gemm(dt, nt, dk, bufs, nullptr, (int *)c->derr.p, c->bf16, MIX_TNS[k], c->st));
      c->launches += 1;
    }
    CK(cudaEventRecord(T.e1[k], c->st));
  }
  CK(cudaStreamSynchronize(c->st));
  for (int k = 0; k < MIX_NTN; ++k) {
    CK(cudaEventElapsedTime(&T.ms[k], T.e0[k], T.e1[k]));
    if (T.ms[k] < T.ms[T.choice]) T.choice = k;
  }
  c->tc_tunes += 1;
  if (stage == 3) {
    for (int p = 0; p < P; ++p) c->hbufs[p * NBUF + BUF_OUT] = keep[p];
    NOMEM(c->upload(c->dbufs, c->hbufs));
  }
  return check_dev_err(c);
}

idmrg_status plan_mixed(idmrg_ctx *c) {
  const int P = c->P, d = c->d, target = c->o.target_charge, dd = d * d;
  const int GA = 16;
  // one packed K block is 128 bytes of every row: TA floats per hi or lo A
  // tile, 32 per row of a B tile
  const int64_t TA = 128 * 32;
  const int kblk = c->bf16 ? 64 : 32;
  auto cdiv = [](int64_t a, int64_t b) { return (a + b - 1) / b; };
  c->pk_L.clear();
  for (int k = 0; k < MIX_NTN; ++k) {
    c->pk_psi[k].clear();
    c->pk_R[k].clear();
    c->tc1k[k].clear();
    c->tc1t[k].clear();
    c->tc3k[k].clear();
    c->tc3t[k].clear();
  }
  c->wtp.clear();
  c->wtpm.clear();
  c->pk_L_rows = c->pk_psi_rows = c->pk_R_rows = c->wtp_rows = 0;
  double work1 = 0.0, work3 = 0.0;
  int64_t max_psi = 1;
  auto seg = [&](std::vector<PackSeg> &v, int &mr, int sb, int dst_buf, int64_t dst_off, int src_buf,
                 int64_t src_off, int row0, int k0, int rows, int ks, int ld, int trans, int KB, int G) {
    if (rows <= 0 || ks <= 0) return;
    PackSeg p{};
    p.dst_off = dst_off;
    p.src_off = src_off;
    p.row0 = row0;
    p.k0 = k0;
    p.rows = rows;
    p.ks = ks;
    p.src_ld = ld;
    p.trans = trans;
    p.KB = KB;
    p.G = G;
    p.sb = sb;
    p.src_buf = src_buf;
    p.dst_buf = dst_buf;
    p.src_fp32 = 0;
    v.push_back(p);
    mr = std::max(mr, rows);
  };
  for (int p = 0; p < P; ++p) {
    if (!c->owns(p)) continue;
    SBPlan &S = c->plan[p];
    const Env &L = c->envL[p];
    const Env &R = c->envR[c->nxt(p)];
    const Basis &BL = L.lay.b, &BR = R.lay.b;
    const PsiLayout &psi = S.psi;
    const int SL = BL.S(), SR = BR.S();
    const int wa = L.lay.w, wc = R.lay.w;
    // ---------------- stage 1
    std::vector<int64_t> pa1(SL, -1), t1f(SL, -1);
    std::vector<std::vector<int>> rs1(SL, std::vector<int>(wa, -1));
    int64_t pa1n = 0, pb1n[MIX_NTN] = {0, 0, 0}, t1fn = 0;
    max_psi = std::max<int64_t>(max_psi, psi.N);
    for (int si = 0; si < SL; ++si) {
      if (psi.C[si] == 0) continue;
      int M = 0;
      for (int a = 0; a < wa; ++a) {
        const int so = L.lay.so[a * SL + si];
        if (so < 0) continue;
        rs1[si][a] = M;
        M += BL.dim[so];
      }
      if (M == 0) continue;
      const int K = BL.dim[si], N = psi.C[si];
      const int KB = (int)cdiv(K, kblk), MT = (int)cdiv(M, 128);
      pa1[si] = pa1n;
      pa1n += (int64_t)MT * KB * 2 * TA;
      t1f[si] = t1fn;
      t1fn += (int64_t)M * N;
      work1 += 2.0 * M * K * N;
      for (int a = 0; a < wa; ++a) {
        if (rs1[si][a] < 0) continue;
        const int so = L.lay.so[a * SL + si];
        seg(c->pk_L, c->pk_L_rows, p, BUF_PA1, pa1[si], BUF_L, L.lay.off[a * SL + si], rs1[si][a], 0,
            BL.dim[so], K, K, 0, KB, GA);
      }
      for (int k = 0; k < MIX_NTN; ++k) {  // B (psi) layout, task and tiles per N tile
        const int TN = MIX_TNS[k], NT = (int)cdiv(N, TN);
        const int64_t pb = pb1n[k];
        pb1n[k] += (int64_t)NT * KB * 2 * TN * 32;
        seg(c->pk_psi[k], c->pk_psi_rows, p, BUF_PB1, pb, BUF_IN, psi.roff[si], 0, 0, N, K, N, 1, KB, TN / 8);
        TcTask t{};
        t.a_off = pa1[si];
        t.b_off = pb;
        t.c_off = t1f[si];
        t.sb = p;
        t.M = M;
        t.N = N;
        t.KB = KB;
        t.a_buf = BUF_PA1;
        t.b_buf = BUF_PB1;
        t.c_buf = BUF_T1F;
        t.mode = 0;
        t.ldc = N;
        const int id = (int)c->tc1k[k].size();
        c->tc1k[k].push_back(t);
        for (int mt = 0; mt < MT; ++mt)
          for (int nt = 0; nt < NT; ++nt) c->tc1t[k].push_back(TcTile{id, mt, nt, 0});
      }
    }
    // ---------------- stage 3
    std::vector<int64_t> pa3(SR, -1), rmo(SR, -1);
    std::vector<int64_t> rmap;
    int64_t pa3n = 0, pb3n[MIX_NTN] = {0, 0, 0};
    for (int jo = 0; jo < SR; ++jo) {
      // K: channels c whose R_c block lands in jo
      std::vector<int> ks(wc, -1);
      int K = 0;
      for (int cc = 0; cc < wc; ++cc) {
        const int jin = BR.find(BR.q[jo] - R.lay.chq[cc]);
        if (jin < 0 || R.lay.so[cc * SR + jin] != jo) continue;
        ks[cc] = K;
        K += BR.dim[jin];
      }
      // rows: sub-blocks (i, s, t) with right sector jo
      std::vector<int> rows_of(SL * dd, -1);
      int M = 0;
      const int64_t r0 = (int64_t)rmap.size();
      for (int i = 0; i < SL; ++i)
        for (int s = 0; s < d; ++s)
          for (int t = 0; t < d; ++t) {
            const int k = psi.sub(i, s, t);
            if (psi.sj[k] != jo) continue;
            rows_of[k] = M;
            for (int x = 0; x < BL.dim[i]; ++x) rmap.push_back(psi.roff[i] + (int64_t)x * psi.C[i] + psi.scol[k]);
            M += BL.dim[i];
          }
      if (M == 0) continue;
      const int N = BR.dim[jo];
      const int KB = (int)cdiv(std::max(K, 1), kblk), MT = (int)cdiv(M, 128);
      pa3[jo] = pa3n;
      pa3n += (int64_t)MT * KB * 2 * TA;
      rmo[jo] = r0;
      work3 += 2.0 * M * K * N;
      int64_t pb3[MIX_NTN];
      for (int k = 0; k < MIX_NTN; ++k) {  // B (R) layout per N tile
        const int TN = MIX_TNS[k], NT = (int)cdiv(N, TN);
        pb3[k] = pb3n[k];
        pb3n[k] += (int64_t)NT * KB * 2 * TN * 32;
        for (int cc = 0; cc < wc; ++cc) {
          if (ks[cc] < 0) continue;
          const int jin = BR.find(BR.q[jo] - R.lay.chq[cc]);
          seg(c->pk_R[k], c->pk_R_rows, p, BUF_PB3, pb3[k], BUF_R, R.lay.off[cc * SR + jin], 0, ks[cc], N,
              BR.dim[jin], BR.dim[jin], 0, KB, TN / 8);
        }
      }
      // W stage: T3[c](i,s,t) into rows rows_of(i,s,t), columns ks[c]
      for (int i = 0; i < SL; ++i)
        for (int s = 0; s < d; ++s)
          for (int t = 0; t < d; ++t) {
            const int k = psi.sub(i, s, t);
            if (rows_of[k] < 0) continue;
            for (int cc = 0; cc < wc; ++cc) {
              if (ks[cc] < 0) continue;
              const int jin = BR.find(BR.q[jo] - R.lay.chq[cc]);
              WTaskP w{};
              w.dst_off = pa3[jo];
              w.row0 = rows_of[k];
              w.k0 = ks[cc];
              w.KB = KB;
              w.G = GA;
              w.sb = p;
              w.rows = BL.dim[i];
              w.cols = BR.dim[jin];
              w.in_buf = BUF_T1F;
              w.dst_buf = BUF_PA3;
              w.term0 = (int)c->wtpm.size();
              for (int a = 0; a < wa; ++a) {
                const int si = BL.find(BL.q[i] - L.lay.chq[a]);
                if (si < 0 || L.lay.so[a * SL + si] != i || rs1[si][a] < 0) continue;
                for (int s2 = 0; s2 < d; ++s2)
                  for (int t2 = 0; t2 < d; ++t2) {
                    const double cf = S.W12[(((size_t)a * wc + cc) * dd + s * d + t) * dd + s2 * d + t2];
                    if (cf == 0.0) continue;
                    const int k2 = psi.sub(si, s2, t2);
                    if (psi.sj[k2] != jin) continue;
                    WTerm term{};
                    term.in_off = t1f[si] + (int64_t)rs1[si][a] * psi.C[si] + psi.scol[k2];
                    term.in_ld = psi.C[si];
                    term.coef = cf;
                    c->wtpm.push_back(term);
                  }
              }
              w.nterm = (int)c->wtpm.size() - w.term0;
              if (w.nterm == 0) continue;  // the packed rectangle stays zero
              c->wtp.push_back(w);
              c->wtp_rows = std::max(c->wtp_rows, w.rows);
            }
          }
      for (int k = 0; k < MIX_NTN; ++k) {
        const int NT = (int)cdiv(N, MIX_TNS[k]);
        TcTask t{};
        t.a_off = pa3[jo];
        t.b_off = pb3[k];
        t.rmap_off = rmo[jo];
        t.sb = p;
        t.M = M;
        t.N = N;
        t.KB = K > 0 ? KB : 0;
        t.a_buf = BUF_PA3;
        t.b_buf = BUF_PB3;
        t.c_buf = BUF_OUT;
        t.rmap_buf = BUF_RMAP;
        t.mode = 1;
        const int id = (int)c->tc3k[k].size();
        c->tc3k[k].push_back(t);
        for (int mt = 0; mt < MT; ++mt)
          for (int nt = 0; nt < NT; ++nt) c->tc3t[k].push_back(TcTile{id, mt, nt, 0});
      }
    }
    // B operands sized for the widest layout of any candidate
    const int64_t pb1max = std::max({pb1n[0], pb1n[1], pb1n[2]}), pb3max = std::max({pb3n[0], pb3n[1], pb3n[2]});
    NOMEM(c->ensure(c->bPA1[p], 4 * std::max<int64_t>(pa1n, 4)) &&
          c->ensure(c->bPB1[p], 4 * std::max<int64_t>(pb1max, 4)) &&
          c->ensure(c->bT1F[p], 4 * std::max<int64_t>(t1fn, 4)) &&
          c->ensure(c->bPA3[p], 4 * std::max<int64_t>(pa3n, 4)) &&
          c->ensure(c->bPB3[p], 4 * std::max<int64_t>(pb3max, 4)) && c->upload(c->bRMAP[p], rmap));
    // zero padding of every packed operand (only real elements are rewritten
    // later; a K block's padding is zero in A, so B's padding only has to
    // hold finite values, which a switch of B layouts leaves behind)
    CK(cudaMemsetAsync(c->bPA1[p].p, 0, 4 * pa1n, c->st));
    CK(cudaMemsetAsync(c->bPB1[p].p, 0, 4 * pb1max, c->st));
    CK(cudaMemsetAsync(c->bPA3[p].p, 0, 4 * pa3n, c->st));
    CK(cudaMemsetAsync(c->bPB3[p].p, 0, 4 * pb3max, c->st));
    c->hbufs[p * NBUF + BUF_PA1] = c->dp(c->bPA1[p]);
    c->hbufs[p * NBUF + BUF_PB1] = c->dp(c->bPB1[p]);
    c->hbufs[p * NBUF + BUF_T1F] = c->dp(c->bT1F[p]);
    c->hbufs[p * NBUF + BUF_PA3] = c->dp(c->bPA3[p]);
    c->hbufs[p * NBUF + BUF_PB3] = c->dp(c->bPB3[p]);
    c->hbufs[p * NBUF + BUF_RMAP] = c->dp(c->bRMAP[p]);
  }
  // W stage units: windows of 32 rows x 64 packed K columns of each rectangle
  c->wunits.clear();
  for (size_t k = 0; k < c->wtp.size(); ++k) {
    const WTaskP &w = c->wtp[k];
    for (int r0 = 0; r0 < w.rows; r0 += 32)
      for (int kw = w.k0 / 64; kw <= (w.k0 + w.cols - 1) / 64; ++kw) c->wunits.push_back(make_int4((int)k, r0, kw, 0));
  }
  NOMEM(c->upload(c->dwunits, c->wunits));
  NOMEM(c->upload(c->dpkL, c->pk_L) && c->upload(c->dwtp, c->wtp) && c->upload(c->dwtpm, c->wtpm));
  for (int k = 0; k < MIX_NTN; ++k)
    NOMEM(c->upload(c->dpkp[k], c->pk_psi[k]) && c->upload(c->dpkR[k], c->pk_R[k]) &&
          c->upload(c->dtc1k[k], c->tc1k[k]) && c->upload(c->dtc1t[k], c->tc1t[k]) &&
          c->upload(c->dtc3k[k], c->tc3k[k]) && c->upload(c->dtc3t[k], c->tc3t[k]));
  NOMEM(c->upload(c->dbufs, c->hbufs));
  // split L once for this iteration
  c->kbegin(IDMRG_K_HEFF_WSTAGE);
  CK(launch_pack((const PackSeg *)c->dpkL.p, (int)c->pk_L.size(), c->pk_L_rows, (double *const *)c->dbufs.p,
                 nullptr, c->bf16, c->st));
  c->kend(IDMRG_K_HEFF_WSTAGE);
  c->launches += 1;
  // N tiles: tuned whenever a stage's work moved by more than 10 % since
  // its last tuning (every iteration while the blocks grow, rarely after)
  idmrg_status ts = tc_tune(c, c->tt1, 1, work1, max_psi);
  if (ts != IDMRG_OK) return ts;
  ts = tc_tune(c, c->tt3, 3, work3, max_psi);
  if (ts != IDMRG_OK) return ts;
  // split R once for this iteration, in the chosen stage-3 layout
  const int k3 = c->tt3.choice;
  c->kbegin(IDMRG_K_HEFF_WSTAGE);
  CK(launch_pack((const PackSeg *)c->dpkR[k3].p, (int)c->pk_R[k3].size(), c->pk_R_rows,
                 (double *const *)c->dbufs.p, nullptr, c->bf16, c->st));
  c->kend(IDMRG_K_HEFF_WSTAGE);
  c->launches += 1;
  return IDMRG_OK;
}

// Digit-slice form (FP64-accurate, see kernels_tc.cu): the stage-1 / W /
// stage-3 structure of plan_mixed with 32-element K blocks of eight BF16
// digit planes and one exponent per packed row.  Exponents of every
// superblock live in one array: [stage-1 A and B rows | stage-3 B rows |
// stage-3 A rows]; the last two ranges are reset before their atomic
// maxima are taken.  Tasks whose K exceeds OZ_MAX_K (the bound of exact
// digit sums) run in K chunks, one launch per chunk, later chunks adding
// their FP64 results.
idmrg_status plan_oz(idmrg_ctx *c) {
  const int P = c->P, d = c->d, target = c->o.target_charge, dd = d * d;
  const int GA = 16, GB = TC_TN / 8;
  const int64_t TA = (int64_t)128 * OZ_KBLK * OZ_PLANES, TB = (int64_t)TC_TN * OZ_KBLK * OZ_PLANES;
  auto cdiv = [](int64_t a, int64_t b) { return (a + b - 1) / b; };
  c->oz_ok = false;
  c->oz_step_w.clear();
  c->oz_step_p.clear();
  c->oz_psi.clear();
  c->oz1k.clear();
  c->oz1t.clear();
  c->oz3k.clear();
  c->oz3t.clear();
  c->ozw.clear();
  c->wtpm_oz.clear();
  c->oz_step_w_rows = c->oz_step_p_rows = c->oz_psi_rows = c->ozw_rows = 0;
  auto seg = [&](std::vector<PackSeg> &v, int &mr, int sb, int dst_buf, int64_t dst_off, int src_buf,
                 int64_t src_off, int64_t exp_off, int row0, int k0, int rows, int ks, int ld, int trans, int KB,
                 int G, int whole) {
    if (rows <= 0 || ks <= 0) return;
    PackSeg q{};
    q.dst_off = dst_off;
    q.src_off = src_off;
    q.exp_off = exp_off;
    q.row0 = row0;
    q.k0 = k0;
    q.rows = rows;
    q.ks = ks;
    q.src_ld = ld;
    q.trans = trans;
    q.KB = KB;
    q.G = G;
    q.sb = sb;
    q.src_buf = src_buf;
    q.dst_buf = dst_buf;
    q.whole = whole;
    q.exp_buf = BUF_OEXP;
    q.alpha = 1.0;
    v.push_back(q);
    mr = std::max(mr, rows);
  };
  // a task in K chunks of at most OZ_MAX_K (exact digit sums); the tiles of
  // chunk c go to lists[c], launched one chunk after the other
  std::vector<std::vector<TcTile>> t1c, t3c;
  auto add_task = [&](std::vector<TcTask> &tasks, std::vector<std::vector<TcTile>> &lists, TcTask t, int MT,
                      int NT) {
    const int KBt = t.KB, per = OZ_MAX_K / OZ_KBLK;
    const int nch = KBt > 0 ? (KBt + per - 1) / per : 1;
    if ((int)lists.size() < nch) lists.resize(nch);
    for (int ch = 0; ch < nch; ++ch) {
      TcTask u = t;
      u.kb_stride = KBt;
      u.kb0 = ch * per;
      u.KB = KBt > 0 ? std::min(per, KBt - u.kb0) : 0;
      u.accum = (t.accum || ch > 0) ? 1 : 0;
      const int id = (int)tasks.size();
      tasks.push_back(u);
      for (int mt = 0; mt < MT; ++mt)
        for (int nt = 0; nt < NT; ++nt) lists[ch].push_back(TcTile{id, mt, nt, 0});
    }
  };
  int64_t ex1 = 0, exb3 = 0, exa3 = 0;  // the three exponent ranges, relative
  const size_t b3seg0 = 0;
  std::vector<size_t> a3_tasks, b3_tasks;  // tasks / items whose offsets get the range bases
  std::vector<std::vector<int64_t>> rmaps(P);
  std::vector<int64_t> na1(P), nb1(P), nt1(P), na3(P), nb3(P), nt3(P);
  for (int p = 0; p < P; ++p) {
    if (!c->owns(p)) continue;
    SBPlan &S = c->plan[p];
    const Env &L = c->envL[p];
    const Env &R = c->envR[c->nxt(p)];
    const Basis &BL = L.lay.b, &BR = R.lay.b;
    const PsiLayout &psi = S.psi;
    const int SL = BL.S(), SR = BR.S();
    const int wa = L.lay.w, wc = R.lay.w;
    // ---------------- stage 1
    std::vector<int64_t> t1f(SL, -1);
    std::vector<std::vector<int>> rs1(SL, std::vector<int>(wa, -1));
    int64_t pa1n = 0, pb1n = 0, t1n = 0;
    for (int si = 0; si < SL; ++si) {
      if (psi.C[si] == 0) continue;
      int M = 0;
      for (int a = 0; a < wa; ++a) {
        const int so = L.lay.so[a * SL + si];
        if (so < 0) continue;
        rs1[si][a] = M;
        M += BL.dim[so];
      }
      if (M == 0) continue;
      const int K = BL.dim[si], N = psi.C[si];
      const int KB = (int)cdiv(K, OZ_KBLK), MT = (int)cdiv(M, 128), NT = (int)cdiv(N, TC_TN);
      const int64_t pa = pa1n, pb = pb1n, ea = ex1, eb = ex1 + M;
      pa1n += (int64_t)MT * KB * TA;
      pb1n += (int64_t)NT * KB * TB;
      ex1 += M + N;
      t1f[si] = t1n;
      t1n += (int64_t)M * N;
      for (int a = 0; a < wa; ++a) {
        if (rs1[si][a] < 0) continue;
        const int so = L.lay.so[a * SL + si];
        seg(c->oz_step_w, c->oz_step_w_rows, p, BUF_OA1, pa, BUF_L, L.lay.off[a * SL + si], ea, rs1[si][a], 0,
            BL.dim[so], K, K, 0, KB, GA, 1);
      }
      seg(c->oz_psi, c->oz_psi_rows, p, BUF_OB1, pb, BUF_IN, psi.roff[si], eb, 0, 0, N, K, N, 1, KB, GB, 1);
      TcTask t{};
      t.a_off = pa;
      t.b_off = pb;
      t.c_off = t1f[si];
      t.a_exp = ea;
      t.b_exp = eb;
      t.sb = p;
      t.M = M;
      t.N = N;
      t.KB = KB;
      t.a_buf = BUF_OA1;
      t.b_buf = BUF_OB1;
      t.c_buf = BUF_OT1;
      t.exp_buf = BUF_OEXP;
      t.mode = 2;
      t.ldc = N;
      add_task(c->oz1k, t1c, t, MT, NT);
    }
    // ---------------- stage 3
    int64_t pa3n = 0, pb3n = 0, nt3s = 0;
    std::vector<int64_t> &rmap = rmaps[p];
    for (int jo = 0; jo < SR; ++jo) {
      std::vector<int> ks(wc, -1);
      int K = 0;
      for (int cc = 0; cc < wc; ++cc) {
        const int jin = BR.find(BR.q[jo] - R.lay.chq[cc]);
        if (jin < 0 || R.lay.so[cc * SR + jin] != jo) continue;
        ks[cc] = K;
        K += BR.dim[jin];
      }
      std::vector<int> rows_of(SL * dd, -1);
      int M = 0;
      const int64_t r0 = (int64_t)rmap.size();
      for (int i = 0; i < SL; ++i)
        for (int s = 0; s < d; ++s)
          for (int t = 0; t < d; ++t) {
            const int k = psi.sub(i, s, t);
            if (psi.sj[k] != jo) continue;
            rows_of[k] = M;
            for (int x = 0; x < BL.dim[i]; ++x) rmap.push_back(psi.roff[i] + (int64_t)x * psi.C[i] + psi.scol[k]);
            M += BL.dim[i];
          }
      if (M == 0) continue;
      const int N = BR.dim[jo];
      const int KB = (int)cdiv(std::max(K, 1), OZ_KBLK), MT = (int)cdiv(M, 128), NT = (int)cdiv(N, TC_TN);
      const int64_t pa = pa3n, pb = pb3n, ea = exa3, eb = exb3;
      const int64_t t3n = nt3s;
      nt3s += (int64_t)M * K;
      pa3n += (int64_t)MT * KB * TA;
      pb3n += (int64_t)NT * KB * TB;
      exa3 += M;
      exb3 += N;
      for (int cc = 0; cc < wc; ++cc) {
        if (ks[cc] < 0) continue;
        const int jin = BR.find(BR.q[jo] - R.lay.chq[cc]);
        seg(c->oz_step_p, c->oz_step_p_rows, p, BUF_OB3, pb, BUF_R, R.lay.off[cc * SR + jin], eb, 0, ks[cc], N,
            BR.dim[jin], BR.dim[jin], 0, KB, GB, 0);
      }
      for (int i = 0; i < SL; ++i)
        for (int s = 0; s < d; ++s)
          for (int t = 0; t < d; ++t) {
            const int k = psi.sub(i, s, t);
            if (rows_of[k] < 0) continue;
            for (int cc = 0; cc < wc; ++cc) {
              if (ks[cc] < 0) continue;
              const int jin = BR.find(BR.q[jo] - R.lay.chq[cc]);
              WTaskP w{};
              w.dst_off = pa;
              w.exp_off = ea;
              w.row0 = rows_of[k];
              w.k0 = ks[cc];
              w.KB = KB;
              w.G = GA;
              w.sb = p;
              w.rows = BL.dim[i];
              w.cols = BR.dim[jin];
              w.in_buf = BUF_OT1;
              w.dst_buf = BUF_OA3;
              w.t3_off = t3n;
              w.t3_ld = K;
              w.term0 = (int)c->wtpm_oz.size();
              for (int a = 0; a < wa; ++a) {
                const int si = BL.find(BL.q[i] - L.lay.chq[a]);
                if (si < 0 || L.lay.so[a * SL + si] != i || rs1[si][a] < 0) continue;
                for (int s2 = 0; s2 < d; ++s2)
                  for (int t2 = 0; t2 < d; ++t2) {
                    const double cf = S.W12[(((size_t)a * wc + cc) * dd + s * d + t) * dd + s2 * d + t2];
                    if (cf == 0.0) continue;
                    const int k2 = psi.sub(si, s2, t2);
                    if (psi.sj[k2] != jin) continue;
                    WTerm term{};
                    term.in_off = t1f[si] + (int64_t)rs1[si][a] * psi.C[si] + psi.scol[k2];
                    term.in_ld = psi.C[si];
                    term.coef = cf;
                    c->wtpm_oz.push_back(term);
                  }
              }
              w.nterm = (int)c->wtpm_oz.size() - w.term0;
              if (w.nterm == 0) continue;
              c->ozw.push_back(w);
              c->ozw_rows = std::max(c->ozw_rows, w.rows);
            }
          }
      TcTask t{};
      t.a_off = pa;
      t.b_off = pb;
      t.rmap_off = r0;
      t.a_exp = ea;
      t.b_exp = eb;
      t.sb = p;
      t.M = M;
      t.N = N;
      t.KB = K > 0 ? KB : 0;
      t.a_buf = BUF_OA3;
      t.b_buf = BUF_OB3;
      t.c_buf = BUF_OUT;
      t.rmap_buf = BUF_ORMAP;
      t.exp_buf = BUF_OEXP;
      t.mode = 1;
      add_task(c->oz3k, t3c, t, MT, NT);
    }
    na1[p] = pa1n;
    nb1[p] = pb1n;
    nt1[p] = t1n;
    na3[p] = pa3n;
    nb3[p] = pb3n;
    nt3[p] = nt3s;
  }
  (void)b3seg0;
  (void)target;
  auto flatten = [](const std::vector<std::vector<TcTile>> &lists, std::vector<TcTile> &out, std::vector<int> &lo) {
    out.clear();
    lo.assign(1, 0);
    for (const auto &l : lists) {
      out.insert(out.end(), l.begin(), l.end());
      lo.push_back((int)out.size());
    }
  };
  flatten(t1c, c->oz1t, c->oz1_lo);
  flatten(t3c, c->oz3t, c->oz3_lo);
  // exponent ranges: stage-3 B after stage 1, stage-3 A last
  c->oz_b3_lo = ex1;
  c->oz_b3_hi = ex1 + exb3;
  c->oz_a3_lo = c->oz_b3_hi;
  c->oz_a3_hi = c->oz_a3_lo + exa3;
  for (PackSeg &q : c->oz_step_p) q.exp_off += c->oz_b3_lo;
  for (WTaskP &w : c->ozw) w.exp_off += c->oz_a3_lo;
  for (TcTask &t : c->oz3k) {
    t.a_exp += c->oz_a3_lo;
    t.b_exp += c->oz_b3_lo;
  }
  NOMEM(c->ensure(c->oexp, 4 * (size_t)std::max<int64_t>(c->oz_a3_hi, 4)));
  for (int p = 0; p < P; ++p) {
    NOMEM(c->ensure(c->bOA1[p], 2 * std::max<int64_t>(na1[p], 8)) &&
          c->ensure(c->bOB1[p], 2 * std::max<int64_t>(nb1[p], 8)) &&
          c->ensure(c->bOT1[p], 8 * std::max<int64_t>(nt1[p], 1)) &&
          c->ensure(c->bOA3[p], 2 * std::max<int64_t>(na3[p], 8)) &&
          c->ensure(c->bOB3[p], 2 * std::max<int64_t>(nb3[p], 8)) &&
          c->ensure(c->bOT3[p], 8 * std::max<int64_t>(nt3[p], 1)) && c->upload(c->bORMAP[p], rmaps[p]));
    // zero digits in the padding (only real elements are rewritten later)
    CK(cudaMemsetAsync(c->bOA1[p].p, 0, 2 * na1[p], c->st));
    CK(cudaMemsetAsync(c->bOB1[p].p, 0, 2 * nb1[p], c->st));
    CK(cudaMemsetAsync(c->bOA3[p].p, 0, 2 * na3[p], c->st));
    CK(cudaMemsetAsync(c->bOB3[p].p, 0, 2 * nb3[p], c->st));
    c->hbufs[p * NBUF + BUF_OA1] = c->dp(c->bOA1[p]);
    c->hbufs[p * NBUF + BUF_OB1] = c->dp(c->bOB1[p]);
    c->hbufs[p * NBUF + BUF_OT1] = c->dp(c->bOT1[p]);
    c->hbufs[p * NBUF + BUF_OA3] = c->dp(c->bOA3[p]);
    c->hbufs[p * NBUF + BUF_OB3] = c->dp(c->bOB3[p]);
    c->hbufs[p * NBUF + BUF_ORMAP] = c->dp(c->bORMAP[p]);
    c->hbufs[p * NBUF + BUF_OEXP] = c->dp(c->oexp);
    c->hbufs[p * NBUF + BUF_OT3] = c->dp(c->bOT3[p]);
  }
  NOMEM(c->upload(c->dozsw, c->oz_step_w) && c->upload(c->dozsp, c->oz_step_p) && c->upload(c->dozp, c->oz_psi) &&
        c->upload(c->doz1k, c->oz1k) && c->upload(c->doz1t, c->oz1t) && c->upload(c->doz3k, c->oz3k) &&
        c->upload(c->doz3t, c->oz3t) && c->upload(c->dozw, c->ozw) && c->upload(c->dozwm, c->wtpm_oz));
  NOMEM(c->upload(c->dbufs, c->hbufs));
  // digits of L and R once for this iteration (R's rows span several channel
  // segments: exponents first)
  c->kbegin(IDMRG_K_HEFF_WSTAGE);
  CK(cudaMemsetAsync((int *)c->oexp.p + c->oz_b3_lo, 0x80, 4 * (c->oz_b3_hi - c->oz_b3_lo), c->st));
  double *const *bufs = (double *const *)c->dbufs.p;
  CK(launch_oz_exp((const PackSeg *)c->dozsp.p, (int)c->oz_step_p.size(), c->oz_step_p_rows, bufs, nullptr, c->st));
  CK(launch_oz_pack((const PackSeg *)c->dozsp.p, (int)c->oz_step_p.size(), c->oz_step_p_rows, bufs, nullptr, c->st));
  CK(launch_oz_pack((const PackSeg *)c->dozsw.p, (int)c->oz_step_w.size(), c->oz_step_w_rows, bufs, nullptr, c->st));
  c->kend(IDMRG_K_HEFF_WSTAGE);
  c->launches += 3;
  c->oz_ok = true;
  return IDMRG_OK;
}

// FP64-accurate H_eff psi from digit slices on the tensor cores
idmrg_status heff_launch_oz(idmrg_ctx *c, const int *active_dev, const int *act) {
  double *const *bufs = (double *const *)c->dbufs.p;
  double gf = 0, by = 0, wf = 0;
  for (int q = 0; q < c->P; ++q)
    if (!act || act[q]) { gf += c->plan[q].gemm_flops; wf += c->plan[q].w_flops; by += c->plan[q].heff_bytes; }
  c->kbegin(IDMRG_K_HEFF_WSTAGE);
  CK(launch_oz_pack((const PackSeg *)c->dozp.p, (int)c->oz_psi.size(), c->oz_psi_rows, bufs, active_dev, c->st));
  c->kend(IDMRG_K_HEFF_WSTAGE);
  // booked as the restart matvecs of a mixed context, as the H_eff GEMMs of FP64_TC
  const int kg = c->mixed ? IDMRG_K_HEFF_F64 : IDMRG_K_HEFF_GEMM;
  c->kbegin(kg);
  for (size_t ch = 0; ch + 1 < c->oz1_lo.size(); ++ch) {
    CK(launch_oz_gemm((const TcTile *)c->doz1t.p + c->oz1_lo[ch], c->oz1_lo[ch + 1] - c->oz1_lo[ch],
                      (const TcTask *)c->doz1k.p, bufs, active_dev, (int *)c->derr.p, c->st));
    c->launches += 1;
  }
  c->kend(kg);
  c->kbegin(IDMRG_K_HEFF_WSTAGE);
  CK(cudaMemsetAsync((int *)c->oexp.p + c->oz_a3_lo, 0x80, 4 * (c->oz_a3_hi - c->oz_a3_lo), c->st));
  CK(launch_wstage_oz((const WTaskP *)c->dozw.p, (int)c->ozw.size(), c->ozw_rows, (const WTerm *)c->dozwm.p, bufs,
                      active_dev, 0, c->st));
  CK(launch_wstage_oz((const WTaskP *)c->dozw.p, (int)c->ozw.size(), c->ozw_rows, (const WTerm *)c->dozwm.p, bufs,
                      active_dev, 1, c->st));
  c->kend(IDMRG_K_HEFF_WSTAGE, wf, 0.0);
  c->kbegin(kg);
  for (size_t ch = 0; ch + 1 < c->oz3_lo.size(); ++ch) {
    CK(launch_oz_gemm((const TcTile *)c->doz3t.p + c->oz3_lo[ch], c->oz3_lo[ch + 1] - c->oz3_lo[ch],
                      (const TcTask *)c->doz3k.p, bufs, active_dev, (int *)c->derr.p, c->st));
    c->launches += 1;
  }
  c->kend(kg, gf, by);
  c->launches += 3;
  c->fp64_matvecs += 1;
  return IDMRG_OK;
}

// heff on every superblock whose active flag is set (device array); the host
// copy `act` (may be null = all) only feeds the flop/byte accounting
idmrg_status heff_launch_fp64(idmrg_ctx *c, const int *active_dev, const int *act);
idmrg_status heff_launch_mixed(idmrg_ctx *c, const int *active_dev, const int *act) {
  double *const *bufs = (double *const *)c->dbufs.p;
  double gf = 0, by = 0, wf = 0, pb = 0, wb = 0;
  const double hl = c->bf16 ? 4.0 : 8.0;  // bytes of one hi/lo pair
  for (int q = 0; q < c->P; ++q)
    if (!act || act[q]) {
      const SBPlan &S = c->plan[q];
      gf += S.gemm_flops;
      wf += S.w_flops;
      by += S.heff_bytes;
      pb += (8.0 + hl) * S.wpack_elems;
      wb += 4.0 * S.wt1_elems + hl * S.wt3_elems;
    }
  const int k1 = std::max(c->tt1.choice, 0), k3 = std::max(c->tt3.choice, 0);
  c->kbegin(IDMRG_K_HEFF_WSTAGE);
  CK(launch_pack((const PackSeg *)c->dpkp[k1].p, (int)c->pk_psi[k1].size(), c->pk_psi_rows, bufs, active_dev,
                 c->bf16, c->st));
  c->kend(IDMRG_K_HEFF_WSTAGE, 0.0, pb);
  c->kbegin(IDMRG_K_HEFF_GEMM);
  CK(launch_tc_gemm((const TcTile *)c->dtc1t[k1].p, (int)c->tc1t[k1].size(), (const TcTask *)c->dtc1k[k1].p, bufs,
                    active_dev, (int *)c->derr.p, c->bf16, MIX_TNS[k1], c->st));
  c->kend(IDMRG_K_HEFF_GEMM);
  c->kbegin(IDMRG_K_HEFF_WSTAGE);
  CK(launch_wstage_tc((const int4 *)c->dwunits.p, (int)c->wunits.size(), (const WTaskP *)c->dwtp.p,
                      (const WTerm *)c->dwtpm.p, bufs, active_dev, c->bf16, c->st));
  c->kend(IDMRG_K_HEFF_WSTAGE, wf, wb);
  c->kbegin(IDMRG_K_HEFF_GEMM);
  CK(launch_tc_gemm((const TcTile *)c->dtc3t[k3].p, (int)c->tc3t[k3].size(), (const TcTask *)c->dtc3k[k3].p, bufs,
                    active_dev, (int *)c->derr.p, c->bf16, MIX_TNS[k3], c->st));
  c->kend(IDMRG_K_HEFF_GEMM, gf, by);
  c->launches += 4;
  c->mixed_matvecs += 1;
  return IDMRG_OK;
}
idmrg_status heff_launch(idmrg_ctx *c, const int *active_dev, const int *act, bool fp64) {
  if (c->mixed && !fp64) return heff_launch_mixed(c, active_dev, act);
  return heff_launch_fp64(c, active_dev, act);
}
idmrg_status heff_launch_oz(idmrg_ctx *c, const int *active_dev, const int *act);
idmrg_status heff_launch_fp64(idmrg_ctx *c, const int *active_dev, const int *act) {
  if (c->oz_active()) return heff_launch_oz(c, active_dev, act);
  c->fp64_matvecs += 1;
  double *const *bufs = (double *const *)c->dbufs.p;
  double gf = 0, wf = 0, by = 0;
  for (int q = 0; q < c->P; ++q)
    if (!act || act[q]) { gf += c->plan[q].gemm_flops; wf += c->plan[q].w_flops; by += c->plan[q].heff_bytes; }
  const int kg = c->mixed ? IDMRG_K_HEFF_F64 : IDMRG_K_HEFF_GEMM;  // (FP64 GEMMs)
  c->kbegin(kg);
  {
    idmrg_status sg_ = gemm_run(c, c->tn_g1, c->dg1k, c->dg1s, active_dev);
    if (sg_ != IDMRG_OK) return sg_;
  }
  c->kend(kg, 0.0, 0.0);
  c->kbegin(IDMRG_K_HEFF_WSTAGE);
  CK(launch_wstage_f64((const WTask *)c->dwt.p, (int)c->wl.tasks.size(), c->wl.max_rows, (const WTerm *)c->dwm.p,
                       bufs, active_dev, c->st));
  c->kend(IDMRG_K_HEFF_WSTAGE, wf, 0.0);
  c->kbegin(kg);
  {
    idmrg_status sg_ = gemm_run(c, c->tn_g3, c->dg3k, c->dg3s, active_dev);
    if (sg_ != IDMRG_OK) return sg_;
  }
  c->kend(kg, gf, by);
  c->launches += 3;
  return IDMRG_OK;
}

idmrg_status check_dev_err(idmrg_ctx *c) {
  int e = 0;
  CK(c->d2h_copy(&e, c->derr.p, sizeof(int)));
  CK(cudaStreamSynchronize(c->st));
  if (e & IDMRG_DEV_ERR_TIMEOUT) return c->fail(IDMRG_ETIMEOUT, "device wait exceeded its budget");
  if (e & IDMRG_DEV_ERR_NUMERIC) return c->fail(IDMRG_ENUMERIC, "non-finite Lanczos coefficient (n=%d)", c->n);
  if (e & IDMRG_DEV_ERR_ZERONORM)
    return c->fail(IDMRG_ENUMERIC, "start vector with zero norm (n=%d, superblock mask 0x%x)", c->n, e >> 4);
  if (e & IDMRG_DEV_ERR_JACOBI)
    return c->fail(IDMRG_ENUMERIC, "SVD: sweeps exhausted, or a rotation beyond FP32-pair range (n=%d)", c->n);
  return IDMRG_OK;
}

bool want(const idmrg_ctx *c, int p, int q) { return p < 0 ? c->owns(q) : p == q; }

idmrg_status check_p(idmrg_ctx *c, int p) {
  if (p < -1 || p >= c->P) return c->fail(IDMRG_EINVAL, "superblock index %d out of range", p);
  if (p >= 0 && !c->owns(p)) return c->fail(IDMRG_EINVAL, "superblock %d is outside this context's range", p);
  if (c->plan_pending) return c->fail(IDMRG_ESTATE, "the boundary pair of this range has not been imported");
  return IDMRG_OK;
}

// ------------------------------------------------------------------------
// Step 3': start vectors
// ------------------------------------------------------------------------
idmrg_status predict(idmrg_ctx *c, int p) {
  const int P = c->P, d = c->d;
  const bool use_pred = c->o.predict && c->n >= 3;
  for (int q = 0; q < P; ++q)
    if (want(c, p, q) && c->stage[q] != ST_READY && c->stage[q] != ST_STARTED)
      return c->fail(IDMRG_ESTATE, "predict_wavefunction: superblock %d already past its start", q);
  double *const *bufs = (double *const *)c->dbufs.p;
  if (!use_pred) {
    // SplitMix64 numbers on every charge-allowed element; one launch for all
    // requested superblocks (blocks of other superblocks are filtered on host)
    std::vector<RandBlock> rb;
    int mr = 0;
    for (const RandBlock &b : c->rblocks)
      if (want(c, p, b.sb)) { rb.push_back(b); mr = std::max(mr, b.rows); }
    c->kbegin(IDMRG_K_PREDICT);
    if (p >= 0) {
      NOMEM(c->upload(c->dst, rb));
      CK(launch_rand_blocks((const RandBlock *)c->dst.p, (int)rb.size(), mr, bufs, BUF_PSI, c->st));
    } else {
      CK(launch_rand_blocks((const RandBlock *)c->drb.p, (int)c->rblocks.size(), c->rmax_rows, bufs, BUF_PSI, c->st));
    }
    c->kend(IDMRG_K_PREDICT);
    c->launches += 1;
  } else {
    // Eq. wfprediction: psi~ = sum_B [lam_i v_i]^T [u_{i+1} lam_{i+1} / lam''_{i+1}]
    c->stasks.clear();
    c->stable.clear();
    c->smax_rows = 0;
    c->gp.clear();
    for (int q = 0; q < P; ++q) {
      if (!want(c, p, q)) continue;
      const int q1 = c->nxt(q);
      const TruncRec &A = c->prev[q], &B = c->prev[q1], &B2 = c->prev2[q1];
      if (!A.valid || !B.valid || !B2.valid) return c->fail(IDMRG_ESTATE, "prediction needs two earlier iterations");
      NOMEM(c->ensure(c->bVT[q], 8 * std::max<int64_t>(A.vsize, 1)));
      NOMEM(c->ensure(c->bUT[q], 8 * std::max<int64_t>(B.usize, 1)));
      c->hbufs[q * NBUF + BUF_VPREV] = (double *)A.V.p;
      c->hbufs[q * NBUF + BUF_UPREV] = (double *)B.U.p;
      c->hbufs[q * NBUF + BUF_VT] = c->dp(c->bVT[q]);
      c->hbufs[q * NBUF + BUF_UT] = c->dp(c->bUT[q]);
      const int t_lamA = (int)c->stable.size();
      c->stable.insert(c->stable.end(), A.lam.begin(), A.lam.end());
      const int t_lamB = (int)c->stable.size();
      c->stable.insert(c->stable.end(), B.lam.begin(), B.lam.end());
      const int t_lamB2 = (int)c->stable.size();
      c->stable.insert(c->stable.end(), B2.lam.begin(), B2.lam.end());
      const int t_max = (int)c->stable.size();
      c->stable.push_back(B2.lam_all.empty() ? 0.0 : B2.lam_all[0]);
      // v~ = v_i lam_i (columns)
      for (const SecInfo &s : A.sec) {
        ScaleTask t{};
        t.off = s.v_off;
        t.rows = s.c;
        t.cols = s.k;
        t.ld = s.k;
        t.sb = q;
        t.src_buf = BUF_VPREV;
        t.dst_buf = BUF_VT;
        t.rs_off = -1;
        t.cs_off = t_lamA + s.lam_off;
        t.rs_inv = 0;
        t.max_off = t_max;
        c->stasks.push_back(t);
        c->smax_rows = std::max(c->smax_rows, t.rows);
      }
      // u~ = u_{i+1} lam_{i+1} (columns) / lam''_{i+1} (rows, zero rule)
      for (const SecInfo &s : B.sec)
        for (const auto &g : s.rg) {
          ScaleTask t{};
          t.off = s.u_off + (int64_t)g[2] * s.k;
          t.rows = B.leftB.dim[g[0]];
          t.cols = s.k;
          t.ld = s.k;
          t.sb = q;
          t.src_buf = BUF_UPREV;
          t.dst_buf = BUF_UT;
          t.rs_off = t_lamB2 + B.leftB.off[g[0]];
          t.cs_off = t_lamB + s.lam_off;
          t.rs_inv = 1;
          t.max_off = t_max;
          c->stasks.push_back(t);
          c->smax_rows = std::max(c->smax_rows, t.rows);
        }
      // products, one task per psi~ sub-block (left sector a, s, t)
      const PsiLayout &psi = c->plan[q].psi;
      for (int a = 0; a < (int)A.sec.size(); ++a)
        for (int s = 0; s < d; ++s)
          for (int t = 0; t < d; ++t) {
            const int k = psi.sub(a, s, t);
            const int g = psi.sj[k];
            if (g < 0) continue;
            const SecInfo &sa = A.sec[a], &sg = B.sec[g];
            c->gp.task(q, BUF_PSI, psi.roff[a] + psi.scol[k], sa.k, sg.k, psi.C[a]);
            int jB = -1, startV = 0;
            for (const auto &cg : sa.cg)
              if (cg[0] == s) { jB = cg[1]; startV = cg[2]; }
            if (jB < 0) continue;
            for (const auto &rg : sg.rg)
              if (rg[1] == t && rg[0] == jB)
                c->gp.seg(BUF_VT, sa.v_off + (int64_t)startV * sa.k, sa.k, BUF_UT, sg.u_off + (int64_t)rg[2] * sg.k,
                          sg.k, A.rightB.dim[jB], 1);
          }
    }

    NOMEM(sync_bufs(c) == IDMRG_OK);
    NOMEM(c->upload(c->dst, c->stasks) && c->upload(c->dstab, c->stable));
    {
      idmrg_status sg = gemm_upload(c, c->gp, c->dgpk, c->dgps, c->tn_gp);
      if (sg != IDMRG_OK) return sg;
    }
    c->kbegin(IDMRG_K_PREDICT);
    CK(launch_scale_tasks((const ScaleTask *)c->dst.p, (int)c->stasks.size(), c->smax_rows,
                          (const double *)c->dstab.p, c->o.lambda_zero_rel, bufs, c->st));
    {
    idmrg_status sg_ = gemm_run(c, c->tn_gp, c->dgpk, c->dgps, nullptr);
    if (sg_ != IDMRG_OK) return sg_;
  }
    c->kend(IDMRG_K_PREDICT, c->gp.flops, 0.0);
    c->launches += 2;
  }
  for (int q = 0; q < P; ++q)
    if (want(c, p, q)) c->stage[q] = ST_STARTED;
  return IDMRG_OK;
}

// ------------------------------------------------------------------------
// Step 3: batched Lanczos
// ------------------------------------------------------------------------
// One Lanczos iteration of every active superblock: matvec (FP64 or on the
// tensor cores), three-term step, full re-orthogonalisation pass,
// tridiagonal solve and convergence test, next Krylov vector.  `act` and
// `vb` only feed the per-class timers (act may be null).
idmrg_status lanczos_iteration(idmrg_ctx *c, const LanczosDev &L, bool fp64, const int *act, double vb) {
  idmrg_status s = heff_launch(c, L.active, act, fp64);
  if (s != IDMRG_OK) return s;
  c->kbegin(IDMRG_K_LANCZOS_VEC);
  CK(lanczos_project(L, 0, c->st));
  CK(lanczos_reduce(L, 0, c->st));
  CK(lanczos_sub0_proj1(L, c->st));
  CK(lanczos_reduce(L, 1, c->st));
  CK(lanczos_subtract(L, 1, c->st));
  c->kend(IDMRG_K_LANCZOS_VEC, 0.0, vb);
  c->kbegin(IDMRG_K_LANCZOS_TRI);
  CK(lanczos_finalize(L, c->st));
  c->kend(IDMRG_K_LANCZOS_TRI);
  c->kbegin(IDMRG_K_LANCZOS_VEC);
  CK(lanczos_next(L, c->st));
  c->kend(IDMRG_K_LANCZOS_VEC);
  c->launches += 7;
  return IDMRG_OK;
}

idmrg_status lanczos(idmrg_ctx *c, int p) {
  const int P = c->P;
  for (int q = 0; q < P; ++q)
    if (want(c, p, q) && c->stage[q] != ST_STARTED)
      return c->fail(IDMRG_ESTATE, "lanczos_solve: superblock %d has no start vector", q);
  // a mixed-precision run stops after 80 iterations and restarts: its Krylov
  // basis never holds more than 81 vectors
  const int kmax = c->mixed ? std::min(c->o.lanczos_maxit, 81) : c->o.lanczos_maxit;
  std::vector<int64_t> N(P);
  int64_t nmax = 1;
  for (int q = 0; q < P; ++q) {
    N[q] = c->plan[q].psi.N;
    nmax = std::max(nmax, N[q]);
  }
  const int CHK = 1024;
  const int nchunk = (int)((nmax + CHK - 1) / CHK);
  std::vector<double *> Vp(P), wp(P), psip(P), v0p(P), startp(P, nullptr);
  for (int q = 0; q < P; ++q) {
    NOMEM(c->ensure(c->bV[q], 8 * std::max<int64_t>((int64_t)kmax * N[q], 1)));
    Vp[q] = c->dp(c->bV[q]);
    wp[q] = c->dp(c->bW[q]);
    psip[q] = c->dp(c->bPsi[q]);
    v0p[q] = Vp[q];
    if (c->mixed) {
      NOMEM(c->ensure(c->bStart[q], 8 * std::max<int64_t>(N[q], 1)));
      startp[q] = c->dp(c->bStart[q]);
    }
  }
  NOMEM(c->upload(c->lN, N) && c->upload(c->lV, Vp) && c->upload(c->lw, wp) && c->upload(c->lpsi, psip) &&
        c->upload(c->lv0, v0p));
  NOMEM(c->ensure(c->lalpha, 8 * (size_t)P * kmax) && c->ensure(c->lbeta, 8 * (size_t)P * kmax) &&
        c->ensure(c->libeta, 8 * (size_t)P * kmax) &&
        c->ensure(c->lh, 8 * 2 * (size_t)P * kmax) && c->ensure(c->ly, 8 * (size_t)P * kmax) &&
        c->ensure(c->lpart, 8 * 3 * (size_t)P * kmax * nchunk) && c->ensure(c->ltheta, 8 * P) &&
        c->ensure(c->lresid, 8 * P) && c->ensure(c->ldot, 8 * P) && c->ensure(c->lk, 4 * P) &&
        c->ensure(c->lactive, 4 * P) && c->ensure(c->lconv, 4 * P));
  std::vector<int> member(P);
  for (int q = 0; q < P; ++q) member[q] = want(c, p, q) ? 1 : 0;
  NOMEM(c->upload(c->lmember, member));
  if (!c->pin_act) {
    CK(cudaHostAlloc((void **)&c->pin_act, 2 * 4 * (size_t)P, cudaHostAllocDefault));
    for (auto &e : c->ev_act) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  LanczosDev L{};
  L.S = P;
  L.kmax = kmax;
  L.N = (const int64_t *)c->lN.p;
  L.V = (double *const *)c->lV.p;
  L.w = (double *const *)c->lw.p;
  L.alpha = c->dp(c->lalpha);
  L.beta = c->dp(c->lbeta);
  L.ibeta = c->dp(c->libeta);
  L.h = c->dp(c->lh);
  L.part = c->dp(c->lpart);
  L.k = (int *)c->lk.p;
  L.member = (int *)c->lmember.p;
  L.active = (int *)c->lactive.p;
  L.conv = (int *)c->lconv.p;
  L.theta = c->dp(c->ltheta);
  L.y = c->dp(c->ly);
  L.resid = c->dp(c->lresid);
  L.err = (int *)c->derr.p;
  L.nchunk_max = nchunk;
  L.tol = c->o.lanczos_tol;
  NOMEM(c->ensure(c->dtarget, 8 * P));
  L.target = c->dp(c->dtarget);
  L.bufs = (double **)c->dbufs.p;
  // FP64: one Lanczos run.  Mixed precision: restarts.  Each restart begins
  // with an FP64 matvec on its start vector, so k = 0 checks the true residual
  // against tol (and its alpha_0 is the FP64 Rayleigh quotient); the following
  // matvecs run on the tensor cores until the residual estimate falls by the
  // inner factor; the Ritz vector starts the next restart.
  // (BF16 splits carry ~16 bits per product against ~21 for TF32: each
  // restart gains less, so more of them are allowed)
  L.inner_factor = c->mixed ? c->inner_factor : 0.0;
  const int max_restarts = c->mixed ? (c->bf16 ? 12 : 8) : 1;
  const int inner_cap = c->mixed ? std::min(kmax, c->inner_cap) : kmax;
  for (int q = 0; q < P; ++q) c->hbufs[q * NBUF + BUF_PSI] = psip[q];
  NOMEM(sync_bufs(c) == IDMRG_OK);
  std::vector<double> nrm2(P, 0.0), theta(P, 0.0), dots(P, 0.0);
  std::vector<int> act(P), kk(P), conv(P), total(P, 0), final_(P, 0);
  bool allconv = true;
  // graphs of one iteration ([1]: FP64 matvec, [0]: reduced precision),
  // captured on first use in this solve
  cudaGraphExec_t iter_graph[2] = {nullptr, nullptr};
  uint64_t graph_launches[2] = {0, 0};
  bool graph_ok = true;
  struct GraphGuard {
    cudaGraphExec_t *g;
    ~GraphGuard() {
      for (int k = 0; k < 2; ++k)
        if (g[k]) cudaGraphExecDestroy(g[k]);
    }
  } graph_guard{iter_graph};
  for (int r = 0; r < max_restarts; ++r) {
    bool anym = false;
    for (int q = 0; q < P; ++q) anym |= member[q] != 0;
    if (!anym) break;
    NOMEM(c->upload(c->lmember, member));
    CK(lanczos_init(L, (const double *const *)c->lpsi.p, c->st));
    CK(lanczos_set_ptrs(L, (double **)c->dbufs.p, c->st));  // later ones: next_kernel
    c->launches += 4;
    if (r == 0) CK(c->d2h_copy(nrm2.data(), c->lresid.p, 8 * P));  // ||psi~|| for the report
    for (int it = 0; it < inner_cap; ++it) {
      // the same iteration as a graph once the kernels of its matvec are
      // fixed (reduced precision, or FP64 with tuned GEMM tiles)
      const bool fp64 = it == 0 || !c->mixed;
      const bool as_graph = graph_ok && !c->prof &&
                            (fp64 ? (c->oz_active() || (!c->mixed && c->tn_g1.choice >= 0 && c->tn_g3.choice >= 0))
                                  : true);
      if (as_graph && !iter_graph[fp64]) {
        const uint64_t l0 = c->launches, mm0 = c->mixed_matvecs, fm0 = c->fp64_matvecs;
        cudaGraph_t g = nullptr;
        bool okc = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeRelaxed) == cudaSuccess;
        idmrg_status sc = okc ? lanczos_iteration(c, L, fp64, nullptr, 0.0) : IDMRG_ECUDA;
        okc = (cudaStreamEndCapture(c->st, &g) == cudaSuccess) && okc && sc == IDMRG_OK;
        okc = okc && cudaGraphInstantiate(&iter_graph[fp64], g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        graph_launches[fp64] = c->launches - l0;
        c->launches = l0;
        c->mixed_matvecs = mm0;
        c->fp64_matvecs = fm0;
        if (!okc) {  // capture refused: stay with direct launches
          cudaGetLastError();
          iter_graph[fp64] = nullptr;
          graph_ok = false;
        }
      }
      if (as_graph && iter_graph[fp64]) {
        CK(cudaGraphLaunch(iter_graph[fp64], c->st));
        c->launches += graph_launches[fp64];
        (fp64 ? c->fp64_matvecs : c->mixed_matvecs) += 1;
      } else {
        double vb = 0.0;
        for (int q = 0; q < P; ++q)
          // three-term step 6 N, full pass (k + 2) N + (k + 3) N, k = it
          if (it == 0 ? member[q] : act[q]) vb += 8.0 * (double)N[q] * (2.0 * it + 11.0);
        idmrg_status s = lanczos_iteration(c, L, fp64, it == 0 ? member.data() : act.data(), vb);
        if (s != IDMRG_OK) return s;
      }
      // the active flags after this iteration go to pinned memory; the host
      // reads those of the previous iteration, so the next iteration is
      // already queued while it waits (an iteration launched after the last
      // superblock stopped finds every superblock inactive and does nothing)
      int *flags = c->pin_act + (it & 1) * P;
      CK(cudaMemcpyAsync(flags, c->lactive.p, 4 * P, cudaMemcpyDeviceToHost, c->st));
      c->d2h += 4 * P;
      CK(cudaEventRecord(c->ev_act[it & 1], c->st));
      if (it == 0) continue;
      CK(cudaEventSynchronize(c->ev_act[(it - 1) & 1]));
      const int *prevf = c->pin_act + ((it - 1) & 1) * P;
      bool any = false;
      for (int q = 0; q < P; ++q) {
        act[q] = prevf[q];
        any |= (act[q] != 0);
      }
      if (!any) break;
    }
    CK(lanczos_ritz(L, (double *const *)c->lpsi.p, c->st));
    c->launches += 4;
    if (r == 0 && !c->mixed) {  // one run: V[0] is still the normalised start vector
      CK(lanczos_dot(L, (const double *const *)c->lv0.p, (const double *const *)c->lpsi.p, c->dp(c->ldot), c->st));
      c->launches += 2;
      CK(c->d2h_copy(dots.data(), c->ldot.p, 8 * P));
    }
    if (r == 0 && c->mixed)  // restarts overwrite V[0]: keep the normalised start for Eq. fid1
      for (int q = 0; q < P; ++q)
        if (want(c, p, q) && N[q] > 0)
          CK(cudaMemcpyAsync(startp[q], Vp[q], 8 * (size_t)N[q], cudaMemcpyDeviceToDevice, c->st));
    std::vector<double> th(P);
    CK(c->d2h_copy(th.data(), c->ltheta.p, 8 * P));
    CK(c->d2h_copy(kk.data(), c->lk.p, 4 * P));
    CK(c->d2h_copy(conv.data(), c->lconv.p, 4 * P));
    idmrg_status s = check_dev_err(c);
    if (s != IDMRG_OK) return s;
    for (int q = 0; q < P; ++q) {
      if (!member[q]) continue;
      total[q] += kk[q] + 1;
      theta[q] = th[q];
      // FP64 mode: done.  Mixed: done only when the FP64 check at k = 0 passed
      const bool done = !c->mixed || (conv[q] && kk[q] == 0);
      if (done) {
        final_[q] = conv[q];
        member[q] = 0;
      }
    }
  }
  if (c->mixed) {  // Eq. fid1 against the final Ritz vector
    std::vector<int> all(P);
    for (int q = 0; q < P; ++q) all[q] = want(c, p, q) ? 1 : 0;
    NOMEM(c->upload(c->lmember, all) && c->upload(c->lv0, startp));
    CK(lanczos_dot(L, (const double *const *)c->lv0.p, (const double *const *)c->lpsi.p, c->dp(c->ldot), c->st));
    c->launches += 2;
    CK(c->d2h_copy(dots.data(), c->ldot.p, 8 * P));
    CK(cudaStreamSynchronize(c->st));
  }
  for (int q = 0; q < P; ++q) {
    if (!want(c, p, q)) continue;
    c->energy[q] = theta[q];
    c->iters[q] = total[q];
    c->conv[q] = final_[q];
    c->startnorm[q] = sqrt(nrm2[q]);
    c->fidelity[q] = (c->o.predict && c->n >= 3) ? 1.0 - fabs(dots[q]) : NAN;
    c->stage[q] = ST_SOLVED;
    allconv &= final_[q] != 0;
  }
  // centre-bond energies <psi|h|psi>
  std::vector<DotTerm> dt;
  std::vector<int> dsb;
  for (size_t k = 0; k < c->dterms.size(); ++k)
    if (want(c, p, c->dterm_sb[k])) { dt.push_back(c->dterms[k]); dsb.push_back(c->dterm_sb[k]); }
  if (!dt.empty()) {
    NOMEM(c->upload(c->dst, dt) && c->ensure(c->ddp, 8 * dt.size()));
    CK(launch_dot_terms((const DotTerm *)c->dst.p, (int)dt.size(), (double *const *)c->dbufs.p, c->dp(c->ddp), c->st));
    c->launches += 1;
    std::vector<double> part(dt.size());
    CK(c->d2h_copy(part.data(), c->ddp.p, 8 * dt.size()));
    CK(cudaStreamSynchronize(c->st));
    for (int q = 0; q < P; ++q)
      if (want(c, p, q)) c->bond[q] = 0.0;
    for (size_t k = 0; k < dt.size(); ++k) c->bond[dsb[k]] += part[k];
  } else {
    for (int q = 0; q < P; ++q)
      if (want(c, p, q)) c->bond[q] = 0.0;
  }
  return allconv ? IDMRG_OK : c->fail(IDMRG_ENOCONV, "Lanczos reached lanczos_maxit before converging");
}

// ------------------------------------------------------------------------
// Step 4: sector SVD, cut, compaction
// ------------------------------------------------------------------------
// Jacobi launch groups of jobs listed largest first (ord[0..m)): a job's
// time is about (columns) x (latency of a sub-round) whatever the cluster
// size, so only the largest sectors need 16 CTAs; smaller ones take 8, 4 or
// 1 and finish within the same time on fewer SMs.  g[k] ends group k (0:
// global-memory kernel for sectors beyond the block kernel's shared memory,
// 1..4: block kernel on 16, 8, 4, 1 CTAs); gcols[k] is the largest column
// count of block group k+1.
void jacobi_groups(const idmrg_ctx *c, const int *ord, int m, int g[4], int gcols[4]) {
  for (int k = 0; k < 4; ++k) g[k] = gcols[k] = 0;
  if (c->svd_global) {  // every job on the global-memory kernels
    for (int k = 0; k < 4; ++k) g[k] = m;
    return;
  }
  for (int j = 0; j < m; ++j) {
    const int ca = c->jobs[ord[j]].cols_a;
    if (ca >= 128 && svd_block_smem(ca, 16) > SVD_BLOCK_SMEM_MAX) g[0] = j + 1;
    if (ca >= 128) g[1] = j + 1;
    if (ca >= 64) g[2] = j + 1;
    if (ca >= 24) g[3] = j + 1;
  }
  if (g[1] > g[0]) gcols[0] = c->jobs[ord[g[0]]].cols_a;
  if (g[2] > g[1]) gcols[1] = c->jobs[ord[g[1]]].cols_a;
  if (g[3] > g[2]) gcols[2] = c->jobs[ord[g[2]]].cols_a;
  if (m > g[3]) gcols[3] = c->jobs[ord[g[3]]].cols_a;
}

// SVD jobs of every superblock of `p`: one job per charge sector Q of the
// left half, (x s) rows of charge Q against (t y) columns of charge
// target - Q.  Uploads the jobs, the global and the per-superblock orders
// (largest first) and sizes every work array; nothing depends on psi.
idmrg_status trunc_plan(idmrg_ctx *c, int p) {
  const int P = c->P, d = c->d, target = c->o.target_charge;
  c->jobs.clear();
  c->tsecs.assign(P, {});
  c->tjob0.assign(P, 0);
  c->tnjob.assign(P, 0);
  c->tentries.assign(P, 1);
  c->tmaxel.assign(P, 0);
  c->tg.assign(P, {0, 0, 0, 0});
  c->tgcols.assign(P, {0, 0, 0, 0});
  int64_t work = 0;
  int sv = 0, iw = 0;
  c->tentries_max = 1;
  c->tmaxel_all = 0;
  for (int q = 0; q < P; ++q) {
    c->tjob0[q] = (int)c->jobs.size();
    if (!want(c, p, q)) continue;
    const Env &L = c->envL[q];
    const Env &R = c->envR[c->nxt(q)];
    const Basis &BL = L.lay.b, &BR = R.lay.b;
    const PsiLayout &psi = c->plan[q].psi;
    std::vector<int> Qs;
    for (int i = 0; i < BL.S(); ++i)
      for (int s = 0; s < d; ++s) Qs.push_back(BL.q[i] + c->qp[s]);
    std::sort(Qs.begin(), Qs.end());
    Qs.erase(std::unique(Qs.begin(), Qs.end()), Qs.end());
    int entries = 0;
    for (int Q : Qs) {
      SecInfo si;
      si.Q = Q;
      for (int i = 0; i < BL.S(); ++i)
        for (int s = 0; s < d; ++s)
          if (BL.q[i] + c->qp[s] == Q) { si.rg.push_back({i, s, si.r}); si.r += BL.dim[i]; }
      for (int t = 0; t < d; ++t)
        for (int j = 0; j < BR.S(); ++j)
          if (c->qp[t] + BR.q[j] == target - Q) { si.cg.push_back({t, j, si.c}); si.c += BR.dim[j]; }
      if (si.r == 0 || si.c == 0) continue;
      if (si.rg.size() > 4 || si.cg.size() > 4) return c->fail(IDMRG_EINVAL, "local dimension above 4 is not supported");
      SvdJob J{};
      J.sb = q;
      J.Q = Q;
      J.r = si.r;
      J.c = si.c;
      J.transposed = si.r < si.c;
      J.rows_a = std::max(si.r, si.c);
      J.cols_a = std::min(si.r, si.c);
      J.ngr = (int)si.rg.size();
      J.ngc = (int)si.cg.size();
      for (int g = 0; g < J.ngr; ++g) {
        J.gr_start[g] = si.rg[g][2];
        J.gr_len[g] = BL.dim[si.rg[g][0]];
        J.gr_stride[g] = psi.C[si.rg[g][0]];
      }
      for (int h = 0; h < J.ngc; ++h) {
        J.gc_start[h] = si.cg[h][2];
        J.gc_len[h] = BR.dim[si.cg[h][1]];
      }
      for (int g = 0; g < J.ngr; ++g)
        for (int h = 0; h < J.ngc; ++h) {
          const int i = si.rg[g][0], s = si.rg[g][1], t = si.cg[h][0], j = si.cg[h][1];
          const int k = psi.sub(i, s, t);
          if (psi.sj[k] != j) return c->fail(IDMRG_EINVAL, "internal: sector bookkeeping mismatch");
          J.base[g * 4 + h] = psi.roff[i] + psi.scol[k];
        }
      if (J.cols_a > 4096) return c->fail(IDMRG_EINVAL, "charge sector with more than 4096 states per side");
      J.a_off = work;
      work += (int64_t)J.rows_a * J.cols_a;
      J.x_off = work;
      work += (int64_t)J.rows_a * J.cols_a;
      J.j_off = work;
      work += (int64_t)J.cols_a * J.cols_a;
      J.b_off = work;
      work += (int64_t)J.cols_a * J.cols_a;
      J.tau_off = work;
      work += J.cols_a;
      J.w_off = work;
      work += (int64_t)J.cols_a * J.cols_a;
      J.perm_off = iw;
      iw += J.cols_a + 3;  // permutation, rank, FP64 and FP32 Jacobi sweeps
      J.sv_off = sv;
      sv += J.cols_a;
      entries += J.cols_a;
      c->tmaxel[q] = std::max<int64_t>(c->tmaxel[q], (int64_t)J.r * J.c);
      si.job = (int)c->jobs.size();
      c->jobs.push_back(J);
      c->tsecs[q].push_back(si);
    }
    c->tnjob[q] = (int)c->jobs.size() - c->tjob0[q];
    c->tentries[q] = std::max(1, entries);
    c->tentries_max = std::max(c->tentries_max, entries);
    c->tmaxel_all = std::max(c->tmaxel_all, c->tmaxel[q]);
  }
  const int nj = (int)c->jobs.size();
  c->tiw = iw;
  c->tsv = sv;
  // largest sector matrices first: they set the length of the SVD phase
  auto bigger = [&](int a, int b) {
    const SvdJob &x = c->jobs[a], &y = c->jobs[b];
    if (x.cols_a != y.cols_a) return x.cols_a > y.cols_a;
    return x.rows_a > y.rows_a;
  };
  c->torder.resize(nj);
  for (int j = 0; j < nj; ++j) c->torder[j] = j;
  std::stable_sort(c->torder.begin(), c->torder.end(), bigger);
  c->torderq.clear();
  c->to0.assign(P, 0);
  for (int q = 0; q < P; ++q) {
    c->to0[q] = (int)c->torderq.size();
    for (int j = 0; j < c->tnjob[q]; ++j) c->torderq.push_back(c->tjob0[q] + j);
    std::stable_sort(c->torderq.begin() + c->to0[q], c->torderq.end(), bigger);
  }
  for (int q = 0; q < P; ++q)
    jacobi_groups(c, c->torderq.data() + c->to0[q], c->tnjob[q], c->tg[q].data(), c->tgcols[q].data());
  // Newton-Schulz steps and X = B V of the FP32-preconditioned Jacobi.  V is
  // column-major cols_a x cols_a, i.e. the row-major matrix V^T:
  // G = V^T V (x_off), W^T = G V^T (w_off), X^T = V^T B^T (w_off)
  c->svdG.clear();
  c->svdW.clear();
  c->svdX.clear();
  c->tmaxcols = 0;
  for (const SvdJob &J : c->jobs) {
    const int ca = J.cols_a;
    c->tmaxcols = std::max(c->tmaxcols, ca);
    c->svdG.task(J.sb, BUF_SVD, J.x_off, ca, ca, ca);
    c->svdG.seg(BUF_SVD, J.j_off, ca, BUF_SVD, J.j_off, ca, ca, 2);
    c->svdW.task(J.sb, BUF_SVD, J.w_off, ca, ca, ca);
    c->svdW.seg(BUF_SVD, J.x_off, ca, BUF_SVD, J.j_off, ca, ca, 0);
    c->svdX.task(J.sb, BUF_SVD, J.w_off, ca, ca, ca);
    c->svdX.seg(BUF_SVD, J.j_off, ca, BUF_SVD, J.b_off, ca, ca, 0);
  }
  NOMEM(c->ensure(c->siw, 4 * std::max(iw, 1)));
  NOMEM(c->upload(c->sjobs, c->jobs) && c->ensure(c->swork, 8 * std::max<int64_t>(work, 1)) &&
        c->ensure(c->ssv, 8 * std::max(sv, 1)) && c->upload(c->sjob0, c->tjob0) && c->upload(c->snjob, c->tnjob) &&
        c->ensure(c->skpj, 4 * std::max(nj, 1)) && c->ensure(c->sperm, 4 * std::max(sv, 1)) &&
        c->ensure(c->slam, 8 * std::max(sv, 1)) && c->ensure(c->seps, 8 * P) && c->ensure(c->sepsb, 8 * P) &&
        c->ensure(c->skept, 4 * P) && c->upload(c->sorder, c->torder) && c->upload(c->sorderq, c->torderq) &&
        c->ensure(c->slamk, 8 * (size_t)P * std::max(1, c->o.m)));
  for (auto [L, dk, ds, T] : {std::make_tuple(&c->svdG, &c->dsgk, &c->dsgs, &c->tn_svdG),
                               std::make_tuple(&c->svdW, &c->dswk, &c->dsws, &c->tn_svdW),
                               std::make_tuple(&c->svdX, &c->dsxk, &c->dsxs, &c->tn_svdX)}) {
    idmrg_status sg = gemm_upload(c, *L, *dk, *ds, *T);
    if (sg != IDMRG_OK) return sg;
  }
  for (int q = 0; q < P; ++q) c->hbufs[q * NBUF + BUF_SVD] = c->dp(c->swork);
  NOMEM(sync_bufs(c) == IDMRG_OK);
  return IDMRG_OK;
}

// algorithmic flops of the sector SVDs of superblock q (all if q < 0): the
// R-SVD count 6 r c^2 + 20 c^3 for singular values and both thin factors of
// an r x c matrix, r >= c
double svd_flops(const idmrg_ctx *c, int q) {
  double f = 0.0;
  for (const SvdJob &j : c->jobs) {
    if (q >= 0 && j.sb != q) continue;
    const double r = j.rows_a, cc = j.cols_a;
    f += 6.0 * r * cc * cc + 20.0 * cc * cc * cc;
  }
  return f;
}

SelectOut select_out(idmrg_ctx *c, int q0) {
  SelectOut so{};
  so.kept_per_job = (int *)c->skpj.p;
  so.perm = (int *)c->sperm.p;
  so.lam_sorted = c->dp(c->slam);
  so.eps = c->dp(c->seps) + q0;
  so.eps_best = c->dp(c->sepsb) + q0;
  so.kept = (int *)c->skept.p + q0;
  return so;
}

// New bases of superblock q from the selection (host arrays indexed like the
// device ones: kpj per job, lam per singular value, iw per job slot, eps and
// eps_best per superblock); appends q's compaction jobs to cj.
idmrg_status trunc_host(idmrg_ctx *c, int q, const int *kpj, const double *lam, const int *iwh, const double *eps,
                        const double *epsb, std::vector<CompactJob> &cj) {
  const int P = c->P, target = c->o.target_charge;
  for (int j = c->tjob0[q]; j < c->tjob0[q] + c->tnjob[q]; ++j) {
    const SvdJob &J = c->jobs[j];
    const int rk = iwh[J.perm_off + J.cols_a], sw = iwh[J.perm_off + J.cols_a + 1];
    c->svd_max_cols = std::max(c->svd_max_cols, J.cols_a);
    c->svd_max_rank = std::max(c->svd_max_rank, rk);
    c->svd_max_sweeps = std::max(c->svd_max_sweeps, sw);
    c->svd_mean_sweeps += (double)sw / std::max(c->svd_jobs, 1);
    if (rk >= 2) {
      const int s32 = iwh[J.perm_off + J.cols_a + 2];
      c->svd_max_sweeps32 = std::max(c->svd_max_sweeps32, s32);
      c->svd_mean_sweeps32 += s32;
      c->svd_jobs32 += 1;
    }
  }
  TruncRec &T = c->cur[q];
  {
    const DevBuf keepU = T.U, keepV = T.V;  // recycle the device buffers
    T = TruncRec();
    T.U = keepU;
    T.V = keepV;
  }
  T.valid = true;
  T.leftB = c->envL[q].lay.b;
  T.rightB = c->envR[c->nxt(q)].lay.b;
  T.eps = eps[q];
  T.eps_best = epsb[q];
  int lam_off = 0;
  int64_t uo = 0, vo = 0;
  for (SecInfo si : c->tsecs[q]) {
    si.k = kpj[si.job];
    if (si.k == 0) continue;
    si.u_off = uo;
    si.v_off = vo;
    si.lam_off = lam_off;
    uo += (int64_t)si.r * si.k;
    vo += (int64_t)si.c * si.k;
    lam_off += si.k;
    T.bU.add(si.Q, si.k);
    T.bV.add(target - si.Q, si.k);
    T.sec.push_back(si);
  }
  T.bU.finish();
  T.bV.finish();
  T.usize = uo;
  T.vsize = vo;
  if (c->tnjob[q] > 0) {
    const SvdJob &J0 = c->jobs[c->tjob0[q]], &J1 = c->jobs[c->tjob0[q] + c->tnjob[q] - 1];
    T.lam_all.assign(lam + J0.sv_off, lam + J1.sv_off + J1.cols_a);
  }
  NOMEM(c->ensure(T.U, 8 * std::max<int64_t>(uo, 1)) && c->ensure(T.V, 8 * std::max<int64_t>(vo, 1)));
  c->hbufs[q * NBUF + BUF_U] = (double *)T.U.p;
  c->hbufs[q * NBUF + BUF_V] = (double *)T.V.p;
  // kept lambdas go to one device array: per superblock at a fixed stride
  const int stride = std::max(1, c->o.m);
  for (const SecInfo &si : T.sec) {
    CompactJob j{};
    j.job = si.job;
    j.u_off = si.u_off;
    j.v_off = si.v_off;
    j.lam_off = si.lam_off + q * stride;
    cj.push_back(j);
  }
  return IDMRG_OK;
}

idmrg_status trunc_compact(idmrg_ctx *c, DevBuf &dcj, const std::vector<CompactJob> &cj, int max_kept,
                           cudaStream_t s) {
  if (cj.empty()) return IDMRG_OK;
  NOMEM(c->ensure(dcj, std::max<size_t>(cj.size() * sizeof(CompactJob), 16)));
  CK(cudaMemcpyAsync(dcj.p, cj.data(), cj.size() * sizeof(CompactJob), cudaMemcpyHostToDevice, s));
  c->h2d += cj.size() * sizeof(CompactJob);
  int max_rows = 0;
  for (const CompactJob &j : cj) max_rows = std::max(max_rows, c->jobs[j.job].rows_a);
  CK(launch_svd_compact((const SvdJob *)c->sjobs.p, (const CompactJob *)dcj.p, (int)cj.size(), std::max(1, max_kept),
                        max_rows, c->dp(c->swork), (const int *)c->siw.p, c->dp(c->ssv), (const int *)c->sperm.p,
                        (const int *)c->skpj.p, (double *const *)c->dbufs.p, c->dp(c->slamk), s));
  c->launches += 1;
  return IDMRG_OK;
}

void svd_stats_reset(idmrg_ctx *c) {
  c->svd_jobs = (int)c->jobs.size();
  c->svd_max_cols = c->svd_max_rank = c->svd_max_sweeps = 0;
  c->svd_mean_sweeps = 0.0;
  c->svd_max_sweeps32 = 0;
  c->svd_mean_sweeps32 = 0.0;
  c->svd_jobs32 = 0;
}

idmrg_status truncate(idmrg_ctx *c, int p) {
  const int P = c->P;
  for (int q = 0; q < P; ++q)
    if (want(c, p, q) && c->stage[q] != ST_SOLVED)
      return c->fail(IDMRG_ESTATE, "truncate: superblock %d has not been solved", q);
  idmrg_status s0 = trunc_plan(c, p);
  if (s0 != IDMRG_OK) return s0;
  const int nj = (int)c->jobs.size();
  double *const *bufs = (double *const *)c->dbufs.p;
  const int PH = IDMRG_K_COUNT;  // SVD phases: 0 gather + QR, 1 FP32 Jacobi, 2 Newton-Schulz + X = B V,
                                // 3 FP64 Jacobi, 4 select, 5 compact
  c->kbegin(IDMRG_K_SVD);
  c->kbegin(PH + 0);
  CK(launch_svd_gather_sized((const SvdJob *)c->sjobs.p, nj, c->tmaxel_all, bufs, BUF_PSI, c->dp(c->swork), c->st));
  // groups over all jobs (largest first across superblocks): the pivoted QR
  // and both Jacobi stages run each group on clusters of the same size
  int g[4], gcols[4], grows[4] = {0, 0, 0, 0}, rows0 = 0, cols0 = 0;
  jacobi_groups(c, c->torder.data(), nj, g, gcols);
  for (int k = 1; k < 5; ++k) {
    const int lo = g[k - 1], hi = k < 4 ? g[k] : nj;
    for (int j = lo; j < hi; ++j) grows[k - 1] = std::max(grows[k - 1], c->jobs[c->torder[j]].rows_a);
  }
  for (int j = 0; j < g[0]; ++j) {
    rows0 = std::max(rows0, c->jobs[c->torder[j]].rows_a);
    cols0 = std::max(cols0, c->jobs[c->torder[j]].cols_a);
  }
  if (c->side_streams() != IDMRG_OK) return c->fail(IDMRG_ECUDA, "truncate: cannot create the SVD side streams");
  CK(launch_svd_qrcp_grouped((const SvdJob *)c->sjobs.p, (const int *)c->sorder.p, nj, g, grows, gcols, rows0, cols0,
                             c->dp(c->swork), (int *)c->siw.p, c->o.lambda_zero_rel, c->svd_global, c->st, c->side,
                             c->sev));
  if (c->side_streams() != IDMRG_OK) return c->fail(IDMRG_ECUDA, "truncate: cannot create the SVD side streams");
  // FP32 stage: rotations V to FP32 accuracy; Newton-Schulz makes V
  // orthogonal to FP64 precision (V <- 1.5 V - 0.5 V V^T V, twice); X = B V;
  // the FP64 stage starts from X with its rotations initialised to V
  const SvdJob *dj = (const SvdJob *)c->sjobs.p;
  double *sw = c->dp(c->swork);
  double *const *svb = (double *const *)c->dbufs.p;
  c->kend(PH + 0);
  c->kbegin(PH + 1);
  CK(launch_svd_elementwise(dj, nj, c->tmaxcols, 0, sw, c->st));
  {
    // group 0 from g0b on fits the shared-memory FP32 tournament (none in
    // the forced large-sector mode, which exercises the all-global kernel)
    const int bmax = c->svd_global ? 0 : svd_jacobi32_big_max_cols();
    int g0b = 0;
    while (g0b < g[0] && c->jobs[c->torder[g0b]].cols_a > bmax) ++g0b;
    const int cols0b = g0b < g[0] ? c->jobs[c->torder[g0b]].cols_a : 0;
    CK(launch_svd_jacobi32(dj, (const int *)c->sorder.p, nj, g, gcols, cols0, g0b, cols0b, sw, (const int *)c->siw.p,
                           c->st, c->side, c->sev));
  }
  c->kend(PH + 1);
  c->kbegin(PH + 2);
  for (int it = 0; it < 2; ++it) {
    {
    idmrg_status sg_ = gemm_run(c, c->tn_svdG, c->dsgk, c->dsgs, nullptr);
    if (sg_ != IDMRG_OK) return sg_;
  }
    {
    idmrg_status sg_ = gemm_run(c, c->tn_svdW, c->dswk, c->dsws, nullptr);
    if (sg_ != IDMRG_OK) return sg_;
  }
    CK(launch_svd_elementwise(dj, nj, c->tmaxcols, 1, sw, c->st));
  }
  {
    idmrg_status sg_ = gemm_run(c, c->tn_svdX, c->dsxk, c->dsxs, nullptr);
    if (sg_ != IDMRG_OK) return sg_;
  }
  CK(launch_svd_elementwise(dj, nj, c->tmaxcols, 2, sw, c->st));
  c->kend(PH + 2);
  c->kbegin(PH + 3);
  CK(launch_svd_jacobi(dj, (const int *)c->sorder.p, nj, g, gcols, sw, (int *)c->siw.p, c->dp(c->ssv),
                       (int *)c->derr.p, 1, c->jac_pairs(), c->st, c->side, c->sev));
  c->kend(PH + 3);
  c->launches += 12;
  // select: one launch, one CTA per superblock (no jobs: nothing kept)
  std::vector<int> sbl;
  for (int q = 0; q < P; ++q)
    if (want(c, p, q)) sbl.push_back(q);
  c->kbegin(PH + 4);
  CK(launch_svd_select((const SvdJob *)c->sjobs.p, (const int *)c->sjob0.p, (const int *)c->snjob.p, P,
                       c->dp(c->ssv), (const int *)c->dmsb.p, c->o.lambda_zero_rel, c->o.tie_rel, select_out(c, 0),
                       c->tentries_max,
                       c->st));
  c->kend(PH + 4);
  c->kend(IDMRG_K_SVD, svd_flops(c, -1), 0.0);
  c->launches += 3;
  std::vector<int> kpj(std::max(nj, 1)), iwh(std::max(c->tiw, 1));
  std::vector<double> lam_sorted(std::max(c->tsv, 1)), eps(P), epsb(P);
  CK(c->d2h_copy(iwh.data(), c->siw.p, 4 * (size_t)c->tiw));
  CK(c->d2h_copy(kpj.data(), c->skpj.p, 4 * (size_t)nj));
  CK(c->d2h_copy(lam_sorted.data(), c->slam.p, 8 * (size_t)c->tsv));
  CK(c->d2h_copy(eps.data(), c->seps.p, 8 * P));
  CK(c->d2h_copy(epsb.data(), c->sepsb.p, 8 * P));
  idmrg_status s = check_dev_err(c);
  if (s != IDMRG_OK) return s;
  svd_stats_reset(c);
  std::vector<CompactJob> cj;
  for (int q : sbl) {
    s = trunc_host(c, q, kpj.data(), lam_sorted.data(), iwh.data(), eps.data(), epsb.data(), cj);
    if (s != IDMRG_OK) return s;
  }
  NOMEM(sync_bufs(c) == IDMRG_OK);
  int max_kept = 1;
  for (int v : kpj) max_kept = std::max(max_kept, v);
  c->kbegin(IDMRG_K_SVD);
  c->kbegin(PH + 5);
  s = trunc_compact(c, c->scj, cj, max_kept, c->st);
  if (s != IDMRG_OK) return s;
  c->kend(PH + 5);
  c->kend(IDMRG_K_SVD);
  const int stride = std::max(1, c->o.m);
  std::vector<double> lamk((size_t)P * stride);
  CK(c->d2h_copy(lamk.data(), c->slamk.p, 8 * lamk.size()));
  CK(cudaStreamSynchronize(c->st));
  for (int q : sbl) {
    TruncRec &T = c->cur[q];
    T.lam.assign(lamk.begin() + (size_t)q * stride, lamk.begin() + (size_t)q * stride + T.bU.D);
    c->stage[q] = ST_TRUNCATED;
  }
  return IDMRG_OK;
}

// ------------------------------------------------------------------------
// Step 6: block-spin transformation (Eqs. L, R)
// ------------------------------------------------------------------------
// Step 6 task lists of pair q: X = env . U (V), Y = W . X, new env = U^T Y
// (V Y); appends to g1, w, g3 and sizes the pair's new environments and
// scratch (pointer table entries LNEW, RNEW, X, Y of q).
idmrg_status env_build(idmrg_ctx *c, int q, GemmList &g1, GemmList &g3, WList &w) {
  const int P = c->P, d = c->d, target = c->o.target_charge;
  const SBPlan &S = c->plan[q];
  const Env &L = c->envL[q];
  const Env &R = c->envR[c->nxt(q)];
  const Basis &BL = L.lay.b, &BR = R.lay.b;
  const TruncRec &T = c->cur[q];
  const int SL = BL.S(), SR = BR.S();
  const int wa = L.lay.w, wb = c->adim[c->bond_right(S.c1)], wc = R.lay.w;
  std::map<int, int> secQ;
  for (int k = 0; k < (int)T.sec.size(); ++k) secQ[T.sec[k].Q] = k;
  auto sec_of = [&](int Q) { auto it = secQ.find(Q); return it == secQ.end() ? -1 : it->second; };
  int64_t xs = 0, ys = 0;
  // ---------------- left: X[a](so, s') = L_a(so,si) U[(si,s')]
  std::vector<int64_t> xl((size_t)wa * SL * d, -1), yl((size_t)wb * SL * d, -1);
  for (int a = 0; a < wa; ++a)
    for (int si = 0; si < SL; ++si) {
      const int so = L.lay.so[a * SL + si];
      if (so < 0) continue;
      for (int s2 = 0; s2 < d; ++s2) {
        const int k = sec_of(BL.q[si] + c->qp[s2]);
        if (k < 0) continue;
        const SecInfo &sc = T.sec[k];
        int rs = -1;
        for (const auto &g : sc.rg)
          if (g[0] == si && g[1] == s2) rs = g[2];
        if (rs < 0) continue;
        xl[((size_t)a * SL + so) * d + s2] = xs;
        g1.task(q, BUF_X, xs, BL.dim[so], sc.k, sc.k);
        g1.seg(BUF_L, L.lay.off[a * SL + si], BL.dim[si], BUF_U, sc.u_off + (int64_t)rs * sc.k, sc.k,
                     BL.dim[si], 0);
        xs += (int64_t)BL.dim[so] * sc.k;
      }
    }
  // Y[b](so, s) = sum_{a,s'} W_c1(a,b,s,s') X[a](so,s')
  std::vector<int> bchq(c->bq[c->bond_right(S.c1)]);
  for (int b = 0; b < wb; ++b)
    for (int so = 0; so < SL; ++so)
      for (int s = 0; s < d; ++s) {
        const int ko = sec_of(BL.q[so] + c->qp[s]);
        const int ki = sec_of(BL.q[so] + c->qp[s] - bchq[b]);
        if (ko < 0 || ki < 0) continue;
        const int kin = T.sec[ki].k;
        yl[((size_t)b * SL + so) * d + s] = ys;
        w.task(q, BUF_Y, ys, kin, BUF_X, BL.dim[so], kin);
        for (int a = 0; a < wa; ++a)
          for (int s2 = 0; s2 < d; ++s2) {
            const double cf = c->Wat(S.c1, a, b, s, s2);
            if (cf == 0.0) continue;
            const int64_t xo = xl[((size_t)a * SL + so) * d + s2];
            if (xo < 0) continue;
            w.term(xo, kin, cf);
          }
        ys += (int64_t)BL.dim[so] * kin;
      }
  // L'[b](Qo, Qi) = sum_{(so,s) in Qo} U[(so,s)]^T Y[b](so,s)
  Env &NL = c->newL[q];
  NL.lay.build(T.bU, bchq);
  NOMEM(c->ensure(NL.data, 8 * std::max<int64_t>(NL.lay.size, 1)));
  c->hbufs[q * NBUF + BUF_LNEW] = c->dp(NL.data);
  const int SU = T.bU.S();
  for (int b = 0; b < wb; ++b)
    for (int si = 0; si < SU; ++si) {
      const int so = NL.lay.so[b * SU + si];
      if (so < 0) continue;
      const SecInfo &o = T.sec[so];
      const int kin = T.sec[si].k;
      g3.task(q, BUF_LNEW, NL.lay.off[b * SU + si], o.k, kin, kin);
      for (const auto &g : o.rg) {
        const int64_t y = yl[((size_t)b * SL + g[0]) * d + g[1]];
        if (y < 0) continue;
        g3.seg(BUF_U, o.u_off + (int64_t)g[2] * o.k, o.k, BUF_Y, y, kin, BL.dim[g[0]], 1);
      }
    }
  // ---------------- right: X[c](jo, t') = R_c(jo,ji) V[(t',ji)]
  std::vector<int64_t> xr((size_t)wc * SR * d, -1), yr((size_t)wb * SR * d, -1);
  for (int cc = 0; cc < wc; ++cc)
    for (int ji = 0; ji < SR; ++ji) {
      const int jo = R.lay.so[cc * SR + ji];
      if (jo < 0) continue;
      for (int t2 = 0; t2 < d; ++t2) {
        const int k = sec_of(target - (c->qp[t2] + BR.q[ji]));
        if (k < 0) continue;
        const SecInfo &sc = T.sec[k];
        int cs = -1;
        for (const auto &g : sc.cg)
          if (g[0] == t2 && g[1] == ji) cs = g[2];
        if (cs < 0) continue;
        xr[((size_t)cc * SR + jo) * d + t2] = xs;
        g1.task(q, BUF_X, xs, BR.dim[jo], sc.k, sc.k);
        g1.seg(BUF_R, R.lay.off[cc * SR + ji], BR.dim[ji], BUF_V, sc.v_off + (int64_t)cs * sc.k, sc.k,
                     BR.dim[ji], 0);
        xs += (int64_t)BR.dim[jo] * sc.k;
      }
    }
  // Y[b](jo, t) = sum_{c,t'} W_c2(b,c,t,t') X[c](jo,t')
  std::vector<int> rchq(wb);
  for (int b = 0; b < wb; ++b) rchq[b] = -c->bq[S.c2][b];
  for (int b = 0; b < wb; ++b)
    for (int jo = 0; jo < SR; ++jo)
      for (int t = 0; t < d; ++t) {
        const int qo = c->qp[t] + BR.q[jo];           // right charge of row (t, jo)
        const int ko = sec_of(target - qo);
        const int ki = sec_of(target - (qo - rchq[b]));
        if (ko < 0 || ki < 0) continue;
        const int kin = T.sec[ki].k;
        yr[((size_t)b * SR + jo) * d + t] = ys;
        w.task(q, BUF_Y, ys, kin, BUF_X, BR.dim[jo], kin);
        for (int cc = 0; cc < wc; ++cc)
          for (int t2 = 0; t2 < d; ++t2) {
            const double cf = c->Wat(S.c2, b, cc, t, t2);
            if (cf == 0.0) continue;
            const int64_t xo = xr[((size_t)cc * SR + jo) * d + t2];
            if (xo < 0) continue;
            w.term(xo, kin, cf);
          }
        ys += (int64_t)BR.dim[jo] * kin;
      }
  Env &NR = c->newR[q];
  NR.lay.build(T.bV, rchq);
  NOMEM(c->ensure(NR.data, 8 * std::max<int64_t>(NR.lay.size, 1)));
  c->hbufs[q * NBUF + BUF_RNEW] = c->dp(NR.data);
  const int SV = T.bV.S();
  for (int b = 0; b < wb; ++b)
    for (int si = 0; si < SV; ++si) {
      const int so = NR.lay.so[b * SV + si];
      if (so < 0) continue;
      const SecInfo &o = T.sec[so];
      const int kin = T.sec[si].k;
      g3.task(q, BUF_RNEW, NR.lay.off[b * SV + si], o.k, kin, kin);
      for (const auto &g : o.cg) {
        const int64_t y = yr[((size_t)b * SR + g[1]) * d + g[0]];
        if (y < 0) continue;
        g3.seg(BUF_V, o.v_off + (int64_t)g[2] * o.k, o.k, BUF_Y, y, kin, BR.dim[g[1]], 1);
      }
    }
  NOMEM(c->ensure(c->bX[q], 8 * std::max<int64_t>(xs, 1)) && c->ensure(c->bY[q], 8 * std::max<int64_t>(ys, 1)));
  c->hbufs[q * NBUF + BUF_X] = c->dp(c->bX[q]);
  c->hbufs[q * NBUF + BUF_Y] = c->dp(c->bY[q]);
  return IDMRG_OK;
}

idmrg_status update_envs(idmrg_ctx *c, int p) {
  const int P = c->P;
  for (int q = 0; q < P; ++q)
    if (want(c, p, q) && c->stage[q] != ST_TRUNCATED)
      return c->fail(IDMRG_ESTATE, "update_environments: superblock %d is not truncated", q);
  c->genv1.clear();
  c->genv3.clear();
  c->wenv.clear();
  for (int q = 0; q < P; ++q) {
    if (!want(c, p, q)) continue;
    idmrg_status s = env_build(c, q, c->genv1, c->genv3, c->wenv);
    if (s != IDMRG_OK) return s;
  }
  NOMEM(sync_bufs(c) == IDMRG_OK);
  {
    idmrg_status sg = gemm_upload(c, c->genv1, c->dge1k, c->dge1s, c->tn_env1);
    if (sg != IDMRG_OK) return sg;
    sg = gemm_upload(c, c->genv3, c->dge3k, c->dge3s, c->tn_env3);
    if (sg != IDMRG_OK) return sg;
  }
  NOMEM(c->upload(c->dwet, c->wenv.tasks) && c->upload(c->dwem, c->wenv.terms));
  double *const *bufs = (double *const *)c->dbufs.p;
  c->kbegin(IDMRG_K_ENV);
  {
    idmrg_status sg_ = gemm_run(c, c->tn_env1, c->dge1k, c->dge1s, nullptr);
    if (sg_ != IDMRG_OK) return sg_;
  }
  CK(launch_wstage_f64((const WTask *)c->dwet.p, (int)c->wenv.tasks.size(), c->wenv.max_rows,
                       (const WTerm *)c->dwem.p, bufs, nullptr, c->st));
  {
    idmrg_status sg_ = gemm_run(c, c->tn_env3, c->dge3k, c->dge3s, nullptr);
    if (sg_ != IDMRG_OK) return sg_;
  }
  c->kend(IDMRG_K_ENV, c->genv1.flops + c->wenv.flops + c->genv3.flops, 0.0);
  c->launches += 3;
  for (int q = 0; q < P; ++q)
    if (want(c, p, q)) c->stage[q] = ST_UPDATED;
  return IDMRG_OK;
}

// ------------------------------------------------------------------------
// Step 7 and the rotation of Step 2'
// ------------------------------------------------------------------------
idmrg_status advance(idmrg_ctx *c) {
  const int P = c->P;
  for (int q = 0; q < P; ++q)
    if (c->owns(q) && c->stage[q] != ST_UPDATED)
      return c->fail(IDMRG_ESTATE, "advance: superblock %d is not updated", q);
  CK(cudaStreamSynchronize(c->st));
  c->obs.valid = c->obs.fixed = false;
  for (int q = 0; q < P; ++q) {
    std::swap(c->envL[q], c->newL[q]);
    std::swap(c->envR[q], c->newR[q]);
  }
  // lambda history: cur -> prev -> prev2 (buffers recycled); for another
  // worker's pair the stale record moves along and the import replaces prev
  for (int q = 0; q < P; ++q) {
    std::swap(c->prev2[q], c->prev[q]);
    std::swap(c->prev[q], c->cur[q]);
  }
  for (idmrg_ctx::Ring &R : c->rings) {
    if (!c->owns(R.p0)) continue;  // Step 5' (superblock 1 of the paper) of each ring
    R.eps1[c->n] = c->prev[R.p0].eps;
    R.e1[c->n] = c->energy[R.p0];
    if ((c->n + 1) % R.ell == 0) {
      const double before = (c->n - R.ell == -1) ? 0.0 : R.e1[c->n - R.ell];
      R.eg_last = (R.e1[c->n] - before) / (2.0 * R.ell);
      R.eg_n = c->n;
    }
  }
  c->n += 1;
  if (!c->owns_all()) {  // the right block of the last superblock comes from the next worker
    c->plan_pending = true;
    for (int q = 0; q < P; ++q) c->stage[q] = ST_READY;
    return IDMRG_OK;
  }
  return plan_iteration(c);
}

// ------------------------------------------------------------------------
// Uniform-MPS observables (Sec. 3, Eq. mps2)
// ------------------------------------------------------------------------
// The unit after iteration n is V^(n)_1^T u~^(n)_2 V^(n)_2^T u~^(n)_3 ... with
// u~^(n)_{i+1} = (lam^(n-1)_{i+1})^-1 u^(n)_{i+1} lam^(n)_{i+1}, the tensors
// Eq. wfprediction scales for iteration n + 1 (same zero rule); A_2p = V_p^T
// carries lattice site f(2p + n + 1), A_2p+1 = u~_p+1 the next one.  The unit
// is not exactly right-normalised, so expectation values use the dominant
// left and right eigenvectors of its transfer map.  Environments are D x D
// dense; the site tensors are multiplied block by block (charge blocks).
enum ObsBuf { OB_A = 0, OB_Y = 1, OB_EL = 2, OB_ER = 3, OB_X0 = 4 };  // X_i at OB_X0 + i

double *obs_x(idmrg_ctx *c, int i) { return (double *)c->obs.X[i].p; }

// out = alpha sum_{s,t} O[s][t] A_k[s]^T in A_k[t]   (O null: identity)
void obs_left_map(const ObsState &S, int d, int k, const double *O, double alpha, int in_buf, int64_t in_off,
                  int out_buf, int64_t out_off, GemmList &g1, GemmList &g2) {
  const int Dk = S.D[k], Dk1 = S.D[k + 1];
  const int64_t plane = (int64_t)Dk * Dk1;
  const auto &B0 = S.bb[k], &B1 = S.bb[k + 1];
  const int nb1 = (int)B1.size();
  auto o_at = [&](int s, int t) { return O ? O[s * d + t] : (s == t ? 1.0 : 0.0); };
  g1.clear();
  g2.clear();
  // Y[t] = in A_k[t], every column block written (zero where A has no block)
  for (int t = 0; t < d; ++t) {
    bool used = false;
    for (int s = 0; s < d; ++s) used = used || o_at(s, t) != 0.0;
    if (!used) continue;
    for (int cb = 0; cb < nb1; ++cb) {
      g1.task(0, OB_Y, t * plane + B1[cb].first, Dk, B1[cb].second, Dk1);
      const int rb = S.rb_of[k][t * nb1 + cb];
      if (rb >= 0)
        g1.seg(in_buf, in_off + B0[rb].first, Dk, OB_A, S.aoff[k] + t * plane + (int64_t)B0[rb].first * Dk1 +
               B1[cb].first, Dk1, B0[rb].second, 0);
    }
  }
  // out[cb rows] = sum_{s,t} alpha O[s][t] A_k[s][rb, cb]^T Y[t][rb rows]
  for (int cb = 0; cb < nb1; ++cb) {
    g2.task(0, out_buf, out_off + (int64_t)B1[cb].first * Dk1, B1[cb].second, Dk1, Dk1);
    for (int s = 0; s < d; ++s) {
      const int rb = S.rb_of[k][s * nb1 + cb];
      if (rb < 0) continue;
      for (int t = 0; t < d; ++t) {
        const double o = o_at(s, t);
        if (o == 0.0) continue;
        g2.seg(OB_A, S.aoff[k] + s * plane + (int64_t)B0[rb].first * Dk1 + B1[cb].first, Dk1, OB_Y,
               t * plane + (int64_t)B0[rb].first * Dk1, Dk1, B0[rb].second, 1, alpha * o);
      }
    }
  }
  g1.finish(32, 32);
  g2.finish(32, 32);
}

// out = alpha sum_t A_k[t] in A_k[t]^T
void obs_right_map(const ObsState &S, int d, int k, double alpha, int in_buf, int64_t in_off, int out_buf,
                   int64_t out_off, GemmList &g1, GemmList &g2) {
  const int Dk = S.D[k], Dk1 = S.D[k + 1];
  const int64_t plane = (int64_t)Dk * Dk1;
  const auto &B0 = S.bb[k], &B1 = S.bb[k + 1];
  const int nb0 = (int)B0.size();
  g1.clear();
  g2.clear();
  // Y[t] = A_k[t] in, every row block written
  for (int t = 0; t < d; ++t)
    for (int rb = 0; rb < nb0; ++rb) {
      g1.task(0, OB_Y, t * plane + (int64_t)B0[rb].first * Dk1, B0[rb].second, Dk1, Dk1);
      const int cb = S.cb_of[k][t * nb0 + rb];
      if (cb >= 0)
        g1.seg(OB_A, S.aoff[k] + t * plane + (int64_t)B0[rb].first * Dk1 + B1[cb].first, Dk1, in_buf,
               in_off + (int64_t)B1[cb].first * Dk1, Dk1, B1[cb].second, 0);
    }
  // out[:, rb] = sum_t alpha Y[t][:, cb] A_k[t][rb, cb]^T
  for (int rb = 0; rb < nb0; ++rb) {
    g2.task(0, out_buf, out_off + B0[rb].first, Dk, B0[rb].second, Dk);
    for (int t = 0; t < d; ++t) {
      const int cb = S.cb_of[k][t * nb0 + rb];
      if (cb < 0) continue;
      g2.seg(OB_Y, t * plane + B1[cb].first, Dk1, OB_A,
             S.aoff[k] + t * plane + (int64_t)B0[rb].first * Dk1 + B1[cb].first, Dk1, B1[cb].second, 2, alpha);
    }
  }
  g1.finish(32, 32);
  g2.finish(32, 32);
}

idmrg_status obs_upload(idmrg_ctx *c, ObsArena &a) {
  NOMEM(c->upload(a.dtasks, a.G.tasks) && c->upload(a.dsegs, a.G.segs) && c->upload(a.dtiles, a.G.tiles));
  return IDMRG_OK;
}

idmrg_status obs_run(idmrg_ctx *c, ObsArena &a, const ObsList &L) {
  CK(launch_gemm_f64((const GemmTile *)a.dtiles.p + L.tile0, L.ntile, (const GemmTask *)a.dtasks.p,
                     (const GemmSeg *)a.dsegs.p, (double *const *)c->obs.tab.p, nullptr, c->st, GEMM_32x32));
  c->launches += 1;
  return IDMRG_OK;
}

idmrg_status obs_read(idmrg_ctx *c, double *host, int n) {
  CK(c->d2h_copy(host, c->obs.res.p, sizeof(double) * n));
  CK(cudaStreamSynchronize(c->st));
  return IDMRG_OK;
}

idmrg_status obs_dot(idmrg_ctx *c, const double *x, const double *y, int64_t n, double coef, int slot, int acc) {
  CK(launch_obs_dot(x, y, n, coef, (double *)c->obs.res.p + slot, acc, c->st));
  c->launches += 1;
  return IDMRG_OK;
}

idmrg_status obs_axpby(idmrg_ctx *c, const double *x, double *y, int64_t n, double a, double b) {
  CK(launch_obs_axpby(x, y, n, a, b, c->st));
  c->launches += 1;
  return IDMRG_OK;
}

#define OBS_TRY(call)                  \
  do {                                 \
    const idmrg_status s_ = (call);    \
    if (s_ != IDMRG_OK) return s_;     \
  } while (0)

// Embeds the unit of the last completed iteration and builds its block tables
// and the unit-map task lists.
idmrg_status obs_build(idmrg_ctx *c) {
  ObsState &S = c->obs;
  if (S.valid) return IDMRG_OK;
  const int P = c->P, d = c->d, ell = c->ell;
  if (c->n < 3) return c->fail(IDMRG_ESTATE, "observables need two completed iterations");
  for (int q = 0; q < P; ++q)
    if (!c->prev[q].valid || !c->prev2[q].valid)
      return c->fail(IDMRG_ESTATE, "observables need two completed iterations");
  S.fixed = false;
  S.s0 = (c->n - 1 + 1) % ell;
  S.D.assign(ell + 1, 0);
  S.bb.assign(ell + 1, {});
  S.blk.assign(ell, {});
  for (int p = 0; p < P; ++p) {
    const TruncRec &A = c->prev[p], &B = c->prev[c->nxt(p)];
    if (A.rightB.D != B.leftB.D || A.rightB.dim != B.leftB.dim)
      return c->fail(IDMRG_ESTATE, "observables: bases of superblocks %d and %d do not meet", p, c->nxt(p));
    if ((int)c->prev2[c->nxt(p)].lam.size() != B.leftB.D)
      return c->fail(IDMRG_ESTATE, "observables: lambda^(n-1) of superblock %d has the wrong length", c->nxt(p));
    for (const SecInfo &s : A.sec) S.bb[2 * p].push_back({s.lam_off, s.k});
    for (int j = 0; j < (int)A.rightB.dim.size(); ++j) S.bb[2 * p + 1].push_back({A.rightB.off[j], A.rightB.dim[j]});
    S.D[2 * p] = (int)A.lam.size();
    S.D[2 * p + 1] = A.rightB.D;
    for (int a = 0; a < (int)A.sec.size(); ++a)
      for (const auto &g : A.sec[a].cg) S.blk[2 * p].push_back({g[0], a, g[1]});
    for (int g = 0; g < (int)B.sec.size(); ++g)
      for (const auto &r : B.sec[g].rg) S.blk[2 * p + 1].push_back({r[1], r[0], g});
  }
  S.D[ell] = S.D[0];
  S.bb[ell] = S.bb[0];
  S.q0.clear();
  for (const SecInfo &s : c->prev[0].sec) S.q0.insert(S.q0.end(), s.k, s.Q);
  NOMEM(c->upload(S.dq0, S.q0));
  S.aoff.assign(ell + 1, 0);
  S.eoff.assign(ell + 2, 0);
  S.ysize = S.xsize = 0;
  S.rb_of.assign(ell, {});
  S.cb_of.assign(ell, {});
  for (int k = 0; k < ell; ++k) {
    const int64_t plane = (int64_t)S.D[k] * S.D[k + 1];
    S.aoff[k + 1] = S.aoff[k] + d * plane;
    S.ysize = std::max<int64_t>(S.ysize, d * plane);
    const int nb0 = (int)S.bb[k].size(), nb1 = (int)S.bb[k + 1].size();
    S.rb_of[k].assign((size_t)d * nb1, -1);
    S.cb_of[k].assign((size_t)d * nb0, -1);
    for (const ObsBlock &b : S.blk[k]) {
      S.rb_of[k][b.s * nb1 + b.cb] = b.rb;
      S.cb_of[k][b.s * nb0 + b.rb] = b.cb;
    }
  }
  for (int k = 0; k <= ell; ++k) {
    S.eoff[k + 1] = S.eoff[k] + (int64_t)S.D[k] * S.D[k];
    S.xsize = std::max<int64_t>(S.xsize, (int64_t)S.D[k] * S.D[k]);
  }
  NOMEM(c->ensure(S.A, 8 * std::max<int64_t>(S.aoff[ell], 1)) && c->ensure(S.Y, 8 * std::max<int64_t>(S.ysize, 1)) &&
        c->ensure(S.envl, 8 * S.eoff[ell + 1]) && c->ensure(S.envr, 8 * S.eoff[ell + 1]) &&
        c->ensure(S.res, 8 * 64));
  for (auto &x : S.X) NOMEM(c->ensure(x, 8 * S.xsize));
  // pointer table of the GEMM lists (superblock 0, slots OB_*)
  std::vector<double *> tab(NBUF, nullptr);
  tab[OB_A] = (double *)S.A.p;
  tab[OB_Y] = (double *)S.Y.p;
  tab[OB_EL] = (double *)S.envl.p;
  tab[OB_ER] = (double *)S.envr.p;
  for (int i = 0; i < 7; ++i) tab[OB_X0 + i] = (double *)S.X[i].p;
  NOMEM(c->upload(S.tab, tab));
  // embed: V^T (transposed copy) and u~ (rows / lam'', columns * lam)
  std::vector<double> scal;
  std::vector<EmbedTask> et;
  int max_rows = 0;
  double *Abase = (double *)S.A.p;
  for (int p = 0; p < P; ++p) {
    const int q = c->nxt(p);
    const TruncRec &A = c->prev[p], &B = c->prev[q], &B2 = c->prev2[q];
    {
      const int k = 2 * p, D1 = S.D[k + 1];
      const int64_t plane = (int64_t)S.D[k] * D1;
      for (const SecInfo &s : A.sec)
        for (const auto &g : s.cg) {
          EmbedTask t{};
          t.src = (const double *)A.V.p + s.v_off + (int64_t)g[2] * s.k;
          t.dst = Abase + S.aoff[k] + g[0] * plane + (int64_t)s.lam_off * D1 + A.rightB.off[g[1]];
          t.rows = s.k;
          t.cols = A.rightB.dim[g[1]];
          t.src_ld = s.k;
          t.dst_ld = D1;
          t.trans = 1;
          t.rs = t.cs = -1;
          et.push_back(t);
          max_rows = std::max(max_rows, t.rows);
        }
    }
    {
      const int k = 2 * p + 1, D1 = S.D[k + 1];
      const int64_t plane = (int64_t)S.D[k] * D1;
      const int lam_at = (int)scal.size();
      scal.insert(scal.end(), B.lam.begin(), B.lam.end());
      const int lam2_at = (int)scal.size();
      scal.insert(scal.end(), B2.lam.begin(), B2.lam.end());
      const double thr = c->o.lambda_zero_rel * (B2.lam_all.empty() ? 0.0 : B2.lam_all[0]);
      for (const SecInfo &s : B.sec)
        for (const auto &r : s.rg) {
          EmbedTask t{};
          t.src = (const double *)B.U.p + s.u_off + (int64_t)r[2] * s.k;
          t.dst = Abase + S.aoff[k] + r[1] * plane + (int64_t)B.leftB.off[r[0]] * D1 + s.lam_off;
          t.rows = B.leftB.dim[r[0]];
          t.cols = s.k;
          t.src_ld = s.k;
          t.dst_ld = D1;
          t.trans = 0;
          t.rs = lam2_at + B.leftB.off[r[0]];
          t.cs = lam_at + s.lam_off;
          t.thr = thr;
          et.push_back(t);
          max_rows = std::max(max_rows, t.rows);
        }
    }
  }
  NOMEM(c->upload(S.emb, et) && c->upload(S.scal, scal));
  CK(cudaMemsetAsync(S.A.p, 0, 8 * S.aoff[ell], c->st));
  CK(launch_obs_embed((const EmbedTask *)S.emb.p, (int)et.size(), max_rows, (const double *)S.scal.p, c->st));
  c->launches += 1;
  // unit maps (alpha 1), ping-pong X0 <-> X1, ending in X0 (l is even)
  S.unit.clear();
  S.unit_l.clear();
  S.unit_r.clear();
  GemmList g1, g2;
  for (int k = 0; k < ell; ++k) {
    const int in = (k % 2 == 0) ? OB_X0 : OB_X0 + 1, out = (k % 2 == 0) ? OB_X0 + 1 : OB_X0;
    obs_left_map(S, d, k, nullptr, 1.0, in, 0, out, 0, g1, g2);
    S.unit_l.push_back({S.unit.add(g1), S.unit.add(g2)});
  }
  for (int i = 0; i < ell; ++i) {
    const int k = ell - 1 - i;
    const int in = (i % 2 == 0) ? OB_X0 : OB_X0 + 1, out = (i % 2 == 0) ? OB_X0 + 1 : OB_X0;
    obs_right_map(S, d, k, 1.0, in, 0, out, 0, g1, g2);
    S.unit_r.push_back({S.unit.add(g1), S.unit.add(g2)});
  }
  OBS_TRY(obs_upload(c, S.unit));
  S.valid = true;
  return IDMRG_OK;
}

idmrg_status obs_unit_map(idmrg_ctx *c, bool left) {
  for (const auto &pr : left ? c->obs.unit_l : c->obs.unit_r) {
    OBS_TRY(obs_run(c, c->obs.unit, pr.first));
    OBS_TRY(obs_run(c, c->obs.unit, pr.second));
  }
  return IDMRG_OK;
}

// Two-vector subspace iteration of the unit map on charge-difference sector
// `delta` of bond 0 (the map keeps the charge difference of an environment's
// entries), Rayleigh-Ritz on the 2 x 2 projection H = X^T T X.
//  mode 0 (fixed point): the unscaled left or right map on sector 0 until the
//    dominant Ritz pair (theta real, largest) has |T x - theta x| <= tol theta
//    |x|; x (unit Frobenius norm) is written to dst, theta to *lam.  Its error
//    falls as |t3 / t1| per iteration, not |t2 / t1| as in a power iteration.
//  mode 1 (spectrum): the left map scaled by 1/t1, on sector 0 also deflated
//    of the fixed point (T(x)/t1 - l_0 (r_0|x), (l_0|r_0) = 1), until the
//    largest Ritz modulus changes by at most tol (relative) three times in a
//    row; it is written to *lam (a complex pair gives sqrt(det H)).
idmrg_status obs_subspace(idmrg_ctx *c, bool left, int delta, int mode, double tol, int maxit, double *lam,
                          int *iters, double *dst) {
  ObsState &S = c->obs;
  const int ell = c->ell, D0 = S.D[0];
  const int64_t n = (int64_t)D0 * D0;
  const double *l0 = (const double *)S.envl.p, *r0 = (const double *)S.envr.p + S.eoff[ell];
  double *x0 = obs_x(c, 0), *xr = obs_x(c, 2), *v[2] = {obs_x(c, 3), obs_x(c, 4)}, *y[2] = {obs_x(c, 5), obs_x(c, 6)};
  double h[4];
  const double tiny = 1e-280;
  const bool deflated = mode == 1 && delta == 0;
  for (int a = 0; a < 2; ++a) {
    CK(launch_obs_fill(v[a], D0, 1, 0.0, c->o.seed * 2654435761ull + 7919ull * (a + 1) + 104729ull * delta +
                       15485863ull * (left ? 1 : 2) * (mode + 1), c->st));
    CK(launch_obs_mask(v[a], D0, (const int *)S.dq0.p, delta, c->st));
    c->launches += 2;
  }
  auto deflate = [&](double *w) -> idmrg_status {
    if (!deflated) return IDMRG_OK;
    OBS_TRY(obs_dot(c, r0, w, n, 1.0, 0, 0));
    OBS_TRY(obs_read(c, h, 1));
    return obs_axpby(c, l0, w, n, -h[0], 1.0);
  };
  // orthonormalise (w0, w1) into (v0, v1); a vanishing second direction
  // becomes zero, a vanishing first one ends the iteration
  auto orth = [&](double *w0, double *w1, bool *dead) -> idmrg_status {
    OBS_TRY(obs_dot(c, w0, w0, n, 1.0, 0, 0));
    OBS_TRY(obs_read(c, h, 1));
    if (!(h[0] > tiny)) {
      *dead = true;
      return IDMRG_OK;
    }
    OBS_TRY(obs_axpby(c, w0, v[0], n, 1.0 / std::sqrt(h[0]), 0.0));
    OBS_TRY(obs_dot(c, v[0], w1, n, 1.0, 0, 0));
    OBS_TRY(obs_read(c, h, 1));
    OBS_TRY(obs_axpby(c, v[0], w1, n, -h[0], 1.0));
    OBS_TRY(obs_dot(c, w1, w1, n, 1.0, 0, 0));
    OBS_TRY(obs_read(c, h, 1));
    if (h[0] > tiny)
      OBS_TRY(obs_axpby(c, w1, v[1], n, 1.0 / std::sqrt(h[0]), 0.0));
    else
      OBS_TRY(obs_axpby(c, w1, v[1], n, 0.0, 0.0));
    return IDMRG_OK;
  };
  bool dead = false;
  OBS_TRY(deflate(v[0]));
  OBS_TRY(deflate(v[1]));
  OBS_TRY(orth(v[0], v[1], &dead));
  double last = -1.0;
  int stable = 0;
  bool done = false;
  *lam = 0.0;
  *iters = 0;
  for (int it = 1; it <= maxit && !dead && !done; ++it) {
    for (int a = 0; a < 2; ++a) {
      CK(cudaMemcpyAsync(x0, v[a], 8 * n, cudaMemcpyDeviceToDevice, c->st));
      OBS_TRY(obs_unit_map(c, left));
      OBS_TRY(obs_axpby(c, x0, y[a], n, mode == 1 ? 1.0 / S.t1 : 1.0, 0.0));
      OBS_TRY(deflate(y[a]));
    }
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) OBS_TRY(obs_dot(c, v[a], y[b], n, 1.0, 2 * a + b, 0));
    OBS_TRY(obs_read(c, h, 4));
    // H = [[h0, h1], [h2, h3]] (H[a][b] = (v_a | T v_b))
    const double tr = h[0] + h[3], det = h[0] * h[3] - h[1] * h[2];
    const double disc = 0.25 * tr * tr - det;
    if (!std::isfinite(tr) || !std::isfinite(det))
      return c->fail(IDMRG_ENUMERIC, "observables: transfer map gave non-finite values");
    *iters = it;
    if (mode == 1) {
      const double m = disc >= 0.0 ? std::max(std::fabs(0.5 * tr + std::sqrt(disc)), std::fabs(0.5 * tr - std::sqrt(disc)))
                                   : std::sqrt(std::max(det, 0.0));
      stable = (std::fabs(m - last) <= tol * std::max(m, tiny)) ? stable + 1 : 0;
      last = m;
      *lam = m;
      done = stable >= 3;
    } else if (disc >= 0.0) {
      // dominant real Ritz pair: theta, y with H y = theta y; x = V y
      const double th = 0.5 * tr + std::sqrt(disc);
      double ya = h[1], yb = th - h[0];          // from the first row of (H - theta)
      const double za = th - h[3], zb = h[2];    // from the second row
      if (za * za + zb * zb > ya * ya + yb * yb) { ya = za; yb = zb; }
      if (ya * ya + yb * yb > tiny && th > 0.0) {
        // x = ya v0 + yb v1 (in xr), T x = ya y0 + yb y1 (in x0), residual in x0
        OBS_TRY(obs_axpby(c, v[0], xr, n, ya, 0.0));
        OBS_TRY(obs_axpby(c, v[1], xr, n, yb, 1.0));
        OBS_TRY(obs_axpby(c, y[0], x0, n, ya, 0.0));
        OBS_TRY(obs_axpby(c, y[1], x0, n, yb, 1.0));
        OBS_TRY(obs_axpby(c, xr, x0, n, -th, 1.0));
        OBS_TRY(obs_dot(c, x0, x0, n, 1.0, 0, 0));
        OBS_TRY(obs_dot(c, xr, xr, n, 1.0, 1, 0));
        OBS_TRY(obs_read(c, h, 2));
        *lam = th;
        if (h[1] > tiny && std::sqrt(h[0]) <= tol * th * std::sqrt(h[1])) {
          double tracev[1];
          // unit norm, sign fixed by the trace (the fixed point is positive semidefinite)
          CK(launch_obs_fill(x0, D0, 0, 1.0, 0, c->st));
          c->launches += 1;
          OBS_TRY(obs_dot(c, x0, xr, n, 1.0, 0, 0));
          OBS_TRY(obs_read(c, tracev, 1));
          const double sg = tracev[0] < 0.0 ? -1.0 : 1.0;
          OBS_TRY(obs_axpby(c, xr, dst, n, sg / std::sqrt(h[1]), 0.0));
          done = true;
        }
      }
    }
    if (!done) OBS_TRY(orth(y[0], y[1], &dead));
  }
  if (mode == 1) {
    if (dead) *lam = 0.0;
    if (!dead && !done)
      return c->fail(IDMRG_ENOCONV, "observables: subspace iteration (charge difference %d) did not converge in %d "
                     "steps", delta, maxit);
    return IDMRG_OK;
  }
  if (dead) return c->fail(IDMRG_ENUMERIC, "observables: the transfer map annihilated its start vectors");
  if (!done)
    return c->fail(IDMRG_ENOCONV, "observables: fixed point of the transfer map not converged in %d steps", maxit);
  return IDMRG_OK;
}

// Fixed points l_0, r_0 with (l_0|r_0) = 1, the per-site factor t1^(-1/l)
// and the environments l_k (k = 0..l-1), r_k (k = 1..l) of the scaled maps.
idmrg_status obs_fixed(idmrg_ctx *c, double tol, int maxit) {
  OBS_TRY(obs_build(c));
  ObsState &S = c->obs;
  if (S.fixed) return IDMRG_OK;
  const int ell = c->ell, d = c->d, D0 = S.D[0];
  const int64_t n = (int64_t)D0 * D0;
  double *EL = (double *)S.envl.p, *ER = (double *)S.envr.p;
  OBS_TRY(obs_subspace(c, true, 0, 0, tol, maxit, &S.t1, &S.it_left, EL));
  OBS_TRY(obs_subspace(c, false, 0, 0, tol, maxit, &S.t1r, &S.it_right, ER + S.eoff[ell]));
  double h[1];
  OBS_TRY(obs_dot(c, EL, ER + S.eoff[ell], n, 1.0, 0, 0));
  OBS_TRY(obs_read(c, h, 1));
  if (!(std::fabs(h[0]) > 0.0) || !std::isfinite(h[0]))
    return c->fail(IDMRG_ENUMERIC, "observables: fixed points with overlap %g", h[0]);
  OBS_TRY(obs_axpby(c, ER + S.eoff[ell], ER + S.eoff[ell], n, 0.0, 1.0 / h[0]));
  S.scale = std::pow(S.t1, -1.0 / ell);
  S.env.clear();
  GemmList g1, g2;
  std::vector<std::pair<ObsList, ObsList>> le, re;
  for (int k = 0; k + 1 < ell; ++k) {
    obs_left_map(S, d, k, nullptr, S.scale, OB_EL, S.eoff[k], OB_EL, S.eoff[k + 1], g1, g2);
    le.push_back({S.env.add(g1), S.env.add(g2)});
  }
  for (int k = ell - 1; k >= 1; --k) {
    obs_right_map(S, d, k, S.scale, OB_ER, S.eoff[k + 1], OB_ER, S.eoff[k], g1, g2);
    re.push_back({S.env.add(g1), S.env.add(g2)});
  }
  OBS_TRY(obs_upload(c, S.env));
  for (const auto &pr : le) {
    OBS_TRY(obs_run(c, S.env, pr.first));
    OBS_TRY(obs_run(c, S.env, pr.second));
  }
  for (const auto &pr : re) {
    OBS_TRY(obs_run(c, S.env, pr.first));
    OBS_TRY(obs_run(c, S.env, pr.second));
  }
  S.fixed = true;
  return IDMRG_OK;
}

constexpr double OBS_TOL = 1e-12;
constexpr int OBS_MAXIT = 5000;

// Two-point functions: one walk per distinct first site and term.  The left
// environment at site i's bond takes O^a_i, then every later site an identity
// step; at each requested j a branch applies O^b_j and closes with r_{j+1}.
idmrg_status obs_correlation(idmrg_ctx *c, int nterms, const double *opa, const double *opb, const double *coef,
                             int npairs, const int64_t *si, const int64_t *sj, double *out) {
  OBS_TRY(obs_fixed(c, OBS_TOL, OBS_MAXIT));
  ObsState &S = c->obs;
  const int ell = c->ell, d = c->d;
  std::map<int64_t, std::vector<int64_t>> groups;  // i -> sorted distinct j
  for (int k = 0; k < npairs; ++k) groups[si[k]].push_back(sj[k]);
  std::map<std::pair<int64_t, int64_t>, int> slot;  // (i, j) -> result slot
  for (auto &g : groups) {
    std::sort(g.second.begin(), g.second.end());
    g.second.erase(std::unique(g.second.begin(), g.second.end()), g.second.end());
    for (int64_t j : g.second) slot.emplace(std::make_pair(g.first, j), (int)slot.size());
  }
  NOMEM(c->ensure(S.res, 8 * std::max<size_t>(slot.size(), 64)));
  // operations: a map (two lists) or a closing dot
  struct Op {
    int kind;  // 0 map, 1 dot
    ObsList a, b;
    int x_buf, slot;
    int64_t r_off, n;
    double coef;
  };
  std::vector<Op> ops;
  S.walk.clear();
  GemmList g1, g2;
  std::map<std::tuple<int, int, int>, std::pair<ObsList, ObsList>> idmaps;  // (site, in, out)
  auto unit_pos = [&](int64_t x) { return (int)(((x - S.s0) % ell + ell) % ell); };
  auto push_map = [&](int k, const double *O, int in_buf, int64_t in_off, int out_buf) {
    Op o{};
    o.kind = 0;
    if (!O && in_buf != OB_EL) {
      auto key = std::make_tuple(k, in_buf, out_buf);
      auto it = idmaps.find(key);
      if (it == idmaps.end()) {
        obs_left_map(S, d, k, nullptr, S.scale, in_buf, in_off, out_buf, 0, g1, g2);
        it = idmaps.emplace(key, std::make_pair(S.walk.add(g1), S.walk.add(g2))).first;
      }
      o.a = it->second.first;
      o.b = it->second.second;
    } else {
      obs_left_map(S, d, k, O, S.scale, in_buf, in_off, out_buf, 0, g1, g2);
      o.a = S.walk.add(g1);
      o.b = S.walk.add(g2);
    }
    ops.push_back(o);
  };
  const int XM = OB_X0 + 6;  // measurement branch
  for (const auto &g : groups) {
    const int64_t i = g.first;
    const std::vector<int64_t> &js = g.second;
    for (int t = 0; t < nterms; ++t) {
      const double *Oa = opa + (size_t)t * d * d, *Ob = opb + (size_t)t * d * d;
      int cur = OB_X0, other = OB_X0 + 1;
      const int ki = unit_pos(i);
      push_map(ki, Oa, OB_EL, S.eoff[ki], cur);
      size_t next = 0;
      for (int64_t x = i + 1; x <= js.back(); ++x) {
        const int kx = unit_pos(x);
        if (js[next] == x) {
          push_map(kx, Ob, cur, 0, XM);
          Op o{};
          o.kind = 1;
          o.x_buf = XM;
          o.r_off = S.eoff[kx + 1];
          o.n = (int64_t)S.D[kx + 1] * S.D[kx + 1];
          o.slot = slot[{i, x}];
          o.coef = coef[t];
          ops.push_back(o);
          ++next;
        }
        if (x < js.back()) {
          push_map(kx, nullptr, cur, 0, other);
          std::swap(cur, other);
        }
      }
    }
  }
  OBS_TRY(obs_upload(c, S.walk));
  CK(cudaMemsetAsync(S.res.p, 0, 8 * slot.size(), c->st));
  const double *ER = (const double *)S.envr.p;
  for (const Op &o : ops) {
    if (o.kind == 0) {
      OBS_TRY(obs_run(c, S.walk, o.a));
      OBS_TRY(obs_run(c, S.walk, o.b));
    } else {
      OBS_TRY(obs_dot(c, obs_x(c, o.x_buf - OB_X0), ER + o.r_off, o.n, o.coef, o.slot, 1));
    }
  }
  std::vector<double> h(slot.size());
  if (!h.empty()) OBS_TRY(obs_read(c, h.data(), (int)h.size()));
  for (int k = 0; k < npairs; ++k) out[k] = h[slot[{si[k], sj[k]}]];
  return IDMRG_OK;
}

// |t2| / t1 of the unit's transfer map: finite-m truncation splits SU(2)
// multiplets across the charge-difference sectors by small amounts, so each
// sector (differences 0, 1 and 2 steps of the smallest one present at bond 0)
// is iterated on its own (mode 1 of obs_subspace) and the largest modulus
// over the sectors is taken.
idmrg_status obs_spectrum(idmrg_ctx *c, double tol, int maxit, double *ratio, int *iters) {
  OBS_TRY(obs_fixed(c, OBS_TOL, OBS_MAXIT));
  const std::vector<int> &q = c->obs.q0;
  std::vector<int> diffs;
  for (int a : q)
    for (int b : q)
      if (a > b) diffs.push_back(a - b);
  int step = 0;
  for (int x : diffs) step = step == 0 ? x : std::min(step, x);
  idmrg_status worst = IDMRG_OK;
  *ratio = 0.0;
  *iters = 0;
  for (int k = 0; k < 3; ++k) {
    const int delta = k * step;
    if (k > 0 && (step == 0 || std::find(diffs.begin(), diffs.end(), delta) == diffs.end())) continue;
    double r = 0.0;
    int it = 0;
    const idmrg_status s = obs_subspace(c, true, delta, 1, tol, maxit, &r, &it, nullptr);
    if (s != IDMRG_OK && s != IDMRG_ENOCONV) return s;
    if (s == IDMRG_ENOCONV) worst = s;
    *ratio = std::max(*ratio, r);
    *iters += it;
  }
  return worst;
}

}  // namespace

// ==========================================================================
// C ABI
// ==========================================================================
// checkpoint file helpers (idmrg_save / idmrg_load)
namespace {
constexpr char CK_MAGIC[8] = {'I', 'D', 'M', 'R', 'G', 'C', 'K', '1'};

struct CkFile {
  FILE *f = nullptr;
  bool ok = true;
  ~CkFile() {
    if (f) fclose(f);
  }
  template <class T>
  void put(const T &v) {
    ok = ok && fwrite(&v, sizeof(T), 1, f) == 1;
  }
  template <class T>
  void putv(const std::vector<T> &v) {
    put((int64_t)v.size());
    if (!v.empty()) ok = ok && fwrite(v.data(), sizeof(T), v.size(), f) == v.size();
  }
  template <class T>
  void get(T &v) {
    ok = ok && fread(&v, sizeof(T), 1, f) == 1;
  }
  template <class T>
  void getv(std::vector<T> &v, int64_t cap = (int64_t)1 << 40) {
    int64_t n = 0;
    get(n);
    if (!ok || n < 0 || n > cap) {
      ok = false;
      return;
    }
    v.resize((size_t)n);
    if (n > 0) ok = ok && fread(v.data(), sizeof(T), (size_t)n, f) == (size_t)n;
  }
};

void ck_put_basis(CkFile &F, const Basis &b) {
  F.putv(b.q);
  F.putv(b.dim);
}
void ck_get_basis(CkFile &F, Basis &b) {
  b.clear();
  F.getv(b.q);
  F.getv(b.dim);
  if (b.q.size() != b.dim.size()) F.ok = false;
  b.finish();
}
void ck_put_sec(CkFile &F, const SecInfo &si) {
  F.put(si.Q);
  F.put(si.k);
  F.put(si.r);
  F.put(si.c);
  F.put(si.job);
  F.put(si.u_off);
  F.put(si.v_off);
  F.put(si.lam_off);
  F.putv(si.rg);
  F.putv(si.cg);
}
void ck_get_sec(CkFile &F, SecInfo &si) {
  F.get(si.Q);
  F.get(si.k);
  F.get(si.r);
  F.get(si.c);
  F.get(si.job);
  F.get(si.u_off);
  F.get(si.v_off);
  F.get(si.lam_off);
  F.getv(si.rg);
  F.getv(si.cg);
}
}  // namespace

idmrg_status ck_put_dev(idmrg_ctx *c, CkFile &F, const DevBuf &b, int64_t n) {
  std::vector<double> h((size_t)std::max<int64_t>(n, 0));
  if (n > 0) CK(cudaMemcpy(h.data(), b.p, 8 * (size_t)n, cudaMemcpyDeviceToHost));
  F.putv(h);
  return IDMRG_OK;
}

idmrg_status ck_get_dev(idmrg_ctx *c, CkFile &F, DevBuf &b, int64_t n) {
  std::vector<double> h;
  F.getv(h, n);
  if (!F.ok || (int64_t)h.size() != n) return c->fail(IDMRG_EINVAL, "load: checkpoint truncated or inconsistent");
  NOMEM(c->ensure(b, 8 * (size_t)std::max<int64_t>(n, 1)));
  if (n > 0) CK(cudaMemcpy(b.p, h.data(), 8 * (size_t)n, cudaMemcpyHostToDevice));
  return IDMRG_OK;
}

namespace {
// one truncation record (bases, sector tables, lambda, U and V)
idmrg_status ck_put_trunc_dev(idmrg_ctx *c, CkFile &F, const TruncRec &T) {
  F.put((int)T.valid);
  ck_put_basis(F, T.leftB);
  ck_put_basis(F, T.rightB);
  ck_put_basis(F, T.bU);
  ck_put_basis(F, T.bV);
  F.put((int64_t)T.sec.size());
  for (const SecInfo &si : T.sec) ck_put_sec(F, si);
  F.putv(T.lam);
  F.putv(T.lam_all);
  F.put(T.eps);
  F.put(T.eps_best);
  F.put(T.usize);
  F.put(T.vsize);
  idmrg_status s = ck_put_dev(c, F, T.U, T.valid ? T.usize : 0);
  if (s != IDMRG_OK) return s;
  return ck_put_dev(c, F, T.V, T.valid ? T.vsize : 0);
}

idmrg_status ck_get_trunc(idmrg_ctx *c, CkFile &F, TruncRec &T) {
  const DevBuf keepU = T.U, keepV = T.V;  // device buffers are recycled
  T = TruncRec();
  T.U = keepU;
  T.V = keepV;
  int valid = 0;
  F.get(valid);
  T.valid = valid != 0;
  ck_get_basis(F, T.leftB);
  ck_get_basis(F, T.rightB);
  ck_get_basis(F, T.bU);
  ck_get_basis(F, T.bV);
  int64_t ns = 0;
  F.get(ns);
  if (!F.ok || ns < 0 || ns > (1 << 20)) return c->fail(IDMRG_EINVAL, "truncation record damaged");
  T.sec.resize((size_t)ns);
  for (SecInfo &si : T.sec) ck_get_sec(F, si);
  F.getv(T.lam);
  F.getv(T.lam_all);
  F.get(T.eps);
  F.get(T.eps_best);
  F.get(T.usize);
  F.get(T.vsize);
  if (!F.ok) return c->fail(IDMRG_EINVAL, "truncation record truncated");
  idmrg_status s = ck_get_dev(c, F, T.U, T.valid ? T.usize : 0);
  if (s != IDMRG_OK) return s;
  return ck_get_dev(c, F, T.V, T.valid ? T.vsize : 0);
}
}  // namespace

extern "C" {

void idmrg_default_opts(idmrg_opts *o) {
  if (!o) return;
  o->m = 64;
  o->target_charge = 0;
  o->lanczos_tol = 1e-12;
  o->lanczos_maxit = 300;
  o->prec = IDMRG_FP64;
  o->predict = 1;
  o->seed = 0;
  o->lambda_zero_rel = 1e-12;
  o->tie_rel = 1e-7;
}

idmrg_status idmrg_create(const idmrg_mpo *mpo, const idmrg_opts *opts, void *cuda_stream,
                          const idmrg_allocator *alloc, idmrg_ctx **out) {
  return idmrg_create_batch(mpo, 1, nullptr, opts, cuda_stream, alloc, out);
}

idmrg_status idmrg_create_batch(const idmrg_mpo *mpos, int nmpo, const int *m_per, const idmrg_opts *opts,
                                void *cuda_stream, const idmrg_allocator *alloc, idmrg_ctx **out) {
  if (!mpos || nmpo < 1 || !opts || !out) return IDMRG_EINVAL;
  *out = nullptr;
  idmrg_ctx *c = new idmrg_ctx();
  auto bail = [&](idmrg_status s) {
    // the ABI returns no context on failure: free everything
    idmrg_destroy(c);
    return s;
  };
  c->o = *opts;
  c->st = (cudaStream_t)cuda_stream;
  if (alloc && alloc->alloc && alloc->free) {
    c->alloc = *alloc;
    c->own_alloc = false;
  }
  const int d = mpos[0].d;
  if (d < 1 || d > 4 || !mpos[0].phys_charge) return bail(IDMRG_EINVAL);
  for (int r = 0; r < nmpo; ++r) {
    const idmrg_mpo &M = mpos[r];
    if (M.ell < 2 || M.ell % 2 || M.d != d || !M.bond_dim || !M.W || !M.phys_charge || !M.bond_charge)
      return bail(IDMRG_EINVAL);
    for (int s = 0; s < d; ++s)
      if (M.phys_charge[s] != mpos[0].phys_charge[s]) return bail(IDMRG_EINVAL);  // one local basis
    if (m_per && m_per[r] < 1) return bail(IDMRG_EINVAL);
  }
  if (opts->m < 1 || opts->lanczos_maxit < 2 || opts->lanczos_maxit > 600 || !(opts->lanczos_tol > 0))
    return bail(IDMRG_EINVAL);
  if (opts->prec != IDMRG_FP64 && opts->prec != IDMRG_TF32X3 && opts->prec != IDMRG_BF16X3 &&
      opts->prec != IDMRG_FP64_TC)
    return bail(IDMRG_EINVAL);
  c->mixed = opts->prec == IDMRG_TF32X3 || opts->prec == IDMRG_BF16X3;
  c->fp64tc = opts->prec == IDMRG_FP64_TC;
  for (GemmTune *t : {&c->tn_gp, &c->tn_env1, &c->tn_env3, &c->tn_svdG, &c->tn_svdW, &c->tn_svdX}) t->oz_use = true;
  c->bf16 = opts->prec == IDMRG_BF16X3 ? 1 : 0;
  c->inner_factor = c->bf16 ? 1e-2 : 1e-3;
  c->d = d;
  c->ell = mpos[0].ell;
  // rings: superblocks and sites numbered problem after problem
  int nsb = 0, nsite = 0, mmax = 0;
  for (int r = 0; r < nmpo; ++r) {
    idmrg_ctx::Ring R;
    R.p0 = nsb;
    R.np = mpos[r].ell / 2;
    R.s0 = nsite;
    R.ell = mpos[r].ell;
    R.m = m_per ? m_per[r] : opts->m;
    mmax = std::max(mmax, R.m);
    nsb += R.np;
    nsite += R.ell;
    c->rings.push_back(R);
  }
  c->o.m = mmax;  // the largest m: strides of the per-superblock lambda arrays
  c->P = nsb;
  c->own0 = 0;
  c->own1 = c->P;
  c->ring_of.resize(nsb);
  c->ring_of_site.resize(nsite);
  for (int r = 0; r < nmpo; ++r) {
    const idmrg_ctx::Ring &R = c->rings[r];
    for (int q = 0; q < R.np; ++q) c->ring_of[R.p0 + q] = r;
    for (int k = 0; k < R.ell; ++k) c->ring_of_site[R.s0 + k] = r;
  }
  c->qp.assign(mpos[0].phys_charge, mpos[0].phys_charge + d);
  for (int s = 0; s < d; ++s)
    for (int t = s + 1; t < d; ++t)
      if (c->qp[s] == c->qp[t]) return bail(IDMRG_EINVAL);  // one state per physical charge
  c->adim.resize(nsite);
  c->W.resize(nsite);
  c->bq.resize(nsite);
  for (int r = 0; r < nmpo; ++r) {
    const idmrg_mpo &M = mpos[r];
    const int ell = M.ell, s0 = c->rings[r].s0;
    if (M.bond_dim[ell] != M.bond_dim[0]) return bail(IDMRG_EINVAL);
    for (int k = 0; k <= ell; ++k)
      if (M.bond_dim[k] < 2) return bail(IDMRG_EINVAL);
    size_t woff = 0, qoff = 0;
    for (int k = 0; k < ell; ++k) {
      c->adim[s0 + k] = M.bond_dim[k];
      const size_t n = (size_t)M.bond_dim[k] * M.bond_dim[k + 1] * d * d;
      c->W[s0 + k].assign(M.W + woff, M.W + woff + n);
      woff += n;
      c->bq[s0 + k].assign(M.bond_charge + qoff, M.bond_charge + qoff + M.bond_dim[k]);
      qoff += M.bond_dim[k];
    }
  }
  // lower-triangular FSA form and charge conservation (Sec. 2, Eq. mpo)
  for (int k = 0; k < nsite; ++k) {
    const int kb = c->bond_right(k);
    const int A = c->adim[k], B = c->adim[kb];
    const std::vector<int> &qa = c->bq[k], &qb = c->bq[kb];
    for (int a = 0; a < A; ++a)
      for (int b = 0; b < B; ++b)
        for (int s = 0; s < d; ++s)
          for (int t = 0; t < d; ++t) {
            const double w = c->Wat(k, a, b, s, t);
            const double id = (s == t) ? 1.0 : 0.0;
            if ((a == 0 && b == 0) || (a == A - 1 && b == B - 1)) {
              if (w != id) { c->fail(IDMRG_EINVAL, "W_%d: corner channels must be the identity", k); return bail(IDMRG_EINVAL); }
              continue;
            }
            if (w == 0.0) continue;
            if (a == 0 || b == B - 1) return bail(IDMRG_EINVAL);
            if (c->qp[s] - c->qp[t] != qb[b] - qa[a]) return bail(IDMRG_EINVAL);
          }
  }
  {
    std::vector<int> msb(nsb);
    for (int q = 0; q < nsb; ++q) msb[q] = c->rings[c->ring_of[q]].m;
    if (!c->upload(c->dmsb, msb)) return bail(IDMRG_ENOMEM);
  }
  const int P = c->P;
  c->stage.assign(P, ST_READY);
  c->envL.resize(P);
  c->envR.resize(P);
  c->newL.resize(P);
  c->newR.resize(P);
  c->cur.resize(P);
  c->prev.resize(P);
  c->prev2.resize(P);
  c->energy.assign(P, NAN);
  c->fidelity.assign(P, NAN);
  c->bond.assign(P, NAN);
  c->startnorm.assign(P, NAN);
  c->iters.assign(P, 0);
  c->conv.assign(P, 0);
  c->bT1.resize(P);
  c->bT3.resize(P);
  c->bX.resize(P);
  c->bY.resize(P);
  c->bV.resize(P);
  c->bW.resize(P);
  c->bPsi.resize(P);
  c->bUT.resize(P);
  c->bVT.resize(P);
  c->bStart.resize(P);
  for (auto *v : {&c->bPA1, &c->bPB1, &c->bT1F, &c->bPA3, &c->bPB3, &c->bRMAP, &c->bOA1, &c->bOB1, &c->bOT1,
                  &c->bOA3, &c->bOB3, &c->bORMAP, &c->bOT3})
    v->resize(P);
  c->hbufs.assign((size_t)P * NBUF, nullptr);
  if (!c->ensure(c->derr, 256)) return bail(IDMRG_ENOMEM);
  if (cudaMemsetAsync(c->derr.p, 0, sizeof(int), c->st) != cudaSuccess) return bail(IDMRG_ECUDA);
  // Step 1: L^(0) of pair p = last row of W at site 2p, R^(0) = first column of W at 2p+1
  for (int p = 0; p < P; ++p) {
    Basis b;
    for (int s = 0; s < d; ++s) b.add(c->qp[s], 1);
    b.finish();
    const int sL = 2 * p, sR = 2 * p + 1;
    Env &L = c->envL[p];
    L.lay.build(b, c->bq[c->bond_right(sL)]);
    std::vector<double> hl(L.lay.size, 0.0);
    for (int a = 0; a < L.lay.w; ++a)
      for (int si = 0; si < d; ++si) {
        const int so = L.lay.so[a * d + si];
        if (so >= 0) hl[L.lay.off[a * d + si]] = c->Wat(sL, c->adim[sL] - 1, a, so, si);
      }
    std::vector<int> rq(c->adim[sR]);
    for (int a = 0; a < c->adim[sR]; ++a) rq[a] = -c->bq[sR][a];
    Env &R = c->envR[p];
    R.lay.build(b, rq);
    std::vector<double> hr(R.lay.size, 0.0);
    for (int a = 0; a < R.lay.w; ++a)
      for (int si = 0; si < d; ++si) {
        const int so = R.lay.so[a * d + si];
        if (so >= 0) hr[R.lay.off[a * d + si]] = c->Wat(sR, a, 0, so, si);
      }
    if (!c->upload(L.data, hl) || !c->upload(R.data, hr)) return bail(IDMRG_ENOMEM);
  }
  c->n = 1;
  for (idmrg_ctx::Ring &R : c->rings) R.e1[-1] = 0.0;
  if (plan_iteration(c) != IDMRG_OK) return bail(IDMRG_ENOMEM);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return bail(IDMRG_ECUDA);
  *out = c;
  return IDMRG_OK;
}

void idmrg_destroy(idmrg_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  auto rel = [&](DevBuf &b) { c->release(b); };
  for (auto &e : c->envL) rel(e.data);
  for (auto &e : c->envR) rel(e.data);
  for (auto &e : c->newL) rel(e.data);
  for (auto &e : c->newR) rel(e.data);
  for (auto *v : {&c->cur, &c->prev, &c->prev2})
    for (auto &t : *v) { rel(t.U); rel(t.V); }
  for (auto *v : {&c->bT1, &c->bT3, &c->bX, &c->bY, &c->bV, &c->bW, &c->bPsi, &c->bUT, &c->bVT, &c->bStart, &c->bPA1,
                  &c->bPB1, &c->bT1F, &c->bPA3, &c->bPB3, &c->bRMAP, &c->bOA1, &c->bOB1, &c->bOT1, &c->bOA3,
                  &c->bOB3, &c->bORMAP, &c->bOT3})
    for (auto &b : *v) rel(b);
  for (DevBuf *b : {&c->dbufs, &c->dg1k, &c->dg1s, &c->dg3k, &c->dg3s, &c->dwt, &c->dwm, &c->ddt,
                    &c->ddp, &c->drb, &c->dgpk, &c->dgps, &c->dst, &c->dstab, &c->dge1k,
                    &c->dge1s, &c->dge3k, &c->dge3s, &c->dwet, &c->dwem, &c->dmask, &c->derr, &c->lN,
                    &c->lV, &c->lw, &c->lalpha, &c->lbeta, &c->libeta, &c->lh, &c->lpart, &c->lk, &c->lmember, &c->lactive,
                    &c->lconv, &c->ltheta, &c->ly, &c->lresid, &c->lpsi, &c->lv0, &c->ldot, &c->sjobs, &c->swork,
                    &c->ssv, &c->sjob0, &c->snjob, &c->skpj, &c->sperm, &c->slam, &c->seps, &c->sepsb, &c->skept,
                    &c->scj, &c->slamk, &c->siw, &c->sorder, &c->sorderq, &c->dsgk, &c->dsgs,
                    &c->dswk, &c->dsws, &c->dsxk, &c->dsxs, &c->dpkL, &c->dtune_out, &c->dmsb,
                    &c->dwtp, &c->dwtpm, &c->dwunits, &c->dtarget, &c->dozsw, &c->dozsp, &c->dozp,
                    &c->doz1k,
                    &c->doz1t, &c->doz3k, &c->doz3t, &c->dozw, &c->dozwm, &c->oexp, &c->goz_planes,
                    &c->goz_exps})
    rel(*b);
  for (int k = 0; k < MIX_NTN; ++k)
    for (DevBuf *b : {&c->dpkp[k], &c->dpkR[k], &c->dtc1k[k], &c->dtc1t[k], &c->dtc3k[k], &c->dtc3t[k]}) rel(*b);
  for (auto *t : {&c->tt1, &c->tt3})
    for (int k = 0; k < MIX_NTN; ++k) {
      if (t->e0[k]) cudaEventDestroy(t->e0[k]);
      if (t->e1[k]) cudaEventDestroy(t->e1[k]);
    }
  {
    ObsState &S = c->obs;
    for (DevBuf *b : {&S.A, &S.Y, &S.envl, &S.envr, &S.res, &S.tab, &S.emb, &S.scal, &S.dq0, &S.unit.dtasks, &S.unit.dsegs,
                      &S.unit.dtiles, &S.env.dtasks, &S.env.dsegs, &S.env.dtiles, &S.walk.dtasks, &S.walk.dsegs,
                      &S.walk.dtiles})
      rel(*b);
    for (auto &x : S.X) rel(x);
  }
  for (int k = 0; k < idmrg_ctx::KT_ALL; ++k) c->collapse(k);
  for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
  for (cudaStream_t x : c->side)
    if (x) cudaStreamDestroy(x);
  if (c->pin_act) cudaFreeHost(c->pin_act);
  for (GemmTune *t : {&c->tn_g1, &c->tn_g3, &c->tn_gp, &c->tn_env1, &c->tn_env3, &c->tn_svdG, &c->tn_svdW, &c->tn_svdX}) {
    for (auto &b : t->tiles) rel(b);
    rel(t->oz.dsegs);
    rel(t->oz.dtasks);
    rel(t->oz.dtiles);
    for (int k = 0; k < GEMM_NSHAPE; ++k) {
      if (t->e0[k]) cudaEventDestroy(t->e0[k]);
      if (t->e1[k]) cudaEventDestroy(t->e1[k]);
    }
  }
  for (cudaEvent_t e : c->ev_act)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : c->sev)
    if (e) cudaEventDestroy(e);
  delete c;
}

const char *idmrg_last_error(const idmrg_ctx *c) { return c ? c->err.c_str() : "null context"; }

idmrg_status idmrg_set_stream(idmrg_ctx *c, void *s) {
  if (!c) return IDMRG_EINVAL;
  c->st = (cudaStream_t)s;
  return IDMRG_OK;
}

idmrg_status idmrg_iteration(const idmrg_ctx *c, int *n) {
  if (!c || !n) return IDMRG_EINVAL;
  *n = c->n;
  return IDMRG_OK;
}

idmrg_status idmrg_psi_layout(const idmrg_ctx *cc, int p, int *desc, int cap, int *nblocks, size_t *nelem) {
  idmrg_ctx *c = const_cast<idmrg_ctx *>(cc);
  if (!c || p < 0 || p >= c->P) return IDMRG_EINVAL;
  const PsiLayout &psi = c->plan[p].psi;
  const Basis &BL = c->envL[p].lay.b, &BR = c->envR[c->nxt(p)].lay.b;
  int nb = 0;
  for (int i = 0; i < BL.S(); ++i)
    for (int s = 0; s < c->d; ++s)
      for (int t = 0; t < c->d; ++t) {
        const int k = psi.sub(i, s, t);
        const int j = psi.sj[k];
        if (j < 0) continue;
        if (desc && nb < cap) {
          int *e = desc + 8 * nb;
          e[0] = BL.off[i];
          e[1] = BL.dim[i];
          e[2] = s;
          e[3] = t;
          e[4] = BR.off[j];
          e[5] = BR.dim[j];
          e[6] = (int)(psi.roff[i] + psi.scol[k]);
          e[7] = psi.C[i];
        }
        ++nb;
      }
  if (nblocks) *nblocks = nb;
  if (nelem) *nelem = (size_t)psi.N;
  return IDMRG_OK;
}

idmrg_status idmrg_block_basis(const idmrg_ctx *c, int p, int side, int *charges, int cap, int *dim, int *channels) {
  if (!c || p < 0 || p >= c->P || (side != 0 && side != 1)) return IDMRG_EINVAL;
  const Env &E = side == 0 ? c->envL[p] : c->envR[c->nxt(p)];
  const Basis &b = E.lay.b;
  if (charges) {
    int k = 0;
    for (int i = 0; i < b.S(); ++i)
      for (int x = 0; x < b.dim[i]; ++x)
        if (k < cap) charges[k++] = b.q[i];
  }
  if (dim) *dim = b.D;
  if (channels) *channels = E.lay.w;
  return IDMRG_OK;
}

idmrg_status idmrg_block_to_host(const idmrg_ctx *cc, int p, int side, double *host, size_t cap) {
  idmrg_ctx *c = const_cast<idmrg_ctx *>(cc);
  if (!c || !host || p < 0 || p >= c->P || (side != 0 && side != 1)) return IDMRG_EINVAL;
  const Env &E = side == 0 ? c->envL[p] : c->envR[c->nxt(p)];
  const Basis &b = E.lay.b;
  const size_t D = b.D;
  if (cap < (size_t)E.lay.w * D * D) return c->fail(IDMRG_EINVAL, "block_to_host: buffer too small");
  std::vector<double> blocks(E.lay.size);
  CK(cudaStreamSynchronize(c->st));
  CK(cudaMemcpy(blocks.data(), E.data.p, 8 * blocks.size(), cudaMemcpyDeviceToHost));
  memset(host, 0, sizeof(double) * E.lay.w * D * D);
  const int S = b.S();
  for (int a = 0; a < E.lay.w; ++a)
    for (int si = 0; si < S; ++si) {
      const int so = E.lay.so[a * S + si];
      if (so < 0) continue;
      const double *blk = blocks.data() + E.lay.off[a * S + si];
      for (int x = 0; x < b.dim[so]; ++x)
        for (int y = 0; y < b.dim[si]; ++y)
          host[((size_t)a * D + b.off[so] + x) * D + b.off[si] + y] = blk[(size_t)x * b.dim[si] + y];
    }
  return IDMRG_OK;
}

// form -1: the context's own arithmetic; 0: FP64 GEMMs; 1: digit slices
static idmrg_status heff_apply_form(idmrg_ctx *c, int p, const double *psi_dev, double *out_dev, int form) {
  if (!c || !psi_dev || !out_dev) return IDMRG_EINVAL;
  if (check_p(c, p) != IDMRG_OK) return IDMRG_EINVAL;
  if (form == 1 && !c->oz_ok) return c->fail(IDMRG_EINVAL, "digit-slice form not available");
  std::vector<int> mask(c->P, 0);
  int64_t off = 0;
  std::vector<double *> save_in(c->P), save_out(c->P);
  for (int q = 0; q < c->P; ++q) {
    save_in[q] = c->hbufs[q * NBUF + BUF_IN];
    save_out[q] = c->hbufs[q * NBUF + BUF_OUT];
    if (!want(c, p, q)) continue;
    mask[q] = 1;
    c->hbufs[q * NBUF + BUF_IN] = const_cast<double *>(psi_dev) + off;
    c->hbufs[q * NBUF + BUF_OUT] = out_dev + off;
    if (p < 0) off += c->plan[q].psi.N;
  }
  NOMEM(c->upload(c->dmask, mask));
  NOMEM(sync_bufs(c) == IDMRG_OK);
  const bool keep_oz = c->o_oz;
  if (form >= 0) c->o_oz = form == 1;
  idmrg_status s = heff_launch(c, (const int *)c->dmask.p, mask.data(), form >= 0);
  c->o_oz = keep_oz;
  for (int q = 0; q < c->P; ++q) {
    c->hbufs[q * NBUF + BUF_IN] = save_in[q];
    c->hbufs[q * NBUF + BUF_OUT] = save_out[q];
  }
  return s;
}

idmrg_status idmrg_heff_apply(idmrg_ctx *c, int p, const double *psi_dev, double *out_dev) {
  return heff_apply_form(c, p, psi_dev, out_dev, -1);
}

idmrg_status idmrg_heff_apply_fp64(idmrg_ctx *c, int p, const double *psi_dev, double *out_dev, int form) {
  if (form != 0 && form != 1) return IDMRG_EINVAL;
  return heff_apply_form(c, p, psi_dev, out_dev, form);
}

idmrg_status idmrg_predict_wavefunction(idmrg_ctx *c, int p, double *norm_out) {
  if (!c) return IDMRG_EINVAL;
  if (check_p(c, p) != IDMRG_OK) return IDMRG_EINVAL;
  idmrg_status s = predict(c, p);
  if (s != IDMRG_OK || !norm_out) return s;
  // ||psi~|| on request: one device reduction per requested superblock
  const int P = c->P;
  std::vector<int64_t> N(P);
  std::vector<double *> x(P);
  std::vector<int> mask(P);
  int64_t nmax = 1;
  for (int q = 0; q < P; ++q) {
    N[q] = c->plan[q].psi.N;
    x[q] = c->dp(c->bPsi[q]);
    mask[q] = want(c, p, q) ? 1 : 0;
    nmax = std::max(nmax, N[q]);
  }
  const int nchunk = (int)((nmax + norm_chunk() - 1) / norm_chunk());
  NOMEM(c->upload(c->lN, N) && c->upload(c->lpsi, x) && c->upload(c->lmember, mask) &&
        c->ensure(c->lpart, 8 * (size_t)P * nchunk) && c->ensure(c->lresid, 8 * (size_t)P));
  CK(launch_norms((const int64_t *)c->lN.p, P, (const double *const *)c->lpsi.p, (const int *)c->lmember.p,
                  c->dp(c->lpart), nchunk, c->dp(c->lresid), c->st));
  c->launches += 2;
  std::vector<double> nr(P);
  CK(c->d2h_copy(nr.data(), c->lresid.p, 8 * (size_t)P));
  CK(cudaStreamSynchronize(c->st));
  int k = 0;
  for (int q = 0; q < P; ++q)
    if (want(c, p, q)) norm_out[k++] = nr[q];
  return IDMRG_OK;
}

idmrg_status idmrg_set_start_vector(idmrg_ctx *c, int p, const double *psi_dev) {
  if (!c || !psi_dev) return IDMRG_EINVAL;
  if (check_p(c, p) != IDMRG_OK) return IDMRG_EINVAL;
  for (int q = 0; q < c->P; ++q)
    if (want(c, p, q) && c->stage[q] != ST_READY && c->stage[q] != ST_STARTED)
      return c->fail(IDMRG_ESTATE, "set_start_vector: superblock %d already past its start", q);
  int64_t off = 0;
  for (int q = 0; q < c->P; ++q) {
    if (!want(c, p, q)) continue;
    const int64_t N = c->plan[q].psi.N;
    if (N > 0) CK(cudaMemcpyAsync(c->bPsi[q].p, psi_dev + off, 8 * (size_t)N, cudaMemcpyDeviceToDevice, c->st));
    off += N;
    c->stage[q] = ST_STARTED;
  }
  return IDMRG_OK;
}

idmrg_status idmrg_lanczos_solve(idmrg_ctx *c, int p, double *e_out, int *iters_out) {
  if (!c) return IDMRG_EINVAL;
  if (check_p(c, p) != IDMRG_OK) return IDMRG_EINVAL;
  idmrg_status s = lanczos(c, p);
  if (s != IDMRG_OK && s != IDMRG_ENOCONV) return s;
  int k = 0;
  for (int q = 0; q < c->P; ++q) {
    if (!want(c, p, q)) continue;
    if (e_out) e_out[k] = c->energy[q];
    if (iters_out) iters_out[k] = c->iters[q];
    ++k;
  }
  return s;
}

idmrg_status idmrg_get_psi(const idmrg_ctx *cc, int p, double *host, size_t cap) {
  idmrg_ctx *c = const_cast<idmrg_ctx *>(cc);
  if (!c || !host || p < 0 || p >= c->P) return IDMRG_EINVAL;
  if (c->stage[p] < ST_SOLVED) return c->fail(IDMRG_ESTATE, "get_psi: superblock %d not solved", p);
  const size_t N = c->plan[p].psi.N;
  if (cap < N) return c->fail(IDMRG_EINVAL, "get_psi: buffer too small");
  CK(cudaStreamSynchronize(c->st));
  CK(cudaMemcpy(host, c->bPsi[p].p, 8 * N, cudaMemcpyDeviceToHost));
  return IDMRG_OK;
}

idmrg_status idmrg_truncate(idmrg_ctx *c, int p, double *eps_out, double *eps_best_out, int *kept_out) {
  if (!c) return IDMRG_EINVAL;
  if (check_p(c, p) != IDMRG_OK) return IDMRG_EINVAL;
  idmrg_status s = truncate(c, p);
  if (s != IDMRG_OK) return s;
  int k = 0;
  for (int q = 0; q < c->P; ++q) {
    if (!want(c, p, q)) continue;
    if (eps_out) eps_out[k] = c->cur[q].eps;
    if (eps_best_out) eps_best_out[k] = c->cur[q].eps_best;
    if (kept_out) kept_out[k] = c->cur[q].bU.D;
    ++k;
  }
  return IDMRG_OK;
}

idmrg_status idmrg_get_lambda(const idmrg_ctx *c, int p, double *host, int cap, int *len) {
  if (!c || p < 0 || p >= c->P) return IDMRG_EINVAL;
  const TruncRec &T = c->stage[p] >= ST_TRUNCATED ? c->cur[p] : c->prev[p];
  if (!T.valid) return IDMRG_ESTATE;
  const int n = (int)T.lam_all.size();
  if (host)
    for (int i = 0; i < std::min(n, cap); ++i) host[i] = T.lam_all[i];
  if (len) *len = n;
  return IDMRG_OK;
}

idmrg_status idmrg_update_environments(idmrg_ctx *c, int p) {
  if (!c) return IDMRG_EINVAL;
  if (check_p(c, p) != IDMRG_OK) return IDMRG_EINVAL;
  return update_envs(c, p);
}

idmrg_status idmrg_advance(idmrg_ctx *c) {
  if (!c) return IDMRG_EINVAL;
  return advance(c);
}

idmrg_status idmrg_batch_step(idmrg_ctx *const *ctxs, int n, int threads, idmrg_step_report *reps) {
  if (!ctxs || n < 0 || threads < 1) return IDMRG_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i]) return IDMRG_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IDMRG_ECUDA;
  std::vector<idmrg_status> st(n, IDMRG_OK);
  std::atomic<int> next(0);
  auto work = [&]() {
    cudaSetDevice(dev);
    for (int i = next++; i < n; i = next++) st[i] = idmrg_unit_cell_step(ctxs[i], reps ? &reps[i] : nullptr);
  };
  const int nt = std::min(threads, std::max(n, 1));
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(work);
  work();
  for (auto &t : pool) t.join();
  for (int i = 0; i < n; ++i)
    if (st[i] != IDMRG_OK) return st[i];
  return IDMRG_OK;
}

idmrg_status idmrg_unit_cell_step(idmrg_ctx *c, idmrg_step_report *rep) {
  if (!c) return IDMRG_EINVAL;
  if (c->plan_pending) return c->fail(IDMRG_ESTATE, "unit_cell_step: the boundary pair has not been imported");
  for (int q = 0; q < c->P; ++q)
    if (c->owns(q) && c->stage[q] != ST_READY)
      return c->fail(IDMRG_ESTATE, "unit_cell_step: iteration %d already in progress", c->n);
  idmrg_status s = predict(c, -1);
  if (s != IDMRG_OK) return s;
  idmrg_status sl = lanczos(c, -1);
  if (sl != IDMRG_OK && sl != IDMRG_ENOCONV) return sl;
  s = truncate(c, -1);
  if (s != IDMRG_OK) return s;
  s = update_envs(c, -1);
  if (s != IDMRG_OK) return s;
  const int n_done = c->n;
  std::vector<double> eps(c->P), epsb(c->P);
  std::vector<int> kept(c->P);
  for (int q = 0; q < c->P; ++q) {
    eps[q] = c->cur[q].eps;
    epsb[q] = c->cur[q].eps_best;
    kept[q] = c->cur[q].bU.D;
  }
  s = advance(c);
  if (s != IDMRG_OK) return s;
  if (rep) {
    rep->n = n_done;
    for (int q = 0; q < c->P; ++q) {
      if (rep->energy) rep->energy[q] = c->energy[q];
      if (rep->iters) rep->iters[q] = c->iters[q];
      if (rep->eps) rep->eps[q] = eps[q];
      if (rep->eps_best) rep->eps_best[q] = epsb[q];
      if (rep->fidelity) rep->fidelity[q] = c->fidelity[q];
      if (rep->bond) rep->bond[q] = c->bond[q];
      if (rep->kept) rep->kept[q] = kept[q];
    }
    rep->e_g = (c->rings[0].eg_n == n_done) ? c->rings[0].eg_last : NAN;
  }
  return sl;
}

// ------------------------------------------------------------------------
// One problem over several workers (Sec. 3, Step 2'): a context steps a
// contiguous range of pairs; after each step the first pair of the range is
// exported (R^(n) of that pair and its truncation: U^(n), V^(n), lambda^(n),
// bases and sector tables) and imported by the worker whose range ends just
// before it.  The byte layout is the checkpoint's, for one pair.
// ------------------------------------------------------------------------
idmrg_status idmrg_set_pair_range(idmrg_ctx *c, int p0, int p1) {
  if (!c) return IDMRG_EINVAL;
  if (!c->one_ring()) return c->fail(IDMRG_EINVAL, "set_pair_range: needs a context of one problem");
  if (p0 < 0 || p1 > c->P || p0 >= p1) return c->fail(IDMRG_EINVAL, "pair range %d..%d outside 0..%d", p0, p1, c->P);
  for (int q = 0; q < c->P; ++q)
    if (c->stage[q] != ST_READY) return c->fail(IDMRG_ESTATE, "set_pair_range: a step is in progress");
  if (c->plan_pending) return c->fail(IDMRG_ESTATE, "set_pair_range: the boundary pair has not been imported");
  c->own0 = p0;
  c->own1 = p1;
  c->obs.valid = c->obs.fixed = false;
  return IDMRG_OK;
}

idmrg_status idmrg_export_pair(const idmrg_ctx *cc, int q, void *host, size_t cap, size_t *len) {
  idmrg_ctx *c = const_cast<idmrg_ctx *>(cc);
  if (!c || !len || q < 0 || q >= c->P) return IDMRG_EINVAL;
  if (!c->one_ring()) return c->fail(IDMRG_EINVAL, "export_pair: needs a context of one problem");
  if (!c->owns(q)) return c->fail(IDMRG_EINVAL, "export_pair: pair %d is not stepped by this context", q);
  for (int k = 0; k < c->P; ++k)
    if (c->stage[k] != ST_READY) return c->fail(IDMRG_ESTATE, "export_pair: a step is in progress");
  if (!c->prev[q].valid) return c->fail(IDMRG_ESTATE, "export_pair: pair %d has no completed iteration", q);
  CK(cudaStreamSynchronize(c->st));
  char *buf = nullptr;
  size_t n = 0;
  CkFile F;
  F.f = open_memstream(&buf, &n);
  if (!F.f) return c->fail(IDMRG_ENOMEM, "export_pair: no host memory");
  F.put(c->n);
  F.put(q);
  const Env &E = c->envR[q];
  ck_put_basis(F, E.lay.b);
  F.putv(E.lay.chq);
  idmrg_status s = ck_put_dev(c, F, E.data, E.lay.size);
  if (s == IDMRG_OK) s = ck_put_trunc_dev(c, F, c->prev[q]);
  fclose(F.f);
  F.f = nullptr;
  if (s == IDMRG_OK && !F.ok) s = c->fail(IDMRG_ENOMEM, "export_pair: serialisation failed");
  if (s == IDMRG_OK) {
    *len = n;
    if (host && cap >= n) memcpy(host, buf, n);
    else if (host) s = c->fail(IDMRG_EINVAL, "export_pair: %zu bytes needed, %zu given", n, cap);
  }
  free(buf);
  return s;
}

idmrg_status idmrg_import_pair(idmrg_ctx *c, int q, const void *host, size_t len) {
  if (!c || !host || q < 0 || q >= c->P) return IDMRG_EINVAL;
  if (!c->one_ring()) return c->fail(IDMRG_EINVAL, "import_pair: needs a context of one problem");
  if (c->owns(q)) return c->fail(IDMRG_EINVAL, "import_pair: pair %d is stepped by this context", q);
  if (q != c->own1 % c->P) return c->fail(IDMRG_EINVAL, "import_pair: pair %d does not follow this range", q);
  CkFile F;
  F.f = fmemopen(const_cast<void *>(host), len, "rb");
  if (!F.f) return c->fail(IDMRG_EINVAL, "import_pair: cannot read the buffer");
  int n = 0, qq = -1;
  F.get(n);
  F.get(qq);
  if (!F.ok || qq != q || n != c->n)  // both sides have advanced to the next iteration
    return c->fail(IDMRG_EINVAL, "import_pair: data of pair %d for iteration %d, expected pair %d for %d", qq, n, q,
                   c->n);
  Env &E = c->envR[q];
  Basis b;
  std::vector<int> chq;
  ck_get_basis(F, b);
  F.getv(chq, 1 << 20);
  if (!F.ok) return c->fail(IDMRG_EINVAL, "import_pair: data truncated");
  E.lay.build(b, chq);
  idmrg_status s = ck_get_dev(c, F, E.data, E.lay.size);
  if (s != IDMRG_OK) return s;
  s = ck_get_trunc(c, F, c->prev[q]);
  if (s != IDMRG_OK) return s;
  if (c->plan_pending) {
    c->plan_pending = false;
    return plan_iteration(c);
  }
  return IDMRG_OK;
}

// ------------------------------------------------------------------------
// Checkpoint between unit-cell steps: n, the e_g bookkeeping, every pair's
// current environments and the last two truncations (bases, sector tables,
// U, V, lambda) that the prediction reads.  Binary, host byte order.
// ------------------------------------------------------------------------
idmrg_status idmrg_save(const idmrg_ctx *cc, const char *path) {
  if (!cc || !path) return IDMRG_EINVAL;
  idmrg_ctx *c = const_cast<idmrg_ctx *>(cc);  // errors are recorded in the context
  if (!c->one_ring()) return c->fail(IDMRG_EINVAL, "save: needs a context of one problem");
  if (!c->owns_all()) return c->fail(IDMRG_ESTATE, "save: the context steps only superblocks %d..%d", c->own0, c->own1 - 1);
  for (int q = 0; q < c->P; ++q)
    if (c->stage[q] != ST_READY) return c->fail(IDMRG_ESTATE, "save: a step is in progress");
  CK(cudaStreamSynchronize(c->st));
  CkFile F;
  F.f = fopen(path, "wb");
  if (!F.f) return c->fail(IDMRG_EINVAL, "save: cannot open %s", path);
  F.ok = fwrite(CK_MAGIC, 1, 8, F.f) == 8;
  F.put(c->ell);
  F.put(c->d);
  F.put(c->P);
  F.put(c->o.m);
  F.put((int)c->o.prec);
  F.put(c->o.target_charge);
  {  // the bond dimensions of the unit cell with its closing bond (l + 1 entries)
    std::vector<int> ad(c->adim);
    ad.push_back(c->adim[0]);
    F.putv(ad);
  }
  F.put(c->n);
  F.put(c->rings[0].eg_n);
  F.put(c->rings[0].eg_last);
  std::vector<int> e1n;
  std::vector<double> e1v;
  for (const auto &kv : c->rings[0].e1) {
    e1n.push_back(kv.first);
    e1v.push_back(kv.second);
  }
  F.putv(e1n);
  F.putv(e1v);
  std::vector<int> ern;
  std::vector<double> erv;
  for (const auto &kv : c->rings[0].eps1) {
    ern.push_back(kv.first);
    erv.push_back(kv.second);
  }
  F.putv(ern);
  F.putv(erv);
  for (int q = 0; q < c->P; ++q) {
    for (const Env *E : {&c->envL[q], &c->envR[q]}) {
      ck_put_basis(F, E->lay.b);
      F.putv(E->lay.chq);
      idmrg_status s = ck_put_dev(c, F, E->data, E->lay.size);
      if (s != IDMRG_OK) return s;
    }
    for (const TruncRec *T : {&c->prev[q], &c->prev2[q]}) {
      idmrg_status s = ck_put_trunc_dev(c, F, *T);
      if (s != IDMRG_OK) return s;
    }
  }
  if (!F.ok) return c->fail(IDMRG_EINVAL, "save: write to %s failed", path);
  return IDMRG_OK;
}

idmrg_status idmrg_load(idmrg_ctx *c, const char *path) {
  if (!c || !path) return IDMRG_EINVAL;
  if (!c->one_ring()) return c->fail(IDMRG_EINVAL, "load: needs a context of one problem");
  if (!c->owns_all()) return c->fail(IDMRG_ESTATE, "load: the context steps only superblocks %d..%d", c->own0, c->own1 - 1);
  for (int q = 0; q < c->P; ++q)
    if (c->stage[q] != ST_READY) return c->fail(IDMRG_ESTATE, "load: a step is in progress");
  c->obs.valid = c->obs.fixed = false;
  CkFile F;
  F.f = fopen(path, "rb");
  if (!F.f) return c->fail(IDMRG_EINVAL, "load: cannot open %s", path);
  char magic[8] = {};
  F.ok = fread(magic, 1, 8, F.f) == 8 && memcmp(magic, CK_MAGIC, 8) == 0;
  int ell = 0, d = 0, P = 0, m = 0, prec = 0, target = 0;
  std::vector<int> adim;
  F.get(ell);
  F.get(d);
  F.get(P);
  F.get(m);
  F.get(prec);
  F.get(target);
  F.getv(adim, 1 << 20);
  (void)prec;  // every precision keeps the state in FP64: a state moves between precisions
  if (!F.ok || ell != c->ell || d != c->d || P != c->P || m != c->o.m || target != c->o.target_charge ||
      adim.size() != c->adim.size() + 1 || !std::equal(c->adim.begin(), c->adim.end(), adim.begin()) ||
      adim.back() != c->adim[0])
    return c->fail(IDMRG_EINVAL, "load: %s is not a checkpoint of this MPO and these options", path);
  int n = 0, eg_n = 0;
  double eg_last = 0.0;
  std::vector<int> e1n;
  std::vector<double> e1v;
  F.get(n);
  F.get(eg_n);
  F.get(eg_last);
  F.getv(e1n, 1 << 30);
  F.getv(e1v, 1 << 30);
  std::vector<int> ern;
  std::vector<double> erv;
  F.getv(ern, 1 << 30);
  F.getv(erv, 1 << 30);
  if (!F.ok || n < 1 || e1n.size() != e1v.size() || ern.size() != erv.size())
    return c->fail(IDMRG_EINVAL, "load: checkpoint header damaged");
  for (int q = 0; q < P; ++q) {
    for (Env *E : {&c->envL[q], &c->envR[q]}) {
      Basis b;
      std::vector<int> chq;
      ck_get_basis(F, b);
      F.getv(chq, 1 << 20);
      if (!F.ok) return c->fail(IDMRG_EINVAL, "load: checkpoint truncated");
      E->lay.build(b, chq);
      idmrg_status s = ck_get_dev(c, F, E->data, E->lay.size);
      if (s != IDMRG_OK) return s;
    }
    for (TruncRec *T : {&c->prev[q], &c->prev2[q]}) {
      idmrg_status s = ck_get_trunc(c, F, *T);
      if (s != IDMRG_OK) return s;
    }
  }
  c->n = n;
  c->rings[0].eg_n = eg_n;
  c->rings[0].eg_last = eg_last;
  c->rings[0].e1.clear();
  for (size_t k = 0; k < e1n.size(); ++k) c->rings[0].e1[e1n[k]] = e1v[k];
  c->rings[0].eps1.clear();
  for (size_t k = 0; k < ern.size(); ++k) c->rings[0].eps1[ern[k]] = erv[k];
  return plan_iteration(c);
}

idmrg_status idmrg_truncation_error(const idmrg_ctx *c, double *eps) {
  if (!c || !eps) return IDMRG_EINVAL;
  if (!c->one_ring()) return IDMRG_EINVAL;
  if (c->rings[0].eps1.empty()) return IDMRG_ESTATE;
  double e = 0.0;
  int k = 0;
  for (auto it = c->rings[0].eps1.rbegin(); it != c->rings[0].eps1.rend() && k < c->ell; ++it, ++k) e = std::max(e, it->second);
  *eps = e;
  return IDMRG_OK;
}

idmrg_status idmrg_run(idmrg_ctx *c, int max_steps, double de_tol, double *e_g, double *eps, int *steps) {
  if (!c || max_steps < 1 || !(de_tol > 0)) return IDMRG_EINVAL;
  if (!c->one_ring()) return c->fail(IDMRG_EINVAL, "run: needs a context of one problem");
  double last = NAN;
  int last_n = -1, k = 0;
  bool done = false;
  for (; k < max_steps && !done; ++k) {
    const idmrg_status s = idmrg_unit_cell_step(c, nullptr);
    if (s != IDMRG_OK && s != IDMRG_ENOCONV) return s;
    if (c->rings[0].eg_n >= 0 && c->rings[0].eg_n != last_n) {  // a new estimate of e_g
      done = std::isfinite(last) && fabs(c->rings[0].eg_last - last) < de_tol;
      last = c->rings[0].eg_last;
      last_n = c->rings[0].eg_n;
    }
  }
  if (steps) *steps = k;
  if (e_g) *e_g = c->rings[0].eg_last;
  if (eps) idmrg_truncation_error(c, eps);
  return done ? IDMRG_OK : IDMRG_ENOCONV;
}

idmrg_status idmrg_correlation(idmrg_ctx *c, int nterms, const double *op_a, const double *op_b, const double *coef,
                               int npairs, const int64_t *site_i, const int64_t *site_j, double *out) {
  if (!c || nterms < 1 || nterms > 64 || npairs < 0 || !op_a || !op_b || !coef) return IDMRG_EINVAL;
  if (!c->one_ring()) return c->fail(IDMRG_EINVAL, "correlation: needs a context of one problem");
  if (npairs > 0 && (!site_i || !site_j || !out)) return IDMRG_EINVAL;
  if (!c->owns_all() || c->plan_pending) return c->fail(IDMRG_ESTATE, "correlation: needs the whole unit cell");
  for (int k = 0; k < npairs; ++k)
    if (site_i[k] < 0 || site_j[k] <= site_i[k] || site_j[k] - site_i[k] > (int64_t)1 << 20)
      return c->fail(IDMRG_EINVAL, "correlation: pair %d needs 0 <= i < j <= i + 2^20", k);
  for (int q = 0; q < c->P; ++q)
    if (c->stage[q] != ST_READY) return c->fail(IDMRG_ESTATE, "correlation: a step is in progress");
  if (npairs == 0) return IDMRG_OK;
  return obs_correlation(c, nterms, op_a, op_b, coef, npairs, site_i, site_j, out);
}

idmrg_status idmrg_transfer_spectrum(idmrg_ctx *c, double tol, int maxit, double *t1, double *t2_abs, double *xi,
                                     int *iters) {
  if (!c || !(tol > 0.0) || maxit < 1) return IDMRG_EINVAL;
  if (!c->one_ring()) return c->fail(IDMRG_EINVAL, "transfer_spectrum: needs a context of one problem");
  if (!c->owns_all() || c->plan_pending) return c->fail(IDMRG_ESTATE, "transfer_spectrum: needs the whole unit cell");
  for (int q = 0; q < c->P; ++q)
    if (c->stage[q] != ST_READY) return c->fail(IDMRG_ESTATE, "transfer_spectrum: a step is in progress");
  double ratio = 0.0;
  int it = 0;
  const idmrg_status s = obs_spectrum(c, tol, maxit, &ratio, &it);
  if (s != IDMRG_OK && s != IDMRG_ENOCONV) return s;
  if (t1) *t1 = c->obs.t1;
  if (t2_abs) *t2_abs = ratio * c->obs.t1;
  if (xi) *xi = ratio > 0.0 ? -1.0 / std::log(ratio) : 0.0;
  if (iters) *iters = it;
  return s;
}

idmrg_status idmrg_ring_energy(const idmrg_ctx *c, int r, double *e_g, int *n_of_estimate) {
  if (!c || r < 0 || r >= (int)c->rings.size()) return IDMRG_EINVAL;
  const idmrg_ctx::Ring &R = c->rings[r];
  if (R.eg_n < 0) return IDMRG_ESTATE;
  if (e_g) *e_g = R.eg_last;
  if (n_of_estimate) *n_of_estimate = R.eg_n;
  return IDMRG_OK;
}

idmrg_status idmrg_energy_per_site(const idmrg_ctx *c, double *e_g, int *n_of_estimate) {
  if (!c) return IDMRG_EINVAL;
  if (c->rings[0].eg_n < 0) return IDMRG_ESTATE;
  if (e_g) *e_g = c->rings[0].eg_last;
  if (n_of_estimate) *n_of_estimate = c->rings[0].eg_n;
  return IDMRG_OK;
}

idmrg_status idmrg_heff_cost(const idmrg_ctx *c, int p, double *flops, double *bytes) {
  if (!c || p < -1 || p >= c->P) return IDMRG_EINVAL;
  double f = 0, b = 0;
  for (int q = 0; q < c->P; ++q)
    if (want(c, p, q)) { f += c->plan[q].heff_flops; b += c->plan[q].heff_bytes; }
  if (flops) *flops = f;
  if (bytes) *bytes = b;
  return IDMRG_OK;
}

idmrg_status idmrg_launch_count(const idmrg_ctx *c, uint64_t *count) {
  if (!c || !count) return IDMRG_EINVAL;
  *count = c->launches;
  return IDMRG_OK;
}

idmrg_status idmrg_profile_enable(idmrg_ctx *c, int on) {
  if (!c) return IDMRG_EINVAL;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return IDMRG_ECUDA;
  for (int k = 0; k < idmrg_ctx::KT_ALL; ++k) {
    c->collapse(k);
    c->kt[k].ms = c->kt[k].flops = c->kt[k].bytes = 0.0;
    c->kt[k].n = 0;
    c->kt[k].pending = nullptr;
  }
  c->prof = on != 0;
  return IDMRG_OK;
}

idmrg_status idmrg_profile_read(idmrg_ctx *c, int k, double *ms, uint64_t *launches, double *flops, double *bytes) {
  if (!c || k < 0 || k >= IDMRG_K_COUNT) return IDMRG_EINVAL;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return IDMRG_ECUDA;
  c->collapse(k);
  if (ms) *ms = c->kt[k].ms;
  if (launches) *launches = c->kt[k].n;
  if (flops) *flops = c->kt[k].flops;
  if (bytes) *bytes = c->kt[k].bytes;
  return IDMRG_OK;
}

idmrg_status idmrg_svd_phase_ms(idmrg_ctx *c, double *ms) {
  if (!c || !ms) return IDMRG_EINVAL;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return IDMRG_ECUDA;
  for (int k = 0; k < idmrg_ctx::SVD_PHASES; ++k) {
    c->collapse(IDMRG_K_COUNT + k);
    ms[k] = c->kt[IDMRG_K_COUNT + k].ms;
  }
  return IDMRG_OK;
}

idmrg_status idmrg_set_svd_path(idmrg_ctx *c, int global_only) {
  if (!c) return IDMRG_EINVAL;
  c->svd_global = global_only != 0;
  return IDMRG_OK;
}

idmrg_status idmrg_set_jacobi_arithmetic(idmrg_ctx *c, int mode) {
  if (!c) return IDMRG_EINVAL;
  if (mode < 0 || mode > 2) return c->fail(IDMRG_EINVAL, "set_jacobi_arithmetic: mode %d is not 0, 1 or 2", mode);
  c->jac_arith = mode;
  return IDMRG_OK;
}

idmrg_status idmrg_svd_sweeps32(const idmrg_ctx *c, int *max_sweeps, double *mean_sweeps) {
  if (!c) return IDMRG_EINVAL;
  if (max_sweeps) *max_sweeps = c->svd_max_sweeps32;
  if (mean_sweeps) *mean_sweeps = c->svd_jobs32 ? c->svd_mean_sweeps32 / c->svd_jobs32 : 0.0;
  return IDMRG_OK;
}

idmrg_status idmrg_svd_stats(const idmrg_ctx *c, int *jobs, int *max_cols, int *max_rank, int *max_sweeps,
                             double *mean_sweeps) {
  if (!c) return IDMRG_EINVAL;
  if (jobs) *jobs = c->svd_jobs;
  if (max_cols) *max_cols = c->svd_max_cols;
  if (max_rank) *max_rank = c->svd_max_rank;
  if (max_sweeps) *max_sweeps = c->svd_max_sweeps;
  if (mean_sweeps) *mean_sweeps = c->svd_mean_sweeps;
  return IDMRG_OK;
}

idmrg_status idmrg_set_mixed_restart(idmrg_ctx *c, double inner_factor, int inner_cap) {
  if (!c) return IDMRG_EINVAL;
  if (!(inner_factor > 0.0 && inner_factor < 1.0) || inner_cap < 2)
    return c->fail(IDMRG_EINVAL, "set_mixed_restart: need 0 < inner_factor < 1 and inner_cap >= 2");
  c->inner_factor = inner_factor;
  c->inner_cap = inner_cap;
  return IDMRG_OK;
}

idmrg_status idmrg_set_gemm_tile(idmrg_ctx *c, int tn1, int tn3) {
  if (!c) return IDMRG_EINVAL;
  auto ok = [](int t) { return t == 0 || t == 64 || t == 128 || t == 256; };
  if (!ok(tn1) || !ok(tn3)) return c->fail(IDMRG_EINVAL, "set_gemm_tile: N tiles are 0 (tuned), 64, 128 or 256");
  c->force_tn[0] = tn1;
  c->force_tn[1] = tn3;
  return IDMRG_OK;
}

idmrg_status idmrg_gemm_tuning(const idmrg_ctx *c, int stage, int *tn, float *ms, int *tunings) {
  if (!c || (stage != 1 && stage != 3)) return IDMRG_EINVAL;
  const idmrg_ctx::TcTune &T = stage == 1 ? c->tt1 : c->tt3;
  if (tn) *tn = T.choice >= 0 ? MIX_TNS[T.choice] : 0;
  if (ms)
    for (int k = 0; k < MIX_NTN; ++k) ms[k] = T.ms[k];
  if (tunings) *tunings = c->tc_tunes;
  return IDMRG_OK;
}

idmrg_status idmrg_transfer_bytes(const idmrg_ctx *c, uint64_t *h2d, uint64_t *d2h) {
  if (!c) return IDMRG_EINVAL;
  if (h2d) *h2d = c->h2d;
  if (d2h) *d2h = c->d2h;
  return IDMRG_OK;
}

}  // extern "C"

// --------------------------------------------------------------------------
// H_eff psi without device allocation.
//
// Some callers cannot allocate device memory once they are running: code
// inside a memory-capped or pre-partitioned pool, callers that must not touch
// the allocator while other work is queued, or embedders whose allocator may
// not be called from this thread.  This entry point serves them: it applies
// one superblock's H_eff in FP64 with its intermediates (the T1 and T3
// contractions) and its pointer table in the file-scope device array below,
// a fixed 16 MiB that every GPU loading this library holds until the process
// exits.  Host code sees the array's name only as a stand-in for the symbol,
// so every call looks its device address up with cudaGetSymbolAddress (with
// the context's device current; the lookup allocates nothing), and the
// pointer table is built on the device from the context's own device table
// and values passed to a one-thread kernel, so no host memory is read by the
// queued work.
// --------------------------------------------------------------------------
namespace {
constexpr size_t kNoallocBytes = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// table = src (all P * NBUF entries), then superblock p's operands patched in;
// active[q] = (q == p).  One block; the entries are independent.
__global__ void noalloc_table_kernel(double *const *src, double **table, int *active, int P, int p, double *L,
                                     double *R, double *in, double *out, double *t1, double *t3) {
  for (int i = threadIdx.x; i < P * NBUF; i += blockDim.x) {
    const int q = i / NBUF, b = i % NBUF;
    double *v = src[i];
    if (q == p) {
      if (b == BUF_L) v = L;
      else if (b == BUF_R) v = R;
      else if (b == BUF_IN) v = in;
      else if (b == BUF_OUT) v = out;
      else if (b == BUF_T1) v = t1;
      else if (b == BUF_T3) v = t3;
    }
    table[i] = v;
  }
  for (int q = threadIdx.x; q < P; q += blockDim.x) active[q] = q == p ? 1 : 0;
}
}  // namespace

extern "C" idmrg_status idmrg_heff_apply_noalloc(idmrg_ctx *c, int p, const double *psi_dev, double *out_dev) {
  if (!c || !psi_dev || !out_dev || p < 0 || p >= c->P) return IDMRG_EINVAL;
  if (!c->owns(p) || c->plan_pending)
    return c->fail(IDMRG_ESTATE, "heff_apply_noalloc: superblock %d is not planned in this context", p);
  for (int q = 0; q < c->P; ++q)
    if (c->stage[q] >= ST_TRUNCATED)
      return c->fail(IDMRG_ESTATE, "heff_apply_noalloc: iteration %d is being truncated; call after idmrg_advance",
                     c->n);
  void *ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess || !ptr)
    return c->fail(IDMRG_ECUDA, "heff_apply_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  unsigned char *base = (unsigned char *)ptr;
  const SBPlan &S = c->plan[p];
  const size_t table_bytes = round256(sizeof(double *) * (size_t)c->P * NBUF);
  const size_t mask_bytes = round256(sizeof(int) * (size_t)c->P);
  const size_t t1_bytes = round256(8 * (size_t)std::max<int64_t>(S.t1size, 1));
  const size_t t3_bytes = round256(8 * (size_t)std::max<int64_t>(S.t3size, 1));
  const size_t need = table_bytes + mask_bytes + t1_bytes + t3_bytes;
  if (need > kNoallocBytes)
    return c->fail(IDMRG_EINVAL, "heff_apply_noalloc: superblock %d needs %zu bytes of scratch, the limit is %zu", p,
                   need, kNoallocBytes);
  double **bufs = (double **)base;
  int *active = (int *)(base + table_bytes);
  double *t1 = (double *)(base + table_bytes + mask_bytes);
  double *t3 = (double *)(base + table_bytes + mask_bytes + t1_bytes);
  noalloc_table_kernel<<<1, 256, 0, c->st>>>((double *const *)c->dbufs.p, bufs, active, c->P, p,
                                             c->hbufs[p * NBUF + BUF_L], c->hbufs[p * NBUF + BUF_R],
                                             const_cast<double *>(psi_dev), out_dev, t1, t3);
  CK(cudaGetLastError());
  CK(launch_gemm_f64((const GemmTile *)c->tn_g1.tiles[GEMM_64x64].p, c->tn_g1.ntiles[GEMM_64x64],
                     (const GemmTask *)c->dg1k.p, (const GemmSeg *)c->dg1s.p, bufs, active, c->st, GEMM_64x64));
  CK(launch_wstage_f64((const WTask *)c->dwt.p, (int)c->wl.tasks.size(), c->wl.max_rows, (const WTerm *)c->dwm.p,
                       bufs, active, c->st));
  CK(launch_gemm_f64((const GemmTile *)c->tn_g3.tiles[GEMM_64x64].p, c->tn_g3.ntiles[GEMM_64x64],
                     (const GemmTask *)c->dg3k.p, (const GemmSeg *)c->dg3s.p, bufs, active, c->st, GEMM_64x64));
  c->launches += 4;
  return IDMRG_OK;
}

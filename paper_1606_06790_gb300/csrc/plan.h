// Host-side block tables of the U(1) (2 S^z) block-sparse tensors and the task
// lists the batched kernels consume.  Pure C++ (no CUDA calls).
#pragma once
#include <stdint.h>

#include <array>
#include <vector>

#include "common.h"

namespace idmrg {

// Basis of a renormalised block: contiguous charge sectors in a fixed order.
struct Basis {
  std::vector<int> q, dim, off;
  int D = 0;
  void clear() { q.clear(); dim.clear(); off.clear(); D = 0; }
  void add(int charge, int d) { q.push_back(charge); dim.push_back(d); }
  void finish() {
    off.assign(q.size(), 0);
    D = 0;
    for (size_t i = 0; i < q.size(); ++i) { off[i] = D; D += dim[i]; }
  }
  int find(int charge) const {
    for (size_t i = 0; i < q.size(); ++i)
      if (q[i] == charge) return (int)i;
    return -1;
  }
  int S() const { return (int)q.size(); }
};

// Block-sparse operator list O_a[x][y] on a basis: channel a connects in-sector
// si to out-sector so[a*S+si] (charge q_out - q_in = chq[a]); each block is a
// dense row-major D_out x D_in matrix at element offset off[a*S+si].
struct EnvLayout {
  Basis b;
  int w = 0;
  std::vector<int> chq, so;
  std::vector<int64_t> off;
  int64_t size = 0;
  void build(const Basis &basis, const std::vector<int> &ch);
};

// Superblock wavefunction psi[x][s][t][y]: one dense row block per left sector
// i (D_i rows, C[i] columns made of the (s,t) sub-blocks), sub-block (i,s,t)
// holding right sector sj[(i*d+s)*d+t] at column scol[...].
struct PsiLayout {
  int d = 0;
  std::vector<int64_t> roff;
  std::vector<int> C, sj, scol;
  int64_t N = 0;
  void build(const Basis &L, const Basis &R, const std::vector<int> &qp, int target);
  int sub(int i, int s, int t) const { return (i * d + s) * d + t; }
};

// Grouped-GEMM task list (see GemmTask / GemmSeg).
struct GemmList {
  std::vector<GemmTask> tasks;
  std::vector<GemmSeg> segs;
  std::vector<GemmTile> tiles;
  double flops = 0.0;
  void clear() { tasks.clear(); segs.clear(); tiles.clear(); flops = 0.0; }
  int task(int sb, int c_buf, int64_t c_off, int M, int N, int ldc, int accumulate = 0);
  void seg(int a_buf, int64_t a_off, int lda, int b_buf, int64_t b_off, int ldb, int K, int flags,
           double alpha = 1.0);
  void finish(int tm, int tn);  // output tiles
};

struct WList {
  std::vector<WTask> tasks;
  std::vector<WTerm> terms;
  int max_rows = 0;
  double flops = 0.0;
  void clear() { tasks.clear(); terms.clear(); max_rows = 0; flops = 0.0; }
  void task(int sb, int out_buf, int64_t out_off, int out_ld, int in_buf, int rows, int cols);
  void term(int64_t in_off, int in_ld, double coef);
};

// Kept sector of one truncation (Step 4): left charge Q, k states.  Rows of U
// are the (left sector i, s) groups rg = {i, s, first row}; rows of V the
// (t, right sector j) groups cg = {t, j, first row}.
struct SecInfo {
  int Q = 0, k = 0, r = 0, c = 0, job = -1;
  std::vector<std::array<int, 3>> rg, cg;
  int64_t u_off = 0, v_off = 0;
  int lam_off = 0;
};

}  // namespace idmrg

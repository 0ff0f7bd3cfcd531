// Host-side block tables; see plan.h.
#include "plan.h"

#include <algorithm>

namespace idmrg {

void EnvLayout::build(const Basis &basis, const std::vector<int> &ch) {
  b = basis;
  chq = ch;
  w = (int)ch.size();
  const int S = b.S();
  so.assign((size_t)w * S, -1);
  off.assign((size_t)w * S, -1);
  size = 0;
  for (int a = 0; a < w; ++a)
    for (int si = 0; si < S; ++si) {
      const int o = b.find(b.q[si] + chq[a]);
      if (o < 0) continue;
      so[a * S + si] = o;
      off[a * S + si] = size;
      size += (int64_t)b.dim[o] * b.dim[si];
    }
}

void PsiLayout::build(const Basis &L, const Basis &R, const std::vector<int> &qp, int target) {
  d = (int)qp.size();
  const int SL = L.S();
  roff.assign(SL, 0);
  C.assign(SL, 0);
  sj.assign((size_t)SL * d * d, -1);
  scol.assign((size_t)SL * d * d, -1);
  N = 0;
  for (int i = 0; i < SL; ++i) {
    int c = 0;
    for (int s = 0; s < d; ++s)
      for (int t = 0; t < d; ++t) {
        const int j = R.find(target - L.q[i] - qp[s] - qp[t]);
        const int k = sub(i, s, t);
        if (j < 0) continue;
        sj[k] = j;
        scol[k] = c;
        c += R.dim[j];
      }
    C[i] = c;
    roff[i] = N;
    N += (int64_t)L.dim[i] * c;
  }
}

int GemmList::task(int sb, int c_buf, int64_t c_off, int M, int N, int ldc, int accumulate) {
  GemmTask t{};
  t.c_off = c_off;
  t.c_buf = c_buf;
  t.sb = sb;
  t.M = M;
  t.N = N;
  t.ldc = ldc;
  t.seg0 = (int)segs.size();
  t.nseg = 0;
  t.accumulate = accumulate;
  tasks.push_back(t);
  return (int)tasks.size() - 1;
}

void GemmList::seg(int a_buf, int64_t a_off, int lda, int b_buf, int64_t b_off, int ldb, int K, int flags,
                   double alpha) {
  GemmSeg s{};
  s.a_off = a_off;
  s.b_off = b_off;
  s.a_buf = a_buf;
  s.b_buf = b_buf;
  s.lda = lda;
  s.ldb = ldb;
  s.K = K;
  s.flags = flags;
  s.alpha = alpha;
  segs.push_back(s);
  GemmTask &t = tasks.back();
  t.nseg += 1;
  flops += 2.0 * t.M * (double)t.N * K;
}

void GemmList::finish(int tm, int tn) {
  tiles.clear();
  for (size_t i = 0; i < tasks.size(); ++i) {
    const GemmTask &t = tasks[i];
    for (int m0 = 0; m0 < t.M; m0 += tm)
      for (int n0 = 0; n0 < t.N; n0 += tn) tiles.push_back(GemmTile{(int)i, m0, n0, 0});
  }
}

void WList::task(int sb, int out_buf, int64_t out_off, int out_ld, int in_buf, int rows, int cols) {
  WTask t{};
  t.out_off = out_off;
  t.out_ld = out_ld;
  t.sb = sb;
  t.rows = rows;
  t.cols = cols;
  t.term0 = (int)terms.size();
  t.nterm = 0;
  t.out_buf = out_buf;
  t.in_buf = in_buf;
  tasks.push_back(t);
  max_rows = std::max(max_rows, rows);
}

void WList::term(int64_t in_off, int in_ld, double coef) {
  WTerm w{};
  w.in_off = in_off;
  w.in_ld = in_ld;
  w.coef = coef;
  terms.push_back(w);
  WTask &t = tasks.back();
  t.nterm += 1;
  flops += 2.0 * t.rows * (double)t.cols;
}

}  // namespace idmrg

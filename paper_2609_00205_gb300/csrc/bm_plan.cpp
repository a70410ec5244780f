// Host-side plan: hierarchy sizes, global-level tables and error constants.
// Compiled without floating-point contraction so every result is the same on
// every host architecture.
#include "bm_plan.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>

namespace bm {
namespace {

// Coarse nodes of a dimension with n nodes: even indices plus the last node,
// floor(n/2)+1 of them (Sec. II-B).
std::vector<int> coarse_of(int n) {
  std::vector<int> c;
  for (int i = 0; i < n; i += 2) c.push_back(i);
  if ((n - 1) % 2 != 0) c.push_back(n - 1);
  return c;
}

// Tridiagonal mass matrix of hats on x: diag d, off-diagonal o (o[i] = M(i,i+1)).
void mass(const std::vector<double>& x, std::vector<double>& d, std::vector<double>& o) {
  const int n = (int)x.size();
  d.assign(n, 0.0);
  o.assign(n, 0.0);
  for (int i = 0; i + 1 < n; ++i) {
    const double h = x[i + 1] - x[i];
    d[i] += h / 3.0;
    d[i + 1] += h / 3.0;
    o[i] = h / 6.0;
  }
}

Dim1DHost make_dim(const std::vector<double>& x) {
  Dim1DHost D;
  D.n = (int)x.size();
  D.x = x;
  D.cidx = coarse_of(D.n);
  D.c = (int)D.cidx.size();
  D.isc.assign(D.n, 0);
  for (int j : D.cidx) D.isc[j] = 1;
  D.jlo.resize(D.n); D.jhi.resize(D.n); D.wl.resize(D.n); D.wr.resize(D.n); D.cb.resize(D.n);
  int J = 0;
  for (int i = 0; i < D.n; ++i) {
    D.cb[i] = J;  // coarse indices strictly below i
    if (D.isc[i]) {
      D.jlo[i] = D.jhi[i] = J;
      D.wl[i] = 1.0;
      D.wr[i] = 0.0;
      ++J;
    } else {
      D.jlo[i] = J - 1;
      D.jhi[i] = J;
      const double a = x[i - 1], b = x[i + 1];
      D.wl[i] = (b - x[i]) / (b - a);
      D.wr[i] = (x[i] - a) / (b - a);
    }
  }
  std::vector<double> md, mo;
  mass(x, md, mo);
  D.md = md;
  D.mo = mo;
  auto Mf = [&](int r, int c) -> double {
    if (r < 0 || c < 0 || r >= D.n || c >= D.n) return 0.0;
    if (r == c) return md[r];
    if (r + 1 == c) return mo[r];
    if (c + 1 == r) return mo[c];
    return 0.0;
  };
  D.f0.resize(D.c);
  D.band.assign(5 * (size_t)D.c, 0.0);
  for (int Jc = 0; Jc < D.c; ++Jc) {
    const int f = D.cidx[Jc];
    D.f0[Jc] = std::max(0, f - 2);
    for (int m = 0; m < 5; ++m) {
      const int col = D.f0[Jc] + m;
      if (col >= D.n || col > f + 2) continue;
      // row Jc of I^T M_f = M_f(f, :) + sum over fine neighbours of I(nb, Jc) M_f(nb, :)
      double v = Mf(f, col);
      if (f - 1 >= 0 && !D.isc[f - 1]) v += D.wr[f - 1] * Mf(f - 1, col);
      if (f + 1 < D.n && !D.isc[f + 1]) v += D.wl[f + 1] * Mf(f + 1, col);
      D.band[5 * Jc + m] = v;
    }
  }
  // coarse mass matrix and its Thomas factors
  std::vector<double> xc(D.c);
  for (int Jc = 0; Jc < D.c; ++Jc) xc[Jc] = x[D.cidx[Jc]];
  std::vector<double> cd, co;
  mass(xc, cd, co);
  D.tm.assign(D.c, 0.0); D.tib.assign(D.c, 0.0); D.tsup.assign(D.c, 0.0);
  double bp = cd[0];
  D.tib[0] = 1.0 / bp;
  for (int i = 1; i < D.c; ++i) {
    const double mul = co[i - 1] / bp;
    bp = cd[i] - mul * co[i - 1];
    D.tm[i] = mul;
    D.tib[i] = 1.0 / bp;
  }
  for (int i = 0; i + 1 < D.c; ++i) D.tsup[i] = co[i];
  return D;
}

// nb copies of the level on block-local coordinates xs side by side, with
// no coupling between them: every index table shifted by the segment, the
// band rows kept inside their segment (make_dim zeroes columns beyond it),
// and the Thomas factors restarting at each segment (tm = 0 at its first
// coarse node, tsup = 0 at its last), so one solve along the whole line is
// nb independent solves.
Dim1DHost make_blocked_dim(int nb, const std::vector<double>& xs) {
  const Dim1DHost S = make_dim(xs);
  Dim1DHost D;
  const int n = S.n, c = S.c;
  D.n = nb * n;
  D.c = nb * c;
  for (int b = 0; b < nb; ++b) {
    for (int i = 0; i < n; ++i) {
      D.x.push_back((double)b * (xs.back() + 1.0) + xs[(size_t)i]);
      D.jlo.push_back(b * c + S.jlo[(size_t)i]);
      D.jhi.push_back(b * c + S.jhi[(size_t)i]);
      D.cb.push_back(b * c + S.cb[(size_t)i]);
      D.isc.push_back(S.isc[(size_t)i]);
      D.wl.push_back(S.wl[(size_t)i]);
      D.wr.push_back(S.wr[(size_t)i]);
      D.md.push_back(S.md[(size_t)i]);
      D.mo.push_back(S.mo[(size_t)i]);  // 0 at the segment's last node
    }
    for (int J = 0; J < c; ++J) {
      D.cidx.push_back(b * n + S.cidx[(size_t)J]);
      D.f0.push_back(b * n + S.f0[(size_t)J]);
      for (int m = 0; m < 5; ++m) D.band.push_back(S.band[5 * (size_t)J + m]);
      D.tm.push_back(S.tm[(size_t)J]);    // 0 at the segment's first coarse node
      D.tib.push_back(S.tib[(size_t)J]);
      D.tsup.push_back(S.tsup[(size_t)J]);  // 0 at its last
    }
  }
  return D;
}

// P = M_c^{-1} I^T M_f as a dense c x n matrix, column by column (Thomas).
std::vector<double> projection(const Dim1DHost& D) {
  std::vector<double> P((size_t)D.c * D.n, 0.0);
  if (D.c == D.n) {
    for (int i = 0; i < D.n; ++i) P[(size_t)i * D.n + i] = 1.0;
    return P;
  }
  std::vector<double> r(D.c), y(D.c);
  for (int col = 0; col < D.n; ++col) {
    for (int J = 0; J < D.c; ++J) {
      const int m = col - D.f0[J];
      r[J] = (m >= 0 && m < 5) ? D.band[5 * J + m] : 0.0;
    }
    y[0] = r[0];
    for (int J = 1; J < D.c; ++J) y[J] = r[J] - D.tm[J] * y[J - 1];
    double z = y[D.c - 1] * D.tib[D.c - 1];
    P[(size_t)(D.c - 1) * D.n + col] = z;
    for (int J = D.c - 2; J >= 0; --J) {
      z = (y[J] - D.tsup[J] * z) * D.tib[J];
      P[(size_t)J * D.n + col] = z;
    }
  }
  return P;
}

// Per fine row r of Q = I P: abs row sum S, abs sum over coarse columns SC,
// diagonal entry q, coarse flag.
struct RowStat {
  double S, SC, q;
  int coarse;
  bool operator<(const RowStat& o) const { return std::tie(S, SC, q, coarse) < std::tie(o.S, o.SC, o.q, o.coarse); }
};

std::vector<RowStat> row_stats(const Dim1DHost& D) {
  const std::vector<double> P = projection(D);
  std::vector<RowStat> st;
  for (int r = 0; r < D.n; ++r) {
    RowStat s{0.0, 0.0, 0.0, D.isc[r]};
    for (int col = 0; col < D.n; ++col) {
      // Q(r, col) = wl P(jlo, col) + wr P(jhi, col)  (one row at coarse nodes)
      double q = D.isc[r] ? P[(size_t)D.jlo[r] * D.n + col]
                          : D.wl[r] * P[(size_t)D.jlo[r] * D.n + col] + D.wr[r] * P[(size_t)D.jhi[r] * D.n + col];
      s.S += std::fabs(q);
      if (D.isc[col]) s.SC += std::fabs(q);
      if (col == r) s.q = q;
    }
    st.push_back(s);
  }
  std::sort(st.begin(), st.end());
  st.erase(std::unique(st.begin(), st.end(),
                       [](const RowStat& a, const RowStat& b) { return !(a < b) && !(b < a); }),
           st.end());
  return st;
}

// Level error constant: max over fine nodes of the abs row sum of
// R = (Id - I P) restricted to the coefficient (non all-coarse) columns,
// rounded up onto the 2^-16 grid.
double error_constant(const Dim1DHost* D3) {
  std::vector<RowStat> s0 = row_stats(D3[0]), s1 = row_stats(D3[1]), s2 = row_stats(D3[2]);
  double best = 0.0;
  for (const RowStat& a : s0)
    for (const RowStat& b : s1)
      for (const RowStat& c : s2) {
        const double full = a.S * b.S * c.S;
        const double coarse = a.SC * b.SC * c.SC;
        double v;
        if (a.coarse && b.coarse && c.coarse) {
          v = full - coarse;
        } else {
          const double q = a.q * b.q * c.q;
          v = full - std::fabs(q) + std::fabs(1.0 - q) - coarse;
        }
        best = std::max(best, v);
      }
  return std::ceil(best * 65536.0 + 0.5) / 65536.0;
}

}  // namespace

std::string make_plan(const int64_t* shape, int B, int K, int M, int R, PlanHost& p) {
  if (B < 3 || B > 64) return "block size must be in [3, 64]";
  if (R < 1) return "at least one round";
  p = PlanHost{};
  for (int d = 0; d < 3; ++d) p.shape[d] = shape[d];
  p.B = B; p.K = K; p.M = M; p.R = R;
  // a dimension of extent 1 (the missing dimensions of a 1-D or 2-D field)
  // is neither blocked nor coarsened
  int nonunit = 0;
  for (int d = 0; d < 3; ++d) {
    if (shape[d] < 1) return "every extent must be at least 1";
    p.Bd[d] = shape[d] == 1 ? 1 : B;
    if (shape[d] > 1) {
      if (nonunit < 2) p.ax[nonunit] = d;
      ++nonunit;
    }
  }
  if (nonunit == 0) return "a field needs at least two values";
  p.reduced = nonunit < 3;
  if (p.reduced && nonunit == 1) { p.ax[1] = p.ax[0]; p.ax[0] = -1; }
  if (p.reduced && R > 1) return "re-blocking rounds need a 3-D field without extents of 1";
  p.nblocks = 1;
  for (int d = 0; d < 3; ++d) {
    const int64_t nb = (shape[d] + p.Bd[d] - 1) / p.Bd[d];
    if (nb > (1 << 30)) return "shape too large";
    p.nb[d] = (int)nb;
    p.nblocks *= nb;
  }
  // block-local coordinates through K levels (uniform: every other node kept)
  std::vector<double> xl(B);
  for (int j = 0; j < B; ++j) xl[j] = j;
  p.per_block = 0;
  const Dim1DHost one = make_dim(std::vector<double>{0.0});
  std::vector<int64_t> lvl_cnt;
  std::vector<Dim1DHost> lvl_dim;
  for (int l = 0; l < K; ++l) {
    const int n = (int)xl.size();
    if (n < 3) return "too many in-cache levels for this block size";
    std::vector<int> ci = coarse_of(n);
    int64_t nn = 1, cc = 1;
    for (int d = 0; d < 3; ++d) {
      nn *= p.Bd[d] == 1 ? 1 : n;
      cc *= p.Bd[d] == 1 ? 1 : (int64_t)ci.size();
    }
    lvl_cnt.push_back(nn - cc);
    p.per_block += nn - cc;
    Dim1DHost D = make_dim(xl);
    const Dim1DHost D3[3] = {p.Bd[0] == 1 ? one : D, p.Bd[1] == 1 ? one : D, p.Bd[2] == 1 ? one : D};
    p.A.push_back(error_constant(D3));
    lvl_dim.push_back(D);
    std::vector<double> nx;
    for (int j : ci) nx.push_back(xl[j]);
    xl = nx;
  }
  p.m = (int)xl.size();
  for (int d = 0; d < 3; ++d) p.md[d] = p.Bd[d] == 1 ? 1 : p.m;
  if (p.reduced) {
    int64_t off = 0;
    for (int l = 0; l < K; ++l) {
      RLevelHost rl;
      rl.nblk = p.nblocks;
      rl.da = p.ax[0] < 0 ? one : lvl_dim[(size_t)l];
      rl.db = lvl_dim[(size_t)l];
      rl.off = off;
      rl.blk_extra = p.per_block - lvl_cnt[(size_t)l];
      off += lvl_cnt[(size_t)l];
      p.rlev.push_back(rl);
    }
  }
  // re-blocking rounds (Sec. III-C): round r+1 blocks round r's gathered grid
  int64_t S[3] = {shape[0], shape[1], shape[2]};
  int64_t pos = 0;
  p.nblocks_all = 0;
  for (int r = 0; r < R; ++r) {
    RoundHost rd{};
    rd.nblocks = 1;
    for (int d = 0; d < 3; ++d) {
      const int64_t nb = (S[d] + p.Bd[d] - 1) / p.Bd[d];
      if (nb > (1 << 30)) return "shape too large";
      rd.shape[d] = S[d];
      rd.nb[d] = (int)nb;
      rd.nblocks *= nb;
      rd.gshape[d] = nb * p.md[d];
    }
    rd.off = pos;
    pos += rd.nblocks * p.per_block;
    p.nblocks_all += rd.nblocks;
    p.rounds.push_back(rd);
    for (int d = 0; d < 3; ++d) S[d] = rd.gshape[d];
  }
  // block sizes without a fused kernel: per round and level, the padded grid
  // and its block-diagonal operators
  p.generic = !p.reduced && !fused_block(B);
  if (p.generic) {
    std::vector<std::vector<double>> xs;  // block coordinates per level (K + 1)
    std::vector<double> x0(B);
    for (int j = 0; j < B; ++j) x0[j] = j;
    xs.push_back(x0);
    for (int l = 0; l < K; ++l) {
      std::vector<double> nx;
      for (int j : coarse_of((int)xs.back().size())) nx.push_back(xs.back()[(size_t)j]);
      xs.push_back(nx);
    }
    for (const RoundHost& rd : p.rounds) {
      std::vector<XLevelHost> lv;
      int64_t off = rd.off;
      for (int l = 0; l < K; ++l) {
        XLevelHost X;
        const int e = (int)xs[(size_t)l].size(), ce = (int)xs[(size_t)l + 1].size();
        for (int d = 0; d < 3; ++d) {
          X.e[d] = e;
          X.ce[d] = ce;
          X.nb[d] = rd.nb[d];
          X.shape[d] = (int64_t)rd.nb[d] * e;
          X.d[d] = make_blocked_dim(rd.nb[d], xs[(size_t)l]);
          if (X.d[d].c > 544) X.d[d].P = projection(X.d[d]);  // lines longer than the scan kernel takes
        }
        X.sym_off = off;
        off += (int64_t)e * e * e - (int64_t)ce * ce * ce;
        lv.push_back(X);
      }
      p.xlev.push_back(lv);
    }
  }
  // coordinates of the global levels' input: physical for one round (block
  // offset plus the coarse node's in-block coordinate), index coordinates of
  // the last gathered grid for several
  std::vector<double> gx[3];
  for (int d = 0; d < 3; ++d) {
    p.gshape[d] = S[d];
    if (R == 1) {
      for (int b = 0; b < p.nb[d]; ++b)
        for (int j = 0; j < p.md[d]; ++j) gx[d].push_back((double)b * p.Bd[d] + (p.Bd[d] == 1 ? 0.0 : xl[j]));
    } else {
      for (int64_t i = 0; i < S[d]; ++i) gx[d].push_back((double)i);
    }
  }
  for (int l = 0; l <= M; ++l) {
    for (int d = 0; d < 3; ++d) p.lshape.push_back((int64_t)gx[d].size());
    p.sym_off.push_back(pos);
    if (l == M) break;
    std::vector<Dim1DHost> L3;
    for (int d = 0; d < 3; ++d) {
      L3.push_back(make_dim(gx[d]));
      L3.back().P = projection(L3.back());
    }
    const int64_t cnt = (int64_t)L3[0].n * L3[1].n * L3[2].n - (int64_t)L3[0].c * L3[1].c * L3[2].c;
    pos += cnt;
    p.A.push_back(error_constant(L3.data()));
    for (int d = 0; d < 3; ++d) {
      std::vector<double> nx;
      for (int j : L3[d].cidx) nx.push_back(gx[d][j]);
      gx[d] = nx;
    }
    p.glev.push_back(L3);
  }
  const int64_t coarsest = p.lshape[3 * M] * p.lshape[3 * M + 1] * p.lshape[3 * M + 2];
  p.sym_off.push_back(pos + coarsest);  // end marker
  p.n_coeffs = pos + coarsest;
  return "";
}

}  // namespace bm

// BlockMGARD CPU oracle — TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, FP64 implementation of what the compressor computes, written
// from the paper's method description so the CUDA path can be checked against
// it.  Only tests/, the smoke check and the bench's CPU-baseline leg may load
// it; the product path never does.  It shares no code, header, table or
// constant generator with the CUDA library.
//
// What each part follows (section numbers of the BlockMGARD paper):
//   * nested grids, n -> floor(n/2)+1 nodes per level ............ Sec. II-B
//   * multilevel coefficients: fine values minus the interpolant of the
//     coarse values; coarse correction by the mass-matrix (L2) projection,
//     applied as one 1-D pass per dimension ........................ Sec. II-B
//   * level-dependent error shares giving an L-inf bound .......... Sec. II-B
//   * fixed-size blocks, zero fill outside the domain ........ Sec. III-A, III-D
//   * hybrid hierarchy: K in-cache levels per block, then M global levels on
//     the gathered block-coarse nodes ............................. Sec. III-B
//   * per-block ROI tolerance, tau_global = min_i tau_i ............ Sec. III-C
//   * Huffman coding of the quantised symbols (outliers, histogram,
//     codebook, encoding, concatenation) .......................... Sec. III-B
// Where the paper is silent this oracle takes these readings: the global
// levels use the physical coordinates of the gathered nodes; the error budget
// gives every level an equal share tau'/(N+1) divided by the level's exact
// L-inf operator constant A_l; tau' = tau minus a round-off margin of
// kappa*eps*(N+1)*max|u| (kappa = 8); quantisation rounds half up
// (floor(c/q + 1/2)); Huffman merging takes a leaf before an internal node of
// equal weight, and canonical codes are assigned in (length, symbol) order;
// the byte layout of the stream is the one written by compress() below.
//
// Everything is dense and direct: the 1-D operators are assembled as full
// matrices (I, M_f, M_c, P = M_c^{-1} I^T M_f) and applied as mode products.
//
// Parity pins: every function below is pinned by tests in tests/test_oracle_*.py
// (closed forms, invariants, independent quadrature assembly, brute force).

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <stdexcept>
#include <string>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Dense matrices and 3-D arrays
// ---------------------------------------------------------------------------
struct Mat {
  int r = 0, c = 0;
  std::vector<double> a;
  Mat() = default;
  Mat(int r_, int c_) : r(r_), c(c_), a((size_t)r_ * c_, 0.0) {}
  double& operator()(int i, int j) { return a[(size_t)i * c + j]; }
  double operator()(int i, int j) const { return a[(size_t)i * c + j]; }
};

struct Grid {
  int64_t n[3] = {0, 0, 0};
  std::vector<double> v;
  Grid() = default;
  Grid(int64_t a, int64_t b, int64_t c) { n[0] = a; n[1] = b; n[2] = c; v.assign((size_t)(a * b * c), 0.0); }
  double& at(int64_t i, int64_t j, int64_t k) { return v[(size_t)((i * n[1] + j) * n[2] + k)]; }
  double at(int64_t i, int64_t j, int64_t k) const { return v[(size_t)((i * n[1] + j) * n[2] + k)]; }
};

// B = A with dimension `dim` multiplied by Mat (out x in).
Grid mode_product(const Grid& A, int dim, const Mat& T) {
  if (T.c != A.n[dim]) throw std::runtime_error("mode_product: size mismatch");
  int64_t m[3] = {A.n[0], A.n[1], A.n[2]};
  m[dim] = T.r;
  Grid B(m[0], m[1], m[2]);
  for (int64_t i = 0; i < m[0]; ++i)
    for (int64_t j = 0; j < m[1]; ++j)
      for (int64_t k = 0; k < m[2]; ++k) {
        int64_t o = dim == 0 ? i : (dim == 1 ? j : k);
        double s = 0.0;
        for (int t = 0; t < T.c; ++t) {
          double w = T((int)o, t);
          if (w == 0.0) continue;
          double x = dim == 0 ? A.at(t, j, k) : (dim == 1 ? A.at(i, t, k) : A.at(i, j, t));
          s += w * x;
        }
        B.at(i, j, k) = s;
      }
  return B;
}

// Solve A X = R (A square, dense) by Gaussian elimination with partial pivoting.
Mat solve(Mat A, Mat R) {
  const int n = A.r;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int i = col + 1; i < n; ++i)
      if (std::fabs(A(i, col)) > std::fabs(A(piv, col))) piv = i;
    if (piv != col) {
      for (int j = 0; j < n; ++j) std::swap(A(col, j), A(piv, j));
      for (int j = 0; j < R.c; ++j) std::swap(R(col, j), R(piv, j));
    }
    for (int i = col + 1; i < n; ++i) {
      double f = A(i, col) / A(col, col);
      if (f == 0.0) continue;
      for (int j = col; j < n; ++j) A(i, j) -= f * A(col, j);
      for (int j = 0; j < R.c; ++j) R(i, j) -= f * R(col, j);
    }
  }
  for (int i = n - 1; i >= 0; --i)
    for (int j = 0; j < R.c; ++j) {
      double s = R(i, j);
      for (int t = i + 1; t < n; ++t) s -= A(i, t) * R(t, j);
      R(i, j) = s / A(i, i);
    }
  return R;
}

// ---------------------------------------------------------------------------
// 1-D level operator (Sec. II-B)
// ---------------------------------------------------------------------------
// A dimension of n nodes coarsens to floor(n/2)+1 nodes: the even indices plus
// the last node.  The coefficients live on the remaining (odd, non-last) nodes.
std::vector<int> coarse_indices(int n) {
  std::vector<int> c;
  for (int i = 0; i < n; i += 2) c.push_back(i);
  if ((n - 1) % 2 != 0) c.push_back(n - 1);
  return c;
}

// Piecewise-linear finite-element mass matrix on nodes x (hat functions).
Mat mass_matrix(const std::vector<double>& x) {
  const int n = (int)x.size();
  Mat M(n, n);
  for (int i = 0; i + 1 < n; ++i) {
    double h = x[i + 1] - x[i];
    M(i, i) += h / 3.0;
    M(i + 1, i + 1) += h / 3.0;
    M(i, i + 1) += h / 6.0;
    M(i + 1, i) += h / 6.0;
  }
  return M;
}

struct Level1D {
  int n = 0, nc = 0;
  std::vector<int> cidx;
  std::vector<char> is_coarse;
  std::vector<double> x, xc;
  Mat I;   // n x nc: interpolation of coarse nodal values onto the fine nodes
  Mat Mf;  // n x n
  Mat Mc;  // nc x nc
  Mat P;   // nc x n: P = Mc^{-1} I^T Mf (L2 projection of a fine function onto the coarse space)
};

Level1D make_level(const std::vector<double>& x) {
  Level1D L;
  L.n = (int)x.size();
  L.x = x;
  L.cidx = coarse_indices(L.n);
  L.nc = (int)L.cidx.size();
  L.is_coarse.assign(L.n, 0);
  for (int j : L.cidx) L.is_coarse[j] = 1;
  for (int j : L.cidx) L.xc.push_back(x[j]);
  L.I = Mat(L.n, L.nc);
  int J = 0;
  for (int i = 0; i < L.n; ++i) {
    if (L.is_coarse[i]) {
      L.I(i, J) = 1.0;
      ++J;
    } else {
      // Coarse hats at x[i-1] (index J-1) and x[i+1] (index J) evaluated at x[i].
      double a = x[i - 1], b = x[i + 1], t = x[i];
      L.I(i, J - 1) = (b - t) / (b - a);
      L.I(i, J) = (t - a) / (b - a);
    }
  }
  L.Mf = mass_matrix(L.x);
  L.Mc = mass_matrix(L.xc);
  if (L.nc == L.n) {  // no node to coarsen: the pass is the identity
    L.P = Mat(L.nc, L.n);
    for (int i = 0; i < L.n; ++i) L.P(i, i) = 1.0;
  } else {
    Mat R(L.nc, L.n);  // I^T Mf
    for (int a = 0; a < L.nc; ++a)
      for (int b = 0; b < L.n; ++b) {
        double s = 0.0;
        for (int t = 0; t < L.n; ++t) s += L.I(t, a) * L.Mf(t, b);
        R(a, b) = s;
      }
    L.P = solve(L.Mc, R);
  }
  return L;
}

double inf_norm(const Mat& A) {
  double m = 0.0;
  for (int i = 0; i < A.r; ++i) {
    double s = 0.0;
    for (int j = 0; j < A.c; ++j) s += std::fabs(A(i, j));
    m = std::max(m, s);
  }
  return m;
}

// ---------------------------------------------------------------------------
// One d-dimensional level (Sec. II-B), tensor product of the 1-D operators.
// ---------------------------------------------------------------------------
bool node_coarse(const Level1D* L, int64_t i, int64_t j, int64_t k) {
  return L[0].is_coarse[i] && L[1].is_coarse[j] && L[2].is_coarse[k];
}

Grid restrict_coarse(const Grid& u, const Level1D* L) {
  Grid c(L[0].nc, L[1].nc, L[2].nc);
  for (int a = 0; a < L[0].nc; ++a)
    for (int b = 0; b < L[1].nc; ++b)
      for (int d = 0; d < L[2].nc; ++d) c.at(a, b, d) = u.at(L[0].cidx[a], L[1].cidx[b], L[2].cidx[d]);
  return c;
}

Grid interpolate(const Grid& c, const Level1D* L) {
  Grid t = mode_product(c, 2, L[2].I);
  t = mode_product(t, 1, L[1].I);
  return mode_product(t, 0, L[0].I);
}

Grid project(const Grid& D, const Level1D* L) {  // z = (P0 x P1 x P2) D, last dim first
  Grid t = mode_product(D, 2, L[2].P);
  t = mode_product(t, 1, L[1].P);
  return mode_product(t, 0, L[0].P);
}

// Decompose one level: appends the coefficients (row-major over the
// non-coarse nodes) to `coef` and returns the corrected coarse values.
Grid decompose_level(const Grid& u, const Level1D* L, std::vector<double>& coef) {
  Grid uc = restrict_coarse(u, L);
  Grid E = interpolate(uc, L);
  Grid D(u.n[0], u.n[1], u.n[2]);
  for (int64_t i = 0; i < u.n[0]; ++i)
    for (int64_t j = 0; j < u.n[1]; ++j)
      for (int64_t k = 0; k < u.n[2]; ++k) {
        if (node_coarse(L, i, j, k)) continue;
        double d = u.at(i, j, k) - E.at(i, j, k);
        D.at(i, j, k) = d;
        coef.push_back(d);
      }
  Grid z = project(D, L);
  for (size_t t = 0; t < uc.v.size(); ++t) uc.v[t] += z.v[t];
  return uc;
}

// Inverse of decompose_level: coarse values and the level's coefficients
// (read from coef[pos...]) give the fine values.
Grid recompose_level(const Grid& c_hat, const Level1D* L, const double* coef, size_t& pos) {
  Grid D(L[0].n, L[1].n, L[2].n);
  for (int64_t i = 0; i < D.n[0]; ++i)
    for (int64_t j = 0; j < D.n[1]; ++j)
      for (int64_t k = 0; k < D.n[2]; ++k)
        if (!node_coarse(L, i, j, k)) D.at(i, j, k) = coef[pos++];
  Grid z = project(D, L);
  Grid uc = c_hat;
  for (size_t t = 0; t < uc.v.size(); ++t) uc.v[t] -= z.v[t];
  Grid u = interpolate(uc, L);
  for (size_t t = 0; t < u.v.size(); ++t) u.v[t] += D.v[t];  // D is 0 at coarse nodes
  return u;
}

size_t level_detail_count(const Level1D* L) {
  return (size_t)L[0].n * L[1].n * L[2].n - (size_t)L[0].nc * L[1].nc * L[2].nc;
}

// ---------------------------------------------------------------------------
// Hybrid hierarchy plan: R rounds of K in-cache levels per B^3 block (round
// r+1 re-blocks the gathered coarse values of round r, Sec. III-C), then M
// global levels.
// ---------------------------------------------------------------------------
struct Round {
  int64_t shape[3];  // the round's input grid
  int64_t nb[3];
  int64_t nblocks;
  size_t off;        // first coefficient of the round
};

struct Plan {
  int64_t shape[3];
  int B, K, M, R = 1;
  int Bd[3];         // block edge per dimension: B, or 1 for a dimension of extent 1
  int md[3];         // coarse nodes per block edge after K levels, per dimension
  int64_t nb[3];     // round 0
  int64_t nblocks;   // round 0
  std::vector<Round> rounds;
  int m;                          // coarse nodes per block dim after K levels (B-node dimensions)
  std::vector<std::vector<double>> block_coords;  // per local level (K+1 entries), B-node dimensions
  std::vector<Level1D> local;     // per local level: the 1-D level of a B-node dimension
  std::vector<std::array<Level1D, 3>> local3;     // per local level, per dimension (identity where Bd = 1)
  std::vector<std::array<Level1D, 3>> global;     // per global level
  size_t per_block = 0;           // coefficients per block
  std::vector<size_t> global_counts;
  size_t coarsest = 0;
  int64_t gshape[3];              // gathered coarse grid G
  int64_t cshape[3];              // coarsest grid
  size_t n_coeffs = 0;
};

Plan make_plan(const int64_t* shape, int B, int K, int M, int R = 1) {
  if (B < 2 || K < 0 || M < 0 || R < 1) throw std::runtime_error("bad parameters");
  Plan p;
  for (int d = 0; d < 3; ++d) p.shape[d] = shape[d];
  p.B = B; p.K = K; p.M = M; p.R = R;
  // A dimension of extent 1 (the missing dimensions of a 1-D or 2-D field) is
  // neither blocked nor coarsened: its blocks are one node thick and its level
  // operators are the identity of one node.
  for (int d = 0; d < 3; ++d) {
    if (shape[d] < 1) throw std::runtime_error("bad shape");
    p.Bd[d] = shape[d] == 1 ? 1 : B;
  }
  p.nblocks = 1;
  for (int d = 0; d < 3; ++d) {
    p.nb[d] = (shape[d] + p.Bd[d] - 1) / p.Bd[d];
    p.nblocks *= p.nb[d];
  }
  std::vector<double> xl(B);
  for (int j = 0; j < B; ++j) xl[j] = j;  // block-local coordinates x_j = j
  p.block_coords.push_back(xl);
  const Level1D one = make_level(std::vector<double>{0.0});
  for (int l = 0; l < K; ++l) {
    Level1D L = make_level(xl);
    p.local.push_back(L);
    std::array<Level1D, 3> L3;
    for (int d = 0; d < 3; ++d) L3[d] = p.Bd[d] == 1 ? one : L;
    p.per_block += level_detail_count(L3.data());
    p.local3.push_back(L3);
    xl = L.xc;
    p.block_coords.push_back(xl);
  }
  p.m = (int)xl.size();
  for (int d = 0; d < 3; ++d) p.md[d] = p.Bd[d] == 1 ? 1 : p.m;
  // rounds: each re-blocks the previous round's gathered grid (zero fill
  // beyond its extent)
  int64_t S[3] = {shape[0], shape[1], shape[2]};
  size_t off = 0;
  for (int r = 0; r < R; ++r) {
    Round rd;
    rd.nblocks = 1;
    for (int d = 0; d < 3; ++d) {
      rd.shape[d] = S[d];
      rd.nb[d] = (S[d] + p.Bd[d] - 1) / p.Bd[d];
      rd.nblocks *= rd.nb[d];
    }
    rd.off = off;
    off += (size_t)rd.nblocks * p.per_block;
    p.rounds.push_back(rd);
    for (int d = 0; d < 3; ++d) S[d] = rd.nb[d] * p.md[d];
  }
  // Coordinates of the gathered grid the global levels start from.  One
  // round: physical, block offset plus the coarse node's local coordinate, in
  // finest-grid index units.  Several rounds: index coordinates of the last
  // round's gathered grid (the paper's re-blocking works in index space).
  std::vector<double> gx[3];
  for (int d = 0; d < 3; ++d) {
    p.gshape[d] = S[d];
    if (R == 1) {
      for (int64_t b = 0; b < p.nb[d]; ++b)
        for (int j = 0; j < p.md[d]; ++j) gx[d].push_back((double)(b * p.Bd[d]) + (p.Bd[d] == 1 ? 0.0 : xl[j]));
    } else {
      for (int64_t i = 0; i < S[d]; ++i) gx[d].push_back((double)i);
    }
  }
  for (int l = 0; l < M; ++l) {
    std::array<Level1D, 3> L3{make_level(gx[0]), make_level(gx[1]), make_level(gx[2])};
    p.global_counts.push_back(level_detail_count(L3.data()));
    for (int d = 0; d < 3; ++d) gx[d] = L3[d].xc;
    p.global.push_back(L3);
  }
  for (int d = 0; d < 3; ++d) p.cshape[d] = (int64_t)gx[d].size();
  p.coarsest = (size_t)(p.cshape[0] * p.cshape[1] * p.cshape[2]);
  p.n_coeffs = off;
  for (size_t c : p.global_counts) p.n_coeffs += c;
  p.n_coeffs += p.coarsest;
  return p;
}

// Coefficient order: round by round, blocks row-major; inside a block levels
// finest->coarsest, each level's non-coarse nodes row-major; then global
// levels finest->coarsest; then the coarsest array row-major.
Grid decompose_round(const Grid& in, const Plan& p, const Round& rd, std::vector<double>& coef) {
  const int* Bd = p.Bd;
  const int* md = p.md;
  Grid G(rd.nb[0] * md[0], rd.nb[1] * md[1], rd.nb[2] * md[2]);
  for (int64_t b0 = 0; b0 < rd.nb[0]; ++b0)
    for (int64_t b1 = 0; b1 < rd.nb[1]; ++b1)
      for (int64_t b2 = 0; b2 < rd.nb[2]; ++b2) {
        Grid blk(Bd[0], Bd[1], Bd[2]);
        for (int i = 0; i < Bd[0]; ++i)
          for (int j = 0; j < Bd[1]; ++j)
            for (int k = 0; k < Bd[2]; ++k) {
              int64_t gi = b0 * Bd[0] + i, gj = b1 * Bd[1] + j, gk = b2 * Bd[2] + k;
              bool inside = gi < rd.shape[0] && gj < rd.shape[1] && gk < rd.shape[2];
              blk.at(i, j, k) = inside ? in.at(gi, gj, gk) : 0.0;  // zero fill
            }
        for (int l = 0; l < p.K; ++l) blk = decompose_level(blk, p.local3[l].data(), coef);
        for (int i = 0; i < md[0]; ++i)
          for (int j = 0; j < md[1]; ++j)
            for (int k = 0; k < md[2]; ++k)
              G.at(b0 * md[0] + i, b1 * md[1] + j, b2 * md[2] + k) = blk.at(i, j, k);
      }
  return G;
}

std::vector<double> decompose(const double* u, const Plan& p) {
  std::vector<double> coef;
  coef.reserve(p.n_coeffs);
  Grid G(p.shape[0], p.shape[1], p.shape[2]);
  std::copy(u, u + G.v.size(), G.v.begin());
  for (const Round& rd : p.rounds) G = decompose_round(G, p, rd, coef);
  for (int l = 0; l < p.M; ++l) G = decompose_level(G, p.global[l].data(), coef);
  for (double v : G.v) coef.push_back(v);
  return coef;
}

// Inverse of decompose_round: the round's gathered grid G and its
// coefficients give the round's input grid (in-domain nodes only).
Grid recompose_round(const Grid& G, const Plan& p, const Round& rd, const double* coef) {
  Grid out(rd.shape[0], rd.shape[1], rd.shape[2]);
  std::vector<size_t> lpos(p.K);
  for (int64_t b0 = 0; b0 < rd.nb[0]; ++b0)
    for (int64_t b1 = 0; b1 < rd.nb[1]; ++b1)
      for (int64_t b2 = 0; b2 < rd.nb[2]; ++b2) {
        int64_t bid = (b0 * rd.nb[1] + b1) * rd.nb[2] + b2;
        size_t q = rd.off + (size_t)bid * p.per_block;
        const int* Bd = p.Bd;
        const int* md = p.md;
        for (int l = 0; l < p.K; ++l) {
          lpos[l] = q;
          q += level_detail_count(p.local3[l].data());
        }
        Grid blk(md[0], md[1], md[2]);
        for (int i = 0; i < md[0]; ++i)
          for (int j = 0; j < md[1]; ++j)
            for (int k = 0; k < md[2]; ++k) blk.at(i, j, k) = G.at(b0 * md[0] + i, b1 * md[1] + j, b2 * md[2] + k);
        for (int l = p.K - 1; l >= 0; --l) {
          size_t r = lpos[l];
          blk = recompose_level(blk, p.local3[l].data(), coef, r);
        }
        for (int i = 0; i < Bd[0]; ++i)
          for (int j = 0; j < Bd[1]; ++j)
            for (int k = 0; k < Bd[2]; ++k) {
              int64_t gi = b0 * Bd[0] + i, gj = b1 * Bd[1] + j, gk = b2 * Bd[2] + k;
              if (gi < rd.shape[0] && gj < rd.shape[1] && gk < rd.shape[2]) out.at(gi, gj, gk) = blk.at(i, j, k);
            }
      }
  return out;
}

std::vector<double> recompose(const double* coef, const Plan& p) {
  // Coarsest, then global levels coarsest->finest, then the rounds last to first.
  size_t pos = p.rounds.back().off + (size_t)p.rounds.back().nblocks * p.per_block;
  std::vector<size_t> gpos(p.M);
  for (int l = 0; l < p.M; ++l) { gpos[l] = pos; pos += p.global_counts[l]; }
  Grid G(p.cshape[0], p.cshape[1], p.cshape[2]);
  for (size_t t = 0; t < G.v.size(); ++t) G.v[t] = coef[pos + t];
  for (int l = p.M - 1; l >= 0; --l) {
    size_t q = gpos[l];
    G = recompose_level(G, p.global[l].data(), coef, q);
  }
  for (int r = p.R - 1; r >= 0; --r) G = recompose_round(G, p, p.rounds[(size_t)r], coef);
  return G.v;
}

// Block tiers of every round (Sec. III-C): a block of round r+1 takes the
// smallest tolerance (lowest tier) among the round-r blocks whose coarse
// values it holds.  Empty with a single tier.
std::vector<std::vector<uint8_t>> round_tiers(const Plan& p, const std::vector<uint8_t>& tier0) {
  std::vector<std::vector<uint8_t>> t(p.rounds.size());
  if (tier0.empty()) return t;
  t[0] = tier0;
  for (size_t r = 0; r + 1 < p.rounds.size(); ++r) {
    const Round& a = p.rounds[r];
    const Round& b = p.rounds[r + 1];
    t[r + 1].assign((size_t)b.nblocks, 255);
    for (int64_t j0 = 0; j0 < b.nb[0]; ++j0)
      for (int64_t j1 = 0; j1 < b.nb[1]; ++j1)
        for (int64_t j2 = 0; j2 < b.nb[2]; ++j2) {
          const int64_t j[3] = {j0, j1, j2};
          int64_t lo[3], hi[3];  // contributing round-r blocks per dimension
          for (int d = 0; d < 3; ++d) {
            const int64_t first = j[d] * p.Bd[d], last = std::min((j[d] + 1) * p.Bd[d], b.shape[d]) - 1;
            lo[d] = first / p.md[d];
            hi[d] = last / p.md[d];
          }
          uint8_t v = 255;
          for (int64_t i0 = lo[0]; i0 <= hi[0]; ++i0)
            for (int64_t i1 = lo[1]; i1 <= hi[1]; ++i1)
              for (int64_t i2 = lo[2]; i2 <= hi[2]; ++i2)
                v = std::min(v, t[r][(size_t)((i0 * a.nb[1] + i1) * a.nb[2] + i2)]);
          t[r + 1][(size_t)((j0 * b.nb[1] + j1) * b.nb[2] + j2)] = v;
        }
  }
  return t;
}

// ---------------------------------------------------------------------------
// Error budget (Sec. II-B level shares, Sec. III-C tau_global)
// ---------------------------------------------------------------------------
// Level error constant A_l: the exact inf-norm of the map from a level's
// coefficient errors to the fine-grid error when the level is recomposed,
//   R = E_F - (I_0 P_0) x (I_1 P_1) x (I_2 P_2) E_F,
// E_F embedding the non-coarse nodes.  With coarse errors e_c bounded by E and
// coefficient errors by delta, recomposition gives |e| <= E + A_l delta, since
// the interpolation I is a convex combination.  Row r of R has abs sum
//   prod_k S_k(r_k) - prod_k SC_k(r_k)                        (r all-coarse)
//   prod_k S_k(r_k) - |q_r| + |1 - q_r| - prod_k SC_k(r_k)   (otherwise)
// with Q_k = I_k P_k, S_k = row abs sums of Q_k, SC_k = the same over coarse
// columns, q_r = prod_k Q_k(r_k, r_k).  A_l is rounded up onto the 2^-16 grid
// by ceil(A * 65536 + 0.5) / 65536 so independent implementations agree bitwise.
double round_constant(double C) { return std::ceil(C * 65536.0 + 0.5) / 65536.0; }

double level_error_constant(const Level1D* L) {
  std::vector<double> S[3], SC[3], dq[3];
  for (int k = 0; k < 3; ++k) {
    const int n = L[k].n;
    S[k].assign(n, 0.0); SC[k].assign(n, 0.0); dq[k].assign(n, 0.0);
    for (int r = 0; r < n; ++r)
      for (int j = 0; j < n; ++j) {
        double q = 0.0;  // Q(r, j) = sum_J I(r, J) P(J, j)
        for (int J = 0; J < L[k].nc; ++J) q += L[k].I(r, J) * L[k].P(J, j);
        S[k][r] += std::fabs(q);
        if (L[k].is_coarse[j]) SC[k][r] += std::fabs(q);
        if (j == r) dq[k][r] = q;
      }
  }
  double best = 0.0;
  for (int a = 0; a < L[0].n; ++a)
    for (int b = 0; b < L[1].n; ++b)
      for (int c = 0; c < L[2].n; ++c) {
        double full = S[0][a] * S[1][b] * S[2][c];
        double coarse = SC[0][a] * SC[1][b] * SC[2][c];
        double v;
        if (L[0].is_coarse[a] && L[1].is_coarse[b] && L[2].is_coarse[c]) {
          v = full - coarse;
        } else {
          double q = dq[0][a] * dq[1][b] * dq[2][c];
          v = full - std::fabs(q) + std::fabs(1.0 - q) - coarse;
        }
        best = std::max(best, v);
      }
  return best;
}

std::vector<double> level_constants(const Plan& p) {  // local 1..K then global 1..M
  std::vector<double> C;
  for (int l = 0; l < p.K; ++l) C.push_back(round_constant(level_error_constant(p.local3[l].data())));
  for (int l = 0; l < p.M; ++l) C.push_back(round_constant(level_error_constant(p.global[l].data())));
  return C;
}

constexpr double kKappa = 8.0;                 // round-off margin factor
constexpr double kEps32 = 5.9604644775390625e-08;  // 2^-24
constexpr double kEps64 = 1.1102230246251565e-16;  // 2^-53

struct Budget {
  std::vector<double> tau;     // per tier, absolute (before the margin)
  double margin = 0.0;
  bool raw = false;            // margin too large for some tier
  std::vector<double> q;       // [tier*K + l] local, then M global, then coarsest
};

// q for one share: delta = tau' / ((N+1) * A), q = 2 delta.
double q_of(double tau_p, int N, double A) {
  double t = (double)(N + 1);
  double denom = t * A;
  double delta = tau_p / denom;
  return 2.0 * delta;
}

Budget make_budget(const Plan& p, const std::vector<double>& tau, double max_abs, bool f64) {
  Budget b;
  b.tau = tau;
  const int N = p.R * p.K + p.M;
  double eps = f64 ? kEps64 : kEps32;
  b.margin = ((kKappa * eps) * (double)(N + 1)) * max_abs;
  std::vector<double> C = level_constants(p);
  double tau_g = INFINITY;
  std::vector<double> taup(tau.size());
  for (size_t t = 0; t < tau.size(); ++t) {
    taup[t] = tau[t] - b.margin;
    if (!(taup[t] > 0.5 * tau[t])) b.raw = true;
    tau_g = std::min(tau_g, taup[t]);
  }
  for (size_t t = 0; t < tau.size(); ++t)
    for (int l = 0; l < p.K; ++l) b.q.push_back(q_of(taup[t], N, C[l]));
  for (int l = 0; l < p.M; ++l) b.q.push_back(q_of(tau_g, N, C[p.K + l]));
  {
    double t = (double)(N + 1);
    b.q.push_back(2.0 * (tau_g / t));
  }
  return b;
}

// ---------------------------------------------------------------------------
// Quantiser (Sec. III-C/III-D): code = floor(c * (1/q) + 1/2), decided in the
// field's precision (fused multiply-add, round to nearest).
// ---------------------------------------------------------------------------
struct QResult { int64_t code; bool overflow; };

QResult quantize(double c, double q, bool f64) {
  QResult r{0, false};
  if (f64) {
    double rq = 1.0 / q;
    double y = std::fma(c, rq, 0.5);
    if (!(std::fabs(y) < 1073741824.0)) { r.overflow = true; return r; }
    r.code = (int64_t)std::floor(y);
  } else {
    float rq = (float)(1.0 / q);
    float cf = (float)c;
    float y = std::fmaf(cf, rq, 0.5f);
    if (!(std::fabs(y) < 1073741824.0f)) { r.overflow = true; return r; }
    r.code = (int64_t)std::floor(y);
  }
  return r;
}

// Index into the q table of every coefficient, in coefficient order: local
// levels use the block's tier, global levels and the coarsest array follow.
std::vector<uint32_t> coeff_q_index(const Plan& p, const std::vector<std::vector<uint8_t>>& block_tier,
                                    int ntiers) {
  std::vector<uint32_t> qi(p.n_coeffs);
  size_t pos = 0;
  for (size_t r = 0; r < p.rounds.size(); ++r)
    for (int64_t b = 0; b < p.rounds[r].nblocks; ++b) {
      int tier = block_tier[r].empty() ? 0 : block_tier[r][(size_t)b];
      for (int l = 0; l < p.K; ++l) {
        size_t cnt = level_detail_count(p.local3[l].data());
        for (size_t t = 0; t < cnt; ++t) qi[pos++] = (uint32_t)(tier * p.K + l);
      }
    }
  for (int l = 0; l < p.M; ++l)
    for (size_t t = 0; t < p.global_counts[l]; ++t) qi[pos++] = (uint32_t)(ntiers * p.K + l);
  for (size_t t = 0; t < p.coarsest; ++t) qi[pos++] = (uint32_t)(ntiers * p.K + p.M);
  return qi;
}

// ---------------------------------------------------------------------------
// Huffman coding (Sec. III-B lossless stage; cuSZ-style chunked "deflate" =
// concatenation of codes, no zlib)
// ---------------------------------------------------------------------------
// Code lengths by the two-queue Huffman construction: leaves sorted by
// (frequency, symbol); on equal weight a leaf is taken before an internal
// node; internal nodes are taken in creation order.  One present symbol gets
// length 1.  If the longest code exceeds 32 bits, frequencies are replaced by
// max(1, f >> t) for t = 1, 2, ... until it fits.
std::vector<uint8_t> huffman_lengths_once(const std::vector<uint64_t>& freq, int* maxlen) {
  const int S = (int)freq.size();
  std::vector<uint8_t> len(S, 0);
  std::vector<int> leaves;
  for (int s = 0; s < S; ++s)
    if (freq[s] > 0) leaves.push_back(s);
  *maxlen = 0;
  if (leaves.empty()) return len;
  if (leaves.size() == 1) { len[leaves[0]] = 1; *maxlen = 1; return len; }
  std::stable_sort(leaves.begin(), leaves.end(), [&](int a, int b) { return freq[a] < freq[b]; });
  const int n = (int)leaves.size();
  // nodes 0..n-1 = leaves (in sorted order), n.. = internal nodes
  std::vector<uint64_t> w(2 * n - 1);
  std::vector<int> parent(2 * n - 1, -1);
  for (int i = 0; i < n; ++i) w[i] = freq[leaves[i]];
  int lp = 0, qp = n, qe = n;
  auto take = [&]() {
    if (lp < n && (qp >= qe || w[lp] <= w[qp])) return lp++;
    return qp++;
  };
  while (qe < 2 * n - 1) {
    int a = take();
    int b = take();
    w[qe] = w[a] + w[b];
    parent[a] = qe;
    parent[b] = qe;
    ++qe;
  }
  std::vector<int> depth(2 * n - 1, 0);
  for (int v = 2 * n - 3; v >= 0; --v) depth[v] = depth[parent[v]] + 1;
  for (int i = 0; i < n; ++i) {
    len[leaves[i]] = (uint8_t)std::min(depth[i], 255);
    *maxlen = std::max(*maxlen, depth[i]);
  }
  return len;
}

std::vector<uint8_t> huffman_lengths(const std::vector<uint64_t>& freq) {
  int maxlen = 0;
  std::vector<uint8_t> len = huffman_lengths_once(freq, &maxlen);
  for (int t = 1; maxlen > 32; ++t) {
    std::vector<uint64_t> f2(freq.size());
    for (size_t s = 0; s < freq.size(); ++s) f2[s] = freq[s] ? std::max<uint64_t>(1, freq[s] >> t) : 0;
    len = huffman_lengths_once(f2, &maxlen);
  }
  return len;
}

// Canonical codes: symbols ordered by (length, symbol), consecutive code values.
std::vector<uint32_t> canonical_codes(const std::vector<uint8_t>& len) {
  std::vector<uint32_t> code(len.size(), 0);
  std::vector<int> order;
  for (size_t s = 0; s < len.size(); ++s)
    if (len[s]) order.push_back((int)s);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return len[a] < len[b]; });
  uint64_t c = 0;
  int prev = order.empty() ? 0 : len[order[0]];
  for (size_t i = 0; i < order.size(); ++i) {
    int L = len[order[i]];
    if (i > 0) c = (c + 1) << (L - prev);
    code[order[i]] = (uint32_t)c;
    prev = L;
  }
  return code;
}

// ---------------------------------------------------------------------------
// Byte stream.  A 256-byte header (magic, flags, shape, parameters, counts and
// the byte offset of every section), then, each padded to 8 bytes: tolerance
// tiers (f64), q table (f64), block tiers (u8, only with several tiers), chunk
// word counts (u32), split offsets (u16, 7 per chunk), codebook runs, escape
// counts per chunk (u32, only with outliers), outlier codes (i32), bitstream
// (u32 words).  A raw stream is the header followed by the field.
// ---------------------------------------------------------------------------
constexpr uint32_t kMagic = 0x31474D42u;  // "BMG1"
constexpr size_t kHeader = 256;

struct Writer {
  std::vector<uint8_t> b;
  void pad8() { while (b.size() % 8) b.push_back(0); }
  void pad4() { while (b.size() % 4) b.push_back(0); }
  template <class T> void put(const T& v) {
    const uint8_t* p = reinterpret_cast<const uint8_t*>(&v);
    b.insert(b.end(), p, p + sizeof(T));
  }
  template <class T> void put_at(size_t off, const T& v) { std::memcpy(b.data() + off, &v, sizeof(T)); }
};

// The Huffman section: codebook runs, chunk word counts, bitstream.
struct HuffOut {
  std::vector<uint8_t> codebook;  // runs {u32 first, u32 count, u8 len[count], pad4}
  uint32_t n_runs = 0;
  std::vector<uint32_t> chunk_words;
  std::vector<uint32_t> chunk_esc;  // symbols 0 (escapes) per chunk
  std::vector<uint16_t> splits;     // per chunk: bit offsets of its eighths 1..7 from the chunk start
  std::vector<uint32_t> words;
};

// A chunk is split into eight equal runs of chunk/8 symbols; the stream keeps
// where runs 1..7 start so a decoder can work on the eight runs in parallel.
constexpr int kSplits = 8;

HuffOut huffman_encode(const uint16_t* sym, size_t n, int dict, int chunk) {
  HuffOut h;
  std::vector<uint64_t> freq(dict, 0);
  for (size_t i = 0; i < n; ++i) freq[sym[i]]++;
  std::vector<uint8_t> len = huffman_lengths(freq);
  std::vector<uint32_t> code = canonical_codes(len);
  for (int s = 0; s < dict;) {
    if (!len[s]) { ++s; continue; }
    int e = s;
    while (e < dict && len[e]) ++e;
    Writer w;
    w.put<uint32_t>((uint32_t)s);
    w.put<uint32_t>((uint32_t)(e - s));
    for (int t = s; t < e; ++t) w.put<uint8_t>(len[t]);
    w.pad4();
    h.codebook.insert(h.codebook.end(), w.b.begin(), w.b.end());
    h.n_runs++;
    s = e;
  }
  size_t nchunks = (n + chunk - 1) / chunk;
  for (size_t c = 0; c < nchunks; ++c) {
    size_t s0 = c * chunk, s1 = std::min(n, s0 + (size_t)chunk);
    uint64_t bitpos = 0;
    std::vector<uint32_t> cw;
    uint32_t nesc = 0;
    const size_t sub = std::max<size_t>(1, (size_t)chunk / kSplits);
    uint16_t split[kSplits] = {};
    for (size_t i = s0; i < s1; ++i) {
      if ((i - s0) % sub == 0 && (i - s0) / sub > 0) split[(i - s0) / sub] = (uint16_t)bitpos;
      nesc += sym[i] == 0;
      int L = len[sym[i]];
      uint32_t cd = code[sym[i]];
      for (int t = L - 1; t >= 0; --t) {  // MSB first
        uint32_t bit = (cd >> t) & 1u;
        size_t wi = bitpos / 32;
        if (wi >= cw.size()) cw.push_back(0);
        if (bit) cw[wi] |= 1u << (31 - (bitpos % 32));
        ++bitpos;
      }
    }
    // runs past the end of a short last chunk start where the chunk ends
    for (int k = 1; k < kSplits; ++k)
      if (s0 + k * sub >= s1) split[k] = (uint16_t)bitpos;
    for (int k = 1; k < kSplits; ++k) h.splits.push_back(split[k]);
    h.chunk_words.push_back((uint32_t)cw.size());
    h.chunk_esc.push_back(nesc);
    h.words.insert(h.words.end(), cw.begin(), cw.end());
  }
  return h;
}

// Read back runs into a length table.
bool parse_codebook(const uint8_t* p, size_t nbytes, uint32_t n_runs, int dict, std::vector<uint8_t>& len) {
  len.assign(dict, 0);
  size_t off = 0;
  for (uint32_t r = 0; r < n_runs; ++r) {
    if (off + 8 > nbytes) return false;
    uint32_t first, count;
    std::memcpy(&first, p + off, 4);
    std::memcpy(&count, p + off + 4, 4);
    off += 8;
    if ((uint64_t)first + count > (uint64_t)dict || off + count > nbytes) return false;
    for (uint32_t t = 0; t < count; ++t) len[first + t] = p[off + t];
    off += (count + 3) & ~3u;
  }
  return true;
}

bool huffman_decode(const std::vector<uint8_t>& len, const uint32_t* chunk_words, const uint32_t* words,
                    uint64_t n_words, uint16_t* out, size_t n, int chunk) {
  std::vector<uint32_t> code = canonical_codes(len);
  // Decode by brute-force matching of (length, code) pairs: slow and simple.
  std::vector<std::vector<std::pair<uint32_t, int>>> by_len(33);
  for (size_t s = 0; s < len.size(); ++s)
    if (len[s]) {
      if (len[s] > 32) return false;
      by_len[len[s]].push_back({code[s], (int)s});
    }
  for (auto& v : by_len) std::sort(v.begin(), v.end());
  size_t nchunks = (n + chunk - 1) / chunk;
  uint64_t wbase = 0;
  for (size_t c = 0; c < nchunks; ++c) {
    size_t s0 = c * chunk, s1 = std::min(n, s0 + (size_t)chunk);
    uint64_t nw = chunk_words[c];
    if (wbase + nw > n_words) return false;
    uint64_t bitpos = 0, nbits = nw * 32;
    for (size_t i = s0; i < s1; ++i) {
      uint32_t cur = 0;
      int L = 0;
      int found = -1;
      while (found < 0) {
        if (bitpos >= nbits || L >= 32) return false;
        uint32_t w = words[wbase + bitpos / 32];
        uint32_t bit = (w >> (31 - (bitpos % 32))) & 1u;
        ++bitpos;
        cur = (cur << 1) | bit;
        ++L;
        auto& v = by_len[L];
        auto it = std::lower_bound(v.begin(), v.end(), std::make_pair(cur, -1));
        if (it != v.end() && it->first == cur) found = it->second;
      }
      out[i] = (uint16_t)found;
    }
    wbase += nw;
  }
  return true;
}

struct CompressOpts {
  int B = 9, K = 1, M = 2, chunk = 2048, radius = 32768, R = 1;
  int ndim = 3;  // dimensions of the caller's field (the shape holds it with leading extents of 1)
};

thread_local std::string g_err;

// Full compression of an FP64 copy of the field (f64 says what the original dtype was).
std::vector<uint8_t> compress(const double* u, const int64_t* shape, bool f64, double tol, int rel,
                              const double* roi, const CompressOpts& o, std::vector<int64_t>* codes_out) {
  Plan p = make_plan(shape, o.B, o.K, o.M, o.R);
  const size_t nel = (size_t)(shape[0] * shape[1] * shape[2]);
  double max_abs = 0.0;
  bool finite = true;
  for (size_t i = 0; i < nel; ++i) {
    if (!std::isfinite(u[i])) finite = false;
    max_abs = std::max(max_abs, std::fabs(u[i]));
  }
  // Per-block tolerances min(tol, roi_i), deduplicated into ascending tiers;
  // a tier's absolute tolerance is its value times max|u| in REL mode.
  std::vector<double> btau((size_t)p.nblocks);
  for (int64_t b = 0; b < p.nblocks; ++b) {
    double t = tol;
    if (roi) t = std::min(t, roi[b]);
    btau[(size_t)b] = t;
  }
  std::vector<double> tiers = btau;
  std::sort(tiers.begin(), tiers.end());
  tiers.erase(std::unique(tiers.begin(), tiers.end()), tiers.end());
  if (tiers.size() > 255) throw std::runtime_error("more than 255 distinct tolerances");
  std::vector<uint8_t> block_tier((size_t)p.nblocks);
  for (int64_t b = 0; b < p.nblocks; ++b)
    block_tier[(size_t)b] = (uint8_t)(std::lower_bound(tiers.begin(), tiers.end(), btau[(size_t)b]) - tiers.begin());
  if (rel)
    for (double& t : tiers) t = t * max_abs;
  const int ntiers = (int)tiers.size();
  Budget bud = make_budget(p, tiers, max_abs, f64);
  bool raw = bud.raw || !finite;

  std::vector<uint16_t> sym;
  std::vector<int32_t> out_code;  // codes of the escaped symbols, in stream order
  if (!raw) {
    std::vector<double> coef = decompose(u, p);
    std::vector<uint32_t> qi = coeff_q_index(p, round_tiers(p, ntiers > 1 ? block_tier : std::vector<uint8_t>()), ntiers);
    sym.resize(p.n_coeffs);
    if (codes_out) codes_out->resize(p.n_coeffs);
    for (size_t i = 0; i < p.n_coeffs && !raw; ++i) {
      QResult r = quantize(coef[i], bud.q[qi[i]], f64);
      if (r.overflow) { raw = true; break; }
      if (codes_out) (*codes_out)[i] = r.code;
      if (r.code > -o.radius && r.code < o.radius) {
        sym[i] = (uint16_t)(r.code + o.radius);
      } else {
        sym[i] = 0;
        out_code.push_back((int32_t)r.code);
      }
    }
  }
  const size_t esize = f64 ? 8 : 4;
  Writer w;
  w.b.assign(kHeader, 0);
  w.put_at<uint32_t>(0, kMagic);
  w.put_at<uint16_t>(4, 1);
  w.put_at<int32_t>(8, o.ndim);
  w.put_at<int32_t>(12, o.B);
  for (int d = 0; d < 3; ++d) w.put_at<int64_t>(16 + 8 * d, shape[d]);
  w.put_at<double>(80, max_abs);
  w.put_at<double>(88, tol);
  w.put_at<int32_t>(76, rel);
  auto finish_raw = [&]() {
    w.b.assign(kHeader, 0);
    w.put_at<uint32_t>(0, kMagic);
    w.put_at<uint16_t>(4, 1);
    w.put_at<uint16_t>(6, (uint16_t)(1 | (f64 ? 2 : 0)));
    w.put_at<int32_t>(8, o.ndim);
    w.put_at<int32_t>(12, o.B);
    for (int d = 0; d < 3; ++d) w.put_at<int64_t>(16 + 8 * d, shape[d]);
    w.put_at<int32_t>(76, rel);
    w.put_at<double>(80, max_abs);
    w.put_at<double>(88, tol);
    for (size_t i = 0; i < nel; ++i) {
      if (f64) w.put<double>(u[i]);
      else w.put<float>((float)u[i]);
    }
    w.put_at<uint64_t>(168, (uint64_t)kHeader);
    w.put_at<uint64_t>(184, (uint64_t)w.b.size());
    return w.b;
  };
  if (raw) return finish_raw();

  HuffOut h = huffman_encode(sym.data(), sym.size(), 2 * o.radius, o.chunk);
  w.put_at<uint16_t>(6, (uint16_t)(f64 ? 2 : 0));
  w.put_at<int32_t>(40, o.K);
  w.put_at<int32_t>(44, o.M);
  w.put_at<int32_t>(48, o.chunk);
  w.put_at<int32_t>(52, o.radius);
  w.put_at<int32_t>(56, ntiers);
  w.put_at<int32_t>(60, p.m);
  for (int d = 0; d < 3; ++d) w.put_at<int32_t>(64 + 4 * d, (int32_t)p.nb[d]);
  w.put_at<uint64_t>(96, (uint64_t)sym.size());
  w.put_at<uint64_t>(104, (uint64_t)h.chunk_words.size());
  w.put_at<uint64_t>(112, (uint64_t)out_code.size());
  w.put_at<uint64_t>(120, (uint64_t)h.words.size());
  w.put_at<uint32_t>(192, (uint32_t)h.codebook.size());
  w.put_at<uint32_t>(196, h.n_runs);
  w.put_at<double>(200, bud.margin);
  w.put_at<uint32_t>(224, (uint32_t)(o.R - 1));
  w.put_at<uint64_t>(128, (uint64_t)w.b.size());
  for (double t : tiers) w.put<double>(t);
  w.pad8();
  w.put_at<uint64_t>(136, (uint64_t)w.b.size());
  for (double q : bud.q) w.put<double>(q);
  w.pad8();
  w.put_at<uint64_t>(144, (uint64_t)w.b.size());
  if (ntiers > 1)
    for (const auto& rt : round_tiers(p, block_tier))
      for (uint8_t t : rt) w.put<uint8_t>(t);
  w.pad8();
  w.put_at<uint64_t>(152, (uint64_t)w.b.size());
  for (uint32_t c : h.chunk_words) w.put<uint32_t>(c);
  w.pad8();
  w.put_at<uint64_t>(216, (uint64_t)w.b.size());
  for (uint16_t v : h.splits) w.put<uint16_t>(v);
  w.pad8();
  w.put_at<uint64_t>(160, (uint64_t)w.b.size());
  w.b.insert(w.b.end(), h.codebook.begin(), h.codebook.end());
  w.pad8();
  // escape counts per chunk, present only when there are outliers
  w.put_at<uint64_t>(208, (uint64_t)w.b.size());
  if (!out_code.empty())
    for (uint32_t c : h.chunk_esc) w.put<uint32_t>(c);
  w.pad8();
  w.put_at<uint64_t>(176, (uint64_t)w.b.size());
  for (int32_t x : out_code) w.put<int32_t>(x);
  w.pad8();
  // the bitstream comes last: every offset before it follows from the
  // codebook and the number of outliers alone
  w.put_at<uint64_t>(168, (uint64_t)w.b.size());
  for (uint32_t x : h.words) w.put<uint32_t>(x);
  w.pad8();
  w.put_at<uint64_t>(184, (uint64_t)w.b.size());
  if (w.b.size() >= kHeader + nel * esize) return finish_raw();
  return w.b;
}

template <class T> T rd(const uint8_t* p, size_t off) { T v; std::memcpy(&v, p + off, sizeof(T)); return v; }

// Decompression to FP64; the caller rounds to the original dtype.
bool decompress(const uint8_t* s, size_t nbytes, std::vector<double>& u, int64_t shape[3], bool* f64,
                std::vector<int64_t>* codes_out) {
  if (nbytes < kHeader || rd<uint32_t>(s, 0) != kMagic) { g_err = "bad magic"; return false; }
  uint16_t flags = rd<uint16_t>(s, 6);
  *f64 = (flags & 2) != 0;
  for (int d = 0; d < 3; ++d) shape[d] = rd<int64_t>(s, 16 + 8 * d);
  const size_t nel = (size_t)(shape[0] * shape[1] * shape[2]);
  const size_t esize = *f64 ? 8 : 4;
  if (rd<uint64_t>(s, 184) != nbytes) { g_err = "length mismatch"; return false; }
  u.assign(nel, 0.0);
  if (flags & 1) {
    if (nbytes != kHeader + nel * esize) { g_err = "raw size"; return false; }
    for (size_t i = 0; i < nel; ++i)
      u[i] = *f64 ? rd<double>(s, kHeader + 8 * i) : (double)rd<float>(s, kHeader + 4 * i);
    return true;
  }
  CompressOpts o;
  o.B = rd<int32_t>(s, 12);
  o.K = rd<int32_t>(s, 40);
  o.M = rd<int32_t>(s, 44);
  o.chunk = rd<int32_t>(s, 48);
  o.radius = rd<int32_t>(s, 52);
  int ntiers = rd<int32_t>(s, 56);
  o.R = (int)rd<uint32_t>(s, 224) + 1;
  if (o.R > 16) { g_err = "rounds"; return false; }
  Plan p = make_plan(shape, o.B, o.K, o.M, o.R);
  uint64_t nsym = rd<uint64_t>(s, 96), nch = rd<uint64_t>(s, 104), nout = rd<uint64_t>(s, 112),
           nwords = rd<uint64_t>(s, 120);
  if (nsym != p.n_coeffs) { g_err = "symbol count"; return false; }
  const double* q = reinterpret_cast<const double*>(s + rd<uint64_t>(s, 136));
  std::vector<double> qv(q, q + (size_t)ntiers * o.K + o.M + 1);
  std::vector<std::vector<uint8_t>> block_tier(p.rounds.size());
  if (ntiers > 1) {
    const uint8_t* bt = s + rd<uint64_t>(s, 144);
    for (size_t r = 0; r < p.rounds.size(); ++r) {
      block_tier[r].assign(bt, bt + p.rounds[r].nblocks);
      bt += p.rounds[r].nblocks;
    }
  }
  std::vector<uint32_t> chunk_words(nch);
  std::memcpy(chunk_words.data(), s + rd<uint64_t>(s, 152), nch * 4);
  std::vector<uint8_t> len;
  if (!parse_codebook(s + rd<uint64_t>(s, 160), rd<uint32_t>(s, 192), rd<uint32_t>(s, 196), 2 * o.radius, len)) {
    g_err = "codebook";
    return false;
  }
  std::vector<uint32_t> words(nwords);
  std::memcpy(words.data(), s + rd<uint64_t>(s, 168), nwords * 4);
  std::vector<uint16_t> sym(nsym);
  if (!huffman_decode(len, chunk_words.data(), words.data(), nwords, sym.data(), nsym, o.chunk)) {
    g_err = "bitstream";
    return false;
  }
  // escaped symbols take the outlier codes in stream order
  std::vector<int64_t> code(nsym);
  size_t ooff = rd<uint64_t>(s, 176);
  uint64_t next = 0;
  for (size_t i = 0; i < nsym; ++i) {
    if (sym[i]) {
      code[i] = (int64_t)sym[i] - o.radius;
    } else {
      if (next >= nout) { g_err = "more escapes than outliers"; return false; }
      code[i] = rd<int32_t>(s, ooff + 4 * next);
      ++next;
    }
  }
  if (next != nout) { g_err = "outlier count"; return false; }
  if (codes_out) *codes_out = code;
  std::vector<uint32_t> qi = coeff_q_index(p, block_tier, ntiers);
  std::vector<double> coef(nsym);
  for (size_t i = 0; i < nsym; ++i) coef[i] = (double)code[i] * qv[qi[i]];
  u = recompose(coef.data(), p);
  return true;
}

}  // namespace

// ===========================================================================
// extern "C" surface used by tests/ through ctypes
// ===========================================================================
extern "C" {

const char* or_last_error() { return g_err.c_str(); }

// 1-D operator matrices for coordinates x[0..n): I (n*nc), Mf (n*n), Mc (nc*nc), P (nc*n).
int or_level_1d(int n, const double* x, double* I, double* Mf, double* Mc, double* P, int* nc) {
  std::vector<double> xv(x, x + n);
  Level1D L = make_level(xv);
  *nc = L.nc;
  if (I) std::memcpy(I, L.I.a.data(), L.I.a.size() * 8);
  if (Mf) std::memcpy(Mf, L.Mf.a.data(), L.Mf.a.size() * 8);
  if (Mc) std::memcpy(Mc, L.Mc.a.data(), L.Mc.a.size() * 8);
  if (P) std::memcpy(P, L.P.a.data(), L.P.a.size() * 8);
  return 0;
}

// Sizes of the hierarchy: out[0]=n_coeffs, [1]=per_block, [2]=nblocks, [3]=m,
// [4..6]=gathered grid, [7..9]=coarsest grid, [10]=coarsest count,
// [11..11+M) = global level counts.
int or_plan_r(const int64_t* shape, int B, int K, int M, int R, int64_t* out) {
  try {
    Plan p = make_plan(shape, B, K, M, R);
    out[0] = (int64_t)p.n_coeffs;
    out[1] = (int64_t)p.per_block;
    out[2] = p.nblocks;
    out[3] = p.m;
    for (int d = 0; d < 3; ++d) { out[4 + d] = p.gshape[d]; out[7 + d] = p.cshape[d]; }
    out[10] = (int64_t)p.coarsest;
    for (int l = 0; l < M; ++l) out[11 + l] = (int64_t)p.global_counts[l];
    return 0;
  } catch (const std::exception& e) { g_err = e.what(); return 1; }
}

int or_plan(const int64_t* shape, int B, int K, int M, int64_t* out) { return or_plan_r(shape, B, K, M, 1, out); }

// Blocks of every round (out[r]) and the tiers of every round's blocks
// propagated from round 0's (tier_out, concatenated; only if tier0 != null).
int or_rounds(const int64_t* shape, int B, int K, int R, const uint8_t* tier0, int64_t* nblocks_out,
              uint8_t* tier_out) {
  try {
    Plan p = make_plan(shape, B, K, 0, R);
    for (int r = 0; r < R; ++r) nblocks_out[r] = p.rounds[(size_t)r].nblocks;
    if (tier0 && tier_out) {
      std::vector<uint8_t> t0(tier0, tier0 + p.nblocks);
      size_t o = 0;
      for (const auto& rt : round_tiers(p, t0)) {
        std::memcpy(tier_out + o, rt.data(), rt.size());
        o += rt.size();
      }
    }
    return 0;
  } catch (const std::exception& e) { g_err = e.what(); return 1; }
}

int or_decompose_r(const double* u, const int64_t* shape, int B, int K, int M, int R, double* coef_out) {
  try {
    Plan p = make_plan(shape, B, K, M, R);
    std::vector<double> c = decompose(u, p);
    std::memcpy(coef_out, c.data(), c.size() * 8);
    return 0;
  } catch (const std::exception& e) { g_err = e.what(); return 1; }
}

int or_decompose(const double* u, const int64_t* shape, int B, int K, int M, double* coef_out) {
  return or_decompose_r(u, shape, B, K, M, 1, coef_out);
}

int or_recompose_r(const double* coef, const int64_t* shape, int B, int K, int M, int R, double* u_out) {
  try {
    Plan p = make_plan(shape, B, K, M, R);
    std::vector<double> u = recompose(coef, p);
    std::memcpy(u_out, u.data(), u.size() * 8);
    return 0;
  } catch (const std::exception& e) { g_err = e.what(); return 1; }
}

int or_recompose(const double* coef, const int64_t* shape, int B, int K, int M, double* u_out) {
  return or_recompose_r(coef, shape, B, K, M, 1, u_out);
}

// Coefficients of one block (its K local levels, in stream order) and its m^3 coarse values.
int or_block_coeffs(const double* u, const int64_t* shape, int B, int K, int64_t block, double* coef_out,
                    double* coarse_out) {
  try {
    Plan p = make_plan(shape, B, K, 0);
    int64_t b2 = block % p.nb[2], b1 = (block / p.nb[2]) % p.nb[1], b0 = block / (p.nb[1] * p.nb[2]);
    Grid blk(B, B, B);
    for (int i = 0; i < B; ++i)
      for (int j = 0; j < B; ++j)
        for (int k = 0; k < B; ++k) {
          int64_t gi = b0 * B + i, gj = b1 * B + j, gk = b2 * B + k;
          bool in = gi < shape[0] && gj < shape[1] && gk < shape[2];
          blk.at(i, j, k) = in ? u[(gi * shape[1] + gj) * shape[2] + gk] : 0.0;
        }
    std::vector<double> coef;
    for (int l = 0; l < K; ++l) {
      Level1D L3[3] = {p.local[l], p.local[l], p.local[l]};
      blk = decompose_level(blk, L3, coef);
    }
    std::memcpy(coef_out, coef.data(), coef.size() * 8);
    if (coarse_out) std::memcpy(coarse_out, blk.v.data(), blk.v.size() * 8);
    return 0;
  } catch (const std::exception& e) { g_err = e.what(); return 1; }
}

// Level constants C_l (rounded), local 1..K then global 1..M.
int or_level_constants(const int64_t* shape, int B, int K, int M, double* out) {
  try {
    Plan p = make_plan(shape, B, K, M);
    std::vector<double> C = level_constants(p);
    std::memcpy(out, C.data(), C.size() * 8);
    return 0;
  } catch (const std::exception& e) { g_err = e.what(); return 1; }
}

// Quantiser widths for tiers tau[0..ntiers): out = [tier*K + l], M global, coarsest;
// meta[0] = margin, meta[1] = raw flag.
int or_budget_r(const int64_t* shape, int B, int K, int M, int R, const double* tau, int ntiers, double max_abs,
                int f64, double* q_out, double* meta) {
  try {
    Plan p = make_plan(shape, B, K, M, R);
    std::vector<double> t(tau, tau + ntiers);
    Budget b = make_budget(p, t, max_abs, f64 != 0);
    std::memcpy(q_out, b.q.data(), b.q.size() * 8);
    meta[0] = b.margin;
    meta[1] = b.raw ? 1.0 : 0.0;
    return 0;
  } catch (const std::exception& e) { g_err = e.what(); return 1; }
}

int or_budget(const int64_t* shape, int B, int K, int M, const double* tau, int ntiers, double max_abs, int f64,
              double* q_out, double* meta) {
  return or_budget_r(shape, B, K, M, 1, tau, ntiers, max_abs, f64, q_out, meta);
}

int64_t or_quantize(double c, double q, int f64, int* overflow) {
  QResult r = quantize(c, q, f64 != 0);
  *overflow = r.overflow ? 1 : 0;
  return r.code;
}

// The quantiser applied element by element (codes of given coefficients and
// bin widths; overflowing entries are reported through their own flag).
int or_quantize_array(const double* c, const double* q, int64_t n, int f64, int64_t* code_out, uint8_t* ovf_out) {
  for (int64_t i = 0; i < n; ++i) {
    QResult r = quantize(c[i], q[i], f64 != 0);
    code_out[i] = r.code;
    ovf_out[i] = r.overflow ? 1 : 0;
  }
  return 0;
}

int or_huffman_lengths(const uint64_t* freq, int nsym, uint8_t* len_out) {
  std::vector<uint64_t> f(freq, freq + nsym);
  std::vector<uint8_t> l = huffman_lengths(f);
  std::memcpy(len_out, l.data(), l.size());
  return 0;
}

int or_canonical_codes(const uint8_t* len, int nsym, uint32_t* code_out) {
  std::vector<uint8_t> l(len, len + nsym);
  std::vector<uint32_t> c = canonical_codes(l);
  std::memcpy(code_out, c.data(), c.size() * 4);
  return 0;
}

// Huffman section for symbols sym[0..n): chunk word counts, split offsets,
// codebook runs, bitstream, concatenated in that order (each padded to 8
// bytes), the order these parts take inside a stream.
// sizes[0..3] = codebook bytes, n_runs, n_chunks, n_words.
int or_huffman_encode(const uint16_t* sym, uint64_t n, int dict, int chunk, uint8_t* out, uint64_t cap,
                      uint64_t* sizes) {
  HuffOut h = huffman_encode(sym, n, dict, chunk);
  Writer w;
  for (uint32_t c : h.chunk_words) w.put<uint32_t>(c);
  w.pad8();
  for (uint16_t v : h.splits) w.put<uint16_t>(v);
  w.pad8();
  w.b.insert(w.b.end(), h.codebook.begin(), h.codebook.end());
  w.pad8();
  for (uint32_t x : h.words) w.put<uint32_t>(x);
  w.pad8();
  sizes[0] = h.codebook.size();
  sizes[1] = h.n_runs;
  sizes[2] = h.chunk_words.size();
  sizes[3] = h.words.size();
  sizes[4] = w.b.size();
  if (w.b.size() > cap) { g_err = "capacity"; return 1; }
  std::memcpy(out, w.b.data(), w.b.size());
  return 0;
}

int or_huffman_decode(const uint8_t* codebook, uint64_t cb_bytes, uint32_t n_runs, int dict, const uint32_t* chunk_words,
                      const uint32_t* words, uint64_t n_words, uint64_t n, int chunk, uint16_t* out) {
  std::vector<uint8_t> len;
  if (!parse_codebook(codebook, cb_bytes, n_runs, dict, len)) { g_err = "codebook"; return 1; }
  return huffman_decode(len, chunk_words, words, n_words, out, n, chunk) ? 0 : 1;
}

// Compress a field given as FP64 values (dtype_f64 = 1 if the original is FP64).
// roi may be null (one tolerance per block otherwise). codes_out (optional,
// n_coeffs entries) receives the integer codes.
// The same for a field of ndim (1..3) dimensions, held in `shape` as a 3-D
// shape with leading extents of 1; the header records ndim.
int or_compress_nd(const double* u, const int64_t* shape, int ndim, int dtype_f64, double tol, int rel,
                   const double* roi, int B, int K, int M, int R, int chunk, int radius, uint8_t* out, uint64_t cap,
                   uint64_t* out_bytes, int64_t* codes_out) {
  try {
    if (ndim < 1 || ndim > 3) throw std::runtime_error("ndim must be 1, 2 or 3");
    for (int d = 0; d < 3 - ndim; ++d)
      if (shape[d] != 1) throw std::runtime_error("leading extents of a field with fewer than 3 dimensions must be 1");
    CompressOpts o;
    o.B = B; o.K = K; o.M = M; o.R = R; o.chunk = chunk; o.radius = radius; o.ndim = ndim;
    std::vector<int64_t> codes;
    std::vector<uint8_t> s = compress(u, shape, dtype_f64 != 0, tol, rel, roi, o, codes_out ? &codes : nullptr);
    *out_bytes = s.size();
    if (s.size() > cap) { g_err = "capacity"; return 2; }
    std::memcpy(out, s.data(), s.size());
    if (codes_out && !codes.empty()) std::memcpy(codes_out, codes.data(), codes.size() * 8);
    return 0;
  } catch (const std::exception& e) { g_err = e.what(); return 1; }
}

int or_compress_r(const double* u, const int64_t* shape, int dtype_f64, double tol, int rel, const double* roi, int B,
                  int K, int M, int R, int chunk, int radius, uint8_t* out, uint64_t cap, uint64_t* out_bytes,
                  int64_t* codes_out) {
  try {
    CompressOpts o;
    o.B = B; o.K = K; o.M = M; o.R = R; o.chunk = chunk; o.radius = radius;
    std::vector<int64_t> codes;
    std::vector<uint8_t> s = compress(u, shape, dtype_f64 != 0, tol, rel, roi, o, codes_out ? &codes : nullptr);
    *out_bytes = s.size();
    if (s.size() > cap) { g_err = "capacity"; return 2; }
    std::memcpy(out, s.data(), s.size());
    if (codes_out && !codes.empty()) std::memcpy(codes_out, codes.data(), codes.size() * 8);
    return 0;
  } catch (const std::exception& e) { g_err = e.what(); return 1; }
}

int or_compress(const double* u, const int64_t* shape, int dtype_f64, double tol, int rel, const double* roi, int B,
                int K, int M, int chunk, int radius, uint8_t* out, uint64_t cap, uint64_t* out_bytes,
                int64_t* codes_out) {
  return or_compress_r(u, shape, dtype_f64, tol, rel, roi, B, K, M, 1, chunk, radius, out, cap, out_bytes, codes_out);
}

// Decompress into FP64 values u_out (shape from the header); codes_out optional.
int or_decompress(const uint8_t* s, uint64_t n, double* u_out, int64_t* codes_out) {
  try {
    std::vector<double> u;
    int64_t shape[3];
    bool f64;
    std::vector<int64_t> codes;
    if (!decompress(s, n, u, shape, &f64, codes_out ? &codes : nullptr)) return 1;
    std::memcpy(u_out, u.data(), u.size() * 8);
    if (codes_out && !codes.empty()) std::memcpy(codes_out, codes.data(), codes.size() * 8);
    return 0;
  } catch (const std::exception& e) { g_err = e.what(); return 1; }
}

}  // extern "C"

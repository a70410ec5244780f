// Host-side plan of one hierarchy: sizes, stream-order offsets, the tables of
// the global levels and the level error constants.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace bm {

// One dimension of one global level, in double precision (converted to the
// field's dtype when uploaded).
struct Dim1DHost {
  int n = 0, c = 0;
  std::vector<double> x;       // node coordinates
  std::vector<int> cidx, jlo, jhi, cb, f0;
  std::vector<uint8_t> isc;
  std::vector<double> wl, wr;  // interpolation weights
  std::vector<double> band;    // [5c] rows of I^T M_f
  std::vector<double> tm, tib, tsup;  // Thomas factors of M_c
  std::vector<double> md, mo;  // M_f: diagonal, and mo[i] = M_f(i, i+1) (adjoint passes)
  std::vector<double> P;       // [c x n] row-major: M_c^{-1} I^T M_f (global levels)
};

// One re-blocking round: B-node blocks over the round's input grid (the field
// for round 0, the previous round's gathered coarse grid after that).
struct RoundHost {
  int64_t shape[3];  // input grid
  int nb[3];
  int64_t nblocks;
  int64_t off;       // first coefficient of the round
  int64_t gshape[3]; // gathered coarse grid (nb * m)
};

// One in-cache level of a field with a dimension of extent 1, run on the
// block-major grid (block, a, b): the block index is an identity dimension
// (not tabulated), a and b the block's two remaining axes (a has one node for
// a 1-D field).
struct RLevelHost {
  int64_t nblk;                 // blocks (identity dimension)
  Dim1DHost da, db;             // the level's operators along the in-block axes
  int64_t off;                  // first symbol of the level inside block 0
  int64_t blk_extra;            // per block: symbols of the other levels (block-major order)
};

// One in-cache level of one round of a field whose block size has no fused
// block kernel, run on the zero-padded grid of the round's blocks: along
// every dimension the level operator is block-diagonal (nb segments of the
// block-local level), which makes the whole-grid passes the blockwise
// transform; the coarse part after the last level is the gathered grid.
struct XLevelHost {
  int64_t shape[3];             // padded grid of the level (nb * block extent of the level)
  Dim1DHost d[3];               // block-diagonal operators
  int e[3], ce[3], nb[3];       // per dimension: block extent, its coarse count, blocks
  int64_t sym_off;              // first symbol of the level inside the round's first block
};

struct PlanHost {
  int64_t shape[3];
  int B, K, M, R;
  bool generic = false;         // no fused block kernel for B: in-cache levels as padded whole-grid passes
  std::vector<std::vector<XLevelHost>> xlev;  // [round][level] (generic only)
  int Bd[3];         // block edge per dimension: B, or 1 for a dimension of extent 1
  int md[3];         // coarse nodes per block edge after K levels, per dimension
  bool reduced = false;         // some dimension has extent 1: in-cache levels on the block-major grid
  int ax[2] = {-1, -1};         // field dimensions of the block-major grid's axes a and b (-1: one node)
  std::vector<RLevelHost> rlev; // [K] (reduced only)
  int nb[3];         // round 0
  int64_t nblocks;   // round 0
  std::vector<RoundHost> rounds;
  int64_t nblocks_all;  // blocks of all rounds
  int m;                 // coarse nodes per block edge after K levels
  int64_t per_block;
  int64_t gshape[3];     // gathered grid of the last round (the global levels' input)
  std::vector<int64_t> lshape;  // [3*(M+1)]: grid of global level l (l = 0 is G), last = coarsest
  std::vector<int64_t> sym_off; // [M+2]: first symbol of global level l; sym_off[M] = coarsest
  int64_t n_coeffs;
  std::vector<std::vector<Dim1DHost>> glev;  // [M][3]
  std::vector<double> A;  // level error constants: local 1..K then global 1..M (rounded)
};

// Whether the fused In-cache Block kernels exist for a block size.
inline bool fused_block(int B) { return B == 9 || B == 17; }

// Builds the plan; returns an empty string on success, else a message.
std::string make_plan(const int64_t* shape, int B, int K, int M, int R, PlanHost& p);

}  // namespace bm

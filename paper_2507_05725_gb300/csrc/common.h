// Shared host/device descriptors of the FTH-MS library (plain structs, no CUDA types).
#pragma once
#include <cstdint>

namespace fthms {

// One (arc j, frequency l) open-arc system: N first-kind nodes, matrix A_j(omega_l).
struct SysDesc {
  int arc;
  int l;            // frequency index, 1..L-1
  int N;
  int panel;        // node panel (arc, N)
  long long mat_off;  // complex offset of the N x N matrix / LU factor (column-major)
  long long vec_off;  // complex offset of the Q x N data / density block ([q][i])
  long long piv_off;  // int offset of the N pivots
  long long rlog_off; // double offset of the N x N self log-weight table
  double kappa;
};

// Nodes of arc `arc` at first-kind Chebyshev size N: t_i, x(t_i), |x'(t_i)|.
struct Panel {
  int arc;
  int N;
  long long off;    // offset into the node arrays
};

// Target of a cross-evaluation block (receiving arc k or the observation set).
struct CrossTgt {
  double x, y;
  double tstar;     // parameter of the target on the source arc's curve (near rule), else 0
  int near;         // 1: near rule (same curve, 1 < |t*| <= 3)
  int out;          // transfer-node index on arc k (or observation index)
};

// A (source arc j -> receiver k) block at one frequency: rows = targets, cols = N_j(omega_l).
struct CrossBlk {
  int j;            // source arc
  int sys;          // system index of (j, l)
  int N;
  int nrows;
  int tgt_off;      // first CrossTgt of the (k, j) pair
  int pad;
  long long e_off;  // complex offset of the row-major nrows x N block
};

// Group of blocks sharing (l, k): one launch unit of the cross matvec.
struct CrossGrp {
  int l;
  int k;            // receiving arc, or P for the observation points
  int blk_begin, blk_end;
};

// Row slice of a group for the double-float cross apply: rows [row0, row0 + nrows) of the group's
// concatenated block rows, overlapping blocks b0..b1 (indices into the block list, inclusive), the
// first of which starts at group row rowb0.
constexpr int kApplySlice = 256;
struct ApplySlice {
  int grp;
  int row0, nrows;
  int b0, b1;
  int rowb0;
};

// Mixed-form refinement residuals: 32 consecutive rows of one system (one warp, a row per lane).
struct ResidChunk {
  int sys, row0;
};

// Receiver/source pair (k, j), k = P for the observation points.
struct PairDesc {
  int k, j;
  int tgt_off;      // first CrossTgt
  int nrows;
};

// Assembly task: rows [row0, row0+nrows) of pair `pair` for the band of frequencies l0..l1
// (inclusive) that share the same N_j(omega_l); E offsets come from e_off[pair*L + l].
struct CrossAsm {
  int pair;
  int l0, l1;
  int N;
  int row0, nrows;
  int panel;        // node panel of source arc j at N
  int pad;
};

// On-the-fly cross task (cross_mode 1): assembly task `task`, restricted to the frequencies l0..l1
// (at most otf_band(Q) of them: the per-frequency sums of a CTA take 128 x Q x otf_band(Q) complex
// values of shared memory, at most 32 KB).
constexpr int kOtfBand = 16;
template <int Q> struct OtfBand { static constexpr int value = kOtfBand / Q > 4 ? kOtfBand / Q : 4; };
inline int otf_band(int Q) { return kOtfBand / Q > 4 ? kOtfBand / Q : 4; }   // host side of OtfBand
// Mixed forms: the double-float every-step kernel evaluates a (row, source) pair for bands of up to
// kOtfBandDf frequencies (its per-pair set-up amortised over the band; 16 rather than 32 leaves room for more
// CTAs per SM).
constexpr int kOtfBandDf = 16;
struct CrossOtf {
  int task;
  int l0, l1;
  int pad;
};

// Upper-triangular tile of the self matrices of a band of consecutive systems (same arc, same N,
// consecutive frequencies sys .. sys+nsys-1).
struct SelfTile {
  int sys;
  int nsys;
  int ti, tl;       // tile row / column (tile edge = kSelfTile)
};

// LU paths: one CTA per system in shared memory up to N = kLuSmallMax (FP64) / any N below kLuBigMin
// (mixed forms); the mixed forms factor N >= kLuBigMin (up to kLuBigMax) with tensor-core updates.
constexpr int kLuSmallMax = 800;
constexpr int kLuBigMin = 801;
constexpr int kLuBigMax = 2048;

constexpr int kSelfTile = 16;
constexpr int kSelfBand = 32;

}  // namespace fthms

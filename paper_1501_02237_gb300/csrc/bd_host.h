// Host front end: Smith form, consistency, LLL-reduced kernel points, Hadamard bound,
// work-list construction.  Plain C++ (no CUDA), shared by the C ABI and the host emulation.
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "bd_core.cuh"

namespace bd {

struct Reduction {
  int rank = 0, dim = 0;
  uint64_t torsion = 1;
  bool consistent = true;
  std::vector<int64_t> points;  // (n + 1) x dim, row-major; last row the origin
  int64_t max_abs_coord = 0;
};

// Returns BD_OK or an error code; message in `err`.
int reduce_system(const int64_t* A, int n, int m, const int64_t* coef, Reduction& out, std::string& err);

// log2 of Hadamard bounds on every minor of the lifted difference matrices [a_q - a_s, w_q - w_s]
// (K+1 rows) that the enumeration forms: `coord` for minors of coordinate columns only, the
// return value for all minors (lift column included).  lifts == nullptr: lift differences are
// bounded by max_lift_spread.
double hadamard_log2(const int64_t* pts, const int64_t* lifts, int npts, int k, int64_t max_lift_spread,
                     double* coord = nullptr);

// Integer path for the bounds: 0 (int32 coordinate minors, int64 lift minors), 1 (int64, int64),
// 2 (int128), -1 (too large).
int choose_path(double coord_bits, double full_bits);

// Depth of the deepest work item of the walk on integer path `path` (0: int32 coordinate
// minors, 1: int64, 2: int128): the depth at which its bottom stage starts.  The 5-D stage
// (int32 coordinate minors, k >= 4, when `five`) starts at k-3, the 4-D stage at k-2.
int item_depth(int k, int path, bool five);

// Whether the walk on the 32-bit coordinate path should end in the 5-D stage for these npts x k
// points (row-major) rather than the 4-D stage.  The 5-D stage skips one Bareiss level per node
// but tests every quadruple with a det4 and every nonsingular one with five 4x4 cofactors.  Rule,
// from timings of both stages on random, quiver-style, master-space and batch systems on a
// GB300: where the system's items share launches with other systems (teams = 0) the 5-D stage
// for k >= 4 (it took fewer SM cycles on every class of the uneven batch); where the system
// fills a launch alone (teams = its resident warps), k >= 6 and at most half of 256 sampled
// (k+1)-subsets full-dimensional (64 or 128 when at most 35 % or at least 65 % of them are; exact
// rank by fraction-free elimination in 64 bits, so the points must be on the 32-bit coordinate
// path; a fixed seed, so the choice is a function of the points): mostly nonsingular systems run
// faster on the 4-D stage's finer work list.  Allocation-free.
bool prefer_five(const int64_t* points, int npts, int k, uint64_t teams);

// Prefix work list: every (k+1)-subset of {0..npts-1} lies below exactly one item; items are
// split until each holds at most `max_subsets` subsets (or reaches length `depth`), then
// sorted by decreasing size.  With depth = k-3 (the 5-D stage), an item of that length holding
// more than 16 times `max_subsets` is split once more (length k-2: its last index is then the
// first point of the quadruples it takes).
// sorted = false: in generation (lexicographic) order, for callers that order items themselves.
std::vector<Item> build_items(int npts, int k, uint64_t max_subsets, int depth, bool sorted = true);

// The work-item split threshold for a launch of `teams` warps over `total` subsets: fine enough
// for the packing of ranges (1/32 of a warp's share), between 64 and 2^20 subsets.
uint64_t default_item_subsets(uint64_t total, uint64_t teams);

// The same items in lexicographic order, grouped into ranges of consecutive items for `teams`
// teams: runs packed up to 1/8 of a team's share of the estimated work (the bottom stage's
// warp rounds and level steps, not subsets, which misjudge regions of small nodes), taken
// largest first.  A team builds the prefixes its range's items share once.
void build_ranges(int npts, int k, uint64_t max_subsets, uint64_t teams, int depth, std::vector<Item>& items,
                  std::vector<Range>& ranges);

// The same list written into a caller-owned array of `cap` items (no allocation); false when
// it does not fit.
bool build_items_into(int npts, int k, uint64_t max_subsets, int depth, Item* out, size_t cap, size_t* count);

// Host emulation of the warp enumeration on `threads` CPU threads (one single-lane team
// each), for an integer path; team_width > 1 instead runs one team of that many lanes as
// threads in lockstep.  With ranges, teams take whole ranges of consecutive items.  `five`
// selects the 5-D bottom stage where it applies; the items must come from item_depth(K, path, five).
void host_enumerate(int path, bool five, const int64_t* P, int N, int K, const std::vector<Item>& items, int threads, Acc& acc,
                    int team_width = 1, const std::vector<Range>* ranges = nullptr, const CellSink* sink = nullptr);

}  // namespace bd

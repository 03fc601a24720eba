// Output-sensitive enumeration of the lifting's cells by simplicial pivoting (Sec. 4.2,
// Eq. pivot), shared by the CUDA warp kernel and its host emulation.
//
// A cell is a lower facet {s_0 < .. < s_d} of the lifted points (Eq. lower-d-face).  Dropping
// the equality of vertex s_i frees the inner normal by one degree (Eq. pivot); turning it about
// the ridge until it meets another point gives the neighbouring cell across that ridge, the
// basic feasible solution the paper obtains by a Phase One step.  This file takes that step
// without a linear program: with lambda(p) the barycentric coordinates of p in the cell's
// simplex and h(p) the height of p above the cell's lifted hyperplane, turning about the ridge
// opposite s_i lowers the height of p by t * (-lambda_i(p)), so the first point met is the one
// with lambda_i(p) < 0 that minimises h(p) / (-lambda_i(p)); no such point means the ridge lies
// on the boundary of conv(points).
//
// Exactness.  M^T lambda = p - s_0 (M the cell's difference rows) is solved for every point at
// once by fraction-free Gauss-Jordan elimination of [M^T | a_p - a_{s_0}], whose entries stay
// minors of that matrix (bounded on the host by Hadamard's inequality): at the end the left
// block is D I with D = +-det M and the right block holds g(p) = D lambda(p) (g_0 = D - sum g_j).
// The height is s(p) = D h(p) = D (w_p - w_{s_0}) - sum_j g_j(p) (w_{s_j} - w_{s_0}) in 128 bits,
// and ratios are compared by 256-bit cross products (s_A g_B > s_B g_A means A comes first,
// both g of the far side having the sign opposite to D).  A point other than the cell's with
// s(p) of the wrong sign, a zero height or two equal ratios mean the lifting is not generic.
//
// Parallel layout: a warp owns one cell; its lanes own the matrix columns in the elimination
// and the points in the height and ridge stages; each ridge's minimum is a tree reduction over
// the lanes' candidates in shared memory.
#pragma once

#include "bd_core.cuh"
#include "bd_lifts.h"

namespace bd {

constexpr int kPivotDMax = 30;  // dimension limit of the pivoting path (N <= 64 points)

enum { PV_OK = 0, PV_TIE = 1, PV_INVALID = 2 };

// one lane's best candidate for a ridge
struct PivotCand {
  i128 s;      // height numerator s(p)
  int64_t g;   // barycentric numerator of the dropped vertex, g_i(p)
  int32_t p;   // point index, -1 for none
  int32_t pad;
};

// per-warp scratch of the pivoting stage
struct PivotScratch {
  PivotCand cand[32];
  uint8_t cidx[kPivotDMax + 2];  // the cell's points in increasing order
  int32_t piv;                   // pivot row of the current elimination step
  int32_t flags;                 // PV_TIE | PV_INVALID found by any lane
};

// signed 256-bit comparison of two products: a * b > c * d
BD_HD bool prod_greater(i128 a, i128 b, i128 c, i128 d) {
  u128 h1, l1, h2, l2;
  mul_wide(a, b, h1, l1);
  mul_wide(c, d, h2, l2);
  if (h1 != h2) return (i128)h1 > (i128)h2;
  return l1 > l2;
}

BD_HD bool prod_equal(i128 a, i128 b, i128 c, i128 d) {
  u128 h1, l1, h2, l2;
  mul_wide(a, b, h1, l1);
  mul_wide(c, d, h2, l2);
  return h1 == h2 && l1 == l2;
}

// merge candidate B into A (both for the same ridge); sets *tie on equal ratios
BD_HD void pivot_merge(PivotCand& A, const PivotCand& B, int32_t* flags) {
  if (B.p < 0) return;
  if (A.p < 0) {
    A = B;
    return;
  }
  // A first iff s_A g_B > s_B g_A (g_A, g_B of the same sign)
  if (prod_equal(A.s, (i128)B.g, B.s, (i128)A.g)) {
#ifdef __CUDA_ARCH__
    atomicOr(flags, PV_TIE);
#else
    __atomic_fetch_or(flags, PV_TIE, __ATOMIC_RELAXED);
#endif
    if (B.p < A.p) A = B;  // either choice is wrong: the lifting is re-drawn
    return;
  }
  if (!prod_greater(A.s, (i128)B.g, B.s, (i128)A.g)) A = B;
}

struct PivotAcc {
  u128 nvol;          // sum of |D| over the cells processed
  uint64_t cells;     // cells processed
  uint64_t boundary;  // ridges on the boundary of conv(points)
};

// Process one cell (bitmask of its d+1 points): eliminate, check it, add |D|, and hand every
// neighbour across a ridge to insert(mask) (called by lane 0).  P holds the points
// coordinate-major (P[r * N + p]), L the lifts.  Per team: W, d x (d+N) int64; S, N heights;
// G0, N values of g_0; sc, the scratch.  Returns PV_OK, or PV_TIE / PV_INVALID bits.
#ifdef __CUDACC__
#pragma nv_exec_check_disable  // instantiated with host-only teams by the host emulation
#endif
template <class Team, class Insert>
BD_HD int pivot_cell(Team tm, const int64_t* P, const int64_t* L, int N, int d, uint64_t mask, int64_t* W, i128* S,
                     int64_t* G0, PivotScratch* sc, PivotAcc& acc, Insert insert) {
  const int lane = tm.lane(), nl = tm.lanes(), width = d + N;
  tm.sync();  // the previous cell's readers are done with the scratch
  if (lane == 0) sc->flags = 0;
  for (int b = lane; b < 64; b += nl)
    if ((mask >> b) & 1) sc->cidx[popc64(mask & ((1ull << b) - 1))] = (uint8_t)b;
  tm.sync();
  const int s0 = sc->cidx[0];
  // W = [M^T | a_p - a_{s_0}]: row r holds coordinate r
  for (int c = lane; c < width; c += nl) {
    const int src = c < d ? sc->cidx[c + 1] : c - d;
    for (int r = 0; r < d; ++r) W[r * width + c] = P[r * N + src] - P[r * N + s0];
  }
  tm.sync();
  // fraction-free Gauss-Jordan: after step k, rows i != k have no entry in column k
  int64_t prev = 1;
  for (int k = 0; k < d; ++k) {
    if (lane == 0) {
      int r = k;
      while (r < d && W[r * width + k] == 0) ++r;
      sc->piv = r;
    }
    tm.sync();
    const int pr = sc->piv;
    if (pr == d) {  // no pivot: the points are affinely dependent, not a cell
      if (lane == 0) sc->flags |= PV_INVALID;
      tm.sync();
      return sc->flags;
    }
    if (pr != k) {
      for (int c = lane; c < width; c += nl) {
        const int64_t t = W[k * width + c];
        W[k * width + c] = W[pr * width + c];
        W[pr * width + c] = t;
      }
      tm.sync();
    }
    const int64_t pk = W[k * width + k];
    const Div64 D = make_div(prev);
    for (int c = k + 1 + lane; c < width; c += nl) {
      const int64_t top = W[k * width + c];
      for (int i = 0; i < d; ++i)
        if (i != k) W[i * width + c] = bareiss(W[i * width + c], pk, W[i * width + k], top, D);
    }
    tm.sync();
    prev = pk;
  }
  const int64_t Dv = prev;  // +-det M: the cell's normalized volume up to sign
  const int sd = Dv > 0 ? 1 : -1;
  // heights and g_0 of every point
  int fl = 0;
  for (int p = lane; p < N; p += nl) {
    i128 s = (i128)Dv * (L[p] - L[s0]), gs = 0;
    for (int j = 0; j < d; ++j) {
      const int64_t g = W[j * width + d + p];
      gs += g;
      s -= (i128)g * (L[sc->cidx[j + 1]] - L[s0]);
    }
    S[p] = s;
    G0[p] = (int64_t)((i128)Dv - gs);  // itself a minor: fits
    if (!((mask >> p) & 1)) {
      const int sg = (s > 0) - (s < 0);
      if (sg == 0) fl |= PV_TIE;
      else if (sg != sd) fl |= PV_INVALID;
    }
  }
  if (fl) {
#ifdef __CUDA_ARCH__
    atomicOr(&sc->flags, fl);
#else
    __atomic_fetch_or(&sc->flags, fl, __ATOMIC_RELAXED);
#endif
  }
  tm.sync();
  if (sc->flags) return sc->flags;  // uniform: read after the sync
  if (lane == 0) {
    acc.nvol += (u128)(Dv < 0 ? -Dv : Dv);
    ++acc.cells;
  }
  // every ridge: the far-side point of least h / (-lambda_i)
  for (int i = 0; i <= d; ++i) {
    PivotCand best{0, 0, -1, 0};
    for (int p = lane; p < N; p += nl) {
      if ((mask >> p) & 1) continue;
      const int64_t gi = i == 0 ? G0[p] : W[(i - 1) * width + d + p];
      if (gi == 0 || (gi > 0 ? 1 : -1) == sd) continue;  // not beyond the ridge
      PivotCand c{S[p], gi, p, 0};
      pivot_merge(best, c, &sc->flags);
    }
    sc->cand[lane] = best;
    tm.sync();
    for (int h = 1; h < nl; h *= 2) {
      if (lane % (2 * h) == 0 && lane + h < nl) pivot_merge(sc->cand[lane], sc->cand[lane + h], &sc->flags);
      tm.sync();
    }
    if (lane == 0) {
      const PivotCand b = sc->cand[0];
      if (b.p < 0) ++acc.boundary;
      else insert((mask & ~(1ull << sc->cidx[i])) | (1ull << b.p));
    }
    tm.sync();  // cand[0] is read before the next ridge overwrites the candidates
  }
  return sc->flags;
}

BD_HD uint64_t pivot_hash(uint64_t m) { return splitmix_mix(m); }  // a cell mask spread over the table

}  // namespace bd

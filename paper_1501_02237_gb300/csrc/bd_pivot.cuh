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
// The tableau holds 64-bit entries while that bound stays below 2^62 and 128-bit entries above
// it (TE, the entry type).  The height is s(p) = D h(p) = D (w_p - w_{s_0}) - sum_j g_j(p)
// (w_{s_j} - w_{s_0}) in 128 bits (the host also bounds it: minors times 2^41 heights, d+1
// terms), and ratios are compared by 256-bit cross products (s_A g_B > s_B g_A means A comes
// first, both g of the far side having the sign opposite to D).  A point other than the cell's with
// s(p) of the wrong sign, a zero height or two equal ratios mean the lifting is not generic.
//
// Parallel layout: a warp owns one cell; its lanes own the matrix columns in the elimination and
// the points in the height stage; in the ridge stage lane r takes ridge r and scans every point
// for its minimum, and the lanes claim their neighbours concurrently.
#pragma once

#include "bd_core.cuh"
#include "bd_lifts.h"

namespace bd {

constexpr int kPivotDMax = 30;   // dimension limit of the pivoting path
constexpr int kPivotNMax = 127;  // point limit: a cell is a mask of up to 127 point bits

// A cell is the set of its d+1 points, kept as a bit mask: one 64-bit word while there are at
// most 64 points, two words (every shift below 64) up to 127.  The walk is generic in the mask.
struct WideMask {
  uint64_t lo, hi;  // bits 0..63 and 64..126
};
BD_HD bool operator==(WideMask a, WideMask b) { return a.lo == b.lo && a.hi == b.hi; }

BD_HD bool mhas(uint64_t m, int p) { return (m >> p) & 1ull; }
BD_HD bool mhas(WideMask m, int p) { return ((p < 64 ? m.lo >> p : m.hi >> (p - 64)) & 1ull) != 0; }
// number of the mask's points below point b
BD_HD int mrank(uint64_t m, int b) { return popc64(m & ((1ull << b) - 1)); }
BD_HD int mrank(WideMask m, int b) {
  return b < 64 ? popc64(m.lo & ((1ull << b) - 1)) : popc64(m.lo) + popc64(m.hi & ((1ull << (b - 64)) - 1));
}
// the mask without point `out`, with point `in`
BD_HD uint64_t mswap(uint64_t m, int out, int in) { return (m & ~(1ull << out)) | (1ull << in); }
BD_HD WideMask mswap(WideMask m, int out, int in) {
  if (out < 64) m.lo &= ~(1ull << out);
  else m.hi &= ~(1ull << (out - 64));
  if (in < 64) m.lo |= 1ull << in;
  else m.hi |= 1ull << (in - 64);
  return m;
}
BD_HD void madd(uint64_t& m, int p) { m |= 1ull << p; }
BD_HD void madd(WideMask& m, int p) {
  if (p < 64) m.lo |= 1ull << p;
  else m.hi |= 1ull << (p - 64);
}

enum { PV_OK = 0, PV_TIE = 1, PV_INVALID = 2 };

// one lane's best candidate for a ridge (TE: the tableau's entry type, int64_t or i128)
template <class TE>
struct PivotCand {
  i128 s;      // height numerator s(p)
  TE g;        // barycentric numerator of the dropped vertex, g_i(p)
  int32_t p;   // point index, -1 for none
  int32_t pad;
};

// per-warp scratch of the pivoting stage
// deepest in-place walk below an eliminated cell: 32 levels keep the per-warp stack at ~1.2 KB
// (W4,5 walks at 12 instead of 10 warps per SM: 4.11 -> 3.44 s; 64 levels gained nothing)
#ifndef BD_WALK_DEPTH
#define BD_WALK_DEPTH 32
#endif
constexpr int kWalkDepth = BD_WALK_DEPTH;

template <class TE>
struct PivotScratch {
  i128 sq;                       // the entering point's height numerator during a pivot
  TE colq[kPivotDMax + 1];       // the entering point's tableau column during a pivot
  TE D;                          // the current cell's +-det M
  uint8_t cidx[kPivotDMax + 2];  // the current cell's vertices; tableau row r belongs to cidx[r]
  uint8_t st_slot[kWalkDepth], st_old[kWalkDepth];  // the walk's stack: replaced row and point
  uint32_t st_todo[kWalkDepth];  // the parent's new neighbours still to handle
  uint8_t nbr[kWalkDepth][32];   // per stack level: the point beyond each ridge (255: boundary)
  int32_t piv;                   // pivot row of the current elimination step
  int32_t flags;                 // PV_TIE | PV_INVALID found by any lane
  int32_t claimed;               // lane 0's claim of a neighbour, read by every lane
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

// a float near x (relative error below 2^-23.9): the top 62 bits through an int64 conversion
BD_HD float approx_f(i128 x);
BD_HD float approx_f(int64_t x) { return (float)x; }  // rounded once
BD_HD float approx_f(i128 x) {
  const bool neg = x < 0;
  const u128 a = neg ? (u128)(-x) : (u128)x;
  int sh = 0;
  if (a >> 62) {
    const uint64_t hi = (uint64_t)(a >> 64);
#ifdef __CUDA_ARCH__
    const int lz = hi ? __clzll((long long)hi) : 64;
#else
    const int lz = hi ? __builtin_clzll(hi) : 64;
#endif
    sh = 66 - lz;  // leaves the value below 2^62
  }
  const float f = ldexpf((float)(int64_t)(a >> sh), sh);
  return neg ? -f : f;
}

// a / b in single precision: the device's fast division (within 2 ulp for |b| below 2^126),
// the host's IEEE division (within half an ulp)
BD_HD float ratio_f(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fdividef(a, b);
#else
  return a / b;
#endif
}

// merge candidate B into A (both for the same ridge); sets *tie on equal ratios
template <class TE>
BD_HD void pivot_merge(PivotCand<TE>& A, const PivotCand<TE>& B, int32_t* flags) {
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

// Process one cell (bitmask of its d+1 points) and up to `budget` of its descendants: eliminate
// it, check it, add |D|; then walk its ridges.  A neighbour that claim(mask) reports as new is
// either entered in place (one rank-one pivot of the tableau, Sec. 4.2's pivot taken literally;
// one more pivot leads back) or, past the budget or the stack depth, handed to push(mask) for a
// later launch.  claim and push are called by any lane, concurrently.  P holds the points coordinate-major
// (P[r * N + p], 32-bit: the pivoting path takes coordinates below 2^20), L the lifts.  Per team: W, d x N entries; S, N heights and Sf, their
// single-precision values; G0, N values of g_0; sc, the scratch.  Rows 1..d of the tableau are W's right block, row 0 is G0.  TE is int64_t
// (cell minors below 2^62) or i128 (below 2^126; the host checks the bounds).  Returns PV_OK,
// or PV_TIE / PV_INVALID bits.
#ifdef __CUDACC__
#pragma nv_exec_check_disable  // instantiated with host-only teams by the host emulation
#endif
template <class TE, class Team, class Mask, class Claim, class Push>
BD_HD int pivot_cell(Team tm, const int32_t* P, const int64_t* L, int N, int d, Mask mask, TE* W, i128* S,
                     float* Sf, TE* G0, PivotScratch<TE>* sc, PivotAcc& acc, Claim claim, Push push, int budget) {
  typedef typename DivOf<TE>::type Div;
  const int lane = tm.lane(), nl = tm.lanes();
  tm.sync();  // the previous cell's readers are done with the scratch
  if (lane == 0) sc->flags = 0;
  for (int b = lane; b < N; b += nl)
    if (mhas(mask, b)) sc->cidx[mrank(mask, b)] = (uint8_t)b;
  tm.sync();
  const int s0 = sc->cidx[0];
  // W = [a_p - a_{s_0}] for every point p (row r: coordinate r; d x N, row stride N).  The
  // columns of the cell's own points s_1 .. s_d are M^T, so fraction-free Gauss-Jordan runs on W
  // alone: step k pivots on the column of s_{k+1}, which then holds p_k e_k, and at the end
  // every column is D lambda(p) (the cell's own columns D e_j)
  for (int p = lane; p < N; p += nl)
    for (int r = 0; r < d; ++r) W[r * N + p] = (TE)(P[r * N + p] - P[r * N + s0]);
  tm.sync();
  TE prev = 1;
  for (int k = 0; k < d; ++k) {
    const int kc = sc->cidx[k + 1];  // the pivot column
    if (lane == 0) {
      int r = k;
      while (r < d && W[r * N + kc] == 0) ++r;
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
      for (int c = lane; c < N; c += nl) {
        const TE t = W[k * N + c];
        W[k * N + c] = W[pr * N + c];
        W[pr * N + c] = t;
      }
      tm.sync();
    }
    const TE pk = W[k * N + kc];
    const Div D = make_div(prev);
    for (int c = lane; c < N; c += nl) {
      if (c == kc) continue;  // the multipliers: read by every lane, rewritten below
      const TE top = W[k * N + c];
      for (int i = 0; i < d; ++i)
        if (i != k) W[i * N + c] = bareiss(W[i * N + c], pk, W[i * N + kc], top, D);
    }
    tm.sync();
    for (int i = lane; i < d; i += nl) W[i * N + kc] = i == k ? pk : (TE)0;
    tm.sync();
    prev = pk;
  }
  const TE Dv = prev;  // +-det M: the cell's normalized volume up to sign
  // heights and g_0 of every point
  int fl = 0;
  for (int p = lane; p < N; p += nl) {
    i128 s = (i128)Dv * (L[p] - L[s0]), gs = 0;
    for (int j = 0; j < d; ++j) {
      const TE g = W[j * N + p];
      gs += g;
      s -= (i128)g * (L[sc->cidx[j + 1]] - L[s0]);
    }
    S[p] = s;
    Sf[p] = approx_f(s);
    G0[p] = (TE)((i128)Dv - gs);  // itself a minor: fits
    if (!mhas(mask, p)) {
      const int sg = (s > 0) - (s < 0);
      if (sg == 0) fl |= PV_TIE;
      else if (sg != (Dv > 0 ? 1 : -1)) fl |= PV_INVALID;
    }
  }
  auto raise = [&](int f) {
    if (!f) return;
#ifdef __CUDA_ARCH__
    atomicOr(&sc->flags, f);
#else
    __atomic_fetch_or(&sc->flags, f, __ATOMIC_RELAXED);
#endif
  };
  raise(fl);
  if (lane == 0) sc->D = Dv;
  tm.sync();
  if (sc->flags) return sc->flags;  // uniform: read after the sync
  if (lane == 0) {
    acc.nvol += (u128)(Dv < 0 ? -Dv : Dv);
    ++acc.cells;
  }
  auto T = [&](int r, int p) -> TE& { return r == 0 ? G0[p] : W[(r - 1) * N + p]; };
  // Pivot row i onto point q: T'[r][p] = (T[r][p] T[i][q] - T[r][q] T[i][p]) / D for r != i,
  // T'[i][p] = T[i][p], S'[p] = (S[p] T[i][q] - S[q] T[i][p]) / D, D' = T[i][q] (every entry
  // again a minor, or D' times a height, of the new cell).
  auto pivot_to = [&](int i, int q) {
    for (int r = lane; r <= d; r += nl) sc->colq[r] = T(r, q);
    if (lane == 0) sc->sq = S[q];
    tm.sync();
    const TE Dold = sc->D, piv = sc->colq[i];
    const Div Dd = make_div(Dold);
    const Div128 Dw = make_div((i128)Dold);
    const i128 sq = sc->sq;
    for (int p = lane; p < N; p += nl) {
      const TE ti = T(i, p);
      for (int r = 0; r <= d; ++r)
        if (r != i) T(r, p) = bareiss(T(r, p), piv, sc->colq[r], ti, Dd);
      S[p] = bareiss(S[p], (i128)piv, sq, (i128)ti, Dw);
      Sf[p] = approx_f(S[p]);
    }
    tm.sync();
    if (lane == 0) {
      sc->D = piv;
      sc->cidx[i] = (uint8_t)q;
    }
    tm.sync();
  };
  // The ridges of the current cell: lane l takes ridges l, l + lanes, .. and scans every point
  // for the least h / (-lambda_r); all lanes then claim their neighbours at once, and one vote
  // gives the ridges whose neighbour is new (bit r).
  auto scan = [&](int lvl) -> uint32_t {
    const int sd = sc->D > 0 ? 1 : -1;
    uint64_t fresh = 0;
    for (int r = lane; r <= d; r += nl) {
      int bp = -1;     // the best candidate so far: its point, g_r and ratio in single precision
      TE bg = 0;
      float bf = 0.f;
      for (int p = 0; p < N; ++p) {
        if (mhas(mask, p)) continue;
        const TE gi = T(r, p);
        if (gi == 0 || (gi > 0 ? 1 : -1) == sd) continue;  // not beyond the ridge
        // Ratios in single precision first: the height within 2^-23.9 of its value (Sf, formed
        // once per cell), g_r within 2^-23.9, the quotient within 2 ulp (2^-22), so a ratio is
        // within 2^-21.2 of the exact one and ratios apart by more than 2^-16 of their size are
        // ordered correctly.  Closer ones: the exact test.
        const float cf = ratio_f(Sf[p], approx_f((TE)-gi));
        if (bp < 0 || cf < bf * (1.f - 0x1p-16f)) {
          bp = p;
          bg = gi;
          bf = cf;
          continue;
        }
        if (cf > bf * (1.f + 0x1p-16f)) continue;
        PivotCand<TE> best{S[bp], bg, bp, 0};
        pivot_merge(best, PivotCand<TE>{S[p], gi, p, 0}, &sc->flags);
        bp = best.p;
        bg = best.g;
        bf = ratio_f(Sf[bp], approx_f((TE)-bg));
      }
      sc->nbr[lvl][r] = bp < 0 ? (uint8_t)255 : (uint8_t)bp;
      if (bp >= 0 && claim(mswap(mask, sc->cidx[r], bp))) fresh |= 1ull << r;
    }
    fresh = tm.or_all(fresh);
    tm.sync();  // the neighbours are visible to every lane
    return (uint32_t)fresh;
  };
  int depth = 0, entered = 0;
  uint32_t todo = scan(0);  // new neighbours of the current cell not yet handled
  for (;;) {
    if (!todo) {  // this cell is done
      if (depth == 0) break;
      --depth;
      const int i = sc->st_slot[depth], o = sc->st_old[depth], q = sc->cidx[i];
      todo = sc->st_todo[depth];
      pivot_to(i, o);  // back to the parent cell
      mask = mswap(mask, q, o);
      continue;
    }
    const int r = ctz64((uint64_t)todo);
    if (depth + 1 < kWalkDepth && entered < budget) {  // enter the neighbour in place
      todo &= todo - 1;
      const int q = sc->nbr[depth][r];
      const Mask nm = mswap(mask, sc->cidx[r], q);
      if (lane == 0) {
        sc->st_slot[depth] = (uint8_t)r;
        sc->st_old[depth] = sc->cidx[r];
        sc->st_todo[depth] = todo;
      }
      pivot_to(r, q);
      mask = nm;
      ++depth;
      ++entered;
      const int sdn = sc->D > 0 ? 1 : -1;
      int f2 = 0;
      for (int p = lane; p < N; p += nl) {
        if (mhas(mask, p)) continue;
        const int sg = (S[p] > 0) - (S[p] < 0);
        if (sg == 0) f2 |= PV_TIE;
        else if (sg != sdn) f2 |= PV_INVALID;
      }
      raise(f2);
      tm.sync();
      if (sc->flags) return sc->flags;
      if (lane == 0) {
        const TE Dn = sc->D;
        acc.nvol += (u128)(Dn < 0 ? -Dn : Dn);
        ++acc.cells;
      }
      todo = scan(depth);
      continue;
    }
    // past the budget or the depth: this cell's remaining new neighbours go to the next level
    for (int rr = lane; rr <= d; rr += nl)
      if ((todo >> rr) & 1) push(mswap(mask, sc->cidx[rr], sc->nbr[depth][rr]));
    todo = 0;
    tm.sync();
  }
  tm.sync();
  return sc->flags;
}

BD_HD uint64_t pivot_hash(uint64_t m) { return splitmix_mix(m); }  // a cell mask spread over the table
// a two-word mask's fingerprint, never 0 (0 marks an empty slot of the two-word table)
BD_HD uint64_t pivot_hash(WideMask m) { return splitmix_mix(m.lo ^ splitmix_mix(m.hi + 0x632BE59BD9B4E019ull)) | 1ull; }

}  // namespace bd

// Exact mixed volume by enumerating the fine mixed cells of a random lifting, shared by the
// CUDA warp kernel and its host emulation.
//
// Method (the BKK generalisation of the degree, Appendix A; mixed cells of a lifting as in
// Huber-Sturmfels 1995, on which Sec. 4's remark on earlier work builds): K point sets
// A_0..A_{K-1} in Z^K, every point lifted to (a, w(a)).  A tuple of pairs C = (C_0..C_{K-1}),
// C_i = {p_i, q_i} a 2-subset of A_i, is a fine mixed cell iff M = [a_{q_i} - a_{p_i}]_i is
// nonsingular and the alpha with <a_{q_i} - a_{p_i}, alpha> = -(w(q_i) - w(p_i)) puts every
// other point b of every A_i strictly above: <b - a_{p_i}, alpha> + w(b) - w(p_i) > 0.
// MV = sum |det M| over the fine mixed cells.
//
// Exact test.  Let R be the K x (K+1) matrix of lifted pair rows r_i = z(q_i) - z(p_i),
// z(a) = (a, w(a)), and f(r) = det [R ; r].  Then f(z(b) - z(p_i)) = det M * (height of b
// above the cell's plane in A_i's lifting) (Cramer's rule on [R ; z(b) - z(p_i)] (alpha, 1)),
// so b is strictly above iff sign(f(z(b)) - f(z(p_i))) = sign(det M); f is linear, so every
// point's row is reduced once, whatever its component.
//
// Evaluation order (this file's design): a depth-first walk over the components in level
// order; level j fixes the pair of component j.  The state at level j is the fraction-free
// (Bareiss) reduction of every point's row z(a) - z(base of its component) against the pivot
// rows of levels 0..j-1; the pivot row of level j is the difference of the reduced rows of
// q_j and p_j (the reduction is linear in the row).  An entry of state j equals the
// (j+1) x (j+1) minor of (pivot rows, the point's row) on (pivot columns, its column)
// (Sylvester's identity).  A pivot row with no nonzero coordinate entry makes det M = 0 for
// the whole subtree (counted singular, skipped).  After K-1 levels every point carries
// (x, y): its K x K minors on the last coordinate column and on the lift column.  For a
// pair (p, q) of the last component, X = x_q - x_p is det M up to the column-permutation
// sign sigma, and f(z(b)) = sigma (X y_b - x_b Y) / d with Y = y_q - y_p and d the previous
// pivot, so the test of b is a 2 x 2 cross product and a sign compare.
//
// Parallel layout: a warp owns one subtree at a time; its lanes own points round-robin for
// the state updates, and the pairs of the last component are dealt to lanes, each lane
// scanning the points with early exit.
#pragma once

#include "bd_core.cuh"

namespace bd {

// the shape of one mixed problem, in level order (component j = the j-th level)
struct MixedShape {
  int K, N;                  // dimension, points in all components
  int first[KMAX + 1];       // component j owns points first[j] .. first[j+1]-1
  uint32_t npairs[KMAX];     // C(|A_j|, 2)
  uint64_t below[KMAX + 1];  // tuples under one node of level j: prod_{i >= j} npairs[i]
  int prefix;                // levels fixed by a work item (0 <= prefix <= K-1)
  uint64_t items;            // prod_{j < prefix} npairs[j]
};

// a fine mixed cell as reported: the pair of each level as point indices, and |det M|
struct MixedCellRec {
  uint8_t idx[2 * KMAX];  // p_j, q_j (global point indices in level order), j = 0..K-1
  uint8_t pad[32 - 2 * KMAX];
  int64_t absdet;         // |det M|, or -1 when it needs more than 63 bits
};
static_assert(sizeof(MixedCellRec) == 40, "record layout");

struct MixedSink {
  MixedCellRec* out;
  unsigned long long* count;
  unsigned long long cap;
};

// pairs (p, q), p < q, of n points in lexicographic order: rank -> (p, q)
BD_HD void pair_of_rank(uint32_t r, int n, int& p, int& q) {
  p = 0;
  for (;;) {
    const uint32_t c = (uint32_t)(n - 1 - p);
    if (r < c) break;
    r -= c;
    ++p;
  }
  q = p + 1 + (int)r;
}

// Up to KMAX pairs of six-bit point indices in three registers (ten fields per word): the walk's
// cursor, kept out of per-thread local arrays.
struct Pairs14 {
  uint64_t w0 = 0, w1 = 0, w2 = 0;
  BD_HD int get(int f) const {
    const uint64_t w = f < 10 ? w0 : (f < 20 ? w1 : w2);
    return (int)((w >> (6 * (f % 10))) & 63u);
  }
  BD_HD void set(int f, int v) {
    const int sh = 6 * (f % 10);
    const uint64_t m = ~(63ull << sh), b = (uint64_t)v << sh;
    if (f < 10) w0 = (w0 & m) | b;
    else if (f < 20) w1 = (w1 & m) | b;
    else w2 = (w2 & m) | b;
  }
  BD_HD int p(int j) const { return get(2 * j); }
  BD_HD int q(int j) const { return get(2 * j + 1); }
  BD_HD void set_pair(int j, int p, int q) {
    set(2 * j, p);
    set(2 * j + 1, q);
  }
};

// per-warp values every lane needs after a level is built (written by lane 0)
template <class T> struct MixedUniform {
  T dv[KMAX + 1];  // dv[j]: the pivot of level j-1 (the divisor of level j's update); dv[0] = 1
};

struct MixedAcc {
  u128 mv;            // sum |det M| over accepted tuples
  uint64_t cells, singular, ties;
};

template <class T> BD_HD int sgn(T x) { return (x > 0) - (x < 0); }

template <class T, class Team> struct MixedWalker {
  typedef typename DivOf<T>::type Div;
  Team tm;
  const T* P;              // raw rows, column-major: P[c * N + g], c < K coordinates, c = K lift
  const MixedShape* sh;
  T* st;                   // this team's stack: level j >= 1 at st[(off(j) + e) * N + g]
  MixedUniform<T>* uni;
  const uint16_t* last_pairs;  // pairs of the last component as p | q << 8 (global indices)
  MixedSink sink{nullptr, nullptr, 0};
  Pairs14 cur;             // the pairs of the built levels
  int built = 0;           // levels 0..built-1 are reduced (state `built` is valid)
  int K, N;

  BD_HD MixedWalker(Team t, const T* P_, const MixedShape* s, T* stack, MixedUniform<T>* u, const uint16_t* lp)
      : tm(t), P(P_), sh(s), st(stack), uni(u), last_pairs(lp), K(s->K), N(s->N) {
    if (tm.lane() == 0) uni->dv[0] = T(1);
    tm.sync();
  }

  BD_HD int off(int j) const { return (j - 1) * (K + 1) - (j - 1) * j / 2; }  // sum_{i=1}^{j-1} (K+1-i)
  BD_HD T at(int j, int e, int g) const { return j == 0 ? P[e * N + g] : st[(off(j) + e) * N + g]; }
  BD_HD T& put(int j, int e, int g) { return st[(off(j) + e) * N + g]; }

  // Build level j+1 from level j with the pair (p, q) of component j.  Returns false when the
  // pivot row has no nonzero coordinate entry (det M = 0 below this node).
  BD_HD bool descend(int j, int p, int q) {
    const int slots = K + 1 - j;  // surviving columns at level j, the lift last
    int c = -1;
    T vc = 0;
    for (int e = 0; e < slots - 1; ++e) {
      const T v = at(j, e, q) - at(j, e, p);
      if (v != 0) {
        c = e;
        vc = v;
        break;
      }
    }
    if (c < 0) return false;
    const Div D = make_div(uni->dv[j]);
    tm.sync();  // readers of the old level j+1 (a sibling's subtree) are done
    for (int e = 0; e < slots; ++e) {
      if (e == c) continue;
      const T ve = at(j, e, q) - at(j, e, p);
      const int en = e - (e > c ? 1 : 0);
      for (int g = tm.lane(); g < N; g += tm.lanes()) put(j + 1, en, g) = bareiss(at(j, e, g), vc, at(j, c, g), ve, D);
    }
    if (tm.lane() == 0) uni->dv[j + 1] = vc;
    tm.sync();
    cur.set_pair(j, p, q);
    built = j + 1;
    return true;
  }

  // All pairs of the last component under the built prefix (levels 0..K-2 fixed).
  BD_HD void leaves(MixedAcc& acc) {
    const int j = K - 1;
    const uint32_t np = sh->npairs[j];
    const int sd = sgn(uni->dv[j]);
    for (uint32_t t = tm.lane(); t < np; t += tm.lanes()) {
      const uint16_t pq = last_pairs[t];
      const int p = pq & 255, q = pq >> 8;
      const T X = at(j, 0, q) - at(j, 0, p);
      if (X == 0) {
        ++acc.singular;
        continue;
      }
      const T Y = at(j, 1, q) - at(j, 1, p);
      const int want = sgn(X) * sd;  // sign of f(b) - f(base) for a point strictly above
      bool below = false, on = false;
      for (int i = 0; i < K && !below; ++i) {
        const int pi = i == j ? p : cur.p(i), qi = i == j ? q : cur.q(i);
        const T cb = X * at(j, 1, pi) - at(j, 0, pi) * Y;
        for (int g = sh->first[i]; g < sh->first[i + 1]; ++g) {
          if (g == pi || g == qi) continue;
          const int s = sgn(X * at(j, 1, g) - at(j, 0, g) * Y - cb);
          if (s != want) {
            if (s == 0) {
              on = true;
            } else {
              below = true;
              break;
            }
          }
        }
      }
      if (below) continue;
      if (on) {
        ++acc.ties;
        continue;
      }
      const T ax = X < 0 ? -X : X;
      acc.mv += (u128)ax;
      ++acc.cells;
      if (sink.out) record(p, q, ax);
    }
  }

  BD_HD void record(int p, int q, T ax) {
#ifdef __CUDA_ARCH__
    const unsigned long long slot = atomicAdd(sink.count, 1ull);
#else
    const unsigned long long slot = __atomic_fetch_add(sink.count, 1ull, __ATOMIC_RELAXED);
#endif
    if (slot >= sink.cap) return;
    MixedCellRec r;
    memset(&r, 0, sizeof(r));
    for (int i = 0; i < K - 1; ++i) {
      r.idx[2 * i] = (uint8_t)cur.p(i);
      r.idx[2 * i + 1] = (uint8_t)cur.q(i);
    }
    r.idx[2 * (K - 1)] = (uint8_t)p;
    r.idx[2 * (K - 1) + 1] = (uint8_t)q;
    r.absdet = ax > (T)INT64_MAX ? -1 : (int64_t)ax;
    sink.out[slot] = r;
  }

  // Depth-first walk of every tuple under the prefix `it` (levels 0..prefix-1 fixed by the
  // item's mixed-radix digits, the last level least significant).
  BD_HD void run_item(uint64_t it, MixedAcc& acc) {
    const int L = sh->prefix;
    const bool lead = tm.lane() == 0;  // uniform counts are added once per team
    // digits of the item, most significant first; reuse the built levels they share
    Pairs14 want;
    {
      uint64_t r = it;
      for (int j = L - 1; j >= 0; --j) {
        const uint32_t np = sh->npairs[j];
        const uint32_t d = (uint32_t)(r % np);
        r /= np;
        int p, q;
        pair_of_rank(d, sh->first[j + 1] - sh->first[j], p, q);
        want.set_pair(j, sh->first[j] + p, sh->first[j] + q);
      }
    }
    int f = 0;
    while (f < L && f < built && want.p(f) == cur.p(f) && want.q(f) == cur.q(f)) ++f;
    built = f;
    for (int j = f; j < L; ++j) {
      if (!descend(j, want.p(j), want.q(j))) {
        if (lead) acc.singular += sh->below[L];  // this item's tuples (its siblings count theirs)
        built = j;  // levels 0..j-1 stay valid
        return;
      }
    }
    if (L == K - 1) {
      leaves(acc);
      return;
    }
    // walk levels L..K-2; pair (p, q) of level j runs over component j in lexicographic order
    int j = L;
    int p = sh->first[j], q = p + 1;
    for (;;) {
      bool down = false;
      if (descend(j, p, q)) {
        if (j + 1 == K - 1) {
          leaves(acc);
        } else {
          ++j;
          p = sh->first[j];
          q = p + 1;
          down = true;
        }
      } else if (lead) {
        acc.singular += sh->below[j + 1];
      }
      if (down) continue;
      // next pair at level j, climbing while a level is exhausted
      for (;;) {
        const int end = sh->first[j + 1];
        if (++q >= end) {
          ++p;
          q = p + 1;
        }
        if (q < end) break;
        if (j == L) {
          built = L;  // the prefix levels stay valid for the next item
          return;
        }
        --j;
        p = cur.p(j);
        q = cur.q(j);
      }
    }
  }
};

// stack entries per point: sum over levels 1..K-1 of (K+1-j) surviving columns
BD_HD int mixed_stack_entries(int K) { return K <= 1 ? 0 : (K - 1) * (K + 1) - (K - 1) * K / 2; }

}  // namespace bd

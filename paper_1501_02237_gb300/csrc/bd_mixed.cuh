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
// scanning the points with early exit, in single precision with a rigorous error bound and an
// exact fallback (see leaves()).
#pragma once

#include "bd_core.cuh"

namespace bd {

// the shape of one mixed problem, in level order (component j = the j-th level)
struct MixedShape {
  int K, N;                  // dimension, points in all components
  int first[KMAX + 1];       // component j owns points first[j] .. first[j+1]-1
  uint32_t npairs[KMAX];     // C(|A_j|, 2)
  uint64_t below[KMAX + 1];  // tuples under one node of level j: prod_{i >= j} npairs[i]
  int prefix;                // levels fixed by a work item (0 <= prefix <= K-1; <= K-2 with leaf3)
  int leaf3;                 // 1: the last two levels are tested together from level K-2
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
  float xmax, ymax, wmax;  // upper bounds of the magnitudes of the leaf level's columns
};

BD_HD uint32_t f2u(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
}
BD_HD float u2f(uint32_t u) {
  float f;
  memcpy(&f, &u, 4);
  return f;
}

// nearest float (relative error below 2^-23 in every case)
BD_HD float to_float(int64_t v) { return (float)v; }
BD_HD float to_float(i128 v) {
  const u128 a = v < 0 ? (u128)(-v) : (u128)v;
  const float r = (float)((double)(uint64_t)(a >> 64) * 18446744073709551616.0 + (double)(uint64_t)a);
  return v < 0 ? -r : r;
}

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
  float* fl;               // the leaf level in single precision: level K-1 as fl[g] = x_g,
                           // fl[N + g] = y_g; with leaf3, level K-2 as float4 (u, v, w, 0) per point
  float* rl;               // leaf3: per point of the fixed sets, F(g) - F(base) and the base index
  MixedUniform<T>* uni;
  const uint16_t* last_pairs;  // pairs of the last component as p | q << 8 (global indices)
  const uint16_t* prev_pairs;  // pairs of component K-2 (leaf3)
  MixedSink sink{nullptr, nullptr, 0};
  Pairs14 cur;             // the pairs of the built levels
  int built = 0;           // levels 0..built-1 are reduced (state `built` is valid)
  int K, N;
  int kill = -1, kill_c = 0;  // this lane's last point found below a candidate, and its set

  BD_HD MixedWalker(Team t, const T* P_, const MixedShape* s, T* stack, float* f, MixedUniform<T>* u,
                    const uint16_t* lp, const uint16_t* pp)
      : tm(t), P(P_), sh(s), st(stack), fl(f), rl(f + 4 * s->N), uni(u), last_pairs(lp), prev_pairs(pp), K(s->K),
        N(s->N) {
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
    if (sh->leaf3 && j + 3 == K) {  // level K-2 for the 3-D leaf stage: (u, v, w) as float4
      uint32_t mu = 0, mv = 0, mw = 0;
      for (int g = tm.lane(); g < N; g += tm.lanes()) {
        const float u = to_float(put(j + 1, 0, g)), v = to_float(put(j + 1, 1, g)), w = to_float(put(j + 1, 2, g));
        fl[4 * g] = u;
        fl[4 * g + 1] = v;
        fl[4 * g + 2] = w;
        fl[4 * g + 3] = 0.f;
        mu = f2u(fabsf(u)) > mu ? f2u(fabsf(u)) : mu;
        mv = f2u(fabsf(v)) > mv ? f2u(fabsf(v)) : mv;
        mw = f2u(fabsf(w)) > mw ? f2u(fabsf(w)) : mw;
      }
      mu = tm.max_u32(mu);
      mv = tm.max_u32(mv);
      mw = tm.max_u32(mw);
      if (tm.lane() == 0) {
        uni->xmax = u2f(mu) * 1.0000005f;
        uni->ymax = u2f(mv) * 1.0000005f;
        uni->wmax = u2f(mw) * 1.0000005f;
      }
    }
    if (!sh->leaf3 && j + 2 == K) {  // the leaf level: single-precision copies and bounds of their magnitudes
      uint32_t mx = 0, my = 0;
      for (int g = tm.lane(); g < N; g += tm.lanes()) {
        const float x = to_float(put(j + 1, 0, g)), y = to_float(put(j + 1, 1, g));
        fl[g] = x;
        fl[N + g] = y;
        mx = f2u(fabsf(x)) > mx ? f2u(fabsf(x)) : mx;  // non-negative floats order as their bits
        my = f2u(fabsf(y)) > my ? f2u(fabsf(y)) : my;
      }
      mx = tm.max_u32(mx);
      my = tm.max_u32(my);
      if (tm.lane() == 0) {  // rounded up past the conversion error
        uni->xmax = u2f(mx) * 1.0000005f;
        uni->ymax = u2f(my) * 1.0000005f;
      }
    }
    if (tm.lane() == 0) uni->dv[j + 1] = vc;
    tm.sync();
    cur.set_pair(j, p, q);
    built = j + 1;
    return true;
  }

  // exact sign of f(z(g)) - f(z(b)) times sigma / d at the leaf (X, Y)
  BD_HD int exact_sign(T X, T Y, int g, int b) const {
    const int j = K - 1;
    return sgn(X * at(j, 1, g) - at(j, 0, g) * Y - (X * at(j, 1, b) - at(j, 0, b) * Y));
  }

  // All pairs of the last component under the built prefix (levels 0..K-2 fixed).
  //
  // Filter: with w = +-1 the wanted sign, t = w (X y_g - Y x_g - (X y_b - Y x_b)) is evaluated
  // in single precision from the rounded copies.  Every operand carries a conversion error below
  // u = 2^-24, so each of the four products is within 3.01 u of its exact value, and the three
  // differences add at most 3 u of the sum of the products' magnitudes: the computed t is within
  // 6.1 u (|X| (|y_g| + |y_b|) + |Y| (|x_g| + |x_b|)) <= 12.2 u (|X| ymax + |Y| xmax) of the
  // exact value.  eps = 2^-19 (|X| ymax + |Y| xmax) = 32 u (..) keeps a factor 2.6 over that for
  // the rounding of eps and of the bounds.  |t| > eps decides the sign; otherwise the point is
  // tested exactly.  Each lane first retries the point that rejected its previous candidate.
  BD_HD void leaves(MixedAcc& acc) {
    const int j = K - 1;
    const uint32_t np = sh->npairs[j];
    const int sd = sgn(uni->dv[j]);
    const bool filt = K >= 2;  // the raw level 0 has no single-precision copy
    const float xmax = filt ? uni->xmax : 0.f, ymax = filt ? uni->ymax : 0.f;
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
      const float wf = want > 0 ? 1.f : -1.f;
      const float Xw = to_float(X) * wf, Yw = to_float(Y) * wf;
      const float eps = 0x1p-19f * (fabsf(Xw) * ymax + fabsf(Yw) * xmax);
      // 1: strictly above, 0: on the cell's plane, -1: strictly below
      auto verdict = [&](int g, int b, float cbw) -> int {
        if (filt) {
          const float tt = (Xw * fl[N + g] - Yw * fl[g]) - cbw;
          if (tt > eps) return 1;
          if (tt < -eps) return -1;
        }
        return exact_sign(X, Y, g, b) * want;
      };
      bool below = false, on = false;
      if (kill >= 0) {
        const int i = kill_c;
        const int pi = i == j ? p : cur.p(i), qi = i == j ? q : cur.q(i);
        if (kill != pi && kill != qi)
          below = verdict(kill, pi, filt ? Xw * fl[N + pi] - Yw * fl[pi] : 0.f) < 0;
      }
      for (int i = 0; i < K && !below; ++i) {
        const int pi = i == j ? p : cur.p(i), qi = i == j ? q : cur.q(i);
        const float cbw = filt ? Xw * fl[N + pi] - Yw * fl[pi] : 0.f;
        for (int g = sh->first[i]; g < sh->first[i + 1]; ++g) {
          if (g == pi || g == qi) continue;
          const int v = verdict(g, pi, cbw);
          if (v < 0) {
            below = true;
            kill = g;
            kill_c = i;
            break;
          }
          on |= v == 0;
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
      if (sink.out) record(-1, -1, p, q, ax);
    }
  }

  // Exact verdict of point g against base b for the tuple whose last two pivot rows are
  // a = r(q1) - r(p1), c = r(q) - r(p) at level K-2 (1 above, 0 on, -1 below): level K-1 is
  // formed for the four rows only, and the test is the one of leaves().
  BD_HD int exact3(int p1, int q1, int p, int q, int g, int b, const Div& D) const {
    const int j = K - 2;
    const T a0 = at(j, 0, q1) - at(j, 0, p1), a1 = at(j, 1, q1) - at(j, 1, p1), a2 = at(j, 2, q1) - at(j, 2, p1);
    const int c = a0 != 0 ? 0 : 1, o = 1 - c;  // a's pivot column (det M != 0: a has one)
    const T ac = c == 0 ? a0 : a1, ao = c == 0 ? a1 : a0;
    auto x = [&](int r) { return bareiss(at(j, o, r), ac, at(j, c, r), ao, D); };
    auto y = [&](int r) { return bareiss(at(j, 2, r), ac, at(j, c, r), a2, D); };
    const T xp = x(p), X = x(q) - xp, Y = y(q) - y(p);
    const int want = sgn(X) * sgn(ac);
    return sgn(X * (y(g) - y(b)) - (x(g) - x(b)) * Y) * want;
  }

  // The 3-D leaf stage: every pair (p1, q1) of component K-2 with every pair (p, q) of the
  // last component, tested from level K-2 without forming level K-1.  With a, c the two pivot
  // rows and e = r(b) - r(base) (columns u, v, w of level K-2, d its divisor), eliminating a
  // and then c gives (Sylvester) X = det2 / d, det2 = a_u c_v - a_v c_u, and the test value of
  // the two-level rule a_piv det[a; c; e] / d^2, so b is above iff det[a; c; e] * det2 *
  // sign(d) > 0, and |det M| = |det2 / d|.
  //
  // Filter: a, c, n = a x c and n . e in single precision from the rounded copies F (and, for
  // the sets fixed above this node, from e = F(b) - F(base) formed once per node).  With U, V,
  // W bounds of |u|, |v|, |w|: each entry of a or c is within 4 u U (V, W) of its exact value
  // (u = 2^-24), each component of n within 48 u of its bound 8 V W (8 W U, 8 U V), and n . F(b)
  // - n . F(base) within 624 u U V W (n . e within 528 u U V W) of det[a; c; e] < 2^-14.7 U V W:
  // eps3 = 2^-13 U V W.  When U, V <= 2^22 and U V <= 2^21 every value in det2 is an integer
  // below 2^24 and det2 is exact in single precision; otherwise it is within 48 u U V <
  // 2^-18.4 U V, eps2 = 2^-16 U V, and values inside are taken from the stored integers.  Values
  // inside eps3 are decided exactly (exact3).
  //
  // Lane l takes the l-th contiguous block of the combinations, so consecutive candidates of a
  // lane share the pair of set K-2 (its row a is formed once) and, mostly, the point that
  // rejects them, which each lane retries first.
  BD_HD void leaves3(MixedAcc& acc) {
    const int j = K - 2;
    const uint32_t n1 = sh->npairs[j], n2 = sh->npairs[j + 1], total = n1 * n2;
    const int f2 = sh->first[j], f3 = sh->first[j + 1];
    const T d = uni->dv[j];
    const Div D = make_div(d);
    const int sd = sgn(d);
    const float U = uni->xmax, V = uni->ymax, Wm = uni->wmax;
    const float eps2 = 0x1p-16f * U * V, eps3 = 0x1p-13f * U * V * Wm;
    const bool small2 = U <= 0x1p22f && V <= 0x1p22f && U * V <= 0x1p21f;
    // the fixed sets: members and, per point, e = F(g) - F(base) with the base's index in .w
    uint64_t members = 0;
    for (int i = 0; i < j; ++i) members |= (1ull << cur.p(i)) | (1ull << cur.q(i));
    tm.sync();  // readers of the previous node's relative rows are done
    for (int g = tm.lane(); g < f2; g += tm.lanes()) {
      int i = 0;
      while (g >= sh->first[i + 1]) ++i;
      const int b = cur.p(i);
      rl[4 * g] = fl[4 * g] - fl[4 * b];
      rl[4 * g + 1] = fl[4 * g + 1] - fl[4 * b + 1];
      rl[4 * g + 2] = fl[4 * g + 2] - fl[4 * b + 2];
      rl[4 * g + 3] = (float)b;
    }
    tm.sync();
    const uint32_t lo = (uint32_t)(((uint64_t)total * tm.lane()) / tm.lanes());
    const uint32_t hi = (uint32_t)(((uint64_t)total * (tm.lane() + 1)) / tm.lanes());
    uint32_t t1 = lo / n2, t2 = lo % n2;
    int p1 = -1, q1 = -1;
    float a0 = 0, a1 = 0, a2 = 0;
    for (uint32_t t = lo; t < hi; ++t, ++t2) {
      if (t2 == n2) {
        t2 = 0;
        ++t1;
      }
      if ((int)(prev_pairs[t1] & 255) != p1 || (int)(prev_pairs[t1] >> 8) != q1) {
        p1 = prev_pairs[t1] & 255;
        q1 = prev_pairs[t1] >> 8;
        a0 = fl[4 * q1] - fl[4 * p1];
        a1 = fl[4 * q1 + 1] - fl[4 * p1 + 1];
        a2 = fl[4 * q1 + 2] - fl[4 * p1 + 2];
      }
      const uint16_t pc = last_pairs[t2];
      const int p = pc & 255, q = pc >> 8;
      const float c0 = fl[4 * q] - fl[4 * p], c1 = fl[4 * q + 1] - fl[4 * p + 1], c2 = fl[4 * q + 2] - fl[4 * p + 2];
      const float det2f = a0 * c1 - a1 * c0;
      int s2;
      T det2 = 0;
      bool have2 = false;
      if (small2) {
        if (det2f == 0.f) {
          ++acc.singular;
          continue;
        }
        s2 = det2f > 0 ? 1 : -1;
      } else if (fabsf(det2f) > eps2) {
        s2 = det2f > 0 ? 1 : -1;
      } else {
        det2 = (at(j, 0, q1) - at(j, 0, p1)) * (at(j, 1, q) - at(j, 1, p)) -
               (at(j, 1, q1) - at(j, 1, p1)) * (at(j, 0, q) - at(j, 0, p));
        have2 = true;
        if (det2 == 0) {
          ++acc.singular;
          continue;
        }
        s2 = sgn(det2);
      }
      s2 *= sd;  // b is above iff s2 * det[a; c; e] > 0
      const float w = s2 > 0 ? 1.f : -1.f;
      const float n0 = (a1 * c2 - a2 * c1) * w, n1v = (a2 * c0 - a0 * c2) * w, n2v = (a0 * c1 - a1 * c0) * w;
      const float nb1 = n0 * fl[4 * p1] + n1v * fl[4 * p1 + 1] + n2v * fl[4 * p1 + 2];
      const float nb2 = n0 * fl[4 * p] + n1v * fl[4 * p + 1] + n2v * fl[4 * p + 2];
      // the single-precision value tested for point g, and the point's base
      auto tval = [&](int g) -> float {
        const bool fixed = g < f2;
        const float* src = fixed ? rl : fl;
        const float sub = fixed ? 0.f : (g >= f3 ? nb2 : nb1);
        return n0 * src[4 * g] + n1v * src[4 * g + 1] + n2v * src[4 * g + 2] - sub;
      };
      auto member = [&](int g) -> bool {
        if (g < f2) return (members >> g) & 1;
        return g >= f3 ? (g == p || g == q) : (g == p1 || g == q1);
      };
      // 1 above, 0 on, -1 below
      auto decide = [&](int g, float tt) -> int {
        if (tt > eps3) return 1;
        if (tt < -eps3) return -1;
        return exact3(p1, q1, p, q, g, g < f2 ? (int)rl[4 * g + 3] : (g >= f3 ? p : p1), D);
      };
      bool below = kill >= 0 && !member(kill) && decide(kill, tval(kill)) == -1;
      bool on = false;
      for (int g = 0; g < N && !below; ++g) {
        if (member(g)) continue;
        const int v = decide(g, tval(g));
        if (v == -1) {
          below = true;
          kill = g;
        }
        on |= v == 0;
      }
      if (below) continue;
      if (on) {
        ++acc.ties;
        continue;
      }
      if (!have2)
        det2 = small2 ? (T)(int64_t)det2f
                      : (at(j, 0, q1) - at(j, 0, p1)) * (at(j, 1, q) - at(j, 1, p)) -
                            (at(j, 1, q1) - at(j, 1, p1)) * (at(j, 0, q) - at(j, 0, p));
      T ax = det2 / d;  // |det M| = |det2 / d|, an exact quotient
      ax = ax < 0 ? -ax : ax;
      acc.mv += (u128)ax;
      ++acc.cells;
      if (sink.out) record(p1, q1, p, q, ax);
    }
  }

  BD_HD void record(int p1, int q1, int p, int q, T ax) {
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
    if (p1 >= 0) {  // leaf3: level K-2's pair is not in the cursor
      r.idx[2 * (K - 2)] = (uint8_t)p1;
      r.idx[2 * (K - 2) + 1] = (uint8_t)q1;
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
    const int leaf_at = sh->leaf3 ? K - 2 : K - 1;  // the level whose state feeds the leaf stage
    if (L == leaf_at) {
      if (sh->leaf3) leaves3(acc);
      else leaves(acc);
      return;
    }
    // walk levels L..leaf_at-1; pair (p, q) of level j runs over component j in lexicographic order
    int j = L;
    int p = sh->first[j], q = p + 1;
    for (;;) {
      bool down = false;
      if (descend(j, p, q)) {
        if (j + 1 == leaf_at) {
          if (sh->leaf3) leaves3(acc);
          else leaves(acc);
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

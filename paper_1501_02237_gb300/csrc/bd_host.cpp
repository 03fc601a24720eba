// Host front end of the degree computation (Sec. 2-3 of the paper) and the CPU emulation of
// the GPU enumeration.  Plain C++17, no CUDA.
#include "bd_host.h"
#include "bd_teams.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <mutex>
#include <thread>
#ifdef BD_DEBUG
#include <cstdio>
#endif

#include "../../include/binodeg.h"

namespace bd {

namespace {

const i128 ENTRY_LIMIT = (i128)1 << 62;  // Smith-form entries stay below 2^62 so products fit i128

struct Mat {
  int r = 0, c = 0;
  std::vector<i128> a;
  Mat() {}
  Mat(int r_, int c_) : r(r_), c(c_), a((size_t)r_ * c_, 0) {}
  i128& at(int i, int j) { return a[(size_t)i * c + j]; }
  i128 at(int i, int j) const { return a[(size_t)i * c + j]; }
  static Mat eye(int n) {
    Mat m(n, n);
    for (int i = 0; i < n; ++i) m.at(i, i) = 1;
    return m;
  }
};

i128 iabs(i128 x) { return x < 0 ? -x : x; }

// extended Euclid: g = s a + t b = gcd(a, b) >= 0
void xgcd(i128 a, i128 b, i128& g, i128& s, i128& t) {
  i128 r0 = a, r1 = b, s0 = 1, s1 = 0, t0 = 0, t1 = 1;
  while (r1 != 0) {
    i128 q = r0 / r1;
    i128 tmp = r0 - q * r1; r0 = r1; r1 = tmp;
    tmp = s0 - q * s1; s0 = s1; s1 = tmp;
    tmp = t0 - q * t1; t0 = t1; t1 = tmp;
  }
  if (r0 < 0) { r0 = -r0; s0 = -s0; t0 = -t0; }
  g = r0; s = s0; t = t0;
}

// unimodular [[s, t], [u, v]] sending (a1, a2) to (g, 0) (Sec. 3); plain elimination when a1 | a2
void bezout2(i128 a1, i128 a2, i128& s, i128& t, i128& u, i128& v) {
  if (a2 % a1 == 0) { s = 1; t = 0; u = -(a2 / a1); v = 1; return; }
  i128 g;
  xgcd(a1, a2, g, s, t);
  u = -(a2 / g);
  v = a1 / g;
}

bool rows_op(Mat& X, int i, int j, i128 s, i128 t, i128 u, i128 v) {
  for (int c = 0; c < X.c; ++c) {
    i128 x = X.at(i, c), y = X.at(j, c);
    i128 nx = s * x + t * y, ny = u * x + v * y;
    if (iabs(nx) >= ENTRY_LIMIT || iabs(ny) >= ENTRY_LIMIT) return false;
    X.at(i, c) = nx; X.at(j, c) = ny;
  }
  return true;
}

bool cols_op(Mat& X, int i, int j, i128 s, i128 t, i128 u, i128 v) {
  for (int r = 0; r < X.r; ++r) {
    i128 x = X.at(r, i), y = X.at(r, j);
    i128 nx = s * x + t * y, ny = u * x + v * y;
    if (iabs(nx) >= ENTRY_LIMIT || iabs(ny) >= ENTRY_LIMIT) return false;
    X.at(r, i) = nx; X.at(r, j) = ny;
  }
  return true;
}

u128 ugcd(u128 a, u128 b) {
  while (b) { u128 r = a % b; a = b; b = r; }
  return a;
}

// b^{Q_0} == 1 exactly (Eq. consistency), b_i = -c_{i,2} / c_{i,1}.  Numbers are split over a
// coprime base (repeated gcd refinement), so exponents can be compared without factoring.
bool consistent(const int64_t* coef, int m, const Mat& R, std::string& err, bool& ok) {
  std::vector<u128> num(m), den(m);
  std::vector<int> neg(m);
  for (int i = 0; i < m; ++i) {
    const int64_t n1 = coef[4 * i], d1 = coef[4 * i + 1], n2 = coef[4 * i + 2], d2 = coef[4 * i + 3];
    if (n1 == 0 || d1 == 0 || n2 == 0 || d2 == 0) { err = "coefficients and denominators must be nonzero"; return false; }
    i128 p = -(i128)n2 * d1, q = (i128)d2 * n1;  // b_i = p / q
    neg[i] = (p < 0) != (q < 0);
    u128 up = (u128)iabs(p), uq = (u128)iabs(q);
    u128 g = ugcd(up, uq);
    num[i] = up / g;
    den[i] = uq / g;
  }
  std::vector<u128> base;
  for (int i = 0; i < m; ++i) {
    if (num[i] > 1) base.push_back(num[i]);
    if (den[i] > 1) base.push_back(den[i]);
  }
  for (bool changed = true; changed;) {
    changed = false;
    std::sort(base.begin(), base.end());
    base.erase(std::unique(base.begin(), base.end()), base.end());
    for (size_t i = 0; i < base.size() && !changed; ++i)
      for (size_t j = i + 1; j < base.size() && !changed; ++j) {
        u128 g = ugcd(base[i], base[j]);
        if (g > 1) {
          u128 x = base[i] / g, y = base[j] / g;
          base.erase(base.begin() + j);
          base.erase(base.begin() + i);
          if (x > 1) base.push_back(x);
          if (y > 1) base.push_back(y);
          base.push_back(g);
          changed = true;
        }
      }
  }
  auto val = [](u128 x, u128 b) {
    int v = 0;
    while (x % b == 0) { x /= b; ++v; }
    return v;
  };
  ok = true;
  for (int j = 0; j < R.r && ok; ++j) {
    i128 sgn = 0;
    for (int i = 0; i < m; ++i)
      if (neg[i]) sgn += R.at(j, i);
    if (sgn % 2 != 0) ok = false;
    for (size_t b = 0; b < base.size() && ok; ++b) {
      i128 e = 0;
      for (int i = 0; i < m; ++i) {
        const int v = val(num[i], base[b]) - val(den[i], base[b]);
        if (v) e += R.at(j, i) * v;
      }
      if (e != 0) ok = false;
    }
  }
  return true;
}

// LLL reduction (delta = 0.99) of the rows of B (d x n).  Row operations are exact integer
// operations; Gram-Schmidt data is kept in double only to steer them (every operation is
// unimodular, so the rows always span the same lattice whatever the doubles decide).  To keep
// the doubles trustworthy with large entries, the coefficients of row k are recomputed from the
// exact integer row before each use and size reduction is repeated until it makes only small
// corrections (the usual floating-point LLL safeguard).
template <class T>
bool lll_t(std::vector<T>& B, int d, int n) {
  const T limit = (T)1 << 62;
  auto tabs_ = [](T x) { return x < 0 ? -x : x; };
  if (d <= 1) return true;
  std::vector<double> bs((size_t)d * n), bn(d, 0.0), mu((size_t)d * d, 0.0);
  auto row = [&](int i) { return &B[(size_t)i * n]; };
  auto set_row = [&](int k) -> bool {  // size-reduce b_k, then b*_k and |b*_k|^2
    for (int iter = 0; iter < 100; ++iter) {
      for (int j = 0; j < k; ++j) {
        double dot = 0;
        for (int c = 0; c < n; ++c) dot += (double)row(k)[c] * bs[(size_t)j * n + c];
        mu[(size_t)k * d + j] = bn[j] > 0 ? dot / bn[j] : 0.0;
      }
      bool large = false;
      for (int j = k - 1; j >= 0; --j) {
        const double m = mu[(size_t)k * d + j];
        if (std::fabs(m) <= 0.51) continue;
        if (std::fabs(m) > 4e18) return false;
        const T q = (T)std::llround(m);
        for (int c = 0; c < n; ++c) {
          T t, v;
          if (__builtin_mul_overflow(q, row(j)[c], &t) || __builtin_sub_overflow(row(k)[c], t, &v)) return false;
          if (tabs_(v) >= limit) return false;
          row(k)[c] = v;
        }
        for (int l = 0; l < j; ++l) mu[(size_t)k * d + l] -= (double)q * mu[(size_t)j * d + l];
        mu[(size_t)k * d + j] -= (double)q;
        if (tabs_(q) > ((T)1 << 20)) large = true;
      }
      if (!large) break;
    }
    for (int c = 0; c < n; ++c) {
      double v = (double)row(k)[c];
      for (int j = 0; j < k; ++j) v -= mu[(size_t)k * d + j] * bs[(size_t)j * n + c];
      bs[(size_t)k * n + c] = v;
    }
    double s2 = 0;
    for (int c = 0; c < n; ++c) s2 += bs[(size_t)k * n + c] * bs[(size_t)k * n + c];
    bn[k] = s2;
    return true;
  };
  if (!set_row(0)) return false;
  int k = 1;
  long guard = 0;
  while (k < d) {
    if (++guard > 2000000) return true;  // still a basis of the same lattice
    if (!set_row(k)) return false;
    const double m = mu[(size_t)k * d + k - 1];
    if (bn[k] < (0.99 - m * m) * bn[k - 1]) {
      for (int c = 0; c < n; ++c) std::swap(row(k)[c], row(k - 1)[c]);
      k = std::max(k - 1, 1);
      if (k == 1 && !set_row(0)) return false;
    } else {
      ++k;
    }
  }
  return true;
}

bool lll(std::vector<i128>& B, int d, int n) { return lll_t<i128>(B, d, n); }

// checked i128 arithmetic
bool mul_ok(i128 a, i128 b, i128& r) { return !__builtin_mul_overflow(a, b, &r); }
bool add_ok(i128 a, i128 b, i128& r) { return !__builtin_add_overflow(a, b, &r); }

// Basis (rows of U, d x rows) of the lattice {p in Z^rows : p M = 0} for M (rows x cols).
// Column by column: the values v = U m_j of the current basis are sent to (g, 0, .., 0) by the
// unimodular 2x2 Bezout steps of Sec. 3 applied to the basis rows; the row carrying g leaves
// the basis, the others span exactly the vectors of the old lattice orthogonal to m_j.  The
// basis is LLL-reduced whenever its entries grow, and after the last column when reduce_last
// (the kernel points themselves; bases used only for determinants skip it).  The result is
// saturated: it is a basis of ker(M) intersected with Z^rows.
template <class T>
bool kernel_rows_t(const Mat& M, Mat& U, std::string& err, bool reduce_last) {
  auto tabs_ = [](T x) { return x < 0 ? -x : x; };
  auto mul_t = [](T a, T b, T& r) { return !__builtin_mul_overflow(a, b, &r); };
  auto add_t = [](T a, T b, T& r) { return !__builtin_add_overflow(a, b, &r); };
  auto entry = [&](int t, int j, T& x) {  // M's entry in T
    const i128 v = M.at(t, j);
    x = (T)v;
    return (i128)x == v;
  };
  const int n = M.r, m = M.c;
  std::vector<std::vector<T>> B(n, std::vector<T>(n, 0));
  for (int i = 0; i < n; ++i) B[i][i] = 1;
  for (int j = 0; j < m && !B.empty(); ++j) {
    const int d = (int)B.size();
    std::vector<T> v(d, 0);
    for (int i = 0; i < d; ++i)
      for (int t = 0; t < n; ++t) {
        T pr, mt;
        if (!entry(t, j, mt) || !mul_t(B[i][t], mt, pr) || !add_t(v[i], pr, v[i])) { err = "kernel values overflow"; return false; }
      }
    // Euclid on the value vector: reduce every value modulo the smallest nonzero one (row
    // operations b_i -= q b_min) until a single nonzero value g = gcd remains; this keeps the
    // multipliers no larger than the values themselves.  If the rows still grow, LLL-reduce
    // them (a unimodular change of basis; the values are recomputed) and continue.
    bool all_zero = true;
    for (int i = 0; i < d; ++i)
      if (v[i] != 0) all_zero = false;
    if (all_zero) continue;  // the whole current lattice is orthogonal to this column
    int resets = 0;  // mid-way LLL passes on this column (bounded: a lattice whose kernel
                     // rows must be long would otherwise cycle between growth and reduction)
    for (int guard = 0;; ++guard) {
      int piv = -1, nz = 0;
      for (int i = 0; i < d; ++i)
        if (v[i] != 0) {
          ++nz;
          if (piv < 0 || tabs_(v[i]) < tabs_(v[piv])) piv = i;
        }
      if (nz <= 1) {
        std::swap(B[0], B[piv]);
        std::swap(v[0], v[piv]);
        break;
      }
      T big = 0;
      for (int i = 0; i < d; ++i) {
        if (i == piv || v[i] == 0) continue;
        const bool narrow = v[i] > -((T)1 << 62) && v[i] < ((T)1 << 62) && v[piv] > -((T)1 << 62) &&
                            v[piv] < ((T)1 << 62);
        if (!narrow && sizeof(T) == 8) { err = "kernel values leave 62 bits"; return false; }
        T q = narrow ? (T)((int64_t)v[i] / (int64_t)v[piv]) : v[i] / v[piv];  // truncation
        const T r = v[i] - q * v[piv];  // smaller than |v_piv|
        if (tabs_(r) > tabs_(v[piv]) - tabs_(r)) q += ((r > 0) == (v[piv] > 0)) ? 1 : -1;  // nearest quotient
        for (int c = 0; c < n; ++c) {
          T t;
          if (!mul_t(q, B[piv][c], t) || __builtin_sub_overflow(B[i][c], t, &B[i][c])) { err = "kernel basis overflow"; return false; }
          big = std::max(big, tabs_(B[i][c]));
        }
        v[i] -= q * v[piv];
      }
      if (big > ((T)1 << 40) && resets < 3) {
        ++resets;
        std::vector<T> flat;
        for (auto& row : B) flat.insert(flat.end(), row.begin(), row.end());
        if (!lll_t<T>(flat, d, n)) { err = "kernel basis entries exceed 2^62"; return false; }
        for (int i = 0; i < d; ++i) {
          v[i] = 0;
          for (int c = 0; c < n; ++c) {
            B[i][c] = flat[(size_t)i * n + c];
            T pr, mt;
            if (!entry(c, j, mt) || !mul_t(B[i][c], mt, pr) || !add_t(v[i], pr, v[i])) { err = "kernel values overflow"; return false; }
          }
        }
      }
      if (guard > 8000) { err = "kernel elimination did not converge"; return false; }
    }
    B.erase(B.begin());
    T big = 0;
    for (auto& r : B)
      for (T x : r) big = std::max(big, tabs_(x));
    const bool last_col = reduce_last && (j == m - 1);
#ifdef BD_DEBUG
    {
      double lb = 0;
      for (auto& r : B) for (T x : r) lb = std::max(lb, (double)tabs_(x));
      double vb = 0;
      fprintf(stderr, "kernel_rows %dx%d col %d d=%zu big=%.3g\n", n, m, j, B.size(), lb);
    }
#endif
    if (!B.empty() && (big > ((T)1 << 16) || last_col)) {
      std::vector<T> flat;
      for (auto& row : B) flat.insert(flat.end(), row.begin(), row.end());
      if (!lll_t<T>(flat, (int)B.size(), n)) { err = "kernel basis entries exceed 2^62"; return false; }
      for (size_t i = 0; i < B.size(); ++i)
        for (int c = 0; c < n; ++c) B[i][c] = flat[i * n + c];
    }
  }
  U = Mat((int)B.size(), n);
  for (size_t i = 0; i < B.size(); ++i)
    for (int c = 0; c < n; ++c) {
      if (tabs_(B[i][c]) >= ((T)1 << 62)) { err = "kernel basis entries exceed 2^62"; return false; }
      U.at((int)i, c) = (i128)B[i][c];
    }
  return true;
}

// int64 arithmetic while every value fits (the common case), else the same steps in int128
// (identical decisions, so identical results)
bool kernel_rows(const Mat& M, Mat& U, std::string& err, bool reduce_last = true) {
  if (kernel_rows_t<int64_t>(M, U, err, reduce_last)) return true;
  err.clear();
  return kernel_rows_t<i128>(M, U, err, reduce_last);
}

Mat transpose(const Mat& A) {
  Mat T(A.c, A.r);
  for (int i = 0; i < A.r; ++i)
    for (int j = 0; j < A.c; ++j) T.at(j, i) = A.at(i, j);
  return T;
}

// exact determinant of a k x k i128 matrix (fraction-free elimination, overflow-checked).
// Every intermediate value is a minor of a, bounded by the product of its row norms
// (Hadamard); below 2^62 the elimination runs in 64 bits with the exact 2-adic division of
// the GPU walker, otherwise in checked 128-bit arithmetic.
bool det_exact(std::vector<i128> a, int k, i128& det) {
  double lg = 0;
  bool small = true;
  for (int r = 0; r < k && small; ++r) {
    double n2 = 0;
    for (int j = 0; j < k; ++j) {
      const i128 x = a[(size_t)r * k + j];
      if (iabs(x) >= ((i128)1 << 62)) small = false;
      n2 += (double)x * (double)x;
    }
    lg += 0.5 * std::log2(std::max(n2, 1.0));
  }
  if (small && lg < 61.9) {
    std::vector<int64_t> b(a.begin(), a.end());
    Div64 D = make_div((int64_t)1);
    int sign = 1;
    for (int c = 0; c < k; ++c) {
      int p = -1;
      for (int r = c; r < k; ++r)
        if (b[(size_t)r * k + c] != 0) { p = r; break; }
      if (p < 0) { det = 0; return true; }
      if (p != c) {
        for (int j = 0; j < k; ++j) std::swap(b[(size_t)c * k + j], b[(size_t)p * k + j]);
        sign = -sign;
      }
      const int64_t pc = b[(size_t)c * k + c];
      for (int r = c + 1; r < k; ++r) {
        const int64_t rc = b[(size_t)r * k + c];
        for (int j = c + 1; j < k; ++j)
          b[(size_t)r * k + j] = bareiss(b[(size_t)r * k + j], pc, rc, b[(size_t)c * k + j], D);
        b[(size_t)r * k + c] = 0;
      }
      D = make_div(pc);
    }
    det = k == 0 ? 1 : (i128)sign * b[(size_t)(k - 1) * k + (k - 1)];
    return true;
  }
  i128 prev = 1;
  int sign = 1;
  for (int c = 0; c < k; ++c) {
    int p = -1;
    for (int r = c; r < k; ++r)
      if (a[(size_t)r * k + c] != 0) { p = r; break; }
    if (p < 0) { det = 0; return true; }
    if (p != c) {
      for (int j = 0; j < k; ++j) std::swap(a[(size_t)c * k + j], a[(size_t)p * k + j]);
      sign = -sign;
    }
    for (int r = c + 1; r < k; ++r) {
      for (int j = c + 1; j < k; ++j) {
        i128 x, y;
        if (!mul_ok(a[(size_t)r * k + j], a[(size_t)c * k + c], x) || !mul_ok(a[(size_t)r * k + c], a[(size_t)c * k + j], y))
          return false;
        a[(size_t)r * k + j] = (x - y) / prev;  // exact (Bareiss)
      }
      a[(size_t)r * k + c] = 0;
    }
    prev = a[(size_t)c * k + c];
  }
  det = sign * a[(size_t)(k - 1) * k + (k - 1)];
  if (k == 0) det = 1;
  return true;
}

// rows I and columns J of an r x r submatrix of A that is nonsingular modulo a prime.  The
// primes are below 2^31 (products reduce with 64-bit arithmetic); the rank drops modulo p only
// when p divides every r x r minor, i.e. the torsion, and torsion < 2^63 is divisible by at
// most two of them, so one of the first three always serves.
bool pivot_sets(const Mat& A, int r, std::vector<int>& I, std::vector<int>& J) {
  const uint64_t primes[4] = {2147483647ull, 2147483629ull, 2147483587ull, 2147483579ull};
  for (uint64_t pr : primes) {
    const int n = A.r, m = A.c;
    std::vector<uint64_t> M((size_t)n * m);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < m; ++j) {
        const i128 a = A.at(i, j);
        int64_t x = (a >= -((i128)1 << 62) && a < ((i128)1 << 62)) ? (int64_t)a % (int64_t)pr
                                                                    : (int64_t)(a % (i128)pr);
        if (x < 0) x += (int64_t)pr;
        M[(size_t)i * m + j] = (uint64_t)x;
      }
    auto mulmod = [pr](uint64_t a, uint64_t b) { return a * b % pr; };
    auto inv = [&](uint64_t a) {
      uint64_t r = 1, e = pr - 2;
      while (e) { if (e & 1) r = mulmod(r, a); a = mulmod(a, a); e >>= 1; }
      return r;
    };
    std::vector<int> used(n, 0);
    I.clear();
    J.clear();
    for (int c = 0; c < m && (int)I.size() < r; ++c) {
      int p = -1;
      for (int i = 0; i < n; ++i)
        if (!used[i] && M[(size_t)i * m + c]) { p = i; break; }
      if (p < 0) continue;
      used[p] = 1;
      I.push_back(p);
      J.push_back(c);
      const uint64_t ip = inv(M[(size_t)p * m + c]);
      for (int i = 0; i < n; ++i) {
        if (used[i] || !M[(size_t)i * m + c]) continue;
        const uint64_t f = mulmod(M[(size_t)i * m + c], ip);
        for (int cc = c; cc < m; ++cc)
          M[(size_t)i * m + cc] = (M[(size_t)i * m + cc] + pr - mulmod(f, M[(size_t)p * m + cc])) % pr;
      }
    }
    if ((int)I.size() == r) {
      std::sort(I.begin(), I.end());
      return true;
    }
  }
  return false;
}

}  // namespace

// The invariants of the Smith form P A Q = D (Eq. smith) that the degree needs, computed
// without forming P and Q (whose entries can grow to hundreds of bits):
//   * P_0: any basis of the saturated left kernel {p : p A = 0} (the rows of P_0 in
//     Eq. rank-decomp are one such basis; Prop. 4's volume is the same for every basis);
//   * rank r = n - dim of that kernel;
//   * Q_0: a basis of the right kernel {q : A q = 0}, for the consistency test b^{Q_0} = 1;
//   * |prod d_j| = gcd of the r x r minors of A (Prop. 1).  With X a basis of the saturated
//     column lattice (n x r) and S of the saturated row lattice (r x m), A = X Y and Y = T S
//     with T r x r integer, so by Cauchy-Binet, for any nonsingular A_{I,J}:
//         |prod d_j| = |det T| = |det A_{I,J}| / (|det X_I| |det S_J|).
int reduce_system(const int64_t* A, int n, int m, const int64_t* coef, Reduction& out, std::string& err) {
  Mat M(n, m);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) M.at(i, j) = A[(size_t)i * m + j];
  Mat P0, R;
  if (!kernel_rows(M, P0, err)) return BD_ERR_OVERFLOW;
  const int d = P0.r, rank = n - d;
  if (!kernel_rows(transpose(M), R, err, false)) return BD_ERR_OVERFLOW;
  if (R.r != m - rank) { err = "inconsistent kernel dimensions"; return BD_ERR_OVERFLOW; }
  out.rank = rank;
  out.dim = d;
  out.torsion = 1;
  if (rank > 0) {
    // |det X_I| and |det S_J| from the complementary minors of the orthogonal complements
    // already at hand: for a saturated lattice and its saturated orthogonal complement the
    // Plucker coordinates agree up to sign on complementary index sets (Jacobi's complementary
    // minor theorem applied to a unimodular completion of a basis), so
    // |det X_I| = |det P_0 restricted to the columns outside I| and likewise for S and R.
    std::vector<int> I, J;
    if (!pivot_sets(M, rank, I, J)) { err = "rank selection failed"; return BD_ERR_OVERFLOW; }
    std::vector<int> Ic, Jc;
    for (int t = 0, u = 0; t < n; ++t) {
      if (u < rank && I[u] == t) ++u;
      else Ic.push_back(t);
    }
    std::vector<int> Js(J);
    std::sort(Js.begin(), Js.end());
    for (int t = 0, u = 0; t < m; ++t) {
      if (u < rank && Js[u] == t) ++u;
      else Jc.push_back(t);
    }
    std::vector<i128> a((size_t)rank * rank), x((size_t)d * d), sm(Jc.size() * Jc.size());
    for (int u = 0; u < rank; ++u)
      for (int v = 0; v < rank; ++v) a[(size_t)u * rank + v] = M.at(I[u], J[v]);
    for (int u = 0; u < d; ++u)
      for (int v = 0; v < d; ++v) x[(size_t)u * d + v] = P0.at(u, Ic[v]);
    const int e = (int)Jc.size();
    for (int u = 0; u < e; ++u)
      for (int v = 0; v < e; ++v) sm[(size_t)u * e + v] = R.at(u, Jc[v]);
    i128 da, dx, ds;
    if (!det_exact(a, rank, da) || !det_exact(x, d, dx) || !det_exact(sm, e, ds)) {
      err = "torsion determinants exceed 2^127";
      return BD_ERR_OVERFLOW;
    }
    if (da == 0 || dx == 0 || ds == 0 || da % (dx * ds) != 0) { err = "torsion identity failed"; return BD_ERR_OVERFLOW; }
    const i128 t = iabs(da / (dx * ds));
    if (t >> 63) { err = "torsion exceeds 2^63"; return BD_ERR_OVERFLOW; }
    out.torsion = (uint64_t)t;
  }
  out.consistent = true;
  if (coef && rank < m) {
    bool ok = true;
    if (!consistent(coef, m, R, err, ok)) return BD_ERR_ARG;
    out.consistent = ok;
  }
  out.points.assign((size_t)(n + 1) * d, 0);
  out.max_abs_coord = 0;
  if (d == 0) return BD_OK;
  // the points are the columns of the (LLL-reduced) kernel basis (Prop. 4), then the origin
  for (int q = 0; q < n; ++q)
    for (int i = 0; i < d; ++i) {
      const i128 v = P0.at(i, q);
      // the enumeration takes coordinates below 2^40; a segment (d = 1) has a closed form
      if (d > 1 && iabs(v) >= ((i128)1 << 40)) { err = "kernel point coordinate exceeds 2^40"; return BD_ERR_OVERFLOW; }
      out.points[(size_t)q * d + i] = (int64_t)v;
      out.max_abs_coord = std::max<int64_t>(out.max_abs_coord, (int64_t)iabs(v));
    }
  return BD_OK;
}

double hadamard_log2(const int64_t* pts, const int64_t* lifts, int npts, int k, int64_t max_lift_spread,
                     double* coord) {
  // Column-wise Hadamard bound for the (K+1) x (K+1) lifted difference matrices: for column c
  // and base point s, the K+1 largest squared differences |a_q[c] - a_s[c]|^2 bound the
  // squared column norm; the bound is the product over columns of the worst base point
  // (each factor at least 1, so it also bounds every smaller minor).
  double total = 0, coords = 0;
  std::vector<double> sq(npts);
  for (int c = 0; c <= k; ++c) {
    double best = 1.0;
    for (int s = 0; s < npts; ++s) {
      for (int q = 0; q < npts; ++q) {
        double diff;
        if (c < k) diff = (double)(pts[(size_t)q * k + c] - pts[(size_t)s * k + c]);
        else if (lifts) diff = (double)(lifts[q] - lifts[s]);
        else diff = (double)max_lift_spread;
        sq[q] = diff * diff;
      }
      std::sort(sq.begin(), sq.end(), [](double a, double b) { return a > b; });
      double sum = 0;
      for (int i = 0; i < std::min(k + 1, npts); ++i) sum += sq[i];
      best = std::max(best, sum);
    }
    total += 0.5 * std::log2(best);
    if (c < k) coords = total;
  }
  if (coord) *coord = coords;
  return total;
}

int choose_path(double coord_bits, double full_bits) {
  // margins cover the rounding of the double-precision logarithms
  if (full_bits < 126.99) {
    if (full_bits < 62.99) return coord_bits < 30.99 ? 0 : 1;
    return 2;
  }
  return -1;
}



// the colex decode table the enumeration kernel reads, for the host emulation
const uint32_t* colex_table() {
  static const std::vector<uint32_t> t = [] {
    std::vector<uint32_t> v(kTriEntries);
    fill_colex_table(v.data());
    return v;
  }();
  return t.data();
}

template <class TC, class TL>
void lockstep_run(bool five, const int64_t* P, int N, int K, const std::vector<Item>& items,
                  const std::vector<Range>* ranges, int width, Acc& acc, const CellSink* sink) {
  LockstepShared sh(width);
  std::vector<TC> sc((size_t)N * stack_entries(K));
  std::vector<TL> sl((size_t)N * K);
  std::vector<float> fl((size_t)8 * N);
  std::vector<Uniform<TC>> uni(1);  // one copy for the team, as in a warp's shared memory
  std::vector<Acc> part(width);
  std::vector<std::thread> th;
  for (int l = 0; l < width; ++l)
    th.emplace_back([&, l] {
      LockstepTeam tm{&sh, l};
      Walker<TC, TL, LockstepTeam> W(tm, P, N, K, N, sc.data(), sl.data(), fl.data(), uni.data());
      W.tri = colex_table();
      W.use5 = five;
      if (sink) W.sink = *sink;
      Acc a{};
      if (ranges) {
        for (const Range& r : *ranges)
          for (uint32_t i = r.first; i < r.first + r.count; ++i) W.run_item(items[i], a);
      } else {
        for (const Item& it : items) W.run_item(it, a);
      }
      part[l] = a;
    });
  for (auto& t : th) t.join();
  acc = Acc{};
  for (auto& a : part) {
    acc.nvol += a.nvol;
    acc.cells += a.cells;
    acc.singular += a.singular;
    acc.ties += a.ties;
  }
}

template <class TC, class TL>
void host_run(bool five, const int64_t* P, int N, int K, const std::vector<Item>& items,
              const std::vector<Range>* ranges, int threads, Acc& acc, const CellSink* sink) {
  std::atomic<size_t> next(0);
  std::vector<Acc> part(std::max(1, threads));
  const size_t units = ranges ? ranges->size() : items.size();
  auto work = [&](int tid) {
    HostTeam tm;
    std::vector<TC> sc((size_t)N * stack_entries(K));
    std::vector<TL> sl((size_t)N * K);
    std::vector<float> fl((size_t)8 * N);
    std::vector<Uniform<TC>> uni(1);
    Walker<TC, TL, HostTeam> W(tm, P, N, K, N, sc.data(), sl.data(), fl.data(), uni.data());
    W.tri = colex_table();
    W.use5 = five;
    if (sink) W.sink = *sink;
    Acc a{};
    for (;;) {
      const size_t u = next.fetch_add(1);
      if (u >= units) break;
      const Range r = ranges ? (*ranges)[u] : Range{(uint32_t)u, 1};
      for (uint32_t i = r.first; i < r.first + r.count; ++i) W.run_item(items[i], a);
    }
    part[tid] = a;
  };
  if (threads <= 1) {
    work(0);
  } else {
    std::vector<std::thread> th;
    for (int t = 0; t < threads; ++t) th.emplace_back(work, t);
    for (auto& t : th) t.join();
  }
  acc = Acc{};
  for (auto& a : part) {
    acc.nvol += a.nvol;
    acc.cells += a.cells;
    acc.singular += a.singular;
    acc.ties += a.ties;
  }
}

void host_enumerate(int path, bool five, const int64_t* P, int N, int K, const std::vector<Item>& items, int threads, Acc& acc,
                    int team_width, const std::vector<Range>* ranges, const CellSink* sink) {
  if (team_width > 1) {  // one team walks every range in order
    if (path == 0) lockstep_run<int32_t, int64_t>(five, P, N, K, items, ranges, team_width, acc, sink);
    else if (path == 1) lockstep_run<int64_t, int64_t>(five, P, N, K, items, ranges, team_width, acc, sink);
    else lockstep_run<i128, i128>(five, P, N, K, items, ranges, team_width, acc, sink);
    return;
  }
  if (path == 0) host_run<int32_t, int64_t>(five, P, N, K, items, ranges, threads, acc, sink);
  else if (path == 1) host_run<int64_t, int64_t>(five, P, N, K, items, ranges, threads, acc, sink);
  else host_run<i128, i128>(five, P, N, K, items, ranges, threads, acc, sink);
}

}  // namespace bd

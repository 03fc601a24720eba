// Start solutions of the witness-set homotopy, cell by cell (Sec. 6): for a cell {a_0 .. a_k}
// of the lifting's triangulation and generic coefficients C, the start system
// C (y^{a_0}, .., y^{a_k})^T = 0 (Eq. affine-cut-starting) reduces to the binomial system
// y^{a_j - a_k} = kappa_j / kappa_k, j < k, kappa_j = (-1)^j det(C without column j)
// (Eq. affine-cut-eliminated), whose |det E| solutions (E: rows a_j - a_k) are
//     y = exp(E^-1 (log b + 2 pi i m)),  m over representatives of Z^k / E Z^k.
// The representatives are the box 0 <= m_i < h_i of the lower-triangular column Hermite form
// of E (h_i its diagonal), and E^-1 = adj(E) / det E is exact, so the phase of every solution
// is an exact fraction of a turn.  Per cell, the host prepares a StartCell; every solution is
// then independent (start_solution), one GPU thread each.
#pragma once

#include <math.h>
#include <stdint.h>

#include "bd_core.cuh"
#include "bd_lifts.h"

namespace bd {

struct StartCell {
  int64_t det;               // nonzero; E^-1 = adj / det (sign from the elimination's row order)
  int64_t h[KMAX];           // diagonal of the column Hermite form of E (positive)
  int64_t adj[KMAX * KMAX];  // det E^-1, row-major
  int32_t E[KMAX * KMAX];    // the exponent matrix, row-major (rows: equations)
  double base_re[KMAX];      // Re E^-1 log b = adj log|b| / det
  double base_im[KMAX];      // Im E^-1 log b = adj arg b / det
  double b_re[KMAX], b_im[KMAX];  // the right-hand sides (residual check)
};

// the coefficient generator: unit complex numbers exp(2 pi i u) on a SplitMix64 stream of their own
BD_HD uint64_t coef_stream_seed(uint64_t coef_seed) { return splitmix_mix(coef_seed ^ 0xC2B2AE3D27D4EB4Full); }
BD_HD double coef_turns(uint64_t stream, int npts, int i, int q) {
  const uint64_t h = splitmix_mix(stream + (uint64_t)(i * npts + q + 1) * 0x9E3779B97F4A7C15ull);
  return (double)(h >> 11) * (1.0 / 9007199254740992.0);  // 2^-53
}

// solution t (0 <= t < |det|) of cell sc, written as k complex numbers (re, im interleaved)
BD_HD void start_solution(const StartCell& sc, int k, uint64_t t, double* out) {
  int64_t m[KMAX];
  for (int i = 0; i < k; ++i) {  // mixed-radix digits of t in the box of the Hermite diagonal
    m[i] = (int64_t)(t % (uint64_t)sc.h[i]);
    t /= (uint64_t)sc.h[i];
  }
  const int64_t D = sc.det < 0 ? -sc.det : sc.det;
  for (int i = 0; i < k; ++i) {
    i128 num = 0;
    for (int j = 0; j < k; ++j) num += (i128)sc.adj[i * k + j] * m[j];
    if (sc.det < 0) num = -num;
    int64_t r = (int64_t)(num % D);
    if (r < 0) r += D;
    const double turns = (double)r / (double)D;  // exact fraction of a turn, rounded once
    const double ang = sc.base_im[i] + 6.283185307179586 * turns;
    const double mag = exp(sc.base_re[i]);
    out[2 * i] = mag * cos(ang);
    out[2 * i + 1] = mag * sin(ang);
  }
}

// A complex number as (re + i im) * 2^ex, rescaled to max(|re|, |im|) in [0.5, 1) whenever the
// mantissa drifts far from 1, so that the powers and products below neither overflow nor
// underflow however far |y| is from 1.
struct ScaledCx {
  double re, im;
  int64_t ex;
};

BD_HD void rescale(ScaledCx& z) {
  const double a = fabs(z.re) > fabs(z.im) ? fabs(z.re) : fabs(z.im);
  if (a == 0 || !(a < INFINITY)) return;
  int s;
  frexp(a, &s);
  z.re = ldexp(z.re, -s);
  z.im = ldexp(z.im, -s);
  z.ex += s;
}

// Mantissas are kept within [2^-400, 2^400], so one product of two of them is still a normal
// double; only a mantissa that leaves the range is rescaled.
BD_HD void keep_in_range(ScaledCx& z) {
  const double m = fabs(z.re) > fabs(z.im) ? fabs(z.re) : fabs(z.im);
  if (!(m > 0x1p-400 && m < 0x1p+400)) rescale(z);
}

BD_HD ScaledCx scaled_mul(const ScaledCx& a, const ScaledCx& b) {
  ScaledCx z{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re, a.ex + b.ex};
  keep_in_range(z);
  return z;
}

// max over the cell's equations of |y^{E_j} / b_j - 1| for one solution y (k complex numbers)
BD_HD double start_residual(const StartCell& sc, int k, const double* y) {
  ScaledCx pos[KMAX], neg[KMAX];  // y_i and 1 / y_i, scaled
  for (int i = 0; i < k; ++i) {
    pos[i] = ScaledCx{y[2 * i], y[2 * i + 1], 0};
    keep_in_range(pos[i]);
    const double n2 = pos[i].re * pos[i].re + pos[i].im * pos[i].im;  // 1/y = conj(y) / |y|^2
    neg[i] = ScaledCx{pos[i].re / n2, -pos[i].im / n2, -pos[i].ex};
    keep_in_range(neg[i]);
  }
  double worst = 0;
  for (int j = 0; j < k; ++j) {
    ScaledCx p{1, 0, 0};
    for (int i = 0; i < k; ++i) {
      int64_t e = sc.E[j * k + i];
      ScaledCx base = e < 0 ? neg[i] : pos[i];
      e = e < 0 ? -e : e;
      while (e) {  // square and multiply
        if (e & 1) p = scaled_mul(p, base);
        e >>= 1;
        if (e) base = scaled_mul(base, base);
      }
    }
    // |p / b - 1| = |p - b| / |b|, both brought to b's binary exponent
    ScaledCx b{sc.b_re[j], sc.b_im[j], 0};
    keep_in_range(b);
    const int64_t d = p.ex - b.ex;
    double v;
    if (d > 2000) {
      v = INFINITY;
    } else {
      const double scale = d == 0 ? 1.0 : (d < -2000 ? 0.0 : ldexp(1.0, (int)d));
      const double dr = p.re * scale - b.re, di = p.im * scale - b.im;
      v = sqrt((dr * dr + di * di) / (b.re * b.re + b.im * b.im));
    }
    worst = (v > worst || v != v) ? v : worst;  // a NaN stays visible
  }
  return worst;
}

// a complex number for the setup (plain doubles on host and device)
struct Cx {
  double re, im;
};
BD_HD Cx cx_mul(Cx a, Cx b) { return Cx{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
BD_HD Cx cx_div(Cx a, Cx b) {
  const double n = b.re * b.re + b.im * b.im;
  return Cx{(a.re * b.re + a.im * b.im) / n, (a.im * b.re - a.re * b.im) / n};
}

// determinant of a k x k complex matrix (Gaussian elimination with partial pivoting; a is
// overwritten)
BD_HD Cx cx_det(Cx* a, int k) {
  Cx d{1, 0};
  for (int c = 0; c < k; ++c) {
    int p = c;
    double best = a[c * k + c].re * a[c * k + c].re + a[c * k + c].im * a[c * k + c].im;
    for (int r = c + 1; r < k; ++r) {
      const double v = a[r * k + c].re * a[r * k + c].re + a[r * k + c].im * a[r * k + c].im;
      if (v > best) {
        best = v;
        p = r;
      }
    }
    if (best == 0) return Cx{0, 0};
    if (p != c) {
      for (int j = 0; j < k; ++j) {
        const Cx t = a[c * k + j];
        a[c * k + j] = a[p * k + j];
        a[p * k + j] = t;
      }
      d = Cx{-d.re, -d.im};
    }
    d = cx_mul(d, a[c * k + c]);
    for (int r = c + 1; r < k; ++r) {
      const Cx f = cx_div(a[r * k + c], a[c * k + c]);
      for (int j = c; j < k; ++j) {
        const Cx t = cx_mul(f, a[c * k + j]);
        a[r * k + j] = Cx{a[r * k + j].re - t.re, a[r * k + j].im - t.im};
      }
    }
  }
  return d;
}

// The StartCell of the cell with point indices idx[0..k] (row-major points); false when the
// cell is flat or an exact value would leave 64 bits (every exact value is a minor of
// [E | I], bounded by the Hadamard bound of E, which is checked first).
BD_HD bool start_setup(const int64_t* pts, int npts, int k, const uint8_t* idx, uint64_t coef_seed, StartCell& out) {
  int64_t E[KMAX * KMAX];
  double lg = 0;
  for (int j = 0; j < k; ++j) {
    double n2 = 0;
    for (int c = 0; c < k; ++c) {
      const int64_t v = pts[(size_t)idx[j] * k + c] - pts[(size_t)idx[k] * k + c];
      if (v >= ((int64_t)1 << 31) || v <= -((int64_t)1 << 31)) return false;
      E[j * k + c] = v;
      out.E[j * k + c] = (int32_t)v;
      n2 += (double)v * (double)v;
    }
    lg += 0.5 * log2(n2 > 1 ? n2 : 1.0);
  }
  if (lg > 61.0) return false;
  // fraction-free Gauss-Jordan on [E | I]: ends at [d I | d E^-1], d = det of the row-permuted E
  int64_t A[KMAX * 2 * KMAX];
  const int w = 2 * k;
  for (int r = 0; r < k; ++r)
    for (int c = 0; c < w; ++c) A[r * w + c] = c < k ? E[r * k + c] : (c - k == r ? 1 : 0);
  Div64 D = make_div((int64_t)1);
  for (int c = 0; c < k; ++c) {
    int p = -1;
    for (int r = c; r < k; ++r)
      if (A[r * w + c] != 0) { p = r; break; }
    if (p < 0) return false;
    if (p != c)
      for (int j = 0; j < w; ++j) {
        const int64_t t = A[c * w + j];
        A[c * w + j] = A[p * w + j];
        A[p * w + j] = t;
      }
    const int64_t pc = A[c * w + c];
    for (int r = 0; r < k; ++r) {
      if (r == c) continue;
      const int64_t rc = A[r * w + c];
      for (int j = 0; j < w; ++j)
        if (j != c) A[r * w + j] = bareiss(A[r * w + j], pc, rc, A[c * w + j], D);
      A[r * w + c] = 0;
    }
    D = make_div(pc);
  }
  // every diagonal entry is now d (fraction-free Gauss-Jordan keeps the rows on one scale)
  const int64_t d = A[(k - 1) * w + (k - 1)];
  for (int r = 0; r < k; ++r)
    if (A[r * w + r] != d) return false;
  out.det = d;
  for (int r = 0; r < k; ++r)
    for (int j = 0; j < k; ++j) out.adj[r * k + j] = A[r * w + k + j];
  // diagonal of the lower-triangular column Hermite form, computed modulo R = |det E| (the
  // lattice E Z^k contains R Z^k, so entries may be reduced mod R, which keeps them small; the
  // modulus drops to R / h_i after row i): row i's entries right of the diagonal are cleared by
  // extended-Euclid column steps, then h_i = gcd(H_ii, R)
  int64_t H[KMAX * KMAX];
  for (int t = 0; t < k * k; ++t) H[t] = E[t];
  int64_t R = d < 0 ? -d : d;
  auto modR = [&](i128 x) { int64_t r = (int64_t)(x % R); return r < 0 ? r + R : r; };
  for (int i = 0; i < k; ++i) {
    for (int r = 0; r < k; ++r) H[r * k + i] = modR(H[r * k + i]);
    for (int j = i + 1; j < k; ++j) {
      const int64_t hij = modR(H[i * k + j]);
      if (hij == 0) {
        for (int r = 0; r < k; ++r) H[r * k + j] = modR(H[r * k + j]);
        continue;
      }
      // u H_ii + v H_ij = g = gcd(H_ii, H_ij)
      int64_t r0 = H[i * k + i], r1 = hij, s0 = 1, s1 = 0, t0 = 0, t1 = 1;
      while (r1 != 0) {
        const int64_t q = r0 / r1;
        int64_t t = r0 - q * r1; r0 = r1; r1 = t;
        t = s0 - q * s1; s0 = s1; s1 = t;
        t = t0 - q * t1; t0 = t1; t1 = t;
      }
      const int64_t g = r0, a = H[i * k + i] / g, bq = hij / g;
      for (int r = 0; r < k; ++r) {
        const int64_t ci = H[r * k + i], cj = H[r * k + j];
        H[r * k + i] = modR((i128)s0 * ci + (i128)t0 * cj);
        H[r * k + j] = modR((i128)a * cj - (i128)bq * ci);
      }
    }
    int64_t x = H[i * k + i], y = R;  // h_i = gcd(H_ii, R)
    while (y != 0) {
      const int64_t t = x % y;
      x = y;
      y = t;
    }
    out.h[i] = x;
    R /= x;
  }
  if (R != 1) return false;
  // right-hand sides: b_j = kappa_j / kappa_k, kappa_j = (-1)^j det(C without column j)
  const uint64_t cs = coef_stream_seed(coef_seed);
  Cx C[KMAX * (KMAX + 1)];
  for (int i = 0; i < k; ++i)
    for (int j = 0; j <= k; ++j) {
      const double th = 6.283185307179586 * coef_turns(cs, npts, i, idx[j]);
      C[i * (k + 1) + j] = Cx{cos(th), sin(th)};
    }
  Cx kappa[KMAX + 1], sub[KMAX * KMAX];
  for (int j = 0; j <= k; ++j) {
    for (int i = 0; i < k; ++i)
      for (int c = 0, t = 0; c <= k; ++c)
        if (c != j) sub[i * k + t++] = C[i * (k + 1) + c];
    const Cx dj = cx_det(sub, k);
    kappa[j] = (j & 1) ? Cx{-dj.re, -dj.im} : dj;
  }
  if (kappa[k].re == 0 && kappa[k].im == 0) return false;
  double lmag[KMAX], larg[KMAX];
  for (int j = 0; j < k; ++j) {
    const Cx b = cx_div(kappa[j], kappa[k]);
    if (b.re == 0 && b.im == 0) return false;
    out.b_re[j] = b.re;
    out.b_im[j] = b.im;
    lmag[j] = 0.5 * log(b.re * b.re + b.im * b.im);
    larg[j] = atan2(b.im, b.re);
  }
  // E^-1 log b = adj log b / det
  for (int i = 0; i < k; ++i) {
    double re = 0, im = 0;
    for (int j = 0; j < k; ++j) {
      re += (double)out.adj[i * k + j] * lmag[j];
      im += (double)out.adj[i * k + j] * larg[j];
    }
    out.base_re[i] = re / (double)d;
    out.base_im[i] = im / (double)d;
  }
  return true;
}

}  // namespace bd

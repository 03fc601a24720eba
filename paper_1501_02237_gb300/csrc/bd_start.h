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
  uint64_t first;            // index of this cell's first solution in the global order
  int64_t det;               // det E (nonzero)
  int64_t h[KMAX];           // diagonal of the column Hermite form of E (positive)
  int64_t adj[KMAX * KMAX];  // adj(E), row-major: E^-1 = adj / det
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

// max over the cell's equations of |y^{E_j} / b_j - 1| for one solution y (k complex numbers)
BD_HD double start_residual(const StartCell& sc, int k, const double* y) {
  double worst = 0;
  for (int j = 0; j < k; ++j) {
    double pr = 1, pi = 0;
    for (int i = 0; i < k; ++i) {
      int e = sc.E[j * k + i];
      double br = y[2 * i], bi = y[2 * i + 1];
      if (e < 0) {  // y^-1 = conj(y) / |y|^2
        const double n2 = br * br + bi * bi;
        br = br / n2;
        bi = -bi / n2;
        e = -e;
      }
      while (e) {  // square and multiply
        if (e & 1) {
          const double r = pr * br - pi * bi;
          pi = pr * bi + pi * br;
          pr = r;
        }
        const double r = br * br - bi * bi;
        bi = 2 * br * bi;
        br = r;
        e >>= 1;
      }
    }
    // |p / b - 1| = |p - b| / |b|
    const double dr = pr - sc.b_re[j], di = pi - sc.b_im[j];
    const double v = sqrt((dr * dr + di * di) / (sc.b_re[j] * sc.b_re[j] + sc.b_im[j] * sc.b_im[j]));
    worst = v > worst ? v : worst;
  }
  return worst;
}

// Host: the StartCell of the cell with point indices idx[0..k] (row-major points); false when
// the cell is flat or an exact value leaves 64 bits.
bool start_setup(const int64_t* pts, int npts, int k, const uint8_t* idx, uint64_t coef_seed, StartCell& out);

}  // namespace bd

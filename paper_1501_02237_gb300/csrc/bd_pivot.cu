// Output-sensitive volume by simplicial pivoting (Sec. 4.2): the start cell (host), the
// breadth-first traversal of the cells on the GPU (one warp per cell, a hash set of cell
// bitmasks, one launch per level), its host emulation, and the C ABI (bd_volume_pivot,
// bd_volume_pivot_lifted, bd_host_volume_pivot, bd_degree_pivot).  The per-cell step is in
// bd_pivot.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <unordered_set>
#include <vector>

#include "../../include/binodeg.h"
#include "bd_host.h"
#include "bd_internal.h"
#include "bd_lifts.h"
#include "bd_pivot.cuh"
#include "bd_teams.h"

using bd::i128;
using bd::u128;

namespace {

constexpr int kPivotMaxWarps = 8;  // warps per block: chosen per problem, at most this

std::atomic<int> g_force_wide{0};  // bd_pivot_force_wide: 128-bit tableau entries whatever the bound

struct PivotWarp {
  __device__ int lane() const { return threadIdx.x & 31; }
  __device__ int lanes() const { return 32; }
  __device__ void sync() const { __syncwarp(); }
  __device__ uint64_t or_all(uint64_t x) const {  // ridge bits: below 2^31
    return __reduce_or_sync(0xffffffffu, (uint32_t)x);
  }
};

enum { START_OK = 0, START_TIE = 1, START_FLAT = 2, START_OVERFLOW = 3 };

// The heights of the pivoting path: the top 40 bits of the lift stream (bd_lifts.h), in
// [1, 2^40].  The path walks up to ~1e8 cells, where the 20-bit heights of the subset
// enumeration tie too often (one relift at 7e6 cells, every lifting at 5e7).
int64_t lift_height_wide(uint64_t stream_seed, int i) {
  return 1 + (int64_t)(bd::splitmix_mix(stream_seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull) >> 24);
}

i128 iabs(i128 x) { return x < 0 ? -x : x; }

i128 gcd128(i128 a, i128 b) {
  a = iabs(a);
  b = iabs(b);
  while (b) {
    const i128 t = a % b;
    a = b;
    b = t;
  }
  return a;
}

bool mul_ok(i128 a, i128 b, i128& r) { return !__builtin_mul_overflow(a, b, &r); }
bool add_ok(i128 a, i128 b, i128& r) { return !__builtin_add_overflow(a, b, &r); }

// Signed 256-bit values as sign and magnitude, for the start cell's support function: the
// coefficients of one extension step are formed exactly in 256 bits and reduced by their gcd
// before they are stored back in 128 bits.
struct U256 {
  u128 lo = 0, hi = 0;
};
struct S256 {
  bool neg = false;
  U256 m;
};

bool u_zero(const U256& a) { return a.lo == 0 && a.hi == 0; }
bool u_less(const U256& a, const U256& b) { return a.hi != b.hi ? a.hi < b.hi : a.lo < b.lo; }
U256 u_add(const U256& a, const U256& b) {  // the callers keep the sum below 2^256
  U256 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (r.lo < a.lo ? 1 : 0);
  return r;
}
U256 u_sub(const U256& a, const U256& b) {  // a >= b
  U256 r;
  r.lo = a.lo - b.lo;
  r.hi = a.hi - b.hi - (a.lo < b.lo ? 1 : 0);
  return r;
}
U256 u_shr(const U256& a, int k) {  // 0 <= k < 256
  if (k == 0) return a;
  U256 r;
  if (k >= 128) {
    r.lo = a.hi >> (k - 128);
  } else {
    r.lo = (a.lo >> k) | (a.hi << (128 - k));
    r.hi = a.hi >> k;
  }
  return r;
}
U256 u_shl(const U256& a, int k) {  // 0 <= k < 256, no bit shifted out
  if (k == 0) return a;
  U256 r;
  if (k >= 128) {
    r.hi = a.lo << (k - 128);
  } else {
    r.hi = (a.hi << k) | (a.lo >> (128 - k));
    r.lo = a.lo << k;
  }
  return r;
}
int u_ctz(const U256& a) { return a.lo ? bd::ctz128(a.lo) : 128 + bd::ctz128(a.hi); }
U256 u_mul(u128 a, u128 b) {  // the full product of two 128-bit magnitudes
  const u128 a0 = (uint64_t)a, a1 = a >> 64, b0 = (uint64_t)b, b1 = b >> 64;
  const u128 p00 = a0 * b0, p01 = a0 * b1, p10 = a1 * b0, p11 = a1 * b1;
  const u128 mid = (p00 >> 64) + (uint64_t)p01 + (uint64_t)p10;
  U256 r;
  r.lo = (u128)(uint64_t)p00 | (mid << 64);
  r.hi = p11 + (p01 >> 64) + (p10 >> 64) + (mid >> 64);
  return r;
}
u128 uabs128(i128 x) { return x < 0 ? (u128)0 - (u128)x : (u128)x; }
S256 s_mul(i128 a, i128 b) {
  S256 r;
  r.m = u_mul(uabs128(a), uabs128(b));
  r.neg = !u_zero(r.m) && ((a < 0) != (b < 0));
  return r;
}
S256 s_add(const S256& a, const S256& b) {  // magnitudes below 2^255
  S256 r;
  if (a.neg == b.neg) {
    r.neg = a.neg;
    r.m = u_add(a.m, b.m);
  } else if (u_less(a.m, b.m)) {
    r.neg = b.neg;
    r.m = u_sub(b.m, a.m);
  } else {
    r.neg = a.neg;
    r.m = u_sub(a.m, b.m);
  }
  if (u_zero(r.m)) r.neg = false;
  return r;
}
S256 s_negate(S256 a) {
  if (!u_zero(a.m)) a.neg = !a.neg;
  return a;
}
U256 u_gcd(U256 a, U256 b) {  // binary gcd
  if (u_zero(a)) return b;
  if (u_zero(b)) return a;
  const int za = u_ctz(a), zb = u_ctz(b), sh = za < zb ? za : zb;
  a = u_shr(a, za);
  while (!u_zero(b)) {
    b = u_shr(b, u_ctz(b));
    if (u_less(b, a)) std::swap(a, b);
    b = u_sub(b, a);
  }
  return u_shl(a, sh);
}
U256 u_div(const U256& x, const U256& g) {  // floor(x / g), g != 0, by binary long division
  U256 q, r;
  for (int i = 255; i >= 0; --i) {
    r = u_shl(r, 1);  // r < g < 2^256 before the shift: r stays below 2^256 while g < 2^255
    const bool bit = i >= 128 ? ((x.hi >> (i - 128)) & 1) : ((x.lo >> i) & 1);
    if (bit) r.lo |= 1;
    if (!u_less(r, g)) {
      r = u_sub(r, g);
      if (i >= 128) q.hi |= (u128)1 << (i - 128);
      else q.lo |= (u128)1 << i;
    }
  }
  return q;
}
// v / g as a 128-bit integer; false if it does not fit
bool s_div_fit(const S256& v, const U256& g, i128& out) {
  const U256 q = u_div(v.m, g);
  if (q.hi != 0 || (q.lo >> 127) != 0) return false;
  out = v.neg ? -(i128)q.lo : (i128)q.lo;
  return true;
}

// A lower facet to start from, by extension (the paper's extension process, Sec. 4.1, done
// here without a linear program): from the lowest lifted point, a lower face F with an integer
// support function H(p) = c w_p - <A, a_p> - B (>= 0 on all points, 0 exactly on F) is tilted
// about F in a direction u orthogonal to F's affine span until a further point joins:
// H' = w_q H - H(q) <u, a_p - a_f0> for the point q minimising H(q) / <u, a_q - a_f0> among
// those with <u, .> > 0.  d steps give a cell.  pts is row-major (npts x d).
template <class Mask>
int start_cell(const int64_t* pts, const int64_t* lifts, int N, int d, Mask& mask) {
  int v0 = 0;
  for (int p = 1; p < N; ++p)
    if (lifts[p] < lifts[v0]) v0 = p;
  for (int p = 0; p < N; ++p)
    if (p != v0 && lifts[p] == lifts[v0]) return START_TIE;
  std::vector<int> F{v0};
  i128 c = 1, B = lifts[v0];
  std::vector<i128> A(d, 0);
  std::vector<i128> H(N);
  auto eval = [&]() {  // false on overflow
    for (int p = 0; p < N; ++p) {
      i128 h, t;
      if (!mul_ok(c, (i128)lifts[p], h) || __builtin_sub_overflow(h, B, &h)) return false;
      for (int e = 0; e < d; ++e)
        if (!mul_ok(A[e], (i128)pts[p * d + e], t) || __builtin_sub_overflow(h, t, &h)) return false;
      H[p] = h;
    }
    return true;
  };
  while ((int)F.size() < d + 1) {
    const int j = (int)F.size() - 1, f0 = F[0];
    // the difference rows of F, reduced by fraction-free Gauss-Jordan to find free columns
    std::vector<std::vector<i128>> R(j, std::vector<i128>(d));
    for (int r = 0; r < j; ++r)
      for (int e = 0; e < d; ++e) R[r][e] = (i128)pts[F[r + 1] * d + e] - pts[f0 * d + e];
    std::vector<int> pivcol;
    i128 prev = 1;
    for (int col = 0; col < d && (int)pivcol.size() < j; ++col) {
      const int rk = (int)pivcol.size();
      int r = rk;
      while (r < j && R[r][col] == 0) ++r;
      if (r == j) continue;
      std::swap(R[r], R[rk]);
      const i128 pk = R[rk][col];
      for (int i = 0; i < j; ++i) {
        if (i == rk) continue;
        for (int e = 0; e < d; ++e) {
          if (e == col) continue;
          i128 t1, t2, t;
          if (!mul_ok(pk, R[i][e], t1) || !mul_ok(R[i][col], R[rk][e], t2) || __builtin_sub_overflow(t1, t2, &t))
            return START_OVERFLOW;
          R[i][e] = t / prev;  // exact (Bareiss)
        }
        R[i][col] = 0;
      }
      prev = pk;
      pivcol.push_back(col);
    }
    if ((int)pivcol.size() < j) return START_TIE;  // F not affinely independent
    if (!eval()) return START_OVERFLOW;
    bool extended = false;
    for (int fcol = 0; fcol < d && !extended; ++fcol) {
      if (std::find(pivcol.begin(), pivcol.end(), fcol) != pivcol.end()) continue;
      // u: prev at the free column, -R[r][fcol] at pivot column r (R's pivots all equal prev)
      std::vector<i128> u(d, 0);
      u[fcol] = prev;
      for (int r = 0; r < j; ++r) u[pivcol[r]] = -R[r][fcol];
      i128 g = 0;
      for (int e = 0; e < d; ++e) g = gcd128(g, u[e]);
      for (int e = 0; e < d; ++e) u[e] /= g;
      std::vector<i128> w(N);
      bool pos = false, neg = false;
      for (int p = 0; p < N; ++p) {
        i128 s = 0, t;
        for (int e = 0; e < d; ++e)
          if (!mul_ok(u[e], (i128)pts[p * d + e] - pts[f0 * d + e], t) || !add_ok(s, t, s)) return START_OVERFLOW;
        w[p] = s;
        pos |= s > 0;
        neg |= s < 0;
      }
      if (!pos && !neg) continue;
      const int sg = pos ? 1 : -1;
      int q = -1;
      for (int p = 0; p < N; ++p) {
        if (sg * w[p] <= 0) continue;
        if (H[p] <= 0) return START_TIE;  // a point on the face's plane outside the face
        if (q < 0) {
          q = p;
          continue;
        }
        // H[p] / (sg w[p]) against H[q] / (sg w[q])
        if (bd::prod_equal(H[p], sg * w[q], H[q], sg * w[p])) return START_TIE;
        if (bd::prod_greater(H[q], sg * w[p], H[p], sg * w[q])) q = p;
      }
      // H' = wq H - hq sg <u, a - a_f0>, formed exactly in 256 bits, then divided by the gcd of
      // its coefficients (the products overflow 128 bits on large coordinates long before the
      // reduced support function does)
      const i128 wq = sg * w[q], hq = H[q];  // wq > 0, hq > 0
      i128 uf0 = 0, t;
      for (int e = 0; e < d; ++e)
        if (!mul_ok(u[e], (i128)pts[f0 * d + e], t) || !add_ok(uf0, t, uf0)) return START_OVERFLOW;
      const S256 nc = s_mul(wq, c);
      std::vector<S256> nA(d);
      for (int e = 0; e < d; ++e) nA[e] = s_add(s_mul(wq, A[e]), s_mul(hq * sg, u[e]));
      const S256 nB = s_add(s_mul(wq, B), s_negate(s_mul(hq * sg, uf0)));
      U256 gg = u_gcd(nc.m, nB.m);
      for (int e = 0; e < d; ++e) gg = u_gcd(gg, nA[e].m);
      if (!s_div_fit(nc, gg, c) || !s_div_fit(nB, gg, B)) return START_OVERFLOW;
      for (int e = 0; e < d; ++e)
        if (!s_div_fit(nA[e], gg, A[e])) return START_OVERFLOW;
      F.push_back(q);
      extended = true;
    }
    if (!extended) return START_FLAT;  // every point lies in F's affine span
  }
  if (!eval()) return START_OVERFLOW;
  mask = Mask{};
  for (int f : F) bd::madd(mask, f);
  for (int p = 0; p < N; ++p)
    if (!bd::mhas(mask, p) && H[p] <= 0) return START_TIE;
  return START_OK;
}

// log2 of a Hadamard bound on every minor (of order <= d) of [M^T | a_p - a_s0] over all cells:
// every column is a_x - a_s0 for one base s0 and distinct points x, so a minor is at most the
// product of the d largest norms ||a_x - a_s0|| (each taken >= 1), maximised over s0
double pivot_bound_log2(const int64_t* pts, int N, int d) {
  double best = 0;
  std::vector<double> lg(N);
  for (int s0 = 0; s0 < N; ++s0) {
    for (int x = 0; x < N; ++x) {
      double s = 0;
      for (int e = 0; e < d; ++e) {
        const double v = (double)(pts[x * d + e] - pts[s0 * d + e]);
        s += v * v;
      }
      lg[x] = 0.5 * std::log2(std::max(s, 1.0));
    }
    std::sort(lg.begin(), lg.end(), [](double u, double v) { return u > v; });
    double t = 0;
    for (int i = 0; i < d && i < N; ++i) t += lg[i];
    best = std::max(best, t);
  }
  return best;
}

// per-warp shared memory of the walk with tableau entries of type TE: the scratch, the heights
// S (i128), then G0 and W (TE)
template <class TE>
__host__ __device__ size_t pivot_warp_bytes(int N, int d) {
  size_t b = sizeof(bd::PivotScratch<TE>);
  b = (b + 15) / 16 * 16 + 16 * (size_t)N;     // S: heights (i128)
  b += sizeof(TE) * (size_t)N;                 // G0
  b += sizeof(TE) * (size_t)d * N;             // W: the d x N tableau rows
  b += sizeof(float) * (size_t)N;              // Sf: the heights in single precision
  return (b + 15) / 16 * 16;
}

// the block's points: 32-bit coordinates (below 2^20), coordinate-major, then the 64-bit lifts
__host__ __device__ size_t pivot_points_bytes(int N, int d) {
  return (4 * (size_t)d * N + 15) / 16 * 16 + (8 * (size_t)N + 15) / 16 * 16;
}

template <class TE>
size_t pivot_smem(int N, int d, int warps) {
  return pivot_points_bytes(N, d) + warps * pivot_warp_bytes<TE>(N, d);
}

struct PivotDev {
  unsigned long long nvol_lo, nvol_hi, cells, boundary, next_count, flags, claimed;
};

constexpr int kWalkBudget = 64;  // cells a warp enters in place below each cell it eliminates

enum { PF_TIE = 1, PF_INVALID = 2, PF_FULL = 4 };

constexpr unsigned long long kMaxProbes = 4096;  // linear probing below half load: ~2.5 on average

// The hash set of claimed cells, one slot per cell.  Claims stay at most half the capacity
// (counting every claimed cell); past that, after kMaxProbes, or after a bounded wait for a
// slot being written, the level reports PF_FULL and the traversal restarts with a larger table.
template <class Mask>
struct CellTable;

// one-word masks (at most 64 points): a slot holds the mask itself, 0 when empty
template <>
struct CellTable<uint64_t> {
  unsigned long long* slot = nullptr;

  cudaError_t alloc(unsigned long long cap) { return bd::dev_malloc(&slot, sizeof(unsigned long long) * cap); }
  cudaError_t clear(unsigned long long cap, cudaStream_t st) {
    return cudaMemsetAsync(slot, 0, sizeof(unsigned long long) * cap, st);
  }
  void release() { cudaFree(slot); }
  __device__ void seed(unsigned long long cap, uint64_t m) const { slot[bd::pivot_hash(m) & (cap - 1)] = m; }
  // true if m was not in the table and now is
  __device__ bool claim(unsigned long long cap, uint64_t m, unsigned long long* claimed, unsigned long long* flags) const {
    unsigned long long h = bd::pivot_hash(m) & (cap - 1);
    for (unsigned long long probe = 0; probe < kMaxProbes; ++probe) {
      const unsigned long long cur = slot[h];
      if (cur == m) return false;
      if (cur == 0ull) {
        if (2 * *(volatile unsigned long long*)claimed >= cap) break;  // too full
        const unsigned long long old = atomicCAS(slot + h, 0ull, m);
        if (old == 0ull) {
          atomicAdd(claimed, 1ull);
          return true;
        }
        if (old == m) return false;
      }
      h = (h + 1) & (cap - 1);
    }
    atomicOr(flags, (unsigned long long)PF_FULL);
    return false;
  }
};

// two-word masks (up to 127 points): per slot a fingerprint (0: empty) and the two words; the
// high word carries kReady once both are written.  A claim takes a slot by compare-and-swap on
// the fingerprint; a reader meeting an equal fingerprint waits (bounded) for the words and
// compares them in full.
constexpr unsigned long long kReady = 1ull << 63;  // bit 127 of a mask: never a point

template <>
struct CellTable<bd::WideMask> {
  unsigned long long *fp = nullptr, *lo = nullptr, *hi = nullptr;

  cudaError_t alloc(unsigned long long cap) {
    cudaError_t e = bd::dev_malloc(&fp, sizeof(unsigned long long) * cap);
    if (e == cudaSuccess) e = bd::dev_malloc(&lo, sizeof(unsigned long long) * cap);
    if (e == cudaSuccess) e = bd::dev_malloc(&hi, sizeof(unsigned long long) * cap);
    return e;
  }
  cudaError_t clear(unsigned long long cap, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(fp, 0, sizeof(unsigned long long) * cap, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(hi, 0, sizeof(unsigned long long) * cap, st);
    return e;
  }
  void release() {
    cudaFree(fp);
    cudaFree(lo);
    cudaFree(hi);
  }
  __device__ void seed(unsigned long long cap, bd::WideMask m) const {
    const unsigned long long h = bd::pivot_hash(m) & (cap - 1);
    fp[h] = bd::pivot_hash(m);
    lo[h] = m.lo;
    hi[h] = m.hi | kReady;
  }
  __device__ bool claim(unsigned long long cap, bd::WideMask m, unsigned long long* claimed,
                        unsigned long long* flags) const {
    const unsigned long long f = bd::pivot_hash(m);
    unsigned long long h = f & (cap - 1);
    for (unsigned long long probe = 0; probe < kMaxProbes; ++probe) {
      unsigned long long cur = *(volatile unsigned long long*)(fp + h);
      if (cur == 0ull) {
        if (2 * *(volatile unsigned long long*)claimed >= cap) break;  // too full
        cur = atomicCAS(fp + h, 0ull, f);
        if (cur == 0ull) {
          lo[h] = m.lo;
          __threadfence();
          *(volatile unsigned long long*)(hi + h) = m.hi | kReady;
          atomicAdd(claimed, 1ull);
          return true;
        }
      }
      if (cur == f) {  // maybe m: wait for the slot's words
        unsigned long long hv = 0;
        for (int spin = 0; spin < (1 << 22); ++spin) {
          hv = *(volatile unsigned long long*)(hi + h);
          if (hv & kReady) break;
        }
        if (!(hv & kReady)) break;  // gave up waiting: report and restart
        __threadfence();
        if ((hv & ~kReady) == m.hi && *(volatile unsigned long long*)(lo + h) == m.lo) return false;
      }
      h = (h + 1) & (cap - 1);
    }
    atomicOr(flags, (unsigned long long)PF_FULL);
    return false;
  }
};

// append a claimed cell to the next level's list
template <class Mask>
__device__ void frontier_push(Mask* next, unsigned long long cap, Mask m, PivotDev* dv) {
  const unsigned long long pos = atomicAdd(&dv->next_count, 1ull);
  if (pos < cap) next[pos] = m;
  else atomicOr(&dv->flags, (unsigned long long)PF_FULL);
}

// One breadth-first level: every cell of `cur` is processed by one warp; its new neighbours
// enter the table and `next`.
template <class Mask, class TE>
__global__ void __launch_bounds__(32 * kPivotMaxWarps) k_pivot(const int64_t* pts, const int64_t* lifts, int N, int d,
                                                            const Mask* cur, unsigned long long ncur,
                                                            CellTable<Mask> table, unsigned long long cap,
                                                            int budget, Mask* next, PivotDev* dv) {
  extern __shared__ __align__(16) unsigned char smem[];
  int32_t* P = reinterpret_cast<int32_t*>(smem);  // coordinate-major, then the lifts
  int64_t* L = reinterpret_cast<int64_t*>(smem + (4 * (size_t)d * N + 15) / 16 * 16);
  for (int i = threadIdx.x; i < d * N; i += blockDim.x) P[i] = (int32_t)pts[(i % N) * d + i / N];
  for (int i = threadIdx.x; i < N; i += blockDim.x) L[i] = lifts[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* wb = smem + pivot_points_bytes(N, d) + warp * pivot_warp_bytes<TE>(N, d);
  auto* sc = reinterpret_cast<bd::PivotScratch<TE>*>(wb);
  size_t at = (sizeof(bd::PivotScratch<TE>) + 15) / 16 * 16;
  i128* S = reinterpret_cast<i128*>(wb + at);
  at += 16 * (size_t)N;
  TE* G0 = reinterpret_cast<TE*>(wb + at);
  at += sizeof(TE) * (size_t)N;
  TE* W = reinterpret_cast<TE*>(wb + at);
  at += sizeof(TE) * (size_t)d * N;
  float* Sf = reinterpret_cast<float*>(wb + at);
  PivotWarp tm;
  bd::PivotAcc acc{};
  int flags = 0;
  const int wpb = blockDim.x >> 5;
  const unsigned long long gw = (unsigned long long)blockIdx.x * wpb + warp;
  const unsigned long long nw = (unsigned long long)gridDim.x * wpb;
  for (unsigned long long c = gw; c < ncur; c += nw) {
    flags |= bd::pivot_cell<TE>(
        tm, P, L, N, d, cur[c], W, S, Sf, G0, sc, acc,
        [&](Mask m) { return table.claim(cap, m, &dv->claimed, &dv->flags); },
        [&](Mask m) { frontier_push(next, cap, m, dv); }, budget);
  }
  if (lane == 0) {
    const unsigned long long lo = (uint64_t)acc.nvol, hi = (uint64_t)(acc.nvol >> 64);
    if (lo || hi) {
      const unsigned long long old = atomicAdd(&dv->nvol_lo, lo);
      const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
      if (hi + carry) atomicAdd(&dv->nvol_hi, hi + carry);
    }
    if (acc.cells) atomicAdd(&dv->cells, (unsigned long long)acc.cells);
    if (acc.boundary) atomicAdd(&dv->boundary, (unsigned long long)acc.boundary);
    if (flags & bd::PV_TIE) atomicOr(&dv->flags, (unsigned long long)PF_TIE);
    if (flags & bd::PV_INVALID) atomicOr(&dv->flags, (unsigned long long)PF_INVALID);
  }
}

template <class Mask>
__global__ void k_pivot_seed(CellTable<Mask> t, unsigned long long cap, Mask m, Mask* frontier, PivotDev* dv) {
  t.seed(cap, m);
  frontier[0] = m;
  dv->claimed = 1;
}

struct PivotRun {
  u128 nvol = 0;
  uint64_t cells = 0, boundary = 0;
  int flags = 0;  // PF_*
  int levels = 0;
  double ms = 0;
  std::vector<uint64_t> masks;  // host emulation: every cell
};

// The traversal on the GPU from `start`; the table grows (and the traversal restarts) while it
// would be more than half full.
template <class Mask, class TE>
int device_pivot(const int64_t* pts, const int64_t* lifts, int N, int d, Mask start, PivotRun& run) {
  cudaStream_t st = bd::thread_stream();
  int dev = 0, sms = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);  // no device: a CUDA error, never a host fallback
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return bd::cuda_error(e);
  if (pivot_smem<TE>(N, d, 1) > (size_t)optin) return bd::set_error(BD_ERR_ARG, "the pivoting state exceeds shared memory");
  e = cudaFuncSetAttribute(k_pivot<Mask, TE>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  // warps per block: the most resident warps per SM (the state is per warp)
  int wpb = 1, per_sm = 0, best = 0;
  for (int w = 1; w <= kPivotMaxWarps && e == cudaSuccess; ++w) {
    const size_t sm_w = pivot_smem<TE>(N, d, w);
    if (sm_w > (size_t)optin) break;
    int b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pivot<Mask, TE>, 32 * w, sm_w);
    if (b * w > best) {
      best = b * w;
      wpb = w;
      per_sm = b;
    }
  }
  if (e != cudaSuccess) return bd::cuda_error(e);
  per_sm = std::max(per_sm, 1);
  const size_t smem = pivot_smem<TE>(N, d, wpb);
  // the table starts at 2^22 slots (2^26 for two-word masks: point sets past 64 points are the
  // large walks) and grows 8-fold (4-fold) per restart
  const bool two_words = std::is_same<Mask, bd::WideMask>::value;
  for (unsigned long long cap = two_words ? 1ull << 26 : 1ull << 22; cap <= (1ull << 31); cap <<= (two_words ? 2 : 3)) {
    int64_t *d_pts = nullptr, *d_lifts = nullptr;
    CellTable<Mask> table;
    Mask *d_a = nullptr, *d_b = nullptr;
    PivotDev* d_dv = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto release = [&]() {
      cudaFree(d_pts);
      cudaFree(d_lifts);
      table.release();
      cudaFree(d_a);
      cudaFree(d_b);
      cudaFree(d_dv);
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
    };
    e = bd::dev_malloc(&d_pts, sizeof(int64_t) * N * d);
    if (e == cudaSuccess) e = bd::dev_malloc(&d_lifts, sizeof(int64_t) * N);
    if (e == cudaSuccess) e = table.alloc(cap);
    if (e == cudaSuccess) e = bd::dev_malloc(&d_a, sizeof(Mask) * cap);
    if (e == cudaSuccess) e = bd::dev_malloc(&d_b, sizeof(Mask) * cap);
    if (e == cudaSuccess) e = bd::dev_malloc(&d_dv, sizeof(PivotDev));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_pts, pts, sizeof(int64_t) * N * d, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_lifts, lifts, sizeof(int64_t) * N, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = table.clear(cap, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_dv, 0, sizeof(PivotDev), st);
    if (e == cudaSuccess) {
      k_pivot_seed<Mask><<<1, 1, 0, st>>>(table, cap, start, d_a, d_dv);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    unsigned long long ncur = 1, total = 1;
    PivotDev h{};
    run.levels = 0;
    while (e == cudaSuccess && ncur > 0) {
      const unsigned long long zero = 0;
      e = cudaMemcpyAsync(&d_dv->next_count, &zero, sizeof(zero), cudaMemcpyHostToDevice, st);
      const unsigned long long blocks =
          std::min<unsigned long long>((unsigned long long)sms * per_sm, (ncur + wpb - 1) / wpb);
      // while a level has fewer cells than resident warps, push every new neighbour to the next
      // level (the list grows about d-fold per level) instead of walking from a few cells alone
      const unsigned long long warps = (unsigned long long)sms * per_sm * wpb;
      const int budget = ncur * 4 < warps ? 0 : kWalkBudget;
      if (e == cudaSuccess) {
        k_pivot<Mask, TE><<<(unsigned int)blocks, 32 * wpb, smem, st>>>(d_pts, d_lifts, N, d, d_a, ncur, table, cap,
                                                                           budget, d_b, d_dv);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_dv, sizeof(h), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      ++run.levels;
      if (e != cudaSuccess || h.flags) break;
      ncur = h.next_count;
      total = h.claimed;
      if (2 * total > cap) {  // too full for cheap probing: restart with a larger table
        h.flags = PF_FULL;
        break;
      }
      std::swap(d_a, d_b);
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    release();
    if (e != cudaSuccess) return bd::cuda_error(e);
    if (h.flags & PF_FULL) continue;
    run.nvol = ((u128)h.nvol_hi << 64) | h.nvol_lo;
    run.cells = h.cells;
    run.boundary = h.boundary;
    run.flags = (int)h.flags;
    run.ms = ms;
    return BD_OK;
  }
  return bd::set_error(BD_ERR_NOMEM, "more than 2^30 cells");
}

// The same traversal on the host: one team (one lane, or `width` lanes run as threads in
// lockstep), cells in breadth-first order.
struct MaskHash {
  size_t operator()(uint64_t m) const { return (size_t)bd::pivot_hash(m); }
  size_t operator()(bd::WideMask m) const { return (size_t)bd::pivot_hash(m); }
};

template <class Mask, class TE>
int host_pivot(const int64_t* pts, const int64_t* lifts, int N, int d, Mask start, int width, int budget,
               PivotRun& run) {
  std::vector<int32_t> P((size_t)d * N);
  for (int r = 0; r < d; ++r)
    for (int p = 0; p < N; ++p) P[(size_t)r * N + p] = (int32_t)pts[p * d + r];
  std::vector<TE> W((size_t)d * N), G0(N);
  std::vector<i128> S(N);
  std::vector<float> Sf(N);
  bd::PivotScratch<TE> sc{};
  std::unordered_set<Mask, MaskHash> seen{start};
  std::vector<Mask> cur{start}, next;
  bd::PivotAcc acc{};
  int flags = 0;
  std::mutex mu;
  auto step = [&](auto tm) {  // neighbours go to `next` under the mutex
    for (const Mask m : cur) {
      const int f = bd::pivot_cell<TE>(
          tm, P.data(), lifts, N, d, m, W.data(), S.data(), Sf.data(), G0.data(), &sc, acc,
          [&](Mask nb) {
            std::lock_guard<std::mutex> g(mu);  // lanes of a lockstep team claim concurrently
            return seen.insert(nb).second;
          },
          [&](Mask nb) {
            std::lock_guard<std::mutex> g(mu);
            next.push_back(nb);
          },
          budget);
      if (tm.lane() == 0) flags |= f;
    }
  };
  while (!cur.empty() && !flags) {
    next.clear();
    if (width <= 1) {
      step(bd::HostTeam{});
    } else {
      bd::LockstepShared shl(width);
      std::vector<std::thread> th;
      for (int l = 1; l < width; ++l) th.emplace_back([&, l] { step(bd::LockstepTeam{&shl, l}); });
      step(bd::LockstepTeam{&shl, 0});
      for (auto& t : th) t.join();
    }

    ++run.levels;
    cur.swap(next);
  }
  run.nvol = acc.nvol;
  run.cells = acc.cells;
  run.boundary = acc.boundary;
  run.flags = (flags & bd::PV_TIE ? PF_TIE : 0) | (flags & bd::PV_INVALID ? PF_INVALID : 0);
  if constexpr (std::is_same<Mask, uint64_t>::value) {  // cell lists: at most 64 points
    run.masks.assign(seen.begin(), seen.end());             // every claimed cell was processed once
    std::sort(run.masks.begin(), run.masks.end());
  }
  return BD_OK;
}

int pivot_common(const int64_t* points, const int64_t* given_lifts, int32_t npts, int32_t k, uint64_t seed,
                 int host_width, int host_budget, bd_volume_out* out, uint64_t* cells, int64_t capacity,
                 double* device_ms) {
  if (!out || !points) return bd::set_error(BD_ERR_ARG, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  if (k < 1 || k > bd::kPivotDMax) return bd::set_error(BD_ERR_ARG, "need 1 <= k <= 30 for the pivoting path");
  if (npts < k + 1 || npts > bd::kPivotNMax) return bd::set_error(BD_ERR_ARG, "need k+1 <= npts <= 127");
  if (cells && npts > 64) return bd::set_error(BD_ERR_ARG, "cell lists take at most 64 points");
  for (int i = 0; i < npts * k; ++i)
    if (points[i] >= (1 << 20) || points[i] <= -(1 << 20))
      return bd::set_error(BD_ERR_ARG, "coordinates must stay below 2^20 in magnitude on the pivoting path");
  const double bits = pivot_bound_log2(points, npts, k);
  out->bound_bits = (int32_t)std::ceil(bits);
  // the tableau's entries are cell minors: 64-bit while the bound stays below 2^62, else 128-bit;
  // the heights D h(p) (d+1 terms of a minor times a lift difference below 2^41) are 128-bit
  const bool wide = bits >= 61.99 || g_force_wide.load() != 0;
  if (bits + 41.0 + std::log2((double)(k + 1)) >= 125.99)
    return bd::set_error(BD_ERR_OVERFLOW, "cell heights may leave 127 bits (cell minors past 2^84)");
  std::vector<int64_t> lifts(npts);
  const int attempts = given_lifts ? 1 : 8;
  for (int a = 0; a < attempts; ++a) {
    if (given_lifts) {
      for (int i = 0; i < npts; ++i) {
        if (given_lifts[i] > (int64_t(1) << 40) || given_lifts[i] < -(int64_t(1) << 40))
          return bd::set_error(BD_ERR_ARG, "lifts must stay within 2^40 in magnitude on the pivoting path");
        lifts[i] = given_lifts[i];
      }
    } else {
      const uint64_t ss = bd::lift_stream_seed(seed, (uint32_t)a);
      for (int i = 0; i < npts; ++i) lifts[i] = lift_height_wide(ss, i);
    }
    out->relifts = a;
    uint64_t start = 0;        // at most 64 points: one-word masks
    bd::WideMask wmask{0, 0};  // more: two words
    const int sr = npts <= 64 ? start_cell(points, lifts.data(), npts, k, start)
                              : start_cell(points, lifts.data(), npts, k, wmask);
    if (sr == START_FLAT) {
      out->flags = BD_FLAG_DEGENERATE;
      return BD_OK;
    }
    if (sr == START_OVERFLOW) return bd::set_error(BD_ERR_OVERFLOW, "the start cell's support function left 128 bits");
    if (sr == START_TIE) {
      out->ties = 1;
      continue;
    }
    PivotRun run;
    int rc;
    if (npts <= 64 && !wide)
      rc = host_width > 0 ? host_pivot<uint64_t, int64_t>(points, lifts.data(), npts, k, start, host_width, host_budget, run)
                          : device_pivot<uint64_t, int64_t>(points, lifts.data(), npts, k, start, run);
    else if (npts <= 64)
      rc = host_width > 0 ? host_pivot<uint64_t, i128>(points, lifts.data(), npts, k, start, host_width, host_budget, run)
                          : device_pivot<uint64_t, i128>(points, lifts.data(), npts, k, start, run);
    else if (!wide)
      rc = host_width > 0 ? host_pivot<bd::WideMask, int64_t>(points, lifts.data(), npts, k, wmask, host_width, host_budget, run)
                          : device_pivot<bd::WideMask, int64_t>(points, lifts.data(), npts, k, wmask, run);
    else
      rc = host_width > 0 ? host_pivot<bd::WideMask, i128>(points, lifts.data(), npts, k, wmask, host_width, host_budget, run)
                          : device_pivot<bd::WideMask, i128>(points, lifts.data(), npts, k, wmask, run);
    if (rc) return rc;
    if (run.flags & PF_INVALID) return bd::set_error(BD_ERR_ARG, "pivoting reached a non-cell (internal error)");
    if (run.flags & PF_TIE) {
      out->ties = 1;
      continue;
    }
    out->ties = 0;
    if (wide) out->flags |= BD_FLAG_INT128;
    out->nvol_lo = (uint64_t)run.nvol;
    out->nvol_hi = (uint64_t)(run.nvol >> 64);
    out->cells = run.cells;
    out->subsets = run.cells * (uint64_t)(k + 1);  // ridges examined
    if (device_ms) *device_ms = run.ms;
    if (cells) {
      if ((int64_t)run.masks.size() > capacity)
        return bd::set_error(BD_ERR_ARG, "capacity is below the number of cells (out->cells holds it)");
      std::copy(run.masks.begin(), run.masks.end(), cells);
    }
    return BD_OK;
  }
  return bd::set_error(BD_ERR_TIES, given_lifts ? "the given lifting is not generic" : "every lifting had a tie");
}

}  // namespace

extern "C" {

int bd_volume_pivot(const int64_t* points, int32_t npts, int32_t k, uint64_t seed, bd_volume_out* out,
                    double* device_ms) {
  return pivot_common(points, nullptr, npts, k, seed, 0, 0, out, nullptr, 0, device_ms);
}

int bd_host_volume_pivot(const int64_t* points, const int64_t* lifts, int32_t npts, int32_t k, int32_t team_width,
                         int32_t walk_budget, bd_volume_out* out, uint64_t* cells, int64_t capacity) {
  if (!lifts) return bd::set_error(BD_ERR_ARG, "NULL argument");
  if (team_width < 1 || team_width > 32) return bd::set_error(BD_ERR_ARG, "team width must be 1..32");
  if (walk_budget < 0) return bd::set_error(BD_ERR_ARG, "negative walk budget");
  if (cells && capacity < 0) return bd::set_error(BD_ERR_ARG, "negative capacity");
  return pivot_common(points, lifts, npts, k, 0, team_width, walk_budget, out, cells, capacity, nullptr);
}

int bd_pivot_force_wide(int32_t on) { return g_force_wide.exchange(on != 0 ? 1 : 0); }

int bd_degree_pivot(const int64_t* A, int32_t n, int32_t m, const int64_t* coef, uint64_t seed, bd_degree_out* out) {
  if (!out) return bd::set_error(BD_ERR_ARG, "out is NULL");
  if (!A && m > 0) return bd::set_error(BD_ERR_ARG, "A is NULL");
  if (n < 1 || n >= bd::kPivotNMax || m < 0 || m > 256)
    return bd::set_error(BD_ERR_ARG, "need 1 <= n <= 126, 0 <= m <= 256 on the pivoting path");
  std::memset(out, 0, sizeof(*out));
  bd::Reduction r;
  std::string err;
  int rc = bd::reduce_system(A, n, m, coef, r, err);
  if (rc) return bd::set_error(rc, err.c_str());
  out->rank = r.rank;
  out->dim = r.dim;
  out->torsion = r.torsion;
  out->consistent = r.consistent ? 1 : 0;
  out->max_abs_coord = (int32_t)r.max_abs_coord;
  if (!r.consistent) {
    out->flags = BD_FLAG_INCONSISTENT;
    return BD_OK;
  }
  u128 nvol = 1;
  if (r.dim >= 1) {
    bd_volume_out v;
    rc = pivot_common(r.points.data(), nullptr, n + 1, r.dim, seed, 0, 0, &v, nullptr, 0, nullptr);
    if (rc) return rc;
    nvol = ((u128)v.nvol_hi << 64) | v.nvol_lo;
    out->relifts = v.relifts;
    out->subsets = v.subsets;
    out->cells = v.cells;
    out->flags = v.flags;
  }
  const u128 deg = nvol * r.torsion;
  if (r.torsion && deg / r.torsion != nvol) return bd::set_error(BD_ERR_OVERFLOW, "degree exceeds 2^128");
  out->nvol_lo = (uint64_t)nvol;
  out->nvol_hi = (uint64_t)(nvol >> 64);
  out->degree_lo = (uint64_t)deg;
  out->degree_hi = (uint64_t)(deg >> 64);
  return BD_OK;
}

}  // extern "C"

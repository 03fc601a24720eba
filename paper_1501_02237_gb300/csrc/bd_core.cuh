// Exact lower-facet enumeration core, shared by the CUDA warp kernel and its host emulation.
//
// Method (Sec. 4, Eq. lower-face; strict form Sec. 5, Eq. lower-d-face-again): for a lifted
// point set S^ = {(a_q, w_q)} in Z^{K+1}, a (K+1)-subset {s_0 < .. < s_K} is a lower facet iff
// its coordinate simplex is full-dimensional (D0 = det(a_{s_j} - a_{s_0}) != 0) and every
// other lifted point lies strictly above the hyperplane through the lifted subset.  With
// M = [a_{s_j} - a_{s_0}], w = [w_{s_j} - w_{s_0}] and z_q = (a_q - a_{s_0}, w_q - w_{s_0}),
//     s(q) = det [[M, w], [z_q]]  =  D0 * (height of q above the hyperplane),
// so q is strictly above iff sign s(q) = sign D0.  NVol = sum |D0| over accepted cells
// (Eq. simplex-vol read as |det|).
//
// Evaluation order (this file's own design, not the paper's LP traversal):
//   * subsets are enumerated depth-first in lexicographic order; level j fixes s_j;
//   * the state at level j is the fraction-free (Bareiss) reduction of EVERY point's
//     lifted difference row z_q against the pivot rows of s_1..s_j: an entry of state j at
//     a surviving column c equals the (j+1)x(j+1) minor det(rows s_1..s_j, q ; pivot cols, c)
//     (Sylvester's identity), so each level costs one update per point and surviving column
//     and is shared by the whole subtree below it;
//   * pivots are taken in coordinate columns only; a pivot row with no nonzero coordinate
//     entry means every subset extending the prefix has D0 = 0 (counted as singular, skipped);
//   * after K-1 levels each point q carries two numbers (C_q, L_q): the K x K minors with the
//     last coordinate column and with the lift column.  For the last point p,
//         D0 = sigma * C_p,   s(q) = sigma * (C_p L_q - C_q L_p) / p_{K-1},
//     (sigma = column-permutation sign, common to both) so the test of q is one more
//     Bareiss step and a sign compare;
//   * a warp owns one subtree; lane l holds points l, l+32, ...; a warp vote decides each cell.
//
// Exactness: entries are minors bounded by a Hadamard bound checked on the host, so each fits
// the entry type (int64 or int128).  The Bareiss division (a p - b r) / d is exact; it is done
// modulo 2^64 (2^128) as in T. Jebelean, "An algorithm for exact division", J. Symbolic
// Computation 15 (1993): drop the t trailing zero bits of d (t = ctz d, using the high product
// bits when t > 0) and multiply by the inverse of the odd part of d modulo 2^64, obtained by
// Newton-Hensel lifting x <- x (2 - d x).
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define BD_HD __host__ __device__ __forceinline__
#define BD_COLD __host__ __device__ __noinline__
#else
#define BD_HD inline
#define BD_COLD __attribute__((noinline))
#endif

namespace bd {

typedef __int128 i128;
typedef unsigned __int128 u128;

BD_HD int ctz64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __ffsll((long long)x) - 1;
#else
  return __builtin_ctzll(x);
#endif
}

BD_HD int popc64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __popcll(x);
#else
  return __builtin_popcountll(x);
#endif
}

BD_HD int popc32(uint32_t x) {
#ifdef __CUDA_ARCH__
  return __popc(x);
#else
  return __builtin_popcount(x);
#endif
}

// position of the r-th set bit (from 0) of m, which has more than r set bits: a binary search
// over popcounts of the word's halves
BD_HD int nth_set(uint64_t m, int r) {
  int pos = 0;
  uint32_t w = (uint32_t)m;
  const int lo = popc32(w);
  if (r >= lo) {
    r -= lo;
    w = (uint32_t)(m >> 32);
    pos = 32;
  }
  for (int sh = 16; sh >= 1; sh >>= 1) {
    const uint32_t low = w & ((1u << sh) - 1u);
    const int c = popc32(low);
    if (r >= c) {
      r -= c;
      w >>= sh;
      pos += sh;
    } else {
      w = low;
    }
  }
  return pos;
}

BD_HD int ctz128(u128 x) {
  uint64_t lo = (uint64_t)x;
  return lo ? ctz64(lo) : 64 + ctz64((uint64_t)(x >> 64));
}

// ---------------------------------------------------------------------------------------------
// exact division by a fixed nonzero divisor
// ---------------------------------------------------------------------------------------------
struct Div64 {
  uint64_t inv;  // inverse of the odd part of d modulo 2^64
  int shift;     // number of trailing zero bits of d
};

BD_HD Div64 make_div(int64_t d) {
  Div64 r;
  r.shift = ctz64((uint64_t)d);
  const uint64_t odd = (uint64_t)(d >> r.shift);  // exact: 2^shift divides d
  // (3 odd) xor 2 is an inverse modulo 2^5; each Newton-Hensel step doubles the correct bits:
  // three 32-bit steps reach 40 >= 32 bits, one 64-bit step reaches 64
  const uint32_t o32 = (uint32_t)odd;
  uint32_t y = (3u * o32) ^ 2u;
  y *= 2u - o32 * y;
  y *= 2u - o32 * y;
  y *= 2u - o32 * y;
  uint64_t x = y;
  x *= 2u - odd * x;
  r.inv = x;
  return r;
}

struct Div128 {
  u128 inv;
  int shift;
};

BD_HD Div128 make_div(i128 d) {
  Div128 r;
  r.shift = ctz128((u128)d);
  const u128 odd = (u128)(d >> r.shift);
  const Div64 lo = make_div((int64_t)(uint64_t)odd);  // inverse modulo 2^64 (odd: shift 0)
  u128 x = lo.inv;
  x *= (u128)2 - odd * x;  // 128 bits
  r.inv = x;
  return r;
}

// (a*p - b*r) / d, exact, for a quotient that fits int64.
BD_HD int64_t bareiss(int64_t a, int64_t p, int64_t b, int64_t r, const Div64& D) {
  if (D.shift == 0) {
    uint64_t v = (uint64_t)a * (uint64_t)p - (uint64_t)b * (uint64_t)r;  // mod 2^64
    return (int64_t)(v * D.inv);
  }
  i128 v = (i128)a * p - (i128)b * r;  // |a p|, |b r| < 2^126: exact
  uint64_t lo = (uint64_t)(v >> D.shift);
  return (int64_t)(lo * D.inv);
}

// divider for 32-bit coordinate minors, also usable for the 64-bit lift minors
struct Div32 {
  uint32_t inv32;  // inverse of the odd part modulo 2^32
  uint64_t inv64;  // the same odd part (sign-extended) inverted modulo 2^64
  int shift;
};

BD_HD Div32 make_div(int32_t d) {
  Div32 r;
  r.shift = ctz64((uint64_t)(uint32_t)d);
  const int64_t odd = (int64_t)(d >> r.shift);
  const uint32_t o32 = (uint32_t)odd;
  uint32_t y = (3u * o32) ^ 2u;  // 5 bits
  y *= 2u - o32 * y;             // 10
  y *= 2u - o32 * y;             // 20
  y *= 2u - o32 * y;             // 40 >= 32
  r.inv32 = y;
  uint64_t x = y;
  x *= 2u - (uint64_t)odd * x;   // 80 >= 64
  r.inv64 = x;
  return r;
}

// (a*p - b*r) / d for 32-bit minors: the products are exact in 64 bits
BD_HD int32_t bareiss(int32_t a, int32_t p, int32_t b, int32_t r, const Div32& D) {
  const int64_t v = (int64_t)a * p - (int64_t)b * r;
  return (int32_t)((uint32_t)(v >> D.shift) * D.inv32);
}

// (a*p - b*r) / d for a 64-bit lift minor a, r with 32-bit coordinate minors p, b, d
BD_HD int64_t bareiss(int64_t a, int32_t p, int32_t b, int64_t r, const Div32& D) {
  if (D.shift == 0) {
    const uint64_t v = (uint64_t)a * (uint64_t)(int64_t)p - (uint64_t)(int64_t)b * (uint64_t)r;
    return (int64_t)(v * D.inv64);
  }
  const i128 v = (i128)a * p - (i128)b * r;  // < 2^95 in magnitude
  return (int64_t)((uint64_t)(v >> D.shift) * D.inv64);
}

// signed 128 x 128 -> 256 product as (hi, lo)
BD_HD void mul_wide(i128 a, i128 b, u128& hi, u128& lo) {
  u128 ua = (u128)a, ub = (u128)b;
  uint64_t a0 = (uint64_t)ua, a1 = (uint64_t)(ua >> 64);
  uint64_t b0 = (uint64_t)ub, b1 = (uint64_t)(ub >> 64);
  u128 p00 = (u128)a0 * b0, p01 = (u128)a0 * b1, p10 = (u128)a1 * b0, p11 = (u128)a1 * b1;
  u128 mid = (p00 >> 64) + (uint64_t)p01 + (uint64_t)p10;
  lo = (u128)(uint64_t)p00 | ((u128)(uint64_t)mid << 64);
  hi = p11 + (p01 >> 64) + (p10 >> 64) + (mid >> 64);
  if (a < 0) hi -= ub;  // two's-complement correction of the unsigned product
  if (b < 0) hi -= ua;
}

// (a*p - b*r) / d, exact, for a quotient that fits int128.
BD_HD i128 bareiss(i128 a, i128 p, i128 b, i128 r, const Div128& D) {
  if (D.shift == 0) {
    u128 v = (u128)a * (u128)p - (u128)b * (u128)r;  // mod 2^128
    return (i128)(v * D.inv);
  }
  u128 h1, l1, h2, l2;
  mul_wide(a, p, h1, l1);
  mul_wide(b, r, h2, l2);
  u128 lo = l1 - l2;
  u128 hi = h1 - h2 - (u128)(l1 < l2);
  int t = D.shift;  // 0 < t < 127
  u128 q = (lo >> t) | (hi << (128 - t));
  return (i128)(q * D.inv);
}

// read-only load through the non-coherent cache on the device
BD_HD uint32_t ldg_u32(const uint32_t* p) {
#ifdef __CUDA_ARCH__
  return __ldg(p);
#else
  return *p;
#endif
}

// Number of triples i < j < k < 63: the colex decode table covers every node (R <= 63).
constexpr int kTriEntries = 63 * 62 * 61 / 6;

// entry t of the colex order of triples i < j < k (by k, then j, then i), packed
// i | j << 8 | k << 16 (host side: the table the device reads)
inline void fill_colex_table(uint32_t* out) {
  int t = 0;
  for (int k = 2; k < 63; ++k)
    for (int j = 1; j < k; ++j)
      for (int i = 0; i < j; ++i) out[t++] = (uint32_t)i | ((uint32_t)j << 8) | ((uint32_t)k << 16);
}

// four single-precision values loaded as one 16-byte word (16-byte aligned address)
#ifdef __CUDACC__
typedef float4 F4;
#else
struct alignas(16) F4 {
  float x, y, z, w;
};
#endif
BD_HD F4 ld4(const float* p) { return *reinterpret_cast<const F4*>(p); }

// square root of v >= 1 to a few ulps (the callers correct the integer part they take from it)
BD_HD float approx_sqrt(float v) {
#ifdef __CUDA_ARCH__
  return v * rsqrtf(v);
#else
  return sqrtf(v);
#endif
}

// single-precision value of a 64-bit integer without a 64-bit conversion instruction: the
// magnitude is split into 32-bit halves, each converted (one rounding each) and recombined by
// one fused multiply-add, so the relative error is at most 2^-23.
BD_HD float f32_of(int64_t x) {
  const uint64_t a = x < 0 ? (uint64_t)0 - (uint64_t)x : (uint64_t)x;
  const float f = fmaf((float)(uint32_t)(a >> 32), 4294967296.0f, (float)(uint32_t)a);
  return x < 0 ? -f : f;
}
BD_HD float f32_of(int32_t x) { return (float)x; }
BD_HD float f32_of(i128 x) { return (float)x; }

// sign of a*b - c*d, exact (-1, 0, 1)
BD_HD int cross_sign(int64_t a, int64_t b, int64_t c, int64_t d) {
  const i128 v = (i128)a * b - (i128)c * d;  // |a b|, |c d| < 2^126
  return (v > 0) - (v < 0);
}

BD_HD int cross_sign(i128 a, i128 b, i128 c, i128 d) {
  u128 h1, l1, h2, l2;
  mul_wide(a, b, h1, l1);
  mul_wide(c, d, h2, l2);
  const u128 lo = l1 - l2;
  const i128 hi = (i128)(h1 - h2 - (u128)(l1 < l2));
  if (hi != 0) return hi > 0 ? 1 : -1;
  return lo != 0 ? 1 : 0;
}

// Sign of a*b - c*d from single-precision copies (af = fl(a) etc.), or 2 when the rounded
// value is too close to zero to decide.  Each copy has relative error <= 2^-24, each product
// and the fused difference add at most 2^-24 more, so the computed value is within
// 2^-21 (|ab| + |cd|) of the exact one; a larger magnitude fixes the sign.  Copies of values
// below 2^63 keep every product below 2^126 < FLT_MAX.
BD_HD int cross_sign_filtered(float af, float bf, float cf, float df) {
  const float p = af * bf;
  const float v = fmaf(-cf, df, p);
  const float bound = 4.8e-7f * (fabsf(p) + fabsf(cf * df));  // 2^-21 ~ 4.77e-7
  if (v > bound) return 1;
  if (v < -bound) return -1;
  return 2;
}

// ---------------------------------------------------------------------------------------------
// work items and per-team accumulators
// ---------------------------------------------------------------------------------------------
constexpr int KMAX = 14;           // largest lattice dimension K (a work item is 16 bytes)

constexpr int NMAX = 64;           // largest number of points (one 64-bit membership mask)

struct Item {                      // a subset prefix s_0 < .. < s_{L-1}, 1 <= L <= max(K-2, 1)
  uint8_t len;
  uint8_t idx[15];
};

struct Range {                     // items first .. first+count-1 of a lexicographic work list
  uint32_t first, count;
};

struct Acc {
  u128 nvol;         // sum of |D0| over accepted cells
  uint64_t cells;    // accepted cells
  uint64_t singular; // subsets with D0 = 0
  uint64_t ties;     // subsets with no point below and at least one point on the hyperplane
#ifdef BD_COUNT
  uint64_t builds[KMAX + 1], fails[KMAX + 1], leaves, leaf_singular, exact_fallbacks;
  uint64_t bottoms, pairs, qtests;
#endif
};

// Accumulators are per lane: uniform counts are added by lane 0 only, per-pair results by the
// lane that decided them; the kernels sum them over the warp before flushing.  The kernels of
// the 5-D stage keep the rare results of that stage (accepted cells, their |D0| and ties) in the
// team's shared state instead (Uniform::rare), so that no register holds them during the walk.

// Binomial coefficients C(n, k), n <= 64, k <= 15, by Pascal's rule at compile time; the device
// reads them from constant memory (a division loop costs dozens of instructions per step there).
struct BinomTable {
  uint64_t v[NMAX + 1][KMAX + 2];
};
constexpr BinomTable make_binom_table() {
  BinomTable t{};
  for (int n = 0; n <= NMAX; ++n) {
    t.v[n][0] = 1;
    for (int k = 1; k <= KMAX + 1; ++k) t.v[n][k] = n == 0 ? 0 : t.v[n - 1][k - 1] + t.v[n - 1][k];
  }
  return t;
}
#ifdef __CUDACC__
static __constant__ BinomTable c_binom = make_binom_table();
#endif
static constexpr BinomTable h_binom = make_binom_table();  // the host's copy (work-list builders)

BD_HD uint64_t binom(int n, int k) {
  if (k < 0 || n < k) return 0;
#ifdef __CUDA_ARCH__
  if (n <= NMAX && k <= KMAX + 1) return c_binom.v[n][k];
#else
  if (n <= NMAX && k <= KMAX + 1) return h_binom.v[n][k];
#endif
  if (k > n - k) k = n - k;
  uint64_t r = 1;
  for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
  return r;
}

// number of (K+1)-subsets below a prefix whose last index is `last` and length `len`
BD_HD uint64_t subtree_size(int N, int K, int last, int len) { return binom(N - 1 - last, K + 1 - len); }

// offset of level j inside a point's coordinate stack: sum_{i<j} (K-i) (level j keeps K-j
// coordinate minors; the lift minor of level j is kept apart, one per level)
BD_HD int level_offset(int K, int j) { return j * K - (j * (j - 1)) / 2; }
BD_HD int stack_entries(int K) { return level_offset(K, K); }

template <class T> struct DivOf;
template <> struct DivOf<int32_t> { typedef Div32 type; };
template <> struct DivOf<int64_t> { typedef Div64 type; };
template <> struct DivOf<i128> { typedef Div128 type; };

template <class T> BD_HD T tabs(T x) { return x < 0 ? -x : x; }

// ---------------------------------------------------------------------------------------------
// The DFS state of one team (a warp on the GPU, one thread in the host emulation).
//
// Team provides lane(), lanes(), any(bool), sync().  Points are owned round-robin by lanes;
// `st` is this team's stack: entry (level j, column e, point q) at st[(off_j + e) * SLOTS + q].
// `P` holds the lifted points column-major: P[c * N + q], c < K coordinates, c = K the lift.
// ---------------------------------------------------------------------------------------------
enum { ST_SINGULAR = 0, ST_REJECTED = 1, ST_ACCEPTED = 2, ST_TIE = 3 };

// wider exact type for a 2x2 determinant of coordinate minors
template <class TC> struct Wide2;
template <> struct Wide2<int32_t> { typedef int64_t type; };
template <> struct Wide2<int64_t> { typedef i128 type; };
template <> struct Wide2<i128> { typedef i128 type; };  // unused: the 128-bit path tests in 2-D

// Up to 15 point indices below 64, six bits each, in two registers (entries 0..9 in lo,
// 10..14 in hi): the walk's prefix and cursor live here instead of in per-thread local arrays,
// which the compiler would place in local memory (dynamic indices).
struct Idx15 {
  uint64_t lo = 0, hi = 0;
  BD_HD int get(int j) const {
    return j < 10 ? (int)((lo >> (6 * j)) & 63u) : (int)((hi >> (6 * (j - 10))) & 63u);
  }
  BD_HD void set(int j, int v) {
    if (j < 10) lo = (lo & ~(63ull << (6 * j))) | ((uint64_t)v << (6 * j));
    else hi = (hi & ~(63ull << (6 * (j - 10)))) | ((uint64_t)v << (6 * (j - 10)));
  }
};

// the first field at which two packed index lists differ (15 when none of the 15 does)
constexpr uint64_t kIdxHiMask = (1ull << 30) - 1;
BD_HD int first_difference(const Idx15& a, const Idx15& b) {
  const uint64_t x = a.lo ^ b.lo;
  if (x) return ctz64(x) / 6;
  const uint64_t y = (a.hi ^ b.hi) & kIdxHiMask;
  return y ? 10 + ctz64(y) / 6 : 15;
}

// A work item as the device reads it: the prefix as six-bit fields (entries 0..9 in lo, 10..14
// in the low 30 bits of hi) and its length in the top byte of hi.
struct PackedItem {
  uint64_t lo, hi;
};
BD_HD int packed_len(const PackedItem& p) { return (int)(p.hi >> 56); }
BD_HD PackedItem pack_item(const Item& it) {
  Idx15 x;
  for (int i = 0; i < it.len; ++i) x.set(i, it.idx[i]);
  return PackedItem{x.lo, x.hi | ((uint64_t)it.len << 56)};
}

// The pivots and exact dividers of the levels: the same for every lane of a team, so one copy
// per team (in shared memory on the GPU), written by lane 0 and read after a team sync.
template <class TC>
struct Uniform {
  TC piv[KMAX];                        // the pivots p_j (piv[0] = 1)
  typename DivOf<TC>::type dv[KMAX];   // exact divider by p_j (dv[0]: by 1)
  uint64_t taken[KMAX];                // taken[j]: the points s_0 .. s_j (bit q for point q)
  uint32_t queue[64];                  // the 5-D stage's nonsingular quadruples awaiting their test
  unsigned long long rare[4];          // 5-D stage, Stage 5 kernels: sum |D0| (low, high word), cells, ties
};
constexpr size_t kUniformBytes = 1088;  // room for Uniform<TC> of every coordinate type

// ---------------------------------------------------------------------------------------------
// Cells of the triangulation and their inner normals (Sec. 6, Eq. lower-d-face-again): the
// witness-set construction needs, for every cell {a_0 .. a_k}, the unique alpha^ = (alpha, 1)
// with <a^_j, alpha^> = beta on the cell (and > beta off it, which the lower-facet test has
// established).
// ---------------------------------------------------------------------------------------------

// A cell sink: accepted cells are appended as 16-byte records (the K+1 increasing indices,
// then zeros); records past cap are counted but not written.
struct CellSink {
  uint8_t* out;
  unsigned long long* count;
  unsigned long long cap;
};

static BD_COLD void record_cell(CellSink sink, Idx15 s, int pre, int a, int b, int c, int d = -1) {
#ifdef __CUDA_ARCH__
  const unsigned long long slot = atomicAdd(sink.count, 1ull);
#else
  const unsigned long long slot = __atomic_fetch_add(sink.count, 1ull, __ATOMIC_RELAXED);
#endif
  if (slot >= sink.cap) return;
  uint8_t rec[16] = {};
  int n = 0;
  for (int i = 0; i < pre; ++i) rec[n++] = (uint8_t)s.get(i);
  if (a >= 0) rec[n++] = (uint8_t)a;
  if (b >= 0) rec[n++] = (uint8_t)b;
  if (c >= 0) rec[n++] = (uint8_t)c;
  if (d >= 0) rec[n++] = (uint8_t)d;
  memcpy(sink.out + 16 * slot, rec, 16);
}

// 256-bit accumulator for the exact back substitution
struct Acc256 {
  u128 hi = 0, lo = 0;
  BD_HD void add(i128 a, i128 b, bool negate) {  // += (or -=) a * b, modulo 2^256
    u128 h, l;
    mul_wide(a, b, h, l);
    if (negate) {  // two's complement of (h, l)
      l = ~l + 1;
      h = ~h + (l == 0 ? 1 : 0);
    }
    const u128 nl = lo + l;
    hi += h + (nl < lo ? 1 : 0);
    lo = nl;
  }
  BD_HD i128 div_exact(const Div128& D) const {  // quotient known to fit 128 bits
    const int t = D.shift;
    const u128 q = t == 0 ? lo : ((lo >> t) | (hi << (128 - t)));
    return (i128)(q * D.inv);
  }
};

// The inner normal of the cell with indices idx[0..K] over points pts (row-major N x K) lifted
// by lifts: alpha = y / den, beta = beta_num / den with den > 0.  It solves
// (a_j - a_0) . alpha = w_0 - w_j (j = 1..K) by fraction-free elimination (every entry a minor
// of the lifted system) and fraction-free back substitution (y_i = den alpha_i, Cramer), then
// beta = a_0 . alpha + w_0.  false when the cell is flat or a value leaves the output range
// (den and y in int64, beta_num in int128).
BD_HD bool cell_normal_exact(const int64_t* pts, const int64_t* lifts, int K, const uint8_t* idx, int64_t& den,
                             int64_t* y_out, i128& beta_num) {
  i128 A[KMAX][KMAX + 1];
  const int i0 = idx[0];
  for (int r = 0; r < K; ++r) {
    const int q = idx[r + 1];
    for (int c = 0; c < K; ++c) A[r][c] = (i128)pts[(size_t)q * K + c] - pts[(size_t)i0 * K + c];
    A[r][K] = (i128)lifts[i0] - lifts[q];
  }
  Div128 D = make_div((i128)1);
  for (int c = 0; c < K; ++c) {
    int p = -1;
    for (int r = c; r < K; ++r)
      if (A[r][c] != 0) { p = r; break; }
    if (p < 0) return false;
    if (p != c)
      for (int j = 0; j <= K; ++j) {
        const i128 t = A[c][j];
        A[c][j] = A[p][j];
        A[p][j] = t;
      }
    for (int r = c + 1; r < K; ++r) {
      for (int j = c + 1; j <= K; ++j) A[r][j] = bareiss(A[r][j], A[c][c], A[r][c], A[c][j], D);
      A[r][c] = 0;
    }
    D = make_div(A[c][c]);
  }
  const i128 dd = A[K - 1][K - 1];
  i128 y[KMAX];
  for (int i = K - 1; i >= 0; --i) {
    Acc256 num;
    num.add(dd, A[i][K], false);
    for (int j = i + 1; j < K; ++j) num.add(A[i][j], y[j], true);
    y[i] = i == K - 1 ? A[i][K] : num.div_exact(make_div(A[i][i]));
  }
  const bool flip = dd < 0;
  const i128 lim = (i128)1 << 63;
  const i128 dpos = flip ? -dd : dd;
  if (dpos >= lim) return false;
  den = (int64_t)dpos;
  Acc256 b;
  b.add((i128)lifts[i0], dd, false);
  for (int i = 0; i < K; ++i) {
    const i128 yi = flip ? -y[i] : y[i];
    if (yi >= lim || yi < -lim) return false;
    y_out[i] = (int64_t)yi;
    b.add((i128)pts[(size_t)i0 * K + i], y[i], false);
  }
  // beta_num = (a_0 . y + w_0 dd), sign-normalised; it must fit int128
  const bool hi_ok = (b.hi == 0 && (b.lo >> 127) == 0) || (b.hi == ~(u128)0 && (b.lo >> 127) == 1);
  if (!hi_ok) return false;
  beta_num = flip ? -(i128)b.lo : (i128)b.lo;
  return true;
}

static_assert(sizeof(Uniform<i128>) <= kUniformBytes, "uniform state area too small");
static_assert(sizeof(Item) == 16, "an item is four words");

// The reduced state that a walker's exact routes read.  The routes run out of line and take it
// by value: a pointer to the walker itself would pin the whole walker in local memory.
template <class TC, class TL>
struct StateView {
  const TC* sc;
  const TL* sl;
  const Uniform<TC>* u;
  int SLOTS, K;
};

// level K-1 minors of point x for pivot row c on state K-2 (the exact route of a Bareiss step
// for one point)
template <class TC, class TL>
BD_HD void exact_pair_minors(const StateView<TC, TL>& v, int c, int x, TL& C, TL& L) {
  const int o = level_offset(v.K, v.K - 2), S = v.SLOTS;
  const TC xc = v.sc[o * S + c], yc = v.sc[(o + 1) * S + c];
  const int pi = xc != 0 ? 0 : 1;
  const TC a = pi == 0 ? xc : yc, b = pi == 0 ? yc : xc;
  const TC ex_pi = v.sc[(o + pi) * S + x], ex_o = v.sc[(o + 1 - pi) * S + x];
  const typename DivOf<TC>::type D = v.u->dv[v.K - 2];
  C = (TL)bareiss(ex_o, a, ex_pi, b, D);
  L = bareiss(v.sl[(v.K - 2) * S + x], a, ex_pi, v.sl[(v.K - 2) * S + c], D);
}

// exact: C_p L_q - C_q L_p on the reduced state K-2, with the 2-D sign rule (rarely reached)
template <class TC, class TL>
BD_COLD int side3_exact(StateView<TC, TL> v, int c, int p, int q, int sig, TC xc, TC yc) {
  TL Cp, Lp, Cq, Lq;
  exact_pair_minors(v, c, p, Cp, Lp);
  exact_pair_minors(v, c, q, Cq, Lq);
  const int cs = cross_sign(Cp, Lq, Cq, Lp);
  const int pc = (xc != 0 ? xc : yc) < 0 ? -1 : 1;
  // below iff cs != 0 and cs != sign(C_p) * sign(pivot of c); map onto sig's convention
  return cs == 0 ? 0 : ((cs == ((Cp < 0 ? -1 : 1) * pc)) ? sig : -sig);
}

// A point's values on the reduced state K-3 (three coordinate minors and the lift minor) and on
// state K-4 (four coordinate minors and the lift minor), read from the stack or produced by an
// exact Bareiss step.
template <class TC, class TL>
struct Row3 {
  TC x[3];
  TL l;
};
template <class TC, class TL>
struct Row4 {
  TC x[4];
  TL l;
};

template <class TC, class TL>
BD_HD Row3<TC, TL> row3(const StateView<TC, TL>& v, int x) {
  const int o = level_offset(v.K, v.K - 3), S = v.SLOTS;
  return Row3<TC, TL>{{v.sc[o * S + x], v.sc[(o + 1) * S + x], v.sc[(o + 2) * S + x]}, v.sl[(v.K - 3) * S + x]};
}
template <class TC, class TL>
BD_HD Row4<TC, TL> row4(const StateView<TC, TL>& v, int x) {
  const int o = level_offset(v.K, v.K - 4), S = v.SLOTS;
  return Row4<TC, TL>{{v.sc[o * S + x], v.sc[(o + 1) * S + x], v.sc[(o + 2) * S + x], v.sc[(o + 3) * S + x]},
                      v.sl[(v.K - 4) * S + x]};
}

// level K-2 values of row x (two coordinate minors X, Y and the lift minor L) after the Bareiss
// step with pivot row c1, both rows on state K-3, whose pivot D divides; a is c1's pivot and pi
// its column (-1: none)
template <class TC, class TL, class Div>
BD_HD void after3(const Row3<TC, TL>& c1, const Row3<TC, TL>& x, const Div& D, TC& X, TC& Y, TL& L, TC& a,
                  int& pi) {
  pi = c1.x[0] != 0 ? 0 : (c1.x[1] != 0 ? 1 : (c1.x[2] != 0 ? 2 : -1));
  if (pi < 0) {
    X = Y = 0;
    L = 0;
    a = 0;
    return;
  }
  a = c1.x[pi];
  const TC bq = x.x[pi];
  const int r0 = pi == 0 ? 1 : 0, r1 = pi == 2 ? 1 : 2;
  X = bareiss(x.x[r0], a, bq, c1.x[r0], D);
  Y = bareiss(x.x[r1], a, bq, c1.x[r1], D);
  L = bareiss(x.l, a, bq, c1.l, D);
}

// exact K x K minor of the prefix with rows c1, c, p (on state K-3, pivot divider D), carrying
// the sign of the coordinate det3 of the three rows: moving c1's pivot column pi to the front
// permutes the columns by (-1)^pi
template <class TC, class TL, class Div>
BD_HD typename Wide2<TC>::type minor3(const Row3<TC, TL>& c1, const Row3<TC, TL>& c, const Row3<TC, TL>& p,
                                      const Div& D) {
  typedef typename Wide2<TC>::type W2;
  TC Xc, Yc, Xp, Yp, a;
  TL Lc, Lp;
  int pi;
  after3(c1, c, D, Xc, Yc, Lc, a, pi);
  if (pi < 0) return 0;
  after3(c1, p, D, Xp, Yp, Lp, a, pi);
  const W2 m = ((W2)Xc * Yp - (W2)Yc * Xp) / (W2)a;  // exact
  return pi == 1 ? -m : m;
}

// exact side of q for the nonsingular rows (c1, c, p) on state K-3 (pivot divider D), in the
// convention of sig (0 on the hyperplane, sig above, -sig below): two more Bareiss steps (pivot
// rows c1, then c) and the 2-D rule
template <class TC, class TL, class Div>
BD_HD int side_rows(const Row3<TC, TL>& c1, const Row3<TC, TL>& c, const Row3<TC, TL>& p, const Row3<TC, TL>& q,
                    const Div& D, int sig) {
  TC Xc, Yc, Xp, Yp, Xq, Yq, a;
  TL Lc, Lp, Lq;
  int pi;
  after3(c1, c, D, Xc, Yc, Lc, a, pi);
  after3(c1, p, D, Xp, Yp, Lp, a, pi);
  after3(c1, q, D, Xq, Yq, Lq, a, pi);
  const typename DivOf<TC>::type Da = make_div(a);
  const bool px = Xc != 0;  // c's pivot column on state K-2
  const TC b = px ? Xc : Yc, ob = px ? Yc : Xc;
  const TL Cp = (TL)bareiss(px ? Yp : Xp, b, px ? Xp : Yp, ob, Da);
  const TL Cq = (TL)bareiss(px ? Yq : Xq, b, px ? Xq : Yq, ob, Da);
  const TL Mp = bareiss(Lp, b, px ? Xp : Yp, Lc, Da);
  const TL Mq = bareiss(Lq, b, px ? Xq : Yq, Lc, Da);
  const int cs = cross_sign(Cp, Mq, Cq, Mp);
  if (cs == 0) return 0;
  const bool below = cs != (Cp < 0 ? -1 : 1) * (b < 0 ? -1 : 1);  // the 2-D rule
  return below ? -sig : sig;
}

// exact K x K minor of {s_0 .. s_{K-3}, c1, c, p} with the sign of the coordinate det3 on state K-3
template <class TC, class TL>
BD_COLD typename Wide2<TC>::type exact_minor(StateView<TC, TL> v, int c1, int c, int p) {
  return minor3(row3(v, c1), row3(v, c), row3(v, p), v.u->dv[v.K - 3]);
}

// exact side of q for the nonsingular triple (c1, c, p) on state K-3
template <class TC, class TL>
BD_COLD int side4_exact(StateView<TC, TL> v, int c1, int c, int p, int q, int sig) {
  return side_rows(row3(v, c1), row3(v, c), row3(v, p), row3(v, q), v.u->dv[v.K - 3], sig);
}

// state K-3 row of x from state K-4 after the Bareiss step with pivot row c0 (column pi0, its
// first nonzero coordinate), divided by the pivot of state K-4; the other three columns keep
// their order, as in the walker's own step
template <class TC, class TL, class Div>
BD_HD Row3<TC, TL> step43(const Row4<TC, TL>& c0, int pi0, const Row4<TC, TL>& x, const Div& D) {
  const TC a0 = c0.x[pi0], bq = x.x[pi0];
  const int e0 = pi0 == 0 ? 1 : 0, e1 = pi0 <= 1 ? 2 : 1, e2 = pi0 <= 2 ? 3 : 2;
  Row3<TC, TL> r;
  r.x[0] = bareiss(x.x[e0], a0, bq, c0.x[e0], D);
  r.x[1] = bareiss(x.x[e1], a0, bq, c0.x[e1], D);
  r.x[2] = bareiss(x.x[e2], a0, bq, c0.x[e2], D);
  r.l = bareiss(x.l, a0, bq, c0.l, D);
  return r;
}

template <class TC, class TL>
BD_HD int first_nonzero4(const Row4<TC, TL>& r) {
  return r.x[0] != 0 ? 0 : (r.x[1] != 0 ? 1 : (r.x[2] != 0 ? 2 : (r.x[3] != 0 ? 3 : -1)));
}

// The exact 5-D routes of a quadruple c0 < c1 < c < p on state K-4: one Bareiss step with pivot
// row c0 reduces them to the 4-D routes on state K-3 (whose pivot is c0's, a0).  The coordinate
// det4 D4 of the four rows satisfies D4 a0^2 = det3 p^3 (-1)^pi0 (det3 of the reduced rows, p
// the pivot of state K-4), so sign(D4) = sign(det3) sign(p) (-1)^pi0, and the normalized volume
// |D0| = |D4| / |p|^3 = |det3| / a0^2 is the reduced routes' minor.
template <class TC, class TL>
BD_COLD typename Wide2<TC>::type quad_minor(StateView<TC, TL> v, int c0, int c1, int c, int p, int& s4) {
  const Row4<TC, TL> r0 = row4(v, c0);
  const int pi0 = first_nonzero4(r0);
  if (pi0 < 0) {
    s4 = 0;
    return 0;
  }
  const auto& D = v.u->dv[v.K - 4];
  const typename DivOf<TC>::type D3 = make_div(r0.x[pi0]);
  const typename Wide2<TC>::type m =
      minor3(step43(r0, pi0, row4(v, c1), D), step43(r0, pi0, row4(v, c), D), step43(r0, pi0, row4(v, p), D), D3);
  const int sd = v.u->piv[v.K - 4] < 0 ? -1 : 1;
  s4 = m == 0 ? 0 : (m > 0 ? 1 : -1) * sd * ((pi0 & 1) ? -1 : 1);
  return m < 0 ? -m : m;
}

// the exact sign of D4 alone (no division): sign(det3) = sign(Xc Yp - Yc Xp) sign(a) (-1)^pi
// with the second step's values, as minor3 computes them before its exact division
template <class TC, class TL>
BD_COLD int quad_sign(StateView<TC, TL> v, int c0, int c1, int c, int p) {
  const Row4<TC, TL> r0 = row4(v, c0);
  const int pi0 = first_nonzero4(r0);
  if (pi0 < 0) return 0;
  const auto& D = v.u->dv[v.K - 4];
  const typename DivOf<TC>::type D3 = make_div(r0.x[pi0]);
  const Row3<TC, TL> a1 = step43(r0, pi0, row4(v, c1), D);
  TC Xc, Yc, Xp, Yp, a;
  TL Lc, Lp;
  int pi;
  after3(a1, step43(r0, pi0, row4(v, c), D), D3, Xc, Yc, Lc, a, pi);
  if (pi < 0) return 0;
  after3(a1, step43(r0, pi0, row4(v, p), D), D3, Xp, Yp, Lp, a, pi);
  const int cs = cross_sign((TL)Xc, (TL)Yp, (TL)Yc, (TL)Xp);
  const int sd = v.u->piv[v.K - 4] < 0 ? -1 : 1;
  return cs * (a < 0 ? -1 : 1) * (pi == 1 ? -1 : 1) * sd * ((pi0 & 1) ? -1 : 1);
}

// exact side of q for the nonsingular quadruple (c0, c1, c, p) on state K-4
template <class TC, class TL>
BD_COLD int side5_exact(StateView<TC, TL> v, int c0, int c1, int c, int p, int q, int sig) {
  const Row4<TC, TL> r0 = row4(v, c0);
  const int pi0 = first_nonzero4(r0);
  const auto& D = v.u->dv[v.K - 4];
  const typename DivOf<TC>::type D3 = make_div(r0.x[pi0]);
  return side_rows(step43(r0, pi0, row4(v, c1), D), step43(r0, pi0, row4(v, c), D), step43(r0, pi0, row4(v, p), D),
                   step43(r0, pi0, row4(v, q), D), D3, sig);
}

// Stage: the bottom stage, fixed at compile time (4: the 4-D test only; 5: the 5-D test only,
// for callers that guarantee the 32-bit coordinate path and K >= 4) or chosen at run time by
// use5 (0).  A fixed stage keeps the other stage's code out of the kernel.
template <class TC, class TL, class Team, int Stage = 0>
struct Walker {
  typedef typename DivOf<TC>::type Div;
  Team& tm;
  const int64_t* P;
  int N, K, SLOTS;
  TC* sc;           // coordinate minors: (level j, entry e, point q) at sc[(off_j + e) * SLOTS + q]
  TL* sl;           // lift minor of level j for point q at sl[j * SLOTS + q]
  float* fl;        // single-precision copies for the filters: 4 rows of SLOTS floats
  Uniform<TC>* u;   // pivots and dividers (team-shared)
  const uint32_t* tri = nullptr;  // optional colex decode table (device memory; see bottom4)
  CellSink sink{nullptr, nullptr, 0};  // optional: where accepted cells are recorded
  Idx15 s;          // chosen indices s_0 .. s_j
  int psign;        // sign of the level K-1 pivot p_{K-1} (2-D test)
  int valid = 0;    // states 0 .. valid-1 are those of s_0 .. s_{valid-1} (kept across items)
#ifdef BD_COUNT
  Acc* cnt = nullptr;
#endif

  BD_HD Walker(Team& t, const int64_t* P_, int N_, int K_, int SLOTS_, TC* sc_, TL* sl_, float* fl_, void* uni)
      : tm(t), P(P_), N(N_), K(K_), SLOTS(SLOTS_), sc(sc_), sl(sl_), fl(fl_), u(static_cast<Uniform<TC>*>(uni)) {}

  BD_HD StateView<TC, TL> view() const { return StateView<TC, TL>{sc, sl, u, SLOTS, K}; }

  // the single-precision filtered tests run for the int32 and int64 coordinate paths: the 5-D
  // test on state K-4 (int32 coordinate minors, K >= 4), the 4-D test on state K-3 (int64
  // coordinate minors, or K = 3), the 3-D test on state 0 when K = 2; the 128-bit path and K = 1
  // use the 2-D test on the fully reduced state.  The 5-D test saves the Bareiss step of state
  // K-3 at every node and rejects a singular quadruple for a det4, but its single-precision
  // bound is looser (one exact elimination fewer removes cancellation); where the minors are
  // 64-bit numbers its exact routes, in 128-bit arithmetic, cost more than the step it saves.
  static constexpr bool kFiltered = sizeof(TL) == 8;
  static constexpr bool kFive = kFiltered && sizeof(TC) == 4 && Stage != 4;
  bool use5 = true;  // Stage 0: the 5-D stage where it applies (else the 4-D test); the work list must agree
  BD_HD bool five() const { return Stage == 5 ? kFive : (kFive && use5 && K >= 4); }
  // DFS depth at which the bottom stage takes over (the chosen prefix is s_0 .. s_{depth-1}):
  // the 5-D test finishes the last four levels, the 4-D test three, the 3-D and 2-D tests two
  BD_HD int bottom_depth() const {
    return five() ? K - 3 : (kFiltered && K >= 3 ? K - 2 : (K >= 2 ? K - 1 : 1));
  }
  // The filtered tests read single-precision copies of their input state, point-major: the
  // coordinate minors of point q at fl[FS q + e], its lift minor at fl[FS q + LI] (FS = 8,
  // LI = 4 for the 5-D test's five values; FS = 4, LI = 3 for the 4-D test's four).  The Bareiss
  // step that builds that state writes them.
  BD_HD int copy_level() const { return five() ? K - 4 : K - 3; }
  BD_HD int copy_stride() const { return five() ? 8 : 4; }

  // state 0: lifted differences z_q = (a_q - a_{s_0}, w_q - w_{s_0})
  BD_HD void start(int s0) {
    tm.sync();  // the previous item's readers are done with the stack
    s.set(0, s0);
    const bool conv = kFiltered && K >= 3 && copy_level() == 0;  // state 0 is the filter's input
    const int FS = copy_stride();
    for (int q = tm.lane(); q < N; q += tm.lanes()) {
      for (int c = 0; c < K; ++c) {
        const TC v = (TC)(P[c * N + q] - P[c * N + s0]);
        sc[c * SLOTS + q] = v;
        if (conv) fl[FS * q + c] = f32_of(v);
      }
      const TL l = (TL)(P[K * N + q] - P[K * N + s0]);
      sl[q] = l;
      if (conv) fl[FS * q + K] = f32_of(l);  // K coordinates at state 0: the lift minor at index K
    }
    if (tm.lane() == 0) {
      u->dv[0] = make_div((TC)1);
      u->piv[0] = 1;
      u->taken[0] = 1ull << s0;
    }
    psign = 1;
    tm.sync();
  }

  // Bareiss step: state j (j < K-1, or j = K-1 on the 2-D path via build_last) from state j-1
  // with pivot point c (s_j = c).  false when the pivot row has no nonzero coordinate minor
  // (every extension is singular).
  BD_HD bool build(int j, int c) {
    const int po = level_offset(K, j - 1), no = level_offset(K, j);
    const int ncoord = K - j + 1;  // coordinate minors of state j-1
    int pi = -1;
    for (int e = 0; e < ncoord; ++e)
      if (sc[(po + e) * SLOTS + c] != 0) { pi = e; break; }
#ifdef BD_COUNT
    if (cnt) { if (pi < 0) cnt->fails[j]++; else cnt->builds[j]++; }
#endif
    if (pi < 0) return false;
    const TC pj = sc[(po + pi) * SLOTS + c];
    const TL rl = sl[(j - 1) * SLOTS + c];
    const Div D = u->dv[j - 1];
    tm.sync();  // readers of the old state j (a sibling's subtree) are done
    // the filtered test's input state: its single-precision copies are written here too (K - j
    // coordinate minors at fl[FS q + e], the lift minor at fl[FS q + K - j])
    const bool conv = kFiltered && K >= 3 && j == copy_level();
    const int FS = copy_stride(), LI = K - j;
    // state j's pivot, exact divider and point set, for the levels below; every lane forms the
    // divider (a chain of dependent multiplies) before the point loop, so that its latency
    // overlaps the loop's independent work, and lane 0 stores it (read after the closing sync)
    {
      const Div Dj = make_div(pj);
      if (tm.lane() == 0) {
        u->piv[j] = pj;
        u->dv[j] = Dj;
        u->taken[j] = u->taken[j - 1] | (1ull << c);
      }
    }
    auto whole_point = [&](int q) {
      const TC bq = sc[(po + pi) * SLOTS + q];
      auto entry = [&](int e) {
        const int ep = e < pi ? e : e + 1;
        const TC v = bareiss(sc[(po + ep) * SLOTS + q], pj, bq, sc[(po + ep) * SLOTS + c], D);
        sc[(no + e) * SLOTS + q] = v;
        if (conv) fl[FS * q + e] = f32_of(v);
      };
      if constexpr (Stage == 4) {
        // the 4-D kernel interleaves pairs of independent entries (measured: n=24/k=8 0.190 ->
        // 0.179 ms); the 5-D kernel, whose registers are scarcer, keeps them one at a time
#pragma unroll 2
        for (int e = 0; e < ncoord - 1; ++e) entry(e);
      } else {
        for (int e = 0; e < ncoord - 1; ++e) entry(e);
      }
      const TL l = bareiss(sl[(j - 1) * SLOTS + q], pj, bq, rl, D);
      sl[j * SLOTS + q] = l;
      if (conv) fl[FS * q + LI] = f32_of(l);
    };
    // Only the points outside s_0 .. s_{j-1}, c are built: the rows of those vanish from state j
    // on, and no reader of state j or later touches them.  When the rest fit one pass of the
    // team (the team is narrower than N), lane l builds the l-th of them.
    const int W = tm.lanes();
    const uint64_t taken = u->taken[j - 1] | (1ull << c);
    const uint64_t rest = (N >= 64 ? ~0ull : ((1ull << N) - 1)) & ~taken;
    const int nrest = popc64(rest);
    const bool compact = N > W && nrest <= W;
    // otherwise whole points one per lane; when N exceeds the team width, the last N mod width
    // points have their entries dealt across the lanes instead (one lane would carry them alone)
    const int whole = compact ? 0 : (N > W ? N - N % W : N);
    if (compact && (int)tm.lane() < nrest) whole_point(nth_set(rest, tm.lane()));
    for (int q = tm.lane(); q < whole; q += W) whole_point(q);
    for (int t = tm.lane(); !compact && t < (N - whole) * ncoord; t += W) {
      const int q = whole + t / ncoord, e = t % ncoord;  // entry e < ncoord-1: coordinate; last: lift
      const TC bq = sc[(po + pi) * SLOTS + q];
      if (e < ncoord - 1) {
        const int ep = e < pi ? e : e + 1;
        const TC v = bareiss(sc[(po + ep) * SLOTS + q], pj, bq, sc[(po + ep) * SLOTS + c], D);
        sc[(no + e) * SLOTS + q] = v;
        if (conv) fl[FS * q + e] = f32_of(v);
      } else {
        const TL l = bareiss(sl[(j - 1) * SLOTS + q], pj, bq, rl, D);
        sl[j * SLOTS + q] = l;
        if (conv) fl[FS * q + LI] = f32_of(l);
      }
    }
    s.set(j, c);
    tm.sync();
    return true;
  }

  BD_HD uint64_t member_mask(int upto) const {
    uint64_t mask = 0;
    for (int i = 0; i < upto; ++i) mask |= 1ull << s.get(i);
    return mask;
  }

  // ---------------------------------------------------------------------------------------
  // 2-D test on the fully reduced state K-1: each point q carries (C_q, L_q); for the last
  // point p, s(q) = sigma (C_p L_q - C_q L_p) / p_{K-1} and D0 = sigma C_p.
  // ---------------------------------------------------------------------------------------
  BD_HD uint64_t build_last(int c) {  // state K-1 with pivot c; returns the candidate mask
    if (K == 1) {
      uint64_t mine = 0;
      for (int q = tm.lane(); q < N; q += tm.lanes()) {
        if (q > s.get(0) && sc[q] != 0) mine |= 1ull << q;
        fl[q] = (float)sc[q];
        fl[SLOTS + q] = (float)sl[q];
      }
      const uint64_t cand = tm.or_all(mine);
      tm.sync();
      return cand;
    }
    if (!build(K - 1, c)) return 0;
    psign = u->piv[K - 1] < 0 ? -1 : 1;
    const int o = level_offset(K, K - 1);
    uint64_t mine = 0;
    for (int q = tm.lane(); q < N; q += tm.lanes()) {
      const TC v = sc[o * SLOTS + q];
      if (v != 0 && q > c) mine |= 1ull << q;
      fl[q] = (float)v;
      fl[SLOTS + q] = (float)sl[(K - 1) * SLOTS + q];
    }
    const uint64_t cand = tm.or_all(mine);
    tm.sync();
    return cand;
  }

  BD_HD int leaf2(int p, uint64_t mask, TL& absdet) {
    const int lo = level_offset(K, K - 1);
    const TL Cp = (TL)sc[lo * SLOTS + p];
    const TL Lp = sl[(K - 1) * SLOTS + p];
    absdet = tabs(Cp);
    if (Cp == 0) return ST_SINGULAR;
    const float Cpf = fl[p], Lpf = fl[SLOTS + p];
    const int sig = (Cp < 0 ? -1 : 1) * psign;
    bool below = false, on = false;
    for (int q = tm.lane(); q < N; q += tm.lanes()) {
      if (((mask >> q) & 1ull) || q == p) continue;
      int sg = sizeof(TL) == 8 ? cross_sign_filtered(Cpf, fl[SLOTS + q], fl[q], Lpf) : 2;
      if (sg == 2) sg = cross_sign(Cp, sl[(K - 1) * SLOTS + q], (TL)sc[lo * SLOTS + q], Lp);
      if (sg == 0) on = true;
      else if (sg != sig) below = true;
    }
    if (tm.any(below)) return ST_REJECTED;
    return tm.any(on) ? ST_TIE : ST_ACCEPTED;
  }

  // all cells below a state-(K-2) node on the 2-D path (every child c, then every p > c)
  BD_HD void bottom2(Acc& acc) {
    const bool lead = tm.lane() == 0;
    if (K == 1) {
      const uint64_t cand = build_last(0);
      if (lead) acc.singular += (uint64_t)(N - 1 - s.get(0)) - (uint64_t)popc64(cand);
      leaves2(cand, acc);
      return;
    }
    for (int c = s.get(K - 2) + 1; c <= N - 2; ++c) {
      const uint64_t cand = build_last(c);
      if (lead) acc.singular += (uint64_t)(N - 1 - c) - (uint64_t)popc64(cand);
      if (cand) leaves2(cand, acc);
    }
  }

  BD_HD void leaves2(uint64_t cand, Acc& acc) {
    const uint64_t mask = member_mask(K);
    while (cand) {
      const int p = ctz64(cand);
      cand &= cand - 1;
      TL ad;
      const int stt = leaf2(p, mask, ad);
      if (tm.lane() != 0) continue;  // uniform verdict: counted once per team
      if (stt == ST_ACCEPTED) {
        acc.cells += 1;
        acc.nvol += (u128)ad;
        if (sink.out) record_cell(sink, s, K, p, -1, -1);
      }
      else if (stt == ST_TIE) acc.ties += 1;
    }
  }

  // ---------------------------------------------------------------------------------------
  // 3-D test on state K-2.  Each point is v_q = (x_q, y_q, l_q) (two coordinate minors and the
  // lift minor).  Eliminating one more pivot row c (Sylvester) turns the 2-D test into
  //     C_p L_q - C_q L_p = x_c det3(v_c, v_p, v_q) / p_{K-2}^2,   C_p = det2(c, p) / p_{K-2},
  // (for pivot column x; the y-pivot case flips both signs), so q lies strictly below the
  // lifted cell {s_0..s_{K-2}, c, p} iff  sign(det2) sign(p_{K-2}) det3 < 0, and
  // |D0| = |det2| / |p_{K-2}|.  det3 = v_q . (v_c x v_p) is evaluated in single precision with a
  // rigorous error bound; undecided signs use the exact 2-D formulation for that (c, p, q).
  // ---------------------------------------------------------------------------------------
  typedef typename Wide2<TC>::type W2;

  // the test of one lane-owned point q against the pair (c, p); 0 tie, +-1 side, computed
  // exactly when the single-precision value is too close to zero
  BD_HD int side3(int c, int p, int q, float nx, float ny, float nz, float ax, float ay, float az, float xq,
                  float yq, float lq, int sig, TC xc, TC yc) const {
    const float v = fmaf(nx, xq, fmaf(ny, yq, nz * lq));
    // Error budget with u = 2^-24: point copies 2u (f32_of), products 5u, the components of
    // n 6u of their magnitude sums a_*, then one more copy and three roundings: 11u in all of
    // sum a_i |v_qi|.  The bound 2^-17 * sum (32u) leaves a factor ~3 of slack.
    const float bound = 7.63e-6f * fmaf(ax, fabsf(xq), fmaf(ay, fabsf(yq), az * fabsf(lq)));
    if (v > bound) return 1;
    if (v < -bound) return -1;
    return side3_exact(view(), c, p, q, sig, xc, yc);
  }

  // The pairs (c, p), s_{K-2} < c < p < N, are taken in lexicographic order, one per lane and a
  // warp-width of them per round; each lane walks the points q in index order and stops at the
  // first one strictly below its cell, and the round ends when every lane has a verdict.  A
  // rejected pair usually meets a point below within a few steps, so this costs far less than
  // testing every point for every pair.  Per-lane results go into the lane's own accumulator
  // (summed over the warp by the caller).
  BD_HD void bottom3(Acc& acc) {
    const int o = level_offset(K, K - 2);
    const TC dp = u->piv[K - 2];
    const int sd = dp < 0 ? -1 : 1;
    const uint64_t prefix = member_mask(K - 1);
    for (int q = tm.lane(); q < N; q += tm.lanes()) {
      fl[q] = f32_of(sc[o * SLOTS + q]);
      fl[SLOTS + q] = f32_of(sc[(o + 1) * SLOTS + q]);
      fl[2 * SLOTS + q] = f32_of(sl[(K - 2) * SLOTS + q]);
    }
    tm.sync();
    // this lane's pair: the lane-th pair, then every lanes()-th one
    int c = s.get(K - 2) + 1, p = c + 1 + tm.lane();
    for (;;) {
      while (p >= N && c < N - 2) {  // carry into the next c: N-1-c pairs per c
        p -= N - c - 2;
        ++c;
      }
      bool live = p < N;
      if (!tm.any(live)) break;
      W2 d2 = 0;
      TC xc = 0, yc = 0;
      float nx = 0, ny = 0, nz = 0, ax = 0, ay = 0, az = 0;
      int sig = 1;
      if (live) {
        xc = sc[o * SLOTS + c];
        yc = sc[(o + 1) * SLOTS + c];
        d2 = (W2)xc * sc[(o + 1) * SLOTS + p] - (W2)yc * sc[o * SLOTS + p];
        if (d2 == 0) {  // also every pair whose c has no pivot left
          acc.singular += 1;
          live = false;
        }
      }
      if (live) {
        const float xcf = fl[c], ycf = fl[SLOTS + c], lcf = fl[2 * SLOTS + c];
        const float xpf = fl[p], ypf = fl[SLOTS + p], lpf = fl[2 * SLOTS + p];
        const float t1 = ycf * lpf, t2 = lcf * ypf, t3 = lcf * xpf, t4 = xcf * lpf, t5 = xcf * ypf, t6 = ycf * xpf;
        nx = t1 - t2;
        ny = t3 - t4;
        nz = t5 - t6;
        ax = fabsf(t1) + fabsf(t2);
        ay = fabsf(t3) + fabsf(t4);
        az = fabsf(t5) + fabsf(t6);
        sig = (d2 < 0 ? -1 : 1) * sd;  // q is below iff sig * det3 < 0
      }
      const uint64_t excl = prefix | (1ull << c) | (1ull << (live ? p : c));
      bool below = false, on = false;
#ifdef BD_COUNT
      int qt = 0;
#endif
      for (int q = 0; q < N; ++q) {
        if (tm.all(!live || below)) break;
        if (!live || below || ((excl >> q) & 1ull)) continue;
#ifdef BD_COUNT
        ++qt;
#endif
        const int sg = side3(c, p, q, nx, ny, nz, ax, ay, az, fl[q], fl[SLOTS + q], fl[2 * SLOTS + q], sig, xc, yc);
        if (sg == 0) on = true;
        else if (sg != sig) below = true;
      }
#ifdef BD_COUNT
      if (cnt && live) { cnt->pairs++; cnt->qtests += qt; }
#endif
      if (live && !below) {
        if (on) {
          acc.ties += 1;
        } else {
          acc.cells += 1;
          const W2 ad = d2 < 0 ? -d2 : d2;
          const W2 dd = dp < 0 ? -(W2)dp : (W2)dp;
          acc.nvol += (u128)(ad / dd);  // exact: det2 = p_{K-2} * C_p
          if (sink.out) record_cell(sink, s, K - 1, c, p, -1);
        }
      }
      p += tm.lanes();
    }
  }

  // ---------------------------------------------------------------------------------------
  // 4-D test on state K-3.  Each point is v_q = (x_q, y_q, z_q, l_q) (three coordinate minors
  // and the lift minor, all scaled by the pivot p_{K-3}).  For a triple c1 < c < p the simplex
  // {s_0 .. s_{K-3}, c1, c, p} is full-dimensional iff D = det3(x, y, z of c1, c, p) != 0, and
  // then its normalized volume is |D| / p_{K-3}^2 (Sylvester's identity).  The lifted hyperplane
  // through its vertices has height det4(v_c1, v_c, v_p, v_q) / D above q (in the scaled
  // coordinates), so q lies strictly below the lifted cell iff
  //     sign(D) sign(p_{K-3}) det4(v_c1, v_c, v_p, v_q) < 0.
  // det4 = n . v_q with n the cofactor vector of the rows c1, c, p, evaluated in single
  // precision with a rigorous error bound; undecided signs take two exact Bareiss steps
  // (pivot rows c1, then c) and the 2-D rule, as the 2-D path would.
  // ---------------------------------------------------------------------------------------

  // The triples (c1, c, p), s_{K-3} < c1 < c < p < N, are dealt to lanes in colex order, a
  // warp-width per round; each lane walks the points q in index order and stops at the first
  // one strictly below its cell; the round ends when every lane has a verdict.
  BD_HD void bottom4(Acc& acc) {
    const int sd = u->piv[K - 3] < 0 ? -1 : 1;
    const uint64_t prefix = member_mask(K - 2);
    // fl holds the single-precision copies of state K-3 (written by the step that built it),
    // point-major: the four values of point q at fl[4q .. 4q+3], one 16-byte load per point.
    // Error bounds, u = 2^-24: every term of det4 is a product of four point copies (2u each,
    // f32_of) through at most nine roundings (2x2 minor: product and difference; cofactor:
    // product and two sums; det4: product and three sums), so |error| <= 17.001u T with T the
    // sum of the magnitudes of all 24 terms; T evaluated in single precision (same depth, one
    // more rounding for the scale) is at least (1 - 19u) T, so eps = 2^-19 = 32u covers it with
    // a factor ~1.9 to spare.  The cofactor det3 (11u) uses the same eps.  Below 2^23 every
    // operand and partial result is an integer held exactly, and the single-precision value is
    // the exact one.
    const float eps = 1.9073486328125e-6f;  // 2^-19
    // Triple number t in colex order (by p, then c, then c1) is decoded directly:
    // C(k,3) <= t < C(k+1,3), then C(j,2) <= t - C(k,3) < C(j+1,2), i = t - C(k,3) - C(j,2),
    // and (c1, c, p) = s_{K-3} + 1 + (i, j, k).  k never decreases for a lane.
    const int base = s.get(K - 3) + 1, R = N - base;
    const int total = R * (R - 1) * (R - 2) / 6;
    int k = 2;
    // with a decode table (colex triples packed i | j << 8 | k << 16), the next round's entry
    // is loaded while this round runs
    uint32_t nxt = 0;
    if (tri && (int)tm.lane() < total) nxt = ldg_u32(tri + tm.lane());
    for (int t0 = 0; t0 < total; t0 += tm.lanes()) {
      const int t = t0 + tm.lane();
      bool live = t < total;
      int c1 = base, c = base, p = base;
      if (tri) {
        const uint32_t w = nxt;
        if (t + (int)tm.lanes() < total) nxt = ldg_u32(tri + t + tm.lanes());
        if (live) {
          c1 = base + (int)(w & 255u);
          c = base + (int)((w >> 8) & 255u);
          p = base + (int)(w >> 16);
        }
      } else if (live) {
        while ((k + 1) * k * (k - 1) / 6 <= t) ++k;
        const int u = t - k * (k - 1) * (k - 2) / 6;
        int jj = (int)((1.0f + approx_sqrt(8.0f * (float)u + 1.0f)) * 0.5f);
        if (jj * (jj - 1) / 2 > u) --jj;
        else if ((jj + 1) * jj / 2 <= u) ++jj;
        c1 = base + u - jj * (jj - 1) / 2;
        c = base + jj;
        p = base + k;
      }
      float n0 = 0, n1 = 0, n2 = 0, n3 = 0, e0 = 0, e1 = 0, e2 = 0, e3 = 0;
      int sig = 1, s3 = 0;
      if (live) {
        const F4 A = ld4(fl + 4 * c1), U = ld4(fl + 4 * c), Wp = ld4(fl + 4 * p);
        const float a0 = A.x, a1 = A.y, a2 = A.z, a3 = A.w;
        const float u0 = U.x, u1 = U.y, u2 = U.z, u3 = U.w;
        const float w0 = Wp.x, w1 = Wp.y, w2 = Wp.z, w3 = Wp.w;
        // 2x2 minors of rows (c, p) and their magnitude sums
        const float m01 = u0 * w1 - u1 * w0, m02 = u0 * w2 - u2 * w0, m12 = u1 * w2 - u2 * w1;
        const float M01 = fabsf(u0 * w1) + fabsf(u1 * w0), M02 = fabsf(u0 * w2) + fabsf(u2 * w0),
                    M12 = fabsf(u1 * w2) + fabsf(u2 * w1);
        const float D3 = a0 * m12 - a1 * m02 + a2 * m01;
        const float B3 = fabsf(a0) * M12 + fabsf(a1) * M02 + fabsf(a2) * M01;
        if (fabsf(D3) > eps * B3 || B3 < 8388608.0f) s3 = (D3 > 0) - (D3 < 0);
        else {
          const W2 m = exact_minor(view(), c1, c, p);
          s3 = (m > 0) - (m < 0);
        }
        if (s3 == 0) {
          acc.singular += 1;
          live = false;
        } else {
          const float m03 = u0 * w3 - u3 * w0, m13 = u1 * w3 - u3 * w1, m23 = u2 * w3 - u3 * w2;
          const float M03 = fabsf(u0 * w3) + fabsf(u3 * w0), M13 = fabsf(u1 * w3) + fabsf(u3 * w1),
                      M23 = fabsf(u2 * w3) + fabsf(u3 * w2);
          // det4(c1, c, p, q) = -q0 D0 + q1 D1 - q2 D2 + q3 D3, D_i the det3 without column i
          n0 = -(a1 * m23 - a2 * m13 + a3 * m12);
          n1 = a0 * m23 - a2 * m03 + a3 * m02;
          n2 = -(a0 * m13 - a1 * m03 + a3 * m01);
          n3 = D3;
          e0 = eps * (fabsf(a1) * M23 + fabsf(a2) * M13 + fabsf(a3) * M12);
          e1 = eps * (fabsf(a0) * M23 + fabsf(a2) * M03 + fabsf(a3) * M02);
          e2 = eps * (fabsf(a0) * M13 + fabsf(a1) * M03 + fabsf(a3) * M01);
          e3 = eps * B3;
          sig = s3 * sd;  // q is below iff sig * det4 < 0
        }
      }
      const uint64_t excl = prefix | (1ull << c1) | (1ull << c) | (live ? 1ull << p : 0ull);
      bool below = false, on = false;
#ifdef BD_COUNT
      int qt = 0;
#endif
      // single-precision scan; undecided points are noted and decided exactly afterwards,
      // unless a point strictly below was found (as in the 5-D test's scan)
      uint64_t und = 0;
      for (int q = 0; q < N; ++q) {
        if (tm.all(!live || below)) break;
        if (!live || below || ((excl >> q) & 1ull)) continue;
#ifdef BD_COUNT
        ++qt;
#endif
        const F4 X = ld4(fl + 4 * q);
        const float x0 = X.x, x1 = X.y, x2 = X.z, x3 = X.w;
        const float v = fmaf(n0, x0, fmaf(n1, x1, fmaf(n2, x2, n3 * x3)));
        const float bound = fmaf(e0, fabsf(x0), fmaf(e1, fabsf(x1), fmaf(e2, fabsf(x2), e3 * fabsf(x3))));
        if (v > bound) {
          if (sig < 0) below = true;
        } else if (v < -bound) {
          if (sig > 0) below = true;
        } else {
          und |= 1ull << q;
        }
      }
      if (live && !below) {
        for (; und; und &= und - 1) {
          const int sg = side4_exact(view(), c1, c, p, ctz64(und), sig);
          if (sg == 0) {
            on = true;
          } else if (sg != sig) {
            below = true;
            break;
          }
        }
      }
#ifdef BD_COUNT
      if (cnt && live) { cnt->pairs++; cnt->qtests += qt; }
#endif
      if (live && !below) {
        if (on) {
          acc.ties += 1;
        } else {
          acc.cells += 1;
          const W2 m = exact_minor(view(), c1, c, p);
          acc.nvol += (u128)(m < 0 ? -m : m);
          if (sink.out) record_cell(sink, s, K - 2, c1, c, p);
        }
      }
    }
  }

  // ---------------------------------------------------------------------------------------
  // 5-D test on state K-4.  Each point is v_q = (x0, x1, x2, x3, l) (four coordinate minors and
  // the lift minor, all scaled by the pivot p of state K-4).  For a quadruple c0 < c1 < c < p
  // the simplex {s_0 .. s_{K-4}, c0, c1, c, p} is full-dimensional iff the coordinate det4
  // D4 of the four rows is nonzero, and then its normalized volume is |D4| / |p|^3
  // (Sylvester's identity: a k x k determinant of state-j rows is the full minor times the
  // state's pivot to the power k-1).  The lifted hyperplane through its vertices puts q
  // strictly below the cell iff
  //     sign(D4) sign(p) det5(v_c0, v_c1, v_c, v_p, v_q) < 0,
  // det5 = n . v_q with n the five signed cofactors of the rows c0, c1, c, p.
  // Phase A deals the triples c1 < c < p (the three largest points of a quadruple) to lanes, a
  // warp-width per round; each lane forms the four 3x3 minors of its triple's coordinate rows
  // once and then, for every c0 < c1 in turn, decides sign(D4) = sign(v_c0 . minors) (single
  // precision with a rigorous error bound, exactly when undecided); the nonsingular
  // quadruples go to the team's queue.  The triples are taken with their smallest point c1 in
  // descending order, so that the lanes of a round loop over similar counts of c0.  Phase B
  // takes a warp-width of queued quadruples, one per lane, forms n and its error bounds and
  // walks the points as the 4-D test does.  Most quadruples are singular, and a singular one
  // costs its lane a four-term dot product of Phase A.
  // ---------------------------------------------------------------------------------------

  static BD_HD uint32_t c3(int n) { return n < 3 ? 0u : (uint32_t)(n * (n - 1) * (n - 2) / 6); }

  // colex triple of rank t (i < j < k) packed i | j << 8 | k << 16, from the decode table when
  // present
  BD_HD uint32_t colex3(uint32_t t) const {
    if (tri) return ldg_u32(tri + t);
    int k = 2;
    while ((uint32_t)((k + 1) * k * (k - 1) / 6) <= t) ++k;
    const uint32_t u = t - (uint32_t)(k * (k - 1) * (k - 2) / 6);
    int j = 1;
    while ((uint32_t)((j + 1) * j / 2) <= u) ++j;
    const uint32_t i = u - (uint32_t)(j * (j - 1) / 2);
    return i | (uint32_t)j << 8 | (uint32_t)k << 16;
  }

  // sign of the coordinate det4 of rows c0, c1, c, p, from the single-precision copies.
  // Error bound, u = 2^-24: every term is a product of four copies (2u each, f32_of) through at
  // most nine roundings (2x2 minor: product and difference; 3x3: product and two sums; det4:
  // product and three sums), so |error| <= 17.001u T with T the sum of the magnitudes of the 24
  // terms; T evaluated in single precision (same depth) is at least (1 - 19u) T, and
  // eps = 2^-19 = 32u covers it with a factor ~1.9.  Below 2^23 every operand and partial result
  // is an integer held exactly.  Undecided (or overflowed) values take the exact route.
  BD_HD int d4_sign(int c0, int c1, int c, int p) const {
    const float eps = 1.9073486328125e-6f;  // 2^-19
    const F4 A = ld4(fl + 8 * c0), B = ld4(fl + 8 * c1), U = ld4(fl + 8 * c), V = ld4(fl + 8 * p);
    const float m01 = U.x * V.y - U.y * V.x, m02 = U.x * V.z - U.z * V.x, m03 = U.x * V.w - U.w * V.x;
    const float m12 = U.y * V.z - U.z * V.y, m13 = U.y * V.w - U.w * V.y, m23 = U.z * V.w - U.w * V.z;
    const float M01 = fabsf(U.x * V.y) + fabsf(U.y * V.x), M02 = fabsf(U.x * V.z) + fabsf(U.z * V.x);
    const float M03 = fabsf(U.x * V.w) + fabsf(U.w * V.x), M12 = fabsf(U.y * V.z) + fabsf(U.z * V.y);
    const float M13 = fabsf(U.y * V.w) + fabsf(U.w * V.y), M23 = fabsf(U.z * V.w) + fabsf(U.w * V.z);
    const float t123 = B.y * m23 - B.z * m13 + B.w * m12, t023 = B.x * m23 - B.z * m03 + B.w * m02;
    const float t013 = B.x * m13 - B.y * m03 + B.w * m01, t012 = B.x * m12 - B.y * m02 + B.z * m01;
    const float T123 = fabsf(B.y) * M23 + fabsf(B.z) * M13 + fabsf(B.w) * M12;
    const float T023 = fabsf(B.x) * M23 + fabsf(B.z) * M03 + fabsf(B.w) * M02;
    const float T013 = fabsf(B.x) * M13 + fabsf(B.y) * M03 + fabsf(B.w) * M01;
    const float T012 = fabsf(B.x) * M12 + fabsf(B.y) * M02 + fabsf(B.z) * M01;
    const float D4 = A.x * t123 - A.y * t023 + A.z * t013 - A.w * t012;
    const float B4 = fabsf(A.x) * T123 + fabsf(A.y) * T023 + fabsf(A.z) * T013 + fabsf(A.w) * T012;
    if (fabsf(D4) > eps * B4 || B4 < 8388608.0f) return (D4 > 0) - (D4 < 0);
    return quad_sign(view(), c0, c1, c, p);
  }

  // Phase B on the first `take` of the qlen queued quadruples (one per lane); the rest move to
  // the front of the queue.
  // Error bound of det5, u = 2^-24: every term is a product of five copies (10u) through at most
  // fourteen roundings (2x2: 2, 3x3: 3, cofactor: 4, det5: 5), so |error| <= 24.001u T with T
  // the magnitude sum; the bound evaluated in single precision (cofactor magnitudes, then the
  // sum against |q|) is at least (1 - 19u) eps T, and eps = 2^-19 = 32u covers the error with a
  // factor ~1.3.  Undecided (or overflowed) values take the exact route.
  BD_HD void quads(Acc& acc, int take, int qlen, int sd, uint64_t rest) {
    const int lane = tm.lane();
    const bool busy = lane < take;
    const uint32_t rec = busy ? u->queue[lane] : 0u;
    tm.sync();  // every lane has its entry
    if (lane + take < qlen) u->queue[lane] = u->queue[lane + take];
    tm.sync();
    const int c0 = rec & 63u, c1 = (rec >> 6) & 63u, c = (rec >> 12) & 63u, p = (rec >> 18) & 63u;
    const int sig = ((rec >> 31) ? -1 : 1) * sd;  // q is below iff sig * det5 < 0
    float n0 = 0, n1 = 0, n2 = 0, n3 = 0, n4 = 0, e0 = 0, e1 = 0, e2 = 0, e3 = 0, e4 = 0;
    if (busy) {
      const float eps = 1.9073486328125e-6f;  // 2^-19
      const F4 A = ld4(fl + 8 * c0), B = ld4(fl + 8 * c1), U = ld4(fl + 8 * c), V = ld4(fl + 8 * p);
      const float A4 = fl[8 * c0 + 4], B4 = fl[8 * c1 + 4], U4 = fl[8 * c + 4], V4 = fl[8 * p + 4];
      // 2x2 minors of rows (c, p) on columns a < b (column 4: the lift), and their magnitudes
      const float m01 = U.x * V.y - U.y * V.x, m02 = U.x * V.z - U.z * V.x, m03 = U.x * V.w - U.w * V.x;
      const float m04 = U.x * V4 - U4 * V.x, m12 = U.y * V.z - U.z * V.y, m13 = U.y * V.w - U.w * V.y;
      const float m14 = U.y * V4 - U4 * V.y, m23 = U.z * V.w - U.w * V.z, m24 = U.z * V4 - U4 * V.z;
      const float m34 = U.w * V4 - U4 * V.w;
      const float M01 = fabsf(U.x * V.y) + fabsf(U.y * V.x), M02 = fabsf(U.x * V.z) + fabsf(U.z * V.x);
      const float M03 = fabsf(U.x * V.w) + fabsf(U.w * V.x), M04 = fabsf(U.x * V4) + fabsf(U4 * V.x);
      const float M12 = fabsf(U.y * V.z) + fabsf(U.z * V.y), M13 = fabsf(U.y * V.w) + fabsf(U.w * V.y);
      const float M14 = fabsf(U.y * V4) + fabsf(U4 * V.y), M23 = fabsf(U.z * V.w) + fabsf(U.w * V.z);
      const float M24 = fabsf(U.z * V4) + fabsf(U4 * V.z), M34 = fabsf(U.w * V4) + fabsf(U4 * V.w);
      // 3x3 minors of rows (c1, c, p) on columns a < b < c
      const float b0 = B.x, b1 = B.y, b2 = B.z, b3 = B.w;
      const float ab0 = fabsf(b0), ab1 = fabsf(b1), ab2 = fabsf(b2), ab3 = fabsf(b3), ab4 = fabsf(B4);
      const float t012 = b0 * m12 - b1 * m02 + b2 * m01, T012 = ab0 * M12 + ab1 * M02 + ab2 * M01;
      const float t013 = b0 * m13 - b1 * m03 + b3 * m01, T013 = ab0 * M13 + ab1 * M03 + ab3 * M01;
      const float t014 = b0 * m14 - b1 * m04 + B4 * m01, T014 = ab0 * M14 + ab1 * M04 + ab4 * M01;
      const float t023 = b0 * m23 - b2 * m03 + b3 * m02, T023 = ab0 * M23 + ab2 * M03 + ab3 * M02;
      const float t024 = b0 * m24 - b2 * m04 + B4 * m02, T024 = ab0 * M24 + ab2 * M04 + ab4 * M02;
      const float t034 = b0 * m34 - b3 * m04 + B4 * m03, T034 = ab0 * M34 + ab3 * M04 + ab4 * M03;
      const float t123 = b1 * m23 - b2 * m13 + b3 * m12, T123 = ab1 * M23 + ab2 * M13 + ab3 * M12;
      const float t124 = b1 * m24 - b2 * m14 + B4 * m12, T124 = ab1 * M24 + ab2 * M14 + ab4 * M12;
      const float t134 = b1 * m34 - b3 * m14 + B4 * m13, T134 = ab1 * M34 + ab3 * M14 + ab4 * M13;
      const float t234 = b2 * m34 - b3 * m24 + B4 * m23, T234 = ab2 * M34 + ab3 * M24 + ab4 * M23;
      // cofactors along q's row: n_e = (-1)^e det4(rows c0, c1, c, p without column e)
      const float a0 = A.x, a1 = A.y, a2 = A.z, a3 = A.w;
      const float aa0 = fabsf(a0), aa1 = fabsf(a1), aa2 = fabsf(a2), aa3 = fabsf(a3), aa4 = fabsf(A4);
      n0 = a1 * t234 - a2 * t134 + a3 * t124 - A4 * t123;
      n1 = -(a0 * t234 - a2 * t034 + a3 * t024 - A4 * t023);
      n2 = a0 * t134 - a1 * t034 + a3 * t014 - A4 * t013;
      n3 = -(a0 * t124 - a1 * t024 + a2 * t014 - A4 * t012);
      n4 = a0 * t123 - a1 * t023 + a2 * t013 - a3 * t012;
      e0 = eps * (aa1 * T234 + aa2 * T134 + aa3 * T124 + aa4 * T123);
      e1 = eps * (aa0 * T234 + aa2 * T034 + aa3 * T024 + aa4 * T023);
      e2 = eps * (aa0 * T134 + aa1 * T034 + aa3 * T014 + aa4 * T013);
      e3 = eps * (aa0 * T124 + aa1 * T024 + aa2 * T014 + aa4 * T012);
      e4 = eps * (aa0 * T123 + aa1 * T023 + aa2 * T013 + aa3 * T012);
    }
    const uint64_t own = busy ? (1ull << c0) | (1ull << c1) | (1ull << c) | (1ull << p) : 0ull;
    bool below = false, on = false;
    // The scan decides each point in single precision; a point whose value lies inside the
    // error bound is noted in `und` and decided exactly after the scan, and only if no point
    // was found strictly below (the exact routes are calls: out of the loop, they do not
    // constrain its registers).
    uint64_t und = 0;
    for (uint64_t f = rest; f; f &= f - 1) {
      if (tm.all(!busy || below)) break;
      const int q = ctz64(f);  // the same point for every lane
      if (!busy || below || ((own >> q) & 1ull)) continue;
      const F4 X = ld4(fl + 8 * q);
      const float x4 = fl[8 * q + 4];
      const float v = fmaf(n0, X.x, fmaf(n1, X.y, fmaf(n2, X.z, fmaf(n3, X.w, n4 * x4))));
      const float bound = fmaf(e0, fabsf(X.x), fmaf(e1, fabsf(X.y), fmaf(e2, fabsf(X.z), fmaf(e3, fabsf(X.w), e4 * fabsf(x4)))));
      if (v > bound) {
        if (sig < 0) below = true;  // side +1 against sig -1
      } else if (v < -bound) {
        if (sig > 0) below = true;
      } else {
        und |= 1ull << q;
      }
    }
    if (busy && !below) {
      for (; und; und &= und - 1) {
        const int sg = side5_exact(view(), c0, c1, c, p, ctz64(und), sig);
        if (sg == 0) {
          on = true;
        } else if (sg != sig) {
          below = true;
          break;
        }
      }
    }
#ifdef BD_COUNT
    if (cnt && busy) cnt->pairs++;
#endif
    if (busy && !below) {
      int s4;
      const W2 m = on ? (W2)0 : quad_minor(view(), c0, c1, c, p, s4);
      if (!on && sink.out) record_cell(sink, s, K - 3, c0, c1, c, p);
#ifdef __CUDA_ARCH__
      if (Stage == 5) {  // into the team's shared accumulators (several lanes may decide at once)
        if (on) {
          atomicAdd(&u->rare[3], 1ull);
        } else {
          const unsigned long long lo = (unsigned long long)(uint64_t)(u128)m;
          const unsigned long long hi = (unsigned long long)(uint64_t)((u128)m >> 64);
          const unsigned long long old = atomicAdd(&u->rare[0], lo);
          const unsigned long long carry = old + lo < old ? 1ull : 0ull;
          if (hi + carry) atomicAdd(&u->rare[1], hi + carry);
          atomicAdd(&u->rare[2], 1ull);
        }
      } else
#endif
      if (on) {
        acc.ties += 1;
      } else {
        acc.cells += 1;
        acc.nvol += (u128)m;
      }
    }
  }


  // the four 3x3 minors of the coordinate rows c1, c, p on state K-4 (t_abc: columns a < b < c)
  // and their magnitude sums, the factors of D4 along the row of c0 (the same single-precision
  // expression as d4_sign)
  BD_HD void minors3(int c1, int c, int p, float& t123, float& t023, float& t013, float& t012, float& T123,
                     float& T023, float& T013, float& T012) const {
    const F4 B = ld4(fl + 8 * c1), U = ld4(fl + 8 * c), V = ld4(fl + 8 * p);
    const float m01 = U.x * V.y - U.y * V.x, m02 = U.x * V.z - U.z * V.x, m03 = U.x * V.w - U.w * V.x;
    const float m12 = U.y * V.z - U.z * V.y, m13 = U.y * V.w - U.w * V.y, m23 = U.z * V.w - U.w * V.z;
    const float M01 = fabsf(U.x * V.y) + fabsf(U.y * V.x), M02 = fabsf(U.x * V.z) + fabsf(U.z * V.x);
    const float M03 = fabsf(U.x * V.w) + fabsf(U.w * V.x), M12 = fabsf(U.y * V.z) + fabsf(U.z * V.y);
    const float M13 = fabsf(U.y * V.w) + fabsf(U.w * V.y), M23 = fabsf(U.z * V.w) + fabsf(U.w * V.z);
    t123 = B.y * m23 - B.z * m13 + B.w * m12;
    t023 = B.x * m23 - B.z * m03 + B.w * m02;
    t013 = B.x * m13 - B.y * m03 + B.w * m01;
    t012 = B.x * m12 - B.y * m02 + B.z * m01;
    T123 = fabsf(B.y) * M23 + fabsf(B.z) * M13 + fabsf(B.w) * M12;
    T023 = fabsf(B.x) * M23 + fabsf(B.z) * M03 + fabsf(B.w) * M02;
    T013 = fabsf(B.x) * M13 + fabsf(B.y) * M03 + fabsf(B.w) * M01;
    T012 = fabsf(B.x) * M12 + fabsf(B.y) * M02 + fabsf(B.z) * M01;
  }

  BD_HD void bottom5(Acc& acc) {
    const int sd = u->piv[K - 4] < 0 ? -1 : 1;
    const uint64_t rest = (N >= 64 ? ~0ull : ((1ull << N) - 1)) & ~u->taken[K - 4];  // the points q to test
    const int base = s.get(K - 4) + 1, R = N - base;
    // triples whose smallest point is not the node's first (each has c0 candidates below it):
    // colex rank t over R-1 positions counted from the node's last point down, so that (i, j, k)
    // is the triple c1 = base + R-1-k < c = base + R-1-j < p = base + R-1-i; the ranks ascend
    // with k, i.e. c1 descends
    const uint32_t total = c3(R - 1);
    const int W = tm.lanes(), lane = tm.lane();
    const float eps = 1.9073486328125e-6f;  // 2^-19: the error bound of d4_sign
    int qlen = 0;
    for (uint32_t t0 = 0; t0 < total; t0 += (uint32_t)W) {
      const uint32_t t = t0 + (uint32_t)lane;
      const bool live = t < total;
      int r1 = 0, c1 = base, c = base, p = base;  // r1: the number of c0 candidates (c0 < c1)
      if (live) {
        const uint32_t w = colex3(t);
        r1 = R - 1 - (int)(w >> 16);
        c1 = base + r1;
        c = base + R - 1 - (int)((w >> 8) & 255u);
        p = base + R - 1 - (int)(w & 255u);
      }
      float t123, t023, t013, t012, T123, T023, T013, T012;
      minors3(c1, c, p, t123, t023, t013, t012, T123, T023, T013, T012);
      const int rounds = (int)tm.max_u32(live ? (uint32_t)r1 : 0u);  // lane 0's: the round's largest c1
      for (int i0 = 0; i0 < rounds; ++i0) {
        const int c0 = base + i0;  // the same point for every lane: a broadcast read
        bool act = live && i0 < r1;
        uint32_t rec = 0;
        if (act) {
          const F4 A = ld4(fl + 8 * c0);
          const float D4 = A.x * t123 - A.y * t023 + A.z * t013 - A.w * t012;
          const float B4 = fabsf(A.x) * T123 + fabsf(A.y) * T023 + fabsf(A.z) * T013 + fabsf(A.w) * T012;
          const int s4 = (fabsf(D4) > eps * B4 || B4 < 8388608.0f) ? (D4 > 0) - (D4 < 0) : quad_sign(view(), c0, c1, c, p);
          if (s4 == 0) {
            acc.singular += 1;
            act = false;
          } else {
            rec = (uint32_t)c0 | (uint32_t)c1 << 6 | (uint32_t)c << 12 | (uint32_t)p << 18 | (s4 < 0 ? 1u << 31 : 0u);
          }
        }
        const uint64_t bal = tm.ballot(act);
        if (act) u->queue[qlen + popc64(bal & ((1ull << lane) - 1ull))] = rec;
        qlen += popc64(bal);
        if (qlen >= W) {
          tm.sync();
          quads(acc, W, qlen, sd, rest);
          qlen -= W;
        }
      }
    }
    if (qlen > 0) {
      tm.sync();
      quads(acc, qlen, qlen, sd, rest);
    }
  }

  // The quadruples of the node on state K-4 whose first point is `first` (a work item one level
  // below the node: a large node's quadruples are split this way over several warps).  The
  // triples (a1, a2, a3) after `first` are dealt in colex order, as in bottom4.
  BD_COLD void bottom5_first(Acc& acc, int first) {
    const int sd = u->piv[K - 4] < 0 ? -1 : 1;
    const uint64_t rest = (N >= 64 ? ~0ull : ((1ull << N) - 1)) & ~u->taken[K - 4];
    const int base = first + 1, R = N - base;
    const uint32_t total = c3(R);
    const int W = tm.lanes(), lane = tm.lane();
    int qlen = 0;
    for (uint32_t t0 = 0; t0 < total; t0 += (uint32_t)W) {
      const uint32_t t = t0 + (uint32_t)lane;
      bool live = t < total;
      uint32_t rec = 0;
      if (live) {
        const uint32_t w = colex3(t);
        const int a1 = base + (int)(w & 255u), a2 = base + (int)((w >> 8) & 255u), a3 = base + (int)(w >> 16);
        const int s4 = d4_sign(first, a1, a2, a3);
        if (s4 == 0) {
          acc.singular += 1;
          live = false;
        } else {
          rec = (uint32_t)first | (uint32_t)a1 << 6 | (uint32_t)a2 << 12 | (uint32_t)a3 << 18 | (s4 < 0 ? 1u << 31 : 0u);
        }
      }
      const uint64_t bal = tm.ballot(live);
      if (live) u->queue[qlen + popc64(bal & ((1ull << lane) - 1ull))] = rec;
      qlen += popc64(bal);
      if (qlen >= W) {
        tm.sync();
        quads(acc, W, qlen, sd, rest);
        qlen -= W;
      }
    }
    if (qlen > 0) {
      tm.sync();
      quads(acc, qlen, qlen, sd, rest);
    }
  }

  BD_HD void bottom(Acc& acc) {
    if (five()) bottom5(acc);
    else if (kFiltered && K >= 3) bottom4(acc);
    else if (kFiltered && K == 2) bottom3(acc);
    else bottom2(acc);
  }

  // every (K+1)-subset extending the prefix it.idx[0 .. it.len-1] (len <= bottom depth, or
  // bottom depth + 1 for the 5-D stage: then the last index is the first point of the
  // quadruples taken).  The states of a prefix shared with the previous item are still in place
  // and are not rebuilt (the depth-first walk below an item only rewrites levels >= its length).
  BD_HD void run_item(const Item& it, Acc& acc) { run_item(pack_item(it), acc); }

  BD_HD void run_item(const PackedItem& it, Acc& acc) {
    const Idx15 pre{it.lo, it.hi & kIdxHiMask};
    const int L = packed_len(it);
    const int B = bottom_depth();
    const int LB = L < B ? L : B;  // the levels built from the prefix
    const bool lead = tm.lane() == 0;  // uniform counts are added once per team
    const int last = pre.get(L - 1);
    // the first level whose index differs from the built prefix (six-bit fields compared at once)
    int m = first_difference(s, pre);
    m = m < valid ? m : valid;
    m = m < LB ? m : LB;
    if (m == 0) {
      start(pre.get(0));
      m = 1;
    }
    valid = m;
    for (int j = m; j < LB; ++j) {
      if (!build(j, pre.get(j))) {
        if (lead) acc.singular += subtree_size(N, K, last, L);
        return;
      }
      valid = j + 1;
    }
    if (kFive && L > B) {  // a 5-D item below its node (the work list goes that deep only there)
      bottom5_first(acc, last);
      return;
    }
    Idx15 cur;  // cur[j]: the last index tried at level j
    int j = L;
    cur.set(j, last);
    for (;;) {
      if (j == B) {
        bottom(acc);
        if (--j < L) break;
        continue;
      }
      const int c = cur.get(j) + 1;
      cur.set(j, c);
      if (c > N - 1 - (K - j)) {
        if (--j < L) break;
        continue;
      }
      if (!build(j, c)) {
        if (lead) acc.singular += binom(N - 1 - c, K - j);
        continue;
      }
      ++j;
      cur.set(j, c);
    }
  }

  // status of one given subset sub[0] < .. < sub[K] (2-D route)
  BD_HD int classify(const uint8_t* sub, TL& absdet) {
    valid = 0;
    start(sub[0]);
    for (int j = 1; j < K - 1; ++j)
      if (!build(j, sub[j])) { absdet = 0; return ST_SINGULAR; }
    if (K >= 2) s.set(K - 1, sub[K - 1]);
    const uint64_t cand = build_last(K >= 2 ? sub[K - 1] : 0);
    if (!((cand >> sub[K]) & 1ull)) { absdet = 0; return ST_SINGULAR; }
    return leaf2(sub[K], member_mask(K), absdet);
  }
};

}  // namespace bd

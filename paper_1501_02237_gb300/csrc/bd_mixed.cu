// Mixed volume (the BKK bound, Appendix A): host preparation, the enumeration kernel, the
// C ABI (bd_mixed_volume, bd_mixed_volume_lifted) and the host emulation of the same walker
// (bd_host_mixed_volume_lifted).  The method and the exact test are in bd_mixed.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>
#include <vector>

#include "../../include/binodeg.h"
#include "bd_internal.h"
#include "bd_lifts.h"
#include "bd_mixed.cuh"
#include "bd_teams.h"

using bd::i128;
using bd::u128;

namespace {

constexpr int kMixedMaxWarps = 8;  // warps per block: chosen per problem, at most this

struct MixedWarp {
  __device__ int lane() const { return threadIdx.x & 31; }
  __device__ int lanes() const { return 32; }
  __device__ void sync() const { __syncwarp(); }
  __device__ uint32_t max_u32(uint32_t x) const { return __reduce_max_sync(0xffffffffu, x); }
};

// One problem ready for a launch: rows in level order, relative to each component's first
// point (coordinates and lift), and the shape.
struct MixedPrep {
  bd::MixedShape shape{};
  std::vector<int> order;        // level j <- caller's component order[j]
  std::vector<int> orig_first;   // caller's component c starts at orig_first[c] in the flat input
  std::vector<int> level_point;  // global point index (level order) -> flat input index
  std::vector<uint16_t> last_pairs;
  std::vector<uint16_t> prev_pairs;  // component K-2's pairs (the 3-D leaf stage)
  int path = 0;                  // 0: int64, 1: int128
  double bound_bits = 0;
  bool zero = false;             // some component has fewer than two distinct points
};

uint64_t choose2(uint64_t n) { return n * (n - 1) / 2; }

int prepare(const int64_t* pts, const int32_t* counts, int k, bool force128, double lift_span, int prefix_levels,
            int leaf3, MixedPrep& mp) {
  if (!pts || !counts) return bd::set_error(BD_ERR_ARG, "NULL argument");
  if (k < 1 || k > BD_KMAX) return bd::set_error(BD_ERR_ARG, "need 1 <= k <= BD_KMAX");
  int n = 0;
  for (int c = 0; c < k; ++c) {
    if (counts[c] < 1) return bd::set_error(BD_ERR_ARG, "every component needs at least one point");
    n += counts[c];
  }
  if (n > BD_NMAX) return bd::set_error(BD_ERR_ARG, "more than BD_NMAX points in all components");
  for (int i = 0; i < n * k; ++i)
    if (pts[i] >= (int64_t(1) << 40) || pts[i] <= -(int64_t(1) << 40))
      return bd::set_error(BD_ERR_ARG, "coordinates must stay below 2^40 in magnitude");
  mp.orig_first.assign(k + 1, 0);
  for (int c = 0; c < k; ++c) mp.orig_first[c + 1] = mp.orig_first[c] + counts[c];
  // a component whose points all coincide has no nonsingular pair: MV = 0
  for (int c = 0; c < k; ++c) {
    bool spread = false;
    for (int a = mp.orig_first[c] + 1; a < mp.orig_first[c + 1] && !spread; ++a)
      for (int e = 0; e < k; ++e) spread |= pts[a * k + e] != pts[mp.orig_first[c] * k + e];
    if (!spread) mp.zero = true;
  }
  // level order: fewest pairs first, so the tree is narrow at the top and the last level,
  // whose pairs are dealt to lanes, is the widest
  mp.order.resize(k);
  std::iota(mp.order.begin(), mp.order.end(), 0);
  std::stable_sort(mp.order.begin(), mp.order.end(), [&](int a, int b) { return counts[a] < counts[b]; });
  bd::MixedShape& s = mp.shape;
  s.K = k;
  s.N = n;
  s.first[0] = 0;
  mp.level_point.clear();
  for (int j = 0; j < k; ++j) {
    const int c = mp.order[j];
    s.first[j + 1] = s.first[j] + counts[c];
    s.npairs[j] = (uint32_t)choose2((uint64_t)counts[c]);
    for (int a = 0; a < counts[c]; ++a) mp.level_point.push_back(mp.orig_first[c] + a);
  }
  double lg = 0;
  for (int j = 0; j < k; ++j) lg += std::log2((double)std::max<uint32_t>(s.npairs[j], 1));
  if (lg > 62) return bd::set_error(BD_ERR_ARG, "more than 2^62 tuples of pairs");
  s.below[k] = 1;
  for (int j = k - 1; j >= 0; --j) s.below[j] = s.below[j + 1] * s.npairs[j];
  // Hadamard bound.  Every row of a minor is a pair difference within one component (the
  // point rows are taken relative to the component's first point), so with m_j the largest
  // pair distance of component j and W the largest lift difference within a component (with
  // a factor 2 of margin), a K x K coordinate minor
  // is at most prod_j m_j * max m / min m, a minor with the lift column at most K W times the
  // (K-1)-minors, and the leaf test forms 4 * (coordinate minor) * (lift minor).
  std::vector<double> m(k, 1.0);
  for (int j = 0; j < k; ++j) {
    const int c = mp.order[j];
    double best = 0;
    for (int a = mp.orig_first[c]; a < mp.orig_first[c + 1]; ++a)
      for (int b = a + 1; b < mp.orig_first[c + 1]; ++b) {
        double d2 = 0;
        for (int e = 0; e < k; ++e) {
          const double d = (double)(pts[b * k + e] - pts[a * k + e]);
          d2 += d * d;
        }
        best = std::max(best, std::sqrt(d2));
      }
    m[j] = std::max(best, 1.0);
  }
  const double mx = *std::max_element(m.begin(), m.end()), mn = *std::min_element(m.begin(), m.end());
  double lgc = std::log2(mx / mn);
  for (double v : m) lgc += std::log2(v);
  const double lgw = std::log2(2.0 * lift_span * k) + lgc - std::log2(mn);
  mp.bound_bits = 2 + lgc + lgw;
  mp.path = (force128 || mp.bound_bits >= 62.99) ? 1 : 0;
  if (mp.bound_bits >= 126.99) return bd::set_error(BD_ERR_OVERFLOW, "the exact minors may leave 128 bits");
  // the 3-D leaf stage (64-bit path) when the nodes above it are enough to spread the work
  double nodes3 = 1;
  for (int j = 0; j + 2 < k; ++j) nodes3 *= s.npairs[j];
  s.leaf3 = (mp.path == 0 && k >= 3 && (leaf3 > 0 || (leaf3 < 0 && nodes3 >= 1024))) ? 1 : 0;
  // items: fix levels until there are enough subtrees to spread over the GPU
  const int deepest = s.leaf3 ? k - 2 : k - 1;
  s.prefix = 0;
  s.items = 1;
  const int want = prefix_levels > 0 ? std::min(prefix_levels, deepest) : deepest;
  while (s.prefix < want && (prefix_levels > 0 || s.items < (1u << 17))) s.items *= s.npairs[s.prefix++];
  auto pairs_of = [&](int j, std::vector<uint16_t>& out) {
    out.clear();
    const int n = s.first[j + 1] - s.first[j];
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) out.push_back((uint16_t)((s.first[j] + p) | ((s.first[j] + q) << 8)));
  };
  pairs_of(k - 1, mp.last_pairs);
  if (k >= 2) pairs_of(k - 2, mp.prev_pairs);
  else mp.prev_pairs.clear();
  return BD_OK;
}

// rows in level order for the given flat lifts: P[c * N + g], relative to the component base
template <class T> void make_rows(const int64_t* pts, const int64_t* lifts, const MixedPrep& mp, std::vector<T>& P) {
  const int K = mp.shape.K, N = mp.shape.N;
  P.assign((size_t)(K + 1) * N, T(0));
  for (int j = 0; j < K; ++j) {
    const int base = mp.level_point[mp.shape.first[j]];
    for (int g = mp.shape.first[j]; g < mp.shape.first[j + 1]; ++g) {
      const int a = mp.level_point[g];
      for (int e = 0; e < K; ++e) P[(size_t)e * N + g] = T(pts[a * K + e] - pts[base * K + e]);
      P[(size_t)K * N + g] = T(lifts[a] - lifts[base]);
    }
  }
}

size_t smem_bytes(const MixedPrep& mp, int elem, int warps) {
  const int K = mp.shape.K, N = mp.shape.N;
  size_t b = (size_t)(K + 1) * N * elem;                                  // rows
  b += sizeof(bd::MixedShape);
  b += (mp.last_pairs.size() * sizeof(uint16_t) + 15) / 16 * 16;          // last level's pairs
  b += (mp.prev_pairs.size() * sizeof(uint16_t) + 15) / 16 * 16;          // level K-2's pairs
  b = (b + 15) / 16 * 16;
  const size_t per_warp = sizeof(bd::MixedUniform<i128>) + 32 * (size_t)N + (size_t)bd::mixed_stack_entries(K) * N * elem;
  return b + warps * ((per_warp + 15) / 16 * 16);
}

struct MixedDevAcc {
  unsigned long long mv_lo, mv_hi, cells, singular, ties;
};

template <class T>
__global__ void __launch_bounds__(32 * kMixedMaxWarps) k_mixed(const T* rows, bd::MixedShape shape,
                                                            const uint16_t* last_pairs, const uint16_t* prev_pairs,
                                                            unsigned long long* next,
                                                            unsigned long long chunk, bd::MixedSink sink,
                                                            MixedDevAcc* out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int K = shape.K, N = shape.N;
  T* P = reinterpret_cast<T*>(smem);
  size_t at = (size_t)(K + 1) * N * sizeof(T);
  bd::MixedShape* sh = reinterpret_cast<bd::MixedShape*>(smem + at);
  at += sizeof(bd::MixedShape);
  uint16_t* lp = reinterpret_cast<uint16_t*>(smem + at);
  const uint32_t npl = shape.npairs[K - 1], npp = K >= 2 ? shape.npairs[K - 2] : 0;
  at += ((size_t)npl * sizeof(uint16_t) + 15) / 16 * 16;
  uint16_t* pp = reinterpret_cast<uint16_t*>(smem + at);
  at += ((size_t)npp * sizeof(uint16_t) + 15) / 16 * 16;
  at = (at + 15) / 16 * 16;
  const size_t stack_bytes = (size_t)bd::mixed_stack_entries(K) * N * sizeof(T);
  const size_t per_warp = ((sizeof(bd::MixedUniform<i128>) + 32 * (size_t)N + stack_bytes) + 15) / 16 * 16;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* wbase = smem + at + warp * per_warp;
  auto* uni = reinterpret_cast<bd::MixedUniform<T>*>(wbase);
  float* fl = reinterpret_cast<float*>(wbase + sizeof(bd::MixedUniform<i128>));  // 16-byte aligned
  T* stack = reinterpret_cast<T*>(wbase + sizeof(bd::MixedUniform<i128>) + 32 * (size_t)N);
  for (int i = threadIdx.x; i < (K + 1) * N; i += blockDim.x) P[i] = rows[i];
  for (uint32_t i = threadIdx.x; i < npl; i += blockDim.x) lp[i] = last_pairs[i];
  for (uint32_t i = threadIdx.x; i < npp; i += blockDim.x) pp[i] = prev_pairs[i];
  if (threadIdx.x == 0) *sh = shape;
  __syncthreads();

  MixedWarp tm;
  bd::MixedWalker<T, MixedWarp> W(tm, P, sh, stack, fl, uni, lp, pp);
  W.sink = sink;
  bd::MixedAcc acc{};
  for (;;) {
    unsigned long long start = 0;
    if (lane == 0) start = atomicAdd(next, chunk);
    start = __shfl_sync(0xffffffffu, start, 0);
    if (start >= shape.items) break;
    const unsigned long long end = min(start + chunk, (unsigned long long)shape.items);
    for (unsigned long long it = start; it < end; ++it) W.run_item(it, acc);
  }
  // warp sum, then one set of atomics per warp
  unsigned long long lo = (uint64_t)acc.mv, hi = (uint64_t)(acc.mv >> 64);
  unsigned long long c = acc.cells, s = acc.singular, t = acc.ties;
  for (int o = 16; o; o >>= 1) {
    const unsigned long long lo2 = __shfl_xor_sync(0xffffffffu, lo, o), hi2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const unsigned long long nl = lo + lo2;
    hi += hi2 + (nl < lo ? 1ull : 0ull);
    lo = nl;
    c += __shfl_xor_sync(0xffffffffu, c, o);
    s += __shfl_xor_sync(0xffffffffu, s, o);
    t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  if (lane == 0) {
    const unsigned long long old = atomicAdd(&out->mv_lo, lo);
    const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
    if (hi + carry) atomicAdd(&out->mv_hi, hi + carry);
    if (c) atomicAdd(&out->cells, c);
    if (s) atomicAdd(&out->singular, s);
    if (t) atomicAdd(&out->ties, t);
  }
}

struct RunResult {
  u128 mv = 0;
  uint64_t cells = 0, singular = 0, ties = 0;
  double ms = 0;
  std::vector<bd::MixedCellRec> recs;
};

// One lifting on the GPU.  cap: records to keep (0: none).
template <class T>
int device_run(const MixedPrep& mp, const std::vector<T>& rows, uint64_t cap, RunResult& rr) {
  cudaStream_t st = bd::thread_stream();
  int dev = 0, sms = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);  // no device: a CUDA error, never a host fallback
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return bd::cuda_error(e);
  if (smem_bytes(mp, sizeof(T), 1) > (size_t)optin)
    return bd::set_error(BD_ERR_ARG, "the problem's walk state exceeds shared memory");
  e = cudaFuncSetAttribute(k_mixed<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  // warps per block: the most resident warps per SM (the walk state is per warp, so the
  // block size decides how much of the shared memory is left unused)
  int wpb = 1, per_sm = 0, best = 0;
  for (int w = 1; w <= kMixedMaxWarps && e == cudaSuccess; ++w) {
    const size_t sm_w = smem_bytes(mp, sizeof(T), w);
    if (sm_w > (size_t)optin) break;
    int b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_mixed<T>, 32 * w, sm_w);
    if (b * w > best) {
      best = b * w;
      wpb = w;
      per_sm = b;
    }
  }
  if (e != cudaSuccess) return bd::cuda_error(e);
  per_sm = std::max(per_sm, 1);
  const size_t smem = smem_bytes(mp, sizeof(T), wpb);
  const unsigned long long items = mp.shape.items;
  const unsigned long long warps = (unsigned long long)sms * per_sm * wpb;
  const unsigned long long blocks = std::min<unsigned long long>((unsigned long long)sms * per_sm,
                                                                 (items + wpb - 1) / wpb);
  // runs of consecutive items share their prefix levels, which a warp builds once
  const unsigned long long chunk = std::max<unsigned long long>(1, items / (warps * 8));
  T* d_rows = nullptr;
  uint16_t* d_lp = nullptr;
  uint16_t* d_pp = nullptr;
  unsigned long long* d_next = nullptr;
  MixedDevAcc* d_acc = nullptr;
  bd::MixedCellRec* d_recs = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto release = [&]() {
    cudaFree(d_rows);
    cudaFree(d_lp);
    cudaFree(d_pp);
    cudaFree(d_next);
    cudaFree(d_acc);
    cudaFree(d_recs);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  e = bd::dev_malloc(&d_rows, sizeof(T) * rows.size());
  if (e == cudaSuccess) e = bd::dev_malloc(&d_lp, sizeof(uint16_t) * std::max<size_t>(mp.last_pairs.size(), 1));
  if (e == cudaSuccess) e = bd::dev_malloc(&d_pp, sizeof(uint16_t) * std::max<size_t>(mp.prev_pairs.size(), 1));
  if (e == cudaSuccess) e = bd::dev_malloc(&d_next, sizeof(unsigned long long) * 2);
  if (e == cudaSuccess) e = bd::dev_malloc(&d_acc, sizeof(MixedDevAcc));
  if (e == cudaSuccess && cap) e = bd::dev_malloc(&d_recs, sizeof(bd::MixedCellRec) * cap);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_rows, rows.data(), sizeof(T) * rows.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !mp.last_pairs.empty())
    e = cudaMemcpyAsync(d_lp, mp.last_pairs.data(), sizeof(uint16_t) * mp.last_pairs.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !mp.prev_pairs.empty())
    e = cudaMemcpyAsync(d_pp, mp.prev_pairs.data(), sizeof(uint16_t) * mp.prev_pairs.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_next, 0, sizeof(unsigned long long) * 2, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_acc, 0, sizeof(MixedDevAcc), st);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    bd::MixedSink sink{d_recs, d_next + 1, cap};
    k_mixed<T><<<(unsigned int)blocks, 32 * wpb, smem, st>>>(d_rows, mp.shape, d_lp, d_pp, d_next, chunk, sink,
                                                                       d_acc);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  MixedDevAcc h{};
  unsigned long long nrec = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_acc, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nrec, d_next + 1, sizeof(nrec), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && cap) {
    rr.recs.resize((size_t)std::min<unsigned long long>(nrec, cap));
    if (!rr.recs.empty())
      e = cudaMemcpy(rr.recs.data(), d_recs, sizeof(bd::MixedCellRec) * rr.recs.size(), cudaMemcpyDeviceToHost);
  }
  float ms = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  release();
  if (e != cudaSuccess) return bd::cuda_error(e);
  rr.mv = ((u128)h.mv_hi << 64) | h.mv_lo;
  rr.cells = h.cells;
  rr.singular = h.singular;
  rr.ties = h.ties;
  rr.ms = ms;
  return BD_OK;
}

// One lifting on the host: the same walker, one-lane teams on `threads` threads (items taken
// in turn), or one lockstep team of `width` lane threads.
template <class T>
int host_run(const MixedPrep& mp, const std::vector<T>& rows, uint64_t cap, int width, RunResult& rr) {
  const int K = mp.shape.K, N = mp.shape.N;
  const size_t entries = (size_t)std::max(bd::mixed_stack_entries(K), 1) * N;
  std::vector<bd::MixedCellRec> recs((size_t)cap);
  unsigned long long nrec = 0;
  bd::MixedSink sink{cap ? recs.data() : nullptr, &nrec, cap};
  std::vector<bd::MixedAcc> part;
  if (width > 1) {
    bd::LockstepShared shl(width);
    std::vector<T> stack(entries);
    std::vector<float> fl(8 * (size_t)N);
    bd::MixedUniform<T> uni{};
    part.assign(width, bd::MixedAcc{});
    std::vector<std::thread> th;
    for (int l = 0; l < width; ++l)
      th.emplace_back([&, l] {
        bd::LockstepTeam tm{&shl, l};
        bd::MixedWalker<T, bd::LockstepTeam> W(tm, rows.data(), &mp.shape, stack.data(), fl.data(), &uni,
                                               mp.last_pairs.data(), mp.prev_pairs.data());
        W.sink = sink;
        for (uint64_t it = 0; it < mp.shape.items; ++it) W.run_item(it, part[l]);
      });
    for (auto& t : th) t.join();
  } else {
    const int nt = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    part.assign(nt, bd::MixedAcc{});
    std::atomic<uint64_t> next(0);
    auto work = [&](int w) {
      std::vector<T> stack(entries);
      std::vector<float> fl(8 * (size_t)N);
      bd::MixedUniform<T> uni{};
      bd::HostTeam tm;
      bd::MixedWalker<T, bd::HostTeam> W(tm, rows.data(), &mp.shape, stack.data(), fl.data(), &uni,
                                         mp.last_pairs.data(), mp.prev_pairs.data());
      W.sink = sink;
      for (;;) {
        const uint64_t it = next.fetch_add(1);
        if (it >= mp.shape.items) break;
        W.run_item(it, part[w]);
      }
    };
    std::vector<std::thread> th;
    for (int w = 1; w < nt; ++w) th.emplace_back(work, w);
    work(0);
    for (auto& t : th) t.join();
  }
  for (const auto& a : part) {
    rr.mv += a.mv;
    rr.cells += a.cells;
    rr.singular += a.singular;
    rr.ties += a.ties;
  }
  recs.resize((size_t)std::min<unsigned long long>(nrec, cap));
  rr.recs = std::move(recs);
  return BD_OK;
}

template <class T>
int run_lifting(const int64_t* pts, const int64_t* lifts, const MixedPrep& mp, uint64_t cap, int host_width,
                RunResult& rr) {
  std::vector<T> rows;
  make_rows<T>(pts, lifts, mp, rows);
  return host_width > 0 ? host_run<T>(mp, rows, cap, host_width, rr) : device_run<T>(mp, rows, cap, rr);
}

void fill_out(const MixedPrep& mp, const RunResult& rr, int relifts, bd_mixed_out* out) {
  out->mv_lo = (uint64_t)rr.mv;
  out->mv_hi = (uint64_t)(rr.mv >> 64);
  out->cells = rr.cells;
  out->singular = rr.singular;
  out->ties = rr.ties;
  out->tuples = mp.shape.below[0];
  out->relifts = relifts;
  out->flags = mp.path == 1 ? BD_FLAG_INT128 : 0;
  out->bound_bits = (int32_t)std::ceil(mp.bound_bits);
  out->device_ms = rr.ms;
}

// cells back in the caller's component order, as local indices
int write_cells(const MixedPrep& mp, const RunResult& rr, int k, int32_t* cells, int64_t capacity, int64_t* absdet) {
  if (!cells) return BD_OK;
  if ((int64_t)rr.cells > capacity)
    return bd::set_error(BD_ERR_ARG, "capacity is below the number of cells (out->cells holds it)");
  std::vector<size_t> ord(rr.recs.size());
  std::iota(ord.begin(), ord.end(), 0);
  std::vector<std::vector<int32_t>> rows(rr.recs.size(), std::vector<int32_t>(2 * k));
  for (size_t r = 0; r < rr.recs.size(); ++r)
    for (int j = 0; j < k; ++j) {
      const int c = mp.order[j];
      const int p = mp.level_point[rr.recs[r].idx[2 * j]] - mp.orig_first[c];
      const int q = mp.level_point[rr.recs[r].idx[2 * j + 1]] - mp.orig_first[c];
      rows[r][2 * c] = std::min(p, q);
      rows[r][2 * c + 1] = std::max(p, q);
    }
  std::sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return rows[a] < rows[b]; });
  for (size_t i = 0; i < ord.size(); ++i) {
    std::memcpy(cells + i * 2 * k, rows[ord[i]].data(), sizeof(int32_t) * 2 * k);
    if (absdet) absdet[i] = rr.recs[ord[i]].absdet;
  }
  return BD_OK;
}

int mixed_common(const int64_t* pts, const int32_t* counts, int32_t k, const int64_t* given_lifts, uint64_t seed,
                 int host_width, int force128, int prefix_levels, int leaf3, bd_mixed_out* out, int32_t* cells,
                 int64_t capacity, int64_t* absdet) {
  if (!out) return bd::set_error(BD_ERR_ARG, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  if (cells && capacity < 0) return bd::set_error(BD_ERR_ARG, "negative capacity");
  // the largest lift difference within a component: 2^20 for generated lifts
  double span = (double)(1 << 20);
  if (given_lifts && counts && k >= 1 && k <= BD_KMAX) {
    span = 1;
    int at = 0;
    for (int c = 0; c < k; ++c) {
      if (counts[c] < 1 || at + counts[c] > BD_NMAX) break;
      const auto mm = std::minmax_element(given_lifts + at, given_lifts + at + counts[c]);
      span = std::max(span, (double)*mm.second - (double)*mm.first);
      at += counts[c];
    }
  }
  MixedPrep mp;
  int rc = prepare(pts, counts, k, force128 != 0, span, prefix_levels, leaf3, mp);
  if (rc) return rc;
  if (mp.zero) {
    out->tuples = mp.shape.below[0];
    out->singular = out->tuples;
    out->flags = BD_FLAG_DEGENERATE;
    return BD_OK;
  }
  const int n = mp.shape.N;
  const uint64_t cap = cells ? (uint64_t)capacity : 0;
  std::vector<int64_t> lifts(n);
  const int attempts = given_lifts ? 1 : 8;
  RunResult rr;
  for (int a = 0; a < attempts; ++a) {
    if (given_lifts) {
      for (int i = 0; i < n; ++i) {
        if (given_lifts[i] >= (int64_t(1) << 40) || given_lifts[i] <= -(int64_t(1) << 40))
          return bd::set_error(BD_ERR_ARG, "lifts must stay below 2^40 in magnitude");
        lifts[i] = given_lifts[i];
      }
    } else {
      const uint64_t ss = bd::lift_stream_seed(seed, (uint32_t)a);
      for (int i = 0; i < n; ++i) lifts[i] = bd::lift_height(ss, i);
    }
    rr = RunResult{};
    rc = mp.path == 0 ? run_lifting<int64_t>(pts, lifts.data(), mp, cap, host_width, rr)
                      : run_lifting<i128>(pts, lifts.data(), mp, cap, host_width, rr);
    if (rc) return rc;
    fill_out(mp, rr, a, out);
    if (rr.ties == 0) return write_cells(mp, rr, k, cells, capacity, absdet);
  }
  return bd::set_error(BD_ERR_TIES, given_lifts ? "the given lifting has a tie" : "every lifting had a tie");
}

}  // namespace

extern "C" {

int bd_mixed_volume(const int64_t* points, const int32_t* counts, int32_t k, uint64_t seed, bd_mixed_out* out) {
  return mixed_common(points, counts, k, nullptr, seed, 0, 0, 0, -1, out, nullptr, 0, nullptr);
}

int bd_mixed_volume_lifted(const int64_t* points, const int32_t* counts, int32_t k, const int64_t* lifts,
                           int32_t force_int128, bd_mixed_out* out, int32_t* cells, int64_t capacity,
                           int64_t* absdet) {
  if (!lifts) return bd::set_error(BD_ERR_ARG, "NULL argument");
  return mixed_common(points, counts, k, lifts, 0, 0, force_int128, 0, -1, out, cells, capacity, absdet);
}

int bd_host_mixed_volume_lifted(const int64_t* points, const int32_t* counts, int32_t k, const int64_t* lifts,
                                int32_t team_width, int32_t force_int128, int32_t prefix_levels, int32_t leaf3,
                                bd_mixed_out* out, int32_t* cells, int64_t capacity, int64_t* absdet) {
  if (!lifts) return bd::set_error(BD_ERR_ARG, "NULL argument");
  if (team_width < 1 || team_width > 32) return bd::set_error(BD_ERR_ARG, "team width must be 1..32");
  if (prefix_levels < 0) return bd::set_error(BD_ERR_ARG, "negative prefix_levels");
  return mixed_common(points, counts, k, lifts, 0, team_width, force_int128, prefix_levels, leaf3 < 0 ? -1 : leaf3,
                      out, cells, capacity, absdet);
}

}  // extern "C"

// CUDA kernels of the lower-facet enumeration (sm_103a).
//
// k_enumerate is persistent: every warp repeatedly takes the next work item (a subset prefix,
// largest first) from a global counter and walks all (K+1)-subsets below it with the exact
// level-by-level Bareiss state of bd_core.cuh.  The lifted points sit in shared memory
// (column-major, one int64 per coordinate); each warp has its own stack of reduced rows in
// shared memory, laid out [level entry][point] so that lane l touches consecutive 8-byte
// (16-byte for the wide path) words and a pivot row is a broadcast read.  Per-warp results
// stay in registers and are added once to the global accumulators at the end (128-bit sum
// by two 64-bit atomics with carry).
#include "bd_kernels.cuh"
#include "bd_lifts.h"

namespace bd {

namespace {

struct WarpTeam {
  BD_HD int lane() const {
#ifdef __CUDA_ARCH__
    return threadIdx.x & 31;
#else
    return 0;
#endif
  }
  BD_HD int lanes() const { return 32; }
  BD_HD bool any(bool b) const {
#ifdef __CUDA_ARCH__
    return __any_sync(0xffffffffu, b);
#else
    return b;
#endif
  }
  BD_HD void sync() const {
#ifdef __CUDA_ARCH__
    __syncwarp();
#endif
  }
  BD_HD bool all(bool b) const {
#ifdef __CUDA_ARCH__
    return __all_sync(0xffffffffu, b);
#else
    return b;
#endif
  }
  BD_HD uint64_t ballot(bool b) const {  // bit l: lane l's vote
#ifdef __CUDA_ARCH__
    return (uint64_t)__ballot_sync(0xffffffffu, b);
#else
    return b ? 1ull : 0ull;
#endif
  }
  BD_HD uint32_t max_u32(uint32_t x) const {
#ifdef __CUDA_ARCH__
    return __reduce_max_sync(0xffffffffu, x);
#else
    return x;
#endif
  }
  BD_HD uint64_t or_all(uint64_t x) const {
#ifdef __CUDA_ARCH__
    const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)x);
    const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(x >> 32));
    return ((uint64_t)hi << 32) | lo;
#else
    return x;
#endif
  }
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
// point slots of a warp stack: N rounded up to 4 (rows stay 16-byte aligned for every entry
// type; lane l owns points l and l + 32 whatever the stride)
__host__ __device__ inline int slots_of(int N) { return (N + 3) & ~3; }

// at most 256 threads per block and at least 2 resident blocks: up to 128 registers per thread
#ifndef BD_LB_BLOCKS
#define BD_LB_BLOCKS 2
#endif
#define BD_ENUM_BOUNDS __launch_bounds__(256, BD_LB_BLOCKS)

// one warp's shared memory: its coordinate-minor stack, lift-minor stack, eight floats per
// point for the single-precision filters and the walker's team-shared state (pivots, dividers,
// prefix sets, the 5-D queue), each 16-byte aligned
template <class TC, class TL>
__host__ __device__ inline size_t warp_bytes(int slots, int K) {
  return align16((size_t)slots * stack_entries(K) * sizeof(TC)) + align16((size_t)slots * K * sizeof(TL)) +
         align16((size_t)8 * slots * sizeof(float)) + kUniformBytes;
}

// the uniform-state area of a warp region laid out as in warp_bytes, given its float rows
__device__ inline void* uniform_after(float* fl, int slots) {
  return reinterpret_cast<unsigned char*>(fl) + align16((size_t)8 * slots * sizeof(float));
}

// The shared accumulators of the 5-D stage in a warp's uniform area (the walker of a Stage 5
// kernel adds accepted cells, their |D0| and ties there): cleared before the warp's first
// item, added into lane 0's accumulator and cleared again where the kernel flushes.
template <class TC>
__device__ void rare_clear(void* uni) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) {
    unsigned long long* r = static_cast<Uniform<TC>*>(uni)->rare;
    r[0] = r[1] = r[2] = r[3] = 0;
  }
  __syncwarp();
}
template <class TC>
__device__ void rare_fold(void* uni, Acc& acc) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) {
    const unsigned long long* r = static_cast<Uniform<TC>*>(uni)->rare;
    acc.nvol += ((u128)r[1] << 64) | (u128)r[0];
    acc.cells += r[2];
    acc.ties += r[3];
  }
  rare_clear<TC>(uni);
}

template <class TC, class TL>
struct WarpMem {
  TC* sc;
  TL* sl;
  float* fl;
  void* uni;
  __device__ WarpMem(unsigned char* smem, int N, int K, int slots, int warp) {
    unsigned char* b = smem + align16((size_t)(K + 1) * N * sizeof(int64_t)) + (size_t)warp * warp_bytes<TC, TL>(slots, K);
    sc = reinterpret_cast<TC*>(b);
    b += align16((size_t)slots * stack_entries(K) * sizeof(TC));
    sl = reinterpret_cast<TL*>(b);
    b += align16((size_t)slots * K * sizeof(TL));
    fl = reinterpret_cast<float*>(b);
    uni = uniform_after(fl, slots);
  }
};

__device__ void load_points(int64_t* P, const EnumParams& p) {
  const int N = p.N, K = p.K;
  for (int i = threadIdx.x; i < N * K; i += blockDim.x) {
    const int q = i / K, c = i - q * K;
    P[c * N + q] = p.pts[i];
  }
  for (int q = threadIdx.x; q < N; q += blockDim.x)
    P[K * N + q] = p.lifts ? p.lifts[q] : lift_height(p.lift_seed, q);
  __syncthreads();
}

// sum of the lanes' accumulators, valid in lane 0
__device__ Acc warp_sum(Acc a) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long lo = __shfl_down_sync(0xffffffffu, (unsigned long long)(uint64_t)a.nvol, o);
    const unsigned long long hi = __shfl_down_sync(0xffffffffu, (unsigned long long)(uint64_t)(a.nvol >> 64), o);
    a.nvol += ((u128)hi << 64) | lo;
    a.cells += __shfl_down_sync(0xffffffffu, (unsigned long long)a.cells, o);
    a.singular += __shfl_down_sync(0xffffffffu, (unsigned long long)a.singular, o);
    a.ties += __shfl_down_sync(0xffffffffu, (unsigned long long)a.ties, o);
  }
  return a;
}

__device__ void flush(const Acc& a, DevAcc* g, unsigned long long items) {
  const unsigned long long lo = (unsigned long long)(uint64_t)a.nvol;
  const unsigned long long hi = (unsigned long long)(uint64_t)(a.nvol >> 64);
  const unsigned long long old = atomicAdd(&g->nvol_lo, lo);
  const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
  if (hi + carry) atomicAdd(&g->nvol_hi, hi + carry);
  if (a.cells) atomicAdd(&g->cells, (unsigned long long)a.cells);
  if (a.singular) atomicAdd(&g->singular, (unsigned long long)a.singular);
  if (a.ties) atomicAdd(&g->ties, (unsigned long long)a.ties);
  if (items) atomicAdd(&g->items_done, items);
}

// Stage: the walker's bottom stage (4 or 5; see Walker), one kernel each, so that neither carries
// the other's code
template <class TC, class TL, int Stage>
__global__ void BD_ENUM_BOUNDS k_enumerate(EnumParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  int64_t* P = reinterpret_cast<int64_t*>(smem);
  const int N = p.N, K = p.K;
  const int slots = slots_of(N);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpMem<TC, TL> m(smem, N, K, slots, warp);
  load_points(P, p);

  WarpTeam tm;
  Walker<TC, TL, WarpTeam, Stage> W(tm, P, N, K, slots, m.sc, m.sl, m.fl, m.uni);
  W.tri = p.tri;
  W.sink = p.sink;
  Acc acc{};
  if (Stage == 5) rare_clear<TC>(m.uni);
  unsigned long long done = 0;
  const unsigned int units = p.ranges ? (unsigned int)p.nranges : (unsigned int)p.nitems;
  const unsigned int shards = p.shards > 1 ? (unsigned int)p.shards : 1u;
  for (;;) {
    unsigned int u = 0;
    if (lane == 0) u = atomicAdd(p.counter, 1u);
    u = __shfl_sync(0xffffffffu, u, 0);
    u = u * shards + (unsigned int)p.shard;  // this shard's units only
    if (u >= units) break;
    const Range r = p.ranges ? p.ranges[u] : Range{u, 1u};
    for (unsigned int i = r.first; i < r.first + r.count; ++i) {
      const PackedItem it = p.items[i];
      W.run_item(it, acc);
      ++done;
    }
  }
  if (Stage == 5) rare_fold<TC>(m.uni, acc);
  acc = warp_sum(acc);
  if (lane == 0) flush(acc, p.acc, done);
}

template <class TC, class TL>
__global__ void k_classify(const int64_t* pts, const int64_t* lifts, int N, int K, const uint8_t* subsets,
                           int count, int32_t* status, int64_t* absdet) {
  extern __shared__ __align__(16) unsigned char smem[];
  int64_t* P = reinterpret_cast<int64_t*>(smem);
  EnumParams p{};
  p.pts = pts;
  p.lifts = lifts;
  p.N = N;
  p.K = K;
  load_points(P, p);
  const int slots = slots_of(N);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, warps = blockDim.x >> 5;
  WarpMem<TC, TL> m(smem, N, K, slots, warp);
  WarpTeam tm;
  Walker<TC, TL, WarpTeam, 4> W(tm, P, N, K, slots, m.sc, m.sl, m.fl, m.uni);
  for (int i = blockIdx.x * warps + warp; i < count; i += gridDim.x * warps) {
    TL ad = 0;
    const int s = W.classify(subsets + (size_t)i * (K + 1), ad);
    if (lane == 0) {
      status[i] = s;
      absdet[i] = (ad >> 63) != 0 ? -1 : (int64_t)ad;
    }
  }
}

template <class TC, class TL>
cudaError_t configure(int smem) {
  cudaError_t e = cudaFuncSetAttribute(k_enumerate<TC, TL, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if constexpr (sizeof(TC) == 4) {  // the 5-D stage exists on the 32-bit coordinate path only
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_enumerate<TC, TL, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  }
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_classify<TC, TL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

// The dynamic shared-memory ceiling of every kernel is raised once to the device's opt-in
// maximum, so that launch shapes computed (and cached) at different times never invalidate
// each other.
cudaError_t configure_path(int path, int /*smem*/) {
  int dev = 0, max_optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (path == PATH_NARROW) return configure<int32_t, int64_t>(max_optin);
  if (path == PATH_MID) return configure<int64_t, int64_t>(max_optin);
  return configure<i128, i128>(max_optin);
}

}  // namespace

size_t enum_smem_bytes(int N, int K, int warps, int path) {
  const size_t pts = align16((size_t)(K + 1) * N * sizeof(int64_t));
  const int slots = slots_of(N);
  const size_t per_warp = path == PATH_NARROW ? warp_bytes<int32_t, int64_t>(slots, K)
                          : path == PATH_MID  ? warp_bytes<int64_t, int64_t>(slots, K)
                                              : warp_bytes<i128, i128>(slots, K);
  return pts + per_warp * warps;
}

LaunchShape enum_shape(int N, int K, int path, bool five, int warps_req, int blocks_per_sm_req, int sms,
                       cudaError_t* err) {
  LaunchShape s;
  *err = cudaSuccess;
  int dev = 0, max_optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  int warps = warps_req > 0 ? warps_req : 4;
  while (warps > 1 && enum_smem_bytes(N, K, warps, path) > (size_t)max_optin) warps /= 2;
  s.warps = warps;
  s.smem = enum_smem_bytes(N, K, warps, path);
  s.slots = slots_of(N);
  if (s.smem > (size_t)max_optin) { *err = cudaErrorInvalidConfiguration; return s; }
  cudaError_t e = configure_path(path, (int)s.smem);
  if (e != cudaSuccess) { *err = e; return s; }
  int per_sm = blocks_per_sm_req;
  if (per_sm <= 0) {
    if (path == PATH_NARROW && five)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_enumerate<int32_t, int64_t, 5>, warps * 32, s.smem);
    else if (path == PATH_NARROW)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_enumerate<int32_t, int64_t, 4>, warps * 32, s.smem);
    else if (path == PATH_MID)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_enumerate<int64_t, int64_t, 4>, warps * 32, s.smem);
    else
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_enumerate<i128, i128, 4>, warps * 32, s.smem);
    if (e != cudaSuccess) { *err = e; return s; }
    if (per_sm < 1) per_sm = 1;
  }
  s.blocks = per_sm * sms;
  return s;
}

cudaError_t launch_enumerate(const EnumParams& p, const LaunchShape& s, int path, cudaStream_t st) {
  if (path == PATH_NARROW && p.five && p.K >= 4) k_enumerate<int32_t, int64_t, 5><<<s.blocks, s.warps * 32, s.smem, st>>>(p);
  else if (path == PATH_NARROW) k_enumerate<int32_t, int64_t, 4><<<s.blocks, s.warps * 32, s.smem, st>>>(p);
  else if (path == PATH_MID) k_enumerate<int64_t, int64_t, 4><<<s.blocks, s.warps * 32, s.smem, st>>>(p);
  else k_enumerate<i128, i128, 4><<<s.blocks, s.warps * 32, s.smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_classify(const int64_t* pts, const int64_t* lifts, int N, int K, const uint8_t* subsets,
                            int count, int32_t* status, int64_t* absdet, int path, cudaStream_t st) {
  const int warps = 4;
  const size_t smem = enum_smem_bytes(N, K, warps, path);
  cudaError_t e = configure_path(path, (int)smem);
  if (e != cudaSuccess) return e;
  int blocks = (count + warps - 1) / warps;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  if (path == PATH_NARROW)
    k_classify<int32_t, int64_t><<<blocks, warps * 32, smem, st>>>(pts, lifts, N, K, subsets, count, status, absdet);
  else if (path == PATH_MID)
    k_classify<int64_t, int64_t><<<blocks, warps * 32, smem, st>>>(pts, lifts, N, K, subsets, count, status, absdet);
  else
    k_classify<i128, i128><<<blocks, warps * 32, smem, st>>>(pts, lifts, N, K, subsets, count, status, absdet);
  return cudaGetLastError();
}

// ---- batches --------------------------------------------------------------------------------

namespace {

__device__ void flush_sys(const Acc& a, unsigned long long items, unsigned long long cyc, const BatchParams& p,
                          int sys) {
  flush(a, p.acc + sys, items);
  if (cyc) atomicAdd(p.cycles + sys, cyc);
  if (items) atomicAdd(p.done + sys, (unsigned int)items);
}

// Persistent: every warp takes the next (system, prefix) item; when the system changes it
// loads that system's lifted points into its own shared-memory buffer (so warps of one block
// may work on different systems) and flushes its accumulators for the previous one.
template <class TC, class TL, int Stage>
__global__ void BD_ENUM_BOUNDS k_batch(BatchParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slots = slots_of(p.maxN);
  const size_t pbytes = align16((size_t)(p.maxK + 1) * p.maxN * sizeof(int64_t));
  unsigned char* base = smem + (size_t)warp * (pbytes + warp_bytes<TC, TL>(slots, p.maxK));
  int64_t* P = reinterpret_cast<int64_t*>(base);
  TC* sc = reinterpret_cast<TC*>(base + pbytes);
  TL* sl = reinterpret_cast<TL*>(base + pbytes + align16((size_t)slots * stack_entries(p.maxK) * sizeof(TC)));
  float* fl = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(sl) + align16((size_t)slots * p.maxK * sizeof(TL)));
  WarpTeam tm;
  int cur = -1, N = 0, K = 0;
  Acc acc{};
  if (Stage == 5) rare_clear<TC>(uniform_after(fl, slots));
  unsigned long long items = 0, cyc = 0;
  for (;;) {
    unsigned int i = 0;
    if (lane == 0) i = atomicAdd(p.counter, 1u);
    i = __shfl_sync(0xffffffffu, i, 0);
    if (i >= (unsigned int)p.nitems) break;
    const BatchItem bi = p.items[i];
    if ((int)bi.sys != cur) {
      if (cur >= 0) {
        if (Stage == 5) rare_fold<TC>(uniform_after(fl, slots), acc);
        const Acc s = warp_sum(acc);
        if (lane == 0) flush_sys(s, items, cyc, p, cur);
      }
      acc = Acc{};
      items = cyc = 0;
      cur = (int)bi.sys;
      const BatchDesc d = p.desc[cur];
      N = d.N;
      K = d.K;
      __syncwarp();
      for (int t = lane; t < N * K; t += 32) {
        const int q = t / K, c = t - q * K;
        P[c * N + q] = p.pts[d.pts_off + t];
      }
      for (int q = lane; q < N; q += 32) P[K * N + q] = lift_height(d.lift_seed, q);
      __syncwarp();
    }
    Item it{};
    it.len = bi.len;
    for (int t = 0; t < bi.len; ++t) it.idx[t] = bi.idx[t];
    Walker<TC, TL, WarpTeam, Stage> W(tm, P, N, K, slots, sc, sl, fl, uniform_after(fl, slots));
    W.tri = p.tri;
    const long long t0 = clock64();
    W.run_item(it, acc);
    cyc += (unsigned long long)(clock64() - t0);
    ++items;
  }
  if (cur >= 0) {
    if (Stage == 5) rare_fold<TC>(uniform_after(fl, slots), acc);
    const Acc s = warp_sum(acc);
    if (lane == 0) flush_sys(s, items, cyc, p, cur);
  }
}

template <class TC, class TL, int Stage>
cudaError_t configure_batch() {
  int dev = 0, max_optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return cudaFuncSetAttribute(k_batch<TC, TL, Stage>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin);
}

}  // namespace

size_t batch_smem_bytes(int maxN, int maxK, int warps, int path) {
  const int slots = slots_of(maxN);
  const size_t pbytes = align16((size_t)(maxK + 1) * maxN * sizeof(int64_t));
  const size_t per_warp = path == PATH_NARROW ? warp_bytes<int32_t, int64_t>(slots, maxK)
                          : path == PATH_MID  ? warp_bytes<int64_t, int64_t>(slots, maxK)
                                              : warp_bytes<i128, i128>(slots, maxK);
  return (pbytes + per_warp) * warps;
}

LaunchShape batch_shape(int maxN, int maxK, int path, bool five, int warps_req, int blocks_per_sm_req, int sms,
                        cudaError_t* err) {
  LaunchShape s;
  *err = cudaSuccess;
  int dev = 0, max_optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  int warps = warps_req > 0 ? warps_req : 4;
  while (warps > 1 && batch_smem_bytes(maxN, maxK, warps, path) > (size_t)max_optin) warps /= 2;
  s.warps = warps;
  s.smem = batch_smem_bytes(maxN, maxK, warps, path);
  s.slots = slots_of(maxN);
  if (s.smem > (size_t)max_optin) { *err = cudaErrorInvalidConfiguration; return s; }
  cudaError_t e = path == PATH_NARROW && five ? configure_batch<int32_t, int64_t, 5>()
                  : path == PATH_NARROW       ? configure_batch<int32_t, int64_t, 4>()
                  : path == PATH_MID          ? configure_batch<int64_t, int64_t, 4>()
                                              : configure_batch<i128, i128, 4>();
  if (e != cudaSuccess) { *err = e; return s; }
  int per_sm = blocks_per_sm_req;
  if (per_sm <= 0) {
    if (path == PATH_NARROW && five)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<int32_t, int64_t, 5>, warps * 32, s.smem);
    else if (path == PATH_NARROW)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<int32_t, int64_t, 4>, warps * 32, s.smem);
    else if (path == PATH_MID)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<int64_t, int64_t, 4>, warps * 32, s.smem);
    else
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<i128, i128, 4>, warps * 32, s.smem);
    if (e != cudaSuccess) { *err = e; return s; }
    if (per_sm < 1) per_sm = 1;
  }
  s.blocks = per_sm * sms;
  return s;
}

cudaError_t launch_batch(const BatchParams& p, const LaunchShape& s, int path, bool five, cudaStream_t st) {
  if (path == PATH_NARROW && five) k_batch<int32_t, int64_t, 5><<<s.blocks, s.warps * 32, s.smem, st>>>(p);
  else if (path == PATH_NARROW) k_batch<int32_t, int64_t, 4><<<s.blocks, s.warps * 32, s.smem, st>>>(p);
  else if (path == PATH_MID) k_batch<int64_t, int64_t, 4><<<s.blocks, s.warps * 32, s.smem, st>>>(p);
  else k_batch<i128, i128, 4><<<s.blocks, s.warps * 32, s.smem, st>>>(p);
  return cudaGetLastError();
}

// ---- serving ---------------------------------------------------------------------------------

namespace {

// One item of a request with the walker of its integer path (32- or 64-bit coordinate minors),
// starting from the prefix levels the warp built for the same system (valid, lo, hi), which are
// updated for the next item.
template <class TC>
__device__ void serve_item(WarpTeam& tm, const int64_t* P, int N, int K, int slots, unsigned char* sc, int64_t* sl,
                           float* fl, const Item& it, Acc& acc, const uint32_t* tri, bool five, int& valid,
                           uint64_t& lo, uint64_t& hi) {
  Walker<TC, int64_t, WarpTeam> W(tm, P, N, K, slots, reinterpret_cast<TC*>(sc), sl, fl, uniform_after(fl, slots));
  W.tri = tri;
  W.use5 = five;
  W.valid = valid;
  W.s = Idx15{lo, hi};
  W.run_item(it, acc);
  valid = W.valid;
  lo = W.s.lo;
  hi = W.s.hi;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Persistent: every warp takes the next ticket by fetch-and-add (no retries, so claims do not
// contend however many warps wait) and waits, napping, until the host has published it.  The
// unpublished tickets are always the top ones, [tail, head); once nothing has been published for
// idle_ns, a waiting warp gives its ticket back when every later ticket has been given back
// (head == ticket + 1, by compare-and-swap) and exits, so an idle kernel leaves the GPU with
// head == tail and the next launch claims from there.  A given-back ticket published in the meantime
// is claimed again (head moved below it), never processed twice.  Consecutive items of one
// request (same slot, admission and lifting) keep the warp's points in shared memory and the
// walker's built prefix levels.
__global__ void BD_ENUM_BOUNDS k_serve(ServeParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slots = slots_of(p.maxN);
  const size_t pbytes = align16((size_t)(p.maxK + 1) * p.maxN * sizeof(int64_t));
  // each warp's region is laid out for the 64-bit coordinate path (the larger stack); the 32-bit
  // path uses the front of the same bytes
  unsigned char* base = smem + (size_t)warp * (pbytes + warp_bytes<int64_t, int64_t>(slots, p.maxK));
  int64_t* P = reinterpret_cast<int64_t*>(base);
  unsigned char* sc = base + pbytes;
  int64_t* sl = reinterpret_cast<int64_t*>(sc + align16((size_t)slots * stack_entries(p.maxK) * sizeof(int64_t)));
  float* fl = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(sl) + align16((size_t)slots * p.maxK * sizeof(int64_t)));
  WarpTeam tm;
  // the system whose points and prefix states this warp holds
  int cur_slot = -1, cur_gen = 0;
  uint64_t cur_seed = 0;
  int pv_valid = 0;
  uint64_t pv_lo = 0, pv_hi = 0;
  for (;;) {
    unsigned long long got = 0;
    int quit = 0;
    if (lane == 0) {
      got = atomicAdd(p.head, 1ull);
      unsigned nap = 128;
      unsigned long long seen = *p.tail, t_seen = globaltimer_ns();
      for (;;) {
        if (*(volatile unsigned long long*)p.fault_dev) {
          quit = 1;  // a publication wait ran out: every warp leaves and the host resets the ring
          break;
        }
        const unsigned long long tail = *p.tail;
        if (got < tail) break;
        if (*p.stop) {
          quit = 1;
          break;
        }
        // idle means no publication at all for idle_ns (not just this ticket's wait), so that
        // warps do not leave one by one while work still flows
        const unsigned long long now = globaltimer_ns();
        if (tail != seen) {
          seen = tail;
          t_seen = now;
        } else if (now - t_seen > p.idle_ns && atomicCAS(p.head, got + 1, got) == got + 1) {
          quit = 1;  // the ticket is given back
          break;
        }
        __nanosleep(nap);
        nap = nap < 8192 ? 2 * nap : nap;
      }
    }
    got = __shfl_sync(0xffffffffu, got, 0);
    quit = __shfl_sync(0xffffffffu, quit, 0);
    if (quit) break;
    __threadfence();  // the item and its slot were published before the tail
    {
      const unsigned long long tk = got;
      int lost = 0;
      // The item's publication stamp (written after the item, before the tail) confirms that the
      // ring position holds this ticket's item.  It is normally there already; the wait for it is
      // bounded, and when the bound runs out the warp records the ticket and leaves without
      // touching the item (the host fails its request and resets the ring).
      if (lane == 0) {
        const unsigned long long want = tk + 1;
        const volatile unsigned long long* sp = p.seq + (tk % p.ring_cap);
        if (*sp != want) {
          const unsigned long long t0 = globaltimer_ns();
          while (*sp != want) {
            if (globaltimer_ns() - t0 > p.wait_ns) {
              lost = 1;
              break;
            }
            __nanosleep(1000);
          }
        }
        if (lost && atomicCAS(p.fault_dev, 0ull, want) == 0ull) {
          *p.fault_host = want;
          __threadfence_system();
        }
      }
      lost = __shfl_sync(0xffffffffu, lost, 0);
      if (lost) break;
      __threadfence();
      const volatile unsigned int* rp = reinterpret_cast<const volatile unsigned int*>(p.ring + (tk % p.ring_cap));
      BatchItem bi;
      unsigned int* bw = reinterpret_cast<unsigned int*>(&bi);
      for (int t = 0; t < 4; ++t) bw[t] = rp[t];
      const int slot = (int)bi.sys;
      // a slot is reused for other systems and liftings: its descriptor and points are read past L1
      const unsigned long long* dw = reinterpret_cast<const unsigned long long*>(p.desc + slot);
      BatchDesc d;
      unsigned long long* dd = reinterpret_cast<unsigned long long*>(&d);
      for (int t = 0; t < (int)(sizeof(BatchDesc) / 8); ++t) dd[t] = __ldcg(dw + t);
      const int N = d.N, K = d.K;
      const bool same = slot == cur_slot && d.gen == cur_gen && d.lift_seed == cur_seed;
      if (!same) {
        __syncwarp();  // the previous system's readers are done
        for (int t = lane; t < N * K; t += 32) {
          const int q = t / K, c = t - q * K;
          P[c * N + q] = __ldcg(p.pts + (size_t)slot * BD_SERVE_PTS + t);
        }
        for (int q = lane; q < N; q += 32) P[K * N + q] = lift_height(d.lift_seed, q);
        __syncwarp();
        cur_slot = slot;
        cur_gen = d.gen;
        cur_seed = d.lift_seed;
        pv_valid = 0;
      }
      Item it{};
      it.len = bi.len;
      for (int t = 0; t < bi.len; ++t) it.idx[t] = bi.idx[t];
      Acc acc{};
      const long long t0 = clock64();
      if (d.path == PATH_NARROW)
        serve_item<int32_t>(tm, P, N, K, slots, sc, sl, fl, it, acc, p.tri, d.five != 0, pv_valid, pv_lo, pv_hi);
      else
        serve_item<int64_t>(tm, P, N, K, slots, sc, sl, fl, it, acc, p.tri, false, pv_valid, pv_lo, pv_hi);
      const unsigned long long cyc = (unsigned long long)(clock64() - t0);
      acc = warp_sum(acc);
      if (lane == 0) {
        flush(acc, p.acc + slot, 1);
        atomicAdd(p.cycles + slot, cyc);
        __threadfence();
        if (atomicSub(p.remaining + slot, 1u) == 1u) {  // the slot's last item: publish its completion
          __threadfence();
          // the slot's sums (every other item's atomics are done) into host-mapped memory, so
          // that the host reads the result without a copy
          const unsigned long long* a = reinterpret_cast<const unsigned long long*>(p.acc + slot);
          volatile unsigned long long* out = p.res + (size_t)slot * kServeResWords;
          for (int w = 0; w < (int)(sizeof(DevAcc) / 8); ++w) out[w] = __ldcg(a + w);
          out[sizeof(DevAcc) / 8] = __ldcg(p.cycles + slot);
          __threadfence_system();
          const unsigned long long i = atomicAdd(p.comp_count, 1ull);
          p.comp[i % p.comp_cap] = ((i + 1) << 32) | (unsigned long long)(unsigned)slot;
          __threadfence_system();
        }
      }
    }
  }
}

}  // namespace

size_t serve_smem_bytes(int maxN, int maxK, int warps) {
  const int slots = slots_of(maxN);
  return (align16((size_t)(maxK + 1) * maxN * sizeof(int64_t)) + warp_bytes<int64_t, int64_t>(slots, maxK)) * warps;
}

LaunchShape serve_shape(int maxN, int maxK, int warps_req, int blocks_per_sm_req, int sms, cudaError_t* err) {
  LaunchShape s;
  *err = cudaSuccess;
  int dev = 0, max_optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  int warps = warps_req > 0 ? warps_req : 4;
  while (warps > 1 && serve_smem_bytes(maxN, maxK, warps) > (size_t)max_optin) warps /= 2;
  s.warps = warps;
  s.smem = serve_smem_bytes(maxN, maxK, warps);
  s.slots = slots_of(maxN);
  cudaError_t e = cudaFuncSetAttribute(k_serve, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin);
  if (e != cudaSuccess) { *err = e; return s; }
  int per_sm = blocks_per_sm_req;
  if (per_sm <= 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_serve, warps * 32, s.smem);
    if (e != cudaSuccess) { *err = e; return s; }
    per_sm = per_sm > 2 ? per_sm - 1 : per_sm;  // leave room for other kernels (the side route, the cost model)
  }
  s.blocks = per_sm * sms;
  return s;
}

cudaError_t launch_serve(const ServeParams& p, const LaunchShape& s, cudaStream_t st) {
  k_serve<<<s.blocks, s.warps * 32, s.smem, st>>>(p);
  return cudaGetLastError();
}

// ---- cell normals ----------------------------------------------------------------------------

namespace {

__global__ void k_cell_normals(const int64_t* pts, const int64_t* lifts, uint64_t lift_seed, int N, int K,
                               const uint8_t* cells, unsigned long long count, int64_t* den, int64_t* alpha,
                               int64_t* beta, int32_t* status) {
  const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  int64_t lf[NMAX];
  for (int q = 0; q < N; ++q) lf[q] = lifts ? lifts[q] : lift_height(lift_seed, q);
  uint8_t idx[16];
  for (int t = 0; t < 16; ++t) idx[t] = cells[16 * i + t];
  int64_t d = 0;
  i128 b = 0;
  const bool ok = cell_normal_exact(pts, lf, K, idx, d, alpha + i * K, b);
  den[i] = ok ? d : 0;
  beta[2 * i] = (int64_t)(uint64_t)(u128)b;
  beta[2 * i + 1] = (int64_t)(b >> 64);
  status[i] = ok ? 0 : 1;
}

}  // namespace

cudaError_t launch_cell_normals(const int64_t* pts, const int64_t* lifts, uint64_t lift_seed, int N, int K,
                                const uint8_t* cells, unsigned long long count, int64_t* den, int64_t* alpha,
                                int64_t* beta, int32_t* status, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const unsigned int threads = 64;
  const unsigned long long blocks = (count + threads - 1) / threads;
  k_cell_normals<<<(unsigned int)blocks, threads, 0, st>>>(pts, lifts, lift_seed, N, K, cells, count, den, alpha,
                                                           beta, status);
  return cudaGetLastError();
}

}  // namespace bd

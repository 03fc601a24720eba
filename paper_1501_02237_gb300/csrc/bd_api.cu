// C ABI of libbinodeg.so (declarations and contracts in include/binodeg.h).
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <algorithm>
#include <vector>

#include "../../include/binodeg.h"
#include "bd_host.h"
#include "bd_internal.h"
#include "bd_kernels.cuh"
#include "bd_lifts.h"

using bd::i128;
using bd::u128;

namespace {

thread_local std::string g_err;
thread_local cudaStream_t g_stream = nullptr;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(e == cudaErrorMemoryAllocation ? BD_ERR_NOMEM : BD_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

// device allocations still to succeed before the injected failure (-1: none armed); armed by
// bd_inject_alloc_failure or, at load, by the environment variable BD_INJECT_ALLOC_FAILURE
std::atomic<long long> g_alloc_fail_after{[] {
  const char* v = std::getenv("BD_INJECT_ALLOC_FAILURE");
  return v && *v ? std::atoll(v) : -1ll;
}()};

#define BD_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

constexpr int MAX_LIFTINGS = 8;

int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

int check_points(const int64_t* points, int32_t npts, int32_t k) {
  if (!points) return fail(BD_ERR_ARG, "points is NULL");
  if (k < 1 || k > BD_KMAX) return fail(BD_ERR_ARG, "k must be in [1, BD_KMAX]");
  if (npts < 1 || npts > BD_NMAX) return fail(BD_ERR_ARG, "npts must be in [1, BD_NMAX]");
  for (int64_t i = 0; i < (int64_t)npts * k; ++i)
    if (points[i] >= ((int64_t)1 << 40) || points[i] <= -((int64_t)1 << 40))
      return fail(BD_ERR_ARG, "|coordinate| must be below 2^40");
  return BD_OK;
}

void set_u128(uint64_t& lo, uint64_t& hi, u128 v) {
  lo = (uint64_t)v;
  hi = (uint64_t)(v >> 64);
}

// Work lists depend only on (N, K, split size): built once per process and device, kept on the
// device and shared by every plan that needs them.
struct ItemList {
  std::vector<bd::Item> host;  // lexicographic order
  std::vector<bd::Range> ranges;
  bd::PackedItem* dev = nullptr;  // the same items, packed, on the device
  bd::Range* dev_ranges = nullptr;
};
std::mutex g_cache_mu;
std::map<std::tuple<int, int, int64_t, int64_t, int, int>, std::shared_ptr<ItemList>> g_items;
std::map<std::tuple<int, int, int, int, int, int, bool>, bd::LaunchShape> g_shapes;

int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}

int get_items(int N, int K, int64_t thr, int64_t teams, int depth, std::shared_ptr<ItemList>& out) {
  const auto key = std::make_tuple(N, K, thr, teams, current_device(), depth);
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto it = g_items.find(key);
  if (it != g_items.end()) {
    out = it->second;
    return BD_OK;
  }
  auto L = std::make_shared<ItemList>();
  bd::build_ranges(N, K, (uint64_t)thr, (uint64_t)teams, depth, L->host, L->ranges);
  std::vector<bd::PackedItem> packed(L->host.size());
  for (size_t i = 0; i < packed.size(); ++i) packed[i] = bd::pack_item(L->host[i]);
  cudaError_t e = bd::dev_malloc(&L->dev, sizeof(bd::PackedItem) * std::max<size_t>(1, L->host.size()));
  if (e == cudaSuccess) e = bd::dev_malloc(&L->dev_ranges, sizeof(bd::Range) * std::max<size_t>(1, L->ranges.size()));
  if (e == cudaSuccess && !L->host.empty())
    e = cudaMemcpy(L->dev, packed.data(), sizeof(bd::PackedItem) * packed.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !L->ranges.empty())
    e = cudaMemcpy(L->dev_ranges, L->ranges.data(), sizeof(bd::Range) * L->ranges.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {  // not cached: free what was allocated
    cudaFree(L->dev);
    cudaFree(L->dev_ranges);
    return cuda_fail(e, "work list upload");
  }
  g_items[key] = L;
  out = L;
  return BD_OK;
}

// the colex triple decode table, uploaded once per device
std::map<int, uint32_t*> g_tri;

int get_tri(const uint32_t*& out) {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto it = g_tri.find(dev);
  if (it != g_tri.end()) {
    out = it->second;
    return BD_OK;
  }
  std::vector<uint32_t> h(bd::kTriEntries);
  bd::fill_colex_table(h.data());
  uint32_t* d = nullptr;
  cudaError_t e = bd::dev_malloc(&d, sizeof(uint32_t) * h.size());
  if (e == cudaSuccess) e = cudaMemcpy(d, h.data(), sizeof(uint32_t) * h.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "decode table upload");
  g_tri[dev] = d;
  out = d;
  return BD_OK;
}

int get_shape(int N, int K, int path, bool five, int warps_req, int bps_req, bd::LaunchShape& out) {
  const auto key = std::make_tuple(N, K, path, warps_req, bps_req, current_device(), five);
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto it = g_shapes.find(key);
  if (it != g_shapes.end()) {
    out = it->second;
    return BD_OK;
  }
  cudaError_t e;
  out = bd::enum_shape(N, K, path, five, warps_req, bps_req, sm_count(), &e);
  if (e != cudaSuccess) return cuda_fail(e, "launch shape");
  g_shapes[key] = out;
  return BD_OK;
}

}  // namespace

namespace bd {
int set_error(int code, const char* msg) { return fail(code, msg); }
cudaStream_t thread_stream() { return g_stream; }
int device_tri_table(const uint32_t** out) { return get_tri(*out); }

cudaError_t dev_malloc_raw(void** p, size_t bytes) {
  long long n = g_alloc_fail_after.load();
  while (n >= 0 && !g_alloc_fail_after.compare_exchange_weak(n, n - 1)) {
  }
  if (n == 0) {  // the armed allocation: fail as the device would when out of memory
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation) cudaGetLastError();
  return e;
}

int cuda_error(cudaError_t e, const char* where) {
  const std::string msg = where ? std::string(where) + ": " + cudaGetErrorString(e) : std::string(cudaGetErrorString(e));
  return fail(e == cudaErrorMemoryAllocation ? BD_ERR_NOMEM : BD_ERR_CUDA, msg);
}
}  // namespace bd

// A plan owns small fixed-size device buffers (points of up to BD_NMAX x BD_KMAX coordinates,
// lifts, accumulators) and pinned host staging; it can be re-targeted at another point set
// without allocating, which is what the synchronous calls do through one plan per thread.
struct bd_plan {
  int N = 0, K = 0;
  int path = 0;  // bd::PATH_NARROW / MID / WIDE
  bool five = false;  // the walk's bottom stage is the 5-D test (32-bit coordinate path, k >= 4)
  double bound = 0;
  int64_t max_abs = 0;
  bool explicit_lifts = false;
  int device = -1;
  std::shared_ptr<ItemList> items;
  int64_t* d_pts = nullptr;          // BD_NMAX * BD_KMAX
  int64_t* d_lifts = nullptr;        // BD_NMAX
  unsigned char* d_state = nullptr;  // [DevAcc][counter]
  bd::DevAcc* h_acc = nullptr;       // pinned
  int64_t* h_stage = nullptr;        // pinned: points then lifts
  bd::LaunchShape shape;
  cudaStream_t stream = nullptr;
  bool launched = false;
  int attempt = 0;
  int shard = 0, shards = 1;  // of the last launch
  const uint32_t* tri = nullptr;  // the device's colex decode table
  uint64_t items_expected = 0;
};

namespace {

size_t state_bytes() { return sizeof(bd::DevAcc) + 16; }
constexpr size_t STAGE_WORDS = (size_t)BD_NMAX * BD_KMAX + BD_NMAX;

void plan_release(bd_plan* p) {
  cudaFree(p->d_pts);
  cudaFree(p->d_lifts);
  cudaFree(p->d_state);
  cudaFreeHost(p->h_acc);
  cudaFreeHost(p->h_stage);
  p->d_pts = p->d_lifts = nullptr;
  p->d_state = nullptr;
  p->h_acc = nullptr;
  p->h_stage = nullptr;
  p->device = -1;
}

void plan_free(bd_plan* p) {
  if (!p) return;
  plan_release(p);
  delete p;
}

int plan_alloc(bd_plan* p) {
  const int dev = current_device();
  if (p->device == dev) return BD_OK;
  if (p->device >= 0) plan_release(p);
  cudaError_t e = bd::dev_malloc(&p->d_pts, sizeof(int64_t) * BD_NMAX * BD_KMAX);
  if (e == cudaSuccess) e = bd::dev_malloc(&p->d_lifts, sizeof(int64_t) * BD_NMAX);
  if (e == cudaSuccess) e = bd::dev_malloc(&p->d_state, state_bytes());
  if (e == cudaSuccess) e = cudaMallocHost(&p->h_acc, sizeof(bd::DevAcc));
  if (e == cudaSuccess) e = cudaMallocHost(&p->h_stage, sizeof(int64_t) * STAGE_WORDS);
  if (e != cudaSuccess) {
    plan_release(p);
    return cuda_fail(e, "plan buffers");
  }
  p->device = dev;
  return BD_OK;
}

// point the plan at a point set: bound, integer path, launch shape, work list, and the
// asynchronous upload of points (and explicit lifts) on stream st
int plan_prepare(bd_plan* p, const int64_t* points, const int64_t* lifts, int32_t npts, int32_t k,
                 const bd_plan_opts* opts, cudaStream_t st) {
  int rc = check_points(points, npts, k);
  if (rc) return rc;
  if (npts < k + 1) return fail(BD_ERR_ARG, "a plan needs at least k+1 points");
  rc = plan_alloc(p);
  if (rc) return rc;
  if (p->launched) {  // the staging buffer may still feed the previous launch
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    p->launched = false;
  }
  p->N = npts;
  p->K = k;
  p->max_abs = 0;
  for (int64_t i = 0; i < (int64_t)npts * k; ++i) p->max_abs = std::max<int64_t>(p->max_abs, std::llabs(points[i]));
  int64_t spread = (1 << 20) - 1;
  if (lifts) {
    int64_t lo = lifts[0], hi = lifts[0];
    for (int i = 0; i < npts; ++i) {
      if (lifts[i] >= ((int64_t)1 << 40) || lifts[i] <= -((int64_t)1 << 40)) return fail(BD_ERR_ARG, "|lift| must be below 2^40");
      lo = std::min(lo, lifts[i]);
      hi = std::max(hi, lifts[i]);
    }
    spread = hi - lo;
  }
  double coord_bits = 0;
  p->bound = bd::hadamard_log2(points, lifts, npts, k, spread, &coord_bits);
  p->path = bd::choose_path(coord_bits, p->bound);
  if (p->path < 0) return fail(BD_ERR_OVERFLOW, "Hadamard bound of the lifted minors exceeds 2^127");
  if (opts && opts->force_int128) p->path = bd::PATH_WIDE;
  const int wreq = opts ? opts->warps_per_block : 0, breq = opts ? opts->blocks_per_sm : 0;
  const int stage = opts ? opts->bottom_stage : 0;
  if (stage != 0 && stage != 4 && stage != 5) return fail(BD_ERR_ARG, "bottom_stage must be 0, 4 or 5");
  rc = get_shape(npts, k, p->path, false, wreq, breq, p->shape);
  if (rc) return rc;
  p->five = p->path == bd::PATH_NARROW && k >= 4 &&
            (stage == 5 || (stage == 0 && bd::prefer_five(points, npts, k, (uint64_t)p->shape.blocks * p->shape.warps)));
  if (p->five) {  // the 5-D kernel's own occupancy
    rc = get_shape(npts, k, p->path, true, wreq, breq, p->shape);
    if (rc) return rc;
  }
  const uint64_t total = bd::binom(npts, k + 1);
  const uint64_t warps = (uint64_t)p->shape.blocks * p->shape.warps;
  const int64_t thr = opts && opts->item_subsets > 0 ? opts->item_subsets : (int64_t)bd::default_item_subsets(total, warps);
  rc = get_items(npts, k, thr, (int64_t)warps, bd::item_depth(k, p->path, p->five), p->items);
  if (rc) return rc;
  rc = get_tri(p->tri);
  if (rc) return rc;
  std::memcpy(p->h_stage, points, sizeof(int64_t) * npts * k);
  cudaError_t e = cudaMemcpyAsync(p->d_pts, p->h_stage, sizeof(int64_t) * npts * k, cudaMemcpyHostToDevice, st);
  p->explicit_lifts = lifts != nullptr;
  if (e == cudaSuccess && lifts) {
    std::memcpy(p->h_stage + (size_t)BD_NMAX * BD_KMAX, lifts, sizeof(int64_t) * npts);
    e = cudaMemcpyAsync(p->d_lifts, p->h_stage + (size_t)BD_NMAX * BD_KMAX, sizeof(int64_t) * npts,
                        cudaMemcpyHostToDevice, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "point upload");
  p->stream = st;
  return BD_OK;
}

int plan_make(const int64_t* points, const int64_t* lifts, int32_t npts, int32_t k, const bd_plan_opts* opts,
              bd_plan** out) {
  bd_plan* p = new (std::nothrow) bd_plan();
  if (!p) return fail(BD_ERR_NOMEM, "host allocation");
  int rc = plan_prepare(p, points, lifts, npts, k, opts, g_stream);
  if (rc) {
    plan_free(p);
    return rc;
  }
  cudaError_t e = cudaStreamSynchronize(g_stream);  // the plan owns its inputs from here on
  if (e != cudaSuccess) {
    plan_free(p);
    return cuda_fail(e, "cudaStreamSynchronize");
  }
  *out = p;
  return BD_OK;
}

// the calling thread's plan for the synchronous calls
bd_plan* thread_plan() {
  struct Holder {
    bd_plan* p = nullptr;
    ~Holder() {
      if (p) plan_free(p);
    }
  };
  thread_local Holder h;
  if (!h.p) h.p = new (std::nothrow) bd_plan();
  return h.p;
}

int plan_launch(bd_plan* p, uint64_t seed, int attempt, cudaStream_t st, int shard = 0, int shards = 1,
                const bd::CellSink* sink = nullptr) {
  BD_CUDA(cudaMemsetAsync(p->d_state, 0, state_bytes(), st));
  bd::EnumParams ep{};
  ep.pts = p->d_pts;
  ep.lifts = p->explicit_lifts ? p->d_lifts : nullptr;
  ep.lift_seed = bd::lift_stream_seed(seed, (uint32_t)attempt);
  ep.items = p->items->dev;
  ep.nitems = (int)p->items->host.size();
  ep.ranges = p->items->dev_ranges;
  ep.nranges = (int)p->items->ranges.size();
  ep.shard = shard;
  ep.shards = shards;
  ep.tri = p->tri;
  if (sink) ep.sink = *sink;
  uint64_t expected = 0;
  for (size_t u = (size_t)shard; u < p->items->ranges.size(); u += (size_t)shards) expected += p->items->ranges[u].count;
  ep.N = p->N;
  ep.K = p->K;
  ep.five = p->five ? 1 : 0;
  ep.acc = reinterpret_cast<bd::DevAcc*>(p->d_state);
  ep.counter = reinterpret_cast<unsigned int*>(p->d_state + sizeof(bd::DevAcc));
  BD_CUDA(bd::launch_enumerate(ep, p->shape, p->path, st));
  BD_CUDA(cudaMemcpyAsync(p->h_acc, p->d_state, sizeof(bd::DevAcc), cudaMemcpyDeviceToHost, st));
  p->stream = st;
  p->launched = true;
  p->attempt = attempt;
  p->shard = shard;
  p->shards = shards;
  p->items_expected = expected;
  return BD_OK;
}

int plan_read(bd_plan* p, bd_volume_out* out) {
  if (!p->launched) return fail(BD_ERR_STATE, "plan has not been launched");
  BD_CUDA(cudaStreamSynchronize(p->stream));
  std::memset(out, 0, sizeof(*out));
  const bd::DevAcc& a = *p->h_acc;
  out->nvol_lo = a.nvol_lo;
  out->nvol_hi = a.nvol_hi;
  out->cells = a.cells;
  out->singular = a.singular;
  out->ties = a.ties;
  out->subsets = bd::binom(p->N, p->K + 1);
  out->relifts = p->attempt;
  out->flags = (p->path == bd::PATH_WIDE ? BD_FLAG_INT128 : 0) | ((a.nvol_lo | a.nvol_hi) == 0 ? BD_FLAG_DEGENERATE : 0);
  out->max_abs_coord = (int32_t)std::min<int64_t>(p->max_abs, INT32_MAX);
  out->bound_bits = (int32_t)std::ceil(p->bound);
  if (a.items_done != p->items_expected) return fail(BD_ERR_CUDA, "enumeration did not process every work item");
  return BD_OK;
}

int plan_volume(bd_plan* p, uint64_t seed, cudaStream_t st, bd_volume_out* out) {
  const int tries = p->explicit_lifts ? 1 : MAX_LIFTINGS;
  for (int attempt = 0; attempt < tries; ++attempt) {
    int rc = plan_launch(p, seed, attempt, st);
    if (rc) return rc;
    rc = plan_read(p, out);
    if (rc) return rc;
    if (out->ties == 0) return BD_OK;
  }
  return fail(BD_ERR_TIES, p->explicit_lifts ? "the given lifting has ties" : "every allowed lifting had ties");
}

void degenerate_volume(int32_t npts, int32_t k, const int64_t* points, bd_volume_out* out) {
  std::memset(out, 0, sizeof(*out));
  out->flags = BD_FLAG_DEGENERATE;
  out->subsets = bd::binom(npts, k + 1);
  int64_t mx = 0;
  for (int64_t i = 0; i < (int64_t)npts * k; ++i) mx = std::max<int64_t>(mx, std::llabs(points[i]));
  out->max_abs_coord = (int32_t)std::min<int64_t>(mx, INT32_MAX);
}

}  // namespace

extern "C" {

const char* bd_last_error(void) { return g_err.c_str(); }

int bd_inject_alloc_failure(int32_t after) {
  g_alloc_fail_after.store(after < 0 ? -1 : after);
  return BD_OK;
}

int bd_set_stream(void* stream) {
  g_stream = reinterpret_cast<cudaStream_t>(stream);
  return BD_OK;
}

int bd_plan_create(const int64_t* points, int32_t npts, int32_t k, const bd_plan_opts* opts, bd_plan** plan) {
  if (!plan) return fail(BD_ERR_ARG, "plan is NULL");
  return plan_make(points, nullptr, npts, k, opts, plan);
}

int bd_plan_launch(bd_plan* plan, uint64_t seed, int32_t attempt, void* stream) {
  if (!plan) return fail(BD_ERR_ARG, "plan is NULL");
  return plan_launch(plan, seed, attempt, stream ? reinterpret_cast<cudaStream_t>(stream) : g_stream);
}

int bd_plan_launch_shard(bd_plan* plan, uint64_t seed, int32_t attempt, int32_t shard, int32_t shards,
                         void* stream) {
  if (!plan) return fail(BD_ERR_ARG, "plan is NULL");
  if (shards < 1 || shard < 0 || shard >= shards) return fail(BD_ERR_ARG, "need 0 <= shard < shards");
  return plan_launch(plan, seed, attempt, stream ? reinterpret_cast<cudaStream_t>(stream) : g_stream, shard, shards);
}

int bd_plan_read(bd_plan* plan, bd_volume_out* out) {
  if (!plan || !out) return fail(BD_ERR_ARG, "NULL argument");
  return plan_read(plan, out);
}

int bd_plan_volume(bd_plan* plan, uint64_t seed, bd_volume_out* out) {
  if (!plan || !out) return fail(BD_ERR_ARG, "NULL argument");
  return plan_volume(plan, seed, g_stream, out);
}

int bd_plan_info(const bd_plan* plan, int64_t* info) {
  if (!plan || !info) return fail(BD_ERR_ARG, "NULL argument");
  info[0] = (int64_t)plan->items->host.size();
  info[1] = plan->shape.blocks;
  info[2] = plan->shape.warps;
  info[3] = (int64_t)plan->shape.smem;
  info[4] = plan->path;
  info[5] = plan->shape.slots;
  info[6] = (int64_t)plan->items->ranges.size();
  // the walker's bottom test: 5-D, 4-D (filtered paths, k >= 3), 3-D (k = 2), else 2-D
  info[7] = plan->five ? 5 : plan->path != bd::PATH_WIDE && plan->K >= 3 ? 4 : plan->path != bd::PATH_WIDE && plan->K == 2 ? 3 : 2;
  return BD_OK;
}

int bd_plan_destroy(bd_plan* plan) {
  plan_free(plan);
  return BD_OK;
}

int bd_volume(const int64_t* points, int32_t npts, int32_t k, uint64_t seed, bd_volume_out* out) {
  if (!out) return fail(BD_ERR_ARG, "out is NULL");
  int rc = check_points(points, npts, k);
  if (rc) return rc;
  if (npts < k + 1) {
    degenerate_volume(npts, k, points, out);
    return BD_OK;
  }
  bd_plan* p = thread_plan();
  if (!p) return fail(BD_ERR_NOMEM, "host allocation");
  rc = plan_prepare(p, points, nullptr, npts, k, nullptr, g_stream);
  if (rc) return rc;
  return plan_volume(p, seed, g_stream, out);
}

int bd_volume_lifted(const int64_t* points, const int64_t* lifts, int32_t npts, int32_t k, bd_volume_out* out) {
  if (!out || !lifts) return fail(BD_ERR_ARG, "NULL argument");
  int rc = check_points(points, npts, k);
  if (rc) return rc;
  if (npts < k + 1) {
    degenerate_volume(npts, k, points, out);
    return BD_OK;
  }
  bd_plan* p = thread_plan();
  if (!p) return fail(BD_ERR_NOMEM, "host allocation");
  rc = plan_prepare(p, points, lifts, npts, k, nullptr, g_stream);
  if (rc) return rc;
  return plan_volume(p, 0, g_stream, out);
}

int bd_reduce(const int64_t* A, int32_t n, int32_t m, const int64_t* coef, int64_t* points, int64_t* info) {
  if (!A && m > 0) return fail(BD_ERR_ARG, "A is NULL");
  if (!points || !info) return fail(BD_ERR_ARG, "NULL output");
  if (n < 1 || n > 126 || m < 0 || m > 256) return fail(BD_ERR_ARG, "need 1 <= n <= 126, 0 <= m <= 256");
  bd::Reduction r;
  std::string err;
  int rc = bd::reduce_system(A, n, m, coef, r, err);
  if (rc) return fail(rc, err);
  std::memcpy(points, r.points.data(), sizeof(int64_t) * r.points.size());
  info[0] = r.rank;
  info[1] = r.dim;
  info[2] = (int64_t)r.torsion;
  info[3] = r.consistent ? 1 : 0;
  info[4] = r.max_abs_coord;
  info[5] = info[6] = info[7] = 0;
  return BD_OK;
}

int bd_degree(const int64_t* A, int32_t n, int32_t m, const int64_t* coef, uint64_t seed, bd_degree_out* out) {
  if (!out) return fail(BD_ERR_ARG, "out is NULL");
  if (!A && m > 0) return fail(BD_ERR_ARG, "A is NULL");
  if (n < 1 || n > 126 || m < 0 || m > 256) return fail(BD_ERR_ARG, "need 1 <= n <= 126, 0 <= m <= 256");
  std::memset(out, 0, sizeof(*out));
  bd::Reduction r;
  std::string err;
  int rc = bd::reduce_system(A, n, m, coef, r, err);
  if (rc) return fail(rc, err);
  return bd::degree_from_reduction(r, n, seed, out);
}

}  // extern "C"

namespace bd {

int degree_from_reduction(const Reduction& r, int n, uint64_t seed, bd_degree_out* out) {
  int rc = BD_OK;
  std::memset(out, 0, sizeof(*out));
  out->rank = r.rank;
  out->dim = r.dim;
  out->torsion = r.torsion;
  out->consistent = r.consistent ? 1 : 0;
  out->max_abs_coord = (int32_t)r.max_abs_coord;
  if (!r.consistent) {
    out->flags = BD_FLAG_INCONSISTENT;
    return BD_OK;
  }
  if (r.dim == 0) {  // isolated points (Prop. 1)
    set_u128(out->nvol_lo, out->nvol_hi, 1);
    set_u128(out->degree_lo, out->degree_hi, r.torsion);
    return BD_OK;
  }
  // beyond the subset enumeration (dimension above BD_KMAX, or more than BD_NMAX points in two
  // or more dimensions): walk the cells by pivoting instead
  if (r.dim > BD_KMAX || (r.dim > 1 && n + 1 > BD_NMAX)) {
    bd_volume_out v;
    double ms = 0;
    rc = bd_volume_pivot(r.points.data(), n + 1, r.dim, seed, &v, &ms);
    if (rc) return rc;
    const u128 nvol = ((u128)v.nvol_hi << 64) | v.nvol_lo;
    const u128 deg = nvol * r.torsion;
    if (r.torsion && deg / r.torsion != nvol) return fail(BD_ERR_OVERFLOW, "degree exceeds 2^128");
    set_u128(out->nvol_lo, out->nvol_hi, nvol);
    set_u128(out->degree_lo, out->degree_hi, deg);
    out->relifts = v.relifts;
    out->subsets = v.subsets;
    out->cells = v.cells;
    out->flags = v.flags | BD_FLAG_PIVOT;
    return BD_OK;
  }
  if (r.dim == 1) {  // a segment: NVol_1(conv{0, p_1 .. p_n}) = max - min, cells = distinct values - 1
    std::vector<int64_t> x(r.points.begin(), r.points.end());  // n kernel points, then the origin
    std::sort(x.begin(), x.end());
    const u128 nvol = (u128)((i128)x.back() - (i128)x.front());
    set_u128(out->nvol_lo, out->nvol_hi, nvol);
    set_u128(out->degree_lo, out->degree_hi, nvol * r.torsion);
    out->cells = (uint64_t)(std::unique(x.begin(), x.end()) - x.begin()) - 1;
    out->subsets = bd::binom(n + 1, 2);
    return BD_OK;
  }
  bd_volume_out v;
  rc = bd_volume(r.points.data(), n + 1, r.dim, seed, &v);
  if (rc) return rc;
  const u128 nvol = ((u128)v.nvol_hi << 64) | v.nvol_lo;
  const u128 deg = nvol * r.torsion;
  if (r.torsion && deg / r.torsion != nvol) return fail(BD_ERR_OVERFLOW, "degree exceeds 2^128");
  set_u128(out->nvol_lo, out->nvol_hi, nvol);
  set_u128(out->degree_lo, out->degree_hi, deg);
  out->relifts = v.relifts;
  out->subsets = v.subsets;
  out->cells = v.cells;
  out->flags = v.flags;
  return BD_OK;
}

}  // namespace bd

extern "C" {

int bd_classify(const int64_t* points, const int64_t* lifts, int32_t npts, int32_t k, const uint8_t* subsets,
                int32_t count, int32_t* status, int64_t* absdet) {
  int rc = check_points(points, npts, k);
  if (rc) return rc;
  if (!lifts || !subsets || !status || !absdet || count < 0) return fail(BD_ERR_ARG, "NULL argument");
  if (npts < k + 1) return fail(BD_ERR_ARG, "need at least k+1 points");
  for (int64_t i = 0; i < (int64_t)count; ++i) {
    const uint8_t* s = subsets + i * (k + 1);
    for (int j = 0; j <= k; ++j)
      if (s[j] >= npts || (j && s[j] <= s[j - 1])) return fail(BD_ERR_ARG, "subset indices must increase and be < npts");
  }
  if (count == 0) return BD_OK;
  int64_t lo = lifts[0], hi = lifts[0];
  for (int i = 0; i < npts; ++i) {
    lo = std::min(lo, lifts[i]);
    hi = std::max(hi, lifts[i]);
  }
  double coord_bits = 0;
  const double bound = bd::hadamard_log2(points, lifts, npts, k, hi - lo, &coord_bits);
  const int path = bd::choose_path(coord_bits, bound);
  if (path < 0) return fail(BD_ERR_OVERFLOW, "Hadamard bound exceeds 2^127");
  cudaStream_t st = g_stream;
  int64_t *d_pts = nullptr, *d_lifts = nullptr, *d_abs = nullptr;
  uint8_t* d_sub = nullptr;
  int32_t* d_status = nullptr;
  auto cleanup = [&]() {
    cudaFree(d_pts);
    cudaFree(d_lifts);
    cudaFree(d_abs);
    cudaFree(d_sub);
    cudaFree(d_status);
  };
  cudaError_t e = cudaSuccess;
  const char* where = "";
#define CL(call)                 \
  if (e == cudaSuccess) {        \
    e = (call);                  \
    if (e != cudaSuccess) where = #call; \
  }
  CL(bd::dev_malloc(&d_pts, sizeof(int64_t) * npts * k));
  CL(bd::dev_malloc(&d_lifts, sizeof(int64_t) * npts));
  CL(bd::dev_malloc(&d_abs, sizeof(int64_t) * count));
  CL(bd::dev_malloc(&d_sub, (size_t)count * (k + 1)));
  CL(bd::dev_malloc(&d_status, sizeof(int32_t) * count));
  CL(cudaMemcpyAsync(d_pts, points, sizeof(int64_t) * npts * k, cudaMemcpyHostToDevice, st));
  CL(cudaMemcpyAsync(d_lifts, lifts, sizeof(int64_t) * npts, cudaMemcpyHostToDevice, st));
  CL(cudaMemcpyAsync(d_sub, subsets, (size_t)count * (k + 1), cudaMemcpyHostToDevice, st));
  CL(bd::launch_classify(d_pts, d_lifts, npts, k, d_sub, count, d_status, d_abs, path, st));
  CL(cudaMemcpyAsync(status, d_status, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, st));
  CL(cudaMemcpyAsync(absdet, d_abs, sizeof(int64_t) * count, cudaMemcpyDeviceToHost, st));
  CL(cudaStreamSynchronize(st));
#undef CL
  cleanup();
  if (e != cudaSuccess) return cuda_fail(e, where);
  return BD_OK;
}

int bd_host_volume_lifted(const int64_t* points, const int64_t* lifts, int32_t npts, int32_t k,
                          const bd_host_opts* opts, bd_volume_out* out) {
  if (!out || !lifts) return fail(BD_ERR_ARG, "NULL argument");
  const bd_host_opts o = opts ? *opts : bd_host_opts{};
  if (o.team_width > 64) return fail(BD_ERR_ARG, "team_width above 64");
  const int shards = o.shards > 1 ? o.shards : 1;
  if (o.shard < 0 || o.shard >= shards) return fail(BD_ERR_ARG, "need 0 <= shard < shards");
  int rc = check_points(points, npts, k);
  if (rc) return rc;
  if (npts < k + 1) {
    degenerate_volume(npts, k, points, out);
    return BD_OK;
  }
  int64_t lo = lifts[0], hi = lifts[0];
  for (int i = 0; i < npts; ++i) {
    lo = std::min(lo, lifts[i]);
    hi = std::max(hi, lifts[i]);
  }
  double coord_bits = 0;
  const double bound = bd::hadamard_log2(points, lifts, npts, k, hi - lo, &coord_bits);
  int path = bd::choose_path(coord_bits, bound);
  if (path < 0) return fail(BD_ERR_OVERFLOW, "Hadamard bound exceeds 2^127");
  if (o.force_int128) path = bd::PATH_WIDE;
  if (o.bottom_stage != 0 && o.bottom_stage != 4 && o.bottom_stage != 5)
    return fail(BD_ERR_ARG, "bottom_stage must be 0, 4 or 5");
  const bool five = path == bd::PATH_NARROW && k >= 4 &&
                    (o.bottom_stage == 5 || (o.bottom_stage == 0 && bd::prefer_five(points, npts, k, 0)));
  std::vector<int64_t> P((size_t)(k + 1) * npts);
  for (int q = 0; q < npts; ++q) {
    for (int c = 0; c < k; ++c) P[(size_t)c * npts + q] = points[(size_t)q * k + c];
    P[(size_t)k * npts + q] = lifts[q];
  }
  // the device's work list: items in lexicographic order, taken in ranges (8 teams' worth of
  // guided ranges, so that range boundaries and prefix reuse are exercised on one thread too)
  std::vector<bd::Item> items;
  std::vector<bd::Range> ranges;
  bd::build_ranges(npts, k, o.item_subsets ? o.item_subsets : 4096, 8, bd::item_depth(k, path, five), items, ranges);
  if (shards > 1) {  // this shard's ranges only (u % shards == shard, as on the device)
    std::vector<bd::Range> mine;
    for (size_t u = (size_t)o.shard; u < ranges.size(); u += (size_t)shards) mine.push_back(ranges[u]);
    ranges.swap(mine);
  }
  bd::Acc acc{};
  bd::host_enumerate(path, five, P.data(), npts, k, items, std::max(1, o.threads), acc, o.team_width, &ranges);
  std::memset(out, 0, sizeof(*out));
  set_u128(out->nvol_lo, out->nvol_hi, acc.nvol);
  out->cells = acc.cells;
  out->singular = acc.singular;
  out->ties = acc.ties;
  out->subsets = bd::binom(npts, k + 1);
  out->flags = (path == bd::PATH_WIDE ? BD_FLAG_INT128 : 0) | (acc.nvol == 0 ? BD_FLAG_DEGENERATE : 0);
  int64_t mx = 0;
  for (int64_t i = 0; i < (int64_t)npts * k; ++i) mx = std::max<int64_t>(mx, std::llabs(points[i]));
  out->max_abs_coord = (int32_t)std::min<int64_t>(mx, INT32_MAX);
  out->bound_bits = (int32_t)std::ceil(bound);
  if (acc.ties) return fail(BD_ERR_TIES, "the given lifting has ties");
  return BD_OK;
}

int bd_cells(const int64_t* points, int32_t npts, int32_t k, uint64_t seed, int64_t capacity, uint8_t* cells,
             int64_t* den, int64_t* alpha, int64_t* beta, int64_t* count, bd_volume_out* out) {
  if (!out || !count) return fail(BD_ERR_ARG, "NULL argument");
  if (capacity < 0 || (capacity > 0 && (!cells || !den || !alpha || !beta))) return fail(BD_ERR_ARG, "NULL output array");
  *count = 0;
  int rc = check_points(points, npts, k);
  if (rc) return rc;
  if (npts < k + 1) {
    degenerate_volume(npts, k, points, out);
    return BD_OK;
  }
  bd_plan* p = thread_plan();
  if (!p) return fail(BD_ERR_NOMEM, "plan");
  cudaStream_t st = g_stream;
  rc = plan_prepare(p, points, nullptr, npts, k, nullptr, st);
  if (rc) return rc;
  const size_t cap = (size_t)std::max<int64_t>(capacity, 1);
  uint8_t* d_cells = nullptr;
  unsigned long long* d_count = nullptr;
  int64_t *d_den = nullptr, *d_alpha = nullptr, *d_beta = nullptr;
  int32_t* d_status = nullptr;
  auto release = [&]() {
    cudaFree(d_cells);
    cudaFree(d_count);
    cudaFree(d_den);
    cudaFree(d_alpha);
    cudaFree(d_beta);
    cudaFree(d_status);
  };
#define CC(x)                                              \
  do {                                                     \
    cudaError_t e_ = (x);                                  \
    if (e_ != cudaSuccess) {                               \
      release();                                           \
      return cuda_fail(e_, #x);                            \
    }                                                      \
  } while (0)
  CC(bd::dev_malloc(&d_cells, 16 * cap));
  CC(bd::dev_malloc(&d_count, sizeof(unsigned long long)));
  CC(bd::dev_malloc(&d_den, sizeof(int64_t) * cap));
  CC(bd::dev_malloc(&d_alpha, sizeof(int64_t) * cap * k));
  CC(bd::dev_malloc(&d_beta, sizeof(int64_t) * 2 * cap));
  CC(bd::dev_malloc(&d_status, sizeof(int32_t) * cap));
  const bd::CellSink sink{d_cells, d_count, (unsigned long long)capacity};
  int attempt = 0;
  for (;; ++attempt) {
    if (attempt == MAX_LIFTINGS) {
      release();
      return fail(BD_ERR_TIES, "every allowed lifting had ties");
    }
    CC(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), st));
    rc = plan_launch(p, seed, attempt, st, 0, 1, &sink);
    if (!rc) rc = plan_read(p, out);
    if (rc) {
      release();
      return rc;
    }
    if (out->ties == 0) break;
  }
  out->relifts = attempt;
  unsigned long long n = 0;
  CC(cudaMemcpy(&n, d_count, sizeof(n), cudaMemcpyDeviceToHost));
  *count = (int64_t)n;
  if (n > (unsigned long long)capacity) {
    release();
    return fail(BD_ERR_ARG, "capacity is below the number of cells (count holds it)");
  }
  CC(bd::launch_cell_normals(p->d_pts, nullptr, bd::lift_stream_seed(seed, (uint32_t)attempt), npts, k, d_cells, n,
                             d_den, d_alpha, d_beta, d_status, st));
  std::vector<uint8_t> hc(16 * std::max<size_t>(n, 1));
  std::vector<int64_t> hd(std::max<size_t>(n, 1)), ha(std::max<size_t>(n, 1) * k), hb(2 * std::max<size_t>(n, 1));
  std::vector<int32_t> hs(std::max<size_t>(n, 1));
  CC(cudaStreamSynchronize(st));
  if (n) {
    CC(cudaMemcpy(hc.data(), d_cells, 16 * n, cudaMemcpyDeviceToHost));
    CC(cudaMemcpy(hd.data(), d_den, sizeof(int64_t) * n, cudaMemcpyDeviceToHost));
    CC(cudaMemcpy(ha.data(), d_alpha, sizeof(int64_t) * n * k, cudaMemcpyDeviceToHost));
    CC(cudaMemcpy(hb.data(), d_beta, sizeof(int64_t) * 2 * n, cudaMemcpyDeviceToHost));
    CC(cudaMemcpy(hs.data(), d_status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
  }
#undef CC
  release();
  for (unsigned long long i = 0; i < n; ++i)
    if (hs[i]) return fail(BD_ERR_OVERFLOW, "a cell normal leaves the int64/int128 output range");
  // cells in lexicographic order of their index records (the device appends them in any order)
  std::vector<size_t> ord(n);
  for (size_t i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return std::memcmp(&hc[16 * a], &hc[16 * b], 16) < 0; });
  for (size_t r = 0; r < n; ++r) {
    const size_t i = ord[r];
    std::memcpy(cells + r * (k + 1), &hc[16 * i], (size_t)k + 1);
    den[r] = hd[i];
    for (int c = 0; c < k; ++c) alpha[r * k + c] = ha[i * k + c];
    beta[2 * r] = hb[2 * i];
    beta[2 * r + 1] = hb[2 * i + 1];
  }
  return BD_OK;
}

int bd_host_cells(const int64_t* points, const int64_t* lifts, int32_t npts, int32_t k, int64_t capacity,
                  uint8_t* cells, int64_t* den, int64_t* alpha, int64_t* beta, int64_t* count) {
  if (!count || !lifts) return fail(BD_ERR_ARG, "NULL argument");
  if (capacity < 0 || (capacity > 0 && (!cells || !den || !alpha || !beta))) return fail(BD_ERR_ARG, "NULL output array");
  *count = 0;
  int rc = check_points(points, npts, k);
  if (rc) return rc;
  if (npts < k + 1) return BD_OK;
  int64_t lo = lifts[0], hi = lifts[0];
  for (int i = 0; i < npts; ++i) {
    lo = std::min(lo, lifts[i]);
    hi = std::max(hi, lifts[i]);
  }
  double coord_bits = 0;
  const double bound = bd::hadamard_log2(points, lifts, npts, k, hi - lo, &coord_bits);
  const int path = bd::choose_path(coord_bits, bound);
  if (path < 0) return fail(BD_ERR_OVERFLOW, "Hadamard bound exceeds 2^127");
  std::vector<int64_t> P((size_t)(k + 1) * npts);
  for (int q = 0; q < npts; ++q) {
    for (int c = 0; c < k; ++c) P[(size_t)c * npts + q] = points[(size_t)q * k + c];
    P[(size_t)k * npts + q] = lifts[q];
  }
  std::vector<bd::Item> items;
  std::vector<bd::Range> ranges;
  const bool five = path == bd::PATH_NARROW && k >= 4 && bd::prefer_five(points, npts, k, 0);
  bd::build_ranges(npts, k, 4096, 8, bd::item_depth(k, path, five), items, ranges);
  const size_t cap = (size_t)std::max<int64_t>(capacity, 1);
  std::vector<uint8_t> rec(16 * cap);
  unsigned long long n = 0;
  const bd::CellSink sink{rec.data(), &n, (unsigned long long)capacity};
  bd::Acc acc{};
  bd::host_enumerate(path, five, P.data(), npts, k, items, 1, acc, 1, &ranges, &sink);
  *count = (int64_t)n;
  if (acc.ties) return fail(BD_ERR_TIES, "the given lifting has ties");
  if (n > (unsigned long long)capacity) return fail(BD_ERR_ARG, "capacity is below the number of cells (count holds it)");
  std::vector<size_t> ord(n);
  for (size_t i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return std::memcmp(&rec[16 * a], &rec[16 * b], 16) < 0; });
  for (size_t r = 0; r < n; ++r) {
    const uint8_t* c = &rec[16 * ord[r]];
    std::memcpy(cells + r * (k + 1), c, (size_t)k + 1);
    i128 b = 0;
    if (!bd::cell_normal_exact(points, lifts, k, c, den[r], alpha + r * k, b))
      return fail(BD_ERR_OVERFLOW, "a cell normal leaves the int64/int128 output range");
    beta[2 * r] = (int64_t)(uint64_t)(u128)b;
    beta[2 * r + 1] = (int64_t)(b >> 64);
  }
  return BD_OK;
}

}  // extern "C"

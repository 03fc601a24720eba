// Batches: many binomial systems, reduced on host threads, enumerated by one persistent launch
// per integer path over a shared work list of (system, prefix) items (largest predicted cost
// first), optionally captured in a CUDA graph, with an autotuner for the launch geometry and the
// item size.  The plain alternative (one synchronous bd_volume call per system) is kept as a
// mode of the same entry point for comparison.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/binodeg.h"
#include "bd_host.h"
#include "bd_internal.h"
#include "bd_kernels.cuh"
#include "bd_lifts.h"

using bd::i128;
using bd::u128;

namespace {

struct BatchSys {
  // input
  std::vector<int64_t> A, coef;
  int n = 0, m = 0;
  bool has_coef = false, from_points = false;
  uint64_t seed = 0;
  // reduction
  bool reduced = false;
  int status = BD_OK;
  std::string err;
  int rank = 0, dim = 0, N = 0, K = 0, path = 0;
  bool prefer5 = false;  // the 5-D bottom stage is expected to be faster (prefer_five)
  bool five = false;     // this run's bottom stage is the 5-D test
  uint64_t torsion = 1;
  bool consistent = true;
  double bound = 0, coord_bits = 0;
  int64_t max_abs = 0;
  std::vector<int64_t> pts;
  // result of the last run
  u128 nvol = 0;
  uint64_t cells = 0, singular = 0, ties = 0, cycles = 0;
  int attempt = 0;
  bool done = false;
};

// autotuned (warps, items per warp) by (path, maxN, maxK)
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tuned;

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace

struct bd_batch {
  std::vector<BatchSys> sys;
  // device buffers (grown on demand)
  size_t cap_sys = 0, cap_pts = 0, cap_items = 0;
  bd::BatchDesc* d_desc = nullptr;
  int64_t* d_pts = nullptr;
  bd::BatchItem* d_items = nullptr;
  bd::DevAcc* d_acc = nullptr;
  unsigned long long* d_cycles = nullptr;
  unsigned int* d_done = nullptr;
  unsigned int* d_counter = nullptr;  // one per launch group (integer path and bottom stage)
  bd::DevAcc* h_acc = nullptr;        // pinned, cap_sys
  unsigned long long* h_cycles = nullptr;
  cudaGraphExec_t graph = nullptr;
  std::string graph_key;
  bd_batch_stats last{};
};

namespace {

void free_dev(bd_batch* b) {
  cudaFree(b->d_desc);
  cudaFree(b->d_pts);
  cudaFree(b->d_items);
  cudaFree(b->d_acc);
  cudaFree(b->d_cycles);
  cudaFree(b->d_done);
  cudaFree(b->d_counter);
  cudaFreeHost(b->h_acc);
  cudaFreeHost(b->h_cycles);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->d_desc = nullptr;
  b->d_pts = nullptr;
  b->d_items = nullptr;
  b->d_acc = nullptr;
  b->d_cycles = nullptr;
  b->d_done = nullptr;
  b->d_counter = nullptr;
  b->h_acc = nullptr;
  b->h_cycles = nullptr;
  b->cap_sys = b->cap_pts = b->cap_items = 0;
}

int ensure(bd_batch* b, size_t nsys, size_t npts, size_t nitems) {
  cudaError_t e = cudaSuccess;
  if (nsys > b->cap_sys) {
    size_t c = std::max(nsys, b->cap_sys * 2);
    cudaFree(b->d_desc);
    cudaFree(b->d_acc);
    cudaFree(b->d_cycles);
    cudaFree(b->d_done);
    cudaFreeHost(b->h_acc);
    cudaFreeHost(b->h_cycles);
    b->d_desc = nullptr; b->d_acc = nullptr; b->d_cycles = nullptr; b->d_done = nullptr;
    b->h_acc = nullptr; b->h_cycles = nullptr;
    if (e == cudaSuccess) e = bd::dev_malloc(&b->d_desc, sizeof(bd::BatchDesc) * c);
    if (e == cudaSuccess) e = bd::dev_malloc(&b->d_acc, sizeof(bd::DevAcc) * c);
    if (e == cudaSuccess) e = bd::dev_malloc(&b->d_cycles, sizeof(unsigned long long) * c);
    if (e == cudaSuccess) e = bd::dev_malloc(&b->d_done, sizeof(unsigned int) * c);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_acc, sizeof(bd::DevAcc) * c);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_cycles, sizeof(unsigned long long) * c);
    b->cap_sys = c;
  }
  if (e == cudaSuccess && npts > b->cap_pts) {
    size_t c = std::max(npts, b->cap_pts * 2);
    cudaFree(b->d_pts);
    b->d_pts = nullptr;
    e = bd::dev_malloc(&b->d_pts, sizeof(int64_t) * c);
    b->cap_pts = c;
  }
  if (e == cudaSuccess && nitems > b->cap_items) {
    size_t c = std::max(nitems, b->cap_items * 2);
    cudaFree(b->d_items);
    b->d_items = nullptr;
    e = bd::dev_malloc(&b->d_items, sizeof(bd::BatchItem) * c);
    b->cap_items = c;
  }
  if (e == cudaSuccess && !b->d_counter) e = bd::dev_malloc(&b->d_counter, sizeof(unsigned int) * 4);
  if (e != cudaSuccess) {
    free_dev(b);
    return bd::set_error(e == cudaErrorMemoryAllocation ? BD_ERR_NOMEM : BD_ERR_CUDA, cudaGetErrorString(e));
  }
  return BD_OK;
}

void reduce_one(BatchSys& s) {
  if (s.reduced) return;
  s.reduced = true;
  if (!s.from_points) {
    bd::Reduction r;
    std::string err;
    int rc = bd::reduce_system(s.A.data(), s.n, s.m, s.has_coef ? s.coef.data() : nullptr, r, err);
    if (rc) {
      s.status = rc;
      s.err = err;
      return;
    }
    s.rank = r.rank;
    s.dim = r.dim;
    s.torsion = r.torsion;
    s.consistent = r.consistent;
    s.max_abs = r.max_abs_coord;
    s.pts = std::move(r.points);
    s.N = s.n + 1;
    s.K = s.dim;
  }
  if (!s.consistent || s.K == 0) {  // no enumeration: empty set or isolated points
    s.done = true;
    return;
  }
  if (s.K > bd::BATCH_KMAX || s.N > BD_NMAX) {
    s.status = BD_ERR_ARG;
    s.err = "batch systems need dimension <= 12 and at most 64 points";
    return;
  }
  s.bound = bd::hadamard_log2(s.pts.data(), nullptr, s.N, s.K, (1 << 20) - 1, &s.coord_bits);
  s.path = bd::choose_path(s.coord_bits, s.bound);
  s.prefer5 = s.path == bd::PATH_NARROW && s.K >= 4 && bd::prefer_five(s.pts.data(), s.N, s.K, 0);
  if (s.path < 0) {
    s.status = BD_ERR_OVERFLOW;
    s.err = "Hadamard bound of the lifted minors exceeds 2^127";
  }
}

// closed-form cost of one system (the fallback of the cost model): subsets times the work of
// the plain per-subset test, C(N, K+1) (K^3/3 + (N-K)(K+1))
double closed_form_cost(const BatchSys& s) {
  const double sub = (double)bd::binom(s.N, s.K + 1);
  return sub * ((double)s.K * s.K * s.K / 3.0 + (double)(s.N - s.K) * (s.K + 1));
}

struct Group {
  int path = 0, maxN = 0, maxK = 0;
  bool five = false;            // the group's launch runs the 5-D bottom stage
  size_t first = 0, count = 0;  // range in the item array
};

// Work list of the active systems: per system, prefixes of at most `thr_s` subsets where
// thr_s gives each item about `target` predicted cost; all items ordered by decreasing cost.
void build_batch_items(bd_batch* b, const std::vector<int>& active, const float* cost, int items_per_warp,
                       int warps_total, std::vector<bd::BatchItem>& items, std::vector<Group>& groups) {
  items.clear();
  groups.clear();
  // one launch per (integer path, bottom stage): the 32-bit path with the 5-D stage, the 32-bit
  // path with the 4-D stage, the 64-bit and the 128-bit paths
  for (int kind = 0; kind < 4; ++kind) {
    const int path = kind == 0 ? 0 : kind - 1;
    const bool five = kind == 0;
    std::vector<int> in;
    double total = 0;
    for (int i : active)
      if (b->sys[i].path == path && b->sys[i].five == five) {
        in.push_back(i);
        total += cost ? std::max(1e-9, (double)cost[i]) : closed_form_cost(b->sys[i]);
      }
    if (in.empty()) continue;
    Group g;
    g.path = path;
    g.five = five;
    g.first = items.size();
    const double target = total / ((double)warps_total * items_per_warp + 1.0);
    std::vector<std::pair<double, bd::BatchItem>> tmp;
    for (int i : in) {
      const BatchSys& s = b->sys[i];
      g.maxN = std::max(g.maxN, s.N);
      g.maxK = std::max(g.maxK, s.K);
      const double sub = (double)bd::binom(s.N, s.K + 1);
      const double c = cost ? std::max(1e-9, (double)cost[i]) : closed_form_cost(s);
      const double per_subset = c / std::max(1.0, sub);
      uint64_t thr = (uint64_t)std::max(64.0, std::min(4e9, target / per_subset));
      // generation order: the items of every system are ordered by predicted cost below
      for (const bd::Item& it : bd::build_items(s.N, s.K, thr, bd::item_depth(s.K, s.path, s.five), false)) {
        bd::BatchItem x{};
        x.sys = (uint32_t)i;
        x.len = it.len;
        for (int t = 0; t < it.len && t < 11; ++t) x.idx[t] = it.idx[t];
        tmp.push_back({(double)bd::subtree_size(s.N, s.K, it.idx[it.len - 1], it.len) * per_subset, x});
      }
    }
    // largest predicted cost first, by a counting sort on quarter octaves of the cost (items
    // within 19 % of each other keep their generation order; a comparison sort of the ~200,000
    // items of a 4096-system batch cost more host time than the order is worth)
    std::vector<int> key(tmp.size());
    int kmin = INT32_MAX, kmax = INT32_MIN;
    for (size_t t = 0; t < tmp.size(); ++t) {
      int e = 0;
      const double m = std::frexp(std::max(tmp[t].first, 1e-300), &e);  // m in [0.5, 1)
      key[t] = 4 * e + (m >= 0.8408964152537145 ? 3 : m >= 0.7071067811865476 ? 2 : m >= 0.5946035575013605 ? 1 : 0);
      kmin = std::min(kmin, key[t]);
      kmax = std::max(kmax, key[t]);
    }
    std::vector<size_t> start((size_t)(kmax - kmin) + 2, 0);
    for (size_t t = 0; t < tmp.size(); ++t) ++start[(size_t)(kmax - key[t]) + 1];
    for (size_t b2 = 1; b2 < start.size(); ++b2) start[b2] += start[b2 - 1];
    items.resize(g.first + tmp.size());
    for (size_t t = 0; t < tmp.size(); ++t) items[g.first + start[(size_t)(kmax - key[t])]++] = tmp[t].second;
    g.count = items.size() - g.first;
    groups.push_back(g);
  }
}

// one batched pass over `active` (their current liftings); results into the systems
int run_batched(bd_batch* b, const std::vector<int>& active, const float* cost, int warps_req, int items_per_warp,
                bool use_graph, cudaStream_t st, double* gpu_ms, int* launches, size_t* nitems_out) {
  // the launch geometry of the largest group sizes the work list
  const int sms = sm_count();
  std::vector<bd::BatchItem> items;
  std::vector<Group> groups;
  {
    int maxN = 0, maxK = 0;
    for (int i : active) {
      maxN = std::max(maxN, b->sys[i].N);
      maxK = std::max(maxK, b->sys[i].K);
    }
    cudaError_t e;
    bd::LaunchShape s0 = bd::batch_shape(std::max(maxN, 2), std::max(maxK, 1), bd::PATH_NARROW, false, warps_req, 0, sms, &e);
    if (e != cudaSuccess) return bd::cuda_error(e);
    build_batch_items(b, active, cost, items_per_warp, s0.blocks * s0.warps, items, groups);
  }
  // packed descriptors and points (all systems, so that indices stay global)
  const size_t nsys = b->sys.size();
  std::vector<bd::BatchDesc> desc(nsys);
  std::vector<int64_t> pts;
  for (size_t i = 0; i < nsys; ++i) {
    const BatchSys& s = b->sys[i];
    desc[i].N = s.N;
    desc[i].K = s.K;
    desc[i].pts_off = (int)pts.size();
    desc[i].path = s.path;
    desc[i].five = s.five ? 1 : 0;
    desc[i].lift_seed = bd::lift_stream_seed(s.seed, (uint32_t)s.attempt);
    pts.insert(pts.end(), s.pts.begin(), s.pts.begin() + (size_t)s.N * s.K);
  }
  int rc = ensure(b, nsys, std::max<size_t>(1, pts.size()), std::max<size_t>(1, items.size()));
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(b->d_desc, desc.data(), sizeof(bd::BatchDesc) * nsys, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !pts.empty())
    e = cudaMemcpyAsync(b->d_pts, pts.data(), sizeof(int64_t) * pts.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !items.empty())
    e = cudaMemcpyAsync(b->d_items, items.data(), sizeof(bd::BatchItem) * items.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host vectors go out of scope
  if (e != cudaSuccess) return bd::cuda_error(e);

  // the timed part: clear, one persistent launch per path group, copy the results back
  std::vector<bd::LaunchShape> shapes;
  for (const Group& g : groups) {
    bd::LaunchShape s = bd::batch_shape(g.maxN, g.maxK, g.path, g.five, warps_req, 0, sms, &e);
    if (e != cudaSuccess) return bd::cuda_error(e);
    shapes.push_back(s);
  }
  const uint32_t* tri = nullptr;  // fetched before any stream capture
  {
    const int trc = bd::device_tri_table(&tri);
    if (trc) return trc;
  }
  auto enqueue = [&](cudaStream_t s) -> cudaError_t {
    cudaError_t r = cudaMemsetAsync(b->d_acc, 0, sizeof(bd::DevAcc) * nsys, s);
    if (r == cudaSuccess) r = cudaMemsetAsync(b->d_cycles, 0, sizeof(unsigned long long) * nsys, s);
    if (r == cudaSuccess) r = cudaMemsetAsync(b->d_done, 0, sizeof(unsigned int) * nsys, s);
    if (r == cudaSuccess) r = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned int) * 4, s);
    for (size_t gi = 0; gi < groups.size() && r == cudaSuccess; ++gi) {
      const Group& g = groups[gi];
      bd::BatchParams p{};
      p.desc = b->d_desc;
      p.pts = b->d_pts;
      p.items = b->d_items + g.first;
      p.nitems = (int)g.count;
      p.maxN = g.maxN;
      p.maxK = g.maxK;
      p.counter = b->d_counter + gi;
      p.acc = b->d_acc;
      p.cycles = b->d_cycles;
      p.done = b->d_done;
      p.tri = tri;
      r = bd::launch_batch(p, shapes[gi], g.path, g.five, s);
    }
    if (r == cudaSuccess) r = cudaMemcpyAsync(b->h_acc, b->d_acc, sizeof(bd::DevAcc) * nsys, cudaMemcpyDeviceToHost, s);
    if (r == cudaSuccess)
      r = cudaMemcpyAsync(b->h_cycles, b->d_cycles, sizeof(unsigned long long) * nsys, cudaMemcpyDeviceToHost, s);
    return r;
  };
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  if (use_graph) {
    // the graph is keyed by everything its nodes capture (buffers, sizes, shapes)
    std::string key = std::to_string(nsys) + ":" + std::to_string((uintptr_t)b->d_acc) + ":" +
                      std::to_string((uintptr_t)b->d_items);
    for (size_t gi = 0; gi < groups.size(); ++gi)
      key += ":" + std::to_string(groups[gi].path) + "," + std::to_string(groups[gi].five) + "," +
             std::to_string(groups[gi].first) + "," +
             std::to_string(groups[gi].count) + "," + std::to_string(groups[gi].maxN) + "," +
             std::to_string(groups[gi].maxK) + "," + std::to_string(shapes[gi].blocks) + "," +
             std::to_string(shapes[gi].warps);
    if (!b->graph || key != b->graph_key) {
      if (b->graph) cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
      cudaStream_t cs;
      e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
      cudaGraph_t g = nullptr;
      if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t r = enqueue(cs);
        e = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess) e = r;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
      if (g) cudaGraphDestroy(g);
      cudaStreamDestroy(cs);
      if (e != cudaSuccess) return bd::cuda_error(e);
      b->graph_key = key;
    }
    e = cudaGraphLaunch(b->graph, st);
  } else {
    e = enqueue(st);
  }
  cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return bd::cuda_error(e);
  *gpu_ms += ms;
  *launches += (int)groups.size();
  *nitems_out += items.size();
  for (int i : active) {
    BatchSys& s = b->sys[i];
    const bd::DevAcc& a = b->h_acc[i];
    s.nvol = ((u128)a.nvol_hi << 64) | a.nvol_lo;
    s.cells = a.cells;
    s.singular = a.singular;
    s.ties = a.ties;
    s.cycles = b->h_cycles[i];
  }
  return BD_OK;
}

void fill_degree(const BatchSys& s, bd_degree_out* out) {
  std::memset(out, 0, sizeof(*out));
  out->rank = s.rank;
  out->dim = s.dim;
  out->torsion = s.torsion;
  out->consistent = s.consistent ? 1 : 0;
  out->max_abs_coord = (int32_t)std::min<int64_t>(s.max_abs, INT32_MAX);
  if (!s.consistent) {
    out->flags = BD_FLAG_INCONSISTENT;
    return;
  }
  if (s.K == 0) {
    out->nvol_lo = 1;
    out->degree_lo = s.torsion;
    return;
  }
  const u128 deg = s.nvol * (u128)s.torsion;
  out->nvol_lo = (uint64_t)s.nvol;
  out->nvol_hi = (uint64_t)(s.nvol >> 64);
  out->degree_lo = (uint64_t)deg;
  out->degree_hi = (uint64_t)(deg >> 64);
  out->relifts = s.attempt;
  out->subsets = bd::binom(s.N, s.K + 1);
  out->cells = s.cells;
  out->flags = (s.path == bd::PATH_WIDE ? BD_FLAG_INT128 : 0) | (s.nvol == 0 ? BD_FLAG_DEGENERATE : 0);
}

}  // namespace

extern "C" {

int bd_batch_create(bd_batch** out) {
  if (!out) return bd::set_error(BD_ERR_ARG, "NULL argument");
  *out = new (std::nothrow) bd_batch();
  return *out ? BD_OK : bd::set_error(BD_ERR_NOMEM, "host allocation");
}

int bd_batch_destroy(bd_batch* b) {
  if (!b) return BD_OK;
  free_dev(b);
  delete b;
  return BD_OK;
}

int bd_batch_add(bd_batch* b, const int64_t* A, int32_t n, int32_t m, const int64_t* coef, uint64_t seed,
                 int32_t* index) {
  if (!b || (!A && m > 0)) return bd::set_error(BD_ERR_ARG, "NULL argument");
  if (n < 1 || n >= BD_NMAX || m < 0 || m > 256) return bd::set_error(BD_ERR_ARG, "need 1 <= n < BD_NMAX, 0 <= m <= 256");
  BatchSys s;
  s.n = n;
  s.m = m;
  s.A.assign(A, A + (size_t)n * m);
  if (coef) {
    s.has_coef = true;
    s.coef.assign(coef, coef + (size_t)4 * m);
  }
  s.seed = seed;
  b->sys.push_back(std::move(s));
  if (index) *index = (int32_t)b->sys.size() - 1;
  return BD_OK;
}

int bd_batch_add_points(bd_batch* b, const int64_t* points, int32_t npts, int32_t k, uint64_t seed, int32_t* index) {
  if (!b || !points) return bd::set_error(BD_ERR_ARG, "NULL argument");
  if (k < 1 || k > bd::BATCH_KMAX || npts < k + 1 || npts > BD_NMAX)
    return bd::set_error(BD_ERR_ARG, "batch point sets need 1 <= k <= 12 and k+1 <= npts <= BD_NMAX");
  BatchSys s;
  s.from_points = true;
  s.N = npts;
  s.K = k;
  s.dim = k;
  s.pts.assign(points, points + (size_t)npts * k);
  for (int64_t v : s.pts) {
    if (v >= ((int64_t)1 << 40) || v <= -((int64_t)1 << 40)) return bd::set_error(BD_ERR_ARG, "|coordinate| must be below 2^40");
    s.max_abs = std::max<int64_t>(s.max_abs, std::llabs(v));
  }
  s.seed = seed;
  b->sys.push_back(std::move(s));
  if (index) *index = (int32_t)b->sys.size() - 1;
  return BD_OK;
}

int bd_batch_size(const bd_batch* b, int32_t* count) {
  if (!b || !count) return bd::set_error(BD_ERR_ARG, "NULL argument");
  *count = (int32_t)b->sys.size();
  return BD_OK;
}

int bd_batch_prepare(bd_batch* b, int32_t threads) {
  if (!b) return bd::set_error(BD_ERR_ARG, "NULL argument");
  const double t0 = now_ms();
  int nt = threads > 0 ? threads : (int)std::max(1u, std::thread::hardware_concurrency());
  nt = std::min<int>(nt, (int)std::max<size_t>(1, b->sys.size()));
  std::atomic<size_t> next(0);
  auto work = [&]() {
    for (;;) {
      const size_t i = next.fetch_add(1);
      if (i >= b->sys.size()) break;
      reduce_one(b->sys[i]);
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
  b->last.host_ms = now_ms() - t0;
  for (const BatchSys& s : b->sys)
    if (s.status != BD_OK) return bd::set_error(s.status, s.err.c_str());
  return BD_OK;
}

int bd_batch_features(const bd_batch* b, float* features) {
  if (!b || !features) return bd::set_error(BD_ERR_ARG, "NULL argument");
  for (size_t i = 0; i < b->sys.size(); ++i) {
    const BatchSys& s = b->sys[i];
    if (!s.reduced) return bd::set_error(BD_ERR_STATE, "bd_batch_prepare must run first");
    float* f = features + i * BD_FEATURES;
    const double sub = (double)bd::binom(s.N, s.K + 1);
    // integer-derived descriptors of the reduced system (see include/binodeg.h)
    int zeros = 0, ones = 0;
    for (int64_t v : s.pts) {
      zeros += v == 0;
      ones += v == 1 || v == -1;
    }
    const double cnt = std::max<size_t>(1, s.pts.size());
    double rowspread = 0;  // mean over coordinates of (max - min)
    for (int c = 0; c < s.K; ++c) {
      int64_t lo = 0, hi = 0;
      for (int q = 0; q < s.N; ++q) {
        lo = std::min(lo, s.pts[(size_t)q * s.K + c]);
        hi = std::max(hi, s.pts[(size_t)q * s.K + c]);
      }
      rowspread += (double)(hi - lo);
    }
    rowspread /= std::max(1, s.K);
    f[0] = (float)s.N;
    f[1] = (float)s.K;
    f[2] = (float)std::log2(std::max(1.0, sub));
    f[3] = (float)std::log2(std::max(1.0, closed_form_cost(s)));
    f[4] = (float)s.path;
    f[5] = (float)s.bound;
    f[6] = (float)s.coord_bits;
    f[7] = (float)std::log2(1.0 + (double)s.max_abs);
    f[8] = (float)(zeros / cnt);
    f[9] = (float)(ones / cnt);
    f[10] = (float)rowspread;
    f[11] = (float)(s.N - s.K);
    f[12] = (float)s.n;
    f[13] = (float)s.m;
    f[14] = (float)s.rank;
    f[15] = (float)std::log2((double)std::max<uint64_t>(1, s.torsion));
  }
  return BD_OK;
}

int bd_batch_run(bd_batch* b, const bd_batch_opts* opts, bd_batch_stats* stats) {
  if (!b) return bd::set_error(BD_ERR_ARG, "NULL argument");
  bd_batch_opts o{};
  if (opts) o = *opts;
  cudaStream_t st = bd::thread_stream();
  for (const BatchSys& s : b->sys)
    if (!s.reduced) return bd::set_error(BD_ERR_STATE, "bd_batch_prepare must run first");
    else if (s.status != BD_OK) return bd::set_error(s.status, s.err.c_str());
  bd_batch_stats S{};
  S.host_ms = b->last.host_ms;
  std::vector<int> active;
  for (size_t i = 0; i < b->sys.size(); ++i) {
    BatchSys& s = b->sys[i];
    s.attempt = 0;
    s.done = !s.consistent || s.K == 0;
    if (!s.done) active.push_back((int)i);
  }
  if (o.bottom_stage != 0 && o.bottom_stage != 4 && o.bottom_stage != 5)
    return bd::set_error(BD_ERR_ARG, "bottom_stage must be 0, 4 or 5");
  for (BatchSys& s : b->sys)
    s.five = s.path == bd::PATH_NARROW && s.K >= 4 && (o.bottom_stage == 5 || (o.bottom_stage == 0 && s.prefer5));
  const double w0 = now_ms();
  if (o.mode == 1) {  // the plain form: one synchronous bd_volume per system
    for (int i : active) {
      BatchSys& s = b->sys[i];
      bd_volume_out v;
      int rc = bd_volume(s.pts.data(), s.N, s.K, s.seed, &v);
      if (rc) return rc;
      s.nvol = ((u128)v.nvol_hi << 64) | v.nvol_lo;
      s.cells = v.cells;
      s.singular = v.singular;
      s.ties = 0;
      s.attempt = v.relifts;
      s.cycles = 0;
      s.done = true;
      S.launches += 1 + v.relifts;
    }
  } else {
    int warps = o.warps_per_block, ipw = o.item_factor > 0 ? o.item_factor : 4;
    if (o.autotune && !active.empty()) {
      int maxN = 0, maxK = 0;
      for (int i : active) {
        maxN = std::max(maxN, b->sys[i].N);
        maxK = std::max(maxK, b->sys[i].K);
      }
      const auto key = std::make_tuple(0, maxN, maxK, (int)std::min<size_t>(active.size(), 1u << 20));
      bool have = false;
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
          warps = it->second.first;
          ipw = it->second.second;
          have = true;
        }
      }
      if (!have) {
        // time each candidate on a sample of the batch (every system if it is small)
        std::vector<int> sample;
        const size_t step = std::max<size_t>(1, active.size() / 256);
        for (size_t t = 0; t < active.size(); t += step) sample.push_back(active[t]);
        double best = 1e300;
        for (int w : {2, 4, 8})
          for (int f : {2, 4, 8, 16}) {
            double ms = 0;
            int l = 0;
            size_t ni = 0;
            int rc = run_batched(b, sample, o.cost, w, f, false, st, &ms, &l, &ni);
            if (rc) return rc;
            S.tune_ms += ms;
            if (ms < best) {
              best = ms;
              warps = w;
              ipw = f;
            }
          }
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = {warps, ipw};
      }
    }
    S.warps_per_block = warps;
    S.item_factor = ipw;
    for (int attempt = 0; attempt < 8 && !active.empty(); ++attempt) {
      size_t ni = 0;
      int rc = run_batched(b, active, o.cost, warps, ipw, o.use_graph != 0 && attempt == 0, st, &S.gpu_ms,
                           &S.launches, &ni);
      if (rc) return rc;
      S.items += (int64_t)ni;
      std::vector<int> again;
      for (int i : active) {
        BatchSys& s = b->sys[i];
        if (s.ties) {
          s.attempt += 1;
          again.push_back(i);
          S.relifted += 1;
        } else {
          s.done = true;
        }
      }
      active.swap(again);
    }
    if (!active.empty()) return bd::set_error(BD_ERR_TIES, "every allowed lifting had ties");
  }
  S.wall_ms = now_ms() - w0;
  for (const BatchSys& s : b->sys)
    if (s.consistent && s.K > 0) S.subsets += bd::binom(s.N, s.K + 1);
  b->last = S;
  if (stats) *stats = S;
  return BD_OK;
}

int bd_batch_result(const bd_batch* b, int32_t index, bd_degree_out* out, uint64_t* cycles) {
  if (!b || !out || index < 0 || (size_t)index >= b->sys.size()) return bd::set_error(BD_ERR_ARG, "bad index");
  const BatchSys& s = b->sys[index];
  if (!s.done) return bd::set_error(BD_ERR_STATE, "system has no result yet");
  fill_degree(s, out);
  if (cycles) *cycles = s.cycles;
  return BD_OK;
}

}  // extern "C"

// Serving with continuous batching.  One persistent kernel (k_serve) claims work items from a
// device ring while the host keeps appending to it: a pump thread admits submitted systems into
// free slots as long as the device budget (slots and ring capacity) allows, publishes their
// items, watches completion records the kernel writes to host-mapped memory, re-lifts ties and
// hands finished degrees to bd_server_poll.  Systems that arrive while others run are admitted
// immediately, so their items interleave with the running ones on the device.  Systems the
// persistent kernel does not carry (128-bit minors, dimension above its stack, more than 64
// points) go to a side worker thread that runs bd_degree's volume path on a stream of its own,
// beside the persistent kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/binodeg.h"
#include "bd_host.h"
#include "bd_internal.h"
#include "bd_kernels.cuh"
#include "bd_lifts.h"

using bd::u128;

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
  int64_t ticket = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int rank = 0, dim = 0, N = 0, K = 0, path = 0, attempt = 0;
  bool five = false;    // the walk's bottom stage is the 5-D test (set when its items are built)
  bool alone5 = false;  // the 5-D stage is preferred when the request has the GPU to itself
  bool pooled5 = false; // ... and when it shares the persistent kernel with other requests
  uint64_t torsion = 1, seed = 0;
  bool consistent = true;
  int64_t max_abs = 0;
  double cost = 0;
  std::vector<int64_t> pts;
  std::vector<bd::BatchItem> items;
  uint64_t ring_start = 0;  // first ring ticket of the current publication
  int slot = -1;
  int64_t admission = 0;    // 1-based admission number (the test hook withholds one of them)
  bd_degree_out out{};
  int status = BD_OK;
  std::string err;          // message of a failed request
  uint64_t cycles = 0;
  bd::Reduction red;        // side route only: the host reduction, for bd_degree's volume path
};

}  // namespace

struct bd_server {
  bd_server_opts opts{};
  int slots = 0;
  uint64_t ring_cap = 0, comp_cap = 0;
  int maxN = 32, maxK = 10;  // the systems the persistent kernel carries (its shared-memory layout)
  bd::LaunchShape shape;
  const uint32_t* tri = nullptr;  // the device's colex decode table
  // device
  bd::BatchDesc* d_desc = nullptr;
  int64_t* d_pts = nullptr;
  bd::BatchItem* d_ring = nullptr;
  unsigned long long* d_head = nullptr;
  unsigned long long* d_tail = nullptr;
  unsigned int* d_remaining = nullptr;
  bd::DevAcc* d_acc = nullptr;
  unsigned long long* d_cycles = nullptr;
  unsigned long long* d_comp_count = nullptr;
  // host-mapped
  volatile unsigned long long* h_comp = nullptr;
  unsigned long long* d_comp = nullptr;
  int* d_stop = nullptr;  // device word: 1 asks the kernel's waiting warps to exit (server stop)
  unsigned long long* d_seq = nullptr;           // per ring position: ticket + 1 once published
  unsigned long long* h_seq = nullptr;           // pinned mirror of the stamps
  unsigned long long* d_fault = nullptr;         // device fault word (see ServeParams)
  volatile unsigned long long* h_fault = nullptr;  // host-mapped copy
  unsigned long long* d_fault_map = nullptr;
  int64_t admissions = 0;
  // pinned staging
  bd::BatchDesc* h_desc = nullptr;   // per slot
  int64_t* h_pts = nullptr;          // per slot
  unsigned int* h_rem = nullptr;     // per slot
  bd::BatchItem* h_ring = nullptr;   // mirror of the ring
  unsigned long long* h_tails = nullptr;   // tail values, one per publication (kTailStage entries)
  uint64_t publications = 0;
  volatile unsigned long long* h_res = nullptr;  // host-mapped: per slot, the kernel's final sums
  unsigned long long* d_res = nullptr;
  cudaStream_t s_kernel = nullptr, s_ctl = nullptr, s_side = nullptr;
  int device = 0;
  // host state
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req*> waiting, done;
  std::vector<Req*> in_slot;
  std::vector<int> free_slots;
  uint64_t tail = 0, ring_used = 0, comp_read = 0, inflight_items = 0;
  int64_t next_ticket = 0;
  std::atomic<bool> running{false};
  bool kernel_live = false;
  // work lists by (N, K, integer path, 5-D stage), built once (pump thread, under mu)
  std::map<std::tuple<int, int, int, bool>, std::vector<bd::BatchItem>> item_cache;
  std::thread pump;
  // side route: a queue served by its own thread and stream
  std::deque<Req*> side_q;
  std::condition_variable side_cv;
  bool side_running = true;
  std::thread side_worker;
  int resident = 0;  // requests holding a slot (their items on the device)
  bd_server_stats stats{};
  std::string error;
};

namespace {

int cu(cudaError_t e, const char* what) {
  return e == cudaSuccess ? BD_OK : bd::cuda_error(e, what);
}

constexpr uint64_t kTailStage = 1024;  // staged tail values (see publish)

// publish one request's items (it already owns a slot) and its slot state
int publish(bd_server* s, Req* r) {
  const int slot = r->slot;
  bd::BatchDesc& d = s->h_desc[slot];
  d.N = r->N;
  d.K = r->K;
  d.pts_off = 0;
  d.path = r->path;
  d.five = r->five ? 1 : 0;
  d.gen = (int)r->admission;
  d.lift_seed = bd::lift_stream_seed(r->seed, (uint32_t)r->attempt);
  std::memcpy(s->h_pts + (size_t)slot * bd::BD_SERVE_PTS, r->pts.data(), sizeof(int64_t) * r->pts.size());
  s->h_rem[slot] = (unsigned)r->items.size();
  cudaError_t e = cudaMemcpyAsync(s->d_desc + slot, &d, sizeof(d), cudaMemcpyHostToDevice, s->s_ctl);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_pts + (size_t)slot * bd::BD_SERVE_PTS, s->h_pts + (size_t)slot * bd::BD_SERVE_PTS,
                        sizeof(int64_t) * r->pts.size(), cudaMemcpyHostToDevice, s->s_ctl);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_acc + slot, 0, sizeof(bd::DevAcc), s->s_ctl);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_cycles + slot, 0, sizeof(unsigned long long), s->s_ctl);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_remaining + slot, s->h_rem + slot, sizeof(unsigned), cudaMemcpyHostToDevice, s->s_ctl);
  // items into the ring (possibly wrapping), then the new tail: same stream, so in this order
  const uint64_t n = r->items.size();
  r->ring_start = s->tail;
  for (uint64_t i = 0; i < n; ++i) {
    bd::BatchItem it = r->items[i];
    it.sys = (uint32_t)slot;
    s->h_ring[(s->tail + i) % s->ring_cap] = it;
  }
  uint64_t start = s->tail % s->ring_cap, first = std::min<uint64_t>(n, s->ring_cap - start);
  if (e == cudaSuccess && first)
    e = cudaMemcpyAsync(s->d_ring + start, s->h_ring + start, sizeof(bd::BatchItem) * first, cudaMemcpyHostToDevice, s->s_ctl);
  if (e == cudaSuccess && n > first)
    e = cudaMemcpyAsync(s->d_ring, s->h_ring, sizeof(bd::BatchItem) * (n - first), cudaMemcpyHostToDevice, s->s_ctl);
  // the publication stamps, after the items (same stream) and before the tail; the test hook
  // withholds those of one admission so that the kernel's bounded wait for them runs out
  if (r->admission != s->opts.test_withhold) {
    for (uint64_t i = 0; i < n; ++i) s->h_seq[(s->tail + i) % s->ring_cap] = s->tail + i + 1;
    if (e == cudaSuccess && first)
      e = cudaMemcpyAsync(s->d_seq + start, s->h_seq + start, sizeof(unsigned long long) * first,
                          cudaMemcpyHostToDevice, s->s_ctl);
    if (e == cudaSuccess && n > first)
      e = cudaMemcpyAsync(s->d_seq, s->h_seq, sizeof(unsigned long long) * (n - first), cudaMemcpyHostToDevice, s->s_ctl);
  }
  // Every staging buffer is pinned and owned by the slot or the ring position until the request
  // completes, except the tail value: each publication copies its own entry of a small ring of
  // them, and every half turn of that ring waits for the copies in flight, so that no entry is
  // rewritten before its copy has run.  The pump thus never waits for a publication.
  s->tail += n;
  const uint64_t ti = s->publications++ % kTailStage;
  if (ti % (kTailStage / 2) == 0 && e == cudaSuccess) e = cudaStreamSynchronize(s->s_ctl);
  s->h_tails[ti] = s->tail;
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_tail, s->h_tails + ti, sizeof(unsigned long long), cudaMemcpyHostToDevice, s->s_ctl);
  s->ring_used += n;
  s->inflight_items += n;
  return cu(e, "publish");
}

void build_request_items(bd_server* s, Req* r) {
  // the list depends only on (N, K, integer path, stage) for a given server: built once
  const auto key = std::make_tuple(r->N, r->K, r->path, r->five);
  auto hit = s->item_cache.find(key);
  if (hit != s->item_cache.end()) {
    r->items = hit->second;
    return;
  }
  const uint64_t sub = bd::binom(r->N, r->K + 1);
  const uint64_t warps = (uint64_t)s->shape.blocks * s->shape.warps;
  // eight items per resident warp: enough to spread one system over the GPU with balance
  const uint64_t want = std::max<uint64_t>(1, 8 * warps);
  uint64_t thr = std::max<uint64_t>(s->opts.item_subsets > 0 ? (uint64_t)s->opts.item_subsets : 256, sub / want);
  // a request must fit the ring and the in-flight limit on an idle device, or it would wait
  // forever: the split is coarsened until it does (the coarsest list, one item per first index,
  // has at most 64 items; the ring holds at least 1024)
  const uint64_t limit = s->opts.max_inflight_items > 0 ? std::min<uint64_t>(s->ring_cap, (uint64_t)s->opts.max_inflight_items)
                                                        : s->ring_cap;
  std::vector<bd::Item> list;
  for (;;) {
    list = bd::build_items(r->N, r->K, thr, bd::item_depth(r->K, r->path, r->five));
    if (list.size() <= limit || thr >= sub) break;
    thr *= 2;
  }
  r->items.clear();
  for (const bd::Item& it : list) {
    bd::BatchItem x{};
    x.len = it.len;
    for (int t = 0; t < it.len && t < 11; ++t) x.idx[t] = it.idx[t];
    r->items.push_back(x);
  }
  if (s->item_cache.size() >= 4096) s->item_cache.clear();
  s->item_cache[key] = r->items;
}

void finish(bd_server* s, Req* r) {
  r->t_done = now_ms();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->done.push_back(r);
    s->stats.completed += 1;
  }
  s->cv.notify_all();
}

// completion records the kernel has published: results, re-lifts, freed slots
bool take_completions(bd_server* s) {
  bool progress = false;
  for (;;) {
    const unsigned long long rec = s->h_comp[s->comp_read % s->comp_cap];
    if ((rec >> 32) != (unsigned long long)(s->comp_read + 1)) break;
    const int slot = (int)(rec & 0xffffffffull);
    s->comp_read += 1;
    progress = true;
    Req* r = s->in_slot[slot];
    // the slot's sums, written by the kernel to host-mapped memory before the record
    std::atomic_thread_fence(std::memory_order_acquire);
    bd::DevAcc acc;
    unsigned long long* aw = reinterpret_cast<unsigned long long*>(&acc);
    const volatile unsigned long long* src = s->h_res + (size_t)slot * bd::kServeResWords;
    for (size_t w = 0; w < sizeof(bd::DevAcc) / 8; ++w) aw[w] = src[w];
    const unsigned long long cyc = src[sizeof(bd::DevAcc) / 8];
    const bd::DevAcc* a = &acc;
    cudaError_t e = cudaSuccess;
    s->ring_used -= r->items.size();
    s->inflight_items -= r->items.size();
    if (e != cudaSuccess) {
      r->status = BD_ERR_CUDA;
    } else if (a->ties && r->attempt < 7) {  // re-lift in the same slot
      r->attempt += 1;
      s->stats.relifted += 1;
      if (publish(s, r) != BD_OK) r->status = BD_ERR_CUDA;
      else continue;
    } else if (a->ties) {
      r->status = BD_ERR_TIES;
    } else if (a->items_done != r->items.size()) {
      r->status = BD_ERR_CUDA;
    } else {
      const u128 nvol = ((u128)a->nvol_hi << 64) | a->nvol_lo;
      const u128 deg = nvol * (u128)r->torsion;
      r->out.nvol_lo = (uint64_t)nvol;
      r->out.nvol_hi = (uint64_t)(nvol >> 64);
      r->out.degree_lo = (uint64_t)deg;
      r->out.degree_hi = (uint64_t)(deg >> 64);
      r->out.cells = a->cells;
      r->out.relifts = r->attempt;
      r->out.flags = nvol == 0 ? BD_FLAG_DEGENERATE : 0;
      r->cycles = cyc;
    }
    s->in_slot[slot] = nullptr;
    s->free_slots.push_back(slot);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->resident -= 1;
    }
    finish(s, r);
  }
  return progress;
}

// A publication wait in the kernel ran out: every warp has left or is leaving.  Once the kernel
// has exited, finished requests are taken, the request that owns the lost ticket fails with
// BD_ERR_TIMEOUT, the other admitted requests go back to the front of the queue (their partial
// sums are discarded and they run again from the start), and the ring, its stamps and the
// completion records start over.
void recover_from_fault(bd_server* s) {
  const unsigned long long ticket = *s->h_fault - 1;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stats.faults += 1;  // counted before any request of this fault is handed back
  }
  cudaStreamSynchronize(s->s_kernel);
  s->kernel_live = false;
  take_completions(s);
  std::vector<Req*> requeue;
  for (int slot = 0; slot < s->slots; ++slot) {
    Req* r = s->in_slot[slot];
    if (!r) continue;
    s->in_slot[slot] = nullptr;
    s->free_slots.push_back(slot);
    if (ticket >= r->ring_start && ticket < r->ring_start + r->items.size()) {
      r->status = BD_ERR_TIMEOUT;
      r->err = "the device-side wait for the publication of work item " + std::to_string(ticket) +
               " ran out";
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->resident -= 1;
      }
      finish(s, r);
    } else {
      requeue.push_back(r);
    }
  }
  cudaError_t e = cudaMemsetAsync(s->d_head, 0, sizeof(unsigned long long), s->s_ctl);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_tail, 0, sizeof(unsigned long long), s->s_ctl);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_comp_count, 0, sizeof(unsigned long long), s->s_ctl);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_seq, 0, sizeof(unsigned long long) * s->ring_cap, s->s_ctl);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_fault, 0, sizeof(unsigned long long), s->s_ctl);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->s_ctl);
  std::memset((void*)s->h_comp, 0, sizeof(unsigned long long) * s->comp_cap);
  std::memset(s->h_seq, 0, sizeof(unsigned long long) * s->ring_cap);
  s->comp_read = 0;
  s->tail = 0;
  s->ring_used = 0;
  s->inflight_items = 0;
  *s->h_fault = 0;
  std::lock_guard<std::mutex> lk(s->mu);
  s->resident -= (int)requeue.size();
  for (auto it = requeue.rbegin(); it != requeue.rend(); ++it) s->waiting.push_front(*it);
  if (e != cudaSuccess) s->error = cudaGetErrorString(e);
}

// one pump iteration; returns true if it made progress
bool pump_once(bd_server* s) {
  if (*s->h_fault) {
    recover_from_fault(s);
    return true;
  }
  bool progress = take_completions(s);
  // admissions: FIFO or shortest predicted cost first, while a slot and ring room are free and
  // the in-flight work stays below the budget
  for (;;) {
    Req* r = nullptr;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->waiting.empty() || s->free_slots.empty()) break;
      auto it = s->waiting.begin();
      if (s->opts.order == 1)
        it = std::min_element(s->waiting.begin(), s->waiting.end(), [](Req* a, Req* b) { return a->cost < b->cost; });
      r = *it;
      if (r->items.empty()) {
        // the bottom stage by the load at admission: alone on the GPU (latency: the standalone
        // choice) or sharing it with requests in flight or waiting (throughput: the pooled one)
        r->five = s->resident > 0 || s->waiting.size() > 1 ? r->pooled5 : r->alone5;
        build_request_items(s, r);
      }
      const uint64_t limit = s->opts.max_inflight_items > 0 ? (uint64_t)s->opts.max_inflight_items : s->ring_cap;
      // ring room: requests finish out of order, so the oldest publication still in a slot
      // bounds what may be overwritten
      uint64_t oldest = s->tail;
      for (Req* q : s->in_slot)
        if (q) oldest = std::min(oldest, q->ring_start);
      if (s->tail + r->items.size() - oldest > s->ring_cap ||
          (s->inflight_items > 0 && s->inflight_items + r->items.size() > limit))
        break;
      s->waiting.erase(it);
    }
    r->slot = s->free_slots.back();
    s->free_slots.pop_back();
    s->in_slot[r->slot] = r;
    r->t_admit = now_ms();
    r->admission = ++s->admissions;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->resident += 1;
      s->stats.peak_resident = std::max(s->stats.peak_resident, (int32_t)s->resident);
    }
    if (publish(s, r) != BD_OK) {
      r->status = BD_ERR_CUDA;
      r->err = "publish failed";
      s->in_slot[r->slot] = nullptr;
      s->free_slots.push_back(r->slot);
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->resident -= 1;
      }
      finish(s, r);
    }
    progress = true;
  }
  // the kernel: relaunch when work is in flight and the previous launch has exited
  if (s->inflight_items > 0) {
    if (s->kernel_live && cudaStreamQuery(s->s_kernel) == cudaSuccess) s->kernel_live = false;
    if (!s->kernel_live) {
      bd::ServeParams p{};
      p.desc = s->d_desc;
      p.pts = s->d_pts;
      p.ring = s->d_ring;
      p.ring_cap = s->ring_cap;
      p.head = s->d_head;
      p.tail = s->d_tail;
      p.remaining = s->d_remaining;
      p.acc = s->d_acc;
      p.cycles = s->d_cycles;
      p.comp_count = s->d_comp_count;
      p.comp = s->d_comp;
      p.comp_cap = s->comp_cap;
      p.res = s->d_res;
      p.stop = s->d_stop;
      p.idle_ns = 40000000ull;  // ~40 ms without a publication: waiting warps give their tickets back
      p.seq = s->d_seq;
      p.fault_dev = s->d_fault;
      p.fault_host = s->d_fault_map;
      p.wait_ns = (unsigned long long)(s->opts.publish_wait_ms > 0 ? s->opts.publish_wait_ms : 1000) * 1000000ull;
      p.maxN = s->maxN;
      p.maxK = s->maxK;
      p.tri = s->tri;
      if (bd::launch_serve(p, s->shape, s->s_kernel) == cudaSuccess) {
        s->kernel_live = true;
        s->stats.launches += 1;
      }
    }
  }
  return progress;
}

void pump_loop(bd_server* s) {
  cudaSetDevice(s->device);
  while (s->running.load()) {
    if (!pump_once(s)) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  // drain: finish what was admitted and what still waits
  for (;;) {
    bool busy;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      busy = !s->waiting.empty();
    }
    busy = busy || s->inflight_items > 0;
    if (!busy) break;
    if (!pump_once(s)) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

// the side route: requests the persistent kernel does not carry, one at a time through
// bd_degree's volume path on the server's side stream (concurrent with the persistent kernel,
// which leaves room on every SM); drains the queue before it exits
void side_loop(bd_server* s) {
  cudaSetDevice(s->device);
  bd_set_stream(s->s_side);
  for (;;) {
    Req* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->side_cv.wait(lk, [&] { return !s->side_q.empty() || !s->side_running; });
      if (s->side_q.empty()) break;
      r = s->side_q.front();
      s->side_q.pop_front();
    }
    r->t_admit = now_ms();
    bd_degree_out o;
    const int rc = bd::degree_from_reduction(r->red, r->N - 1, r->seed, &o);
    if (rc) {
      r->status = rc;
      r->err = bd_last_error();
    } else {
      r->out = o;
    }
    finish(s, r);
  }
}

void release(bd_server* s) {
  cudaFree(s->d_desc);
  cudaFree(s->d_pts);
  cudaFree(s->d_ring);
  cudaFree(s->d_head);
  cudaFree(s->d_tail);
  cudaFree(s->d_remaining);
  cudaFree(s->d_acc);
  cudaFree(s->d_cycles);
  cudaFree(s->d_comp_count);
  cudaFree(s->d_seq);
  cudaFree(s->d_fault);
  cudaFreeHost((void*)s->h_fault);
  cudaFreeHost(s->h_seq);
  cudaFreeHost((void*)s->h_comp);
  cudaFree(s->d_stop);
  cudaFreeHost(s->h_desc);
  cudaFreeHost(s->h_pts);
  cudaFreeHost(s->h_rem);
  cudaFreeHost(s->h_ring);
  cudaFreeHost(s->h_tails);
  cudaFreeHost((void*)s->h_res);
  if (s->s_kernel) cudaStreamDestroy(s->s_kernel);
  if (s->s_ctl) cudaStreamDestroy(s->s_ctl);
  if (s->s_side) cudaStreamDestroy(s->s_side);
  for (Req* r : s->waiting) delete r;
  for (Req* r : s->side_q) delete r;
  for (Req* r : s->done) delete r;
  for (Req* r : s->in_slot) delete r;
}

}  // namespace

extern "C" {

int bd_server_start(const bd_server_opts* opts, bd_server** out) {
  if (!out) return bd::set_error(BD_ERR_ARG, "NULL argument");
  if (opts && opts->bottom_stage != 0 && opts->bottom_stage != 4 && opts->bottom_stage != 5)
    return bd::set_error(BD_ERR_ARG, "bottom_stage must be 0, 4 or 5");
  bd_server* s = new (std::nothrow) bd_server();
  if (!s) return bd::set_error(BD_ERR_NOMEM, "host allocation");
  if (opts) s->opts = *opts;
  s->slots = s->opts.slots > 0 ? s->opts.slots : 256;
  s->ring_cap = s->opts.ring_items > 0 ? (uint64_t)s->opts.ring_items : (1u << 20);
  if (s->opts.memory_budget > 0) {  // admission by device memory: the ring shrinks to the budget
    const int64_t per_slot = sizeof(int64_t) * bd::BD_SERVE_PTS + sizeof(bd::BatchDesc) + sizeof(bd::DevAcc) + 12;
    const int64_t left = s->opts.memory_budget - per_slot * s->slots;
    const int64_t per_item = sizeof(bd::BatchItem) + sizeof(unsigned long long);  // the item and its stamp
    if (left < per_item * 1024) {
      delete s;
      return bd::set_error(BD_ERR_ARG, "memory budget below the slot table plus 1024 ring items");
    }
    s->ring_cap = std::min<uint64_t>(s->ring_cap, (uint64_t)(left / per_item));
  }
  s->comp_cap = 4096;
  cudaGetDevice(&s->device);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
  cudaError_t e;
  s->shape = bd::serve_shape(s->maxN, s->maxK, s->opts.warps_per_block, s->opts.blocks_per_sm, sms, &e);
  int rc = cu(e, "serve shape");
  if (!rc) rc = bd::device_tri_table(&s->tri);
  auto A = [&](cudaError_t x) {
    if (rc == BD_OK && x != cudaSuccess) rc = cu(x, "server allocation");
  };
  A(bd::dev_malloc(&s->d_desc, sizeof(bd::BatchDesc) * s->slots));
  A(bd::dev_malloc(&s->d_pts, sizeof(int64_t) * bd::BD_SERVE_PTS * s->slots));
  A(bd::dev_malloc(&s->d_ring, sizeof(bd::BatchItem) * s->ring_cap));
  A(bd::dev_malloc(&s->d_head, sizeof(unsigned long long)));
  A(bd::dev_malloc(&s->d_tail, sizeof(unsigned long long)));
  A(bd::dev_malloc(&s->d_remaining, sizeof(unsigned) * s->slots));
  A(bd::dev_malloc(&s->d_acc, sizeof(bd::DevAcc) * s->slots));
  A(bd::dev_malloc(&s->d_cycles, sizeof(unsigned long long) * s->slots));
  A(bd::dev_malloc(&s->d_comp_count, sizeof(unsigned long long)));
  A(bd::dev_malloc(&s->d_seq, sizeof(unsigned long long) * s->ring_cap));
  A(bd::dev_malloc(&s->d_fault, sizeof(unsigned long long)));
  A(cudaHostAlloc((void**)&s->h_fault, sizeof(unsigned long long), cudaHostAllocMapped));
  A(cudaMallocHost(&s->h_seq, sizeof(unsigned long long) * s->ring_cap));
  A(cudaHostAlloc((void**)&s->h_comp, sizeof(unsigned long long) * s->comp_cap, cudaHostAllocMapped));
  A(bd::dev_malloc(&s->d_stop, sizeof(int)));
  A(cudaMallocHost(&s->h_desc, sizeof(bd::BatchDesc) * s->slots));
  A(cudaMallocHost(&s->h_pts, sizeof(int64_t) * bd::BD_SERVE_PTS * s->slots));
  A(cudaMallocHost(&s->h_rem, sizeof(unsigned) * s->slots));
  A(cudaMallocHost(&s->h_ring, sizeof(bd::BatchItem) * s->ring_cap));
  A(cudaMallocHost(&s->h_tails, sizeof(unsigned long long) * kTailStage));
  A(cudaHostAlloc((void**)&s->h_res, sizeof(unsigned long long) * bd::kServeResWords * s->slots, cudaHostAllocMapped));
  A(cudaStreamCreateWithFlags(&s->s_kernel, cudaStreamNonBlocking));
  A(cudaStreamCreateWithFlags(&s->s_ctl, cudaStreamNonBlocking));
  A(cudaStreamCreateWithFlags(&s->s_side, cudaStreamNonBlocking));
  if (rc == BD_OK) {
    std::memset((void*)s->h_comp, 0, sizeof(unsigned long long) * s->comp_cap);
    A(cudaMemset(s->d_stop, 0, sizeof(int)));
    A(cudaHostGetDevicePointer((void**)&s->d_comp, (void*)s->h_comp, 0));
    A(cudaHostGetDevicePointer((void**)&s->d_res, (void*)s->h_res, 0));

    *s->h_fault = 0;
    A(cudaHostGetDevicePointer((void**)&s->d_fault_map, (void*)s->h_fault, 0));
    A(cudaMemset(s->d_seq, 0, sizeof(unsigned long long) * s->ring_cap));
    A(cudaMemset(s->d_fault, 0, sizeof(unsigned long long)));
    std::memset(s->h_seq, 0, sizeof(unsigned long long) * s->ring_cap);
    A(cudaMemset(s->d_head, 0, sizeof(unsigned long long)));
    A(cudaMemset(s->d_tail, 0, sizeof(unsigned long long)));
    A(cudaMemset(s->d_comp_count, 0, sizeof(unsigned long long)));
  }
  if (rc != BD_OK) {
    release(s);
    delete s;
    return rc;
  }
  s->in_slot.assign(s->slots, nullptr);
  for (int i = s->slots - 1; i >= 0; --i) s->free_slots.push_back(i);
  s->stats.ring_items = (int64_t)s->ring_cap;
  s->stats.slots = s->slots;
  s->stats.blocks = s->shape.blocks;
  s->stats.warps_per_block = s->shape.warps;
  s->running = true;
  s->pump = std::thread(pump_loop, s);
  s->side_worker = std::thread(side_loop, s);
  *out = s;
  return BD_OK;
}

int bd_server_submit(bd_server* s, const int64_t* A, int32_t n, int32_t m, const int64_t* coef, uint64_t seed,
                     double predicted_cost, int64_t* ticket) {
  if (!s || (!A && m > 0)) return bd::set_error(BD_ERR_ARG, "NULL argument");
  if (n < 1 || n > 126 || m < 0 || m > 256) return bd::set_error(BD_ERR_ARG, "need 1 <= n <= 126, 0 <= m <= 256");
  Req* r = new (std::nothrow) Req();
  if (!r) return bd::set_error(BD_ERR_NOMEM, "host allocation");
  r->t_submit = now_ms();
  bd::Reduction red;
  std::string err;
  int rc = bd::reduce_system(A, n, m, coef, red, err);
  if (rc) {
    delete r;
    return bd::set_error(rc, err.c_str());
  }
  r->rank = red.rank;
  r->dim = red.dim;
  r->torsion = red.torsion;
  r->consistent = red.consistent;
  r->max_abs = red.max_abs_coord;
  r->N = n + 1;
  r->K = red.dim;
  r->seed = seed;
  r->out.rank = r->rank;
  r->out.dim = r->dim;
  r->out.torsion = r->torsion;
  r->out.consistent = r->consistent ? 1 : 0;
  r->out.max_abs_coord = (int32_t)std::min<int64_t>(r->max_abs, INT32_MAX);
  r->out.subsets = r->K > 0 && r->K <= BD_KMAX && r->N <= BD_NMAX ? bd::binom(r->N, r->K + 1) : 0;
  const bool direct = !r->consistent || r->K == 0;
  bool side = false;
  if (!direct) {
    if (r->K > s->maxK || r->N > s->maxN) {
      side = true;
    } else {
      double coord = 0;
      const double bound = bd::hadamard_log2(red.points.data(), nullptr, r->N, r->K, (1 << 20) - 1, &coord);
      r->path = bd::choose_path(coord, bound);
      const int stage = s->opts.bottom_stage;
      const bool narrow = r->path == bd::PATH_NARROW && r->K >= 4;
      r->alone5 = narrow && (stage == 5 || (stage == 0 && bd::prefer_five(red.points.data(), r->N, r->K,
                                                                         (uint64_t)s->shape.blocks * s->shape.warps)));
      r->pooled5 = narrow && (stage == 5 || (stage == 0 && bd::prefer_five(red.points.data(), r->N, r->K, 0)));
      // the persistent kernel carries the 32- and 64-bit coordinate walkers; 128-bit systems take
      // the side route
      side = r->path < 0 || r->path == bd::PATH_WIDE;
    }
    if (!side) {
      const double sub = (double)bd::binom(r->N, r->K + 1);
      r->cost = predicted_cost > 0 ? predicted_cost
                                   : sub * ((double)r->K * r->K * r->K / 3.0 + (double)(r->N - r->K) * (r->K + 1));
    }
  }
  if (side) r->red = std::move(red);
  else r->pts = std::move(red.points);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->ticket = s->next_ticket++;
    s->stats.submitted += 1;
    if (direct) {
      if (!r->consistent) r->out.flags = BD_FLAG_INCONSISTENT;
      else {
        r->out.nvol_lo = 1;
        r->out.degree_lo = r->torsion;
      }
    } else if (side) {
      s->side_q.push_back(r);
      s->stats.routed += 1;
    } else {
      s->waiting.push_back(r);
    }
  }
  if (ticket) *ticket = r->ticket;
  if (direct) finish(s, r);
  if (side) s->side_cv.notify_all();
  return BD_OK;
}

int bd_server_poll(bd_server* s, int32_t wait_ms, int64_t* ticket, bd_degree_out* out, double* latency_ms) {
  if (!s || !out) return bd::set_error(BD_ERR_ARG, "NULL argument");
  Req* r = nullptr;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && wait_ms > 0) s->cv.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
    if (s->done.empty()) return bd::set_error(BD_ERR_STATE, "no finished request");
    r = s->done.front();
    s->done.pop_front();
  }
  const int st = r->status;
  *out = r->out;
  if (ticket) *ticket = r->ticket;
  if (latency_ms) *latency_ms = r->t_done - r->t_submit;
  const std::string msg = "request " + std::to_string(r->ticket) + " failed: " + r->err;
  delete r;
  return st == BD_OK ? BD_OK : bd::set_error(st, msg.c_str());
}

int bd_server_stats_get(bd_server* s, bd_server_stats* out) {
  if (!s || !out) return bd::set_error(BD_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->waiting = (int32_t)s->waiting.size();
  return BD_OK;
}

int bd_server_stop(bd_server* s) {
  if (!s) return BD_OK;
  s->running = false;
  if (s->pump.joinable()) s->pump.join();  // drains admitted and waiting requests first
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->side_running = false;
  }
  s->side_cv.notify_all();
  if (s->side_worker.joinable()) s->side_worker.join();  // and the side route's queue
  const int one = 1;  // the copy engine delivers the flag while the kernel runs
  cudaMemcpyAsync(s->d_stop, &one, sizeof(one), cudaMemcpyHostToDevice, s->s_ctl);
  cudaStreamSynchronize(s->s_ctl);
  cudaStreamSynchronize(s->s_kernel);
  release(s);
  delete s;
  return BD_OK;
}

}  // extern "C"

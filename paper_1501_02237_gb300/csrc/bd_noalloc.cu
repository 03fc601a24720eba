// bd_volume_noalloc: the lower-facet enumeration with every piece of device scratch memory in
// one file-scope static device array, for callers that must not allocate device memory.
//
// The array is part of the library image: every GPU that loads the library holds it until the
// process exits.  Host code cannot use the array's name as a device address (it names a host
// shadow), so the address is obtained once per device with cudaGetSymbolAddress while that
// device is current, and cached for the life of the process (a device reset unloads the library
// image from that device and invalidates it: the call is not valid after one).  The call never
// calls cudaMalloc, cudaFree or any other allocating routine: inputs are staged into the array
// with plain copies, the work counter and accumulators are cleared with a memset, and the result
// is copied back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "../../include/binodeg.h"
#include "bd_host.h"
#include "bd_internal.h"
#include "bd_kernels.cuh"
#include "bd_lifts.h"

namespace {

constexpr size_t kPointsOffset = 256;                                  // after the accumulators and counter
constexpr size_t kItemsOffset = 8192;                                  // after BD_NMAX x BD_KMAX points
constexpr size_t kItemsMax = BD_NOALLOC_MAX_ITEMS;
constexpr size_t kScratchBytes = kItemsOffset + kItemsMax * sizeof(bd::PackedItem);
static_assert(kPointsOffset >= sizeof(bd::DevAcc) + sizeof(unsigned int), "scratch header");
static_assert(kPointsOffset + sizeof(int64_t) * BD_NMAX * BD_KMAX <= kItemsOffset, "scratch points");
static_assert(kScratchBytes == BD_NOALLOC_SCRATCH_BYTES, "scratch size");

// [DevAcc accumulators][work counter] ... [points, N x K int64] ... [work list]
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;                     // one call at a time in this process
void* g_addr[256] = {};              // device address of g_scratch, per device ordinal
bd::Item g_host_items[kItemsMax];          // host-side work list (static, no heap)
bd::PackedItem g_host_packed[kItemsMax];   // the same, packed as the device reads it

int scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return bd::set_error(BD_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= 256) return bd::set_error(BD_ERR_ARG, "device ordinal above 255");
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);  // with `dev` current: that device's copy
    if (e != cudaSuccess || !p)
      return bd::set_error(BD_ERR_CUDA, e != cudaSuccess ? cudaGetErrorString(e) : "no symbol address");
    g_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_addr[dev]);
  return BD_OK;
}

}  // namespace

extern "C" int bd_volume_noalloc(const int64_t* points, int32_t npts, int32_t k, uint64_t seed,
                                 bd_volume_out* out) {
  if (!points || !out) return bd::set_error(BD_ERR_ARG, "NULL argument");
  if (k < 1 || k > BD_KMAX) return bd::set_error(BD_ERR_ARG, "k must be in [1, BD_KMAX]");
  if (npts < 1 || npts > BD_NMAX) return bd::set_error(BD_ERR_ARG, "npts must be in [1, BD_NMAX]");
  int64_t max_abs = 0;
  for (int64_t i = 0; i < (int64_t)npts * k; ++i) {
    if (points[i] >= ((int64_t)1 << 40) || points[i] <= -((int64_t)1 << 40))
      return bd::set_error(BD_ERR_ARG, "|coordinate| must be below 2^40");
    max_abs = std::max<int64_t>(max_abs, std::llabs(points[i]));
  }
  std::memset(out, 0, sizeof(*out));
  out->subsets = bd::binom(npts, k + 1);
  out->max_abs_coord = (int32_t)std::min<int64_t>(max_abs, INT32_MAX);
  if (npts < k + 1) {
    out->flags = BD_FLAG_DEGENERATE;
    return BD_OK;
  }
  double coord_bits = 0;
  const double bound = bd::hadamard_log2(points, nullptr, npts, k, (1 << 20) - 1, &coord_bits);
  const int path = bd::choose_path(coord_bits, bound);
  if (path < 0) return bd::set_error(BD_ERR_OVERFLOW, "Hadamard bound of the lifted minors exceeds 2^127");
  out->bound_bits = (int32_t)std::ceil(bound);

  std::lock_guard<std::mutex> lk(g_mu);
  unsigned char* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  bd::LaunchShape shape = bd::enum_shape(npts, k, path, false, 0, 0, sms > 0 ? sms : 1, &e);
  if (e != cudaSuccess) return bd::set_error(BD_ERR_CUDA, cudaGetErrorString(e));
  const bool five = path == bd::PATH_NARROW && k >= 4 && bd::prefer_five(points, npts, k, (uint64_t)shape.blocks * shape.warps);
  if (five) {  // the 5-D kernel's own occupancy
    shape = bd::enum_shape(npts, k, path, true, 0, 0, sms > 0 ? sms : 1, &e);
    if (e != cudaSuccess) return bd::set_error(BD_ERR_CUDA, cudaGetErrorString(e));
  }
  // the work list must fit the array: coarsen the split until it does (the coarsest list,
  // one prefix per first index, always fits)
  const uint64_t total = bd::binom(npts, k + 1);
  uint64_t thr = std::max<uint64_t>(256, total / ((uint64_t)shape.blocks * shape.warps * 4 + 1));
  size_t nitems = 0;
  while (!bd::build_items_into(npts, k, thr, bd::item_depth(k, path, five), g_host_items, kItemsMax, &nitems)) thr *= 4;

  cudaStream_t st = bd::thread_stream();
  bd::DevAcc* d_acc = reinterpret_cast<bd::DevAcc*>(base);
  unsigned int* d_counter = reinterpret_cast<unsigned int*>(base + sizeof(bd::DevAcc));
  int64_t* d_pts = reinterpret_cast<int64_t*>(base + kPointsOffset);
  bd::PackedItem* d_items = reinterpret_cast<bd::PackedItem*>(base + kItemsOffset);
  for (size_t i = 0; i < nitems; ++i) g_host_packed[i] = bd::pack_item(g_host_items[i]);
  // once work is queued, every return first waits for it, so that the array is idle whenever
  // the lock is free (a later call may use another stream)
  auto fail_idle = [&](int code, const char* msg) {
    cudaStreamSynchronize(st);
    return bd::set_error(code, msg);
  };
  e = cudaMemcpyAsync(d_pts, points, sizeof(int64_t) * npts * k, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_items, g_host_packed, sizeof(bd::PackedItem) * nitems, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail_idle(BD_ERR_CUDA, cudaGetErrorString(e));
  for (int attempt = 0; attempt < 8; ++attempt) {
    bd::DevAcc acc{};
    e = cudaMemsetAsync(base, 0, kPointsOffset, st);  // accumulators and work counter start at zero
    bd::EnumParams ep{};
    ep.pts = d_pts;
    ep.lifts = nullptr;
    ep.lift_seed = bd::lift_stream_seed(seed, (uint32_t)attempt);
    ep.items = d_items;
    ep.nitems = (int)nitems;
    ep.N = npts;
    ep.K = k;
    ep.five = five ? 1 : 0;
    ep.counter = d_counter;
    ep.acc = d_acc;
    if (e == cudaSuccess) e = bd::launch_enumerate(ep, shape, path, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&acc, d_acc, sizeof(acc), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_idle(BD_ERR_CUDA, cudaGetErrorString(e));
    if (acc.items_done != nitems) return bd::set_error(BD_ERR_CUDA, "enumeration did not process every work item");
    out->nvol_lo = acc.nvol_lo;
    out->nvol_hi = acc.nvol_hi;
    out->cells = acc.cells;
    out->singular = acc.singular;
    out->ties = acc.ties;
    out->relifts = attempt;
    out->flags = (path == bd::PATH_WIDE ? BD_FLAG_INT128 : 0) | ((acc.nvol_lo | acc.nvol_hi) == 0 ? BD_FLAG_DEGENERATE : 0);
    if (acc.ties == 0) return BD_OK;
  }
  return bd::set_error(BD_ERR_TIES, "every allowed lifting had ties");
}

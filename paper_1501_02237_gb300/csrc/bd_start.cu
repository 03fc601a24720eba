// Start solutions of the witness-set homotopy (Sec. 6): the cells come from the enumeration;
// one GPU thread prepares each cell (start_setup: exact inverse and Hermite diagonal of its
// exponent matrix, the right-hand sides from its generic coefficients), then one thread per
// solution writes it, and a third kernel checks every residual.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/binodeg.h"
#include "bd_host.h"
#include "bd_internal.h"
#include "bd_start.h"

namespace {

using bd::StartCell;

__global__ void k_start_prepare(const int64_t* pts, int npts, int k, const uint8_t* recs, int ncells,
                                uint64_t coef_seed, StartCell* cells, int32_t* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ncells) return;
  uint8_t idx[16];
  for (int t = 0; t < 16; ++t) idx[t] = recs[16 * i + t];
  status[i] = bd::start_setup(pts, npts, k, idx, coef_seed, cells[i]) ? 0 : 1;
}

// the cell holding global solution g: the last cell whose first solution is <= g
__device__ int cell_of(const unsigned long long* first, int ncells, unsigned long long g) {
  int lo = 0, hi = ncells - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (first[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void k_start_solutions(const StartCell* cells, const unsigned long long* first, int ncells, int k,
                                  unsigned long long total, double* out) {
  const unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int c = cell_of(first, ncells, g);
  bd::start_solution(cells[c], k, g - first[c], out + 2ull * k * g);
}

__global__ void k_start_residual(const StartCell* cells, const unsigned long long* first, int ncells, int k,
                                 unsigned long long total, const double* sols, unsigned long long* worst_bits) {
  const unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int c = cell_of(first, ncells, g);
  const double r = bd::start_residual(cells[c], k, sols + 2ull * k * g);
  // nonnegative doubles order like their bit patterns; NaN (a broken solution) sorts above all
  atomicMax(worst_bits, (unsigned long long)__double_as_longlong(r != r ? 1e300 : r));
}

// the cells of bd_cells as 16-byte records, lexicographic (retrying once with the exact count)
int device_cells(const int64_t* points, int32_t npts, int32_t k, uint64_t seed, std::vector<uint8_t>& recs,
                 size_t& n) {
  int64_t cap = 4096, count = 0;
  for (int pass = 0; pass < 2; ++pass) {
    const size_t c1 = (size_t)std::max<int64_t>(cap, 1);
    std::vector<uint8_t> packed(c1 * (k + 1));
    std::vector<int64_t> den(c1), al(c1 * k), be(2 * c1);
    bd_volume_out vol;
    const int rc = bd_cells(points, npts, k, seed, cap, packed.data(), den.data(), al.data(), be.data(), &count, &vol);
    if (rc == BD_OK) {
      n = (size_t)count;
      recs.assign(16 * std::max<size_t>(n, 1), 0);
      for (size_t i = 0; i < n; ++i) std::memcpy(&recs[16 * i], &packed[i * (k + 1)], (size_t)k + 1);
      return BD_OK;
    }
    if (rc != BD_ERR_ARG || count <= cap) return rc;
    cap = count;
  }
  return bd::set_error(BD_ERR_ARG, "cell count changed between calls");
}

}  // namespace

extern "C" {

int bd_start_solutions(const int64_t* points, int32_t npts, int32_t k, uint64_t seed, uint64_t coef_seed,
                       int64_t capacity, double* sols, int32_t sols_on_device, int64_t* count, double* max_residual) {
  if (!count || capacity < 0 || (capacity > 0 && !sols)) return bd::set_error(BD_ERR_ARG, "NULL argument");
  *count = 0;
  if (k < 1 || k > BD_KMAX || npts < k + 1) return bd::set_error(BD_ERR_ARG, "need 1 <= k <= BD_KMAX and k+1 points");
  std::vector<uint8_t> recs;
  size_t n = 0;
  int rc = device_cells(points, npts, k, seed, recs, n);
  if (rc) return rc;
  if (n == 0) return BD_OK;
  cudaStream_t st = bd::thread_stream();
  int64_t* d_pts = nullptr;
  uint8_t* d_recs = nullptr;
  StartCell* d_cells = nullptr;
  int32_t* d_status = nullptr;
  unsigned long long *d_first = nullptr, *d_worst = nullptr;
  double* d_sols = sols_on_device ? sols : nullptr;
  auto release = [&]() {
    cudaFree(d_pts);
    cudaFree(d_recs);
    cudaFree(d_cells);
    cudaFree(d_status);
    cudaFree(d_first);
    cudaFree(d_worst);
    if (!sols_on_device) cudaFree(d_sols);
    d_sols = nullptr;
  };
  auto fail_cuda = [&](cudaError_t e) {
    release();
    return bd::cuda_error(e);
  };
  cudaError_t e = bd::dev_malloc(&d_pts, sizeof(int64_t) * npts * k);
  if (e == cudaSuccess) e = bd::dev_malloc(&d_recs, 16 * n);
  if (e == cudaSuccess) e = bd::dev_malloc(&d_cells, sizeof(StartCell) * n);
  if (e == cudaSuccess) e = bd::dev_malloc(&d_status, sizeof(int32_t) * n);
  if (e == cudaSuccess) e = bd::dev_malloc(&d_first, sizeof(unsigned long long) * n);
  if (e == cudaSuccess) e = bd::dev_malloc(&d_worst, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_pts, points, sizeof(int64_t) * npts * k, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_recs, recs.data(), 16 * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_start_prepare<<<(unsigned int)((n + 63) / 64), 64, 0, st>>>(d_pts, npts, k, d_recs, (int)n, coef_seed, d_cells,
                                                                 d_status);
    e = cudaGetLastError();
  }
  // the solution count of each cell is |det|: the offsets are a prefix sum on the host
  std::vector<int32_t> status(n);
  std::vector<int64_t> dets(n);
  if (e == cudaSuccess) e = cudaMemcpyAsync(status.data(), d_status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(dets.data(), sizeof(int64_t), &d_cells->det, sizeof(StartCell), sizeof(int64_t), n,
                          cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail_cuda(e);
  std::vector<unsigned long long> first(n);
  uint64_t total = 0;
  for (size_t i = 0; i < n; ++i) {
    if (status[i]) {
      release();
      return bd::set_error(BD_ERR_OVERFLOW, "a start system's exact data leaves 64 bits");
    }
    first[i] = total;
    total += (uint64_t)(dets[i] < 0 ? -dets[i] : dets[i]);
  }
  *count = (int64_t)total;
  if (total > (uint64_t)capacity) {
    release();
    return bd::set_error(BD_ERR_ARG, "capacity is below the number of solutions (count holds it)");
  }
  if (!sols_on_device) e = bd::dev_malloc(&d_sols, sizeof(double) * 2 * k * total);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_first, first.data(), sizeof(unsigned long long) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_worst, 0, sizeof(unsigned long long), st);
  const unsigned int threads = 128;
  const unsigned long long blocks = (total + threads - 1) / threads;
  if (e == cudaSuccess) {
    k_start_solutions<<<(unsigned int)blocks, threads, 0, st>>>(d_cells, d_first, (int)n, k, total, d_sols);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && max_residual) {
    k_start_residual<<<(unsigned int)blocks, threads, 0, st>>>(d_cells, d_first, (int)n, k, total, d_sols, d_worst);
    e = cudaGetLastError();
  }
  unsigned long long worst = 0;
  if (e == cudaSuccess && max_residual) e = cudaMemcpyAsync(&worst, d_worst, sizeof(worst), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && !sols_on_device)
    e = cudaMemcpyAsync(sols, d_sols, sizeof(double) * 2 * k * total, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail_cuda(e);
  release();
  if (max_residual) {
    double wv;
    std::memcpy(&wv, &worst, sizeof(wv));
    *max_residual = wv;
  }
  return BD_OK;
}

int bd_host_start_solutions(const int64_t* points, const int64_t* lifts, int32_t npts, int32_t k, uint64_t coef_seed,
                            int64_t capacity, double* sols, int64_t* count, double* max_residual) {
  if (!count || capacity < 0 || (capacity > 0 && !sols)) return bd::set_error(BD_ERR_ARG, "NULL argument");
  *count = 0;
  if (k < 1 || k > BD_KMAX || npts < k + 1) return bd::set_error(BD_ERR_ARG, "need 1 <= k <= BD_KMAX and k+1 points");
  int64_t cap = 4096, nc = 0;
  std::vector<uint8_t> packed;
  int rc = BD_OK;
  for (int pass = 0; pass < 2; ++pass) {
    const size_t c1 = (size_t)std::max<int64_t>(cap, 1);
    packed.assign(c1 * (k + 1), 0);
    std::vector<int64_t> den(c1), al(c1 * k), be(2 * c1);
    rc = bd_host_cells(points, lifts, npts, k, cap, packed.data(), den.data(), al.data(), be.data(), &nc);
    if (rc != BD_ERR_ARG || nc <= cap) break;
    cap = nc;
  }
  if (rc) return rc;
  std::vector<StartCell> cells((size_t)nc);
  std::vector<uint64_t> first((size_t)nc);
  uint64_t total = 0;
  for (int64_t i = 0; i < nc; ++i) {
    uint8_t idx[16] = {};
    std::memcpy(idx, &packed[(size_t)i * (k + 1)], (size_t)k + 1);
    if (!bd::start_setup(points, npts, k, idx, coef_seed, cells[i]))
      return bd::set_error(BD_ERR_OVERFLOW, "a start system's exact data leaves 64 bits");
    first[i] = total;
    total += (uint64_t)(cells[i].det < 0 ? -cells[i].det : cells[i].det);
  }
  *count = (int64_t)total;
  if (total > (uint64_t)capacity) return bd::set_error(BD_ERR_ARG, "capacity is below the number of solutions (count holds it)");
  // cells dealt round-robin to the host threads, each with its own worst residual
  const int nt = (int)std::max<int64_t>(1, std::min<int64_t>(nc, std::max(1u, std::thread::hardware_concurrency())));
  std::vector<double> worst_of(nt, 0.0);
  auto work = [&](int w) {
    double worst = 0;
    for (int64_t c = w; c < nc; c += nt) {
      const uint64_t m = (uint64_t)(cells[c].det < 0 ? -cells[c].det : cells[c].det);
      for (uint64_t t = 0; t < m; ++t) {
        double* y = sols + 2ull * k * (first[c] + t);
        bd::start_solution(cells[c], k, t, y);
        const double r = bd::start_residual(cells[c], k, y);
        worst = (r != r) ? 1e300 : (r > worst ? r : worst);
      }
    }
    worst_of[w] = worst;
  };
  std::vector<std::thread> th;
  for (int w = 1; w < nt; ++w) th.emplace_back(work, w);
  work(0);
  for (auto& t : th) t.join();
  if (max_residual) *max_residual = *std::max_element(worst_of.begin(), worst_of.end());
  return BD_OK;
}

}  // extern "C"

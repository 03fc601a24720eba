// Start solutions of the witness-set homotopy (Sec. 6): cells from the enumeration, per-cell
// preparation on the host (bd_host.cpp: start_setup), then one GPU thread per solution.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "../../include/binodeg.h"
#include "bd_host.h"
#include "bd_internal.h"
#include "bd_start.h"

// ---- per-cell preparation on the host -----------------------------------------------------

namespace {

using bd::i128;

// exact determinant of a k x k integer matrix (fraction-free elimination, checked 128-bit)
bool det128(std::vector<i128> a, int k, i128& det) {
  if (k == 0) {
    det = 1;
    return true;
  }
  i128 prev = 1;
  int sign = 1;
  for (int c = 0; c < k; ++c) {
    int p = -1;
    for (int r = c; r < k; ++r)
      if (a[(size_t)r * k + c] != 0) { p = r; break; }
    if (p < 0) { det = 0; return true; }
    if (p != c) {
      for (int j = 0; j < k; ++j) std::swap(a[(size_t)c * k + j], a[(size_t)p * k + j]);
      sign = -sign;
    }
    for (int r = c + 1; r < k; ++r) {
      for (int j = c + 1; j < k; ++j) {
        i128 x, y;
        if (__builtin_mul_overflow(a[(size_t)r * k + j], a[(size_t)c * k + c], &x) ||
            __builtin_mul_overflow(a[(size_t)r * k + c], a[(size_t)c * k + j], &y))
          return false;
        a[(size_t)r * k + j] = (x - y) / prev;  // exact (Bareiss)
      }
      a[(size_t)r * k + c] = 0;
    }
    prev = a[(size_t)c * k + c];
  }
  det = sign * a[(size_t)(k - 1) * k + (k - 1)];
  return true;
}

i128 iabs128(i128 x) { return x < 0 ? -x : x; }

// determinant of a k x k complex matrix (Gaussian elimination with partial pivoting)
std::complex<double> cdet(std::vector<std::complex<double>> a, int k) {
  std::complex<double> d = 1;
  for (int c = 0; c < k; ++c) {
    int p = c;
    for (int r = c + 1; r < k; ++r)
      if (std::abs(a[(size_t)r * k + c]) > std::abs(a[(size_t)p * k + c])) p = r;
    if (a[(size_t)p * k + c] == 0.0) return 0;
    if (p != c) {
      for (int j = 0; j < k; ++j) std::swap(a[(size_t)c * k + j], a[(size_t)p * k + j]);
      d = -d;
    }
    d *= a[(size_t)c * k + c];
    for (int r = c + 1; r < k; ++r) {
      const std::complex<double> f = a[(size_t)r * k + c] / a[(size_t)c * k + c];
      for (int j = c; j < k; ++j) a[(size_t)r * k + j] -= f * a[(size_t)c * k + j];
    }
  }
  return d;
}

}  // namespace

namespace bd {

bool start_setup(const int64_t* pts, int npts, int k, const uint8_t* idx, uint64_t coef_seed, StartCell& out) {
  out = StartCell{};
  // the exponent matrix: rows a_j - a_k
  std::vector<i128> E((size_t)k * k);
  for (int j = 0; j < k; ++j)
    for (int c = 0; c < k; ++c) E[(size_t)j * k + c] = (i128)pts[(size_t)idx[j] * k + c] - pts[(size_t)idx[k] * k + c];
  i128 det;
  if (!det128(E, k, det) || det == 0 || iabs128(det) >= ((i128)1 << 62)) return false;
  out.det = (int64_t)det;
  for (int j = 0; j < k; ++j)
    for (int c = 0; c < k; ++c) {
      if (iabs128(E[(size_t)j * k + c]) >= ((i128)1 << 31)) return false;
      out.E[j * k + c] = (int32_t)E[(size_t)j * k + c];
    }
  // adj(E)[i][j] = (-1)^(i+j) det(E without row j and column i)
  if (k == 1) {
    out.adj[0] = 1;
  } else {
    std::vector<i128> minor((size_t)(k - 1) * (k - 1));
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) {
        size_t t = 0;
        for (int r = 0; r < k; ++r)
          if (r != j)
            for (int c = 0; c < k; ++c)
              if (c != i) minor[t++] = E[(size_t)r * k + c];
        i128 m;
        if (!det128(minor, k - 1, m) || iabs128(m) >= ((i128)1 << 62)) return false;
        out.adj[i * k + j] = (int64_t)(((i + j) & 1) ? -m : m);
      }
  }
  // diagonal of the lower-triangular column Hermite form (column operations only)
  std::vector<i128> H(E);
  auto col_axpy = [&](int dst, int src, i128 q) -> bool {  // column dst -= q column src
    for (int r = 0; r < k; ++r) {
      i128 t;
      if (__builtin_mul_overflow(q, H[(size_t)r * k + src], &t)) return false;
      H[(size_t)r * k + dst] -= t;
      if (iabs128(H[(size_t)r * k + dst]) >= ((i128)1 << 100)) return false;
    }
    return true;
  };
  auto col_swap = [&](int a, int b) {
    for (int r = 0; r < k; ++r) std::swap(H[(size_t)r * k + a], H[(size_t)r * k + b]);
  };
  uint64_t count = 1;
  for (int i = 0; i < k; ++i) {
    for (int j = i + 1; j < k; ++j) {
      while (H[(size_t)i * k + j] != 0) {
        if (H[(size_t)i * k + i] == 0 || iabs128(H[(size_t)i * k + j]) < iabs128(H[(size_t)i * k + i])) col_swap(i, j);
        if (H[(size_t)i * k + j] == 0) break;
        if (!col_axpy(j, i, H[(size_t)i * k + j] / H[(size_t)i * k + i])) return false;
      }
    }
    if (H[(size_t)i * k + i] < 0)
      for (int r = 0; r < k; ++r) H[(size_t)r * k + i] = -H[(size_t)r * k + i];
    if (H[(size_t)i * k + i] <= 0) return false;
    out.h[i] = (int64_t)H[(size_t)i * k + i];
    count *= (uint64_t)out.h[i];
  }
  if ((i128)count != iabs128(det)) return false;
  // the right-hand sides: b_j = kappa_j / kappa_k, kappa_j = (-1)^j det(C without column j)
  const uint64_t cs = coef_stream_seed(coef_seed);
  std::vector<std::complex<double>> C((size_t)k * (k + 1));
  for (int i = 0; i < k; ++i)
    for (int j = 0; j <= k; ++j) {
      const double th = 6.283185307179586 * coef_turns(cs, npts, i, idx[j]);
      C[(size_t)i * (k + 1) + j] = std::complex<double>(std::cos(th), std::sin(th));
    }
  std::vector<std::complex<double>> kappa(k + 1), sub((size_t)k * k);
  for (int j = 0; j <= k; ++j) {
    for (int i = 0; i < k; ++i)
      for (int c = 0, t = 0; c <= k; ++c)
        if (c != j) sub[(size_t)i * k + t++] = C[(size_t)i * (k + 1) + c];
    kappa[j] = ((j & 1) ? -1.0 : 1.0) * cdet(sub, k);
  }
  if (kappa[k] == 0.0) return false;
  for (int j = 0; j < k; ++j) {
    const std::complex<double> b = kappa[j] / kappa[k];
    if (b == 0.0) return false;
    out.b_re[j] = b.real();
    out.b_im[j] = b.imag();
  }
  // E^-1 log b = adj log b / det (real and imaginary parts)
  for (int i = 0; i < k; ++i) {
    double re = 0, im = 0;
    for (int j = 0; j < k; ++j) {
      const std::complex<double> b(out.b_re[j], out.b_im[j]);
      re += (double)out.adj[i * k + j] * std::log(std::abs(b));
      im += (double)out.adj[i * k + j] * std::arg(b);
    }
    out.base_re[i] = re / (double)out.det;
    out.base_im[i] = im / (double)out.det;
  }
  return true;
}

}  // namespace bd

namespace {

using bd::StartCell;

// the cell holding global solution g: the last cell whose first solution is <= g
__device__ int cell_of(const StartCell* cells, int ncells, unsigned long long g) {
  int lo = 0, hi = ncells - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (cells[mid].first <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void k_start_solutions(const StartCell* cells, int ncells, int k, unsigned long long total, double* out) {
  const unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int c = cell_of(cells, ncells, g);
  bd::start_solution(cells[c], k, g - cells[c].first, out + 2ull * k * g);
}

__global__ void k_start_residual(const StartCell* cells, int ncells, int k, unsigned long long total,
                                 const double* sols, unsigned long long* worst_bits) {
  const unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int c = cell_of(cells, ncells, g);
  const double r = bd::start_residual(cells[c], k, sols + 2ull * k * g);
  // nonnegative doubles order like their bit patterns; NaN (a broken solution) sorts above all
  atomicMax(worst_bits, (unsigned long long)__double_as_longlong(r != r ? 1e300 : r));
}

// cells (lexicographic) from the given cell records, prepared; total = sum of |det|
int prepare(const int64_t* points, int32_t npts, int32_t k, const std::vector<uint8_t>& recs, size_t ncells,
            uint64_t coef_seed, std::vector<StartCell>& cells, uint64_t& total) {
  cells.resize(ncells);
  total = 0;
  for (size_t i = 0; i < ncells; ++i) {
    if (!bd::start_setup(points, npts, k, &recs[i * (k + 1)], coef_seed, cells[i]))
      return bd::set_error(BD_ERR_OVERFLOW, "a start system's exact data leaves 64 bits");
    cells[i].first = total;
    total += (uint64_t)(cells[i].det < 0 ? -cells[i].det : cells[i].det);
  }
  return BD_OK;
}

// the cells of bd_cells (retrying once with the exact count)
int device_cells(const int64_t* points, int32_t npts, int32_t k, uint64_t seed, std::vector<uint8_t>& recs,
                 size_t& n) {
  int64_t cap = 4096, count = 0;
  for (int pass = 0; pass < 2; ++pass) {
    recs.assign((size_t)std::max<int64_t>(cap, 1) * (k + 1), 0);
    std::vector<int64_t> den((size_t)std::max<int64_t>(cap, 1)), al((size_t)std::max<int64_t>(cap, 1) * k),
        be(2 * (size_t)std::max<int64_t>(cap, 1));
    bd_volume_out vol;
    const int rc = bd_cells(points, npts, k, seed, cap, recs.data(), den.data(), al.data(), be.data(), &count, &vol);
    if (rc == BD_OK) {
      n = (size_t)count;
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
  if (k < 1 || npts < k + 1) return bd::set_error(BD_ERR_ARG, "need k >= 1 and at least k+1 points");
  std::vector<uint8_t> recs;
  size_t n = 0;
  int rc = device_cells(points, npts, k, seed, recs, n);
  if (rc) return rc;
  std::vector<StartCell> cells;
  uint64_t total = 0;
  rc = prepare(points, npts, k, recs, n, coef_seed, cells, total);
  if (rc) return rc;
  *count = (int64_t)total;
  if (total > (uint64_t)capacity) return bd::set_error(BD_ERR_ARG, "capacity is below the number of solutions (count holds it)");
  if (total == 0) return BD_OK;
  cudaStream_t st = bd::thread_stream();
  StartCell* d_cells = nullptr;
  double* d_sols = sols_on_device ? sols : nullptr;
  unsigned long long* d_worst = nullptr;
  auto release = [&]() {
    cudaFree(d_cells);
    if (!sols_on_device) cudaFree(d_sols);
    cudaFree(d_worst);
  };
  cudaError_t e = cudaMalloc(&d_cells, sizeof(StartCell) * n);
  if (e == cudaSuccess && !sols_on_device) e = cudaMalloc(&d_sols, sizeof(double) * 2 * k * total);
  if (e == cudaSuccess) e = cudaMalloc(&d_worst, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_cells, cells.data(), sizeof(StartCell) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_worst, 0, sizeof(unsigned long long), st);
  const unsigned int threads = 128;
  const unsigned long long blocks = (total + threads - 1) / threads;
  if (e == cudaSuccess) {
    k_start_solutions<<<(unsigned int)blocks, threads, 0, st>>>(d_cells, (int)n, k, total, d_sols);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && max_residual) {
    k_start_residual<<<(unsigned int)blocks, threads, 0, st>>>(d_cells, (int)n, k, total, d_sols, d_worst);
    e = cudaGetLastError();
  }
  unsigned long long worst = 0;
  if (e == cudaSuccess && max_residual) e = cudaMemcpyAsync(&worst, d_worst, sizeof(worst), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && !sols_on_device)
    e = cudaMemcpyAsync(sols, d_sols, sizeof(double) * 2 * k * total, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  release();
  if (e != cudaSuccess) return bd::set_error(BD_ERR_CUDA, cudaGetErrorString(e));
  if (max_residual) {
    double w;
    std::memcpy(&w, &worst, sizeof(w));
    *max_residual = w;
  }
  return BD_OK;
}

int bd_host_start_solutions(const int64_t* points, const int64_t* lifts, int32_t npts, int32_t k, uint64_t coef_seed,
                            int64_t capacity, double* sols, int64_t* count, double* max_residual) {
  if (!count || capacity < 0 || (capacity > 0 && !sols)) return bd::set_error(BD_ERR_ARG, "NULL argument");
  *count = 0;
  if (k < 1 || npts < k + 1) return bd::set_error(BD_ERR_ARG, "need k >= 1 and at least k+1 points");
  int64_t cap = 4096, nc = 0;
  std::vector<uint8_t> recs;
  int rc = BD_OK;
  for (int pass = 0; pass < 2; ++pass) {
    const size_t c1 = (size_t)std::max<int64_t>(cap, 1);
    recs.assign(c1 * (k + 1), 0);
    std::vector<int64_t> den(c1), al(c1 * k), be(2 * c1);
    rc = bd_host_cells(points, lifts, npts, k, cap, recs.data(), den.data(), al.data(), be.data(), &nc);
    if (rc != BD_ERR_ARG || nc <= cap) break;
    cap = nc;
  }
  if (rc) return rc;
  std::vector<StartCell> cells;
  uint64_t total = 0;
  rc = prepare(points, npts, k, recs, (size_t)nc, coef_seed, cells, total);
  if (rc) return rc;
  *count = (int64_t)total;
  if (total > (uint64_t)capacity) return bd::set_error(BD_ERR_ARG, "capacity is below the number of solutions (count holds it)");
  double worst = 0;
  for (size_t c = 0; c < cells.size(); ++c) {
    const uint64_t m = (uint64_t)(cells[c].det < 0 ? -cells[c].det : cells[c].det);
    for (uint64_t t = 0; t < m; ++t) {
      double* y = sols + 2ull * k * (cells[c].first + t);
      bd::start_solution(cells[c], k, t, y);
      const double r = bd::start_residual(cells[c], k, y);
      worst = (r != r || r > worst) ? (r != r ? 1e300 : r) : worst;
    }
  }
  if (max_residual) *max_residual = worst;
  return BD_OK;
}

}  // extern "C"

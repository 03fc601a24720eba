// The learned cost model: a 16 -> 64 -> 64 -> 1 fully connected network with ReLU, FP32,
// trained on the GPU by these kernels (forward, backward with per-block gradient sums, Adam).
// It predicts log2 of a system's enumeration cost from integer-derived features; the batch
// engine uses the prediction only to size and order work items (never for the answer).
//
// Parameter layout (5313 floats): W1[64][16], b1[64], W2[64][64], b2[64], W3[64], b3.
// Inputs are standardized with a stored mean and standard deviation per feature.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/binodeg.h"
#include "bd_internal.h"

namespace {

constexpr int F = BD_FEATURES, H = 64;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * F, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H, NPARAM = OFF_B3 + 1;
static_assert(NPARAM == BD_MLP_PARAMS, "parameter count");
constexpr int SPB = 4;  // samples per block: 4 x 64 = 256 threads (static shared memory stays below 48 KB)

// one block: SPB samples, thread (s, j) owns hidden unit j of sample s
__device__ void forward_block(const float* __restrict__ w, const float* __restrict__ X, const float* __restrict__ mean,
                              const float* __restrict__ stdv, int n, int base, float (*x)[F], float (*h1)[H],
                              float (*h2)[H], float* out) {
  const int s = threadIdx.x / H, j = threadIdx.x % H;
  const int idx = base + s;
  if (j < F) x[s][j] = idx < n ? (X[(size_t)idx * F + j] - mean[j]) / stdv[j] : 0.f;
  __syncthreads();
  float a = w[OFF_B1 + j];
  for (int f = 0; f < F; ++f) a = fmaf(w[OFF_W1 + j * F + f], x[s][f], a);
  h1[s][j] = fmaxf(a, 0.f);
  __syncthreads();
  float b = w[OFF_B2 + j];
  for (int i = 0; i < H; ++i) b = fmaf(w[OFF_W2 + j * H + i], h1[s][i], b);
  h2[s][j] = fmaxf(b, 0.f);
  __syncthreads();
  // output: warp-level sum of W3[j] h2[s][j] over the two warps of the sample
  float c = w[OFF_W3 + j] * h2[s][j];
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  __shared__ float part[SPB * 2];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
  __syncthreads();
  if (j == 0) out[s] = part[2 * s] + part[2 * s + 1] + w[OFF_B3];
  __syncthreads();
}

__global__ void __launch_bounds__(SPB * H) k_mlp_forward(const float* w, const float* X, const float* mean,
                                                         const float* stdv, int n, float* y) {
  __shared__ float sw[NPARAM];
  __shared__ float x[SPB][F], h1[SPB][H], h2[SPB][H], out[SPB];
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) sw[i] = w[i];
  __syncthreads();
  for (int base = blockIdx.x * SPB; base < n; base += gridDim.x * SPB) {
    forward_block(sw, X, mean, stdv, n, base, x, h1, h2, out);
    if (threadIdx.x < SPB && base + (int)threadIdx.x < n) y[base + threadIdx.x] = out[threadIdx.x];
    __syncthreads();
  }
}

// gradient of L = (1/count) sum_i (f(x_i) - y_i)^2 over samples [0, n) of this launch, summed
// per block in shared memory and added to g once; loss sum added to *loss
__global__ void __launch_bounds__(SPB * H) k_mlp_backward(const float* w, const float* X, const float* Y,
                                                          const float* mean, const float* stdv, int n, float inv_count,
                                                          float* g, float* loss) {
  __shared__ float sw[NPARAM];
  __shared__ float sg[NPARAM];
  __shared__ float x[SPB][F], h1[SPB][H], h2[SPB][H], out[SPB], d2[SPB][H];
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) {
    sw[i] = w[i];
    sg[i] = 0.f;
  }
  __syncthreads();
  const int s = threadIdx.x / H, j = threadIdx.x % H;
  float lsum = 0.f;
  for (int base = blockIdx.x * SPB; base < n; base += gridDim.x * SPB) {
    forward_block(sw, X, mean, stdv, n, base, x, h1, h2, out);
    const int idx = base + s;
    const bool valid = idx < n;
    const float r = valid ? out[s] - Y[idx] : 0.f;
    const float dout = 2.f * r * inv_count;
    if (j == 0 && valid) lsum += r * r;
    // layer 3
    const float dh2 = (h2[s][j] > 0.f) ? dout * sw[OFF_W3 + j] : 0.f;
    d2[s][j] = dh2;
    __syncthreads();
    // thread (s, j) now owns hidden unit j of layer 1 for sample s: d h1_j = sum_k W2[k][j] dh2_k
    float dh1 = 0.f;
    for (int k = 0; k < H; ++k) dh1 = fmaf(sw[OFF_W2 + k * H + j], d2[s][k], dh1);
    dh1 = (h1[s][j] > 0.f) ? dh1 : 0.f;
    // accumulate parameter gradients over the block's samples (one thread per output row)
    __syncthreads();
    if (s == 0) {
      for (int t = 0; t < SPB; ++t) {
        if (base + t >= n) break;
        const float dt2 = d2[t][j];
        sg[OFF_W3 + j] += 2.f * (out[t] - Y[base + t]) * inv_count * h2[t][j];
        sg[OFF_B2 + j] += dt2;
        for (int i = 0; i < H; ++i) sg[OFF_W2 + j * H + i] += dt2 * h1[t][i];
        if (j == 0) sg[OFF_B3] += 2.f * (out[t] - Y[base + t]) * inv_count;
      }
    }
    // layer 1 rows: thread (s, j) holds dh1 for sample s; reduce over samples with shared atomics
    atomicAdd(&sg[OFF_B1 + j], dh1);
    for (int f = 0; f < F; ++f) atomicAdd(&sg[OFF_W1 + j * F + f], dh1 * x[s][f]);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) atomicAdd(&g[i], sg[i]);
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, lsum);
}

// Adam (Kingma & Ba 2015) with bias correction; clears the gradient for the next step
__global__ void k_mlp_adam(float* w, float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps,
                           float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    g[i] = 0.f;
  }
}

uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

struct bd_mlp {
  float* d_w = nullptr;  // params, grads, adam m, adam v, mean, std, loss
  float* d_g = nullptr;
  float* d_m = nullptr;
  float* d_v = nullptr;
  float* d_norm = nullptr;  // mean[F], std[F]
  float* d_loss = nullptr;
  int step = 0;
};

namespace {

int cuda_err(cudaError_t e) { return bd::cuda_error(e); }

int upload_xy(const float* X, const float* y, int count, float** dX, float** dY, cudaStream_t st) {
  cudaError_t e = bd::dev_malloc(dX, sizeof(float) * (size_t)count * F);
  if (e == cudaSuccess && y) e = bd::dev_malloc(dY, sizeof(float) * (size_t)count);
  if (e == cudaSuccess) e = cudaMemcpyAsync(*dX, X, sizeof(float) * (size_t)count * F, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && y) e = cudaMemcpyAsync(*dY, y, sizeof(float) * (size_t)count, cudaMemcpyHostToDevice, st);
  return e == cudaSuccess ? BD_OK : cuda_err(e);
}

}  // namespace

extern "C" {

int bd_mlp_create(uint64_t seed, bd_mlp** out) {
  if (!out) return bd::set_error(BD_ERR_ARG, "NULL argument");
  bd_mlp* m = new (std::nothrow) bd_mlp();
  if (!m) return bd::set_error(BD_ERR_NOMEM, "host allocation");
  cudaError_t e = bd::dev_malloc(&m->d_w, sizeof(float) * NPARAM * 4 + sizeof(float) * (2 * F + 1));
  if (e != cudaSuccess) {
    delete m;
    return cuda_err(e);
  }
  m->d_g = m->d_w + NPARAM;
  m->d_m = m->d_g + NPARAM;
  m->d_v = m->d_m + NPARAM;
  m->d_norm = m->d_v + NPARAM;
  m->d_loss = m->d_norm + 2 * F;
  // He initialisation from a counter-based generator: uniform(-a, a), a = sqrt(6 / fan_in)
  std::vector<float> w(NPARAM, 0.f);
  auto uni = [&](uint64_t i) { return (float)((mix64(seed * 0x9E3779B97F4A7C15ull + i) >> 11) * 0x1.0p-53) * 2.f - 1.f; };
  for (int i = 0; i < H * F; ++i) w[OFF_W1 + i] = uni(i) * sqrtf(6.f / F);
  for (int i = 0; i < H * H; ++i) w[OFF_W2 + i] = uni(100000 + i) * sqrtf(6.f / H);
  for (int i = 0; i < H; ++i) w[OFF_W3 + i] = uni(200000 + i) * sqrtf(6.f / H);
  std::vector<float> rest(NPARAM * 3 + 2 * F + 1, 0.f);
  for (int f = 0; f < F; ++f) rest[NPARAM * 3 + F + f] = 1.f;  // std = 1
  e = cudaMemcpy(m->d_w, w.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->d_g, rest.data(), sizeof(float) * rest.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(m->d_w);
    delete m;
    return cuda_err(e);
  }
  *out = m;
  return BD_OK;
}

int bd_mlp_destroy(bd_mlp* m) {
  if (!m) return BD_OK;
  cudaFree(m->d_w);
  delete m;
  return BD_OK;
}

int bd_mlp_get_params(const bd_mlp* m, float* params, float* norm) {
  if (!m || !params) return bd::set_error(BD_ERR_ARG, "NULL argument");
  cudaError_t e = cudaMemcpy(params, m->d_w, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && norm) e = cudaMemcpy(norm, m->d_norm, sizeof(float) * 2 * F, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? BD_OK : cuda_err(e);
}

int bd_mlp_set_params(bd_mlp* m, const float* params, const float* norm) {
  if (!m || !params) return bd::set_error(BD_ERR_ARG, "NULL argument");
  for (int f = 0; norm && f < F; ++f)
    if (!(norm[F + f] > 0.f)) return bd::set_error(BD_ERR_ARG, "standard deviations must be positive");
  cudaError_t e = cudaMemcpy(m->d_w, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && norm) e = cudaMemcpy(m->d_norm, norm, sizeof(float) * 2 * F, cudaMemcpyHostToDevice);
  return e == cudaSuccess ? BD_OK : cuda_err(e);
}

int bd_mlp_predict(bd_mlp* m, const float* X, int32_t count, float* y) {
  if (!m || !X || !y || count < 0) return bd::set_error(BD_ERR_ARG, "bad argument");
  if (count == 0) return BD_OK;
  cudaStream_t st = bd::thread_stream();
  float *dX = nullptr, *dY = nullptr;
  int rc = upload_xy(X, nullptr, count, &dX, &dY, st);
  cudaError_t e = cudaSuccess;
  if (!rc) e = bd::dev_malloc(&dY, sizeof(float) * count);
  if (!rc && e == cudaSuccess) {
    const int blocks = std::min(1024, (count + SPB - 1) / SPB);
    k_mlp_forward<<<blocks, SPB * H, 0, st>>>(m->d_w, dX, m->d_norm, m->d_norm + F, count, dY);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(y, dY, sizeof(float) * count, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFree(dX);
  cudaFree(dY);
  if (rc) return rc;
  return e == cudaSuccess ? BD_OK : cuda_err(e);
}

int bd_mlp_gradient(bd_mlp* m, const float* X, const float* y, int32_t count, float* grad, float* loss) {
  if (!m || !X || !y || !grad || count <= 0) return bd::set_error(BD_ERR_ARG, "bad argument");
  cudaStream_t st = bd::thread_stream();
  float *dX = nullptr, *dY = nullptr;
  int rc = upload_xy(X, y, count, &dX, &dY, st);
  cudaError_t e = cudaSuccess;
  if (!rc) {
    e = cudaMemsetAsync(m->d_g, 0, sizeof(float) * NPARAM, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->d_loss, 0, sizeof(float), st);
    const int blocks = std::min(256, (count + SPB - 1) / SPB);
    if (e == cudaSuccess)
      k_mlp_backward<<<blocks, SPB * H, 0, st>>>(m->d_w, dX, dY, m->d_norm, m->d_norm + F, count, 1.f / count, m->d_g,
                                                  m->d_loss);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(grad, m->d_g, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, st);
    float l = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l, m->d_loss, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (loss) *loss = l / count;
    if (e == cudaSuccess) e = cudaMemsetAsync(m->d_g, 0, sizeof(float) * NPARAM, st);
  }
  cudaFree(dX);
  cudaFree(dY);
  if (rc) return rc;
  return e == cudaSuccess ? BD_OK : cuda_err(e);
}

int bd_mlp_train(bd_mlp* m, const float* X, const float* y, int32_t count, int32_t epochs, int32_t batch, float lr,
                 uint64_t seed, float* final_loss) {
  if (!m || !X || !y || count <= 0 || epochs < 0 || batch <= 0 || !(lr > 0.f)) return bd::set_error(BD_ERR_ARG, "bad argument");
  cudaStream_t st = bd::thread_stream();
  // feature standardisation from the training set
  std::vector<float> norm(2 * F, 0.f);
  for (int f = 0; f < F; ++f) {
    double s = 0, s2 = 0;
    for (int i = 0; i < count; ++i) {
      const double v = X[(size_t)i * F + f];
      s += v;
      s2 += v * v;
    }
    const double mu = s / count, var = std::max(0.0, s2 / count - mu * mu);
    norm[f] = (float)mu;
    norm[F + f] = (float)std::max(1e-3, std::sqrt(var));
  }
  cudaError_t e = cudaMemcpyAsync(m->d_norm, norm.data(), sizeof(float) * 2 * F, cudaMemcpyHostToDevice, st);
  // per epoch the samples are permuted on the host (seeded) and uploaded in that order
  std::vector<float> Xp((size_t)count * F), yp(count);
  std::vector<int> perm(count);
  for (int i = 0; i < count; ++i) perm[i] = i;
  float *dX = nullptr, *dY = nullptr;
  if (e == cudaSuccess) e = bd::dev_malloc(&dX, sizeof(float) * Xp.size());
  if (e == cudaSuccess) e = bd::dev_malloc(&dY, sizeof(float) * count);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->d_g, 0, sizeof(float) * NPARAM, st);
  float lsum = 0;
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    for (int i = count - 1; i > 0; --i) {
      const int j = (int)(mix64(seed ^ ((uint64_t)ep << 32) ^ (uint64_t)i) % (uint64_t)(i + 1));
      std::swap(perm[i], perm[j]);
    }
    for (int i = 0; i < count; ++i) {
      std::memcpy(&Xp[(size_t)i * F], &X[(size_t)perm[i] * F], sizeof(float) * F);
      yp[i] = y[perm[i]];
    }
    e = cudaMemcpyAsync(dX, Xp.data(), sizeof(float) * Xp.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dY, yp.data(), sizeof(float) * count, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->d_loss, 0, sizeof(float), st);
    for (int b0 = 0; b0 < count && e == cudaSuccess; b0 += batch) {
      const int nb = std::min(batch, count - b0);
      const int blocks = std::min(64, (nb + SPB - 1) / SPB);
      k_mlp_backward<<<blocks, SPB * H, 0, st>>>(m->d_w, dX + (size_t)b0 * F, dY + b0, m->d_norm, m->d_norm + F, nb,
                                                  1.f / nb, m->d_g, m->d_loss);
      ++m->step;
      const float c1 = 1.f - powf(0.9f, (float)m->step), c2 = 1.f - powf(0.999f, (float)m->step);
      k_mlp_adam<<<(NPARAM + 255) / 256, 256, 0, st>>>(m->d_w, m->d_g, m->d_m, m->d_v, NPARAM, lr, 0.9f, 0.999f, 1e-8f,
                                                       c1, c2);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&lsum, m->d_loss, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFree(dX);
  cudaFree(dY);
  if (e != cudaSuccess) return cuda_err(e);
  if (final_loss) *final_loss = lsum / count;  // mean squared error over the last epoch
  return BD_OK;
}

}  // extern "C"

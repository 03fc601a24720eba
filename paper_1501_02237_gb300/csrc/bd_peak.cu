// Issue-rate microbenchmark: the denominator of the integer roofline (measurement only; no
// part of the volume computation).
//
// Every thread runs eight coupled recurrences of one 32-bit instruction kind, written as
// inline PTX so that each step is exactly one instruction of that kind: step j of a round
// updates register j from itself, register j+1 (mod 8) and a loop-invariant operand, so two
// dependent steps always have at least four distinct inputs and no pair of them can be fused
// into one instruction, and no operation used is associative in the way the chain is built
// (majority for the logic kind, multiply-add for the multiply kind), so no chain collapses.
// Eight chains with 64 warps per SM give each scheduler enough independent instructions to
// issue every cycle.  Kinds:
//   0  LOP3 (lop3.b32, majority)              ALU pipe
//   1  IMAD (mad.lo.u32)                      multiply-add pipe
//   2  LOP3 and IMAD alternating              both integer pipes
//   3  FFMA (fma.rn.f32)                      for context: the single-precision filter's pipe
//   4  LOP3 and FFMA alternating              the filter's mix
// SM cycles come from clock64() around the loop in every block; the wall time from CUDA events
// on the library's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "../../include/binodeg.h"
#include "bd_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 16;  // rounds per loop iteration

__device__ __forceinline__ uint32_t op_lop3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm volatile("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}
__device__ __forceinline__ uint32_t op_imad(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}
__device__ __forceinline__ uint32_t op_ffma(uint32_t a, uint32_t b, uint32_t c) {
  float r;
  asm volatile("fma.rn.f32 %0, %1, %2, %3;"
               : "=f"(r)
               : "f"(__uint_as_float(a)), "f"(__uint_as_float(b)), "f"(__uint_as_float(c)));
  return __float_as_uint(r);
}

template <int KIND>
__device__ __forceinline__ uint32_t step(int j, uint32_t a, uint32_t next, uint32_t b) {
  if (KIND == 0) return op_lop3(a, next, b);
  if (KIND == 1) return op_imad(a, b, next);
  if (KIND == 2) return (j & 1) ? op_imad(a, b, next) : op_lop3(a, next, b);
  if (KIND == 3) return op_ffma(a, b, next);
  return (j & 1) ? op_ffma(a, b, next) : op_lop3(a, next, b);
}

template <int KIND>
__global__ void __launch_bounds__(kThreads) k_issue(uint32_t seed, int iters, uint32_t* sink,
                                                    unsigned long long* cycles) {
  uint32_t a[kChains];
  const uint32_t t = blockIdx.x * kThreads + threadIdx.x;
  // small positive floats for the floating kinds (bounded recurrences), arbitrary words otherwise
  const bool fp = KIND >= 3;
  for (int j = 0; j < kChains; ++j) {
    const uint32_t w = (seed ^ (t * 0x9E3779B9u)) + 0x85EBCA6Bu * (uint32_t)j;
    a[j] = fp ? __float_as_uint(0.25f + (float)(w & 1023u) * (1.0f / 4096.0f)) : w;
  }
  const uint32_t b = fp ? __float_as_uint(0.5f) : (seed | 1u) * 0x2545F491u;
  __syncthreads();
  const long long c0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = step<KIND>(j, a[j], a[(j + 1) % kChains], b);
    }
  }
  const long long c1 = clock64();
  uint32_t x = 0;
  for (int j = 0; j < kChains; ++j) x ^= a[j];
  if (x == 0x6A09E667u) sink[t] = x;  // keeps the chains live; practically never stored
  __syncthreads();
  if (threadIdx.x == 0) cycles[blockIdx.x] = (unsigned long long)(c1 - c0);
}

template <int KIND>
cudaError_t launch(int blocks, cudaStream_t st, uint32_t seed, int iters, uint32_t* sink, unsigned long long* cyc) {
  k_issue<KIND><<<blocks, kThreads, 0, st>>>(seed, iters, sink, cyc);
  return cudaGetLastError();
}

}  // namespace

extern "C" int bd_issue_peak(int32_t kind, int32_t blocks_per_sm, int32_t iters, bd_peak_out* out) {
  if (!out) return bd::set_error(BD_ERR_ARG, "out is NULL");
  if (kind < 0 || kind > 4) return bd::set_error(BD_ERR_ARG, "kind must be in [0, 4]");
  if (iters < 1 || iters > (1 << 20)) return bd::set_error(BD_ERR_ARG, "iters must be in [1, 2^20]");
  int dev = 0, sms = 0, maxb = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxb, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  if (e != cudaSuccess) return bd::set_error(BD_ERR_CUDA, cudaGetErrorString(e));
  const int resident = std::max(1, maxb / kThreads);
  if (blocks_per_sm <= 0) blocks_per_sm = resident;
  if (blocks_per_sm > resident) return bd::set_error(BD_ERR_ARG, "blocks_per_sm above the resident limit");
  const int blocks = sms * blocks_per_sm;
  cudaStream_t st = bd::thread_stream();
  uint32_t* sink = nullptr;
  unsigned long long* cyc = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  e = cudaMalloc(&sink, sizeof(uint32_t) * (size_t)blocks * kThreads);
  if (e == cudaSuccess) e = cudaMalloc(&cyc, sizeof(unsigned long long) * blocks);
  if (e == cudaSuccess) e = cudaEventCreate(&ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&ev1);
  std::vector<unsigned long long> hc(blocks);
  if (e == cudaSuccess) e = cudaEventRecord(ev0, st);
  if (e == cudaSuccess) {
    switch (kind) {
      case 0: e = launch<0>(blocks, st, 12345u, iters, sink, cyc); break;
      case 1: e = launch<1>(blocks, st, 12345u, iters, sink, cyc); break;
      case 2: e = launch<2>(blocks, st, 12345u, iters, sink, cyc); break;
      case 3: e = launch<3>(blocks, st, 12345u, iters, sink, cyc); break;
      default: e = launch<4>(blocks, st, 12345u, iters, sink, cyc); break;
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(ev1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
  if (e == cudaSuccess) e = cudaMemcpy(hc.data(), cyc, sizeof(unsigned long long) * blocks, cudaMemcpyDeviceToHost);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (sink) cudaFree(sink);
  if (cyc) cudaFree(cyc);
  if (e != cudaSuccess) return bd::set_error(BD_ERR_CUDA, cudaGetErrorString(e));
  double cmax = 0, csum = 0;
  for (unsigned long long c : hc) {
    cmax = std::max(cmax, (double)c);
    csum += (double)c;
  }
  const double ops = (double)blocks * kThreads * (double)iters * kUnroll * kChains;
  out->lane_ops = ops;
  out->ms = ms;
  out->lane_ops_per_s = ops / (ms * 1e-3);
  out->sm_cycles = cmax;
  out->sm_mhz = cmax / (ms * 1e3);
  // per SM per cycle over the whole run: the slowest block spans the kernel (block start times
  // differ, so the mean block span would overstate the rate)
  (void)csum;
  out->lane_ops_per_sm_clk = ops / ((double)sms * cmax);
  out->sms = sms;
  out->blocks = blocks;
  out->threads_per_block = kThreads;
  out->kind = kind;
  return BD_OK;
}

// Library-internal helpers shared by the C ABI translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/binodeg.h"

namespace bd {

struct Reduction;

// records the message returned by bd_last_error() on this thread and returns `code`
int set_error(int code, const char* msg);
// the stream chosen with bd_set_stream() on this thread
cudaStream_t thread_stream();
// the current device's colex decode table for the enumeration's 4-D stage (uploaded on first
// use; call outside stream capture)
int device_tri_table(const uint32_t** out);
// bd_degree after its host reduction of an n-variable system: the volume by the subset
// enumeration, the pivoting walk or the segment rule, times the torsion, on the thread's stream
int degree_from_reduction(const Reduction& r, int n, uint64_t seed, bd_degree_out* out);

// Every device allocation of the library goes through dev_malloc: cudaMalloc, except that an
// allocation armed by bd_inject_alloc_failure fails as cudaErrorMemoryAllocation without
// calling it (host-side fault injection for tests), and a real out-of-memory error is cleared
// from the runtime's last-error slot so that it cannot be reported again by a later check.
cudaError_t dev_malloc_raw(void** p, size_t bytes);
template <class T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc_raw(reinterpret_cast<void**>(p), bytes);
}
// records a CUDA failure for bd_last_error(): BD_ERR_NOMEM for cudaErrorMemoryAllocation,
// BD_ERR_CUDA otherwise; returns that code
int cuda_error(cudaError_t e, const char* where = nullptr);

}  // namespace bd

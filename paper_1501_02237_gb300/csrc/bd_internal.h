// Library-internal helpers shared by the C ABI translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bd {

// records the message returned by bd_last_error() on this thread and returns `code`
int set_error(int code, const char* msg);
// the stream chosen with bd_set_stream() on this thread
cudaStream_t thread_stream();
// the current device's colex decode table for the enumeration's 4-D stage (uploaded on first
// use; call outside stream capture)
int device_tri_table(const uint32_t** out);

}  // namespace bd

// Lift heights from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014), the counter-based generator used for the generic lifting of
// Sec. 4.1.  The paper fixes neither values nor generator; this library's convention:
//     seed'    = mix(seed ^ attempt * 0xD1B54A32D192ED03)
//     omega(i) = 1 + (mix(seed' + (i + 1) * 0x9E3779B97F4A7C15) >> 44)   in [1, 2^20]
// where mix is SplitMix64's output function.  `attempt` counts re-lifts after a tie.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define BD_LIFT_HD __host__ __device__ __forceinline__
#else
#define BD_LIFT_HD inline
#endif

namespace bd {

BD_LIFT_HD uint64_t splitmix_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

BD_LIFT_HD uint64_t lift_stream_seed(uint64_t seed, uint32_t attempt) {
  return splitmix_mix(seed ^ ((uint64_t)attempt * 0xD1B54A32D192ED03ull));
}

BD_LIFT_HD int64_t lift_height(uint64_t stream_seed, int i) {
  return 1 + (int64_t)(splitmix_mix(stream_seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull) >> 44);
}

}  // namespace bd

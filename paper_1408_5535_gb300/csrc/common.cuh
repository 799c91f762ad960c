// Shared device helpers of the PHSVDS GB300 library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#define PH_WARP 32

namespace ph {

// SplitMix64 finaliser (Vigna); counter-based use: element i of stream s under
// seed k is mix(k ^ (s * 0xD1B54A32D192ED03) + (i + 1) * 0x9E3779B97F4A7C15).
__host__ __device__ inline uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
// Uniform in [-1, 1): 2 * (top 53 bits * 2^-53) - 1.
__host__ __device__ inline double sm64_pm1(uint64_t seed, uint64_t stream, uint64_t i) {
  uint64_t key = seed ^ (stream * 0xD1B54A32D192ED03ULL);
  uint64_t z = sm64_mix(key + (i + 1) * 0x9E3779B97F4A7C15ULL);
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

template <typename T>
__device__ inline T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// A warp's sum of per-thread partials in the element precision (FP32
// butterflies for the FP32 inner solves: GB300's FP64 pipe is narrow, and
// FP64 butterflies bound those kernels), widened to FP64 for the block and
// grid levels of the sum.
template <typename T>
__device__ inline double warp_sum_wide(T v) {
  return (double)warp_sum(v);
}

// Vectorised row access for b values per row (b in {1,2,4,8}).
template <typename T, int B> struct Row { T v[B]; };

template <typename T, int B>
__device__ inline void load_row(const T* __restrict__ p, T (&r)[B]) {
  if constexpr (sizeof(T) * B % 16 == 0) {
#pragma unroll
    for (int q = 0; q < B; q += 16 / sizeof(T)) {
      if constexpr (sizeof(T) == 8) {
        double2 t = *reinterpret_cast<const double2*>(p + q);
        r[q] = t.x; r[q + 1] = t.y;
      } else {
        float4 t = *reinterpret_cast<const float4*>(p + q);
        r[q] = t.x; r[q + 1] = t.y; r[q + 2] = t.z; r[q + 3] = t.w;
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < B; ++q) r[q] = p[q];
  }
}

template <typename T, int B>
__device__ inline void store_row(T* __restrict__ p, const T (&r)[B]) {
  if constexpr (sizeof(T) * B % 16 == 0) {
#pragma unroll
    for (int q = 0; q < B; q += 16 / sizeof(T)) {
      if constexpr (sizeof(T) == 8) {
        *reinterpret_cast<double2*>(p + q) = make_double2(r[q], r[q + 1]);
      } else {
        *reinterpret_cast<float4*>(p + q) = make_float4(r[q], r[q + 1], r[q + 2], r[q + 3]);
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < B; ++q) p[q] = r[q];
  }
}

// Atomic accumulation of a row of B values (float: 128-bit vector atomics).
template <typename T, int B>
__device__ inline void atomic_add_row(T* p, const T (&r)[B]) {
  if constexpr (sizeof(T) == 4 && B % 4 == 0) {
#pragma unroll
    for (int q = 0; q < B; q += 4)
      atomicAdd(reinterpret_cast<float4*>(p + q), make_float4(r[q], r[q + 1], r[q + 2], r[q + 3]));
  } else if constexpr (sizeof(T) == 4 && B == 2) {
    atomicAdd(reinterpret_cast<float2*>(p), make_float2(r[0], r[1]));
  } else {
#pragma unroll
    for (int q = 0; q < B; ++q) atomicAdd(p + q, r[q]);
  }
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }


}  // namespace ph

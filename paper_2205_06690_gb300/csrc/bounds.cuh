// Debug bounds checks, compiled in with -DSBSE_DEBUG_BOUNDS (the debug build of the library).
// SBSE_IDX(i, n) is i when 0 <= i < n. Otherwise it records the first such access of this
// translation unit (site = SBSE_TU * 100000 + source line, and the low 40 bits of the index) in a
// device word and yields 0, so the access stays inside the array and the kernel runs on to its end:
// no trap, no fault, the host reads the record through sbse_debug_bounds. Without the flag
// SBSE_IDX(i, n) is i and costs nothing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sbse {
// collects the readers of the translation units' records (sbse_api.cu)
void register_bounds_reader(int (*reader)(unsigned long long *));
}  // namespace sbse

#ifdef SBSE_DEBUG_BOUNDS
#ifndef SBSE_TU
#define SBSE_TU 0
#endif
namespace {
__device__ unsigned long long g_bounds_fault;

__device__ __forceinline__ long long sbse_bounds_check(long long i, long long n, unsigned long long site) {
  if (i >= 0 && i < n) return i;
  atomicCAS(&g_bounds_fault, 0ull, (site << 40) | ((unsigned long long)i & 0xFFFFFFFFFFull));
  return 0;
}

// the record of this translation unit, cleared once read; returns 1 if there was one
int read_bounds_fault(unsigned long long *out) {
  unsigned long long v = 0;
  if (cudaMemcpyFromSymbol(&v, g_bounds_fault, sizeof v) != cudaSuccess) return -1;
  if (v) {
    const unsigned long long z = 0;
    cudaMemcpyToSymbol(g_bounds_fault, &z, sizeof z);
  }
  *out = v;
  return v != 0;
}

struct BoundsReaderRegistration {
  BoundsReaderRegistration() { sbse::register_bounds_reader(&read_bounds_fault); }
} g_bounds_reader_registration;
}  // namespace
#define SBSE_IDX(i, n) sbse_bounds_check((long long)(i), (long long)(n), (unsigned long long)(SBSE_TU * 100000 + __LINE__))
#else
#define SBSE_IDX(i, n) (i)
#endif

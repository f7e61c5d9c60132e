// Optional bounds-checked build (-DSNAP_BOUNDS_CHECK, library libsnap_bc.so): the kernels'
// global-memory accesses that derive their index from a loop, a lane or a slice number go
// through snap_in_bounds(site, i, n).  In the checked build an index outside [0, n) records
// (site, index) in the error word -- the first failure only -- and the access is skipped, so
// a wrong index shows up as a status the host reads (snap_bounds_error) instead of a fault.
// In the normal build the check compiles to `true`.
//
// Error word: bits 63..48 the site number, bits 47..0 the index (two's complement, truncated),
// 0 = no failure.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#ifdef SNAP_BOUNDS_CHECK
#ifdef __CUDACC__
extern __device__ unsigned long long g_snap_bounds_err;
#endif
#endif

__host__ __device__ __forceinline__ unsigned long long snap_bounds_word(int site, long long i) {
  return ((unsigned long long)(site & 0xFFFF) << 48) | ((unsigned long long)i & 0xFFFFFFFFFFFFull);
}

// Records the first failure in *err (atomically on the device) and returns false when
// i is outside [0, n).
__host__ __device__ __forceinline__ bool snap_check_index(unsigned long long *err, int site,
                                                          long long i, long long n) {
  if (i >= 0 && i < n) return true;
#if defined(__CUDA_ARCH__)
  atomicCAS(err, 0ull, snap_bounds_word(site, i));
#else
  if (*err == 0ull) *err = snap_bounds_word(site, i);
#endif
  return false;
}

#if defined(SNAP_BOUNDS_CHECK) && defined(__CUDA_ARCH__)
#define snap_in_bounds(site, i, n) snap_check_index(&g_snap_bounds_err, (site), (long long)(i), (long long)(n))
#else
#define snap_in_bounds(site, i, n) true
#endif

// Check sites (one number per checked access).
enum {
  SNAP_SITE_HEAT_G = 1,        // k_heat_*: params row of a sample
  SNAP_SITE_HEAT_U = 2,        // k_heat_*: u / u_hat / dL/du of a slice
  SNAP_SITE_HEAT_LAM = 3,      // k_heat_forward: multiplier rows
  SNAP_SITE_MOMENT_ROW = 4,    // k1d_mixed: u_hat row of a slice (moments)
  SNAP_SITE_MIXED_ROW = 6      // k1d_mixed: slice index / write-back of a slice row
};

// Host build of the bounds-check helper of the library (compiled by nvcc as host code with
// -DSNAP_BOUNDS_CHECK; no kernels): the same snap_check_index the checked kernels call, and a
// checked copy loop shaped like their row accesses, for CPU tests.
#include "../../paper_2607_00095_b300/csrc/snap_bounds.cuh"

extern "C" int harness_check(unsigned long long *err, int site, long long i, long long n) {
  return snap_check_index(err, site, i, n) ? 1 : 0;
}

// dst[j] = src[j] for j in [first, first + count) of arrays of n elements: an access whose
// index leaves [0, n) is skipped and recorded (site 7), as in the checked build.
extern "C" int harness_checked_copy(const double *src, double *dst, long long n, long long first,
                                    long long count, unsigned long long *err) {
  int done = 0;
  for (long long j = first; j < first + count; ++j)
    if (snap_check_index(err, 7, j, n)) {
      dst[j] = src[j];
      ++done;
    }
  return done;
}

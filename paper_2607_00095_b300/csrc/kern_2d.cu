// 2-D family C (divergence + kinetic energy): placeholder until the 2-D kernels land.
#include "snap_internal.h"

cudaError_t setup_2d(snap_problem *p) { (void)p; return cudaSuccess; }
void teardown_2d(snap_problem *p) { (void)p; }
size_t ws_bytes_2d(const snap_problem *p, int B) { (void)p; (void)B; return 256; }
size_t cache_bytes_2d(const snap_problem *p, int B) { (void)p; (void)B; return 0; }
cudaError_t launch_2d_forward(const snap_problem *, int, const double *, const double *,
                              const double *, double *, double *, snap_stats *, void *,
                              const SolverOpts &, int, void *, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_2d_backward(const snap_problem *, int, const double *, const double *,
                               const double *, const double *, const snap_stats *, const void *,
                               double *, double *, void *, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_2d_residual(const snap_problem *, int, const double *, const double *,
                               double *, double *, void *, cudaStream_t) {
  return cudaErrorNotSupported;
}

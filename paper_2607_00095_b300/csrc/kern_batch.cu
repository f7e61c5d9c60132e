// Uneven batches: placeholder until the persistent kernel lands.
#include "snap_internal.h"

struct snap_batch { int n; };

extern "C" {
snap_status snap_batch_create(int, const snap_problem_t *, int, const int *, snap_batch_t *) {
  return SNAP_ERR_UNSUPPORTED;
}
void snap_batch_destroy(snap_batch_t) {}
snap_status snap_batch_bind(snap_batch_t, const double *const *, const double *const *,
                            double *const *, double *const *, snap_stats *) {
  return SNAP_ERR_UNSUPPORTED;
}
snap_status snap_batch_workspace_size(snap_batch_t, size_t *) { return SNAP_ERR_UNSUPPORTED; }
snap_status snap_batch_project(snap_batch_t, const snap_options *, unsigned long long *, void *,
                               size_t, snap_stream_t) {
  return SNAP_ERR_UNSUPPORTED;
}
snap_status snap_batch_project_grouped(snap_batch_t, const snap_options *, void *, size_t,
                                       snap_stream_t) {
  return SNAP_ERR_UNSUPPORTED;
}
}

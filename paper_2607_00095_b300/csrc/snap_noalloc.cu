// snap_project_noalloc: the 1-D forward projection with its scratch memory in a fixed,
// library-owned device array instead of a caller-provided workspace.
//
// Who needs it: callers that cannot allocate device memory at the point where they project,
// for example code running inside a host callback or a driver-level plugin that forbids
// cudaMalloc, or an embedding that has no allocator of its own and cannot size a workspace
// per batch.  They still pass every input and output buffer; only the scratch is provided
// by the library.
//
// The scratch is one file-scope __device__ array of SNAP_NOALLOC_SCRATCH_BYTES bytes.  Every
// GPU that loads the library holds it until the process exits.  In host code the array's
// name is only a host-side handle, not a device address, so its device address is looked up
// with cudaGetSymbolAddress once per device (with that device current) and cached; the first
// call on each device does this look-up.
#include <cuda_runtime.h>
#include <stdio.h>

#include <mutex>

#include "snap_internal.h"

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[SNAP_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" {

SNAP_API snap_status snap_project_noalloc(snap_problem_t p, int B, const double *u_hat,
                                          const double *params, double *u, double *lambda,
                                          snap_stats *stats, const snap_options *opt,
                                          snap_stream_t stream) {
  snap_clear_error();
  snap_reset_launches();
  if (!p) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null problem");
  if (p->desc.family != SNAP_FAMILY_A_MASS_ENERGY && p->desc.family != SNAP_FAMILY_B_BURGERS_BOUNDARY)
    return snap_fail_msg(SNAP_ERR_UNSUPPORTED, "snap_project_noalloc supports families A and B only");
  if (B < 0 || (p->desc.max_batch > 0 && B > p->desc.max_batch))
    return snap_fail_msg(SNAP_ERR_INVALID_ARG, "batch size out of range");
  if (B == 0) return SNAP_OK;
  if (!u_hat || !params || !u || !lambda)
    return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null u_hat / params / u / lambda");
  if ((((uintptr_t)u_hat) & 15u) || (((uintptr_t)u) & 15u))
    return snap_fail_msg(SNAP_ERR_INVALID_ARG, "u_hat and u must be 16-byte aligned");
  // the prepare kernel writes the IC slice of u while the tile kernel may still be reading
  // u_hat (programmatic dependent launch), so an in-place call would be undefined
  if (u == u_hat || (const double *)lambda == u || (const double *)lambda == u_hat)
    return snap_fail_msg(SNAP_ERR_INVALID_ARG, "outputs may not alias inputs");
  const size_t need = ws_bytes_1d(p, B);
  if (need > (size_t)SNAP_NOALLOC_SCRATCH_BYTES) {
    char msg[160];
    snprintf(msg, sizeof(msg),
             "snap_project_noalloc: this batch needs %zu bytes of scratch; the static array holds %d",
             need, SNAP_NOALLOC_SCRATCH_BYTES);
    return snap_fail_msg(SNAP_ERR_WORKSPACE, msg);
  }
  snap_options o;
  snap_options_default(&o);
  if (opt) o = *opt;
  if (snap_check_options(o) != SNAP_OK) return SNAP_ERR_INVALID_ARG;
  if (o.path == SNAP_PATH_GENERAL || o.path == SNAP_PATH_AUTO) o.path = SNAP_PATH_MIXED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return snap_fail_msg(SNAP_ERR_CUDA, "no usable current device");
  void *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void *ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr)
        return snap_fail_msg(SNAP_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
      g_noalloc_ptr[dev] = ptr;
    }
    scratch = g_noalloc_ptr[dev];
  }
  SolverOpts so;
  so.tol_kkt = o.tol_kkt;
  so.tol_h = o.tol_h;
  so.c1 = o.armijo_c1;
  so.delta0 = o.delta0;
  so.w_keep = o.w_keep;
  so.max_iter = o.max_iter;
  so.max_backtracks = o.max_backtracks;
  so.max_corrections = o.max_corrections;
  so.pad = 0;
  const cudaError_t e = launch_1d_forward(p, B, u_hat, params, nullptr, u, lambda, stats,
                                          so, o.path, scratch, (cudaStream_t)stream);
  if (e == cudaErrorNotSupported)
    return snap_fail_msg(SNAP_ERR_UNSUPPORTED, "unsupported request for this family");
  if (e != cudaSuccess) return snap_fail_msg(SNAP_ERR_CUDA, cudaGetErrorString(e));
  return SNAP_OK;
}

}  // extern "C"

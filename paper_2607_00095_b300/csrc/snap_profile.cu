// Optional per-kernel timing with CUDA events recorded on the launching stream around each
// kernel.  Off by default.  Mode 1 skips launches that are being captured into a graph;
// mode 2 records the events into the graph as event nodes, so that after a replay the
// recorded pairs hold that replay's kernel durations.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "snap_internal.h"

namespace {

struct Rec {
  std::string name;
  cudaEvent_t a, b;
};

std::mutex g_mu;
bool g_on = false;
bool g_in_graph = false;   // also record (as graph event nodes) while a stream is captured
std::vector<Rec> g_recs;

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return true;
  return st != cudaStreamCaptureStatusNone;
}

}  // namespace

int snap_prof_begin(cudaStream_t s, const char *name) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on || (capturing(s) && !g_in_graph)) return -1;
  Rec r;
  r.name = name;
  if (cudaEventCreate(&r.a) != cudaSuccess) return -1;
  if (cudaEventCreate(&r.b) != cudaSuccess) { cudaEventDestroy(r.a); return -1; }
  cudaEventRecord(r.a, s);
  g_recs.push_back(r);
  return (int)g_recs.size() - 1;
}

void snap_prof_end(cudaStream_t s, int id) {
  if (id < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (id < (int)g_recs.size()) cudaEventRecord(g_recs[id].b, s);
}

extern "C" {

SNAP_API snap_status snap_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = on != 0;
  g_in_graph = on == 2;
  return SNAP_OK;
}

SNAP_API snap_status snap_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto &r : g_recs) {
    cudaEventSynchronize(r.b);
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_recs.clear();
  return SNAP_OK;
}

SNAP_API snap_status snap_profile_read(const char *name, double *total_ms, long long *launches) {
  if (!name || !total_ms || !launches) return SNAP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  double t = 0.0;
  long long n = 0;
  for (auto &r : g_recs) {
    if (r.name != name) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return SNAP_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return SNAP_ERR_CUDA;
    t += ms;
    n++;
  }
  *total_ms = t;
  *launches = n;
  return SNAP_OK;
}

}  // extern "C"

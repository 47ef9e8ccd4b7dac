// mr_lbm_project_noalloc: the uniform-level reconstruction of
// mr_lbm_project without any memory allocation.
//
// mr_lbm_project allocates its two dense level buffers with cudaMalloc the
// first time it is called on a handle.  Some callers cannot allocate at that
// point: a process whose device memory is owned by another allocator (a
// framework's caching allocator, a memory pool with a hard budget) that must
// not see a foreign cudaMalloc in the middle of a run, or a serving loop on
// a shared GPU that cannot afford the device-wide synchronisation that
// allocating and freeing device memory may cause.  This entry point uses
// instead one file-scope device array of fixed size,
// MR_NOALLOC_SCRATCH_DOUBLES doubles (16 MiB), that every GPU which loads
// the library holds until the process exits.
//
// Set-up: the first call on each device, with that device current, looks up
// the device address of the array with cudaGetSymbolAddress (in host code the
// array's name is only a host-side stand-in, not a device address) and keeps
// it for later calls on that device.  Make that first call before any stream
// capture begins.
//
// Sharing: every call on a device uses the same array, which keeps the
// contents of the last call.  Nothing in it needs to start at zero: each
// level is written in full before it is read.  Calls whose work overlaps on
// the GPU (different streams, or different handles on concurrent streams)
// race on the array; serialise them.
#include <mutex>

#include "mr_handle.cuh"

#define MR_NOALLOC_SCRATCH_DOUBLES (1u << 21)  // two halves of 2^20 doubles
#define MR_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) double g_noalloc_scratch[MR_NOALLOC_SCRATCH_DOUBLES];

namespace {

std::mutex g_setup_mutex;
double* g_scratch_addr[MR_NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (set up on the
// first call for that device); nullptr on failure.
double* scratch_address() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MR_NOALLOC_MAX_DEVICES) return nullptr;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return nullptr;
    g_scratch_addr[dev] = (double*)p;
  }
  return g_scratch_addr[dev];
}

}  // namespace

extern "C" mr_status mr_lbm_project_noalloc(mr_lbm_t h, int level, double* out, int on_device) {
  if (!h || !out) return MR_EINVAL;
  if (h->sticky != MR_OK) return h->sticky;
  if (!h->initialized) return mr_handle_fail(h, MR_ESTATE);
  const Geo& g = h->g;
  if (level < g.Jmin || level > g.J) return MR_EINVAL;
  const size_t half = MR_NOALLOC_SCRATCH_DOUBLES / 2;
  const size_t per_level = (size_t)g.ncons * g.ncode[level];
  if (per_level > half) return MR_ECAPACITY;  // rejected before any work; the handle stays usable
  double* base = scratch_address();
  if (!base) return mr_handle_fail(h, MR_ECUDA);
  double* buf[2] = {base, base + half};
  mr_handle_projection(h);
  const MeshDev& A = h->mesh[h->cur];
  int pb = 0;
  for (int l = g.Jmin; l <= level; ++l) {
    mr_launch_project_dense(g, A, h->fstate, l, buf[pb], buf[1 - pb], h->st, h->nsm * 4);
    h->launches += 1;
    pb = 1 - pb;
  }
  if (cudaGetLastError() != cudaSuccess) return mr_handle_fail(h, MR_ECUDA);
  if (cudaMemcpyAsync(out, buf[pb], per_level * sizeof(double),
                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st) != cudaSuccess)
    return mr_handle_fail(h, MR_ECUDA);
  if (!on_device) {
    MeshCounts hc[2];
    return mr_handle_read_counts(h, hc);
  }
  return MR_OK;
}

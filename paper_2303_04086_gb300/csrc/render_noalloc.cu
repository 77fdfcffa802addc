// Allocation-free variant of inolf_render_rays.
//
// Some callers cannot allocate device memory at the point where they render:
// a frame loop whose memory budget is fixed at start-up, a plug-in whose host
// application owns every device allocation, or a latency-critical thread
// that cannot afford the device-wide synchronisation cudaMalloc/cudaFree may
// imply.  inolf_render_rays needs a caller-provided workspace (the hit list
// between the trace and shade kernels); this entry point instead uses a
// fixed array compiled into the library's device image, so it needs no
// workspace and calls no allocator.  The array exists on every GPU that
// loads the library, from module load until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "inolf_internal.h"

// Hit-list scratch of the allocation-free path: a 256-byte header (hit
// counter and error flags) followed by one 8-byte (ray, t) record per ray,
// for at most INOLF_NOALLOC_MAX_RAYS rays: 8 MiB + 256 B in total.  Objects
// with density cubes need 12 bytes per ray (alpha_c alongside); for them the
// array holds 699 050 rays per pass and larger batches take several passes.
static constexpr size_t kNoAllocBytes = 256 + 8 * (size_t)INOLF_NOALLOC_MAX_RAYS;
static __device__ __align__(256) unsigned char inolf_noalloc_scratch[kNoAllocBytes];

namespace {

// Zeroes the scratch header (counters must start at zero on every call; the
// array otherwise keeps whatever the previous call left in it).
__global__ void k_noalloc_clear_header() {
  if (threadIdx.x < 64) reinterpret_cast<uint32_t*>(inolf_noalloc_scratch)[threadIdx.x] = 0u;
}

std::mutex g_mu;
void* g_scratch[inolf::kMaxDevices] = {};

}  // namespace

// Device address of the scratch array on the current device.  In host code
// the symbol names a host-side stand-in, not device memory, so the address
// is looked up once per device with cudaGetSymbolAddress while that device is
// current, then cached.
inolf_status inolf::noalloc_scratch_address(void** out) {
  const int dev = inolf::device_index();
  if (dev < 0)
    return inolf::fail(INOLF_E_UNSUPPORTED, "inolf_render_rays_noalloc: no current device, or an index beyond 63");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, inolf_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return inolf::fail(INOLF_E_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_scratch[dev] = p;
  }
  *out = g_scratch[dev];
  return INOLF_OK;
}

extern "C" inolf_status inolf_render_rays_noalloc(const inolf_object* obj, const float* o, const float* d,
                                                  int64_t n, inolf_precision prec, float* rgba_out,
                                                  int32_t* tri_out, float* t_out, void* stream) {
  inolf::clear_error();
  if (!obj || n < 0 || (n > 0 && (!o || !d || !rgba_out)))
    return inolf::fail(INOLF_E_INVALID, "inolf_render_rays_noalloc: bad argument");
  if (n > INOLF_NOALLOC_MAX_RAYS)
    return inolf::fail(INOLF_E_INVALID, "inolf_render_rays_noalloc: n = " + std::to_string(n) +
                                            " rays exceeds the fixed scratch limit of " +
                                            std::to_string(INOLF_NOALLOC_MAX_RAYS) +
                                            " rays; split the batch or use inolf_render_rays");
  if (n == 0) return INOLF_OK;
  void* ws = nullptr;
  inolf_status s = inolf::noalloc_scratch_address(&ws);
  if (s != INOLF_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  k_noalloc_clear_header<<<1, 64, 0, st>>>();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return inolf::fail(INOLF_E_CUDA, std::string("k_noalloc_clear_header: ") + cudaGetErrorString(e));
  inolf::RayBatch rb{};
  rb.mode = 1;
  rb.o = o;
  rb.d = d;
  rb.n = n;
  s = inolf::launch_render(obj->o, rb, prec, rgba_out, tri_out, t_out, nullptr, nullptr, ws, kNoAllocBytes, stream);
  if (s != INOLF_OK) return s;
  // the failure flags sit in the scratch header, out of the caller's reach,
  // and the next call clears them: read them now (this synchronises `stream`)
  uint32_t flags = 0;
  s = inolf::read_device_flags(ws, stream, &flags);
  if (s != INOLF_OK) return s;
  return inolf::flags_status(flags, "inolf_render_rays_noalloc");
}

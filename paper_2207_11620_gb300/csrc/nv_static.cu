// nv_static.cu -- nv_render_raw_noalloc: the raw-volume ray march for callers
// that must not allocate device memory, with its scratch in a fixed static
// device array instead of an nv_renderer.
//
// Some callers cannot call cudaMalloc: real-time loops whose memory budget is
// fixed up front (an allocation may synchronise the device and take unbounded
// time inside a frame), plugins inside a host application that owns every
// allocation and budgets the GPU's memory itself, or callers that would
// otherwise have to keep a renderer object alive just to draw an occasional
// small image.  This entry point serves them: it allocates nothing (no
// cudaMalloc, cudaFree, cudaMallocHost, event or stream creation) and takes
// its ray buffers, sample batches and counters from the array below.  It runs
// the fixed-step emission-absorption march only (no adaptive step, no
// shadows).
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (NV_NOALLOC_SCRATCH_BYTES, about 16 MB) until the process
// exits.  In host code its name is only a host-side stand-in, not a device
// address, so the address is looked up with cudaGetSymbolAddress once per
// device, with that device current, the first time the entry point runs on
// it; that first call should therefore come before any stream capture.
// Every call shares the array and it keeps the last call's contents: the
// counters that must start at zero are cleared by each call, and two calls
// whose work overlaps on the GPU (different streams, or different host
// threads) race on the same scratch.
#include <mutex>

#include "nv_internal.cuh"

namespace {

constexpr int64_t kMaxPix = NV_NOALLOC_MAX_PIXELS;
constexpr int kMaxK = NV_NOALLOC_MAX_K;

constexpr int64_t align256(int64_t b) { return (b + 255) & ~int64_t(255); }
// layout of the scratch, in bytes from its start
constexpr int64_t kRayBytes = align256(kMaxPix * 13 * 4);       // one ray buffer
constexpr int64_t kNextKBytes = align256(kMaxPix * 4);          // one next-sample buffer
constexpr int64_t kCoordBytes = align256(kMaxPix * kMaxK * 12);
constexpr int64_t kValueBytes = align256(kMaxPix * kMaxK * 4);
constexpr int64_t kValidBytes = align256(kMaxPix * 4);
constexpr int64_t kOffRay0 = 0, kOffRay1 = kOffRay0 + kRayBytes;
constexpr int64_t kOffNext0 = kOffRay1 + kRayBytes, kOffNext1 = kOffNext0 + kNextKBytes;
constexpr int64_t kOffCoords = kOffNext1 + kNextKBytes;
constexpr int64_t kOffValues = kOffCoords + kCoordBytes;
constexpr int64_t kOffValid = kOffValues + kValueBytes;
constexpr int64_t kOffCounters = kOffValid + kValidBytes;  // 2 x int
constexpr int64_t kOffSamples = kOffCounters + 256;         // int64
constexpr int64_t kTotal = kOffSamples + 256;
static_assert(kTotal == NV_NOALLOC_SCRATCH_BYTES, "scratch size in nv.h is out of date");

__device__ __align__(256) unsigned char g_noalloc_scratch[kTotal];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_dev[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up once per device).
nv_status scratch_for_current_device(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nv_cuda_check(e, "nv_render_raw_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return nv_fail(NV_ERR_UNSUPPORTED, "nv_render_raw_noalloc: device %d", dev);
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_dev[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return nv_cuda_check(e, "nv_render_raw_noalloc: cudaGetSymbolAddress");
    g_scratch_dev[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_scratch_dev[dev];
  return NV_OK;
}

}  // namespace

extern "C" nv_status nv_render_raw_noalloc(const nv_volume *raw, const nv_camera *cam, const float *lut,
                                           const nv_macrocells *mc, const nv_render_opts *opts, float *rgba,
                                           void *stream) {
  if (!raw || !raw->data_dev || raw->nx < 1 || raw->ny < 1 || raw->nz < 1)
    return nv_fail(NV_ERR_ARG, "nv_render_raw_noalloc: bad volume");
  if (!cam || !lut || !opts || !rgba) return nv_fail(NV_ERR_ARG, "nv_render_raw_noalloc: NULL argument");
  if (cam->width < 1 || cam->height < 1) return nv_fail(NV_ERR_ARG, "nv_render_raw_noalloc: image %dx%d", cam->width, cam->height);
  if ((int64_t)cam->width * cam->height > kMaxPix)
    return nv_fail(NV_ERR_ARG, "nv_render_raw_noalloc: %dx%d = %lld pixels exceeds the static maximum of %lld",
                   cam->width, cam->height, (long long)cam->width * cam->height, (long long)kMaxPix);
  if (opts->K < 1 || opts->K > kMaxK)
    return nv_fail(NV_ERR_ARG, "nv_render_raw_noalloc: K=%d not in [1, %d]", opts->K, kMaxK);
  if (!(opts->step > 0.f) || !(opts->alpha_exp > 0.f) || !(opts->et > 0.f))
    return nv_fail(NV_ERR_ARG, "nv_render_raw_noalloc: step, alpha_exp and et must be > 0");
  if (!(cam->tan_half_fovy >= 0.f)) return nv_fail(NV_ERR_ARG, "nv_render_raw_noalloc: tan_half_fovy < 0");
  if (opts->step_max > 0.f || opts->shade != 0)
    return nv_fail(NV_ERR_UNSUPPORTED, "nv_render_raw_noalloc: emission-absorption with the fixed step only");
  if (mc && (!mc->mu_max_dev || mc->cell < 1 || mc->nx < 1 || mc->ny < 1 || mc->nz < 1))
    return nv_fail(NV_ERR_ARG, "nv_render_raw_noalloc: bad macrocell grid");
  unsigned char *base = nullptr;
  nv_status s = scratch_for_current_device(&base);
  if (s != NV_OK) return s;
  // a renderer view of the static scratch (nothing is allocated)
  nv_renderer r{};
  r.max_pixels = kMaxPix;
  r.K = opts->K;
  r.stream = (cudaStream_t)stream;
  r.ray[0] = reinterpret_cast<float *>(base + kOffRay0);
  r.ray[1] = reinterpret_cast<float *>(base + kOffRay1);
  r.next_k[0] = reinterpret_cast<int *>(base + kOffNext0);
  r.next_k[1] = reinterpret_cast<int *>(base + kOffNext1);
  r.coords = reinterpret_cast<float *>(base + kOffCoords);
  r.values = reinterpret_cast<float *>(base + kOffValues);
  r.nvalid = reinterpret_cast<int *>(base + kOffValid);
  r.counters = reinterpret_cast<int *>(base + kOffCounters);
  r.d_samples = reinterpret_cast<int64_t *>(base + kOffSamples);
  r.h_count = nullptr;
  return render_raw_sync_loop(r, *raw, *cam, lut, mc, *opts, rgba, (cudaStream_t)stream);
}

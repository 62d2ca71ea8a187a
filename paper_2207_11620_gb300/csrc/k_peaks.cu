// k_peaks.cu -- measurement kernels for the rooflines of the scatter and the
// gather (the paper has no counterpart): the rate at which this GPU completes
// scattered 16-byte FP32 vector reductions, and scattered 16-byte loads, into
// a buffer of a given size, with nothing else in the way.  Addresses come from
// a 32-bit mixing function of (thread, op), so every access lands on an
// unpredictable 16-byte slot, as the hash grid's do.
#include "nv_internal.cuh"
#include "tc_grid.cuh"

namespace {

__device__ __forceinline__ uint32_t mix32(uint32_t x) {  // a bijective integer mixer (xorshift-multiply)
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

constexpr int kOps = 32;  // accesses per thread, all issued back to back

__global__ void __launch_bounds__(256) k_peak_scatter(float *buf, uint32_t mask16, uint32_t seed) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll 8
  for (int k = 0; k < kOps; ++k) {
    const uint32_t slot = mix32(t * kOps + k + seed) & mask16;
    red_v4(buf + 4 * (size_t)slot, 1.f, 1.f, 1.f, 1.f);
  }
}

__global__ void __launch_bounds__(256) k_peak_gather(const uint4 *__restrict__ buf, uint32_t mask16, uint32_t seed,
                                                     uint32_t *sink) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
#pragma unroll 8
  for (int k = 0; k < kOps; ++k) {
    const uint4 v = __ldg(buf + (mix32(t * kOps + k + seed) & mask16));
    acc ^= v.x ^ v.y ^ v.z ^ v.w;
  }
  if (acc == 0x9e3779b9u) sink[t & 1023] = acc;  // keeps the loads; practically never stores
}

}  // namespace

// ops = threads * kOps; the grid covers ceil(ops / (256 kOps)) CTAs
extern "C" nv_status nv_peak_scatter(float *buf, int64_t n16, int64_t ops, uint64_t seed, void *stream) {
  if (!buf || n16 < 1 || (n16 & (n16 - 1)) || n16 > (int64_t(1) << 32) || ops < 1)
    return nv_fail(NV_ERR_ARG, "nv_peak_scatter: n16 must be a power of two <= 2^32, ops >= 1");
  const int64_t blocks = (ops + 256 * kOps - 1) / (256 * kOps);
  if (blocks > (int64_t(1) << 24)) return nv_fail(NV_ERR_ARG, "nv_peak_scatter: ops too large");
  k_peak_scatter<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(buf, (uint32_t)(n16 - 1), (uint32_t)seed);
  return nv_cuda_check(cudaGetLastError(), "k_peak_scatter launch");
}

extern "C" nv_status nv_peak_gather(const void *buf, int64_t n16, int64_t ops, uint64_t seed, void *sink,
                                    void *stream) {
  if (!buf || !sink || n16 < 1 || (n16 & (n16 - 1)) || n16 > (int64_t(1) << 32) || ops < 1)
    return nv_fail(NV_ERR_ARG, "nv_peak_gather: n16 must be a power of two <= 2^32, ops >= 1");
  const int64_t blocks = (ops + 256 * kOps - 1) / (256 * kOps);
  if (blocks > (int64_t(1) << 24)) return nv_fail(NV_ERR_ARG, "nv_peak_gather: ops too large");
  k_peak_gather<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
      reinterpret_cast<const uint4 *>(buf), (uint32_t)(n16 - 1), (uint32_t)seed, reinterpret_cast<uint32_t *>(sink));
  return nv_cuda_check(cudaGetLastError(), "k_peak_gather launch");
}

// k_ooc.cu -- A-17: out-of-core training samples (Sec. 4.1, Fig. 2).
//
// The volume stays in pinned host memory as bricks of B^3 voxels plus a
// one-voxel ghost layer ((B+2)^3 floats each).  The device keeps a ring of R
// brick slots.  A refresh replaces `count` slots (round robin) with randomly
// chosen bricks: one gather kernel on the ring's own high-priority stream reads
// the bricks straight from the pinned host memory (its mapped address) over the
// host link, ordered after the work already on the compute stream (the last
// reads of the ring) and waited for by the next sample on it -- called right
// after a sample, the copies overlap the training step that follows.  A sample picks a slot, a voxel of the slot's brick and
// a jitter of +-0.5 voxel, all from Philox, and interpolates the target inside
// the brick (its ghost layer holds every voxel the lookup can read).
#include <cmath>
#include <new>
#include <vector>

#include "nv_internal.cuh"

struct nv_ooc {
  const float *host;        // pinned [nbz][nby][nbx][(B+2)^3]
  const float *host_dev;    // the same memory as the device sees it (mapped)
  int64_t *job_pinned[2];   // per refresh: [count] source brick, [count] destination slot (pinned, mapped)
  int nx, ny, nz, B, nbx, nby, nbz;
  int64_t n_bricks, brick_floats;
  int R;
  float *ring;              // device [R][(B+2)^3]
  int *slot_brick_dev;      // device [R]
  std::vector<int> slot_brick;
  int *table_pinned[2];     // pinned copies of the slot table, alternating per refresh
  cudaEvent_t table_done[2];
  int next_slot;
  uint64_t refreshes;
  cudaStream_t copy;
  cudaEvent_t read_done, copies_done;
  static const int kPairs = 64;   // copy-timing event pairs
  cudaEvent_t t0[kPairs], t1[kPairs];
  int pair_head, pair_count;
  int64_t bytes_copied;
  double copy_ms;
  bool sample_must_wait;    // a refresh is in flight: the next sample waits for it
};

namespace {

__global__ void k_brick_sample(const float *__restrict__ ring, const int *__restrict__ slot_brick, int R, int B,
                               int nbx, int nby, int nx, int ny, int nz, int64_t n, uint64_t seed, uint32_t step,
                               float *xyz, float *target) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const uint4 u = nv_philox(make_uint4((uint32_t)i, (uint32_t)((uint64_t)i >> 32), step, 1u), k0, k1);
  const uint4 w = nv_philox(make_uint4((uint32_t)i, (uint32_t)((uint64_t)i >> 32), step, 2u), k0, k1);
  const int s = (int)(u.x % (uint32_t)R);
  const int b = slot_brick[s];
  const int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
  const int v[3] = {bx * B + (int)((u.y & 255u) % (uint32_t)B), by * B + (int)(((u.y >> 8) & 255u) % (uint32_t)B),
                    bz * B + (int)(((u.y >> 16) & 255u) % (uint32_t)B)};
  const uint32_t jw[3] = {u.z, u.w, w.x};
  const int dims[3] = {nx, ny, nz};
  const int org[3] = {bx * B - 1, by * B - 1, bz * B - 1};  // global index of the brick's first (ghost) voxel
  float p[3];
  int i0[3];
  float wt[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float j = __fsub_rn(__fmul_rn((float)(jw[a] >> 8), 1.0f / 16777216.0f), 0.5f);
    p[a] = __fdiv_rn(__fadd_rn(__fadd_rn((float)v[a], 0.5f), j), (float)dims[a]);
    // the cell-centred lookup of the whole volume (q = x n - 0.5, clamped), moved into the brick
    int g0, g1;
    nv_voxel_axis(p[a], dims[a], g0, g1, wt[a]);
    i0[a] = g0 - org[a];
  }
  const int E = B + 2;
  const float *br = ring + (int64_t)s * E * E * E;
  const float *r00 = br + ((int64_t)i0[2] * E + i0[1]) * E + i0[0];
  const float *r01 = r00 + E, *r10 = r00 + (int64_t)E * E, *r11 = r10 + E;
  float c00 = __ldg(r00) + wt[0] * (__ldg(r00 + 1) - __ldg(r00));
  float c01 = __ldg(r01) + wt[0] * (__ldg(r01 + 1) - __ldg(r01));
  float c10 = __ldg(r10) + wt[0] * (__ldg(r10 + 1) - __ldg(r10));
  float c11 = __ldg(r11) + wt[0] * (__ldg(r11 + 1) - __ldg(r11));
  float c0 = c00 + wt[1] * (c01 - c00);
  float c1 = c10 + wt[1] * (c11 - c10);
  if (xyz) {
    xyz[3 * i] = p[0];
    xyz[3 * i + 1] = p[1];
    xyz[3 * i + 2] = p[2];
  }
  if (target) target[i] = c0 + wt[2] * (c1 - c0);
}

// Refresh copies: a small persistent grid walks the (job, part) items -- job =
// source brick -> destination slot, part = a contiguous eighth of the brick --
// with 16-byte loads straight from the pinned host bricks over the host link,
// four in flight per thread.  64 CTAs of 128 threads carry the link's rate
// (256 bricks of 66^3 floats in 1.49 ms alone) and leave the SMs to the
// training kernels that run meanwhile: on the 2048^3 ring workload a grid of one
// 256-thread CTA per item ran after the training step rather than beside it
// (2.9 + 1.4 -> 4.3 ms), 64 CTAs overlap it (3.1 ms), 16-32 starve the link and
// 128-512 crowd the training kernels again.
constexpr int kGatherThreads = 128;
constexpr int kGatherCtas = 64;
constexpr int kGatherParts = 8;

__global__ void __launch_bounds__(kGatherThreads) k_brick_gather(const float4 *__restrict__ host,
                                                                 const int64_t *__restrict__ jobs, int count,
                                                                 int64_t brick_f4, float4 *ring) {
  const int64_t items = (int64_t)count * kGatherParts;
  const int64_t per = (brick_f4 + kGatherParts - 1) / kGatherParts;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int j = (int)(it / kGatherParts), q = (int)(it % kGatherParts);
    const int64_t src = jobs[j], dst = jobs[count + j];
    const float4 *s = host + src * brick_f4;
    float4 *d = ring + dst * brick_f4;
    const int64_t lo = q * per, hi = min(brick_f4, lo + per);
    for (int64_t i = lo + threadIdx.x; i < hi; i += 4 * blockDim.x) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t k = i + u * blockDim.x;
        if (k < hi) v[u] = __ldcs(s + k);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t k = i + u * blockDim.x;
        if (k < hi) d[k] = v[u];
      }
    }
  }
}

// Brick choice of one refreshed slot: splitmix64 of (seed, refresh, slot).
uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

nv_status copy_slots(nv_ooc *o, int first, int count, uint64_t seed) {
  const size_t bb = (size_t)o->brick_floats * sizeof(float);
  // the job list and slot table travel from one of two pinned buffers; the
  // work that read the same buffer two refreshes ago has finished before it
  // is rewritten
  const int tb = (int)(o->refreshes & 1);
  cudaError_t e = cudaEventSynchronize(o->table_done[tb]);
  if (e != cudaSuccess) return nv_cuda_check(e, "nv_ooc: refresh buffers");
  int64_t *jobs = o->job_pinned[tb];
  for (int k = 0; k < count; ++k) {
    const int s = (first + k) % o->R;
    const uint64_t h = mix64(seed ^ mix64(o->refreshes * 0x100000001B3ull + (uint64_t)s));
    const int64_t b = (int64_t)(h % (uint64_t)o->n_bricks);
    o->slot_brick[s] = (int)b;
    jobs[k] = b;
    jobs[count + k] = s;
  }
  int64_t *jobs_dev = nullptr;
  e = cudaHostGetDevicePointer((void **)&jobs_dev, jobs, 0);
  if (e != cudaSuccess) return nv_cuda_check(e, "nv_ooc: job list");
  // jobs[0..count) source bricks, jobs[count..2 count) destination slots
  const int64_t brick_f4 = o->brick_floats / 4;
  const int64_t items = (int64_t)count * kGatherParts;
  const unsigned grid = (unsigned)(items < kGatherCtas ? items : kGatherCtas);
  if (o->brick_floats % 4 == 0) {
    k_brick_gather<<<grid, kGatherThreads, 0, o->copy>>>(reinterpret_cast<const float4 *>(o->host_dev), jobs_dev,
                                                         count, brick_f4, reinterpret_cast<float4 *>(o->ring));
    e = cudaGetLastError();
  } else {
    for (int k = 0; k < count && e == cudaSuccess; ++k)
      e = cudaMemcpyAsync(o->ring + jobs[count + k] * o->brick_floats, o->host + jobs[k] * o->brick_floats, bb,
                          cudaMemcpyHostToDevice, o->copy);
  }
  if (e != cudaSuccess) return nv_cuda_check(e, "nv_ooc: brick copies");
  o->bytes_copied += (int64_t)count * (int64_t)bb;
  for (int s = 0; s < o->R; ++s) o->table_pinned[tb][s] = o->slot_brick[s];
  e = cudaMemcpyAsync(o->slot_brick_dev, o->table_pinned[tb], sizeof(int) * o->R, cudaMemcpyHostToDevice, o->copy);
  if (e == cudaSuccess) e = cudaEventRecord(o->table_done[tb], o->copy);
  return nv_cuda_check(e, "nv_ooc: slot table copy");
}

void ooc_free(nv_ooc *o) {
  if (!o) return;
  if (o->copy) cudaStreamSynchronize(o->copy);
  cudaFree(o->ring);
  cudaFree(o->slot_brick_dev);
  for (int b = 0; b < 2; ++b) {
    if (o->job_pinned[b]) cudaFreeHost(o->job_pinned[b]);
    if (o->table_pinned[b]) cudaFreeHost(o->table_pinned[b]);
    if (o->table_done[b]) cudaEventDestroy(o->table_done[b]);
  }
  if (o->read_done) cudaEventDestroy(o->read_done);
  if (o->copies_done) cudaEventDestroy(o->copies_done);
  for (int k = 0; k < nv_ooc::kPairs; ++k) {
    if (o->t0[k]) cudaEventDestroy(o->t0[k]);
    if (o->t1[k]) cudaEventDestroy(o->t1[k]);
  }
  if (o->copy) cudaStreamDestroy(o->copy);
  delete o;
}

// Fold the oldest recorded copy interval into copy_ms (waits for it).
void retire_pair(nv_ooc *o) {
  const int k = (o->pair_head - o->pair_count + nv_ooc::kPairs) % nv_ooc::kPairs;
  float ms = 0.f;
  if (cudaEventSynchronize(o->t1[k]) == cudaSuccess && cudaEventElapsedTime(&ms, o->t0[k], o->t1[k]) == cudaSuccess)
    o->copy_ms += ms;
  --o->pair_count;
}

}  // namespace

extern "C" nv_status nv_ooc_create(const float *host_bricks, int nx, int ny, int nz, int brick, int ring_slots,
                                   uint64_t seed, nv_ooc **out) {
  if (!out) return nv_fail(NV_ERR_ARG, "nv_ooc_create: out is NULL");
  *out = nullptr;
  if (!host_bricks) return nv_fail(NV_ERR_ARG, "nv_ooc_create: host_bricks is NULL");
  if (brick < 2 || brick > 256) return nv_fail(NV_ERR_ARG, "nv_ooc_create: brick=%d not in [2, 256]", brick);
  if (nx < brick || ny < brick || nz < brick || nx % brick || ny % brick || nz % brick)
    return nv_fail(NV_ERR_ARG, "nv_ooc_create: volume %dx%dx%d is not a multiple of the brick %d", nx, ny, nz,
                   brick);
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, host_bricks) != cudaSuccess || at.type != cudaMemoryTypeHost) {
    cudaGetLastError();
    return nv_fail(NV_ERR_ARG, "nv_ooc_create: host_bricks must be pinned host memory");
  }
  nv_ooc *o = new (std::nothrow) nv_ooc();
  if (!o) return nv_fail(NV_ERR_OOM, "nv_ooc_create: host allocation");
  o->host = host_bricks;
  o->nx = nx;
  o->ny = ny;
  o->nz = nz;
  o->B = brick;
  o->nbx = nx / brick;
  o->nby = ny / brick;
  o->nbz = nz / brick;
  o->n_bricks = (int64_t)o->nbx * o->nby * o->nbz;
  o->brick_floats = (int64_t)(brick + 2) * (brick + 2) * (brick + 2);
  if (ring_slots < 1 || ring_slots > o->n_bricks) {
    int64_t nb = o->n_bricks;
    delete o;
    return nv_fail(NV_ERR_ARG, "nv_ooc_create: ring_slots=%d not in [1, %lld]", ring_slots, (long long)nb);
  }
  o->R = ring_slots;
  o->slot_brick.assign(ring_slots, 0);
  cudaError_t e = cudaMalloc(&o->ring, (size_t)ring_slots * o->brick_floats * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&o->slot_brick_dev, sizeof(int) * ring_slots);
  // the refresh copies run as a kernel on a high-priority stream so their CTAs are
  // scheduled ahead of the training kernels they overlap
  int prio_lo = 0, prio_hi = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&o->copy, cudaStreamNonBlocking, prio_hi);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&o->host_dev, (void *)host_bricks, 0);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&o->read_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&o->copies_done, cudaEventDisableTiming);
  for (int k = 0; k < nv_ooc::kPairs && e == cudaSuccess; ++k) {
    e = cudaEventCreate(&o->t0[k]);
    if (e == cudaSuccess) e = cudaEventCreate(&o->t1[k]);
  }
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaMallocHost(&o->table_pinned[b], sizeof(int) * ring_slots);
    if (e == cudaSuccess) e = cudaMallocHost(&o->job_pinned[b], sizeof(int64_t) * 2 * ring_slots);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&o->table_done[b], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    nv_status s = nv_cuda_check(e, "nv_ooc_create");
    ooc_free(o);
    return s;
  }
  // the first sampling step needs every slot filled (Sec. 4.1: the buffer is warmed up once)
  nv_status s = copy_slots(o, 0, ring_slots, seed);
  if (s == NV_OK) s = nv_cuda_check(cudaStreamSynchronize(o->copy), "nv_ooc_create: warm-up");
  if (s != NV_OK) {
    ooc_free(o);
    return s;
  }
  o->refreshes = 1;
  o->bytes_copied = 0;
  *out = o;
  return NV_OK;
}

extern "C" nv_status nv_ooc_destroy(nv_ooc *o) {
  ooc_free(o);
  return NV_OK;
}

extern "C" nv_status nv_ooc_refresh(nv_ooc *o, int count, uint64_t seed, void *stream) {
  if (!o) return nv_fail(NV_ERR_ARG, "nv_ooc_refresh: ooc is NULL");
  if (count < 0 || count > o->R) return nv_fail(NV_ERR_ARG, "nv_ooc_refresh: count=%d not in [0, %d]", count, o->R);
  if (count == 0) return NV_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (o->pair_count == nv_ooc::kPairs) retire_pair(o);
  const int k = o->pair_head;
  // copies start only after the compute stream's earlier work (the last ring reads)
  cudaError_t e = cudaEventRecord(o->read_done, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(o->copy, o->read_done, 0);
  if (e == cudaSuccess) e = cudaEventRecord(o->t0[k], o->copy);
  if (e != cudaSuccess) return nv_cuda_check(e, "nv_ooc_refresh: ordering");
  nv_status s = copy_slots(o, o->next_slot, count, seed);
  if (s != NV_OK) return s;
  o->next_slot = (o->next_slot + count) % o->R;
  ++o->refreshes;
  e = cudaEventRecord(o->t1[k], o->copy);
  if (e == cudaSuccess) e = cudaEventRecord(o->copies_done, o->copy);
  if (e != cudaSuccess) return nv_cuda_check(e, "nv_ooc_refresh: ordering");
  o->sample_must_wait = true;  // the next sample (not the work in between) waits for the copies
  o->pair_head = (o->pair_head + 1) % nv_ooc::kPairs;
  ++o->pair_count;
  return NV_OK;
}

extern "C" nv_status nv_ooc_sample(nv_ooc *o, int64_t n, uint64_t seed, uint32_t step, float *xyz, float *target,
                                   void *stream) {
  if (!o) return nv_fail(NV_ERR_ARG, "nv_ooc_sample: ooc is NULL");
  if (n < 0) return nv_fail(NV_ERR_ARG, "nv_ooc_sample: n < 0");
  if (n == 0) return NV_OK;
  if (o->sample_must_wait) {
    cudaError_t e = cudaStreamWaitEvent((cudaStream_t)stream, o->copies_done, 0);
    if (e != cudaSuccess) return nv_cuda_check(e, "nv_ooc_sample: wait for refresh");
    o->sample_must_wait = false;
  }
  const unsigned blocks = (unsigned)((n + 255) / 256);
  k_brick_sample<<<blocks, 256, 0, (cudaStream_t)stream>>>(o->ring, o->slot_brick_dev, o->R, o->B, o->nbx, o->nby,
                                                            o->nx, o->ny, o->nz, n, seed, step, xyz, target);
  return nv_cuda_check(cudaGetLastError(), "k_brick_sample launch");
}

extern "C" nv_status nv_ooc_slots(nv_ooc *o, int *slot_brick) {
  if (!o || !slot_brick) return nv_fail(NV_ERR_ARG, "nv_ooc_slots: NULL argument");
  for (int s = 0; s < o->R; ++s) slot_brick[s] = o->slot_brick[s];
  return NV_OK;
}

extern "C" nv_status nv_ooc_stats(nv_ooc *o, int64_t *bytes_copied, double *copy_ms) {
  if (!o) return nv_fail(NV_ERR_ARG, "nv_ooc_stats: ooc is NULL");
  cudaError_t e = cudaStreamSynchronize(o->copy);
  if (e != cudaSuccess) return nv_cuda_check(e, "nv_ooc_stats: sync");
  while (o->pair_count > 0) retire_pair(o);
  if (bytes_copied) *bytes_copied = o->bytes_copied;
  if (copy_ms) *copy_ms = o->copy_ms;
  return NV_OK;
}

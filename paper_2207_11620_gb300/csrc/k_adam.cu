// k_adam.cu -- A-8: Adam over the parameters in one HBM pass.
//
// Per parameter the kernel reads p, g, m, v (16 B) and writes p, m, v, g = 0
// (16 B) plus the FP16/BF16 shadow (2 B) in tensor-core precisions: 32-34 B of
// algorithmic traffic per parameter, in blocks of 128 parameters (512 B of
// each array).  Persistent CTAs (as many as fit: three per SM) stream tiles of kCW blocks
// through a kStages-deep shared-memory ring: one producer warp brings p, g, m
// and v of a tile in with bulk asynchronous copies (the copy engine; runs of
// consecutive blocks in one copy per array) counted on an mbarrier, and each of
// the kCW consumer warps updates one block from shared memory and stores the
// results straight to global memory.  The loads of p, m and v are marked to
// leave L2 first and those of g to stay: the 64 MiB table gradient this kernel
// zeroes is what the next step's scatter reduces into (0.180 -> 0.173 ms for
// that kernel on L16 F2 T2^19).  Groups of four parameters that no
// gradient has reached yet (zero g, m and v) are read but not rewritten.
//
// Blocks no gradient can reach are not visited at all.  A point of [0,1]^3 has
// its cell corners at integer coordinates 0..N_l+1 of level l, so a hash slot
// that none of those vertices maps to never receives a gradient; on the coarse
// levels, with far fewer vertices than T slots, most 128-parameter blocks hold
// no such slot (about 4.4 of the 16 levels' blocks for L16 T2^19 Nmin16
// b1.38).  With zero g, m and v and no L2 term an Adam update leaves p, m, v
// and g as they are, bit for bit, so skipping those blocks is exact.  The block
// list is built once per network; Adam falls back to every block, for good,
// once that premise may fail: an L2 term, a gradient or moment buffer handed
// to the caller, or a gradient scattered from a point outside [0,1]^3 (the
// kernels that read given training points set a device flag).
//
// The step counter, the overflow flag and the loss scale live on the device,
// so a step whose gradient overflowed is skipped without a host round trip
// (the gradient is still cleared); the last CTA of the launch does the step's
// book-keeping.
#include <algorithm>
#include <vector>

#include "nv_internal.cuh"
#include "tc_ptx.cuh"

namespace {

struct AdamHP {
  float lr, b1, b2, eps, l2;
  int decay_start, decay_interval;
  float decay_base;
};

constexpr int kBlk = 32;                              // float4 groups per block: 128 parameters, one per lane
constexpr int kCW = 8;                                // consumer warps = blocks per tile
constexpr int kStages = 4;                            // tiles in flight per CTA
constexpr int kAdamThreads = (kCW + 1) * 32;          // + the producer warp
constexpr int kStageF4 = 4 * kCW * kBlk;              // float4 of p, g, m, v of one tile (16 KB)
constexpr size_t kAdamSmem = (size_t)kStages * kStageF4 * 16 + 2 * kStages * 8 + kStages * kCW * 8;
constexpr uint32_t kWaitLimit = 1u << 24;             // mbarrier polls before a wait gives up

// Bulk global -> shared copy with an L2 eviction policy (createpolicy).
__device__ __forceinline__ void bulk_g2s_stream(void *dst_smem, const void *src, uint32_t bytes, uint64_t *mbar,
                                                uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          tc::smem_u32(dst_smem)),
      "l"(src), "r"(bytes), "r"(tc::smem_u32(mbar)), "l"(policy)
      : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// b^e for an integer e >= 0 by binary exponentiation: about 2 log2(e) FP64
// multiplies (the library pow's FP64 log and exp took ~6 us of dependent FP64
// work on this GPU at the head of every launch); within a few ulps of pow.
__device__ __forceinline__ double ipow(double b, int e) {
  double r = 1.0;
  for (; e > 0; e >>= 1) {
    if (e & 1) r *= b;
    b *= b;
  }
  return r;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(mbar)) : "memory");
}

template <int SHADOW>
__device__ __forceinline__ void put_shadow(void *shadow, int64_t i, float4 pp) {
  if (SHADOW == 0) return;
  uint2 u;
  if (SHADOW == 1) {
    __half2 a = __floats2half2_rn(pp.x, pp.y), b = __floats2half2_rn(pp.z, pp.w);
    u.x = *reinterpret_cast<uint32_t *>(&a);
    u.y = *reinterpret_cast<uint32_t *>(&b);
  } else {
    __nv_bfloat162 a = __floats2bfloat162_rn(pp.x, pp.y), b = __floats2bfloat162_rn(pp.z, pp.w);
    u.x = *reinterpret_cast<uint32_t *>(&a);
    u.y = *reinterpret_cast<uint32_t *>(&b);
  }
  reinterpret_cast<uint2 *>(shadow)[i] = u;
}

// Book-keeping after the update, by the last CTA to finish: count the step or,
// after an overflow, halve the loss scale; publish the batch loss.
__device__ __forceinline__ void step_finish(DevState *ds, double inv_n, double *loss_out) {
  if (ds->overflow) {
    ds->loss_scale *= 0.5f;
    ds->overflow = 0;
  } else {
    ds->step += 1;
  }
  ds->loss_mean = ds->loss_acc * inv_n;
  ds->loss_acc = 0.0;
  if (loss_out) *loss_out = ds->loss_mean;
}

template <int SHADOW>  // 0 none, 1 fp16, 2 bf16
__global__ void __launch_bounds__(kAdamThreads) k_adam(float *__restrict__ p, float *__restrict__ g,
                                                       float *__restrict__ m, float *__restrict__ v,
                                                       void *__restrict__ shadow, int64_t n, AdamHP hp,
                                                       DevState *ds, const int32_t *__restrict__ blocks,
                                                       int64_t nblocks, double inv_n, double *loss_out) {
  extern __shared__ __align__(128) uint8_t smem[];
  float4 *ring = reinterpret_cast<float4 *>(smem);  // [kStages][p g m v][kCW][kBlk]
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)kStages * kStageF4 * 16);
  uint64_t *empty = full + kStages;
  int64_t *ids = reinterpret_cast<int64_t *>(empty + kStages);  // [kStages][kCW] block of each slot, -1: none
  __shared__ float s_bc[3];
  __shared__ int s_skip, s_all, s_step;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    s_step = ds->step;
    s_skip = ds->overflow != 0;
    s_all = blocks == nullptr || ds->off_domain != 0;
    for (int st = 0; st < kStages; ++st) {
      tc::mbar_init(full + st, 1);
      tc::mbar_init(empty + st, kCW);
    }
    tc::mbar_fence_init();
  }
  __syncthreads();
  const bool skip = s_skip != 0, all = s_all != 0;
  const int64_t n4 = n >> 2;
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nb = all ? (n4 + kBlk - 1) / kBlk : nblocks;
  const int64_t ntile = (nb + kCW - 1) / kCW;
  bool failed = false;
  float4 *go = reinterpret_cast<float4 *>(g);
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  if (skip) {  // an overflowed step: only clear the gradient
    for (int64_t i = t0; i < n4; i += nthr) go[i] = zero;
    for (int64_t i = (n4 << 2) + t0; i < n; i += nthr) g[i] = 0.f;
  } else if (warp == kCW) {
    // ---- producer: tile j of this CTA into stage it % kStages ----
    const float4 *src[4] = {reinterpret_cast<const float4 *>(p), reinterpret_cast<const float4 *>(g),
                            reinterpret_cast<const float4 *>(m), reinterpret_cast<const float4 *>(v)};
    // p, m, v stream through L2 once per step; the table gradient stays: the
    // next step's scatter reduces into the lines this step zeroes
    const uint64_t pol = policy_evict_first(), pol_g = policy_evict_last();
    auto block_of = [&](int64_t j) -> int64_t {  // this lane's block of tile j
      const int64_t jj = j * kCW + lane;
      return (lane < kCW && j < ntile && jj < nb) ? (all ? jj : (int64_t)__ldg(blocks + jj)) : -1;
    };
    int64_t it = 0;
    int64_t b_next = block_of(blockIdx.x);
    for (int64_t j = blockIdx.x; j < ntile; j += gridDim.x, ++it) {
      const int st = (int)(it % kStages);
      const int64_t b = b_next;
      b_next = block_of(j + gridDim.x);  // in flight while this stage is waited for and filled
      if (it >= kStages && !tc::mbar_wait(empty + st, (uint32_t)(it / kStages - 1) & 1u, kWaitLimit)) {
        failed = true;
        break;
      }
      if (lane < kCW) ids[st * kCW + lane] = b;
      __syncwarp();  // orders the ids before lane 0 arms the stage (its arrive releases them)
      // a lane heads a run unless the lane before it holds block b - 1; the run
      // covers the following lanes that continue it
      const int64_t prev = __shfl_up_sync(0xffffffffu, b, 1);
      const bool cont = b >= 0 && lane > 0 && prev == b - 1;
      const uint32_t cmask = __ballot_sync(0xffffffffu, cont);
      const bool head = b >= 0 && !cont;
      int64_t f4 = 0;  // float4 per array the head's copy carries
      if (head) {
        const uint32_t after = lane < 31 ? ~(cmask >> (lane + 1)) : 0xffffffffu;
        const int run = __ffs((int)after);  // 1 + continuing lanes
        const int64_t end = (b + run) * kBlk < n4 ? (b + run) * kBlk : n4;
        f4 = end - b * kBlk;
      }
      const uint32_t bytes = __reduce_add_sync(0xffffffffu, (uint32_t)(f4 * 16 * 4));
      if (lane == 0) tc::mbar_expect_tx(full + st, bytes);
      __syncwarp();
      if (head) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
          bulk_g2s_stream(ring + ((size_t)(st * 4 + a) * kCW + lane) * kBlk, src[a] + b * kBlk, (uint32_t)(f4 * 16),
                          full + st, a == 1 ? pol_g : pol);
      }
    }
    // the copies of the last stages armed must land before the CTA may end
    if (lane == 0) {
      const int64_t first = it > kStages ? it - kStages : 0;
      for (int64_t u = first; u < it; ++u)
        if (!tc::mbar_wait(full + (int)(u % kStages), (uint32_t)(u / kStages) & 1u, kWaitLimit)) failed = true;
    }
  } else {
    // ---- consumers: warp w updates block w of each tile ----
    // bias corrections of step t (Kingma & Ba) and the decayed learning rate
    // of step index t - 1 (App. B): one FP64 evaluation per CTA, while the
    // producer's first copies are in flight (t >= 1, d >= 0)
    if (threadIdx.x == 0) {
      const int t = s_step + 1;
      s_bc[0] = (float)(1.0 / (1.0 - ipow((double)hp.b1, t)));
      s_bc[1] = (float)(1.0 / (1.0 - ipow((double)hp.b2, t)));
      const int k = t - 1;
      const int d = (k < hp.decay_start || hp.decay_interval <= 0) ? 0 : (k - hp.decay_start) / hp.decay_interval + 1;
      s_bc[2] = (float)((double)hp.lr * ipow((double)hp.decay_base, d));
    }
    asm volatile("bar.sync 1, %0;" ::"n"(kCW * 32) : "memory");  // the consumer warps only
    const float inv_bc1 = s_bc[0], inv_bc2 = s_bc[1], lr = s_bc[2];
    float4 *po = reinterpret_cast<float4 *>(p), *mo = reinterpret_cast<float4 *>(m);
    float4 *vo = reinterpret_cast<float4 *>(v);
    auto upd = [&](float &pp, float gg, float &mm, float &vv) {
      gg += hp.l2 * pp;
      mm = hp.b1 * mm + (1.f - hp.b1) * gg;
      vv = hp.b2 * vv + (1.f - hp.b2) * gg * gg;
      const float mh = mm * inv_bc1, vh = vv * inv_bc2;
      pp -= lr * mh / (sqrtf(vh) + hp.eps);
    };
    int64_t it = 0;
    for (int64_t j = blockIdx.x; j < ntile; j += gridDim.x, ++it) {
      const int st = (int)(it % kStages);
      if (!tc::mbar_wait(full + st, (uint32_t)(it / kStages) & 1u, kWaitLimit)) {
        failed = true;
        break;
      }
      const int64_t b = ids[st * kCW + warp];  // written by the producer before it armed the stage
      const int64_t i = b * kBlk + lane;
      if (b >= 0 && i < n4) {
        const float4 *sl = ring + ((size_t)(st * 4) * kCW + warp) * kBlk + lane;
        float4 pp = sl[0], gg = sl[kCW * kBlk], mm = sl[2 * kCW * kBlk], vv = sl[3 * kCW * kBlk];
        // four parameters with zero gradient and zero moments leave Adam
        // unchanged bit for bit when there is no L2 term; no stores
        const bool idle = hp.l2 == 0.f && (gg.x == 0.f) & (gg.y == 0.f) & (gg.z == 0.f) & (gg.w == 0.f) &
                                                (mm.x == 0.f) & (mm.y == 0.f) & (mm.z == 0.f) & (mm.w == 0.f) &
                                                (vv.x == 0.f) & (vv.y == 0.f) & (vv.z == 0.f) & (vv.w == 0.f);
        if (!idle) {
          upd(pp.x, gg.x, mm.x, vv.x);
          upd(pp.y, gg.y, mm.y, vv.y);
          upd(pp.z, gg.z, mm.z, vv.z);
          upd(pp.w, gg.w, mm.w, vv.w);
          go[i] = zero;
          __stcs(po + i, pp);
          __stcs(mo + i, mm);
          __stcs(vo + i, vv);
          put_shadow<SHADOW>(shadow, i, pp);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(empty + st);
    }
  }
  if (failed) atomicExch(&ds->err, 1);
  __syncthreads();
  // tail (n not a multiple of 4)
  if (!skip) {
    const float inv_bc1 = s_bc[0], inv_bc2 = s_bc[1], lr = s_bc[2];
    for (int64_t i = (n4 << 2) + t0; i < n; i += nthr) {
      float gg = g[i];
      g[i] = 0.f;
      float pp = p[i], mm = m[i], vv = v[i];
      gg += hp.l2 * pp;
      mm = hp.b1 * mm + (1.f - hp.b1) * gg;
      vv = hp.b2 * vv + (1.f - hp.b2) * gg * gg;
      pp -= lr * (mm * inv_bc1) / (sqrtf(vv * inv_bc2) + hp.eps);
      p[i] = pp;
      m[i] = mm;
      v[i] = vv;
      if (SHADOW == 1) reinterpret_cast<__half *>(shadow)[i] = __float2half_rn(pp);
      else if (SHADOW == 2) reinterpret_cast<__nv_bfloat16 *>(shadow)[i] = __float2bfloat16_rn(pp);
    }
  }
  // every CTA has read step and overflow above; the last one to get here
  // updates them for the next step
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&ds->adam_done, 1u) == gridDim.x - 1) {
      __threadfence();
      step_finish(ds, inv_n, loss_out);
      ds->adam_done = 0;
    }
  }
}

template <int SHADOW>
__global__ void k_shadow(const float *__restrict__ p, void *__restrict__ shadow, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (SHADOW == 1) reinterpret_cast<__half *>(shadow)[i] = __float2half_rn(p[i]);
    else reinterpret_cast<__nv_bfloat16 *>(shadow)[i] = __float2bfloat16_rn(p[i]);
  }
}

// Reachable blocks, step 1: a block is visited when it holds a weight or a
// parameter of a level whose vertices are not enumerated (lvl_enum bit clear).
__global__ void k_reach_fixed(uint32_t *bits, int64_t nblk, int64_t n4, int64_t n_table, int64_t level_span,
                              uint32_t lvl_enum) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q0 = b * (4 * kBlk), q1 = (q0 + 4 * kBlk < 4 * n4 ? q0 + 4 * kBlk : 4 * n4) - 1;  // its parameters
    bool on = q1 >= n_table;
    for (int64_t l = q0 / level_span; !on && l * level_span <= q1 && l * level_span < n_table; ++l)
      on = ((lvl_enum >> l) & 1u) == 0;
    if (on) atomicOr(bits + (b >> 5), 1u << (b & 31));
  }
}

// Step 2, one level: every vertex (x, y, z) in 0..n1-1 marks the block of its
// hash slot (F divides the block's 128 parameters, so an entry lies in one).
__global__ void k_reach_vertices(uint32_t *bits, int n1, uint32_t tmask, int F, int64_t level_base) {
  const int64_t nv = (int64_t)n1 * n1 * n1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t x = (uint32_t)(i % n1), y = (uint32_t)((i / n1) % n1), z = (uint32_t)(i / ((int64_t)n1 * n1));
    const int64_t q = level_base + (int64_t)(nv_hash3(x, y, z) & tmask) * F;
    const int64_t b = q / (4 * kBlk);
    atomicOr(bits + (b >> 5), 1u << (b & 31));
  }
}

}  // namespace

template <int SHADOW>
static nv_status launch_adam_t(nv_ctx *c, const AdamHP &hp, const int32_t *blocks, double inv_n,
                               double *loss_out) {
  static int per_sm = 0;  // resident CTAs per SM with the ring
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k_adam<SHADOW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdamSmem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adam<SHADOW>, kAdamThreads, kAdamSmem);
    if (e != cudaSuccess) return nv_cuda_check(e, "k_adam setup");
    if (per_sm < 1) return nv_fail(NV_ERR_CUDA, "k_adam: the %zu-byte ring does not fit an SM", kAdamSmem);
  }
  const int64_t n = c->n_params;
  // persistent, one wave: each CTA walks the tiles grid-stride (the tiles of
  // all blocks bound the count)
  const int64_t tiles = ((n >> 2) / kBlk + kCW) / kCW;
  const int64_t grid = std::min<int64_t>((int64_t)c->num_sms * per_sm, std::max<int64_t>(tiles, 1));
  k_adam<SHADOW><<<(unsigned)grid, kAdamThreads, kAdamSmem, c->stream>>>(
      c->params, c->grads, c->adam_m, c->adam_v, c->shadow, n, hp, c->ds, blocks, c->adam_nblocks, inv_n, loss_out);
  return nv_cuda_check(cudaGetLastError(), "k_adam launch");
}

nv_status launch_adam(nv_ctx *c, double inv_n, double *loss_out) {
  if (c->adam.l2_reg != 0.f) c->adam_dense = 1;  // weight decay moves every parameter
  const int32_t *blocks = c->adam_dense ? nullptr : c->adam_blocks;
  AdamHP hp{c->adam.lr,          c->adam.beta1,          c->adam.beta2,     c->adam.eps,
            c->adam.l2_reg,      c->adam.decay_start,    c->adam.decay_interval, c->adam.decay_base};
  switch (c->prec) {
    case NV_FP16: return launch_adam_t<1>(c, hp, blocks, inv_n, loss_out);
    case NV_BF16: return launch_adam_t<2>(c, hp, blocks, inv_n, loss_out);
    default: return launch_adam_t<0>(c, hp, blocks, inv_n, loss_out);
  }
}

nv_status launch_shadow(nv_ctx *c) {
  if (c->prec == NV_FP32) return NV_OK;
  int64_t n = c->n_params;
  unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 8);
  if (c->prec == NV_FP16) k_shadow<1><<<grid, 256, 0, c->stream>>>(c->params, c->shadow, n);
  else k_shadow<2><<<grid, 256, 0, c->stream>>>(c->params, c->shadow, n);
  return nv_cuda_check(cudaGetLastError(), "k_shadow launch");
}

// The sorted list of blocks Adam visits while every gradient comes from points
// of [0,1]^3 (see the head of this file).  Levels with more than 4 T vertices
// are not enumerated (all their blocks visited); none is left out when nearly
// every block is reachable anyway.
nv_status build_adam_blocks(nv_ctx *c) {
  const NetDesc &nd = c->nd;
  const int64_t n4 = c->n_params >> 2, nblk = (n4 + kBlk - 1) / kBlk;
  c->adam_blocks = nullptr;
  c->adam_nblocks = 0;
  if (nblk < 1 || nblk > INT32_MAX) return NV_OK;
  uint32_t lvl_enum = 0;
  for (int l = 0; l < nd.L; ++l) {
    const double n1 = (double)nd.res[l] + 2.0;
    if (n1 * n1 * n1 <= 4.0 * (double)nd.T) lvl_enum |= 1u << l;
  }
  if (!lvl_enum) return NV_OK;
  const int64_t nwords = (nblk + 31) / 32;
  uint32_t *bits = nullptr;
  cudaError_t e = cudaMalloc(&bits, nwords * sizeof(uint32_t));
  if (e != cudaSuccess) return nv_cuda_check(e, "build_adam_blocks: alloc");
  auto grid_for = [&](int64_t work) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)c->num_sms * 16));
  };
  e = cudaMemsetAsync(bits, 0, nwords * sizeof(uint32_t), c->stream);
  if (e == cudaSuccess) {
    k_reach_fixed<<<grid_for(nblk), 256, 0, c->stream>>>(bits, nblk, n4, nd.n_table, (int64_t)nd.T * nd.F, lvl_enum);
    e = cudaGetLastError();
  }
  for (int l = 0; l < nd.L && e == cudaSuccess; ++l) {
    if (!((lvl_enum >> l) & 1u)) continue;
    const int n1 = nd.res[l] + 2;
    k_reach_vertices<<<grid_for((int64_t)n1 * n1 * n1), 256, 0, c->stream>>>(bits, n1, nd.T - 1, nd.F,
                                                                              (int64_t)l * nd.T * nd.F);
    e = cudaGetLastError();
  }
  std::vector<uint32_t> h(nwords);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), bits, nwords * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(bits);
  if (e != cudaSuccess) return nv_cuda_check(e, "build_adam_blocks");
  std::vector<int32_t> list;
  for (int64_t b = 0; b < nblk; ++b)
    if ((h[b >> 5] >> (b & 31)) & 1u) list.push_back((int32_t)b);
  if ((double)list.size() > 0.97 * (double)nblk) return NV_OK;  // not worth the indirection
  if (list.empty()) return NV_OK;
  int32_t *d = nullptr;
  e = cudaMalloc(&d, list.size() * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemcpy(d, list.data(), list.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return nv_cuda_check(e, "build_adam_blocks: list");
  }
  c->adam_blocks = d;
  c->adam_nblocks = (int64_t)list.size();
  return NV_OK;
}

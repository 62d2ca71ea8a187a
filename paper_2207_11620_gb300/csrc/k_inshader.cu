// k_inshader.cu -- in-shader inference (Sec. 5.1, App. A): one ray-marching
// kernel in which every thread owns a ray and the network is evaluated inside
// the march, with no sample batches in global memory.
//
// A CTA is 128 threads = 128 rays = one tensor-core tile.  Per iteration each
// live thread finds its ray's next sample (march_step, the macrocell skip of
// the streaming path), gathers its hash-grid features into row `thread` of the
// tile in shared memory, one thread issues the layer-0 and layer-1 products
// (tcgen05, accumulators in tensor memory), every thread reads its row back,
// applies ReLU / the FP32 output layer / the sigmoid and composites the
// sample.  The CTA iterates until none of its rays is live (the paper's
// block-wide "any" over the rays), so a CTA runs as long as its longest ray
// and the rays that finished early leave their rows idle: the cost the
// sample-streaming path avoids by compacting live rays across the whole image
// (Sec. 5.2.1).
//
// Every per-sample step -- positions, features, products, epilogue order,
// output layer and compositing -- is the one the streaming path takes, so for
// the same network and camera both paths produce the same image.
#include "nv_internal.cuh"
#include "render_common.cuh"
#include "tc_grid.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int kH = 64;    // hidden width
constexpr int kTP = 128;  // rays (threads) per CTA = tile rows
constexpr int kIsTW = 16;  // a CTA's rays: a kIsTW x (kTP / kIsTW) pixel tile
constexpr uint32_t kWaitLimit = 1u << 24;
// D1 and D2 share 64 columns: layer 1's product is issued only after every
// thread's loads of D1 have completed, so a CTA needs 64 columns and seven CTAs
// (72 registers, 31 KB of shared memory at L*F = 32) share an SM.
constexpr uint32_t kTmemCols = 64;

template <int D0>
struct IsPlan {
  static constexpr int W0 = 0;                  // B [64][D0]
  static constexpr int W1 = W0 + kH * D0 * 2;   // B [64][64]
  static constexpr int A0 = W1 + kH * kH * 2;   // A [128][D0] features of this iteration's samples
  // A [128][64] h1, over the features: written after layer 0's product has
  // read them, and the next features are written after layer 1's has read it
  static constexpr int A1 = A0;
  static constexpr int W2 = A1 + kTP * kH * 2;  // float [64]
  static constexpr int BAR = W2 + kH * 4;       // mbarrier + tensor-memory slot
  static constexpr int TOTAL = BAR + 16;
};

// SH: single-shot shadows compiled in (the emission-absorption kernel keeps
// none of their state)
template <int D0, int F, bool BF, bool SH>
__global__ void __launch_bounds__(kTP, 7) k_render_is(NetDesc nd, const float *__restrict__ params,
                                                   const uint16_t *__restrict__ shadow, nv_camera cam, McView mc,
                                                   const float *__restrict__ lut, float step, float alpha_exp,
                                                   float et, ShadeArgs sh, float4 *__restrict__ rgba,
                                                   unsigned long long *samples, int *err) {
  using P = IsPlan<D0>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + P::BAR);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + P::BAR + 8);
  float *sW2 = reinterpret_cast<float *>(sm + P::W2);
  const uint32_t sbase = tc::smem_u32(sm);

  // ---- weights (FP16/BF16 shadow) as B operands, the output layer in FP32 ----
  const uint16_t *w0g = shadow + nd.n_table + nd.w_off[0];
  const uint16_t *w1g = shadow + nd.n_table + nd.w_off[1];
  for (int i = tid; i < kH * D0 / 8; i += kTP) {
    const int nn = i / (D0 / 8), c = i % (D0 / 8);
    *reinterpret_cast<uint4 *>(sm + P::W0 + tile_off(nn, c * 8, D0)) =
        __ldg(reinterpret_cast<const uint4 *>(w0g + nn * D0 + c * 8));
  }
  for (int i = tid; i < kH * kH / 8; i += kTP) {
    const int nn = i / (kH / 8), c = i % (kH / 8);
    *reinterpret_cast<uint4 *>(sm + P::W1 + tile_off(nn, c * 8, kH)) =
        __ldg(reinterpret_cast<const uint4 *>(w1g + nn * kH + c * 8));
  }
  for (int i = tid; i < kH; i += kTP) sW2[i] = params[nd.n_table + nd.w_off[2] + i];
  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    tc::mbar_fence_init();
  }
  tc::fence_async_smem();
  __syncthreads();
  if (warp == 0) {
    tc::tmem_alloc(tslot, kTmemCols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint32_t tD1 = tmem, tD2 = tmem;
  const uint32_t id_fwd = tc::idesc_f16(128, kH, BF, false, false);

  // ---- this thread's ray (A-11): a CTA takes a 16 x 8 pixel tile, so its
  // rays' samples share table lines at the mid levels ----
  const int tiles_x = (cam.width + kIsTW - 1) / kIsTW;
  const int px = (int)(blockIdx.x % tiles_x) * kIsTW + tid % kIsTW;
  const int py = (int)(blockIdx.x / tiles_x) * (kTP / kIsTW) + tid / kIsTW;
  const int64_t pix = (int64_t)py * cam.width + px;
  float o[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 1.f}, t0 = 0.f, t1 = 0.f;
  bool live = false;
  if (px < cam.width && py < cam.height) {
    nv_camera_ray(cam, px, py, o, d);
    live = nv_box(o, d, t0, t1);
    if (!live) rgba[pix] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  float cr = 0.f, cg = 0.f, cb = 0.f, ca = 0.f;
  int k = 0;
  McCache cache;  // cells and their mu_max are the same for the primary and the shadow march
  // single-shot shadows (Sec. 5): the largest contribution (1 - A) a' so far and
  // its position; as < 0 during the primary march, then the shadow march's opacity
  float bw = 0.f, bp[3] = {0.f, 0.f, 0.f}, as = -1.f;
  // the primary march has ended: march on towards the light from the sample of
  // largest contribution (same sampling rules, opacity only) if there is one
  auto start_shadow = [&]() -> bool {
    float s0, s1;
    if (!(SH && bw > 0.f && nv_box(bp, sh.light, s0, s1))) return false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      o[a] = bp[a];
      d[a] = sh.light[a];
    }
    t0 = s0;
    t1 = s1;
    k = 0;
    as = 0.f;
    return true;
  };
  auto finish = [&]() {
    if (SH && as >= 0.f) shade_colour(sh, as, cr, cg, cb);  // shaded at the point of largest contribution
    rgba[pix] = make_float4(cr, cg, cb, ca);
    live = false;
  };
  unsigned nsamp = 0;
  uint32_t phase = 0;
  bool failed = false;

  auto wait_mma = [&]() -> bool {
    const bool ok = tc::mbar_wait(mbar, phase, kWaitLimit);
    phase ^= 1u;
    tc::fence_after_sync();
    return __syncthreads_or(!ok) != 0;
  };

  for (;;) {
    // ---- next sample of the ray (A-12) ----
    float pos[3] = {0.f, 0.f, 0.f};
    while (live) {
      int m;
      while ((m = march_step(o, d, t0, t1, step, mc, k, pos, &cache)) == kMarchSkip) {
      }
      if (m != kMarchEnd) break;
      // left the volume: the primary march may hand over to the shadow march
      if (!(as < 0.f && start_shadow())) finish();
    }
    if (!__syncthreads_or(live)) break;
    // ---- its features, row `tid` of the tile (A-1..A-3; zero for idle rows) ----
#pragma unroll
    for (int c = 0; c < D0 / 8; ++c) {
      uint4 u = make_uint4(0u, 0u, 0u, 0u);
      if (live) {
        float f8[8];
        gather_corners<F, BF, 8 / F>(shadow, nd, c * (8 / F), pos[0], pos[1], pos[2], f8);
        u.x = pack16x2<BF>(f8[0], f8[1]);
        u.y = pack16x2<BF>(f8[2], f8[3]);
        u.z = pack16x2<BF>(f8[4], f8[5]);
        u.w = pack16x2<BF>(f8[6], f8[7]);
      }
      *reinterpret_cast<uint4 *>(sm + P::A0 + tile_off(tid, c * 8, D0)) = u;
    }
    tc::fence_async_smem();
    __syncthreads();
    // ---- layer 0: D1 = A0 W0^T ----
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < D0 / 16; ++kk)
        tc::mma_f16(tD1, desc_k(sbase + P::A0 + kk * 256, D0), desc_k(sbase + P::W0 + kk * 256, D0), id_fwd,
                    kk > 0);
      tc::mma_commit(mbar);
    }
    if (wait_mma()) { failed = true; break; }
#pragma unroll
    for (int c = 0; c < kH / 32; ++c) {  // 32 columns in flight per wait
      float v[32];
      tc::tmem_ld16(tD1 + lane_base + c * 32, v);
      tc::tmem_ld16(tD1 + lane_base + c * 32 + 16, v + 16);
      tc::tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < 4; ++j) st_row8_relu<BF>(sm + P::A1, tid, 4 * c + j, kH, v + 8 * j);
    }
    tc::fence_before_sync();
    tc::fence_async_smem();
    __syncthreads();
    // ---- layer 1: D2 = A1 W1^T ----
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < kH / 16; ++kk)
        tc::mma_f16(tD2, desc_k(sbase + P::A1 + kk * 256, kH), desc_k(sbase + P::W1 + kk * 256, kH), id_fwd,
                    kk > 0);
      tc::mma_commit(mbar);
    }
    if (wait_mma()) { failed = true; break; }
    // ---- output layer in FP32, summed over the two halves of the hidden
    // columns in the order the streaming kernel uses, then the sigmoid ----
    float zh[2];
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      float h2[32];
      tc::tmem_ld16(tD2 + lane_base + hh * 32, h2);
      tc::tmem_ld16(tD2 + lane_base + hh * 32 + 16, h2 + 16);
      tc::tmem_ld_wait();
      float zp = 0.f;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        h2[i] = fmaxf(h2[i], 0.f);
        zp += sW2[hh * 32 + i] * h2[i];
      }
      zh[hh] = zp;
    }
    tc::fence_before_sync();
    const float z3 = zh[0] + zh[1];
    const float yv = 1.f / (1.f + expf(-z3));
    // ---- A-14: composite; a ray that reaches et is done ----
    if (live) {
      ++nsamp;
      bool stop;
      if (as < 0.f) {
        float w;
        stop = composite_one(yv, lut, alpha_exp, et, cr, cg, cb, ca, &w);
        if (SH && w > bw) {
          bw = w;
          bp[0] = pos[0];
          bp[1] = pos[1];
          bp[2] = pos[2];
        }
      } else if constexpr (SH) {
        stop = shadow_one(yv, lut, alpha_exp, et, as);
      } else {
        stop = false;  // no shadow march without SH (as stays < 0)
      }
      ++k;
      if (stop && !(as < 0.f && start_shadow())) finish();
    }
  }

  // evaluated samples, for the statistics
  unsigned sw = nsamp;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) sw += __shfl_xor_sync(0xffffffffu, sw, s);
  if (lane == 0 && sw && samples) atomicAdd(samples, (unsigned long long)sw);
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
    // give an MMA that may still be in flight one more bounded chance to finish
    tc::mbar_wait(mbar, phase ^ 1u, kWaitLimit);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

template <int D0, int F, bool BF>
nv_status launch_is(nv_ctx *c, const nv_camera &cam, const float *lut, const McView &mv, const nv_render_opts &o,
                    float *rgba, unsigned long long *samples) {
  using P = IsPlan<D0>;
  // tensor memory holds 512 columns per SM: size the shared-memory request so
  // that at most 512 / kTmemCols CTAs share an SM
  const int tmem_cap = 512 / (int)kTmemCols;
  size_t bytes = P::TOTAL + 1024;
  const size_t min_bytes = 233472 / (tmem_cap + 1) + 1024;
  if (bytes < min_bytes) bytes = min_bytes;
  auto kern = o.shade ? k_render_is<D0, F, BF, true> : k_render_is<D0, F, BF, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return nv_cuda_check(e, "cudaFuncSetAttribute(k_render_is)");
  e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return nv_cuda_check(e, "cudaFuncSetAttribute(carveout)");
  const int64_t tiles_x = (cam.width + kIsTW - 1) / kIsTW, tiles_y = (cam.height + kTP / kIsTW - 1) / (kTP / kIsTW);
  const unsigned grid = (unsigned)(tiles_x * tiles_y);
  const ShadeArgs sh{o.shade, {o.light[0], o.light[1], o.light[2]}, o.ambient};
  kern<<<grid, kTP, bytes, c->stream>>>(c->nd, c->params, reinterpret_cast<const uint16_t *>(c->shadow), cam, mv,
                                        lut, o.step, o.alpha_exp, o.et, sh, reinterpret_cast<float4 *>(rgba),
                                        samples, &c->ds->err);
  return nv_cuda_check(cudaGetLastError(), "k_render_is launch");
}

template <bool BF>
nv_status dispatch_is(nv_ctx *c, const nv_camera &cam, const float *lut, const McView &mv, const nv_render_opts &o,
                      float *rgba, unsigned long long *samples) {
  const int D0 = c->nd.dims[0], F = c->nd.F;
  if (F == 2 && D0 == 16) return launch_is<16, 2, BF>(c, cam, lut, mv, o, rgba, samples);
  if (F == 2 && D0 == 32) return launch_is<32, 2, BF>(c, cam, lut, mv, o, rgba, samples);
  if (F == 2 && D0 == 64) return launch_is<64, 2, BF>(c, cam, lut, mv, o, rgba, samples);
  if (F == 4 && D0 == 32) return launch_is<32, 4, BF>(c, cam, lut, mv, o, rgba, samples);
  if (F == 4 && D0 == 64) return launch_is<64, 4, BF>(c, cam, lut, mv, o, rgba, samples);
  return nv_fail(NV_ERR_UNSUPPORTED, "in-shader render: no kernel for F=%d, L*F=%d", F, D0);
}

}  // namespace

nv_status render_inshader(nv_ctx *c, const nv_camera &cam, const float *lut, const nv_macrocells *mc,
                          const nv_render_opts &o, float *rgba, unsigned long long *samples) {
  if (c->prec == NV_FP32) return nv_fail(NV_ERR_UNSUPPORTED, "in-shader render: needs an FP16 or BF16 network");
  if (!tc_supported(c->nd)) return nv_fail(NV_ERR_UNSUPPORTED, "in-shader render: unsupported network shape");
  if (samples) {
    cudaError_t e = cudaMemsetAsync(samples, 0, sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return nv_cuda_check(e, "cudaMemsetAsync(samples)");
  }
  const McView mv = mc_view(mc);
  const int tk = prof_begin(c);
  const nv_status s = c->prec == NV_BF16 ? dispatch_is<true>(c, cam, lut, mv, o, rgba, samples)
                                         : dispatch_is<false>(c, cam, lut, mv, o, rgba, samples);
  prof_end(c, NV_K_RENDER, tk);
  return s;
}

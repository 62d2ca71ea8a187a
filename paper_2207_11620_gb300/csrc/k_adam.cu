// k_adam.cu -- A-8: dense Adam over every parameter in one HBM pass.
//
// Per parameter the kernel reads p, g, m, v (16 B) and writes p, m, v, g = 0
// (16 B) plus the FP16/BF16 shadow (2 B) in tensor-core precisions: 32-34 B of
// algorithmic traffic per parameter, float4-vectorised, grid-stride over a
// grid of a few CTAs per SM.  Groups of four parameters that no gradient has
// reached yet (zero g, m and v) are read but not rewritten.  The step counter, the overflow flag and the loss
// scale live on the device, so a step whose gradient overflowed is skipped
// without a host round trip (the gradient is still cleared); the last CTA of
// the launch does the step's book-keeping.
#include <algorithm>

#include "nv_internal.cuh"

namespace {

struct AdamHP {
  float lr, b1, b2, eps, l2;
  int decay_start, decay_interval;
  float decay_base;
};

constexpr int kU = 4;  // float4 iterations per thread kept in flight

template <int SHADOW>
__device__ __forceinline__ void put_shadow(void *shadow, int64_t i, float4 pp) {
  if (SHADOW == 1) {
    __half2 a = __floats2half2_rn(pp.x, pp.y), b = __floats2half2_rn(pp.z, pp.w);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t *>(&a);
    u.y = *reinterpret_cast<uint32_t *>(&b);
    reinterpret_cast<uint2 *>(shadow)[i] = u;
  } else if (SHADOW == 2) {
    __nv_bfloat162 a = __floats2bfloat162_rn(pp.x, pp.y), b = __floats2bfloat162_rn(pp.z, pp.w);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t *>(&a);
    u.y = *reinterpret_cast<uint32_t *>(&b);
    reinterpret_cast<uint2 *>(shadow)[i] = u;
  }
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
__global__ void __launch_bounds__(256) k_adam(float *__restrict__ p, float *__restrict__ g,
                                              float *__restrict__ m, float *__restrict__ v,
                                              void *__restrict__ shadow, int64_t n, AdamHP hp, DevState *ds,
                                              double inv_n, double *loss_out) {
  // bias corrections of step t (Kingma & Ba) and the decayed learning rate of
  // step index t - 1 (App. B): one FP64 evaluation per CTA
  __shared__ float s_bc[3];
  __shared__ int s_skip;
  if (threadIdx.x == 0) {
    const int t = ds->step + 1;
    s_bc[0] = (float)(1.0 / (1.0 - pow((double)hp.b1, (double)t)));
    s_bc[1] = (float)(1.0 / (1.0 - pow((double)hp.b2, (double)t)));
    const int k = t - 1;
    const int d = (k < hp.decay_start || hp.decay_interval <= 0) ? 0 : (k - hp.decay_start) / hp.decay_interval + 1;
    s_bc[2] = (float)((double)hp.lr * pow((double)hp.decay_base, (double)d));
    s_skip = ds->overflow != 0;
  }
  __syncthreads();
  const bool skip = s_skip != 0;
  const float inv_bc1 = s_bc[0], inv_bc2 = s_bc[1], lr = s_bc[2];
  const int64_t n4 = n >> 2;
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const float4 *p4 = reinterpret_cast<const float4 *>(p), *g4 = reinterpret_cast<const float4 *>(g);
  const float4 *m4 = reinterpret_cast<const float4 *>(m), *v4 = reinterpret_cast<const float4 *>(v);
  float4 *po = reinterpret_cast<float4 *>(p), *go = reinterpret_cast<float4 *>(g);
  float4 *mo = reinterpret_cast<float4 *>(m), *vo = reinterpret_cast<float4 *>(v);
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  auto upd = [&](float &pp, float gg, float &mm, float &vv) {
    gg += hp.l2 * pp;
    mm = hp.b1 * mm + (1.f - hp.b1) * gg;
    vv = hp.b2 * vv + (1.f - hp.b2) * gg * gg;
    const float mh = mm * inv_bc1, vh = vv * inv_bc2;
    pp -= lr * mh / (sqrtf(vh) + hp.eps);
  };
  if (skip) {  // an overflowed step: only clear the gradient
    for (int64_t i = t0; i < n4; i += nthr) go[i] = zero;
    for (int64_t i = (n4 << 2) + t0; i < n; i += nthr) g[i] = 0.f;
  }
  // kU float4 of each of p, g, m, v are loaded before anything is stored
  for (int64_t base = skip ? n4 : t0; base < n4; base += nthr * kU) {
    float4 gg[kU], pp[kU], mm[kU], vv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = base + u * nthr;
      if (i < n4) {
        gg[u] = __ldcs(g4 + i);
        pp[u] = __ldcs(p4 + i);
        mm[u] = __ldcs(m4 + i);
        vv[u] = __ldcs(v4 + i);
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = base + u * nthr;
      // four parameters with zero gradient and zero moments (never reached by
      // a gradient: hash slots no point has touched) leave Adam unchanged bit
      // for bit when there is no L2 term; their stores are skipped
      const bool idle = hp.l2 == 0.f && (gg[u].x == 0.f) & (gg[u].y == 0.f) & (gg[u].z == 0.f) &
                                              (gg[u].w == 0.f) & (mm[u].x == 0.f) & (mm[u].y == 0.f) &
                                              (mm[u].z == 0.f) & (mm[u].w == 0.f) & (vv[u].x == 0.f) &
                                              (vv[u].y == 0.f) & (vv[u].z == 0.f) & (vv[u].w == 0.f);
      if (i < n4 && !idle) {
        upd(pp[u].x, gg[u].x, mm[u].x, vv[u].x);
        upd(pp[u].y, gg[u].y, mm[u].y, vv[u].y);
        upd(pp[u].z, gg[u].z, mm[u].z, vv[u].z);
        upd(pp[u].w, gg[u].w, mm[u].w, vv[u].w);
        __stcs(go + i, zero);
        po[i] = pp[u];
        __stcs(mo + i, mm[u]);
        __stcs(vo + i, vv[u]);
        put_shadow<SHADOW>(shadow, i, pp[u]);
      }
    }
  }
  // tail (n not a multiple of 4)
  for (int64_t i = (n4 << 2) + t0; i < n && !skip; i += nthr) {
    float gg = g[i];
    g[i] = 0.f;
    float pp = p[i], mm = m[i], vv = v[i];
    upd(pp, gg, mm, vv);
    p[i] = pp;
    m[i] = mm;
    v[i] = vv;
    if (SHADOW == 1) reinterpret_cast<__half *>(shadow)[i] = __float2half_rn(pp);
    else if (SHADOW == 2) reinterpret_cast<__nv_bfloat16 *>(shadow)[i] = __float2bfloat16_rn(pp);
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

}  // namespace

nv_status launch_adam(nv_ctx *c, double inv_n, double *loss_out) {
  AdamHP hp{c->adam.lr,          c->adam.beta1,          c->adam.beta2,     c->adam.eps,
            c->adam.l2_reg,      c->adam.decay_start,    c->adam.decay_interval, c->adam.decay_base};
  int64_t n = c->n_params;
  // one wave of resident CTAs: each thread walks the vector grid-stride
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adam<0>, 256, 0);
  if (per_sm < 1) per_sm = 1;
  int64_t want = ((n >> 2) / kU + 255) / 256;
  int64_t grid = (int64_t)c->num_sms * per_sm;
  if (want < grid) grid = want;
  if (grid < 1) grid = 1;
  switch (c->prec) {
    case NV_FP16:
      k_adam<1><<<(unsigned)grid, 256, 0, c->stream>>>(c->params, c->grads, c->adam_m, c->adam_v, c->shadow, n,
                                                        hp, c->ds, inv_n, loss_out);
      break;
    case NV_BF16:
      k_adam<2><<<(unsigned)grid, 256, 0, c->stream>>>(c->params, c->grads, c->adam_m, c->adam_v, c->shadow, n,
                                                        hp, c->ds, inv_n, loss_out);
      break;
    default:
      k_adam<0><<<(unsigned)grid, 256, 0, c->stream>>>(c->params, c->grads, c->adam_m, c->adam_v, nullptr, n, hp,
                                                        c->ds, inv_n, loss_out);
  }
  return nv_cuda_check(cudaGetLastError(), "k_adam launch");
}

nv_status launch_shadow(nv_ctx *c) {
  if (c->prec == NV_FP32) return NV_OK;
  int64_t n = c->n_params;
  unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 8);
  if (c->prec == NV_FP16) k_shadow<1><<<grid, 256, 0, c->stream>>>(c->params, c->shadow, n);
  else k_shadow<2><<<grid, 256, 0, c->stream>>>(c->params, c->shadow, n);
  return nv_cuda_check(cudaGetLastError(), "k_shadow launch");
}

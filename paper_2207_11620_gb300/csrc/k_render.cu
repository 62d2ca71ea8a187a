// k_render.cu -- training-sample generation (A-9), macrocell build (A-10), the
// sample-streaming ray march (A-11..A-15, Sec. 5.2.1) and the FP64 quality
// reductions (A-16).
//
// Streaming loop per iteration (Sec. 5.2.1, batched ray marching):
//   k_coords     next K sample positions of each live ray, skipping samples
//                whose macrocell is transparent (mu_max == 0, Sec. 5.3)
//   inference    the network on the n_live*K positions (FP32 or tensor-core
//                kernel), or trilinear lookups of the raw volume
//   k_composite  front-to-back compositing with opacity correction and early
//                termination; finished rays write their pixel, live rays are
//                compacted into the other ray buffer (warp-aggregated atomic)
// The live count stays on the device: every kernel reads it there, and the
// host learns it through a pinned copy a few iterations late, so the loop
// never waits on the GPU inside a frame.
#include <algorithm>
#include <cmath>

#include "nv_internal.cuh"
#include "render_common.cuh"

namespace {

enum { R_OX = 0, R_OY, R_OZ, R_DX, R_DY, R_DZ, R_T0, R_T1, R_CR, R_CG, R_CB, R_CA, R_PIX, R_NFIELDS };

__global__ void k_sample(nv_volume v, int64_t n, uint64_t seed, uint32_t step, float *xyz, float *t) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float3 p = nv_sample_point(seed, step, (uint64_t)i);
  if (xyz) {
    xyz[3 * i] = p.x;
    xyz[3 * i + 1] = p.y;
    xyz[3 * i + 2] = p.z;
  }
  if (t) t[i] = nv_trilinear(v.data_dev, v.nx, v.ny, v.nz, p.x, p.y, p.z);
}

// Largest LUT opacity over the entries floor(255 lo) .. ceil(255 hi) of a value
// range clamped to [0, 1] (FP32 products decide the indices); an empty range
// (lo = +inf, hi = -inf) covers no entry and gives 0.
__device__ __forceinline__ float mu_of_range(float lo, float hi, const float *__restrict__ lut) {
  const float a0 = fminf(fmaxf(lo, 0.f), 1.f), a1 = fminf(fmaxf(hi, 0.f), 1.f);
  const int e0 = (int)floorf(__fmul_rn(a0, 255.0f)), e1 = min((int)ceilf(__fmul_rn(a1, 255.0f)), 255);
  float m = 0.f;
  for (int e = e0; e <= e1; ++e) m = fmaxf(m, lut[4 * e + 3]);
  return m;
}

// One CTA per macrocell: min/max over the aproned voxel range, then mu_max
// from the transfer function over the covered LUT entries.
__global__ void __launch_bounds__(256) k_macrocells(nv_volume v, int cell, int ncx, int ncy,
                                                    const float *__restrict__ lut, float *minmax, float *mu) {
  const int c = blockIdx.x;
  const int cx = c % ncx, cy = (c / ncx) % ncy, cz = c / (ncx * ncy);
  const int x0 = max(cx * cell - 1, 0), x1 = min(cx * cell + cell, v.nx - 1);
  const int y0 = max(cy * cell - 1, 0), y1 = min(cy * cell + cell, v.ny - 1);
  const int z0 = max(cz * cell - 1, 0), z1 = min(cz * cell + cell, v.nz - 1);
  const int wx = x1 - x0 + 1, wy = y1 - y0 + 1, wz = z1 - z0 + 1;
  const int total = wx * wy * wz;
  float lo = __int_as_float(0x7f800000), hi = -lo;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    int ix = i % wx, iy = (i / wx) % wy, iz = i / (wx * wy);
    float val = __ldg(v.data_dev + ((int64_t)(z0 + iz) * v.ny + (y0 + iy)) * v.nx + (x0 + ix));
    lo = fminf(lo, val);
    hi = fmaxf(hi, val);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  __shared__ float slo[8], shi[8];
  if ((threadIdx.x & 31) == 0) {
    slo[threadIdx.x >> 5] = lo;
    shi[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      lo = fminf(lo, slo[w]);
      hi = fmaxf(hi, shi[w]);
    }
    if (minmax) {
      minmax[2 * c] = lo;
      minmax[2 * c + 1] = hi;
    }
    if (mu) mu[c] = mu_of_range(lo, hi, lut);
  }
}

// Online macrocells (Sec. 5.3): training samples widen the value range of the
// macrocell that holds them (the cell of the position, as the march looks it
// up), with float atomic min / max.
struct McGrid {
  int ncx, ncy, ncz;
  float sx, sy, sz;  // cells per unit length (n / cell, FP32)
};

__device__ __forceinline__ void atomic_min_f(float *a, float v) {
  if (v >= 0.f) atomicMin(reinterpret_cast<int *>(a), __float_as_int(v));
  else atomicMax(reinterpret_cast<unsigned *>(a), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_f(float *a, float v) {
  if (v >= 0.f) atomicMax(reinterpret_cast<int *>(a), __float_as_int(v));
  else atomicMin(reinterpret_cast<unsigned *>(a), __float_as_uint(v));
}

__device__ __forceinline__ void mc_widen(float *minmax, const McGrid &g, float x, float y, float z, float v) {
  if (v != v) return;  // NaN widens nothing
  v += 0.0f;           // -0 -> +0, so the integer orderings above hold
  const int cx = min(max((int)floorf(__fmul_rn(x, g.sx)), 0), g.ncx - 1);
  const int cy = min(max((int)floorf(__fmul_rn(y, g.sy)), 0), g.ncy - 1);
  const int cz = min(max((int)floorf(__fmul_rn(z, g.sz)), 0), g.ncz - 1);
  float *m = minmax + 2 * (((int64_t)cz * g.ncy + cy) * g.ncx + cx);
  if (v < m[0]) atomic_min_f(m, v);
  if (v > m[1]) atomic_max_f(m + 1, v);
}

__global__ void k_mc_reset(float2 *minmax, int64_t nc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nc) minmax[i] = make_float2(__int_as_float(0x7f800000), __int_as_float(0xff800000));
}

// xyz (nullable: Philox training sample of (seed, step), target from vol) and val
__global__ void k_mc_update(const float *__restrict__ xyz, const float *__restrict__ val, int64_t n, nv_volume vol,
                            uint64_t seed, uint32_t step, McGrid g, float *minmax) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x, y, z, v;
  if (xyz) {
    x = xyz[3 * i];
    y = xyz[3 * i + 1];
    z = xyz[3 * i + 2];
    v = val[i];
  } else {
    const float3 p = nv_sample_point(seed, step, (uint64_t)i);
    x = p.x;
    y = p.y;
    z = p.z;
    v = nv_trilinear(vol.data_dev, vol.nx, vol.ny, vol.nz, x, y, z);
  }
  mc_widen(minmax, g, x, y, z, v);
}

__global__ void k_mc_mu(const float2 *__restrict__ minmax, int64_t nc, const float *__restrict__ lut, float *mu) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nc) {
    const float2 r = minmax[i];
    mu[i] = mu_of_range(r.x, r.y, lut);
  }
}

__device__ __forceinline__ int warp_append(int *counter, bool pred) {
  const unsigned mask = __ballot_sync(0xffffffffu, pred);
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (mask) {
    const int leader = __ffs(mask) - 1;
    if (lane == leader) base = atomicAdd(counter, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
  }
  return base + __popc(mask & ((1u << lane) - 1u));
}

// Rays are generated in 8 x 4 pixel tiles, one warp per tile and the tiles in
// row-major order, so a ray's slot neighbours are its image neighbours in both
// directions: the 32 consecutive rays a gather CTA takes cover a compact patch,
// and their samples share more table lines in L1 at the mid levels than a
// 32-pixel row would.  Compaction appends a warp's survivors together, which
// keeps the patches together in later iterations.
constexpr int RG_TW = 8, RG_TH = 4;

inline int64_t raygen_threads(int width, int rows) {
  const int64_t tx = (width + RG_TW - 1) / RG_TW, ty = (rows + RG_TH - 1) / RG_TH;
  return tx * ty * (RG_TW * RG_TH);
}

// next_k starts at sample 0, or, for the adaptive step, at the ray parameter t0
// (float bits); aux (nullable) gets the initial single-shot shadow state.
// Rows [row0, row0 + rows) of the image: pix indexes the band (row-major).
__global__ void k_raygen(nv_camera cam, int row0, int rows, float *ray, int *next_k, int64_t cap, int *count,
                         float4 *rgba, bool adaptive, float *aux) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int tiles_x = (cam.width + RG_TW - 1) / RG_TW;
  const int64_t tile = t / (RG_TW * RG_TH);
  const int within = (int)(t % (RG_TW * RG_TH));
  const int px = (int)(tile % tiles_x) * RG_TW + within % RG_TW;
  const int64_t py = (tile / tiles_x) * RG_TH + within / RG_TW;
  const int64_t pix = py * cam.width + px;
  bool hit = false;
  float o[3], d[3], t0 = 0.f, t1 = 0.f;
  if (px < cam.width && py < rows) {
    nv_camera_ray(cam, px, row0 + (int)py, o, d);
    hit = nv_box(o, d, t0, t1);
    if (!hit) rgba[pix] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  const int slot = warp_append(count, hit);
  if (hit) {
    ray[R_OX * cap + slot] = o[0];
    ray[R_OY * cap + slot] = o[1];
    ray[R_OZ * cap + slot] = o[2];
    ray[R_DX * cap + slot] = d[0];
    ray[R_DY * cap + slot] = d[1];
    ray[R_DZ * cap + slot] = d[2];
    ray[R_T0 * cap + slot] = t0;
    ray[R_T1 * cap + slot] = t1;
    ray[R_CR * cap + slot] = 0.f;
    ray[R_CG * cap + slot] = 0.f;
    ray[R_CB * cap + slot] = 0.f;
    ray[R_CA * cap + slot] = 0.f;
    ray[R_PIX * cap + slot] = __int_as_float((int)pix);
    next_k[slot] = adaptive ? __float_as_int(t0) : 0;
    if (aux) {
      aux[AUX_BW * cap + slot] = 0.f;
      aux[AUX_AS * cap + slot] = -1.f;  // primary march
    }
  }
}

// Threads per CTA of k_coords (32, 64 and 128 measured alike on the 1080p
// frame, although rays take different numbers of march steps and a CTA holds
// its SM slot until its slowest warp ends).
constexpr int kCoordsThreads = 128;

// Next K sample positions of each live ray (A-12, march_step).
// seg_exp (non-NULL: adaptive step between step and step_max): the opacity
// exponent of each emitted sample; next_k then holds the ray parameter t.
// A ray's K positions are contiguous (96 B at K = 8), so the positions are
// staged in shared memory ([thread][3K + 1] floats) and each warp writes its 32
// rays' block with coalesced stores: one store per sample from every thread hit
// a different sector per lane and kept the load/store queue full.
__global__ void __launch_bounds__(kCoordsThreads) k_coords(const float *__restrict__ ray, int *next_k, int64_t cap,
                                                const int *count, int K, float step, float step_max,
                                                float alpha_exp, McView mc, float *coords, float *seg_exp,
                                                int *nvalid) {
  extern __shared__ float s_pos[];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int n = *count;
  const int stride = 3 * K + 1;  // odd: the per-thread rows fall in different banks
  float *mine = s_pos + threadIdx.x * stride;
  if (i < n) {
    const float o[3] = {ray[R_OX * cap + i], ray[R_OY * cap + i], ray[R_OZ * cap + i]};
    const float d[3] = {ray[R_DX * cap + i], ray[R_DY * cap + i], ray[R_DZ * cap + i]};
    const float t0 = ray[R_T0 * cap + i], t1 = ray[R_T1 * cap + i];
    int k = next_k[i];
    int cnt = 0;
    float pos[3];
    if (seg_exp) {
      float t = __int_as_float(k);
      while (cnt < K) {
        float e;
        const int m = march_step_adaptive(o, d, t1, step, step_max, alpha_exp, mc, t, pos, e);
        if (m == kMarchEnd) break;
        if (m == kMarchSkip) continue;
        mine[3 * cnt] = pos[0];
        mine[3 * cnt + 1] = pos[1];
        mine[3 * cnt + 2] = pos[2];
        seg_exp[i * K + cnt] = e;
        ++cnt;
      }
      k = __float_as_int(t);
    } else {
      while (cnt < K) {
        const int m = march_step(o, d, t0, t1, step, mc, k, pos);
        if (m == kMarchEnd) break;
        if (m == kMarchSkip) continue;
        mine[3 * cnt] = pos[0];
        mine[3 * cnt + 1] = pos[1];
        mine[3 * cnt + 2] = pos[2];
        ++cnt;
        ++k;
      }
    }
    for (int j = 3 * cnt; j < 3 * K; ++j) mine[j] = 0.f;
    nvalid[i] = cnt;
    next_k[i] = k;
  }
  __syncwarp();
  // this warp's rays [w0, w0 + nr) are one contiguous block of nr * 3K floats
  const int lane = threadIdx.x & 31;
  const int64_t w0 = i - lane;
  const int64_t left = (int64_t)n - w0;
  const int nr = left < 0 ? 0 : (left > 32 ? 32 : (int)left);
  const int per = 3 * K;
  const float *wbase = s_pos + (threadIdx.x - lane) * stride;
  float *dst = coords + w0 * per;
  if ((per & 3) == 0) {  // K a multiple of 4: float4 stores (the block starts 16-byte aligned)
    const int q = per / 4, nq = nr * q;
    for (int f = lane; f < nq; f += 32) {
      const int r = f / q, w = (f - r * q) * 4;
      const float *src = wbase + r * stride + w;
      reinterpret_cast<float4 *>(dst)[f] = make_float4(src[0], src[1], src[2], src[3]);
    }
  } else {
    const int nf = nr * per;
    for (int f = lane; f < nf; f += 32) {
      const int r = f / per;
      dst[f] = wbase[r * stride + (f - r * per)];
    }
  }
}

// k_coords needs more than the default 48 KB of dynamic shared memory for K > 31
// (the renderer allows K up to 64): raise its limit once.
nv_status coords_kernel_setup() {
  static int done = 0;
  if (done) return NV_OK;
  cudaError_t e = cudaFuncSetAttribute(k_coords, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)((size_t)kCoordsThreads * (3 * 64 + 1) * sizeof(float)));
  if (e != cudaSuccess) return nv_cuda_check(e, "cudaFuncSetAttribute(k_coords)");
  done = 1;
  return NV_OK;
}

__global__ void k_values_raw(nv_volume v, const float *__restrict__ coords, const int *count, int K,
                             float *values) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)(*count) * K) return;
  values[i] = nv_trilinear(v.data_dev, v.nx, v.ny, v.nz, coords[3 * i], coords[3 * i + 1], coords[3 * i + 2]);
}


// A-14 + A-15: transfer function (linear between the 256 LUT entries), opacity
// correction a' = 1 - (1 - a)^e, front-to-back compositing, early termination
// at A >= et, and compaction of the rays that stay alive.
__global__ void k_composite(const float *__restrict__ ray, const int *__restrict__ next_k_in, int64_t cap,
                            const int *count, const float *__restrict__ values, const int *__restrict__ nvalid,
                            const float *__restrict__ seg_exp, int K, const float *__restrict__ lut,
                            float alpha_exp, float et, ShadeArgs sh, const float *__restrict__ coords,
                            const float *__restrict__ aux, float *aux_out, float *ray_out, int *next_k_out,
                            int *count_out, float4 *rgba, unsigned long long *samples) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int n = *count;
  bool live = false;
  int nv = 0;
  float cr = 0.f, cg = 0.f, cb = 0.f, ca = 0.f;
  float geo[8];  // o, d, t0, t1 of the ray that continues
  int nk = 0;
  float bw = 0.f, bp[3] = {0.f, 0.f, 0.f}, as = -1.f;
  if (i < n) {
    cr = ray[R_CR * cap + i];
    cg = ray[R_CG * cap + i];
    cb = ray[R_CB * cap + i];
    ca = ray[R_CA * cap + i];
#pragma unroll
    for (int f = 0; f < 8; ++f) geo[f] = ray[(R_OX + f) * cap + i];
    nk = next_k_in[i];
    nv = nvalid[i];
    if (sh.on) {
      bw = aux[AUX_BW * cap + i];
      bp[0] = aux[AUX_BX * cap + i];
      bp[1] = aux[AUX_BY * cap + i];
      bp[2] = aux[AUX_BZ * cap + i];
      as = aux[AUX_AS * cap + i];
    }
    bool done = false;
    const float *vrow = values + i * K;  // this ray's K values, contiguous: read 4 at a time when K % 4 == 0
    if (as < 0.f) {  // the primary march (A-14)
      for (int j0 = 0; j0 < nv && !done; j0 += 4) {
        float vv[4];
        if ((K & 3) == 0) {
          const float4 t4 = *reinterpret_cast<const float4 *>(vrow + j0);
          vv[0] = t4.x;
          vv[1] = t4.y;
          vv[2] = t4.z;
          vv[3] = t4.w;
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u) vv[u] = (j0 + u < nv) ? vrow[j0 + u] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + u;
          if (j >= nv || done) break;
          const float ex = seg_exp ? seg_exp[i * K + j] : alpha_exp;
          float w;
          const bool stop = composite_one(vv[u], lut, ex, et, cr, cg, cb, ca, &w);
          if (sh.on && w > bw) {
            bw = w;
            const float *p = coords + (i * K + j) * 3;
            bp[0] = p[0];
            bp[1] = p[1];
            bp[2] = p[2];
          }
          if (stop) done = true;
        }
      }
      if (nv < K) done = true;  // the ray left the volume during this batch
      if (done && sh.on && bw > 0.f) {
        // single-shot shadow: march on from the sample of largest contribution
        float s0, s1;
        if (nv_box(bp, sh.light, s0, s1)) {
          geo[0] = bp[0];
          geo[1] = bp[1];
          geo[2] = bp[2];
          geo[3] = sh.light[0];
          geo[4] = sh.light[1];
          geo[5] = sh.light[2];
          geo[6] = s0;
          geo[7] = s1;
          nk = seg_exp ? __float_as_int(s0) : 0;
          as = 0.f;
          done = false;
        }
      }
    } else {  // the shadow march: opacity only
      for (int j = 0; j < nv; ++j) {
        const float ex = seg_exp ? seg_exp[i * K + j] : alpha_exp;
        if (shadow_one(values[i * K + j], lut, ex, et, as)) {
          done = true;
          break;
        }
      }
      if (nv < K) done = true;
    }
    if (done) {
      if (as >= 0.f) shade_colour(sh, as, cr, cg, cb);  // shaded at the point of largest contribution
      rgba[__float_as_int(ray[R_PIX * cap + i])] = make_float4(cr, cg, cb, ca);
    }
    live = !done;
  }
  // evaluated samples of this warp, for the statistics
  int sw = nv;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sw += __shfl_xor_sync(0xffffffffu, sw, o);
  if ((threadIdx.x & 31) == 0 && sw) atomicAdd(samples, (unsigned long long)sw);
  const int slot = warp_append(count_out, live);
  if (live) {
#pragma unroll
    for (int f = 0; f < 8; ++f) ray_out[(R_OX + f) * cap + slot] = geo[f];
    ray_out[R_CR * cap + slot] = cr;
    ray_out[R_CG * cap + slot] = cg;
    ray_out[R_CB * cap + slot] = cb;
    ray_out[R_CA * cap + slot] = ca;
    ray_out[R_PIX * cap + slot] = ray[R_PIX * cap + i];
    next_k_out[slot] = nk;
    if (sh.on) {
      aux_out[AUX_BW * cap + slot] = bw;
      aux_out[AUX_BX * cap + slot] = bp[0];
      aux_out[AUX_BY * cap + slot] = bp[1];
      aux_out[AUX_BZ * cap + slot] = bp[2];
      aux_out[AUX_AS * cap + slot] = as;
    }
  }
}

// A-16: FP64 sum of squared RGB differences; each CTA adds its partial / (3n).
__global__ void __launch_bounds__(256) k_image_mse(const float4 *__restrict__ a, const float4 *__restrict__ b,
                                                   int64_t n, double scale, double *out) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float4 x = a[i], y = b[i];
    double dr = (double)x.x - (double)y.x, dg = (double)x.y - (double)y.y, db = (double)x.z - (double)y.z;
    s += dr * dr + dg * dg + db * db;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double part[8];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    atomicAdd(out, t * scale);
  }
}

__global__ void k_scale_double(double *x, double s) { *x *= s; }

inline unsigned blocks_for(int64_t n, int bs) { return (unsigned)std::max<int64_t>(1, (n + bs - 1) / bs); }

// Dynamic shared memory of k_coords: kCoordsThreads x (3K + 1) floats.
inline size_t coords_smem(int K) { return (size_t)kCoordsThreads * (3 * K + 1) * sizeof(float); }

}  // namespace

nv_status launch_scale_double(double *x, double s, cudaStream_t st) {
  k_scale_double<<<1, 1, 0, st>>>(x, s);
  return nv_cuda_check(cudaGetLastError(), "k_scale_double launch");
}

nv_status launch_sample(const nv_volume &v, int64_t n, uint64_t seed, uint32_t step, float *xyz, float *t,
                        cudaStream_t s) {
  if (n == 0) return NV_OK;
  k_sample<<<blocks_for(n, 256), 256, 0, s>>>(v, n, seed, step, xyz, t);
  return nv_cuda_check(cudaGetLastError(), "k_sample launch");
}

nv_status launch_macrocells(const nv_volume &v, int cell, const float *lut, float *minmax, float *mu,
                            cudaStream_t s) {
  int ncx = (v.nx + cell - 1) / cell, ncy = (v.ny + cell - 1) / cell, ncz = (v.nz + cell - 1) / cell;
  int64_t nc = (int64_t)ncx * ncy * ncz;
  k_macrocells<<<(unsigned)nc, 256, 0, s>>>(v, cell, ncx, ncy, lut, minmax, mu);
  return nv_cuda_check(cudaGetLastError(), "k_macrocells launch");
}

static McGrid mc_grid(int nx, int ny, int nz, int cell) {
  return McGrid{(nx + cell - 1) / cell, (ny + cell - 1) / cell, (nz + cell - 1) / cell,
                (float)nx / (float)cell, (float)ny / (float)cell, (float)nz / (float)cell};
}

nv_status launch_mc_reset(float *minmax, int nx, int ny, int nz, int cell, cudaStream_t s) {
  const McGrid g = mc_grid(nx, ny, nz, cell);
  const int64_t nc = (int64_t)g.ncx * g.ncy * g.ncz;
  k_mc_reset<<<blocks_for(nc, 256), 256, 0, s>>>(reinterpret_cast<float2 *>(minmax), nc);
  return nv_cuda_check(cudaGetLastError(), "k_mc_reset launch");
}

nv_status launch_mc_update(const float *xyz, const float *val, int64_t n, const nv_volume &vol, uint64_t seed,
                           uint32_t step, int nx, int ny, int nz, int cell, float *minmax, cudaStream_t s) {
  if (n == 0) return NV_OK;
  k_mc_update<<<blocks_for(n, 256), 256, 0, s>>>(xyz, val, n, vol, seed, step, mc_grid(nx, ny, nz, cell), minmax);
  return nv_cuda_check(cudaGetLastError(), "k_mc_update launch");
}

nv_status launch_mc_mu(const float *minmax, int nx, int ny, int nz, int cell, const float *lut, float *mu,
                       cudaStream_t s) {
  const McGrid g = mc_grid(nx, ny, nz, cell);
  const int64_t nc = (int64_t)g.ncx * g.ncy * g.ncz;
  k_mc_mu<<<blocks_for(nc, 256), 256, 0, s>>>(reinterpret_cast<const float2 *>(minmax), nc, lut, mu);
  return nv_cuda_check(cudaGetLastError(), "k_mc_mu launch");
}

nv_status launch_image_mse(const float *a, const float *b, int64_t n, double *out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
  if (e != cudaSuccess) return nv_cuda_check(e, "cudaMemsetAsync");
  if (n == 0) return NV_OK;
  unsigned grid = (unsigned)std::min<int64_t>(blocks_for(n, 256), 1216);
  k_image_mse<<<grid, 256, 0, s>>>(reinterpret_cast<const float4 *>(a), reinterpret_cast<const float4 *>(b), n,
                                   1.0 / (3.0 * (double)n), out);
  return nv_cuda_check(cudaGetLastError(), "k_image_mse launch");
}

nv_status render_impl(nv_renderer *r, nv_ctx *net, const nv_volume *raw, const nv_camera &cam, const float *lut,
                      const nv_macrocells *mc, const nv_render_opts &o, int row0, int rows, float *rgba) {
  const int64_t npix = (int64_t)cam.width * rows;
  const int64_t cap = r->max_pixels;
  const int K = r->K;
  cudaStream_t st = net ? net->stream : r->stream;
  {
    const nv_status cs = coords_kernel_setup();
    if (cs != NV_OK) return cs;
  }
  cudaError_t e = cudaMemsetAsync(r->counters, 0, 2 * sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(r->d_samples, 0, sizeof(int64_t), st);
  if (e != cudaSuccess) return nv_cuda_check(e, "render memset");
  float4 *out = reinterpret_cast<float4 *>(rgba);
  const bool adaptive = o.step_max > 0.f;
  float *seg_exp = adaptive ? r->seg_exp : nullptr;
  ShadeArgs sh{o.shade, {o.light[0], o.light[1], o.light[2]}, o.ambient};
  k_raygen<<<blocks_for(raygen_threads(cam.width, rows), 256), 256, 0, st>>>(
      cam, row0, rows, r->ray[0], r->next_k[0], cap, &r->counters[0], out, adaptive, sh.on ? r->aux[0] : nullptr);
  nv_status s = nv_cuda_check(cudaGetLastError(), "k_raygen launch");
  if (s != NV_OK) return s;

  const McView mv = mc_view(mc);
  // every iteration consumes at least one sample of each live ray, or ends it;
  // adaptive segments also end at every cell face a ray crosses
  int64_t max_samples = (int64_t)std::ceil(1.7320509 / (double)o.step);
  if (adaptive) max_samples = max_samples * 1025 / 1024 + 3 * (int64_t)(mv.ncx + mv.ncy + mv.ncz) + 8;
  // a shadow march follows the primary one
  const int64_t max_iter = (sh.on ? 2 : 1) * ((max_samples + K - 1) / K + 4);
  const int R = 4;  // iterations in flight before the host waits for a count
  cudaEvent_t ev[R];
  for (int j = 0; j < R; ++j) {
    e = cudaEventCreateWithFlags(&ev[j], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      for (int q = 0; q < j; ++q) cudaEventDestroy(ev[q]);
      return nv_cuda_check(e, "cudaEventCreate");
    }
  }
  int64_t bound = npix;  // upper bound of the live rays (counts only decrease)
  int64_t issued = 0, known = 0;  // iterations launched / whose count the host has read
  int cur = 0;
  while (bound > 0 && issued < max_iter) {
    const int nxt = cur ^ 1;
    int tk = net ? prof_begin(net) : -1;
    k_coords<<<blocks_for(bound, kCoordsThreads), kCoordsThreads, coords_smem(K), st>>>(
        r->ray[cur], r->next_k[cur], cap, &r->counters[cur], K, o.step, o.step_max, o.alpha_exp, mv, r->coords,
        seg_exp, r->nvalid);
    if (net) prof_end(net, NV_K_OTHER, tk);
    if ((s = nv_cuda_check(cudaGetLastError(), "k_coords launch")) != NV_OK) break;
    if (net) {
      MlpArgs a{};
      a.xyz = r->coords;
      a.y = r->values;
      a.ds = net->ds;
      a.coherent = 1;
      s = (net->prec == NV_FP32)
              ? launch_mlp_f32_ext(net, MODE_INFER, a, &r->counters[cur], K, bound * K, nullptr)
              : launch_mlp_tc_ext(net, MODE_INFER, a, &r->counters[cur], K, bound * K, nullptr);
      if (s != NV_OK) break;
    } else {
      k_values_raw<<<blocks_for(bound * K, 256), 256, 0, st>>>(*raw, r->coords, &r->counters[cur], K, r->values);
      if ((s = nv_cuda_check(cudaGetLastError(), "k_values_raw launch")) != NV_OK) break;
    }
    if ((e = cudaMemsetAsync(&r->counters[nxt], 0, sizeof(int), st)) != cudaSuccess) {
      s = nv_cuda_check(e, "cudaMemsetAsync");
      break;
    }
    tk = net ? prof_begin(net) : -1;
    k_composite<<<blocks_for(bound, 128), 128, 0, st>>>(
        r->ray[cur], r->next_k[cur], cap, &r->counters[cur], r->values, r->nvalid, seg_exp, K, lut, o.alpha_exp, o.et,
        sh, r->coords, r->aux[cur], r->aux[nxt], r->ray[nxt], r->next_k[nxt], &r->counters[nxt], out,
        reinterpret_cast<unsigned long long *>(r->d_samples));
    if (net) prof_end(net, NV_K_RENDER, tk);
    if ((s = nv_cuda_check(cudaGetLastError(), "k_composite launch")) != NV_OK) break;
    const int slot = (int)(issued % R);
    cudaMemcpyAsync(&r->h_count[slot], &r->counters[nxt], sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaEventRecord(ev[slot], st);
    ++issued;
    cur = nxt;
    // learn counts of finished iterations; block only when R iterations are in flight
    while (known < issued) {
      const int ks = (int)(known % R);
      cudaError_t q = (issued - known >= R) ? cudaEventSynchronize(ev[ks]) : cudaEventQuery(ev[ks]);
      if (q == cudaErrorNotReady) break;
      if (q != cudaSuccess) {
        s = nv_cuda_check(q, "render event");
        break;
      }
      bound = r->h_count[ks];
      ++known;
      if (bound == 0) break;
    }
    if (s != NV_OK) break;
  }
  if (s == NV_OK && bound > 0 && issued >= max_iter) {
    // the loop stopped on the iteration cap: the last live count decides
    e = cudaEventSynchronize(ev[(int)((issued - 1) % R)]);
    if (e != cudaSuccess) s = nv_cuda_check(e, "render event");
    else if (r->h_count[(int)((issued - 1) % R)] > 0)
      s = nv_fail(NV_ERR_STATE, "ray march did not finish within %lld iterations", (long long)max_iter);
  }
  r->last_iters = (int)issued;
  for (int j = 0; j < R; ++j) cudaEventDestroy(ev[j]);
  return s;
}

// The ray march of render_impl on the raw volume, for scratch the caller
// provides in `r` (ray buffers, sample batches, counters) and without any host
// allocation: no events and no pinned buffer -- the live count of each
// iteration is copied into a host stack variable and the stream synchronised.
nv_status render_raw_sync_loop(const nv_renderer &r, const nv_volume &raw, const nv_camera &cam, const float *lut,
                               const nv_macrocells *mc, const nv_render_opts &o, float *rgba, cudaStream_t st) {
  const int64_t cap = r.max_pixels;
  const int K = r.K;
  {
    const nv_status cs = coords_kernel_setup();
    if (cs != NV_OK) return cs;
  }
  cudaError_t e = cudaMemsetAsync(r.counters, 0, 2 * sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(r.d_samples, 0, sizeof(int64_t), st);
  if (e != cudaSuccess) return nv_cuda_check(e, "render memset");
  float4 *out = reinterpret_cast<float4 *>(rgba);
  k_raygen<<<blocks_for(raygen_threads(cam.width, cam.height), 256), 256, 0, st>>>(
      cam, 0, cam.height, r.ray[0], r.next_k[0], cap, &r.counters[0], out, false, nullptr);
  nv_status s = nv_cuda_check(cudaGetLastError(), "k_raygen launch");
  if (s != NV_OK) return s;
  const McView mv = mc_view(mc);
  const int64_t max_iter = (int64_t)std::ceil(1.7320509 / (double)o.step / (double)K) + 4;
  int live = 0;
  if ((e = cudaMemcpyAsync(&live, &r.counters[0], sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return nv_cuda_check(e, "render live count");
  int cur = 0;
  for (int64_t it = 0; live > 0; ++it) {
    if (it >= max_iter) return nv_fail(NV_ERR_STATE, "ray march did not finish within %lld iterations", (long long)max_iter);
    const int nxt = cur ^ 1;
    const int64_t bound = live;
    k_coords<<<blocks_for(bound, kCoordsThreads), kCoordsThreads, coords_smem(K), st>>>(
        r.ray[cur], r.next_k[cur], cap, &r.counters[cur], K, o.step, 0.f, o.alpha_exp, mv, r.coords, nullptr,
        r.nvalid);
    if ((s = nv_cuda_check(cudaGetLastError(), "k_coords launch")) != NV_OK) return s;
    k_values_raw<<<blocks_for(bound * K, 256), 256, 0, st>>>(raw, r.coords, &r.counters[cur], K, r.values);
    if ((s = nv_cuda_check(cudaGetLastError(), "k_values_raw launch")) != NV_OK) return s;
    if ((e = cudaMemsetAsync(&r.counters[nxt], 0, sizeof(int), st)) != cudaSuccess)
      return nv_cuda_check(e, "cudaMemsetAsync");
    k_composite<<<blocks_for(bound, 128), 128, 0, st>>>(
        r.ray[cur], r.next_k[cur], cap, &r.counters[cur], r.values, r.nvalid, nullptr, K, lut, o.alpha_exp, o.et,
        ShadeArgs{}, r.coords, nullptr, nullptr, r.ray[nxt],
        r.next_k[nxt], &r.counters[nxt], out, reinterpret_cast<unsigned long long *>(r.d_samples));
    if ((s = nv_cuda_check(cudaGetLastError(), "k_composite launch")) != NV_OK) return s;
    if ((e = cudaMemcpyAsync(&live, &r.counters[nxt], sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return nv_cuda_check(e, "render live count");
    cur = nxt;
  }
  return NV_OK;
}

namespace {
// A-16: FP64 sum of squared differences of two float arrays; each CTA adds partial / n.
__global__ void __launch_bounds__(256) k_mse(const float *__restrict__ a, const float *__restrict__ b, int64_t n,
                                             double scale, double *out) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = (double)a[i] - (double)b[i];
    s += d * d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double part[8];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    atomicAdd(out, t * scale);
  }
}
}  // namespace

nv_status launch_mse(const float *a, const float *b, int64_t n, double *out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
  if (e != cudaSuccess) return nv_cuda_check(e, "cudaMemsetAsync");
  if (n == 0) return NV_OK;
  unsigned grid = (unsigned)std::min<int64_t>(blocks_for(n, 256), 1216);
  k_mse<<<grid, 256, 0, s>>>(a, b, n, 1.0 / (double)n, out);
  return nv_cuda_check(cudaGetLastError(), "k_mse launch");
}

// k_pt.cu -- volumetric path tracing with sample streaming (Sec. 5.2.2,
// Alg. 1, Eq. 1-2).
//
// Each live path holds one tentative collision at a time.  Per iteration:
//   network inference on the tentative collision points of all live paths
//   (the tensor-core or FP32 MLP kernels; the raw volume is read inline)
//   k_pt_shade  accept or reject each collision (Woodcock: probability
//               sigma(x) / majorant), advance the path's state machine
//               (scattering ray -> shadow ray towards the light -> scattering
//               with roulette and an isotropic direction), find its next
//               tentative collision by a Hofmann macrocell flight, and compact
//               the paths that continue
// The ray-generation kernel runs the first flight itself, as the paper's
// ray-generation and shading kernels absorb the sample computation.
//
// Readings (the paper names the method, not its constants; the oracle's
// or_render_pt states the same): extinction sigma = D * LUT opacity per unit
// length, albedo = LUT colour, isotropic phase, one directional light whose
// irradiance cancels the phase factor, black background.  Random numbers are
// Philox4x32-10 blocks, key = seed, counter = (pixel, event, frame, 0).  Every
// decision (cell walk, collision point, acceptance, roulette) is taken in FP32
// with each operation rounded on its own, and for the raw volume the density
// is evaluated the same way, so paths match the oracle's.
#include "nv_internal.cuh"
#include "render_common.cuh"

namespace {

constexpr float kTiny = 9.5367431640625e-07f;  // 2^-20: cell lookups just past a position

// per-path state, [kPtN][cap] floats (integers as bits)
enum {
  P_OX = 0, P_OY, P_OZ, P_DX, P_DY, P_DZ, P_T, P_T1,  // the current ray and its parameter range
  P_XX, P_XY, P_XZ,                                   // the last real scattering point
  P_AR, P_AG, P_AB,                                   // its albedo
  P_BR, P_BG, P_BB,                                   // throughput
  P_LR, P_LG, P_LB,                                   // radiance
  P_TC, P_MU, P_XI,                                   // pending tentative collision: t, majorant, accept draw
  P_MODE, P_BOUNCE, P_EV, P_PIX, P_HIT,
  kPtN
};

struct PtArgs {
  float density;
  float light[3];
  int max_bounces;
  uint2 key;
  uint32_t frame;
  McView mc;
};

__device__ __forceinline__ float u01(uint32_t x) { return __fmul_rn((float)(x >> 8), 5.9604644775390625e-08f); }

__device__ __forceinline__ uint4 pt_block(uint32_t pix, uint32_t ev, const PtArgs &a) {
  return nv_philox(make_uint4(pix, ev, a.frame, 0u), a.key.x, a.key.y);
}

// FP32 trilinear of the raw volume with every operation rounded on its own.
__device__ __forceinline__ float trilinear_rn(const nv_volume &v, const float *x) {
  const int n[3] = {v.nx, v.ny, v.nz};
  int i0[3], i1[3];
  float w[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (n[a] == 1) {
      i0[a] = 0;
      i1[a] = 0;
      w[a] = 0.f;
      continue;
    }
    float q = __fadd_rn(__fmul_rn(x[a], (float)n[a]), -0.5f);
    q = fminf(fmaxf(q, 0.0f), (float)(n[a] - 1));
    const int i = min((int)floorf(q), n[a] - 2);
    i0[a] = i;
    i1[a] = i + 1;
    w[a] = __fsub_rn(q, (float)i);
  }
  const int64_t sy = v.nx, sz = (int64_t)v.nx * v.ny;
  float c[2][2];
#pragma unroll
  for (int zz = 0; zz < 2; ++zz)
#pragma unroll
    for (int yy = 0; yy < 2; ++yy) {
      const float *row = v.data_dev + (int64_t)(zz ? i1[2] : i0[2]) * sz + (int64_t)(yy ? i1[1] : i0[1]) * sy;
      const float a0 = __ldg(row + i0[0]), a1 = __ldg(row + i1[0]);
      c[zz][yy] = __fadd_rn(a0, __fmul_rn(w[0], __fsub_rn(a1, a0)));
    }
  const float e0 = __fadd_rn(c[0][0], __fmul_rn(w[1], __fsub_rn(c[0][1], c[0][0])));
  const float e1 = __fadd_rn(c[1][0], __fmul_rn(w[1], __fsub_rn(c[1][1], c[1][0])));
  return __fadd_rn(e0, __fmul_rn(w[2], __fsub_rn(e1, e0)));
}

// Transfer function with every operation rounded on its own.
__device__ __forceinline__ float4 tf_rn(const float *__restrict__ lut, float v) {
  const float u = __fmul_rn(fminf(fmaxf(v, 0.0f), 1.0f), 255.0f);
  const int e = min((int)floorf(u), 254);
  const float w = __fsub_rn(u, (float)e);
  const float4 l0 = __ldg(reinterpret_cast<const float4 *>(lut) + e);
  const float4 l1 = __ldg(reinterpret_cast<const float4 *>(lut) + e + 1);
  return make_float4(__fadd_rn(l0.x, __fmul_rn(w, __fsub_rn(l1.x, l0.x))),
                     __fadd_rn(l0.y, __fmul_rn(w, __fsub_rn(l1.y, l0.y))),
                     __fadd_rn(l0.z, __fmul_rn(w, __fsub_rn(l1.z, l0.z))),
                     __fadd_rn(l0.w, __fmul_rn(w, __fsub_rn(l1.w, l0.w))));
}

// One Woodcock flight from t (Hofmann's macrocell walk, Eq. 1-2): the target
// optical thickness tau is spent cell by cell; true with the tentative
// collision *tc inside the cell where it runs out and that cell's majorant.
__device__ __forceinline__ bool flight(const float *o, const float *d, float t, float t1, float tau, float D,
                                       const McView &mc, float &tc, float &muc) {
  const float sc[3] = {mc.sx, mc.sy, mc.sz};
  const int nc[3] = {mc.ncx, mc.ncy, mc.ncz};
  float acc = 0.f;
  for (int guard = 0; guard < (1 << 20); ++guard) {
    if (!(t < t1)) return false;
    const float tl = __fadd_rn(t, kTiny);
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float p = __fadd_rn(o[a], __fmul_rn(tl, d[a]));
      c[a] = min(max((int)floorf(__fmul_rn(p, sc[a])), 0), nc[a] - 1);
    }
    float texit = __int_as_float(0x7f800000);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (d[a] != 0.f) {
        const float face = __fdiv_rn((float)(d[a] > 0.f ? c[a] + 1 : c[a]), sc[a]);
        texit = fminf(texit, __fdiv_rn(__fsub_rn(face, o[a]), d[a]));
      }
    }
    texit = fminf(texit, t1);
    float seg = __fsub_rn(texit, t);
    if (!(seg > kTiny)) seg = kTiny;
    const float mu = __fmul_rn(D, __ldg(mc.mu + ((int64_t)c[2] * mc.ncy + c[1]) * mc.ncx + c[0]));
    const float next = __fadd_rn(acc, __fmul_rn(mu, seg));
    if (mu > 0.f && next >= tau) {
      const float tcol = __fadd_rn(t, __fdiv_rn(__fsub_rn(tau, acc), mu));
      tc = fminf(tcol, __fadd_rn(t, seg));
      muc = mu;
      return true;
    }
    acc = next;
    t = __fadd_rn(t, seg);
  }
  return false;
}

struct Path {
  float o[3], d[3], t, t1;
  float xs[3], al[3], beta[3], L[3];
  float tc, muc, xi;
  int mode, bounce;
  uint32_t ev, pix;
  float hit;
};

__device__ __forceinline__ void load(const float *s, int64_t cap, int64_t i, Path &p) {
  p.o[0] = s[P_OX * cap + i]; p.o[1] = s[P_OY * cap + i]; p.o[2] = s[P_OZ * cap + i];
  p.d[0] = s[P_DX * cap + i]; p.d[1] = s[P_DY * cap + i]; p.d[2] = s[P_DZ * cap + i];
  p.t = s[P_T * cap + i]; p.t1 = s[P_T1 * cap + i];
  p.xs[0] = s[P_XX * cap + i]; p.xs[1] = s[P_XY * cap + i]; p.xs[2] = s[P_XZ * cap + i];
  p.al[0] = s[P_AR * cap + i]; p.al[1] = s[P_AG * cap + i]; p.al[2] = s[P_AB * cap + i];
  p.beta[0] = s[P_BR * cap + i]; p.beta[1] = s[P_BG * cap + i]; p.beta[2] = s[P_BB * cap + i];
  p.L[0] = s[P_LR * cap + i]; p.L[1] = s[P_LG * cap + i]; p.L[2] = s[P_LB * cap + i];
  p.tc = s[P_TC * cap + i]; p.muc = s[P_MU * cap + i]; p.xi = s[P_XI * cap + i];
  p.mode = __float_as_int(s[P_MODE * cap + i]);
  p.bounce = __float_as_int(s[P_BOUNCE * cap + i]);
  p.ev = (uint32_t)__float_as_int(s[P_EV * cap + i]);
  p.pix = (uint32_t)__float_as_int(s[P_PIX * cap + i]);
  p.hit = s[P_HIT * cap + i];
}

__device__ __forceinline__ void store(float *s, int64_t cap, int64_t i, const Path &p) {
  s[P_OX * cap + i] = p.o[0]; s[P_OY * cap + i] = p.o[1]; s[P_OZ * cap + i] = p.o[2];
  s[P_DX * cap + i] = p.d[0]; s[P_DY * cap + i] = p.d[1]; s[P_DZ * cap + i] = p.d[2];
  s[P_T * cap + i] = p.t; s[P_T1 * cap + i] = p.t1;
  s[P_XX * cap + i] = p.xs[0]; s[P_XY * cap + i] = p.xs[1]; s[P_XZ * cap + i] = p.xs[2];
  s[P_AR * cap + i] = p.al[0]; s[P_AG * cap + i] = p.al[1]; s[P_AB * cap + i] = p.al[2];
  s[P_BR * cap + i] = p.beta[0]; s[P_BG * cap + i] = p.beta[1]; s[P_BB * cap + i] = p.beta[2];
  s[P_LR * cap + i] = p.L[0]; s[P_LG * cap + i] = p.L[1]; s[P_LB * cap + i] = p.L[2];
  s[P_TC * cap + i] = p.tc; s[P_MU * cap + i] = p.muc; s[P_XI * cap + i] = p.xi;
  s[P_MODE * cap + i] = __int_as_float(p.mode);
  s[P_BOUNCE * cap + i] = __int_as_float(p.bounce);
  s[P_EV * cap + i] = __int_as_float((int)p.ev);
  s[P_PIX * cap + i] = __int_as_float((int)p.pix);
  s[P_HIT * cap + i] = p.hit;
}

// The scattering after a real collision has been resolved by its shadow ray:
// throughput *= albedo, bounce count, roulette and an isotropic direction.
// False when the path ends.
__device__ __forceinline__ bool scatter(Path &p, const PtArgs &a) {
#pragma unroll
  for (int c = 0; c < 3; ++c) p.beta[c] = __fmul_rn(p.beta[c], p.al[c]);
  ++p.bounce;
  if (p.bounce >= a.max_bounces) return false;
  const uint4 u = pt_block(p.pix, p.ev++, a);
  if (p.bounce >= 3) {
    const float q = fminf(1.0f, fmaxf(p.beta[0], fmaxf(p.beta[1], p.beta[2])));
    if (!(u01(u.z) < q)) return false;
#pragma unroll
    for (int c = 0; c < 3; ++c) p.beta[c] = __fdiv_rn(p.beta[c], q);
  }
  const double z = 1.0 - 2.0 * (double)u01(u.x);
  const double r = sqrt(fmax(0.0, 1.0 - z * z));
  const double phi = 6.283185307179586 * (double)u01(u.y);
#pragma unroll
  for (int c = 0; c < 3; ++c) p.o[c] = p.xs[c];
  p.d[0] = (float)(r * cos(phi));
  p.d[1] = (float)(r * sin(phi));
  p.d[2] = (float)z;
  p.mode = 0;
  float t0, t1;
  if (!nv_box(p.o, p.d, t0, t1)) return false;
  p.t = t0;
  p.t1 = t1;
  return true;
}

// Find the path's next tentative collision (its flight draws one block).  A
// shadow ray that leaves the volume makes the light visible and hands over to
// the scattering.  False when the path ends; else pos = the collision point.
__device__ __forceinline__ bool next_collision(Path &p, const PtArgs &a, float *pos) {
  for (int guard = 0; guard < 4 * 64 + 8; ++guard) {
    const uint4 u = pt_block(p.pix, p.ev++, a);
    const float tau = (float)(-log1p(-(double)u01(u.x)));
    float tc, muc;
    if (flight(p.o, p.d, p.t, p.t1, tau, a.density, a.mc, tc, muc)) {
      p.tc = tc;
      p.muc = muc;
      p.xi = u01(u.y);
#pragma unroll
      for (int c = 0; c < 3; ++c) pos[c] = __fadd_rn(p.o[c], __fmul_rn(tc, p.d[c]));
      return true;
    }
    if (p.mode == 0) return false;  // the scattering ray left the volume
    // the shadow ray left the volume: the light is visible from the scattering point
#pragma unroll
    for (int c = 0; c < 3; ++c) p.L[c] = __fadd_rn(p.L[c], __fmul_rn(p.beta[c], p.al[c]));
    if (!scatter(p, a)) return false;
  }
  return false;
}

__device__ __forceinline__ int warp_append_pt(int *counter, bool pred) {
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

__device__ __forceinline__ void finish(const Path &p, float4 *rgba) {
  rgba[p.pix] = make_float4(p.L[0], p.L[1], p.L[2], p.hit);
}

__global__ void k_pt_raygen(nv_camera cam, PtArgs a, float *st, int64_t cap, float *coords, int *count,
                            float4 *rgba) {
  const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t npix = (int64_t)cam.width * cam.height;
  bool live = false;
  Path p;
  float pos[3] = {0.f, 0.f, 0.f};
  if (pix < npix) {
    float t0 = 0.f, t1 = 0.f;
    nv_camera_ray(cam, (int)(pix % cam.width), (int)(pix / cam.width), p.o, p.d);
    const bool hit = nv_box(p.o, p.d, t0, t1);
    p.t = t0;
    p.t1 = t1;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      p.xs[c] = 0.f;
      p.al[c] = 0.f;
      p.beta[c] = 1.f;
      p.L[c] = 0.f;
    }
    p.tc = p.muc = p.xi = 0.f;
    p.mode = 0;
    p.bounce = 0;
    p.ev = 0;
    p.pix = (uint32_t)pix;
    p.hit = 0.f;
    live = hit && next_collision(p, a, pos);
    if (!live) finish(p, rgba);
  }
  const int slot = warp_append_pt(count, live);
  if (live) {
    store(st, cap, slot, p);
    coords[3 * slot] = pos[0];
    coords[3 * slot + 1] = pos[1];
    coords[3 * slot + 2] = pos[2];
  }
}

// values (nullable): network values of the pending collisions; NULL: raw volume inline.
__global__ void k_pt_shade(PtArgs a, const float *__restrict__ lut, const float *__restrict__ values,
                           nv_volume raw, const float *__restrict__ st, int64_t cap, const float *__restrict__ coords,
                           const int *count, float *st_out, float *coords_out, int *count_out, float4 *rgba,
                           unsigned long long *samples) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int n = *count;
  bool live = false;
  Path p;
  float pos[3] = {0.f, 0.f, 0.f};
  if (i < n) {
    load(st, cap, i, p);
    const float x[3] = {coords[3 * i], coords[3 * i + 1], coords[3 * i + 2]};
    const float v = values ? values[i] : trilinear_rn(raw, x);
    const float4 c = tf_rn(lut, v);
    const float ratio = __fdiv_rn(__fmul_rn(a.density, c.w), p.muc);
    bool go;
    if (!(p.xi < ratio)) {  // null collision: fly on from it
      p.t = p.tc;
      go = true;
    } else if (p.mode == 0) {  // real scattering collision: a shadow ray towards the light
      p.hit = 1.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) p.xs[k] = x[k];
      p.al[0] = c.x;
      p.al[1] = c.y;
      p.al[2] = c.z;
      p.mode = 1;
      float s0, s1;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        p.o[k] = x[k];
        p.d[k] = a.light[k];
      }
      if (nv_box(p.o, p.d, s0, s1)) {
        p.t = s0;
        p.t1 = s1;
        go = true;
      } else {  // no interval in the volume: nothing blocks the light
#pragma unroll
        for (int k = 0; k < 3; ++k) p.L[k] = __fadd_rn(p.L[k], __fmul_rn(p.beta[k], p.al[k]));
        go = scatter(p, a);
      }
    } else {  // the shadow ray hit the medium: the light is blocked
      go = scatter(p, a);
    }
    live = go && next_collision(p, a, pos);
    if (!live) finish(p, rgba);
  }
  const unsigned m = __ballot_sync(0xffffffffu, i < n);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(samples, (unsigned long long)__popc(m));
  const int slot = warp_append_pt(count_out, live);
  if (live) {
    store(st_out, cap, slot, p);
    coords_out[3 * slot] = pos[0];
    coords_out[3 * slot + 1] = pos[1];
    coords_out[3 * slot + 2] = pos[2];
  }
}

inline unsigned blocks_for(int64_t n, int bs) { return (unsigned)std::max<int64_t>(1, (n + bs - 1) / bs); }

}  // namespace

nv_status render_pt_impl(nv_renderer *r, nv_ctx *net, const nv_volume *raw, const nv_camera &cam, const float *lut,
                         const nv_macrocells &mc, const nv_pt_opts &o, float *rgba) {
  const int64_t npix = (int64_t)cam.width * cam.height;
  const int64_t cap = r->max_pixels;
  cudaStream_t st = net ? net->stream : r->stream;
  if (!r->pt[0]) {
    cudaError_t e = cudaMalloc(&r->pt[0], (size_t)cap * kPtN * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&r->pt[1], (size_t)cap * kPtN * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&r->pt_coords, (size_t)cap * 3 * sizeof(float));
    if (e != cudaSuccess) return nv_cuda_check(e, "path-tracer state");
  }
  PtArgs a;
  a.density = o.density;
  a.light[0] = o.light[0];
  a.light[1] = o.light[1];
  a.light[2] = o.light[2];
  a.max_bounces = o.max_bounces;
  a.key = make_uint2((uint32_t)o.seed, (uint32_t)(o.seed >> 32));
  a.frame = o.frame;
  a.mc = mc_view(&mc);
  cudaError_t e = cudaMemsetAsync(r->counters, 0, 2 * sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(r->d_samples, 0, sizeof(int64_t), st);
  if (e != cudaSuccess) return nv_cuda_check(e, "path-tracer memset");
  float4 *out = reinterpret_cast<float4 *>(rgba);
  float *coords[2] = {r->coords, r->pt_coords};
  k_pt_raygen<<<blocks_for(npix, 128), 128, 0, st>>>(cam, a, r->pt[0], cap, coords[0], &r->counters[0], out);
  nv_status s = nv_cuda_check(cudaGetLastError(), "k_pt_raygen launch");
  if (s != NV_OK) return s;
  const int64_t max_iter = 1 << 16;
  const int R = 4;
  cudaEvent_t ev[R];
  for (int j = 0; j < R; ++j) {
    e = cudaEventCreateWithFlags(&ev[j], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      for (int q = 0; q < j; ++q) cudaEventDestroy(ev[q]);
      return nv_cuda_check(e, "cudaEventCreate");
    }
  }
  int64_t bound = npix, issued = 0, known = 0;
  int cur = 0;
  while (bound > 0 && issued < max_iter) {
    const int nxt = cur ^ 1;
    const float *vals = nullptr;
    if (net) {
      MlpArgs m{};
      m.xyz = coords[cur];
      m.y = r->values;
      m.ds = net->ds;
      s = (net->prec == NV_FP32) ? launch_mlp_f32_ext(net, MODE_INFER, m, &r->counters[cur], 1, bound, nullptr)
                                 : launch_mlp_tc_ext(net, MODE_INFER, m, &r->counters[cur], 1, bound, nullptr);
      if (s != NV_OK) break;
      vals = r->values;
    }
    if ((e = cudaMemsetAsync(&r->counters[nxt], 0, sizeof(int), st)) != cudaSuccess) {
      s = nv_cuda_check(e, "cudaMemsetAsync");
      break;
    }
    const int tk = net ? prof_begin(net) : -1;
    k_pt_shade<<<blocks_for(bound, 128), 128, 0, st>>>(a, lut, vals, raw ? *raw : nv_volume{}, r->pt[cur], cap,
                                                       coords[cur], &r->counters[cur], r->pt[nxt], coords[nxt],
                                                       &r->counters[nxt], out,
                                                       reinterpret_cast<unsigned long long *>(r->d_samples));
    if (net) prof_end(net, NV_K_RENDER, tk);
    if ((s = nv_cuda_check(cudaGetLastError(), "k_pt_shade launch")) != NV_OK) break;
    const int slot = (int)(issued % R);
    cudaMemcpyAsync(&r->h_count[slot], &r->counters[nxt], sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaEventRecord(ev[slot], st);
    ++issued;
    cur = nxt;
    while (known < issued) {
      const int ks = (int)(known % R);
      cudaError_t q = (issued - known >= R) ? cudaEventSynchronize(ev[ks]) : cudaEventQuery(ev[ks]);
      if (q == cudaErrorNotReady) break;
      if (q != cudaSuccess) {
        s = nv_cuda_check(q, "path-tracer event");
        break;
      }
      bound = r->h_count[ks];
      ++known;
      if (bound == 0) break;
    }
    if (s != NV_OK) break;
  }
  if (s == NV_OK && bound > 0 && issued >= max_iter) {
    e = cudaEventSynchronize(ev[(int)((issued - 1) % R)]);
    if (e != cudaSuccess) s = nv_cuda_check(e, "path-tracer event");
    else if (r->h_count[(int)((issued - 1) % R)] > 0)
      s = nv_fail(NV_ERR_STATE, "path tracing did not finish within %lld iterations", (long long)max_iter);
  }
  r->last_iters = (int)issued;
  for (int j = 0; j < R; ++j) cudaEventDestroy(ev[j]);
  return s;
}

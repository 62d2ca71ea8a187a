// render_common.cuh -- per-ray pieces of the emission-absorption ray march
// shared by the sample-streaming kernels (k_render.cu) and the in-shader
// megakernel (k_inshader.cu), so both take the same samples and composite
// them with the same arithmetic.
#pragma once

#include "nv_internal.cuh"

struct McView {
  const float *mu;  // nullptr: no skipping
  int ncx, ncy, ncz;
  float sx, sy, sz;  // cells per unit length along each axis (n / cell)
};

inline McView mc_view(const nv_macrocells *mc) {
  McView mv{nullptr, 1, 1, 1, 0.f, 0.f, 0.f};
  if (mc) {
    mv.mu = mc->mu_max_dev;
    mv.ncx = (mc->nx + mc->cell - 1) / mc->cell;
    mv.ncy = (mc->ny + mc->cell - 1) / mc->cell;
    mv.ncz = (mc->nz + mc->cell - 1) / mc->cell;
    mv.sx = (float)mc->nx / (float)mc->cell;
    mv.sy = (float)mc->ny / (float)mc->cell;
    mv.sz = (float)mc->nz / (float)mc->cell;
  }
  return mv;
}

// A-12, one step of the walk along a ray.  Sample k sits at t_k = t0 + (k +
// 1/2) step (FP32, the same operations as the oracle).  A sample inside a
// transparent macrocell (mu_max == 0, Sec. 5.3) is skipped: the walk jumps to
// two samples before the cell's exit, so every sample near a cell face is
// still tested on its own, which makes the skipped set exactly the per-sample
// definition.  Returns kMarchEnd once t_k >= t1, kMarchSkip after moving k
// past a transparent stretch, kMarchSample with pos = the position of sample k
// (k unchanged).  Callers loop one step per iteration, so the lanes of a warp
// that skip and the lanes that take samples advance together.
enum { kMarchEnd = 0, kMarchSample = 1, kMarchSkip = 2 };

// McCache: the last macrocell a ray looked up and its mu_max (idx -1: none), so
// the run of samples inside one cell loads its value once.  The in-shader
// kernel keeps it across its iterations; the streaming march's walk (whose
// lookups hit L1) measured 2-4% slower with it and passes none.
struct McCache {
  int idx = -1;
  float mu = 0.f;
};

__device__ __forceinline__ float mc_lookup(const McView &mc, int cx, int cy, int cz, McCache *cache) {
  const int ci = (cz * mc.ncy + cy) * mc.ncx + cx;
  if (!cache) return __ldg(mc.mu + ci);
  if (ci != cache->idx) {
    cache->idx = ci;
    cache->mu = __ldg(mc.mu + ci);
  }
  return cache->mu;
}

__device__ __forceinline__ int march_step(const float *o, const float *d, float t0, float t1, float step,
                                          const McView &mc, int &k, float *pos, McCache *cache = nullptr) {
  const float tk = __fadd_rn(t0, __fmul_rn(__fadd_rn((float)k, 0.5f), step));
  if (!(tk < t1)) return kMarchEnd;
#pragma unroll
  for (int a = 0; a < 3; ++a) pos[a] = __fadd_rn(o[a], __fmul_rn(tk, d[a]));
  if (!mc.mu) return kMarchSample;
  const int cx = min(max((int)floorf(__fmul_rn(pos[0], mc.sx)), 0), mc.ncx - 1);
  const int cy = min(max((int)floorf(__fmul_rn(pos[1], mc.sy)), 0), mc.ncy - 1);
  const int cz = min(max((int)floorf(__fmul_rn(pos[2], mc.sz)), 0), mc.ncz - 1);
  if (mc_lookup(mc, cx, cy, cz, cache) != 0.0f) return kMarchSample;
  // exit distance of this cell along the ray, approximate (fast divisions: a
  // few units in the last place, far inside the two-sample margin below); it
  // only decides how far to jump, never which samples are taken
  const int cc[3] = {cx, cy, cz};
  const float sc[3] = {mc.sx, mc.sy, mc.sz};
  float texit = __int_as_float(0x7f800000);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (d[a] > 0.f) texit = fminf(texit, __fdividef(__fdividef((float)(cc[a] + 1), sc[a]) - o[a], d[a]));
    else if (d[a] < 0.f) texit = fminf(texit, __fdividef(__fdividef((float)cc[a], sc[a]) - o[a], d[a]));
  }
  const float kf = ceilf(__fdividef(texit - t0, step) - 0.5f) - 2.0f;
  int kj = k + 1;
  if (kf > (float)kj) kj = (kf < 2.0e9f) ? (int)kf : 2000000000;
  k = kj;
  return kMarchSkip;
}

// Adaptive step (Sec. 5.3, Eq. 3), one step of the walk from the ray
// parameter t, every FP32 operation rounded on its own as in the oracle.  The
// cell is looked up just past the start (t + s1 / 1024), so a ray standing on
// a face moves on into the next cell; the segment runs to the nearest of that
// cell's exit, t1 and t + s_bar, s_bar = max(s1 + (s2 - s1) (1 - min(mu, 1))^2,
// s1), and is at least s1 / 1024 long.  A transparent cell (mu == 0) is crossed
// without a sample (kMarchSkip).  kMarchSample: pos = the segment midpoint and
// e = alpha_exp * seg / s1, the opacity-correction exponent of its length;
// t moves to the end of the segment.  Needs macrocells (mc.mu != NULL).
__device__ __forceinline__ int march_step_adaptive(const float *o, const float *d, float t1, float s1, float s2,
                                                   float alpha_exp, const McView &mc, float &t, float *pos,
                                                   float &e) {
  if (!(t < t1)) return kMarchEnd;
  const float tiny = __fmul_rn(s1, 0.0009765625f);
  const float tc = __fadd_rn(t, tiny);
  const float sc[3] = {mc.sx, mc.sy, mc.sz};
  const int nc[3] = {mc.ncx, mc.ncy, mc.ncz};
  int c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float p = __fadd_rn(o[a], __fmul_rn(tc, d[a]));
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
  float room = __fsub_rn(texit, t);
  if (!(room > tiny)) room = tiny;
  const float mu = __ldg(mc.mu + ((int64_t)c[2] * mc.ncy + c[1]) * mc.ncx + c[0]);
  if (mu == 0.0f) {
    t = __fadd_rn(t, room);
    return kMarchSkip;
  }
  const float q = __fsub_rn(1.0f, fminf(mu, 1.0f));
  const float grow = __fmul_rn(__fsub_rn(s2, s1), __fmul_rn(q, q));
  const float sbar = fmaxf(__fadd_rn(s1, grow), s1);
  const float seg = fminf(sbar, room);
  const float tm = __fadd_rn(t, __fmul_rn(0.5f, seg));
#pragma unroll
  for (int a = 0; a < 3; ++a) pos[a] = __fadd_rn(o[a], __fmul_rn(tm, d[a]));
  e = __fmul_rn(alpha_exp, __fdiv_rn(seg, s1));
  t = __fadd_rn(t, seg);
  return kMarchSample;
}

// A-14 for one sample value v: transfer function (linear between the 256 LUT
// entries), opacity correction a' = 1 - (1 - a)^e, front-to-back compositing.
// Returns true once the accumulated opacity reaches et (early termination).
__device__ __forceinline__ void tf_lookup(float v, const float *__restrict__ lut, float alpha_exp, float &r,
                                          float &g, float &b, float &ac) {
  const float u = __fmul_rn(fminf(fmaxf(v, 0.f), 1.f), 255.0f);
  const int e = min((int)floorf(u), 254);
  const float w = u - (float)e;
  const float4 l0 = __ldg(reinterpret_cast<const float4 *>(lut) + e);
  const float4 l1 = __ldg(reinterpret_cast<const float4 *>(lut) + e + 1);
  r = l0.x + w * (l1.x - l0.x);
  g = l0.y + w * (l1.y - l0.y);
  b = l0.z + w * (l1.z - l0.z);
  const float al = l0.w + w * (l1.w - l0.w);
  // a' = 1 - (1 - a)^e, as -expm1(e log1p(-a)) to keep small opacities accurate
  ac = (alpha_exp == 1.0f) ? al : -expm1f(alpha_exp * log1pf(-al));
}

// w (nullable) receives the sample's contribution (1 - A) a'.
__device__ __forceinline__ bool composite_one(float v, const float *__restrict__ lut, float alpha_exp, float et,
                                              float &cr, float &cg, float &cb, float &ca, float *w = nullptr) {
  float r, g, b, ac;
  tf_lookup(v, lut, alpha_exp, r, g, b, ac);
  const float tr = (1.0f - ca) * ac;
  cr += tr * r;
  cg += tr * g;
  cb += tr * b;
  ca += tr;
  if (w) *w = tr;
  return ca >= et;
}

// Single-shot heuristic shadows (Sec. 5): per-ray state beside the ray
// buffers, [kAuxN][cap] floats: the best contribution so far, its position,
// and the opacity of the shadow march (negative during the primary march).
enum { AUX_BW = 0, AUX_BX, AUX_BY, AUX_BZ, AUX_AS, kAuxN };
struct ShadeArgs {
  int on;          // 1: single-shot shadows
  float light[3];  // unit direction towards the directional light
  float ambient;   // colour scale where the light is fully blocked
};

// One sample of the shadow march (opacity only): as += (1 - as) a', every
// operation rounded on its own so the streaming and in-shader marches agree
// bit for bit; returns whether the march stops (as >= et).
__device__ __forceinline__ bool shadow_one(float v, const float *__restrict__ lut, float alpha_exp, float et,
                                           float &as) {
  float r, g, b, ac;
  tf_lookup(v, lut, alpha_exp, r, g, b, ac);
  as = __fadd_rn(as, __fmul_rn(__fsub_rn(1.0f, as), ac));
  return as >= et;
}

// The colour of a shaded ray: C (ambient + (1 - ambient) T), T = 1 - as.
__device__ __forceinline__ void shade_colour(const ShadeArgs &sh, float as, float &cr, float &cg, float &cb) {
  const float k = __fadd_rn(sh.ambient, __fmul_rn(__fsub_rn(1.0f, sh.ambient), __fsub_rn(1.0f, as)));
  cr = __fmul_rn(cr, k);
  cg = __fmul_rn(cg, k);
  cb = __fmul_rn(cb, k);
}

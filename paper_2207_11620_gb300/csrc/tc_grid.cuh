// tc_grid.cuh -- device pieces shared by the tensor-core path's kernels: the
// source of a work item's point, the chunk a launch covers, the tensor-core
// tile layout of features in memory, 16-bit packing, and the x-paired hash
// gather (A-1..A-3) and scatter (A-7).
#pragma once

#include "nv_internal.cuh"
#include "tc_ptx.cuh"

// Where the points of a launch come from.
struct PointSrc {
  const float *xyz;   // kind 0: [n][3] (point p at row p - xyz_off)
  int64_t xyz_off;
  int kind;           // 0: xyz array, 1: voxel centres of vol, 2: Philox training sample
  nv_volume vol;      // kind 1 and the training target of kind 2
  uint64_t seed;      // kind 2
  uint32_t step;      // kind 2
};

__device__ __forceinline__ float3 point_at(const PointSrc &s, int64_t p) {
  if (s.kind == 0) {
    const float *r = s.xyz + 3 * (p - s.xyz_off);
    return make_float3(r[0], r[1], r[2]);
  }
  if (s.kind == 1) {
    const int64_t nx = s.vol.nx, ny = s.vol.ny;
    const int ix = (int)(p % nx), iy = (int)((p / nx) % ny), iz = (int)(p / (nx * ny));
    return make_float3(__fdiv_rn(__fadd_rn((float)ix, 0.5f), (float)s.vol.nx),
                       __fdiv_rn(__fadd_rn((float)iy, 0.5f), (float)s.vol.ny),
                       __fdiv_rn(__fadd_rn((float)iz, 0.5f), (float)s.vol.nz));
  }
  return nv_sample_point(s.seed, s.step, (uint64_t)p);
}

// The points [off, off + cap) of a launch; the total is n_host, or read on the
// device as *n_dev * n_mult (the live samples of a render iteration).
struct ChunkSpan {
  const int *n_dev;
  int n_mult;
  int64_t n_host;
  int64_t off;
  int64_t cap;
};

__device__ __forceinline__ int64_t chunk_count(const ChunkSpan &c) {
  const int64_t tot = c.n_dev ? (int64_t)(*c.n_dev) * c.n_mult : c.n_host;
  int64_t n = tot - c.off;
  if (n < 0) n = 0;
  if (n > c.cap) n = c.cap;
  return n;
}

// Byte offset of element (r, k) of a [rows][K] 16-bit operand stored as
// no-swizzle core matrices: 8 rows x 16 B blocks, K-chunks adjacent, 8-row
// groups K * 16 B apart.
__host__ __device__ __forceinline__ uint32_t tile_off(int r, int k, int K) {
  return (uint32_t)((r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

template <bool BF>
struct Half;
template <>
struct Half<false> {
  using T = __half;
  using T2 = __half2;
  static __device__ __forceinline__ T2 pack(float a, float b) { return __floats2half2_rn(a, b); }
  static __device__ __forceinline__ float2 unpack(T2 v) { return __half22float2(v); }
  static __device__ __forceinline__ float lo(T v) { return __half2float(v); }
};
template <>
struct Half<true> {
  using T = __nv_bfloat16;
  using T2 = __nv_bfloat162;
  static __device__ __forceinline__ T2 pack(float a, float b) { return __floats2bfloat162_rn(a, b); }
  static __device__ __forceinline__ float2 unpack(T2 v) { return __bfloat1622float2(v); }
  static __device__ __forceinline__ float lo(T v) { return __bfloat162float(v); }
};

template <bool BF>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  typename Half<BF>::T2 h = Half<BF>::pack(a, b);
  return *reinterpret_cast<uint32_t *>(&h);
}

template <bool BF>
__device__ __forceinline__ uint32_t pack16x2(float a, float b) {
  typename Half<BF>::T2 h = Half<BF>::pack(a, b);
  return *reinterpret_cast<uint32_t *>(&h);
}

// Store 8 consecutive K values (one 16-byte core-matrix row) of row r.
template <bool BF>
__device__ __forceinline__ void st_row8(uint8_t *base, int r, int c, int K, const float *v) {
  uint4 u;
  u.x = pack16x2<BF>(v[0], v[1]);
  u.y = pack16x2<BF>(v[2], v[3]);
  u.z = pack16x2<BF>(v[4], v[5]);
  u.w = pack16x2<BF>(v[6], v[7]);
  *reinterpret_cast<uint4 *>(base + tile_off(r, c * 8, K)) = u;
}

// max(a, 0) and max(b, 0) rounded to 16 bits and packed (a in the low half):
// one conversion with the ReLU built in.  Rounding commutes with the clamp, so
// this equals pack16x2(fmaxf(a, 0), fmaxf(b, 0)) but for the sign of a zero.
template <bool BF>
__device__ __forceinline__ uint32_t pack16x2_relu(float a, float b) {
  uint32_t r;
  if constexpr (BF) asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  else asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}

// st_row8 of max(v, 0).
template <bool BF>
__device__ __forceinline__ void st_row8_relu(uint8_t *base, int r, int c, int K, const float *v) {
  uint4 u;
  u.x = pack16x2_relu<BF>(v[0], v[1]);
  u.y = pack16x2_relu<BF>(v[2], v[3]);
  u.z = pack16x2_relu<BF>(v[4], v[5]);
  u.w = pack16x2_relu<BF>(v[6], v[7]);
  *reinterpret_cast<uint4 *>(base + tile_off(r, c * 8, K)) = u;
}

// Shared-memory descriptor of a K-major [rows][K] no-swizzle operand: the next
// 8 K values are 128 B on, the next 8 rows K * 16 B on.
__device__ __forceinline__ uint64_t desc_k(uint32_t saddr, int K) {
  return tc::smem_desc(saddr, 128, (uint32_t)K * 16);
}

template <int F>
struct Raw;  // raw 16-bit storage of one entry (single) and of two adjacent entries (pair)
template <>
struct Raw<1> {
  using S = uint16_t;
  using P = uint32_t;
};
template <>
struct Raw<2> {
  using S = uint32_t;
  using P = uint2;
};
template <>
struct Raw<4> {
  using S = uint2;
  using P = uint4;
};

template <int F, bool BF, typename T>
__device__ __forceinline__ void unpack16(const T &u, float *e) {
  using T2 = typename Half<BF>::T2;
  const uint16_t *h = reinterpret_cast<const uint16_t *>(&u);
  constexpr int n = (int)(sizeof(T) / 2);
  if constexpr (n == 1) {
    typename Half<BF>::T v = *reinterpret_cast<const typename Half<BF>::T *>(h);
    e[0] = Half<BF>::lo(v);
  } else {
#pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      float2 f = Half<BF>::unpack(*reinterpret_cast<const T2 *>(h + 2 * i));
      e[2 * i] = f.x;
      e[2 * i + 1] = f.y;
    }
  }
}

// Weights of the x-corners of corner row q (dy = q & 1, dz = q >> 1) and the
// row's contribution, every operation rounded on its own: all gathers below
// blend in this order, so they give the same features bit for bit whatever
// loads they use.
__device__ __forceinline__ void row_weights(int q, float wx, float wy, float wz, float &w0, float &w1) {
  const float wyz = __fmul_rn((q & 1) ? wy : __fsub_rn(1.f, wy), (q >> 1) ? wz : __fsub_rn(1.f, wz));
  w0 = __fmul_rn(__fsub_rn(1.f, wx), wyz);
  w1 = __fmul_rn(wx, wyz);
}
__device__ __forceinline__ float blend2(float acc, float w0, float v0, float w1, float v1) {
  return __fmaf_rn(w1, v1, __fmaf_rn(w0, v0, acc));
}

// A-1..A-3 for G consecutive levels, x-paired: corners (cx, .) and (cx + 1, .)
// hash to entries h and h ^ 1 when cx is even (the x prime is 1), so one
// aligned 2-entry load serves both; for odd cx the second corner is loaded
// alone.  Every load of the G levels is issued before any is consumed, so a
// thread waits for one memory round trip per G levels.
template <int F, bool BF, int G>
__device__ __forceinline__ void gather_levels(const uint16_t *__restrict__ shadow, const NetDesc &nd, int l0,
                                              float x, float y, float z, float *out) {
  using PT = typename Raw<F>::P;
  using ST = typename Raw<F>::S;
  const uint32_t mask = nd.T - 1;
  PT pr[G][4];
  ST sg[G][4];
  uint32_t odd0 = 0, evenm = 0;
  float wxs[G], wys[G], wzs[G];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int l = l0 + g;
    int cx, cy, cz;
    const float N = (float)nd.res[l];
    nv_cell(x, N, cx, wxs[g]);
    nv_cell(y, N, cy, wys[g]);
    nv_cell(z, N, cz, wzs[g]);
    const bool even = (cx & 1) == 0;
    if (even) evenm |= 1u << g;
    const uint16_t *tab = shadow + (size_t)l * nd.T * F;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int dy = q & 1, dz = q >> 1;
      const uint32_t hy = ((uint32_t)(cy + dy) * 2654435761u) ^ ((uint32_t)(cz + dz) * 805459861u);
      const uint32_t h0 = ((uint32_t)cx ^ hy) & mask;
      if (h0 & 1u) odd0 |= 1u << (g * 4 + q);
      pr[g][q] = __ldg(reinterpret_cast<const PT *>(tab + (size_t)(h0 & ~1u) * F));
      if (!even) {
        const uint32_t h1 = ((uint32_t)(cx + 1) ^ hy) & mask;
        sg[g][q] = __ldg(reinterpret_cast<const ST *>(tab + (size_t)h1 * F));
      }
    }
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {
    float acc[F];
#pragma unroll
    for (int j = 0; j < F; ++j) acc[j] = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float pv[2 * F], e1[F];
      unpack16<F, BF>(pr[g][q], pv);
      const int o0 = ((odd0 >> (g * 4 + q)) & 1u) ? F : 0;
      if ((evenm >> g) & 1u) {
#pragma unroll
        for (int j = 0; j < F; ++j) e1[j] = pv[F - o0 + j];
      } else {
        unpack16<F, BF>(sg[g][q], e1);
      }
      float w0, w1;
      row_weights(q, wxs[g], wys[g], wzs[g], w0, w1);
#pragma unroll
      for (int j = 0; j < F; ++j) acc[j] = blend2(acc[j], w0, pv[o0 + j], w1, e1[j]);
    }
#pragma unroll
    for (int j = 0; j < F; ++j) out[g * F + j] = acc[j];
  }
}

// Fire-and-forget FP32 reductions (no value returned, so the issuing thread
// never waits for L2): 1, 2 or 4 floats at a 4-, 8- or 16-byte aligned address.
__device__ __forceinline__ void red_f32(float *p, float a) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(a) : "memory");
}
__device__ __forceinline__ void red_v2(float *p, float a, float b) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}
__device__ __forceinline__ void red_v4(float *p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

// Entry k (0..3) of a 16-byte group of four 4-byte entries.
__device__ __forceinline__ uint32_t pick4(const uint4 &g, uint32_t k) {
  const uint32_t lo = (k & 1u) ? g.y : g.x, hi = (k & 1u) ? g.w : g.z;
  return (k & 2u) ? hi : lo;
}

// A-1..A-3 for G consecutive levels of an F = 2 table with 16-bit features
// (4-byte entries).  The x-corners of a cell hash to h0 = cx ^ hy and h1 =
// (cx + 1) ^ hy (the x prime is 1), so h0 ^ h1 = cx ^ (cx + 1): 1 for even cx,
// 3 for cx = 1 mod 4, 7 or more otherwise.  One aligned 16-byte load of the
// four entries around h0 therefore serves both corners in three cells of four,
// and only cx = 3 mod 4 needs a second load: 5 loads per point and level on
// average instead of 6 with pairs.  Every load of the G levels is issued before
// any is consumed.
template <bool BF, int G>
__device__ __forceinline__ void gather_levels_f2(const uint16_t *__restrict__ shadow, const NetDesc &nd, int l0,
                                                 float x, float y, float z, float *out) {
  const uint32_t mask = nd.T - 1;
  uint4 grp[G][4];
  uint32_t sg[G][4];
  uint32_t sel[G];  // per corner row q: bits 8q..8q+7 = h0 & 3 | (h1 & 3) << 2 | (same group) << 4
  float wxs[G], wys[G], wzs[G];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int l = l0 + g;
    int cx, cy, cz;
    const float N = (float)nd.res[l];
    nv_cell(x, N, cx, wxs[g]);
    nv_cell(y, N, cy, wys[g]);
    nv_cell(z, N, cz, wzs[g]);
    const uint16_t *tab = shadow + (size_t)l * nd.T * 2;
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int dy = q & 1, dz = q >> 1;
      const uint32_t hy = ((uint32_t)(cy + dy) * 2654435761u) ^ ((uint32_t)(cz + dz) * 805459861u);
      const uint32_t h0 = ((uint32_t)cx ^ hy) & mask;
      const uint32_t h1 = ((uint32_t)(cx + 1) ^ hy) & mask;
      const bool same = (h0 >> 2) == (h1 >> 2);
      s |= ((h0 & 3u) | ((h1 & 3u) << 2) | ((same ? 1u : 0u) << 4)) << (8 * q);
      grp[g][q] = __ldg(reinterpret_cast<const uint4 *>(tab + (size_t)(h0 & ~3u) * 2));
      if (!same) sg[g][q] = __ldg(reinterpret_cast<const uint32_t *>(tab + (size_t)h1 * 2));
    }
    sel[g] = s;
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t s = sel[g] >> (8 * q);
      const uint32_t e0 = pick4(grp[g][q], s & 3u);
      const uint32_t e1 = (s & 16u) ? pick4(grp[g][q], (s >> 2) & 3u) : sg[g][q];
      const float2 v0 = Half<BF>::unpack(*reinterpret_cast<const typename Half<BF>::T2 *>(&e0));
      const float2 v1 = Half<BF>::unpack(*reinterpret_cast<const typename Half<BF>::T2 *>(&e1));
      float w0, w1;
      row_weights(q, wxs[g], wys[g], wzs[g], w0, w1);
      a0 = blend2(a0, w0, v0.x, w1, v1.x);
      a1 = blend2(a1, w0, v0.y, w1, v1.y);
    }
    out[2 * g] = a0;
    out[2 * g + 1] = a1;
  }
}

// A-1..A-3 for G consecutive levels with each of the 8 corners loaded on its
// own (8 one-entry loads per level, no selection among loaded entries).  For
// the sample batches of a ray march -- the K samples of a ray in adjacent work
// items, neighbouring rays in neighbouring items -- most corner loads hit in
// L1 and the x-paired gathers above are bound by the integer work of picking
// entries out of their 16-byte groups, not by memory; this one issues about
// 40% fewer instructions per level.  The hash of corner (cx + dx, cy + dy,
// cz + dz) is formed from the per-axis products (cy + 1) P1 = cy P1 + P1
// (mod 2^32).
template <int F, bool BF, int G>
__device__ __forceinline__ void gather_corners(const uint16_t *__restrict__ shadow, const NetDesc &nd, int l0,
                                               float x, float y, float z, float *out) {
  using ST = typename Raw<F>::S;
  const uint32_t mask = nd.T - 1;
  ST e[G][8];
  float wxs[G], wys[G], wzs[G];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int l = l0 + g;
    int cx, cy, cz;
    const float N = (float)nd.res[l];
    nv_cell(x, N, cx, wxs[g]);
    nv_cell(y, N, cy, wys[g]);
    nv_cell(z, N, cz, wzs[g]);
    const ST *tab = reinterpret_cast<const ST *>(shadow + (size_t)l * nd.T * F);
    const uint32_t y0 = (uint32_t)cy * 2654435761u, y1 = y0 + 2654435761u;
    const uint32_t z0 = (uint32_t)cz * 805459861u, z1 = z0 + 805459861u;
    const uint32_t x0 = (uint32_t)cx, x1 = x0 + 1u;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t hy = ((q & 1) ? y1 : y0) ^ ((q >> 1) ? z1 : z0);
      e[g][2 * q] = __ldg(tab + ((x0 ^ hy) & mask));
      e[g][2 * q + 1] = __ldg(tab + ((x1 ^ hy) & mask));
    }
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {
    float acc[F];
#pragma unroll
    for (int j = 0; j < F; ++j) acc[j] = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float v0[F], v1[F], w0, w1;
      unpack16<F, BF>(e[g][2 * q], v0);
      unpack16<F, BF>(e[g][2 * q + 1], v1);
      row_weights(q, wxs[g], wys[g], wzs[g], w0, w1);
#pragma unroll
      for (int j = 0; j < F; ++j) acc[j] = blend2(acc[j], w0, v0[j], w1, v1[j]);
    }
#pragma unroll
    for (int j = 0; j < F; ++j) out[g * F + j] = acc[j];
  }
}

template <int F>
__device__ __forceinline__ void red_entry(float *p, const float *g) {
  if constexpr (F == 1) {
    red_f32(p, g[0]);
  } else if constexpr (F == 2) {
    red_v2(p, g[0], g[1]);
  } else if constexpr (F == 4) {
    red_v4(p, g[0], g[1], g[2], g[3]);
  } else {
    red_v4(p, g[0], g[1], g[2], g[3]);
    red_v4(p + 4, g[4], g[5], g[6], g[7]);
  }
}

// A-7 at one level into a dense vertex grid (x fastest, n1 even): the two
// x-corners of an even cell are adjacent and 16-byte aligned at F = 2, one
// vector reduction; otherwise one per corner.  Only for points of [0,1]^3
// (corners 0..N+1 < n1).
template <int F>
__device__ __forceinline__ void scatter_dense(float *rep, int n1, float N, float x, float y, float z,
                                              const float *df) {
  int cx, cy, cz;
  float wx, wy, wz;
  nv_cell(x, N, cx, wx);
  nv_cell(y, N, cy, wy);
  nv_cell(z, N, cz, wz);
  const bool even = (cx & 1) == 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int dy = q & 1, dz = q >> 1;
    const float wyz = (dy ? wy : 1.f - wy) * (dz ? wz : 1.f - wz);
    const float w0 = (1.f - wx) * wyz, w1 = wx * wyz;
    float g0[F], g1[F];
#pragma unroll
    for (int j = 0; j < F; ++j) {
      g0[j] = w0 * df[j];
      g1[j] = w1 * df[j];
    }
    float *dst = rep + (((int64_t)(cz + dz) * n1 + (cy + dy)) * n1 + cx) * F;
    if (F == 2 && even) {
      red_v4(dst, g0[0], g0[1], g1[0], g1[1]);
    } else {
      red_entry<F>(dst, g0);
      red_entry<F>(dst + F, g1);
    }
  }
}

// A-7 for one level, x-paired like the gather: for even cx and F = 2 both
// x-corners land in one 16-byte aligned pair of FP32 entries and take one
// vector atomic.
template <int F>
__device__ __forceinline__ void scatter_level(float *gt, uint32_t mask, float N, float x, float y, float z,
                                              const float *df) {
  int cx, cy, cz;
  float wx, wy, wz;
  nv_cell(x, N, cx, wx);
  nv_cell(y, N, cy, wy);
  nv_cell(z, N, cz, wz);
  const bool even = (cx & 1) == 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int dy = q & 1, dz = q >> 1;
    const float wyz = (dy ? wy : 1.f - wy) * (dz ? wz : 1.f - wz);
    const uint32_t hy = ((uint32_t)(cy + dy) * 2654435761u) ^ ((uint32_t)(cz + dz) * 805459861u);
    const uint32_t h0 = ((uint32_t)cx ^ hy) & mask;
    const float w0 = (1.f - wx) * wyz, w1 = wx * wyz;
    float g0[F], g1[F];
#pragma unroll
    for (int j = 0; j < F; ++j) {
      g0[j] = w0 * df[j];
      g1[j] = w1 * df[j];
    }
    if (F == 2 && even) {
      const bool odd0 = (h0 & 1u) != 0;
      float *dst = gt + (size_t)(h0 & ~1u) * 2;
      if (odd0) red_v4(dst, g1[0], g1[1], g0[0], g0[1]);
      else red_v4(dst, g0[0], g0[1], g1[0], g1[1]);
    } else {
      const uint32_t h1 = ((uint32_t)(cx + 1) ^ hy) & mask;
      red_entry<F>(gt + (size_t)h0 * F, g0);
      red_entry<F>(gt + (size_t)h1 * F, g1);
    }
  }
}


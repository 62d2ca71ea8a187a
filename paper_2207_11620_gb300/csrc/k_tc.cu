// k_tc.cu -- fused hash encoding + MLP on the tcgen05 tensor cores (FP16 or
// BF16 operands, FP32 accumulation in tensor memory), for networks with
// L*F = D0 in {16, 32, 64} inputs and two hidden layers of 64 (Sec. 3.1's
// fully fused MLP, re-designed for sm_103a).
//
// One CTA = 128 threads = one warpgroup; a tile is 128 points, point r of the
// tile is TMEM lane r and thread r.  Per tile (training):
//   encode         each thread gathers its point's 8L corners from the FP16/BF16
//                  table shadow, interpolates in FP32, writes its feature row
//                  into shared memory (K-major core matrices)
//   layer 0, 1     one thread issues D1 = A0 W0^T and D2 = A1 W1^T
//                  (M=128, N=64); the rows come back with tcgen05.ld, ReLU in
//                  registers, h1 goes back to shared memory as the next A
//   output         z3 = W2 . h2 and the sigmoid in FP32 registers
//   backward       dZ2 rows to shared memory; dH1 = dZ2 W1 (M=128) and
//                  dW1 += dZ2^T H1 (M=64, the same shared buffers read
//                  MN-major); dZ1 rows; dF = dZ1 W0 and dW0 += dZ1^T F;
//                  dW2 by a warp reduce-scatter
//   scatter        every corner gets w * dF with vector atomics into the FP32
//                  table gradient
// The weight gradients accumulate in tensor memory across all tiles of the
// persistent CTA and reach global memory once, at the end.
//
// Shared-memory operands use no swizzle: a core matrix is 8 rows x 16 B.  A
// [rows][K] operand stores element (r, k) at
//   (r / 8) * SBO + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,
// with SBO = K / 8 * 128.  Read K-major: LBO = 128 (next 8 K), SBO (next 8
// rows).  Read MN-major (the transposed operand of a weight-gradient product,
// rows are then the K dimension): LBO = SBO of the K-major view (next 8 K),
// SBO = 128 (next 8 M/N).
#include "nv_internal.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int kH = 64;            // hidden width
constexpr int kTP = 128;          // points per tile
constexpr uint32_t kWaitLimit = 1u << 24;

// Descriptor field order of an MN-major no-swizzle operand: the leading byte
// offset holds the K-direction core-matrix stride and the stride byte offset
// the M/N-direction one, the same roles as for a K-major operand (checked on
// sm_103a with small in-bounds products against a host reference).
constexpr bool kMnLboIsMn = false;
// Tensor-memory rows of an M=64 product: true when row 16q + i sits in lane
// 32q + i (16 rows per warp quarter).
constexpr bool kM64Quarters = true;

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

// Gather one table entry of F 16-bit features and return them as FP32.
template <int F, bool BF>
__device__ __forceinline__ void load_entry16(const uint16_t *__restrict__ p, float *e) {
  using T2 = typename Half<BF>::T2;
  if constexpr (F == 1) {
    uint16_t u = __ldg(p);
    typename Half<BF>::T h = *reinterpret_cast<typename Half<BF>::T *>(&u);
    e[0] = Half<BF>::lo(h);
  } else if constexpr (F == 2) {
    uint32_t u = __ldg(reinterpret_cast<const uint32_t *>(p));
    float2 f = Half<BF>::unpack(*reinterpret_cast<T2 *>(&u));
    e[0] = f.x; e[1] = f.y;
  } else if constexpr (F == 4) {
    uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
    float2 a = Half<BF>::unpack(*reinterpret_cast<T2 *>(&u.x)), b = Half<BF>::unpack(*reinterpret_cast<T2 *>(&u.y));
    e[0] = a.x; e[1] = a.y; e[2] = b.x; e[3] = b.y;
  } else {
    uint4 u = __ldg(reinterpret_cast<const uint4 *>(p));
    float2 a = Half<BF>::unpack(*reinterpret_cast<T2 *>(&u.x)), b = Half<BF>::unpack(*reinterpret_cast<T2 *>(&u.y));
    float2 c = Half<BF>::unpack(*reinterpret_cast<T2 *>(&u.z)), d = Half<BF>::unpack(*reinterpret_cast<T2 *>(&u.w));
    e[0] = a.x; e[1] = a.y; e[2] = b.x; e[3] = b.y; e[4] = c.x; e[5] = c.y; e[6] = d.x; e[7] = d.y;
  }
}

template <int F>
__device__ __forceinline__ void red_entry(float *p, const float *g) {
  if constexpr (F == 1) {
    atomicAdd(p, g[0]);
  } else if constexpr (F == 2) {
    atomicAdd(reinterpret_cast<float2 *>(p), make_float2(g[0], g[1]));
  } else if constexpr (F == 4) {
    atomicAdd(reinterpret_cast<float4 *>(p), make_float4(g[0], g[1], g[2], g[3]));
  } else {
    atomicAdd(reinterpret_cast<float4 *>(p), make_float4(g[0], g[1], g[2], g[3]));
    atomicAdd(reinterpret_cast<float4 *>(p) + 1, make_float4(g[4], g[5], g[6], g[7]));
  }
}

// Shared-memory plan (bytes from a 1024-aligned base).
template <int D0, int MODE>
struct Plan {
  static constexpr bool kBwd = (MODE == MODE_TRAIN || MODE == MODE_BACKWARD);
  static constexpr int W0 = 0;                       // B [64][D0]
  static constexpr int W1 = W0 + kH * D0 * 2;        // B [64][64]
  static constexpr int A0 = W1 + kH * kH * 2;        // A [128][D0]  features
  static constexpr int A1 = A0 + kTP * D0 * 2;       // A [128][64]  h1
  static constexpr int W1T = A1 + kTP * kH * 2;      // B [64][64]   W1^T
  static constexpr int W0T = W1T + (kBwd ? kH * kH * 2 : 0);   // B [D0][64] W0^T
  static constexpr int DZ2 = W0T + (kBwd ? D0 * kH * 2 : 0);   // A [128][64]
  static constexpr int DZ1 = DZ2 + (kBwd ? kTP * kH * 2 : 0);  // A [128][64]
  static constexpr int W2 = DZ1 + (kBwd ? kTP * kH * 2 : 0);   // float [64]
  static constexpr int BAR = W2 + kH * 4;                      // mbarrier (8 B) + tmem slot
  static constexpr int TOTAL = BAR + 64;
  static constexpr uint32_t kTmemCols = kBwd ? 256 : 128;
  static constexpr int kColD1 = 0, kColD2 = 64, kColG1 = 128, kColG0 = 192;
};

// Highest byte (from the buffer start) an MMA sequence can read: K-major over a
// [rows][Kphys] buffer, K = 16 per MMA advancing 256 B; or MN-major over a
// [128 pts][Kphys] buffer with M/N = mn, 16 points per MMA advancing
// 2 * Kphys * 16 B.  Every product below is checked against its buffer size.
constexpr int span_k(int rows, int Kphys, int ksteps) {
  return (ksteps - 1) * 256 + (rows / 8 - 1) * Kphys * 16 + 128 + 127;
}
constexpr int span_mn(int mn, int Kphys) { return 7 * 2 * Kphys * 16 + (mn / 8 - 1) * 128 + Kphys * 16 + 127; }
template <int D0>
struct SpanCheck {
  static_assert(span_k(kTP, D0, D0 / 16) < kTP * D0 * 2, "layer 0 A");
  static_assert(span_k(kH, D0, D0 / 16) < kH * D0 * 2, "layer 0 B");
  static_assert(span_k(kTP, kH, kH / 16) < kTP * kH * 2, "layer 1 A / dZ A");
  static_assert(span_k(kH, kH, kH / 16) < kH * kH * 2, "layer 1 B / W1^T");
  static_assert(span_k(D0, kH, kH / 16) < D0 * kH * 2, "W0^T");
  static_assert(span_mn(kH, kH) < kTP * kH * 2, "dZ^T and H1^T");
  static_assert(span_mn(D0, D0) < kTP * D0 * 2, "F^T");
  static constexpr bool ok = true;
};
static_assert(SpanCheck<16>::ok && SpanCheck<32>::ok && SpanCheck<64>::ok, "operand spans");

// element (r, k) of a [rows][K] operand, byte offset
__device__ __forceinline__ uint32_t op_off(int r, int k, int K) {
  return (uint32_t)((r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Store 8 consecutive K values (one 16-byte core-matrix row) of row r.
template <bool BF>
__device__ __forceinline__ void st_row8(uint8_t *base, int r, int c, int K, const float *v) {
  uint4 u;
  u.x = pack2<BF>(v[0], v[1]);
  u.y = pack2<BF>(v[2], v[3]);
  u.z = pack2<BF>(v[4], v[5]);
  u.w = pack2<BF>(v[6], v[7]);
  *reinterpret_cast<uint4 *>(base + op_off(r, c * 8, K)) = u;
}

__device__ __forceinline__ uint64_t desc_k(uint32_t saddr, int K) {  // K-major [rows][K]
  return tc::smem_desc(saddr, 128, (uint32_t)K * 16);
}
__device__ __forceinline__ uint64_t desc_mn(uint32_t saddr, int Kphys) {  // MN-major view of [pts][Kphys]
  const uint32_t mn = 128, kk = (uint32_t)Kphys * 16;
  return kMnLboIsMn ? tc::smem_desc(saddr, mn, kk) : tc::smem_desc(saddr, kk, mn);
}

// Reduce 64 per-lane values across the warp; lane l ends with the sums of
// indices 2l and 2l+1 (reduce-scatter by halving: 62 shuffles).
__device__ __forceinline__ void warp_reduce_scatter64(float *v, float &o0, float &o1) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 16, n = 64; s >= 1; s >>= 1, n >>= 1) {
    const bool up = (lane & s) != 0;
    const int h = n >> 1;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      float give = up ? v[i] : v[i + h];
      float keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, give, s);
    }
  }
  o0 = v[0];
  o1 = v[1];
}

template <int F, int D0, bool BF, int MODE>
__global__ void __launch_bounds__(kTP) k_mlp_tc(NetDesc nd, const float *__restrict__ params,
                                                const uint16_t *__restrict__ shadow, MlpArgs a,
                                                const int *__restrict__ n_dev, int n_mult, double *acc) {
  using P = Plan<D0, MODE>;
  constexpr bool kBwd = P::kBwd;
  constexpr int L = D0 / F;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + P::BAR);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + P::BAR + 8);
  float *sW2 = reinterpret_cast<float *>(sm + P::W2);
  const uint32_t sbase = tc::smem_u32(sm);

  // ---- stage the weights (FP16/BF16 shadow) as B operands ----
  const uint16_t *w0g = shadow + nd.n_table + nd.w_off[0];
  const uint16_t *w1g = shadow + nd.n_table + nd.w_off[1];
  for (int i = tid; i < kH * D0 / 8; i += kTP) {  // W0 [64][D0] rows, 16 B at a time
    const int n = i / (D0 / 8), c = i % (D0 / 8);
    *reinterpret_cast<uint4 *>(sm + P::W0 + op_off(n, c * 8, D0)) =
        __ldg(reinterpret_cast<const uint4 *>(w0g + n * D0 + c * 8));
  }
  for (int i = tid; i < kH * kH / 8; i += kTP) {
    const int n = i / (kH / 8), c = i % (kH / 8);
    *reinterpret_cast<uint4 *>(sm + P::W1 + op_off(n, c * 8, kH)) =
        __ldg(reinterpret_cast<const uint4 *>(w1g + n * kH + c * 8));
  }
  if constexpr (kBwd) {
    for (int i = tid; i < kH * kH; i += kTP) {  // W1^T: B[n][k] = W1[k][n]
      const int n = i / kH, k = i % kH;
      *reinterpret_cast<uint16_t *>(sm + P::W1T + op_off(n, k, kH)) = w1g[k * kH + n];
    }
    for (int i = tid; i < D0 * kH; i += kTP) {  // W0^T: B[n][k] = W0[k][n], n < D0, k < 64
      const int n = i / kH, k = i % kH;
      *reinterpret_cast<uint16_t *>(sm + P::W0T + op_off(n, k, kH)) = w0g[k * D0 + n];
    }
  }
  for (int i = tid; i < kH; i += kTP) sW2[i] = params[nd.n_table + nd.w_off[2] + i];
  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    tc::mbar_fence_init();
  }
  tc::fence_async_smem();
  __syncthreads();
  if (warp == 0) {
    tc::tmem_alloc(tslot, P::kTmemCols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint32_t tD1 = tmem + P::kColD1, tD2 = tmem + P::kColD2;

  const int64_t n = n_dev ? (int64_t)(*n_dev) * n_mult : a.n;
  const int64_t ntiles = (n + kTP - 1) / kTP;
  float scale = 1.f, inv_scale = 1.f;
  if constexpr (kBwd) {
    scale = a.ds->loss_scale;
    inv_scale = (MODE == MODE_TRAIN ? a.inv_n : 1.f) / scale;
  }
  const uint32_t id_fwd = tc::idesc_f16(128, kH, BF, false, false);
  const uint32_t id_df = tc::idesc_f16(128, D0, BF, false, false);
  const uint32_t id_g1 = tc::idesc_f16(64, kH, BF, true, true);
  const uint32_t id_g0 = tc::idesc_f16(64, D0, BF, true, true);
  uint32_t phase = 0;
  bool failed = false;
  double local_acc = 0.0;
  float gw2a = 0.f, gw2b = 0.f;
  bool first = true;
  bool bad = false;

  auto wait_mma = [&]() -> bool {
    bool ok = tc::mbar_wait(mbar, phase, kWaitLimit);
    phase ^= 1u;
    tc::fence_after_sync();
    return __syncthreads_or(!ok) != 0;
  };

  for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const int64_t p = tile * kTP + tid;
    const bool valid = p < n;
    float x = 0.f, y = 0.f, z = 0.f, tgt = 0.f;
    if (valid) {
      if (MODE == 3) {
        const int64_t nx = a.vol.nx, ny = a.vol.ny;
        int ix = (int)(p % nx), iy = (int)((p / nx) % ny), iz = (int)(p / (nx * ny));
        x = __fdiv_rn(__fadd_rn((float)ix, 0.5f), (float)a.vol.nx);
        y = __fdiv_rn(__fadd_rn((float)iy, 0.5f), (float)a.vol.ny);
        z = __fdiv_rn(__fadd_rn((float)iz, 0.5f), (float)a.vol.nz);
        tgt = a.vol.data_dev[p];
      } else if (a.xyz) {
        x = a.xyz[3 * p];
        y = a.xyz[3 * p + 1];
        z = a.xyz[3 * p + 2];
        if (MODE == MODE_TRAIN) tgt = a.in[p];
      } else {
        float3 s = nv_sample_point(a.seed, a.sample_step, (uint64_t)p);
        x = s.x; y = s.y; z = s.z;
        tgt = nv_trilinear(a.vol.data_dev, a.vol.nx, a.vol.ny, a.vol.nz, x, y, z);
      }
    }
    // ---- encode: 8 features (one core-matrix row) at a time ----
#pragma unroll
    for (int c = 0; c < D0 / 8; ++c) {
      float f8[8];
#pragma unroll
      for (int q = 0; q < 8 / F; ++q) {
        const int l = c * (8 / F) + q;
        int cx, cy, cz;
        float wx, wy, wz;
        const float N = (float)nd.res[l];
        nv_cell(x, N, cx, wx);
        nv_cell(y, N, cy, wy);
        nv_cell(z, N, cz, wz);
        const uint16_t *tab = shadow + (size_t)l * nd.T * F;
        float acc_f[F];
#pragma unroll
        for (int j = 0; j < F; ++j) acc_f[j] = 0.f;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
          const int dx = d & 1, dy = (d >> 1) & 1, dz = (d >> 2) & 1;
          const float w = (dx ? wx : 1.f - wx) * (dy ? wy : 1.f - wy) * (dz ? wz : 1.f - wz);
          const uint32_t h = nv_hash3((uint32_t)(cx + dx), (uint32_t)(cy + dy), (uint32_t)(cz + dz)) & (nd.T - 1);
          float e[F];
          load_entry16<F, BF>(tab + (size_t)h * F, e);
#pragma unroll
          for (int j = 0; j < F; ++j) acc_f[j] += w * e[j];
        }
#pragma unroll
        for (int j = 0; j < F; ++j) f8[q * F + j] = acc_f[j];
      }
      st_row8<BF>(sm + P::A0, tid, c, D0, f8);
    }
    tc::fence_async_smem();
    __syncthreads();
    // ---- layer 0: D1 = A0 W0^T ----
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int k = 0; k < D0 / 16; ++k)
        tc::mma_f16(tD1, desc_k(sbase + P::A0 + k * 256, D0), desc_k(sbase + P::W0 + k * 256, D0), id_fwd, k > 0);
      tc::mma_commit(mbar);
    }
    if (wait_mma()) { failed = true; break; }
    uint64_t m1 = 0;  // ReLU mask of z1
#pragma unroll
    for (int c = 0; c < kH / 16; ++c) {
      float v[16];
      tc::tmem_ld16(tD1 + lane_base + c * 16, v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        if (v[i] > 0.f) m1 |= 1ull << (c * 16 + i);
        v[i] = fmaxf(v[i], 0.f);
      }
      st_row8<BF>(sm + P::A1, tid, 2 * c, kH, v);
      st_row8<BF>(sm + P::A1, tid, 2 * c + 1, kH, v + 8);
    }
    tc::fence_before_sync();
    tc::fence_async_smem();
    __syncthreads();
    // ---- layer 1: D2 = A1 W1^T ----
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int k = 0; k < kH / 16; ++k)
        tc::mma_f16(tD2, desc_k(sbase + P::A1 + k * 256, kH), desc_k(sbase + P::W1 + k * 256, kH), id_fwd, k > 0);
      tc::mma_commit(mbar);
    }
    if (wait_mma()) { failed = true; break; }
    float h2[kH];
#pragma unroll
    for (int c = 0; c < kH / 16; ++c) {
      tc::tmem_ld16(tD2 + lane_base + c * 16, h2 + c * 16);
    }
    tc::tmem_ld_wait();
    float z3 = 0.f;
#pragma unroll
    for (int i = 0; i < kH; ++i) {
      h2[i] = fmaxf(h2[i], 0.f);
      z3 += sW2[i] * h2[i];
    }
    const float yv = 1.f / (1.f + expf(-z3));
    if constexpr (MODE == MODE_INFER) {
      if (valid) a.y[p] = yv;
      tc::fence_before_sync();
      continue;
    }
    if constexpr (MODE == 3) {
      if (valid) {
        double dd = (double)yv - (double)tgt;
        local_acc += dd * dd;
      }
      tc::fence_before_sync();
      continue;
    }
    if constexpr (kBwd) {
      // ---- output delta (scaled by the loss scale S) ----
      float g = 0.f;
      if (valid) {
        if (MODE == MODE_TRAIN) {
          const float diff = yv - tgt;
          local_acc += (double)diff * (double)diff;
          g = 2.f * diff * scale;
        } else {
          g = a.in[p] * scale;
        }
      }
      const float dz3 = g * yv * (1.f - yv);
      // dW2 (FP32): reduce dz3 * h2 over the warp's 32 points
      {
        float v[kH];
#pragma unroll
        for (int i = 0; i < kH; ++i) v[i] = dz3 * h2[i];
        float s0, s1;
        warp_reduce_scatter64(v, s0, s1);
        gw2a += s0;
        gw2b += s1;
      }
      // dZ2 = dz3 W2 * 1[z2 > 0] -> shared memory
#pragma unroll
      for (int c = 0; c < kH / 8; ++c) {
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int k = c * 8 + i;
          v[i] = h2[k] > 0.f ? dz3 * sW2[k] : 0.f;
        }
        st_row8<BF>(sm + P::DZ2, tid, c, kH, v);
      }
      tc::fence_before_sync();
      tc::fence_async_smem();
      __syncthreads();
      // ---- dH1 = dZ2 W1 (-> D1) and dW1 += dZ2^T H1 (-> G1, M = 64) ----
      if (tid == 0) {
        tc::fence_after_sync();
#pragma unroll
        for (int k = 0; k < kH / 16; ++k)
          tc::mma_f16(tD1, desc_k(sbase + P::DZ2 + k * 256, kH), desc_k(sbase + P::W1T + k * 256, kH), id_fwd,
                      k > 0);
#pragma unroll
        for (int k = 0; k < kTP / 16; ++k)
          tc::mma_f16(tmem + P::kColG1, desc_mn(sbase + P::DZ2 + k * 2 * kH * 16, kH),
                      desc_mn(sbase + P::A1 + k * 2 * kH * 16, kH), id_g1, (!first || k > 0) ? 1u : 0u);
        tc::mma_commit(mbar);
      }
      if (wait_mma()) { failed = true; break; }
      // dZ1 = dH1 * 1[z1 > 0] -> shared memory
#pragma unroll
      for (int c = 0; c < kH / 16; ++c) {
        float v[16];
        tc::tmem_ld16(tD1 + lane_base + c * 16, v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (!((m1 >> (c * 16 + i)) & 1ull)) v[i] = 0.f;
        st_row8<BF>(sm + P::DZ1, tid, 2 * c, kH, v);
        st_row8<BF>(sm + P::DZ1, tid, 2 * c + 1, kH, v + 8);
      }
      tc::fence_before_sync();
      tc::fence_async_smem();
      __syncthreads();
      // ---- dF = dZ1 W0 (-> D2, N = D0) and dW0 += dZ1^T F (-> G0, M = 64) ----
      if (tid == 0) {
        tc::fence_after_sync();
#pragma unroll
        for (int k = 0; k < kH / 16; ++k)
          tc::mma_f16(tD2, desc_k(sbase + P::DZ1 + k * 256, kH), desc_k(sbase + P::W0T + k * 256, kH), id_df,
                      k > 0);
#pragma unroll
        for (int k = 0; k < kTP / 16; ++k)
          tc::mma_f16(tmem + P::kColG0, desc_mn(sbase + P::DZ1 + k * 2 * kH * 16, kH),
                      desc_mn(sbase + P::A0 + k * 2 * D0 * 16, D0), id_g0, (!first || k > 0) ? 1u : 0u);
        tc::mma_commit(mbar);
      }
      if (wait_mma()) { failed = true; break; }
      first = false;
      // ---- dF back to FP32 (unscaled) and scattered into the table gradient ----
      float df[D0];
#pragma unroll
      for (int c = 0; c < D0 / 16; ++c) tc::tmem_ld16(tD2 + lane_base + c * 16, df + c * 16);
      tc::tmem_ld_wait();
      tc::fence_before_sync();
      if (valid) {
#pragma unroll
        for (int i = 0; i < D0; ++i) {
          df[i] *= inv_scale;
          if (!isfinite(df[i])) bad = true;
        }
        if (!bad) {
#pragma unroll
          for (int l = 0; l < L; ++l) {
            int cx, cy, cz;
            float wx, wy, wz;
            const float N = (float)nd.res[l];
            nv_cell(x, N, cx, wx);
            nv_cell(y, N, cy, wy);
            nv_cell(z, N, cz, wz);
            float *gt = a.grads + (size_t)l * nd.T * F;
#pragma unroll
            for (int d = 0; d < 8; ++d) {
              const int dx = d & 1, dy = (d >> 1) & 1, dz = (d >> 2) & 1;
              const float w = (dx ? wx : 1.f - wx) * (dy ? wy : 1.f - wy) * (dz ? wz : 1.f - wz);
              const uint32_t h =
                  nv_hash3((uint32_t)(cx + dx), (uint32_t)(cy + dy), (uint32_t)(cz + dz)) & (nd.T - 1);
              float gg[F];
#pragma unroll
              for (int j = 0; j < F; ++j) gg[j] = w * df[l * F + j];
              red_entry<F>(gt + (size_t)h * F, gg);
            }
          }
        }
      }
    }
  }

  if (failed && tid == 0) atomicExch(&a.ds->err, 1);
  if constexpr (MODE == MODE_TRAIN || MODE == 3) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local_acc += __shfl_xor_sync(0xffffffffu, local_acc, o);
    if (lane == 0 && local_acc != 0.0) atomicAdd(acc, local_acc);
  }
  if constexpr (kBwd) {
    if (!failed && !first) {
      // weight gradients: dW2 from the lanes' registers, dW1 / dW0 from tensor memory
      float *gw = a.grads + nd.n_table;
      float w2a = gw2a * inv_scale, w2b = gw2b * inv_scale;
      if (!isfinite(w2a) || !isfinite(w2b)) bad = true;
      else {
        atomicAdd(gw + nd.w_off[2] + 2 * lane, w2a);
        atomicAdd(gw + nd.w_off[2] + 2 * lane + 1, w2b);
      }
      // M = 64 rows: which rows this warp's lanes hold
      int row = -1;
      if (kM64Quarters) {
        if (lane < 16) row = warp * 16 + lane;
      } else {
        if (warp < 2) row = warp * 32 + lane;
      }
#pragma unroll
      for (int c = 0; c < kH / 16; ++c) {
        float v[16];
        tc::tmem_ld16(tmem + P::kColG1 + lane_base + c * 16, v);
        tc::tmem_ld_wait();
        if (row >= 0) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            float g = v[i] * inv_scale;
            if (!isfinite(g)) bad = true;
            else if (g != 0.f) atomicAdd(gw + nd.w_off[1] + row * kH + c * 16 + i, g);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < D0 / 16; ++c) {
        float v[16];
        tc::tmem_ld16(tmem + P::kColG0 + lane_base + c * 16, v);
        tc::tmem_ld_wait();
        if (row >= 0) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            float g = v[i] * inv_scale;
            if (!isfinite(g)) bad = true;
            else if (g != 0.f) atomicAdd(gw + nd.w_off[0] + row * D0 + c * 16 + i, g);
          }
        }
      }
    }
    if (bad) atomicExch(&a.ds->overflow, 1);
  }
  if (failed) {
    // give an MMA that may still be in flight one more bounded chance to finish
    tc::mbar_wait(mbar, phase ^ 1u, kWaitLimit);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, P::kTmemCols);
}

template <int F, int D0, bool BF, int MODE>
nv_status launch_t(const nv_ctx *c, const MlpArgs &a, const int *n_dev, int n_mult, int64_t n_upper, double *acc) {
  using P = Plan<D0, MODE>;
  // tensor memory holds 512 columns per SM: size the shared-memory request so
  // that no more CTAs fit on an SM than their columns allow
  const int tmem_cap = 512 / (int)P::kTmemCols;
  size_t bytes = P::TOTAL + 1024;
  const size_t min_bytes = 233472 / (tmem_cap + 1) + 1024;
  if (bytes < min_bytes) bytes = min_bytes;
  auto kern = k_mlp_tc<F, D0, BF, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return nv_cuda_check(e, "cudaFuncSetAttribute(k_mlp_tc)");
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTP, bytes);
  if (per_sm > tmem_cap) per_sm = tmem_cap;
  if (per_sm < 1) per_sm = 1;
  const int64_t ntiles = (n_upper + kTP - 1) / kTP;
  int64_t grid = (int64_t)c->num_sms * per_sm;
  if (ntiles < grid) grid = ntiles;
  if (grid < 1) return NV_OK;
  kern<<<(unsigned)grid, kTP, bytes, c->stream>>>(c->nd, c->params, reinterpret_cast<const uint16_t *>(c->shadow),
                                                   a, n_dev, n_mult, acc);
  return nv_cuda_check(cudaGetLastError(), "k_mlp_tc launch");
}

template <int F, int D0, bool BF>
nv_status dispatch_mode(const nv_ctx *c, int mode, const MlpArgs &a, const int *n_dev, int n_mult, int64_t n_upper,
                        double *acc) {
  switch (mode) {
    case MODE_INFER: return launch_t<F, D0, BF, MODE_INFER>(c, a, n_dev, n_mult, n_upper, acc);
    case MODE_BACKWARD: return launch_t<F, D0, BF, MODE_BACKWARD>(c, a, n_dev, n_mult, n_upper, acc);
    case MODE_TRAIN: return launch_t<F, D0, BF, MODE_TRAIN>(c, a, n_dev, n_mult, n_upper, acc);
    case 3: return launch_t<F, D0, BF, 3>(c, a, n_dev, n_mult, n_upper, acc);
  }
  return nv_fail(NV_ERR_ARG, "bad MLP mode %d", mode);
}

template <bool BF>
nv_status dispatch_shape(const nv_ctx *c, int mode, const MlpArgs &a, const int *n_dev, int n_mult, int64_t n_upper,
                         double *acc) {
  const int F = c->nd.F, D0 = c->nd.dims[0];
  if (F == 2 && D0 == 16) return dispatch_mode<2, 16, BF>(c, mode, a, n_dev, n_mult, n_upper, acc);
  if (F == 2 && D0 == 32) return dispatch_mode<2, 32, BF>(c, mode, a, n_dev, n_mult, n_upper, acc);
  if (F == 4 && D0 == 64) return dispatch_mode<4, 64, BF>(c, mode, a, n_dev, n_mult, n_upper, acc);
  if (F == 4 && D0 == 32) return dispatch_mode<4, 32, BF>(c, mode, a, n_dev, n_mult, n_upper, acc);
  if (F == 2 && D0 == 64) return dispatch_mode<2, 64, BF>(c, mode, a, n_dev, n_mult, n_upper, acc);
  return nv_fail(NV_ERR_UNSUPPORTED, "tensor-core MLP: no kernel for F=%d, L*F=%d", F, D0);
}

}  // namespace

bool tc_supported(const NetDesc &nd) {
  if (nd.n_dims != 4 || nd.dims[1] != kH || nd.dims[2] != kH || nd.dims[3] != 1) return false;
  const int F = nd.F, D0 = nd.dims[0];
  return (F == 2 && (D0 == 16 || D0 == 32 || D0 == 64)) || (F == 4 && (D0 == 32 || D0 == 64));
}

nv_status launch_mlp_tc_ext(const nv_ctx *c, int mode, const MlpArgs &a, const int *n_dev, int n_mult,
                            int64_t n_upper, double *acc) {
  if (!tc_supported(c->nd)) return nv_fail(NV_ERR_UNSUPPORTED, "tensor-core MLP: unsupported network shape");
  return c->prec == NV_BF16 ? dispatch_shape<true>(c, mode, a, n_dev, n_mult, n_upper, acc)
                            : dispatch_shape<false>(c, mode, a, n_dev, n_mult, n_upper, acc);
}

nv_status launch_mlp_tc(const nv_ctx *c, int mode, const MlpArgs &a) {
  return launch_mlp_tc_ext(c, mode, a, nullptr, 1, a.n, mode == MODE_TRAIN ? &a.ds->loss_acc : nullptr);
}

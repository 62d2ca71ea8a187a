// k_tc.cu -- the MLP of the hash-encoded network on the tcgen05 tensor cores
// (FP16 or BF16 operands, FP32 accumulation in tensor memory), for L*F = D0 in
// {16, 32, 64} inputs and two hidden layers of 64 (Sec. 3.1's fully fused MLP,
// re-designed for sm_103a), and the launch sequence of the tensor-core path:
//
//   k_encode_tiles   gather + trilinear blend -> features in tile layout, and
//                    the targets of a sampled training batch (k_grid.cu)
//   k_mlp_tc         per 128-point tile: features arrive by one bulk async copy
//                    (double-buffered, the next tile's copy overlaps this one),
//                    layer 0 / 1 products, ReLU and the FP32 output layer; in
//                    training the backward products, the weight gradients
//                    accumulated in tensor memory over all tiles of the CTA,
//                    and the per-point input gradient dF, which each thread
//                    scatters straight into the FP32 table gradient (A-7)
//
// The two run on chunks of points.  Passes that scatter gradients take at
// most kChunk = 2^19 points (16 MB of features at D0 = 32, L2-resident
// between the kernels).  Inference takes up to kChunkInfer = 2^23 (512 MB):
// a render iteration's samples then go through in one or two launches, and
// the ramp and tail every launch of either kernel pays cost more, at
// 2^19-point chunks, than the features' round trip through HBM.  The
// scatter's vector reductions keep the load/store path busy while the CTA's
// other phases wait on the tensor core, so the MLP and the scatter overlap
// inside one kernel.
//
// One CTA = 256 threads; a tile is 128 points.  Point r of the tile is TMEM
// lane r and is shared by threads r and r + 128: each handles half of the 64
// hidden columns (and of the D0 input-gradient columns) in every epilogue.
//
// Shared-memory operands use no swizzle: a core matrix is 8 rows x 16 B.  A
// [rows][K] operand stores element (r, k) at
//   (r / 8) * SBO + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,
// with SBO = K / 8 * 128.  Read K-major: LBO = 128 (next 8 K), SBO (next 8
// rows).  Read MN-major (the transposed operand of a weight-gradient product,
// rows are then the K dimension): LBO = SBO of the K-major view (next 8 K),
// SBO = 128 (next 8 M/N).
#include "nv_internal.cuh"
#include "tc_grid.cuh"
#include "tc_ptx.cuh"

nv_status launch_encode_tiles(const nv_ctx *c, const PointSrc &ps, const ChunkSpan &cs, uint8_t *feat,
                              float *tgt, float *xyz_out, int *off_flag, bool coherent, cudaStream_t st);

namespace {

constexpr int kH = 64;            // hidden width
constexpr int kTP = 128;          // points per tile
constexpr int kThreads = 256;     // two threads per point
constexpr int64_t kChunk = 1 << 19;
constexpr int64_t kChunkInfer = 1 << 23;
constexpr uint32_t kWaitLimit = 1u << 24;

// Descriptor field order of an MN-major no-swizzle operand: the leading byte
// offset holds the K-direction core-matrix stride and the stride byte offset
// the M/N-direction one, the same roles as for a K-major operand (checked on
// sm_103a with small in-bounds products against a host reference).
constexpr bool kMnLboIsMn = false;
// Tensor-memory rows of an M=64 product: row 16q + i sits in lane 32q + i
// (16 rows per warp quarter; checked the same way).
constexpr bool kM64Quarters = true;

// Shared-memory plan (bytes from a 1024-aligned base).
template <int D0, int MODE>
struct Plan {
  static constexpr bool kBwd = (MODE == MODE_TRAIN || MODE == MODE_BACKWARD);
  static constexpr int kTile = kTP * D0 * 2;                   // one feature tile
  static constexpr int W0 = 0;                                 // B [64][D0]
  static constexpr int W1 = W0 + kH * D0 * 2;                  // B [64][64]
  static constexpr int A0 = W1 + kH * kH * 2;                  // A [128][D0] features, two buffers
  static constexpr int A1 = A0 + 2 * kTile;                    // A [128][64]  h1
  static constexpr int W1T = A1 + kTP * kH * 2;                // B [64][64]   W1^T
  static constexpr int W0T = W1T + (kBwd ? kH * kH * 2 : 0);   // B [D0][64] W0^T
  static constexpr int DZ2 = W0T + (kBwd ? D0 * kH * 2 : 0);   // A [128][64]
  static constexpr int DZ1 = DZ2 + (kBwd ? kTP * kH * 2 : 0);  // A [128][64]
  static constexpr int W2 = DZ1 + (kBwd ? kTP * kH * 2 : 0);   // float [64]
  static constexpr int Z3 = W2 + kH * 4;                       // float [2][128] partial output sums
  static constexpr int TG = Z3 + 2 * kTP * 4;                  // float [128] targets of the tile
  static constexpr int BAR = TG + kTP * 4;                     // 3 mbarriers + tmem slot
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

// Add n scaled values to 16-byte aligned dst with n / 4 vector reductions,
// skipping all-zero groups; returns whether any value is not finite (that
// group is then left out).
template <int n>
__device__ __forceinline__ bool red_row(float *dst, const float *v, float s) {
  bool bad = false;
#pragma unroll
  for (int j = 0; j < n; j += 4) {
    const float4 g = make_float4(v[j] * s, v[j + 1] * s, v[j + 2] * s, v[j + 3] * s);
    if (!isfinite(g.x) || !isfinite(g.y) || !isfinite(g.z) || !isfinite(g.w)) {
      bad = true;
      continue;
    }
    if (g.x != 0.f || g.y != 0.f || g.z != 0.f || g.w != 0.f) red_v4(dst + j, g.x, g.y, g.z, g.w);
  }
  return bad;
}

__device__ __forceinline__ uint64_t desc_mn(uint32_t saddr, int Kphys) {  // MN-major view of [pts][Kphys]
  const uint32_t mn = 128, kk = (uint32_t)Kphys * 16;
  return kMnLboIsMn ? tc::smem_desc(saddr, mn, kk) : tc::smem_desc(saddr, kk, mn);
}

constexpr int kHotR = 8;  // dense replicas of the coarsest levels' gradient

// Fold the dense replicas into the hashed table gradient, after the kernel
// that scattered into them: one thread per vertex of the replicated levels
// sums the R copies (in copy order), clears them and adds the sum to the
// vertex's hash slot.
__global__ void __launch_bounds__(256) k_fold_replicas(const __grid_constant__ NetDesc nd, const __grid_constant__ HotRep h,
                                                       float *grads) {
  const int F = nd.F;
  const int64_t vtot = h.vbase[h.levels];
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < vtot; v += (int64_t)gridDim.x * blockDim.x) {
    int l = 0;
    while (l + 1 < h.levels && v >= h.vbase[l + 1]) ++l;
    const int n1 = h.n1[l];
    const int64_t loc = v - h.vbase[l];
    const int x = (int)(loc % n1), y = (int)((loc / n1) % n1), z = (int)(loc / ((int64_t)n1 * n1));
    const int lim = nd.res[l] + 1;  // corners of cells of [0,1]^3 reach N_l + 1
    if (x > lim || y > lim || z > lim) continue;
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    bool any = false;
    if (F == 2) {
      float2 t[kHotR];
#pragma unroll
      for (int r = 0; r < kHotR; ++r) t[r] = __ldcg(reinterpret_cast<const float2 *>(h.buf + ((int64_t)r * vtot + v) * 2));
#pragma unroll
      for (int r = 0; r < kHotR; ++r) {
        if (t[r].x != 0.f || t[r].y != 0.f) {
          s[0] += t[r].x;
          s[1] += t[r].y;
          any = true;
          *reinterpret_cast<float2 *>(h.buf + ((int64_t)r * vtot + v) * 2) = make_float2(0.f, 0.f);
        }
      }
    } else {
      float4 t[kHotR];
#pragma unroll
      for (int r = 0; r < kHotR; ++r) t[r] = __ldcg(reinterpret_cast<const float4 *>(h.buf + ((int64_t)r * vtot + v) * 4));
#pragma unroll
      for (int r = 0; r < kHotR; ++r) {
        if (t[r].x != 0.f || t[r].y != 0.f || t[r].z != 0.f || t[r].w != 0.f) {
          s[0] += t[r].x;
          s[1] += t[r].y;
          s[2] += t[r].z;
          s[3] += t[r].w;
          any = true;
          *reinterpret_cast<float4 *>(h.buf + ((int64_t)r * vtot + v) * 4) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    }
    if (!any) continue;
    const uint32_t hs = nv_hash3((uint32_t)x, (uint32_t)y, (uint32_t)z) & (nd.T - 1);
    float *g = grads + ((size_t)l * nd.T + hs) * F;
    if (F == 2) red_v2(g, s[0], s[1]);
    else red_v4(g, s[0], s[1], s[2], s[3]);
  }
}

// MODE_INFER: y = sigmoid(MLP(f)).  MODE 3: accumulate (y - vol)^2 into acc.
// MODE_TRAIN: loss += (y - t)^2, dF = d(loss / n)/df.  MODE_BACKWARD: dF = dL/dy * dy/df.
// TRAIN / BACKWARD add the weight gradients and the table gradient w_corner * dF
// into a.grads.  tgt_buf: the targets of a sampled training batch, [chunk rows].
template <int D0, bool BF, int MODE>
__global__ void __launch_bounds__(kThreads, (MODE == MODE_INFER || MODE == 3) ? 4 : 2) k_mlp_tc(NetDesc nd, const float *__restrict__ params,
                                                        const uint16_t *__restrict__ shadow, MlpArgs a,
                                                        PointSrc ps, ChunkSpan cs,
                                                        const uint8_t *__restrict__ feat,
                                                        const float *__restrict__ tgt_buf, double *acc) {
  using P = Plan<D0, MODE>;
  constexpr bool kBwd = P::kBwd;
  constexpr int HH = kH / 2;  // hidden columns per thread
  constexpr int DH = D0 / 2;  // input-gradient columns per thread
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r = tid & (kTP - 1);  // point row == TMEM lane
  const int hh = tid >> 7;        // half: hidden columns [hh*HH, ..)
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + P::BAR);       // MMA completion
  uint64_t *lbar = reinterpret_cast<uint64_t *>(sm + P::BAR + 8);   // [2] feature tile arrival
  uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + P::BAR + 24);
  float *sW2 = reinterpret_cast<float *>(sm + P::W2);
  float *sZ3 = reinterpret_cast<float *>(sm + P::Z3);
  float *sTG = reinterpret_cast<float *>(sm + P::TG);
  const uint32_t sbase = tc::smem_u32(sm);
  const int64_t n = chunk_count(cs);
  const int64_t ntiles = (n + kTP - 1) / kTP;
  // a CTA with no tile -- all of them for a chunk with no points, which the
  // renderer launches for an upper bound of the live samples -- has nothing to
  // do: leave before staging weights or tensor memory
  if ((int64_t)blockIdx.x >= ntiles) return;

  // ---- stage the weights (FP16/BF16 shadow) as B operands ----
  const uint16_t *w0g = shadow + nd.n_table + nd.w_off[0];
  const uint16_t *w1g = shadow + nd.n_table + nd.w_off[1];
  for (int i = tid; i < kH * D0 / 8; i += kThreads) {  // W0 [64][D0] rows, 16 B at a time
    const int nn = i / (D0 / 8), c = i % (D0 / 8);
    *reinterpret_cast<uint4 *>(sm + P::W0 + tile_off(nn, c * 8, D0)) =
        __ldg(reinterpret_cast<const uint4 *>(w0g + nn * D0 + c * 8));
  }
  for (int i = tid; i < kH * kH / 8; i += kThreads) {
    const int nn = i / (kH / 8), c = i % (kH / 8);
    *reinterpret_cast<uint4 *>(sm + P::W1 + tile_off(nn, c * 8, kH)) =
        __ldg(reinterpret_cast<const uint4 *>(w1g + nn * kH + c * 8));
  }
  if constexpr (kBwd) {
    // the transposes read consecutive elements of a weight row per warp (coalesced)
    for (int i = tid; i < kH * kH; i += kThreads) {  // W1^T: B[n][k] = W1[k][n]
      const int nn = i % kH, k = i / kH;
      *reinterpret_cast<uint16_t *>(sm + P::W1T + tile_off(nn, k, kH)) = w1g[k * kH + nn];
    }
    for (int i = tid; i < D0 * kH; i += kThreads) {  // W0^T: B[n][k] = W0[k][n], n < D0, k < 64
      const int nn = i % D0, k = i / D0;
      *reinterpret_cast<uint16_t *>(sm + P::W0T + tile_off(nn, k, kH)) = w0g[k * D0 + nn];
    }
  }
  for (int i = tid; i < kH; i += kThreads) sW2[i] = params[nd.n_table + nd.w_off[2] + i];
  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    tc::mbar_init(lbar, 1);
    tc::mbar_init(lbar + 1, 1);
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
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const uint32_t tD1 = tmem + P::kColD1, tD2 = tmem + P::kColD2;

  // feature copies issued (by thread 0) into each buffer, and which are not yet
  // waited for (scalars rather than arrays indexed by the buffer, which would
  // live in local memory on the MMA-issuing thread's path)
  uint32_t uses0 = 0, uses1 = 0;
  bool pend0 = false, pend1 = false;
  auto issue_tile = [&](int b, int64_t t) {
    tc::mbar_expect_tx(lbar + b, P::kTile);
    tc::bulk_g2s(sm + P::A0 + b * P::kTile, feat + t * P::kTile, P::kTile, lbar + b);
    if (b) {
      ++uses1;
      pend1 = true;
    } else {
      ++uses0;
      pend0 = true;
    }
  };
  // first feature tile of this CTA
  if (tid == 0 && (int64_t)blockIdx.x < ntiles) issue_tile(0, blockIdx.x);

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
  float gw2 = 0.f;
  bool first = true;
  bool bad = false;

  auto wait_mma = [&]() -> bool {
    bool ok = tc::mbar_wait(mbar, phase, kWaitLimit);
    phase ^= 1u;
    tc::fence_after_sync();
    return __syncthreads_or(!ok) != 0;
  };

  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x, ++it) {
    const int buf = it & 1;
    const uint32_t a0 = P::A0 + buf * P::kTile;
    const int64_t q = tile * kTP + r;   // row within the chunk
    const int64_t p = cs.off + q;       // point index of the launch
    const bool valid = q < n;
    // per-point target of the output delta (read while the features arrive)
    float tgt = 0.f;
    if (valid && hh == 0) {
      if (MODE == 3) {
        tgt = a.vol.data_dev[p];
      } else if (MODE == MODE_TRAIN) {
        tgt = a.in ? a.in[p] : tgt_buf[q];
      } else if (MODE == MODE_BACKWARD) {
        tgt = a.in[p];
      }
    }
    // the point itself, for the table scatter at the end of the tile: loaded now,
    // so its round trip hides under the tile's products instead of delaying the
    // scatter
    float3 xs = make_float3(0.f, 0.f, 0.f);
    if (kBwd && valid) xs = point_at(ps, p);
    // ---- this tile's features; start the next tile's copy into the other buffer ----
    const bool ok_ld = tc::mbar_wait(lbar + buf, (uint32_t)(it >> 1) & 1u, kWaitLimit);
    if (__syncthreads_or(!ok_ld)) { failed = true; break; }
    if (tid == 0) {
      if (buf) pend1 = false;
      else pend0 = false;
      const int64_t nt = tile + gridDim.x;
      if (nt < ntiles) issue_tile(buf ^ 1, nt);
      // ---- layer 0: D1 = A0 W0^T ----
      tc::fence_after_sync();
#pragma unroll
      for (int k = 0; k < D0 / 16; ++k)
        tc::mma_f16(tD1, desc_k(sbase + a0 + k * 256, D0), desc_k(sbase + P::W0 + k * 256, D0), id_fwd, k > 0);
      tc::mma_commit(mbar);
    }
    if (wait_mma()) { failed = true; break; }
    uint32_t m1 = 0;  // ReLU mask of this thread's 32 columns of z1
    {
      // both halves of the thread's columns in flight before the one wait
      float v[HH];
#pragma unroll
      for (int c = 0; c < HH / 16; ++c) tc::tmem_ld16(tD1 + lane_base + hh * HH + c * 16, v + c * 16);
      tc::tmem_ld_wait();
      if constexpr (kBwd) {
#pragma unroll
        for (int i = 0; i < HH; ++i)
          if (v[i] > 0.f) m1 |= 1u << i;
      }
#pragma unroll
      for (int c = 0; c < HH / 8; ++c) st_row8_relu<BF>(sm + P::A1, r, hh * (HH / 8) + c, kH, v + c * 8);
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
    float h2[HH];
#pragma unroll
    for (int c = 0; c < HH / 16; ++c) tc::tmem_ld16(tD2 + lane_base + hh * HH + c * 16, h2 + c * 16);
    tc::tmem_ld_wait();
    tc::fence_before_sync();
    float zp = 0.f;
#pragma unroll
    for (int i = 0; i < HH; ++i) {
      h2[i] = fmaxf(h2[i], 0.f);
      zp += sW2[hh * HH + i] * h2[i];
    }
    sZ3[hh * kTP + r] = zp;
    if (hh == 0) sTG[r] = tgt;
    __syncthreads();
    const float z3 = sZ3[r] + sZ3[kTP + r];
    const float yv = 1.f / (1.f + expf(-z3));
    const float tv = sTG[r];
    if constexpr (MODE == MODE_INFER) {
      if (valid && hh == 0) a.y[p] = yv;
      continue;
    }
    if constexpr (MODE == 3) {
      if (valid && hh == 0) {
        const double dd = (double)yv - (double)tv;
        local_acc += dd * dd;
      }
      continue;
    }
    if constexpr (kBwd) {
      // ---- output delta (scaled by the loss scale S) ----
      float g = 0.f;
      if (valid) {
        if (MODE == MODE_TRAIN) {
          const float diff = yv - tv;
          if (a.l1) {
            if (hh == 0) local_acc += fabs((double)diff);
            g = (float)((diff > 0.f) - (diff < 0.f)) * scale;
          } else {
            if (hh == 0) local_acc += (double)diff * (double)diff;
            g = 2.f * diff * scale;
          }
        } else {
          g = tv * scale;
        }
      }
      const float dz3 = g * yv * (1.f - yv);
      // dW2 (FP32): reduce dz3 * h2 over the warp's 32 points, lane l keeps column hh*32 + l
      {
        float v[HH];
#pragma unroll
        for (int i = 0; i < HH; ++i) v[i] = dz3 * h2[i];
#pragma unroll
        for (int s2 = 16, m = HH; s2 >= 1; s2 >>= 1, m >>= 1) {
          const bool up = (lane & s2) != 0;
          const int h = m >> 1;
#pragma unroll
          for (int i = 0; i < h; ++i) {
            const float give = up ? v[i] : v[i + h];
            const float keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, give, s2);
          }
        }
        gw2 += v[0];
      }
      // dZ2 = dz3 W2 * 1[z2 > 0] -> shared memory
#pragma unroll
      for (int c = 0; c < HH / 8; ++c) {
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int k = c * 8 + i;
          v[i] = h2[k] > 0.f ? dz3 * sW2[hh * HH + k] : 0.f;
        }
        st_row8<BF>(sm + P::DZ2, r, hh * (HH / 8) + c, kH, v);
      }
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
      for (int c = 0; c < HH / 16; ++c) {
        float v[16];
        tc::tmem_ld16(tD1 + lane_base + hh * HH + c * 16, v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (!((m1 >> (c * 16 + i)) & 1u)) v[i] = 0.f;
        st_row8<BF>(sm + P::DZ1, r, hh * (HH / 8) + 2 * c, kH, v);
        st_row8<BF>(sm + P::DZ1, r, hh * (HH / 8) + 2 * c + 1, kH, v + 8);
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
                      desc_mn(sbase + a0 + k * 2 * D0 * 16, D0), id_g0, (!first || k > 0) ? 1u : 0u);
        tc::mma_commit(mbar);
      }
      if (wait_mma()) { failed = true; break; }
      first = false;
      // ---- this thread's half of dF, unscaled, scattered into the table gradient ----
      float df[DH];
#pragma unroll
      for (int c = 0; c < DH / 8; ++c) tc::tmem_ld8(tD2 + lane_base + hh * DH + c * 8, df + c * 8);
      tc::tmem_ld_wait();
      tc::fence_before_sync();
      if (valid) {
#pragma unroll
        for (int i = 0; i < DH; ++i) {
          df[i] *= inv_scale;
          if (!isfinite(df[i])) bad = true;
        }
        if (MODE == MODE_BACKWARD && a.df_out) {  // this thread's half of dL/df, level-major
          float4 *dst = reinterpret_cast<float4 *>(a.df_out + p * D0 + hh * DH);
#pragma unroll
          for (int i = 0; i < DH; i += 4) dst[i / 4] = make_float4(df[i], df[i + 1], df[i + 2], df[i + 3]);
        }
        const float3 x = xs;
        // the coarsest levels (all in half 0) go to this CTA's dense replica
        const bool dense = hh == 0 && a.hot.levels > 0 && x.x >= 0.f && x.x <= 1.f && x.y >= 0.f && x.y <= 1.f &&
                           x.z >= 0.f && x.z <= 1.f;
        const int64_t rep_off = dense ? (int64_t)(blockIdx.x % a.hot.R) * a.hot.vbase[a.hot.levels] : 0;
        if (nd.F == 2) {
#pragma unroll
          for (int k = 0; k < DH / 2; ++k) {
            const int l = hh * (DH / 2) + k;
            if (k < 4 && dense && k < a.hot.levels)
              scatter_dense<2>(a.hot.buf + (rep_off + a.hot.vbase[k < 4 ? k : 0]) * 2, a.hot.n1[k < 4 ? k : 0],
                               (float)nd.res[l], x.x, x.y, x.z, df + 2 * k);
            else
              scatter_level<2>(a.grads + (size_t)l * nd.T * 2, nd.T - 1, (float)nd.res[l], x.x, x.y, x.z,
                               df + 2 * k);
          }
        } else {
#pragma unroll
          for (int k = 0; k < DH / 4; ++k) {
            const int l = hh * (DH / 4) + k;
            if (k < 4 && dense && k < a.hot.levels)
              scatter_dense<4>(a.hot.buf + (rep_off + a.hot.vbase[k < 4 ? k : 0]) * 4, a.hot.n1[k < 4 ? k : 0],
                               (float)nd.res[l], x.x, x.y, x.z, df + 4 * k);
            else
              scatter_level<4>(a.grads + (size_t)l * nd.T * 4, nd.T - 1, (float)nd.res[l], x.x, x.y, x.z,
                               df + 4 * k);
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
      const float w2 = gw2 * inv_scale;
      if (!isfinite(w2)) bad = true;
      else atomicAdd(gw + nd.w_off[2] + hh * HH + lane, w2);
      if (hh == 0) {
        // M = 64 rows: which rows this warp's lanes hold
        int row = -1;
        if (kM64Quarters) {
          if (lane < 16) row = warp * 16 + lane;
        } else {
          if (warp < 2) row = warp * 32 + lane;
        }
        // 16-byte vector reductions: all CTAs add into the same few thousand
        // addresses, so fewer, wider reductions shorten the kernel's tail
        // (the weight offsets are multiples of 4 floats, checked on the host)
#pragma unroll
        for (int c = 0; c < kH / 16; ++c) {
          float v[16];
          tc::tmem_ld16(tmem + P::kColG1 + lane_base + c * 16, v);
          tc::tmem_ld_wait();
          if (row >= 0) bad |= red_row<16>(gw + nd.w_off[1] + row * kH + c * 16, v, inv_scale);
        }
#pragma unroll
        for (int c = 0; c < D0 / 8; ++c) {
          float v[8];
          tc::tmem_ld8(tmem + P::kColG0 + lane_base + c * 8, v);
          tc::tmem_ld_wait();
          if (row >= 0) bad |= red_row<8>(gw + nd.w_off[0] + row * D0 + c * 8, v, inv_scale);
        }
      }
    }
    if (bad) atomicExch(&a.ds->overflow, 1);
  }
  if (tid == 0) {
    // a feature copy still in flight (only after an early exit) must land
    // before the CTA's shared memory is released
    if (pend0) tc::mbar_wait(lbar, (uses0 - 1) & 1u, kWaitLimit);
    if (pend1) tc::mbar_wait(lbar + 1, (uses1 - 1) & 1u, kWaitLimit);
  }
  if (failed) {
    // give an MMA that may still be in flight one more bounded chance to finish
    tc::mbar_wait(mbar, phase ^ 1u, kWaitLimit);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, P::kTmemCols);
}

template <int D0, bool BF, int MODE>
nv_status launch_mlp(const nv_ctx *c, const MlpArgs &a, const PointSrc &ps, const ChunkSpan &cs,
                     const uint8_t *feat, const float *tgt, double *acc) {
  using P = Plan<D0, MODE>;
  // tensor memory holds 512 columns per SM: size the shared-memory request so
  // that no more CTAs fit on an SM than their columns allow
  const int tmem_cap = 512 / (int)P::kTmemCols;
  size_t bytes = P::TOTAL + 1024;
  const size_t min_bytes = 233472 / (tmem_cap + 1) + 1024;
  if (bytes < min_bytes) bytes = min_bytes;
  auto kern = k_mlp_tc<D0, BF, MODE>;
  // set up once per kernel instance (device attributes of the first device used)
  static int per_sm = 0;
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return nv_cuda_check(e, "cudaFuncSetAttribute(k_mlp_tc)");
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return nv_cuda_check(e, "cudaFuncSetAttribute(carveout)");
    // resident CTAs per SM: the tightest of registers, shared memory and tensor memory
    int dev = 0, regs_sm = 0, smem_sm = 0, smem_rsv = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return nv_cuda_check(e, "cudaFuncGetAttributes(k_mlp_tc)");
    const int by_regs = regs_sm / (((fa.numRegs + 7) & ~7) * kThreads);
    const int by_smem = smem_sm / (int)(bytes + smem_rsv);
    int n = by_regs < by_smem ? by_regs : by_smem;
    if (n > tmem_cap) n = tmem_cap;
    per_sm = n < 1 ? 1 : n;
  }
  const int64_t ntiles = (cs.cap + kTP - 1) / kTP;
  int64_t grid = (int64_t)c->num_sms * per_sm;
  if (ntiles < grid) grid = ntiles;
  if (grid < 1) return NV_OK;
  kern<<<(unsigned)grid, kThreads, bytes, c->stream>>>(c->nd, c->params,
                                                        reinterpret_cast<const uint16_t *>(c->shadow), a, ps, cs,
                                                        feat, tgt, acc);
  return nv_cuda_check(cudaGetLastError(), "k_mlp_tc launch");
}

template <int D0, bool BF>
nv_status dispatch_mode(const nv_ctx *c, int mode, const MlpArgs &a, const PointSrc &ps, const ChunkSpan &cs,
                        const uint8_t *feat, const float *tgt, double *acc) {
  switch (mode) {
    case MODE_INFER: return launch_mlp<D0, BF, MODE_INFER>(c, a, ps, cs, feat, tgt, acc);
    case MODE_BACKWARD: return launch_mlp<D0, BF, MODE_BACKWARD>(c, a, ps, cs, feat, tgt, acc);
    case MODE_TRAIN: return launch_mlp<D0, BF, MODE_TRAIN>(c, a, ps, cs, feat, tgt, acc);
    case 3: return launch_mlp<D0, BF, 3>(c, a, ps, cs, feat, tgt, acc);
  }
  return nv_fail(NV_ERR_ARG, "bad MLP mode %d", mode);
}

template <bool BF>
nv_status dispatch_shape(const nv_ctx *c, int mode, const MlpArgs &a, const PointSrc &ps, const ChunkSpan &cs,
                         const uint8_t *feat, const float *tgt, double *acc) {
  switch (c->nd.dims[0]) {
    case 16: return dispatch_mode<16, BF>(c, mode, a, ps, cs, feat, tgt, acc);
    case 32: return dispatch_mode<32, BF>(c, mode, a, ps, cs, feat, tgt, acc);
    case 64: return dispatch_mode<64, BF>(c, mode, a, ps, cs, feat, tgt, acc);
  }
  return nv_fail(NV_ERR_UNSUPPORTED, "tensor-core MLP: no kernel for L*F=%d", c->nd.dims[0]);
}

}  // namespace

bool tc_supported(const NetDesc &nd) {
  if (nd.n_dims != 4 || nd.dims[1] != kH || nd.dims[2] != kH || nd.dims[3] != 1) return false;
  const int F = nd.F, D0 = nd.dims[0];
  // the weight-gradient reductions are 16-byte vectors
  if (nd.n_table % 4 || nd.w_off[0] % 4 || nd.w_off[1] % 4) return false;
  return (F == 2 && (D0 == 16 || D0 == 32 || D0 == 64)) || (F == 4 && (D0 == 32 || D0 == 64));
}

// Scratch of the tensor-core path: one chunk of features (16-bit, tile layout)
// and of sampled training points and targets (FP32), allocated on first use;
// chunks of at most `chunk` points.
static nv_status tc_scratch(nv_ctx *c, int64_t points, int64_t chunk) {
  const int64_t cap = points < chunk ? ((points + kTP - 1) / kTP) * kTP : chunk;
  if (c->tc_cap >= cap) return NV_OK;
  cudaFree(c->tc_feat);
  cudaFree(c->tc_tgt);
  cudaFree(c->tc_xyz);
  c->tc_feat = nullptr;
  c->tc_tgt = nullptr;
  c->tc_xyz = nullptr;
  c->tc_cap = 0;
  const int D0 = c->nd.dims[0];
  cudaError_t e = cudaMalloc(&c->tc_feat, (size_t)cap * D0 * 2);
  if (e == cudaSuccess) e = cudaMalloc(&c->tc_tgt, (size_t)cap * 4);
  if (e == cudaSuccess) e = cudaMalloc(&c->tc_xyz, (size_t)cap * 12);
  if (e != cudaSuccess) return nv_cuda_check(e, "tensor-core scratch");
  c->tc_cap = cap;
  return NV_OK;
}

nv_status launch_mlp_tc_ext(const nv_ctx *cc, int mode, const MlpArgs &a, const int *n_dev, int n_mult,
                            int64_t n_upper, double *acc) {
  nv_ctx *c = const_cast<nv_ctx *>(cc);
  if (!tc_supported(c->nd)) return nv_fail(NV_ERR_UNSUPPORTED, "tensor-core MLP: unsupported network shape");
  if (n_upper <= 0) return NV_OK;
  const int64_t chunk_max = (mode == MODE_INFER || mode == 3) ? kChunkInfer : kChunk;
  nv_status s = tc_scratch(c, n_upper, chunk_max);
  if (s != NV_OK) return s;
  const int64_t chunk = c->tc_cap < chunk_max ? c->tc_cap : chunk_max;
  PointSrc ps{};
  if (mode == 3) {
    ps.kind = 1;
    ps.vol = a.vol;
  } else if (a.xyz) {
    ps.kind = 0;
    ps.xyz = a.xyz;
  } else {
    ps.kind = 2;
    ps.vol = a.vol;
    ps.seed = a.seed;
    ps.step = a.sample_step;
  }
  MlpArgs am = a;  // the MLP kernel's arguments: backward passes scatter the coarsest levels into replicas
  if (mode == MODE_TRAIN || mode == MODE_BACKWARD) am.hot = c->hot;
  // a sampled training batch: the gather kernel computes each Philox point
  // once for the MLP kernel too (its points and targets)
  const bool sampled = mode == MODE_TRAIN && ps.kind == 2;
  float *tgt = sampled ? c->tc_tgt : nullptr;
  float *xyz_out = sampled ? c->tc_xyz : nullptr;
  // given points of a pass that scatters table gradients: the gather kernel
  // flags any outside [0,1]^3 (sampled ones never are)
  int *off_flag = (mode == MODE_TRAIN || mode == MODE_BACKWARD) && ps.kind == 0 ? &c->ds->off_domain : nullptr;
  for (int64_t off = 0; off < n_upper; off += chunk) {
    ChunkSpan cs{n_dev, n_mult, a.n, off, n_upper - off < chunk ? n_upper - off : chunk};
    int tk = prof_begin(c);
    s = launch_encode_tiles(c, ps, cs, c->tc_feat, tgt, xyz_out, off_flag, a.coherent != 0 || mode == 3,
                            c->stream);
    prof_end(c, NV_K_ENCODE, tk);
    if (s != NV_OK) return s;
    tk = prof_begin(c);
    PointSrc pm = ps;
    if (sampled) {
      pm.kind = 0;
      pm.xyz = c->tc_xyz;
      pm.xyz_off = off;
    }
    s = c->prec == NV_BF16 ? dispatch_shape<true>(c, mode, am, pm, cs, c->tc_feat, tgt, acc)
                           : dispatch_shape<false>(c, mode, am, pm, cs, c->tc_feat, tgt, acc);
    prof_end(c, NV_K_MLP, tk);
    if (s != NV_OK) return s;
    if (am.hot.levels > 0) {
      tk = prof_begin(c);
      const int64_t vtot = am.hot.vbase[am.hot.levels];
      k_fold_replicas<<<(unsigned)((vtot + 255) / 256), 256, 0, c->stream>>>(c->nd, am.hot, am.grads);
      s = nv_cuda_check(cudaGetLastError(), "k_fold_replicas launch");
      prof_end(c, NV_K_SCATTER, tk);
      if (s != NV_OK) return s;
    }
  }
  return NV_OK;
}

nv_status launch_mlp_tc(const nv_ctx *c, int mode, const MlpArgs &a) {
  return launch_mlp_tc_ext(c, mode, a, nullptr, 1, a.n, mode == MODE_TRAIN ? &a.ds->loss_acc : nullptr);
}

// Dense replicas of the coarsest levels' table gradient: consecutive levels
// from 0 whose padded vertex grid holds at most 2^15 vertices (at most four,
// all in the first half of the levels), kHotR copies.
nv_status build_hot_replicas(nv_ctx *c) {
  HotRep h{};
  const NetDesc &nd = c->nd;
  int64_t v = 0;
  for (int l = 0; l < 4 && l < nd.L / 2; ++l) {
    const int n1 = (nd.res[l] + 3) & ~1;
    if ((int64_t)n1 * n1 * n1 > 32768) break;
    h.n1[l] = n1;
    h.vbase[l] = v;
    v += (int64_t)n1 * n1 * n1;
    h.levels = l + 1;
  }
  h.vbase[h.levels] = v;
  h.R = kHotR;
  c->hot = HotRep{};
  if (h.levels == 0 || c->prec == NV_FP32 || !tc_supported(nd)) return NV_OK;
  cudaError_t e = cudaMalloc(&h.buf, (size_t)h.R * v * nd.F * sizeof(float));
  if (e == cudaSuccess) e = cudaMemsetAsync(h.buf, 0, (size_t)h.R * v * nd.F * sizeof(float), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    cudaFree(h.buf);
    return nv_cuda_check(e, "replicas of the coarse levels' gradient");
  }
  c->hot = h;
  return NV_OK;
}

// k_simt64.cu -- the FP32 CUDA-core MLP (A-4..A-7 of the FP32 path) for the
// network shape the workloads use: D0 = L*F in {16, 32, 64} inputs, two
// hidden layers of 64, one output (Sec. 3.1), F in {2, 4}.  Other shapes take
// the generic kernel in k_simt.cu.
//
// A CTA of 256 threads takes 128-point tiles (persistent).  Every product of
// the forward and backward pass is a small FP32 matrix product over the tile,
// computed from shared memory with register blocking:
//   point-major products (Z1 = F W0^T, Z2 = H1 W1^T, dH1 = dZ2 W1, dF = dZ1 W0):
//     thread (pg, cg) = (tid / 16, tid % 16) owns points 8 pg .. 8 pg + 7 and
//     output columns cg + 16 j; per reduction index it loads 8 activations (two
//     broadcast float4) and 4 weights (consecutive over the lanes) for 32 FMAs
//   weight gradients (dW1 = dZ2^T H1, dW0 = dZ1^T F; the reduction runs over the
//     tile's points): thread (ng, cg) owns rows ng + 16 s and columns cg + 16 j,
//     4 points per step from float4 loads of both operands
// Activations live feature-major ([feature][132] floats: rows of 128 points plus
// 4 of padding, so the rows of consecutive features fall in different banks);
// W0 and W1 are stored [out][in + 1] so both their row and their column walks
// are conflict-free.  The weight gradients accumulate in registers over all tiles
// of the CTA and reach global memory once.  The table gradient is the x-paired
// vector-reduction scatter of the tensor-core path (tc_grid.cuh).  Every sum is
// an FP32 sum of the same terms as the oracle's, in another order.
#include "nv_internal.cuh"
#include "tc_grid.cuh"

namespace {

constexpr int kT = 256;   // threads per CTA
constexpr int kPts = 128; // points per tile
constexpr int kPp = 132;  // row stride (floats) of the feature-major activation buffers
constexpr int kHid = 64;

template <int D0>
struct Plan64 {
  static constexpr int W0 = 0;                          // [64][D0 + 1]
  static constexpr int W1 = W0 + kHid * (D0 + 1);       // [64][65]
  static constexpr int W2 = W1 + kHid * (kHid + 1);     // [64]
  static constexpr int FT = (W2 + kHid + 3) & ~3;       // [D0][kPp]: features, later dF
  static constexpr int H1T = FT + D0 * kPp;             // [64][kPp]: h1, later dZ1
  static constexpr int D2T = H1T + kHid * kPp;          // [64][kPp]: dZ2
  static constexpr int XYZ = D2T + kHid * kPp;          // [128][3] the tile's points
  static constexpr int DZ3 = XYZ + kPts * 3;            // [128] output deltas
  static constexpr int TOTAL = DZ3 + kPts;              // floats
};

// Point-major product: acc[i][j] += sum_k A[k][8 pg + i] * B[k][cg + 16 j] with A
// feature-major ([K][kPp]) and B read as B(k, col) through a functor.
template <int K, int J, typename BF>
__device__ __forceinline__ void pm_product(const float *A, BF B, int pg, int cg, float (&acc)[8][J]) {
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    const float4 a0 = *reinterpret_cast<const float4 *>(A + k * kPp + 8 * pg);
    const float4 a1 = *reinterpret_cast<const float4 *>(A + k * kPp + 8 * pg + 4);
    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const float b = B(k, cg + 16 * j);
#pragma unroll
      for (int i = 0; i < 8; ++i) acc[i][j] = fmaf(av[i], b, acc[i][j]);
    }
  }
}

// Weight-gradient product over the tile's points: acc[s][j] += sum_p X[ng + 16 s][p] * Y[cg + 16 j][p],
// X and Y feature-major.
template <int S, int J>
__device__ __forceinline__ void wg_product(const float *X, const float *Y, int ng, int cg, float (&acc)[S][J]) {
#pragma unroll 2
  for (int p = 0; p < kPts; p += 4) {
    float4 xv[S], yv[J];
#pragma unroll
    for (int s = 0; s < S; ++s) xv[s] = *reinterpret_cast<const float4 *>(X + (ng + 16 * s) * kPp + p);
#pragma unroll
    for (int j = 0; j < J; ++j) yv[j] = *reinterpret_cast<const float4 *>(Y + (cg + 16 * j) * kPp + p);
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int j = 0; j < J; ++j) {
        acc[s][j] = fmaf(xv[s].x, yv[j].x, acc[s][j]);
        acc[s][j] = fmaf(xv[s].y, yv[j].y, acc[s][j]);
        acc[s][j] = fmaf(xv[s].z, yv[j].z, acc[s][j]);
        acc[s][j] = fmaf(xv[s].w, yv[j].w, acc[s][j]);
      }
  }
}

// A-1..A-3 at one level from the FP32 master table: trilinear blend of the 8 corners.
template <int F>
__device__ __forceinline__ void encode_level64(const float *__restrict__ tab, uint32_t Tmask, float N, float x,
                                               float y, float z, float *out) {
  int cx, cy, cz;
  float wx, wy, wz;
  nv_cell(x, N, cx, wx);
  nv_cell(y, N, cy, wy);
  nv_cell(z, N, cz, wz);
#pragma unroll
  for (int j = 0; j < F; ++j) out[j] = 0.f;
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    const int dx = d & 1, dy = (d >> 1) & 1, dz = (d >> 2) & 1;
    const float w = (dx ? wx : 1.f - wx) * (dy ? wy : 1.f - wy) * (dz ? wz : 1.f - wz);
    const uint32_t h = nv_hash3((uint32_t)(cx + dx), (uint32_t)(cy + dy), (uint32_t)(cz + dz)) & Tmask;
    float e[4];
    if constexpr (F == 2) {
      const float2 v = __ldg(reinterpret_cast<const float2 *>(tab) + h);
      e[0] = v.x;
      e[1] = v.y;
    } else {
      const float4 v = __ldg(reinterpret_cast<const float4 *>(tab) + h);
      e[0] = v.x;
      e[1] = v.y;
      e[2] = v.z;
      e[3] = v.w;
    }
#pragma unroll
    for (int j = 0; j < F; ++j) out[j] += w * e[j];
  }
}

// MODE_INFER: y = net(x).  MODE_BACKWARD: grads += d(sum dL/dy * y)/dparams (and dL/df into a.df_out).
// MODE_TRAIN: loss += sum (y - t)^2 or |y - t|; grads += d(loss / n)/dparams.
// Mode 3 (volume MSE): x = voxel centre of point index p, accumulates (y - vol)^2.
template <int D0, int F, int MODE>
__global__ void __launch_bounds__(kT) k_mlp_f32x(NetDesc nd, const float *__restrict__ params, MlpArgs a,
                                                 const int *__restrict__ n_dev, int n_mult, double *acc) {
  using P = Plan64<D0>;
  constexpr bool kBwd = (MODE == MODE_BACKWARD || MODE == MODE_TRAIN);
  constexpr int JD = D0 / 16;  // dF / dW0 columns per thread
  constexpr int L = D0 / F;
  extern __shared__ float sm[];
  const int tid = threadIdx.x;
  const int pg = tid >> 4, cg = tid & 15;  // point group / column group of the point-major products
  const int r = tid & (kPts - 1), hh = tid >> 7;  // point and half of the levels in the encode / scatter

  // weights: W0 [64][D0 + 1], W1 [64][65], W2 [64]
  const float *wg = params + nd.n_table;
  for (int i = tid; i < kHid * D0; i += kT) sm[P::W0 + (i / D0) * (D0 + 1) + i % D0] = wg[nd.w_off[0] + i];
  for (int i = tid; i < kHid * kHid; i += kT) sm[P::W1 + (i / kHid) * (kHid + 1) + i % kHid] = wg[nd.w_off[1] + i];
  for (int i = tid; i < kHid; i += kT) sm[P::W2 + i] = wg[nd.w_off[2] + i];
  __syncthreads();
  const float *W0 = sm + P::W0;
  const float *W1 = sm + P::W1;
  const float *W2 = sm + P::W2;
  float *FT = sm + P::FT;
  float *H1T = sm + P::H1T;
  float *D2T = sm + P::D2T;
  float *sX = sm + P::XYZ;
  float *sDz3 = sm + P::DZ3;

  float gW1[4][4] = {}, gW0[4][JD > 0 ? JD : 1] = {}, gW2[4] = {};
  double local_acc = 0.0;
  const int64_t n = n_dev ? (int64_t)(*n_dev) * n_mult : a.n;
  const int64_t ntiles = (n + kPts - 1) / kPts;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // ---- the tile's points and features (thread r, half hh: half of the levels) ----
    const int64_t p = tile * kPts + r;
    const bool valid = p < n;
    float x = 0.f, y = 0.f, z = 0.f, tgt = 0.f;
    if (valid) {
      if (MODE == 3) {
        const int64_t nx = a.vol.nx, ny = a.vol.ny;
        const int ix = (int)(p % nx), iy = (int)((p / nx) % ny), iz = (int)(p / (nx * ny));
        x = __fdiv_rn(__fadd_rn((float)ix, 0.5f), (float)a.vol.nx);
        y = __fdiv_rn(__fadd_rn((float)iy, 0.5f), (float)a.vol.ny);
        z = __fdiv_rn(__fadd_rn((float)iz, 0.5f), (float)a.vol.nz);
        if (hh == 0) tgt = a.vol.data_dev[p];
      } else if (a.xyz) {
        x = a.xyz[3 * p];
        y = a.xyz[3 * p + 1];
        z = a.xyz[3 * p + 2];
        if (MODE == MODE_TRAIN && hh == 0) tgt = a.in[p];
        if (MODE == MODE_BACKWARD && hh == 0) tgt = a.in[p];  // dL/dy
      } else {
        const float3 s = nv_sample_point(a.seed, a.sample_step, (uint64_t)p);
        x = s.x;
        y = s.y;
        z = s.z;
        if (hh == 0) tgt = nv_trilinear(a.vol.data_dev, a.vol.nx, a.vol.ny, a.vol.nz, x, y, z);
      }
    }
#pragma unroll 1
    for (int l = hh * (L / 2); l < (hh + 1) * (L / 2); ++l) {
      float out[F];
      if (valid) {
        encode_level64<F>(params + (size_t)l * nd.T * F, nd.T - 1, (float)nd.res[l], x, y, z, out);
      } else {
#pragma unroll
        for (int j = 0; j < F; ++j) out[j] = 0.f;
      }
#pragma unroll
      for (int j = 0; j < F; ++j) FT[(l * F + j) * kPp + r] = out[j];
    }
    if (hh == 0) {
      sX[3 * r] = x;
      sX[3 * r + 1] = y;
      sX[3 * r + 2] = z;
      sDz3[r] = tgt;  // the target (or dL/dy) until the output delta replaces it
    }
    __syncthreads();

    // ---- layer 0: Z1 = F W0^T, h1 = ReLU -> H1T ----
    {
      float acc[8][4] = {};
      pm_product<D0, 4>(FT, [&](int k, int c) { return W0[c * (D0 + 1) + k]; }, pg, cg, acc);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float *dst = H1T + (cg + 16 * j) * kPp + 8 * pg;
        *reinterpret_cast<float4 *>(dst) = make_float4(fmaxf(acc[0][j], 0.f), fmaxf(acc[1][j], 0.f),
                                                       fmaxf(acc[2][j], 0.f), fmaxf(acc[3][j], 0.f));
        *reinterpret_cast<float4 *>(dst + 4) = make_float4(fmaxf(acc[4][j], 0.f), fmaxf(acc[5][j], 0.f),
                                                           fmaxf(acc[6][j], 0.f), fmaxf(acc[7][j], 0.f));
      }
    }
    __syncthreads();
    // ---- layer 1: Z2 = H1 W1^T (kept in registers), output layer, loss, output delta ----
    float z2[8][4] = {};
    pm_product<kHid, 4>(H1T, [&](int k, int c) { return W1[c * (kHid + 1) + k]; }, pg, cg, z2);
    float zo[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float s = 0.f;
#pragma unroll
      for (int j = 0; j < 4; ++j) s = fmaf(W2[cg + 16 * j], fmaxf(z2[i][j], 0.f), s);
      zo[i] = s;
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1)
#pragma unroll
      for (int i = 0; i < 8; ++i) zo[i] += __shfl_xor_sync(0xffffffffu, zo[i], o);
    float dz3[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int pt = 8 * pg + i;
      const int64_t pp = tile * kPts + pt;
      const bool v = pp < n;
      const float yv = 1.f / (1.f + expf(-zo[i]));
      const float tv = sDz3[pt];
      float g = 0.f;
      if (MODE == MODE_INFER) {
        if (v && cg == i) a.y[pp] = yv;
      } else if (MODE == 3) {
        if (v && cg == i) {
          const double dd = (double)yv - (double)tv;
          local_acc += dd * dd;
        }
      } else if (MODE == MODE_TRAIN) {
        if (v) {
          const float diff = yv - tv;
          if (a.l1) {
            if (cg == i) local_acc += fabs((double)diff);
            g = (float)((diff > 0.f) - (diff < 0.f)) * a.inv_n;
          } else {
            if (cg == i) local_acc += (double)diff * (double)diff;
            g = 2.f * diff * a.inv_n;
          }
        }
      } else {  // MODE_BACKWARD
        if (v) g = tv;
      }
      dz3[i] = g * yv * (1.f - yv);
    }
    if constexpr (kBwd) {
      // dW2 and dZ2 = dz3 W2 * 1[z2 > 0] -> D2T
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float w2 = W2[cg + 16 * j];
        float d[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          gW2[j] = fmaf(dz3[i], fmaxf(z2[i][j], 0.f), gW2[j]);
          d[i] = z2[i][j] > 0.f ? dz3[i] * w2 : 0.f;
        }
        float *dst = D2T + (cg + 16 * j) * kPp + 8 * pg;
        *reinterpret_cast<float4 *>(dst) = make_float4(d[0], d[1], d[2], d[3]);
        *reinterpret_cast<float4 *>(dst + 4) = make_float4(d[4], d[5], d[6], d[7]);
      }
      __syncthreads();
      // dW1 += dZ2^T H1 (rows ng + 16 s = pg + 16 s of dZ2's features, columns cg + 16 j of H1's)
      wg_product<4, 4>(D2T, H1T, pg, cg, gW1);
      // dH1 = dZ2 W1, dZ1 = dH1 * 1[h1 > 0]
      float dh[8][4] = {};
      pm_product<kHid, 4>(D2T, [&](int k, int c) { return W1[k * (kHid + 1) + c]; }, pg, cg, dh);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float *hrow = H1T + (cg + 16 * j) * kPp + 8 * pg;
        const float4 h0 = *reinterpret_cast<const float4 *>(hrow);
        const float4 h1 = *reinterpret_cast<const float4 *>(hrow + 4);
        const float hv[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (!(hv[i] > 0.f)) dh[i][j] = 0.f;
      }
      __syncthreads();  // every thread has read H1T (dW1, the masks): dZ1 may replace it
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float *dst = H1T + (cg + 16 * j) * kPp + 8 * pg;
        *reinterpret_cast<float4 *>(dst) = make_float4(dh[0][j], dh[1][j], dh[2][j], dh[3][j]);
        *reinterpret_cast<float4 *>(dst + 4) = make_float4(dh[4][j], dh[5][j], dh[6][j], dh[7][j]);
      }
      __syncthreads();
      // dW0 += dZ1^T F
      wg_product<4, JD>(H1T, FT, pg, cg, gW0);
      // dF = dZ1 W0
      float df[8][JD] = {};
      pm_product<kHid, JD>(H1T, [&](int k, int c) { return W0[k * (D0 + 1) + c]; }, pg, cg, df);
      __syncthreads();  // every thread has read FT (dW0): dF may replace it
#pragma unroll
      for (int j = 0; j < JD; ++j) {
        float *dst = FT + (cg + 16 * j) * kPp + 8 * pg;
        *reinterpret_cast<float4 *>(dst) = make_float4(df[0][j], df[1][j], df[2][j], df[3][j]);
        *reinterpret_cast<float4 *>(dst + 4) = make_float4(df[4][j], df[5][j], df[6][j], df[7][j]);
      }
      __syncthreads();
      // ---- table-gradient scatter: thread r, half hh of the levels ----
      const int64_t pp = tile * kPts + r;
      if (pp < n) {
        const float px = sX[3 * r], py = sX[3 * r + 1], pz = sX[3 * r + 2];
        if (hh == 0 && !(px >= 0.f && px <= 1.f && py >= 0.f && py <= 1.f && pz >= 0.f && pz <= 1.f))
          a.ds->off_domain = 1;  // corners outside the vertex range the optimizer's block list covers
#pragma unroll 1
        for (int l = hh * (L / 2); l < (hh + 1) * (L / 2); ++l) {
          float d[F];
#pragma unroll
          for (int j = 0; j < F; ++j) {
            d[j] = FT[(l * F + j) * kPp + r];
            if (MODE == MODE_BACKWARD && a.df_out) a.df_out[pp * D0 + l * F + j] = d[j];
          }
          scatter_level<F>(a.grads + (size_t)l * nd.T * F, nd.T - 1, (float)nd.res[l], px, py, pz, d);
        }
      }
    }
    __syncthreads();  // the next tile rewrites the buffers
  }

  if (MODE == MODE_TRAIN || MODE == 3) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local_acc += __shfl_xor_sync(0xffffffffu, local_acc, o);
    if ((tid & 31) == 0 && local_acc != 0.0) atomicAdd(acc, local_acc);
  }
  if constexpr (kBwd) {
    float *g = a.grads + nd.n_table;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (gW1[s][j] != 0.f) atomicAdd(g + nd.w_off[1] + (pg + 16 * s) * kHid + cg + 16 * j, gW1[s][j]);
#pragma unroll
      for (int j = 0; j < JD; ++j)
        if (gW0[s][j] != 0.f) atomicAdd(g + nd.w_off[0] + (pg + 16 * s) * D0 + cg + 16 * j, gW0[s][j]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (gW2[j] != 0.f) atomicAdd(g + nd.w_off[2] + cg + 16 * j, gW2[j]);
  }
}

template <int D0, int F, int MODE>
nv_status launch64(const nv_ctx *c, const MlpArgs &a, const int *n_dev, int n_mult, int64_t n_upper, double *acc) {
  using P = Plan64<D0>;
  const size_t bytes = (size_t)P::TOTAL * sizeof(float);
  auto kern = k_mlp_f32x<D0, F, MODE>;
  static int per_sm = 0;
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return nv_cuda_check(e, "cudaFuncSetAttribute(k_mlp_f32x)");
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kT, bytes);
    if (e != cudaSuccess) return nv_cuda_check(e, "occupancy(k_mlp_f32x)");
    per_sm = n < 1 ? 1 : n;
  }
  const int64_t ntiles = (n_upper + kPts - 1) / kPts;
  int64_t grid = (int64_t)c->num_sms * per_sm;
  if (ntiles < grid) grid = ntiles;
  if (grid < 1) return NV_OK;
  kern<<<(unsigned)grid, kT, bytes, c->stream>>>(c->nd, c->params, a, n_dev, n_mult, acc);
  return nv_cuda_check(cudaGetLastError(), "k_mlp_f32x launch");
}

template <int D0, int F>
nv_status by_mode(const nv_ctx *c, int mode, const MlpArgs &a, const int *n_dev, int n_mult, int64_t n_upper,
                  double *acc) {
  switch (mode) {
    case MODE_INFER: return launch64<D0, F, MODE_INFER>(c, a, n_dev, n_mult, n_upper, acc);
    case MODE_BACKWARD: return launch64<D0, F, MODE_BACKWARD>(c, a, n_dev, n_mult, n_upper, acc);
    case MODE_TRAIN: return launch64<D0, F, MODE_TRAIN>(c, a, n_dev, n_mult, n_upper, acc);
    case 3: return launch64<D0, F, 3>(c, a, n_dev, n_mult, n_upper, acc);
  }
  return nv_fail(NV_ERR_ARG, "bad MLP mode %d", mode);
}

}  // namespace

bool f32x_supported(const NetDesc &nd) {
  if (nd.n_dims != 4 || nd.dims[1] != kHid || nd.dims[2] != kHid || nd.dims[3] != 1) return false;
  const int F = nd.F, D0 = nd.dims[0];
  if (D0 != nd.L * F || nd.L % 2) return false;
  return (F == 2 && (D0 == 16 || D0 == 32 || D0 == 64)) || (F == 4 && (D0 == 32 || D0 == 64));
}

nv_status launch_mlp_f32x(const nv_ctx *c, int mode, const MlpArgs &a, const int *n_dev, int n_mult,
                          int64_t n_upper, double *acc) {
  const int F = c->nd.F, D0 = c->nd.dims[0];
  if (F == 2 && D0 == 16) return by_mode<16, 2>(c, mode, a, n_dev, n_mult, n_upper, acc);
  if (F == 2 && D0 == 32) return by_mode<32, 2>(c, mode, a, n_dev, n_mult, n_upper, acc);
  if (F == 2 && D0 == 64) return by_mode<64, 2>(c, mode, a, n_dev, n_mult, n_upper, acc);
  if (F == 4 && D0 == 32) return by_mode<32, 4>(c, mode, a, n_dev, n_mult, n_upper, acc);
  if (F == 4 && D0 == 64) return by_mode<64, 4>(c, mode, a, n_dev, n_mult, n_upper, acc);
  return nv_fail(NV_ERR_UNSUPPORTED, "k_mlp_f32x: L*F=%d, F=%d", D0, F);
}

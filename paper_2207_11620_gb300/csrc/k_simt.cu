// k_simt.cu -- FP32 CUDA-core kernels: hash indices, encoding, and the fused
// encode + MLP forward / backward / training step (the FP32 parity path).
//
// Fused MLP kernel layout: a persistent grid, one CTA per SM, 128 threads; a
// tile is 128 points, one point per thread.  Shared memory holds all weights,
// every layer's activations of the tile ([P][width+1] rows, the +1 keeps the
// per-thread row walks and the cross-point weight-gradient sweeps free of
// bank conflicts), the output deltas and the CTA's weight-gradient
// accumulator, which is flushed to global memory once at the end.
#include "nv_internal.cuh"

namespace {

constexpr int kP = 128;  // points per tile == threads per CTA

template <int F>
__device__ __forceinline__ void load_entry(const float *__restrict__ p, float *e) {
  if constexpr (F == 1) {
    e[0] = __ldg(p);
  } else if constexpr (F == 2) {
    float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    e[0] = v.x; e[1] = v.y;
  } else if constexpr (F == 4) {
    float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    e[0] = v.x; e[1] = v.y; e[2] = v.z; e[3] = v.w;
  } else {
    float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    float4 u = __ldg(reinterpret_cast<const float4 *>(p) + 1);
    e[0] = v.x; e[1] = v.y; e[2] = v.z; e[3] = v.w;
    e[4] = u.x; e[5] = u.y; e[6] = u.z; e[7] = u.w;
  }
}

template <int F>
__device__ __forceinline__ void add_entry(float *p, const float *g) {
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

// A-1..A-3 at one level: trilinear blend of the 8 hashed corner entries.
template <int F>
__device__ __forceinline__ void encode_level(const float *__restrict__ tab, uint32_t Tmask, float N,
                                             float x, float y, float z, float *out) {
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
    float w = (dx ? wx : 1.f - wx) * (dy ? wy : 1.f - wy) * (dz ? wz : 1.f - wz);
    uint32_t h = nv_hash3((uint32_t)(cx + dx), (uint32_t)(cy + dy), (uint32_t)(cz + dz)) & Tmask;
    float e[F];
    load_entry<F>(tab + (size_t)h * F, e);
#pragma unroll
    for (int j = 0; j < F; ++j) out[j] += w * e[j];
  }
}

// A-7 at one level: scatter w_corner * df into the 8 corner gradients.
template <int F>
__device__ __forceinline__ void scatter_level(float *gtab, uint32_t Tmask, float N, float x, float y,
                                              float z, const float *df) {
  int cx, cy, cz;
  float wx, wy, wz;
  nv_cell(x, N, cx, wx);
  nv_cell(y, N, cy, wy);
  nv_cell(z, N, cz, wz);
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    const int dx = d & 1, dy = (d >> 1) & 1, dz = (d >> 2) & 1;
    float w = (dx ? wx : 1.f - wx) * (dy ? wy : 1.f - wy) * (dz ? wz : 1.f - wz);
    uint32_t h = nv_hash3((uint32_t)(cx + dx), (uint32_t)(cy + dy), (uint32_t)(cz + dz)) & Tmask;
    float g[F];
#pragma unroll
    for (int j = 0; j < F; ++j) g[j] = w * df[j];
    add_entry<F>(gtab + (size_t)h * F, g);
  }
}

__global__ void k_hash_indices(NetDesc nd, const float *__restrict__ xyz, int64_t n, uint32_t *idx) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
  for (int l = 0; l < nd.L; ++l) {
    int cx, cy, cz;
    float wx, wy, wz;
    float N = (float)nd.res[l];
    nv_cell(x, N, cx, wx);
    nv_cell(y, N, cy, wy);
    nv_cell(z, N, cz, wz);
    for (int d = 0; d < 8; ++d)
      idx[(i * nd.L + l) * 8 + d] =
          nv_hash3((uint32_t)(cx + (d & 1)), (uint32_t)(cy + ((d >> 1) & 1)), (uint32_t)(cz + ((d >> 2) & 1))) &
          (nd.T - 1);
  }
}

template <int F>
__global__ void k_encode_f32(NetDesc nd, const float *__restrict__ params, const float *__restrict__ xyz,
                             int64_t n, float *feat) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
  const int LF = nd.L * F;
  for (int l = 0; l < nd.L; ++l) {
    float out[F];
    encode_level<F>(params + (size_t)l * nd.T * F, nd.T - 1, (float)nd.res[l], x, y, z, out);
#pragma unroll
    for (int j = 0; j < F; ++j) feat[i * LF + l * F + j] = out[j];
  }
}

struct SmemPlan {
  int act_off[NV_MAX_LAYERS + 1];  // float offset of act_k (rows of dims[k]+1)
  int dout_off, gw_off, total;      // floats
};

__host__ __device__ inline SmemPlan plan_smem(const NetDesc &nd, int mode) {
  SmemPlan s;
  int off = (int)nd.n_weights;
  for (int k = 0; k + 1 < nd.n_dims; ++k) {  // act_k is the input of layer k
    s.act_off[k] = off;
    off += kP * (nd.dims[k] + 1);
  }
  s.dout_off = off;
  if (mode != MODE_INFER) off += kP;
  off = (off + 1) & ~1;  // the FP64 accumulator needs 8-byte alignment
  s.gw_off = off;
  if (mode == MODE_BACKWARD || mode == MODE_TRAIN) off += 2 * (int)nd.n_weights;
  s.total = off;
  return s;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// MODE_INFER: y = net(x).  MODE_BACKWARD: grads += d(sum dL/dy * y)/dparams.
// MODE_TRAIN: loss += sum (y - t)^2; grads += d(loss / n)/dparams.
// Mode 3 (volume MSE): x = voxel centre of point index p, accumulates (y - vol)^2.
template <int F, int MODE>
__global__ void __launch_bounds__(kP) k_mlp_f32(NetDesc nd, const float *__restrict__ params, MlpArgs a,
                                                 const int *__restrict__ n_dev, int n_mult, double *acc) {
  extern __shared__ float sm[];
  const SmemPlan sp = plan_smem(nd, MODE == 3 ? MODE_INFER : MODE);
  const int tid = threadIdx.x;
  const int nl = nd.n_dims - 1;
  float *sW = sm;
  for (int64_t i = tid; i < nd.n_weights; i += kP) sW[i] = params[nd.n_table + i];
  // the CTA's weight-gradient accumulator is FP64: it sums one FP32 partial per tile
  double *sGW = reinterpret_cast<double *>(sm + sp.gw_off);
  if (MODE == MODE_BACKWARD || MODE == MODE_TRAIN)
    for (int64_t i = tid; i < nd.n_weights; i += kP) sGW[i] = 0.0;
  __syncthreads();

  const int64_t n = n_dev ? (int64_t)(*n_dev) * n_mult : a.n;
  const int64_t ntiles = (n + kP - 1) / kP;
  const int d0 = nd.dims[0];
  double local_acc = 0.0;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t p = tile * kP + tid;
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
        x = a.xyz[3 * p]; y = a.xyz[3 * p + 1]; z = a.xyz[3 * p + 2];
        if (MODE == MODE_TRAIN) tgt = a.in[p];
      } else {
        float3 s = nv_sample_point(a.seed, a.sample_step, (uint64_t)p);
        x = s.x; y = s.y; z = s.z;
        tgt = nv_trilinear(a.vol.data_dev, a.vol.nx, a.vol.ny, a.vol.nz, x, y, z);
      }
    }
    // encode into act_0 row
    float *a0 = sm + sp.act_off[0] + tid * (d0 + 1);
    for (int l = 0; l < nd.L; ++l) {
      float out[F];
      encode_level<F>(params + (size_t)l * nd.T * F, nd.T - 1, (float)nd.res[l], x, y, z, out);
#pragma unroll
      for (int j = 0; j < F; ++j) a0[l * F + j] = out[j];
    }
    // forward
    float zlast = 0.f;
    for (int k = 0; k < nl; ++k) {
      const int din = nd.dims[k], dout = nd.dims[k + 1];
      const float *in = sm + sp.act_off[k] + tid * (din + 1);
      const float *W = sW + nd.w_off[k];
      if (k + 1 < nl) {
        float *out = sm + sp.act_off[k + 1] + tid * (dout + 1);
        for (int j = 0; j < dout; ++j) {
          float s = 0.f;
          for (int i = 0; i < din; ++i) s += W[j * din + i] * in[i];
          out[j] = fmaxf(s, 0.f);
        }
      } else {
        float s = 0.f;
        for (int i = 0; i < din; ++i) s += W[i] * in[i];
        zlast = s;
      }
    }
    const float yv = 1.f / (1.f + expf(-zlast));
    if (MODE == MODE_INFER) {
      if (valid) a.y[p] = yv;
      continue;
    }
    if (MODE == 3) {
      if (valid) { double dd = (double)yv - (double)tgt; local_acc += dd * dd; }
      continue;
    }
    // output delta
    float g = 0.f;
    if (valid) {
      if (MODE == MODE_TRAIN) {
        float diff = yv - tgt;
        if (a.l1) {
          local_acc += fabs((double)diff);
          g = (float)((diff > 0.f) - (diff < 0.f)) * a.inv_n;
        } else {
          local_acc += (double)diff * (double)diff;
          g = 2.f * diff * a.inv_n;
        }
      } else {
        g = a.in[p];
      }
    }
    float *sDout = sm + sp.dout_off;
    sDout[tid] = g * yv * (1.f - yv);
    // backward, layer by layer from the output
    for (int k = nl - 1; k >= 0; --k) {
      const int din = nd.dims[k], dout = nd.dims[k + 1];
      const float *act = sm + sp.act_off[k];
      const float *dl = (k == nl - 1) ? sDout : sm + sp.act_off[k + 1];
      const int dstride = (k == nl - 1) ? 1 : dout + 1;
      __syncthreads();
      // dW_k += sum over the tile's points of delta_k (x) act_k
      for (int e = tid; e < dout * din; e += kP) {
        const int j = e / din, i = e - j * din;
        float s = 0.f;
        for (int q = 0; q < kP; ++q) s += dl[q * dstride + j] * act[q * (din + 1) + i];
        sGW[nd.w_off[k] + e] += (double)s;
      }
      __syncthreads();
      const float *W = sW + nd.w_off[k];
      const float *myd = dl + tid * dstride;
      if (k > 0) {
        // delta_{k-1} = (W_k^T delta_k) * 1[a_k > 0], written over this thread's act_k row
        float *row = sm + sp.act_off[k] + tid * (din + 1);
        for (int i = 0; i < din; ++i) {
          float s = 0.f;
          for (int j = 0; j < dout; ++j) s += W[j * din + i] * myd[j];
          row[i] = row[i] > 0.f ? s : 0.f;
        }
      } else if (valid) {
        // df = W_0^T delta_0, scattered level by level into the table gradients
        if (!(x >= 0.f && x <= 1.f && y >= 0.f && y <= 1.f && z >= 0.f && z <= 1.f))
          a.ds->off_domain = 1;  // corners outside the vertex range the optimizer's block list covers
        for (int l = 0; l < nd.L; ++l) {
          float df[F];
#pragma unroll
          for (int jf = 0; jf < F; ++jf) {
            const int i = l * F + jf;
            float s = 0.f;
            for (int j = 0; j < dout; ++j) s += W[j * din + i] * myd[j];
            df[jf] = s;
            if (a.df_out) a.df_out[p * din + i] = s;
          }
          scatter_level<F>(a.grads + (size_t)l * nd.T * F, nd.T - 1, (float)nd.res[l], x, y, z, df);
        }
      }
    }
    __syncthreads();  // act rows are rewritten by the next tile's encode
  }

  if (MODE == MODE_TRAIN || MODE == 3) {
    double v = warp_sum_d(local_acc);
    if ((tid & 31) == 0 && v != 0.0) atomicAdd(acc, v);
  }
  if (MODE == MODE_BACKWARD || MODE == MODE_TRAIN) {
    __syncthreads();
    for (int64_t i = tid; i < nd.n_weights; i += kP) {
      float v = (float)sGW[i];
      if (v != 0.f) atomicAdd(a.grads + nd.n_table + i, v);
    }
  }
}

template <int F, int MODE>
nv_status launch_mode(const nv_ctx *c, const MlpArgs &a, const int *n_dev, int n_mult, int64_t n_upper,
                      double *acc) {
  SmemPlan sp = plan_smem(c->nd, MODE == 3 ? MODE_INFER : MODE);
  size_t bytes = (size_t)sp.total * sizeof(float);
  if (bytes > 227 * 1024)
    return nv_fail(NV_ERR_UNSUPPORTED, "FP32 MLP needs %zu B of shared memory (> 227 KiB)", bytes);
  auto kern = k_mlp_f32<F, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return nv_cuda_check(e, "cudaFuncSetAttribute(k_mlp_f32)");
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kP, bytes);
  if (per_sm < 1) per_sm = 1;
  int64_t ntiles = (n_upper + kP - 1) / kP;
  int64_t grid = (int64_t)c->num_sms * per_sm;
  if (ntiles < grid) grid = ntiles;
  if (grid < 1) return NV_OK;
  kern<<<(unsigned)grid, kP, bytes, c->stream>>>(c->nd, c->params, a, n_dev, n_mult, acc);
  return nv_cuda_check(cudaGetLastError(), "k_mlp_f32 launch");
}

template <int MODE>
nv_status dispatch_f(const nv_ctx *c, const MlpArgs &a, const int *n_dev, int n_mult, int64_t n_upper,
                     double *acc) {
  switch (c->nd.F) {
    case 1: return launch_mode<1, MODE>(c, a, n_dev, n_mult, n_upper, acc);
    case 2: return launch_mode<2, MODE>(c, a, n_dev, n_mult, n_upper, acc);
    case 4: return launch_mode<4, MODE>(c, a, n_dev, n_mult, n_upper, acc);
    case 8: return launch_mode<8, MODE>(c, a, n_dev, n_mult, n_upper, acc);
  }
  return nv_fail(NV_ERR_UNSUPPORTED, "F=%d (supported: 1, 2, 4, 8)", c->nd.F);
}

// Gradient of the loss in the point coordinates from dL/df (the Jacobian of
// A-3): within a cell of level l, the weight of corner d is a product of w_a
// or 1 - w_a with w_a = x_a N_l - c_a, so its derivative in x_a is N_l times
// +1 (upper corner) or -1 (lower) times the other two axes' factors; dL/dx_a
// sums that times <theta_l[h_d], dL/df_l> over levels and corners.  FP32
// master tables, one thread per point.
template <int F>
__global__ void __launch_bounds__(256) k_coord_grad(NetDesc nd, const float *__restrict__ params,
                                                    const float *__restrict__ xyz, int64_t n,
                                                    const float *__restrict__ df, float *__restrict__ dxyz) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
  const int D0 = nd.L * F;
  float gx = 0.f, gy = 0.f, gz = 0.f;
  for (int l = 0; l < nd.L; ++l) {
    const float N = (float)nd.res[l];
    int cx, cy, cz;
    float wx, wy, wz;
    nv_cell(x, N, cx, wx);
    nv_cell(y, N, cy, wy);
    nv_cell(z, N, cz, wz);
    float d[F];
#pragma unroll
    for (int j = 0; j < F; ++j) d[j] = df[i * D0 + l * F + j];
    const float *tab = params + (size_t)l * nd.T * F;
    float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
      const uint32_t h = nv_hash3((uint32_t)(cx + dx), (uint32_t)(cy + dy), (uint32_t)(cz + dz)) & (nd.T - 1);
      float e[F];
      load_entry<F>(tab + (size_t)h * F, e);
      float dot = 0.f;
#pragma unroll
      for (int j = 0; j < F; ++j) dot += e[j] * d[j];
      const float fx = dx ? wx : 1.f - wx, fy = dy ? wy : 1.f - wy, fz = dz ? wz : 1.f - wz;
      sx += (dx ? fy : -fy) * fz * dot;
      sy += (dy ? fx : -fx) * fz * dot;
      sz += (dz ? fx : -fx) * fy * dot;
    }
    gx += N * sx;
    gy += N * sy;
    gz += N * sz;
  }
  dxyz[3 * i] = gx;
  dxyz[3 * i + 1] = gy;
  dxyz[3 * i + 2] = gz;
}

}  // namespace

nv_status launch_hash_indices(const nv_ctx *c, const float *xyz, int64_t n, uint32_t *idx) {
  if (n == 0) return NV_OK;
  int64_t blocks = (n + 255) / 256;
  k_hash_indices<<<(unsigned)blocks, 256, 0, c->stream>>>(c->nd, xyz, n, idx);
  return nv_cuda_check(cudaGetLastError(), "k_hash_indices launch");
}

nv_status launch_encode_f32(const nv_ctx *c, const float *xyz, int64_t n, float *feat) {
  if (n == 0) return NV_OK;
  unsigned blocks = (unsigned)((n + 255) / 256);
  switch (c->nd.F) {
    case 1: k_encode_f32<1><<<blocks, 256, 0, c->stream>>>(c->nd, c->params, xyz, n, feat); break;
    case 2: k_encode_f32<2><<<blocks, 256, 0, c->stream>>>(c->nd, c->params, xyz, n, feat); break;
    case 4: k_encode_f32<4><<<blocks, 256, 0, c->stream>>>(c->nd, c->params, xyz, n, feat); break;
    case 8: k_encode_f32<8><<<blocks, 256, 0, c->stream>>>(c->nd, c->params, xyz, n, feat); break;
    default: return nv_fail(NV_ERR_UNSUPPORTED, "F=%d", c->nd.F);
  }
  return nv_cuda_check(cudaGetLastError(), "k_encode_f32 launch");
}

// The register-blocked kernel for the D0 -> 64 -> 64 -> 1 networks (k_simt64.cu).
bool f32x_supported(const NetDesc &nd);
nv_status launch_mlp_f32x(const nv_ctx *c, int mode, const MlpArgs &a, const int *n_dev, int n_mult,
                          int64_t n_upper, double *acc);

// mode: MODE_INFER / MODE_BACKWARD / MODE_TRAIN, or 3 = volume MSE into acc.
nv_status launch_mlp_f32_ext(const nv_ctx *c, int mode, const MlpArgs &a, const int *n_dev, int n_mult,
                             int64_t n_upper, double *acc) {
  if (f32x_supported(c->nd)) return launch_mlp_f32x(c, mode, a, n_dev, n_mult, n_upper, acc);
  switch (mode) {
    case MODE_INFER: return dispatch_f<MODE_INFER>(c, a, n_dev, n_mult, n_upper, acc);
    case MODE_BACKWARD: return dispatch_f<MODE_BACKWARD>(c, a, n_dev, n_mult, n_upper, acc);
    case MODE_TRAIN: return dispatch_f<MODE_TRAIN>(c, a, n_dev, n_mult, n_upper, acc);
    case 3: return dispatch_f<3>(c, a, n_dev, n_mult, n_upper, acc);
  }
  return nv_fail(NV_ERR_ARG, "bad MLP mode %d", mode);
}

nv_status launch_mlp_f32(const nv_ctx *c, int mode, const MlpArgs &a) {
  return launch_mlp_f32_ext(c, mode, a, nullptr, 1, a.n, mode == MODE_TRAIN ? &a.ds->loss_acc : nullptr);
}

// df: [n][L*F] dL/df of nv_backward; dxyz: [n][3] written.
nv_status launch_coord_grad(const nv_ctx *c, const float *xyz, int64_t n, const float *df, float *dxyz) {
  if (n == 0) return NV_OK;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  switch (c->nd.F) {
    case 1: k_coord_grad<1><<<blocks, 256, 0, c->stream>>>(c->nd, c->params, xyz, n, df, dxyz); break;
    case 2: k_coord_grad<2><<<blocks, 256, 0, c->stream>>>(c->nd, c->params, xyz, n, df, dxyz); break;
    case 4: k_coord_grad<4><<<blocks, 256, 0, c->stream>>>(c->nd, c->params, xyz, n, df, dxyz); break;
    case 8: k_coord_grad<8><<<blocks, 256, 0, c->stream>>>(c->nd, c->params, xyz, n, df, dxyz); break;
    default: return nv_fail(NV_ERR_UNSUPPORTED, "F=%d", c->nd.F);
  }
  return nv_cuda_check(cudaGetLastError(), "k_coord_grad launch");
}

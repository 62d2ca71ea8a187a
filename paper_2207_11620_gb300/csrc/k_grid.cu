// k_grid.cu -- the memory-bound halves of the tensor-core path: the hash-grid
// gather that produces FP16/BF16 features in the tensor-core tile layout
// (A-1..A-3), and the scatter of the input gradient into the FP32 table
// gradient (A-7).  Both are kept out of the tensor-core kernel so that they
// run at full occupancy: each thread issues all the loads (or atomics) of its
// levels back to back and dozens of warps per SM keep the L1-to-L2 request
// path busy.
//
// Work item = (point, chunk of 8 features): with F features per level a chunk
// covers 8 / F levels.  Items are chunk-major, so neighbouring threads handle
// neighbouring points at the same levels (coarse-level table lines are shared
// in L1) and write one 16-byte core-matrix row each.
#include "nv_internal.cuh"
#include "tc_grid.cuh"

namespace {

template <int F, bool BF>
__global__ void __launch_bounds__(256) k_encode_tiles(NetDesc nd, const uint16_t *__restrict__ shadow, PointSrc ps,
                                                      ChunkSpan cs, uint8_t *__restrict__ feat) {
  const int D0 = nd.dims[0];
  const int C = D0 / 8;
  const int64_t n = chunk_count(cs);
  const int64_t npad = (cs.cap + 127) & ~int64_t(127);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad * C) return;
  const int c = (int)(i / npad);
  const int64_t q = i - (int64_t)c * npad;
  uint8_t *dst = feat + (q >> 7) * (int64_t)(128 * D0 * 2) + tile_off((int)(q & 127), c * 8, D0);
  if (q >= n) {
    if (q < npad) *reinterpret_cast<uint4 *>(dst) = make_uint4(0, 0, 0, 0);
    return;
  }
  const float3 x = point_at(ps, cs.off + q);
  float f8[8];
  gather_levels<F, BF, 8 / F>(shadow, nd, c * (8 / F), x.x, x.y, x.z, f8);
  uint4 u;
  u.x = pack16x2<BF>(f8[0], f8[1]);
  u.y = pack16x2<BF>(f8[2], f8[3]);
  u.z = pack16x2<BF>(f8[4], f8[5]);
  u.w = pack16x2<BF>(f8[6], f8[7]);
  *reinterpret_cast<uint4 *>(dst) = u;
}

// dF rows are FP32 [cap][D0], already divided by the loss scale.
template <int F>
__global__ void __launch_bounds__(256) k_scatter_tiles(NetDesc nd, PointSrc ps, ChunkSpan cs,
                                                       const float *__restrict__ dF, float *grads) {
  const int D0 = nd.dims[0];
  const int C = D0 / 8;
  const int64_t n = chunk_count(cs);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * C) return;
  const int c = (int)(i / n);
  const int64_t q = i - (int64_t)c * n;
  const float3 x = point_at(ps, cs.off + q);
  const float4 *src = reinterpret_cast<const float4 *>(dF + q * D0 + c * 8);
  const float4 a = __ldg(src), b = __ldg(src + 1);
  const float g8[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
  for (int k = 0; k < 8 / F; ++k) {
    const int l = c * (8 / F) + k;
    scatter_level<F>(grads + (size_t)l * nd.T * F, nd.T - 1, (float)nd.res[l], x.x, x.y, x.z, g8 + k * F);
  }
}

inline unsigned grid_for(int64_t items) { return (unsigned)((items + 255) / 256); }

}  // namespace

nv_status launch_encode_tiles(const nv_ctx *c, const PointSrc &ps, const ChunkSpan &cs, uint8_t *feat) {
  const int C = c->nd.dims[0] / 8;
  const int64_t npad = (cs.cap + 127) & ~int64_t(127);
  if (npad == 0) return NV_OK;
  const uint16_t *sh = reinterpret_cast<const uint16_t *>(c->shadow);
  const unsigned g = grid_for(npad * C);
  const bool bf = c->prec == NV_BF16;
  switch (c->nd.F) {
    case 2:
      if (bf) k_encode_tiles<2, true><<<g, 256, 0, c->stream>>>(c->nd, sh, ps, cs, feat);
      else k_encode_tiles<2, false><<<g, 256, 0, c->stream>>>(c->nd, sh, ps, cs, feat);
      break;
    case 4:
      if (bf) k_encode_tiles<4, true><<<g, 256, 0, c->stream>>>(c->nd, sh, ps, cs, feat);
      else k_encode_tiles<4, false><<<g, 256, 0, c->stream>>>(c->nd, sh, ps, cs, feat);
      break;
    default:
      return nv_fail(NV_ERR_UNSUPPORTED, "tensor-core encode: F=%d", c->nd.F);
  }
  return nv_cuda_check(cudaGetLastError(), "k_encode_tiles launch");
}

nv_status launch_scatter_tiles(const nv_ctx *c, const PointSrc &ps, const ChunkSpan &cs, const float *dF,
                               float *grads) {
  const int C = c->nd.dims[0] / 8;
  if (cs.cap == 0) return NV_OK;
  const unsigned g = grid_for(cs.cap * C);
  switch (c->nd.F) {
    case 2: k_scatter_tiles<2><<<g, 256, 0, c->stream>>>(c->nd, ps, cs, dF, grads); break;
    case 4: k_scatter_tiles<4><<<g, 256, 0, c->stream>>>(c->nd, ps, cs, dF, grads); break;
    default: return nv_fail(NV_ERR_UNSUPPORTED, "tensor-core scatter: F=%d", c->nd.F);
  }
  return nv_cuda_check(cudaGetLastError(), "k_scatter_tiles launch");
}

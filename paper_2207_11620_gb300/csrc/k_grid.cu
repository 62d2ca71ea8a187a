// k_grid.cu -- the gather half of the tensor-core path: the hash-grid lookup
// that produces FP16/BF16 features in the tensor-core tile layout (A-1..A-3),
// and, for points the training step samples itself, their trilinear ground
// truth (A-9).  It runs ahead of the MLP kernel at full occupancy: each thread
// issues all the loads of its levels back to back and dozens of warps per SM
// keep the L1-to-L2 request path busy, which the tensor-core kernel, with its
// few large CTAs, could not.  The adjoint scatter (A-7) runs inside the MLP
// kernel's backward epilogue (k_tc.cu).
//
// Work item = (point, group of chunks of 8 features): with F features per
// level a chunk covers 8 / F levels.  The grid's y index is the group and its
// x index runs over points, so neighbouring threads handle neighbouring points
// at the same levels (coarse-level table lines are shared in L1) and write
// one 16-byte core-matrix row per chunk.
#include "nv_internal.cuh"
#include "tc_grid.cuh"

namespace {

// CORNERS: every corner loaded on its own (gather_corners), for the coherent
// sample batches of ray marches and voxel sweeps; otherwise the x-paired
// gathers, whose fewer loads suit scattered points (training batches).
// A thread takes kChunksPerThread<CORNERS> consecutive chunks of its point, one
// after the other: the issue-bound coherent gather then computes the point's
// address, coordinates and tile row once for 16 levels instead of 4 (trained
// 1080p frame 19.4 -> 17.2 ms; 18.3 ms with two chunks per thread).
template <bool CORNERS>
constexpr int kChunksPerThread = CORNERS ? 4 : 1;

template <int F, bool BF, bool CORNERS>
__global__ void __launch_bounds__(256, CORNERS ? 6 : 5)
    k_encode_tiles(NetDesc nd, const uint16_t *__restrict__ shadow, PointSrc ps, ChunkSpan cs,
                   uint8_t *__restrict__ feat, float *__restrict__ tgt, float *__restrict__ xyz_out, int *off_flag) {
  const int D0 = nd.dims[0];
  const int64_t n = chunk_count(cs);
  const int64_t npad = (cs.cap + 127) & ~int64_t(127);
  constexpr int CPT = kChunksPerThread<CORNERS>;
  const int c0 = blockIdx.y * CPT;  // the first chunk of 8 features
  const int c1 = c0 + CPT < D0 / 8 ? c0 + CPT : D0 / 8;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= npad) return;
  uint8_t *row = feat + (q >> 7) * (int64_t)(128 * D0 * 2);
  if (q >= n) {
    // rows past n in the last tile the MLP kernel reads are zeroed; tiles past it are never read
    if (q < ((n + 127) & ~int64_t(127)))
      for (int c = c0; c < c1; ++c)
        *reinterpret_cast<uint4 *>(row + tile_off((int)(q & 127), c * 8, D0)) = make_uint4(0, 0, 0, 0);
    return;
  }
  const float3 x = point_at(ps, cs.off + q);
  if (c0 == 0) {
    if (off_flag && !(x.x >= 0.f && x.x <= 1.f && x.y >= 0.f && x.y <= 1.f && x.z >= 0.f && x.z <= 1.f))
      *off_flag = 1;  // its corners may lie outside the vertex range of the optimizer's block list
    if (tgt) tgt[q] = nv_trilinear(ps.vol.data_dev, ps.vol.nx, ps.vol.ny, ps.vol.nz, x.x, x.y, x.z);
    if (xyz_out) {
      xyz_out[3 * q] = x.x;
      xyz_out[3 * q + 1] = x.y;
      xyz_out[3 * q + 2] = x.z;
    }
  }
#pragma unroll 1
  for (int c = c0; c < c1; ++c) {
    float f8[8];
    if constexpr (CORNERS) {
      gather_corners<F, BF, 8 / F>(shadow, nd, c * (8 / F), x.x, x.y, x.z, f8);
    } else if constexpr (F == 2) {
      gather_levels_f2<BF, 4>(shadow, nd, c * 4, x.x, x.y, x.z, f8);
    } else {  // one level at a time: fewer registers, more resident warps
#pragma unroll
      for (int g = 0; g < 8 / F; ++g)
        gather_levels<F, BF, 1>(shadow, nd, c * (8 / F) + g, x.x, x.y, x.z, f8 + g * F);
    }
    uint4 u;
    u.x = pack16x2<BF>(f8[0], f8[1]);
    u.y = pack16x2<BF>(f8[2], f8[3]);
    u.z = pack16x2<BF>(f8[4], f8[5]);
    u.w = pack16x2<BF>(f8[6], f8[7]);
    *reinterpret_cast<uint4 *>(row + tile_off((int)(q & 127), c * 8, D0)) = u;
  }
}

inline dim3 grid_for(int64_t points, int groups) { return dim3((unsigned)((points + 255) / 256), (unsigned)groups); }

}  // namespace

// tgt (nullable): [cap] targets of a Philox training sample (ps.kind == 2);
// xyz_out (nullable): [cap][3] its points, for the MLP kernel's scatter.
// off_flag (nullable): set to 1 when a point lies outside [0,1]^3.  coherent:
// neighbouring points share most corners (ray-march samples, voxel centres).
// Launched on st.
nv_status launch_encode_tiles(const nv_ctx *c, const PointSrc &ps, const ChunkSpan &cs, uint8_t *feat,
                              float *tgt, float *xyz_out, int *off_flag, bool coherent, cudaStream_t st) {
  const int C = c->nd.dims[0] / 8;
  const int64_t npad = (cs.cap + 127) & ~int64_t(127);
  if (npad == 0) return NV_OK;
  const uint16_t *sh = reinterpret_cast<const uint16_t *>(c->shadow);
  const bool bf = c->prec == NV_BF16;
#define NV_ENC(F_, BF_, CO_)                                                                                  \
  k_encode_tiles<F_, BF_, CO_><<<grid_for(npad, (C + kChunksPerThread<CO_> - 1) / kChunksPerThread<CO_>), 256, 0, \
                                 st>>>(c->nd, sh, ps, cs, feat, tgt, xyz_out, off_flag)
  switch (c->nd.F) {
    case 2:
      if (coherent) {
        if (bf) NV_ENC(2, true, true);
        else NV_ENC(2, false, true);
      } else {
        if (bf) NV_ENC(2, true, false);
        else NV_ENC(2, false, false);
      }
      break;
    case 4:
      if (coherent) {
        if (bf) NV_ENC(4, true, true);
        else NV_ENC(4, false, true);
      } else {
        if (bf) NV_ENC(4, true, false);
        else NV_ENC(4, false, false);
      }
      break;
    default:
      return nv_fail(NV_ERR_UNSUPPORTED, "tensor-core encode: F=%d", c->nd.F);
  }
#undef NV_ENC
  return nv_cuda_check(cudaGetLastError(), "k_encode_tiles launch");
}

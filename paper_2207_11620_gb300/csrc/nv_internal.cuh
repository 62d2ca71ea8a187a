// nv_internal.cuh -- shared declarations of the sm_103a neural-volume library:
// the network descriptor passed to kernels, the context and renderer structs,
// device helpers (spatial hash, Philox, trilinear lookup, camera rays) and the
// launchers each kernel file provides.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/nv.h"

#define NV_MAX_LEVELS 32
#define NV_MAX_LAYERS 10

// Everything a kernel needs to know about the network shape, passed by value.
struct NetDesc {
  int L, F, log2T;
  uint32_t T;                       // 2^log2T
  int res[NV_MAX_LEVELS];           // N_l = floor(Nmin b^l), computed on the host in FP64
  int n_dims;                       // MLP widths dims[0..n_dims-1]
  int dims[NV_MAX_LAYERS + 1];
  int64_t n_table;                  // L*T*F
  int64_t w_off[NV_MAX_LAYERS];     // offset of W_k inside the weight block
  int64_t n_weights;
};

// Device-side scalars of a context.
struct DevState {
  double loss_acc;    // sum of squared errors of the current batch
  double loss_mean;   // loss of the last training step (FP64)
  int step;           // optimizer steps taken (skipped overflow steps not counted)
  // the two flags a data-parallel step reduces (maximum) across replicas, adjacent (nv_dp_buffers)
  int overflow;       // set when a gradient contribution was not finite
  int off_domain;     // set (for good) when a table gradient was scattered from a point outside [0,1]^3
  float loss_scale;   // static loss scale of the tensor-core backward
  int err;            // set by a kernel whose bounded wait ran out
  unsigned adam_done; // CTAs of the running Adam launch that have finished (the last one resets it)
};

// Dense replicas of the coarsest levels' table gradient (tensor-core
// training): level l < levels keeps R copies of an n1[l]^3-vertex grid (n1 =
// N_l + 2 rounded up to even, x fastest), F floats per vertex; the backward
// scatters a point of [0,1]^3 into copy (CTA mod R) by vertex index; a
// following kernel folds the copies into the hashed slots.
struct HotRep {
  float *buf;          // [R][vtot][F], zero between launches
  int levels;          // 0: no replicas
  int R;
  int n1[4];
  int64_t vbase[5];    // first vertex of each level; vbase[levels] = vtot
};

struct nv_ctx {
  NetDesc nd;
  int Nmin;
  double b;
  int prec;
  cudaStream_t stream;
  int64_t n_params;
  float *params, *grads, *adam_m, *adam_v;  // FP32 [n_params]
  void *shadow;                             // FP16/BF16 copy of params (tensor-core precisions)
  DevState *ds;
  nv_adam_cfg adam;
  int loss_kind;                            // nv_loss of nv_train_step
  float *mc_minmax;                         // online macrocell ranges the training samples widen (or NULL)
  int mc_nx, mc_ny, mc_nz, mc_cell;
  uint32_t sample_counter;                  // Philox step word of sampled batches
  int params_set;
  float *batch[2];                          // staging for host batches, two slots: [cap][3] xyz + [cap] target
  int64_t batch_cap;
  int batch_slot;                           // slot of the next host batch
  cudaStream_t copy_stream;                 // host-batch copies (created on first use)
  cudaEvent_t batch_copied[2], batch_used[2];
  int num_sms;
  struct Prof *prof;                        // kernel timing (nv_profile_enable), NULL when off
  uint8_t *tc_feat;                         // tensor-core path: one chunk of 16-bit features (tile layout)
  float *tc_tgt;                            // tensor-core path: one chunk of sampled training targets
  float *tc_xyz;                            // tensor-core path: the points of that chunk [cap][3]
  int64_t tc_cap;                           // points per chunk of the two above
  int32_t *adam_blocks;                     // sorted 128-parameter blocks Adam visits (NULL: all of them)
  int64_t adam_nblocks;                     // entries of adam_blocks
  int adam_dense;                           // 1: Adam visits every block from now on (sticky)
  float *df_buf;                            // nv_backward with a coordinate gradient: dL/df [cap][L*F]
  int64_t df_cap;
  HotRep hot;                               // dense replicas of the coarsest levels' gradient (TC path)
};

// Kernel timing hooks (nv_api.cu): bracket a launch on the context stream.
int prof_begin(nv_ctx *c);
void prof_end(nv_ctx *c, int kclass, int token);

struct nv_renderer {
  int64_t max_pixels;
  int K;
  cudaStream_t stream;
  // ray state, two structure-of-arrays copies (ping-pong across compaction)
  float *ray[2];       // [13][max_pixels]: ox oy oz dx dy dz t0 t1 r g b a, (pixel id as int bits)
  int *next_k[2];      // next sample index of each live ray
  float *coords;       // [max_pixels*K][3] sample positions of the current iteration
  float *values;       // [max_pixels*K] sample values
  float *seg_exp;      // [max_pixels*K] opacity exponents of adaptive-step samples (NULL: fixed step only)
  float *aux[2];       // [5][max_pixels] single-shot shadow state, ping-pong with ray (NULL: no shadows)
  float *pt[2];        // path-tracer state [28][max_pixels], ping-pong (allocated on first use)
  float *pt_coords;    // second buffer of pending collision points [max_pixels][3]
  int *nvalid;         // [max_pixels] valid samples of each ray this iteration
  int *counters;       // device: [0] live count (current), [1] live count (next)
  int *h_count;        // pinned host mirror of the live count
  int last_iters;
  int64_t last_samples;
  int64_t *d_samples;  // device counter of evaluated samples
};

// ---- error plumbing (defined in nv_api.cu) ----
nv_status nv_fail(nv_status s, const char *fmt, ...);
nv_status nv_cuda_check(cudaError_t e, const char *what);

// Return a non-OK status from the enclosing function.
#define NV_TRY(x)                      \
  do {                                 \
    nv_status _s = (x);                \
    if (_s != NV_OK) return _s;        \
  } while (0)

#define NV_CUDA(x, what) NV_TRY(nv_cuda_check((x), what))

// ---- device helpers ------------------------------------------------------

// Spatial hash of a grid vertex (Sec. 3.1, instant-NGP primes); the caller masks with T-1.
__device__ __forceinline__ uint32_t nv_hash3(uint32_t x, uint32_t y, uint32_t z) {
  return x ^ (y * 2654435761u) ^ (z * 805459861u);
}

// Scale + cell of one coordinate (A-1): p = fl32(x * N) without contraction,
// c = floor(p), w = p - c (exact in FP32).
__device__ __forceinline__ void nv_cell(float x, float N, int &c, float &w) {
  float p = __fmul_rn(x, N);
  float f = floorf(p);
  c = (int)f;
  w = __fsub_rn(p, f);
}

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds, multipliers 0xD2511F53 /
// 0xCD9E8D57, key schedule 0x9E3779B9 / 0xBB67AE85.
__device__ __forceinline__ uint4 nv_philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    uint4 n;
    n.x = hi1 ^ c.y ^ k0;
    n.y = lo1;
    n.z = hi0 ^ c.w ^ k1;
    n.w = lo0;
    c = n;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Training coordinate of sample `id` at sampler step `step` (A-9).
__device__ __forceinline__ float3 nv_sample_point(uint64_t seed, uint32_t step, uint64_t id) {
  uint4 c = make_uint4((uint32_t)id, (uint32_t)(id >> 32), step, 0u);
  uint4 u = nv_philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const float s = 1.0f / 16777216.0f;
  return make_float3((float)(u.x >> 8) * s, (float)(u.y >> 8) * s, (float)(u.z >> 8) * s);
}

// One axis of a cell-centred trilinear lookup: q = x*n - 0.5 (two FP32 roundings,
// the cell decision), clamped to [0, n-1], lower index capped at n-2.
__device__ __forceinline__ void nv_voxel_axis(float x, int n, int &i0, int &i1, float &w) {
  if (n == 1) { i0 = 0; i1 = 0; w = 0.f; return; }
  float q = __fadd_rn(__fmul_rn(x, (float)n), -0.5f);
  q = fminf(fmaxf(q, 0.0f), (float)(n - 1));
  int i = (int)floorf(q);
  i = min(i, n - 2);
  i0 = i;
  i1 = i + 1;
  w = __fsub_rn(q, (float)i);
}

// Trilinear value of the raw volume at x (Sec. 4 ground truth; raw-volume render path).
__device__ __forceinline__ float nv_trilinear(const float *__restrict__ vol, int nx, int ny, int nz,
                                              float x, float y, float z) {
  int x0, x1, y0, y1, z0, z1;
  float wx, wy, wz;
  nv_voxel_axis(x, nx, x0, x1, wx);
  nv_voxel_axis(y, ny, y0, y1, wy);
  nv_voxel_axis(z, nz, z0, z1, wz);
  const int64_t sy = nx, sz = (int64_t)nx * ny;
  const float *p00 = vol + z0 * sz + y0 * sy, *p01 = vol + z0 * sz + y1 * sy;
  const float *p10 = vol + z1 * sz + y0 * sy, *p11 = vol + z1 * sz + y1 * sy;
  float c00 = __ldg(p00 + x0) + wx * (__ldg(p00 + x1) - __ldg(p00 + x0));
  float c01 = __ldg(p01 + x0) + wx * (__ldg(p01 + x1) - __ldg(p01 + x0));
  float c10 = __ldg(p10 + x0) + wx * (__ldg(p10 + x1) - __ldg(p10 + x0));
  float c11 = __ldg(p11 + x0) + wx * (__ldg(p11 + x1) - __ldg(p11 + x0));
  float c0 = c00 + wy * (c01 - c00);
  float c1 = c10 + wy * (c11 - c10);
  return c0 + wz * (c1 - c0);
}

// Camera ray through the centre of pixel (px, py), every operation rounded on
// its own (no contraction): the sample positions, and with them the macrocell
// and hash-cell decisions, must not depend on the compiler.
__device__ __forceinline__ void nv_norm3(float &x, float &y, float &z) {
  float s = __fmul_rn(x, x);
  s = __fadd_rn(s, __fmul_rn(y, y));
  s = __fadd_rn(s, __fmul_rn(z, z));
  float len = __fsqrt_rn(s);
  x = __fdiv_rn(x, len); y = __fdiv_rn(y, len); z = __fdiv_rn(z, len);
}

__device__ __forceinline__ void nv_cross(float ax, float ay, float az, float bx, float by, float bz,
                                         float &cx, float &cy, float &cz) {
  cx = __fsub_rn(__fmul_rn(ay, bz), __fmul_rn(az, by));
  cy = __fsub_rn(__fmul_rn(az, bx), __fmul_rn(ax, bz));
  cz = __fsub_rn(__fmul_rn(ax, by), __fmul_rn(ay, bx));
}

__device__ __forceinline__ void nv_camera_ray(const nv_camera &cam, int px, int py, float o[3], float d[3]) {
  float fx = __fsub_rn(cam.target[0], cam.eye[0]);
  float fy = __fsub_rn(cam.target[1], cam.eye[1]);
  float fz = __fsub_rn(cam.target[2], cam.eye[2]);
  nv_norm3(fx, fy, fz);
  float rx, ry, rz, ux, uy, uz;
  nv_cross(cam.up[0], cam.up[1], cam.up[2], fx, fy, fz, rx, ry, rz);
  nv_norm3(rx, ry, rz);
  nv_cross(fx, fy, fz, rx, ry, rz, ux, uy, uz);
  float u = __fsub_rn(__fdiv_rn(__fmul_rn(2.0f, __fadd_rn((float)px, 0.5f)), (float)cam.width), 1.0f);
  float v = __fsub_rn(1.0f, __fdiv_rn(__fmul_rn(2.0f, __fadd_rn((float)py, 0.5f)), (float)cam.height));
  float fw[3] = {fx, fy, fz}, rt[3] = {rx, ry, rz}, up2[3] = {ux, uy, uz};
  if (cam.tan_half_fovy > 0.0f) {
    float aspect = __fdiv_rn((float)cam.width, (float)cam.height);
    float su = __fmul_rn(__fmul_rn(u, cam.tan_half_fovy), aspect);
    float sv = __fmul_rn(v, cam.tan_half_fovy);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      d[a] = __fadd_rn(__fadd_rn(fw[a], __fmul_rn(su, rt[a])), __fmul_rn(sv, up2[a]));
      o[a] = cam.eye[a];
    }
    nv_norm3(d[0], d[1], d[2]);
  } else {
    float hu = __fmul_rn(__fmul_rn(u, cam.ortho_w), 0.5f);
    float hv = __fmul_rn(__fmul_rn(v, cam.ortho_h), 0.5f);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      o[a] = __fadd_rn(__fadd_rn(cam.eye[a], __fmul_rn(hu, rt[a])), __fmul_rn(hv, up2[a]));
      d[a] = fw[a];
    }
  }
}

// Slab test against [0,1]^3 clipped to t >= 0 (fminf/fmaxf drop the NaN of 0*inf).
__device__ __forceinline__ bool nv_box(const float o[3], const float d[3], float &t0, float &t1) {
  float tn = 0.0f, tf = __int_as_float(0x7f800000);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float inv = __fdiv_rn(1.0f, d[a]);
    float ta = __fmul_rn(__fsub_rn(0.0f, o[a]), inv);
    float tb = __fmul_rn(__fsub_rn(1.0f, o[a]), inv);
    tn = fmaxf(tn, fminf(ta, tb));
    tf = fminf(tf, fmaxf(ta, tb));
  }
  t0 = tn;
  t1 = tf;
  return tn < tf;
}

// ---- launchers (one per kernel file) ---------------------------------------

enum MlpMode { MODE_INFER = 0, MODE_BACKWARD = 1, MODE_TRAIN = 2 };

struct MlpArgs {
  const float *xyz;      // [n][3] or NULL (TRAIN: sample from vol)
  const float *in;       // TRAIN: targets [n] (NULL when sampling); BACKWARD: dL/dy [n]
  int64_t n;
  float *y;              // INFER output [n]
  float *grads;          // BACKWARD / TRAIN gradient accumulator [n_params]
  DevState *ds;
  nv_volume vol;         // TRAIN with xyz == NULL
  uint64_t seed;
  uint32_t sample_step;
  float inv_n;           // TRAIN: 1/n of the batch mean
  int l1;                // TRAIN: L1 loss (else L2)
  float *df_out;         // BACKWARD (nullable): dL/df of every point, [n][L*F] FP32
  HotRep hot;            // TRAIN / BACKWARD, tensor-core path (levels = 0: none)
  int coherent;          // INFER: the points are ray-march samples (neighbours share corners)
};

// FP32 CUDA-core path
nv_status launch_encode_f32(const nv_ctx *c, const float *xyz, int64_t n, float *feat);
nv_status launch_hash_indices(const nv_ctx *c, const float *xyz, int64_t n, uint32_t *idx);
nv_status launch_mlp_f32(const nv_ctx *c, int mode, const MlpArgs &a);
// n_dev (nullable): the point count is *n_dev * n_mult, read on the device;
// n_upper bounds it for the grid size.  mode 3 = volume MSE accumulated into acc.
nv_status launch_mlp_f32_ext(const nv_ctx *c, int mode, const MlpArgs &a, const int *n_dev, int n_mult,
                             int64_t n_upper, double *acc);
// tcgen05 tensor-core path (FP16 / BF16)
nv_status launch_mlp_tc(const nv_ctx *c, int mode, const MlpArgs &a);
nv_status launch_mlp_tc_ext(const nv_ctx *c, int mode, const MlpArgs &a, const int *n_dev, int n_mult,
                            int64_t n_upper, double *acc);
bool tc_supported(const NetDesc &nd);
// optimizer
// Adam over all parameters; its last CTA counts the step (or halves the loss
// scale after an overflow) and publishes loss_acc * inv_n into loss_out.
nv_status launch_adam(nv_ctx *c, double inv_n, double *loss_out);
nv_status launch_coord_grad(const nv_ctx *c, const float *xyz, int64_t n, const float *df, float *dxyz);
nv_status build_adam_blocks(nv_ctx *c);
nv_status build_hot_replicas(nv_ctx *c);
nv_status launch_scale_double(double *x, double s, cudaStream_t st);
nv_status launch_shadow(nv_ctx *c);
// sampling, macrocells, rendering, reductions
nv_status launch_sample(const nv_volume &v, int64_t n, uint64_t seed, uint32_t step, float *xyz,
                        float *t, cudaStream_t s);
nv_status launch_macrocells(const nv_volume &v, int cell, const float *lut, float *minmax,
                            float *mu, cudaStream_t s);
// rows [row0, row0 + rows) of the camera's image into rgba [rows][width][4]
nv_status render_impl(nv_renderer *r, nv_ctx *net, const nv_volume *raw, const nv_camera &cam,
                      const float *lut, const nv_macrocells *mc, const nv_render_opts &o, int row0, int rows,
                      float *rgba);
// Online macrocells (k_render.cu): ranges reset to empty, widened by samples
// (xyz == NULL: the Philox training sample of (seed, step) with its target from
// vol), mu_max from the ranges.
nv_status launch_mc_reset(float *minmax, int nx, int ny, int nz, int cell, cudaStream_t s);
nv_status launch_mc_update(const float *xyz, const float *val, int64_t n, const nv_volume &vol, uint64_t seed,
                           uint32_t step, int nx, int ny, int nz, int cell, float *minmax, cudaStream_t s);
nv_status launch_mc_mu(const float *minmax, int nx, int ny, int nz, int cell, const float *lut, float *mu,
                       cudaStream_t s);
// Path tracing with sample streaming (k_pt.cu); mc supplies the majorants.
nv_status render_pt_impl(nv_renderer *r, nv_ctx *net, const nv_volume *raw, const nv_camera &cam, const float *lut,
                         const nv_macrocells &mc, const nv_pt_opts &o, float *rgba);
// In-shader ray march (k_inshader.cu); samples (nullable, device) counts the
// evaluated samples.
nv_status render_inshader(nv_ctx *c, const nv_camera &cam, const float *lut, const nv_macrocells *mc,
                          const nv_render_opts &o, float *rgba, unsigned long long *samples);
nv_status render_raw_sync_loop(const nv_renderer &r, const nv_volume &raw, const nv_camera &cam, const float *lut,
                               const nv_macrocells *mc, const nv_render_opts &o, float *rgba, cudaStream_t st);
nv_status launch_image_mse(const float *a, const float *b, int64_t n, double *out, cudaStream_t s);
nv_status launch_mse(const float *a, const float *b, int64_t n, double *out, cudaStream_t s);
nv_status launch_volume_mse(nv_ctx *c, const nv_volume &v, double *out);

/*
 * nv.h -- C ABI of the GB300 (sm_103a) neural-volume library.
 *
 * The library evaluates and trains a multi-resolution hash-encoded neural
 * volume (Sec. 3.1: L hash tables of T entries x F features, trilinear
 * interpolation per level, a small ReLU MLP without biases) and renders it
 * with an emission-absorption ray marcher that streams samples in batches
 * (Sec. 5.2.1), skips empty macrocells (Sec. 5.3) and stops rays at an
 * opacity threshold.
 *
 * Conventions shared by every entry point:
 *  - Every function returns an nv_status; NV_OK is 0.  On any other status a
 *    message is available from nv_last_error() (thread-local, valid until the
 *    next call on the same thread).  No C++ exception crosses this boundary.
 *    After NV_ERR_ARG nothing was launched and the context stays usable.
 *  - Pointers named *_dev are device pointers (cudaMalloc / PyTorch storage)
 *    owned by the caller.  Pointers named *_any may be host or device memory
 *    (the library copies with cudaMemcpyDefault).  The library never frees a
 *    caller pointer.
 *  - Work is enqueued asynchronously on a CUDA stream: the context's stream
 *    (nv_create / nv_set_stream) or the `stream` argument (NULL = the legacy
 *    default stream).  Only nv_sync, nv_get_params and the *_any copies to
 *    host memory synchronise.
 *  - Layouts:
 *      params  one flat float32 vector: tables [L][T][F] (T = 2^log2T),
 *              then the MLP weights W_0, W_1, ... with W_k stored
 *              [mlp_dims[k+1]][mlp_dims[k]] row-major (no biases)
 *      points  [n][3] float32, the normalised domain [0,1)^3 (Sec. 4)
 *      volume  [nz][ny][nx] float32, x fastest, cell-centred voxels,
 *              values normalised to [0,1]
 *      lut     [256][4] float32 RGBA transfer function
 *      image   [height][width][4] float32 RGBA
 */
#ifndef NV_H
#define NV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nv_ctx nv_ctx;           /* network: params, Adam state, scratch */
typedef struct nv_renderer nv_renderer; /* ray-streaming buffers of one image size */

typedef enum {
  NV_OK = 0,
  NV_ERR_ARG = 1,         /* bad argument; nothing launched */
  NV_ERR_OOM = 2,         /* device allocation failed */
  NV_ERR_CUDA = 3,        /* a CUDA call or launch failed */
  NV_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up (kernel returned early) */
  NV_ERR_STATE = 5,       /* call out of order (e.g. params never set) */
  NV_ERR_UNSUPPORTED = 6  /* shape or precision the library has no kernel for */
} nv_status;

typedef enum {
  NV_FP32 = 0, /* MLP on CUDA cores in FP32 (the parity path) */
  NV_FP16 = 1, /* MLP on tcgen05 tensor cores, FP16 operands, FP32 accumulate */
  NV_BF16 = 2  /* MLP on tcgen05 tensor cores, BF16 operands, FP32 accumulate */
} nv_prec;

typedef enum {
  NV_BUF_PARAMS = 0, /* FP32 master parameters */
  NV_BUF_GRADS = 1,  /* FP32 gradient accumulator (zeroed by each optimizer step) */
  NV_BUF_ADAM_M = 2, /* Adam first moment */
  NV_BUF_ADAM_V = 3  /* Adam second moment */
} nv_buffer;

typedef struct {
  const float *data_dev; /* [nz][ny][nx] */
  int nx, ny, nz;
} nv_volume;

typedef struct {
  float eye[3], target[3], up[3];
  float tan_half_fovy;   /* tan(vertical fov / 2) > 0: perspective; 0: orthographic */
  float ortho_w, ortho_h;/* orthographic extent (world units) */
  int width, height;
} nv_camera;

typedef struct {
  float step;      /* sample spacing along a ray, unit-box units (0.5 voxel = 0.5 / n) */
  float alpha_exp; /* opacity correction exponent step / s1 (Sec. 5.3): a' = 1 - (1 - a)^e */
  float et;        /* early termination once accumulated opacity >= et (e.g. 0.99) */
  int K;           /* samples streamed per live ray per iteration (Sec. 5.2.1; ~8) */
  float step_max;  /* > 0: adaptive step (Sec. 5.3, Eq. 3) between `step` (s1) and step_max (s2), p = 2;
                      needs macrocells; 0: fixed step */
  int shade;       /* 0: emission-absorption; 1: single-shot heuristic shadows (Sec. 5) */
  float light[3];  /* shade 1: unit direction towards the directional light */
  float ambient;   /* shade 1: colour scale where the light is fully blocked, in [0, 1] */
} nv_render_opts;

typedef struct {
  const float *mu_max_dev; /* [ceil(nz/cell)][ceil(ny/cell)][ceil(nx/cell)] */
  int cell;                /* macrocell edge in voxels */
  int nx, ny, nz;          /* volume dimensions the grid was built for */
} nv_macrocells;

/* Adam (Kingma & Ba; Sec. 3.1, App. B) with an exponentially decaying rate:
 * the optimizer step with 0-based index k (steps skipped after an FP16
 * overflow are not counted) uses lr * decay_base^d, d = 0 while k <
 * decay_start and d = floor((k - decay_start) / decay_interval) + 1 from then
 * on.  l2_reg * p is added to the gradient before the moments.  decay_base = 1
 * (or decay_interval <= 0) keeps the rate constant. */
typedef struct {
  float lr, beta1, beta2, eps, l2_reg;
  int decay_start, decay_interval;
  float decay_base;
} nv_adam_cfg;

/* Training loss (Sec. 3.1: L1 by default in the paper; L2 where Sec. 7 names it). */
typedef enum { NV_LOSS_L2 = 0, NV_LOSS_L1 = 1 } nv_loss;

/* ---- context ------------------------------------------------------------ */

/* Create a network (Sec. 3.1): L levels, F features per entry, T = 2^log2T
 * entries per level, level resolution N_l = floor(Nmin * b^l) (FP64 on the
 * host), MLP widths mlp_dims[0..n_dims-1] with mlp_dims[0] == L*F and
 * mlp_dims[n_dims-1] == 1 (ReLU hidden layers, sigmoid output, no biases).
 * prec selects the MLP arithmetic (nv_prec).  Parameters start at zero; Adam
 * defaults are lr 1e-2, beta (0.9, 0.999), eps 1e-15, l2 0, with the paper's
 * decay (start 2000, interval 1000, base 0.99); the loss defaults to L2.  Tensor-core
 * precisions need every hidden width == 64 and mlp_dims[0] in {16, 32, 64}.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).  The context
 * owns every buffer it allocates; nv_destroy frees them. */
nv_status nv_create(int L, int F, int log2T, int Nmin, double b, const int *mlp_dims, int n_dims,
                    int prec, void *cuda_stream, nv_ctx **out);
nv_status nv_destroy(nv_ctx *ctx);
nv_status nv_set_stream(nv_ctx *ctx, void *cuda_stream);
/* Sizes: n_params (tables + weights), n_table (L*T*F), and the L level resolutions. */
nv_status nv_info(const nv_ctx *ctx, int64_t *n_params, int64_t *n_table, int *level_res);

/* Copy all parameters in / out (params_any: [n_params] float32).  Setting also
 * refreshes the FP16/BF16 shadow copy used by the tensor-core kernels. */
nv_status nv_set_params(nv_ctx *ctx, const float *params_any);
nv_status nv_get_params(nv_ctx *ctx, float *params_any);
/* Device pointer and length of an internal FP32 buffer (nv_buffer); owned by the context.
 * Writes through the params pointer do not reach the FP16/BF16 shadow (Adam
 * rewrites the shadow only of the parameters it changes): set parameters with
 * nv_set_params.  Handing out NV_BUF_GRADS, NV_BUF_ADAM_M or NV_BUF_ADAM_V
 * makes every later optimizer step visit all parameters (nv_adam_span). */
nv_status nv_buffer_ptr(nv_ctx *ctx, int which, float **ptr_dev, int64_t *n);
/* Adam hyper-parameters (App. B lists beta 0.9 / 0.999, eps 1e-15). */
nv_status nv_set_adam(nv_ctx *ctx, const nv_adam_cfg *cfg);
/* Loss of nv_train_step (default NV_LOSS_L2): L2 = mean((y - t)^2) with
 * dL/dy = 2 (y - t) / n; L1 = mean(|y - t|) with dL/dy = sign(y - t) / n (0 at
 * y == t).  The loss nv_train_step reports follows the choice. */
nv_status nv_set_loss(nv_ctx *ctx, int loss);
/* Static loss scale S of the FP16/BF16 backward (default 128 / 1).  A step whose
 * gradient overflows is skipped and S halved, on the device. */
nv_status nv_set_loss_scale(nv_ctx *ctx, float scale);
/* Optimizer steps taken (skipped ones not counted) and the current loss scale;
 * synchronises the context stream. */
nv_status nv_get_step(nv_ctx *ctx, int *step, float *loss_scale);
/* Parameters the next optimizer step visits (*n_visit).  Adam (Kingma & Ba,
 * App. B settings) leaves a parameter with zero gradient and zero moments
 * unchanged when there is no L2 term, so it skips the 128-parameter blocks
 * that hold no weight and no hash slot a cell corner of a point in [0,1]^3 can
 * map to (on coarse levels most of them); the result equals the dense update
 * bit for bit.  It visits all n_params for good once an L2 term is used, a
 * gradient or moment buffer was handed out by nv_buffer_ptr, or a gradient was
 * scattered from a point outside [0,1]^3.  Synchronises the context stream. */
nv_status nv_adam_span(nv_ctx *ctx, int64_t *n_visit);

/* ---- network evaluation (Sec. 3.1) ---------------------------------------- */

/* A-2 debug output: the 8 corner hash indices of every point at every level,
 * idx_dev [n][L][8] uint32, corner d = dx + 2dy + 4dz of the cell
 * floor(fl32(x * N_l)); h = (x*1 ^ y*2654435761 ^ z*805459861) mod T. */
nv_status nv_hash_indices(nv_ctx *ctx, const float *xyz_dev, int64_t n, uint32_t *idx_dev);
/* A-1..A-3: the encoded feature vector of each point, feat_dev [n][L*F] float32,
 * level-major (feature j of level l at l*F + j), from the FP32 master tables. */
nv_status nv_encode(nv_ctx *ctx, const float *xyz_dev, int64_t n, float *feat_dev);
/* A-1..A-4: network value y = sigmoid(MLP(encode(x))) of each point, y_dev [n]. */
nv_status nv_infer(nv_ctx *ctx, const float *xyz_dev, int64_t n, float *y_dev);
/* A-6/A-7: backward of nv_infer for upstream gradients dL_dy_dev [n]: recomputes
 * the forward (nothing is stored between the calls) and ADDS the parameter
 * gradient into dparams_dev [n_params] (NULL: the context's NV_BUF_GRADS).
 * dxyz_dev (nullable): [n][3], WRITTEN with dL/dx of every point, the adjoint
 * of the trilinear weights of A-3 (within a cell of level l, d w_a / d x_a =
 * N_l) applied to dL/df, with the FP32 master tables; the context keeps an
 * [n][L*F] FP32 scratch for dL/df, grown on demand. */
nv_status nv_backward(nv_ctx *ctx, const float *xyz_dev, int64_t n, const float *dL_dy_dev,
                      float *dparams_dev, float *dxyz_dev);
/* A-8: one Adam step over every parameter (dense, up to the blocks that
 * nv_adam_span describes, which it would leave unchanged) from NV_BUF_GRADS,
 * which it zeroes; refreshes the FP16/BF16 shadow. */
nv_status nv_optimizer_step(nv_ctx *ctx);

/* ---- training (Sec. 4) ---------------------------------------------------- */

/* A-9: n training samples, x ~ U[0,1)^3 from Philox4x32-10 (counter (i lo,
 * i hi, step, 0), key (seed lo, seed hi), coordinate = (u >> 8) 2^-24) and the
 * target interpolated trilinearly from vol (q = x*n - 0.5, clamped).
 * xyz_dev [n][3] and target_dev [n] may be NULL to skip either output. */
nv_status nv_sample(const nv_volume *vol, int64_t n, uint64_t seed, uint32_t step, float *xyz_dev,
                    float *target_dev, void *stream);
/* One training step (Sec. 4): forward, the loss chosen by nv_set_loss
 * (default L2, mean((y - t)^2)), backward, Adam.  Either xyz_any/target_any hold the batch (host or device; a
 * host batch is copied on the context's own copy stream into one of two device staging slots, so the copy
 * overlaps the previous step's kernels; the host memory must stay unchanged until this step has completed,
 * e.g. until nv_sync) or both are NULL and the batch
 * is sampled from vol with nv_sample's generator at the context's sample
 * counter.  loss_dev (nullable): the batch loss before the update, FP64, in
 * device memory or in pinned host memory (the kernel that ends the step writes
 * it there over the host link, so a caller reading every step's loss needs no
 * copy on the stream; the value is there once the step has completed).  Other
 * host memory: NV_ERR_ARG. */
nv_status nv_train_step(nv_ctx *ctx, const float *xyz_any, const float *target_any, int64_t n,
                        const nv_volume *vol, uint64_t seed, double *loss_dev);

/* ---- data-parallel training (Sec. 4's training step split over replicas) ----- */

/* One training step of Sec. 4 split over R replicas of the same network (one
 * per GPU, same shape, parameters and optimizer state): replica r takes a
 * disjoint shard of the global batch of n_total points; each runs
 * nv_train_grad on its shard, the replicas reduce the buffers of
 * nv_dp_buffers (the gradient by sum, the flags by maximum), and each then
 * runs nv_optimizer_step: every replica applies the same update to the same
 * parameters.  Sums of the shards' gradients equal the one-replica gradient of
 * the whole batch up to FP32 summation order.
 *
 * nv_train_grad: forward, the loss chosen by nv_set_loss and backward of
 * nv_train_step on this replica's shard (xyz_dev [n][3], target_dev [n],
 * device memory; n may be 0), without the optimizer step: the gradient of the
 * GLOBAL mean loss (the per-point upstream gradient divided by n_total, not n)
 * is ADDED into NV_BUF_GRADS, and the shard's loss SUM (sum of (y - t)^2, or of
 * |y - t| for L1) is WRITTEN to loss_sum_dev (one device double).  Online
 * macrocells registered with the context are widened by the shard.
 * NV_ERR_ARG if n > n_total or a pointer is host memory. */
nv_status nv_train_grad(nv_ctx *ctx, const float *xyz_dev, const float *target_dev, int64_t n, int64_t n_total,
                        double *loss_sum_dev);
/* The device buffers a data-parallel step reduces across replicas, owned by
 * the context: grads_dev [n] = NV_BUF_GRADS (reduce by sum) and flags_dev [2]
 * int32 = (FP16 gradient overflow, a point outside [0,1]^3 was scattered)
 * (reduce by maximum; every replica then skips the step, or leaves the
 * reachable-block skipping, alike).  Unlike nv_buffer_ptr this keeps Adam's
 * reachable-block skipping (nv_adam_span): the replicas' gradients are zero
 * outside the reachable blocks, so their sum is.  Overwrite the buffers only
 * with such reductions, on the context's stream order, before
 * nv_optimizer_step. */
nv_status nv_dp_buffers(nv_ctx *ctx, float **grads_dev, int64_t *n, int32_t **flags_dev);

/* ---- out-of-core training samples (Sec. 4.1) ------------------------------- */

/* A-17: a device ring of R bricks fed from a volume held in pinned host memory
 * (Sec. 4.1, Fig. 2).  host_bricks: nbx*nby*nbz bricks (nb = n / brick per
 * axis, n a multiple of brick), brick b = (bz*nby + by)*nbx + bx at offset
 * b*(brick+2)^3 floats, each holding voxels brick*b - 1 .. brick*b + brick of
 * its axis range (indices clamped to the volume: the ghost layer), x fastest.
 * The memory stays owned by the caller and must outlive the ring.  Creation
 * fills every slot (the warm-up) and waits; the ring owns a copy stream.
 * Brick choices: splitmix64 of (seed, refresh count, slot) modulo the brick
 * count. */
typedef struct nv_ooc nv_ooc;
nv_status nv_ooc_create(const float *host_bricks, int nx, int ny, int nz, int brick, int ring_slots,
                        uint64_t seed, nv_ooc **out);
nv_status nv_ooc_destroy(nv_ooc *ooc);
/* Replace `count` slots (round robin) with freshly chosen bricks: a gather
 * kernel on the ring's own high-priority stream reads them from the pinned
 * host bricks over the host link.  It starts after the work already enqueued
 * on `stream` (so call it right after the nv_ooc_sample that last reads the
 * ring) and the next nv_ooc_sample waits for it; the training work enqueued in
 * between overlaps the copies. */
nv_status nv_ooc_refresh(nv_ooc *ooc, int count, uint64_t seed, void *stream);
/* n training samples from the resident bricks on `stream`: slot = u0 mod R,
 * voxel = the low three bytes of u1 mod brick, jitter (u >> 8) 2^-24 - 1/2 from
 * u2, u3 and the next draw's u0 (Philox4x32-10, counters (i lo, i hi, step, 1)
 * and (.., 2), key seed); position (v + 1/2 + jitter) / n; target trilinear
 * inside the brick.  xyz_dev [n][3] and target_dev [n] may each be NULL. */
nv_status nv_ooc_sample(nv_ooc *ooc, int64_t n, uint64_t seed, uint32_t step, float *xyz_dev,
                        float *target_dev, void *stream);
/* The brick held by each slot as of the last refresh (host array [R]). */
nv_status nv_ooc_slots(nv_ooc *ooc, int *slot_brick);
/* Bytes copied by refreshes since creation and the copy stream's busy time
 * for them (synchronises the copy stream). */
nv_status nv_ooc_stats(nv_ooc *ooc, int64_t *bytes_copied, double *copy_ms);

/* ---- rendering (Sec. 5) --------------------------------------------------- */

/* A-10: macrocells of `cell` voxels (Sec. 5.3).  minmax_dev [nc][2] holds the
 * value range of the voxels a trilinear lookup inside the cell can read
 * (cell*c - 1 .. cell*c + cell, clamped); mu_max_dev [nc] the largest LUT
 * alpha over entries floor(255 min) .. ceil(255 max).  Either may be NULL. */
nv_status nv_macrocells_build(const nv_volume *vol, int cell, const float *lut_dev,
                              float *minmax_dev, float *mu_max_dev, void *stream);

/* Online macrocells (Sec. 5.3): instead of a pass over the voxels, the value
 * ranges grow from the training samples, so the renderer needs no
 * precomputation over raw data.  minmax_dev [nc][2] (nc = the grid of `cell`
 * voxels over nx*ny*nz, x fastest) as nv_macrocells_build; a sample at unit
 * position x widens the range of the cell floor(fl32(x * fl32(n / cell))) per
 * axis, clamped -- the cell the ray march looks up at that position.
 * reset: every range empty (+inf, -inf).  update: n samples xyz_dev [n][3]
 * with values val_dev [n] (NaN values are ignored).  mu: mu_max_dev [nc] as
 * nv_macrocells_build from the ranges (an empty range gives 0, so cells no
 * sample reached are skipped).  All asynchronous on `stream`. */
nv_status nv_macrocells_reset(float *minmax_dev, int nx, int ny, int nz, int cell, void *stream);
nv_status nv_macrocells_update(const float *xyz_dev, const float *val_dev, int64_t n, int nx, int ny, int nz,
                               int cell, float *minmax_dev, void *stream);
nv_status nv_macrocells_mu(const float *minmax_dev, int nx, int ny, int nz, int cell, const float *lut_dev,
                           float *mu_max_dev, void *stream);
/* Register minmax_dev (NULL = off) so that every later nv_train_step widens it
 * with its batch (given or sampled) on the context stream.  The caller owns
 * the array and keeps it alive while it is registered. */
nv_status nv_set_online_macrocells(nv_ctx *ctx, float *minmax_dev, int nx, int ny, int nz, int cell);

/* A renderer owns the structure-of-arrays ray state for images of up to
 * max_pixels pixels and K samples per ray per iteration. */
nv_status nv_renderer_create(int64_t max_pixels, int K, void *cuda_stream, nv_renderer **out);
nv_status nv_renderer_destroy(nv_renderer *r);

/* A-11..A-15: sample-streaming ray march (Sec. 5.2.1).  Ray generation and
 * box clipping, then per iteration: the next K sample positions of every live
 * ray (t_k = t0 + (k + 1/2) step, skipping samples whose macrocell has
 * mu_max == 0), their values -- from the network `net` (FP32 or tensor-core
 * inference) or, when net is NULL, from the raw volume `raw` by trilinear
 * interpolation -- then front-to-back compositing with opacity correction
 * and early termination, and compaction of the live rays.  mc may be NULL (no
 * skipping).  rgba_dev [height][width][4]; rays that miss are black.
 * opts->step_max > 0 selects the adaptive step (Sec. 5.3, Eq. 3; needs mc):
 * each segment takes s_bar = max(s1 + (s2 - s1) (1 - min(mu, 1))^2, s1) from
 * the macrocell it starts in, ends at that cell's face, t1 or s_bar, samples
 * its midpoint and corrects the opacity by its own length; transparent cells
 * are crossed without samples.  opts->shade == 1 adds single-shot heuristic
 * shadows (Sec. 5): the ray remembers its sample of largest contribution
 * (1 - A) a' and, when its march ends, marches on from that point towards the
 * light (clipped to the volume box, same sampling rules, opacity only); the
 * colour becomes C (ambient + (1 - ambient) T) with T that march's
 * transmittance, A is kept.  A ray with no contribution casts no shadow ray. */
nv_status nv_render(nv_renderer *r, nv_ctx *net, const nv_volume *raw, const nv_camera *cam,
                    const float *lut_dev, const nv_macrocells *mc, const nv_render_opts *opts,
                    float *rgba_dev);
/* Image-tile split of nv_render (Sec. 5.2.1: each pixel's ray is marched and
 * composited on its own, so a frame partitions by pixels with no exchange
 * between the parts): rows [row0, row0 + rows) of the
 * camera's image, each pixel's value equal to nv_render's, into rgba_dev
 * [rows][width][4] (band-local).  0 <= row0, rows >= 1, row0 + rows <= height
 * and width * rows <= the renderer's max_pixels, else NV_ERR_ARG.  Other
 * arguments and errors as nv_render; nv_render_stats reports the band. */
nv_status nv_render_rows(nv_renderer *r, nv_ctx *net, const nv_volume *raw, const nv_camera *cam,
                         const float *lut_dev, const nv_macrocells *mc, const nv_render_opts *opts, int row0,
                         int rows, float *rgba_dev);
/* In-shader inference (Sec. 5.1, App. A): the same ray march as nv_render on
 * the network `net`, as one kernel in which each thread owns a ray and the
 * network is evaluated inside the march -- a CTA of 128 rays (a 16 x 8 pixel
 * tile) gathers one sample per live ray into a tensor-core tile per iteration
 * and runs until its last ray finishes.  Samples, network arithmetic and
 * compositing are those of nv_render, so both give the same image; opts->K is
 * ignored.  The fixed step only (opts->step_max > 0: NV_ERR_UNSUPPORTED);
 * opts->shade == 1 adds nv_render's single-shot shadows, the shadow march run
 * by the same thread after its ray's primary march.  Needs an FP16 or BF16
 * network of a tensor-core shape (NV_ERR_UNSUPPORTED otherwise).  samples_dev
 * (nullable): one int64 on the device, set to the number of evaluated samples
 * (primary and shadow).  Asynchronous on the network's stream. */
nv_status nv_render_inshader(nv_ctx *net, const nv_camera *cam, const float *lut_dev, const nv_macrocells *mc,
                             const nv_render_opts *opts, float *rgba_dev, int64_t *samples_dev);
/* Volumetric path tracing with sample streaming (Sec. 5.2.2, Alg. 1, Eq. 1-2):
 * one path per pixel and call.  Extinction sigma(x) = density * LUT opacity
 * per unit length, single-scattering albedo = LUT colour, isotropic phase, a
 * directional light towards `light` (its irradiance cancels the phase
 * factor), black background.  Free flights are Woodcock tracking against the
 * majorant density * mu_max of each macrocell of `mc` (required), walked
 * cell by cell (Hofmann): tau = -log(1 - zeta) is spent along the ray and
 * the tentative collision accepted with probability sigma / majorant.  Every
 * real collision sends a shadow ray towards the light, tracked the same way
 * (the light counts when it leaves the volume unblocked), then throughput *=
 * albedo, Russian roulette from the third bounce and an isotropic direction;
 * a path ends on leaving the volume or after max_bounces real collisions.
 * Random numbers: Philox4x32-10, key = seed, counter = (pixel, event, frame,
 * 0); per frame the caller averages the images.  rgba_dev: RGB radiance and
 * A = 1 where the camera ray's path had a real collision.  Network values
 * come from `net` (NULL: the raw volume `raw`). */
typedef struct {
  float density;    /* D: extinction per unit length at LUT opacity 1 */
  float light[3];   /* unit direction towards the directional light */
  int max_bounces;  /* real collisions per path, >= 1 */
  uint64_t seed;
  uint32_t frame;
} nv_pt_opts;
nv_status nv_render_pt(nv_renderer *r, nv_ctx *net, const nv_volume *raw, const nv_camera *cam,
                       const float *lut_dev, const nv_macrocells *mc, const nv_pt_opts *opts, float *rgba_dev);
/* Iterations and samples of the last nv_render (synchronises). */
nv_status nv_render_stats(nv_renderer *r, int *iterations, int64_t *samples);

/* The paper has no counterpart to this entry point.  It is nv_render on the
 * raw volume (net = NULL) for callers that cannot allocate device memory:
 * real-time loops whose memory is fixed up front (cudaMalloc and cudaFree may
 * synchronise the device and take unbounded time, which a frame deadline
 * cannot absorb), and plugins inside a host application that owns every
 * allocation and budgets the GPU's memory itself.  It calls no cudaMalloc,
 * cudaFree, cudaMallocHost, event or stream creation; ray buffers, sample
 * batches and counters come from one static device array of
 * NV_NOALLOC_SCRATCH_BYTES (about 16 MB) that every GPU loading the library
 * holds until the process exits.
 *  - Images up to NV_NOALLOC_MAX_PIXELS pixels (256 x 256) and K up to
 *    NV_NOALLOC_MAX_K; larger requests fail with NV_ERR_ARG and a message.
 *  - Only the fixed-step emission-absorption march: opts->step_max > 0
 *    (adaptive step) or opts->shade != 0 (shadows) fail with
 *    NV_ERR_UNSUPPORTED before anything is enqueued.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - Every call shares the array and it keeps the last call's contents; each
 *    call clears the counters that must start at zero.  Calls whose GPU work
 *    overlaps (other streams, other host threads) race on the same scratch.
 *  - The live-ray count is read back synchronously after every iteration, so
 *    the call returns when the image is complete.
 * Other arguments as nv_render; mc may be NULL; stream NULL = legacy default stream. */
#define NV_NOALLOC_MAX_PIXELS 65536
#define NV_NOALLOC_MAX_K 8
#define NV_NOALLOC_SCRATCH_BYTES 15991296
nv_status nv_render_raw_noalloc(const nv_volume *raw, const nv_camera *cam, const float *lut_dev,
                                const nv_macrocells *mc, const nv_render_opts *opts, float *rgba_dev,
                                void *stream);

/* ---- measurement (the paper has no counterpart) ---------------------------- */

/* Reference rates for the rooflines of the scatter and the gather: `ops`
 * (rounded up to a multiple of 8192) scattered 16-byte accesses to slots of a
 * buffer of n16 16-byte slots (a power of two <= 2^32), each slot chosen by a
 * 32-bit integer mixer of (thread, access, seed).  nv_peak_scatter adds
 * (1, 1, 1, 1) to each chosen slot with an FP32 vector reduction (buf_dev:
 * n16 x 4 floats, updated); nv_peak_gather loads each chosen slot (buf_dev:
 * n16 x 16 bytes, read only; sink_dev: 1024 uint32 the kernel may write so the
 * loads are kept).  Asynchronous on `stream`; time them with events. */
nv_status nv_peak_scatter(float *buf_dev, int64_t n16, int64_t ops, uint64_t seed, void *stream);
nv_status nv_peak_gather(const void *buf_dev, int64_t n16, int64_t ops, uint64_t seed, void *sink_dev,
                         void *stream);

/* ---- quality (Sec. 7) ------------------------------------------------------ */

/* A-16: FP64 mean squared error over the RGB channels of two images,
 * mse_dev (one double on the device). */
nv_status nv_image_mse(const float *rgba_a_dev, const float *rgba_b_dev, int64_t n_pixels,
                       double *mse_dev, void *stream);
/* A-16: FP64 mean squared error of two float arrays of n values (e.g. decoded
 * and raw values at the same points), mse_dev (one double on the device). */
nv_status nv_mse_f64(const float *a_dev, const float *b_dev, int64_t n, double *mse_dev, void *stream);
/* A-16: decode the network at every voxel centre (i + 1/2) / n and the FP64 MSE
 * against vol, mse_dev (one double on the device).  No decoded grid is stored. */
nv_status nv_volume_mse(nv_ctx *ctx, const nv_volume *vol, double *mse_dev);

/* ---- misc ------------------------------------------------------------------ */

/* Kernel timing for benchmarks: while enabled, every kernel the context
 * launches is bracketed by CUDA events on the context stream, grouped by
 * class (nv_kclass).  nv_profile_read synchronises, returns the summed device
 * time and launch count of one class since the last read, and clears that
 * class.  Up to 8192 launches are kept; later ones are not recorded. */
typedef enum {
  NV_K_MLP = 0,     /* the MLP kernel (FP32 path: the whole fused encode + MLP + scatter kernel) */
  NV_K_ADAM = 1,
  NV_K_FINISH = 2,  /* no launches: the step's book-keeping runs in the last CTA of Adam */
  NV_K_RENDER = 3,
  NV_K_OTHER = 4,
  NV_K_ENCODE = 5,  /* tensor-core path: hash gather into feature tiles */
  NV_K_SCATTER = 6  /* tensor-core training: the fold of the coarsest levels' gradient replicas into the hashed
                      slots (the scatter itself runs inside the MLP kernel) */
} nv_kclass;
nv_status nv_profile_enable(nv_ctx *ctx, int enable);
nv_status nv_profile_read(nv_ctx *ctx, int kclass, double *total_ms, int *launches);

/* Wait for the context stream; reports NV_ERR_TIMEOUT if a kernel gave up a wait. */
nv_status nv_sync(nv_ctx *ctx);
const char *nv_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* NV_H */

// nv_api.cu -- the C ABI of include/nv.h: argument checks, context and renderer
// lifetime, and the order of kernel launches for each call.  No arithmetic of
// the method happens here except the level resolutions N_l = floor(Nmin b^l),
// computed once in FP64 at creation.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "nv_internal.cuh"

static thread_local char g_err[512] = "";

nv_status nv_fail(nv_status s, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

nv_status nv_cuda_check(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return NV_OK;
  snprintf(g_err, sizeof(g_err), "%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? NV_ERR_OOM : NV_ERR_CUDA;
}

extern "C" const char *nv_last_error(void) { return g_err; }

static bool is_host_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.type == cudaMemoryTypeUnregistered || at.type == cudaMemoryTypeHost;
}

// The address a kernel writes a result to: device memory as given, pinned
// host memory through its device alias (the kernel writes it over the host
// link, with no copy on the stream).  Pageable host memory is refused: no
// kernel may write it.
static nv_status kernel_out_ptr(double *p, double **out, const char *fn) {
  *out = nullptr;
  if (!p) return NV_OK;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nv_fail(NV_ERR_ARG, "%s: loss_dev is neither device nor pinned host memory", fn);
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
    *out = p;
    return NV_OK;
  }
  if (at.type == cudaMemoryTypeHost && at.devicePointer) {
    *out = static_cast<double *>(at.devicePointer);
    return NV_OK;
  }
  return nv_fail(NV_ERR_ARG, "%s: loss_dev is neither device nor pinned host memory", fn);
}

struct Prof {
  static const int kMax = 8192;
  std::vector<cudaEvent_t> ev;   // 2 per recorded launch
  std::vector<int> cls;          // class of each recorded launch
  int used = 0;
  bool on = false;
};

int prof_begin(nv_ctx *c) {
  Prof *p = c->prof;
  if (!p || !p->on || p->used >= Prof::kMax) return -1;
  int i = p->used++;
  cudaEventRecord(p->ev[2 * i], c->stream);
  return i;
}

void prof_end(nv_ctx *c, int kclass, int token) {
  if (token < 0) return;
  Prof *p = c->prof;
  p->cls[token] = kclass;
  cudaEventRecord(p->ev[2 * token + 1], c->stream);
}

static void prof_free(Prof *p) {
  if (!p) return;
  for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
  delete p;
}

static void ctx_free(nv_ctx *c) {
  if (!c) return;
  prof_free(c->prof);
  cudaFree(c->params);
  cudaFree(c->grads);
  cudaFree(c->adam_m);
  cudaFree(c->adam_v);
  cudaFree(c->shadow);
  cudaFree(c->ds);
  cudaFree(c->batch[0]);
  cudaFree(c->batch[1]);
  for (int b = 0; b < 2; ++b) {
    if (c->batch_copied[b]) cudaEventDestroy(c->batch_copied[b]);
    if (c->batch_used[b]) cudaEventDestroy(c->batch_used[b]);
  }
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  cudaFree(c->tc_feat);
  cudaFree(c->tc_tgt);
  cudaFree(c->tc_xyz);
  cudaFree(c->adam_blocks);
  cudaFree(c->df_buf);
  cudaFree(c->hot.buf);
  delete c;
}

extern "C" nv_status nv_create(int L, int F, int log2T, int Nmin, double b, const int *mlp_dims, int n_dims,
                               int prec, void *cuda_stream, nv_ctx **out) {
  if (!out) return nv_fail(NV_ERR_ARG, "nv_create: out is NULL");
  *out = nullptr;
  if (L < 1 || L > NV_MAX_LEVELS) return nv_fail(NV_ERR_ARG, "nv_create: L=%d not in [1, %d]", L, NV_MAX_LEVELS);
  if (F != 1 && F != 2 && F != 4 && F != 8) return nv_fail(NV_ERR_ARG, "nv_create: F=%d not in {1,2,4,8}", F);
  if (log2T < 1 || log2T > 28) return nv_fail(NV_ERR_ARG, "nv_create: log2T=%d not in [1, 28]", log2T);
  if (Nmin < 1 || !(b >= 1.0) || !std::isfinite(b)) return nv_fail(NV_ERR_ARG, "nv_create: Nmin=%d b=%g", Nmin, b);
  if (!mlp_dims || n_dims < 2 || n_dims > NV_MAX_LAYERS + 1)
    return nv_fail(NV_ERR_ARG, "nv_create: n_dims=%d not in [2, %d]", n_dims, NV_MAX_LAYERS + 1);
  if (mlp_dims[0] != L * F) return nv_fail(NV_ERR_ARG, "nv_create: mlp_dims[0]=%d != L*F=%d", mlp_dims[0], L * F);
  if (mlp_dims[n_dims - 1] != 1) return nv_fail(NV_ERR_ARG, "nv_create: the output width must be 1");
  for (int k = 1; k + 1 < n_dims; ++k)
    if (mlp_dims[k] < 1 || mlp_dims[k] > 256) return nv_fail(NV_ERR_ARG, "nv_create: hidden width %d", mlp_dims[k]);
  if (prec != NV_FP32 && prec != NV_FP16 && prec != NV_BF16) return nv_fail(NV_ERR_ARG, "nv_create: prec=%d", prec);

  nv_ctx *c = new (std::nothrow) nv_ctx();
  if (!c) return nv_fail(NV_ERR_OOM, "nv_create: host allocation");
  NetDesc &nd = c->nd;
  nd.L = L;
  nd.F = F;
  nd.log2T = log2T;
  nd.T = 1u << log2T;
  for (int l = 0; l < L; ++l) {
    double r = std::floor((double)Nmin * std::pow(b, (double)l));
    if (!(r < 1073741824.0)) {
      delete c;
      return nv_fail(NV_ERR_ARG, "nv_create: level %d resolution %g too large", l, r);
    }
    nd.res[l] = (int)r;
  }
  nd.n_dims = n_dims;
  for (int k = 0; k < n_dims; ++k) nd.dims[k] = mlp_dims[k];
  nd.n_table = (int64_t)L * nd.T * F;
  int64_t off = 0;
  for (int k = 0; k + 1 < n_dims; ++k) {
    nd.w_off[k] = off;
    off += (int64_t)mlp_dims[k] * mlp_dims[k + 1];
  }
  nd.n_weights = off;
  c->Nmin = Nmin;
  c->b = b;
  c->prec = prec;
  c->stream = (cudaStream_t)cuda_stream;
  c->n_params = nd.n_table + nd.n_weights;
  c->adam = nv_adam_cfg{1e-2f, 0.9f, 0.999f, 1e-15f, 0.0f, 2000, 1000, 0.99f};
  c->loss_kind = NV_LOSS_L2;
  if (prec != NV_FP32 && !tc_supported(nd)) {
    delete c;
    return nv_fail(NV_ERR_UNSUPPORTED,
                   "nv_create: tensor-core MLP needs hidden widths of 64, two hidden layers and L*F in {16,32,64}");
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    delete c;
    return nv_cuda_check(e, "nv_create: device query");
  }
  const size_t pb = (size_t)c->n_params * sizeof(float);
  e = cudaMalloc(&c->params, pb);
  if (e == cudaSuccess) e = cudaMalloc(&c->grads, pb);
  if (e == cudaSuccess) e = cudaMalloc(&c->adam_m, pb);
  if (e == cudaSuccess) e = cudaMalloc(&c->adam_v, pb);
  if (e == cudaSuccess && prec != NV_FP32) e = cudaMalloc(&c->shadow, (size_t)c->n_params * 2 + 16);
  if (e == cudaSuccess) e = cudaMalloc(&c->ds, sizeof(DevState));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->params, 0, pb, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->grads, 0, pb, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->adam_m, 0, pb, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->adam_v, 0, pb, c->stream);
  if (e == cudaSuccess && c->shadow) e = cudaMemsetAsync(c->shadow, 0, (size_t)c->n_params * 2 + 16, c->stream);
  DevState init{};
  init.loss_scale = prec == NV_FP16 ? 128.0f : 1.0f;
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->ds, &init, sizeof(init), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    nv_status s = nv_cuda_check(e, "nv_create: allocation");
    ctx_free(c);
    return s;
  }
  nv_status sb = build_adam_blocks(c);
  if (sb == NV_OK) sb = build_hot_replicas(c);
  if (sb != NV_OK) {
    ctx_free(c);
    return sb;
  }
  *out = c;
  return NV_OK;
}

extern "C" nv_status nv_destroy(nv_ctx *c) {
  if (!c) return NV_OK;
  if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
  cudaStreamSynchronize(c->stream);
  ctx_free(c);
  return NV_OK;
}

extern "C" nv_status nv_set_stream(nv_ctx *c, void *s) {
  if (!c) return nv_fail(NV_ERR_ARG, "nv_set_stream: ctx is NULL");
  c->stream = (cudaStream_t)s;
  return NV_OK;
}

extern "C" nv_status nv_info(const nv_ctx *c, int64_t *n_params, int64_t *n_table, int *level_res) {
  if (!c) return nv_fail(NV_ERR_ARG, "nv_info: ctx is NULL");
  if (n_params) *n_params = c->n_params;
  if (n_table) *n_table = c->nd.n_table;
  if (level_res)
    for (int l = 0; l < c->nd.L; ++l) level_res[l] = c->nd.res[l];
  return NV_OK;
}

extern "C" nv_status nv_set_params(nv_ctx *c, const float *src) {
  if (!c || !src) return nv_fail(NV_ERR_ARG, "nv_set_params: NULL argument");
  NV_CUDA(cudaMemcpyAsync(c->params, src, (size_t)c->n_params * sizeof(float), cudaMemcpyDefault, c->stream),
          "nv_set_params: copy");
  NV_TRY(launch_shadow(c));
  c->params_set = 1;
  return nv_cuda_check(cudaStreamSynchronize(c->stream), "nv_set_params: sync");
}

extern "C" nv_status nv_get_params(nv_ctx *c, float *dst) {
  if (!c || !dst) return nv_fail(NV_ERR_ARG, "nv_get_params: NULL argument");
  NV_CUDA(cudaMemcpyAsync(dst, c->params, (size_t)c->n_params * sizeof(float), cudaMemcpyDefault, c->stream),
          "nv_get_params: copy");
  return nv_cuda_check(cudaStreamSynchronize(c->stream), "nv_get_params: sync");
}

extern "C" nv_status nv_buffer_ptr(nv_ctx *c, int which, float **ptr, int64_t *n) {
  if (!c || !ptr) return nv_fail(NV_ERR_ARG, "nv_buffer_ptr: NULL argument");
  switch (which) {
    case NV_BUF_PARAMS: *ptr = c->params; break;
    case NV_BUF_GRADS: *ptr = c->grads; break;
    case NV_BUF_ADAM_M: *ptr = c->adam_m; break;
    case NV_BUF_ADAM_V: *ptr = c->adam_v; break;
    default: return nv_fail(NV_ERR_ARG, "nv_buffer_ptr: unknown buffer %d", which);
  }
  // whoever holds the gradient or a moment may write any slot: Adam visits all from now on
  if (which != NV_BUF_PARAMS) c->adam_dense = 1;
  if (n) *n = c->n_params;
  return NV_OK;
}

extern "C" nv_status nv_set_adam(nv_ctx *c, const nv_adam_cfg *cfg) {
  if (!c || !cfg) return nv_fail(NV_ERR_ARG, "nv_set_adam: NULL argument");
  if (!(cfg->lr >= 0.f) || !(cfg->beta1 >= 0.f && cfg->beta1 < 1.f) || !(cfg->beta2 >= 0.f && cfg->beta2 < 1.f) ||
      !(cfg->eps >= 0.f) || !(cfg->l2_reg >= 0.f) || !(cfg->decay_base > 0.f && cfg->decay_base <= 1.f) ||
      cfg->decay_start < 0)
    return nv_fail(NV_ERR_ARG, "nv_set_adam: hyper-parameters out of range");
  c->adam = *cfg;
  return NV_OK;
}

extern "C" nv_status nv_set_loss(nv_ctx *c, int loss) {
  if (!c) return nv_fail(NV_ERR_ARG, "nv_set_loss: ctx is NULL");
  if (loss != NV_LOSS_L2 && loss != NV_LOSS_L1) return nv_fail(NV_ERR_ARG, "nv_set_loss: unknown loss %d", loss);
  c->loss_kind = loss;
  return NV_OK;
}

extern "C" nv_status nv_set_loss_scale(nv_ctx *c, float scale) {
  if (!c || !(scale > 0.f) || !std::isfinite(scale)) return nv_fail(NV_ERR_ARG, "nv_set_loss_scale: bad scale");
  NV_CUDA(cudaStreamSynchronize(c->stream), "nv_set_loss_scale: sync");
  NV_CUDA(cudaMemcpy(&c->ds->loss_scale, &scale, sizeof(float), cudaMemcpyHostToDevice), "nv_set_loss_scale");
  return NV_OK;
}

extern "C" nv_status nv_adam_span(nv_ctx *c, int64_t *n_visit) {
  if (!c || !n_visit) return nv_fail(NV_ERR_ARG, "nv_adam_span: NULL argument");
  int off = 0;
  NV_CUDA(cudaStreamSynchronize(c->stream), "nv_adam_span: sync");
  NV_CUDA(cudaMemcpy(&off, &c->ds->off_domain, sizeof(int), cudaMemcpyDeviceToHost), "nv_adam_span: copy");
  if (!c->adam_blocks || c->adam_dense || off || c->adam.l2_reg != 0.f) {
    *n_visit = c->n_params;
  } else {  // the blocks visited, the last one clipped to the vectorised part, plus the scalar tail
    const int64_t n4 = c->n_params >> 2;
    int32_t last = 0;
    NV_CUDA(cudaMemcpy(&last, c->adam_blocks + c->adam_nblocks - 1, sizeof(int32_t), cudaMemcpyDeviceToHost),
            "nv_adam_span: copy");
    int64_t v = c->adam_nblocks * 128;
    if ((int64_t)last * 32 + 32 > n4) v -= ((int64_t)last * 32 + 32 - n4) * 4;
    *n_visit = v + (c->n_params - 4 * n4);
  }
  return NV_OK;
}

extern "C" nv_status nv_get_step(nv_ctx *c, int *step, float *loss_scale) {
  if (!c) return nv_fail(NV_ERR_ARG, "nv_get_step: ctx is NULL");
  DevState h;
  NV_CUDA(cudaStreamSynchronize(c->stream), "nv_get_step: sync");
  NV_CUDA(cudaMemcpy(&h, c->ds, sizeof(h), cudaMemcpyDeviceToHost), "nv_get_step: copy");
  if (step) *step = h.step;
  if (loss_scale) *loss_scale = h.loss_scale;
  return NV_OK;
}

static nv_status check_points(const nv_ctx *c, const void *xyz, int64_t n, const char *fn) {
  if (!c) return nv_fail(NV_ERR_ARG, "%s: ctx is NULL", fn);
  if (n < 0) return nv_fail(NV_ERR_ARG, "%s: n=%lld < 0", fn, (long long)n);
  if (n > 0 && !xyz) return nv_fail(NV_ERR_ARG, "%s: xyz is NULL", fn);
  return NV_OK;
}

extern "C" nv_status nv_hash_indices(nv_ctx *c, const float *xyz, int64_t n, uint32_t *idx) {
  NV_TRY(check_points(c, xyz, n, "nv_hash_indices"));
  if (n > 0 && !idx) return nv_fail(NV_ERR_ARG, "nv_hash_indices: idx is NULL");
  return launch_hash_indices(c, xyz, n, idx);
}

extern "C" nv_status nv_encode(nv_ctx *c, const float *xyz, int64_t n, float *feat) {
  NV_TRY(check_points(c, xyz, n, "nv_encode"));
  if (n > 0 && !feat) return nv_fail(NV_ERR_ARG, "nv_encode: feat is NULL");
  return launch_encode_f32(c, xyz, n, feat);
}

extern "C" nv_status nv_infer(nv_ctx *c, const float *xyz, int64_t n, float *y) {
  NV_TRY(check_points(c, xyz, n, "nv_infer"));
  if (n > 0 && !y) return nv_fail(NV_ERR_ARG, "nv_infer: y is NULL");
  if (n == 0) return NV_OK;
  MlpArgs a{};
  a.xyz = xyz;
  a.n = n;
  a.y = y;
  a.ds = c->ds;
  if (c->prec != NV_FP32) return launch_mlp_tc(c, MODE_INFER, a);  // times its kernels itself
  int tk = prof_begin(c);
  nv_status s = launch_mlp_f32(c, MODE_INFER, a);
  prof_end(c, NV_K_MLP, tk);
  return s;
}

extern "C" nv_status nv_backward(nv_ctx *c, const float *xyz, int64_t n, const float *dy, float *dparams,
                                 float *dxyz) {
  NV_TRY(check_points(c, xyz, n, "nv_backward"));
  if (n > 0 && !dy) return nv_fail(NV_ERR_ARG, "nv_backward: dL_dy is NULL");
  if (n == 0) return NV_OK;
  MlpArgs a{};
  a.xyz = xyz;
  a.in = dy;
  a.n = n;
  a.grads = dparams ? dparams : c->grads;
  a.ds = c->ds;
  if (dxyz) {  // dL/df of every point is kept for the coordinate gradient
    const int64_t need = n * c->nd.dims[0];
    if (c->df_cap < need) {
      cudaFree(c->df_buf);
      c->df_buf = nullptr;
      c->df_cap = 0;
      NV_CUDA(cudaMalloc(&c->df_buf, (size_t)need * sizeof(float)), "nv_backward: dL/df scratch");
      c->df_cap = need;
    }
    a.df_out = c->df_buf;
  }
  if (c->prec != NV_FP32) {
    NV_TRY(launch_mlp_tc(c, MODE_BACKWARD, a));  // times its kernels itself
  } else {
    int tk = prof_begin(c);
    nv_status s = launch_mlp_f32(c, MODE_BACKWARD, a);
    prof_end(c, NV_K_MLP, tk);
    NV_TRY(s);
  }
  if (!dxyz) return NV_OK;
  int tk = prof_begin(c);
  nv_status s = launch_coord_grad(c, xyz, n, c->df_buf, dxyz);
  prof_end(c, NV_K_OTHER, tk);
  return s;
}

extern "C" nv_status nv_optimizer_step(nv_ctx *c) {
  if (!c) return nv_fail(NV_ERR_ARG, "nv_optimizer_step: ctx is NULL");
  int tk = prof_begin(c);
  NV_TRY(launch_adam(c, 0.0, nullptr));
  prof_end(c, NV_K_ADAM, tk);
  return NV_OK;
}

static nv_status check_volume(const nv_volume *v, const char *fn) {
  if (!v || !v->data_dev) return nv_fail(NV_ERR_ARG, "%s: volume is NULL", fn);
  if (v->nx < 1 || v->ny < 1 || v->nz < 1) return nv_fail(NV_ERR_ARG, "%s: volume dims %d %d %d", fn, v->nx, v->ny, v->nz);
  return NV_OK;
}

extern "C" nv_status nv_sample(const nv_volume *vol, int64_t n, uint64_t seed, uint32_t step, float *xyz,
                               float *target, void *stream) {
  NV_TRY(check_volume(vol, "nv_sample"));
  if (n < 0) return nv_fail(NV_ERR_ARG, "nv_sample: n < 0");
  return launch_sample(*vol, n, seed, step, xyz, target, (cudaStream_t)stream);
}

extern "C" nv_status nv_train_step(nv_ctx *c, const float *xyz, const float *target, int64_t n,
                                   const nv_volume *vol, uint64_t seed, double *loss_dev) {
  if (!c) return nv_fail(NV_ERR_ARG, "nv_train_step: ctx is NULL");
  if (n <= 0) return nv_fail(NV_ERR_ARG, "nv_train_step: n=%lld must be > 0", (long long)n);
  if ((xyz == nullptr) != (target == nullptr))
    return nv_fail(NV_ERR_ARG, "nv_train_step: give both xyz and target, or neither (sample from vol)");
  double *loss_k = nullptr;
  NV_TRY(kernel_out_ptr(loss_dev, &loss_k, "nv_train_step"));
  MlpArgs a{};
  a.n = n;
  a.grads = c->grads;
  a.ds = c->ds;
  a.inv_n = (float)(1.0 / (double)n);
  a.l1 = c->loss_kind == NV_LOSS_L1;
  int used_slot = -1;  // staging slot of a host batch
  if (xyz) {
    if (is_host_ptr(xyz) || is_host_ptr(target)) {
      // host batch: copied on a copy stream into one of two staging slots, so
      // this copy overlaps the previous step's kernels; the slot is reused only
      // after the step that read it has finished
      if (!c->copy_stream) {
        NV_CUDA(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking), "nv_train_step: copy stream");
        for (int b = 0; b < 2; ++b) {
          NV_CUDA(cudaEventCreateWithFlags(&c->batch_copied[b], cudaEventDisableTiming), "nv_train_step: event");
          NV_CUDA(cudaEventCreateWithFlags(&c->batch_used[b], cudaEventDisableTiming), "nv_train_step: event");
        }
      }
      if (c->batch_cap < n) {
        NV_CUDA(cudaStreamSynchronize(c->copy_stream), "nv_train_step: staging");
        NV_CUDA(cudaStreamSynchronize(c->stream), "nv_train_step: staging");
        for (int b = 0; b < 2; ++b) {
          cudaFree(c->batch[b]);
          c->batch[b] = nullptr;
        }
        c->batch_cap = 0;
        for (int b = 0; b < 2; ++b)
          NV_CUDA(cudaMalloc(&c->batch[b], (size_t)n * 4 * sizeof(float)), "nv_train_step: staging");
        c->batch_cap = n;
      }
      const int b = c->batch_slot;
      c->batch_slot ^= 1;
      float *bx = c->batch[b], *bt = c->batch[b] + 3 * n;
      NV_CUDA(cudaStreamWaitEvent(c->copy_stream, c->batch_used[b], 0), "nv_train_step: wait");
      NV_CUDA(cudaMemcpyAsync(bx, xyz, (size_t)n * 3 * sizeof(float), cudaMemcpyDefault, c->copy_stream), "H2D xyz");
      NV_CUDA(cudaMemcpyAsync(bt, target, (size_t)n * sizeof(float), cudaMemcpyDefault, c->copy_stream), "H2D target");
      NV_CUDA(cudaEventRecord(c->batch_copied[b], c->copy_stream), "nv_train_step: record");
      NV_CUDA(cudaStreamWaitEvent(c->stream, c->batch_copied[b], 0), "nv_train_step: wait");
      used_slot = b;
      a.xyz = bx;
      a.in = bt;
    } else {
      a.xyz = xyz;
      a.in = target;
    }
  } else {
    NV_TRY(check_volume(vol, "nv_train_step"));
    a.vol = *vol;
    a.seed = seed;
    a.sample_step = c->sample_counter++;
  }
  if (c->prec == NV_FP32) {
    int tk0 = prof_begin(c);
    NV_TRY(launch_mlp_f32(c, MODE_TRAIN, a));
    prof_end(c, NV_K_MLP, tk0);
  } else {
    NV_TRY(launch_mlp_tc(c, MODE_TRAIN, a));  // times its encode and MLP kernels itself
  }
  if (c->mc_minmax) {  // online macrocells (Sec. 5.3): this step's samples widen the ranges
    int tk1 = prof_begin(c);
    NV_TRY(launch_mc_update(a.xyz, a.in, n, a.vol, a.seed, a.sample_step, c->mc_nx, c->mc_ny, c->mc_nz,
                            c->mc_cell, c->mc_minmax, c->stream));
    prof_end(c, NV_K_OTHER, tk1);
  }
  int tk = prof_begin(c);
  NV_TRY(launch_adam(c, 1.0 / (double)n, loss_k));
  prof_end(c, NV_K_ADAM, tk);
  if (used_slot >= 0) NV_CUDA(cudaEventRecord(c->batch_used[used_slot], c->stream), "nv_train_step: record");
  return NV_OK;
}

extern "C" nv_status nv_train_grad(nv_ctx *c, const float *xyz, const float *target, int64_t n, int64_t n_total,
                                   double *loss_sum_dev) {
  if (!c) return nv_fail(NV_ERR_ARG, "nv_train_grad: ctx is NULL");
  if (n < 0 || n_total < 1 || n > n_total)
    return nv_fail(NV_ERR_ARG, "nv_train_grad: need 0 <= n <= n_total, n_total >= 1 (n=%lld, n_total=%lld)",
                   (long long)n, (long long)n_total);
  if (n > 0 && (!xyz || !target)) return nv_fail(NV_ERR_ARG, "nv_train_grad: xyz and target are required");
  if (n > 0 && (is_host_ptr(xyz) || is_host_ptr(target)))
    return nv_fail(NV_ERR_ARG, "nv_train_grad: xyz and target must be device memory");
  if (!loss_sum_dev || is_host_ptr(loss_sum_dev)) return nv_fail(NV_ERR_ARG, "nv_train_grad: loss_sum_dev must be device memory");
  NV_CUDA(cudaMemsetAsync(loss_sum_dev, 0, sizeof(double), c->stream), "nv_train_grad: clear loss");
  if (n == 0) return NV_OK;
  MlpArgs a{};
  a.n = n;
  a.grads = c->grads;
  a.ds = c->ds;
  a.inv_n = (float)(1.0 / (double)n_total);  // the global batch mean
  a.l1 = c->loss_kind == NV_LOSS_L1;
  a.xyz = xyz;
  a.in = target;
  if (c->prec == NV_FP32) {
    int tk = prof_begin(c);
    NV_TRY(launch_mlp_f32_ext(c, MODE_TRAIN, a, nullptr, 1, n, loss_sum_dev));
    prof_end(c, NV_K_MLP, tk);
  } else {
    NV_TRY(launch_mlp_tc_ext(c, MODE_TRAIN, a, nullptr, 1, n, loss_sum_dev));
  }
  if (c->mc_minmax) {
    int tk = prof_begin(c);
    NV_TRY(launch_mc_update(a.xyz, a.in, n, a.vol, a.seed, a.sample_step, c->mc_nx, c->mc_ny, c->mc_nz, c->mc_cell,
                            c->mc_minmax, c->stream));
    prof_end(c, NV_K_OTHER, tk);
  }
  return NV_OK;
}

extern "C" nv_status nv_dp_buffers(nv_ctx *c, float **grads_dev, int64_t *n, int32_t **flags_dev) {
  if (!c || !grads_dev || !n || !flags_dev) return nv_fail(NV_ERR_ARG, "nv_dp_buffers: NULL argument");
  *grads_dev = c->grads;
  *n = c->n_params;
  *flags_dev = &c->ds->overflow;  // [overflow, off_domain], adjacent in DevState
  return NV_OK;
}

static nv_status check_mc_grid(int nx, int ny, int nz, int cell, const char *who) {
  if (nx < 1 || ny < 1 || nz < 1 || cell < 1) return nv_fail(NV_ERR_ARG, "%s: grid %dx%dx%d / cell %d", who, nx, ny, nz, cell);
  return NV_OK;
}

extern "C" nv_status nv_macrocells_reset(float *minmax, int nx, int ny, int nz, int cell, void *stream) {
  if (!minmax) return nv_fail(NV_ERR_ARG, "nv_macrocells_reset: minmax is NULL");
  NV_TRY(check_mc_grid(nx, ny, nz, cell, "nv_macrocells_reset"));
  return launch_mc_reset(minmax, nx, ny, nz, cell, (cudaStream_t)stream);
}

extern "C" nv_status nv_macrocells_update(const float *xyz, const float *val, int64_t n, int nx, int ny, int nz,
                                          int cell, float *minmax, void *stream) {
  if (!xyz || !val || !minmax || n < 0) return nv_fail(NV_ERR_ARG, "nv_macrocells_update: bad argument");
  NV_TRY(check_mc_grid(nx, ny, nz, cell, "nv_macrocells_update"));
  return launch_mc_update(xyz, val, n, nv_volume{}, 0, 0, nx, ny, nz, cell, minmax, (cudaStream_t)stream);
}

extern "C" nv_status nv_macrocells_mu(const float *minmax, int nx, int ny, int nz, int cell, const float *lut,
                                      float *mu, void *stream) {
  if (!minmax || !lut || !mu) return nv_fail(NV_ERR_ARG, "nv_macrocells_mu: NULL argument");
  NV_TRY(check_mc_grid(nx, ny, nz, cell, "nv_macrocells_mu"));
  return launch_mc_mu(minmax, nx, ny, nz, cell, lut, mu, (cudaStream_t)stream);
}

extern "C" nv_status nv_set_online_macrocells(nv_ctx *c, float *minmax, int nx, int ny, int nz, int cell) {
  if (!c) return nv_fail(NV_ERR_ARG, "nv_set_online_macrocells: ctx is NULL");
  if (minmax) NV_TRY(check_mc_grid(nx, ny, nz, cell, "nv_set_online_macrocells"));
  c->mc_minmax = minmax;
  c->mc_nx = nx;
  c->mc_ny = ny;
  c->mc_nz = nz;
  c->mc_cell = cell;
  return NV_OK;
}

extern "C" nv_status nv_macrocells_build(const nv_volume *vol, int cell, const float *lut, float *minmax,
                                         float *mu, void *stream) {
  NV_TRY(check_volume(vol, "nv_macrocells_build"));
  if (cell < 1) return nv_fail(NV_ERR_ARG, "nv_macrocells_build: cell=%d", cell);
  if (mu && !lut) return nv_fail(NV_ERR_ARG, "nv_macrocells_build: mu_max needs the LUT");
  return launch_macrocells(*vol, cell, lut, minmax, mu, (cudaStream_t)stream);
}

static void renderer_free(nv_renderer *r) {
  if (!r) return;
  for (int b = 0; b < 2; ++b) {
    cudaFree(r->ray[b]);
    cudaFree(r->next_k[b]);
  }
  cudaFree(r->coords);
  cudaFree(r->values);
  cudaFree(r->seg_exp);
  cudaFree(r->aux[0]);
  cudaFree(r->aux[1]);
  cudaFree(r->pt[0]);
  cudaFree(r->pt[1]);
  cudaFree(r->pt_coords);
  cudaFree(r->nvalid);
  cudaFree(r->counters);
  cudaFree(r->d_samples);
  cudaFreeHost(r->h_count);
  delete r;
}

extern "C" nv_status nv_renderer_create(int64_t max_pixels, int K, void *stream, nv_renderer **out) {
  if (!out) return nv_fail(NV_ERR_ARG, "nv_renderer_create: out is NULL");
  *out = nullptr;
  if (max_pixels < 1 || max_pixels > (1LL << 28)) return nv_fail(NV_ERR_ARG, "nv_renderer_create: max_pixels");
  if (K < 1 || K > 64) return nv_fail(NV_ERR_ARG, "nv_renderer_create: K=%d not in [1, 64]", K);
  nv_renderer *r = new (std::nothrow) nv_renderer();
  if (!r) return nv_fail(NV_ERR_OOM, "nv_renderer_create: host allocation");
  r->max_pixels = max_pixels;
  r->K = K;
  r->stream = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaMalloc(&r->ray[b], (size_t)max_pixels * 13 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&r->next_k[b], (size_t)max_pixels * sizeof(int));
  }
  if (e == cudaSuccess) e = cudaMalloc(&r->coords, (size_t)max_pixels * K * 3 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&r->values, (size_t)max_pixels * K * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&r->seg_exp, (size_t)max_pixels * K * sizeof(float));
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMalloc(&r->aux[b], (size_t)max_pixels * 5 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&r->nvalid, (size_t)max_pixels * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&r->counters, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&r->d_samples, sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMallocHost(&r->h_count, 4 * sizeof(int));
  if (e != cudaSuccess) {
    nv_status s = nv_cuda_check(e, "nv_renderer_create: allocation");
    renderer_free(r);
    return s;
  }
  *out = r;
  return NV_OK;
}

extern "C" nv_status nv_renderer_destroy(nv_renderer *r) {
  if (!r) return NV_OK;
  cudaStreamSynchronize(r->stream);
  renderer_free(r);
  return NV_OK;
}

// Arguments of nv_render and nv_render_rows, whose image is `pixels` pixels.
static nv_status check_render(const nv_renderer *r, const nv_ctx *net, const nv_volume *raw, const nv_camera *cam,
                              const float *lut, const nv_macrocells *mc, const nv_render_opts *opts,
                              const float *rgba, int64_t pixels) {
  if (!r || !cam || !lut || !opts || !rgba) return nv_fail(NV_ERR_ARG, "nv_render: NULL argument");
  if (!net) NV_TRY(check_volume(raw, "nv_render"));
  if (net && !net->params_set) return nv_fail(NV_ERR_STATE, "nv_render: network parameters never set");
  if (cam->width < 1 || cam->height < 1) return nv_fail(NV_ERR_ARG, "nv_render: image %dx%d", cam->width, cam->height);
  if (pixels > r->max_pixels)
    return nv_fail(NV_ERR_ARG, "nv_render: %lld pixels exceed the renderer's %lld", (long long)pixels,
                   (long long)r->max_pixels);
  if (!(opts->step > 0.f) || !(opts->alpha_exp > 0.f) || !(opts->et > 0.f))
    return nv_fail(NV_ERR_ARG, "nv_render: step, alpha_exp and et must be > 0");
  if (opts->K != r->K) return nv_fail(NV_ERR_ARG, "nv_render: K=%d but the renderer was made for K=%d", opts->K, r->K);
  if (mc && (!mc->mu_max_dev || mc->cell < 1 || mc->nx < 1 || mc->ny < 1 || mc->nz < 1))
    return nv_fail(NV_ERR_ARG, "nv_render: bad macrocell grid");
  if (opts->step_max > 0.f && (!mc || !(opts->step_max >= opts->step)))
    return nv_fail(NV_ERR_ARG, "nv_render: the adaptive step needs macrocells and step_max >= step");
  if (opts->shade != 0 && opts->shade != 1) return nv_fail(NV_ERR_ARG, "nv_render: shade=%d", opts->shade);
  if (opts->shade == 1) {
    const float l2 = opts->light[0] * opts->light[0] + opts->light[1] * opts->light[1] + opts->light[2] * opts->light[2];
    if (!(fabsf(l2 - 1.f) < 1e-3f) || !(opts->ambient >= 0.f && opts->ambient <= 1.f))
      return nv_fail(NV_ERR_ARG, "nv_render: shadows need a unit light direction and ambient in [0, 1]");
  }
  if (!(cam->tan_half_fovy >= 0.f)) return nv_fail(NV_ERR_ARG, "nv_render: tan_half_fovy < 0");
  return NV_OK;
}

extern "C" nv_status nv_render(nv_renderer *r, nv_ctx *net, const nv_volume *raw, const nv_camera *cam,
                               const float *lut, const nv_macrocells *mc, const nv_render_opts *opts,
                               float *rgba) {
  const int64_t pixels = cam ? (int64_t)cam->width * cam->height : 0;
  NV_TRY(check_render(r, net, raw, cam, lut, mc, opts, rgba, pixels));
  return render_impl(r, net, raw, *cam, lut, mc, *opts, 0, cam->height, rgba);
}

extern "C" nv_status nv_render_rows(nv_renderer *r, nv_ctx *net, const nv_volume *raw, const nv_camera *cam,
                                    const float *lut, const nv_macrocells *mc, const nv_render_opts *opts,
                                    int row0, int rows, float *rgba) {
  if (cam && (rows < 1 || row0 < 0 || row0 > cam->height - rows))
    return nv_fail(NV_ERR_ARG, "nv_render_rows: rows [%d, %d + %d) not inside the image's %d", row0, row0, rows,
                   cam->height);
  const int64_t pixels = cam ? (int64_t)cam->width * rows : 0;
  NV_TRY(check_render(r, net, raw, cam, lut, mc, opts, rgba, pixels));
  return render_impl(r, net, raw, *cam, lut, mc, *opts, row0, rows, rgba);
}

extern "C" nv_status nv_render_inshader(nv_ctx *net, const nv_camera *cam, const float *lut,
                                        const nv_macrocells *mc, const nv_render_opts *opts, float *rgba,
                                        int64_t *samples_dev) {
  if (!net || !cam || !lut || !opts || !rgba) return nv_fail(NV_ERR_ARG, "nv_render_inshader: NULL argument");
  if (!net->params_set) return nv_fail(NV_ERR_STATE, "nv_render_inshader: network parameters never set");
  if (cam->width < 1 || cam->height < 1)
    return nv_fail(NV_ERR_ARG, "nv_render_inshader: image %dx%d", cam->width, cam->height);
  if ((int64_t)cam->width * cam->height > ((int64_t)1 << 31) - 256)
    return nv_fail(NV_ERR_ARG, "nv_render_inshader: image too large");
  if (!(opts->step > 0.f) || !(opts->alpha_exp > 0.f) || !(opts->et > 0.f))
    return nv_fail(NV_ERR_ARG, "nv_render_inshader: step, alpha_exp and et must be > 0");
  if (mc && (!mc->mu_max_dev || mc->cell < 1 || mc->nx < 1 || mc->ny < 1 || mc->nz < 1))
    return nv_fail(NV_ERR_ARG, "nv_render_inshader: bad macrocell grid");
  if (opts->step_max > 0.f) return nv_fail(NV_ERR_UNSUPPORTED, "nv_render_inshader: the fixed step only");
  if (opts->shade != 0 && opts->shade != 1) return nv_fail(NV_ERR_ARG, "nv_render_inshader: shade=%d", opts->shade);
  if (opts->shade == 1) {
    const float l2 = opts->light[0] * opts->light[0] + opts->light[1] * opts->light[1] + opts->light[2] * opts->light[2];
    if (!(fabsf(l2 - 1.f) < 1e-3f) || !(opts->ambient >= 0.f && opts->ambient <= 1.f))
      return nv_fail(NV_ERR_ARG, "nv_render_inshader: shadows need a unit light direction and ambient in [0, 1]");
  }
  if (!(cam->tan_half_fovy >= 0.f)) return nv_fail(NV_ERR_ARG, "nv_render_inshader: tan_half_fovy < 0");
  return render_inshader(net, *cam, lut, mc, *opts, rgba, reinterpret_cast<unsigned long long *>(samples_dev));
}

extern "C" nv_status nv_render_pt(nv_renderer *r, nv_ctx *net, const nv_volume *raw, const nv_camera *cam,
                                  const float *lut, const nv_macrocells *mc, const nv_pt_opts *opts, float *rgba) {
  if (!r || !cam || !lut || !mc || !opts || !rgba) return nv_fail(NV_ERR_ARG, "nv_render_pt: NULL argument");
  if (!net) NV_TRY(check_volume(raw, "nv_render_pt"));
  if (net && !net->params_set) return nv_fail(NV_ERR_STATE, "nv_render_pt: network parameters never set");
  if (cam->width < 1 || cam->height < 1) return nv_fail(NV_ERR_ARG, "nv_render_pt: image %dx%d", cam->width, cam->height);
  if ((int64_t)cam->width * cam->height > r->max_pixels)
    return nv_fail(NV_ERR_ARG, "nv_render_pt: %dx%d exceeds the renderer's %lld pixels", cam->width, cam->height,
                   (long long)r->max_pixels);
  if (!mc->mu_max_dev || mc->cell < 1 || mc->nx < 1 || mc->ny < 1 || mc->nz < 1)
    return nv_fail(NV_ERR_ARG, "nv_render_pt: bad macrocell grid");
  const float l2 = opts->light[0] * opts->light[0] + opts->light[1] * opts->light[1] + opts->light[2] * opts->light[2];
  if (!(opts->density > 0.f) || !(fabsf(l2 - 1.f) < 1e-3f) || opts->max_bounces < 1)
    return nv_fail(NV_ERR_ARG, "nv_render_pt: density > 0, a unit light direction and max_bounces >= 1");
  if (!(cam->tan_half_fovy >= 0.f)) return nv_fail(NV_ERR_ARG, "nv_render_pt: tan_half_fovy < 0");
  return render_pt_impl(r, net, raw, *cam, lut, *mc, *opts, rgba);
}

extern "C" nv_status nv_render_stats(nv_renderer *r, int *iterations, int64_t *samples) {
  if (!r) return nv_fail(NV_ERR_ARG, "nv_render_stats: renderer is NULL");
  NV_CUDA(cudaDeviceSynchronize(), "nv_render_stats: sync");
  int64_t s = 0;
  NV_CUDA(cudaMemcpy(&s, r->d_samples, sizeof(s), cudaMemcpyDeviceToHost), "nv_render_stats: copy");
  if (iterations) *iterations = r->last_iters;
  if (samples) *samples = s;
  return NV_OK;
}

extern "C" nv_status nv_image_mse(const float *a, const float *b, int64_t n, double *mse, void *stream) {
  if (!a || !b || !mse || n < 0) return nv_fail(NV_ERR_ARG, "nv_image_mse: bad argument");
  return launch_image_mse(a, b, n, mse, (cudaStream_t)stream);
}

extern "C" nv_status nv_mse_f64(const float *a, const float *b, int64_t n, double *mse, void *stream) {
  if (!a || !b || !mse || n < 0) return nv_fail(NV_ERR_ARG, "nv_mse_f64: bad argument");
  return launch_mse(a, b, n, mse, (cudaStream_t)stream);
}

extern "C" nv_status nv_volume_mse(nv_ctx *c, const nv_volume *vol, double *mse) {
  if (!c || !mse) return nv_fail(NV_ERR_ARG, "nv_volume_mse: NULL argument");
  NV_TRY(check_volume(vol, "nv_volume_mse"));
  const int64_t n = (int64_t)vol->nx * vol->ny * vol->nz;
  NV_CUDA(cudaMemsetAsync(mse, 0, sizeof(double), c->stream), "nv_volume_mse: memset");
  MlpArgs a{};
  a.vol = *vol;
  a.n = n;
  a.ds = c->ds;
  NV_TRY(c->prec == NV_FP32 ? launch_mlp_f32_ext(c, 3, a, nullptr, 1, n, mse)
                            : launch_mlp_tc_ext(c, 3, a, nullptr, 1, n, mse));
  return launch_scale_double(mse, 1.0 / (double)n, c->stream);
}

extern "C" nv_status nv_profile_enable(nv_ctx *c, int enable) {
  if (!c) return nv_fail(NV_ERR_ARG, "nv_profile_enable: ctx is NULL");
  if (!c->prof) {
    Prof *p = new (std::nothrow) Prof();
    if (!p) return nv_fail(NV_ERR_OOM, "nv_profile_enable: host allocation");
    p->ev.resize(2 * Prof::kMax, nullptr);
    p->cls.resize(Prof::kMax, -1);
    for (auto &e : p->ev) {
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) {
        prof_free(p);
        return nv_cuda_check(r, "nv_profile_enable: events");
      }
    }
    c->prof = p;
  }
  c->prof->on = enable != 0;
  return NV_OK;
}

extern "C" nv_status nv_profile_read(nv_ctx *c, int kclass, double *total_ms, int *launches) {
  if (!c || !total_ms || !launches) return nv_fail(NV_ERR_ARG, "nv_profile_read: NULL argument");
  *total_ms = 0.0;
  *launches = 0;
  Prof *p = c->prof;
  if (!p) return NV_OK;
  NV_CUDA(cudaStreamSynchronize(c->stream), "nv_profile_read: sync");
  int keep = 0;
  for (int i = 0; i < p->used; ++i) {
    if (p->cls[i] == kclass) {
      float ms = 0.f;
      NV_CUDA(cudaEventElapsedTime(&ms, p->ev[2 * i], p->ev[2 * i + 1]), "nv_profile_read: elapsed");
      *total_ms += ms;
      ++*launches;
      p->cls[i] = -2;  // consumed
    } else if (p->cls[i] != -2) {
      keep = i + 1;
    }
  }
  if (keep == 0) p->used = 0;
  return NV_OK;
}

extern "C" nv_status nv_sync(nv_ctx *c) {
  if (!c) return nv_fail(NV_ERR_ARG, "nv_sync: ctx is NULL");
  NV_CUDA(cudaStreamSynchronize(c->stream), "nv_sync");
  int err = 0;
  NV_CUDA(cudaMemcpy(&err, &c->ds->err, sizeof(int), cudaMemcpyDeviceToHost), "nv_sync: flag");
  if (err) return nv_fail(NV_ERR_TIMEOUT, "a kernel gave up a bounded wait (code %d)", err);
  return NV_OK;
}

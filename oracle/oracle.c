/*
 * oracle.c -- plain, slow FP64 CPU restatement of the hot path of
 * "Interactive Volume Visualization via Multi-Resolution Hash Encoding based
 * Neural Representation" (Wu, Bauer, Doyle, Ma; arXiv 2207.11620).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py load this library.  The GPU
 * library never links, includes or calls it; the two share no code.
 *
 * Precision.  Everything is FP64, except where a floating-point value decides
 * an integer: the grid cell of a point at a hash level (A-1: p = fl32(x*N_l)),
 * the voxel cell of a trilinear lookup, the macrocell of a ray sample, the
 * ray sample positions themselves and the transfer-function index range of a
 * macrocell.  There the kernel's FP32 operations are restated one by one (this
 * file is compiled with -ffp-contract=off, so no multiply-add is fused) and
 * the integer decision is taken on the FP32 value; all arithmetic that
 * follows the decision is FP64.
 *
 * Pins: every function below is checked in tests/test_oracle.py against
 * values the paper prints, closed forms, brute force or finite differences.
 * Nothing here is "parity unpinned".
 *
 * Data layouts (shared with the GPU path by specification only):
 *   tables  [L][T][F]            T = 2^log2T, entry (l, h) holds F features
 *   weights W_0, W_1, ...        W_k is [dims[k+1]][dims[k]] row-major, no bias
 *   params  = tables followed by weights, one flat vector
 *   points  [n][3] float32 in [0,1)^3
 *   volume  [nz][ny][nx] float32, x fastest, cell-centred voxels
 *   lut     [256][4] float32 RGBA
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Spatial-hash primes of the multi-resolution hash encoding the paper adopts
 * (Sec. 3.1, which cites instant-NGP for the encoding). */
#define OR_PI1 1u
#define OR_PI2 2654435761u
#define OR_PI3 805459861u

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Sec. 3.1 / Fig. 1B: resolution of level l, N_l = floor(Nmin * b^l), FP64. */
void or_level_res(int L, int Nmin, double b, int *res) {
  for (int l = 0; l < L; ++l) res[l] = (int)floor((double)Nmin * pow(b, (double)l));
}

/* Sec. 3.1: spatial hash of an integer grid vertex into a table of T entries:
 * XOR of the per-axis products with the primes (1, 2654435761, 805459861) in
 * uint32 wrap-around arithmetic, reduced mod T. */
uint32_t or_hash(int64_t vx, int64_t vy, int64_t vz, uint32_t T) {
  uint32_t h = ((uint32_t)vx * OR_PI1) ^ ((uint32_t)vy * OR_PI2) ^ ((uint32_t)vz * OR_PI3);
  return h % T;
}

/* Number of parameters of a network as the paper counts them (App. B, table of
 * parameter counts): coarse levels stored densely with N_l^3 entries when that
 * is smaller than T, no biases, output layer padded to out_pad rows. */
int64_t or_param_count_dense_coarse(int L, int F, int log2T, int base, double scale,
                                    int n_neurons, int n_hidden, int out_pad) {
  int64_t T = (int64_t)1 << log2T, total = 0;
  for (int l = 0; l < L; ++l) {
    int64_t N = (int64_t)floor((double)base * pow(scale, (double)l));
    int64_t dense = N * N * N;
    total += (dense < T ? dense : T) * F;
  }
  total += (int64_t)L * F * n_neurons;
  total += (int64_t)(n_hidden - 1) * n_neurons * n_neurons;
  total += (int64_t)n_neurons * out_pad;
  return total;
}

/* ---------------------------------------------------------------- encode -- */

/* A-1: scale and cell of one coordinate at resolution N.  The product is the
 * kernel's single FP32 multiply; the cell and the weight follow from it. */
static void or_cell(float x, int N, int64_t *c, double *w) {
  float p = x * (float)N;
  double fl = floor((double)p);
  *c = (int64_t)fl;
  *w = (double)p - fl;
}

/* A-2: the 8 corner indices of point x at level l (corner d = dx + 2dy + 4dz). */
void or_hash_indices(int L, int log2T, const int *res, const float *xyz, int64_t n, uint32_t *idx) {
  uint32_t T = 1u << log2T;
  for (int64_t i = 0; i < n; ++i)
    for (int l = 0; l < L; ++l) {
      int64_t c[3]; double w[3];
      for (int a = 0; a < 3; ++a) or_cell(xyz[3 * i + a], res[l], &c[a], &w[a]);
      for (int d = 0; d < 8; ++d)
        idx[(i * L + l) * 8 + d] = or_hash(c[0] + (d & 1), c[1] + ((d >> 1) & 1), c[2] + ((d >> 2) & 1), T);
    }
}

/* A-1..A-3 for one point: f[l*F + j] = sum over the 8 corners of the trilinear
 * weight times table entry j (Sec. 3.1, Fig. 1B: interpolate per level,
 * concatenate levels). */
static void or_encode_point(int L, int F, int log2T, const int *res, const double *tables,
                            const float *x, double *f) {
  uint32_t T = 1u << log2T;
  for (int l = 0; l < L; ++l) {
    int64_t c[3]; double w[3];
    for (int a = 0; a < 3; ++a) or_cell(x[a], res[l], &c[a], &w[a]);
    for (int j = 0; j < F; ++j) f[l * F + j] = 0.0;
    for (int d = 0; d < 8; ++d) {
      int dx = d & 1, dy = (d >> 1) & 1, dz = (d >> 2) & 1;
      double wt = (dx ? w[0] : 1.0 - w[0]) * (dy ? w[1] : 1.0 - w[1]) * (dz ? w[2] : 1.0 - w[2]);
      uint32_t h = or_hash(c[0] + dx, c[1] + dy, c[2] + dz, T);
      const double *e = tables + ((int64_t)l * T + h) * F;
      for (int j = 0; j < F; ++j) f[l * F + j] += wt * e[j];
    }
  }
}

void or_encode(int L, int F, int log2T, const int *res, const double *tables,
               const float *xyz, int64_t n, double *feat) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    or_encode_point(L, F, log2T, res, tables, xyz + 3 * i, feat + i * (int64_t)L * F);
}

/* ------------------------------------------------------------------- MLP -- */

static double or_sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

static int or_max_dim(const int *dims, int n_dims) {
  int m = 0;
  for (int k = 0; k < n_dims; ++k) if (dims[k] > m) m = dims[k];
  return m;
}

/* A-4 for one point: a_0 = f; z_{k+1} = W_k a_k; a_{k+1} = ReLU(z_{k+1}) on the
 * hidden layers; y = sigmoid(z_last) (Sec. 3.1: ReLU on all hidden layers, no
 * biases; the sigmoid output is the reading stated in the design notes).
 * act holds every layer's activations back to back (dims[0] + dims[1] + ...)
 * so the backward pass can reuse them. */
static double or_mlp_point(const int *dims, int n_dims, const double *weights, double *act) {
  const double *W = weights;
  double *a = act;
  double z_out = 0.0;
  for (int k = 0; k + 1 < n_dims; ++k) {
    int din = dims[k], dout = dims[k + 1];
    double *an = a + din;
    for (int j = 0; j < dout; ++j) {
      double z = 0.0;
      for (int i = 0; i < din; ++i) z += W[(int64_t)j * din + i] * a[i];
      if (k + 2 < n_dims) an[j] = z > 0.0 ? z : 0.0;
      else { an[j] = z; z_out = z; }
    }
    W += (int64_t)din * dout;
    a = an;
  }
  return or_sigmoid(z_out);
}

static int64_t or_weight_count(const int *dims, int n_dims) {
  int64_t c = 0;
  for (int k = 0; k + 1 < n_dims; ++k) c += (int64_t)dims[k] * dims[k + 1];
  return c;
}

static int or_act_len(const int *dims, int n_dims) {
  int s = 0;
  for (int k = 0; k < n_dims; ++k) s += dims[k];
  return s;
}

/* MLP alone on given inputs (used to pin the MLP separately from the encoding). */
void or_mlp_forward(const int *dims, int n_dims, const double *weights, const double *in,
                    int64_t n, double *y) {
  int alen = or_act_len(dims, n_dims);
#pragma omp parallel
  {
    double *act = (double *)malloc(sizeof(double) * alen);
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      memcpy(act, in + i * dims[0], sizeof(double) * dims[0]);
      y[i] = or_mlp_point(dims, n_dims, weights, act);
    }
    free(act);
  }
}

/* Encode + MLP: the network value at each point (A-1..A-4). */
void or_forward(int L, int F, int log2T, const int *res, const int *dims, int n_dims,
                const double *params, const float *xyz, int64_t n, double *y) {
  int64_t T = (int64_t)1 << log2T;
  const double *weights = params + (int64_t)L * T * F;
  int alen = or_act_len(dims, n_dims);
#pragma omp parallel
  {
    double *act = (double *)malloc(sizeof(double) * alen);
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      or_encode_point(L, F, log2T, res, params, xyz + 3 * i, act);
      y[i] = or_mlp_point(dims, n_dims, weights, act);
    }
    free(act);
  }
}

/* A-5: L2 loss, the mean over the batch of (y - t)^2 (Sec. 7 names L2 for the
 * stability-critical case; the batch mean is the reading stated in the design
 * notes). */
double or_loss_l2(const double *y, const float *t, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) { double d = y[i] - (double)t[i]; s += d * d; }
  return n > 0 ? s / (double)n : 0.0;
}

/* L1 loss, the paper's default (Sec. 3.1, App. B): the mean over the batch of
 * |y - t|.  Its derivative in y is sign(y - t) / n, taken as 0 where y == t. */
double or_loss_l1(const double *y, const float *t, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += fabs(y[i] - (double)t[i]);
  return n > 0 ? s / (double)n : 0.0;
}

/* Exponentially decaying learning rate (App. B: decay start, interval and base
 * around Adam).  Reading: the rate of the optimizer step with 0-based index k
 * is lr0 * base^d with d = 0 while k < start and d = floor((k - start) /
 * interval) + 1 from then on, so the first decay applies to step `start`. */
double or_lr_at(double lr0, int k, int start, int interval, double base) {
  if (k < start || interval <= 0) return lr0;
  return lr0 * pow(base, (double)((k - start) / interval + 1));
}

/* A-6 for one point: the network's forward at x (act: every layer's
 * activations), then the chain rule from dL/dy back to the input features.
 * dz_out = dL/dy * y (1 - y); dW_k += delta_k a_k^T (when gw is given);
 * delta_{k-1} = (W_k^T delta_k) * 1[z > 0]; df = W_0^T delta_0, left in
 * delta[0 .. L*F). */
static void or_point_df(int L, int F, int log2T, const int *res, const int *dims, int n_dims,
                        const double *params, const float *x, double dL_dy, double *gw,
                        double *act, double *delta, double *din) {
  uint32_t T = 1u << log2T;
  const double *weights = params + (int64_t)L * T * F;
  int nl = n_dims - 1;
  or_encode_point(L, F, log2T, res, params, x, act);
  double y = or_mlp_point(dims, n_dims, weights, act);
  delta[0] = dL_dy * y * (1.0 - y);
  /* walk the layers from the output back to the input */
  for (int k = nl - 1; k >= 0; --k) {
    int ind = dims[k], outd = dims[k + 1];
    int64_t woff = 0, aoff = 0;
    for (int q = 0; q < k; ++q) { woff += (int64_t)dims[q] * dims[q + 1]; aoff += dims[q]; }
    const double *Wk = weights + woff;
    const double *ak = act + aoff;
    if (gw) {
      double *gWk = gw + woff;
      for (int j = 0; j < outd; ++j)
        for (int c = 0; c < ind; ++c) gWk[(int64_t)j * ind + c] += delta[j] * ak[c];
    }
    for (int c = 0; c < ind; ++c) {
      double s = 0.0;
      for (int j = 0; j < outd; ++j) s += Wk[(int64_t)j * ind + c] * delta[j];
      /* a_k = ReLU(z_k) for k > 0, so 1[z_k > 0] == 1[a_k > 0] */
      din[c] = (k > 0) ? (ak[c] > 0.0 ? s : 0.0) : s;
    }
    memcpy(delta, din, sizeof(double) * ind);
  }
}

/* A-6 / A-7: analytic backward of encode + MLP for upstream gradients dL/dy.
 * Accumulates (+=) into grads, laid out like params (tables then weights):
 * the weight gradients of or_point_df, and for every corner of every level
 * its trilinear weight times df (the adjoint of A-3).
 * Threads: the per-point chain rule runs over points in parallel (df of every
 * point kept, weight gradients summed per thread, then over the threads in
 * order); the scatter runs over levels in parallel, each level visiting the
 * points in order, so every table entry sums its contributions in point
 * order, as a serial loop would. */
void or_backward(int L, int F, int log2T, const int *res, const int *dims, int n_dims,
                 const double *params, const float *xyz, int64_t n, const double *dL_dy,
                 double *grads) {
  uint32_t T = 1u << log2T;
  int64_t tab = (int64_t)L * T * F;
  int64_t nw = or_weight_count(dims, n_dims);
  int alen = or_act_len(dims, n_dims);
  int mx = or_max_dim(dims, n_dims);
  int LF = L * F;
  double *df = (double *)malloc(sizeof(double) * (n > 0 ? n : 1) * LF);
  int nt = 1;
#ifdef _OPENMP
  nt = omp_get_max_threads();
#endif
  double *gw = (double *)calloc((size_t)nt * nw, sizeof(double));
#pragma omp parallel num_threads(nt)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double *act = (double *)malloc(sizeof(double) * alen);
    double *delta = (double *)malloc(sizeof(double) * mx);
    double *din = (double *)malloc(sizeof(double) * mx);
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      or_point_df(L, F, log2T, res, dims, n_dims, params, xyz + 3 * i, dL_dy[i], gw + (int64_t)tid * nw, act,
                  delta, din);
      memcpy(df + i * LF, delta, sizeof(double) * LF);  /* delta holds df (length L*F) */
    }
    free(act); free(delta); free(din);
  }
  for (int t = 0; t < nt; ++t)
    for (int64_t k = 0; k < nw; ++k) grads[tab + k] += gw[(int64_t)t * nw + k];
  /* the scatter into the table gradients, level by level */
#pragma omp parallel for schedule(dynamic, 1)
  for (int l = 0; l < L; ++l)
    for (int64_t i = 0; i < n; ++i) {
      const float *x = xyz + 3 * i;
      int64_t c[3]; double w[3];
      for (int a = 0; a < 3; ++a) or_cell(x[a], res[l], &c[a], &w[a]);
      for (int d = 0; d < 8; ++d) {
        int dx = d & 1, dy = (d >> 1) & 1, dz = (d >> 2) & 1;
        double wt = (dx ? w[0] : 1.0 - w[0]) * (dy ? w[1] : 1.0 - w[1]) * (dz ? w[2] : 1.0 - w[2]);
        uint32_t h = or_hash(c[0] + dx, c[1] + dy, c[2] + dz, T);
        double *g = grads + ((int64_t)l * T + h) * F;
        for (int j = 0; j < F; ++j) g[j] += wt * df[i * LF + l * F + j];
      }
    }
  free(df); free(gw);
}

/* Gradient of the loss with respect to the point coordinates: dxyz[i][a] =
 * dL/dx_a.  Within a cell of level l the trilinear weights are products of
 * w_a or 1 - w_a with w_a = x_a N_l - c_a, so d(weight)/dx_a = N_l times the
 * product of the other two axes' factors, signed + for the upper corner and -
 * for the lower one (the FP32 rounding of x N_l is taken as having slope N_l).
 * dL/dx_a = sum over levels and corners of that derivative times the dot
 * product of the corner's table entry with df_l. */
void or_backward_x(int L, int F, int log2T, const int *res, const int *dims, int n_dims,
                   const double *params, const float *xyz, int64_t n, const double *dL_dy,
                   double *dxyz) {
  uint32_t T = 1u << log2T;
  int alen = or_act_len(dims, n_dims);
  int mx = or_max_dim(dims, n_dims);
#pragma omp parallel
  {
    double *act = (double *)malloc(sizeof(double) * alen);
    double *delta = (double *)malloc(sizeof(double) * mx);
    double *din = (double *)malloc(sizeof(double) * mx);
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      const float *x = xyz + 3 * i;
      or_point_df(L, F, log2T, res, dims, n_dims, params, x, dL_dy[i], NULL, act, delta, din);
      double gx[3] = {0.0, 0.0, 0.0};
      for (int l = 0; l < L; ++l) {
        int64_t c[3]; double w[3];
        for (int a = 0; a < 3; ++a) or_cell(x[a], res[l], &c[a], &w[a]);
        for (int d = 0; d < 8; ++d) {
          int dd[3] = {d & 1, (d >> 1) & 1, (d >> 2) & 1};
          uint32_t h = or_hash(c[0] + dd[0], c[1] + dd[1], c[2] + dd[2], T);
          const double *e = params + ((int64_t)l * T + h) * F;
          double dot = 0.0;
          for (int j = 0; j < F; ++j) dot += e[j] * delta[l * F + j];
          for (int a = 0; a < 3; ++a) {
            double dw = dd[a] ? 1.0 : -1.0;
            for (int o = 0; o < 3; ++o)
              if (o != a) dw *= dd[o] ? w[o] : 1.0 - w[o];
            gx[a] += (double)res[l] * dw * dot;
          }
        }
      }
      for (int a = 0; a < 3; ++a) dxyz[3 * i + a] = gx[a];
    }
    free(act); free(delta); free(din);
  }
}

/* --------------------------------------------------- error magnitudes -- */

/* Per-element error magnitudes for the parity bounds (test infrastructure).
 * For a quantity q of the path, M(q) >= |q| is the magnitude its rounding
 * errors scale with, propagated in FP64 by the rules of running error
 * analysis (Wilkinson; Higham, "Accuracy and Stability of Numerical
 * Algorithms", ch. 3): an exact input has M = |q|; a sum or a dot product has
 * the sum of its terms' magnitudes (the Sum |terms| of the classical bound
 * |fl(sum) - sum| <= gamma_n Sum |terms|), a product the product of its
 * factors' magnitudes, and a smooth function g of z has |g(z)| + |g'(z)| M(z).
 * An evaluation that rounds each operation to a unit roundoff u, in any order,
 * with chains of at most k dependent roundings, stays within about k u M(q)
 * of q; where nothing cancels, M(q) = |q| and the bound is relative.
 *
 * ReLU: the forward passes M unmasked (a unit whose sign the rounding decides
 * moves its output by at most its own error, which M then still covers).  The
 * backward's masks 1[z > 0] are discontinuous, so a backward magnitude holds
 * only for points whose pre-activations are all clear of zero by more than
 * their error (the kink margin or_forward_mag reports); with masked == 0 every
 * unit is counted instead, a magnitude that covers any masks. */

/* A-1..A-3 with magnitudes: f as or_encode_point, fm = Sum_corners w |theta|. */
static void or_encode_point_mag(int L, int F, int log2T, const int *res, const double *tables,
                                const float *x, double *f, double *fm) {
  uint32_t T = 1u << log2T;
  for (int l = 0; l < L; ++l) {
    int64_t c[3]; double w[3];
    for (int a = 0; a < 3; ++a) or_cell(x[a], res[l], &c[a], &w[a]);
    for (int j = 0; j < F; ++j) { f[l * F + j] = 0.0; fm[l * F + j] = 0.0; }
    for (int d = 0; d < 8; ++d) {
      int dx = d & 1, dy = (d >> 1) & 1, dz = (d >> 2) & 1;
      double wt = (dx ? w[0] : 1.0 - w[0]) * (dy ? w[1] : 1.0 - w[1]) * (dz ? w[2] : 1.0 - w[2]);
      uint32_t h = or_hash(c[0] + dx, c[1] + dy, c[2] + dz, T);
      const double *e = tables + ((int64_t)l * T + h) * F;
      for (int j = 0; j < F; ++j) {
        f[l * F + j] += wt * e[j];
        fm[l * F + j] += wt * fabs(e[j]);
      }
    }
  }
}

/* A-4 with magnitudes: act / actm hold every layer's values and magnitudes
 * (layout of or_mlp_point, the input layer filled by the caller).  Returns y;
 * *ymag = y + y (1 - y) M(z_out); *kink = the smallest |z| / M(z) over the
 * hidden units (infinity if none has M(z) > 0). */
static double or_mlp_point_mag(const int *dims, int n_dims, const double *weights, double *act, double *actm,
                               double *ymag, double *kink) {
  const double *W = weights;
  double *a = act, *am = actm;
  double z_out = 0.0, zm_out = 0.0, margin = INFINITY;
  for (int k = 0; k + 1 < n_dims; ++k) {
    int din = dims[k], dout = dims[k + 1];
    double *an = a + din, *amn = am + din;
    for (int j = 0; j < dout; ++j) {
      double z = 0.0, zm = 0.0;
      for (int i = 0; i < din; ++i) {
        z += W[(int64_t)j * din + i] * a[i];
        zm += fabs(W[(int64_t)j * din + i]) * am[i];
      }
      if (k + 2 < n_dims) {
        an[j] = z > 0.0 ? z : 0.0;
        amn[j] = zm;
        if (zm > 0.0 && fabs(z) / zm < margin) margin = fabs(z) / zm;
      } else {
        an[j] = z; amn[j] = zm; z_out = z; zm_out = zm;
      }
    }
    W += (int64_t)din * dout;
    a = an; am = amn;
  }
  double y = or_sigmoid(z_out);
  *ymag = y + y * (1.0 - y) * zm_out;
  *kink = margin;
  return y;
}

/* Magnitudes of the encoded features, fmag [n][L*F]. */
void or_encode_mag(int L, int F, int log2T, const int *res, const double *tables, const float *xyz, int64_t n,
                   double *fmag) {
#pragma omp parallel
  {
    double *f = (double *)malloc(sizeof(double) * L * F);
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i)
      or_encode_point_mag(L, F, log2T, res, tables, xyz + 3 * i, f, fmag + i * (int64_t)L * F);
    free(f);
  }
}

/* Network values y, their magnitudes ymag and kink margins (all [n]). */
void or_forward_mag(int L, int F, int log2T, const int *res, const int *dims, int n_dims, const double *params,
                    const float *xyz, int64_t n, double *y, double *ymag, double *kink) {
  int64_t T = (int64_t)1 << log2T;
  const double *weights = params + (int64_t)L * T * F;
  int alen = or_act_len(dims, n_dims);
#pragma omp parallel
  {
    double *act = (double *)malloc(sizeof(double) * alen);
    double *actm = (double *)malloc(sizeof(double) * alen);
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      or_encode_point_mag(L, F, log2T, res, params, xyz + 3 * i, act, actm);
      y[i] = or_mlp_point_mag(dims, n_dims, weights, act, actm, &ymag[i], &kink[i]);
    }
    free(act); free(actm);
  }
}

/* The chain of or_point_df with magnitudes for one point, upstream magnitude
 * dym: M(sigma') = y (1 - y) + |1 - 2y| M(y); M(delta_out) = dym M(sigma');
 * M(dW_k[j][c]) += M(delta_k[j]) M(a_k[c]) (into gwm when given);
 * M(delta_{k-1}[c]) = 1[z > 0] Sum_j |W_k[j][c]| M(delta_k[j]) (masked == 0:
 * without 1[z > 0]); M(df) = |W_0|^T M(delta_0), left in dm[0 .. L*F). */
static void or_point_dfmag(int L, int F, int log2T, const int *res, const int *dims, int n_dims,
                           const double *params, const float *x, double dym, int masked, double *gwm,
                           double *act, double *actm, double *dm, double *dinm) {
  uint32_t T = 1u << log2T;
  const double *weights = params + (int64_t)L * T * F;
  int nl = n_dims - 1;
  double ym, kink;
  or_encode_point_mag(L, F, log2T, res, params, x, act, actm);
  double y = or_mlp_point_mag(dims, n_dims, weights, act, actm, &ym, &kink);
  double sp = y * (1.0 - y);
  dm[0] = dym * (sp + fabs(1.0 - 2.0 * y) * ym);
  for (int k = nl - 1; k >= 0; --k) {
    int ind = dims[k], outd = dims[k + 1];
    int64_t woff = 0, aoff = 0;
    for (int q = 0; q < k; ++q) { woff += (int64_t)dims[q] * dims[q + 1]; aoff += dims[q]; }
    const double *Wk = weights + woff;
    const double *ak = act + aoff, *akm = actm + aoff;
    if (gwm) {
      double *gWk = gwm + woff;
      for (int j = 0; j < outd; ++j)
        for (int c = 0; c < ind; ++c) gWk[(int64_t)j * ind + c] += dm[j] * akm[c];
    }
    for (int c = 0; c < ind; ++c) {
      double sm = 0.0;
      for (int j = 0; j < outd; ++j) sm += fabs(Wk[(int64_t)j * ind + c]) * dm[j];
      dinm[c] = (k > 0 && masked && !(ak[c] > 0.0)) ? 0.0 : sm;
    }
    memcpy(dm, dinm, sizeof(double) * ind);
  }
}

/* Magnitudes of the parameter gradient of or_backward for upstream gradients
 * of magnitude dy_mag [n] (|dL/dy| for a given upstream gradient), added into
 * gmag [n_params] (tables, then weights): the weight magnitudes of
 * or_point_dfmag, and M(dtheta) += w M(df) at every corner. */
void or_backward_mag(int L, int F, int log2T, const int *res, const int *dims, int n_dims, const double *params,
                     const float *xyz, int64_t n, const double *dy_mag, int masked, double *gmag) {
  uint32_t T = 1u << log2T;
  int64_t tab = (int64_t)L * T * F;
  int alen = or_act_len(dims, n_dims);
  int mx = or_max_dim(dims, n_dims);
  double *act = (double *)malloc(sizeof(double) * alen);
  double *actm = (double *)malloc(sizeof(double) * alen);
  double *dm = (double *)malloc(sizeof(double) * mx);
  double *dinm = (double *)malloc(sizeof(double) * mx);
  for (int64_t i = 0; i < n; ++i) {
    const float *x = xyz + 3 * i;
    or_point_dfmag(L, F, log2T, res, dims, n_dims, params, x, dy_mag[i], masked, gmag + tab, act, actm, dm, dinm);
    for (int l = 0; l < L; ++l) {
      int64_t c[3]; double w[3];
      for (int a = 0; a < 3; ++a) or_cell(x[a], res[l], &c[a], &w[a]);
      for (int d = 0; d < 8; ++d) {
        int dx = d & 1, dy = (d >> 1) & 1, dz = (d >> 2) & 1;
        double wt = (dx ? w[0] : 1.0 - w[0]) * (dy ? w[1] : 1.0 - w[1]) * (dz ? w[2] : 1.0 - w[2]);
        uint32_t h = or_hash(c[0] + dx, c[1] + dy, c[2] + dz, T);
        double *g = gmag + ((int64_t)l * T + h) * F;
        for (int j = 0; j < F; ++j) g[j] += wt * dm[l * F + j];
      }
    }
  }
  free(act); free(actm); free(dm); free(dinm);
}

/* Magnitudes of or_backward_x's coordinate gradient, dxyz_mag [n][3]: per
 * level and corner, N_l |d(weight)/dx_a| times Sum_j |theta_j| M(df_j), with
 * M(df) from or_point_dfmag (upstream magnitudes dy_mag). */
void or_backward_x_mag(int L, int F, int log2T, const int *res, const int *dims, int n_dims,
                       const double *params, const float *xyz, int64_t n, const double *dy_mag, int masked,
                       double *dxyz_mag) {
  uint32_t T = 1u << log2T;
  int alen = or_act_len(dims, n_dims);
  int mx = or_max_dim(dims, n_dims);
#pragma omp parallel
  {
    double *act = (double *)malloc(sizeof(double) * alen);
    double *actm = (double *)malloc(sizeof(double) * alen);
    double *dm = (double *)malloc(sizeof(double) * mx);
    double *dinm = (double *)malloc(sizeof(double) * mx);
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      const float *x = xyz + 3 * i;
      or_point_dfmag(L, F, log2T, res, dims, n_dims, params, x, dy_mag[i], masked, NULL, act, actm, dm, dinm);
      double gx[3] = {0.0, 0.0, 0.0};
      for (int l = 0; l < L; ++l) {
        int64_t c[3]; double w[3];
        for (int a = 0; a < 3; ++a) or_cell(x[a], res[l], &c[a], &w[a]);
        for (int d = 0; d < 8; ++d) {
          int dd[3] = {d & 1, (d >> 1) & 1, (d >> 2) & 1};
          uint32_t h = or_hash(c[0] + dd[0], c[1] + dd[1], c[2] + dd[2], T);
          const double *e = params + ((int64_t)l * T + h) * F;
          double dot = 0.0;
          for (int j = 0; j < F; ++j) dot += fabs(e[j]) * dm[l * F + j];
          for (int a = 0; a < 3; ++a) {
            double dw = 1.0;
            for (int o = 0; o < 3; ++o)
              if (o != a) dw *= dd[o] ? w[o] : 1.0 - w[o];
            gx[a] += (double)res[l] * dw * dot;
          }
        }
      }
      for (int a = 0; a < 3; ++a) dxyz_mag[3 * i + a] = gx[a];
    }
    free(act); free(actm); free(dm); free(dinm);
  }
}

/* A-8: textbook Adam (Kingma & Ba), as the paper's optimizer (Sec. 3.1, App. B),
 * dense over every parameter, bias-corrected, step t counted from 1.  l2 is the
 * weight-decay term added to the gradient before the moments. */
void or_adam(double *p, const double *g, double *m, double *v, int64_t n, int t,
             double lr, double b1, double b2, double eps, double l2) {
  double bc1 = 1.0 - pow(b1, (double)t), bc2 = 1.0 - pow(b2, (double)t);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double gi = g[i] + l2 * p[i];
    m[i] = b1 * m[i] + (1.0 - b1) * gi;
    v[i] = b2 * v[i] + (1.0 - b2) * gi * gi;
    double mh = m[i] / bc1, vh = v[i] / bc2;
    p[i] -= lr * mh / (sqrt(vh) + eps);
  }
}

/* One training step (Sec. 4): forward on the batch, loss (l1 == 0: L2 with
 * dL/dy = 2 (y - t) / n; l1 != 0: L1 with dL/dy = sign(y - t) / n), backward,
 * Adam at step t (counted from 1) with the learning rate or_lr_at(lr, t - 1,
 * ...).  grads is scratch of the params' size and is left holding this step's
 * gradient.  Returns the loss before the update. */
double or_train_step(int L, int F, int log2T, const int *res, const int *dims, int n_dims,
                     double *params, double *grads, double *m, double *v, int64_t n_params,
                     const float *xyz, const float *target, int64_t n, int t,
                     double lr, double b1, double b2, double eps, double l2,
                     int l1, int decay_start, int decay_interval, double decay_base) {
  double *y = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
  double *dy = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
  or_forward(L, F, log2T, res, dims, n_dims, params, xyz, n, y);
  double loss = l1 ? or_loss_l1(y, target, n) : or_loss_l2(y, target, n);
  for (int64_t i = 0; i < n; ++i) {
    double d = y[i] - (double)target[i];
    dy[i] = l1 ? (double)((d > 0.0) - (d < 0.0)) / (double)n : 2.0 * d / (double)n;
  }
  memset(grads, 0, sizeof(double) * n_params);
  or_backward(L, F, log2T, res, dims, n_dims, params, xyz, n, dy, grads);
  or_adam(params, grads, m, v, n_params, t, or_lr_at(lr, t - 1, decay_start, decay_interval, decay_base),
          b1, b2, eps, l2);
  free(y); free(dy);
  return loss;
}

/* ------------------------------------------------------------- sampling -- */

/* Philox4x32-10 counter-based generator from its published definition
 * (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64 multiplies
 * with the round multipliers 0xD2511F53 / 0xCD9E8D57, the key bumped by the
 * Weyl constants 0x9E3779B9 / 0xBB67AE85 between rounds. */
void or_philox4x32_10(const uint32_t *ctr_in, const uint32_t *key_in, uint32_t *out) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Sec. 4: a training batch of uniform coordinates in [0,1)^3.  Point i of
 * step s draws Philox with counter (i lo, i hi, s, 0) and key (seed lo, seed
 * hi); each of the first three words becomes (u >> 8) * 2^-24. */
void or_sample_points(uint64_t seed, uint32_t step, int64_t first, int64_t n, float *xyz) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int64_t i = 0; i < n; ++i) {
    uint64_t id = (uint64_t)(first + i);
    uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), step, 0u}, u[4];
    or_philox4x32_10(ctr, key, u);
    for (int a = 0; a < 3; ++a) xyz[3 * i + a] = (float)(u[a] >> 8) * (1.0f / 16777216.0f);
  }
}

/* Sec. 4 / Sec. 4.1: the ground-truth value at x, interpolated trilinearly
 * from the voxel and its neighbours.  Voxels are cell centred: q = x*n - 0.5
 * (FP32, the cell decision), clamped to [0, n-1]; the lower index is capped at
 * n-2 so the upper one stays inside, and the blend is FP64. */
static void or_voxel_axis(float x, int nvox, int *i0, double *w) {
  if (nvox == 1) { *i0 = 0; *w = 0.0; return; }
  float q = x * (float)nvox;
  q = q - 0.5f;
  if (q < 0.0f) q = 0.0f;
  if (q > (float)(nvox - 1)) q = (float)(nvox - 1);
  int i = (int)floorf(q);
  if (i > nvox - 2) i = nvox - 2;
  *i0 = i;
  *w = (double)q - (double)i;
}

double or_trilinear_point(const float *vol, int nx, int ny, int nz, const float *x) {
  int i0[3]; double w[3];
  or_voxel_axis(x[0], nx, &i0[0], &w[0]);
  or_voxel_axis(x[1], ny, &i0[1], &w[1]);
  or_voxel_axis(x[2], nz, &i0[2], &w[2]);
  double s = 0.0;
  for (int d = 0; d < 8; ++d) {
    int dx = d & 1, dy = (d >> 1) & 1, dz = (d >> 2) & 1;
    int ix = i0[0] + (nx > 1 ? dx : 0), iy = i0[1] + (ny > 1 ? dy : 0), iz = i0[2] + (nz > 1 ? dz : 0);
    double wt = (dx ? w[0] : 1.0 - w[0]) * (dy ? w[1] : 1.0 - w[1]) * (dz ? w[2] : 1.0 - w[2]);
    s += wt * (double)vol[((int64_t)iz * ny + iy) * nx + ix];
  }
  return s;
}

void or_trilinear(const float *vol, int nx, int ny, int nz, const float *xyz, int64_t n, double *out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = or_trilinear_point(vol, nx, ny, nz, xyz + 3 * i);
}

/* --------------------------------------------------------- macrocells -- */

/* Sec. 5.3: disjoint macrocells of Ng^3 voxels over the volume (the grid may
 * overhang it).  Each holds the value range of the voxels a trilinear lookup
 * inside the cell can touch (voxels Ng*c - 1 .. Ng*c + Ng, clamped) and the
 * largest opacity mu_max the transfer function reaches on that range: the
 * maximum LUT alpha over entries floor(255*min) .. ceil(255*max) (FP32
 * products, the index decision). */
/* Largest LUT opacity over the entries a value range [vmin, vmax] can reach
 * (Sec. 5.3): entries floor(255 vmin) .. ceil(255 vmax) after clamping to
 * [0, 1], FP32 products (the index decision).  An empty range (vmin > vmax,
 * e.g. +inf / -inf) covers no entry and gives 0. */
static float or_mu_of_range(float vmin, float vmax, const float *lut) {
  float a0 = vmin < 0.0f ? 0.0f : (vmin > 1.0f ? 1.0f : vmin);
  float a1 = vmax < 0.0f ? 0.0f : (vmax > 1.0f ? 1.0f : vmax);
  int e0 = (int)floorf(a0 * 255.0f), e1 = (int)ceilf(a1 * 255.0f);
  if (e1 > 255) e1 = 255;
  float mu = 0.0f;
  for (int e = e0; e <= e1; ++e) if (lut[4 * e + 3] > mu) mu = lut[4 * e + 3];
  return mu;
}

void or_macrocells(const float *vol, int nx, int ny, int nz, int Ng, const float *lut,
                   float *minmax, float *mumax) {
  int ncx = (nx + Ng - 1) / Ng, ncy = (ny + Ng - 1) / Ng, ncz = (nz + Ng - 1) / Ng;
  for (int cz = 0; cz < ncz; ++cz)
    for (int cy = 0; cy < ncy; ++cy)
      for (int cx = 0; cx < ncx; ++cx) {
        int lo[3] = {cx * Ng - 1, cy * Ng - 1, cz * Ng - 1};
        int hi[3] = {cx * Ng + Ng, cy * Ng + Ng, cz * Ng + Ng};
        int nn[3] = {nx, ny, nz};
        for (int a = 0; a < 3; ++a) {
          if (lo[a] < 0) lo[a] = 0;
          if (hi[a] > nn[a] - 1) hi[a] = nn[a] - 1;
        }
        float vmin = INFINITY, vmax = -INFINITY;
        for (int z = lo[2]; z <= hi[2]; ++z)
          for (int y = lo[1]; y <= hi[1]; ++y)
            for (int x = lo[0]; x <= hi[0]; ++x) {
              float v = vol[((int64_t)z * ny + y) * nx + x];
              if (v < vmin) vmin = v;
              if (v > vmax) vmax = v;
            }
        int64_t c = ((int64_t)cz * ncy + cy) * ncx + cx;
        minmax[2 * c] = vmin;
        minmax[2 * c + 1] = vmax;
        mumax[c] = or_mu_of_range(vmin, vmax, lut);
      }
}

/* Online macrocells (Sec. 5.3): the value ranges are grown from the training
 * samples themselves instead of a pass over the voxels.  Sample i at position
 * xyz[i] (unit box) with value val[i] widens the range of the macrocell that
 * contains the position, cell index floor(fl32(x * fl32(n / Ng))) per axis
 * clamped to the grid -- the mapping the ray march uses to look cells up.
 * minmax [nc][2] is updated in place (start from +inf / -inf: empty). */
void or_mc_online_update(const float *xyz, const float *val, int64_t n, int nx, int ny, int nz, int Ng,
                         float *minmax) {
  int nc[3] = {(nx + Ng - 1) / Ng, (ny + Ng - 1) / Ng, (nz + Ng - 1) / Ng};
  float sc[3] = {(float)nx / (float)Ng, (float)ny / (float)Ng, (float)nz / (float)Ng};
  for (int64_t i = 0; i < n; ++i) {
    int c[3];
    for (int a = 0; a < 3; ++a) {
      c[a] = (int)floorf(xyz[3 * i + a] * sc[a]);
      if (c[a] < 0) c[a] = 0;
      if (c[a] > nc[a] - 1) c[a] = nc[a] - 1;
    }
    int64_t k = ((int64_t)c[2] * nc[1] + c[1]) * nc[0] + c[0];
    if (val[i] < minmax[2 * k]) minmax[2 * k] = val[i];
    if (val[i] > minmax[2 * k + 1]) minmax[2 * k + 1] = val[i];
  }
}

/* mu_max of every macrocell from its value range (or_mu_of_range). */
void or_mc_mu(const float *minmax, int64_t ncells, const float *lut, float *mumax) {
  for (int64_t c = 0; c < ncells; ++c) mumax[c] = or_mu_of_range(minmax[2 * c], minmax[2 * c + 1], lut);
}

/* ----------------------------------------------------------- renderer -- */

typedef struct {
  float eye[3], target[3], up[3];
  float tan_half_fovy; /* > 0: perspective; 0: orthographic */
  float ortho_w, ortho_h;
  int width, height;
} or_camera;

typedef struct {
  float step;      /* sample spacing along the ray, in units of the unit box */
  float alpha_exp; /* opacity-correction exponent: step / s1 */
  float et;        /* early-termination opacity */
  int mc_cell;     /* macrocell size in voxels (0: no empty-space skipping) */
  float step_max;  /* > 0: adaptive step (Sec. 5.3) between step and step_max; needs macrocells */
  int shade;       /* 0: emission-absorption; 1: single-shot heuristic shadows */
  float light[3];  /* unit direction towards the directional light (shade 1) */
  float ambient;   /* shade 1: colour scale where the light is fully blocked */
} or_opts;

/* One step of the adaptive ray march (Sec. 5.3, Eq. 3) in FP32, every
 * operation rounded on its own.  From the ray parameter *t, in the macrocell
 * c holding o + (t + s1 / 1024) d: the segment runs to the nearest of the
 * cell's exit, t1 and t + s_bar, s_bar = max(s1 + (s2 - s1) (1 - min(mu_c,
 * 1))^2, s1) with p = 2 (readings: the step is taken from the cell the segment
 * starts in -- looked up just past the start, so a ray standing on a face
 * moves on into the next cell -- a segment never crosses a cell face, the
 * sample sits at its midpoint, and a segment is at least s1 / 1024 long).  A
 * cell with mu_c = 0 is
 * crossed without a sample.  Returns 0 at the end of the ray (t >= t1), 2 for
 * a crossed transparent cell, 1 for a sample at pos whose opacity exponent is
 * *e = alpha_exp * seg / s1; *t moves to the end of the segment. */
int or_march_adaptive_step(const float *o, const float *d, float t1, float s1, float s2, float alpha_exp,
                           const float *mumax, int ncx, int ncy, int ncz, float sx, float sy, float sz,
                           float *t, float *pos, float *e) {
  if (!(*t < t1)) return 0;
  float tiny = s1 * 0.0009765625f;
  float tc = *t + tiny;
  float p[3];
  for (int a = 0; a < 3; ++a) { float m = tc * d[a]; p[a] = o[a] + m; }
  int nc[3] = {ncx, ncy, ncz};
  float sc[3] = {sx, sy, sz};
  int c[3];
  for (int a = 0; a < 3; ++a) {
    c[a] = (int)floorf(p[a] * sc[a]);
    if (c[a] < 0) c[a] = 0;
    if (c[a] > nc[a] - 1) c[a] = nc[a] - 1;
  }
  float texit = INFINITY;
  for (int a = 0; a < 3; ++a) {
    float face;
    if (d[a] > 0.f) face = (float)(c[a] + 1) / sc[a];
    else if (d[a] < 0.f) face = (float)c[a] / sc[a];
    else continue;
    float num = face - o[a];
    float ta = num / d[a];
    texit = fminf(texit, ta);
  }
  texit = fminf(texit, t1);
  float room = texit - *t;
  if (!(room > tiny)) room = tiny;
  float mu = mumax[((int64_t)c[2] * ncy + c[1]) * ncx + c[0]];
  if (mu == 0.0f) { *t = *t + room; return 2; }
  float q = 1.0f - fminf(mu, 1.0f);
  float q2 = q * q;
  float ds = s2 - s1;
  float grow = ds * q2;
  float sbar = fmaxf(s1 + grow, s1);
  float seg = fminf(sbar, room);
  float half = 0.5f * seg;
  float tm = *t + half;
  for (int a = 0; a < 3; ++a) { float m = tm * d[a]; pos[a] = o[a] + m; }
  float ratio = seg / s1;
  *e = alpha_exp * ratio;
  *t = *t + seg;
  return 1;
}

/* A-11: the ray through the centre of pixel (px, py), FP32 operation by
 * operation (it decides the sample positions).  forward = normalize(target -
 * eye); right = normalize(up x forward); up' = forward x right; pixel
 * coordinates u = 2(px+0.5)/W - 1, v = 1 - 2(py+0.5)/H. */
static void or_norm3(float *a) {
  float s = a[0] * a[0];
  s = s + a[1] * a[1];
  s = s + a[2] * a[2];
  float len = sqrtf(s);
  a[0] = a[0] / len; a[1] = a[1] / len; a[2] = a[2] / len;
}

static void or_cross(const float *a, const float *b, float *c) {
  float t0 = a[1] * b[2], t1 = a[2] * b[1];
  c[0] = t0 - t1;
  t0 = a[2] * b[0]; t1 = a[0] * b[2];
  c[1] = t0 - t1;
  t0 = a[0] * b[1]; t1 = a[1] * b[0];
  c[2] = t0 - t1;
}

static void or_ray(const or_camera *cam, int px, int py, float *o, float *d) {
  float fw[3] = {cam->target[0] - cam->eye[0], cam->target[1] - cam->eye[1], cam->target[2] - cam->eye[2]};
  or_norm3(fw);
  float rt[3], up2[3];
  or_cross(cam->up, fw, rt);
  or_norm3(rt);
  or_cross(fw, rt, up2);
  float u = (2.0f * ((float)px + 0.5f)) / (float)cam->width - 1.0f;
  float v = 1.0f - (2.0f * ((float)py + 0.5f)) / (float)cam->height;
  if (cam->tan_half_fovy > 0.0f) {
    float aspect = (float)cam->width / (float)cam->height;
    float su = u * cam->tan_half_fovy;
    su = su * aspect;
    float sv = v * cam->tan_half_fovy;
    for (int a = 0; a < 3; ++a) {
      float t0 = su * rt[a];
      float t1 = sv * up2[a];
      float s = fw[a] + t0;
      d[a] = s + t1;
      o[a] = cam->eye[a];
    }
    or_norm3(d);
  } else {
    float hu = u * cam->ortho_w;
    hu = hu * 0.5f;
    float hv = v * cam->ortho_h;
    hv = hv * 0.5f;
    for (int a = 0; a < 3; ++a) {
      float t0 = hu * rt[a];
      float t1 = hv * up2[a];
      float s = cam->eye[a] + t0;
      o[a] = s + t1;
      d[a] = fw[a];
    }
  }
}

/* A-11: slab test against [0,1]^3, clipped to t >= 0 (FP32; NaN from 0*inf is
 * ignored by fminf/fmaxf). */
static int or_box(const float *o, const float *d, float *t0, float *t1) {
  float tn = 0.0f, tf = INFINITY;
  for (int a = 0; a < 3; ++a) {
    float inv = 1.0f / d[a];
    float ta = (0.0f - o[a]) * inv;
    float tb = (1.0f - o[a]) * inv;
    tn = fmaxf(tn, fminf(ta, tb));
    tf = fminf(tf, fmaxf(ta, tb));
  }
  *t0 = tn; *t1 = tf;
  return tn < tf;
}

/* A-14: transfer-function lookup, linear between the 256 LUT entries. */
static void or_tf(const float *lut, double v, double *rgba) {
  double u = (v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v)) * 255.0;
  int i = (int)floor(u);
  if (i > 254) i = 254;
  double w = u - (double)i;
  for (int c = 0; c < 4; ++c) rgba[c] = (1.0 - w) * (double)lut[4 * i + c] + w * (double)lut[4 * (i + 1) + c];
}

/* Magnitudes of or_tf's output for a value of magnitude vm: the two LUT terms
 * plus the slope of the piece times vm (taken whether or not v was clamped:
 * a value at the clamp may fall either side of it). */
static void or_tf_mag(const float *lut, double v, double vm, double *rgbam) {
  double u = (v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v)) * 255.0;
  int i = (int)floor(u);
  if (i > 254) i = 254;
  double w = u - (double)i;
  for (int c = 0; c < 4; ++c) {
    double l0 = (double)lut[4 * i + c], l1 = (double)lut[4 * (i + 1) + c];
    rgbam[c] = (1.0 - w) * fabs(l0) + w * fabs(l1) + 255.0 * fabs(l1 - l0) * vm;
  }
}

/* What one sample sees: the network (use_net) or the raw volume by trilinear
 * interpolation. */
typedef struct {
  int use_net, L, F, log2T;
  const int *res, *dims;
  int n_dims;
  const double *params, *weights;
  const float *vol;
  int nx, ny, nz;
  const float *mumax;
  int Ng, ncx, ncy, ncz;
  float sx, sy, sz;
} or_field;

static double or_field_value(const or_field *f, const float *pos, double *act) {
  if (f->use_net) {
    or_encode_point(f->L, f->F, f->log2T, f->res, f->params, pos, act);
    return or_mlp_point(f->dims, f->n_dims, f->weights, act);
  }
  return or_trilinear_point(f->vol, f->nx, f->ny, f->nz, pos);
}

/* The same value with its magnitude *vm: the network's (or_mlp_point_mag) or,
 * for the raw volume, the trilinear sum of |voxel| (actm: NULL for the raw
 * volume). */
static double or_field_value_mag(const or_field *f, const float *pos, double *act, double *actm, double *vm) {
  if (f->use_net) {
    double kink;
    or_encode_point_mag(f->L, f->F, f->log2T, f->res, f->params, pos, act, actm);
    return or_mlp_point_mag(f->dims, f->n_dims, f->weights, act, actm, vm, &kink);
  }
  int i0[3]; double w[3];
  or_voxel_axis(pos[0], f->nx, &i0[0], &w[0]);
  or_voxel_axis(pos[1], f->ny, &i0[1], &w[1]);
  or_voxel_axis(pos[2], f->nz, &i0[2], &w[2]);
  double m = 0.0;
  for (int d = 0; d < 8; ++d) {
    int dx = d & 1, dy = (d >> 1) & 1, dz = (d >> 2) & 1;
    int ix = i0[0] + (f->nx > 1 ? dx : 0), iy = i0[1] + (f->ny > 1 ? dy : 0), iz = i0[2] + (f->nz > 1 ? dz : 0);
    double wt = (dx ? w[0] : 1.0 - w[0]) * (dy ? w[1] : 1.0 - w[1]) * (dz ? w[2] : 1.0 - w[2]);
    m += wt * fabs((double)f->vol[((int64_t)iz * f->ny + iy) * f->nx + ix]);
  }
  *vm = m;
  return or_trilinear_point(f->vol, f->nx, f->ny, f->nz, pos);
}

/* The march of one ray from t0 to t1 (Sec. 5.2.1, 5.3).  Fixed step: samples
 * at t_k = t0 + (k + 1/2) step while t_k < t1, a sample whose macrocell has
 * mu_max == 0 skipped, opacity exponent alpha_exp.  Adaptive step
 * (step_max > 0): the segments of or_march_adaptive_step.  Each sample's LUT
 * opacity a is corrected to a' = 1 - (1 - a)^e.  transmit == 0: front-to-back
 * compositing C += (1 - A) a' rgb, A += (1 - A) a', stop once A >= et; the
 * sample with the largest contribution (1 - A) a' (the first of equals) is
 * returned in best_pos / *best_w.  transmit != 0: only the opacity, A = 1 - T
 * with T the product of (1 - a'), same stop. */
static void or_march(const or_field *f, const float *lut, const or_opts *opt, const float *o, const float *d,
                     float t0, float t1, int transmit, double *act, double *C, double *A, float *best_pos,
                     double *best_w, double *actm, double *Cm, double *Am) {
  double Ca[3] = {0, 0, 0}, Aa = 0.0, bw = 0.0;
  double Cma[3] = {0, 0, 0}, Ama = 0.0;
  float t = t0;
  for (int64_t k = 0;; ++k) {
    float pos[3];
    double e = (double)opt->alpha_exp;
    if (opt->step_max > 0.0f) {
      float ef;
      int r = or_march_adaptive_step(o, d, t1, opt->step, opt->step_max, opt->alpha_exp, f->mumax, f->ncx,
                                     f->ncy, f->ncz, f->sx, f->sy, f->sz, &t, pos, &ef);
      if (r == 0) break;
      if (r == 2) continue;
      e = (double)ef;
    } else {
      float tk = ((float)k + 0.5f) * opt->step;
      tk = t0 + tk;
      if (!(tk < t1)) break;
      for (int a = 0; a < 3; ++a) { float s = tk * d[a]; pos[a] = o[a] + s; }
      if (f->Ng > 0) {
        int cx = (int)floorf(pos[0] * f->sx), cy = (int)floorf(pos[1] * f->sy), cz = (int)floorf(pos[2] * f->sz);
        cx = cx < 0 ? 0 : (cx > f->ncx - 1 ? f->ncx - 1 : cx);
        cy = cy < 0 ? 0 : (cy > f->ncy - 1 ? f->ncy - 1 : cy);
        cz = cz < 0 ? 0 : (cz > f->ncz - 1 ? f->ncz - 1 : cz);
        if (f->mumax[((int64_t)cz * f->ncy + cy) * f->ncx + cx] == 0.0f) continue;
      }
    }
    double c[4], cm[4], vm = 0.0;
    double v = Am ? or_field_value_mag(f, pos, act, actm, &vm) : or_field_value(f, pos, act);
    or_tf(lut, v, c);
    double a = 1.0 - pow(1.0 - c[3], e);
    double w = (1.0 - Aa) * a;
    if (Am) {
      /* magnitudes: a' = 1 - (1 - a)^e has slope e (1 - a)^(e - 1) (infinite at
       * a = 1 for e < 1); w = (1 - A) a'; C and A sum the w terms */
      or_tf_mag(lut, v, vm, cm);
      double slope = (c[3] < 1.0) ? e * pow(1.0 - c[3], e - 1.0) : (e == 1.0 ? 1.0 : (e > 1.0 ? 0.0 : INFINITY));
      double am = a + slope * cm[3];
      double wm = ((1.0 - Aa) + Ama) * am;
      if (!transmit)
        for (int ch = 0; ch < 3; ++ch) Cma[ch] += wm * cm[ch];
      Ama += wm;
    }
    if (!transmit) {
      for (int ch = 0; ch < 3; ++ch) Ca[ch] += w * c[ch];
      if (w > bw) {
        bw = w;
        for (int q = 0; q < 3; ++q) best_pos[q] = pos[q];
      }
    }
    Aa += w;
    if (Aa >= (double)opt->et) break;
  }
  for (int ch = 0; ch < 3; ++ch) C[ch] = Ca[ch];
  *A = Aa;
  if (best_w) *best_w = bw;
  if (Am) {
    if (Cm)
      for (int ch = 0; ch < 3; ++ch) Cm[ch] = Cma[ch];
    *Am = Ama;
  }
}

/* Sec. 5, 5.2.1, 5.3: the ray march of selected pixels, one ray at a time, every
 * sample evaluated in order (the straightforward march the streaming renderer
 * is compared against, as the paper checks its streaming path against a
 * megakernel).  shade 0: emission-absorption (or_march).  shade 1:
 * single-shot heuristic shadows (Sec. 5: shading only at the point of highest
 * contribution): after the primary march, a second march from that point
 * towards the directional light (light = unit direction to it, clipped to the
 * volume box, same sampling and opacity rules) gives its transmittance T, and
 * the colour becomes C (ambient + (1 - ambient) T); A is kept.  A ray with no
 * contribution casts no shadow ray. */
void or_render_pixels(const or_camera *cam, const float *lut, const or_opts *opt,
                      int use_net, int L, int F, int log2T, const int *res, const int *dims, int n_dims,
                      const double *params,
                      const float *vol, int nx, int ny, int nz, const float *mumax,
                      const int64_t *pix, int64_t npix, double *rgba_out, double *mag_out) {
  or_field f;
  memset(&f, 0, sizeof(f));
  f.use_net = use_net; f.L = L; f.F = F; f.log2T = log2T; f.res = res; f.dims = dims; f.n_dims = n_dims;
  f.params = params;
  f.weights = use_net ? params + (int64_t)L * ((int64_t)1 << log2T) * F : NULL;
  f.vol = vol; f.nx = nx; f.ny = ny; f.nz = nz; f.mumax = mumax;
  f.Ng = opt->mc_cell;
  f.ncx = f.ncy = f.ncz = 1;
  if (f.Ng > 0) {
    f.ncx = (nx + f.Ng - 1) / f.Ng; f.ncy = (ny + f.Ng - 1) / f.Ng; f.ncz = (nz + f.Ng - 1) / f.Ng;
    f.sx = (float)nx / (float)f.Ng; f.sy = (float)ny / (float)f.Ng; f.sz = (float)nz / (float)f.Ng;
  }
  int alen = use_net ? or_act_len(dims, n_dims) : 1;
#pragma omp parallel
  {
    double *act = (double *)malloc(sizeof(double) * alen);
    double *actm = (double *)malloc(sizeof(double) * alen);
#pragma omp for schedule(dynamic, 16)
    for (int64_t q = 0; q < npix; ++q) {
      int64_t p = pix[q];
      int px = (int)(p % cam->width), py = (int)(p / cam->width);
      float o[3], d[3], t0, t1;
      double C[3] = {0, 0, 0}, A = 0.0, Cm[3] = {0, 0, 0}, Am = 0.0;
      double *am = mag_out ? &Am : NULL;
      or_ray(cam, px, py, o, d);
      if (or_box(o, d, &t0, &t1)) {
        float best[3] = {0, 0, 0};
        double bw = 0.0;
        or_march(&f, lut, opt, o, d, t0, t1, 0, act, C, &A, best, &bw, actm, Cm, am);
        if (opt->shade == 1 && bw > 0.0) {
          float s0, s1;
          double Cs[3], As = 0.0, Asm = 0.0;
          if (or_box(best, opt->light, &s0, &s1))
            or_march(&f, lut, opt, best, opt->light, s0, s1, 1, act, Cs, &As, NULL, NULL, actm, NULL,
                     mag_out ? &Asm : NULL);
          double amb = (double)opt->ambient;
          double k = amb + (1.0 - amb) * (1.0 - As);
          double km = amb + (1.0 - amb) * ((1.0 - As) + Asm);
          for (int ch = 0; ch < 3; ++ch) { C[ch] *= k; Cm[ch] *= km; }
        }
      }
      rgba_out[4 * q + 0] = C[0];
      rgba_out[4 * q + 1] = C[1];
      rgba_out[4 * q + 2] = C[2];
      rgba_out[4 * q + 3] = A;
      if (mag_out) {
        for (int ch = 0; ch < 3; ++ch) mag_out[4 * q + ch] = Cm[ch];
        mag_out[4 * q + 3] = Am;
      }
    }
    free(act); free(actm);
  }
}

/* Exit distance of the ray o + t d (o inside the unit box) through the box,
 * by the renderer's slab test; -1 if the test finds no interval. */
float or_box_exit(const float *o, const float *d) {
  float t0, t1;
  return or_box(o, d, &t0, &t1) ? t1 : -1.0f;
}

/* Ray geometry of one pixel, exposed so tests can pin the camera model. */
int or_pixel_ray(const or_camera *cam, int px, int py, float *o, float *d, float *t01) {
  or_ray(cam, px, py, o, d);
  return or_box(o, d, &t01[0], &t01[1]);
}

/* ------------------------------------------------------------- quality -- */

/* A-16: mean squared error in FP64 and PSNR with peak 1 (Sec. 7: PSNR of the
 * decoded volume and of rendered images). */
double or_mse(const double *a, const double *b, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) { double d = a[i] - b[i]; s += d * d; }
  return n > 0 ? s / (double)n : 0.0;
}

double or_psnr(double mse) { return 10.0 * log10(1.0 / mse); }

/* Sec. 5 / Sec. 7: decode the network at every voxel centre (i + 1/2)/n
 * (FP32 division, the position), and the MSE against the raw volume. */
double or_volume_mse(int L, int F, int log2T, const int *res, const int *dims, int n_dims,
                     const double *params, const float *vol, int nx, int ny, int nz) {
  int64_t T = (int64_t)1 << log2T;
  const double *weights = params + (int64_t)L * T * F;
  int alen = or_act_len(dims, n_dims);
  int64_t nvox = (int64_t)nx * ny * nz;
  double total = 0.0;
#pragma omp parallel reduction(+ : total)
  {
    double *act = (double *)malloc(sizeof(double) * alen);
#pragma omp for schedule(static)
    for (int64_t i = 0; i < nvox; ++i) {
      int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / ((int64_t)nx * ny));
      float x[3] = {((float)ix + 0.5f) / (float)nx, ((float)iy + 0.5f) / (float)ny, ((float)iz + 0.5f) / (float)nz};
      or_encode_point(L, F, log2T, res, params, x, act);
      double yv = or_mlp_point(dims, n_dims, weights, act);
      double dlt = yv - (double)vol[i];
      total += dlt * dlt;
    }
    free(act);
  }
  return nvox > 0 ? total / (double)nvox : 0.0;
}

/* ------------------------------------------------------- out of core -- */

/* Sec. 4.1 (out-of-core sampling): a training point is drawn from one of the R
 * blocks resident in the ring: pick a slot, pick a voxel of that block, jitter
 * the voxel centre by U[-0.5, 0.5] per axis; its target is the trilinear value
 * of the volume there (the block's ghost layer makes that value available
 * inside the block).  Random words: Philox4x32-10 with key (seed lo, seed hi);
 * counter (i lo, i hi, step, 1) gives u0 (slot = u0 mod R), u1 (voxel: bits
 * 0-7 / 8-15 / 16-23 mod B per axis), u2, u3 (x and y jitter); counter
 * (i lo, i hi, step, 2) gives u0 (z jitter); jitter = (u >> 8) 2^-24 - 1/2.
 * Blocks are B^3 voxels, block b = (bz nby + by) nbx + bx; slot_brick[s] is
 * the block held by slot s.  The position is (v + 1/2 + jitter) / n per axis
 * in FP32 (it decides the interpolation cell); the target is FP64. */
void or_brick_sample(const float *vol, int nx, int ny, int nz, int B, const int *slot_brick, int R,
                     uint64_t seed, uint32_t step, int64_t n, float *xyz, double *target) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  int nbx = nx / B, nby = ny / B;
  for (int64_t i = 0; i < n; ++i) {
    uint64_t id = (uint64_t)i;
    uint32_t c1[4] = {(uint32_t)id, (uint32_t)(id >> 32), step, 1u}, c2[4] = {(uint32_t)id, (uint32_t)(id >> 32), step, 2u};
    uint32_t u[4], w[4];
    or_philox4x32_10(c1, key, u);
    or_philox4x32_10(c2, key, w);
    int s = (int)(u[0] % (uint32_t)R);
    int b = slot_brick[s];
    int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
    int v[3] = {bx * B + (int)((u[1] & 255u) % (uint32_t)B), by * B + (int)(((u[1] >> 8) & 255u) % (uint32_t)B),
                bz * B + (int)(((u[1] >> 16) & 255u) % (uint32_t)B)};
    uint32_t jw[3] = {u[2], u[3], w[0]};
    int dims[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a) {
      float j = (float)(jw[a] >> 8) * (1.0f / 16777216.0f);
      j = j - 0.5f;
      float p = (float)v[a] + 0.5f;
      p = p + j;
      xyz[3 * i + a] = p / (float)dims[a];
    }
    target[i] = or_trilinear_point(vol, nx, ny, nz, xyz + 3 * i);
  }
}

/* ------------------------------------------------------- path tracing -- */

/* Volumetric path tracing (Sec. 5.2.2, Alg. 1, Eq. 1-2), one path per pixel
 * and frame, as a plain loop.  Readings (the paper names the method, not its
 * constants): extinction sigma(x) = D a(v(x)) per unit length with a the
 * transfer function's opacity and D a density scale; single-scattering albedo
 * = the transfer function's colour; isotropic phase function; one directional
 * light towards `light` whose irradiance cancels the phase factor (a visible
 * light adds throughput * albedo); the background is black.  Free flights use
 * Woodcock tracking with the majorant of each macrocell (Hofmann): the target
 * optical thickness tau = -log(1 - zeta) is spent cell by cell along the ray
 * (tau_n = sum of D mu_max_i s_i), the tentative collision is stepped back into
 * the cell where tau_n first exceeds it, and accepted with probability
 * sigma(x) / (D mu_max_cell); a null collision restarts the flight there.  At
 * every real collision a shadow ray towards the light is tracked the same way
 * (visible when it leaves the volume without a real collision), then the
 * throughput is multiplied by the albedo, Russian roulette from bounce 3
 * keeps the path with probability min(1, max throughput), and an isotropic
 * direction is drawn; paths end on leaving the volume or after max_bounces
 * real collisions.
 * Random numbers: Philox4x32-10 with key = seed and counter = (pixel, event,
 * frame, 0); every flight and every scattering event draws one block of four.
 * The branch decisions (cell walk, collision point, acceptance, roulette) are
 * taken in FP32, every operation rounded on its own, as the GPU takes them --
 * for the raw volume the density is evaluated the same way -- so both sides
 * follow the same paths; -log(1 - zeta) and the direction's trigonometry are
 * evaluated in FP64 and rounded to FP32. */

typedef struct {
  float density;     /* D */
  float light[3];    /* unit direction towards the light */
  int max_bounces;
  uint32_t seed_lo, seed_hi;
  uint32_t frame;
} or_pt_opts;

static const float OR_PT_TINY = 9.5367431640625e-07f; /* 2^-20: cell lookups just past a position */

static float or_u01(uint32_t x) { return (float)(x >> 8) * 5.9604644775390625e-08f; }

/* FP32 trilinear of the raw volume, op by op (the GPU's decision path). */
static float or_trilinear_f32(const float *vol, int nx, int ny, int nz, const float *x) {
  int n[3] = {nx, ny, nz}, i0[3], i1[3];
  float w[3];
  for (int a = 0; a < 3; ++a) {
    if (n[a] == 1) { i0[a] = 0; i1[a] = 0; w[a] = 0.0f; continue; }
    float q = x[a] * (float)n[a];
    q = q + -0.5f;
    q = fminf(fmaxf(q, 0.0f), (float)(n[a] - 1));
    int i = (int)floorf(q);
    if (i > n[a] - 2) i = n[a] - 2;
    i0[a] = i; i1[a] = i + 1;
    w[a] = q - (float)i;
  }
  const int64_t sy = nx, sz = (int64_t)nx * ny;
  float c[2][2];
  for (int zz = 0; zz < 2; ++zz)
    for (int yy = 0; yy < 2; ++yy) {
      const float *row = vol + (int64_t)(zz ? i1[2] : i0[2]) * sz + (int64_t)(yy ? i1[1] : i0[1]) * sy;
      float a0 = row[i0[0]], a1 = row[i1[0]];
      float dlt = a1 - a0;
      float m = w[0] * dlt;
      c[zz][yy] = a0 + m;
    }
  float d0 = c[0][1] - c[0][0], m0 = w[1] * d0, e0 = c[0][0] + m0;
  float d1 = c[1][1] - c[1][0], m1 = w[1] * d1, e1 = c[1][0] + m1;
  float d2 = e1 - e0, m2 = w[2] * d2;
  return e0 + m2;
}

/* FP32 transfer-function lookup, op by op: rgba of value v. */
static void or_tf_f32(const float *lut, float v, float *rgba) {
  float cv = fminf(fmaxf(v, 0.0f), 1.0f);
  float u = cv * 255.0f;
  int e = (int)floorf(u);
  if (e > 254) e = 254;
  float w = u - (float)e;
  for (int c = 0; c < 4; ++c) {
    float l0 = lut[4 * e + c], l1 = lut[4 * (e + 1) + c];
    float dl = l1 - l0, m = w * dl;
    rgba[c] = l0 + m;
  }
}

/* One Woodcock flight from parameter t (Hofmann's macrocell walk): returns 1
 * with the tentative collision parameter *tc and the majorant *mu_c of its
 * cell, or 0 when the ray leaves [t, t1] first. */
int or_pt_flight(const float *o, const float *d, float t, float t1, float tau, float D, const float *mumax,
                 int ncx, int ncy, int ncz, float sx, float sy, float sz, float *tc, float *mu_c) {
  int nc[3] = {ncx, ncy, ncz};
  float sc[3] = {sx, sy, sz};
  float acc = 0.0f;
  for (int guard = 0; guard < 1 << 20; ++guard) {
    if (!(t < t1)) return 0;
    float tl = t + OR_PT_TINY;
    int c[3];
    for (int a = 0; a < 3; ++a) {
      float m = tl * d[a];
      float p = o[a] + m;
      c[a] = (int)floorf(p * sc[a]);
      if (c[a] < 0) c[a] = 0;
      if (c[a] > nc[a] - 1) c[a] = nc[a] - 1;
    }
    float texit = INFINITY;
    for (int a = 0; a < 3; ++a) {
      float face;
      if (d[a] > 0.f) face = (float)(c[a] + 1) / sc[a];
      else if (d[a] < 0.f) face = (float)c[a] / sc[a];
      else continue;
      float num = face - o[a];
      texit = fminf(texit, num / d[a]);
    }
    texit = fminf(texit, t1);
    float seg = texit - t;
    if (!(seg > OR_PT_TINY)) seg = OR_PT_TINY;
    float mu = D * mumax[((int64_t)c[2] * ncy + c[1]) * ncx + c[0]];
    float dtau = mu * seg;
    float next = acc + dtau;
    if (mu > 0.0f && next >= tau) {
      float rem = tau - acc;
      float dt = rem / mu;
      float tcol = t + dt;
      *tc = fminf(tcol, t + seg);
      *mu_c = mu;
      return 1;
    }
    acc = next;
    t = t + seg;
  }
  return 0;
}

static void or_pt_direction(const uint32_t *u, float *d) {
  double z = 1.0 - 2.0 * (double)or_u01(u[0]);
  double r = sqrt(fmax(0.0, 1.0 - z * z));
  double phi = 6.283185307179586 * (double)or_u01(u[1]);
  d[0] = (float)(r * cos(phi));
  d[1] = (float)(r * sin(phi));
  d[2] = (float)z;
}

void or_render_pt(const or_camera *cam, const float *lut, const or_pt_opts *opt, int use_net, int L, int F,
                  int log2T, const int *res, const int *dims, int n_dims, const double *params,
                  const float *vol, int nx, int ny, int nz, const float *mumax, int Ng,
                  const int64_t *pix, int64_t npix, double *rgba_out) {
  or_field f;
  memset(&f, 0, sizeof(f));
  f.use_net = use_net; f.L = L; f.F = F; f.log2T = log2T; f.res = res; f.dims = dims; f.n_dims = n_dims;
  f.params = params;
  f.weights = use_net ? params + (int64_t)L * ((int64_t)1 << log2T) * F : NULL;
  f.vol = vol; f.nx = nx; f.ny = ny; f.nz = nz;
  int ncx = (nx + Ng - 1) / Ng, ncy = (ny + Ng - 1) / Ng, ncz = (nz + Ng - 1) / Ng;
  float sx = (float)nx / (float)Ng, sy = (float)ny / (float)Ng, sz = (float)nz / (float)Ng;
  const uint32_t key[2] = {opt->seed_lo, opt->seed_hi};
  int alen = use_net ? or_act_len(dims, n_dims) : 1;
#pragma omp parallel
  {
    double *act = (double *)malloc(sizeof(double) * alen);
#pragma omp for schedule(dynamic, 4)
    for (int64_t q = 0; q < npix; ++q) {
      int64_t p = pix[q];
      float o[3], d[3], t0, t1;
      double Lr[3] = {0, 0, 0};
      float hit = 0.0f;
      or_ray(cam, (int)(p % cam->width), (int)(p / cam->width), o, d);
      if (or_box(o, d, &t0, &t1)) {
        float beta[3] = {1.0f, 1.0f, 1.0f};
        uint32_t ev = 0;
        float t = t0;
        int bounce = 0;
        for (;;) {
          /* free flight of the scattering ray */
          uint32_t ctr[4] = {(uint32_t)p, ev++, opt->frame, 0u}, u[4];
          or_philox4x32_10(ctr, key, u);
          float tau = (float)(-log1p(-(double)or_u01(u[0])));
          float tc, muc;
          if (!or_pt_flight(o, d, t, t1, tau, opt->density, mumax, ncx, ncy, ncz, sx, sy, sz, &tc, &muc)) break;
          float x[3];
          for (int a = 0; a < 3; ++a) { float m = tc * d[a]; x[a] = o[a] + m; }
          float v = use_net ? (float)or_field_value(&f, x, act) : or_trilinear_f32(vol, nx, ny, nz, x);
          float c[4];
          or_tf_f32(lut, v, c);
          float sig = opt->density * c[3];
          float ratio = sig / muc;
          if (!(or_u01(u[1]) < ratio)) { t = tc; continue; } /* null collision */
          hit = 1.0f;
          /* next-event estimation: a shadow ray towards the light */
          float s0, s1;
          int visible = 1;
          if (or_box(x, opt->light, &s0, &s1)) {
            float ts = s0;
            for (;;) {
              uint32_t c2[4] = {(uint32_t)p, ev++, opt->frame, 0u}, w2[4];
              or_philox4x32_10(c2, key, w2);
              float tau2 = (float)(-log1p(-(double)or_u01(w2[0])));
              float tc2, mu2;
              if (!or_pt_flight(x, opt->light, ts, s1, tau2, opt->density, mumax, ncx, ncy, ncz, sx, sy, sz, &tc2,
                                &mu2))
                break;
              float y[3];
              for (int a = 0; a < 3; ++a) { float m = tc2 * opt->light[a]; y[a] = x[a] + m; }
              float v2 = use_net ? (float)or_field_value(&f, y, act) : or_trilinear_f32(vol, nx, ny, nz, y);
              float c2v[4];
              or_tf_f32(lut, v2, c2v);
              float sig2 = opt->density * c2v[3];
              float r2 = sig2 / mu2;
              if (or_u01(w2[1]) < r2) { visible = 0; break; }
              ts = tc2;
            }
          }
          if (visible)
            for (int ch = 0; ch < 3; ++ch) { float b = beta[ch] * c[ch]; Lr[ch] += (double)b; }
          for (int ch = 0; ch < 3; ++ch) beta[ch] = beta[ch] * c[ch];
          ++bounce;
          if (bounce >= opt->max_bounces) break;
          /* scattering: roulette and an isotropic direction */
          uint32_t c3[4] = {(uint32_t)p, ev++, opt->frame, 0u}, w3[4];
          or_philox4x32_10(c3, key, w3);
          if (bounce >= 3) {
            float qv = fminf(1.0f, fmaxf(beta[0], fmaxf(beta[1], beta[2])));
            if (!(or_u01(w3[2]) < qv)) break;
            for (int ch = 0; ch < 3; ++ch) beta[ch] = beta[ch] / qv;
          }
          for (int a = 0; a < 3; ++a) o[a] = x[a];
          or_pt_direction(w3, d);
          if (!or_box(o, d, &t0, &t1)) break;
          t = t0;
        }
      }
      rgba_out[4 * q + 0] = Lr[0];
      rgba_out[4 * q + 1] = Lr[1];
      rgba_out[4 * q + 2] = Lr[2];
      rgba_out[4 * q + 3] = hit;
    }
    free(act);
  }
}

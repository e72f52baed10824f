// Learned fusion cost model (not in the paper: the paper's fusion, Section
// "Quantum circuit fusion", has no cost model).  A 3-layer tanh perceptron
//   h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = w3 . h2 + b3
// predicts log(ms) of one fusion pass from its features; it is trained on the
// GPU by the kernels below (forward, per-sample backward, per-weight gradient
// sums in sample order, Adam) from timings the library's own kernel log records.
// Weights are flattened W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3.
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include "internal.h"

namespace qs {

struct MlpDims {
  int F, H;
  long long oW1, ob1, oW2, ob2, ow3, ob3, NW;
};

static MlpDims mlp_dims(int F, int H) {
  MlpDims d;
  d.F = F;
  d.H = H;
  d.oW1 = 0;
  d.ob1 = (long long)H * F;
  d.oW2 = d.ob1 + H;
  d.ob2 = d.oW2 + (long long)H * H;
  d.ow3 = d.ob2 + H;
  d.ob3 = d.ow3 + H;
  d.NW = d.ob3 + 1;
  return d;
}

// one thread per sample: activations and the prediction
__global__ void k_mlp_forward(const double* __restrict__ w, const double* __restrict__ x, long long B, MlpDims d,
                              double* __restrict__ h1, double* __restrict__ h2, double* __restrict__ y) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < B; s += (long long)gridDim.x * blockDim.x) {
    const double* xs = x + s * d.F;
    double* a1 = h1 + s * d.H;
    double* a2 = h2 + s * d.H;
    for (int i = 0; i < d.H; ++i) {
      double acc = w[d.ob1 + i];
      for (int j = 0; j < d.F; ++j) acc += w[d.oW1 + (long long)i * d.F + j] * xs[j];
      a1[i] = tanh(acc);
    }
    for (int i = 0; i < d.H; ++i) {
      double acc = w[d.ob2 + i];
      for (int j = 0; j < d.H; ++j) acc += w[d.oW2 + (long long)i * d.H + j] * a1[j];
      a2[i] = tanh(acc);
    }
    double acc = w[d.ob3];
    for (int i = 0; i < d.H; ++i) acc += w[d.ow3 + i] * a2[i];
    y[s] = acc;
  }
}

// one thread per sample: dy = (y - t) / B, d2 = dy w3 (1 - h2^2), d1 = W2^T d2 (1 - h1^2)
__global__ void k_mlp_backward(const double* __restrict__ w, const double* __restrict__ t, long long B, MlpDims d,
                               const double* __restrict__ h1, const double* __restrict__ h2, const double* __restrict__ y,
                               double* __restrict__ dy, double* __restrict__ d1, double* __restrict__ d2) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < B; s += (long long)gridDim.x * blockDim.x) {
    const double r = (y[s] - t[s]) / (double)B;
    dy[s] = r;
    const double* a1 = h1 + s * d.H;
    const double* a2 = h2 + s * d.H;
    double* e2 = d2 + s * d.H;
    double* e1 = d1 + s * d.H;
    for (int i = 0; i < d.H; ++i) e2[i] = r * w[d.ow3 + i] * (1.0 - a2[i] * a2[i]);
    for (int j = 0; j < d.H; ++j) {
      double acc = 0.0;
      for (int i = 0; i < d.H; ++i) acc += w[d.oW2 + (long long)i * d.H + j] * e2[i];
      e1[j] = acc * (1.0 - a1[j] * a1[j]);
    }
  }
}

// one thread per weight: the gradient summed over the samples in sample order
__global__ void k_mlp_weight_grads(const double* __restrict__ x, long long B, MlpDims d, const double* __restrict__ h1,
                                   const double* __restrict__ h2, const double* __restrict__ dy,
                                   const double* __restrict__ d1, const double* __restrict__ d2, double* __restrict__ g) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < d.NW; k += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    if (k < d.ob1) {
      const int i = (int)(k / d.F), j = (int)(k % d.F);
      for (long long s = 0; s < B; ++s) acc += d1[s * d.H + i] * x[s * d.F + j];
    } else if (k < d.oW2) {
      const int i = (int)(k - d.ob1);
      for (long long s = 0; s < B; ++s) acc += d1[s * d.H + i];
    } else if (k < d.ob2) {
      const int i = (int)((k - d.oW2) / d.H), j = (int)((k - d.oW2) % d.H);
      for (long long s = 0; s < B; ++s) acc += d2[s * d.H + i] * h1[s * d.H + j];
    } else if (k < d.ow3) {
      const int i = (int)(k - d.ob2);
      for (long long s = 0; s < B; ++s) acc += d2[s * d.H + i];
    } else if (k < d.ob3) {
      const int i = (int)(k - d.ow3);
      for (long long s = 0; s < B; ++s) acc += dy[s] * h2[s * d.H + i];
    } else {
      for (long long s = 0; s < B; ++s) acc += dy[s];
    }
    g[k] = acc;
  }
}

// loss = (1/B) sum (y - t)^2 / 2, one thread, sample order
__global__ void k_mlp_loss(const double* __restrict__ y, const double* __restrict__ t, long long B, double* loss) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double acc = 0.0;
    for (long long s = 0; s < B; ++s) {
      const double r = y[s] - t[s];
      acc += 0.5 * r * r;
    }
    *loss = acc / (double)B;
  }
}

// Adam (Kingma & Ba 2015) on every weight
__global__ void k_adam(double* __restrict__ w, const double* __restrict__ g, double* __restrict__ m1,
                       double* __restrict__ m2, long long NW, double lr, double b1, double b2, double eps, double c1,
                       double c2) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < NW; k += (long long)gridDim.x * blockDim.x) {
    const double gk = g[k];
    const double a = b1 * m1[k] + (1.0 - b1) * gk;
    const double v = b2 * m2[k] + (1.0 - b2) * gk * gk;
    m1[k] = a;
    m2[k] = v;
    w[k] -= lr * (a / c1) / (sqrt(v / c2) + eps);
  }
}

}  // namespace qs

using namespace qs;

struct qs_mlp {
  MlpDims d;
  double* w = nullptr;   // device weights
  double* m1 = nullptr;  // Adam moments
  double* m2 = nullptr;
  double* g = nullptr;   // gradient
  long long steps = 0;
  cudaStream_t stream = nullptr;
  // per-batch buffers (grown on demand)
  long long cap = 0;
  double *x = nullptr, *t = nullptr, *y = nullptr, *h1 = nullptr, *h2 = nullptr, *dy = nullptr, *d1 = nullptr,
         *d2 = nullptr, *loss = nullptr;
};

static void mlp_free_batch(qs_mlp* m) {
  for (double* p : {m->x, m->t, m->y, m->h1, m->h2, m->dy, m->d1, m->d2}) cudaFree(p);
  m->x = m->t = m->y = m->h1 = m->h2 = m->dy = m->d1 = m->d2 = nullptr;
  m->cap = 0;
}

static int mlp_reserve(qs_mlp* m, long long B) {
  if (B <= m->cap) return QS_OK;
  mlp_free_batch(m);
  const long long F = m->d.F, H = m->d.H;
  QS_CUDA(dmalloc(&m->x, sizeof(double) * B * F));
  QS_CUDA(dmalloc(&m->t, sizeof(double) * B));
  QS_CUDA(dmalloc(&m->y, sizeof(double) * B));
  QS_CUDA(dmalloc(&m->h1, sizeof(double) * B * H));
  QS_CUDA(dmalloc(&m->h2, sizeof(double) * B * H));
  QS_CUDA(dmalloc(&m->dy, sizeof(double) * B));
  QS_CUDA(dmalloc(&m->d1, sizeof(double) * B * H));
  QS_CUDA(dmalloc(&m->d2, sizeof(double) * B * H));
  m->cap = B;
  return QS_OK;
}

static int grid_of(long long items) { return (int)std::max<long long>(1, std::min<long long>((items + 127) / 128, 152 * 8)); }

extern "C" int qs_mlp_create(int n_in, int n_hidden, const double* weights, uint64_t seed, qs_mlp** out) {
  clear_error();
  if (!out) return fail(QS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_in < 1 || n_in > 64 || n_hidden < 1 || n_hidden > 128)
    return fail(QS_ERR_INVALID_ARG, "n_in %d / n_hidden %d outside 1..64 / 1..128", n_in, n_hidden);
  qs_mlp* m = new (std::nothrow) qs_mlp;
  if (!m) return fail(QS_ERR_OOM, "host allocation failed");
  m->d = mlp_dims(n_in, n_hidden);
  const long long NW = m->d.NW;
  std::vector<double> w0(NW);
  if (weights) {
    std::copy(weights, weights + NW, w0.begin());
  } else {
    // seeded SplitMix64 uniform init in +-1/sqrt(fan_in) (LeCun-style scale)
    uint64_t st = seed;
    auto u01 = [&]() {
      st += 0x9E3779B97F4A7C15ull;
      uint64_t z = st;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    for (long long k = 0; k < NW; ++k) {
      double fan = k < m->d.ob1 ? n_in : (k < m->d.ow3 ? n_hidden : n_hidden);
      w0[k] = (2.0 * u01() - 1.0) / sqrt(fan);
    }
    for (long long k = m->d.ob1; k < m->d.oW2; ++k) w0[k] = 0.0;
    for (long long k = m->d.ob2; k < m->d.ow3; ++k) w0[k] = 0.0;
    w0[m->d.ob3] = 0.0;
  }
  cudaError_t e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = dmalloc(&m->w, sizeof(double) * NW);
  if (e == cudaSuccess) e = dmalloc(&m->m1, sizeof(double) * NW);
  if (e == cudaSuccess) e = dmalloc(&m->m2, sizeof(double) * NW);
  if (e == cudaSuccess) e = dmalloc(&m->g, sizeof(double) * NW);
  if (e == cudaSuccess) e = dmalloc(&m->loss, sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(m->w, w0.data(), sizeof(double) * NW, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->m1, 0, sizeof(double) * NW);
  if (e == cudaSuccess) e = cudaMemset(m->m2, 0, sizeof(double) * NW);
  if (e != cudaSuccess) {
    qs_mlp_free(m);
    return cuda_fail(e, "mlp create");
  }
  *out = m;
  return QS_OK;
}

namespace qs {
int mlp_inputs(const qs_mlp* m) { return m ? m->d.F : 0; }
}  // namespace qs

extern "C" int qs_mlp_free(qs_mlp* m) {
  if (!m) return QS_OK;
  if (m->stream) cudaStreamSynchronize(m->stream);
  mlp_free_batch(m);
  for (double* p : {m->w, m->m1, m->m2, m->g, m->loss}) cudaFree(p);
  if (m->stream) cudaStreamDestroy(m->stream);
  delete m;
  return QS_OK;
}

extern "C" int qs_mlp_num_weights(const qs_mlp* m, size_t* out) {
  if (!m || !out) return fail(QS_ERR_INVALID_ARG, "NULL argument");
  *out = (size_t)m->d.NW;
  return QS_OK;
}

extern "C" int qs_mlp_get_weights(const qs_mlp* m, double* out) {
  if (!m || !out) return fail(QS_ERR_INVALID_ARG, "NULL argument");
  QS_CUDA(cudaMemcpyAsync(out, m->w, sizeof(double) * m->d.NW, cudaMemcpyDeviceToHost, m->stream));
  QS_CUDA(cudaStreamSynchronize(m->stream));
  return QS_OK;
}

extern "C" int qs_mlp_set_weights(qs_mlp* m, const double* w) {
  if (!m || !w) return fail(QS_ERR_INVALID_ARG, "NULL argument");
  QS_CUDA(cudaMemcpyAsync(m->w, w, sizeof(double) * m->d.NW, cudaMemcpyHostToDevice, m->stream));
  QS_CUDA(cudaMemsetAsync(m->m1, 0, sizeof(double) * m->d.NW, m->stream));
  QS_CUDA(cudaMemsetAsync(m->m2, 0, sizeof(double) * m->d.NW, m->stream));
  QS_CUDA(cudaStreamSynchronize(m->stream));
  m->steps = 0;
  return QS_OK;
}

static int mlp_upload(qs_mlp* m, const double* x, const double* t, long long B) {
  QS_TRY(mlp_reserve(m, B));
  QS_CUDA(cudaMemcpyAsync(m->x, x, sizeof(double) * B * m->d.F, cudaMemcpyHostToDevice, m->stream));
  if (t) QS_CUDA(cudaMemcpyAsync(m->t, t, sizeof(double) * B, cudaMemcpyHostToDevice, m->stream));
  return QS_OK;
}

static int mlp_fwd(qs_mlp* m, long long B) {
  note_launch(1);
  k_mlp_forward<<<grid_of(B), 128, 0, m->stream>>>(m->w, m->x, B, m->d, m->h1, m->h2, m->y);
  return launch_check("mlp forward");
}

static int mlp_bwd(qs_mlp* m, long long B) {
  note_launch(3);
  k_mlp_backward<<<grid_of(B), 128, 0, m->stream>>>(m->w, m->t, B, m->d, m->h1, m->h2, m->y, m->dy, m->d1, m->d2);
  k_mlp_weight_grads<<<grid_of(m->d.NW), 128, 0, m->stream>>>(m->x, B, m->d, m->h1, m->h2, m->dy, m->d1, m->d2, m->g);
  k_mlp_loss<<<1, 32, 0, m->stream>>>(m->y, m->t, B, m->loss);
  return launch_check("mlp backward");
}

extern "C" int qs_mlp_forward(qs_mlp* m, const double* x, size_t B, double* y) {
  clear_error();
  if (!m || !x || !y || B == 0) return fail(QS_ERR_INVALID_ARG, "NULL argument or empty batch");
  QS_TRY(mlp_upload(m, x, nullptr, (long long)B));
  QS_TRY(mlp_fwd(m, (long long)B));
  QS_CUDA(cudaMemcpyAsync(y, m->y, sizeof(double) * B, cudaMemcpyDeviceToHost, m->stream));
  QS_CUDA(cudaStreamSynchronize(m->stream));
  return QS_OK;
}

extern "C" int qs_mlp_loss_grad(qs_mlp* m, const double* x, const double* t, size_t B, double* loss, double* grad) {
  clear_error();
  if (!m || !x || !t || !loss || !grad || B == 0) return fail(QS_ERR_INVALID_ARG, "NULL argument or empty batch");
  QS_TRY(mlp_upload(m, x, t, (long long)B));
  QS_TRY(mlp_fwd(m, (long long)B));
  QS_TRY(mlp_bwd(m, (long long)B));
  QS_CUDA(cudaMemcpyAsync(grad, m->g, sizeof(double) * m->d.NW, cudaMemcpyDeviceToHost, m->stream));
  QS_CUDA(cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  QS_CUDA(cudaStreamSynchronize(m->stream));
  return QS_OK;
}

extern "C" int qs_mlp_train(qs_mlp* m, const double* x, const double* t, size_t B, int epochs, double lr,
                            double* final_loss) {
  clear_error();
  if (!m || !x || !t || B == 0 || epochs < 1) return fail(QS_ERR_INVALID_ARG, "bad training arguments");
  QS_TRY(mlp_upload(m, x, t, (long long)B));
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  for (int ep = 0; ep < epochs; ++ep) {
    QS_TRY(mlp_fwd(m, (long long)B));
    QS_TRY(mlp_bwd(m, (long long)B));
    ++m->steps;
    const double c1 = 1.0 - pow(b1, (double)m->steps), c2 = 1.0 - pow(b2, (double)m->steps);
    note_launch(1);
    k_adam<<<grid_of(m->d.NW), 128, 0, m->stream>>>(m->w, m->g, m->m1, m->m2, m->d.NW, lr, b1, b2, eps, c1, c2);
    QS_TRY(launch_check("adam"));
  }
  // loss of the final weights
  QS_TRY(mlp_fwd(m, (long long)B));
  QS_TRY(mlp_bwd(m, (long long)B));
  if (final_loss) {
    QS_CUDA(cudaMemcpyAsync(final_loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  }
  QS_CUDA(cudaStreamSynchronize(m->stream));
  return QS_OK;
}

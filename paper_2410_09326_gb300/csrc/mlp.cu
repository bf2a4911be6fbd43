// Learned cost model for pass selection: a 2 x 64 ReLU MLP that predicts the
// natural log of a fused block's device time (ms) from its features.
//
// The paper leaves the mapping from profile data to optimisation flags open
// and points at learned selection of compiler optimisations as the next step
// (Sec. III-A, "PGO design considerations"). Trained on block profiles the
// simulator records itself (QS_PROFILE), the network stands in for repeated
// profiling runs: candidate plans are scored by the sum of predicted block
// times without running them.
//
// Network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = w3 . h2 + b3,
// x standardised with the training set's mean / std, loss = mean squared
// error of y against standardised log-times. Training runs on the GPU with
// the kernels below (layer forward, input / weight gradients, Adam), FP32,
// no atomics (every reduction has a fixed order).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "qs_internal.h"

namespace qs {
std::string &last_error_ref();
}

namespace {

constexpr int kF = QS_MLP_FEATURES;
constexpr int kH = QS_MLP_HIDDEN;

// parameter layout inside one flat array
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kH * kF;
constexpr int kOffW2 = kOffB1 + kH;
constexpr int kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH;
constexpr int kOffB3 = kOffW3 + kH;
constexpr int kParams = kOffB3 + 1;
static_assert(kParams == QS_MLP_PARAMS, "parameter count");

// Y[b][o] = act(sum_i W[o][i] X[b][i] + bias[o]); one thread per (b, o).
__global__ void k_linear_fwd(const float *__restrict__ X, const float *__restrict__ W, const float *__restrict__ bias,
                             float *__restrict__ Y, int B, int in, int out, int relu) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * out) return;
  const int b = t / out, o = t - b * out;
  float s = bias[o];
  for (int i = 0; i < in; i++) s = fmaf(W[o * in + i], X[b * in + i], s);
  Y[t] = relu ? fmaxf(s, 0.f) : s;
}

// dY = 2 (Y - T) / B for the mean squared error; loss_part[b] = (Y - T)^2.
__global__ void k_mse_grad(const float *__restrict__ Y, const float *__restrict__ T, float *__restrict__ dY,
                           float *__restrict__ loss_part, int B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float d = Y[b] - T[b];
  dY[b] = 2.f * d / (float)B;
  loss_part[b] = d * d;
}

// dX[b][i] = (sum_o dY[b][o] W[o][i]) * (X[b][i] > 0 when the input came
// through a ReLU); one thread per (b, i).
__global__ void k_linear_bwd_data(const float *__restrict__ dY, const float *__restrict__ W,
                                  const float *__restrict__ Xact, float *__restrict__ dX, int B, int in, int out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * in) return;
  const int b = t / in, i = t - b * in;
  float s = 0.f;
  for (int o = 0; o < out; o++) s = fmaf(dY[b * out + o], W[o * in + i], s);
  dX[t] = Xact[t] > 0.f ? s : 0.f;
}

// dW[o][i] = sum_b dY[b][o] X[b][i], dbias[o] = sum_b dY[b][o]; one thread
// per weight (i == in computes the bias), samples summed in order.
__global__ void k_linear_bwd_weight(const float *__restrict__ dY, const float *__restrict__ X,
                                    float *__restrict__ dW, float *__restrict__ db, int B, int in, int out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= out * (in + 1)) return;
  const int o = t / (in + 1), i = t - o * (in + 1);
  float s = 0.f;
  if (i < in) {
    for (int b = 0; b < B; b++) s = fmaf(dY[b * out + o], X[b * in + i], s);
    dW[o * in + i] = s;
  } else {
    for (int b = 0; b < B; b++) s += dY[b * out + o];
    db[o] = s;
  }
}

// Adam (Kingma and Ba 2015) with bias correction; step is 1-based.
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int n, float lr, float b1, float b2, float eps, int step) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / (1.f - powf(b1, (float)step));
  const float vh = vi / (1.f - powf(b2, (float)step));
  p[i] -= lr * mh / (sqrtf(vh) + eps);
}

__global__ void k_gather_rows(const float *__restrict__ src, const int *__restrict__ idx, float *__restrict__ dst,
                              int rows, int cols) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * cols) return;
  const int r = t / cols, c = t - r * cols;
  dst[t] = src[(size_t)idx[r] * cols + c];
}

int blocks_for(int n) { return (n + 255) / 256; }

}  // namespace

struct qs_mlp {
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // params, grads, Adam moments
  float *x = nullptr, *t = nullptr, *h1 = nullptr, *h2 = nullptr, *y = nullptr;
  float *dy = nullptr, *dh2 = nullptr, *dh1 = nullptr, *loss = nullptr;
  float *data_x = nullptr, *data_y = nullptr;
  int *idx = nullptr;
  int cap = 0;           // batch rows the work buffers hold
  int data_cap = 0;      // dataset rows on the device
  int step = 0;
  float x_mean[kF], x_std[kF], y_mean = 0.f, y_std = 1.f;
  bool normalised = false;
  cudaStream_t stream = nullptr;
};

namespace {

qs_status mfail(qs_status s, const std::string &m) {
  qs::last_error_ref() = m;
  return s;
}

template <typename T> cudaError_t dalloc(T *&p, size_t n) {
  qs::dev_free(p);
  p = nullptr;
  return qs::dev_malloc((void **)&p, sizeof(T) * (n ? n : 1));
}

cudaError_t ensure_batch(qs_mlp *mm, int B) {
  if (B <= mm->cap) return cudaSuccess;
  cudaError_t e = dalloc(mm->x, (size_t)B * kF);
  if (e == cudaSuccess) e = dalloc(mm->t, (size_t)B);
  if (e == cudaSuccess) e = dalloc(mm->h1, (size_t)B * kH);
  if (e == cudaSuccess) e = dalloc(mm->h2, (size_t)B * kH);
  if (e == cudaSuccess) e = dalloc(mm->y, (size_t)B);
  if (e == cudaSuccess) e = dalloc(mm->dy, (size_t)B);
  if (e == cudaSuccess) e = dalloc(mm->dh2, (size_t)B * kH);
  if (e == cudaSuccess) e = dalloc(mm->dh1, (size_t)B * kH);
  if (e == cudaSuccess) e = dalloc(mm->loss, (size_t)B);
  if (e == cudaSuccess) mm->cap = B;
  return e;
}

cudaError_t forward(qs_mlp *mm, int B) {
  cudaStream_t s = mm->stream;
  const float *p = mm->p;
  k_linear_fwd<<<blocks_for(B * kH), 256, 0, s>>>(mm->x, p + kOffW1, p + kOffB1, mm->h1, B, kF, kH, 1);
  k_linear_fwd<<<blocks_for(B * kH), 256, 0, s>>>(mm->h1, p + kOffW2, p + kOffB2, mm->h2, B, kH, kH, 1);
  k_linear_fwd<<<blocks_for(B), 256, 0, s>>>(mm->h2, p + kOffW3, p + kOffB3, mm->y, B, kH, 1, 0);
  return cudaGetLastError();
}

// forward + backward of the batch in mm->x / mm->t; gradients into mm->g
cudaError_t forward_backward(qs_mlp *mm, int B) {
  cudaStream_t s = mm->stream;
  cudaError_t e = forward(mm, B);
  if (e != cudaSuccess) return e;
  const float *p = mm->p;
  float *g = mm->g;
  k_mse_grad<<<blocks_for(B), 256, 0, s>>>(mm->y, mm->t, mm->dy, mm->loss, B);
  k_linear_bwd_weight<<<blocks_for(1 * (kH + 1)), 256, 0, s>>>(mm->dy, mm->h2, g + kOffW3, g + kOffB3, B, kH, 1);
  k_linear_bwd_data<<<blocks_for(B * kH), 256, 0, s>>>(mm->dy, p + kOffW3, mm->h2, mm->dh2, B, kH, 1);
  k_linear_bwd_weight<<<blocks_for(kH * (kH + 1)), 256, 0, s>>>(mm->dh2, mm->h1, g + kOffW2, g + kOffB2, B, kH, kH);
  k_linear_bwd_data<<<blocks_for(B * kH), 256, 0, s>>>(mm->dh2, p + kOffW2, mm->h1, mm->dh1, B, kH, kH);
  k_linear_bwd_weight<<<blocks_for(kH * (kF + 1)), 256, 0, s>>>(mm->dh1, mm->x, g + kOffW1, g + kOffB1, B, kF, kH);
  return cudaGetLastError();
}

void standardise(const qs_mlp *mm, const float *x, float *out, int n) {
  for (int r = 0; r < n; r++)
    for (int f = 0; f < kF; f++) out[(size_t)r * kF + f] = (x[(size_t)r * kF + f] - mm->x_mean[f]) / mm->x_std[f];
}

}  // namespace

extern "C" {

qs_status qs_mlp_create(uint64_t seed, void *cuda_stream, qs_mlp **out) {
  if (!out) return mfail(QS_EINVAL, "qs_mlp_create: null output");
  *out = nullptr;
  qs_mlp *mm = new (std::nothrow) qs_mlp();
  if (!mm) return mfail(QS_ENOMEM, "qs_mlp_create: host allocation failed");
  mm->stream = (cudaStream_t)cuda_stream;
  for (int f = 0; f < kF; f++) {
    mm->x_mean[f] = 0.f;
    mm->x_std[f] = 1.f;
  }
  // He-uniform initial weights, zero biases, from a seeded generator
  std::vector<float> p(kParams, 0.f);
  std::mt19937_64 rng(seed);
  auto fill = [&](int off, int fan_out, int fan_in) {
    const float lim = std::sqrt(6.f / (float)fan_in);
    std::uniform_real_distribution<float> u(-lim, lim);
    for (int i = 0; i < fan_out * fan_in; i++) p[off + i] = u(rng);
  };
  fill(kOffW1, kH, kF);
  fill(kOffW2, kH, kH);
  fill(kOffW3, 1, kH);
  cudaError_t e = dalloc(mm->p, kParams);
  if (e == cudaSuccess) e = dalloc(mm->g, kParams);
  if (e == cudaSuccess) e = dalloc(mm->m, kParams);
  if (e == cudaSuccess) e = dalloc(mm->v, kParams);
  if (e == cudaSuccess) e = cudaMemcpy(mm->p, p.data(), sizeof(float) * kParams, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(mm->m, 0, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMemset(mm->v, 0, sizeof(float) * kParams);
  if (e != cudaSuccess) {
    qs_mlp_free(mm);
    return mfail(QS_ENOMEM, std::string("qs_mlp_create: ") + cudaGetErrorString(e));
  }
  *out = mm;
  return QS_OK;
}

void qs_mlp_free(qs_mlp *mm) {
  if (!mm) return;
  cudaDeviceSynchronize();
  float *bufs[] = {mm->p, mm->g, mm->m, mm->v, mm->x, mm->t, mm->h1, mm->h2, mm->y, mm->dy, mm->dh2, mm->dh1,
                   mm->loss, mm->data_x, mm->data_y};
  for (float *b : bufs) qs::dev_free(b);
  qs::dev_free(mm->idx);
  delete mm;
}

qs_status qs_mlp_params(qs_mlp *mm, float *host_out, const float *host_in) {
  if (!mm) return mfail(QS_EINVAL, "qs_mlp_params: null model");
  cudaError_t e = cudaSuccess;
  if (host_in) e = cudaMemcpy(mm->p, host_in, sizeof(float) * kParams, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && host_out) e = cudaMemcpy(host_out, mm->p, sizeof(float) * kParams, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return mfail(QS_ECUDA, std::string("qs_mlp_params: ") + cudaGetErrorString(e));
  return QS_OK;
}

qs_status qs_mlp_gradient(qs_mlp *mm, const float *x, const float *y, int n, float *grad_out, float *loss_out) {
  if (!mm || !x || !y || n <= 0 || !grad_out) return mfail(QS_EINVAL, "qs_mlp_gradient: bad arguments");
  cudaError_t e = ensure_batch(mm, n);
  if (e == cudaSuccess) e = cudaMemcpy(mm->x, x, sizeof(float) * (size_t)n * kF, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(mm->t, y, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = forward_backward(mm, n);
  if (e == cudaSuccess) e = cudaStreamSynchronize(mm->stream);
  if (e == cudaSuccess) e = cudaMemcpy(grad_out, mm->g, sizeof(float) * kParams, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && loss_out) {
    std::vector<float> l(n);
    e = cudaMemcpy(l.data(), mm->loss, sizeof(float) * n, cudaMemcpyDeviceToHost);
    double s = 0;
    for (float v : l) s += v;
    *loss_out = (float)(s / n);
  }
  if (e != cudaSuccess) return mfail(QS_ECUDA, std::string("qs_mlp_gradient: ") + cudaGetErrorString(e));
  return QS_OK;
}

qs_status qs_mlp_train(qs_mlp *mm, const float *x, const float *y, int n, int epochs, int batch, float lr,
                       uint64_t seed, float *loss_out) {
  if (!mm || !x || !y || n <= 0 || epochs <= 0 || batch <= 0) return mfail(QS_EINVAL, "qs_mlp_train: bad arguments");
  // standardisation from this training set (features and targets)
  std::vector<double> mu(kF, 0.0), var(kF, 0.0);
  double ym = 0, yv = 0;
  for (int r = 0; r < n; r++) {
    for (int f = 0; f < kF; f++) mu[f] += x[(size_t)r * kF + f];
    ym += y[r];
  }
  for (int f = 0; f < kF; f++) mu[f] /= n;
  ym /= n;
  for (int r = 0; r < n; r++) {
    for (int f = 0; f < kF; f++) {
      const double d = x[(size_t)r * kF + f] - mu[f];
      var[f] += d * d;
    }
    yv += (y[r] - ym) * (y[r] - ym);
  }
  for (int f = 0; f < kF; f++) {
    mm->x_mean[f] = (float)mu[f];
    const double sd = std::sqrt(var[f] / n);
    mm->x_std[f] = sd > 1e-6 ? (float)sd : 1.f;
  }
  mm->y_mean = (float)ym;
  mm->y_std = yv / n > 1e-12 ? (float)std::sqrt(yv / n) : 1.f;
  mm->normalised = true;
  std::vector<float> xs((size_t)n * kF), ys(n);
  standardise(mm, x, xs.data(), n);
  for (int r = 0; r < n; r++) ys[r] = (y[r] - mm->y_mean) / mm->y_std;
  const int B = std::min(batch, n);
  cudaError_t e = ensure_batch(mm, B);
  if (e == cudaSuccess && n > mm->data_cap) {
    e = dalloc(mm->data_x, (size_t)n * kF);
    if (e == cudaSuccess) e = dalloc(mm->data_y, (size_t)n);
    if (e == cudaSuccess) e = dalloc(mm->idx, (size_t)n);
    if (e == cudaSuccess) mm->data_cap = n;
  }
  if (e == cudaSuccess) e = cudaMemcpy(mm->data_x, xs.data(), sizeof(float) * xs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(mm->data_y, ys.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return mfail(QS_ECUDA, std::string("qs_mlp_train: ") + cudaGetErrorString(e));
  std::vector<int> order(n);
  for (int i = 0; i < n; i++) order[i] = i;
  std::mt19937_64 rng(seed);
  std::vector<float> lpart(B);
  double last = 0;
  for (int ep = 0; ep < epochs; ep++) {
    std::shuffle(order.begin(), order.end(), rng);
    // one upload of the epoch's sample order; the host buffer is only reused
    // after the stream has consumed it (synchronised at the end of the epoch)
    e = cudaMemcpyAsync(mm->idx, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, mm->stream);
    if (e != cudaSuccess) break;
    for (int s0 = 0; s0 + B <= n; s0 += B) {
      k_gather_rows<<<blocks_for(B * kF), 256, 0, mm->stream>>>(mm->data_x, mm->idx + s0, mm->x, B, kF);
      k_gather_rows<<<blocks_for(B), 256, 0, mm->stream>>>(mm->data_y, mm->idx + s0, mm->t, B, 1);
      e = forward_backward(mm, B);
      if (e != cudaSuccess) break;
      mm->step++;
      k_adam<<<blocks_for(kParams), 256, 0, mm->stream>>>(mm->p, mm->g, mm->m, mm->v, kParams, lr, 0.9f, 0.999f,
                                                          1e-8f, mm->step);
      e = cudaGetLastError();
      if (e != cudaSuccess) break;
    }
    if (e != cudaSuccess) break;
    if (ep == epochs - 1) {
      // loss of the last batch of the last epoch (standardised units)
      e = cudaMemcpyAsync(lpart.data(), mm->loss, sizeof(float) * B, cudaMemcpyDeviceToHost, mm->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(mm->stream);
    if (e != cudaSuccess) break;
    if (ep == epochs - 1) {
      double esum = 0;
      for (float v : lpart) esum += v;
      last = esum / B;
    }
  }
  if (e != cudaSuccess) return mfail(QS_ECUDA, std::string("qs_mlp_train: ") + cudaGetErrorString(e));
  if (loss_out) *loss_out = (float)last;
  return QS_OK;
}

qs_status qs_mlp_predict(qs_mlp *mm, const float *x, int n, float *y_out) {
  if (!mm || !x || !y_out || n < 0) return mfail(QS_EINVAL, "qs_mlp_predict: bad arguments");
  if (n == 0) return QS_OK;
  std::vector<float> xs((size_t)n * kF);
  standardise(mm, x, xs.data(), n);
  cudaError_t e = ensure_batch(mm, n);
  if (e == cudaSuccess) e = cudaMemcpyAsync(mm->x, xs.data(), sizeof(float) * xs.size(), cudaMemcpyHostToDevice, mm->stream);
  if (e == cudaSuccess) e = forward(mm, n);
  if (e == cudaSuccess) e = cudaMemcpyAsync(y_out, mm->y, sizeof(float) * n, cudaMemcpyDeviceToHost, mm->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(mm->stream);
  if (e != cudaSuccess) return mfail(QS_ECUDA, std::string("qs_mlp_predict: ") + cudaGetErrorString(e));
  for (int i = 0; i < n; i++) y_out[i] = y_out[i] * mm->y_std + mm->y_mean;
  return QS_OK;
}

}  // extern "C"

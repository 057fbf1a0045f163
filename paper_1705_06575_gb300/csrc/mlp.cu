// mlp.cu — the cost model's multilayer perceptron: forward, backward and Adam on the GPU (FP32).
//
// y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3, trained on the mean squared error against
// measured log times. Parameters live in one flat vector (W1 row-major h x nin, b1, W2 h x h,
// b2, w3, b3). Every reduction over the training rows is a fixed sequential loop per output, so
// gradients are deterministic. The network is tiny (a few thousand parameters, a few thousand
// rows): one thread per output element is enough and keeps each kernel a direct statement of
// the formula it computes.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "sym.h"

struct sym_mlp_s {
  int32_t nin = 0, h = 0;
  int64_t np = 0;
  float *theta = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
  float *work = nullptr;
  int64_t work_rows = 0;
  float *loss = nullptr;
  int64_t step = 0;
};

namespace {

constexpr int T = 256;
inline unsigned nblk(int64_t n) { return (unsigned)((n + T - 1) / T); }

// Z = X W^T + b (N x h), H = relu(Z).
__global__ void k_dense_relu(const float *__restrict__ X, int64_t N, int nin, const float *__restrict__ W,
                             const float *__restrict__ b, int h, float *__restrict__ Z, float *__restrict__ H) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * h) return;
  const int64_t i = idx / h;
  const int j = (int)(idx % h);
  float s = b[j];
  for (int k = 0; k < nin; ++k) s = fmaf(X[i * nin + k], W[(int64_t)j * nin + k], s);
  Z[idx] = s;
  H[idx] = s > 0.f ? s : 0.f;
}

// y = H w + b (one output per row).
__global__ void k_dense_out(const float *__restrict__ H, int64_t N, int h, const float *__restrict__ w,
                            const float *__restrict__ b, float *__restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  float s = b[0];
  for (int k = 0; k < h; ++k) s = fmaf(H[i * h + k], w[k], s);
  y[i] = s;
}

// dy = 2 (y - t) / N and the loss mean((y - t)^2), one block, fixed order.
__global__ void k_mse(const float *__restrict__ y, const float *__restrict__ t, int64_t N, float *__restrict__ dy,
                      float *__restrict__ loss) {
  __shared__ float sh[T];
  float s = 0.f;
  for (int64_t i = threadIdx.x; i < N; i += T) {
    const float d = y[i] - t[i];
    dy[i] = 2.f * d / (float)N;
    s = fmaf(d, d, s);
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = T / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = sh[0] / (float)N;
}

// dW[a][c] = sum_i dZ[i][a] Hin[i][c] and db[a] = sum_i dZ[i][a] (one thread per (a, c); the
// c == nin_ slot computes db).
__global__ void k_grad_dense(const float *__restrict__ dZ, const float *__restrict__ Hin, int64_t N, int hout,
                             int hin, float *__restrict__ dW, float *__restrict__ db) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)hout * (hin + 1)) return;
  const int a = (int)(idx / (hin + 1));
  const int c = (int)(idx % (hin + 1));
  float s = 0.f;
  if (c < hin) {
    for (int64_t i = 0; i < N; ++i) s = fmaf(dZ[i * hout + a], Hin[i * hin + c], s);
    dW[(int64_t)a * hin + c] = s;
  } else {
    for (int64_t i = 0; i < N; ++i) s += dZ[i * hout + a];
    db[a] = s;
  }
}

// Output layer: dw3[k] = sum_i dy[i] H2[i][k], db3 = sum_i dy[i].
__global__ void k_grad_out(const float *__restrict__ dy, const float *__restrict__ H, int64_t N, int h,
                           float *__restrict__ dw, float *__restrict__ db) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > h) return;
  float s = 0.f;
  if (k < h)
    for (int64_t i = 0; i < N; ++i) s = fmaf(dy[i], H[i * h + k], s);
  else
    for (int64_t i = 0; i < N; ++i) s += dy[i];
  if (k < h) dw[k] = s;
  else db[0] = s;
}

// dZ2[i][k] = dy[i] w3[k] [Z2 > 0].
__global__ void k_back_out(const float *__restrict__ dy, const float *__restrict__ w, const float *__restrict__ Z,
                           int64_t N, int h, float *__restrict__ dZ) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * h) return;
  dZ[idx] = Z[idx] > 0.f ? dy[idx / h] * w[idx % h] : 0.f;
}

// dZ1[i][c] = (sum_a dZ2[i][a] W2[a][c]) [Z1 > 0].
__global__ void k_back_dense(const float *__restrict__ dZ2, const float *__restrict__ W2, const float *__restrict__ Z1,
                             int64_t N, int h, float *__restrict__ dZ1) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * h) return;
  const int64_t i = idx / h;
  const int c = (int)(idx % h);
  float s = 0.f;
  for (int a = 0; a < h; ++a) s = fmaf(dZ2[i * h + a], W2[(int64_t)a * h + c], s);
  dZ1[idx] = Z1[idx] > 0.f ? s : 0.f;
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, theta -= lr mhat / (sqrt(vhat)+eps).
__global__ void k_adam(float *__restrict__ theta, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int64_t np, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  m[i] = b1 * m[i] + (1.f - b1) * g[i];
  v[i] = b2 * v[i] + (1.f - b2) * g[i] * g[i];
  theta[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
}

struct Views {
  float *W1, *b1, *W2, *b2, *w3, *b3;
};
Views views(float *p, int nin, int h) {
  Views v;
  v.W1 = p;
  v.b1 = v.W1 + (int64_t)h * nin;
  v.W2 = v.b1 + h;
  v.b2 = v.W2 + (int64_t)h * h;
  v.w3 = v.b2 + h;
  v.b3 = v.w3 + h;
  return v;
}

int ensure_work(sym_mlp_s *m, int64_t N) {
  if (N <= m->work_rows) return SYM_OK;
  if (m->work) cudaFree(m->work);
  m->work = nullptr;
  m->work_rows = 0;
  // Z1, H1, Z2, H2, dZ2, dZ1 (N x h each), y and dy (N each)
  if (cudaMalloc(&m->work, sizeof(float) * (6 * N * m->h + 2 * N)) != cudaSuccess) return SYM_ERR_OOM;
  m->work_rows = N;
  return SYM_OK;
}

// Forward pass on N rows; returns pointers into the work area.
void forward(sym_mlp_s *m, const float *X, int64_t N, float **Z1, float **H1, float **Z2, float **H2, float **y) {
  const int h = m->h;
  *Z1 = m->work;
  *H1 = *Z1 + N * h;
  *Z2 = *H1 + N * h;
  *H2 = *Z2 + N * h;
  *y = m->work + 6 * N * h;
  Views p = views(m->theta, m->nin, h);
  k_dense_relu<<<nblk(N * h), T>>>(X, N, m->nin, p.W1, p.b1, h, *Z1, *H1);
  k_dense_relu<<<nblk(N * h), T>>>(*H1, N, h, p.W2, p.b2, h, *Z2, *H2);
  k_dense_out<<<nblk(N), T>>>(*H2, N, h, p.w3, p.b3, *y);
}

// Gradient of the MSE into m->grad; loss into m->loss (device).
void backward(sym_mlp_s *m, const float *X, const float *t, int64_t N) {
  const int h = m->h;
  float *Z1, *H1, *Z2, *H2, *y;
  forward(m, X, N, &Z1, &H1, &Z2, &H2, &y);
  float *dZ2 = H2 + N * h, *dZ1 = dZ2 + N * h, *dy = y + N;
  Views p = views(m->theta, m->nin, h);
  Views g = views(m->grad, m->nin, h);
  k_mse<<<1, T>>>(y, t, N, dy, m->loss);
  k_grad_out<<<nblk(h + 1), T>>>(dy, H2, N, h, g.w3, g.b3);
  k_back_out<<<nblk(N * h), T>>>(dy, p.w3, Z2, N, h, dZ2);
  k_grad_dense<<<nblk((int64_t)h * (h + 1)), T>>>(dZ2, H1, N, h, h, g.W2, g.b2);
  k_back_dense<<<nblk(N * h), T>>>(dZ2, p.W2, Z1, N, h, dZ1);
  k_grad_dense<<<nblk((int64_t)h * (m->nin + 1)), T>>>(dZ1, X, N, h, m->nin, g.W1, g.b1);
}

// Counter-based generator (splitmix64) for the initial weights.
uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

}  // namespace

extern "C" {

int sym_mlp_create(int32_t nin, int32_t hidden, uint64_t seed, sym_mlp *out) {
  if (!out || nin < 1 || hidden < 1 || nin > 4096 || hidden > 4096) return SYM_ERR_INVALID;
  *out = nullptr;
  sym_mlp_s *m = new (std::nothrow) sym_mlp_s();
  if (!m) return SYM_ERR_OOM;
  m->nin = nin;
  m->h = hidden;
  m->np = (int64_t)hidden * nin + hidden + (int64_t)hidden * hidden + hidden + hidden + 1;
  std::vector<float> init(m->np, 0.f);
  // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases
  auto fill = [&](int64_t off, int64_t count, int fan_in) {
    const double a = 1.0 / std::sqrt((double)fan_in);
    for (int64_t i = 0; i < count; ++i) {
      const double u = (double)(splitmix64(seed + (uint64_t)(off + i)) >> 11) * (1.0 / 9007199254740992.0);
      init[off + i] = (float)((2.0 * u - 1.0) * a);
    }
  };
  fill(0, (int64_t)hidden * nin, nin);
  fill((int64_t)hidden * nin + hidden, (int64_t)hidden * hidden, hidden);
  fill((int64_t)hidden * nin + hidden + (int64_t)hidden * hidden + hidden, hidden, hidden);
  if (cudaMalloc(&m->theta, sizeof(float) * m->np) != cudaSuccess ||
      cudaMalloc(&m->grad, sizeof(float) * m->np) != cudaSuccess ||
      cudaMalloc(&m->m1, sizeof(float) * m->np) != cudaSuccess ||
      cudaMalloc(&m->m2, sizeof(float) * m->np) != cudaSuccess || cudaMalloc(&m->loss, sizeof(float)) != cudaSuccess) {
    sym_mlp_free(m);
    return SYM_ERR_OOM;
  }
  cudaMemcpy(m->theta, init.data(), sizeof(float) * m->np, cudaMemcpyHostToDevice);
  cudaMemset(m->m1, 0, sizeof(float) * m->np);
  cudaMemset(m->m2, 0, sizeof(float) * m->np);
  if (cudaGetLastError() != cudaSuccess) {
    sym_mlp_free(m);
    return SYM_ERR_CUDA;
  }
  *out = m;
  return SYM_OK;
}

int64_t sym_mlp_nparams(sym_mlp m) { return m ? m->np : SYM_ERR_INVALID; }

int sym_mlp_set_params(sym_mlp m, const float *theta) {
  if (!m || !theta) return SYM_ERR_INVALID;
  if (cudaMemcpy(m->theta, theta, sizeof(float) * m->np, cudaMemcpyHostToDevice) != cudaSuccess) return SYM_ERR_CUDA;
  cudaMemset(m->m1, 0, sizeof(float) * m->np);
  cudaMemset(m->m2, 0, sizeof(float) * m->np);
  m->step = 0;
  return cudaGetLastError() == cudaSuccess ? SYM_OK : SYM_ERR_CUDA;
}

int sym_mlp_get_params(sym_mlp m, float *theta) {
  if (!m || !theta) return SYM_ERR_INVALID;
  return cudaMemcpy(theta, m->theta, sizeof(float) * m->np, cudaMemcpyDeviceToHost) == cudaSuccess ? SYM_OK
                                                                                                     : SYM_ERR_CUDA;
}

int sym_mlp_predict(sym_mlp m, int64_t nrows, const float *X, float *y) {
  if (!m || nrows < 0 || (nrows > 0 && (!X || !y))) return SYM_ERR_INVALID;
  if (nrows == 0) return SYM_OK;
  if (ensure_work(m, nrows)) return SYM_ERR_OOM;
  float *Z1, *H1, *Z2, *H2, *yy;
  forward(m, X, nrows, &Z1, &H1, &Z2, &H2, &yy);
  cudaMemcpyAsync(y, yy, sizeof(float) * nrows, cudaMemcpyDeviceToDevice);
  return cudaDeviceSynchronize() == cudaSuccess ? SYM_OK : SYM_ERR_CUDA;
}

int sym_mlp_gradient(sym_mlp m, int64_t nrows, const float *X, const float *t, float *grad, float *loss) {
  if (!m || nrows < 1 || !X || !t) return SYM_ERR_INVALID;
  if (ensure_work(m, nrows)) return SYM_ERR_OOM;
  backward(m, X, t, nrows);
  if (grad && cudaMemcpy(grad, m->grad, sizeof(float) * m->np, cudaMemcpyDeviceToHost) != cudaSuccess)
    return SYM_ERR_CUDA;
  if (loss && cudaMemcpy(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return SYM_ERR_CUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? SYM_OK : SYM_ERR_CUDA;
}

int sym_mlp_train(sym_mlp m, int64_t nrows, const float *X, const float *t, int32_t steps, float lr, float *loss) {
  if (!m || nrows < 1 || !X || !t || steps < 0 || !(lr > 0.f)) return SYM_ERR_INVALID;
  if (ensure_work(m, nrows)) return SYM_ERR_OOM;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int32_t s = 0; s < steps; ++s) {
    backward(m, X, t, nrows);
    ++m->step;
    const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
    k_adam<<<nblk(m->np), T>>>(m->theta, m->grad, m->m1, m->m2, m->np, lr, b1, b2, eps, c1, c2);
  }
  if (loss) {
    backward(m, X, t, nrows);  // loss at the final parameters
    if (cudaMemcpy(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return SYM_ERR_CUDA;
  }
  return cudaDeviceSynchronize() == cudaSuccess ? SYM_OK : SYM_ERR_CUDA;
}

void sym_mlp_free(sym_mlp m) {
  if (!m) return;
  float *p[] = {m->theta, m->grad, m->m1, m->m2, m->work, m->loss};
  for (float *q : p)
    if (q) cudaFree(q);
  delete m;
}

}  // extern "C"

// Step/rank controller network: a three-layer FP32 perceptron
//   y = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3   (hidden width 128)
// with hand-written forward, backward (chain rule) and Adam kernels.  Training and
// inference both run on the GPU; weights are stored row-major (out x in) in one
// contiguous buffer [W1 | b1 | W2 | b2 | W3 | b3].  The paper has no network: the
// controller implements its proposed adaptive time stepping (Sec. 6) with a learned rule.
#include "lrei.h"
#include "common.cuh"

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

namespace lrei {

constexpr int MLP_H = 128;

struct MlpShape {
  int n_in, n_out;
  size_t oW1, ob1, oW2, ob2, oW3, ob3, total;
  void init(int i, int o) {
    n_in = i;
    n_out = o;
    oW1 = 0;
    ob1 = oW1 + (size_t)MLP_H * i;
    oW2 = ob1 + MLP_H;
    ob2 = oW2 + (size_t)MLP_H * MLP_H;
    oW3 = ob2 + MLP_H;
    ob3 = oW3 + (size_t)o * MLP_H;
    total = ob3 + o;
  }
};

// Z = X W^T + b, optionally H = tanh(Z).  One thread per output element.
__global__ void dense_fwd_kernel(const float *__restrict__ X, int B, int n_in, const float *__restrict__ W,
                                 const float *__restrict__ b, int n_out, int act, float *__restrict__ Y) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * n_out; e += gridDim.x * blockDim.x) {
    const int bi = e / n_out, o = e % n_out;
    const float *x = X + (size_t)bi * n_in;
    const float *w = W + (size_t)o * n_in;
    float s = b[o];
    for (int i = 0; i < n_in; ++i) s = fmaf(w[i], x[i], s);
    Y[e] = act ? tanhf(s) : s;
  }
}

// dY = w_o (Y - T) / B and the per-element loss terms 0.5 w_o (Y - T)^2 / B.
__global__ void mse_grad_kernel(const float *__restrict__ Y, const float *__restrict__ T, const float *__restrict__ w,
                                int B, int n_out, float *__restrict__ dY, float *__restrict__ lterm) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * n_out; e += gridDim.x * blockDim.x) {
    const int o = e % n_out;
    const float d = Y[e] - T[e];
    dY[e] = w[o] * d / (float)B;
    lterm[e] = 0.5f * w[o] * d * d / (float)B;
  }
}

// dX = dZ W (B x n_in); if H is given, dX is multiplied by (1 - H^2) (tanh derivative of the layer below).
__global__ void dense_bwd_data_kernel(const float *__restrict__ dZ, int B, int n_out, const float *__restrict__ W,
                                      int n_in, const float *__restrict__ Hbelow, float *__restrict__ dX) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * n_in; e += gridDim.x * blockDim.x) {
    const int bi = e / n_in, i = e % n_in;
    float s = 0.f;
    for (int o = 0; o < n_out; ++o) s = fmaf(dZ[(size_t)bi * n_out + o], W[(size_t)o * n_in + i], s);
    if (Hbelow) {
      const float h = Hbelow[e];
      s *= (1.f - h * h);
    }
    dX[e] = s;
  }
}

// dW = dZ^T X (n_out x n_in), db = sum_b dZ.  One thread per weight, fixed summation order.
__global__ void dense_bwd_weight_kernel(const float *__restrict__ dZ, const float *__restrict__ X, int B, int n_out,
                                        int n_in, float *__restrict__ dW, float *__restrict__ db) {
  const int tot = n_out * n_in + n_out;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
    float s = 0.f;
    if (e < n_out * n_in) {
      const int o = e / n_in, i = e % n_in;
      for (int bi = 0; bi < B; ++bi) s = fmaf(dZ[(size_t)bi * n_out + o], X[(size_t)bi * n_in + i], s);
      dW[e] = s;
    } else {
      const int o = e - n_out * n_in;
      for (int bi = 0; bi < B; ++bi) s += dZ[(size_t)bi * n_out + o];
      db[o] = s;
    }
  }
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, size_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void sum_kernel(const float *__restrict__ x, int n, float *__restrict__ out) {
  __shared__ float red[256];
  float s = 0.f;
  for (int e = threadIdx.x; e < n; e += blockDim.x) s += x[e];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

static int grid_of(long long n) {
  long long g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 2048 ? 2048 : g));
}

}  // namespace lrei

using namespace lrei;

struct lrei_mlp {
  MlpShape sh;
  cudaStream_t st = nullptr;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  int cap_B = 0;
  float *H1 = nullptr, *H2 = nullptr, *Y = nullptr, *dY = nullptr, *d2 = nullptr, *d1 = nullptr, *lterm = nullptr,
        *w = nullptr, *lsum = nullptr;
  int t = 0;
};

namespace {
int mlp_reserve(lrei_mlp *net, int B) {
  if (B <= net->cap_B) return LREI_OK;
  float **bufs[] = {&net->H1, &net->H2, &net->d2, &net->d1};
  for (auto b : bufs) {
    if (*b) cudaFree(*b);
    if (cudaMalloc(b, (size_t)B * MLP_H * sizeof(float)) != cudaSuccess) return LREI_ERR_OOM;
  }
  float **obufs[] = {&net->Y, &net->dY, &net->lterm};
  for (auto b : obufs) {
    if (*b) cudaFree(*b);
    if (cudaMalloc(b, (size_t)B * net->sh.n_out * sizeof(float)) != cudaSuccess) return LREI_ERR_OOM;
  }
  net->cap_B = B;
  return LREI_OK;
}

void mlp_forward_into(lrei_mlp *net, const float *X, int B, float *Y) {
  const MlpShape &s = net->sh;
  count_launch(3);
  dense_fwd_kernel<<<grid_of((long long)B * MLP_H), 256, 0, net->st>>>(X, B, s.n_in, net->p + s.oW1, net->p + s.ob1,
                                                                        MLP_H, 1, net->H1);
  dense_fwd_kernel<<<grid_of((long long)B * MLP_H), 256, 0, net->st>>>(net->H1, B, MLP_H, net->p + s.oW2,
                                                                        net->p + s.ob2, MLP_H, 1, net->H2);
  dense_fwd_kernel<<<grid_of((long long)B * s.n_out), 256, 0, net->st>>>(net->H2, B, MLP_H, net->p + s.oW3,
                                                                           net->p + s.ob3, s.n_out, 0, Y);
}
}  // namespace

int lrei_mlp_forward_on(lrei_mlp *net, const float *X, int B, float *Y, cudaStream_t st) {
  if (!net || B < 1) return LREI_ERR_ARG;
  if (mlp_reserve(net, B)) return LREI_ERR_OOM;
  cudaStream_t keep = net->st;
  net->st = st;
  mlp_forward_into(net, X, B, Y);
  net->st = keep;
  return cudaGetLastError() == cudaSuccess ? LREI_OK : LREI_ERR_CUDA;
}

extern "C" {

int lrei_mlp_create(int n_in, int n_out, const float *params_host, void *cuda_stream, lrei_mlp **out) {
  if (!out || n_in < 1 || n_in > 4096 || n_out < 1 || n_out > 64) return LREI_ERR_ARG;
  lrei_mlp *net = new (std::nothrow) lrei_mlp();
  if (!net) return LREI_ERR_OOM;
  net->sh.init(n_in, n_out);
  net->st = reinterpret_cast<cudaStream_t>(cuda_stream);
  const size_t bytes = net->sh.total * sizeof(float);
  float **bufs[] = {&net->p, &net->g, &net->m, &net->v};
  for (auto b : bufs) {
    if (cudaMalloc(b, bytes) != cudaSuccess) {
      lrei_mlp_destroy(net);
      return LREI_ERR_OOM;
    }
    cudaMemsetAsync(*b, 0, bytes, net->st);
  }
  if (cudaMalloc(&net->w, 64 * sizeof(float)) != cudaSuccess || cudaMalloc(&net->lsum, sizeof(float)) != cudaSuccess) {
    lrei_mlp_destroy(net);
    return LREI_ERR_OOM;
  }
  if (params_host) cudaMemcpyAsync(net->p, params_host, bytes, cudaMemcpyHostToDevice, net->st);
  if (cudaStreamSynchronize(net->st) != cudaSuccess) {
    lrei_mlp_destroy(net);
    return LREI_ERR_CUDA;
  }
  *out = net;
  return LREI_OK;
}

int lrei_mlp_destroy(lrei_mlp *net) {
  if (!net) return LREI_OK;
  if (net->st) cudaStreamSynchronize(net->st);
  float *bufs[] = {net->p, net->g, net->m, net->v, net->H1, net->H2, net->Y, net->dY, net->d2, net->d1, net->lterm,
                   net->w, net->lsum};
  for (auto b : bufs)
    if (b) cudaFree(b);
  delete net;
  return LREI_OK;
}

int lrei_mlp_num_params(const lrei_mlp *net) { return net ? (int)net->sh.total : 0; }

int lrei_mlp_get_params(lrei_mlp *net, float *host, int n) {
  if (!net || !host || n != (int)net->sh.total) return LREI_ERR_ARG;
  if (cudaMemcpyAsync(host, net->p, n * sizeof(float), cudaMemcpyDeviceToHost, net->st) != cudaSuccess) return LREI_ERR_CUDA;
  return cudaStreamSynchronize(net->st) == cudaSuccess ? LREI_OK : LREI_ERR_CUDA;
}

int lrei_mlp_set_params(lrei_mlp *net, const float *host, int n) {
  if (!net || !host || n != (int)net->sh.total) return LREI_ERR_ARG;
  if (cudaMemcpyAsync(net->p, host, n * sizeof(float), cudaMemcpyHostToDevice, net->st) != cudaSuccess) return LREI_ERR_CUDA;
  net->t = 0;
  cudaMemsetAsync(net->m, 0, n * sizeof(float), net->st);
  cudaMemsetAsync(net->v, 0, n * sizeof(float), net->st);
  return cudaStreamSynchronize(net->st) == cudaSuccess ? LREI_OK : LREI_ERR_CUDA;
}

int lrei_mlp_forward(lrei_mlp *net, const float *X_dev, int batch, float *Y_dev) {
  if (!net || !X_dev || !Y_dev || batch < 1) return LREI_ERR_ARG;
  if (mlp_reserve(net, batch)) return LREI_ERR_OOM;
  mlp_forward_into(net, X_dev, batch, Y_dev);
  return cudaGetLastError() == cudaSuccess ? LREI_OK : LREI_ERR_CUDA;
}

int lrei_mlp_grads(lrei_mlp *net, const float *X_dev, const float *T_dev, const float *w_host, int batch,
                   float *grad_dev, float *loss_host) {
  if (!net || !X_dev || !T_dev || batch < 1) return LREI_ERR_ARG;
  if (mlp_reserve(net, batch)) return LREI_ERR_OOM;
  const MlpShape &s = net->sh;
  std::vector<float> w(s.n_out, 1.0f);
  if (w_host) std::memcpy(w.data(), w_host, s.n_out * sizeof(float));
  cudaMemcpyAsync(net->w, w.data(), s.n_out * sizeof(float), cudaMemcpyHostToDevice, net->st);
  mlp_forward_into(net, X_dev, batch, net->Y);
  const int B = batch;
  cudaStream_t st = net->st;
  count_launch(8);
  mse_grad_kernel<<<grid_of((long long)B * s.n_out), 256, 0, st>>>(net->Y, T_dev, net->w, B, s.n_out, net->dY,
                                                                    net->lterm);
  // layer 3
  dense_bwd_weight_kernel<<<grid_of((long long)s.n_out * MLP_H + s.n_out), 256, 0, st>>>(
      net->dY, net->H2, B, s.n_out, MLP_H, net->g + s.oW3, net->g + s.ob3);
  dense_bwd_data_kernel<<<grid_of((long long)B * MLP_H), 256, 0, st>>>(net->dY, B, s.n_out, net->p + s.oW3, MLP_H,
                                                                        net->H2, net->d2);
  // layer 2
  dense_bwd_weight_kernel<<<grid_of((long long)MLP_H * MLP_H + MLP_H), 256, 0, st>>>(
      net->d2, net->H1, B, MLP_H, MLP_H, net->g + s.oW2, net->g + s.ob2);
  dense_bwd_data_kernel<<<grid_of((long long)B * MLP_H), 256, 0, st>>>(net->d2, B, MLP_H, net->p + s.oW2, MLP_H,
                                                                        net->H1, net->d1);
  // layer 1
  dense_bwd_weight_kernel<<<grid_of((long long)MLP_H * s.n_in + MLP_H), 256, 0, st>>>(
      net->d1, X_dev, B, MLP_H, s.n_in, net->g + s.oW1, net->g + s.ob1);
  sum_kernel<<<1, 256, 0, st>>>(net->lterm, B * s.n_out, net->lsum);
  if (grad_dev) cudaMemcpyAsync(grad_dev, net->g, s.total * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (loss_host) {
    cudaMemcpyAsync(loss_host, net->lsum, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return LREI_ERR_CUDA;
  }
  return cudaGetLastError() == cudaSuccess ? LREI_OK : LREI_ERR_CUDA;
}

int lrei_mlp_adam(lrei_mlp *net, float lr, float beta1, float beta2, float eps) {
  if (!net || !(lr > 0)) return LREI_ERR_ARG;
  net->t += 1;
  const float c1 = 1.f - std::pow(beta1, (float)net->t), c2 = 1.f - std::pow(beta2, (float)net->t);
  count_launch();
  adam_kernel<<<grid_of((long long)net->sh.total), 256, 0, net->st>>>(net->p, net->g, net->m, net->v, net->sh.total,
                                                                       lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? LREI_OK : LREI_ERR_CUDA;
}

}  // extern "C"

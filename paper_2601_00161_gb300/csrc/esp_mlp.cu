// Kernels and C ABI of the selector's 3-layer perceptron (FP32): dense layers with tanh,
// mean-squared-error loss, back-propagation and Adam.  One thread per output element in
// every kernel; the weight gradients sum over the batch in a fixed order (deterministic).
#include "esp_mlp.h"

#include <cuda_runtime.h>
#include <math.h>

#include <string>

namespace {

constexpr int kT = 256;
std::string g_err;

int fail(const std::string& m, int code = -1) {
  g_err = m;
  return code;
}
int cuda_fail(cudaError_t e, const char* where) {
  return fail(std::string(where) + ": " + cudaGetErrorString(e), -6);
}
#define MLP_CUDA(call)                                 \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

int blocks(int64_t n) { return (int)((n + kT - 1) / kT); }

// out[b][o] = act(b_[o] + sum_i W[o][i] in[b][i])
__global__ void k_dense_fwd(const float* __restrict__ in, const float* __restrict__ W,
                            const float* __restrict__ bias, float* __restrict__ out, int B,
                            int I, int O, int act) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)B * O) return;
  const int b = (int)(e / O), o = (int)(e % O);
  float a = bias[o];
  for (int i = 0; i < I; ++i) a = fmaf(W[o * I + i], in[b * I + i], a);
  out[e] = act ? tanhf(a) : a;
}

// d3 = 2 (y - t) / (B O); loss += sum (y - t)^2 / (B O)
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t,
                      float* __restrict__ d, float* __restrict__ loss, int n) {
  __shared__ float part[kT / 32];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (e < n) {
    const float r = y[e] - t[e];
    d[e] = 2.f * r / n;
    l = r * r / n;
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < kT / 32; ++w) s += part[w];
    atomicAdd(loss, s);
  }
}

// gW[o][i] = sum_b d[b][o] in[b][i] (i < I), gb[o] = sum_b d[b][o] (i == I)
__global__ void k_dense_grad(const float* __restrict__ d, const float* __restrict__ in,
                             float* __restrict__ gW, float* __restrict__ gb, int B, int I,
                             int O) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= O * (I + 1)) return;
  const int o = e / (I + 1), i = e % (I + 1);
  float s = 0.f;
  if (i < I)
    for (int b = 0; b < B; ++b) s = fmaf(d[b * O + o], in[b * I + i], s);
  else
    for (int b = 0; b < B; ++b) s += d[b * O + o];
  if (i < I) gW[o * I + i] = s;
  else gb[o] = s;
}

// d_in[b][i] = (sum_o W[o][i] d[b][o]) (1 - h[b][i]^2): back through tanh
__global__ void k_dense_back(const float* __restrict__ d, const float* __restrict__ W,
                             const float* __restrict__ h, float* __restrict__ d_in, int B, int I,
                             int O) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)B * I) return;
  const int b = (int)(e / I), i = (int)(e % I);
  float s = 0.f;
  for (int o = 0; o < O; ++o) s = fmaf(W[o * I + i], d[b * O + o], s);
  const float hv = h[e];
  d_in[e] = s * (1.f - hv * hv);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float gi = g[e];
  const float mi = b1 * m[e] + (1.f - b1) * gi;
  const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
  m[e] = mi;
  v[e] = vi;
  p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

struct esp_mlp_s {
  int n_in = 0, n_h = 0, n_out = 0, max_batch = 0, n_par = 0;
  int step = 0;
  cudaStream_t st = nullptr;
  float* p = nullptr;   // parameters
  float* g = nullptr;   // gradient
  float* m = nullptr;   // Adam moments
  float* v = nullptr;
  float* h1 = nullptr;  // activations (max_batch x n_h)
  float* h2 = nullptr;
  float* y = nullptr;   // outputs (max_batch x n_out)
  float* d3 = nullptr;  // dL/dy, dL/da2, dL/da1
  float* d2 = nullptr;
  float* d1 = nullptr;
  // views into p / g
  float *W1, *b1, *W2, *b2, *W3, *b3;
  float *gW1, *gb1, *gW2, *gb2, *gW3, *gb3;
};

namespace {

void release(esp_mlp_t n) {
  if (!n) return;
  float* bufs[] = {n->p, n->g, n->m, n->v, n->h1, n->h2, n->y, n->d3, n->d2, n->d1};
  for (float* b : bufs)
    if (b) cudaFree(b);
  delete n;
}

void views(float* base, int I, int H, int O, float** W1, float** b1, float** W2, float** b2,
           float** W3, float** b3) {
  *W1 = base;
  *b1 = *W1 + H * I;
  *W2 = *b1 + H;
  *b2 = *W2 + H * H;
  *W3 = *b2 + H;
  *b3 = *W3 + O * H;
}

int run_forward(esp_mlp_t n, const float* x, int B) {
  k_dense_fwd<<<blocks((int64_t)B * n->n_h), kT, 0, n->st>>>(x, n->W1, n->b1, n->h1, B, n->n_in,
                                                              n->n_h, 1);
  k_dense_fwd<<<blocks((int64_t)B * n->n_h), kT, 0, n->st>>>(n->h1, n->W2, n->b2, n->h2, B,
                                                              n->n_h, n->n_h, 1);
  k_dense_fwd<<<blocks((int64_t)B * n->n_out), kT, 0, n->st>>>(n->h2, n->W3, n->b3, n->y, B,
                                                                n->n_h, n->n_out, 0);
  MLP_CUDA(cudaGetLastError());
  return 0;
}

}  // namespace

extern "C" {

int esp_mlp_n_params(int I, int H, int O) { return H * I + H + H * H + H + O * H + O; }

int esp_mlp_create(esp_mlp_t* out, int I, int H, int O, int max_batch, const float* params_host,
                   void* stream) {
  if (!out || !params_host || I < 1 || H < 1 || O < 1 || max_batch < 1 || I > 4096 ||
      H > 4096 || O > 4096 || (int64_t)max_batch * H > (1 << 28))
    return fail("esp_mlp_create: bad sizes or NULL argument");
  *out = nullptr;
  esp_mlp_t n = new esp_mlp_s;
  n->n_in = I;
  n->n_h = H;
  n->n_out = O;
  n->max_batch = max_batch;
  n->n_par = esp_mlp_n_params(I, H, O);
  n->st = (cudaStream_t)stream;
  const size_t P = (size_t)n->n_par * sizeof(float);
  const size_t BH = (size_t)max_batch * H * sizeof(float), BO = (size_t)max_batch * O * sizeof(float);
  cudaError_t e = cudaSuccess;
  float** bufs[] = {&n->p, &n->g, &n->m, &n->v};
  for (float** b : bufs)
    if (e == cudaSuccess) e = cudaMalloc(b, P);
  if (e == cudaSuccess) e = cudaMalloc(&n->h1, BH);
  if (e == cudaSuccess) e = cudaMalloc(&n->h2, BH);
  if (e == cudaSuccess) e = cudaMalloc(&n->d2, BH);
  if (e == cudaSuccess) e = cudaMalloc(&n->d1, BH);
  if (e == cudaSuccess) e = cudaMalloc(&n->y, BO);
  if (e == cudaSuccess) e = cudaMalloc(&n->d3, BO);
  if (e == cudaSuccess) e = cudaMemcpy(n->p, params_host, P, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(n->m, 0, P);
  if (e == cudaSuccess) e = cudaMemset(n->v, 0, P);
  if (e == cudaSuccess) e = cudaMemset(n->g, 0, P);
  if (e != cudaSuccess) {
    release(n);
    return cuda_fail(e, "esp_mlp_create");
  }
  views(n->p, I, H, O, &n->W1, &n->b1, &n->W2, &n->b2, &n->W3, &n->b3);
  views(n->g, I, H, O, &n->gW1, &n->gb1, &n->gW2, &n->gb2, &n->gW3, &n->gb3);
  *out = n;
  return 0;
}

int esp_mlp_forward(esp_mlp_t n, const float* d_x, int B, float* d_y) {
  if (!n || !d_x || !d_y || B < 1 || B > n->max_batch) return fail("esp_mlp_forward: bad argument");
  int rc = run_forward(n, d_x, B);
  if (rc) return rc;
  MLP_CUDA(cudaMemcpyAsync(d_y, n->y, (size_t)B * n->n_out * sizeof(float), cudaMemcpyDeviceToDevice,
                           n->st));
  return 0;
}

int esp_mlp_loss_grad(esp_mlp_t n, const float* d_x, const float* d_t, int B, float* d_loss,
                      float* d_grad) {
  if (!n || !d_x || !d_t || !d_loss || B < 1 || B > n->max_batch)
    return fail("esp_mlp_loss_grad: bad argument");
  int rc = run_forward(n, d_x, B);
  if (rc) return rc;
  const int I = n->n_in, H = n->n_h, O = n->n_out;
  MLP_CUDA(cudaMemsetAsync(d_loss, 0, sizeof(float), n->st));
  k_mse<<<blocks((int64_t)B * O), kT, 0, n->st>>>(n->y, d_t, n->d3, d_loss, B * O);
  k_dense_grad<<<blocks((int64_t)O * (H + 1)), kT, 0, n->st>>>(n->d3, n->h2, n->gW3, n->gb3, B, H, O);
  k_dense_back<<<blocks((int64_t)B * H), kT, 0, n->st>>>(n->d3, n->W3, n->h2, n->d2, B, H, O);
  k_dense_grad<<<blocks((int64_t)H * (H + 1)), kT, 0, n->st>>>(n->d2, n->h1, n->gW2, n->gb2, B, H, H);
  k_dense_back<<<blocks((int64_t)B * H), kT, 0, n->st>>>(n->d2, n->W2, n->h1, n->d1, B, H, H);
  k_dense_grad<<<blocks((int64_t)H * (I + 1)), kT, 0, n->st>>>(n->d1, d_x, n->gW1, n->gb1, B, I, H);
  MLP_CUDA(cudaGetLastError());
  if (d_grad)
    MLP_CUDA(cudaMemcpyAsync(d_grad, n->g, (size_t)n->n_par * sizeof(float), cudaMemcpyDeviceToDevice,
                             n->st));
  return 0;
}

int esp_mlp_adam(esp_mlp_t n, float lr, float beta1, float beta2, float eps) {
  if (!n || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f))
    return fail("esp_mlp_adam: bad argument");
  n->step += 1;
  const float c1 = 1.f - powf(beta1, (float)n->step), c2 = 1.f - powf(beta2, (float)n->step);
  k_adam<<<blocks(n->n_par), kT, 0, n->st>>>(n->p, n->g, n->m, n->v, n->n_par, lr, beta1, beta2, eps,
                                             c1, c2);
  MLP_CUDA(cudaGetLastError());
  return 0;
}

int esp_mlp_get_params(esp_mlp_t n, float* host) {
  if (!n || !host) return fail("esp_mlp_get_params: NULL argument");
  MLP_CUDA(cudaStreamSynchronize(n->st));
  MLP_CUDA(cudaMemcpy(host, n->p, (size_t)n->n_par * sizeof(float), cudaMemcpyDeviceToHost));
  return 0;
}

int esp_mlp_set_params(esp_mlp_t n, const float* host) {
  if (!n || !host) return fail("esp_mlp_set_params: NULL argument");
  MLP_CUDA(cudaStreamSynchronize(n->st));
  MLP_CUDA(cudaMemcpy(n->p, host, (size_t)n->n_par * sizeof(float), cudaMemcpyHostToDevice));
  return 0;
}

int esp_mlp_destroy(esp_mlp_t n) {
  if (n && n->st) cudaStreamSynchronize(n->st);
  release(n);
  return 0;
}

const char* esp_mlp_last_error(void) { return g_err.c_str(); }

}  // extern "C"

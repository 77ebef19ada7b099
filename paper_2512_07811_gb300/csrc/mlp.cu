// Per-bond rank predictor: a multilayer perceptron with three hidden layers of
// width 64 and ReLU, FP16 weights, FP32 biases, FP32 accumulation, FP32 master
// weights and Adam moments for training (not in the paper; its
// nearest relative is the coarse-grained rank
// of Sec. 5.1).
//
//   h1 = relu(W0 x + b0), h2 = relu(W1 h1 + b1), h3 = relu(W2 h2 + b2),
//   y  = W3 h3 + b3                          (y = predicted log2 rank)
//   L  = (1/B) sum_b w_b (y_b - t_b)^2,  w_b = alpha if y_b < t_b else 1
//
// Packed parameter order (FP32 master copy and gradients):
//   W0 (64 x F), b0 (64), W1 (64 x 64), b1 (64), W2 (64 x 64), b2 (64), W3 (64), b3 (1)
// Weights are row-major (out, in).  One warp handles one sample; lanes own
// neurons l and l + 32 of every hidden layer.
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int H = 64;
constexpr int MAXF = 32;
constexpr int WARPS = 8;

struct Offsets {
  int64_t W0, b0, W1, b1, W2, b2, W3, b3, total;
};

__host__ __device__ inline Offsets offsets(int F) {
  Offsets o;
  o.W0 = 0;
  o.b0 = o.W0 + (int64_t)H * F;
  o.W1 = o.b0 + H;
  o.b1 = o.W1 + H * H;
  o.W2 = o.b1 + H;
  o.b2 = o.W2 + H * H;
  o.W3 = o.b2 + H;
  o.b3 = o.W3 + H;
  o.total = o.b3 + 1;
  return o;
}

__device__ __forceinline__ float wsum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// shared-memory copy of the weights (FP16 weights widened on use)
struct SmemW {
  __half W0[H * MAXF];
  __half W1[H * H];
  __half W2[H * H];
  __half W3[H];
  float b0[H], b1[H], b2[H], b3;
};

__device__ void load_weights(SmemW& s, const __half* Wh, const float* P, int F) {
  const Offsets o = offsets(F);
  for (int i = threadIdx.x; i < H * F; i += blockDim.x) s.W0[i] = Wh[o.W0 + i];
  for (int i = threadIdx.x; i < H * H; i += blockDim.x) {
    s.W1[i] = Wh[o.W1 + i];
    s.W2[i] = Wh[o.W2 + i];
  }
  for (int i = threadIdx.x; i < H; i += blockDim.x) {
    s.W3[i] = Wh[o.W3 + i];
    s.b0[i] = P[o.b0 + i];
    s.b1[i] = P[o.b1 + i];
    s.b2[i] = P[o.b2 + i];
  }
  if (threadIdx.x == 0) s.b3 = P[o.b3];
}

// forward pass of one sample by one warp; stores pre-activations z1..z3 and
// activations h1..h3 in the warp's scratch; returns y on every lane
__device__ float warp_forward(const SmemW& s, const float* x, int F, float* z, float* h) {
  const int lane = threadIdx.x & 31;
  float* z1 = z;
  float* z2 = z + H;
  float* z3 = z + 2 * H;
  float* h1 = h;
  float* h2 = h + H;
  float* h3 = h + 2 * H;
  for (int r = 0; r < 2; ++r) {
    const int n = lane + 32 * r;
    float a = s.b0[n];
    for (int i = 0; i < F; ++i) a = fmaf(__half2float(s.W0[n * F + i]), x[i], a);
    z1[n] = a;
    h1[n] = a > 0.f ? a : 0.f;
  }
  __syncwarp();
  for (int r = 0; r < 2; ++r) {
    const int n = lane + 32 * r;
    float a = s.b1[n];
    for (int i = 0; i < H; ++i) a = fmaf(__half2float(s.W1[n * H + i]), h1[i], a);
    z2[n] = a;
    h2[n] = a > 0.f ? a : 0.f;
  }
  __syncwarp();
  for (int r = 0; r < 2; ++r) {
    const int n = lane + 32 * r;
    float a = s.b2[n];
    for (int i = 0; i < H; ++i) a = fmaf(__half2float(s.W2[n * H + i]), h2[i], a);
    z3[n] = a;
    h3[n] = a > 0.f ? a : 0.f;
  }
  __syncwarp();
  float y = __half2float(s.W3[lane]) * h3[lane] + __half2float(s.W3[lane + 32]) * h3[lane + 32];
  y = wsum(y) + s.b3;
  return y;
}

__global__ void __launch_bounds__(WARPS * 32)
mlp_forward_kernel(const __half* __restrict__ Wh, const float* __restrict__ P, int F, const float* __restrict__ X,
                   int64_t B, float* __restrict__ Y) {
  __shared__ SmemW s;
  __shared__ float xs[WARPS][MAXF];
  __shared__ float zs[WARPS][3 * H];
  __shared__ float hs[WARPS][3 * H];
  load_weights(s, Wh, P, F);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t b = (int64_t)blockIdx.x * WARPS + warp; b < B; b += (int64_t)gridDim.x * WARPS) {
    if (lane < F) xs[warp][lane] = X[b * F + lane];
    __syncwarp();
    float y = warp_forward(s, xs[warp], F, zs[warp], hs[warp]);
    if (lane == 0) Y[b] = y;
    __syncwarp();
  }
}

// Gradients of the asymmetric loss, accumulated per block in shared memory
// and added to the global FP32 gradient buffer G (packed order); the loss sum
// goes to loss_acc.
__global__ void __launch_bounds__(WARPS * 32)
mlp_backward_kernel(const __half* __restrict__ Wh, const float* __restrict__ P, int F, const float* __restrict__ X,
                    const float* __restrict__ T, int64_t B, float alpha, float* __restrict__ G,
                    float* __restrict__ loss_acc) {
  __shared__ SmemW s;
  __shared__ float xs[WARPS][MAXF];
  __shared__ float zs[WARPS][3 * H];
  __shared__ float hs[WARPS][3 * H];
  __shared__ float d3[WARPS][H];
  __shared__ float d2[WARPS][H];
  extern __shared__ float gsm[];  // packed gradient partials, offsets(F).total floats
  const Offsets o = offsets(F);
  load_weights(s, Wh, P, F);
  for (int64_t i = threadIdx.x; i <= o.total; i += blockDim.x) gsm[i] = 0.f;  // gradients and the loss slot
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float lsum = 0.f;
  for (int64_t b = (int64_t)blockIdx.x * WARPS + warp; b < B; b += (int64_t)gridDim.x * WARPS) {
    if (lane < F) xs[warp][lane] = X[b * F + lane];
    __syncwarp();
    const float* x = xs[warp];
    float* z = zs[warp];
    float* h = hs[warp];
    const float y = warp_forward(s, x, F, z, h);
    const float t = T[b];
    const float w = y < t ? alpha : 1.f;
    if (lane == 0) lsum += w * (y - t) * (y - t);  // y is broadcast to all lanes: count it once
    const float g = 2.f / (float)B * w * (y - t);
    // output layer
    if (lane == 0) atomicAdd(&gsm[o.b3], g);
    for (int r = 0; r < 2; ++r) {
      const int n = lane + 32 * r;
      atomicAdd(&gsm[o.W3 + n], g * h[2 * H + n]);
      d3[warp][n] = (z[2 * H + n] > 0.f) ? g * __half2float(s.W3[n]) : 0.f;
    }
    __syncwarp();
    // layer 2 (W2: 64 x 64 from h2 to z3)
    for (int r = 0; r < 2; ++r) {
      const int n = lane + 32 * r;
      const float dn = d3[warp][n];
      atomicAdd(&gsm[o.b2 + n], dn);
      if (dn != 0.f)
        for (int i = 0; i < H; ++i) atomicAdd(&gsm[o.W2 + n * H + i], dn * h[H + i]);
    }
    for (int r = 0; r < 2; ++r) {
      const int m = lane + 32 * r;
      float a = 0.f;
      for (int n = 0; n < H; ++n) a = fmaf(__half2float(s.W2[n * H + m]), d3[warp][n], a);
      d2[warp][m] = (z[H + m] > 0.f) ? a : 0.f;
    }
    __syncwarp();
    // layer 1 (W1 from h1 to z2)
    for (int r = 0; r < 2; ++r) {
      const int n = lane + 32 * r;
      const float dn = d2[warp][n];
      atomicAdd(&gsm[o.b1 + n], dn);
      if (dn != 0.f)
        for (int i = 0; i < H; ++i) atomicAdd(&gsm[o.W1 + n * H + i], dn * h[i]);
    }
    float* d1 = d3[warp];  // reuse
    __syncwarp();
    for (int r = 0; r < 2; ++r) {
      const int m = lane + 32 * r;
      float a = 0.f;
      for (int n = 0; n < H; ++n) a = fmaf(__half2float(s.W1[n * H + m]), d2[warp][n], a);
      d1[m] = (z[m] > 0.f) ? a : 0.f;
    }
    __syncwarp();
    // layer 0 (W0 from x to z1)
    for (int r = 0; r < 2; ++r) {
      const int n = lane + 32 * r;
      const float dn = d1[n];
      atomicAdd(&gsm[o.b0 + n], dn);
      if (dn != 0.f)
        for (int i = 0; i < F; ++i) atomicAdd(&gsm[o.W0 + n * F + i], dn * x[i]);
    }
    __syncwarp();
  }
  lsum = wsum(lsum);
  if (lane == 0) atomicAdd(&gsm[o.total], lsum);  // slot after the gradients
  __syncthreads();
  for (int64_t i = threadIdx.x; i < o.total; i += blockDim.x) atomicAdd(&G[i], gsm[i]);
  if (threadIdx.x == 0) atomicAdd(loss_acc, gsm[o.total]);
}

// Adam (Kingma & Ba 2015) on the FP32 master copy, then the FP16 weights
__global__ void adam_kernel(float* __restrict__ P, __half* __restrict__ Wh, const float* __restrict__ G,
                            float* __restrict__ M, float* __restrict__ V, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float g = G[i];
    const float m = b1 * M[i] + (1.f - b1) * g;
    const float v = b2 * V[i] + (1.f - b2) * g * g;
    M[i] = m;
    V[i] = v;
    const float mh = m / c1, vh = v / c2;
    const float p = P[i] - lr * mh / (sqrtf(vh) + eps);
    P[i] = p;
    Wh[i] = __float2half_rn(p);
  }
}

__global__ void to_half_kernel(const float* __restrict__ P, __half* __restrict__ Wh, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    Wh[i] = __float2half_rn(P[i]);
}

}  // namespace

int64_t qtt_mlp_param_count_f(int F) { return offsets(F).total; }

// The FP16 array mirrors the packed FP32 array element by element (biases are
// read from the FP32 copy).
int qtt_mlp_sync_half(const float* P, __half* Wh, int64_t n, cudaStream_t s) {
  to_half_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P, Wh, n);
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

int qtt_mlp_forward_dev(const __half* Wh, const float* P, int F, const float* X, int64_t B, float* Y, cudaStream_t s) {
  if (F < 1 || F > MAXF) return QTT_ERR_ARG;
  if (B <= 0) return QTT_OK;
  int64_t blocks = (B + WARPS - 1) / WARPS;
  if (blocks > 1024) blocks = 1024;
  mlp_forward_kernel<<<(unsigned)blocks, WARPS * 32, 0, s>>>(Wh, P, F, X, B, Y);
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

int qtt_mlp_backward_dev(const __half* Wh, const float* P, int F, const float* X, const float* T, int64_t B, float alpha,
                         float* G, float* loss_acc, cudaStream_t s) {
  if (F < 1 || F > MAXF) return QTT_ERR_ARG;
  if (B <= 0) return QTT_OK;
  int64_t blocks = (B + WARPS - 1) / WARPS;
  if (blocks > 256) blocks = 256;
  size_t sm = (size_t)(offsets(F).total + 1) * sizeof(float);
  if (qtt_allow_max_smem((const void*)mlp_backward_kernel) != QTT_OK) return QTT_ERR_CUDA;
  mlp_backward_kernel<<<(unsigned)blocks, WARPS * 32, sm, s>>>(Wh, P, F, X, T, B, alpha, G, loss_acc);
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

int qtt_mlp_adam_dev(float* P, __half* Wh, const float* G, float* M, float* V, int64_t n, float lr, int t,
                     cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P, Wh, G, M, V, n, lr, b1, b2, 1e-8f, c1, c2);
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

// Kernels of the learned warm start: a small dilated convolutional network that
// maps (log p, log q, log eps, log lambda) on a grid to initial potentials
// (U0, V0) for the scaling iteration (which replace b = 1 of Algorithm 1).
// Training and inference use only these kernels: 3x3 dilated convolution
// forward, its two backward products, Adam, the squared-error loss and the
// input-feature assembly.  FP32 throughout; activations are leaky ReLU.
//
// Layouts: activations [N][C][H][W] row-major; weights [Cout][Cin][3][3];
// biases [Cout].  Zero padding: out-of-image taps read 0.
#include <string.h>

#include <algorithm>

#include "uot_internal.cuh"

namespace uot {
namespace {

constexpr float kLeak = 0.1f;
constexpr int kCoTile = 8;   // output channels per thread
constexpr int kPixTile = 128; // pixels per block

__device__ __forceinline__ float act(float v, int leaky) { return (leaky && v < 0.0f) ? kLeak * v : v; }
__device__ __forceinline__ float dact(float y, int leaky) { return (leaky && y < 0.0f) ? kLeak : 1.0f; }

// y[n, co, p] = act(b[co] + sum_{ci, tap} w[co, ci, tap] x[n, ci, p + dil*(tap - 1)])
__global__ void __launch_bounds__(kPixTile)
    conv_fwd(const float* __restrict__ x, const float* __restrict__ w, const float* __restrict__ b,
             float* __restrict__ y, int Cin, int Cout, int H, int W, int dil, int leaky) {
  extern __shared__ float sw[];  // [kCoTile][Cin][9]
  const int p = blockIdx.x * kPixTile + threadIdx.x;
  const int co0 = blockIdx.y * kCoTile;
  const int n = blockIdx.z;
  const int HW = H * W;
  for (int t = threadIdx.x; t < kCoTile * Cin * 9; t += kPixTile) {
    const int k = t / (Cin * 9), r = t % (Cin * 9);
    sw[t] = (co0 + k < Cout) ? w[(int64_t)(co0 + k) * Cin * 9 + r] : 0.0f;
  }
  __syncthreads();
  if (p >= HW) return;
  const int h = p / W, wc = p % W;
  float acc[kCoTile];
#pragma unroll
  for (int k = 0; k < kCoTile; ++k) acc[k] = (co0 + k < Cout) ? b[co0 + k] : 0.0f;
  const float* xn = x + (int64_t)n * Cin * HW;
  for (int ci = 0; ci < Cin; ++ci) {
    const float* xc = xn + (int64_t)ci * HW;
#pragma unroll
    for (int kh = 0; kh < 3; ++kh) {
      const int hh = h + (kh - 1) * dil;
      const bool hin = hh >= 0 && hh < H;
#pragma unroll
      for (int kw = 0; kw < 3; ++kw) {
        const int ww = wc + (kw - 1) * dil;
        const float xv = (hin && ww >= 0 && ww < W) ? xc[hh * W + ww] : 0.0f;
        const int tap = kh * 3 + kw;
#pragma unroll
        for (int k = 0; k < kCoTile; ++k) acc[k] = fmaf(sw[(k * Cin + ci) * 9 + tap], xv, acc[k]);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kCoTile; ++k)
    if (co0 + k < Cout) y[((int64_t)n * Cout + co0 + k) * HW + p] = act(acc[k], leaky);
}

// dx[n, ci, p] = sum_{co, tap} w[co, ci, tap] g[n, co, p - dil*(tap - 1)],
// g = dy * act'(y)
__global__ void __launch_bounds__(kPixTile)
    conv_bwd_data(const float* __restrict__ w, const float* __restrict__ y,
                  const float* __restrict__ dy, float* __restrict__ dx, int Cin, int Cout, int H,
                  int W, int dil, int leaky) {
  extern __shared__ float sw[];  // [kCoTile ci][Cout][9]
  const int p = blockIdx.x * kPixTile + threadIdx.x;
  const int ci0 = blockIdx.y * kCoTile;
  const int n = blockIdx.z;
  const int HW = H * W;
  for (int t = threadIdx.x; t < kCoTile * Cout * 9; t += kPixTile) {
    const int k = t / (Cout * 9), r = t % (Cout * 9);
    const int co = r / 9, tap = r % 9;
    sw[t] = (ci0 + k < Cin) ? w[((int64_t)co * Cin + ci0 + k) * 9 + tap] : 0.0f;
  }
  __syncthreads();
  if (p >= HW) return;
  const int h = p / W, wc = p % W;
  float acc[kCoTile];
#pragma unroll
  for (int k = 0; k < kCoTile; ++k) acc[k] = 0.0f;
  for (int co = 0; co < Cout; ++co) {
    const float* dyc = dy + ((int64_t)n * Cout + co) * HW;
    const float* yc = y + ((int64_t)n * Cout + co) * HW;
#pragma unroll
    for (int kh = 0; kh < 3; ++kh) {
      const int hh = h - (kh - 1) * dil;
      const bool hin = hh >= 0 && hh < H;
#pragma unroll
      for (int kw = 0; kw < 3; ++kw) {
        const int ww = wc - (kw - 1) * dil;
        float g = 0.0f;
        if (hin && ww >= 0 && ww < W) {
          const int q = hh * W + ww;
          g = dyc[q] * dact(yc[q], leaky);
        }
        const int tap = kh * 3 + kw;
#pragma unroll
        for (int k = 0; k < kCoTile; ++k) acc[k] = fmaf(sw[(k * Cout + co) * 9 + tap], g, acc[k]);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kCoTile; ++k)
    if (ci0 + k < Cin) dx[((int64_t)n * Cin + ci0 + k) * HW + p] = acc[k];
}

// dw[co, ci, tap] += sum_{n in chunk, p} g[n, co, p] x[n, ci, p + dil*(tap - 1)];
// db[co] += sum g (ci-block 0 only).  One block per (co, ci block, n chunk).
constexpr int kWT = 256;
__global__ void __launch_bounds__(kWT)
    conv_bwd_weight(const float* __restrict__ x, const float* __restrict__ y,
                    const float* __restrict__ dy, float* __restrict__ dw, float* __restrict__ db,
                    int N, int Cin, int Cout, int H, int W, int dil, int leaky, int nchunk) {
  const int co = blockIdx.x;
  const int ci0 = blockIdx.y * kCoTile;
  const int n0 = blockIdx.z * nchunk, n1 = min(N, n0 + nchunk);
  const int HW = H * W;
  float acc[kCoTile][9];
#pragma unroll
  for (int k = 0; k < kCoTile; ++k)
#pragma unroll
    for (int t = 0; t < 9; ++t) acc[k][t] = 0.0f;
  float bacc = 0.0f;
  for (int n = n0; n < n1; ++n) {
    const float* dyc = dy + ((int64_t)n * Cout + co) * HW;
    const float* yc = y + ((int64_t)n * Cout + co) * HW;
    const float* xn = x + (int64_t)n * Cin * HW;
    for (int p = threadIdx.x; p < HW; p += kWT) {
      const float g = dyc[p] * dact(yc[p], leaky);
      bacc += g;
      const int h = p / W, wc = p % W;
#pragma unroll
      for (int kh = 0; kh < 3; ++kh) {
        const int hh = h + (kh - 1) * dil;
        const bool hin = hh >= 0 && hh < H;
#pragma unroll
        for (int kw = 0; kw < 3; ++kw) {
          const int ww = wc + (kw - 1) * dil;
          if (!(hin && ww >= 0 && ww < W)) continue;
          const int q = hh * W + ww;
#pragma unroll
          for (int k = 0; k < kCoTile; ++k)
            if (ci0 + k < Cin) acc[k][kh * 3 + kw] = fmaf(g, xn[(int64_t)(ci0 + k) * HW + q], acc[k][kh * 3 + kw]);
        }
      }
    }
  }
  // block reduction of the 8 x 9 partial sums (+ bias)
  __shared__ float red[kWT / 32];
#pragma unroll
  for (int k = 0; k < kCoTile; ++k) {
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      float v = acc[k][t];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      __syncthreads();
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
      __syncthreads();
      if (threadIdx.x == 0 && ci0 + k < Cin) {
        float s = 0.0f;
        for (int w2 = 0; w2 < kWT / 32; ++w2) s += red[w2];
        atomicAdd(&dw[((int64_t)co * Cin + ci0 + k) * 9 + t], s);
      }
    }
  }
  if (blockIdx.y == 0) {
    float v = bacc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      float s = 0.0f;
      for (int w2 = 0; w2 < kWT / 32; ++w2) s += red[w2];
      atomicAdd(&db[co], s);
    }
  }
}

__global__ void adam_kernel(float* __restrict__ prm, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    prm[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// grad = 2 (pred - target) / n ; loss accumulated in FP64 (one atomic per block)
__global__ void mse_kernel(const float* __restrict__ pred, const float* __restrict__ tgt,
                           float* __restrict__ grad, int64_t n, double* loss) {
  float acc = 0.0f;
  const float inv = 1.0f / (float)n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float d = pred[i] - tgt[i];
    grad[i] = 2.0f * d * inv;
    acc += d * d;
  }
  __shared__ float red[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    atomicAdd(loss, (double)s * (double)inv);
  }
}

// x[n, c, :] *= s[n] for every channel c (per-instance scale)
__global__ void scale_kernel(float* __restrict__ x, const float* __restrict__ sc, int N, int64_t per) {
  const int64_t total = (int64_t)N * per;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x)
    x[t] *= sc[t / per];
}

// features[n] = [clip(log p)/4, clip(log q)/4, log eps / 4, log lambda / 4]
__global__ void features_kernel(const float* __restrict__ p, const float* __restrict__ q,
                                const float* __restrict__ log_eps, const float* __restrict__ log_lam,
                                float* __restrict__ out, int N, int HW) {
  const int64_t total = (int64_t)N * HW;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = t / HW, px = t % HW;
    const float lp = fmaxf(logf(fmaxf(p[t], 1e-30f)), -30.0f);
    const float lq = fmaxf(logf(fmaxf(q[t], 1e-30f)), -30.0f);
    float* o = out + n * 4 * HW;
    o[px] = 0.25f * lp;
    o[HW + px] = 0.25f * lq;
    o[2 * HW + px] = 0.25f * log_eps[n];
    o[3 * HW + px] = 0.25f * log_lam[n];
  }
}

uot_status fail(cudaError_t e) { return e == cudaSuccess ? UOT_OK : (e == cudaErrorMemoryAllocation ? UOT_ENOMEM : UOT_ECUDA); }

}  // namespace
}  // namespace uot

using namespace uot;

extern "C" {

uot_status uot_conv2d_forward(const float* x, const float* w, const float* b, float* y, int N,
                              int Cin, int Cout, int H, int W, int dilation, int leaky, void* stream) {
  if (!x || !w || !b || !y || N < 1 || Cin < 1 || Cout < 1 || H < 1 || W < 1 || dilation < 1)
    return UOT_EINVAL;
  if (N > 65535) return UOT_EUNSUPPORTED;
  const size_t smem = (size_t)kCoTile * Cin * 9 * sizeof(float);
  if (smem > 48 * 1024) return UOT_EUNSUPPORTED;
  dim3 grid((H * W + kPixTile - 1) / kPixTile, (Cout + kCoTile - 1) / kCoTile, N);
  count_launches(1);
  conv_fwd<<<grid, kPixTile, smem, (cudaStream_t)stream>>>(x, w, b, y, Cin, Cout, H, W, dilation, leaky);
  return fail(cudaGetLastError());
}

uot_status uot_conv2d_backward(const float* x, const float* w, const float* y, const float* dy,
                               float* dx, float* dw, float* db, int N, int Cin, int Cout, int H,
                               int W, int dilation, int leaky, void* stream) {
  if (!x || !w || !y || !dy || !dw || !db || N < 1 || Cin < 1 || Cout < 1 || H < 1 || W < 1 ||
      dilation < 1)
    return UOT_EINVAL;
  if (N > 65535) return UOT_EUNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(dw, 0, (size_t)Cout * Cin * 9 * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(db, 0, (size_t)Cout * sizeof(float), s);
  if (e != cudaSuccess) return fail(e);
  if (dx) {
    const size_t smem = (size_t)kCoTile * Cout * 9 * sizeof(float);
    if (smem > 48 * 1024) return UOT_EUNSUPPORTED;
    dim3 grid((H * W + kPixTile - 1) / kPixTile, (Cin + kCoTile - 1) / kCoTile, N);
    count_launches(1);
    conv_bwd_data<<<grid, kPixTile, smem, s>>>(w, y, dy, dx, Cin, Cout, H, W, dilation, leaky);
  }
  const int nchunk = 4;
  dim3 gw(Cout, (Cin + kCoTile - 1) / kCoTile, (N + nchunk - 1) / nchunk);
  count_launches(1);
  conv_bwd_weight<<<gw, kWT, 0, s>>>(x, y, dy, dw, db, N, Cin, Cout, H, W, dilation, leaky, nchunk);
  return fail(cudaGetLastError());
}

uot_status uot_adam_step(float* param, const float* grad, float* m, float* v, long long n,
                         float lr, float beta1, float beta2, float eps, int step, void* stream) {
  if (!param || !grad || !m || !v || n < 1 || step < 1) return UOT_EINVAL;
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
  count_launches(1);
  adam_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(param, grad, m, v, n, lr, beta1, beta2, eps, c1, c2);
  return fail(cudaGetLastError());
}

uot_status uot_mse_grad(const float* pred, const float* target, float* grad, long long n,
                        double* loss_dev, void* stream) {
  if (!pred || !target || !grad || !loss_dev || n < 1) return UOT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(loss_dev, 0, sizeof(double), s);
  if (e != cudaSuccess) return fail(e);
  const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
  count_launches(1);
  mse_kernel<<<blocks, 256, 0, s>>>(pred, target, grad, n, loss_dev);
  return fail(cudaGetLastError());
}

uot_status uot_scale_instances(float* x, const float* scale, int N, long long per_instance,
                               void* stream) {
  if (!x || !scale || N < 1 || per_instance < 1) return UOT_EINVAL;
  const int64_t total = (int64_t)N * per_instance;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 8192);
  count_launches(1);
  scale_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(x, scale, N, per_instance);
  return fail(cudaGetLastError());
}

uot_status uot_warmstart_features(const float* p, const float* q, const float* log_eps,
                                  const float* log_lam, float* out, int N, int H, int W,
                                  void* stream) {
  if (!p || !q || !log_eps || !log_lam || !out || N < 1 || H < 1 || W < 1) return UOT_EINVAL;
  const int64_t total = (int64_t)N * H * W;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 8192);
  count_launches(1);
  features_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(p, q, log_eps, log_lam, out, N, H * W);
  return fail(cudaGetLastError());
}

}  // extern "C"

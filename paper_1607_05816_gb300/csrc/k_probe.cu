// Throughput probes of the pipes the scaling kernels are bound by (FP32 FMA,
// MUFU ex2, FP64 FMA, and the FP64 exponential exp() of the FP64 Gibbs passes
// as the library compiles it), reported in operations per clock per SM so that the
// result does not depend on the clock the GPU runs at.  Each thread runs
// kChains independent dependency chains (enough to cover the pipe latency);
// every block records its elapsed SM cycles with clock64(), and the host
// divides the total operations by SMs x the longest block's cycles.
#include <vector>

#include "uot_internal.cuh"

namespace uot {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) k_probe(int iters, float seed, long long* cycles, float* sink) {
  const long long t0 = clock64();
  float fv[kChains];
  double dv[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    fv[c] = seed + 1e-3f * (float)(threadIdx.x + c);
    dv[c] = (double)fv[c];
  }
  const float fa = 0.999f, fb = 1e-4f;
  const double da = 0.999, db = 1e-4;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        if (KIND == 0) {
          fv[c] = fmaf(fv[c], fa, fb);
        } else if (KIND == 1) {
          float y;
          asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(fv[c]));
          fv[c] = y * -0.5f;  // keeps the argument in [-1, 0]: no denormals or overflow
        } else if (KIND == 2) {
          dv[c] = fma(dv[c], da, db);
        } else {
          dv[c] = -0.5 * exp(dv[c]);  // keeps the argument in [-0.5, 0]
        }
      }
    }
  }
  float acc = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc += fv[c] + (float)dv[c];
  __syncthreads();
  if (threadIdx.x == 0) cycles[blockIdx.x] = clock64() - t0;
  if (acc == 12345.678f) sink[0] = acc;  // keeps the chains live
}

}  // namespace
}  // namespace uot

extern "C" uot_status uot_probe_pipes(double* out, void* stream) {
  using namespace uot;
  if (!out) return UOT_EINVAL;
  (void)cudaGetLastError();
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return UOT_ECUDA;
  // 8 resident blocks of 256 threads per SM: 64 warps, the SM's maximum
  const int blocks = sms * 8;
  long long* dcyc = nullptr;
  float* dsink = nullptr;
  if (cudaMallocAsync((void**)&dcyc, sizeof(long long) * blocks, s) != cudaSuccess) return UOT_ENOMEM;
  if (cudaMallocAsync((void**)&dsink, sizeof(float), s) != cudaSuccess) {
    cudaFreeAsync(dcyc, s);
    return UOT_ENOMEM;
  }
  std::vector<long long> h(blocks);
  uot_status st = UOT_OK;
  const int iters[4] = {4096, 1024, 64, 8};  // a few ms each
  for (int kind = 0; kind < 4 && st == UOT_OK; ++kind) {
    count_launches(1);
    if (kind == 0) k_probe<0><<<blocks, kProbeThreads, 0, s>>>(iters[kind], 0.5f, dcyc, dsink);
    if (kind == 1) k_probe<1><<<blocks, kProbeThreads, 0, s>>>(iters[kind], -0.5f, dcyc, dsink);
    if (kind == 2) k_probe<2><<<blocks, kProbeThreads, 0, s>>>(iters[kind], 0.5f, dcyc, dsink);
    if (kind == 3) k_probe<3><<<blocks, kProbeThreads, 0, s>>>(iters[kind], -0.25f, dcyc, dsink);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(h.data(), dcyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      st = UOT_ECUDA;
      break;
    }
    long long cmax = 1;
    for (long long c : h) cmax = c > cmax ? c : cmax;
    const double ops = (double)blocks * kProbeThreads * (double)iters[kind] * 16.0 * kChains;
    out[kind] = ops / ((double)sms * (double)cmax);
  }
  cudaFreeAsync(dcyc, s);
  cudaFreeAsync(dsink, s);
  return st;
}

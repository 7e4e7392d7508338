// Separable log-domain Gibbs operator on Cartesian grids (Sec. 4.4): for the
// cost |x - y|^2 the kernel is a product of 1-D kernels, so K(b.dy) is taken
// one axis at a time.  In the log domain each axis pass is a batch of 1-D
// log-sum-exp convolutions
//
//   z[i][l] = log sum_j exp(L[l][j] - (xo[i] - yi[j])^2 / eps)
//
// over `nlines` independent lines l.  The result is written transposed
// (point index i*nlines + l), so that d successive passes over the last axis
// cycle a row-major d-dimensional array back to row-major order.
//
// Work per pass: nlines * nout * nin exponentials.  The pass is bound by the
// SFU (MUFU.EX2) throughput in FP32 and by FP64 arithmetic in FP64.
//
// Layout: each warp owns one line and 32*R consecutive outputs (one per lane
// and register slot).  The warp stages its line in shared memory as
// {log2-scaled value, coordinate} pairs, shifted by the line's FP64 maximum, so
// every shared load is a broadcast; each lane then runs a max sweep and a
// sum-of-exponentials sweep over the line for its R outputs.
#include "uot_internal.cuh"

namespace uot {
namespace {

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double load_L(const double* __restrict__ in,
                                         const double* __restrict__ logw, int in_is_pot,
                                         int64_t idx, double inv_eps) {
  const double v = in[idx];
  if (!in_is_pot) return v;
  return (v == -kInf) ? -kInf : v * inv_eps + logw[idx];
}

// FP32 arithmetic, FP64 line values in and out.
template <int R, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
    grid_pass_f32(const double* __restrict__ in, const double* __restrict__ logw, int in_is_pot,
                  int nlines, int nin, const float* __restrict__ yi, int nout,
                  const float* __restrict__ xo, double eps, Epilogue epi) {
  extern __shared__ float2 sm_f2[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l = blockIdx.y * WARPS + warp;
  const int i0 = blockIdx.x * (32 * R);
  const int64_t bz = blockIdx.z;
  in += bz * (int64_t)nlines * nin;
  const double inv_eps = 1.0 / eps;
  double num = 0.0, den = 0.0;
  if (l < nlines) {
    float2* line = sm_f2 + (size_t)warp * nin;
    const int64_t base = (int64_t)l * nin;
    double mx = -kInf;
    for (int j = lane; j < nin; j += 32) mx = fmax(mx, load_L(in, logw, in_is_pot, base + j, inv_eps));
    mx = warp_max(mx);
    if (mx == -kInf) {
      // b = 0 on the whole line: every sum is empty.
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = i0 + lane + 32 * r;
        if (i < nout) {
          double a, b;
          apply_epilogue(epi, bz, (int64_t)i * nlines + l, -kInf, a, b);
          num += a;
          den += b;
        }
      }
    } else {
      for (int j = lane; j < nin; j += 32) {
        const double v = load_L(in, logw, in_is_pot, base + j, inv_eps);
        line[j] = make_float2((float)((v - mx) * (double)kLog2e), yi[j]);
      }
      __syncwarp();
      const float k2 = (float)((double)kLog2e * inv_eps);
      float xr[R], m[R], s[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = i0 + lane + 32 * r;
        xr[r] = xo[i < nout ? i : nout - 1];
        m[r] = -INFINITY;
        s[r] = 0.0f;
      }
      for (int j = 0; j < nin; ++j) {
        const float2 t = line[j];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float dd = xr[r] - t.y;
          m[r] = fmaxf(m[r], fmaf(-k2, dd * dd, t.x));
        }
      }
      for (int j = 0; j < nin; ++j) {
        const float2 t = line[j];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float dd = xr[r] - t.y;
          s[r] += ex2_approx(fmaf(-k2, dd * dd, t.x - m[r]));
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = i0 + lane + 32 * r;
        if (i < nout) {
          const double z = mx + (double)kLn2 * (double)m[r] + log((double)s[r]);
          double a, b;
          apply_epilogue(epi, bz, (int64_t)i * nlines + l, z, a, b);
          num += a;
          den += b;
        }
      }
    }
  }
  if (epi.err) block_add2<WARPS * 32>(num, den, epi.err);
}

// FP64 arithmetic throughout.
template <int R, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
    grid_pass_f64(const double* __restrict__ in, const double* __restrict__ logw, int in_is_pot,
                  int nlines, int nin, const double* __restrict__ yi, int nout,
                  const double* __restrict__ xo, double eps, Epilogue epi) {
  extern __shared__ double2 sm_d2[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l = blockIdx.y * WARPS + warp;
  const int i0 = blockIdx.x * (32 * R);
  const int64_t bz = blockIdx.z;
  in += bz * (int64_t)nlines * nin;
  const double inv_eps = 1.0 / eps;
  double num = 0.0, den = 0.0;
  if (l < nlines) {
    double2* line = sm_d2 + (size_t)warp * nin;
    const int64_t base = (int64_t)l * nin;
    double mx = -kInf;
    for (int j = lane; j < nin; j += 32) {
      const double v = load_L(in, logw, in_is_pot, base + j, inv_eps);
      line[j] = make_double2(v, yi[j]);
      mx = fmax(mx, v);
    }
    mx = warp_max(mx);
    __syncwarp();
    if (mx == -kInf) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = i0 + lane + 32 * r;
        if (i < nout) {
          double a, b;
          apply_epilogue(epi, bz, (int64_t)i * nlines + l, -kInf, a, b);
          num += a;
          den += b;
        }
      }
    } else {
      double xr[R], m[R], s[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = i0 + lane + 32 * r;
        xr[r] = xo[i < nout ? i : nout - 1];
        m[r] = -kInf;
        s[r] = 0.0;
      }
      for (int j = 0; j < nin; ++j) {
        const double2 t = line[j];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const double dd = xr[r] - t.y;
          m[r] = fmax(m[r], t.x - dd * dd * inv_eps);
        }
      }
      for (int j = 0; j < nin; ++j) {
        const double2 t = line[j];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const double dd = xr[r] - t.y;
          s[r] += exp((t.x - m[r]) - dd * dd * inv_eps);
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = i0 + lane + 32 * r;
        if (i < nout) {
          const double z = m[r] + log(s[r]);
          double a, b;
          apply_epilogue(epi, bz, (int64_t)i * nlines + l, z, a, b);
          num += a;
          den += b;
        }
      }
    }
  }
  if (epi.err) block_add2<WARPS * 32>(num, den, epi.err);
}

}  // namespace

cudaError_t launch_grid_pass(int prec, const double* in, const double* logw, int in_is_pot,
                             int nlines, int nin, const void* yi, int nout, const void* xo,
                             double eps, int nbatch, const Epilogue& epi, cudaStream_t s) {
  constexpr int R = 2, WARPS = 4;
  dim3 grid((nout + 32 * R - 1) / (32 * R), (nlines + WARPS - 1) / WARPS, nbatch);
  if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
  prof_mark_begin(PROF_GRID_PASS, s);
  count_launches(1);
  if (prec == UOT_F32) {
    const size_t smem = (size_t)WARPS * nin * sizeof(float2);
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(grid_pass_f32<R, WARPS>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    grid_pass_f32<R, WARPS><<<grid, WARPS * 32, smem, s>>>(
        in, logw, in_is_pot, nlines, nin, (const float*)yi, nout, (const float*)xo, eps, epi);
  } else {
    const size_t smem = (size_t)WARPS * nin * sizeof(double2);
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(grid_pass_f64<R, WARPS>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    grid_pass_f64<R, WARPS><<<grid, WARPS * 32, smem, s>>>(
        in, logw, in_is_pot, nlines, nin, (const double*)yi, nout, (const double*)xo, eps, epi);
  }
  prof_mark_end(PROF_GRID_PASS, s);
  return cudaGetLastError();
}

}  // namespace uot

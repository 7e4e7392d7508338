// Row-wise Gibbs operators for explicit cost matrices and point clouds.
//
// Log domain (Sec. 4.3, absorption after every update):
//   z_i = log sum_j exp(L_j - C_ij/eps),   L_j = W_j/eps + log w_j,
// with C_ij read from a dense row-major matrix or recomputed as |x_i - y_j|^2
// (point clouds; the cost is never stored).  One warp per row: a max sweep and
// a sum sweep over j, lanes strided over j, then warp reductions.  L is first
// shifted by its FP64 maximum (prepare_L) so the FP32 variant only ever sees
// values <= 0.
//
// Algorithm 1 (Sec. 4.2): a_i = proxdiv_F(sum_j K_ij b_j w_j, eps) on a stored
// FP64 kernel K = exp(-C/eps), with the proxdiv column of Table 1 (u = 0).
#include "uot_internal.cuh"

namespace uot {
namespace {

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <typename T>
__device__ __forceinline__ T wmax(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <typename T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// L_j = W_j/eps + log w_j in FP64; then Lt_j = (L_j - max L) in T, scaled by
// log2(e) for the FP32 variant.  Single block; *Lmax receives max L.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) prepare_L(const double* __restrict__ W,
                                                const double* __restrict__ logw, int nin,
                                                double eps, T* __restrict__ Lt,
                                                double* __restrict__ Lmax) {
  __shared__ double red[NT / 32];
  double mx = -kInf;
  for (int j = threadIdx.x; j < nin; j += NT) {
    const double w = W[j];
    const double L = (w == -kInf) ? -kInf : w / eps + logw[j];
    mx = fmax(mx, L);
  }
  mx = wmax(mx);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < NT / 32) ? red[threadIdx.x] : -kInf;
    v = wmax(v);
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  mx = red[0];
  for (int j = threadIdx.x; j < nin; j += NT) {
    const double w = W[j];
    const double L = (w == -kInf) ? -kInf : w / eps + logw[j];
    double v = (mx == -kInf) ? -kInf : L - mx;
    if (sizeof(T) == 4) v *= (double)kLog2e;
    Lt[j] = (T)v;
  }
  if (threadIdx.x == 0) *Lmax = mx;
}

template <typename T, int DMAX>
struct RowCtx {
  T xi[DMAX];
};

// Cost of entry (i, j) in "cost/eps" units scaled as the variant requires.
template <typename T, int DMAX>
__device__ __forceinline__ T cost_ij(int kind, const T* __restrict__ C, const T* __restrict__ y,
                                     int d, int64_t rowbase, int j, const RowCtx<T, DMAX>& c) {
  if (kind == UOT_GEOM_DENSE) return C[rowbase + j];
  T acc = 0;
#pragma unroll
  for (int k = 0; k < DMAX; ++k) {
    if (k < d) {
      const T t = c.xi[k] - y[(int64_t)j * d + k];
      acc = fma(t, t, acc);
    }
  }
  return acc;
}

template <typename T, int DMAX, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
    rows_lse(int kind, const T* __restrict__ C, const T* __restrict__ x, const T* __restrict__ y,
             int d, int nrows, int nin, const T* __restrict__ Lt,
             const double* __restrict__ Lmax_p, double eps, Epilogue epi) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * WARPS + warp;
  double num = 0.0, den = 0.0;
  const double Lmax = *Lmax_p;
  if (i < nrows) {
    if (Lmax == -kInf) {
      if (lane == 0) apply_epilogue(epi, 0, i, -kInf, num, den);
    } else {
      RowCtx<T, DMAX> c;
      if (kind == UOT_GEOM_POINTS) {
#pragma unroll
        for (int k = 0; k < DMAX; ++k) c.xi[k] = (k < d) ? x[(int64_t)i * d + k] : T(0);
      }
      const int64_t rowbase = (int64_t)i * nin;
      // FP32 works in log2 units, FP64 in natural units.
      const T k2 = (sizeof(T) == 4) ? T((double)kLog2e / eps) : T(1.0 / eps);
      T m = -INFINITY;
      for (int j = lane; j < nin; j += 32)
        m = fmax(m, fma(-k2, cost_ij<T, DMAX>(kind, C, y, d, rowbase, j, c), Lt[j]));
      m = wmax(m);
      T s = 0;
      // m = -inf: every term vanishes (C = +inf where the input is finite)
      if (m != -INFINITY)
        for (int j = lane; j < nin; j += 32) {
          const T a = fma(-k2, cost_ij<T, DMAX>(kind, C, y, d, rowbase, j, c), Lt[j] - m);
          if (sizeof(T) == 4)
            s += ex2_approx((float)a);
          else if (a > -746.0)  // below, e^a is 0 in FP64: skip the FP64 exponential
            s += exp((double)a);
        }
      s = wsum(s);
      if (lane == 0 && m == -INFINITY) {
        apply_epilogue(epi, 0, i, -kInf, num, den);
      } else if (lane == 0) {
        const double z = Lmax + ((sizeof(T) == 4) ? (double)kLn2 * (double)m : (double)m) +
                         log((double)s);
        apply_epilogue(epi, 0, i, z, num, den);
      }
    }
  }
  if (epi.err) block_add2<WARPS * 32>(num, den, epi.err);
}

// FP32 path: L_j = W_j/eps + log w_j in float-float; Lt_j = (L_j - max) log2(e)
// in FP32; *Lmax (a float) receives the maximum of the high parts.
template <int NT>
__global__ void __launch_bounds__(NT) prepare_L_ff(const float2* __restrict__ W,
                                                   const float2* __restrict__ logw, int nin,
                                                   float2 inv_eps, float* __restrict__ Lt,
                                                   float* __restrict__ Lmax) {
  __shared__ float red[NT / 32];
  float mx = -INFINITY;
  for (int j = threadIdx.x; j < nin; j += NT) {
    const ff w = ffl(W[j]);
    const ff L = (w.hi == -INFINITY) ? ff_ninf() : ff_add(ff_mul(w, ffl(inv_eps)), ffl(logw[j]));
    mx = fmaxf(mx, L.hi);
  }
  mx = wmax(mx);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = (threadIdx.x < NT / 32) ? red[threadIdx.x] : -INFINITY;
    v = wmax(v);
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  mx = red[0];
  for (int j = threadIdx.x; j < nin; j += NT) {
    const ff w = ffl(W[j]);
    const ff L = (w.hi == -INFINITY) ? ff_ninf() : ff_add(ff_mul(w, ffl(inv_eps)), ffl(logw[j]));
    Lt[j] = (mx == -INFINITY || L.hi == -INFINITY) ? -INFINITY : ((L.hi - mx) + L.lo) * kLog2e;
  }
  if (threadIdx.x == 0) *Lmax = mx;
}

template <int DMAX, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
    rows_lse_f32(int kind, const float* __restrict__ C, const float* __restrict__ x,
                 const float* __restrict__ y, int d, int nrows, int nin,
                 const float* __restrict__ Lt, const float* __restrict__ Lmax_p, float k2,
                 Epilogue epi) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * WARPS + warp;
  float num = 0.0f, den = 0.0f;
  const float Lmax = *Lmax_p;
  if (i < nrows) {
    if (Lmax == -INFINITY) {
      if (lane == 0) apply_epilogue_ff(epi, 0, i, ff_ninf(), num, den);
    } else {
      RowCtx<float, DMAX> c;
      if (kind == UOT_GEOM_POINTS) {
#pragma unroll
        for (int k = 0; k < DMAX; ++k) c.xi[k] = (k < d) ? x[(int64_t)i * d + k] : 0.0f;
      }
      const int64_t rowbase = (int64_t)i * nin;
      float m = -INFINITY;
      for (int j = lane; j < nin; j += 32)
        m = fmaxf(m, fmaf(-k2, cost_ij<float, DMAX>(kind, C, y, d, rowbase, j, c), Lt[j]));
      m = wmax(m);
      float s = 0.0f;
      // m = -inf: every term vanishes (C = +inf where the input is finite)
      if (m != -INFINITY)
        for (int j = lane; j < nin; j += 32)
          s += ex2_approx(fmaf(-k2, cost_ij<float, DMAX>(kind, C, y, d, rowbase, j, c), Lt[j] - m));
      s = wsum(s);
      if (lane == 0 && m == -INFINITY) {
        apply_epilogue_ff(epi, 0, i, ff_ninf(), num, den);
      } else if (lane == 0) {
        const ff ln2 = ff{0.693147182464599609375f, -1.904654323148236017e-09f};
        float lg;
        asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lg) : "f"(s));
        const ff z = ff_add_f(ff_add_f(ff_mul_f(ln2, m), Lmax), kLn2 * lg);
        apply_epilogue_ff(epi, 0, i, z, num, den);
      }
    }
  }
  if (epi.err) block_add2f<WARPS * 32>(num, den, epi.err);
}

// Table 1 proxdiv column with u = 0 (non-log form), 0/0 = 0.
__device__ inline double proxdiv_plain(const DivParams& F, double p, double s, double eps) {
  if (!(s > 0.0)) return 0.0;
  const double ps = p / s;
  switch (F.kind) {
    case UOT_DIV_EQ:
      return ps;
    case UOT_DIV_KL:
      return pow(ps, F.lam / (F.lam + eps));
    case UOT_DIV_TV:
      return fmin(exp(F.lam / eps), fmax(exp(-F.lam / eps), ps));
    default: {
      const double lo = exp(F.log_alpha) * ps;
      const double inner = fmax(lo, 1.0);
      return (F.log_beta == kInf) ? inner : fmin(exp(F.log_beta) * ps, inner);
    }
  }
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
    alg1_half(const double* __restrict__ K, int nrows, int nin, const double* __restrict__ b,
              const double* __restrict__ w, const double* __restrict__ p, DivParams F, double eps,
              double* __restrict__ a, const double* __restrict__ wout, double* err) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * WARPS + warp;
  double num = 0.0, den = 0.0;
  if (i < nrows) {
    const double* row = K + (int64_t)i * nin;
    double s = 0.0;
    for (int j = lane; j < nin; j += 32) s = fma(row[j], b[j] * w[j], s);
    s = wsum(s);
    if (lane == 0) {
      const double aold = a[i];
      const double anew = proxdiv_plain(F, p[i], s, eps);
      a[i] = anew;
      if (err) {
        num = wout[i] * fabs(aold * s - anew * s);
        den = wout[i] * anew * s;
      }
    }
  }
  if (err) block_add2<WARPS * 32>(num, den, err);
}

}  // namespace

cudaError_t launch_rows(int prec, const RowsGeom& g, int nrows, int nin, const double* W,
                        const double* logw, double eps, void* scratch_L, const Epilogue& epi,
                        cudaStream_t s, float* zprev, int use_prev, void* part) {
  // scratch_L: nin elements of the precision's type followed by one double (Lmax).
  constexpr int WARPS = 8;
  const int grid = (nrows + WARPS - 1) / WARPS;
  if (g.kind == UOT_GEOM_POINTS && (g.d < 1 || g.d > 8)) return cudaErrorInvalidValue;
  count_launches(2);
  if (prec == UOT_F32 && g.kind == UOT_GEOM_POINTS && g.d <= 3 && part) {
    // chunked point-cloud kernels; scratch_L holds the block maxima
    count_launches(-2);
    return launch_points((const float*)g.x, (const float*)g.y, g.d, nrows, nin, W, logw, eps,
                         (float*)scratch_L, zprev, use_prev, reinterpret_cast<float2*>(part), epi, s);
  }
  if (prec == UOT_F32) {
    float* Lt = (float*)scratch_L;
    float* Lmax = (float*)((char*)scratch_L + (((size_t)nin * 4 + 255) & ~(size_t)255));
    prepare_L_ff<1024><<<1, 1024, 0, s>>>(reinterpret_cast<const float2*>(W),
                                           reinterpret_cast<const float2*>(logw), nin,
                                           ff2(ff_make(1.0 / eps)), Lt, Lmax);
    prof_mark_begin(PROF_ROWS, s);
    const float* C = (const float*)g.C;
    const float* x = (const float*)g.x;
    const float* y = (const float*)g.y;
    const float k2 = (float)((double)kLog2e / eps);
    if (g.kind == UOT_GEOM_DENSE || g.d <= 4)
      rows_lse_f32<4, WARPS><<<grid, WARPS * 32, 0, s>>>(g.kind, C, x, y, g.d, nrows, nin, Lt, Lmax, k2, epi);
    else
      rows_lse_f32<8, WARPS><<<grid, WARPS * 32, 0, s>>>(g.kind, C, x, y, g.d, nrows, nin, Lt, Lmax, k2, epi);
  } else {
    double* Lt = (double*)scratch_L;
    double* Lmax = (double*)((char*)scratch_L + (((size_t)nin * 8 + 255) & ~(size_t)255));
    prepare_L<double, 1024><<<1, 1024, 0, s>>>(W, logw, nin, eps, Lt, Lmax);
    prof_mark_begin(PROF_ROWS, s);
    const double* C = (const double*)g.C;
    const double* x = (const double*)g.x;
    const double* y = (const double*)g.y;
    if (g.kind == UOT_GEOM_DENSE || g.d <= 4)
      rows_lse<double, 4, WARPS><<<grid, WARPS * 32, 0, s>>>(g.kind, C, x, y, g.d, nrows, nin,
                                                            Lt, Lmax, eps, epi);
    else
      rows_lse<double, 8, WARPS><<<grid, WARPS * 32, 0, s>>>(g.kind, C, x, y, g.d, nrows, nin,
                                                            Lt, Lmax, eps, epi);
  }
  prof_mark_end(PROF_ROWS, s);
  return cudaGetLastError();
}

cudaError_t launch_alg1_half(const double* K, int nrows, int nin, const double* b,
                             const double* w, const double* p, DivParams F, double eps,
                             double* a, const double* wout, double* err, cudaStream_t s) {
  constexpr int WARPS = 8;
  count_launches(1);
  alg1_half<WARPS><<<(nrows + WARPS - 1) / WARPS, WARPS * 32, 0, s>>>(K, nrows, nin, b, w, p, F,
                                                                      eps, a, wout, err);
  return cudaGetLastError();
}

}  // namespace uot

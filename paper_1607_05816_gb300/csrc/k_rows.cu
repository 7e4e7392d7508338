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
#include <string.h>

#include <cooperative_groups.h>

#include <algorithm>

#include "uot_internal.cuh"

namespace uot {
namespace {


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
// log2(e) for the FP32 variant.  Single block; *Lmax receives max L.  Lt32,
// if given, receives an FP32 copy of the FP64 Lt (the prefilter's input).
template <typename T, int NT>
__global__ void __launch_bounds__(NT) prepare_L(const double* __restrict__ W,
                                                const double* __restrict__ logw, int nin,
                                                double eps, T* __restrict__ Lt,
                                                double* __restrict__ Lmax, float* __restrict__ Lt32 = nullptr) {
  __shared__ double red[NT / 32];
  const double inv_eps = 1.0 / eps;
  double mx = -kInf;
  // L_j is stored unshifted first, then shifted in place (one FP64 evaluation each)
  for (int j = threadIdx.x; j < nin; j += NT) {
    const double w = W[j];
    const double L = (w == -kInf) ? -kInf : fma(w, inv_eps, logw[j]);
    mx = fmax(mx, L);
    if (sizeof(T) == 8) reinterpret_cast<double*>(Lt)[j] = L;
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
    double L;
    if (sizeof(T) == 8) {
      L = reinterpret_cast<const double*>(Lt)[j];
    } else {
      const double w = W[j];
      L = (w == -kInf) ? -kInf : fma(w, inv_eps, logw[j]);
    }
    double v = (mx == -kInf) ? -kInf : L - mx;
    if (sizeof(T) == 4) v *= (double)kLog2e;
    Lt[j] = (T)v;
    if (Lt32) Lt32[j] = (float)v;
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

__device__ __forceinline__ void pdl_wait_prev() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch with programmatic dependent launch: the kernel may start while its
// predecessor drains and waits for it (griddepcontrol.wait) before reading
// anything the predecessor writes.
template <typename Kern, typename... Args>
cudaError_t launch_pdl(Kern kern, dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

constexpr int kPfStageMax = 12288;  // inputs staged in shared memory (48 KB)
constexpr int kPfPrepBlocks = 32;   // blocks of the prefilter's line preparation

// Line preparation of the FP64 prefilter, spread over up to kPfPrepBlocks
// blocks: L_j = W_j/eps + log w_j in FP64 (L64, for the surviving terms) and
// as a float-float pair (Lff), and per-block maxima.  The last block to
// finish (an atomic counter, no waiting) merges the maxima into *Lmax and
// writes the shifted FP32 line Lt32_j = L_j - max L from the pairs with FP32
// operations only (the FP64 pipe of one SM would take longer).  With merge =
// 0 only L64 and Lff are written (any number of blocks): the consumer stages
// the line and finds its maximum itself.
__global__ void __launch_bounds__(256) prepare_L_pf(const double* __restrict__ W, const double* __restrict__ logw,
                                                   int nin, double inv_eps, double* __restrict__ L64,
                                                   float2* __restrict__ Lff, double* __restrict__ Lmax,
                                                   float* __restrict__ Lt32, float* __restrict__ lerr,
                                                   double* __restrict__ part, unsigned* __restrict__ count,
                                                   int merge) {
  __shared__ double red[8];
  __shared__ bool last;
  pdl_wait_prev();  // W is the preceding kernel's output
  pdl_release_next();
  double mx = -kInf;
  for (int j = blockIdx.x * 256 + threadIdx.x; j < nin; j += gridDim.x * 256) {
    const double w = W[j];
    const double L = (w == -kInf) ? -kInf : fma(w, inv_eps, logw[j]);
    L64[j] = L;
    const float hi = (float)L;
    Lff[j] = make_float2(hi, (L == -kInf) ? 0.0f : (float)(L - (double)hi));
    mx = fmax(mx, L);
  }
  if (!merge) return;
  mx = wmax(mx);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < 8; ++k) mx = fmax(mx, red[k]);
    part[blockIdx.x] = mx;
    __threadfence();
    last = atomicAdd(count, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < 32) {  // gridDim.x <= 32 partials, one per lane
    mx = (threadIdx.x < gridDim.x) ? __ldcg(&part[threadIdx.x]) : -kInf;
    mx = wmax(mx);
    if (threadIdx.x == 0) red[0] = mx;
  }
  __syncthreads();
  mx = red[0];
  const float mhi = (float)mx;
  const float mlo = (mx == -kInf) ? 0.0f : (float)(mx - (double)mhi);
#pragma unroll 4
  for (int j = threadIdx.x; j < nin; j += 256) {
    const float2 l = __ldcg(&Lff[j]);
    Lt32[j] = (mx == -kInf || l.x == -INFINITY) ? -INFINITY : (l.x - mhi) + (l.y - mlo);
  }
  if (threadIdx.x == 0) {
    *Lmax = mx;
    // the pairs carry |L| 2^-47 of representation error besides the FP32 rounding
    *lerr = (mx == -kInf) ? 4.0f : fmaf(fabsf(mhi), 0x1p-44f, 4.0f);
    *count = 0u;
  }
}

// FP64 rows of a dense cost with an FP32 prefilter.  GB300's FP64 pipe
// issues 2 operations per clock per SM against 128 for FP32, and at small eps
// most terms of a row underflow (e^a = 0 in FP64 for a < -745.2).  The max
// sweep and a conservative skip test therefore run on FP32 copies of C and of
// the shifted input line; the columns that can reach the FP64 range are
// collected per warp (ballot, shared-memory list) and evaluated in FP64 32 at
// a time with every lane active, shifted by the FP32 maximum (converted
// exactly), so the result is the plain FP64 row sum up to FP64 rounding.  The
// warps' leftover lists (< 32 each) are pooled per CTA and evaluated in full
// batches too, and every sum is taken in a fixed order.  WPR warps share a row
// (RPC rows per CTA) so that enough loads are in flight.
template <int WPR, int RPC, bool kRows>
__global__ void __launch_bounds__(WPR * RPC * 32)
    rows_lse_f64_pf(const double* __restrict__ C, const float* __restrict__ C32, int nrows, int nin,
                    const double* __restrict__ L64, const float* __restrict__ Lt32,
                    const double* __restrict__ Lmax_p, const float* __restrict__ lerr_p,
                    const float2* __restrict__ Lff, double k2, Epilogue epi) {
  constexpr int NT = WPR * RPC * 32, NW = WPR * RPC;
  // shared memory: the shifted FP32 input line (when it fits) and, with kRows,
  // the CTA's RPC rows of C32, copied in with cp.async so that every byte is
  // in flight at once and both sweeps read shared memory
  extern __shared__ float sL[];
  __shared__ float sm_m[RPC][WPR];
  __shared__ double sm_s[RPC][WPR];
  __shared__ double rsum[RPC];
  __shared__ int slist[NW][64];
  __shared__ int pool[NW * 32];     // leftover columns, warp by warp (so row by row)
  __shared__ double pval[NW * 32];  // their FP64 terms
  __shared__ int woff[NW + 1];      // exclusive prefix sum of the warps' leftover counts
  __shared__ float sm_lm[NW];       // the warps' maxima of the line (kRows)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rloc = warp / WPR, part = warp % WPR;
  const int i = blockIdx.x * RPC + rloc;
  double num = 0.0, den = 0.0;
  const bool staged = kRows || nin <= kPfStageMax;
  double Lmax;
  float lerr;
  if (kRows) {
    // nin % 4 == 0 and 16-byte aligned C32: 16-byte copies of the rows (the cost does
    // not depend on the preceding kernel, so they are issued before waiting for it)
    const int q = nin >> 2;
    const int nr = min(RPC, nrows - (int)blockIdx.x * RPC);
    for (int t = threadIdx.x; t < q * nr; t += NT) {
      const int r = t / q, c4 = t - r * q;
      const float* src = C32 + ((int64_t)(blockIdx.x * RPC + r) * nin + 4 * c4);
      const unsigned dst = (unsigned)__cvta_generic_to_shared(sL + (size_t)(r + 1) * nin + 4 * c4);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    pdl_wait_prev();
    pdl_release_next();
    // the line from its float-float pairs: every CTA finds the same maximum
    // (mhi, the FP32 rounding of max L, so Lmax = mhi exactly) and writes the
    // shifted line Lt32_j = (hi_j - mhi) + lo_j with FP32 operations only
    float mloc = -INFINITY;
    for (int j = threadIdx.x; j < nin; j += NT) mloc = fmaxf(mloc, Lff[j].x);
    mloc = wmax(mloc);
    if (lane == 0) sm_lm[warp] = mloc;
    __syncthreads();
    float mhi = sm_lm[0];
#pragma unroll
    for (int w = 1; w < NW; ++w) mhi = fmaxf(mhi, sm_lm[w]);
    for (int j = threadIdx.x; j < nin; j += NT) {
      const float2 l = Lff[j];
      sL[j] = (mhi == -INFINITY || l.x == -INFINITY) ? -INFINITY : (l.x - mhi) + l.y;
    }
    Lmax = (mhi == -INFINITY) ? -kInf : (double)mhi;
    // the pairs carry |L| 2^-47 of representation error besides the FP32 rounding
    lerr = (mhi == -INFINITY) ? 4.0f : fmaf(fabsf(mhi), 0x1p-44f, 4.0f);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  } else {
    pdl_wait_prev();
    pdl_release_next();
    if (staged)
      for (int j = threadIdx.x; j < nin; j += NT) sL[j] = Lt32[j];
    Lmax = *Lmax_p;
    lerr = *lerr_p;
  }
  __syncthreads();
  const float* L = staged ? sL : Lt32;
  const bool live = i < nrows && Lmax != -kInf;  // warp-uniform
  const int64_t rowbase = (int64_t)(live ? i : 0) * nin;
  const float* crow = kRows ? sL + (size_t)(1 + rloc) * nin : C32 + rowbase;
  const float k2f = (float)k2;
  float m = -INFINITY;
  if (live) {
#pragma unroll 4
    for (int j = part * 32 + lane; j < nin; j += WPR * 32) m = fmaxf(m, fmaf(-k2f, crow[j], L[j]));
  }
  m = wmax(m);
  if (lane == 0) sm_m[rloc][part] = m;
  __syncthreads();
  m = sm_m[rloc][0];
#pragma unroll
  for (int w = 1; w < WPR; ++w) m = fmaxf(m, sm_m[rloc][w]);
  // FP64 term of column j of CTA row r, relative to that row's FP32 maximum
  auto term = [&](int r, int j) {
    const int64_t ri = (int64_t)(blockIdx.x * RPC + r);
    float mr = sm_m[r][0];
#pragma unroll
    for (int w = 1; w < WPR; ++w) mr = fmaxf(mr, sm_m[r][w]);
    const double a64 = fma(-k2, C[ri * nin + j], L64[j] - Lmax) - (double)mr;
    return a64 > -746.0 ? exp(a64) : 0.0;
  };
  double s = 0.0;
  int cnt = 0;  // warp-uniform
  int* lst = slist[warp];
  if (live && m != -INFINITY) {
    // warp-uniform sweep (the ballots need every lane)
    for (int j0 = part * 32; j0 < nin; j0 += WPR * 32) {
      const int j = j0 + lane;
      bool keep = false;
      if (j < nin) {
        const float c = crow[j], l = L[j];
        const float t = fmaf(-k2f, c, l);
        const float a = t - m;
        // |t - t_FP64| and the error of m are below (k2 c + |l| + |t| + |a|) 2^-22
        // (the roundings of k2, c, l, the fma and the subtraction) plus lerr
        const float tol = fmaf(fabsf(t) + fabsf(a) + fmaf(k2f, c, fabsf(l)), 0x1p-22f, lerr);
        keep = a > -746.0f - tol;
      }
      const unsigned mask = __ballot_sync(0xffffffffu, keep);
      if (mask) {
        if (keep) lst[cnt + __popc(mask & ((1u << lane) - 1u))] = j;
        cnt += __popc(mask);
        if (cnt >= 32) {  // a full batch: every lane evaluates one term
          __syncwarp();
          s += term(rloc, lst[lane]);
          const int rest = cnt - 32;
          const int carry = (lane < rest) ? lst[32 + lane] : 0;
          __syncwarp();
          if (lane < rest) lst[lane] = carry;
          __syncwarp();
          cnt = rest;
        }
      }
    }
  }
  if (__any_sync(0xffffffffu, s != 0.0)) s = wsum(s);  // most warps of a row hold no full batch
  if (lane == 0) sm_s[rloc][part] = s;
  // pool the leftovers (< 32 per warp) of the whole CTA in a fixed order (warp
  // by warp, hence row by row), evaluate them 32 at a time, and sum each row's
  // contiguous segment in a fixed order: the result does not depend on timing
  if (lane == 0) woff[warp] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int o = 0;
    for (int w = 0; w < NW; ++w) {
      const int c = woff[w];
      woff[w] = o;
      o += c;
    }
    woff[NW] = o;
  }
  __syncthreads();
  __syncwarp();
  if (lane < cnt) pool[woff[warp] + lane] = lst[lane];
  __syncthreads();
  const int np = woff[NW];
  for (int b = warp * 32; b < np; b += NT) {
    const int k = b + lane;
    if (k < np) {
      int r = 0;
      while (r + 1 < RPC && k >= woff[(r + 1) * WPR]) ++r;
      pval[k] = term(r, pool[k]);
    }
  }
  __syncthreads();
  if (warp < RPC) {
    double t = 0.0;
    for (int k = woff[warp * WPR] + lane; k < woff[(warp + 1) * WPR]; k += 32) t += pval[k];
    t = wsum(t);
    if (lane == 0) rsum[warp] = t;
  }
  __syncthreads();
  // the CTA's row epilogues (FP64 log and Table 1 row) side by side in the
  // lanes of warp 0: one warp instruction stream for RPC rows instead of one
  // per row on the narrow FP64 pipe
  if (warp == 0 && lane < RPC) {
    const int r = blockIdx.x * RPC + lane;
    if (r < nrows) {
      double z = -kInf;
      float mr = sm_m[lane][0];
      double sr = sm_s[lane][0] + rsum[lane];
#pragma unroll
      for (int w = 1; w < WPR; ++w) {
        mr = fmaxf(mr, sm_m[lane][w]);
        sr += sm_s[lane][w];
      }
      if (Lmax != -kInf && mr != -INFINITY) z = Lmax + (double)mr + log(sr);
      apply_epilogue(epi, 0, r, z, num, den);
    }
  }
  if (epi.err) block_add2<NT>(num, den, epi.err);
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
        const ff ln2 = ln2_ff();
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

// Algorithm 1 for one eps with the stored kernel resident in the shared memory
// of one thread-block cluster (CL CTAs, all iterations in one launch).  CTA r
// holds rows [r R, r R + R) of K and rows [r Q, r Q + Q) of K^T (R = ceil(n/CL),
// Q = ceil(m/CL)) and full copies of b (.) dy and a (.) dx.  A half-step is
// alg1_half's arithmetic (one warp per row, lane-strided FMAs, warp sum), so a
// and b are bit for bit those of the per-launch path.  After each half-step a
// cluster barrier, then every CTA copies the other CTAs' new entries out of
// their shared memory.  The violation sums of a checked iteration are reduced
// per CTA, and every CTA adds the CTAs' sums in the same order, so all of them
// take the same stop decision; there is no spin loop, only hardware barriers.
constexpr int kAlg1Warps = 16;

struct Alg1ClusterArgs {
  const double* K;
  const double* KT;
  int n, m, R, Q;
  const double *p, *dx, *q, *dy;
  DivParams F1, F2;
  double eps;
  double* a;  // [n] in/out
  double* b;  // [m] in/out
  int iters, check_every;  // check_every = 0: no checks
  double tol;
  double* res;  // [3]: violation of the last check, iterations run, converged (0/1)
};

__global__ void __launch_bounds__(kAlg1Warps * 32) alg1_cluster(Alg1ClusterArgs A) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double sh[];
  __shared__ double cpart[2];  // this CTA's violation sums, read by every CTA
  const int CL = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, NT = kAlg1Warps * 32;
  const int n = A.n, m = A.m, R = A.R, Q = A.Q;
  const int r0 = rank * R, nr = max(0, min(R, n - r0));
  const int c0 = rank * Q, nc = max(0, min(Q, m - c0));
  double* sK = sh;                      // [R][m]
  double* sKT = sK + (size_t)R * m;     // [Q][n]
  double* sbw = sKT + (size_t)Q * n;    // [m] b (.) dy
  double* saw = sbw + m;                // [n] a (.) dx
  double* sa = saw + n;                 // [R] this CTA's a
  double* sb = sa + R;                  // [Q] this CTA's b
  double* ssum = sb + Q;                // [max(R, Q)] row sums of the current half-step
  for (size_t t = threadIdx.x; t < (size_t)nr * m; t += NT) sK[t] = A.K[(size_t)r0 * m + t];
  for (size_t t = threadIdx.x; t < (size_t)nc * n; t += NT) sKT[t] = A.KT[(size_t)c0 * n + t];
  for (int j = threadIdx.x; j < m; j += NT) sbw[j] = A.b[j] * A.dy[j];
  for (int i = threadIdx.x; i < nr; i += NT) sa[i] = A.a[r0 + i];
  for (int j = threadIdx.x; j < nc; j += NT) sb[j] = A.b[c0 + j];
  __syncthreads();
  double err = INFINITY;
  int done = 0, conv = 0;
  for (int k = 0; k < A.iters; ++k) {
    const bool check = A.check_every > 0 && ((k + 1) % A.check_every == 0 || k == A.iters - 1);
    // a-update on this CTA's rows: the sums, then Table 1 one row per lane of
    // warp 0 (one FP64 instruction stream for all rows on the narrow FP64 pipe)
    for (int r = warp; r < nr; r += kAlg1Warps) {
      const double* row = sK + (size_t)r * m;
      double sacc = 0.0;
      for (int j = lane; j < m; j += 32) sacc = fma(row[j], sbw[j], sacc);
      sacc = wsum(sacc);
      if (lane == 0) ssum[r] = sacc;
    }
    __syncthreads();
    if (warp == 0) {
      double num = 0.0, den = 0.0;
      for (int r = lane; r < nr; r += 32) {
        const int i = r0 + r;
        const double sv = ssum[r], aold = sa[r];
        const double anew = proxdiv_plain(A.F1, A.p[i], sv, A.eps);
        sa[r] = anew;
        saw[i] = anew * A.dx[i];
        if (check) {
          num += A.dx[i] * fabs(aold * sv - anew * sv);
          den += A.dx[i] * anew * sv;
        }
      }
      if (check) {
        num = wsum(num);
        den = wsum(den);
        if (lane == 0) {
          cpart[0] = num;
          cpart[1] = den;
        }
      }
    }
    cluster.sync();
    // the other CTAs' a (.) dx
    for (int i = threadIdx.x; i < n; i += NT) {
      const int owner = i / R;
      if (owner != rank) saw[i] = *cluster.map_shared_rank(saw + i, owner);
    }
    if (check) {
      double tn = 0.0, td = 0.0;
      for (int c = 0; c < CL; ++c) {
        const double* pc = cluster.map_shared_rank(cpart, c);
        tn += pc[0];
        td += pc[1];
      }
      err = (td > 0.0) ? tn / td : 0.0;
    }
    __syncthreads();
    // b-update on this CTA's columns
    for (int r = warp; r < nc; r += kAlg1Warps) {
      const double* row = sKT + (size_t)r * n;
      double sacc = 0.0;
      for (int i = lane; i < n; i += 32) sacc = fma(row[i], saw[i], sacc);
      sacc = wsum(sacc);
      if (lane == 0) ssum[r] = sacc;
    }
    __syncthreads();
    if (warp == 0) {
      for (int r = lane; r < nc; r += 32) {
        const int j = c0 + r;
        const double bnew = proxdiv_plain(A.F2, A.q[j], ssum[r], A.eps);
        sb[r] = bnew;
        sbw[j] = bnew * A.dy[j];
      }
    }
    cluster.sync();
    for (int j = threadIdx.x; j < m; j += NT) {
      const int owner = j / Q;
      if (owner != rank) sbw[j] = *cluster.map_shared_rank(sbw + j, owner);
    }
    __syncthreads();
    done = k + 1;
    if (check && done > 1 && A.tol > 0.0 && err <= A.tol) {  // the same decision in every CTA
      conv = 1;
      break;
    }
  }
  for (int i = threadIdx.x; i < nr; i += NT) A.a[r0 + i] = sa[i];
  for (int j = threadIdx.x; j < nc; j += NT) A.b[c0 + j] = sb[j];
  if (rank == 0 && threadIdx.x == 0) {
    A.res[0] = err;
    A.res[1] = (double)done;
    A.res[2] = (double)conv;
  }
  cluster.sync();  // no CTA leaves while another may still read its shared memory
}

}  // namespace

size_t rows_pf_scratch_bytes(int64_t nin) {
  return 768 + 2 * (((size_t)nin * 8 + 255) & ~(size_t)255) + (((size_t)nin * 4 + 255) & ~(size_t)255);
}

cudaError_t launch_rows(int prec, const RowsGeom& g, int nrows, int nin, const double* W,
                        const double* logw, double eps, void* scratch_L, const Epilogue& epi,
                        cudaStream_t s, float* zprev, int use_prev, void* part, int precise) {
  if ((precise || precise_forced()) && prec == UOT_F32 && g.kind == UOT_GEOM_POINTS && g.d <= 3)
    return launch_points_ffp((const float*)g.x, (const float*)g.y, g.d, nrows, nin, W, logw, eps,
                             (float*)scratch_L, zprev, epi, s);
  // scratch_L: nin elements of the precision's type followed by one double
  // (Lmax); the FP64 dense prefilter adds nin floats, block maxima and a
  // counter (rows_pf_scratch_bytes).
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
    const double* C = (const double*)g.C;
    // dense rows with an FP32 copy of C: FP32 prefilter (k2 = 1/eps must stay an FP32 number)
    if (g.kind == UOT_GEOM_DENSE && g.C32 && 1.0 / eps < 1e30) {
      // scratch: counter (zeroed by the caller) | block maxima [kPfPrepBlocks] | Lmax, lerr |
      // L64 [nin] | Lff [nin] | Lt32 [nin]; the counter's place does not depend on nin
      char* base = (char*)scratch_L;
      const size_t r8 = ((size_t)nin * 8 + 255) & ~(size_t)255;
      double* Lmx = (double*)(base + 512);
      float* lerr = (float*)(base + 512 + 16);
      double* L64 = (double*)(base + 768);
      float2* Lff = (float2*)(base + 768 + r8);
      float* Lt32 = (float*)(base + 768 + 2 * r8);
      constexpr int WPR = 4, RPC = 4;
      const int grid2 = (nrows + RPC - 1) / RPC;
      // rows and line in shared memory: 16-byte rows (nin % 4 == 0) within 96 KB (opt-in
      // above 48 KB); the rows kernel then finds the line's maximum itself
      const size_t rows_bytes = (size_t)(1 + RPC) * nin * 4;
      const bool rows_smem = (nin % 4 == 0) && rows_bytes <= 96 * 1024 && ((uintptr_t)g.C32 % 16 == 0);
      const int pblk = rows_smem ? (nin + 255) / 256 : std::max(1, std::min(kPfPrepBlocks, (nin + 255) / 256));
      cudaError_t e0 = launch_pdl(prepare_L_pf, dim3(pblk), dim3(256), 0, s, W, logw, nin, 1.0 / eps, L64, Lff,
                                  Lmx, Lt32, lerr, (double*)(base + 256), (unsigned*)base, rows_smem ? 0 : 1);
      if (e0 != cudaSuccess) return e0;
      prof_mark_begin(PROF_ROWS, s);
      const float2* lff = Lff;
      if (rows_smem) {
        {  // opt-in for the current device: rows and line plus the static lists exceed 48 KB from
           // about 1920 columns on
          cudaError_t e = smem_at_least(rows_lse_f64_pf<WPR, RPC, true>, 96 * 1024);
          if (e != cudaSuccess) return e;
        }
        const float* c32 = g.C32;
        const double* l64 = L64;
        const float* lt32 = Lt32;
        const double* lmx = Lmx;
        const float* le = lerr;
        cudaError_t e1 = launch_pdl(rows_lse_f64_pf<WPR, RPC, true>, dim3(grid2), dim3(WPR * RPC * 32), rows_bytes, s,
                                    C, c32, nrows, nin, l64, lt32, lmx, le, lff, 1.0 / eps, epi);
        if (e1 != cudaSuccess) return e1;
      } else {
        const size_t smem = nin <= kPfStageMax ? (size_t)nin * 4 : 0;
        if (smem > 48 * 1024) return cudaErrorInvalidValue;
        // the line (up to 48 KB) and the static lists exceed the default 48 KB per block
        cudaError_t ea = smem_at_least(rows_lse_f64_pf<WPR, RPC, false>, kPfStageMax * 4);
        if (ea != cudaSuccess) return ea;
        const float* c32 = g.C32;
        const double* l64 = L64;
        const float* lt32 = Lt32;
        const double* lmx = Lmx;
        const float* le = lerr;
        cudaError_t e1 = launch_pdl(rows_lse_f64_pf<WPR, RPC, false>, dim3(grid2), dim3(WPR * RPC * 32), smem, s,
                                    C, c32, nrows, nin, l64, lt32, lmx, le, lff, 1.0 / eps, epi);
        if (e1 != cudaSuccess) return e1;
      }
      prof_mark_end(PROF_ROWS, s);
      return cudaGetLastError();
    }
    prepare_L<double, 1024><<<1, 1024, 0, s>>>(W, logw, nin, eps, Lt, Lmax);
    prof_mark_begin(PROF_ROWS, s);
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

size_t alg1_cluster_smem(int n, int m, int CL) {
  const size_t R = (n + CL - 1) / CL, Q = (m + CL - 1) / CL;
  return 8 * (R * m + Q * n + m + n + R + Q + std::max(R, Q));
}

cudaError_t launch_alg1_cluster(const double* K, const double* KT, int n, int m, const double* p,
                                const double* dx, const double* q, const double* dy, DivParams F1,
                                DivParams F2, double eps, double* a, double* b, int iters, int check_every,
                                double tol, double* res, cudaStream_t s, bool* launched) {
  *launched = false;
  for (int CL : {16, 8}) {
    const size_t smem = alg1_cluster_smem(n, m, CL);
    if (smem > 200 * 1024) continue;
    if (CL > 8 && cudaFuncSetAttribute(alg1_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      (void)cudaGetLastError();
      continue;
    }
    if (smem_at_least(alg1_cluster, smem) != cudaSuccess) {
      (void)cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(kAlg1Warps * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, alg1_cluster, &cfg) != cudaSuccess || nclusters < 1) {
      (void)cudaGetLastError();
      continue;
    }
    Alg1ClusterArgs A;
    A.K = K;
    A.KT = KT;
    A.n = n;
    A.m = m;
    A.R = (n + CL - 1) / CL;
    A.Q = (m + CL - 1) / CL;
    A.p = p;
    A.dx = dx;
    A.q = q;
    A.dy = dy;
    A.F1 = F1;
    A.F2 = F2;
    A.eps = eps;
    A.a = a;
    A.b = b;
    A.iters = iters;
    A.check_every = check_every;
    A.tol = tol;
    A.res = res;
    count_launches(1);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, alg1_cluster, A);
    if (e == cudaSuccess) *launched = true;
    return e;
  }
  return cudaSuccess;  // does not fit: the caller runs the per-launch path
}

cudaError_t launch_alg1_half(const double* K, int nrows, int nin, const double* b,
                             const double* w, const double* p, DivParams F, double eps,
                             double* a, const double* wout, double* err, cudaStream_t s) {
  count_launches(1);
  // one row per warp; with few rows, one warp per CTA so that every SM's
  // (narrow) FP64 pipe takes part
  if (nrows < 8 * 152) {
    alg1_half<1><<<nrows, 32, 0, s>>>(K, nrows, nin, b, w, p, F, eps, a, wout, err);
  } else {
    constexpr int WARPS = 8;
    alg1_half<WARPS><<<(nrows + WARPS - 1) / WARPS, WARPS * 32, 0, s>>>(K, nrows, nin, b, w, p, F, eps, a, wout,
                                                                        err);
  }
  return cudaGetLastError();
}

}  // namespace uot

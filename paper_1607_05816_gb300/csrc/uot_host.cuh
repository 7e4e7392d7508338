// Host orchestration shared by the C-ABI entry points (uot_api.cu,
// uot_solve.cu, uot_mass.cu, uot_wf.cu, uot_bary.cu): pointwise conversion and
// update kernels, argument checks, the stream-ordered scratch allocator, the
// Gibbs operator dispatch (grid passes, row kernels, point-cloud kernels),
// CUDA-graph blocks and the FP64 confirmation of FP32 stops.  Everything below
// is internal to each translation unit (anonymous namespace) except the
// process-wide state declared first, defined once in uot_api.cu.
#pragma once
#include <math.h>
#include <string.h>
#include <algorithm>
#include <cmath>
#include <atomic>
#include <mutex>
#include <string>
#include <utility>
#include <vector>
#include "uot_internal.cuh"
#include <cstring>

namespace uot {

// last error of this thread (uot_last_error), kernel launch counter, and the
// optional per-launch event timing of the Gibbs operator kernels
extern thread_local std::string g_last_error;
extern std::atomic<long long> g_launches;
// Optional CUDA-event timing of the Gibbs operator kernels: when enabled, an
// event pair brackets each launch on the launching stream.
struct Prof {
  std::mutex mu;
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> marks[PROF_NFAM];
  cudaEvent_t pending[PROF_NFAM] = {};
};
extern Prof g_prof;

namespace {



bool profiling_on() {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  return g_prof.on;
}

cudaEvent_t prof_event() {
  if (!g_prof.pool.empty()) {
    cudaEvent_t e = g_prof.pool.back();
    g_prof.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

uot_status fail_cuda(cudaError_t e, const char* what = nullptr, const char* file = nullptr, int line = 0) {
  g_last_error = cudaGetErrorString(e);
  if (what) {
    const char* base = file ? strrchr(file, '/') : nullptr;
    g_last_error += std::string(" [") + what + " @" + (base ? base + 1 : (file ? file : "?")) + ":" +
                    std::to_string(line) + "]";
  }
  return (e == cudaErrorMemoryAllocation) ? UOT_ENOMEM : UOT_ECUDA;
}

#define UOT_CK(expr)                                                \
  do {                                                              \
    cudaError_t e_ = (expr);                                        \
    if (e_ != cudaSuccess) return fail_cuda(e_, #expr, __FILE__, __LINE__); \
  } while (0)

// At the start of every entry point: drop a non-sticky CUDA error left by
// other code sharing this runtime, and the previous call's message, so that
// uot_last_error() describes this call only.
inline void clear_stale_error() {
  (void)cudaGetLastError();
  g_last_error.clear();
}

// ---------------------------------------------------------------------------
// pointwise kernels
// ---------------------------------------------------------------------------

// programmatic dependent launch: wait for the preceding kernel, then let the
// next one launch
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

constexpr int kNT = 256;

inline int nblocks(int64_t n) {
  int64_t b = (n + kNT - 1) / kNT;
  return (int)(b < 1 ? 1 : (b > 65535 * 8 ? 65535 * 8 : b));
}

template <typename T>
__global__ void k_to_log(const T* __restrict__ src, int64_t n, double* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)src[i];
    dst[i] = (v > 0.0) ? log(v) : -kInf;
  }
}

// FP32 path: per-point arrays hold float-float pairs in 8-byte slots.
__global__ void k_to_log_ff(const float* __restrict__ src, int64_t n, float2* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)src[i];
    dst[i] = ff2(ff_make(v > 0.0 ? log(v) : -kInf));
  }
}
__global__ void k_to_ff(const float* __restrict__ src, int64_t n, float2* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = make_float2(src[i], 0.0f);
}
__global__ void k_from_ff(const float2* __restrict__ src, int64_t n, float* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = src[i];
    dst[i] = (v.x == -INFINITY) ? v.x : v.x + v.y;
  }
}
// in place: float-float slot -> double slot (for FP64 reductions of FP32-path results)
__global__ void k_ff_to_double(double* __restrict__ a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = reinterpret_cast<const float2*>(a)[i];
    a[i] = (v.x == -INFINITY) ? -kInf : (double)v.x + (double)v.y;
  }
}

template <typename T>
__global__ void k_to_f64(const T* __restrict__ src, int64_t n, double* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

template <typename T>
__global__ void k_from_f64(const double* __restrict__ src, int64_t n, T* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (T)src[i];
}

// *flag = 1 if a and b differ anywhere (bit patterns).
__global__ void k_differs(const double* __restrict__ a, const double* __restrict__ b, int64_t n, int* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (__double_as_longlong(a[i]) != __double_as_longlong(b[i])) *flag = 1;
}

__global__ void k_fill(double* __restrict__ dst, int64_t n, double v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = v;
}

// FP32 path of k_add_logf: float-float V, float f.
__global__ void k_add_logf_ff(const double* __restrict__ Vd, const float* __restrict__ f, int ncols,
                              int col, int64_t n, double eps, double* __restrict__ Wd) {
  const float2* V = reinterpret_cast<const float2*>(Vd);
  float2* W = reinterpret_cast<float2*>(Wd);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const ff v = ffl(V[i]);
    const double fv = f ? (double)f[i * ncols + col] : 1.0;
    W[i] = (v.hi == -INFINITY || !(fv > 0.0)) ? ff2(ff_ninf()) : ff2(ff_add(v, ff_make(eps * log(fv))));
  }
}

// W = V + eps log f[:, col]  (apply_plan: fold a nonnegative function into the input)
template <typename T>
__global__ void k_add_logf(const double* __restrict__ V, const T* __restrict__ f, int ncols,
                           int col, int64_t n, double eps, double* __restrict__ W) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = V[i];
    const double fv = f ? (double)f[i * ncols + col] : 1.0;
    W[i] = (v == -kInf || !(fv > 0.0)) ? -kInf : v + eps * log(fv);
  }
}

template <typename T>
__global__ void k_transpose(const T* __restrict__ A, int n, int m, T* __restrict__ AT) {
  __shared__ T tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = by + r, j = bx + threadIdx.x;
    if (i < n && j < m) tile[r][threadIdx.x] = A[(int64_t)i * m + j];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = bx + r, i = by + threadIdx.x;
    if (i < n && j < m) AT[(int64_t)j * n + i] = tile[threadIdx.x][r];
  }
}

// K = exp(-C/eps) (eq. GibbsKernel) in FP64, and its transpose.
template <typename T>
__global__ void k_gibbs_matrix(const T* __restrict__ C, int n, int m, double eps,
                               double* __restrict__ K, double* __restrict__ KT) {
  const int64_t nm = (int64_t)n * m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nm;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / m, j = t % m;
    const double k = exp(-(double)C[t] / eps);
    K[t] = k;
    KT[j * n + i] = k;
  }
}

// scalings <-> potentials for Algorithm 1: a = exp(U/eps), U = eps log a.
__global__ void k_exp_scale(const double* __restrict__ U, int64_t n, double eps,
                            double* __restrict__ a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = exp(U[i] / eps);
}
__global__ void k_log_scale(const double* __restrict__ a, int64_t n, double eps,
                            double* __restrict__ U) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    U[i] = (a[i] > 0.0) ? eps * log(a[i]) : -kInf;
}

// *flag = 1 where a start potential is NaN or +inf (-inf is a valid zero scaling)
__global__ void k_bad_start(const double* __restrict__ a, int64_t n, int ffmode, int* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = ffmode ? (double)reinterpret_cast<const float2*>(a)[i].x : a[i];
    if (v != v || v == kInf) *flag = 1;
  }
}

__global__ void k_nan_flag(const double* __restrict__ a, int64_t n, int ffmode, int* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (ffmode) {
      const float2 v = reinterpret_cast<const float2*>(a)[i];
      if (v.x != v.x || v.y != v.y) *flag = 1;
    } else if (a[i] != a[i]) {
      *flag = 1;
    }
  }
}

// Barycenter F2 step (Sec. 5.2): from T_k = eps log s_k, the barycenter
//   KL (Table 2 ii): eps log h = (eps+lam) (log sum_k alpha_k e^{T_k/(eps+lam)} - log sum alpha)
//   EQ (Table 2 i):  eps log h = sum_k alpha_k T_k / sum alpha
// and V_k = prox for lam KL(.|h) (resp. the equality row) with p -> h.
// Table 2 (iii), (iv): the barycenter h solves f(w) = 0 for a continuous,
// non-decreasing, piecewise-linear f of w = eps log h (relative to a
// reference), with breakpoints known in closed form.  PLRoot collects, from
// f's values at the breakpoints, the brackets of r1 = min{f >= -tau} and
// r2 = max{f <= tau} (consecutive breakpoints, f being monotone) and returns
// the midpoint of [r1, r2], each end found by linear interpolation to f = 0.
// On a flat zero piece any point minimises the prox problem and the V updates
// do not depend on the choice; the midpoint is this library's reading.
template <typename R>
struct PLRoot {
  R l1b, l1f, r1b, r1f, l2b, l2f, r2b, r2f;
  bool hl1 = false, hr1 = false, hl2 = false, hr2 = false;
  __device__ void add(R b, R fb, R tau) {
    if (fb < -tau) {
      if (!hl1 || b > l1b) { l1b = b; l1f = fb; hl1 = true; }
    } else if (!hr1 || b < r1b) {
      r1b = b; r1f = fb; hr1 = true;
    }
    if (fb <= tau) {
      if (!hl2 || b > l2b) { l2b = b; l2f = fb; hl2 = true; }
    } else if (!hr2 || b < r2b) {
      r2b = b; r2f = fb; hr2 = true;
    }
  }
  __device__ void merge(const PLRoot& o) {
    if (o.hl1 && (!hl1 || o.l1b > l1b)) { l1b = o.l1b; l1f = o.l1f; hl1 = true; }
    if (o.hr1 && (!hr1 || o.r1b < r1b)) { r1b = o.r1b; r1f = o.r1f; hr1 = true; }
    if (o.hl2 && (!hl2 || o.l2b > l2b)) { l2b = o.l2b; l2f = o.l2f; hl2 = true; }
    if (o.hr2 && (!hr2 || o.r2b < r2b)) { r2b = o.r2b; r2f = o.r2f; hr2 = true; }
  }
  __device__ R root() const {
    const R r1 = hl1 ? (hr1 ? l1b + (R(0) - l1f) * (r1b - l1b) / (r1f - l1f) : l1b) : r1b;
    const R r2 = hr2 ? (hl2 ? l2b + (R(0) - l2f) * (r2b - l2b) / (r2f - l2f) : r2b) : l2b;
    return R(0.5) * (r1 + r2);
  }
};

// f of Table 2 (iii) (TV, kind 2) or (iv) (RG, kind 3) at w, from the inputs
// t_k (relative to the same reference; -inf for s_k = 0):
//   TV: A0 + sum_{t_k finite} alpha_k clamp((w - t_k)/lam, -1, 1), A0 = sum of alpha over s_k = 0
//   RG: sum_k alpha_k [b2 min(w - t_k + eps log b2, 0) + b1 max(w - t_k + eps log b1, 0)]
template <typename R>
__device__ R bary_pl_f(int kind, R w, const R* t, int64_t tstride, const R* alpha, int K, R lam, R elb1, R elb2,
                       R b1, R b2) {
  R f = R(0);
  for (int k = 0; k < K; ++k) {
    const R tk = t[k * tstride];
    if (kind == UOT_BARY_TV) {
      if (tk == -R(INFINITY)) f += alpha[k];
      else f += alpha[k] * fmin(R(1), fmax(R(-1), (w - tk) / lam));
    } else {
      f += alpha[k] * (b2 * fmin(w - tk + elb2, R(0)) + b1 * fmax(w - tk + elb1, R(0)));
    }
  }
  return f;
}

__global__ void k_bary_update(const double* __restrict__ T, int K, int64_t m,
                              const double* __restrict__ alpha, double sum_alpha, double lam,
                              double eps, int kind, double b1, double b2, double* __restrict__ logh,
                              double* __restrict__ V) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m;
       j += (int64_t)gridDim.x * blockDim.x) {
    double elogh;
    if (kind == UOT_BARY_TV || kind == UOT_BARY_RG) {
      // roots of Table 2 (iii)/(iv) in w = eps log h, from the 2K breakpoints
      double A0 = 0.0, Ap = 0.0;
      bool any_zero = false;
      for (int k = 0; k < K; ++k) {
        if (T[(int64_t)k * m + j] == -kInf) { A0 += alpha[k]; any_zero = true; }
        else Ap += alpha[k];
      }
      if ((kind == UOT_BARY_TV && A0 >= Ap) || (kind == UOT_BARY_RG && any_zero)) {
        elogh = -kInf;
      } else {
        const double elb1 = (kind == UOT_BARY_RG) ? eps * log(b1) : 0.0;
        const double elb2 = (kind == UOT_BARY_RG) ? eps * log(b2) : 0.0;
        const double tau = 1e-12 * sum_alpha * ((kind == UOT_BARY_TV) ? 1.0 : b2);
        PLRoot<double> pr;
        for (int k = 0; k < K; ++k) {
          const double tk = T[(int64_t)k * m + j];
          if (tk == -kInf) continue;
          for (int side = 0; side < 2; ++side) {
            const double b = (kind == UOT_BARY_TV) ? tk + (side ? lam : -lam) : tk - (side ? elb1 : elb2);
            pr.add(b, bary_pl_f<double>(kind, b, T + j, m, alpha, K, lam, elb1, elb2, b1, b2), tau);
          }
        }
        elogh = pr.root();
      }
    } else if (kind == UOT_BARY_KL) {
      const double c = 1.0 / (eps + lam);
      double mx = -kInf;
      for (int k = 0; k < K; ++k) mx = fmax(mx, log(alpha[k]) + T[(int64_t)k * m + j] * c);
      if (mx == -kInf) {
        elogh = -kInf;
      } else {
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += exp(log(alpha[k]) + T[(int64_t)k * m + j] * c - mx);
        elogh = (eps + lam) * (mx + log(s) - log(sum_alpha));
      }
    } else {
      double s = 0.0;
      for (int k = 0; k < K; ++k) s += alpha[k] * T[(int64_t)k * m + j];
      elogh = s / sum_alpha;
    }
    logh[j] = elogh;
    const double lh = (elogh == -kInf) ? -kInf : elogh / eps;
    DivParams F;
    F.kind = (kind == UOT_BARY_KL) ? UOT_DIV_KL : (kind == UOT_BARY_TV) ? UOT_DIV_TV
             : (kind == UOT_BARY_RG) ? UOT_DIV_RG : UOT_DIV_EQ;
    F.lam = lam;
    F.log_alpha = (kind == UOT_BARY_RG) ? log(b1) : 0.0;
    F.log_beta = (kind == UOT_BARY_RG) ? log(b2) : 0.0;
    for (int k = 0; k < K; ++k) V[(int64_t)k * m + j] = prox_update(F, lh, T[(int64_t)k * m + j], eps);
  }
}

// Barycenter update (Table 2 with Table 1 for the couplings' second marginals),
// float-float.  A CTA of kBJ x kBK threads takes 32 consecutive points j
// (lanes, coalesced over j) and splits the K measures over kBK warps; the
// per-point reductions over k (max and sum of the power mean, or the weighted
// geometric mean) are merged through shared memory.
constexpr int kBJ = 32, kBK = 8;

// TV and RG (Table 2 (iii), (iv)): the inputs of a point are staged relative
// to their largest finite value in dynamic shared memory ([K][kBJ] floats,
// then the K weights), each warp scans the breakpoints of its measures and
// the brackets of the root are merged over the kBK warps.
struct BaryPL {
  float lam, b1, b2, elb1, elb2;  // TV weight; RG range and eps log of its ends
};

__global__ void __launch_bounds__(kBJ * kBK)
    k_bary_update_ff(const double* __restrict__ Td, int K, int64_t m, const float* __restrict__ log_alpha,
                     float log_sum_alpha, float2 epslam, float2 inv_epslam, float2 inv_eps, float2 eps_ff,
                     int kind, DivFF Fh, BaryPL pl, double* __restrict__ loghd, double* __restrict__ Vd) {
  const float2* T = reinterpret_cast<const float2*>(Td);
  float2* logh = reinterpret_cast<float2*>(loghd);
  float2* V = reinterpret_cast<float2*>(Vd);
  __shared__ float r0[kBK][kBJ], r1[kBK][kBJ], r2[kBK][kBJ];
  __shared__ int rneg[kBK][kBJ];
  extern __shared__ float bsm[];  // TV/RG: [K][kBJ] staged inputs, then [K] weights
  const int lane = threadIdx.x, ky = threadIdx.y;
  const bool pwl = (kind == UOT_BARY_TV || kind == UOT_BARY_RG);
  float* sT = bsm;
  float* sAl = bsm + (size_t)K * kBJ;
  __shared__ float pb[kBK][8][kBJ];
  __shared__ unsigned char ph[kBK][4][kBJ];
  float sum_alpha = 0.0f;
  if (pwl) {
    for (int k = ky * kBJ + lane; k < K; k += kBJ * kBK) sAl[k] = expf(log_alpha[k]);
    __syncthreads();
    for (int k = 0; k < K; ++k) sum_alpha += sAl[k];
  }
  for (int64_t jb = (int64_t)blockIdx.x * kBJ; jb < m; jb += (int64_t)gridDim.x * kBJ) {
    const int64_t j = jb + lane;
    const bool valid = j < m;
    ff elogh;
    if (pwl) {
      float ref = -INFINITY, a0 = 0.0f, ap = 0.0f;
      int zero = 0;
      for (int k = ky; k < K && valid; k += kBK) {
        const ff t = ffl(T[(int64_t)k * m + j]);
        if (t.hi == -INFINITY) {
          a0 += sAl[k];
          zero = 1;
        } else {
          ap += sAl[k];
          ref = fmaxf(ref, t.hi);
        }
      }
      r0[ky][lane] = ref;
      r1[ky][lane] = a0;
      r2[ky][lane] = ap;
      rneg[ky][lane] = zero;
      __syncthreads();
      ref = -INFINITY;
      a0 = ap = 0.0f;
      zero = 0;
#pragma unroll
      for (int w = 0; w < kBK; ++w) {
        ref = fmaxf(ref, r0[w][lane]);
        a0 += r1[w][lane];
        ap += r2[w][lane];
        zero |= rneg[w][lane];
      }
      const bool hzero = !valid || ((kind == UOT_BARY_TV) ? (a0 >= ap) : (zero != 0));
      for (int k = ky; k < K && valid; k += kBK) {
        const ff t = ffl(T[(int64_t)k * m + j]);
        sT[(size_t)k * kBJ + lane] = (t.hi == -INFINITY) ? -INFINITY : ((t.hi - ref) + t.lo);
      }
      __syncthreads();
      PLRoot<float> pr;
      if (!hzero) {
        const float tau = 1e-6f * sum_alpha * ((kind == UOT_BARY_TV) ? 1.0f : pl.b2 * fabsf(pl.elb2 - pl.elb1) + 1e-30f);
        for (int k = ky; k < K; k += kBK) {
          const float tk = sT[(size_t)k * kBJ + lane];
          if (tk == -INFINITY) continue;
          for (int side = 0; side < 2; ++side) {
            const float b = (kind == UOT_BARY_TV) ? tk + (side ? pl.lam : -pl.lam) : tk - (side ? pl.elb1 : pl.elb2);
            pr.add(b, bary_pl_f<float>(kind, b, sT + lane, kBJ, sAl, K, pl.lam, pl.elb1, pl.elb2, pl.b1, pl.b2),
                   tau);
          }
        }
      }
      pb[ky][0][lane] = pr.l1b; pb[ky][1][lane] = pr.l1f; pb[ky][2][lane] = pr.r1b; pb[ky][3][lane] = pr.r1f;
      pb[ky][4][lane] = pr.l2b; pb[ky][5][lane] = pr.l2f; pb[ky][6][lane] = pr.r2b; pb[ky][7][lane] = pr.r2f;
      ph[ky][0][lane] = pr.hl1; ph[ky][1][lane] = pr.hr1; ph[ky][2][lane] = pr.hl2; ph[ky][3][lane] = pr.hr2;
      __syncthreads();
      if (hzero) {
        elogh = ff_ninf();
      } else {
        PLRoot<float> tot;
        for (int w = 0; w < kBK; ++w) {
          PLRoot<float> o;
          o.l1b = pb[w][0][lane]; o.l1f = pb[w][1][lane]; o.r1b = pb[w][2][lane]; o.r1f = pb[w][3][lane];
          o.l2b = pb[w][4][lane]; o.l2f = pb[w][5][lane]; o.r2b = pb[w][6][lane]; o.r2f = pb[w][7][lane];
          o.hl1 = ph[w][0][lane]; o.hr1 = ph[w][1][lane]; o.hl2 = ph[w][2][lane]; o.hr2 = ph[w][3][lane];
          tot.merge(o);
        }
        elogh = ff_add_f(ff{ref, 0.0f}, tot.root());
      }
    } else if (kind == UOT_BARY_KL) {
      // eps log h = (eps+lam) (LSE_k(log alpha_k + T_k/(eps+lam)) - log sum alpha)
      float mx = -INFINITY;
      for (int k = ky; k < K && valid; k += kBK) {
        const ff t = ffl(T[(int64_t)k * m + j]);
        if (t.hi != -INFINITY) mx = fmaxf(mx, ff_add_f(ff_mul(t, ffl(inv_epslam)), log_alpha[k]).hi);
      }
      r0[ky][lane] = mx;
      __syncthreads();
      mx = r0[0][lane];
#pragma unroll
      for (int w = 1; w < kBK; ++w) mx = fmaxf(mx, r0[w][lane]);
      float acc = 0.0f;
      if (mx != -INFINITY) {
        for (int k = ky; k < K && valid; k += kBK) {
          const ff t = ffl(T[(int64_t)k * m + j]);
          if (t.hi == -INFINITY) continue;
          const ff a = ff_add_f(ff_mul(t, ffl(inv_epslam)), log_alpha[k]);
          acc += expf((a.hi - mx) + a.lo);
        }
      }
      r1[ky][lane] = acc;
      __syncthreads();
      acc = 0.0f;
#pragma unroll
      for (int w = 0; w < kBK; ++w) acc += r1[w][lane];
      if (mx == -INFINITY) {
        elogh = ff_ninf();
      } else {
        const ff lead = ff_add_f(ff{mx, 0.0f}, logf(acc) - log_sum_alpha);
        elogh = ff_mul(lead, ffl(epslam));
      }
    } else {
      // eps log h = sum_k alpha_k T_k / sum alpha (geometric mean)
      ff acc = ff{0.0f, 0.0f};
      int neg_inf = 0;
      for (int k = ky; k < K && valid; k += kBK) {
        const ff t = ffl(T[(int64_t)k * m + j]);
        if (t.hi == -INFINITY) neg_inf = 1;
        else acc = ff_add(acc, ff_mul_f(t, expf(log_alpha[k] - log_sum_alpha)));
      }
      r0[ky][lane] = acc.hi;
      r1[ky][lane] = acc.lo;
      rneg[ky][lane] = neg_inf;
      __syncthreads();
      acc = ff{0.0f, 0.0f};
      neg_inf = 0;
#pragma unroll
      for (int w = 0; w < kBK; ++w) {
        acc = ff_add(acc, ff{r0[w][lane], r1[w][lane]});
        neg_inf |= rneg[w][lane];
      }
      elogh = neg_inf ? ff_ninf() : acc;
    }
    if (valid) {
      if (ky == 0) logh[j] = ff2(elogh);
      const ff lh = (elogh.hi == -INFINITY) ? ff_ninf() : ff_mul(elogh, ffl(inv_eps));
      for (int k = ky; k < K; k += kBK)
        V[(int64_t)k * m + j] = ff2(prox_update_ff(Fh, lh, ffl(T[(int64_t)k * m + j]), ffl(eps_ff)));
    }
    __syncthreads();  // the reduction buffers are reused by the next points
  }
}

// ---- objective terms (Theorem 3.2, Prop. A.3), FP64 ----

// F(r) = sum w Dbar(r|p) pointwise term
__device__ double div_term(const DivParams& F, double r, double p, double w) {
  switch (F.kind) {
    case UOT_DIV_KL:
      if (p > 0.0) return F.lam * w * ((r > 0.0 ? r * log(r / p) : 0.0) - r + p);
      return (r > 0.0) ? kInf : 0.0;
    case UOT_DIV_TV:
      return F.lam * w * fabs(r - p);
    case UOT_DIV_EQ:
      return (fabs(r - p) <= 1e-9 * fmax(fabs(p), 1e-300)) ? 0.0 : kInf;
    default: {
      const double lo = exp(F.log_alpha) * p, hi = (F.log_beta == kInf) ? kInf : exp(F.log_beta) * p;
      return (r >= lo * (1.0 - 1e-9) - 1e-300 && r <= hi * (1.0 + 1e-9) + 1e-300) ? 0.0 : kInf;
    }
  }
}

// F*(wv) pointwise term for the pairing sum_i w_i wv_i s_i
__device__ double conj_term(const DivParams& F, double wv, double p, double w) {
  if (p == 0.0) {
    // phi'_inf bound only: KL/EQ: no bound; TV: wv <= lam; RG: beta finite no bound
    if (F.kind == UOT_DIV_TV && wv > F.lam * (1.0 + 1e-12)) return kInf;
    return 0.0;
  }
  switch (F.kind) {
    case UOT_DIV_KL:
      return F.lam * w * p * expm1(wv / F.lam);
    case UOT_DIV_TV:
      if (wv > F.lam * (1.0 + 1e-12)) return kInf;
      return w * p * fmax(wv, -F.lam);
    case UOT_DIV_EQ:
      return w * p * wv;
    default: {
      const double a = exp(F.log_alpha);
      if (F.log_beta == kInf) return (wv > 0.0) ? kInf : w * p * a * wv;
      return w * p * fmax(a * wv, exp(F.log_beta) * wv);
    }
  }
}

// acc[0] += F(r) ; acc[1] += F*(-U) ; acc[2] += sum w U r ; acc[3] += sum w r
// acc[4] += sum w e^{zK} (the sum of K against dx dy) ; acc[5..6] violation
__global__ void k_objective_side(const double* __restrict__ r, const double* __restrict__ U,
                                 const double* __restrict__ logp, const double* __restrict__ logw,
                                 const double* __restrict__ zK, const double* __restrict__ S,
                                 DivParams F, double eps, int64_t n, double* acc) {
  double t[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double w = exp(logw[i]);
    const double p = (logp[i] == -kInf) ? 0.0 : exp(logp[i]);
    const double u = U[i];
    t[0] += div_term(F, r[i], p, w);
    t[1] += conj_term(F, (u == -kInf) ? 0.0 : -u, p, w);
    if (u != -kInf && r[i] > 0.0) t[2] += w * u * r[i];
    t[3] += w * r[i];
    if (zK) t[4] += w * exp(zK[i]);
    if (S) {
      double a, b;
      violation_terms(u, prox_update(F, logp[i], S[i], eps), S[i], logw[i], eps, a, b);
      t[5] += a;
      t[6] += b;
    }
  }
  __shared__ double sm[7][kNT / 32];
  for (int k = 0; k < 7; ++k) {
    double v = t[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sm[k][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    double v = 0.0;
    for (int w = 0; w < kNT / 32; ++w) v += sm[threadIdx.x][w];
    atomicAdd(acc + threadIdx.x, v);
  }
}

// ---------------------------------------------------------------------------
// argument checking and problem description
// ---------------------------------------------------------------------------

bool div_ok(const uot_div* F) {
  if (!F) return false;
  switch (F->kind) {
    case UOT_DIV_EQ:
      return true;
    case UOT_DIV_KL:
    case UOT_DIV_TV:
      return F->lambda > 0.0 && isfinite(F->lambda);
    case UOT_DIV_RG:
      return F->alpha >= 0.0 && isfinite(F->alpha) && F->beta >= F->alpha && !(F->beta != F->beta);
    default:
      return false;
  }
}

DivParams make_div(const uot_div& F) {
  DivParams d;
  d.kind = F.kind;
  d.lam = F.lambda;
  d.log_alpha = (F.kind == UOT_DIV_RG) ? (F.alpha > 0.0 ? log(F.alpha) : -kInf) : 0.0;
  d.log_beta = (F.kind == UOT_DIV_RG) ? (isinf(F.beta) ? kInf : log(F.beta)) : 0.0;
  return d;
}

bool prec_ok(int p) { return p == UOT_F64 || p == UOT_F32 || p == UOT_MIXED; }

// Largest second launch-grid dimension: the most lines one grid pass covers.
constexpr int64_t kMaxGridPassLines = 65535;

uot_status check_geom(const uot_geom* g) {
  if (!g) return UOT_EINVAL;
  if (g->n < 1 || g->m < 1) return UOT_EINVAL;
  switch (g->kind) {
    case UOT_GEOM_DENSE:
      return g->C ? UOT_OK : UOT_EINVAL;
    case UOT_GEOM_POINTS:
      return (g->x && g->y && g->d >= 1 && g->d <= 8) ? UOT_OK : UOT_EINVAL;
    case UOT_GEOM_GRID: {
      if (g->ndim < 1 || g->ndim > UOT_MAX_DIM) return UOT_EINVAL;
      int64_t nx = 1, ny = 1;
      for (int k = 0; k < g->ndim; ++k) {
        if (g->shape_x[k] < 1 || g->shape_y[k] < 1) return UOT_EINVAL;
        if (!g->axes_x[k] || !g->axes_y[k]) return UOT_EINVAL;
        // a staged line must fit in shared memory (4 warps x nin x 16 bytes)
        if (g->shape_x[k] > 3000 || g->shape_y[k] > 3000) {
          g_last_error = "grid axis longer than 3000 points";
          return UOT_EUNSUPPORTED;
        }
        nx *= g->shape_x[k];
        ny *= g->shape_y[k];
      }
      if (nx != g->n || ny != g->m) return UOT_EINVAL;
      // The pass kernels put the line index in the launch grid's second
      // dimension.  Passes run from the last axis to the first; the pass along
      // axis a covers the input side's axes before a and the output side's
      // axes after a (in both directions).
      for (int dir = 0; dir < 2; ++dir) {
        const int* in_shape = dir == 0 ? g->shape_y : g->shape_x;
        const int* out_shape = dir == 0 ? g->shape_x : g->shape_y;
        for (int a = 0; a < g->ndim; ++a) {
          int64_t lines = 1;
          for (int t = 0; t < a; ++t) lines *= in_shape[t];
          for (int t = a + 1; t < g->ndim; ++t) lines *= out_shape[t];
          if (lines > kMaxGridPassLines) {
            g_last_error = "a grid pass would run over more than 65535 lines (product of the other axes)";
            return UOT_EUNSUPPORTED;
          }
        }
      }
      return UOT_OK;
    }
    default:
      return UOT_EINVAL;
  }
}

// Device memory carved out of one stream-ordered allocation, released on
// destruction.  Every buffer is reserved with the same element count that is
// later taken, each rounded to 256 bytes; take() refuses to run past the end.
class Scratch {
 public:
  explicit Scratch(cudaStream_t s) : s_(s) {}
  // Carve from caller-provided device memory of `capacity` bytes instead of
  // allocating (used by the no-allocation entry point).
  Scratch(cudaStream_t s, char* fixed_base, size_t capacity)
      : s_(s), fixed_(fixed_base), capacity_(capacity) {}
  ~Scratch() {
    if (base_ && !fixed_) cudaFreeAsync(base_, s_);
  }
  template <typename T>
  void reserve(size_t count) { need_ += round(count * sizeof(T)); }
  size_t needed() const { return need_; }
  cudaError_t allocate() {
    if (need_ == 0) return cudaSuccess;
    if (fixed_) {
      if (need_ > capacity_) return cudaErrorMemoryAllocation;
      base_ = fixed_;
      return cudaSuccess;
    }
    return cudaMallocAsync((void**)&base_, need_, s_);
  }
  template <typename T>
  T* take(size_t count) {
    const size_t b = round(count * sizeof(T));
    if (!base_ || off_ + b > need_) {
      overflow_ = true;
      return nullptr;
    }
    T* p = (T*)(base_ + off_);
    off_ += b;
    return p;
  }
  // false if any take() did not fit what was reserved (a bug: nothing may be launched)
  bool ok() const { return !overflow_; }

 private:
  static size_t round(size_t b) { return (b + 255) & ~(size_t)255; }
  cudaStream_t s_;
  char* fixed_ = nullptr;
  size_t capacity_ = 0;
  char* base_ = nullptr;
  size_t need_ = 0, off_ = 0;
  bool overflow_ = false;
};

#define UOT_SCRATCH_OK(sc)                                         \
  do {                                                             \
    if (!(sc).ok()) {                                              \
      g_last_error = "internal scratch accounting error";          \
      return UOT_ECUDA;                                            \
    }                                                              \
  } while (0)

struct Gibbs {
  uot_geom g;
  int prec;
  size_t esz;
  const void* CT = nullptr;     // dense: C^T in the precision's type
  float* C32[2] = {nullptr, nullptr};  // dense FP64: FP32 copies of C, C^T (row prefilter)
  double* pass[2] = {nullptr, nullptr};  // grid intermediates
  // FP32 grid passes: result of each (direction, pass) from the previous call,
  // reused as the log-sum-exp shift while eps is unchanged (see k_grid.cu)
  float* zbuf[2][UOT_MAX_DIM] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  double zeps[2] = {-1.0, -1.0};
  bool speculate = false;
  // UOT_MIXED: largest coordinate span of 32 consecutive points per axis (X, Y),
  // and a flag set by the tensor-core kernel if a bounded wait gave up
  double span_x[UOT_MAX_DIM] = {0, 0, 0}, span_y[UOT_MAX_DIM] = {0, 0, 0};
  int* tc_err = nullptr;
  bool spans_known = false;
  // FP32 grids: uniform-axis data of each (direction, axis) pass for the
  // block-stabilised kernel; read from the axes at set-up when host_setup
  BlkAxis blk[2][UOT_MAX_DIM] = {};
  bool host_setup = true;
  // UOT_MIXED: once set, the passes run on the FP32 kernels (end of the BF16 phase)
  bool tc_off = false;
  // FP32 grids and point clouds: once set, the passes form their exponents
  // in float-float (grid_pass_ffp, points_ffp), below the FP32 passes'
  // rounding floor
  bool precise = false;
  void* Lscratch = nullptr;     // rows: shifted input line
  void* part = nullptr;         // FP32 point clouds: per-chunk partial sums
  float* zrow[2] = {nullptr, nullptr};  // FP32 point clouds: previous results per direction
  int64_t inter = 0;            // grid intermediate size (elements)
  int nbatch = 1;

  void plan(Scratch& sc, int batch) {
    nbatch = batch;
    esz = (prec == UOT_F64) ? 8 : 4;
    if (g.kind == UOT_GEOM_DENSE) sc.reserve<char>((size_t)g.n * g.m * esz);
    if (g.kind == UOT_GEOM_DENSE && prec == UOT_F64) {
      for (int k = 0; k < 2; ++k) sc.reserve<float>((size_t)g.n * g.m);
      sc.reserve<int>(1);
    }
    if (g.kind == UOT_GEOM_GRID) {
      inter = 1;
      for (int k = 0; k < g.ndim; ++k) inter *= (g.shape_x[k] > g.shape_y[k] ? g.shape_x[k] : g.shape_y[k]);
      if (g.ndim > 1) {
        sc.reserve<double>((size_t)inter * nbatch);
        sc.reserve<double>((size_t)inter * nbatch);
      }
      if (speculate)
        for (int k = 0; k < 2 * g.ndim; ++k) sc.reserve<float>((size_t)inter * nbatch);
      if (prec == UOT_MIXED || prec == UOT_F32) sc.reserve<int>(1);
    } else {
      const int64_t mx = (g.n > g.m ? g.n : g.m);
      sc.reserve<char>(lscratch_bytes(mx));
      if (points_fast()) {
        sc.reserve<float2>(part_elems());
        if (speculate) {
          sc.reserve<float>((size_t)g.n);
          sc.reserve<float>((size_t)g.m);
        }
      }
    }
  }
  bool points_fast() const {
    return g.kind == UOT_GEOM_POINTS && prec != UOT_F64 && g.d <= 3 && points_chunks_fit(g.n) &&
           points_chunks_fit(g.m);
  }
  // shifted input line (+ Lmax) and, for FP64 dense rows, its FP32 copy
  size_t lscratch_bytes(int64_t mx) const {
    if (g.kind == UOT_GEOM_DENSE && prec == UOT_F64) return std::max((size_t)mx * 8 + 512, rows_pf_scratch_bytes(mx));
    return (size_t)mx * 8 + 512;
  }
  size_t part_elems() const {
    return std::max((size_t)points_nchunks(g.m, g.n) * g.n, (size_t)points_nchunks(g.n, g.m) * g.m);
  }
  cudaError_t take(Scratch& sc, cudaStream_t s) {
    if (g.kind == UOT_GEOM_DENSE) {
      void* ct = sc.take<char>((size_t)g.n * g.m * esz);
      if (!ct) return cudaErrorInvalidValue;
      dim3 grid((g.m + 31) / 32, (g.n + 31) / 32), blk(32, 8);
      count_launches(1);
      if (prec == UOT_F64)
        k_transpose<double><<<grid, blk, 0, s>>>((const double*)g.C, g.n, g.m, (double*)ct);
      else
        k_transpose<float><<<grid, blk, 0, s>>>((const float*)g.C, g.n, g.m, (float*)ct);
      CT = ct;
      if (prec == UOT_F64) {
        const int64_t nm = (int64_t)g.n * g.m;
        C32[0] = sc.take<float>((size_t)nm);
        C32[1] = sc.take<float>((size_t)nm);
        int* dflag = sc.take<int>(1);
        if (!C32[0] || !C32[1] || !dflag) return cudaErrorInvalidValue;
        // a symmetric cost (X = Y, e.g. the WF flows) serves both directions from
        // one copy: half the working set, which then stays in L2
        bool sym = false;
        if (g.n == g.m) {
          cudaError_t e = cudaMemsetAsync(dflag, 0, sizeof(int), s);
          if (e != cudaSuccess) return e;
          count_launches(1);
          k_differs<<<nblocks(nm), kNT, 0, s>>>((const double*)g.C, (const double*)CT, nm, dflag);
          int h = 1;
          if ((e = cudaMemcpyAsync(&h, dflag, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
          if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
          sym = (h == 0);
        }
        count_launches(1);
        k_from_f64<float><<<nblocks(nm), kNT, 0, s>>>((const double*)g.C, nm, C32[0]);
        if (sym) {
          CT = g.C;
          C32[1] = C32[0];
        } else {
          count_launches(1);
          k_from_f64<float><<<nblocks(nm), kNT, 0, s>>>((const double*)CT, nm, C32[1]);
        }
      }
    }
    if (g.kind == UOT_GEOM_GRID) {
      if (g.ndim > 1) {
        pass[0] = sc.take<double>((size_t)inter * nbatch);
        pass[1] = sc.take<double>((size_t)inter * nbatch);
      }
      if (speculate)
        for (int d = 0; d < 2; ++d)
          for (int k = 0; k < g.ndim; ++k) zbuf[d][k] = sc.take<float>((size_t)inter * nbatch);
      if (prec == UOT_MIXED || prec == UOT_F32) {
        tc_err = sc.take<int>(1);
        if (!tc_err) return cudaErrorInvalidValue;
        cudaError_t e = cudaMemsetAsync(tc_err, 0, sizeof(int), s);
        if (e != cudaSuccess) return e;
        // largest coordinate span of the 32-point blocks of every axis
        // (tensor-core passes), and uniform axes (block-stabilised pass):
        // both read the axes on the host once
        const bool want_spans = prec == UOT_MIXED || grid_tc3_wanted();
        if (want_spans || host_setup) {
          std::vector<float> h[2][UOT_MAX_DIM];
          for (int side = 0; side < 2; ++side)
            for (int k = 0; k < g.ndim; ++k) {
              const int len = side == 0 ? g.shape_x[k] : g.shape_y[k];
              h[side][k].resize(len);
              e = cudaMemcpyAsync(h[side][k].data(), side == 0 ? g.axes_x[k] : g.axes_y[k], len * sizeof(float),
                                  cudaMemcpyDeviceToHost, s);
              if (e != cudaSuccess) return e;
            }
          if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
          if (want_spans) {
            for (int side = 0; side < 2; ++side)
              for (int k = 0; k < g.ndim; ++k) {
                const std::vector<float>& v = h[side][k];
                const int len = (int)v.size();
                double span = 0.0;
                for (int i0 = 0; i0 < len; i0 += 32)
                  for (int i = i0; i < std::min(len, i0 + 32); ++i)
                    span = std::max(span, std::fabs((double)v[i] - (double)v[i0]));
                (side == 0 ? span_x : span_y)[k] = span;
              }
            spans_known = true;
          }
          if (host_setup) {
            // axis k of a side is uniform when v[i] = v[0] + i h exactly
            double step[2][UOT_MAX_DIM];
            bool uni[2][UOT_MAX_DIM];
            for (int side = 0; side < 2; ++side)
              for (int k = 0; k < g.ndim; ++k) {
                const std::vector<float>& v = h[side][k];
                uni[side][k] = v.size() >= 2;
                step[side][k] = uni[side][k] ? (double)v[1] - (double)v[0] : 0.0;
                for (size_t i = 0; i < v.size() && uni[side][k]; ++i)
                  uni[side][k] = (double)v[i] == (double)v[0] + (double)i * step[side][k];
                uni[side][k] = uni[side][k] && step[side][k] > 0.0 &&
                               (double)(float)step[side][k] == step[side][k];
              }
            for (int dir = 0; dir < 2; ++dir)
              for (int k = 0; k < g.ndim; ++k) {
                const int in = dir == 0 ? 1 : 0, out = 1 - in;
                const double d0 = (double)h[out][k][0] - (double)h[in][k][0];
                BlkAxis& b = blk[dir][k];
                b.ok = uni[in][k] && uni[out][k] && step[in][k] == step[out][k] && (double)(float)d0 == d0;
                b.h = (float)step[in][k];
                b.d0 = (float)d0;
              }
          }
        }
      }
    } else {
      const int64_t mx = (g.n > g.m ? g.n : g.m);
      Lscratch = sc.take<char>(lscratch_bytes(mx));
      if (!Lscratch) return cudaErrorInvalidValue;
      if (g.kind == UOT_GEOM_DENSE && prec == UOT_F64) {
        // the prefilter's block counter (first bytes of the scratch)
        cudaError_t e0 = cudaMemsetAsync(Lscratch, 0, 256, s);
        if (e0 != cudaSuccess) return e0;
      }
      if (points_fast()) {
        part = sc.take<float2>(part_elems());
        if (speculate) {
          zrow[0] = sc.take<float>((size_t)g.n);
          zrow[1] = sc.take<float>((size_t)g.m);
        }
      }
    }
    return cudaGetLastError();
  }

  // dir 0: W on the Y side (size m) -> result on the X side (size n); dir 1: reverse.
  // The tensor-core pass needs the local kernel exp(-(delta - eta)^2/eps) of
  // two 32-point blocks to stay far above the FP32 underflow threshold
  // (2^-100 in log2 units) and the staged lines to fit in shared memory.
  bool tc_ok(int dir, int ax, double eps, int nin) const {
    const double so = (dir == 0 ? span_x : span_y)[ax], si = (dir == 0 ? span_y : span_x)[ax];
    const double reach = (double)kLog2e / eps * (so + si) * (so + si);
    return reach <= 100.0 && grid_pass_tc_smem(nin) <= 200 * 1024;
  }
  // The three-part tensor-core pass keeps its smallest operand parts normal
  // while k (span_out + span_in)^2 <= 90 (log2 units) and takes nin <= 256.
  int tc3_ok(int dir, int ax, double eps, int nin) const {
    if (!spans_known || prec != UOT_F32) return 0;
    const double so = (dir == 0 ? span_x : span_y)[ax], si = (dir == 0 ? span_y : span_x)[ax];
    const double reach = (double)kLog2e / eps * (so + si) * (so + si);
    return (reach <= 90.0 && nin <= grid_pass_tc3_max_nin()) ? 1 : 0;
  }

  // zero_acc: two doubles cleared before the result is produced (violation
  // accumulators of a checked iteration), inside the first kernel when possible.
  cudaError_t apply(int dir, const double* W, const double* logw, double eps, const Epilogue& epi,
                    cudaStream_t s, double* zero_acc = nullptr) {
    if (g.kind == UOT_GEOM_GRID) {
      const int use_prev = (zbuf[dir][0] != nullptr && zeps[dir] == eps) ? 1 : 0;
      const int d = g.ndim;
      const int* in_shape = dir == 0 ? g.shape_y : g.shape_x;
      const int* out_shape = dir == 0 ? g.shape_x : g.shape_y;
      const void* const* in_axes = dir == 0 ? g.axes_y : g.axes_x;
      const void* const* out_axes = dir == 0 ? g.axes_x : g.axes_y;
      const double* cur = W;
      int cur_is_pot = 1;
      for (int k = 0; k < d; ++k) {
        const int ax = d - 1 - k;
        // two short FP32 passes in a row: one fused launch per plane
        const bool f32 = prec == UOT_F32 || (prec == UOT_MIXED && tc_off);
        if (f32 && k + 1 < d && !precise && !precise_forced() &&
            grid_plane_ok(in_shape[ax], out_shape[ax], in_shape[ax - 1], out_shape[ax - 1])) {
          int64_t Pc = 1, S = 1;
          for (int t = 0; t < ax - 1; ++t) Pc *= in_shape[t];
          for (int t = ax + 1; t < d; ++t) S *= out_shape[t];
          const int64_t nlines2 = Pc * out_shape[ax] * S;
          Epilogue e = epi;
          if (k + 1 < d - 1) {
            memset(&e, 0, sizeof(e));
            e.mode = EPI_RAW;
            e.eps = eps;
            e.out = pass[(k + 1) & 1];
            e.bstride = nlines2 * out_shape[ax - 1];
          }
          double* za = nullptr;
          if (k == 0 && zero_acc) {
            if (k + 1 < d - 1) {
              za = zero_acc;  // cleared by the fused launch, accumulated by the last pass
            } else {
              cudaError_t e0 = cudaMemsetAsync(zero_acc, 0, 16 * (size_t)nbatch, s);
              if (e0 != cudaSuccess) return e0;
            }
          }
          cudaError_t err = launch_grid_pass_plane(
              cur, logw, cur_is_pot, Pc * S, (int)S, in_shape[ax], in_axes[ax], out_shape[ax], out_axes[ax],
              zbuf[dir][k], in_shape[ax - 1], in_axes[ax - 1], out_shape[ax - 1], out_axes[ax - 1], zbuf[dir][k + 1],
              eps, nbatch, use_prev, za, e, s);
          if (err != cudaSuccess) return err;
          cur = pass[(k + 1) & 1];
          cur_is_pot = 0;
          ++k;
          continue;
        }
        int64_t nlines = 1;
        for (int t = 0; t < ax; ++t) nlines *= in_shape[t];
        for (int t = ax + 1; t < d; ++t) nlines *= out_shape[t];
        Epilogue e = epi;
        if (k < d - 1) {
          memset(&e, 0, sizeof(e));
          e.mode = EPI_RAW;
          e.eps = eps;
          e.out = pass[k & 1];
          e.bstride = nlines * out_shape[ax];
        }
        double* za = nullptr;
        if (k == 0 && zero_acc) {
          // cleared inside the first pass only when that pass is not also the
          // last one (whose blocks accumulate into it): 2-D and 3-D grids
          if (prec != UOT_F64 && d > 1) {
            za = zero_acc;
          } else {
            cudaError_t e0 = cudaMemsetAsync(zero_acc, 0, 16 * (size_t)nbatch, s);
            if (e0 != cudaSuccess) return e0;
          }
        }
        cudaError_t err;
        if (prec == UOT_MIXED && !tc_off && tc_ok(dir, ax, eps, in_shape[ax])) {
          err = launch_grid_pass_tc(cur, logw, cur_is_pot, (int)nlines, in_shape[ax], in_axes[ax],
                                    out_shape[ax], out_axes[ax], eps, nbatch, e, s, tc_err, za);
        } else {
          err = launch_grid_pass(prec == UOT_F64 ? UOT_F64 : UOT_F32, cur, logw, cur_is_pot,
                                 (int)nlines, in_shape[ax], in_axes[ax], out_shape[ax],
                                 out_axes[ax], eps, nbatch, e, s, zbuf[dir][k], use_prev, za,
                                 tc3_ok(dir, ax, eps, in_shape[ax]), tc_err, &blk[dir][ax], precise ? 1 : 0);
        }
        if (err != cudaSuccess) return err;
        cur = pass[k & 1];
        cur_is_pot = 0;
      }
      if (zbuf[dir][0]) zeps[dir] = eps;
      return cudaSuccess;
    }
    if (zero_acc) {
      cudaError_t e0 = cudaMemsetAsync(zero_acc, 0, 16 * (size_t)nbatch, s);
      if (e0 != cudaSuccess) return e0;
    }
    RowsGeom rg;
    rg.kind = g.kind;
    rg.d = g.d;
    rg.C = (dir == 0) ? g.C : CT;
    rg.C32 = C32[dir];
    rg.x = (dir == 0) ? g.x : g.y;
    rg.y = (dir == 0) ? g.y : g.x;
    const int nrows = (dir == 0) ? g.n : g.m;
    const int nin = (dir == 0) ? g.m : g.n;
    for (int b = 0; b < nbatch; ++b) {
      Epilogue e = epi;
      // batches for rows geometries are run one by one
      if (b > 0) {
        if (e.pot) e.pot += b * e.bstride;
        if (e.out) e.out += b * e.bstride;
        if (e.logp) e.logp += b * e.bstride_p;
        if (e.pot_shift) e.pot_shift += b * e.bstride;
        if (e.err) e.err += 2 * b;
      }
      const int use_prev = (nbatch == 1 && zrow[dir] != nullptr && zeps[dir] == eps) ? 1 : 0;
      cudaError_t err = launch_rows(prec == UOT_F64 ? UOT_F64 : UOT_F32, rg, nrows, nin,
                                    W + (int64_t)b * nin, logw, eps, Lscratch, e, s,
                                    nbatch == 1 ? zrow[dir] : nullptr, use_prev, part, precise ? 1 : 0);
      if (err != cudaSuccess) return err;
    }
    if (zrow[dir] && nbatch == 1) zeps[dir] = eps;
    return cudaSuccess;
  }
};

// A block of launches captured once as a CUDA graph and replayed.  Capture
// runs on a private stream (the caller's may be the legacy default stream,
// which cannot be captured); every replay runs on the caller's stream.  The
// launch counter counts each replayed kernel, not the capture.
struct BlockGraph {
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;
  template <class F>
  cudaError_t capture(F&& body) {
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    const long long before = g_launches.load();
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t eb = body(cs);
      const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
      e = (eb != cudaSuccess) ? eb : ee;
    }
    kernels = g_launches.load() - before;
    g_launches.fetch_sub(kernels);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) exec = nullptr;
    return e;
  }
  cudaError_t launch(cudaStream_t s) {
    count_launches((int)kernels);
    return cudaGraphLaunch(exec, s);
  }
  // forget the captured block (its launches changed); the next use recaptures
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    kernels = 0;
  }
  ~BlockGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

// Per-point state conversions: FP64 path -> double slots; FP32 path ->
// float-float pairs in the same 8-byte slots.
cudaError_t to_log(int prec, const void* src, int64_t n, double* dst, cudaStream_t s) {
  count_launches(1);
  if (prec == UOT_F64)
    k_to_log<double><<<nblocks(n), kNT, 0, s>>>((const double*)src, n, dst);
  else
    k_to_log_ff<<<nblocks(n), kNT, 0, s>>>((const float*)src, n, reinterpret_cast<float2*>(dst));
  return cudaGetLastError();
}
cudaError_t to_f64(int prec, const void* src, int64_t n, double* dst, cudaStream_t s) {
  if (prec == UOT_F64)
    return cudaMemcpyAsync(dst, src, n * 8, cudaMemcpyDeviceToDevice, s);
  count_launches(1);
  k_to_ff<<<nblocks(n), kNT, 0, s>>>((const float*)src, n, reinterpret_cast<float2*>(dst));
  return cudaGetLastError();
}
cudaError_t from_f64(int prec, const double* src, int64_t n, void* dst, cudaStream_t s) {
  if (prec == UOT_F64)
    return cudaMemcpyAsync(dst, src, n * 8, cudaMemcpyDeviceToDevice, s);
  count_launches(1);
  k_from_ff<<<nblocks(n), kNT, 0, s>>>(reinterpret_cast<const float2*>(src), n, (float*)dst);
  return cudaGetLastError();
}

DivFF make_div_ff(const DivParams& F, double eps) {
  DivFF d;
  d.kind = F.kind;
  d.zf = ff2(ff_make(F.lam / (F.lam + eps)));
  d.lam = ff2(ff_make(F.lam));
  d.elog_a = (F.log_alpha == -kInf) ? make_float2(-INFINITY, 0.0f) : ff2(ff_make(eps * F.log_alpha));
  d.elog_b = (F.log_beta == kInf) ? make_float2(INFINITY, 0.0f) : ff2(ff_make(eps * F.log_beta));
  return d;
}

void set_eps(Epilogue& e, double eps) {
  e.eps = eps;
  e.eps_ff = ff2(ff_make(eps));
  e.inv_eps_ff = ff2(ff_make(1.0 / eps));
}

Epilogue prox_epilogue(const DivParams& F, const double* logp, double* pot, const double* logw,
                       double* err, double eps) {
  Epilogue e;
  memset(&e, 0, sizeof(e));
  e.mode = EPI_PROX;
  set_eps(e, eps);
  e.Fff = make_div_ff(F, eps);
  e.F = F;
  e.logp = logp;
  e.pot = pot;
  e.logw = logw;
  e.err = err;
  return e;
}

struct Stage {
  double eps;
  int iters;
};

std::vector<Stage> eps_schedule(const uot_opts& o) {
  std::vector<Stage> st;
  if (o.eps_start > o.eps && o.eps_stages > 0 && o.iters_per_stage > 0) {
    const double rho = pow(o.eps_start / o.eps, 1.0 / o.eps_stages);
    for (int s = 0; s < o.eps_stages; ++s) st.push_back({o.eps_start / pow(rho, s), o.iters_per_stage});
  }
  return st;
}

uot_result empty_result() {
  uot_result r;
  memset(&r, 0, sizeof(r));
  r.marg_err_fp32 = NAN;
  return r;
}

// only uot_solve and uot_solve_many honour out_f64 and verify; uot_solve_batch
// also honours translate and out_f64 (allow_batch)
uot_status check_opts(const uot_opts* o, bool solve_outputs = false, bool allow_batch = false) {
  if (!o || !prec_ok(o->precision)) return UOT_EINVAL;
  if ((o->out_f64 != 0 && o->out_f64 != 1) || (o->verify != 0 && o->verify != 1)) return UOT_EINVAL;
  if (o->translate != 0 && o->translate != 1) return UOT_EINVAL;
  if (!solve_outputs && o->verify) return UOT_EUNSUPPORTED;
  if (!solve_outputs && !allow_batch && (o->out_f64 || o->translate)) return UOT_EUNSUPPORTED;
  if (!(o->eps > 0.0) || !isfinite(o->eps)) return UOT_EINVAL;
  if (o->max_iter < 0 || o->check_every < 0 || !(o->tol >= 0.0)) return UOT_EINVAL;
  if (o->eps_stages < 0 || o->iters_per_stage < 0) return UOT_EINVAL;
  if (o->eps_start > o->eps && !isfinite(o->eps_start)) return UOT_EINVAL;
  return UOT_OK;
}

// ---------------------------------------------------------------------------
// FP64 confirmation of an FP32-path stop (uot_opts.verify), and the FP64
// iterations that finish a solve once the FP32 check has reached its rounding
// floor.  FP64 copies of the geometry and of the state, an FP64 Gibbs
// operator on them; the violation is the stopping criterion of uot_solve
// evaluated in FP64, i.e. the oracle's definition.
// ---------------------------------------------------------------------------
__global__ void k_ff_to_f64(const float2* __restrict__ src, int64_t n, double* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = src[i];
    dst[i] = (v.x == -INFINITY) ? -kInf : (double)v.x + (double)v.y;
  }
}

struct Check64 {
  Scratch sc;
  Gibbs G;
  int batch = 1;
  int64_t n = 0, m = 0;
  double *logp = nullptr, *logq = nullptr, *logdx = nullptr, *logdy = nullptr;
  double *U = nullptr, *V = nullptr, *Ubak = nullptr, *acc = nullptr;
  std::vector<double> acc_h;
  bool ready = false;
  explicit Check64(cudaStream_t s) : sc(s) {}

  // p, q, dx, dy, and the geometry's arrays, are the caller's FP32 inputs.
  cudaError_t setup(const uot_geom& g, int batch_, const void* p, const void* dx, const void* q,
                    const void* dy, cudaStream_t s) {
    batch = batch_;
    n = g.n;
    m = g.m;
    G.g = g;
    G.prec = UOT_F64;
    G.speculate = false;
    // FP64 copies of the geometry
    int64_t glen[2 * UOT_MAX_DIM + 1] = {0};
    int ng = 0;
    if (g.kind == UOT_GEOM_GRID) {
      for (int k = 0; k < g.ndim; ++k) glen[ng++] = g.shape_x[k];
      for (int k = 0; k < g.ndim; ++k) glen[ng++] = g.shape_y[k];
    } else if (g.kind == UOT_GEOM_POINTS) {
      glen[ng++] = (int64_t)g.n * g.d;
      glen[ng++] = (int64_t)g.m * g.d;
    } else {
      glen[ng++] = (int64_t)g.n * g.m;
    }
    for (int k = 0; k < ng; ++k) sc.reserve<double>(glen[k]);
    G.plan(sc, batch);
    sc.reserve<double>(n * batch);  // logp
    sc.reserve<double>(m * batch);  // logq
    sc.reserve<double>(n);          // logdx
    sc.reserve<double>(m);          // logdy
    sc.reserve<double>(n * batch);  // U
    sc.reserve<double>(m * batch);  // V
    sc.reserve<double>(n * batch);  // U before the last a-update
    sc.reserve<double>(2 * (size_t)batch);
    cudaError_t e = sc.allocate();
    if (e != cudaSuccess) return e;
    const void* src[2 * UOT_MAX_DIM + 1];
    ng = 0;
    if (g.kind == UOT_GEOM_GRID) {
      for (int k = 0; k < g.ndim; ++k) src[ng++] = g.axes_x[k];
      for (int k = 0; k < g.ndim; ++k) src[ng++] = g.axes_y[k];
    } else if (g.kind == UOT_GEOM_POINTS) {
      src[ng++] = g.x;
      src[ng++] = g.y;
    } else {
      src[ng++] = g.C;
    }
    for (int k = 0; k < ng; ++k) {
      double* dst = sc.take<double>(glen[k]);
      if (!dst) return cudaErrorInvalidValue;
      count_launches(1);
      k_to_f64<float><<<nblocks(glen[k]), kNT, 0, s>>>((const float*)src[k], glen[k], dst);
      if (g.kind == UOT_GEOM_GRID) {
        if (k < g.ndim) G.g.axes_x[k] = dst;
        else G.g.axes_y[k - g.ndim] = dst;
      } else if (g.kind == UOT_GEOM_POINTS) {
        if (k == 0) G.g.x = dst;
        else G.g.y = dst;
      } else {
        G.g.C = dst;
      }
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = G.take(sc, s)) != cudaSuccess) return e;
    logp = sc.take<double>(n * batch);
    logq = sc.take<double>(m * batch);
    logdx = sc.take<double>(n);
    logdy = sc.take<double>(m);
    U = sc.take<double>(n * batch);
    V = sc.take<double>(m * batch);
    Ubak = sc.take<double>(n * batch);
    acc = sc.take<double>(2 * (size_t)batch);
    if (!sc.ok()) return cudaErrorInvalidValue;
    const void* in[4] = {p, q, dx, dy};
    double* out[4] = {logp, logq, logdx, logdy};
    const int64_t len[4] = {n * batch, m * batch, n, m};
    for (int k = 0; k < 4; ++k) {
      count_launches(1);
      k_to_log<float><<<nblocks(len[k]), kNT, 0, s>>>((const float*)in[k], len[k], out[k]);
    }
    acc_h.assign(2 * (size_t)batch, 0.0);
    ready = true;
    return cudaGetLastError();
  }
  // the FP32 path's float-float state -> FP64
  cudaError_t load_state(const double* Uff, const double* Vff, cudaStream_t s) {
    if (!ready) return cudaErrorInvalidValue;  // setup() first
    count_launches(2);
    k_ff_to_f64<<<nblocks(n * batch), kNT, 0, s>>>(reinterpret_cast<const float2*>(Uff), n * batch, U);
    k_ff_to_f64<<<nblocks(m * batch), kNT, 0, s>>>(reinterpret_cast<const float2*>(Vff), m * batch, V);
    return cudaGetLastError();
  }
  // One FP64 iteration of the log-domain scaling; with `check` the violation
  // of the state it starts from is accumulated (read it with read_err).
  cudaError_t iterate(const DivParams& D1, const DivParams& D2, double eps, bool check, bool v_update,
                      cudaStream_t s) {
    if (!ready) return cudaErrorInvalidValue;  // setup() first
    Epilogue e1 = prox_epilogue(D1, logp, U, logdx, check ? acc : nullptr, eps);
    e1.bstride = e1.bstride_p = n;
    cudaError_t e = G.apply(0, V, logdy, eps, e1, s, check ? acc : nullptr);
    if (e != cudaSuccess || !v_update) return e;
    Epilogue e2 = prox_epilogue(D2, logq, V, logdy, nullptr, eps);
    e2.bstride = e2.bstride_p = m;
    return G.apply(1, U, logdx, eps, e2, s);
  }
  // U <-> its copy taken before an a-update
  cudaError_t save_U(cudaStream_t s) {
    if (!ready) return cudaErrorInvalidValue;
    return cudaMemcpyAsync(Ubak, U, 8 * (size_t)(n * batch), cudaMemcpyDeviceToDevice, s);
  }
  cudaError_t restore_U(cudaStream_t s) {
    if (!ready) return cudaErrorInvalidValue;
    return cudaMemcpyAsync(U, Ubak, 8 * (size_t)(n * batch), cudaMemcpyDeviceToDevice, s);
  }
  // the b-update alone (second half of an iteration)
  cudaError_t b_update(const DivParams& D2, double eps, cudaStream_t s) {
    if (!ready) return cudaErrorInvalidValue;
    Epilogue e2 = prox_epilogue(D2, logq, V, logdy, nullptr, eps);
    e2.bstride = e2.bstride_p = m;
    return G.apply(1, U, logdx, eps, e2, s);
  }
  cudaError_t read_err(double& out, cudaStream_t s) {
    if (!ready) return cudaErrorInvalidValue;  // setup() first
    cudaError_t e = cudaMemcpyAsync(acc_h.data(), acc, 16 * (size_t)batch, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    out = 0.0;
    for (int b = 0; b < batch; ++b) {
      const double v = (acc_h[2 * b + 1] > 0.0) ? acc_h[2 * b] / acc_h[2 * b + 1] : 0.0;
      out = (v > out || v != v) ? v : out;
    }
    return cudaSuccess;
  }
};

}  // namespace
}  // namespace uot

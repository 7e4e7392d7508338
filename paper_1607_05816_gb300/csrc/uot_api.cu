// C-ABI entry points and host orchestration of the scaling iterations.
//
// The host side validates arguments, converts the caller's arrays to the
// internal FP64 per-point state (log densities, log reference weights,
// potentials), and enqueues the iteration on the caller's stream:
//
//   iteration (eq. S, Sec. 3.3, log form of Sec. 4.3):
//     U <- prox_F1(eps log K(e^{V/eps} . dy))     (Gibbs operator + fused Table 1 row)
//     V <- prox_F2(eps log K^T(e^{U/eps} . dx))
//
// eps-scaling (Sec. 4.4) runs `eps_stages` stages of `iters_per_stage`
// iterations at eps_start / rho^s before iterating at eps; potentials carry
// over between stages (they are the absorbed duals of Algorithm 2).
//
// Every kernel on the path is this library's own; no CPU fallback exists.
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

namespace uot {
namespace {

thread_local std::string g_last_error;

std::atomic<long long> g_launches{0};

// Optional CUDA-event timing of the Gibbs operator kernels: when enabled, an
// event pair brackets each launch on the launching stream.
struct Prof {
  std::mutex mu;
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> marks[PROF_NFAM];
  cudaEvent_t pending[PROF_NFAM] = {};
} g_prof;

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

uot_status fail_cuda(cudaError_t e, const char* what = nullptr, int line = 0) {
  g_last_error = cudaGetErrorString(e);
  if (what) g_last_error += std::string(" [") + what + " @uot_api.cu:" + std::to_string(line) + "]";
  return (e == cudaErrorMemoryAllocation) ? UOT_ENOMEM : UOT_ECUDA;
}

#define UOT_CK(expr)                                                \
  do {                                                              \
    cudaError_t e_ = (expr);                                        \
    if (e_ != cudaSuccess) return fail_cuda(e_, #expr, __LINE__);   \
  } while (0)

// Errors raised by other code sharing this CUDA runtime (non-sticky ones) must
// not be attributed to this call: clear them on entry.
inline void clear_stale_error() { (void)cudaGetLastError(); }

// ---------------------------------------------------------------------------
// pointwise kernels
// ---------------------------------------------------------------------------

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
        if (g->shape_x[k] > 3000 || g->shape_y[k] > 3000) return UOT_EUNSUPPORTED;
        nx *= g->shape_x[k];
        ny *= g->shape_y[k];
      }
      return (nx == g->n && ny == g->m) ? UOT_OK : UOT_EINVAL;
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
      if (speculate && (prec == UOT_F32 || prec == UOT_MIXED))
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
  bool points_fast() const { return g.kind == UOT_GEOM_POINTS && prec != UOT_F64 && g.d <= 3; }
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
      if (speculate && (prec == UOT_F32 || prec == UOT_MIXED))
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
          if (prec != UOT_F64) {
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
                                 tc3_ok(dir, ax, eps, in_shape[ax]), tc_err, &blk[dir][ax]);
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
                                    nbatch == 1 ? zrow[dir] : nullptr, use_prev, part);
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

// only uot_solve and uot_solve_many honour out_f64 and verify; translate also uot_solve_batch
uot_status check_opts(const uot_opts* o, bool solve_outputs = false, bool allow_translate = false) {
  if (!o || !prec_ok(o->precision)) return UOT_EINVAL;
  if ((o->out_f64 != 0 && o->out_f64 != 1) || (o->verify != 0 && o->verify != 1)) return UOT_EINVAL;
  if (o->translate != 0 && o->translate != 1) return UOT_EINVAL;
  if (!solve_outputs && (o->out_f64 || o->verify)) return UOT_EUNSUPPORTED;
  if (!solve_outputs && !allow_translate && o->translate) return UOT_EUNSUPPORTED;
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

// ---------------------------------------------------------------------------
// solve
// ---------------------------------------------------------------------------

// `batch` independent problems sharing the geometry, eps and penalties: p, U
// are [batch][n], q, V are [batch][m]; dx, dy are shared.  The iteration stops
// when every problem's violation is <= tol (the reported error is the largest).
uot_status solve_impl(const uot_geom* g, int batch, const void* p, const void* dx, const void* q,
                      const void* dy, const uot_div* F1, const uot_div* F2, const uot_opts* o,
                      void* Uout, void* Vout, uot_result* res, cudaStream_t s) {
  uot_status st = check_geom(g);
  if (st != UOT_OK) return st;
  if ((st = check_opts(o, true)) != UOT_OK) return st;
  if (batch < 1 || !p || !dx || !q || !dy || !Uout || !Vout || !div_ok(F1) || !div_ok(F2))
    return UOT_EINVAL;
  if (o->plain_scaling && (g->kind != UOT_GEOM_DENSE || o->precision != UOT_F64 || batch != 1))
    return UOT_EUNSUPPORTED;
  if (g->kind == UOT_GEOM_GRID && batch > 65535) return UOT_EUNSUPPORTED;
  const bool translate = o->translate != 0;
  if (translate && (F1->kind != UOT_DIV_KL || F2->kind != UOT_DIV_KL || o->plain_scaling || batch > 65535))
    return UOT_EUNSUPPORTED;
  const int prec = o->precision;
  const int64_t n = g->n, m = g->m;
  const int64_t bn = n * batch, bm = m * batch;
  const DivParams D1 = make_div(*F1), D2 = make_div(*F2);

  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  UOT_CK(cudaEventCreate(&ev0));
  UOT_CK(cudaEventCreate(&ev1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } evg{ev0, ev1};
  UOT_CK(cudaEventRecord(ev0, s));

  Scratch sc(s);
  Gibbs G;
  G.g = *g;
  G.prec = prec;
  G.speculate = true;
  G.plan(sc, batch);
  sc.reserve<double>(bn);  // logp
  sc.reserve<double>(n);   // logdx
  sc.reserve<double>(bn);  // U
  sc.reserve<double>(bm);  // logq
  sc.reserve<double>(m);   // logdy
  sc.reserve<double>(bm);  // V
  sc.reserve<double>(2 * (size_t)batch + 4);  // err accumulators + flag
  if (translate) sc.reserve<double2>(kl_translate_part_count(n, m, batch));
  // one persistent cooperative launch for FP32 grid problems
  const std::vector<Stage> stages_p = eps_schedule(*o);
  const int nst = (int)stages_p.size();
  const bool verify = o->verify && prec != UOT_F64 && o->tol > 0.0 && !o->plain_scaling;
  const bool persist = o->launch_mode == 1 && prec == UOT_F32 && g->kind == UOT_GEOM_GRID &&
                       batch == 1 && !o->plain_scaling && !verify && !translate;
  // two kernels per iteration, each fusing two passes on one line (2-D FP32 grids)
  const bool fused2d = o->launch_mode == 3 && prec == UOT_F32 && g->kind == UOT_GEOM_GRID && g->ndim == 2 &&
                       batch == 1 && !o->plain_scaling && !verify && !translate &&
                       grid_fused2_smem(std::max(g->shape_y[0], g->shape_x[1]), std::max(g->shape_x[0], g->shape_y[1])) <=
                           160 * 1024;
  if (persist) {
    sc.reserve<float2>(nst + 1);   // eps
    sc.reserve<float2>(nst + 1);   // 1/eps
    sc.reserve<float>(nst + 1);    // log2(e)/eps
    sc.reserve<DivFF>(2 * (nst + 1));
    sc.reserve<unsigned>(2);       // barrier
    sc.reserve<int>(4);            // status
    sc.reserve<double>(1);         // last violation
  }
  if (o->plain_scaling) {
    sc.reserve<double>((size_t)n * m);  // K
    sc.reserve<double>((size_t)n * m);  // K^T
    for (int k = 0; k < 3; ++k) sc.reserve<double>(n);  // a, p, dx
    for (int k = 0; k < 3; ++k) sc.reserve<double>(m);  // b, q, dy
    sc.reserve<double>(4);                               // cluster solve's result
  }
  UOT_CK(sc.allocate());
  UOT_CK(G.take(sc, s));
  double* logp = sc.take<double>(bn);
  double* logdx = sc.take<double>(n);
  double* U = sc.take<double>(bn);
  double* logq = sc.take<double>(bm);
  double* logdy = sc.take<double>(m);
  double* V = sc.take<double>(bm);
  double* acc = sc.take<double>(2 * (size_t)batch + 4);
  int* flag = (int*)(acc + 2 * (size_t)batch);
  double2* trpart = translate ? sc.take<double2>(kl_translate_part_count(n, m, batch)) : nullptr;
  std::vector<double> acc_h(2 * (size_t)batch);
  UOT_SCRATCH_OK(sc);
  UOT_CK(to_log(prec, p, bn, logp, s));
  UOT_CK(to_log(prec, dx, n, logdx, s));
  UOT_CK(to_log(prec, q, bm, logq, s));
  UOT_CK(to_log(prec, dy, m, logdy, s));
  if (o->U0) {
    UOT_CK(to_f64(prec, o->U0, bn, U, s));
  } else {
    count_launches(1);
    k_fill<<<nblocks(bn), kNT, 0, s>>>(U, bn, 0.0);
  }
  if (o->V0) {
    UOT_CK(to_f64(prec, o->V0, bm, V, s));
  } else {
    count_launches(1);
    k_fill<<<nblocks(bm), kNT, 0, s>>>(V, bm, 0.0);
  }
  UOT_CK(cudaGetLastError());
  if (o->U0 || o->V0) {
    // a NaN or +inf start would spread through the log-sum-exps (all -inf, an empty plan)
    UOT_CK(cudaMemsetAsync(flag, 0, 4, s));
    count_launches(2);
    k_bad_start<<<nblocks(bn), kNT, 0, s>>>(U, bn, prec != UOT_F64, flag);
    k_bad_start<<<nblocks(bm), kNT, 0, s>>>(V, bm, prec != UOT_F64, flag);
    int hbad = 0;
    UOT_CK(cudaMemcpyAsync(&hbad, flag, 4, cudaMemcpyDeviceToHost, s));
    UOT_CK(cudaStreamSynchronize(s));
    if (hbad) {
      g_last_error = "uot_solve: the warm start U0/V0 holds NaN or +inf";
      return UOT_EINVAL;
    }
  }

  const std::vector<Stage> stages = eps_schedule(*o);
  const int check_every = o->check_every > 0 ? o->check_every : 1;
  int it = 0, total = 0;
  double err = INFINITY;
  bool converged = false;
  // opts.verify: FP64 confirmation of the stop, then FP64 iterations past the FP32 floor
  Check64 c64(s);
  double err32 = NAN, err64 = NAN, tol_int = o->tol;
  int nverify = 0, npolish = 0;
  bool polish = false, polished = false;
  // FP32 progress: first check at the final eps, best value so far (1% steps)
  double first_err = NAN, best_err = INFINITY;
  int first_it = 0, best_it = 0;
  // UOT_MIXED: the BF16 (tensor-core) phase, until the violation reaches mixed_switch
  bool mixed_phase = prec == UOT_MIXED && g->kind == UOT_GEOM_GRID && o->tol > 0.0;
  const double mixed_switch = o->mixed_switch > 0.0 ? o->mixed_switch : 1e-3;
  int mixed_iters = 0;
  bool mixed_handover = false;  // set by decide(): the graph block must be recaptured

  auto read_err = [&](double& out) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(acc_h.data(), acc, 16 * (size_t)batch, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    out = 0.0;
    for (int b = 0; b < batch; ++b) {
      const double v = (acc_h[2 * b + 1] > 0.0) ? acc_h[2 * b] / acc_h[2 * b + 1] : 0.0;
      out = (v > out || v != v) ? v : out;
    }
    return cudaSuccess;
  };
  if (persist) {
    std::vector<float2> heps(nst + 1), hieps(nst + 1);
    std::vector<float> hk2(nst + 1);
    std::vector<DivFF> hF(2 * (nst + 1));
    for (int sidx = 0; sidx <= nst; ++sidx) {
      const double e = (sidx < nst) ? stages_p[sidx].eps : o->eps;
      heps[sidx] = ff2(ff_make(e));
      hieps[sidx] = ff2(ff_make(1.0 / e));
      hk2[sidx] = (float)((double)kLog2e / e);
      hF[2 * sidx] = make_div_ff(D1, e);
      hF[2 * sidx + 1] = make_div_ff(D2, e);
    }
    float2* d_eps = sc.take<float2>(nst + 1);
    float2* d_ieps = sc.take<float2>(nst + 1);
    float* d_k2 = sc.take<float>(nst + 1);
    DivFF* d_F = sc.take<DivFF>(2 * (nst + 1));
    unsigned* d_bar = sc.take<unsigned>(2);
    int* d_status = sc.take<int>(4);
    double* d_err = sc.take<double>(1);
    UOT_SCRATCH_OK(sc);
    UOT_CK(cudaMemcpyAsync(d_eps, heps.data(), heps.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
    UOT_CK(cudaMemcpyAsync(d_ieps, hieps.data(), hieps.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
    UOT_CK(cudaMemcpyAsync(d_k2, hk2.data(), hk2.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    UOT_CK(cudaMemcpyAsync(d_F, hF.data(), hF.size() * sizeof(DivFF), cudaMemcpyHostToDevice, s));
    UOT_CK(cudaMemsetAsync(d_bar, 0, 2 * sizeof(unsigned), s));
    UOT_CK(cudaMemsetAsync(d_status, 0, 4 * sizeof(int), s));
    UOT_CK(cudaMemsetAsync(d_err, 0, sizeof(double), s));
    PersistLaunch L;
    memset(&L, 0, sizeof(L));
    L.ndim = g->ndim;
    int nin_max = 1;
    int64_t max_items = 1;
    for (int k = 0; k < g->ndim; ++k) {
      L.shape_x[k] = g->shape_x[k];
      L.shape_y[k] = g->shape_y[k];
      L.axes_x[k] = g->axes_x[k];
      L.axes_y[k] = g->axes_y[k];
      L.zbuf[0][k] = G.zbuf[0][k];
      L.zbuf[1][k] = G.zbuf[1][k];
      nin_max = std::max(nin_max, std::max(g->shape_x[k], g->shape_y[k]));
    }
    for (int dir = 0; dir < 2; ++dir) {
      const int* in_shape = dir == 0 ? g->shape_y : g->shape_x;
      const int* out_shape = dir == 0 ? g->shape_x : g->shape_y;
      for (int ax = 0; ax < g->ndim; ++ax) {
        int64_t nl = 1;
        for (int t = 0; t < ax; ++t) nl *= in_shape[t];
        for (int t = ax + 1; t < g->ndim; ++t) nl *= out_shape[t];
        max_items = std::max<int64_t>(max_items, nl * ((out_shape[ax] + 127) / 128));
      }
    }
    L.U = U;
    L.V = V;
    L.logp = logp;
    L.logq = logq;
    L.logdx = logdx;
    L.logdy = logdy;
    L.pass[0] = G.pass[0];
    L.pass[1] = G.pass[1];
    L.nstage = nst;
    L.iters_per_stage = o->iters_per_stage;
    L.max_iter = o->max_iter;
    L.check_every = check_every;
    L.tol = o->tol;
    L.eps_ff = d_eps;
    L.inv_eps_ff = d_ieps;
    L.k2 = d_k2;
    L.F = d_F;
    L.acc = acc;
    L.bar = d_bar;
    L.status = d_status;
    L.err_out = d_err;
    const int cap = grid_solve_persistent_ctas(nin_max);
    if (cap < 1) return UOT_EUNSUPPORTED;
    const int grid = (int)std::min<int64_t>(cap, max_items);
    UOT_CK(launch_grid_solve_persistent(L, grid, s));
    int hs[4];
    double herr = 0.0;
    UOT_CK(cudaMemcpyAsync(hs, d_status, sizeof(hs), cudaMemcpyDeviceToHost, s));
    UOT_CK(cudaMemcpyAsync(&herr, d_err, sizeof(double), cudaMemcpyDeviceToHost, s));
    UOT_CK(cudaStreamSynchronize(s));
    if (hs[0]) {
      g_last_error = "persistent solve: a grid barrier wait expired";
      return UOT_TIMEOUT;
    }
    converged = hs[1] != 0;
    it = hs[2];
    total = hs[3];
    err = (o->max_iter > 0) ? herr : INFINITY;
  } else if (fused2d) {
    // Pass order per iteration: P1 (contract j2 of V rows) | K_A: P2 (contract j1
    // -> U columns), P3 (contract i1 of the same columns) | K_B: P4 (contract i2
    // -> V rows), P1 of the next iteration (contract j2 of the same rows).
    const int H1 = g->shape_x[0], W1 = g->shape_x[1], H2 = g->shape_y[0], W2 = g->shape_y[1];
    const float* xa0 = (const float*)g->axes_x[0];
    const float* xa1 = (const float*)g->axes_x[1];
    const float* ya0 = (const float*)g->axes_y[0];
    const float* ya1 = (const float*)g->axes_y[1];
    float2* T1 = reinterpret_cast<float2*>(G.pass[0]);
    float2* T2 = reinterpret_cast<float2*>(G.pass[1]);
    float* z[4] = {G.zbuf[0][0], G.zbuf[0][1], G.zbuf[1][0], G.zbuf[1][1]};
    double zeps[4] = {-1.0, -1.0, -1.0, -1.0};
    auto use = [&](int k, double e) {
      const int u = (zeps[k] == e) ? 1 : 0;
      zeps[k] = e;
      return u;
    };
    auto p1 = [&](double e, cudaStream_t st) -> cudaError_t {
      Epilogue r;
      memset(&r, 0, sizeof(r));
      r.mode = EPI_RAW;
      r.eps = e;
      r.ff = 1;
      r.out = G.pass[0];
      r.bstride = (int64_t)H2 * W1;
      const int u = use(0, e);
      return launch_grid_pass(UOT_F32, V, logdy, 1, H2, W2, ya1, W1, xa1, e, 1, r, st, z[0], u);
    };
    auto fused_args = [&](double e) {
      FusedArgs f;
      memset(&f, 0, sizeof(f));
      f.eps1_ff = ff2(ff_make(e));
      f.inv_eps1_ff = ff2(ff_make(1.0 / e));
      f.k2_1 = (float)((double)kLog2e / e);
      f.do2 = 1;
      return f;
    };
    auto ka = [&](double e, bool check, cudaStream_t st) -> cudaError_t {
      if (check) {
        cudaError_t e0 = cudaMemsetAsync(acc, 0, 2 * sizeof(double), st);
        if (e0 != cudaSuccess) return e0;
      }
      FusedArgs f = fused_args(e);
      f.nlines = W1;
      f.in1 = T1;
      f.nin1 = H2;
      f.nout1 = H1;
      f.y1 = ya0;
      f.x1 = xa0;
      f.out1_row = 0;
      f.F1 = make_div_ff(D1, e);
      f.logp1 = reinterpret_cast<const float2*>(logp);
      f.pot1 = reinterpret_cast<float2*>(U);
      f.logw1 = reinterpret_cast<const float2*>(logdx);
      f.err = check ? acc : nullptr;
      f.z1 = z[1];
      f.use_prev1 = use(1, e);
      f.nout2 = H2;
      f.x2 = ya0;
      f.inv_eps2_ff = ff2(ff_make(1.0 / e));
      f.k2_2 = (float)((double)kLog2e / e);
      f.out2 = T2;
      f.z2 = z[2];
      f.use_prev2 = use(2, e);
      return launch_grid_fused2(f, st);
    };
    auto kb = [&](double e, double e_next, cudaStream_t st) -> cudaError_t {
      FusedArgs f = fused_args(e);
      f.nlines = H2;
      f.in1 = T2;
      f.nin1 = W1;
      f.nout1 = W2;
      f.y1 = xa1;
      f.x1 = ya1;
      f.out1_row = 1;
      f.F1 = make_div_ff(D2, e);
      f.logp1 = reinterpret_cast<const float2*>(logq);
      f.pot1 = reinterpret_cast<float2*>(V);
      f.logw1 = reinterpret_cast<const float2*>(logdy);
      f.z1 = z[3];
      f.use_prev1 = use(3, e);
      f.nout2 = W1;
      f.x2 = xa1;
      f.inv_eps2_ff = ff2(ff_make(1.0 / e_next));
      f.k2_2 = (float)((double)kLog2e / e_next);
      f.out2 = T1;
      f.z2 = z[0];
      f.use_prev2 = use(0, e_next);
      return launch_grid_fused2(f, st);
    };
    // eps of the iteration after `total` stage iterations (the final eps after the stages)
    std::vector<double> stage_eps;
    for (const Stage& sg : stages)
      for (int k = 0; k < sg.iters; ++k) stage_eps.push_back(sg.eps);
    auto eps_at = [&](size_t k) { return k < stage_eps.size() ? stage_eps[k] : o->eps; };
    UOT_CK(p1(eps_at(0), s));
    for (size_t k = 0; k < stage_eps.size(); ++k, ++total) {
      UOT_CK(ka(stage_eps[k], false, s));
      UOT_CK(kb(stage_eps[k], eps_at(k + 1), s));
    }
    auto iteration = [&](bool check, cudaStream_t st) -> cudaError_t {
      cudaError_t e = ka(o->eps, check, st);
      if (e != cudaSuccess) return e;
      return kb(o->eps, o->eps, st);
    };
    BlockGraph bg;
    bool graph_ok = !profiling_on();
    while (it < o->max_iter) {
      if (graph_ok && it > 0 && it % check_every == 0 && it + check_every <= o->max_iter) {
        if (!bg.exec) {
          cudaError_t e = bg.capture([&](cudaStream_t cs) -> cudaError_t {
            for (int k = 0; k < check_every; ++k) {
              cudaError_t e2 = iteration(k == check_every - 1, cs);
              if (e2 != cudaSuccess) return e2;
            }
            return cudaSuccess;
          });
          if (e != cudaSuccess) {
            graph_ok = false;
            (void)cudaGetLastError();
            continue;
          }
        }
        UOT_CK(bg.launch(s));
        it += check_every;
        total += check_every;
        UOT_CK(read_err(err));
        if (o->tol > 0.0 && err <= o->tol) {
          converged = true;
          break;
        }
        continue;
      }
      const bool check = ((it + 1) % check_every == 0) || (it == o->max_iter - 1);
      UOT_CK(iteration(check, s));
      ++it;
      ++total;
      if (check) {
        UOT_CK(read_err(err));
        if (it > 1 && o->tol > 0.0 && err <= o->tol) {
          converged = true;
          break;
        }
      }
    }
  } else if (!o->plain_scaling) {
    // The stop decision after a check (err = the FP32 violation just read).
    // No 1% improvement on the best check for W iterations, W = max(50,
    // 5 check_every, 3x the iterations a 1% step took at the rate observed since
    // the first check): the check has reached the rounding floor of the passes.
    auto stalled = [&]() -> bool {
      if (std::isnan(first_err)) {
        first_err = err;
        first_it = it;
      }
      if (err < 0.99 * best_err) {
        best_err = err;
        best_it = it;
        return false;
      }
      double W = std::max(50, 5 * check_every);
      if (best_err < first_err && best_it > first_it) {
        const double rate = std::log(best_err / first_err) / (best_it - first_it);  // < 0
        W = std::max(W, std::min(1e8, 3.0 * std::log(0.99) / rate));
      }
      return it - best_it >= W;
    };
    auto decide = [&](bool& stop) -> cudaError_t {
      stop = false;
      err32 = err;
      if (!(o->tol > 0.0)) return cudaSuccess;
      if (mixed_phase) {
        // BF16 phase: hand over to the FP32 passes at mixed_switch or at the BF16 floor
        if (err <= mixed_switch || stalled()) {
          mixed_phase = false;
          mixed_iters = total;
          G.tc_off = true;
          mixed_handover = true;
          first_err = NAN;
          best_err = INFINITY;
        }
        return cudaSuccess;
      }
      if (!verify) {
        if (err <= o->tol) converged = stop = true;
        return cudaSuccess;
      }
      if (err <= tol_int) {
        cudaError_t e = cudaSuccess;
        if (!c64.ready && (e = c64.setup(*g, batch, p, dx, q, dy, s)) != cudaSuccess) return e;
        if ((e = c64.load_state(U, V, s)) != cudaSuccess) return e;
        if ((e = c64.iterate(D1, D2, o->eps, true, false, s)) != cudaSuccess) return e;
        if ((e = c64.read_err(err64, s)) != cudaSuccess) return e;
        ++nverify;
        if (err64 <= o->tol) {
          converged = stop = true;
          return cudaSuccess;
        }
        // aim the FP32 check proportionally lower
        tol_int = err * std::min(0.7, std::max(0.05, o->tol / err64));
        best_err = err;
        best_it = it;
        return cudaSuccess;
      }
      // the FP32 check's rounding floor: FP64 iterations take over
      if (stalled()) polish = stop = true;
      return cudaSuccess;
    };
    // shift: the translation step after the V-update (opts.translate)
    auto iteration = [&](double eps, bool check, bool shift, cudaStream_t st) -> cudaError_t {
      cudaError_t e;
      Epilogue e1 = prox_epilogue(D1, logp, U, logdx, check ? acc : nullptr, eps);
      e1.bstride = e1.bstride_p = n;
      if ((e = G.apply(0, V, logdy, eps, e1, st, check ? acc : nullptr)) != cudaSuccess) return e;
      Epilogue e2 = prox_epilogue(D2, logq, V, logdy, nullptr, eps);
      e2.bstride = e2.bstride_p = m;
      if ((e = G.apply(1, U, logdx, eps, e2, st)) != cudaSuccess || !shift) return e;
      return launch_kl_translate(U, V, logp, logq, logdx, logdy, n, m, batch, prec != UOT_F64, D1.lam, D2.lam,
                                 trpart, st);
    };
    for (const Stage& sg : stages)
      for (int k = 0; k < sg.iters; ++k, ++total)
        UOT_CK(iteration(sg.eps, false, translate && (k + 1) % check_every == 0, s));
    // launch_mode 2: once a block of check_every iterations (the last one
    // checked) repeats the same launches -- same eps, shifts from the previous
    // iteration -- it is captured once as a CUDA graph and replayed per block.
    BlockGraph bg;
    bool graph_ok = (o->launch_mode == 2 || o->launch_mode == 3) && !profiling_on();
    while (it < o->max_iter) {
      if (graph_ok && it > 0 && it % check_every == 0 && it + check_every <= o->max_iter) {
        if (!bg.exec) {
          cudaError_t e = bg.capture([&](cudaStream_t cs) -> cudaError_t {
            for (int k = 0; k < check_every; ++k) {
              cudaError_t e2 = iteration(o->eps, k == check_every - 1, translate && k == check_every - 1, cs);
              if (e2 != cudaSuccess) return e2;
            }
            return cudaSuccess;
          });
          if (e != cudaSuccess) {
            // not capturable here (e.g. a legacy-stream dependency): per-pass launches
            graph_ok = false;
            (void)cudaGetLastError();
            continue;
          }
        }
        UOT_CK(bg.launch(s));
        it += check_every;
        total += check_every;
        UOT_CK(read_err(err));
        bool stop = false;
        UOT_CK(decide(stop));
        if (stop) break;
        if (mixed_handover) {
          bg.reset();  // the block now launches the FP32 passes
          mixed_handover = false;
        }
        continue;
      }
      const bool check = ((it + 1) % check_every == 0) || (it == o->max_iter - 1);
      UOT_CK(iteration(o->eps, check, translate && check, s));
      ++it;
      ++total;
      if (check) {
        UOT_CK(read_err(err));
        if (it > 1) {
          bool stop = false;
          UOT_CK(decide(stop));
          if (stop) break;
          if (mixed_handover) {
            bg.reset();
            mixed_handover = false;
          }
        } else {
          err32 = err;
        }
      }
    }
    if (polish) {
      // the FP32 check has reached its rounding floor: FP64 iterations from the current state
      // Each check measures the state before its a-update; when it passes,
      // that state is restored and returned, so the reported FP64 violation
      // is the returned potentials' own.
      if (!c64.ready) UOT_CK(c64.setup(*g, batch, p, dx, q, dy, s));
      UOT_CK(c64.load_state(U, V, s));
      while (it < o->max_iter) {
        UOT_CK(c64.save_U(s));
        UOT_CK(c64.iterate(D1, D2, o->eps, true, false, s));
        UOT_CK(c64.read_err(err64, s));
        if (err64 <= o->tol) {
          UOT_CK(c64.restore_U(s));
          converged = true;
          break;
        }
        UOT_CK(c64.b_update(D2, o->eps, s));
        if (translate && (it + 1) % check_every == 0)
          UOT_CK(launch_kl_translate(c64.U, c64.V, c64.logp, c64.logq, c64.logdx, c64.logdy, n, m, batch, 0,
                                     D1.lam, D2.lam, trpart, s));
        ++it;
        ++total;
        ++npolish;
      }
      polished = true;
    }
    if (verify && !std::isnan(err64)) err = err64;
  } else {
    // Algorithm 1 on a stored FP64 kernel.
    double* K = sc.take<double>((size_t)n * m);
    double* KT = sc.take<double>((size_t)n * m);
    double* a = sc.take<double>(n);
    double* b = sc.take<double>(m);
    double* pd = sc.take<double>(n);
    double* qd = sc.take<double>(m);
    double* dxd = sc.take<double>(n);
    double* dyd = sc.take<double>(m);
    double* cres = sc.take<double>(4);
    UOT_SCRATCH_OK(sc);
    UOT_CK(to_f64(prec, p, n, pd, s));
    UOT_CK(to_f64(prec, q, m, qd, s));
    UOT_CK(to_f64(prec, dx, n, dxd, s));
    UOT_CK(to_f64(prec, dy, m, dyd, s));
    auto set_eps = [&](double eps) -> cudaError_t {
      count_launches(1);
      k_gibbs_matrix<double><<<nblocks(n * m), kNT, 0, s>>>((const double*)g->C, (int)n, (int)m, eps, K, KT);
      count_launches(1);
      k_exp_scale<<<nblocks(n), kNT, 0, s>>>(U, n, eps, a);
      count_launches(1);
      k_exp_scale<<<nblocks(m), kNT, 0, s>>>(V, m, eps, b);
      return cudaGetLastError();
    };
    auto to_pot = [&](double eps) -> cudaError_t {
      count_launches(1);
      k_log_scale<<<nblocks(n), kNT, 0, s>>>(a, n, eps, U);
      count_launches(1);
      k_log_scale<<<nblocks(m), kNT, 0, s>>>(b, m, eps, V);
      return cudaGetLastError();
    };
    // launch_mode 1: each eps runs as one launch of a cluster holding K in
    // shared memory (where it fits; the same iterates as the per-launch path)
    const bool cluster_mode = o->launch_mode == 1;
    for (const Stage& sg : stages) {
      UOT_CK(set_eps(sg.eps));
      bool launched = false;
      if (cluster_mode)
        UOT_CK(launch_alg1_cluster(K, KT, (int)n, (int)m, pd, dxd, qd, dyd, D1, D2, sg.eps, a, b, sg.iters, 0, 0.0,
                                   cres, s, &launched));
      if (launched) {
        total += sg.iters;
      } else {
        for (int k = 0; k < sg.iters; ++k, ++total) {
          UOT_CK(launch_alg1_half(K, (int)n, (int)m, b, dyd, pd, D1, sg.eps, a, dxd, nullptr, s));
          UOT_CK(launch_alg1_half(KT, (int)m, (int)n, a, dxd, qd, D2, sg.eps, b, dyd, nullptr, s));
        }
      }
      UOT_CK(to_pot(sg.eps));
    }
    UOT_CK(set_eps(o->eps));
    bool launched = false;
    if (cluster_mode && o->max_iter > 0)
      UOT_CK(launch_alg1_cluster(K, KT, (int)n, (int)m, pd, dxd, qd, dyd, D1, D2, o->eps, a, b, o->max_iter,
                                 check_every, o->tol, cres, s, &launched));
    if (launched) {
      double h[3];
      UOT_CK(cudaMemcpyAsync(h, cres, sizeof(h), cudaMemcpyDeviceToHost, s));
      UOT_CK(cudaStreamSynchronize(s));
      err = h[0];
      it = (int)h[1];
      total += it;
      converged = h[2] != 0.0;
    }
    while (!launched && it < o->max_iter) {
      const bool check = ((it + 1) % check_every == 0) || (it == o->max_iter - 1);
      if (check) UOT_CK(cudaMemsetAsync(acc, 0, 16, s));
      UOT_CK(launch_alg1_half(K, (int)n, (int)m, b, dyd, pd, D1, o->eps, a, dxd, check ? acc : nullptr, s));
      UOT_CK(launch_alg1_half(KT, (int)m, (int)n, a, dxd, qd, D2, o->eps, b, dyd, nullptr, s));
      ++it;
      ++total;
      if (check) {
        double h[2];
        UOT_CK(cudaMemcpyAsync(h, acc, 16, cudaMemcpyDeviceToHost, s));
        UOT_CK(cudaStreamSynchronize(s));
        err = (h[1] > 0.0) ? h[0] / h[1] : 0.0;
        if (it > 1 && o->tol > 0.0 && err <= o->tol) {
          converged = true;
          break;
        }
      }
    }
    UOT_CK(to_pot(o->eps));
  }

  // NaN check and output conversion (after FP64 iterations the state is FP64)
  const double* Ufin = polished ? c64.U : U;
  const double* Vfin = polished ? c64.V : V;
  const bool fin_ff = prec != UOT_F64 && !polished;
  UOT_CK(cudaMemsetAsync(flag, 0, 4, s));
  count_launches(1);
  k_nan_flag<<<nblocks(bn), kNT, 0, s>>>(Ufin, bn, fin_ff, flag);
  count_launches(1);
  k_nan_flag<<<nblocks(bm), kNT, 0, s>>>(Vfin, bm, fin_ff, flag);
  UOT_CK(cudaGetLastError());
  if (fin_ff && o->out_f64) {
    count_launches(2);
    k_ff_to_f64<<<nblocks(bn), kNT, 0, s>>>(reinterpret_cast<const float2*>(Ufin), bn, (double*)Uout);
    k_ff_to_f64<<<nblocks(bm), kNT, 0, s>>>(reinterpret_cast<const float2*>(Vfin), bm, (double*)Vout);
    UOT_CK(cudaGetLastError());
  } else if (!fin_ff && prec != UOT_F64 && !o->out_f64) {
    // FP64 state (after FP64 iterations) to float outputs
    count_launches(2);
    k_from_f64<float><<<nblocks(bn), kNT, 0, s>>>(Ufin, bn, (float*)Uout);
    k_from_f64<float><<<nblocks(bm), kNT, 0, s>>>(Vfin, bm, (float*)Vout);
    UOT_CK(cudaGetLastError());
  } else {
    const int out_prec = fin_ff ? prec : UOT_F64;
    UOT_CK(from_f64(out_prec, Ufin, bn, Uout, s));
    UOT_CK(from_f64(out_prec, Vfin, bm, Vout, s));
  }
  UOT_CK(cudaEventRecord(ev1, s));
  int hflag = 0, htc = 0;
  UOT_CK(cudaMemcpyAsync(&hflag, flag, 4, cudaMemcpyDeviceToHost, s));
  if (G.tc_err) UOT_CK(cudaMemcpyAsync(&htc, G.tc_err, 4, cudaMemcpyDeviceToHost, s));
  UOT_CK(cudaStreamSynchronize(s));
  float ms = 0.f;
  UOT_CK(cudaEventElapsedTime(&ms, ev0, ev1));
  uot_status out = htc ? UOT_TIMEOUT
                       : hflag ? UOT_NUMERICAL
                               : ((o->tol > 0.0 && !converged && o->max_iter > 0) ? UOT_NOT_CONVERGED : UOT_OK);
  if (res) {
    *res = empty_result();
    res->iters = it;
    res->total_iters = total;
    res->marg_err = err;
    res->ms = ms;
    res->status = out;
    res->verifications = nverify;
    res->polish_iters = npolish;
    res->marg_err_fp32 = err32;
    res->mixed_iters = prec != UOT_MIXED ? 0 : (G.tc_off ? mixed_iters : total);
  }
  return out;
}

// ---------------------------------------------------------------------------
// Algorithm 4 (Sec. 4.5): a divergence F3 on the total mass of the plan
// ---------------------------------------------------------------------------
// A scalar z = e^{Z/eps} multiplies the plan; both scaling updates see S + Z
// and T + Z.  z's own update needs the mass of the current plan without z,
// M = sum_i dx_i e^{(U_i + S_i)/eps} with S from the new b.  By Fubini M also
// equals sum_j dy_j e^{(V_j + T_j)/eps} with T from the current a, which the
// b-side of the previous iteration has at hand: when eps does not change,
// k_mass_vupdate computes V and the next Z in one kernel after the raw T pass,
// and the next a-side is the plain prox pass with Z added to S in its
// epilogue (zshift).  At an eps change the z-update takes the direct route:
// raw S pass -> k_mass_reduce (per-block maximum and sum of e^{l_i - max},
// l_i = log dx_i + U_i/eps + z_i, merged by the last block, then F3's row) ->
// k_mass_prox (U = prox_F1(S + Z) and the violation terms).  All kernels wait
// for their predecessor first (programmatic dependent launch).

constexpr int kMassBlocks = kNT;  // partials of the mass reduction: one per block, at most kNT blocks

struct MassArgs {
  int64_t n;
  double eps;
  float2 eps_ff, inv_eps_ff;
  DivParams F3;
  DivFF F3ff;
  double logm0;
  float2 logm0_ff;
  int update;        // 0 in the very first iteration: z = 1 stays
  int check;         // clear acc[0..1] and write the mass violation to acc[2]
  double* Z;         // [1] Z (FP64) or its float-float pair
  double* acc;       // [3] violation accumulators
  double2* part;     // [kMassBlocks] per-block (max, sum); float-float: (max.hi, max.lo) + sum
  unsigned* count;   // blocks finished (the last one sets it back to 0)
};

__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Block-wide maximum and sum (kNT threads), result broadcast to every thread.
__device__ inline double block_max_d(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  v = sh[0];
  for (int k = 1; k < kNT / 32; ++k) v = fmax(v, sh[k]);
  return v;
}
__device__ inline double block_sum_d(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  v = sh[0];
  for (int k = 1; k < kNT / 32; ++k) v += sh[k];
  return v;
}
__device__ inline ff block_max_ff(ff v, float2* sh) {
  for (int o = 16; o > 0; o >>= 1)
    v = ff_max(v, ff{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = ff2(v);
  __syncthreads();
  v = ffl(sh[0]);
  for (int k = 1; k < kNT / 32; ++k) v = ff_max(v, ffl(sh[k]));
  return v;
}
__device__ inline float block_sum_f(float v, float2* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = make_float2(v, 0.0f);
  __syncthreads();
  v = sh[0].x;
  for (int k = 1; k < kNT / 32; ++k) v += sh[k].x;
  return v;
}

constexpr int kMassPerThread = 4;  // elements per thread of the mass reduction (grid cap permitting)

// Per block: the maximum of l_i = log dx_i + U_i/eps + z_i over its
// grid-stride share, then the sum of e^{l_i - max} (a second sweep): two
// block reductions with one exponential per element.  The last block to
// finish merges the partials (one per thread, at most kNT blocks) the same
// way and applies F3's row.
template <bool FF>
__global__ void __launch_bounds__(kNT) k_mass_reduce(const double* __restrict__ U, const double* __restrict__ z,
                                                     const double* __restrict__ logdx, MassArgs a) {
  __shared__ double shd[kNT / 32];
  __shared__ float2 shf[kNT / 32];
  __shared__ bool last;
  pdl_begin();
  if (!a.update) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.check) a.acc[0] = a.acc[1] = 0.0;
    return;
  }
  const int64_t i0 = (int64_t)blockIdx.x * kNT + threadIdx.x, stride = (int64_t)gridDim.x * kNT;
  if constexpr (!FF) {
    auto lval = [&](int64_t i) {
      const double u = U[i], zi = z[i];
      return (u == -kInf || zi == -kInf) ? -kInf : logdx[i] + u / a.eps + zi;
    };
    double mx = -kInf;
    for (int64_t i = i0; i < a.n; i += stride) mx = fmax(mx, lval(i));
    mx = block_max_d(mx, shd);
    double s = 0.0;
    if (mx != -kInf)
      for (int64_t i = i0; i < a.n; i += stride) {
        const double l = lval(i);
        if (l != -kInf) s += exp(l - mx);
      }
    s = block_sum_d(s, shd);
    if (threadIdx.x == 0) {
      a.part[blockIdx.x] = make_double2(mx, s);
      __threadfence();
      last = atomicAdd(a.count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double2 v = make_double2(-kInf, 0.0);
    if (threadIdx.x < gridDim.x) v = __ldcg(&a.part[threadIdx.x]);
    const double M = block_max_d(v.x, shd);
    const double S = block_sum_d((M == -kInf || v.x == -kInf) ? 0.0 : v.y * exp(v.x - M), shd);
    if (threadIdx.x == 0) {
      // eps log M, then Z = prox of F3 at the total mass
      const double SM = (M == -kInf || S == 0.0) ? -kInf : a.eps * (M + log(S));
      a.Z[0] = prox_update(a.F3, a.logm0, SM, a.eps);
      if (a.check) a.acc[0] = a.acc[1] = 0.0;
      *a.count = 0u;
    }
  } else {
    const float2* U2 = reinterpret_cast<const float2*>(U);
    const float2* z2 = reinterpret_cast<const float2*>(z);
    const float2* w2 = reinterpret_cast<const float2*>(logdx);
    const ff inv_eps = ffl(a.inv_eps_ff);
    auto lval = [&](int64_t i) {
      const ff u = ffl(U2[i]), zi = ffl(z2[i]);
      return (u.hi == -INFINITY || zi.hi == -INFINITY) ? ff_ninf()
                                                       : ff_add(ff_add(ffl(w2[i]), ff_mul(u, inv_eps)), zi);
    };
    ff mx = ff_ninf();
    for (int64_t i = i0; i < a.n; i += stride) mx = ff_max(mx, lval(i));
    mx = block_max_ff(mx, shf);
    float s = 0.0f;
    if (mx.hi != -INFINITY)
      for (int64_t i = i0; i < a.n; i += stride) {
        const ff l = lval(i);
        if (l.hi == -INFINITY) continue;
        const ff d = ff_sub(l, mx);
        s += expf(d.hi + d.lo);
      }
    s = block_sum_f(s, shf);
    if (threadIdx.x == 0) {
      reinterpret_cast<float4*>(a.part)[blockIdx.x] = make_float4(mx.hi, mx.lo, s, 0.0f);
      __threadfence();
      last = atomicAdd(a.count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    float4 v = make_float4(-INFINITY, 0.0f, 0.0f, 0.0f);
    if (threadIdx.x < gridDim.x) v = __ldcg(&reinterpret_cast<const float4*>(a.part)[threadIdx.x]);
    const ff vm{v.x, v.y};
    const ff M = block_max_ff(vm, shf);
    float t = 0.0f;
    if (M.hi != -INFINITY && vm.hi != -INFINITY) {
      const ff d = ff_sub(vm, M);
      t = v.z * expf(d.hi + d.lo);
    }
    const float S = block_sum_f(t, shf);
    if (threadIdx.x == 0) {
      const ff eps = ffl(a.eps_ff);
      const ff SM = (M.hi == -INFINITY || S == 0.0f) ? ff_ninf() : ff_mul(eps, ff_add_f(M, logf(S)));
      reinterpret_cast<float2*>(a.Z)[0] = ff2(prox_update_ff(a.F3ff, ffl(a.logm0_ff), SM, eps));
      if (a.check) a.acc[0] = a.acc[1] = 0.0;
      *a.count = 0u;
    }
  }
}

struct MassProx {
  int64_t n;
  double eps;
  float2 eps_ff, inv_eps_ff;
  DivParams F;
  DivFF Fff;
  const double* Z;  // [1] Z (FP64) or its float-float pair
  double* err;      // [2] violation accumulators, NULL: no check
};

// pot_i = prox_F(log p_i, eps z_i + Z), z_i the raw log-sum of the Gibbs pass.
template <bool FF>
__global__ void __launch_bounds__(kNT) k_mass_prox(const double* __restrict__ z, const double* __restrict__ logp,
                                                   double* __restrict__ pot, const double* __restrict__ logw,
                                                   MassProx a) {
  pdl_begin();
  if constexpr (!FF) {
    const double Zv = a.Z[0];
    double num = 0.0, den = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kNT + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * kNT) {
      const double zi = z[i];
      const double Sz = (zi == -kInf || Zv == -kInf) ? -kInf : a.eps * zi + Zv;
      const double Uold = pot[i];
      const double Unew = prox_update(a.F, logp[i], Sz, a.eps);
      pot[i] = Unew;
      if (a.err) {
        double nu, de;
        violation_terms(Uold, Unew, Sz, logw[i], a.eps, nu, de);
        num += nu;
        den += de;
      }
    }
    if (a.err) block_add2<kNT>(num, den, a.err);
  } else {
    const ff Zv = ffl(reinterpret_cast<const float2*>(a.Z)[0]);
    const ff eps = ffl(a.eps_ff), inv_eps = ffl(a.inv_eps_ff);
    float2* pot2 = reinterpret_cast<float2*>(pot);
    float num = 0.0f, den = 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)kNT + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * kNT) {
      const ff zi = ffl(reinterpret_cast<const float2*>(z)[i]);
      const ff Sz = (zi.hi == -INFINITY || Zv.hi == -INFINITY) ? ff_ninf() : ff_add(ff_mul(zi, eps), Zv);
      const ff Uold = ffl(pot2[i]);
      const ff Unew = prox_update_ff(a.Fff, ffl(reinterpret_cast<const float2*>(logp)[i]), Sz, eps);
      pot2[i] = ff2(Unew);
      if (a.err) {
        float nu, de;
        violation_terms_ff(Uold, Unew, Sz, ffl(reinterpret_cast<const float2*>(logw)[i]), inv_eps, nu, de);
        num += nu;
        den += de;
      }
    }
    if (a.err) block_add2f<kNT>(num, den, a.err);
  }
}

// The b-side of an iteration in one kernel, when eps does not change from this
// iteration to the next: V_j = prox_F2(log q_j, T_j + Z), and the mass of the
// plan without z for the next z-update.  By Fubini the sum
// sum_i dx_i e^{(U_i + S_i)/eps}, S from the new b, equals
// sum_j dy_j e^{(V_j + T_j)/eps}, T from the current a, so it is reduced here
// (per block: maximum, then the sum of e^{l_j - max}; the last block merges).
// The last block applies F3's row and keeps the history of Z used for the
// mass violation: zhist[1] <- zhist[0], zhist[0] <- the Z this iteration used.
struct MassV {
  int64_t m;
  double eps;
  float2 eps_ff, inv_eps_ff;
  DivParams F2, F3;
  DivFF F2ff, F3ff;
  double logm0;
  float2 logm0_ff;
  double* Z;      // [1] Z (FP64) or its float-float pair: read, then replaced by the next one
  double* zhist;  // [2] the Z of this iteration and of the one before
  double2* part;  // [kMassBlocks]
  unsigned* count;
};

template <bool FF>
__global__ void __launch_bounds__(kNT) k_mass_vupdate(const double* __restrict__ zT, const double* __restrict__ logq,
                                                      double* __restrict__ V, const double* __restrict__ logdy,
                                                      MassV a) {
  __shared__ double shd[kNT / 32];
  __shared__ float2 shf[kNT / 32];
  __shared__ bool last;
  pdl_begin();
  const int64_t i0 = (int64_t)blockIdx.x * kNT + threadIdx.x, stride = (int64_t)gridDim.x * kNT;
  if constexpr (!FF) {
    const double Zv = a.Z[0];
    double mx = -kInf;
    for (int64_t j = i0; j < a.m; j += stride) {
      const double zj = zT[j];
      const double Sz = (zj == -kInf || Zv == -kInf) ? -kInf : a.eps * zj + Zv;
      const double v = prox_update(a.F2, logq[j], Sz, a.eps);
      V[j] = v;
      if (v != -kInf && zj != -kInf) mx = fmax(mx, logdy[j] + v / a.eps + zj);
    }
    mx = block_max_d(mx, shd);
    double s = 0.0;
    if (mx != -kInf)
      for (int64_t j = i0; j < a.m; j += stride) {
        const double v = V[j], zj = zT[j];
        if (v != -kInf && zj != -kInf) s += exp(logdy[j] + v / a.eps + zj - mx);
      }
    s = block_sum_d(s, shd);
    if (threadIdx.x == 0) {
      a.part[blockIdx.x] = make_double2(mx, s);
      __threadfence();
      last = atomicAdd(a.count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double2 pv = make_double2(-kInf, 0.0);
    if (threadIdx.x < gridDim.x) pv = __ldcg(&a.part[threadIdx.x]);
    const double M = block_max_d(pv.x, shd);
    const double Ssum = block_sum_d((M == -kInf || pv.x == -kInf) ? 0.0 : pv.y * exp(pv.x - M), shd);
    if (threadIdx.x == 0) {
      const double SM = (M == -kInf || Ssum == 0.0) ? -kInf : a.eps * (M + log(Ssum));
      reinterpret_cast<unsigned long long*>(a.zhist)[1] = reinterpret_cast<unsigned long long*>(a.zhist)[0];
      a.zhist[0] = Zv;
      a.Z[0] = prox_update(a.F3, a.logm0, SM, a.eps);
      *a.count = 0u;
    }
  } else {
    const float2* z2 = reinterpret_cast<const float2*>(zT);
    const float2* q2 = reinterpret_cast<const float2*>(logq);
    const float2* w2 = reinterpret_cast<const float2*>(logdy);
    float2* V2 = reinterpret_cast<float2*>(V);
    const ff eps = ffl(a.eps_ff), inv_eps = ffl(a.inv_eps_ff);
    const float2 Zraw = reinterpret_cast<const float2*>(a.Z)[0];
    const ff Zv = ffl(Zraw);
    auto lval = [&](ff v, ff zj, int64_t j) {
      return (v.hi == -INFINITY || zj.hi == -INFINITY) ? ff_ninf() : ff_add(ff_add(ffl(w2[j]), ff_mul(v, inv_eps)), zj);
    };
    ff mx = ff_ninf();
    for (int64_t j = i0; j < a.m; j += stride) {
      const ff zj = ffl(z2[j]);
      const ff Sz = (zj.hi == -INFINITY || Zv.hi == -INFINITY) ? ff_ninf() : ff_add(ff_mul(zj, eps), Zv);
      const ff v = prox_update_ff(a.F2ff, ffl(q2[j]), Sz, eps);
      V2[j] = ff2(v);
      mx = ff_max(mx, lval(v, zj, j));
    }
    mx = block_max_ff(mx, shf);
    float s = 0.0f;
    if (mx.hi != -INFINITY)
      for (int64_t j = i0; j < a.m; j += stride) {
        const ff l = lval(ffl(V2[j]), ffl(z2[j]), j);
        if (l.hi == -INFINITY) continue;
        const ff d = ff_sub(l, mx);
        s += expf(d.hi + d.lo);
      }
    s = block_sum_f(s, shf);
    if (threadIdx.x == 0) {
      reinterpret_cast<float4*>(a.part)[blockIdx.x] = make_float4(mx.hi, mx.lo, s, 0.0f);
      __threadfence();
      last = atomicAdd(a.count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    float4 pv = make_float4(-INFINITY, 0.0f, 0.0f, 0.0f);
    if (threadIdx.x < gridDim.x) pv = __ldcg(&reinterpret_cast<const float4*>(a.part)[threadIdx.x]);
    const ff vm{pv.x, pv.y};
    const ff M = block_max_ff(vm, shf);
    float t = 0.0f;
    if (M.hi != -INFINITY && vm.hi != -INFINITY) {
      const ff d = ff_sub(vm, M);
      t = pv.z * expf(d.hi + d.lo);
    }
    const float Ssum = block_sum_f(t, shf);
    if (threadIdx.x == 0) {
      const ff SM = (M.hi == -INFINITY || Ssum == 0.0f) ? ff_ninf() : ff_mul(eps, ff_add_f(M, logf(Ssum)));
      unsigned long long* zh = reinterpret_cast<unsigned long long*>(a.zhist);
      zh[1] = zh[0];
      reinterpret_cast<float2*>(a.zhist)[0] = Zraw;
      reinterpret_cast<float2*>(a.Z)[0] = ff2(prox_update_ff(a.F3ff, ffl(a.logm0_ff), SM, eps));
      *a.count = 0u;
    }
  }
}

uot_status solve_mass_impl(const uot_geom* g, const void* p, const void* dx, const void* q, const void* dy,
                           const uot_div* F1, const uot_div* F2, const uot_div* F3, double m0,
                           const uot_opts* o, void* Uout, void* Vout, double* Zout, uot_result* res,
                           cudaStream_t s) {
  uot_status st = check_geom(g);
  if (st != UOT_OK) return st;
  if ((st = check_opts(o)) != UOT_OK) return st;
  if (!p || !dx || !q || !dy || !Uout || !Vout || !Zout || !div_ok(F1) || !div_ok(F2) || !div_ok(F3))
    return UOT_EINVAL;
  if (!(m0 > 0.0) || !isfinite(m0)) return UOT_EINVAL;
  if (o->plain_scaling) return UOT_EUNSUPPORTED;
  const int prec = o->precision;
  const bool ffm = prec != UOT_F64;
  const int64_t n = g->n, m = g->m;
  const DivParams D1 = make_div(*F1), D2 = make_div(*F2), D3 = make_div(*F3);

  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  UOT_CK(cudaEventCreate(&ev0));
  UOT_CK(cudaEventCreate(&ev1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } evg{ev0, ev1};
  UOT_CK(cudaEventRecord(ev0, s));

  Scratch sc(s);
  Gibbs G;
  G.g = *g;
  G.prec = prec;
  G.speculate = true;
  G.plan(sc, 1);
  sc.reserve<double>(n);            // logp
  sc.reserve<double>(n);            // logdx
  sc.reserve<double>(n);            // U
  sc.reserve<double>(m);            // logq
  sc.reserve<double>(m);            // logdy
  sc.reserve<double>(m);            // V
  sc.reserve<double>(std::max(n, m));  // raw log-sums of the last pass (S/eps or T/eps)
  sc.reserve<double>(4);            // acc[3] + NaN flag
  sc.reserve<double>(3);            // Z, and the Z of the last two iterations
  sc.reserve<double2>(kMassBlocks); // mass partials
  sc.reserve<unsigned>(1);          // finished-block counter
  UOT_CK(sc.allocate());
  UOT_CK(G.take(sc, s));
  double* logp = sc.take<double>(n);
  double* logdx = sc.take<double>(n);
  double* U = sc.take<double>(n);
  double* logq = sc.take<double>(m);
  double* logdy = sc.take<double>(m);
  double* V = sc.take<double>(m);
  double* zb = sc.take<double>(std::max(n, m));
  double* acc = sc.take<double>(4);
  int* flag = (int*)(acc + 3);
  double* Zd = sc.take<double>(3);
  double* zhist = Zd + 1;
  double2* part = sc.take<double2>(kMassBlocks);
  unsigned* count = sc.take<unsigned>(1);
  UOT_SCRATCH_OK(sc);
  UOT_CK(to_log(prec, p, n, logp, s));
  UOT_CK(to_log(prec, dx, n, logdx, s));
  UOT_CK(to_log(prec, q, m, logq, s));
  UOT_CK(to_log(prec, dy, m, logdy, s));
  if (o->U0) {
    UOT_CK(to_f64(prec, o->U0, n, U, s));
  } else {
    count_launches(1);
    k_fill<<<nblocks(n), kNT, 0, s>>>(U, n, 0.0);
  }
  if (o->V0) {
    UOT_CK(to_f64(prec, o->V0, m, V, s));
  } else {
    count_launches(1);
    k_fill<<<nblocks(m), kNT, 0, s>>>(V, m, 0.0);
  }
  UOT_CK(cudaMemsetAsync(Zd, 0, 3 * sizeof(double), s));  // z = 1 (both layouts)
  UOT_CK(cudaMemsetAsync(acc, 0, 4 * sizeof(double), s));
  UOT_CK(cudaMemsetAsync(count, 0, sizeof(unsigned), s));
  UOT_CK(cudaGetLastError());

  // one partial per block (at most kNT: the last block merges them with one thread each)
  const int64_t per_block = (int64_t)kNT * kMassPerThread;
  const int red_blocks = (int)std::min<int64_t>(kNT, std::max<int64_t>(1, (n + per_block - 1) / per_block));
  bool first = true;
  // programmatic dependent launch (the kernels wait for their predecessor first)
  auto pdl_launch = [&](auto kern, int grid, cudaStream_t st, auto... args) -> cudaError_t {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kNT);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launches(1);
    return cudaLaunchKernelEx(&cfg, kern, args...);
  };
  auto prox_a = [&](double eps, double* err, cudaStream_t st) -> cudaError_t {
    MassProx a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.eps = eps;
    a.eps_ff = ff2(ff_make(eps));
    a.inv_eps_ff = ff2(ff_make(1.0 / eps));
    a.F = D1;
    a.Fff = make_div_ff(D1, eps);
    a.Z = Zd;
    a.err = err;
    const double* zc = zb;
    const double* lp = logp;
    const double* lw = logdx;
    if (ffm) return pdl_launch(k_mass_prox<true>, nblocks(n), st, zc, lp, U, lw, a);
    return pdl_launch(k_mass_prox<false>, nblocks(n), st, zc, lp, U, lw, a);
  };
  // One iteration.  a-side: with eps unchanged since the previous iteration the
  // b-side of that iteration has already computed this iteration's Z (Fubini,
  // k_mass_vupdate), so the prox of S + Z runs in the pass epilogue; otherwise
  // (the first iteration of a new eps stage) the z-update takes the plain route:
  // raw pass, k_mass_reduce, k_mass_prox.  The very first iteration keeps z = 1.
  // b-side: raw pass, then k_mass_vupdate (V and the next Z).
  double prev_eps = -1.0;
  auto iteration = [&](double eps, bool check, cudaStream_t st) -> cudaError_t {
    cudaError_t e;
    Epilogue r;
    memset(&r, 0, sizeof(r));
    r.mode = EPI_RAW;
    set_eps(r, eps);
    r.out = zb;
    r.bstride = n;
    const bool plain = !first && eps != prev_eps;
    if (plain) {
      if ((e = G.apply(0, V, logdy, eps, r, st)) != cudaSuccess) return e;
      MassArgs a;
      memset(&a, 0, sizeof(a));
      a.n = n;
      a.eps = eps;
      a.eps_ff = ff2(ff_make(eps));
      a.inv_eps_ff = ff2(ff_make(1.0 / eps));
      a.F3 = D3;
      a.F3ff = make_div_ff(D3, eps);
      a.logm0 = log(m0);
      a.logm0_ff = ff2(ff_make(log(m0)));
      a.update = 1;
      a.check = check ? 1 : 0;
      a.Z = Zd;
      a.acc = acc;
      a.part = part;
      a.count = count;
      const double* Uc = U;
      const double* zc = zb;
      const double* lw = logdx;
      e = ffm ? pdl_launch(k_mass_reduce<true>, red_blocks, st, Uc, zc, lw, a)
              : pdl_launch(k_mass_reduce<false>, red_blocks, st, Uc, zc, lw, a);
      if (e != cudaSuccess) return e;
      if ((e = prox_a(eps, check ? acc : nullptr, st)) != cudaSuccess) return e;
    } else {
      Epilogue e1 = prox_epilogue(D1, logp, U, logdx, check ? acc : nullptr, eps);
      e1.bstride = e1.bstride_p = n;
      e1.zshift = Zd;
      if ((e = G.apply(0, V, logdy, eps, e1, st, check ? acc : nullptr)) != cudaSuccess) return e;
    }
    first = false;
    prev_eps = eps;
    r.bstride = m;
    if ((e = G.apply(1, U, logdx, eps, r, st)) != cudaSuccess) return e;
    MassV b;
    memset(&b, 0, sizeof(b));
    b.m = m;
    b.eps = eps;
    b.eps_ff = ff2(ff_make(eps));
    b.inv_eps_ff = ff2(ff_make(1.0 / eps));
    b.F2 = D2;
    b.F3 = D3;
    b.F2ff = make_div_ff(D2, eps);
    b.F3ff = make_div_ff(D3, eps);
    b.logm0 = log(m0);
    b.logm0_ff = ff2(ff_make(log(m0)));
    b.Z = Zd;
    b.zhist = zhist;
    b.part = part;
    b.count = count;
    const double* zc = zb;
    const double* lq = logq;
    const double* lw = logdy;
    const int vb = (int)std::min<int64_t>(kNT, std::max<int64_t>(1, (m + per_block - 1) / per_block));
    return ffm ? pdl_launch(k_mass_vupdate<true>, vb, st, zc, lq, V, lw, b)
               : pdl_launch(k_mass_vupdate<false>, vb, st, zc, lq, V, lw, b);
  };
  // the checked iteration's violations: the marginal one from acc, and the mass
  // one |e^{(Z_old - Z)/eps} - 1| of its z-update from the history of Z (after
  // the iteration, zhist = {its Z, the previous Z})
  double hacc[2], hz[2];
  auto zval = [&](double v) {
    if (!ffm) return v;
    float2 f;
    memcpy(&f, &v, sizeof(f));
    return (double)f.x + (double)f.y;
  };
  auto read_err = [&](double& out) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(hacc, acc, sizeof(hacc), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(hz, zhist, sizeof(hz), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    const double v = (hacc[1] > 0.0) ? hacc[0] / hacc[1] : 0.0;
    const double zn = zval(hz[0]), zo = zval(hz[1]);
    const double merr = (std::isfinite(zn) && std::isfinite(zo)) ? std::fabs(std::expm1((zo - zn) / o->eps)) : 0.0;
    out = (v != v) ? NAN : std::max(v, merr);
    return cudaSuccess;
  };

  const std::vector<Stage> stages = eps_schedule(*o);
  const int check_every = o->check_every > 0 ? o->check_every : 1;
  int it = 0, total = 0;
  double err = INFINITY;
  bool converged = false;
  for (const Stage& sg : stages)
    for (int k = 0; k < sg.iters; ++k, ++total) UOT_CK(iteration(sg.eps, false, s));
  // launch_mode 2 (and 1, 3, which have no mass variant): blocks of
  // check_every iterations at the final eps replayed as one CUDA graph.
  BlockGraph bg;
  bool graph_ok = o->launch_mode != 0 && !profiling_on();
  while (it < o->max_iter) {
    if (graph_ok && !first && it > 0 && it % check_every == 0 && it + check_every <= o->max_iter) {
      if (!bg.exec) {
        cudaError_t e = bg.capture([&](cudaStream_t cs) -> cudaError_t {
          for (int k = 0; k < check_every; ++k) {
            cudaError_t e2 = iteration(o->eps, k == check_every - 1, cs);
            if (e2 != cudaSuccess) return e2;
          }
          return cudaSuccess;
        });
        if (e != cudaSuccess) {
          graph_ok = false;
          (void)cudaGetLastError();
          continue;
        }
      }
      UOT_CK(bg.launch(s));
      it += check_every;
      total += check_every;
      UOT_CK(read_err(err));
      if (o->tol > 0.0 && err <= o->tol) {
        converged = true;
        break;
      }
      continue;
    }
    const bool check = ((it + 1) % check_every == 0) || (it == o->max_iter - 1);
    UOT_CK(iteration(o->eps, check, s));
    ++it;
    ++total;
    if (check) {
      UOT_CK(read_err(err));
      if (it > 1 && o->tol > 0.0 && err <= o->tol) {
        converged = true;
        break;
      }
    }
  }

  UOT_CK(cudaMemsetAsync(flag, 0, 4, s));
  count_launches(1);
  k_nan_flag<<<nblocks(n), kNT, 0, s>>>(U, n, ffm, flag);
  count_launches(1);
  k_nan_flag<<<nblocks(m), kNT, 0, s>>>(V, m, ffm, flag);
  UOT_CK(cudaGetLastError());
  UOT_CK(from_f64(prec, U, n, Uout, s));
  UOT_CK(from_f64(prec, V, m, Vout, s));
  UOT_CK(cudaEventRecord(ev1, s));
  int hflag = 0, htc = 0;
  double hZ = 0.0;
  UOT_CK(cudaMemcpyAsync(&hflag, flag, 4, cudaMemcpyDeviceToHost, s));
  UOT_CK(cudaMemcpyAsync(&hZ, zhist, 8, cudaMemcpyDeviceToHost, s));  // the Z of the last iteration
  if (G.tc_err) UOT_CK(cudaMemcpyAsync(&htc, G.tc_err, 4, cudaMemcpyDeviceToHost, s));
  UOT_CK(cudaStreamSynchronize(s));
  if (ffm) {
    float2 zz;
    memcpy(&zz, &hZ, sizeof(zz));
    hZ = (double)zz.x + (double)zz.y;
  }
  *Zout = hZ;
  float ms = 0.f;
  UOT_CK(cudaEventElapsedTime(&ms, ev0, ev1));
  uot_status out = htc ? UOT_TIMEOUT
                       : (hflag || hZ != hZ) ? UOT_NUMERICAL
                                             : ((o->tol > 0.0 && !converged && o->max_iter > 0) ? UOT_NOT_CONVERGED : UOT_OK);
  if (res) {
    *res = empty_result();
    res->iters = it;
    res->total_iters = total;
    res->marg_err = err;
    res->ms = ms;
    res->status = out;
  }
  return out;
}


// ---------------------------------------------------------------------------
// WF gradient flows with growth (Sec. 5.3)
// ---------------------------------------------------------------------------
// Each minimizing-movement step (eq. grad-flow) solves, for S species on the
// same points (X = Y, dy = dx), the scaling iteration with F1 = lam KL(.|p^k)
// per species and the joint F2 of the growth functional
// G = -alpha sum_k mu^k(X) + iota_{<=1}(sum_k d mu^k/dx).  F2's log-form
// proxdiv is the same for every species:
//   V^k = min(-lam log c, -lam Ttot/(lam + eps)),  Ttot = eps log sum_k e^{T^k/eps},
// c = 1 - 2 tau alpha/lam.  The step ends with the next densities
// p^k = r2^k / max(c, sum_k r2^k), r2^k = e^{(V^k + T^k)/eps} the second
// marginals of the step's couplings.

// WF cost (eq. logcost) c = -log cos^2((pi/2)|x - y|/cut), +inf from |x - y| >= cut.
template <typename T>
__global__ void k_wf_cost(const T* __restrict__ x, int n, const T* __restrict__ y, int m, int d, double cut,
                          T* __restrict__ C) {
  const int64_t total = (int64_t)n * m;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / m, j = q - i * m;
    double r2 = 0.0;
    for (int k = 0; k < d; ++k) {
      const double t = (double)x[i * d + k] - (double)y[j * d + k];
      r2 += t * t;
    }
    const double dist = sqrt(r2);
    const double v = (dist >= cut) ? kInf : -2.0 * log(cos(1.5707963267948966 * dist / cut));
    C[q] = (T)v;
  }
}

struct GrowthArgs {
  int S;
  int64_t m;
  double eps, inv_eps, neg_lam_logc, klin, c;  // klin = lam/(lam + eps)
  float2 eps_ff, inv_eps_ff, neg_lam_logc_ff, klin_ff;
};

template <bool FF>
__global__ void __launch_bounds__(kNT) k_growth_prox(const double* __restrict__ Tz, double* __restrict__ V,
                                                     GrowthArgs a) {
  pdl_begin();
  for (int64_t j = blockIdx.x * (int64_t)kNT + threadIdx.x; j < a.m; j += (int64_t)gridDim.x * kNT) {
    if constexpr (!FF) {
      double mx = -kInf;
      for (int k = 0; k < a.S; ++k) mx = fmax(mx, Tz[k * a.m + j]);
      double v = a.neg_lam_logc;
      if (mx != -kInf) {
        double L = mx;  // one species: the log-sum-exp is the value itself
        if (a.S > 1) {
          double s = 0.0;
          for (int k = 0; k < a.S; ++k) s += exp(Tz[k * a.m + j] - mx);
          L += log(s);
        }
        v = fmin(v, -a.klin * (a.eps * L));
      }
      for (int k = 0; k < a.S; ++k) V[k * a.m + j] = v;
    } else {
      const float2* T2 = reinterpret_cast<const float2*>(Tz);
      ff mx = ff_ninf();
      for (int k = 0; k < a.S; ++k) mx = ff_max(mx, ffl(T2[k * a.m + j]));
      ff v = ffl(a.neg_lam_logc_ff);
      if (mx.hi != -INFINITY) {
        ff L = mx;  // one species: the log-sum-exp is the value itself
        if (a.S > 1) {
          float s = 0.0f;
          for (int k = 0; k < a.S; ++k) {
            const ff t = ffl(T2[k * a.m + j]);
            if (t.hi == -INFINITY) continue;
            const ff dlt = ff_sub(t, mx);
            s += expf(dlt.hi + dlt.lo);
          }
          L = ff_add_f(mx, logf(s));
        }
        v = ff_min(v, ff_neg(ff_mul(ffl(a.klin_ff), ff_mul(ffl(a.eps_ff), L))));
      }
      float2* V2 = reinterpret_cast<float2*>(V);
      for (int k = 0; k < a.S; ++k) V2[k * a.m + j] = ff2(v);
    }
  }
}

// Next densities from the plan's second marginals; writes the log densities
// (the next step's F1 targets) and the densities in the caller's type.
template <bool FF>
__global__ void __launch_bounds__(kNT) k_growth_density(const double* __restrict__ Tz, const double* __restrict__ V,
                                                        GrowthArgs a, double* __restrict__ logp, void* __restrict__ pout) {
  for (int64_t j = blockIdx.x * (int64_t)kNT + threadIdx.x; j < a.m; j += (int64_t)gridDim.x * kNT) {
    if constexpr (!FF) {
      double tot = 0.0;
      for (int k = 0; k < a.S; ++k) {
        const double z = Tz[k * a.m + j], v = V[k * a.m + j];
        tot += (z == -kInf || v == -kInf) ? 0.0 : exp(v * a.inv_eps + z);
      }
      const double den = fmax(a.c, tot), lden = log(den);
      for (int k = 0; k < a.S; ++k) {
        const int64_t q = k * a.m + j;
        const double z = Tz[q], v = V[q];
        const bool zero = (z == -kInf || v == -kInf);
        const double lr = zero ? -kInf : v * a.inv_eps + z;
        logp[q] = zero ? -kInf : lr - lden;
        reinterpret_cast<double*>(pout)[q] = zero ? 0.0 : exp(lr) / den;
      }
    } else {
      const float2* T2 = reinterpret_cast<const float2*>(Tz);
      const float2* V2 = reinterpret_cast<const float2*>(V);
      const ff ie = ffl(a.inv_eps_ff);
      float tot = 0.0f;
      for (int k = 0; k < a.S; ++k) {
        const ff z = ffl(T2[k * a.m + j]), v = ffl(V2[k * a.m + j]);
        if (z.hi == -INFINITY || v.hi == -INFINITY) continue;
        const ff lr = ff_add(ff_mul(v, ie), z);
        tot += expf(lr.hi + lr.lo);
      }
      const float den = fmaxf((float)a.c, tot), lden = logf(den);
      for (int k = 0; k < a.S; ++k) {
        const int64_t q = k * a.m + j;
        const ff z = ffl(T2[q]), v = ffl(V2[q]);
        float2* lp2 = reinterpret_cast<float2*>(logp);
        if (z.hi == -INFINITY || v.hi == -INFINITY) {
          lp2[q] = ff2(ff_ninf());
          reinterpret_cast<float*>(pout)[q] = 0.0f;
          continue;
        }
        const ff lp = ff_add_f(ff_add(ff_mul(v, ie), z), -lden);
        lp2[q] = ff2(lp);
        reinterpret_cast<float*>(pout)[q] = expf(lp.hi + lp.lo);
      }
    }
  }
}

uot_status wf_flow_impl(const uot_geom* g, int S, const void* P0, const void* dx, double tau, double alpha,
                        double lam, const uot_opts* o, int nsteps, void* Pout, void* Uout, void* Vout,
                        uot_result* res, cudaStream_t s) {
  uot_status st = check_geom(g);
  if (st != UOT_OK) return st;
  if ((st = check_opts(o)) != UOT_OK) return st;
  if (g->n != g->m || S < 1 || nsteps < 1 || !P0 || !dx || !Pout || !Uout || !Vout) return UOT_EINVAL;
  if (!(tau > 0.0) || !isfinite(tau) || !(alpha >= 0.0) || !isfinite(alpha) || !(lam > 0.0) || !isfinite(lam))
    return UOT_EINVAL;
  const double c = 1.0 - 2.0 * tau * alpha / lam;
  if (!(c > 0.0 && c <= 1.0)) return UOT_EINVAL;
  if (o->tol != 0.0 || o->U0 || o->V0) return UOT_EINVAL;
  if (o->plain_scaling || o->precision == UOT_MIXED) return UOT_EUNSUPPORTED;
  if (g->kind == UOT_GEOM_GRID && S > 65535) return UOT_EUNSUPPORTED;
  const int prec = o->precision;
  const bool ffm = prec != UOT_F64;
  const size_t esz = ffm ? 4 : 8;
  const int64_t n = g->n, Sn = (int64_t)S * n;

  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  UOT_CK(cudaEventCreate(&ev0));
  UOT_CK(cudaEventCreate(&ev1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } evg{ev0, ev1};
  UOT_CK(cudaEventRecord(ev0, s));

  Scratch sc(s);
  Gibbs G;
  G.g = *g;
  G.prec = prec;
  G.speculate = true;
  G.plan(sc, S);
  sc.reserve<double>(Sn);        // log p^k (F1 targets)
  sc.reserve<double>(n);         // log dx
  sc.reserve<double>(Sn);        // U
  sc.reserve<double>(Sn);        // V
  sc.reserve<double>(Sn);        // raw log-sums T^k/eps
  sc.reserve<char>(Sn * esz);    // densities of the current step
  sc.reserve<int>(1);            // NaN flag
  UOT_CK(sc.allocate());
  UOT_CK(G.take(sc, s));
  double* logp = sc.take<double>(Sn);
  double* logdx = sc.take<double>(n);
  double* U = sc.take<double>(Sn);
  double* V = sc.take<double>(Sn);
  double* Tz = sc.take<double>(Sn);
  char* pstep = sc.take<char>(Sn * esz);
  int* flag = sc.take<int>(1);
  UOT_SCRATCH_OK(sc);
  UOT_CK(to_log(prec, P0, Sn, logp, s));
  UOT_CK(to_log(prec, dx, n, logdx, s));

  const DivParams D1 = make_div(uot_div{UOT_DIV_KL, lam, 0.0, 0.0});
  auto gargs = [&](double eps) {
    GrowthArgs a;
    memset(&a, 0, sizeof(a));
    a.S = S;
    a.m = n;
    a.eps = eps;
    a.inv_eps = 1.0 / eps;
    a.neg_lam_logc = -lam * log(c);
    a.klin = lam / (lam + eps);
    a.c = c;
    a.eps_ff = ff2(ff_make(eps));
    a.inv_eps_ff = ff2(ff_make(1.0 / eps));
    a.neg_lam_logc_ff = ff2(ff_make(-lam * log(c)));
    a.klin_ff = ff2(ff_make(lam / (lam + eps)));
    return a;
  };
  auto iteration = [&](double eps, cudaStream_t st) -> cudaError_t {
    cudaError_t e;
    Epilogue e1 = prox_epilogue(D1, logp, U, logdx, nullptr, eps);
    e1.bstride = e1.bstride_p = n;
    if ((e = G.apply(0, V, logdx, eps, e1, st)) != cudaSuccess) return e;
    Epilogue r;
    memset(&r, 0, sizeof(r));
    r.mode = EPI_RAW;
    set_eps(r, eps);
    r.out = Tz;
    r.bstride = n;
    if ((e = G.apply(1, U, logdx, eps, r, st)) != cudaSuccess) return e;
    count_launches(1);
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(nblocks(n));
    cfg.blockDim = dim3(kNT);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const double* tz = Tz;
    return ffm ? cudaLaunchKernelEx(&cfg, k_growth_prox<true>, tz, V, gargs(eps))
               : cudaLaunchKernelEx(&cfg, k_growth_prox<false>, tz, V, gargs(eps));
  };
  const std::vector<Stage> stages = eps_schedule(*o);
  int stage_iters = 0;
  for (const Stage& sg : stages) stage_iters += sg.iters;
  auto step = [&](cudaStream_t st) -> cudaError_t {
    cudaError_t e;
    count_launches(2);
    k_fill<<<nblocks(Sn), kNT, 0, st>>>(U, Sn, 0.0);
    k_fill<<<nblocks(Sn), kNT, 0, st>>>(V, Sn, 0.0);  // b = 1 (both layouts)
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (const Stage& sg : stages)
      for (int k = 0; k < sg.iters; ++k)
        if ((e = iteration(sg.eps, st)) != cudaSuccess) return e;
    for (int k = 0; k < o->max_iter; ++k)
      if ((e = iteration(o->eps, st)) != cudaSuccess) return e;
    count_launches(1);
    if (ffm)
      k_growth_density<true><<<nblocks(n), kNT, 0, st>>>(Tz, V, gargs(o->eps), logp, pstep);
    else
      k_growth_density<false><<<nblocks(n), kNT, 0, st>>>(Tz, V, gargs(o->eps), logp, pstep);
    return cudaGetLastError();
  };
  // launch_mode 2: the first step runs launch by launch; later steps replay
  // it as one CUDA graph (the step repeats the same launches).
  BlockGraph bg;
  bool graph_ok = o->launch_mode != 0 && !profiling_on();
  for (int k = 0; k < nsteps; ++k) {
    if (graph_ok && k > 0) {
      if (!bg.exec) {
        cudaError_t e = bg.capture([&](cudaStream_t cs) { return step(cs); });
        if (e != cudaSuccess) {
          graph_ok = false;
          (void)cudaGetLastError();
        }
      }
    }
    if (graph_ok && bg.exec)
      UOT_CK(bg.launch(s));
    else
      UOT_CK(step(s));
    UOT_CK(cudaMemcpyAsync((char*)Pout + (size_t)k * Sn * esz, pstep, Sn * esz, cudaMemcpyDeviceToDevice, s));
  }

  UOT_CK(cudaMemsetAsync(flag, 0, 4, s));
  count_launches(2);
  k_nan_flag<<<nblocks(Sn), kNT, 0, s>>>(U, Sn, ffm, flag);
  k_nan_flag<<<nblocks(Sn), kNT, 0, s>>>(V, Sn, ffm, flag);
  UOT_CK(cudaGetLastError());
  UOT_CK(from_f64(prec, U, Sn, Uout, s));
  UOT_CK(from_f64(prec, V, Sn, Vout, s));
  UOT_CK(cudaEventRecord(ev1, s));
  int hflag = 0, htc = 0;
  UOT_CK(cudaMemcpyAsync(&hflag, flag, 4, cudaMemcpyDeviceToHost, s));
  if (G.tc_err) UOT_CK(cudaMemcpyAsync(&htc, G.tc_err, 4, cudaMemcpyDeviceToHost, s));
  UOT_CK(cudaStreamSynchronize(s));
  float ms = 0.f;
  UOT_CK(cudaEventElapsedTime(&ms, ev0, ev1));
  const uot_status out = htc ? UOT_TIMEOUT : hflag ? UOT_NUMERICAL : UOT_OK;
  if (res) {
    *res = empty_result();
    res->iters = o->max_iter;
    res->total_iters = nsteps * (stage_iters + o->max_iter);
    res->marg_err = NAN;
    res->ms = ms;
    res->status = out;
  }
  return out;
}


// ---------------------------------------------------------------------------
// Colour transfer (Sec. 5.1): histograms, barycentric projection, bin map
// ---------------------------------------------------------------------------

constexpr int kMaxBinDim = 8;
struct BinGrid {
  int d;
  int shape[kMaxBinDim];
};

// Row-major bin of a point of [0, 1]^d: bin k of axis a covers [k/n_a, (k+1)/n_a);
// the floor is taken on the FP32 product x * n_a, outside points are clamped
// and NaN goes to bin 0.
__device__ __forceinline__ int64_t bin_of(const float* __restrict__ x, const BinGrid& b) {
  int64_t idx = 0;
  for (int a = 0; a < b.d; ++a) {
    const float v = floorf(__fmul_rn(x[a], (float)b.shape[a]));
    const int k = (v != v || v < 0.0f) ? 0 : (v > (float)(b.shape[a] - 1) ? b.shape[a] - 1 : (int)v);
    idx = idx * b.shape[a] + k;
  }
  return idx;
}

__global__ void k_histogram(const float* __restrict__ pts, int64_t npts, BinGrid b, unsigned* __restrict__ counts) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npts; q += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&counts[bin_of(pts + q * b.d, b)], 1u);
}

template <typename T>
__global__ void k_hist_norm(const unsigned* __restrict__ counts, int64_t nb, double npts, T* __restrict__ p) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (T)((double)counts[i] / npts);
}

struct PointsOf {
  int kind, d;  // UOT_GEOM_GRID: axes and shape; UOT_GEOM_POINTS: row-major points
  int shape[UOT_MAX_DIM];
  const void* axes[UOT_MAX_DIM];
  const void* pts;
};

template <typename T>
__device__ __forceinline__ T coord_of(const PointsOf& P, int64_t j, int k) {
  if (P.kind == UOT_GEOM_POINTS) return reinterpret_cast<const T*>(P.pts)[j * P.d + k];
  int64_t r = j;
  for (int a = P.d - 1; a > k; --a) r /= P.shape[a];
  return reinterpret_cast<const T*>(P.axes[k])[r % P.shape[k]];
}

// F[j][0..d-1] = coordinates of point j, F[j][d] = 1.
template <typename T>
__global__ void k_coords1(PointsOf P, int64_t m, T* __restrict__ F) {
  const int c = P.d + 1;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m * c; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = q / c;
    const int k = (int)(q - j * c);
    F[q] = (k == P.d) ? T(1) : coord_of<T>(P, j, k);
  }
}

// T_i = RF[i][0..d-1] / RF[i][d]; rows of zero plan mass keep their own point.
template <typename T>
__global__ void k_bary_divide(const T* __restrict__ RF, PointsOf X, int64_t n, T* __restrict__ Tm) {
  const int d = X.d, c = d + 1;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * d; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / d;
    const int k = (int)(q - i * d);
    const T den = RF[i * c + d];
    Tm[q] = (den > T(0)) ? RF[i * c + k] / den : coord_of<T>(X, i, k);
  }
}

template <typename T>
__global__ void k_apply_bin_map(const float* __restrict__ pts, int64_t npts, BinGrid b, const T* __restrict__ Tm,
                                float* __restrict__ out) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npts; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t bin = bin_of(pts + q * b.d, b);
    for (int c = 0; c < b.d; ++c) out[q * b.d + c] = (float)Tm[bin * b.d + c];
  }
}

uot_status bin_grid(int d, const int* shape, BinGrid& b, int64_t& nb) {
  if (d < 1 || d > kMaxBinDim || !shape) return UOT_EINVAL;
  b.d = d;
  nb = 1;
  for (int a = 0; a < d; ++a) {
    if (shape[a] < 1) return UOT_EINVAL;
    b.shape[a] = shape[a];
    nb *= shape[a];
    if (nb > ((int64_t)1 << 31)) return UOT_EINVAL;
  }
  return UOT_OK;
}

}  // namespace

void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void prof_mark_begin(int family, cudaStream_t s) {
  if (!g_prof.on) return;
  std::lock_guard<std::mutex> lk(g_prof.mu);
  cudaEvent_t e = prof_event();
  cudaEventRecord(e, s);
  g_prof.pending[family] = e;
}

void prof_mark_end(int family, cudaStream_t s) {
  if (!g_prof.on) return;
  std::lock_guard<std::mutex> lk(g_prof.mu);
  cudaEvent_t e = prof_event();
  cudaEventRecord(e, s);
  g_prof.marks[family].push_back({g_prof.pending[family], e});
}

}  // namespace uot

using namespace uot;

extern "C" {

const char* uot_version(void) { return "uot-gb300 0.1 (sm_103a)"; }

const char* uot_last_error(void) { return g_last_error.c_str(); }

long long uot_launch_count(void) { return g_launches.load(); }

int uot_set_autotune(int mode) { return grid_set_autotune(mode); }

uot_status uot_force_grid_tile(int idx) { return grid_force_tile(idx) == 0 ? UOT_OK : UOT_EINVAL; }

int uot_grid_tile_count(void) { return grid_tile_count(); }

uot_status uot_selftest_bounded_wait(double seconds, void* stream) {
  clear_stale_error();
  if (!(seconds > 0.0) || seconds > 10.0) return UOT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  sc.reserve<unsigned>(1);
  sc.reserve<int>(1);
  UOT_CK(sc.allocate());
  unsigned* flag = sc.take<unsigned>(1);
  int* status = sc.take<int>(1);
  UOT_SCRATCH_OK(sc);
  UOT_CK(cudaMemsetAsync(flag, 0, sizeof(unsigned), s));
  UOT_CK(cudaMemsetAsync(status, 0, sizeof(int), s));
  UOT_CK(launch_wait_selftest(flag, (unsigned long long)(seconds * 1e9), status, s));
  int h = 0;
  UOT_CK(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  UOT_CK(cudaStreamSynchronize(s));
  if (h) {
    g_last_error = "bounded device wait expired (self-test: the flag is never set)";
    return UOT_TIMEOUT;
  }
  return UOT_OK;
}

uot_status uot_force_batch_warps(int warps) { return batch_force_warps(warps) == 0 ? UOT_OK : UOT_EINVAL; }

int uot_autotune_table(char* buf, int len) {
  const std::string t = grid_tile_table() + batch_tune_table();
  if (buf && len > 0) {
    const size_t n = std::min((size_t)(len - 1), t.size());
    memcpy(buf, t.data(), n);
    buf[n] = 0;
  }
  return (int)t.size();
}

void uot_profile_begin(void) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  for (auto& v : g_prof.marks) {
    for (auto& pr : v) {
      g_prof.pool.push_back(pr.first);
      g_prof.pool.push_back(pr.second);
    }
    v.clear();
  }
  g_prof.on = true;
}

uot_status uot_profile_end(int family, double* total_ms, long long* launches) {
  if (family < 0 || family >= PROF_NFAM || !total_ms || !launches) return UOT_EINVAL;
  std::lock_guard<std::mutex> lk(g_prof.mu);
  g_prof.on = false;
  double tot = 0.0;
  for (auto& pr : g_prof.marks[family]) {
    cudaError_t e = cudaEventSynchronize(pr.second);
    if (e != cudaSuccess) return fail_cuda(e);
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, pr.first, pr.second);
    if (e != cudaSuccess) return fail_cuda(e);
    tot += ms;
  }
  *total_ms = tot;
  *launches = (long long)g_prof.marks[family].size();
  return UOT_OK;
}

uot_status uot_solve(const uot_geom* g, const void* p, const void* dx, const void* q,
                     const void* dy, const uot_div* F1, const uot_div* F2, const uot_opts* o,
                     void* U, void* V, uot_result* res, void* stream) {
  clear_stale_error();
  return solve_impl(g, 1, p, dx, q, dy, F1, F2, o, U, V, res, (cudaStream_t)stream);
}

uot_status uot_solve_mass(const uot_geom* g, const void* p, const void* dx, const void* q,
                          const void* dy, const uot_div* F1, const uot_div* F2, const uot_div* F3,
                          double m0, const uot_opts* o, void* U, void* V, double* Z, uot_result* res,
                          void* stream) {
  clear_stale_error();
  return solve_mass_impl(g, p, dx, q, dy, F1, F2, F3, m0, o, U, V, Z, res, (cudaStream_t)stream);
}

uot_status uot_wf_cost(const void* x, int n, const void* y, int m, int d, double cut, int precision,
                       void* C, void* stream) {
  clear_stale_error();
  if (!x || !y || !C || n < 1 || m < 1 || d < 1 || d > 8 || !(cut > 0.0) || !isfinite(cut) ||
      (precision != UOT_F64 && precision != UOT_F32))
    return UOT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t total = (int64_t)n * m;
  const int grid = (int)std::min<int64_t>((total + kNT - 1) / kNT, 152 * 16);
  count_launches(1);
  if (precision == UOT_F64)
    k_wf_cost<double><<<grid, kNT, 0, s>>>((const double*)x, n, (const double*)y, m, d, cut, (double*)C);
  else
    k_wf_cost<float><<<grid, kNT, 0, s>>>((const float*)x, n, (const float*)y, m, d, cut, (float*)C);
  UOT_CK(cudaGetLastError());
  return UOT_OK;
}

uot_status uot_wf_flow(const uot_geom* g, int nspecies, const void* P0, const void* dx, double tau,
                       double alpha, double lambda, const uot_opts* o, int nsteps, void* P, void* U,
                       void* V, uot_result* res, void* stream) {
  clear_stale_error();
  return wf_flow_impl(g, nspecies, P0, dx, tau, alpha, lambda, o, nsteps, P, U, V, res, (cudaStream_t)stream);
}

uot_status uot_histogram(const float* pts, long long npts, int d, const int* shape, int precision, void* p,
                         void* stream) {
  clear_stale_error();
  BinGrid b;
  int64_t nb = 0;
  uot_status st = bin_grid(d, shape, b, nb);
  if (st != UOT_OK) return st;
  if (!pts || !p || npts < 1 || (precision != UOT_F64 && precision != UOT_F32)) return UOT_EINVAL;
  if (npts > 0xffffffffLL) return UOT_EINVAL;  // 32-bit counters
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  sc.reserve<unsigned>(nb);
  UOT_CK(sc.allocate());
  unsigned* counts = sc.take<unsigned>(nb);
  UOT_SCRATCH_OK(sc);
  UOT_CK(cudaMemsetAsync(counts, 0, nb * sizeof(unsigned), s));
  count_launches(2);
  k_histogram<<<nblocks(npts), kNT, 0, s>>>(pts, npts, b, counts);
  if (precision == UOT_F64)
    k_hist_norm<double><<<nblocks(nb), kNT, 0, s>>>(counts, nb, (double)npts, (double*)p);
  else
    k_hist_norm<float><<<nblocks(nb), kNT, 0, s>>>(counts, nb, (double)npts, (float*)p);
  UOT_CK(cudaGetLastError());
  return UOT_OK;
}

uot_status uot_barycentric_map(const uot_geom* g, const void* U, const void* V, double eps, const void* dx,
                               const void* dy, int precision, void* T, void* stream) {
  clear_stale_error();
  uot_status st = check_geom(g);
  if (st != UOT_OK) return st;
  if (!U || !V || !dx || !dy || !T || !(eps > 0.0) || (precision != UOT_F64 && precision != UOT_F32))
    return UOT_EINVAL;
  if (g->kind == UOT_GEOM_DENSE) return UOT_EUNSUPPORTED;
  const int d = (g->kind == UOT_GEOM_GRID) ? g->ndim : g->d;
  if (d + 1 > 64) return UOT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = g->n, m = g->m;
  const size_t esz = precision == UOT_F64 ? 8 : 4;
  PointsOf X, Y;
  memset(&X, 0, sizeof(X));
  memset(&Y, 0, sizeof(Y));
  X.kind = Y.kind = g->kind;
  X.d = Y.d = d;
  if (g->kind == UOT_GEOM_GRID) {
    for (int k = 0; k < d; ++k) {
      X.shape[k] = g->shape_x[k];
      X.axes[k] = g->axes_x[k];
      Y.shape[k] = g->shape_y[k];
      Y.axes[k] = g->axes_y[k];
    }
  } else {
    X.pts = g->x;
    Y.pts = g->y;
  }
  Scratch sc(s);
  sc.reserve<char>((size_t)m * (d + 1) * esz);
  sc.reserve<char>((size_t)n * (d + 1) * esz);
  UOT_CK(sc.allocate());
  char* F = sc.take<char>((size_t)m * (d + 1) * esz);
  char* RF = sc.take<char>((size_t)n * (d + 1) * esz);
  UOT_SCRATCH_OK(sc);
  count_launches(1);
  if (precision == UOT_F64)
    k_coords1<double><<<nblocks(m * (d + 1)), kNT, 0, s>>>(Y, m, (double*)F);
  else
    k_coords1<float><<<nblocks(m * (d + 1)), kNT, 0, s>>>(Y, m, (float*)F);
  UOT_CK(cudaGetLastError());
  // R (dy y) and R dy in one pass of d + 1 columns
  st = uot_apply_plan(g, U, V, eps, dx, dy, F, d + 1, 0, precision, RF, stream);
  if (st != UOT_OK) return st;
  count_launches(1);
  if (precision == UOT_F64)
    k_bary_divide<double><<<nblocks(n * d), kNT, 0, s>>>((const double*)RF, X, n, (double*)T);
  else
    k_bary_divide<float><<<nblocks(n * d), kNT, 0, s>>>((const float*)RF, X, n, (float*)T);
  UOT_CK(cudaGetLastError());
  return UOT_OK;
}

uot_status uot_apply_bin_map(const float* pts, long long npts, int d, const int* shape, const void* T,
                             int precision, float* out, void* stream) {
  clear_stale_error();
  BinGrid b;
  int64_t nb = 0;
  uot_status st = bin_grid(d, shape, b, nb);
  if (st != UOT_OK) return st;
  if (!pts || !T || !out || npts < 1 || (precision != UOT_F64 && precision != UOT_F32)) return UOT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  count_launches(1);
  if (precision == UOT_F64)
    k_apply_bin_map<double><<<nblocks(npts), kNT, 0, s>>>(pts, npts, b, (const double*)T, out);
  else
    k_apply_bin_map<float><<<nblocks(npts), kNT, 0, s>>>(pts, npts, b, (const float*)T, out);
  UOT_CK(cudaGetLastError());
  return UOT_OK;
}

uot_status uot_solve_many(const uot_geom* g, int batch, const void* p, const void* dx,
                          const void* q, const void* dy, const uot_div* F1, const uot_div* F2,
                          const uot_opts* o, void* U, void* V, uot_result* res, void* stream) {
  clear_stale_error();
  return solve_impl(g, batch, p, dx, q, dy, F1, F2, o, U, V, res, (cudaStream_t)stream);
}

uot_status uot_gibbs_log(const uot_geom* g, const void* W, const void* w, double eps,
                         int transpose, int precision, void* out, void* stream) {
  clear_stale_error();
  uot_status st = check_geom(g);
  if (st != UOT_OK) return st;
  if (!W || !w || !out || !(eps > 0.0) || !prec_ok(precision)) return UOT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nin = transpose ? g->n : g->m, nout = transpose ? g->m : g->n;
  Scratch sc(s);
  Gibbs G;
  G.g = *g;
  G.prec = precision;
  G.plan(sc, 1);
  sc.reserve<double>(nin);
  sc.reserve<double>(nin);
  sc.reserve<double>(nout);
  UOT_CK(sc.allocate());
  UOT_CK(G.take(sc, s));
  double* Wd = sc.take<double>(nin);
  double* logw = sc.take<double>(nin);
  double* od = sc.take<double>(nout);
  UOT_SCRATCH_OK(sc);
  UOT_CK(to_f64(precision, W, nin, Wd, s));
  UOT_CK(to_log(precision, w, nin, logw, s));
  Epilogue e;
  memset(&e, 0, sizeof(e));
  e.mode = EPI_SCALE;
  set_eps(e, eps);
  e.out = od;
  UOT_CK(G.apply(transpose ? 1 : 0, Wd, logw, eps, e, s));
  UOT_CK(from_f64(precision, od, nout, out, s));
  if (precision == UOT_MIXED && G.tc_err) {
    // the tensor-core pass's bounded waits report through this flag
    int htc = 0;
    UOT_CK(cudaMemcpyAsync(&htc, G.tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    UOT_CK(cudaStreamSynchronize(s));
    if (htc) {
      g_last_error = "uot_gibbs_log: a bounded wait of the tensor-core pass expired";
      return UOT_TIMEOUT;
    }
  }
  return UOT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// No-allocation variant of uot_gibbs_log.
//
// Some callers cannot allocate device memory at all: code running inside a
// CUDA stream capture that must not add allocation nodes, processes whose
// device memory is fully owned by another allocator, or real-time loops where
// an allocation can block.  For them the operator's scratch lives in one
// file-scope device array of fixed size that every GPU loading this library
// holds until the process exits.  In host code the array's name is only a
// host-side stand-in, so its device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernels.
// ---------------------------------------------------------------------------
namespace uot {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)UOT_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
char* g_noalloc_addr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device (set up on the
// first call per device).
cudaError_t noalloc_scratch(char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = (char*)p;
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace uot

extern "C" {

uot_status uot_gibbs_log_noalloc(const uot_geom* g, const void* W, const void* w, double eps,
                                 int transpose, int precision, void* out, void* stream) {
  clear_stale_error();
  // no tuning here: the tuner allocates its scratch inputs
  struct TuneHold {
    TuneHold() { grid_tune_hold(1); }
    ~TuneHold() { grid_tune_hold(0); }
  } hold;
  uot_status st = check_geom(g);
  if (st != UOT_OK) return st;
  if (!W || !w || !out || !(eps > 0.0) || !prec_ok(precision)) return UOT_EINVAL;
  if (g->kind == UOT_GEOM_DENSE) {
    g_last_error = "uot_gibbs_log_noalloc: dense cost matrices are not supported (grid and points only)";
    return UOT_EUNSUPPORTED;
  }
  if (precision == UOT_MIXED) {
    // its set-up copies the grid axes to the host and synchronises the stream
    g_last_error = "uot_gibbs_log_noalloc: UOT_MIXED is not supported (UOT_F64 and UOT_F32 only)";
    return UOT_EUNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  char* base = nullptr;
  UOT_CK(noalloc_scratch(&base));
  const int64_t nin = transpose ? g->n : g->m, nout = transpose ? g->m : g->n;
  Scratch sc(s, base, kNoAllocScratchBytes);
  Gibbs G;
  G.g = *g;
  G.prec = precision;
  G.host_setup = false;  // no read-back of the axes (it would synchronise the stream)
  G.plan(sc, 1);
  sc.reserve<double>(nin);
  sc.reserve<double>(nin);
  sc.reserve<double>(nout);
  if (sc.needed() > kNoAllocScratchBytes) {
    g_last_error = "uot_gibbs_log_noalloc: problem needs " + std::to_string(sc.needed()) +
                   " bytes of scratch, more than the fixed " +
                   std::to_string(kNoAllocScratchBytes) + " bytes (UOT_NOALLOC_SCRATCH_BYTES)";
    return UOT_EINVAL;
  }
  UOT_CK(sc.allocate());
  UOT_CK(G.take(sc, s));
  double* Wd = sc.take<double>(nin);
  double* logw = sc.take<double>(nin);
  double* od = sc.take<double>(nout);
  UOT_SCRATCH_OK(sc);
  // Every buffer carved here is fully written before it is read, so nothing
  // left by an earlier call needs clearing.
  UOT_CK(to_f64(precision, W, nin, Wd, s));
  UOT_CK(to_log(precision, w, nin, logw, s));
  Epilogue e;
  memset(&e, 0, sizeof(e));
  e.mode = EPI_SCALE;
  set_eps(e, eps);
  e.out = od;
  UOT_CK(G.apply(transpose ? 1 : 0, Wd, logw, eps, e, s));
  UOT_CK(from_f64(precision, od, nout, out, s));
  return UOT_OK;
}

uot_status uot_apply_plan(const uot_geom* g, const void* U, const void* V, double eps,
                          const void* dx, const void* dy, const void* f, int ncols,
                          int transpose, int precision, void* out, void* stream) {
  clear_stale_error();
  uot_status st = check_geom(g);
  if (st != UOT_OK) return st;
  if (!U || !V || !dx || !dy || !out || !(eps > 0.0) || !prec_ok(precision)) return UOT_EINVAL;
  if (ncols < 1 || ncols > 64) return UOT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = g->n, m = g->m;
  const int64_t nin = transpose ? n : m, nout = transpose ? m : n;
  Scratch sc(s);
  Gibbs G;
  G.g = *g;
  G.prec = precision;
  G.plan(sc, 1);
  for (int k = 0; k < 3; ++k) sc.reserve<double>(nin);
  sc.reserve<double>(nout);
  sc.reserve<double>(nout * ncols);
  UOT_CK(sc.allocate());
  UOT_CK(G.take(sc, s));
  double* Win = sc.take<double>(nin);
  double* W = sc.take<double>(nin);
  double* logw = sc.take<double>(nin);
  double* Sh = sc.take<double>(nout);
  double* od = sc.take<double>(nout * ncols);
  UOT_SCRATCH_OK(sc);
  UOT_CK(to_f64(precision, transpose ? U : V, nin, Win, s));
  UOT_CK(to_f64(precision, transpose ? V : U, nout, Sh, s));
  UOT_CK(to_log(precision, transpose ? dx : dy, nin, logw, s));
  for (int c = 0; c < ncols; ++c) {
    count_launches(1);
    if (precision == UOT_F64)
      k_add_logf<double><<<nblocks(nin), kNT, 0, s>>>(Win, (const double*)f, ncols, c, nin, eps, W);
    else
      k_add_logf_ff<<<nblocks(nin), kNT, 0, s>>>(Win, (const float*)f, ncols, c, nin, eps, W);
    UOT_CK(cudaGetLastError());
    Epilogue e;
    memset(&e, 0, sizeof(e));
    e.mode = EPI_PLAN;
    set_eps(e, eps);
    e.out = od;
    e.pot_shift = Sh;
    e.ncols = ncols;
    e.col = c;
    UOT_CK(G.apply(transpose ? 1 : 0, W, logw, eps, e, s));
  }
  UOT_CK(from_f64(precision, od, nout * ncols, out, s));
  return UOT_OK;
}

uot_status uot_objective(const uot_geom* g, const void* p, const void* dx, const void* q,
                         const void* dy, const uot_div* F1, const uot_div* F2, double eps,
                         const void* U, const void* V, int precision, double* out, void* stream) {
  clear_stale_error();
  uot_status st = check_geom(g);
  if (st != UOT_OK) return st;
  if (!p || !dx || !q || !dy || !U || !V || !out || !(eps > 0.0) || !prec_ok(precision) ||
      !div_ok(F1) || !div_ok(F2))
    return UOT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = g->n, m = g->m;
  Scratch sc(s);
  Gibbs G;
  G.g = *g;
  G.prec = precision;
  G.plan(sc, 1);
  for (int k = 0; k < 6; ++k) sc.reserve<double>(n);  // Ud logp logdx r1 zK1 S1
  for (int k = 0; k < 4; ++k) sc.reserve<double>(m);  // Vd logq logdy r2
  sc.reserve<double>(n > m ? n : m);                  // zero
  sc.reserve<double>(16);                             // acc
  UOT_CK(sc.allocate());
  UOT_CK(G.take(sc, s));
  double* Ud = sc.take<double>(n);
  double* Vd = sc.take<double>(m);
  double* logp = sc.take<double>(n);
  double* logq = sc.take<double>(m);
  double* logdx = sc.take<double>(n);
  double* logdy = sc.take<double>(m);
  double* r1 = sc.take<double>(n);
  double* r2 = sc.take<double>(m);
  double* zK1 = sc.take<double>(n);
  double* S1 = sc.take<double>(n);
  double* zero = sc.take<double>(n > m ? n : m);
  double* acc = sc.take<double>(16);
  UOT_SCRATCH_OK(sc);
  UOT_CK(to_f64(precision, U, n, Ud, s));
  UOT_CK(to_f64(precision, V, m, Vd, s));
  UOT_CK(to_log(precision, p, n, logp, s));
  UOT_CK(to_log(precision, q, m, logq, s));
  UOT_CK(to_log(precision, dx, n, logdx, s));
  UOT_CK(to_log(precision, dy, m, logdy, s));
  count_launches(1);
  k_fill<<<nblocks(n > m ? n : m), kNT, 0, s>>>(zero, n > m ? n : m, 0.0);
  UOT_CK(cudaMemsetAsync(acc, 0, 16 * 8, s));
  Epilogue e;
  memset(&e, 0, sizeof(e));
  set_eps(e, eps);
  // r1 = R dy, r2 = R^T dx
  e.mode = EPI_PLAN;
  e.ncols = 1;
  e.out = r1;
  e.pot_shift = Ud;
  UOT_CK(G.apply(0, Vd, logdy, eps, e, s));
  e.out = r2;
  e.pot_shift = Vd;
  UOT_CK(G.apply(1, Ud, logdx, eps, e, s));
  // z_i = log sum_j K_ij dy_j  (for sum dx dy K) and S = eps log K(b.dy)
  e.mode = EPI_RAW;
  e.out = zK1;
  UOT_CK(G.apply(0, zero, logdy, eps, e, s));
  e.mode = EPI_SCALE;
  e.out = S1;
  UOT_CK(G.apply(0, Vd, logdy, eps, e, s));
  const DivParams D1 = make_div(*F1), D2 = make_div(*F2);
  if (precision != UOT_F64) {
    double* arrs_n[] = {Ud, logp, logdx, r1, zK1, S1};
    double* arrs_m[] = {Vd, logq, logdy, r2};
    for (double* a : arrs_n) {
      count_launches(1);
      k_ff_to_double<<<nblocks(n), kNT, 0, s>>>(a, n);
    }
    for (double* a : arrs_m) {
      count_launches(1);
      k_ff_to_double<<<nblocks(m), kNT, 0, s>>>(a, m);
    }
    UOT_CK(cudaGetLastError());
  }
  count_launches(1);
  k_objective_side<<<nblocks(n) > 1024 ? 1024 : nblocks(n), kNT, 0, s>>>(r1, Ud, logp, logdx, zK1, S1, D1, eps, n, acc);
  count_launches(1);
  k_objective_side<<<nblocks(m) > 1024 ? 1024 : nblocks(m), kNT, 0, s>>>(r2, Vd, logq, logdy, nullptr, nullptr, D2, eps, m, acc + 8);
  UOT_CK(cudaGetLastError());
  double h[16];
  UOT_CK(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
  UOT_CK(cudaStreamSynchronize(s));
  // eps sum dx dy (R - K) = eps (sum dx r1 - sum dx dy K)
  const double mass_term = eps * (h[3] - h[4]);
  const double primal = h[0] + h[8] + h[2] + h[10] - mass_term;
  const double dual = -h[1] - h[9] - mass_term;
  out[0] = primal;
  out[1] = dual;
  out[2] = (h[0] + h[1] + h[2]) + (h[8] + h[9] + h[10]);
  out[3] = (h[6] > 0.0) ? h[5] / h[6] : 0.0;
  return UOT_OK;
}

uot_status uot_solve_batch(int nprob, const uot_batch_problem* probs, int d, const void* x,
                           const void* p, const void* dx, const void* y, const void* q,
                           const void* dy, const uot_opts* o, void* Uout, void* Vout, int* iters,
                           double* errs, uot_result* res, void* stream) {
  clear_stale_error();
  uot_status st = check_opts(o, false, true);
  if (st != UOT_OK) return st;
  if (nprob < 1 || !probs || d < 1 || d > 3 || !x || !p || !dx || !y || !q || !dy || !Uout || !Vout)
    return UOT_EINVAL;
  if (o->precision != UOT_F32 || o->plain_scaling || o->U0 || o->V0) return UOT_EUNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int> hn(nprob), hm(nprob), order(nprob);
  std::vector<int64_t> hxo(nprob), hyo(nprob);
  int64_t N = 0, M = 0;
  int nmax = 0, mmax = 0;
  for (int k = 0; k < nprob; ++k) {
    const uot_batch_problem& pr = probs[k];
    if (pr.n < 1 || pr.m < 1 || pr.n > 3072 || pr.m > 3072) return UOT_EINVAL;
    if (!div_ok(&pr.F1) || !div_ok(&pr.F2)) return UOT_EINVAL;
    if (o->translate && (pr.F1.kind != UOT_DIV_KL || pr.F2.kind != UOT_DIV_KL)) return UOT_EUNSUPPORTED;
    hn[k] = pr.n;
    hm[k] = pr.m;
    hxo[k] = N;
    hyo[k] = M;
    N += pr.n;
    M += pr.m;
    nmax = pr.n > nmax ? pr.n : nmax;
    mmax = pr.m > mmax ? pr.m : mmax;
    order[k] = k;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (int64_t)hn[a] * hm[a] > (int64_t)hn[b] * hm[b];
  });
  const std::vector<Stage> stages = eps_schedule(*o);
  const int nstage = (int)stages.size();
  std::vector<double> eps_list;
  for (const Stage& sg : stages) eps_list.push_back(sg.eps);
  eps_list.push_back(o->eps);
  std::vector<DivFF> divs((size_t)(nstage + 1) * nprob * 2);
  std::vector<float2> heps(nstage + 1), hieps(nstage + 1);
  std::vector<float> hk2(nstage + 1);
  for (int sidx = 0; sidx <= nstage; ++sidx) {
    const double e = eps_list[sidx];
    heps[sidx] = ff2(ff_make(e));
    hieps[sidx] = ff2(ff_make(1.0 / e));
    hk2[sidx] = (float)((double)kLog2e / e);
    for (int k = 0; k < nprob; ++k) {
      divs[((size_t)sidx * nprob + k) * 2] = make_div_ff(make_div(probs[k].F1), e);
      divs[((size_t)sidx * nprob + k) * 2 + 1] = make_div_ff(make_div(probs[k].F2), e);
    }
  }
  int dev = 0, sms = 0;
  UOT_CK(cudaGetDevice(&dev));
  UOT_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  UOT_CK(cudaEventCreate(&ev0));
  UOT_CK(cudaEventCreate(&ev1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } evg{ev0, ev1};
  UOT_CK(cudaEventRecord(ev0, s));

  Scratch sc(s);
  sc.reserve<int>(nprob);      // order
  sc.reserve<int>(nprob);      // n
  sc.reserve<int>(nprob);      // m
  sc.reserve<int64_t>(nprob);  // xoff
  sc.reserve<int64_t>(nprob);  // yoff
  sc.reserve<DivFF>(divs.size());
  sc.reserve<float2>(nstage + 1);
  sc.reserve<float2>(nstage + 1);
  sc.reserve<float>(nstage + 1);
  sc.reserve<double>(N);  // logp
  sc.reserve<double>(N);  // logdx
  sc.reserve<double>(M);  // logq
  sc.reserve<double>(M);  // logdy
  sc.reserve<int>(nprob);    // iters
  sc.reserve<float>(nprob);  // errs
  sc.reserve<int>(1);        // work counter
  sc.reserve<float2>(N);     // U state (float-float)
  sc.reserve<float2>(M);     // V state
  sc.reserve<float>(N);      // U-side shifts
  sc.reserve<float>(M);      // V-side shifts
  if (o->translate) sc.reserve<double2>(nprob);  // (lambda1, lambda2)
  UOT_CK(sc.allocate());
  int* d_order = sc.take<int>(nprob);
  int* d_n = sc.take<int>(nprob);
  int* d_m = sc.take<int>(nprob);
  int64_t* d_xo = sc.take<int64_t>(nprob);
  int64_t* d_yo = sc.take<int64_t>(nprob);
  DivFF* d_divs = sc.take<DivFF>(divs.size());
  float2* d_eps = sc.take<float2>(nstage + 1);
  float2* d_ieps = sc.take<float2>(nstage + 1);
  float* d_k2 = sc.take<float>(nstage + 1);
  double* d_logp = sc.take<double>(N);
  double* d_logdx = sc.take<double>(N);
  double* d_logq = sc.take<double>(M);
  double* d_logdy = sc.take<double>(M);
  int* d_iters = sc.take<int>(nprob);
  float* d_errs = sc.take<float>(nprob);
  int* d_next = sc.take<int>(1);
  float2* d_Uff = sc.take<float2>(N);
  float2* d_Vff = sc.take<float2>(M);
  float* d_zU = sc.take<float>(N);
  float* d_zV = sc.take<float>(M);
  double2* d_lam = o->translate ? sc.take<double2>(nprob) : nullptr;
  UOT_SCRATCH_OK(sc);
  if (o->translate) {
    std::vector<double2> hl(nprob);
    for (int k = 0; k < nprob; ++k) hl[k] = make_double2(probs[k].F1.lambda, probs[k].F2.lambda);
    UOT_CK(cudaMemcpyAsync(d_lam, hl.data(), nprob * sizeof(double2), cudaMemcpyHostToDevice, s));
  }
  UOT_CK(cudaMemcpyAsync(d_order, order.data(), nprob * sizeof(int), cudaMemcpyHostToDevice, s));
  UOT_CK(cudaMemcpyAsync(d_n, hn.data(), nprob * sizeof(int), cudaMemcpyHostToDevice, s));
  UOT_CK(cudaMemcpyAsync(d_m, hm.data(), nprob * sizeof(int), cudaMemcpyHostToDevice, s));
  UOT_CK(cudaMemcpyAsync(d_xo, hxo.data(), nprob * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  UOT_CK(cudaMemcpyAsync(d_yo, hyo.data(), nprob * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  UOT_CK(cudaMemcpyAsync(d_divs, divs.data(), divs.size() * sizeof(DivFF), cudaMemcpyHostToDevice, s));
  UOT_CK(cudaMemcpyAsync(d_eps, heps.data(), heps.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
  UOT_CK(cudaMemcpyAsync(d_ieps, hieps.data(), hieps.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
  UOT_CK(cudaMemcpyAsync(d_k2, hk2.data(), hk2.size() * sizeof(float), cudaMemcpyHostToDevice, s));
  UOT_CK(cudaMemsetAsync(d_next, 0, sizeof(int), s));
  UOT_CK(to_log(UOT_F32, p, N, d_logp, s));
  UOT_CK(to_log(UOT_F32, dx, N, d_logdx, s));
  UOT_CK(to_log(UOT_F32, q, M, d_logq, s));
  UOT_CK(to_log(UOT_F32, dy, M, d_logdy, s));
  BatchArgs a;
  a.nprob = nprob;
  a.d = d;
  a.nstage = nstage;
  a.iters_per_stage = o->iters_per_stage;
  a.max_iter = o->max_iter;
  a.check_every = o->check_every > 0 ? o->check_every : 1;
  a.nmax = nmax;
  a.mmax = mmax;
  a.ndiv = nprob;
  a.tol = (float)o->tol;
  a.order = d_order;
  a.n = d_n;
  a.m = d_m;
  a.xoff = d_xo;
  a.yoff = d_yo;
  a.x = (const float*)x;
  a.y = (const float*)y;
  a.logp = reinterpret_cast<const float2*>(d_logp);
  a.logdx = reinterpret_cast<const float2*>(d_logdx);
  a.logq = reinterpret_cast<const float2*>(d_logq);
  a.logdy = reinterpret_cast<const float2*>(d_logdy);
  a.divs = d_divs;
  a.eps_ff = d_eps;
  a.inv_eps_ff = d_ieps;
  a.k2 = d_k2;
  a.Uout = (float*)Uout;
  a.Vout = (float*)Vout;
  a.iters_out = d_iters;
  a.err_out = d_errs;
  a.next = d_next;
  a.Uff = d_Uff;
  a.Vff = d_Vff;
  a.zU = d_zU;
  a.zV = d_zV;
  a.translate = o->translate;
  a.lam = d_lam;
  const int variant = batch_pick_variant(a, order.data(), s);
  const int per_sm = batch_ctas_per_sm(d, variant, nmax, mmax);
  if (per_sm < 1) {
    g_last_error = "uot_solve_batch: problem sizes do not fit in shared memory";
    return UOT_EUNSUPPORTED;
  }
  UOT_CK(cudaMemsetAsync(d_next, 0, sizeof(int), s));
  const int grid = (int)std::min<int64_t>(nprob, (int64_t)sms * per_sm);
  UOT_CK(launch_batch(a, variant, grid, s));
  UOT_CK(cudaEventRecord(ev1, s));
  std::vector<int> it_h(nprob);
  std::vector<float> er_h(nprob);
  UOT_CK(cudaMemcpyAsync(it_h.data(), d_iters, nprob * sizeof(int), cudaMemcpyDeviceToHost, s));
  UOT_CK(cudaMemcpyAsync(er_h.data(), d_errs, nprob * sizeof(float), cudaMemcpyDeviceToHost, s));
  UOT_CK(cudaStreamSynchronize(s));
  float ms = 0.f;
  UOT_CK(cudaEventElapsedTime(&ms, ev0, ev1));
  bool all_conv = true;
  int total = 0;
  double worst = 0.0;
  for (int k = 0; k < nprob; ++k) {
    if (iters) iters[k] = it_h[k];
    if (errs) errs[k] = er_h[k];
    total += it_h[k];
    worst = std::max(worst, (double)er_h[k]);
    if (o->tol > 0.0 && !(er_h[k] <= o->tol)) all_conv = false;
  }
  const uot_status out = all_conv ? UOT_OK : UOT_NOT_CONVERGED;
  if (res) {
    *res = empty_result();
    res->iters = total;
    res->total_iters = total + nprob * nstage * o->iters_per_stage;
    res->marg_err = worst;
    res->ms = ms;
    res->status = out;
  }
  return out;
}

static uot_status barycenter_impl(const uot_geom* g, int Kmeas, const double* alpha, const void* P,
                                  const void* dx, const void* dy, const uot_div* F1, double lambda,
                                  int bary_kind, double beta1, double beta2, const uot_opts* o, void* logh_out,
                                  void* Uout, void* Vout, uot_result* res, void* stream);

uot_status uot_barycenter(const uot_geom* g, int Kmeas, const double* alpha, const void* P,
                          const void* dx, const void* dy, const uot_div* F1, double lambda,
                          int bary_kind, const uot_opts* o, void* logh_out, void* Uout,
                          void* Vout, uot_result* res, void* stream) {
  clear_stale_error();
  if (bary_kind == UOT_BARY_RG) return UOT_EINVAL;  // its range needs uot_barycenter_div
  return barycenter_impl(g, Kmeas, alpha, P, dx, dy, F1, lambda, bary_kind, 1.0, 1.0, o, logh_out, Uout, Vout,
                         res, stream);
}

uot_status uot_barycenter_div(const uot_geom* g, int Kmeas, const double* alpha, const void* P,
                              const void* dx, const void* dy, const uot_div* F1, const uot_div* Fh,
                              const uot_opts* o, void* logh_out, void* Uout, void* Vout, uot_result* res,
                              void* stream) {
  clear_stale_error();
  if (!Fh) return UOT_EINVAL;
  switch (Fh->kind) {
    case UOT_DIV_EQ:
      return barycenter_impl(g, Kmeas, alpha, P, dx, dy, F1, 1.0, UOT_BARY_EQ, 1.0, 1.0, o, logh_out, Uout, Vout,
                             res, stream);
    case UOT_DIV_KL:
      return barycenter_impl(g, Kmeas, alpha, P, dx, dy, F1, Fh->lambda, UOT_BARY_KL, 1.0, 1.0, o, logh_out, Uout,
                             Vout, res, stream);
    case UOT_DIV_TV:
      return barycenter_impl(g, Kmeas, alpha, P, dx, dy, F1, Fh->lambda, UOT_BARY_TV, 1.0, 1.0, o, logh_out, Uout,
                             Vout, res, stream);
    case UOT_DIV_RG:
      return barycenter_impl(g, Kmeas, alpha, P, dx, dy, F1, 1.0, UOT_BARY_RG, Fh->alpha, Fh->beta, o, logh_out,
                             Uout, Vout, res, stream);
    default:
      return UOT_EINVAL;
  }
}

}  // extern "C"

static uot_status barycenter_impl(const uot_geom* g, int Kmeas, const double* alpha, const void* P,
                                  const void* dx, const void* dy, const uot_div* F1, double lambda,
                                  int bary_kind, double beta1, double beta2, const uot_opts* o, void* logh_out,
                                  void* Uout, void* Vout, uot_result* res, void* stream) {
  uot_status st = check_geom(g);
  if (st != UOT_OK) return st;
  if ((st = check_opts(o)) != UOT_OK) return st;
  if (Kmeas < 1 || !alpha || !P || !dx || !dy || !div_ok(F1) || !logh_out || !Uout || !Vout)
    return UOT_EINVAL;
  if (bary_kind != UOT_BARY_KL && bary_kind != UOT_BARY_EQ && bary_kind != UOT_BARY_TV && bary_kind != UOT_BARY_RG)
    return UOT_EINVAL;
  if ((bary_kind == UOT_BARY_KL || bary_kind == UOT_BARY_TV) && !(lambda > 0.0)) return UOT_EINVAL;
  if (bary_kind == UOT_BARY_RG && !(beta1 > 0.0 && beta1 <= beta2 && beta2 < kInf)) return UOT_EINVAL;
  if ((bary_kind == UOT_BARY_TV || bary_kind == UOT_BARY_RG) && Kmeas > 1024) return UOT_EINVAL;
  if (o->plain_scaling) return UOT_EUNSUPPORTED;
  double sum_alpha = 0.0;
  for (int k = 0; k < Kmeas; ++k) {
    if (!(alpha[k] > 0.0) || !isfinite(alpha[k])) return UOT_EINVAL;
    sum_alpha += alpha[k];
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int prec = o->precision;
  const int64_t n = g->n, m = g->m;
  const DivParams D1 = make_div(*F1);

  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  UOT_CK(cudaEventCreate(&ev0));
  UOT_CK(cudaEventCreate(&ev1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } evg{ev0, ev1};
  UOT_CK(cudaEventRecord(ev0, s));

  Scratch sc(s);
  Gibbs G;
  G.g = *g;
  G.prec = prec;
  G.speculate = true;
  G.plan(sc, Kmeas);
  sc.reserve<double>(n * Kmeas);  // logP
  sc.reserve<double>(n * Kmeas);  // U
  sc.reserve<double>(n);          // logdx
  sc.reserve<double>(m * Kmeas);  // V
  sc.reserve<double>(m * Kmeas);  // T
  sc.reserve<double>(m);          // logdy
  sc.reserve<double>(m);          // logh
  sc.reserve<double>(Kmeas);      // alpha
  sc.reserve<float>(Kmeas);       // log alpha (FP32 path)
  sc.reserve<double>(2 * (size_t)Kmeas);  // violation accumulators per measure
  UOT_CK(sc.allocate());
  UOT_CK(G.take(sc, s));
  double* logP = sc.take<double>(n * Kmeas);
  double* U = sc.take<double>(n * Kmeas);
  double* logdx = sc.take<double>(n);
  double* V = sc.take<double>(m * Kmeas);
  double* T = sc.take<double>(m * Kmeas);
  double* logdy = sc.take<double>(m);
  double* logh = sc.take<double>(m);
  double* alpha_d = sc.take<double>(Kmeas);
  float* log_alpha_d = sc.take<float>(Kmeas);
  double* acc = sc.take<double>(2 * (size_t)Kmeas);
  std::vector<double> acc_h(2 * (size_t)Kmeas);
  UOT_SCRATCH_OK(sc);
  UOT_CK(to_log(prec, P, n * Kmeas, logP, s));
  UOT_CK(to_log(prec, dx, n, logdx, s));
  UOT_CK(to_log(prec, dy, m, logdy, s));
  UOT_CK(cudaMemcpyAsync(alpha_d, alpha, Kmeas * 8, cudaMemcpyHostToDevice, s));
  std::vector<float> log_alpha_h(Kmeas);
  for (int k = 0; k < Kmeas; ++k) log_alpha_h[k] = (float)log(alpha[k]);
  UOT_CK(cudaMemcpyAsync(log_alpha_d, log_alpha_h.data(), Kmeas * 4, cudaMemcpyHostToDevice, s));
  // pageable source: make sure the copy has consumed it before the vector dies
  UOT_CK(cudaStreamSynchronize(s));
  count_launches(1);
  k_fill<<<nblocks(n * Kmeas), kNT, 0, s>>>(U, n * Kmeas, 0.0);
  count_launches(1);
  k_fill<<<nblocks(m * Kmeas), kNT, 0, s>>>(V, m * Kmeas, 0.0);
  UOT_CK(cudaGetLastError());

  auto iteration = [&](double eps, bool check, cudaStream_t st) -> cudaError_t {
    cudaError_t e;
    Epilogue e1 = prox_epilogue(D1, logP, U, logdx, check ? acc : nullptr, eps);
    e1.bstride = n;
    e1.bstride_p = n;
    if ((e = G.apply(0, V, logdy, eps, e1, st, check ? acc : nullptr)) != cudaSuccess) return e;
    Epilogue e2;
    memset(&e2, 0, sizeof(e2));
    e2.mode = EPI_SCALE;
    set_eps(e2, eps);
    e2.out = T;
    e2.bstride = m;
    count_launches(1);
    if ((e = G.apply(1, U, logdx, eps, e2, st)) != cudaSuccess) return e;
    if (prec == UOT_F64) {
      k_bary_update<<<nblocks(m), kNT, 0, st>>>(T, Kmeas, m, alpha_d, sum_alpha, lambda, eps,
                                                bary_kind, beta1, beta2, logh, V);
    } else {
      DivParams Dh;
      Dh.kind = (bary_kind == UOT_BARY_KL) ? UOT_DIV_KL : (bary_kind == UOT_BARY_TV) ? UOT_DIV_TV
                : (bary_kind == UOT_BARY_RG) ? UOT_DIV_RG : UOT_DIV_EQ;
      Dh.lam = lambda;
      Dh.log_alpha = (bary_kind == UOT_BARY_RG) ? log(beta1) : 0.0;
      Dh.log_beta = (bary_kind == UOT_BARY_RG) ? log(beta2) : 0.0;
      BaryPL pl;
      pl.lam = (float)lambda;
      pl.b1 = (float)beta1;
      pl.b2 = (float)beta2;
      pl.elb1 = (float)(eps * log(beta1));
      pl.elb2 = (float)(eps * log(beta2));
      cudaLaunchConfig_t cfg;
      memset(&cfg, 0, sizeof(cfg));
      cfg.gridDim = dim3((unsigned)std::min<int64_t>((m + kBJ - 1) / kBJ, 1 << 20));
      cfg.blockDim = dim3(kBJ, kBK);
      cfg.stream = st;
      // a plain (fully serialised) launch: measured faster here than a
      // programmatic dependent launch, whose early-launched successor CTAs
      // compete with this small grid
      cfg.attrs = nullptr;
      cfg.numAttrs = 0;
      const bool pwl = bary_kind == UOT_BARY_TV || bary_kind == UOT_BARY_RG;
      cfg.dynamicSmemBytes = pwl ? (size_t)Kmeas * (kBJ + 1) * sizeof(float) : 0;
      if (cfg.dynamicSmemBytes > 48 * 1024) {
        e = cudaFuncSetAttribute(k_bary_update_ff, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)cfg.dynamicSmemBytes);
        if (e != cudaSuccess) return e;
      }
      const double lam_kl = (bary_kind == UOT_BARY_KL) ? lambda : 1.0;
      e = cudaLaunchKernelEx(&cfg, k_bary_update_ff, (const double*)T, Kmeas, (int64_t)m, (const float*)log_alpha_d,
                             (float)log(sum_alpha), ff2(ff_make(eps + lam_kl)), ff2(ff_make(1.0 / (eps + lam_kl))),
                             ff2(ff_make(1.0 / eps)), ff2(ff_make(eps)), bary_kind, make_div_ff(Dh, eps), pl, logh, V);
      if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
  };
  const std::vector<Stage> stages = eps_schedule(*o);
  const int check_every = o->check_every > 0 ? o->check_every : 1;
  int it = 0, total = 0;
  double err = INFINITY;
  bool converged = false;
  for (const Stage& sg : stages)
    for (int k = 0; k < sg.iters; ++k, ++total) UOT_CK(iteration(sg.eps, false, s));
  // launch_mode 2: checked blocks of check_every iterations replayed from a CUDA graph
  BlockGraph bg;
  bool graph_ok = o->launch_mode == 2 && !profiling_on();
  while (it < o->max_iter) {
    bool check;
    if (graph_ok && it > 0 && it % check_every == 0 && it + check_every <= o->max_iter) {
      if (!bg.exec) {
        cudaError_t e = bg.capture([&](cudaStream_t cs) -> cudaError_t {
          for (int k = 0; k < check_every; ++k) {
            cudaError_t e2 = iteration(o->eps, k == check_every - 1, cs);
            if (e2 != cudaSuccess) return e2;
          }
          return cudaSuccess;
        });
        if (e != cudaSuccess) {
          graph_ok = false;
          (void)cudaGetLastError();
          continue;
        }
      }
      UOT_CK(bg.launch(s));
      it += check_every;
      total += check_every;
      check = true;
    } else {
      check = ((it + 1) % check_every == 0) || (it == o->max_iter - 1);
      UOT_CK(iteration(o->eps, check, s));
      ++it;
      ++total;
    }
    if (check) {
      UOT_CK(cudaMemcpyAsync(acc_h.data(), acc, 16 * (size_t)Kmeas, cudaMemcpyDeviceToHost, s));
      UOT_CK(cudaStreamSynchronize(s));
      double h[2] = {0.0, 0.0};
      for (int k = 0; k < Kmeas; ++k) {
        h[0] += acc_h[2 * k];
        h[1] += acc_h[2 * k + 1];
      }
      err = (h[1] > 0.0) ? h[0] / h[1] : 0.0;
      if (it > 1 && o->tol > 0.0 && err <= o->tol) {
        converged = true;
        break;
      }
    }
  }
  UOT_CK(from_f64(prec, U, n * Kmeas, Uout, s));
  UOT_CK(from_f64(prec, V, m * Kmeas, Vout, s));
  UOT_CK(from_f64(prec, logh, m, logh_out, s));
  UOT_CK(cudaEventRecord(ev1, s));
  UOT_CK(cudaStreamSynchronize(s));
  float ms = 0.f;
  UOT_CK(cudaEventElapsedTime(&ms, ev0, ev1));
  uot_status out = (o->tol > 0.0 && !converged && o->max_iter > 0) ? UOT_NOT_CONVERGED : UOT_OK;
  if (res) {
    *res = empty_result();
    res->iters = it;
    res->total_iters = total;
    res->marg_err = err;
    res->ms = ms;
    res->status = out;
  }
  return out;
}

// Translation step for KL penalties on both sides (uot_opts.translate).
//
// Not one of the paper's algorithms: it is the translation step of the
// translation-invariant formulation of unbalanced Sinkhorn (Sejourne,
// Vialard, Peyre 2022), derived here from the dual of Theorem 3.2.  Adding c
// to U and subtracting it from V leaves U_i + V_j, hence the plan and the
// entropic term of the dual, unchanged; along that line only the conjugate
// terms lam1 <dx p, e^{-U/lam1}> and lam2 <dy q, e^{-V/lam2}> move, and the
// dual is maximal at
//   c = lam1 lam2 / (lam1 + lam2) (log A - log B),
//   A = sum_i dx_i p_i e^{-U_i/lam1},  B = sum_j dy_j q_j e^{-V_j/lam2}.
// The scaling iteration damps this direction only by (lam/(lam+eps))^2 per
// iteration, so for lam >> eps it is the slowest mode; one exact step removes
// it.  Entries with p_i = 0 (U_i = -inf) take no part; c = 0 when either
// measure is zero.
//
// Two launches per step: per-block partial log-sum-exps of both sides of
// every problem, then a shift kernel in which every block recombines its
// problem's partials (the same values in the same order, so every block
// applies the same c) and shifts its share of U and V.
#include <string.h>

#include <algorithm>

#include "uot_internal.cuh"

namespace uot {
namespace {

constexpr int kTrThreads = 256;
constexpr int kTrPartialPer = 2;   // elements per thread per block, partial kernel (before the cap)
constexpr int kTrShiftPer = 2;     // the same for the shift kernel
constexpr int kTrMaxBlocks = 256;  // blocks per problem and side: enough loads in flight to hide latency

int blocks_for(int64_t len, int per) {
  const int64_t b = (len + (int64_t)kTrThreads * per - 1) / ((int64_t)kTrThreads * per);
  return (int)std::max<int64_t>(1, std::min<int64_t>(kTrMaxBlocks, b));
}

// a value of the state: FP64, or float-float (hi, lo) in the same buffer
template <bool FF>
__device__ __forceinline__ double load_val(const double* a, int64_t i) {
  if constexpr (FF) {
    const float2 v = reinterpret_cast<const float2*>(a)[i];
    return (v.x == -INFINITY) ? -kInf : (double)v.x + (double)v.y;
  } else {
    return a[i];
  }
}

// running log-sum-exp (mx, s): sum = s e^{mx}, shifts in FP64; exponentials
// of the shifted differences in FP64 on the FP64 path, in FP32 on the
// float-float path (relative error ~1e-7 in the sum, below that path's
// rounding of the potentials)
template <bool FF>
__device__ __forceinline__ double ex(double d) {
  if constexpr (FF) return (double)expf((float)d);
  else return exp(d);
}
template <bool FF>
__device__ __forceinline__ void lse_push(double& mx, double& s, double t) {
  if (t > mx) {
    s = s * ex<FF>(mx - t) + 1.0;
    mx = t;
  } else {
    s += ex<FF>(t - mx);
  }
}
template <bool FF>
__device__ __forceinline__ void lse_merge(double& mx, double& s, double m2, double s2) {
  if (m2 > mx) {
    const double tm = mx, ts = s;
    mx = m2;
    s = s2;
    m2 = tm;
    s2 = ts;
  }
  if (m2 != -kInf) s += s2 * ex<FF>(m2 - mx);
}
template <bool FF>
__device__ __forceinline__ void lse_warp(double& mx, double& s) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double m2 = __shfl_down_sync(0xffffffffu, mx, o);
    const double s2 = __shfl_down_sync(0xffffffffu, s, o);
    lse_merge<FF>(mx, s, m2, s2);
  }
}

struct TrArgs {
  double* pot[2];           // U [batch][n], V [batch][m]
  const double* logm[2];    // log p, log q  ([batch][len])
  const double* logw[2];    // log dx, log dy ([len])
  int64_t len[2];
  int nblk[2];              // partial blocks per problem of each side
  int stride;               // partial entries per (side, problem) = max(nblk)
  double inv_lam[2];
  double w;                 // lam1 lam2 / (lam1 + lam2)
  double2* part;            // [2][batch][stride] (max, sum)
};

// grid (stride, batch, 2): block x of problem y, side z
template <bool FF>
__global__ void __launch_bounds__(kTrThreads) k_tr_partial(TrArgs a) {
  // programmatic dependent launch: wait for the V-update's last pass, then let
  // the shift kernel launch (it waits for this grid in turn)
  pdl_wait();
  pdl_launch_dependents();
  const int side = blockIdx.z;
  const int b = blockIdx.y;
  const int nb = a.nblk[side];
  if ((int)blockIdx.x >= nb) return;  // uniform per block
  const int64_t len = a.len[side];
  const double* pot = a.pot[side];
  const double inv_lam = a.inv_lam[side];
  double mx = -kInf, s = 0.0;
  if constexpr (FF) {
    // float-float terms and running maximum, FP32 sum: no FP64 pipe in the loop
    // (it runs at a small fraction of the FP32 rate); exponentials of the
    // exactly formed differences t - max, rounded to FP32
    const float2* lmf = reinterpret_cast<const float2*>(a.logm[side]) + (int64_t)b * len;
    const float2* uf = reinterpret_cast<const float2*>(pot) + (int64_t)b * len;
    const float2* lwf = reinterpret_cast<const float2*>(a.logw[side]);
    const ff nil = ff_make(-inv_lam);
    ff fmx = ff_ninf();
    float fs = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * kTrThreads + threadIdx.x; i < len; i += (int64_t)nb * kTrThreads) {
      const float2 lm = lmf[i], u = uf[i];
      if (lm.x == -INFINITY || u.x == -INFINITY) continue;
      const ff t = ff_add(ff_add(ffl(lwf[i]), ffl(lm)), ff_mul(ffl(u), nil));
      if (ff_lt(fmx, t)) {
        fs = (fmx.hi == -INFINITY) ? 1.0f : fs * expf(ff_sub(fmx, t).hi) + 1.0f;
        fmx = t;
      } else {
        fs += expf(ff_sub(t, fmx).hi);
      }
    }
    if (fmx.hi != -INFINITY) {
      mx = (double)fmx.hi + (double)fmx.lo;
      s = (double)fs;
    }
  } else {
    for (int64_t i = (int64_t)blockIdx.x * kTrThreads + threadIdx.x; i < len; i += (int64_t)nb * kTrThreads) {
      const double lm = load_val<FF>(a.logm[side], (int64_t)b * len + i);
      const double u = load_val<FF>(pot, (int64_t)b * len + i);
      if (lm == -kInf || u == -kInf) continue;
      lse_push<FF>(mx, s, load_val<FF>(a.logw[side], i) + lm - u * inv_lam);
    }
  }
  lse_warp<FF>(mx, s);
  __shared__ double sm[kTrThreads / 32], ss[kTrThreads / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sm[warp] = mx;
    ss[warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
    mx = (lane < kTrThreads / 32) ? sm[lane] : -kInf;
    s = (lane < kTrThreads / 32) ? ss[lane] : 0.0;
    lse_warp<FF>(mx, s);
    if (lane == 0) a.part[((int64_t)side * gridDim.y + b) * a.stride + blockIdx.x] = make_double2(mx, s);
  }
}

// grid (blocks, batch): c of problem y from its partials, then U += c, V -= c
template <bool FF>
__global__ void __launch_bounds__(kTrThreads) k_tr_shift(TrArgs a) {
  // waits for the partials; never releases its dependents early: the next pass
  // reads the old potentials before its own wait, and this grid rewrites them
  pdl_wait();
  const int b = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ double slog[2];
  __shared__ double sc;
  if (warp < 2) {
    const double2* pp = a.part + ((int64_t)warp * gridDim.y + b) * a.stride;
    double mx = -kInf, s = 0.0;
    for (int k = lane; k < a.nblk[warp]; k += 32) lse_merge<FF>(mx, s, pp[k].x, pp[k].y);
    lse_warp<FF>(mx, s);
    if (lane == 0) slog[warp] = (s > 0.0 && mx != -kInf) ? mx + log(s) : -kInf;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double la = slog[0], lb = slog[1];
    sc = (la != -kInf && lb != -kInf) ? a.w * (la - lb) : 0.0;
  }
  __syncthreads();
  const double c = sc;
  const int64_t n = a.len[0], m = a.len[1];
  const ff cp = ff_make(c), cn = ff_make(-c);
  for (int64_t i = (int64_t)blockIdx.x * kTrThreads + threadIdx.x; i < n + m;
       i += (int64_t)gridDim.x * kTrThreads) {
    const bool onU = i < n;
    const int64_t idx = onU ? (int64_t)b * n + i : (int64_t)b * m + (i - n);
    double* pot = a.pot[onU ? 0 : 1];
    if constexpr (FF) {
      float2* pf = reinterpret_cast<float2*>(pot);
      const float2 v = pf[idx];
      if (isinf(v.x) || v.x != v.x) continue;  // -inf stays -inf
      pf[idx] = ff2(ff_add(ffl(v), onU ? cp : cn));
    } else {
      pot[idx] += onU ? c : -c;
    }
  }
}

}  // namespace

size_t kl_translate_part_count(int64_t n, int64_t m, int batch) {
  const int stride = std::max(blocks_for(n, kTrPartialPer), blocks_for(m, kTrPartialPer));
  return (size_t)2 * (size_t)batch * (size_t)stride;
}

cudaError_t launch_kl_translate(double* U, double* V, const double* logp, const double* logq,
                                const double* logdx, const double* logdy, int64_t n, int64_t m, int batch,
                                int ff, double lam1, double lam2, double2* part, cudaStream_t s) {
  if (batch < 1 || batch > 65535 || n < 1 || m < 1 || !(lam1 > 0.0) || !(lam2 > 0.0) || !part)
    return cudaErrorInvalidValue;
  TrArgs a;
  a.pot[0] = U;
  a.pot[1] = V;
  a.logm[0] = logp;
  a.logm[1] = logq;
  a.logw[0] = logdx;
  a.logw[1] = logdy;
  a.len[0] = n;
  a.len[1] = m;
  a.nblk[0] = blocks_for(n, kTrPartialPer);
  a.nblk[1] = blocks_for(m, kTrPartialPer);
  a.stride = std::max(a.nblk[0], a.nblk[1]);
  a.inv_lam[0] = 1.0 / lam1;
  a.inv_lam[1] = 1.0 / lam2;
  a.w = lam1 * lam2 / (lam1 + lam2);
  a.part = part;
  const dim3 gp(a.stride, batch, 2);
  const dim3 gs(blocks_for(n + m, kTrShiftPer), batch);
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.blockDim = dim3(kTrThreads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launches(2);
  cudaError_t e;
  cfg.gridDim = gp;
  e = ff ? cudaLaunchKernelEx(&cfg, k_tr_partial<true>, a) : cudaLaunchKernelEx(&cfg, k_tr_partial<false>, a);
  if (e != cudaSuccess) return e;
  cfg.gridDim = gs;
  e = ff ? cudaLaunchKernelEx(&cfg, k_tr_shift<true>, a) : cudaLaunchKernelEx(&cfg, k_tr_shift<false>, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace uot

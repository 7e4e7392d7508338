// Internal declarations shared by the library's translation units.
//
// Notation (arXiv:1607.05816): potentials U = eps log a, V = eps log b
// (Sec. 4.3 with every update absorbed), S = eps log K(b.dy),
// T = eps log K^T(a.dx).  Per-point state occupies 8-byte slots: a double on
// the FP64 path, a float-float pair on the FP32 path; the per-entry arithmetic
// of the Gibbs operator is FP32 or FP64 depending on the requested precision.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>

#include "../../include/uot.h"

namespace uot {

constexpr double kInf = __builtin_huge_val();
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// ---------------------------------------------------------------------------
// Float-float numbers (hi + lo, two FP32 values, ~48-bit significand).
// The FP32 path keeps every per-point quantity (potentials, log densities and
// weights, intermediate log-sums) in this form so that the iteration never
// uses the FP64 pipe, which on GB300 runs at a small fraction of the FP32 rate.
// Built from the error-free transformations TwoSum and TwoProd (Knuth, Dekker);
// infinities are carried in `hi` with lo = 0.
// ---------------------------------------------------------------------------
struct ff {
  float hi, lo;
};

__host__ __device__ inline ff ff_make(double x) {
  ff r;
  r.hi = (float)x;
  r.lo = (x == x && x != kInf && x != -kInf) ? (float)(x - (double)r.hi) : 0.0f;
  return r;
}
__host__ __device__ inline float2 ff2(const ff& a) { return make_float2(a.hi, a.lo); }
__device__ __forceinline__ ff ffl(float2 v) { return ff{v.x, v.y}; }
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = a + b;
  if (!isfinite(s)) return ff{s, 0.0f};
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return ff{s, e};
}
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
  const float s = a + b;
  if (!isfinite(s)) return ff{s, 0.0f};
  return ff{s, b - (s - a)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  if (!isfinite(s.hi)) return s;
  return ff_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  const ff s = ff_two_sum(a.hi, b);
  if (!isfinite(s.hi)) return s;
  return ff_fast_two_sum(s.hi, s.lo + a.lo);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = a.hi * b.hi;
  if (!isfinite(p) || p == 0.0f) return ff{p, 0.0f};
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  const float p = a.hi * b;
  if (!isfinite(p) || p == 0.0f) return ff{p, 0.0f};
  const float e = fmaf(a.lo, b, fmaf(a.hi, b, -p));
  return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ bool ff_lt(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ ff ff_min(ff a, ff b) { return ff_lt(b, a) ? b : a; }
__device__ __forceinline__ ff ff_max(ff a, ff b) { return ff_lt(a, b) ? b : a; }
__host__ __device__ constexpr ff ff_ninf() { return ff{-__builtin_huge_valf(), 0.0f}; }

// ln 2 as a float-float pair (hi = the FP32 rounding of ln 2)
__host__ __device__ constexpr ff ln2_ff() { return ff{0.693147182464599609375f, -1.904654323148236017e-09f}; }

// ---------------------------------------------------------------------------
// Device helpers shared by the kernel files.
// ---------------------------------------------------------------------------

// SFU base-2 exponential and logarithm (denormal results flushed to zero).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Packed FP32 pairs: the f32x2 arithmetic of the sm_100 family.
typedef unsigned long long f2p;
__device__ __forceinline__ f2p pk(float a, float b) {
  f2p r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 upk(f2p r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
__device__ __forceinline__ f2p fma2(f2p a, f2p b, f2p c) {
  f2p d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2p add2(f2p a, f2p b) {
  f2p d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2p sub2(f2p a, f2p b) {
  f2p d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2p mul2(f2p a, f2p b) {
  f2p d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

__device__ __forceinline__ float warp_maxf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Programmatic dependent launch: wait until the preceding kernel in the stream
// has completed and its writes are visible / let the next kernel launch early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// tcgen05 operands in shared memory.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// Shared-memory matrix descriptor, K-major operand without swizzle: core
// matrices of 8 rows x 16 bytes; lbo = byte step between core matrices along
// K, sbo = along M/N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// byte offset of element (row, k) in a K-major, no-swizzle tile with K = 32
// bf16 (4 core matrices along K): lbo = 128, sbo = 512
__device__ __forceinline__ uint32_t tile_off(int row, int k) {
  return (uint32_t)((row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// A marginal penalty prepared for the device (Table 1 row + parameters).
struct DivParams {
  int kind;          // uot_div_kind
  double lam;        // KL, TV weight
  double log_alpha;  // RG: log alpha (-inf when alpha == 0)
  double log_beta;   // RG: log beta (+inf when beta == +inf)
};

// eps-dependent constants of one Table 1 row in float-float form (FP32 path).
struct DivFF {
  int kind;
  float2 zf;         // KL: lam/(lam+eps)
  float2 lam;        // TV: lam
  float2 elog_a;     // RG: eps log alpha (hi = -inf when alpha == 0)
  float2 elog_b;     // RG: eps log beta (hi = +inf when beta == +inf)
};

// Table 1 in log form with u = 0: U = eps log proxdiv_F(s, eps) given
// S = eps log s and log p.  Zero masses follow Prop. 5.1 with 0/0 = 0:
// s = 0 (S = -inf) gives a = 0; p = 0 gives U_bar = -inf.
__host__ __device__ inline double prox_update(const DivParams& F, double logp, double S,
                                              double eps) {
  if (S == -kInf) return -kInf;
  const double ubar = (logp == -kInf) ? -kInf : eps * logp - S;
  switch (F.kind) {
    case UOT_DIV_EQ:
      return ubar;
    case UOT_DIV_KL:
      return (F.lam / (F.lam + eps)) * ubar;
    case UOT_DIV_TV:
      return fmin(F.lam, fmax(-F.lam, ubar));
    default: {  // UOT_DIV_RG
      const double inner = fmax(eps * F.log_alpha + ubar, 0.0);
      if (F.log_beta == kInf) return inner;
      return fmin(eps * F.log_beta + ubar, inner);
    }
  }
}

// What the last operator pass does with its LSE result z = log sum (natural
// units) at output point `pt`.
enum EpiMode {
  EPI_RAW = 0,    // out[pt] = z                      (intermediate pass)
  EPI_SCALE = 1,  // out[pt] = eps * z                (Gibbs operator alone)
  EPI_PROX = 2,   // pot[pt] = prox(eps log p - eps z) (+ violation terms)
  EPI_PLAN = 3    // out[pt*ncols+col] = exp(pot_shift[pt]/eps + z)
};

struct Epilogue {
  int mode;
  double eps;
  // FP32 path: arrays hold float-float pairs in their 8-byte slots
  int ff;
  float2 eps_ff, inv_eps_ff;
  DivFF Fff;
  // EPI_PROX
  DivParams F;
  const double* logp;      // log density of the output side
  double* pot;             // potential written (read first as the old value)
  const double* logw;      // log reference weight of the output side (violation)
  double* err;             // [2 per batch entry] = {sum dx |r_old - r_new|, sum dx r_new}; NULL: no check
  const double* zshift;    // device scalar added to S before the prox (Algorithm 4's Z; a
                           // float-float pair on the FP32 path); NULL: none.  Read after the
                           // pass's inputs are complete.
  // EPI_PLAN
  const double* pot_shift; // U (or V) of the output side
  int ncols, col;
  // all modes except PROX
  double* out;
  // batches of independent arrays (barycenters): element (b, pt) of pot/out
  // lives at b*bstride + pt, of logp at b*bstride_p + pt; logw is shared.
  int64_t bstride;
  int64_t bstride_p;
};

// Violation terms of one point: r_old = exp((U_old+S)/eps), r_new = exp((U_new+S)/eps).
__device__ inline void violation_terms(double Uold, double Unew, double S, double logw,
                                       double eps, double& num, double& den) {
  const double w = exp(logw);
  const double ro = (Uold == -kInf || S == -kInf) ? 0.0 : exp((Uold + S) / eps);
  const double rn = (Unew == -kInf || S == -kInf) ? 0.0 : exp((Unew + S) / eps);
  num = w * fabs(ro - rn);
  den = w * rn;
}

// Applies the epilogue to one result; returns the violation terms through num/den.
__device__ inline void apply_epilogue(const Epilogue& e, int64_t b, int64_t pt, double z,
                                      double& num, double& den) {
  num = 0.0;
  den = 0.0;
  const int64_t q = b * e.bstride + pt;
  switch (e.mode) {
    case EPI_RAW:
      e.out[q] = z;
      break;
    case EPI_SCALE:
      e.out[q] = (z == -kInf) ? -kInf : e.eps * z;
      break;
    case EPI_PROX: {
      double S = (z == -kInf) ? -kInf : e.eps * z;
      if (e.zshift) S = (S == -kInf || *e.zshift == -kInf) ? -kInf : S + *e.zshift;
      const double Uold = e.pot[q];
      const double Unew = prox_update(e.F, e.logp[b * e.bstride_p + pt], S, e.eps);
      e.pot[q] = Unew;
      if (e.err) violation_terms(Uold, Unew, S, e.logw[pt], e.eps, num, den);
      break;
    }
    default: {  // EPI_PLAN
      const double u = e.pot_shift[q];
      const double v = (u == -kInf || z == -kInf) ? 0.0 : exp(u / e.eps + z);
      e.out[q * e.ncols + e.col] = v;
      break;
    }
  }
}

// Table 1 in log form, float-float version of prox_update.
__device__ inline ff prox_update_ff(const DivFF& F, ff logp, ff S, ff eps) {
  if (S.hi == -INFINITY) return ff_ninf();
  const ff ubar = (logp.hi == -INFINITY) ? ff_ninf() : ff_sub(ff_mul(eps, logp), S);
  switch (F.kind) {
    case UOT_DIV_EQ:
      return ubar;
    case UOT_DIV_KL:
      return (ubar.hi == -INFINITY) ? ubar : ff_mul(ffl(F.zf), ubar);
    case UOT_DIV_TV: {
      const ff lam = ffl(F.lam);
      return ff_min(lam, ff_max(ff_neg(lam), ubar));
    }
    default: {
      const ff lo = (F.elog_a.x == -INFINITY || ubar.hi == -INFINITY) ? ff_ninf() : ff_add(ffl(F.elog_a), ubar);
      const ff inner = ff_max(lo, ff{0.0f, 0.0f});
      if (F.elog_b.x == INFINITY) return inner;
      const ff hi = (ubar.hi == -INFINITY) ? ff_ninf() : ff_add(ffl(F.elog_b), ubar);
      return ff_min(hi, inner);
    }
  }
}

// FP32 violation terms from float-float potentials: r_new = e^{(U_new+S)/eps},
// |r_old - r_new| = r_new |expm1((U_old - U_new)/eps)|.
__device__ inline void violation_terms_ff(ff Uold, ff Unew, ff S, ff logw, ff inv_eps, float& num,
                                          float& den) {
  const float w = expf(logw.hi + logw.lo);
  if (S.hi == -INFINITY) {
    num = den = 0.0f;
    return;
  }
  float rn = 0.0f, ro = 0.0f;
  if (Unew.hi != -INFINITY) {
    const ff a = ff_mul(ff_add(Unew, S), inv_eps);
    rn = expf(a.hi + a.lo);
  }
  if (Uold.hi != -INFINITY) {
    const ff a = ff_mul(ff_add(Uold, S), inv_eps);
    ro = expf(a.hi + a.lo);
  }
  float diff;
  if (Uold.hi != -INFINITY && Unew.hi != -INFINITY) {
    const ff d = ff_mul(ff_sub(Uold, Unew), inv_eps);
    diff = rn * fabsf(expm1f(d.hi + d.lo));
  } else {
    diff = fabsf(ro - rn);
  }
  num = w * diff;
  den = w * rn;
}

// S + Z with Z a float-float device scalar (-inf absorbs).
__device__ inline ff ff_zshift(ff S, const double* zshift) {
  const ff Zv = ffl(*reinterpret_cast<const float2*>(zshift));
  return (S.hi == -INFINITY || Zv.hi == -INFINITY) ? ff_ninf() : ff_add(S, Zv);
}

// Float-float epilogue (FP32 path): z is the log-sum in natural units.
__device__ inline void apply_epilogue_ff(const Epilogue& e, int64_t b, int64_t pt, ff z, float& num,
                                         float& den) {
  num = 0.0f;
  den = 0.0f;
  const int64_t q = b * e.bstride + pt;
  switch (e.mode) {
    case EPI_RAW:
      reinterpret_cast<float2*>(e.out)[q] = ff2(z);
      break;
    case EPI_SCALE:
      reinterpret_cast<float2*>(e.out)[q] = ff2(z.hi == -INFINITY ? z : ff_mul(z, ffl(e.eps_ff)));
      break;
    case EPI_PROX: {
      const ff eps = ffl(e.eps_ff);
      ff S = (z.hi == -INFINITY) ? ff_ninf() : ff_mul(z, eps);
      if (e.zshift) S = ff_zshift(S, e.zshift);
      float2* pot = reinterpret_cast<float2*>(e.pot);
      const ff Uold = ffl(pot[q]);
      const ff lp = ffl(reinterpret_cast<const float2*>(e.logp)[b * e.bstride_p + pt]);
      const ff Unew = prox_update_ff(e.Fff, lp, S, eps);
      pot[q] = ff2(Unew);
      if (e.err)
        violation_terms_ff(Uold, Unew, S, ffl(reinterpret_cast<const float2*>(e.logw)[pt]),
                           ffl(e.inv_eps_ff), num, den);
      break;
    }
    default: {  // EPI_PLAN
      const ff u = ffl(reinterpret_cast<const float2*>(e.pot_shift)[q]);
      float v = 0.0f;
      if (u.hi != -INFINITY && z.hi != -INFINITY) {
        const ff a = ff_add(ff_mul(u, ffl(e.inv_eps_ff)), z);
        v = expf(a.hi + a.lo);
      }
      reinterpret_cast<float2*>(e.out)[q * e.ncols + e.col] = make_float2(v, 0.0f);
      break;
    }
  }
}

// Block-wide sum of two floats, then one double atomicAdd per block.
template <int NT>
__device__ inline void block_add2f(float a, float b, double* acc) {
  __shared__ float sa[NT / 32], sb[NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (w == 0) {
    a = (l < NT / 32) ? sa[l] : 0.0f;
    b = (l < NT / 32) ? sb[l] : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (l == 0 && acc) {
      atomicAdd(acc, (double)a);
      atomicAdd(acc + 1, (double)b);
    }
  }
}

// Block-wide sum of two doubles, then one atomicAdd per block into acc[0..1].
template <int NT>
__device__ inline void block_add2(double a, double b, double* acc) {
  __shared__ double sa[NT / 32], sb[NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (w == 0) {
    a = (l < NT / 32) ? sa[l] : 0.0;
    b = (l < NT / 32) ? sb[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (l == 0 && acc) {
      atomicAdd(acc, a);
      atomicAdd(acc + 1, b);
    }
  }
}

// ---------------------------------------------------------------------------
// instrumentation: launch counting and optional event timing of the Gibbs
// operator kernels (on the stream they are launched on)
// ---------------------------------------------------------------------------

enum ProfFamily { PROF_GRID_PASS = 0, PROF_ROWS = 1, PROF_GRID_BLK = 2, PROF_NFAM = 3 };
void count_launches(int k);

// Raises, never lowers, a kernel's limit on dynamic shared memory (the
// cudaFuncAttributeMaxDynamicSharedMemorySize attribute) on the current device
// to at least `bytes`.  The attribute is process-wide per kernel: setting it to
// each call's own size would let a concurrent call on another stream or host
// thread lower it between another call's set and launch, which then fails as
// an invalid launch.  Thread-safe; a no-op once the limit is high enough.
cudaError_t smem_limit_at_least(const void* kernel, size_t bytes);
template <typename K>
cudaError_t smem_at_least(K* kernel, size_t bytes) {
  return smem_limit_at_least(reinterpret_cast<const void*>(kernel), bytes);
}
void prof_mark_begin(int family, cudaStream_t s);
void prof_mark_end(int family, cudaStream_t s);

// ---------------------------------------------------------------------------
// launchers implemented in the kernel translation units
// ---------------------------------------------------------------------------

// One separable pass of the log-domain Gibbs operator on a grid axis:
//   z[i][l] = log sum_j exp(L[l][j] - (xo[i] - yi[j])^2 / eps)
// L[l][j] = in[l*nin + j] (in_is_pot = 0) or in[.]/eps + logw[.] (in_is_pot = 1).
// Output layout is transposed: point index i*nlines + l.
// `nbatch` independent arrays: input b at in + b*nlines*nin, results at batch b
// of the epilogue (output batch stride nout*nlines for EPI_RAW).
// FP32 only: zprev (optional, [nbatch][nout*nlines]) receives this pass's
// result; with use_prev = 1 its previous content is used as the shift of the
// log-sum-exp (see k_grid.cu).
// tc3_ok: the tensor-core pass (k_grid_tc3.cu) may be used (the tuner's last
// tile) -- its block-stabilisation condition k (span_out + span_in)^2 <= 90
// holds for 32-point blocks of both axes; tc_err receives its wait flag.
// Uniform axes of one pass, for the block-stabilised kernel: every output
// point is xo[0] + i h and every input point yi[0] + j h, exactly, with the
// same spacing h on both sides.
struct BlkAxis {
  int ok;    // both axes uniform with one spacing (and h, d0 exact in FP32)
  float h;   // the spacing
  float d0;  // xo[0] - yi[0]
};

// Two consecutive FP32 passes over short axes (all four sizes <= 64) fused per
// plane: ngroups = prefixes over the axes before the pair x S, S = the
// contracted suffix; pass 1's intermediate stays in shared memory.
// grid_fuse_short_pairs(mode) sets whether such pairs are fused (1) or run as
// two passes (0, the default); returns the previous mode.
int grid_fuse_short_pairs(int mode);
bool grid_plane_ok(int n1in, int n1out, int n2in, int n2out);
cudaError_t launch_grid_pass_plane(const double* in, const double* logw, int in_is_pot, int64_t ngroups, int S,
                                   int nin1, const void* yi1, int nout1, const void* xo1, float* zprev1,
                                   int nin2, const void* yi2, int nout2, const void* xo2, float* zprev2,
                                   double eps, int nbatch, int use_prev, double* zero_acc, const Epilogue& epi,
                                   cudaStream_t s);
cudaError_t launch_grid_pass(int prec, const double* in, const double* logw, int in_is_pot,
                             int nlines, int nin, const void* yi, int nout, const void* xo,
                             double eps, int nbatch, const Epilogue& epi, cudaStream_t s,
                             float* zprev, int use_prev, double* zero_acc = nullptr, int tc3_ok = 0,
                             int* tc_err = nullptr, const BlkAxis* blk = nullptr, int precise = 0);
// precise = 1 (FP32): the pass with float-float exponents (k_grid.cu,
// grid_pass_ffp), as every FP32 pass runs while grid_force_precise(1) is set;
// returns the previous setting
int grid_force_precise(int on);
int precise_forced();  // the current setting (also read by the point-cloud path)

// Tensor-core convolutions of the warm-start network (k_conv_tc.cu); BF16
// tensors are passed as void pointers.
struct ConvTcLaunch {
  int N, H, W;        // images, image size (W = 64)
  int ldx;            // channel stride of the NHWC input
  int cin_pad;        // K channels per tap (multiple of 64, >= ldx)
  int nout;           // output channels
  int ldy;            // channel stride of the BF16 output (multiple of 16)
  int dil;            // dilation
  int mode;           // 0: + bias, 1: + bias then leaky ReLU, 2: x leaky-ReLU derivative of ref
  const float* bias;
  const void* ref;    // mode 2: BF16 [P][ldref]
  int ldref;
  void* y;            // BF16 [P][ldy] or NULL
  float* yf;          // FP32 [P][nout] or NULL
  int* err;           // bounded-wait flag (may be NULL)
};
int conv_tc_available();
cudaError_t launch_conv_tc(const void* x, const void* wk, int bn, const ConvTcLaunch& L, cudaStream_t s);
cudaError_t launch_wgrad_tc(const void* dyT, int cout_rows, const void* xT, int cin_pad, int N, int H, int W, int dil,
                            int Cout, int Cin, float* part, int splits, float* dw, int* err, cudaStream_t s);
cudaError_t launch_nhwc_to_shifted_cnhw(const void* x, int N, int H, int W, int C, int dil, void* xT,
                                        cudaStream_t s);
cudaError_t launch_nhwc_to_cnhw(const void* y, int64_t P, int C, void* yT, cudaStream_t s);
cudaError_t launch_bias_grad(const void* dy, int64_t P, int ld, int C, float* db, cudaStream_t s);
cudaError_t launch_weights_bf16(const float* w, int Cout, int Cin, int cout_pad, int cin_pad, int cin_rows,
                                int cout_kpad, void* wf, void* wb, cudaStream_t s);

// The tensor-core pass with three-part BF16 operands (k_grid_tc3.cu): same
// result as the FP32 pass to FP32 accuracy; nin <= grid_pass_tc3_max_nin().
int grid_pass_tc3_max_nin();
cudaError_t launch_grid_pass_tc3(const float2* in, const float2* logw, int in_is_pot, int nlines, int nin,
                                 const float* yi, int nout, const float* xo, float2 inv_eps, float k2, int nbatch,
                                 const Epilogue& epi, cudaStream_t s, int* err_flag, double* zero_acc);

// Tile shapes of the FP32 grid pass (warps splitting the contraction x
// outputs per lane) and the tuner that times them once per pass shape
// (nlines, nin, nout, batch) and device, on first use (k_grid.cu).
//  grid_set_autotune(0|1): off = always the first shape; returns the previous mode.
//  grid_force_tile(idx): use shape idx for every pass (-1: back to tuning); -1 if idx is out of range.
//  grid_tune_hold(1|0): nested hold on the calling thread (no tuning, which allocates).
//  grid_tile_table(): the tuned shapes and their measured times, one line per pass shape.
int grid_set_autotune(int mode);
int grid_autotune_enabled();
int grid_tc3_wanted();  // the tensor-core tile may be chosen (tuner on or tile forced), not held
int grid_force_tile(int idx);
int grid_tile_count();
void grid_tune_hold(int on);
std::string grid_tile_table();

// Persistent FP32 grid solve (k_grid.cu): the whole iteration, eps stages and
// convergence test of one grid problem in one cooperative launch.
struct PersistLaunch {
  int ndim;
  int shape_x[UOT_MAX_DIM], shape_y[UOT_MAX_DIM];
  const void* axes_x[UOT_MAX_DIM];
  const void* axes_y[UOT_MAX_DIM];
  double* U;            // float-float state in 8-byte slots
  double* V;
  const double* logp;
  const double* logq;
  const double* logdx;
  const double* logdy;
  double* pass[2];
  float* zbuf[2][UOT_MAX_DIM];
  int nstage, iters_per_stage, max_iter, check_every;
  double tol;
  const float2* eps_ff;
  const float2* inv_eps_ff;
  const float* k2;
  const DivFF* F;       // [nstage+1][2]
  double* acc;
  unsigned* bar;
  int* status;
  double* err_out;
};
int grid_solve_persistent_ctas(int nin_max);
cudaError_t launch_grid_solve_persistent(const PersistLaunch& L, int grid, cudaStream_t s);
// One thread waits (bounded by limit_ns) for *flag to leave 0; *status = 1 on expiry.
cudaError_t launch_wait_selftest(const unsigned* flag, unsigned long long limit_ns, int* status, cudaStream_t s);

// Two fused separable passes per grid line of a 2-D FP32 problem
// (k_grid_fused.cu): pass 1 contracts the line's values (from in1) and
// applies the prox update to the potential pot1 (+ violation); pass 2
// contracts the line of new potentials (pot1/eps2 + log w, from shared memory)
// and writes raw log-sums to out2.  One CTA per line.
struct FusedArgs {
  int nlines;
  // pass 1
  const float2* in1;        // [nlines][nin1] float-float log values
  int nin1, nout1;
  const float* y1;          // [nin1] input coordinates
  const float* x1;          // [nout1] output coordinates (= pass-2 input coordinates)
  float2 eps1_ff, inv_eps1_ff;
  float k2_1;               // log2(e)/eps1
  int out1_row;             // output i of line l at l*nout1 + i (1) or i*nlines + l (0)
  DivFF F1;
  const float2* logp1;      // log density at pass-1 outputs (same indexing)
  float2* pot1;             // potential at pass-1 outputs (old value read, new written)
  const float2* logw1;      // log weights at pass-1 outputs
  double* err;              // violation accumulators [2] or NULL
  float* z1;
  int use_prev1;
  // pass 2
  int do2;
  int nout2;
  const float* x2;          // [nout2] output coordinates
  float2 inv_eps2_ff;
  float k2_2;
  float2* out2;             // output i of line l at i*nlines + l
  float* z2;
  int use_prev2;
  double* zero_acc;         // two doubles cleared by block 0 after the dependency wait, or NULL
};
size_t grid_fused2_smem(int nin1, int nout1);
cudaError_t launch_grid_fused2(const FusedArgs& a, cudaStream_t s);

// Tensor-core (tcgen05) variant of the FP32 grid pass (k_grid_tc.cu); float-
// float lines in, same epilogues; valid while k (2 r)^2 stays in range (see
// grid_tc_valid).  err_flag is set if a bounded wait gave up.
size_t grid_pass_tc_smem(int nin);
cudaError_t launch_grid_pass_tc(const double* in, const double* logw, int in_is_pot, int nlines,
                                int nin, const void* yi, int nout, const void* xo, double eps,
                                int nbatch, const Epilogue& epi, cudaStream_t s, int* err_flag,
                                double* zero_acc);

// Row-wise log-domain Gibbs operator for dense costs and point clouds:
//   z_i = log sum_j exp(L_j - C_ij / eps),  L_j = W_j/eps + logw_j
// C given densely (C row-major [nrows][ncols_c]) or as |x_i - y_j|^2.
struct RowsGeom {
  int kind;          // UOT_GEOM_DENSE or UOT_GEOM_POINTS
  const void* C;     // dense, in the precision's type
  const void* x;     // points [nrows*d]
  const void* y;     // points [nin*d]
  int d;
  const float* C32;  // dense FP64: FP32 copy of C for the row kernel's prefilter (NULL: none)
};
// FP32 point clouds with d <= 3 and a `part` buffer use the chunked kernels of
// k_points.cu (zprev: previous results used as log-sum-exp shifts).
// precise = 1 (FP32 point clouds, d <= 3): the pass with float-float
// exponents (launch_points_ffp) instead of the chunked kernels.
cudaError_t launch_rows(int prec, const RowsGeom& g, int nrows, int nin, const double* W,
                        const double* logw, double eps, void* scratch_L, const Epilogue& epi,
                        cudaStream_t s, float* zprev = nullptr, int use_prev = 0,
                        void* part = nullptr, int precise = 0);
// FP32 point clouds (d <= 3), exponents in float-float (k_points.cu); bmax
// holds ceil(nin / 1024) floats.
cudaError_t launch_points_ffp(const float* x, const float* y, int d, int nout, int nin, const double* W,
                              const double* logw, double eps, float* bmax, float* zprev, const Epilogue& epi,
                              cudaStream_t s);
// Scratch of launch_rows for FP64 dense rows with the FP32 prefilter; its
// first 4 bytes hold a counter that must be zero before the first launch.
size_t rows_pf_scratch_bytes(int64_t nin);
int points_nchunks(int nin, int nout);
bool points_chunks_fit(int nin);
cudaError_t launch_points(const float* x, const float* y, int d, int nout, int nin,
                          const double* W, const double* logw, double eps, float* bmax,
                          float* zprev, int use_prev, float2* part, const Epilogue& epi,
                          cudaStream_t s);

// Persistent batched solver for many point-cloud problems (k_batch.cu).
struct BatchArgs {
  int nprob, d, nstage, iters_per_stage, max_iter, check_every, nmax, mmax;
  int ndiv;  // problems indexed by divs: divs[(stage * ndiv + k) * 2 + side]
  float tol;
  const int* order;
  const int* n;
  const int* m;
  const int64_t* xoff;
  const int64_t* yoff;
  const float* x;
  const float* y;
  const float2* logp;
  const float2* logdx;
  const float2* logq;
  const float2* logdy;
  const DivFF* divs;
  const float2* eps_ff;
  const float2* inv_eps_ff;
  const float* k2;
  float* Uout;
  float* Vout;
  double* Uout64;  // if set (opts.out_f64): the float-float state rounded to FP64 instead of Uout
  double* Vout64;
  int* iters_out;
  float* err_out;
  int* next;
  float2* Uff;  // [sum n] float-float potentials (solver state)
  float2* Vff;  // [sum m]
  float* zU;    // [sum n] last log-sums (shifts)
  float* zV;    // [sum m]
  int translate;        // 1: the translation step (KL / KL problems; uot_opts.translate)
  const double2* lam;   // [nprob] (lambda1, lambda2) when translate
};
// CTA-size variant 0 (8 warps) or 1 (16 warps); the variant for a batch shape
// (d, nmax, mmax) is timed on a sample of the batch on first use when the
// tuner is on (batch_pick_variant: synchronises `s`; a.next is left dirty).
int batch_ctas_per_sm(int d, int variant, int nmax, int mmax);
int batch_pick_variant(const BatchArgs& a, const int* h_order, cudaStream_t s);
int batch_force_warps(int warps);  // 8 or 16 forces a CTA size, 0 returns to the tuned one; -1 if invalid
std::string batch_tune_table();
cudaError_t launch_batch(const BatchArgs& a, int variant, int grid, cudaStream_t s);

// Translation step for lam1 KL / lam2 KL penalties (uot_opts.translate; not
// in the paper): per problem b, c_b = lam1 lam2 / (lam1 + lam2) (log A_b -
// log B_b), A_b = sum_i dx_i p_bi e^{-U_bi/lam1}, B_b = sum_j dy_j q_bj
// e^{-V_bj/lam2}; then U_b += c_b, V_b -= c_b (the plan is unchanged).  U, V,
// log p, log q [batch][n or m], log dx, log dy [n or m], all FP64 or all
// float-float (ff = 1); part holds kl_translate_part_count double2.
size_t kl_translate_part_count(int64_t n, int64_t m, int batch);
cudaError_t launch_kl_translate(double* U, double* V, const double* logp, const double* logq,
                                const double* logdx, const double* logdy, int64_t n, int64_t m, int batch,
                                int ff, double lam1, double lam2, double2* part, cudaStream_t s);

// Algorithm 1 (non-log) half-step on a stored FP64 kernel:
//   a_i = proxdiv_F(sum_j K_ij b_j w_j, eps), also the violation terms.
cudaError_t launch_alg1_half(const double* K, int nrows, int nin, const double* b,
                             const double* w, const double* p, DivParams F, double eps,
                             double* a, const double* wout, double* err, cudaStream_t s);

// Algorithm 1 at one eps, `iters` iterations (a then b) in one launch of one
// thread-block cluster holding K and K^T in shared memory (16 CTAs, else 8).
// check_every > 0: the violation of every check_every-th and of the last
// iteration, stopping once it is <= tol (tol > 0) after more than one
// iteration; res [3] receives the last violation, the iterations run and the
// converged flag.  *launched = false (and nothing queued) when the kernel
// does not fit or no such cluster can be scheduled.
cudaError_t launch_alg1_cluster(const double* K, const double* KT, int n, int m, const double* p,
                                const double* dx, const double* q, const double* dy, DivParams F1,
                                DivParams F2, double eps, double* a, double* b, int iters, int check_every,
                                double tol, double* res, cudaStream_t s, bool* launched);

}  // namespace uot

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
#include <string.h>

#include <algorithm>

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

// ---- packed FP32 pairs (f32x2 arithmetic of sm_100+ family GPUs) ----
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
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// FP32 grid pass.  One CTA = one line x 128 consecutive outputs; its 8 warps
// split the contraction index j into 8 contiguous ranges (so a 256-point axis
// gives 8 x 32 terms per output) and combine their partial (max, sum) pairs
// through shared memory.  Each lane owns 4 outputs handled as two f32x2 pairs.
//
// The log-sum-exp needs a shift m per output; any m with every term's
// exponent <= ~100 and the largest >= ~-90 gives the full FP32 accuracy, and
// the result does not depend on m.  When `zprev` holds this pass's result
// from the previous call at the same eps (potentials move little between
// iterations), that value is used as the shift and each term costs one sweep.
// If any combined sum of the CTA falls outside [2^-90, 2^100], the CTA redoes
// its outputs with the exact per-range maximum (a max sweep and a sum sweep).
constexpr int kNW = 8;                    // warps per CTA = contraction splits
constexpr int kOutCTA = 128;              // outputs per CTA (4 per lane)

struct PassArgs {
  const float2* in;    // float-float line values (or potentials when in_is_pot)
  const float2* logw;  // float-float log weights (in_is_pot only)
  int in_is_pot;
  int nlines, nin, nout;
  const float* yi;
  const float* xo;
  float2 inv_eps;      // 1/eps as float-float
  float k2;            // log2(e)/eps
  float* zprev;        // [nbatch][nout*nlines] approximate result of the previous call, or NULL
  int use_prev;
  double* zero_acc;    // if set, the first block of each batch entry b clears zero_acc[2b..2b+1]
};

__device__ __forceinline__ ff load_L_ff(const PassArgs& a, const float2* in, int64_t idx) {
  const ff v = ffl(in[idx]);
  if (!a.in_is_pot) return v;
  if (v.hi == -INFINITY) return ff_ninf();
  return ff_add(ff_mul(v, ffl(a.inv_eps)), ffl(a.logw[idx]));
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

// Operands of the epilogue that do not depend on the preceding kernel, loaded
// before waiting on it.
struct EpiPre {
  float2 uold, lp, lw;
};

__device__ __forceinline__ void epilogue_prefetch(const Epilogue& e, int64_t b, int64_t pt, EpiPre& o) {
  if (e.mode == EPI_PROX) {
    const int64_t q = b * e.bstride + pt;
    o.uold = reinterpret_cast<const float2*>(e.pot)[q];
    o.lp = reinterpret_cast<const float2*>(e.logp)[b * e.bstride_p + pt];
    o.lw = e.err ? reinterpret_cast<const float2*>(e.logw)[pt] : make_float2(0.0f, 0.0f);
  }
}

__device__ __forceinline__ void epilogue_apply(const Epilogue& e, int64_t b, int64_t pt, ff z,
                                               const EpiPre& o, float& num, float& den) {
  if (e.mode != EPI_PROX) {
    apply_epilogue_ff(e, b, pt, z, num, den);
    return;
  }
  num = den = 0.0f;
  const ff eps = ffl(e.eps_ff);
  const ff S = (z.hi == -INFINITY) ? ff_ninf() : ff_mul(z, eps);
  const ff Unew = prox_update_ff(e.Fff, ffl(o.lp), S, eps);
  reinterpret_cast<float2*>(e.pot)[b * e.bstride + pt] = ff2(Unew);
  if (e.err) violation_terms_ff(ffl(o.uold), Unew, S, ffl(o.lw), ffl(e.inv_eps_ff), num, den);
}

constexpr int kLineRegs = 4;  // line elements held per thread (nin <= 1024 fast path)

// Shared-memory workspace of one work item.
struct ItemSmem {
  float4* sline;               // nin x {t, t, y, y}
  float2 (*part)[kOutCTA];     // [kNW][kOutCTA]
  float* sshift;               // [kOutCTA]
  float* sred;                 // [kNW]
};

// One work item of a grid pass: line l of batch entry bz, outputs i0 .. i0+127.
// With kPDL the item waits for the preceding kernel after its independent
// prologue (programmatic dependent launch) and clears the violation
// accumulators when asked.  Returns the item's violation terms in num, den.
template <bool kPDL>
__device__ __forceinline__ void grid_item_f32(const PassArgs& a, const Epilogue& epi, int l, int64_t bz,
                                              int i0, const ItemSmem& sm, float& num, float& den) {
  float4* sline = sm.sline;
  float2 (*part)[kOutCTA] = sm.part;
  float* sshift = sm.sshift;
  float* sred = sm.sred;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nin = a.nin, nout = a.nout, nlines = a.nlines;
  const float2* in = a.in + bz * (int64_t)nlines * nin;
  const int64_t base = (int64_t)l * nin;
  float* zprev = a.zprev ? a.zprev + bz * (int64_t)nout * nlines : nullptr;
  const bool spec = a.use_prev && zprev;

  // ---- prologue independent of the preceding kernel ----
  const int my_i = i0 + tid;
  const bool owns = (tid < kOutCTA) && (my_i < nout);
  const int64_t my_pt = (int64_t)my_i * nlines + l;
  float zp = 0.0f;
  EpiPre pre;
  if (owns) {
    if (spec) zp = zprev[my_pt];
    epilogue_prefetch(epi, bz, my_pt, pre);
  }
  float yv[kLineRegs];
#pragma unroll
  for (int r = 0; r < kLineRegs; ++r) {
    const int j = tid + r * kNW * 32;
    yv[r] = (j < nin) ? a.yi[j] : 0.0f;
  }
  float xq[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + lane + 32 * q;
    xq[q] = a.xo[i < nout ? i : nout - 1];
  }

  if (kPDL) {
    pdl_wait();
    if (a.zero_acc && blockIdx.x == 0 && blockIdx.y == 0 && tid < 2) a.zero_acc[2 * bz + tid] = 0.0;
    pdl_launch_dependents();
  }

  // ---- line values: one read, kept in registers when the line is short ----
  ff lv[kLineRegs];
  const bool in_regs = nin <= kLineRegs * kNW * 32;
  float mx = -INFINITY;
  if (in_regs) {
#pragma unroll
    for (int r = 0; r < kLineRegs; ++r) {
      const int j = tid + r * kNW * 32;
      lv[r] = (j < nin) ? load_L_ff(a, in, base + j) : ff_ninf();
      mx = fmaxf(mx, lv[r].hi);
    }
  } else {
    for (int j = tid; j < nin; j += kNW * 32) mx = fmaxf(mx, load_L_ff(a, in, base + j).hi);
  }
  mx = warp_maxf(mx);
  if (lane == 0) sred[warp] = mx;
  __syncthreads();
  mx = sred[0];
#pragma unroll
  for (int w = 1; w < kNW; ++w) mx = fmaxf(mx, sred[w]);

  num = 0.0f;
  den = 0.0f;
  if (mx == -INFINITY) {
    // b = 0 on the whole line: every sum is empty.
    if (owns) {
      if (zprev) zprev[my_pt] = -INFINITY;
      epilogue_apply(epi, bz, my_pt, ff_ninf(), pre, num, den);
    }
    return;
  }
  if (in_regs) {
#pragma unroll
    for (int r = 0; r < kLineRegs; ++r) {
      const int j = tid + r * kNW * 32;
      if (j < nin) {
        const float t = (lv[r].hi == -INFINITY) ? -INFINITY : ((lv[r].hi - mx) + lv[r].lo) * kLog2e;
        sline[j] = make_float4(t, t, yv[r], yv[r]);
      }
    }
  } else {
    for (int j = tid; j < nin; j += kNW * 32) {
      const ff v = load_L_ff(a, in, base + j);
      const float t = (v.hi == -INFINITY) ? -INFINITY : ((v.hi - mx) + v.lo) * kLog2e;
      const float y = a.yi[j];
      sline[j] = make_float4(t, t, y, y);
    }
  }
  // speculative shifts in log2 units relative to the staged line
  if (tid < kOutCTA) sshift[tid] = (!owns || zp == -INFINITY) ? 0.0f : (zp - mx) * kLog2e;
  __syncthreads();

  const f2p nk2 = pk(-a.k2, -a.k2);
  const int J = (nin + kNW - 1) / kNW;
  const int j0 = warp * J, j1 = min(nin, j0 + J);
  const f2p X0 = pk(xq[0], xq[1]), X1 = pk(xq[2], xq[3]);

  bool exact = !spec;
  for (int attempt = 0; attempt < 2; ++attempt) {
    float mq[4];
    if (!exact) {
#pragma unroll
      for (int q = 0; q < 4; ++q) mq[q] = sshift[lane + 32 * q];
    } else {
      // exact per-range maximum
      float m4[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
#pragma unroll 4
      for (int j = j0; j < j1; ++j) {
        const float4 v = sline[j];
        const f2p T = pk(v.x, v.y), Y = pk(v.z, v.w);
        const f2p D0 = sub2(X0, Y), D1 = sub2(X1, Y);
        const float2 A0 = upk(fma2(nk2, mul2(D0, D0), T));
        const float2 A1 = upk(fma2(nk2, mul2(D1, D1), T));
        m4[0] = fmaxf(m4[0], A0.x);
        m4[1] = fmaxf(m4[1], A0.y);
        m4[2] = fmaxf(m4[2], A1.x);
        m4[3] = fmaxf(m4[3], A1.y);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) mq[q] = m4[q];
    }
    // sum sweep relative to the shifts (a -inf shift means an empty range)
    const f2p MS0 = pk(mq[0] == -INFINITY ? 0.0f : mq[0], mq[1] == -INFINITY ? 0.0f : mq[1]);
    const f2p MS1 = pk(mq[2] == -INFINITY ? 0.0f : mq[2], mq[3] == -INFINITY ? 0.0f : mq[3]);
    f2p S0 = pk(0.0f, 0.0f), S1 = S0;
#pragma unroll 4
    for (int j = j0; j < j1; ++j) {
      const float4 v = sline[j];
      const f2p T = pk(v.x, v.y), Y = pk(v.z, v.w);
      const f2p D0 = sub2(X0, Y), D1 = sub2(X1, Y);
      const float2 A0 = upk(fma2(nk2, mul2(D0, D0), sub2(T, MS0)));
      const float2 A1 = upk(fma2(nk2, mul2(D1, D1), sub2(T, MS1)));
      S0 = add2(S0, pk(ex2_approx(A0.x), ex2_approx(A0.y)));
      S1 = add2(S1, pk(ex2_approx(A1.x), ex2_approx(A1.y)));
    }
    const float2 s01 = upk(S0), s23 = upk(S1);
    const float sq[4] = {s01.x, s01.y, s23.x, s23.y};
#pragma unroll
    for (int q = 0; q < 4; ++q)
      part[warp][lane + 32 * q] = make_float2(mq[q] == -INFINITY ? 0.0f : mq[q], mq[q] == -INFINITY ? 0.0f : sq[q]);
    __syncthreads();

    // combine the 8 ranges of each output
    bool bad = false;
    float Mo = -INFINITY, So = 0.0f;
    if (tid < kOutCTA) {
#pragma unroll
      for (int w = 0; w < kNW; ++w) {
        const float2 pr = part[w][tid];
        if (pr.y > 0.0f) Mo = fmaxf(Mo, pr.x);
      }
      if (Mo != -INFINITY) {
#pragma unroll
        for (int w = 0; w < kNW; ++w) {
          const float2 pr = part[w][tid];
          if (pr.y > 0.0f) So += pr.y * ex2_approx(pr.x - Mo);
        }
      }
      if (owns && !exact) bad = !(So >= 0x1p-90f && So <= 0x1p100f);
    }
    const int any_bad = __syncthreads_or(bad ? 1 : 0);
    if (any_bad && !exact) {
      exact = true;
      continue;  // block-uniform: redo with exact maxima
    }
    if (owns) {
      ff z = ff_ninf();
      if (So > 0.0f) {
        // z = mx + ln2 Mo + ln2 log2(So), the first product kept exact in float-float
        const ff ln2 = ff{0.693147182464599609375f, -1.904654323148236017e-09f};
        z = ff_add_f(ff_add_f(ff_mul_f(ln2, Mo), mx), kLn2 * lg2_approx(So));
      }
      if (zprev) zprev[my_pt] = z.hi;
      epilogue_apply(epi, bz, my_pt, z, pre, num, den);
    }
    break;
  }
}

__global__ void __launch_bounds__(kNW * 32, 4)
    grid_pass_f32(PassArgs a, Epilogue epi) {
  extern __shared__ float4 sline[];
  __shared__ float2 part[kNW][kOutCTA];
  __shared__ float sshift[kOutCTA];
  __shared__ float sred[kNW];
  const ItemSmem sm{sline, part, sshift, sred};
  float num, den;
  grid_item_f32<true>(a, epi, blockIdx.y, blockIdx.z, blockIdx.x * kOutCTA, sm, num, den);
  if (epi.err) block_add2f<kNW * 32>(num, den, epi.err + 2 * (int64_t)blockIdx.z);
}

// ---------------------------------------------------------------------------
// Persistent solve: the whole iteration of a single FP32 grid problem in one
// cooperative launch (all CTAs co-resident).  Each pass is a set of work items
// (line, 128 outputs) spread over the CTAs, followed by a grid barrier; the
// eps-scaling stages and the convergence test run on the device, so the host
// waits only for the end of the solve.  Barrier waits are bounded in time
// (status[0] = 1 and every CTA returns if one expires).
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Generation-counting barrier: bar[0] arrivals, bar[1] generation.
__device__ bool grid_barrier(unsigned* bar, int* status) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      bar[0] = 0;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*gen == g) {
        __nanosleep(64);
        if (global_ns() - t0 > 2000000000ull) {
          atomicExch(status, 1);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)status == 0;
}

struct PersistArgs {
  int ndim;
  int shape_x[UOT_MAX_DIM], shape_y[UOT_MAX_DIM];
  const float* axes_x[UOT_MAX_DIM];
  const float* axes_y[UOT_MAX_DIM];
  float2* U;
  float2* V;
  const float2* logp;
  const float2* logq;
  const float2* logdx;
  const float2* logdy;
  float2* pass[2];
  float* zbuf[2][UOT_MAX_DIM];
  int nstage, iters_per_stage, max_iter, check_every;
  double tol;
  const float2* eps_ff;      // [nstage+1]
  const float2* inv_eps_ff;  // [nstage+1]
  const float* k2;           // [nstage+1]
  const DivFF* F;            // [nstage+1][2]
  double* acc;               // [2] violation accumulators
  unsigned* bar;             // [2] barrier state (zero before the launch)
  int* status;               // [4] timeout, converged, final iterations, total iterations
  double* err_out;           // last measured violation
};

__global__ void __launch_bounds__(kNW * 32, 4)
    grid_solve_persistent(PersistArgs P) {
  extern __shared__ float4 sline[];
  __shared__ float2 part[kNW][kOutCTA];
  __shared__ float sshift[kOutCTA];
  __shared__ float sred[kNW];
  const ItemSmem sm{sline, part, sshift, sred};
  const int d = P.ndim;
  if (blockIdx.x == 0 && threadIdx.x < 2) P.acc[threadIdx.x] = 0.0;
  if (!grid_barrier(P.bar, P.status)) return;
  int total = 0, it_final = 0;
  bool stop = false;
  for (int s = 0; s <= P.nstage && !stop; ++s) {
    const int iters = (s < P.nstage) ? P.iters_per_stage : P.max_iter;
    const bool final_stage = (s == P.nstage);
    for (int it = 0; it < iters; ++it) {
      const bool check = final_stage && (((it + 1) % P.check_every == 0) || it == iters - 1);
      for (int pidx = 0; pidx < 2 * d; ++pidx) {
        const int dir = pidx / d, k = pidx % d, ax = d - 1 - k;
        const int* in_shape = dir == 0 ? P.shape_y : P.shape_x;
        const int* out_shape = dir == 0 ? P.shape_x : P.shape_y;
        int nlines = 1;
        for (int t = 0; t < ax; ++t) nlines *= in_shape[t];
        for (int t = ax + 1; t < d; ++t) nlines *= out_shape[t];
        PassArgs a;
        a.in = (k == 0) ? (dir == 0 ? P.V : P.U) : P.pass[(k - 1) & 1];
        a.logw = dir == 0 ? P.logdy : P.logdx;
        a.in_is_pot = (k == 0);
        a.nlines = nlines;
        a.nin = in_shape[ax];
        a.nout = out_shape[ax];
        a.yi = dir == 0 ? P.axes_y[ax] : P.axes_x[ax];
        a.xo = dir == 0 ? P.axes_x[ax] : P.axes_y[ax];
        a.inv_eps = P.inv_eps_ff[s];
        a.k2 = P.k2[s];
        a.zprev = P.zbuf[dir][k];
        a.use_prev = it > 0;
        a.zero_acc = nullptr;
        Epilogue e;
        memset(&e, 0, sizeof(e));
        e.ff = 1;
        e.eps_ff = P.eps_ff[s];
        e.inv_eps_ff = P.inv_eps_ff[s];
        if (k < d - 1) {
          e.mode = EPI_RAW;
          e.out = reinterpret_cast<double*>(P.pass[k & 1]);
        } else {
          e.mode = EPI_PROX;
          e.Fff = P.F[2 * s + dir];
          e.logp = reinterpret_cast<const double*>(dir == 0 ? P.logp : P.logq);
          e.pot = reinterpret_cast<double*>(dir == 0 ? P.U : P.V);
          e.logw = reinterpret_cast<const double*>(dir == 0 ? P.logdx : P.logdy);
          e.err = (dir == 0 && check) ? P.acc : nullptr;
        }
        const int nob = (a.nout + kOutCTA - 1) / kOutCTA;
        const int items = nlines * nob;
        for (int item = blockIdx.x; item < items; item += gridDim.x) {
          float num, den;
          grid_item_f32<false>(a, e, item / nob, 0, (item % nob) * kOutCTA, sm, num, den);
          if (e.err) block_add2f<kNW * 32>(num, den, e.err);
        }
        if (!grid_barrier(P.bar, P.status)) return;
      }
      ++total;
      if (final_stage) it_final = it + 1;
      if (check) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
          volatile double* acc = P.acc;
          const double num = acc[0], den = acc[1];
          const double err = (den > 0.0) ? num / den : 0.0;
          *P.err_out = err;
          P.status[1] = (it > 0 && P.tol > 0.0 && err <= P.tol) ? 1 : 0;
          acc[0] = 0.0;
          acc[1] = 0.0;
        }
        if (!grid_barrier(P.bar, P.status)) return;
        if (*(volatile int*)(P.status + 1)) {
          stop = true;
          break;
        }
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    P.status[2] = it_final;
    P.status[3] = total;
  }
}

}  // namespace

int grid_solve_persistent_ctas(int nin_max) {
  int nb = 0, dev = 0, sms = 0;
  const size_t smem = (size_t)nin_max * sizeof(float4);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(grid_solve_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, grid_solve_persistent, kNW * 32, smem) != cudaSuccess) return 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return nb * sms;
}

cudaError_t launch_grid_solve_persistent(const PersistLaunch& L, int grid, cudaStream_t s) {
  PersistArgs P;
  memset(&P, 0, sizeof(P));
  P.ndim = L.ndim;
  for (int k = 0; k < UOT_MAX_DIM; ++k) {
    P.shape_x[k] = L.shape_x[k];
    P.shape_y[k] = L.shape_y[k];
    P.axes_x[k] = (const float*)L.axes_x[k];
    P.axes_y[k] = (const float*)L.axes_y[k];
    P.zbuf[0][k] = L.zbuf[0][k];
    P.zbuf[1][k] = L.zbuf[1][k];
  }
  P.U = reinterpret_cast<float2*>(L.U);
  P.V = reinterpret_cast<float2*>(L.V);
  P.logp = reinterpret_cast<const float2*>(L.logp);
  P.logq = reinterpret_cast<const float2*>(L.logq);
  P.logdx = reinterpret_cast<const float2*>(L.logdx);
  P.logdy = reinterpret_cast<const float2*>(L.logdy);
  P.pass[0] = reinterpret_cast<float2*>(L.pass[0]);
  P.pass[1] = reinterpret_cast<float2*>(L.pass[1]);
  P.nstage = L.nstage;
  P.iters_per_stage = L.iters_per_stage;
  P.max_iter = L.max_iter;
  P.check_every = L.check_every;
  P.tol = L.tol;
  P.eps_ff = L.eps_ff;
  P.inv_eps_ff = L.inv_eps_ff;
  P.k2 = L.k2;
  P.F = L.F;
  P.acc = L.acc;
  P.bar = L.bar;
  P.status = L.status;
  P.err_out = L.err_out;
  int nin_max = 1;
  for (int k = 0; k < L.ndim; ++k) nin_max = std::max(nin_max, std::max(L.shape_x[k], L.shape_y[k]));
  const size_t smem = (size_t)nin_max * sizeof(float4);
  cudaError_t e = cudaFuncSetAttribute(grid_solve_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {&P};
  count_launches(1);
  e = cudaLaunchCooperativeKernel((const void*)grid_solve_persistent, dim3(grid), dim3(kNW * 32), args, smem, s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

namespace {

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
  if (epi.err) block_add2<WARPS * 32>(num, den, epi.err + 2 * bz);
}

}  // namespace

cudaError_t launch_grid_pass(int prec, const double* in, const double* logw, int in_is_pot,
                             int nlines, int nin, const void* yi, int nout, const void* xo,
                             double eps, int nbatch, const Epilogue& epi, cudaStream_t s,
                             float* zprev, int use_prev, double* zero_acc) {
  prof_mark_begin(PROF_GRID_PASS, s);
  count_launches(1);
  if (prec == UOT_F32) {
    dim3 grid((nout + kOutCTA - 1) / kOutCTA, nlines, nbatch);
    if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
    const size_t smem = (size_t)nin * sizeof(float4);
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(grid_pass_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
      if (e != cudaSuccess) return e;
    }
    PassArgs a;
    a.in = reinterpret_cast<const float2*>(in);
    a.logw = reinterpret_cast<const float2*>(logw);
    a.in_is_pot = in_is_pot;
    a.nlines = nlines;
    a.nin = nin;
    a.nout = nout;
    a.yi = (const float*)yi;
    a.xo = (const float*)xo;
    a.inv_eps = ff2(ff_make(1.0 / eps));
    a.k2 = (float)((double)kLog2e / eps);
    a.zprev = zprev;
    a.use_prev = use_prev;
    a.zero_acc = zero_acc;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kNW * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, grid_pass_f32, a, epi);
    if (e != cudaSuccess) return e;
  } else {
    constexpr int R = 2, WARPS = 4;
    dim3 grid((nout + 32 * R - 1) / (32 * R), (nlines + WARPS - 1) / WARPS, nbatch);
    if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
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

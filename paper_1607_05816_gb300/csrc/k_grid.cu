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

__global__ void __launch_bounds__(kNW * 32, 4)
    grid_pass_f32(PassArgs a, Epilogue epi) {
  extern __shared__ float4 sline[];  // nin x {t, t, y, y}
  __shared__ float2 part[kNW][kOutCTA];
  __shared__ float sshift[kOutCTA];
  __shared__ float sred[kNW];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int l = blockIdx.y;
  const int64_t bz = blockIdx.z;
  const int i0 = blockIdx.x * kOutCTA;
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

  pdl_wait();
  if (a.zero_acc && blockIdx.x == 0 && blockIdx.y == 0 && tid < 2) a.zero_acc[2 * bz + tid] = 0.0;
  pdl_launch_dependents();

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

  float num = 0.0f, den = 0.0f;
  if (mx == -INFINITY) {
    // b = 0 on the whole line: every sum is empty.
    if (owns) {
      if (zprev) zprev[my_pt] = -INFINITY;
      epilogue_apply(epi, bz, my_pt, ff_ninf(), pre, num, den);
    }
    if (epi.err) block_add2f<kNW * 32>(num, den, epi.err + 2 * bz);
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
  if (epi.err) block_add2f<kNW * 32>(num, den, epi.err + 2 * bz);
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

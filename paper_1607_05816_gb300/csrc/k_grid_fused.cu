// Two consecutive separable passes of the log-domain Gibbs operator fused on
// one grid line, for 2-D grids (FP32 path).
//
// A 2-D separable operator (Sec. 4.4) contracts one axis, then the other.
// Between the two passes of one half-step the data must be transposed, which
// needs every line of the first pass (a global dependency).  Between the
// half-steps it need not be: if the U-update ends with the pass whose lines
// are columns i2 of U (it contracts j1 and produces U[:, i2] on one line), and
// the V-update starts by contracting i1 -- the same column -- then the second
// pass of that line only needs the first pass's outputs of the same line.
// The same holds between the V-update's last pass (rows j1 of V) and the next
// U-update's first pass (contracting j2 along row j1).  So one Sinkhorn
// iteration is two kernels:
//
//   K_A, line i2:  P2  S[i1] = log sum_j1 exp(T1[i2][j1] - k (x_i1 - y_j1)^2)
//                      U[i1][i2] = prox_F1(...)                (+ violation)
//                  P3  T2[j1][i2] = log sum_i1 exp(U[i1][i2]/eps + log dx - k (y_j1 - x_i1)^2)
//   K_B, line j1:  P4  V[j1][j2] = prox_F2(log sum_i2 exp(T2[j1][i2] - k (y_j2 - x_i2)^2))
//                  P1  T1[i2][j1] = log sum_j2 exp(V[j1][j2]/eps + log dy - k (x_i2 - y_j2)^2)
//
// (contracting the V-update's axes in the order i1, i2 instead of i2, i1 is
// the same operator).  The second pass of each kernel reads its line from
// shared memory, where the first pass's epilogue left it.
//
// CTA = one line, 16 warps in two groups of 8; each group takes items of 128
// outputs in turn, its 8 warps splitting the contraction index and merging
// (max, sum) pairs through shared memory, 4 outputs per lane as two f32x2
// pairs.  Log-sum-exp shifts are the same pass's results from the previous
// call at the same eps, with a block-uniform exact fallback (as in k_grid.cu).
#include <string.h>

#include "uot_internal.cuh"

namespace uot {
namespace {


constexpr int kGW = 8;                 // warps per group
constexpr int kG = 2;                  // groups per CTA
constexpr int kFT = kGW * kG * 32;     // threads per CTA
constexpr int kIO = 128;               // outputs per item (4 per lane)

struct FSmem {
  float4* sline;                 // staged line {t, t, y, y}
  float2* line2;                 // second pass's line values (float-float)
  float2 (*part)[kGW][kIO];      // [kG][kGW][kIO] partial (max, sum)
  float (*sshift)[kIO];          // [kG][kIO]
  float* sred;                   // [16]
};

// Output i of a pass on line l: index i*nlines + l (transposed) or l*nout + i.
struct OutIdx {
  int row, nlines, l, nout;
  __device__ __forceinline__ int64_t operator()(int i) const {
    return row ? (int64_t)l * nout + i : (int64_t)i * nlines + l;
  }
};

__device__ __forceinline__ float cta_max(float v, float* sred) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = sred[0];
#pragma unroll
  for (int w = 1; w < kFT / 32; ++w) r = fmaxf(r, sred[w]);
  __syncthreads();  // sred is reused
  return r;
}

// All outputs of one pass over the staged line (t relative to mx, in log2
// units): z_i = mx + ln2 (M_i + log2 S_i) in natural units, handed to epi(i, z)
// by the thread that owns output i; zprev receives z.hi.
template <class Epi>
__device__ void line_pass(const FSmem& sm, int nin, int nout, const float* __restrict__ xo, float k2, float mx,
                          float* zprev, const OutIdx& oidx, bool spec, Epi&& epi) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = warp / kGW, gw = warp % kGW, gt = tid % (kGW * 32);
  if (mx == -INFINITY) {
    // b = 0 on the whole line: every sum is empty
    for (int i = tid; i < nout; i += kFT) {
      if (zprev) zprev[oidx(i)] = -INFINITY;
      epi(i, ff_ninf());
    }
    return;
  }
  const int nitems = (nout + kIO - 1) / kIO;
  const int rounds = (nitems + kG - 1) / kG;
  const int J = (nin + kGW - 1) / kGW;
  const int j0 = min(nin, gw * J), j1 = min(nin, j0 + J);
  const f2p nk2 = pk(-k2, -k2);
  const ff ln2 = ln2_ff();
  for (int r = 0; r < rounds; ++r) {
    const int item = r * kG + g;
    const bool has = item < nitems;
    const int i0 = item * kIO;
    float xq[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + lane + 32 * q;
      xq[q] = has ? xo[i < nout ? i : nout - 1] : 0.0f;
    }
    const bool owner = has && gt < kIO && i0 + gt < nout;
    if (gt < kIO) {
      float sh = 0.0f;
      if (owner && spec) {
        const float zp = zprev[oidx(i0 + gt)];
        sh = (zp == -INFINITY) ? 0.0f : (zp - mx) * kLog2e;
      }
      sm.sshift[g][gt] = sh;
    }
    __syncthreads();
    const f2p X0 = pk(xq[0], xq[1]), X1 = pk(xq[2], xq[3]);
    bool exact = !spec;
    for (int attempt = 0; attempt < 2; ++attempt) {
      if (has) {
        float mq[4];
        if (!exact) {
#pragma unroll
          for (int q = 0; q < 4; ++q) mq[q] = sm.sshift[g][lane + 32 * q];
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) mq[q] = -INFINITY;
#pragma unroll 4
          for (int j = j0; j < j1; ++j) {
            const float4 v = sm.sline[j];
            const f2p T = pk(v.x, v.y), Y = pk(v.z, v.w);
            const f2p D0 = sub2(X0, Y), D1 = sub2(X1, Y);
            const float2 A0 = upk(fma2(nk2, mul2(D0, D0), T));
            const float2 A1 = upk(fma2(nk2, mul2(D1, D1), T));
            mq[0] = fmaxf(mq[0], A0.x);
            mq[1] = fmaxf(mq[1], A0.y);
            mq[2] = fmaxf(mq[2], A1.x);
            mq[3] = fmaxf(mq[3], A1.y);
          }
        }
        const f2p MS0 = pk(mq[0] == -INFINITY ? 0.0f : mq[0], mq[1] == -INFINITY ? 0.0f : mq[1]);
        const f2p MS1 = pk(mq[2] == -INFINITY ? 0.0f : mq[2], mq[3] == -INFINITY ? 0.0f : mq[3]);
        f2p S0 = pk(0.0f, 0.0f), S1 = S0;
#pragma unroll 4
        for (int j = j0; j < j1; ++j) {
          const float4 v = sm.sline[j];
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
          sm.part[g][gw][lane + 32 * q] =
              make_float2(mq[q] == -INFINITY ? 0.0f : mq[q], mq[q] == -INFINITY ? 0.0f : sq[q]);
      }
      __syncthreads();
      bool bad = false;
      float Mo = -INFINITY, So = 0.0f;
      if (owner) {
#pragma unroll
        for (int w = 0; w < kGW; ++w) {
          const float2 pr = sm.part[g][w][gt];
          if (pr.y > 0.0f) Mo = fmaxf(Mo, pr.x);
        }
        if (Mo != -INFINITY) {
#pragma unroll
          for (int w = 0; w < kGW; ++w) {
            const float2 pr = sm.part[g][w][gt];
            if (pr.y > 0.0f) So += pr.y * ex2_approx(pr.x - Mo);
          }
        }
        if (!exact) bad = !(So >= 0x1p-90f && So <= 0x1p100f);
      }
      const int any_bad = __syncthreads_or(bad ? 1 : 0);
      if (any_bad && !exact) {
        exact = true;  // block-uniform: redo with exact maxima
        continue;
      }
      if (owner) {
        ff z = ff_ninf();
        if (So > 0.0f) z = ff_add_f(ff_add_f(ff_mul_f(ln2, Mo), mx), kLn2 * lg2_approx(So));
        if (zprev) zprev[oidx(i0 + gt)] = z.hi;
        epi(i0 + gt, z);
      }
      break;
    }
  }
}

__global__ void __launch_bounds__(kFT, 2) grid_fused2(FusedArgs a) {
  extern __shared__ float4 fsm[];
  __shared__ float2 part[kG][kGW][kIO];
  __shared__ float sshift[kG][kIO];
  __shared__ float sred[kFT / 32];
  const int l = blockIdx.x;
  const int tid = threadIdx.x;
  const int lmax = a.nin1 > a.nout1 ? a.nin1 : a.nout1;
  FSmem sm{fsm, reinterpret_cast<float2*>(fsm + lmax), part, sshift, sred};

  pdl_wait();
  if (a.zero_acc && blockIdx.x == 0 && tid < 2) a.zero_acc[tid] = 0.0;
  pdl_launch_dependents();

  // ---- pass 1: the line from global memory ----
  const float2* in = a.in1 + (int64_t)l * a.nin1;
  float mx = -INFINITY;
  for (int j = tid; j < a.nin1; j += kFT) {
    const float2 v = in[j];
    sm.sline[j] = make_float4(v.x, v.y, 0.0f, 0.0f);  // rewritten below by the same thread
    mx = fmaxf(mx, v.x);
  }
  mx = cta_max(mx, sred);
  if (mx != -INFINITY) {
    for (int j = tid; j < a.nin1; j += kFT) {
      const float4 v = sm.sline[j];
      const float t = (v.x == -INFINITY) ? -INFINITY : ((v.x - mx) + v.y) * kLog2e;
      const float y = a.y1[j];
      sm.sline[j] = make_float4(t, t, y, y);
    }
  }
  __syncthreads();
  float num = 0.0f, den = 0.0f;
  const OutIdx o1{a.out1_row, (int)gridDim.x, l, a.nout1};
  const ff eps1 = ffl(a.eps1_ff), ieps1 = ffl(a.inv_eps1_ff), ieps2 = ffl(a.inv_eps2_ff);
  line_pass(sm, a.nin1, a.nout1, a.x1, a.k2_1, mx, a.z1, o1, a.use_prev1 != 0, [&](int i, ff z) {
    const int64_t q = o1(i);
    const ff S = (z.hi == -INFINITY) ? ff_ninf() : ff_mul(z, eps1);
    const ff Un = prox_update_ff(a.F1, ffl(a.logp1[q]), S, eps1);
    if (a.err) {
      float va, vb;
      violation_terms_ff(ffl(a.pot1[q]), Un, S, ffl(a.logw1[q]), ieps1, va, vb);
      num += va;
      den += vb;
    }
    a.pot1[q] = ff2(Un);
    if (a.do2)
      sm.line2[i] = (Un.hi == -INFINITY) ? make_float2(-INFINITY, 0.0f)
                                         : ff2(ff_add(ff_mul(Un, ieps2), ffl(a.logw1[q])));
  });
  if (a.err) block_add2f<kFT>(num, den, a.err);
  if (!a.do2) return;
  __syncthreads();

  // ---- pass 2: the first pass's new potentials of this line ----
  float mx2 = -INFINITY;
  for (int j = tid; j < a.nout1; j += kFT) mx2 = fmaxf(mx2, sm.line2[j].x);
  mx2 = cta_max(mx2, sred);
  if (mx2 != -INFINITY) {
    for (int j = tid; j < a.nout1; j += kFT) {
      const float2 v = sm.line2[j];
      const float t = (v.x == -INFINITY) ? -INFINITY : ((v.x - mx2) + v.y) * kLog2e;
      const float y = a.x1[j];
      sm.sline[j] = make_float4(t, t, y, y);
    }
  }
  __syncthreads();
  const OutIdx o2{0, (int)gridDim.x, l, a.nout2};
  line_pass(sm, a.nout1, a.nout2, a.x2, a.k2_2, mx2, a.z2, o2, a.use_prev2 != 0,
            [&](int i, ff z) { a.out2[o2(i)] = ff2(z); });
}

}  // namespace

size_t grid_fused2_smem(int nin1, int nout1) {
  const int lmax = nin1 > nout1 ? nin1 : nout1;
  return (size_t)lmax * sizeof(float4) + (size_t)nout1 * sizeof(float2);
}

cudaError_t launch_grid_fused2(const FusedArgs& a, cudaStream_t s) {
  const size_t smem = grid_fused2_smem(a.nin1, a.nout1);
  if (smem > 48 * 1024) {
    cudaError_t e = smem_at_least(grid_fused2, smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(a.nlines);
  cfg.blockDim = dim3(kFT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  prof_mark_begin(PROF_GRID_PASS, s);
  count_launches(1);
  cudaError_t e = cudaLaunchKernelEx(&cfg, grid_fused2, a);
  if (e != cudaSuccess) return e;
  prof_mark_end(PROF_GRID_PASS, s);
  return cudaGetLastError();
}

}  // namespace uot

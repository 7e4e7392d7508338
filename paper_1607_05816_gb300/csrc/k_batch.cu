// Many independent unbalanced OT problems between point clouds in one
// persistent launch (uneven sizes).
//
// Each CTA takes problems from a device work counter in a host-given order
// (largest n*m first) and runs the whole scaling iteration of that problem
// (eq. S, Sec. 3.3, log form of Sec. 4.3, eps-scaling of Sec. 4.4) with its
// potentials held in shared memory:
//
//   S_i = eps log sum_j exp((V_j - |x_i - y_j|^2)/eps) dy_j ;  U_i = prox_F1(S_i)
//   T_j = eps log sum_i exp((U_i - |x_i - y_j|^2)/eps) dx_i ;  V_j = prox_F2(T_j)
//
// until the marginal violation of the problem is <= tol or the iteration cap.
// There is no communication between CTAs except the atomic work counter, so
// no CTA ever waits on another one.
//
// Per-point state is float-float (no FP64 pipe use); the cost is recomputed on
// the fly from the coordinates; each lane evaluates 4 outputs as two packed
// f32x2 pairs; the log-sum-exp shift of every output is its value from the
// previous iteration of the same stage, with an exact per-warp fallback.
#include <string.h>

#include "uot_internal.cuh"

namespace uot {
namespace {

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

constexpr int kNT = 256;  // threads per CTA

__device__ __forceinline__ float block_max(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = red[0];
#pragma unroll
  for (int w = 1; w < kNT / 32; ++w) r = fmaxf(r, red[w]);
  return r;
}

__device__ __forceinline__ float2 block_sum2(float a, float b, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = a;
    red[kNT / 32 + (threadIdx.x >> 5)] = b;
  }
  __syncthreads();
  float ra = 0.0f, rb = 0.0f;
#pragma unroll
  for (int w = 0; w < kNT / 32; ++w) {
    ra += red[w];
    rb += red[kNT / 32 + w];
  }
  return make_float2(ra, rb);
}

}  // namespace

// One half-step of one problem inside a CTA: outputs on side "out" (nout
// points, coordinates xo), inputs on side "in" (nin points, coordinates yi,
// potential Win, log weights lwin).  Writes Wout (float-float, shared memory),
// zprev (float, shared memory) and returns the violation terms if `check`.
__device__ void batch_half(int d, int nin, int nout, const float* __restrict__ xo,
                           const float* __restrict__ yi, const float2* Win,
                           const float2* __restrict__ lwin, float2* Wout,
                           const float2* __restrict__ lpout, const float2* __restrict__ lwout,
                           float* zprev, bool use_prev, float4* stage, float* red,
                           const DivFF& F, float2 eps_ff, float2 inv_eps_ff, float k2,
                           bool check, float& num, float& den) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // input line: L_j = W_j/eps + log w_j; shift by the block maximum of the high parts
  float mx = -INFINITY;
  for (int j = tid; j < nin; j += kNT) {
    const ff w = ffl(Win[j]);
    if (w.hi != -INFINITY) mx = fmaxf(mx, ff_add(ff_mul(w, ffl(inv_eps_ff)), ffl(lwin[j])).hi);
  }
  mx = block_max(mx, red);
  if (mx == -INFINITY) {
    // b = 0 everywhere: every sum is empty
    for (int i = tid; i < nout; i += kNT) {
      const ff Un = prox_update_ff(F, ffl(lpout[i]), ff_ninf(), ffl(eps_ff));
      if (check) {
        float a, b;
        violation_terms_ff(ffl(Wout[i]), Un, ff_ninf(), ffl(lwout[i]), ffl(inv_eps_ff), a, b);
        num += a;
        den += b;
      }
      Wout[i] = ff2(Un);
      zprev[i] = -INFINITY;
    }
    __syncthreads();
    return;
  }
  for (int j = tid; j < nin; j += kNT) {
    const ff w = ffl(Win[j]);
    float t = -INFINITY;
    if (w.hi != -INFINITY) {
      const ff L = ff_add(ff_mul(w, ffl(inv_eps_ff)), ffl(lwin[j]));
      t = ((L.hi - mx) + L.lo) * kLog2e;
    }
    const float c0 = yi[(int64_t)j * d];
    const float c1 = d > 1 ? yi[(int64_t)j * d + 1] : 0.0f;
    const float c2 = d > 2 ? yi[(int64_t)j * d + 2] : 0.0f;
    stage[2 * j] = make_float4(t, t, c0, c0);
    stage[2 * j + 1] = make_float4(c1, c1, c2, c2);
  }
  __syncthreads();

  const f2p nk2 = pk(-k2, -k2);
  const f2p zero2 = pk(0.0f, 0.0f);
  const ff eps = ffl(eps_ff);
  const ff ln2 = ff{0.693147182464599609375f, -1.904654323148236017e-09f};
  // each warp handles blocks of 128 outputs: lane owns o = base + lane + 32 q
  for (int base = warp * 128; base < nout; base += (kNT / 32) * 128) {
    float xc[3][4];
    bool valid[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = base + lane + 32 * q;
      valid[q] = i < nout;
      const int ii = valid[q] ? i : nout - 1;
#pragma unroll
      for (int k = 0; k < 3; ++k) xc[k][q] = (k < d) ? xo[(int64_t)ii * d + k] : 0.0f;
    }
    const f2p XA0 = pk(xc[0][0], xc[0][1]), XA1 = pk(xc[1][0], xc[1][1]), XA2 = pk(xc[2][0], xc[2][1]);
    const f2p XB0 = pk(xc[0][2], xc[0][3]), XB1 = pk(xc[1][2], xc[1][3]), XB2 = pk(xc[2][2], xc[2][3]);
    float mq[4];
    bool exact = !use_prev;
    if (!exact) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float zp = valid[q] ? zprev[base + lane + 32 * q] : mx;
        mq[q] = (zp == -INFINITY) ? 0.0f : (zp - mx) * kLog2e;
      }
    }
    float sq[4];
    for (int attempt = 0; attempt < 2; ++attempt) {
      if (exact) {
        float m4[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
#pragma unroll 2
        for (int j = 0; j < nin; ++j) {
          const float4 s0 = stage[2 * j], s1 = stage[2 * j + 1];
          const f2p T = pk(s0.x, s0.y), Y0 = pk(s0.z, s0.w), Y1 = pk(s1.x, s1.y), Y2 = pk(s1.z, s1.w);
          f2p DA = sub2(XA0, Y0), DB = sub2(XB0, Y0);
          f2p QA = mul2(DA, DA), QB = mul2(DB, DB);
          if (d > 1) {
            DA = sub2(XA1, Y1);
            DB = sub2(XB1, Y1);
            QA = fma2(DA, DA, QA);
            QB = fma2(DB, DB, QB);
          }
          if (d > 2) {
            DA = sub2(XA2, Y2);
            DB = sub2(XB2, Y2);
            QA = fma2(DA, DA, QA);
            QB = fma2(DB, DB, QB);
          }
          const float2 A = upk(fma2(nk2, QA, T)), B = upk(fma2(nk2, QB, T));
          m4[0] = fmaxf(m4[0], A.x);
          m4[1] = fmaxf(m4[1], A.y);
          m4[2] = fmaxf(m4[2], B.x);
          m4[3] = fmaxf(m4[3], B.y);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) mq[q] = m4[q];
      }
      const f2p MA = pk(mq[0] == -INFINITY ? 0.0f : mq[0], mq[1] == -INFINITY ? 0.0f : mq[1]);
      const f2p MB = pk(mq[2] == -INFINITY ? 0.0f : mq[2], mq[3] == -INFINITY ? 0.0f : mq[3]);
      f2p SA = zero2, SB = zero2;
#pragma unroll 2
      for (int j = 0; j < nin; ++j) {
        const float4 s0 = stage[2 * j], s1 = stage[2 * j + 1];
        const f2p T = pk(s0.x, s0.y), Y0 = pk(s0.z, s0.w), Y1 = pk(s1.x, s1.y), Y2 = pk(s1.z, s1.w);
        f2p DA = sub2(XA0, Y0), DB = sub2(XB0, Y0);
        f2p QA = mul2(DA, DA), QB = mul2(DB, DB);
        if (d > 1) {
          DA = sub2(XA1, Y1);
          DB = sub2(XB1, Y1);
          QA = fma2(DA, DA, QA);
          QB = fma2(DB, DB, QB);
        }
        if (d > 2) {
          DA = sub2(XA2, Y2);
          DB = sub2(XB2, Y2);
          QA = fma2(DA, DA, QA);
          QB = fma2(DB, DB, QB);
        }
        const float2 A = upk(fma2(nk2, QA, sub2(T, MA)));
        const float2 B = upk(fma2(nk2, QB, sub2(T, MB)));
        SA = add2(SA, pk(ex2_approx(A.x), ex2_approx(A.y)));
        SB = add2(SB, pk(ex2_approx(B.x), ex2_approx(B.y)));
      }
      const float2 a = upk(SA), b = upk(SB);
      sq[0] = a.x;
      sq[1] = a.y;
      sq[2] = b.x;
      sq[3] = b.y;
      bool bad = false;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (valid[q] && !exact && !(sq[q] >= 0x1p-90f && sq[q] <= 0x1p100f)) bad = true;
      if (__any_sync(0xffffffffu, bad)) {
        exact = true;  // warp-uniform retry with exact maxima
        continue;
      }
      break;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (!valid[q]) continue;
      const int i = base + lane + 32 * q;
      ff z = ff_ninf();
      if (mq[q] != -INFINITY && sq[q] > 0.0f)
        z = ff_add_f(ff_add_f(ff_mul_f(ln2, mq[q]), mx), kLn2 * lg2_approx(sq[q]));
      zprev[i] = z.hi;
      const ff S = (z.hi == -INFINITY) ? ff_ninf() : ff_mul(z, eps);
      const ff Un = prox_update_ff(F, ffl(lpout[i]), S, eps);
      if (check) {
        float va, vb;
        violation_terms_ff(ffl(Wout[i]), Un, S, ffl(lwout[i]), ffl(inv_eps_ff), va, vb);
        num += va;
        den += vb;
      }
      Wout[i] = ff2(Un);
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kNT) batch_solve(BatchArgs a) {
  extern __shared__ float4 smem4[];
  __shared__ float red[2 * kNT / 32];
  __shared__ int s_prob;
  __shared__ int s_stop;
  const int tid = threadIdx.x;
  // shared layout: stage [2*max(nmax,mmax)] float4 | U [nmax] ff | V [mmax] ff | zU [nmax] | zV [mmax]
  const int lmax = a.nmax > a.mmax ? a.nmax : a.mmax;
  float4* stage = smem4;
  float2* U = reinterpret_cast<float2*>(stage + 2 * lmax);
  float2* V = U + a.nmax;
  float* zU = reinterpret_cast<float*>(V + a.mmax);
  float* zV = zU + a.nmax;
  for (;;) {
    if (tid == 0) {
      const int t = atomicAdd(a.next, 1);
      s_prob = (t < a.nprob) ? a.order[t] : -1;
    }
    __syncthreads();
    const int k = s_prob;
    if (k < 0) break;
    const int n = a.n[k], m = a.m[k];
    const int64_t xo = a.xoff[k], yo = a.yoff[k];
    const float* xk = a.x + xo * a.d;
    const float* yk = a.y + yo * a.d;
    for (int i = tid; i < n; i += kNT) U[i] = make_float2(0.0f, 0.0f);
    for (int j = tid; j < m; j += kNT) V[j] = make_float2(0.0f, 0.0f);
    __syncthreads();
    int it_final = 0;
    float err = INFINITY;
    for (int s = 0; s <= a.nstage; ++s) {
      const int iters = (s < a.nstage) ? a.iters_per_stage : a.max_iter;
      const DivFF F1 = a.divs[((int64_t)s * a.nprob + k) * 2];
      const DivFF F2 = a.divs[((int64_t)s * a.nprob + k) * 2 + 1];
      const float2 eps = a.eps_ff[s], ieps = a.inv_eps_ff[s];
      const float k2 = a.k2[s];
      for (int it = 0; it < iters; ++it) {
        const bool final_stage = (s == a.nstage);
        const bool check = final_stage && (((it + 1) % a.check_every == 0) || it == iters - 1);
        float num = 0.0f, den = 0.0f;
        batch_half(a.d, m, n, xk, yk, V, a.logdy + yo, U, a.logp + xo, a.logdx + xo, zU, it > 0,
                   stage, red, F1, eps, ieps, k2, check, num, den);
        float dn = 0.0f, dd = 0.0f;
        batch_half(a.d, n, m, yk, xk, U, a.logdx + xo, V, a.logq + yo, a.logdy + yo, zV, it > 0,
                   stage, red, F2, eps, ieps, k2, false, dn, dd);
        if (final_stage) it_final = it + 1;
        if (check) {
          const float2 tot = block_sum2(num, den, red);
          err = (tot.y > 0.0f) ? tot.x / tot.y : 0.0f;
          if (tid == 0) s_stop = (it > 0 && a.tol > 0.0f && err <= a.tol) ? 1 : 0;
          __syncthreads();
          if (s_stop) break;
        }
      }
    }
    for (int i = tid; i < n; i += kNT) {
      const float2 u = U[i];
      a.Uout[xo + i] = (u.x == -INFINITY) ? u.x : u.x + u.y;
    }
    for (int j = tid; j < m; j += kNT) {
      const float2 v = V[j];
      a.Vout[yo + j] = (v.x == -INFINITY) ? v.x : v.x + v.y;
    }
    if (tid == 0) {
      a.iters_out[k] = it_final;
      a.err_out[k] = err;
    }
    __syncthreads();
  }
}

size_t batch_smem_bytes(int nmax, int mmax) {
  const int lmax = nmax > mmax ? nmax : mmax;
  return (size_t)2 * lmax * sizeof(float4) + (size_t)(nmax + mmax) * (sizeof(float2) + sizeof(float));
}

cudaError_t launch_batch(const BatchArgs& a, int grid, cudaStream_t s) {
  const size_t smem = batch_smem_bytes(a.nmax, a.mmax);
  cudaError_t e = cudaFuncSetAttribute(batch_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  count_launches(1);
  batch_solve<<<grid, kNT, smem, s>>>(a);
  return cudaGetLastError();
}

int batch_ctas_per_sm(int nmax, int mmax) {
  int nb = 0;
  const size_t smem = batch_smem_bytes(nmax, mmax);
  if (cudaFuncSetAttribute(batch_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_solve, kNT, smem) != cudaSuccess) return 0;
  return nb;
}

}  // namespace uot

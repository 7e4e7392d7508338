// Many independent unbalanced OT problems between point clouds in one
// persistent launch (uneven sizes).
//
// Each CTA takes problems from a device work counter in a host-given order
// (largest n*m first) and runs the whole scaling iteration of that problem
// (eq. S, Sec. 3.3, log form of Sec. 4.3, eps-scaling of Sec. 4.4):
//
//   S_i = eps log sum_j exp((V_j - |x_i - y_j|^2)/eps) dy_j ;  U_i = prox_F1(S_i)
//   T_j = eps log sum_i exp((U_i - |x_i - y_j|^2)/eps) dx_i ;  V_j = prox_F2(T_j)
//
// until the marginal violation of the problem is <= tol or the iteration cap.
// There is no communication between CTAs except the atomic work counter, so
// no CTA ever waits on another one.
//
// Per half-step the CTA stages the input side {t_j, y_j} in shared memory
// (the only per-problem data kept there, so several CTAs share an SM) and
// evaluates the outputs in blocks of 128 (4 per lane, two packed f32x2
// pairs).  A problem with fewer output blocks than warps splits the
// contraction index across warps and merges their partial (max, sum) pairs
// through shared memory, so small problems keep every warp busy.  Per-point
// state (potentials, last log-sums) is float-float in global memory (it stays
// in L2); the cost is recomputed on the fly from the coordinates; the
// log-sum-exp shift of every output is its value from the previous iteration
// of the same stage, with an exact fallback when a sum leaves [2^-90, 2^100].
//
// Two CTA sizes (8 or 16 warps) are compiled for each dimension; the first
// call with a given (d, largest n, largest m) times both on a sample of the
// batch and keeps the faster one.
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "uot_internal.cuh"

namespace uot {
namespace {


constexpr int kOB = 128;  // outputs per warp block (4 per lane)

// Second staged vector of an input point: the remaining coordinates, paired.
template <int D>
struct Stage1 {
  typedef float2 T;  // {y1, y1}
};
template <>
struct Stage1<3> {
  typedef float4 T;  // {y1, y1, y2, y2}
};

template <int D>
__host__ __device__ constexpr size_t stage1_bytes() {
  return D == 1 ? 0 : sizeof(typename Stage1<D>::T);
}

template <int D, int NW>
size_t smem_bytes(int lmax) {
  return (size_t)lmax * (sizeof(float4) + stage1_bytes<D>()) + (size_t)NW * kOB * sizeof(float2);
}

template <int NT>
__device__ __forceinline__ float block_max(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = red[0];
#pragma unroll
  for (int w = 1; w < NT / 32; ++w) r = fmaxf(r, red[w]);
  return r;
}

template <int NT>
__device__ __forceinline__ float2 block_sum2(float a, float b, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = a;
    red[NT / 32 + (threadIdx.x >> 5)] = b;
  }
  __syncthreads();
  float ra = 0.0f, rb = 0.0f;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) {
    ra += red[w];
    rb += red[NT / 32 + w];
  }
  return make_float2(ra, rb);
}

// Output coordinates of a lane's 4 outputs as f32x2 pairs (outputs 0,1 | 2,3).
struct XPairs {
  f2p A[3], B[3];
};

template <int D>
__device__ __forceinline__ void load_x(const float* __restrict__ xo, int nout, int base, int lane, XPairs& X,
                                       bool (&valid)[4]) {
  float xc[3][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = base + lane + 32 * q;
    valid[q] = i < nout;
    const int ii = valid[q] ? i : nout - 1;
#pragma unroll
    for (int k = 0; k < 3; ++k) xc[k][q] = (k < D) ? xo[(int64_t)ii * D + k] : 0.0f;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    X.A[k] = pk(xc[k][0], xc[k][1]);
    X.B[k] = pk(xc[k][2], xc[k][3]);
  }
}

// Squared distances of the pairs A, B to staged point j, times -k2, plus Tm.
template <int D>
__device__ __forceinline__ void term_exponents(const float4* st0, const typename Stage1<D>::T* st1, int j,
                                               const XPairs& X, f2p nk2, f2p MA, f2p MB, f2p& EA, f2p& EB) {
  const float4 s0 = st0[j];
  const f2p T = pk(s0.x, s0.y), Y0 = pk(s0.z, s0.w);
  f2p DA = sub2(X.A[0], Y0), DB = sub2(X.B[0], Y0);
  f2p QA = mul2(DA, DA), QB = mul2(DB, DB);
  if constexpr (D >= 2) {
    const auto s1 = st1[j];
    const f2p Y1 = pk(s1.x, s1.y);
    DA = sub2(X.A[1], Y1);
    DB = sub2(X.B[1], Y1);
    QA = fma2(DA, DA, QA);
    QB = fma2(DB, DB, QB);
    if constexpr (D == 3) {
      const f2p Y2 = pk(s1.z, s1.w);
      DA = sub2(X.A[2], Y2);
      DB = sub2(X.B[2], Y2);
      QA = fma2(DA, DA, QA);
      QB = fma2(DB, DB, QB);
    }
  }
  EA = fma2(nk2, QA, sub2(T, MA));
  EB = fma2(nk2, QB, sub2(T, MB));
}

// Log2-sum-exp of a lane's 4 outputs over staged inputs [j0, j1): with
// `exact` the per-output maxima are computed first (returned in mq), else
// the shifts in mq are used.  Returns the shifted sums in sq.
template <int D>
__device__ __forceinline__ void sweep(const float4* st0, const typename Stage1<D>::T* st1, int j0, int j1,
                                      const XPairs& X, f2p nk2, bool exact, float (&mq)[4], float (&sq)[4]) {
  const f2p zero2 = pk(0.0f, 0.0f);
  if (exact) {
    float m4[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
#pragma unroll 2
    for (int j = j0; j < j1; ++j) {
      f2p EA, EB;
      term_exponents<D>(st0, st1, j, X, nk2, zero2, zero2, EA, EB);
      const float2 A = upk(EA), B = upk(EB);
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
  for (int j = j0; j < j1; ++j) {
    f2p EA, EB;
    term_exponents<D>(st0, st1, j, X, nk2, MA, MB, EA, EB);
    const float2 A = upk(EA), B = upk(EB);
    SA = add2(SA, pk(ex2_approx(A.x), ex2_approx(A.y)));
    SB = add2(SB, pk(ex2_approx(B.x), ex2_approx(B.y)));
  }
  const float2 a = upk(SA), b = upk(SB);
  sq[0] = a.x;
  sq[1] = a.y;
  sq[2] = b.x;
  sq[3] = b.y;
}

// Operands of one half-step: outputs on one side of the current problem,
// inputs on the other.
struct Half {
  int nin, nout;
  const float* xo;      // [nout][D] output coordinates
  const float* yi;      // [nin][D] input coordinates
  const float2* Win;    // [nin] input potential (float-float)
  const float2* lwin;   // [nin] log weights of the inputs
  float2* Wout;         // [nout] output potential (read: old value, written: new)
  const float2* lpout;  // [nout] log densities of the outputs
  const float2* lwout;  // [nout] log weights of the outputs
  float* zprev;         // [nout] last log-sums (shift of the next half-step)
  bool use_prev, check;
  DivFF F;
  float2 eps_ff, inv_eps_ff;
  float k2;
};

// Result of one output: log-sum z = mx + ln2 (Mo + log2 So), prox update and
// violation terms.
__device__ __forceinline__ void output_epilogue(const Half& h, int i, float Mo, float So, float mx, float& num,
                                                float& den) {
  const ff ln2 = ln2_ff();
  ff z = ff_ninf();
  if (Mo != -INFINITY && So > 0.0f) z = ff_add_f(ff_add_f(ff_mul_f(ln2, Mo), mx), kLn2 * lg2_approx(So));
  h.zprev[i] = z.hi;
  const ff eps = ffl(h.eps_ff);
  const ff S = (z.hi == -INFINITY) ? ff_ninf() : ff_mul(z, eps);
  const ff Un = prox_update_ff(h.F, ffl(h.lpout[i]), S, eps);
  if (h.check) {
    float va, vb;
    violation_terms_ff(ffl(h.Wout[i]), Un, S, ffl(h.lwout[i]), ffl(h.inv_eps_ff), va, vb);
    num += va;
    den += vb;
  }
  h.Wout[i] = ff2(Un);
}

template <int D, int NW>
__device__ void half_step(const Half& h, float4* st0, typename Stage1<D>::T* st1, float2* part, float* red,
                          float& num, float& den) {
  constexpr int NT = NW * 32;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nin = h.nin, nout = h.nout;
  // ---- input line L_j = W_j/eps + log w_j (float-float), staged relative to its maximum ----
  float mx = -INFINITY;
  for (int j = tid; j < nin; j += NT) {
    const ff w = ffl(h.Win[j]);
    ff L = ff_ninf();
    if (w.hi != -INFINITY) L = ff_add(ff_mul(w, ffl(h.inv_eps_ff)), ffl(h.lwin[j]));
    st0[j] = make_float4(L.hi, L.lo, 0.0f, 0.0f);  // rewritten below by the same thread
    mx = fmaxf(mx, L.hi);
  }
  mx = block_max<NT>(mx, red);
  if (mx == -INFINITY) {
    // b = 0 everywhere: every sum is empty
    for (int i = tid; i < nout; i += NT) output_epilogue(h, i, -INFINITY, 0.0f, 0.0f, num, den);
    __syncthreads();
    return;
  }
  for (int j = tid; j < nin; j += NT) {
    const float4 v = st0[j];
    const float t = (v.x == -INFINITY) ? -INFINITY : ((v.x - mx) + v.y) * kLog2e;
    const float c0 = h.yi[(int64_t)j * D];
    st0[j] = make_float4(t, t, c0, c0);
    if constexpr (D == 2) {
      const float c1 = h.yi[(int64_t)j * D + 1];
      st1[j] = make_float2(c1, c1);
    }
    if constexpr (D == 3) {
      const float c1 = h.yi[(int64_t)j * D + 1], c2 = h.yi[(int64_t)j * D + 2];
      st1[j] = make_float4(c1, c1, c2, c2);
    }
  }
  __syncthreads();

  const f2p nk2 = pk(-h.k2, -h.k2);
  const int nblk = (nout + kOB - 1) / kOB;
  const int split = nblk >= NW ? 1 : NW / nblk;
  if (split == 1) {
    // one warp per block of 128 outputs, the whole contraction each
    for (int b = warp; b < nblk; b += NW) {
      const int base = b * kOB;
      XPairs X;
      bool valid[4];
      load_x<D>(h.xo, nout, base, lane, X, valid);
      float mq[4], sq[4];
      bool exact = !h.use_prev;
      if (!exact) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float zp = valid[q] ? h.zprev[base + lane + 32 * q] : mx;
          mq[q] = (zp == -INFINITY) ? 0.0f : (zp - mx) * kLog2e;
        }
      }
      for (int attempt = 0; attempt < 2; ++attempt) {
        sweep<D>(st0, st1, 0, nin, X, nk2, exact, mq, sq);
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
      for (int q = 0; q < 4; ++q)
        if (valid[q]) output_epilogue(h, base + lane + 32 * q, mq[q], mq[q] == -INFINITY ? 0.0f : sq[q], mx, num, den);
    }
    __syncthreads();
    return;
  }

  // fewer blocks than warps: `split` warps share each block's contraction
  const bool active = warp < nblk * split;
  const int b = warp % nblk, r = warp / nblk;
  const int J = (nin + split - 1) / split;
  const int j0 = min(nin, r * J), j1 = min(nin, j0 + J);
  const int base = b * kOB;
  XPairs X;
  bool valid[4];
  load_x<D>(h.xo, nout, base, lane, X, valid);
  float shift[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float zp = (h.use_prev && valid[q]) ? h.zprev[base + lane + 32 * q] : mx;
    shift[q] = (zp == -INFINITY) ? 0.0f : (zp - mx) * kLog2e;
  }
  constexpr int OWN = (NW * kOB + NT - 1) / NT;  // combined outputs per thread (4)
  float Mo[OWN], So[OWN];
  bool exact = !h.use_prev;
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (active) {
      float mq[4], sq[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) mq[q] = shift[q];
      sweep<D>(st0, st1, j0, j1, X, nk2, exact, mq, sq);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const bool empty = mq[q] == -INFINITY;
        part[warp * kOB + lane + 32 * q] = make_float2(empty ? 0.0f : mq[q], empty ? 0.0f : sq[q]);
      }
    }
    __syncthreads();
    bool bad = false;
#pragma unroll
    for (int u = 0; u < OWN; ++u) {
      const int o = tid + u * NT;  // output o of the CTA's nblk*128
      Mo[u] = -INFINITY;
      So[u] = 0.0f;
      if (o < nblk * kOB && o < nout) {
        const int bo = o / kOB, oo = o % kOB;
        for (int rr = 0; rr < split; ++rr) {
          const float2 pr = part[(rr * nblk + bo) * kOB + oo];
          if (pr.y > 0.0f) Mo[u] = fmaxf(Mo[u], pr.x);
        }
        if (Mo[u] != -INFINITY) {
          for (int rr = 0; rr < split; ++rr) {
            const float2 pr = part[(rr * nblk + bo) * kOB + oo];
            if (pr.y > 0.0f) So[u] += pr.y * ex2_approx(pr.x - Mo[u]);
          }
        }
        if (!exact && !(So[u] >= 0x1p-90f && So[u] <= 0x1p100f)) bad = true;
      }
    }
    const int any_bad = __syncthreads_or(bad ? 1 : 0);
    if (any_bad && !exact) {
      exact = true;  // block-uniform retry with exact maxima
      continue;
    }
    break;
  }
#pragma unroll
  for (int u = 0; u < OWN; ++u) {
    const int o = tid + u * NT;
    if (o < nblk * kOB && o < nout) output_epilogue(h, o, Mo[u], So[u], mx, num, den);
  }
  __syncthreads();
}

// log sum_i e^{lw_i + lp_i - W_i / lam} over one side of the CTA's problem
// (entries with lp_i = -inf or W_i = -inf take no part); every thread gets
// the result.  Shifts in FP64, exponentials of shifted differences in FP32.
template <int NW>
__device__ double block_side_lse(const float2* W, const float2* lp, const float2* lw, int len, double inv_lam,
                                 double* red) {
  constexpr int NT = NW * 32;
  double mx = -kInf, sm = 0.0;
  for (int i = threadIdx.x; i < len; i += NT) {
    const float2 l = lp[i], w = W[i];
    if (l.x == -INFINITY || w.x == -INFINITY) continue;
    const float2 g = lw[i];
    const double t = ((double)g.x + (double)g.y) + ((double)l.x + (double)l.y) - ((double)w.x + (double)w.y) * inv_lam;
    if (t > mx) {
      sm = sm * (double)expf((float)(mx - t)) + 1.0;
      mx = t;
    } else {
      sm += (double)expf((float)(t - mx));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double m2 = __shfl_down_sync(0xffffffffu, mx, o);
    double s2 = __shfl_down_sync(0xffffffffu, sm, o);
    if (m2 > mx) {
      const double tm = mx, ts = sm;
      mx = m2;
      sm = s2;
      m2 = tm;
      s2 = ts;
    }
    if (m2 != -kInf) sm += s2 * (double)expf((float)(m2 - mx));
  }
  __syncthreads();  // red is free
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = mx;
    red[NW + (threadIdx.x >> 5)] = sm;
  }
  __syncthreads();
  double M = -kInf, S = 0.0;
  for (int w = 0; w < NW; ++w) M = fmax(M, red[w]);
  if (M == -kInf) return -kInf;
  for (int w = 0; w < NW; ++w)
    if (red[w] != -kInf) S += red[NW + w] * (double)expf((float)(red[w] - M));
  return M + log(S);
}

// Translation step (uot_opts.translate; not in the paper: the translation-
// invariant formulation of Sejourne, Vialard, Peyre 2022): U += c, V -= c with
// c = lam1 lam2 / (lam1 + lam2) (log A - log B), the exact maximum of the dual
// along that direction for KL penalties; A = sum dx p e^{-U/lam1}, B = sum dy
// q e^{-V/lam2}.  The plan is unchanged.
template <int NW>
__device__ void translate_problem(float2* U, float2* V, const float2* lpU, const float2* lwU, const float2* lpV,
                                  const float2* lwV, int n, int m, double2 lam, double* red) {
  constexpr int NT = NW * 32;
  const double la = block_side_lse<NW>(U, lpU, lwU, n, 1.0 / lam.x, red);
  const double lb = block_side_lse<NW>(V, lpV, lwV, m, 1.0 / lam.y, red);
  const double c = (la != -kInf && lb != -kInf) ? lam.x * lam.y / (lam.x + lam.y) * (la - lb) : 0.0;
  const ff cp = ff_make(c), cn = ff_make(-c);
  for (int i = threadIdx.x; i < n; i += NT) {
    const float2 u = U[i];
    if (!isinf(u.x)) U[i] = ff2(ff_add(ffl(u), cp));
  }
  for (int j = threadIdx.x; j < m; j += NT) {
    const float2 v = V[j];
    if (!isinf(v.x)) V[j] = ff2(ff_add(ffl(v), cn));
  }
  __syncthreads();
}

template <int D, int NW>
__global__ void __launch_bounds__(NW * 32, NW == 8 ? 3 : 2) batch_solve(BatchArgs a) {
  constexpr int NT = NW * 32;
  typedef typename Stage1<D>::T S1;
  extern __shared__ float4 smem4[];
  __shared__ float red[2 * NW];
  __shared__ int s_prob;
  __shared__ int s_stop;
  __shared__ double tr_red[2 * NW];
  const int tid = threadIdx.x;
  const int lmax = a.nmax > a.mmax ? a.nmax : a.mmax;
  float4* st0 = smem4;
  S1* st1 = reinterpret_cast<S1*>(st0 + lmax);
  float2* part = reinterpret_cast<float2*>(reinterpret_cast<char*>(st0 + lmax) + (size_t)lmax * stage1_bytes<D>());
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
    const float* xk = a.x + xo * D;
    const float* yk = a.y + yo * D;
    float2* U = a.Uff + xo;
    float2* V = a.Vff + yo;
    for (int i = tid; i < n; i += NT) U[i] = make_float2(0.0f, 0.0f);
    for (int j = tid; j < m; j += NT) V[j] = make_float2(0.0f, 0.0f);
    __syncthreads();
    int it_final = 0;
    float err = INFINITY;
    Half h1, h2;
    h1.nin = m;
    h1.nout = n;
    h1.xo = xk;
    h1.yi = yk;
    h1.Win = V;
    h1.lwin = a.logdy + yo;
    h1.Wout = U;
    h1.lpout = a.logp + xo;
    h1.lwout = a.logdx + xo;
    h1.zprev = a.zU + xo;
    h2.nin = n;
    h2.nout = m;
    h2.xo = yk;
    h2.yi = xk;
    h2.Win = U;
    h2.lwin = a.logdx + xo;
    h2.Wout = V;
    h2.lpout = a.logq + yo;
    h2.lwout = a.logdy + yo;
    h2.zprev = a.zV + yo;
    h2.check = false;
    for (int s = 0; s <= a.nstage; ++s) {
      const int iters = (s < a.nstage) ? a.iters_per_stage : a.max_iter;
      h1.F = a.divs[((int64_t)s * a.ndiv + k) * 2];
      h2.F = a.divs[((int64_t)s * a.ndiv + k) * 2 + 1];
      h1.eps_ff = h2.eps_ff = a.eps_ff[s];
      h1.inv_eps_ff = h2.inv_eps_ff = a.inv_eps_ff[s];
      h1.k2 = h2.k2 = a.k2[s];
      for (int it = 0; it < iters; ++it) {
        const bool final_stage = (s == a.nstage);
        const bool check = final_stage && (((it + 1) % a.check_every == 0) || it == iters - 1);
        h1.use_prev = h2.use_prev = it > 0;
        h1.check = check;
        float num = 0.0f, den = 0.0f;
        half_step<D, NW>(h1, st0, st1, part, red, num, den);
        float dn = 0.0f, dd = 0.0f;
        half_step<D, NW>(h2, st0, st1, part, red, dn, dd);
        if (a.translate && (final_stage ? check : (it + 1) % a.check_every == 0))
          translate_problem<NW>(U, V, a.logp + xo, a.logdx + xo, a.logq + yo, a.logdy + yo, n, m, a.lam[k],
                                tr_red);
        if (final_stage) it_final = it + 1;
        if (check) {
          const float2 tot = block_sum2<NT>(num, den, red);
          err = (tot.y > 0.0f) ? tot.x / tot.y : 0.0f;
          if (tid == 0) s_stop = (it > 0 && a.tol > 0.0f && err <= a.tol) ? 1 : 0;
          __syncthreads();
          if (s_stop) break;
        }
      }
    }
    for (int i = tid; i < n; i += NT) {
      const float2 u = U[i];
      if (a.Uout64)
        a.Uout64[xo + i] = (u.x == -INFINITY) ? -kInf : (double)u.x + (double)u.y;
      else
        a.Uout[xo + i] = (u.x == -INFINITY) ? u.x : u.x + u.y;
    }
    for (int j = tid; j < m; j += NT) {
      const float2 v = V[j];
      if (a.Vout64)
        a.Vout64[yo + j] = (v.x == -INFINITY) ? -kInf : (double)v.x + (double)v.y;
      else
        a.Vout[yo + j] = (v.x == -INFINITY) ? v.x : v.x + v.y;
    }
    if (tid == 0) {
      a.iters_out[k] = it_final;
      a.err_out[k] = err;
    }
    __syncthreads();
  }
}

// ---- variants: (dimension, warps per CTA) ----
constexpr int kVariantWarps[2] = {8, 16};

template <int D, int NW>
cudaError_t launch_variant(const BatchArgs& a, int grid, cudaStream_t s) {
  const int lmax = std::max(a.nmax, a.mmax);
  const size_t smem = smem_bytes<D, NW>(lmax);
  cudaError_t e = smem_at_least(batch_solve<D, NW>, smem);
  if (e != cudaSuccess) return e;
  batch_solve<D, NW><<<grid, NW * 32, smem, s>>>(a);
  return cudaGetLastError();
}

template <int D, int NW>
int ctas_variant(int nmax, int mmax) {
  const size_t smem = smem_bytes<D, NW>(std::max(nmax, mmax));
  int nb = 0;
  if (smem_at_least(batch_solve<D, NW>, smem) !=
      cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_solve<D, NW>, NW * 32, smem) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return nb;
}

cudaError_t launch_any(const BatchArgs& a, int variant, int grid, cudaStream_t s) {
  switch (a.d * 2 + variant) {
    case 2: return launch_variant<1, 8>(a, grid, s);
    case 3: return launch_variant<1, 16>(a, grid, s);
    case 4: return launch_variant<2, 8>(a, grid, s);
    case 5: return launch_variant<2, 16>(a, grid, s);
    case 6: return launch_variant<3, 8>(a, grid, s);
    case 7: return launch_variant<3, 16>(a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

int ctas_any(int d, int variant, int nmax, int mmax) {
  switch (d * 2 + variant) {
    case 2: return ctas_variant<1, 8>(nmax, mmax);
    case 3: return ctas_variant<1, 16>(nmax, mmax);
    case 4: return ctas_variant<2, 8>(nmax, mmax);
    case 5: return ctas_variant<2, 16>(nmax, mmax);
    case 6: return ctas_variant<3, 8>(nmax, mmax);
    case 7: return ctas_variant<3, 16>(nmax, mmax);
    default: return 0;
  }
}

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return sms;
}

struct BKey {
  int dev, d, nmax, mmax;
  bool operator<(const BKey& o) const {
    if (dev != o.dev) return dev < o.dev;
    if (d != o.d) return d < o.d;
    if (nmax != o.nmax) return nmax < o.nmax;
    return mmax < o.mmax;
  }
};
struct BEntry {
  int variant;
  float ms[2];
  int sample;
};
std::mutex g_bmu;
std::map<BKey, BEntry> g_btuned;
int g_bforced = -1;  // forced variant, -1: tuned

// Times both CTA sizes on a sample of the batch: every (nprob/S)-th problem
// of the size-ordered queue, six iterations at the first eps, no tolerance
// stop.  The sample's outputs land in the caller's output and state buffers,
// which the full solve overwrites afterwards.
BEntry tune_batch(const BatchArgs& full, const int* h_order, cudaStream_t s) {
  BEntry ent;
  ent.variant = 0;
  ent.ms[0] = ent.ms[1] = -1.0f;
  const int sms = sm_count();
  const int S = std::min(full.nprob, std::max(1, 2 * sms));
  ent.sample = S;
  std::vector<int> samp(S);
  for (int t = 0; t < S; ++t) samp[t] = h_order[(int64_t)t * full.nprob / S];
  int* d_samp = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ok = cudaMallocAsync(&d_samp, S * sizeof(int), s) == cudaSuccess &&
            cudaMemcpyAsync(d_samp, samp.data(), S * sizeof(int), cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  if (ok) {
    BatchArgs a = full;
    a.nprob = S;
    a.order = d_samp;
    a.nstage = 0;
    a.max_iter = 6;
    a.tol = 0.0f;
    a.check_every = 1 << 30;
    a.translate = 0;
    float best = 1e30f;
    for (int v = 0; v < 2; ++v) {
      const int per = ctas_any(a.d, v, a.nmax, a.mmax);
      if (per < 1) continue;
      const int grid = std::min(S, per * sms);
      float tmin = 1e30f;
      bool vok = true;
      for (int rep = 0; rep < 3 && vok; ++rep) {  // the first run warms up
        vok = cudaMemsetAsync(a.next, 0, sizeof(int), s) == cudaSuccess && cudaEventRecord(e0, s) == cudaSuccess &&
              launch_any(a, v, grid, s) == cudaSuccess && cudaEventRecord(e1, s) == cudaSuccess &&
              cudaEventSynchronize(e1) == cudaSuccess;
        float ms = 0.0f;
        vok = vok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        if (vok && rep > 0) tmin = std::min(tmin, ms);
      }
      if (!vok) {
        (void)cudaGetLastError();
        continue;
      }
      ent.ms[v] = tmin;
      if (tmin < best) {
        best = tmin;
        ent.variant = v;
      }
    }
    // the 8-warp CTA stays unless the other is more than 3% faster
    if (ent.ms[0] > 0.0f && ent.ms[0] <= 1.03f * best) ent.variant = 0;
  }
  (void)cudaGetLastError();
  if (d_samp) cudaFreeAsync(d_samp, s);
  cudaStreamSynchronize(s);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  (void)cudaGetLastError();
  return ent;
}

}  // namespace

int batch_force_warps(int warps) {
  std::lock_guard<std::mutex> lk(g_bmu);
  if (warps == 0) {
    g_bforced = -1;
    return 0;
  }
  for (int v = 0; v < 2; ++v) {
    if (kVariantWarps[v] == warps) {
      g_bforced = v;
      return 0;
    }
  }
  return -1;
}

int batch_pick_variant(const BatchArgs& a, const int* h_order, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_bmu);
  if (g_bforced >= 0) return g_bforced;
  BKey key;
  if (cudaGetDevice(&key.dev) != cudaSuccess) return 0;
  key.d = a.d;
  key.nmax = a.nmax;
  key.mmax = a.mmax;
  auto it = g_btuned.find(key);
  if (it != g_btuned.end()) return it->second.variant;
  if (!grid_autotune_enabled()) return 0;
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess || st != cudaStreamCaptureStatusNone) {
    (void)cudaGetLastError();
    return 0;
  }
  const BEntry ent = tune_batch(a, h_order, s);
  g_btuned[key] = ent;
  return ent.variant;
}

std::string batch_tune_table() {
  std::lock_guard<std::mutex> lk(g_bmu);
  std::string s;
  char buf[256];
  for (const auto& kv : g_btuned) {
    snprintf(buf, sizeof(buf), "dev%d batch d=%d nmax=%d mmax=%d sample=%d -> warps=%d; 8:%.3fms 16:%.3fms\n",
             kv.first.dev, kv.first.d, kv.first.nmax, kv.first.mmax, kv.second.sample,
             kVariantWarps[kv.second.variant], kv.second.ms[0], kv.second.ms[1]);
    s += buf;
  }
  return s;
}

int batch_ctas_per_sm(int d, int variant, int nmax, int mmax) { return ctas_any(d, variant, nmax, mmax); }

cudaError_t launch_batch(const BatchArgs& a, int variant, int grid, cudaStream_t s) {
  count_launches(1);
  return launch_any(a, variant, grid, s);
}

}  // namespace uot

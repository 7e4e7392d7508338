// FP32 log-domain Gibbs operator for point clouds (cost |x - y|^2 recomputed on
// the fly, never stored), split into two kernels:
//
//  points_blockmax: per-block maxima of L_j = W_j/eps + log w_j (the shift of
//    the staged values).
//  points_partial: CTA = (1024 outputs, one chunk of the inputs).  The chunk's
//    shifted log-values t_j and coordinates are staged in shared memory as
//    packed pairs; each warp owns 128 outputs (4 per lane, two f32x2 pairs) and
//    sweeps the chunk.  The log-sum-exp shift of an output is its result from
//    the previous call at the same eps; a warp whose partial sum overflows
//    redoes the chunk with the exact chunk maximum.  Writes (shift, sum) per
//    (chunk, output).
//  points_combine: one warp per output merges the chunks' pairs; if the
//    merged sum underflowed (shift far above the result) the warp recomputes
//    that output exactly over all inputs; then the epilogue (Table 1 row,
//    violation terms) runs on the float-float result.
//
// Work: n m exponentials per call, bound by the SFU rate.
#include <string.h>

#include "uot_internal.cuh"

namespace uot {
namespace {


constexpr int kNW = 8;                 // warps per CTA
constexpr int kOutBlk = kNW * 128;     // outputs per CTA
constexpr int kMaxBlk = 1024;          // inputs per block of the max reduction

// The cost is evaluated from coordinate differences, -k |x - y|^2 with
// x - y formed first: the expanded form -k|x|^2 + 2k x.y - k|y|^2 needs fewer
// operations but cancels exponent parts of size ~k |x|^2 in FP32, and at
// eps = 1e-3 in three dimensions that noise kept the marginal violation above
// 1e-6 (measured), so it is not used.

__device__ __forceinline__ ff load_L_pt(const float2* W, const float2* lw, int64_t j, float2 inv_eps) {
  const ff w = ffl(W[j]);
  if (w.hi == -INFINITY) return ff_ninf();
  return ff_add(ff_mul(w, ffl(inv_eps)), ffl(lw[j]));
}

// Per-block maxima of the high parts of L_j = W_j/eps + log w_j.
__global__ void __launch_bounds__(256)
    points_blockmax(const float2* __restrict__ W, const float2* __restrict__ lw, int nin,
                    float2 inv_eps, float* __restrict__ bmax) {
  __shared__ float red[8];
  float m = -INFINITY;
  const int j0 = blockIdx.x * kMaxBlk;
  for (int j = j0 + threadIdx.x; j < min(nin, j0 + kMaxBlk); j += 256) m = fmaxf(m, load_L_pt(W, lw, j, inv_eps).hi);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float r = red[0];
    for (int w = 1; w < 8; ++w) r = fmaxf(r, red[w]);
    bmax[blockIdx.x] = r;
  }
}

__device__ __forceinline__ float all_max(const float* bmax, int nb) {
  float m = -INFINITY;
  for (int b = 0; b < nb; ++b) m = fmaxf(m, bmax[b]);
  return m;
}

struct PtArgs {
  const float* x;     // [nout][d]  output points
  const float* y;     // [nin][d]   input points
  int d, nout, nin, chunk, nbmax;
  const float2* W;    // [nin] float-float input potentials
  const float2* lw;   // [nin] float-float log weights
  float2 inv_eps;
  const float* bmax;  // [nbmax] block maxima of L
  float k2;           // log2(e)/eps
  const float* zprev; // [nout] previous result (natural log), or NULL
  int use_prev;
  float2* part;       // [nchunks][nout] (shift, sum) in log2 units relative to Lmax
};

template <int D>
__global__ void __launch_bounds__(kNW * 32)
    points_partial(PtArgs a) {
  extern __shared__ float4 st[];  // 2 x chunk float4: {t,t,y0,y0}, {y1,y1,y2,y2}
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c = blockIdx.y;
  const int j0 = c * a.chunk, j1 = min(a.nin, j0 + a.chunk);
  constexpr int d = D;  // compile-time: no dimension tests in the sweeps
  const float k2 = a.k2;
  const float Lmax = all_max(a.bmax, a.nbmax);
  for (int j = j0 + tid; j < j1; j += kNW * 32) {
    const ff L = load_L_pt(a.W, a.lw, j, a.inv_eps);
    const float c0 = a.y[(int64_t)j * d];
    const float c1 = d > 1 ? a.y[(int64_t)j * d + 1] : 0.0f;
    const float c2 = d > 2 ? a.y[(int64_t)j * d + 2] : 0.0f;
    const float t = (L.hi == -INFINITY || Lmax == -INFINITY) ? -INFINITY : ((L.hi - Lmax) + L.lo) * kLog2e;
    st[2 * (j - j0)] = make_float4(t, t, c0, c0);
    st[2 * (j - j0) + 1] = make_float4(c1, c1, c2, c2);
  }
  __syncthreads();
  const int base = blockIdx.x * kOutBlk + warp * 128;
  if (base >= a.nout) return;
  float xc[3][4];
  bool valid[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = base + lane + 32 * q;
    valid[q] = i < a.nout;
    const int ii = valid[q] ? i : a.nout - 1;
#pragma unroll
    for (int k = 0; k < 3; ++k) xc[k][q] = (k < d) ? a.x[(int64_t)ii * d + k] : 0.0f;
  }
  const f2p XA0 = pk(xc[0][0], xc[0][1]), XA1 = pk(xc[1][0], xc[1][1]), XA2 = pk(xc[2][0], xc[2][1]);
  const f2p XB0 = pk(xc[0][2], xc[0][3]), XB1 = pk(xc[1][2], xc[1][3]), XB2 = pk(xc[2][2], xc[2][3]);
  const f2p nk2 = pk(-k2, -k2);
  const int nj = j1 - j0;
  float mq[4], sq[4];
  bool exact = !(a.use_prev && a.zprev);
  if (!exact) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float zp = valid[q] ? a.zprev[base + lane + 32 * q] : Lmax;
      mq[q] = (zp == -INFINITY) ? 0.0f : (zp - Lmax) * kLog2e;
    }
  }
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (exact) {
      float m4[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
#pragma unroll 2
      for (int j = 0; j < nj; ++j) {
        const float4 s0 = st[2 * j], s1 = st[2 * j + 1];
        const f2p T = pk(s0.x, s0.y), Y0 = pk(s0.z, s0.w), Y1 = pk(s1.x, s1.y), Y2 = pk(s1.z, s1.w);
        f2p DA = sub2(XA0, Y0), DB = sub2(XB0, Y0);
        f2p QA = mul2(DA, DA), QB = mul2(DB, DB);
        if constexpr (d > 1) {
          DA = sub2(XA1, Y1);
          DB = sub2(XB1, Y1);
          QA = fma2(DA, DA, QA);
          QB = fma2(DB, DB, QB);
        }
        if constexpr (d > 2) {
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
    f2p SA = pk(0.0f, 0.0f), SB = SA;
#pragma unroll 8
    for (int j = 0; j < nj; ++j) {
      const float4 s0 = st[2 * j], s1 = st[2 * j + 1];
      const f2p T = pk(s0.x, s0.y), Y0 = pk(s0.z, s0.w), Y1 = pk(s1.x, s1.y), Y2 = pk(s1.z, s1.w);
      f2p DA = sub2(XA0, Y0), DB = sub2(XB0, Y0);
      f2p QA = mul2(DA, DA), QB = mul2(DB, DB);
      if constexpr (d > 1) {
        DA = sub2(XA1, Y1);
        DB = sub2(XB1, Y1);
        QA = fma2(DA, DA, QA);
        QB = fma2(DB, DB, QB);
      }
      if constexpr (d > 2) {
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
    const float2 s01 = upk(SA), s23 = upk(SB);
    sq[0] = s01.x;
    sq[1] = s01.y;
    sq[2] = s23.x;
    sq[3] = s23.y;
    bool bad = false;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (valid[q] && !exact && !(sq[q] <= 0x1p100f)) bad = true;  // overflow or NaN
    if (__any_sync(0xffffffffu, bad)) {
      exact = true;
      continue;
    }
    break;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (!valid[q]) continue;
    const int i = base + lane + 32 * q;
    a.part[(int64_t)c * a.nout + i] = (mq[q] == -INFINITY) ? make_float2(0.0f, 0.0f) : make_float2(mq[q], sq[q]);
  }
}

struct CombArgs {
  const float* x;
  const float* y;
  int d, nout, nin, nchunks, nbmax;
  const float2* W;
  const float2* lw;
  float2 inv_eps;
  const float* bmax;
  float k2;
  const float2* part;
  float* zprev;  // written (NULL: not kept)
};

// One warp per output: merge chunk partials, exact recomputation if the
// merged sum underflowed, then the epilogue.
__global__ void __launch_bounds__(256)
    points_combine(CombArgs a, Epilogue epi) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + warp;
  float num = 0.0f, den = 0.0f;
  const float Lmax = all_max(a.bmax, a.nbmax);
  if (i < a.nout) {
    float M = -INFINITY;
    for (int c = lane; c < a.nchunks; c += 32) {
      const float2 pr = a.part[(int64_t)c * a.nout + i];
      if (pr.y > 0.0f) M = fmaxf(M, pr.x);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) M = fmaxf(M, __shfl_xor_sync(0xffffffffu, M, o));
    float S = 0.0f;
    if (M != -INFINITY)
      for (int c = lane; c < a.nchunks; c += 32) {
        const float2 pr = a.part[(int64_t)c * a.nout + i];
        if (pr.y > 0.0f) S += pr.y * ex2_approx(pr.x - M);
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
    if (!(S >= 0x1p-90f) && Lmax != -INFINITY) {
      // the shift was far above the result: exact log-sum-exp over all inputs
      float xi[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) xi[k] = (k < a.d) ? a.x[(int64_t)i * a.d + k] : 0.0f;
      auto arg = [&](int j) -> float {
        const ff L = load_L_pt(a.W, a.lw, j, a.inv_eps);
        if (L.hi == -INFINITY) return -INFINITY;
        float q = 0.0f;
        for (int k = 0; k < a.d; ++k) {
          const float t = xi[k] - a.y[(int64_t)j * a.d + k];
          q = fmaf(t, t, q);
        }
        return fmaf(-a.k2, q, ((L.hi - Lmax) + L.lo) * kLog2e);
      };
      float m = -INFINITY;
      for (int j = lane; j < a.nin; j += 32) m = fmaxf(m, arg(j));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      float s = 0.0f;
      if (m != -INFINITY)
        for (int j = lane; j < a.nin; j += 32) s += ex2_approx(arg(j) - m);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      M = m;
      S = s;
    }
    if (lane == 0) {
      ff z = ff_ninf();
      if (Lmax != -INFINITY && M != -INFINITY && S > 0.0f) {
        const ff ln2 = ln2_ff();
        z = ff_add_f(ff_add_f(ff_mul_f(ln2, M), Lmax), kLn2 * lg2_approx(S));
      }
      if (a.zprev) a.zprev[i] = z.hi;
      apply_epilogue_ff(epi, 0, i, z, num, den);
    }
  }
  if (epi.err) block_add2f<256>(num, den, epi.err);
}

// ---------------------------------------------------------------------------
// Precise pass (float-float exponents), used where the FP32 check of a
// verified solve stalls: with lambda >> eps the staged values t_j and the
// costs k |x_i - y_j|^2 are both large and their FP32 difference loses
// ulp(|t_j|) per term.  Here each coordinate difference is an exact TwoSum,
// the squared distance and its product with k = log2(e)/eps are float-float,
// the running maximum is float-float; only the final small difference is
// rounded for ex2.  Eight threads per output, each an online log-sum-exp over
// every eighth input, merged by shuffles (16 outputs per CTA); the inputs are
// staged in chunks of kFfpChunk through shared memory; then the same
// float-float epilogue as points_combine.
// ---------------------------------------------------------------------------
constexpr int kFfpThreads = 128;
constexpr int kFfpSplit = 8;                          // threads per output (input slices)
constexpr int kFfpOut = kFfpThreads / kFfpSplit;      // outputs per CTA
constexpr int kFfpChunk = 1024;
constexpr ff kLog2eFFp{1.44269502162933349609375f, 1.925963033500011e-08f};

struct FfpArgs {
  const float* x;
  const float* y;
  int d, nout, nin, nbmax;
  const float2* W;
  const float2* lw;
  float2 inv_eps;
  const float* bmax;
  float* zprev;
};

// Merges the running (max, sum) of another slice (float-float max).
__device__ __forceinline__ void ffp_merge(float& mh, float& ml, float& sum, float mh2, float ml2, float s2) {
  if (mh2 == -INFINITY) return;
  if (mh == -INFINITY) {
    mh = mh2;
    ml = ml2;
    sum = s2;
    return;
  }
  const ff dq = ff_two_sum(mh2, -mh);
  const float dm = dq.hi + (dq.lo + (ml2 - ml));
  if (dm > 0.0f) {
    sum = fmaf(sum, ex2_approx(-dm), s2);
    mh = mh2;
    ml = ml2;
  } else {
    sum = fmaf(s2, ex2_approx(dm), sum);
  }
}

template <int D>
__global__ void __launch_bounds__(kFfpThreads) points_ffp(FfpArgs a, Epilogue epi) {
  __shared__ float4 st[kFfpChunk];  // {t.hi, t.lo, y0, y1}
  __shared__ float sy2[D == 3 ? kFfpChunk : 1];
  const int slice = threadIdx.x % kFfpSplit;
  const int i = blockIdx.x * kFfpOut + threadIdx.x / kFfpSplit;
  const bool owns = i < a.nout;
  const float Lmax = all_max(a.bmax, a.nbmax);
  const ff k2 = ff_mul(ffl(a.inv_eps), kLog2eFFp);
  float xi[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int k = 0; k < D; ++k) xi[k] = owns ? a.x[(int64_t)i * D + k] : 0.0f;
  float mh = -INFINITY, ml = 0.0f, sum = 0.0f;
  if (Lmax != -INFINITY) {
    for (int j0 = 0; j0 < a.nin; j0 += kFfpChunk) {
      const int nj = min(kFfpChunk, a.nin - j0);
      __syncthreads();  // the previous chunk is no longer read
      for (int jj = threadIdx.x; jj < nj; jj += kFfpThreads) {
        const int j = j0 + jj;
        const ff L = load_L_pt(a.W, a.lw, j, a.inv_eps);
        const ff t = (L.hi == -INFINITY) ? ff_ninf() : ff_mul(ff_add_f(L, -Lmax), kLog2eFFp);
        const float y0 = a.y[(int64_t)j * D];
        const float y1 = D > 1 ? a.y[(int64_t)j * D + 1] : 0.0f;
        st[jj] = make_float4(t.hi, t.lo, y0, y1);
        if (D == 3) sy2[jj] = a.y[(int64_t)j * D + 2];
      }
      __syncthreads();
      for (int jj = slice; jj < nj; jj += kFfpSplit) {
        const float4 tj = st[jj];
        if (tj.x == -INFINITY) continue;
        // q = |x_i - y_j|^2 as an unnormalised float-float pair
        float qh = 0.0f, ql = 0.0f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float yk = (k == 0) ? tj.z : (k == 1) ? tj.w : sy2[D == 3 ? jj : 0];
          const ff dk = ff_two_sum(xi[k], -yk);
          const float p = dk.hi * dk.hi;
          const float pe = fmaf(dk.hi, dk.hi, -p) + 2.0f * dk.hi * dk.lo;
          const ff sq = ff_two_sum(qh, p);
          qh = sq.hi;
          ql += sq.lo + pe;
        }
        const float ch = k2.hi * qh;
        const float ce = fmaf(k2.hi, qh, -ch) + fmaf(k2.hi, ql, k2.lo * qh);
        const ff sa = ff_two_sum(tj.x, -ch);
        ffp_merge(mh, ml, sum, sa.hi, sa.lo + (tj.y - ce), 1.0f);
      }
    }
  }
  // the slices of an output are kFfpSplit consecutive lanes
#pragma unroll
  for (int o = 1; o < kFfpSplit; o <<= 1) {
    const float mh2 = __shfl_xor_sync(0xffffffffu, mh, o);
    const float ml2 = __shfl_xor_sync(0xffffffffu, ml, o);
    const float s2 = __shfl_xor_sync(0xffffffffu, sum, o);
    ffp_merge(mh, ml, sum, mh2, ml2, s2);
  }
  float num = 0.0f, den = 0.0f;
  if (owns && slice == 0) {
    ff z = ff_ninf();
    if (mh != -INFINITY && sum > 0.0f) {
      const ff m2 = ff_add_f(ff_fast_two_sum(mh, ml), lg2_approx(sum));  // log2 units, relative to Lmax
      z = ff_add_f(ff_mul(m2, ln2_ff()), Lmax);
    }
    if (a.zprev) a.zprev[i] = z.hi;
    apply_epilogue_ff(epi, 0, i, z, num, den);
  }
  if (epi.err) block_add2f<kFfpThreads>(num, den, epi.err);
}

}  // namespace

// The chunk index is the launch grid's second dimension.
constexpr int kMaxPointChunks = 65535;

// Inputs of at most 65535 chunks of 1024: larger clouds take the general
// FP32 row kernel instead of the chunked one.
bool points_chunks_fit(int nin) { return (nin + 1023) / 1024 <= kMaxPointChunks; }

// Chunking of the inputs: at most 1024 inputs per chunk; among the counts up
// to 1.5x the least (and at most kMaxPointChunks), the one that best balances
// the grid (output blocks x chunks) over the 152 SMs -- the slowest SM sets
// the pass time -- with a small charge for each extra chunk (more partial sums
// to combine).
int points_nchunks(int nin, int nout) {
  const int least = (nin + 1023) / 1024;
  const int oblocks = (nout + kOutBlk - 1) / kOutBlk;
  const int most = std::min(least + least / 2, std::max(least, kMaxPointChunks));
  int best = least;
  double best_waste = 2.0;
  for (int c = least; c <= most; ++c) {
    if (c > 1 && (nin + c - 1) / c < 256) break;  // chunks of at least 256 inputs
    const long g = (long)oblocks * c;
    const long rounds = (g + 151) / 152;
    const double waste = (double)(rounds * 152 - g) / (double)(rounds * 152) + 0.1 * (c - least) / least;
    if (waste < best_waste - 1e-9) {
      best_waste = waste;
      best = c;
    }
  }
  return best;
}

cudaError_t launch_points(const float* x, const float* y, int d, int nout, int nin,
                          const double* W, const double* logw, double eps, float* bmax,
                          float* zprev, int use_prev, float2* part, const Epilogue& epi,
                          cudaStream_t s) {
  const int nchunks = points_nchunks(nin, nout);
  const int chunk = (nin + nchunks - 1) / nchunks;
  const int nbmax = (nin + kMaxBlk - 1) / kMaxBlk;
  const float2 inv_eps = ff2(ff_make(1.0 / eps));
  const float2* Wf = reinterpret_cast<const float2*>(W);
  const float2* lwf = reinterpret_cast<const float2*>(logw);
  prof_mark_begin(PROF_ROWS, s);
  count_launches(3);
  points_blockmax<<<nbmax, 256, 0, s>>>(Wf, lwf, nin, inv_eps, bmax);
  PtArgs a;
  a.x = x;
  a.y = y;
  a.d = d;
  a.nout = nout;
  a.nin = nin;
  a.chunk = chunk;
  a.nbmax = nbmax;
  a.W = Wf;
  a.lw = lwf;
  a.inv_eps = inv_eps;
  a.bmax = bmax;
  a.k2 = (float)((double)kLog2e / eps);
  a.zprev = zprev;
  a.use_prev = use_prev;
  a.part = part;
  const size_t smem = (size_t)2 * chunk * sizeof(float4);
  dim3 grid((nout + kOutBlk - 1) / kOutBlk, nchunks);
  auto run = [&](auto kern) -> cudaError_t {
    cudaError_t e = smem_at_least(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kNW * 32, smem, s>>>(a);
    return cudaGetLastError();
  };
  cudaError_t e = (d == 1) ? run(points_partial<1>) : (d == 2) ? run(points_partial<2>) : run(points_partial<3>);
  if (e != cudaSuccess) return e;
  CombArgs b;
  b.x = x;
  b.y = y;
  b.d = d;
  b.nout = nout;
  b.nin = nin;
  b.nchunks = nchunks;
  b.nbmax = nbmax;
  b.W = Wf;
  b.lw = lwf;
  b.inv_eps = inv_eps;
  b.bmax = bmax;
  b.k2 = a.k2;
  b.part = part;
  b.zprev = zprev;
  points_combine<<<(nout + 7) / 8, 256, 0, s>>>(b, epi);
  prof_mark_end(PROF_ROWS, s);
  return cudaGetLastError();
}

cudaError_t launch_points_ffp(const float* x, const float* y, int d, int nout, int nin, const double* W,
                              const double* logw, double eps, float* bmax, float* zprev, const Epilogue& epi,
                              cudaStream_t s) {
  if (d < 1 || d > 3) return cudaErrorInvalidValue;
  FfpArgs a;
  a.x = x;
  a.y = y;
  a.d = d;
  a.nout = nout;
  a.nin = nin;
  a.nbmax = (nin + kMaxBlk - 1) / kMaxBlk;
  a.W = reinterpret_cast<const float2*>(W);
  a.lw = reinterpret_cast<const float2*>(logw);
  a.inv_eps = ff2(ff_make(1.0 / eps));
  a.bmax = bmax;
  a.zprev = zprev;
  prof_mark_begin(PROF_ROWS, s);
  count_launches(2);
  points_blockmax<<<a.nbmax, 256, 0, s>>>(a.W, a.lw, nin, a.inv_eps, bmax);
  const dim3 grid((nout + kFfpOut - 1) / kFfpOut);
  if (d == 1) points_ffp<1><<<grid, kFfpThreads, 0, s>>>(a, epi);
  else if (d == 2) points_ffp<2><<<grid, kFfpThreads, 0, s>>>(a, epi);
  else points_ffp<3><<<grid, kFfpThreads, 0, s>>>(a, epi);
  prof_mark_end(PROF_ROWS, s);
  return cudaGetLastError();
}

}  // namespace uot

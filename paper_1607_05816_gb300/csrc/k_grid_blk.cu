// Block-stabilised separable grid pass (FP32) for uniform axes.
//
// A pass of the separable log-domain Gibbs operator (Sec. 4.4, in the log
// domain of Sec. 4.3) is, for every line l,
//
//   z[i][l] = log sum_j exp(L[l][j] - (x_i - y_j)^2 / eps).
//
// When both axes are uniform with one spacing h (x_i = x_0 + i h, y_j =
// y_0 + j h), split the outputs into blocks I of BI = 32 points and the inputs
// into blocks J of BJ points, with midpoints c_I, c_J and D = c_I - c_J.
// With ic, jc the offsets of i, j from their midpoints in units of h,
// x_i - y_j = D + h (ic - jc), and in log2 units (k2 = log2(e)/eps, t = L log2 e)
//
//   t_j - k2 (x_i - y_j)^2 = [t_j + c jc] + [alpha + beta ic] - k2 h^2 (ic - jc)^2,
//   c = 2 k2 D h,  alpha = -k2 D^2,  beta = -2 k2 D h.
//
// The first bracket depends on the line and the input, the second on the
// output only, the last on ic - jc only.  So each block pair contributes
//
//   2^{M + alpha + beta ic} P_li,   P_li = sum_{j in J} A_lj G(ic - jc),
//   A_lj = 2^{t_j + c jc - M} (M its largest exponent, so 0 < A <= 1),
//   G(d) = 2^{-k2 h^2 d^2},
//
// a product of two factors in (0, 1]: one FMA per kernel term, instead of one
// exponential, plus BJ exponentials per (line, input block, output block) for
// A and one per (line, output, input block) to merge the block sums in a
// running (max, scaled sum) pair.  This is the absorption of Sec. 4.3 applied
// per block: the large parts of the exponent are kept in the log domain, only
// bounded factors are multiplied.
//
// G stays a normal FP32 number (>= 2^-90) while k2 h^2 dmax^2 <= 90, dmax the
// largest |ic - jc| of a block pair; every product dropped below 2^-126 is then
// below 2^-30 of its block's sum.  Passes that miss this condition use the
// log-sum-exp tiles of k_grid.cu.
//
// Layout: a CTA = 4 lines x one output block I; its JS warps split the input
// blocks and merge their (max, sum) pairs at the end, and the 4 x 32 results
// are finished (epilogue) by warps 0..3, one line each.  A lane owns one
// output of the block for the CTA's 4 lines; G(lane - jj + const) for the BJ
// inputs of a block sits in registers (the same values for every block
// pair), and the A values of a block are broadcast from shared memory, 4
// lines per load.  At these sizes a pass is latency-bound (one wave of CTAs,
// each a chain load -> stage -> products -> merge -> epilogue), so more warps
// per CTA mean shorter chains.
#include <string.h>

#include <algorithm>

#include "k_grid_pass.cuh"

namespace uot {
namespace {

constexpr int kBI = 32;  // outputs per block (one per lane)
constexpr int kLW = 4;   // lines per CTA
constexpr int kMaxDmax = (kBI + 64) / 2 - 1;

struct BlkArgs {
  PassArgs p;
  float g[kMaxDmax + 1];  // G(d) = 2^{-k2 h^2 d^2}, d = 0 .. dmax
};

template <int BJ>
__host__ __device__ constexpr int blk_dmax() {
  return (kBI + BJ) / 2 - 1;
}

template <int BJ, int JS>
__global__ void __launch_bounds__(JS * 32, 16 / JS) grid_pass_blk(BlkArgs ba, Epilogue epi) {
  constexpr int NT = JS * 32;
  constexpr int DOFF = (BJ - kBI) / 2;  // ic - jc = i_loc - j_loc + DOFF
  constexpr int Q = BJ / 32;            // inputs per lane in the A generation
  const PassArgs& a = ba.p;
  extern __shared__ float smem[];
  __shared__ float sg[kMaxDmax + 1];
  __shared__ float smx[kLW];
  __shared__ float sred[kLW][JS];
  __shared__ float4 sA[JS][BJ];
  __shared__ float2 sx[JS][kLW][32];  // (R, S) of every warp, merged at the end
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int I = blockIdx.x, l0 = blockIdx.y * kLW;
  const int64_t bz = blockIdx.z;
  const int nin = a.nin, nout = a.nout, nlines = a.nlines;
  const int nJ = (nin + BJ - 1) / BJ;
  const int ninp = nJ * BJ;
  float* st = smem;              // [kLW][ninp] t (log2 units, relative to the line maximum)
  float* slo = smem + kLW * ninp;  // [kLW][ninp] staging of the low parts

  // ---- prologue independent of the preceding kernel ----
  for (int k = tid; k <= blk_dmax<BJ>(); k += NT) sg[k] = ba.g[k];
  const int i = I * kBI + lane;
  const bool iok = i < nout;
  // warp w finishes lines w, w + JS, ... of the CTA
  constexpr int LPW = (kLW + JS - 1) / JS;
  EpiPre pre[LPW];
#pragma unroll
  for (int rr = 0; rr < LPW; ++rr) {
    const int r = warp + JS * rr, l = l0 + r;
    if (r < kLW && iok && l < nlines) epilogue_prefetch(epi, bz, (int64_t)i * nlines + l, pre[rr]);
  }
  __syncthreads();
  float G[BJ];
#pragma unroll
  for (int jj = 0; jj < BJ; ++jj) {
    const int d = lane - jj + DOFF;
    G[jj] = sg[d < 0 ? -d : d];
  }

  pdl_wait();
  if (a.zero_acc && blockIdx.x == 0 && blockIdx.y == 0 && tid < 2) a.zero_acc[2 * bz + tid] = 0.0;
  pdl_launch_dependents();

  // ---- the CTA's lines: float-float values, line maxima, t relative to them ----
  const float2* in = a.in + bz * (int64_t)nlines * nin;
  float lmax[kLW];
  {
    // all of a thread's loads are issued before any is used (one L2 round trip)
    constexpr int kB = 4;
    float mx[kLW];
#pragma unroll
    for (int r = 0; r < kLW; ++r) mx[r] = -INFINITY;
    for (int j0 = tid; j0 < ninp; j0 += kB * NT) {
      float2 raw[kLW][kB];
#pragma unroll
      for (int r = 0; r < kLW; ++r)
#pragma unroll
        for (int b = 0; b < kB; ++b) {
          const int j = j0 + b * NT, l = l0 + r;
          raw[r][b] = (l < nlines && j < nin) ? in[(int64_t)l * nin + j] : make_float2(-INFINITY, 0.0f);
        }
#pragma unroll
      for (int r = 0; r < kLW; ++r)
#pragma unroll
        for (int b = 0; b < kB; ++b) {
          const int j = j0 + b * NT, l = l0 + r;
          if (j >= ninp) continue;
          ff v = ffl(raw[r][b]);
          if (a.in_is_pot && l < nlines && j < nin)
            v = (v.hi == -INFINITY) ? ff_ninf()
                                    : ff_add(ff_mul(v, ffl(a.inv_eps)), ffl(a.logw[(int64_t)l * nin + j]));
          st[r * ninp + j] = v.hi;
          slo[r * ninp + j] = v.lo;
          mx[r] = fmaxf(mx[r], v.hi);
        }
    }
#pragma unroll
    for (int r = 0; r < kLW; ++r) {
      lmax[r] = warp_maxf(mx[r]);
      if (lane == 0) sred[r][warp] = lmax[r];
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kLW; ++r) {
    float mx = sred[r][0];
#pragma unroll
    for (int w = 1; w < JS; ++w) mx = fmaxf(mx, sred[r][w]);
    lmax[r] = mx;
    if (tid == 0) smx[r] = mx;
    for (int j = tid; j < ninp; j += NT) {
      const float hi = st[r * ninp + j];
      st[r * ninp + j] = (hi == -INFINITY) ? -INFINITY : ((hi - mx) + slo[r * ninp + j]) * kLog2e;
    }
  }
  __syncthreads();

  // ---- block products over this warp's input blocks ----
  const float h = a.blk.h, k2 = a.k2;
  const float ic = (float)lane - 0.5f * (kBI - 1);
  float R[kLW], S[kLW];
#pragma unroll
  for (int r = 0; r < kLW; ++r) {
    R[r] = -INFINITY;
    S[r] = 0.0f;
  }
  const int J0 = (nJ * warp) / JS, J1 = (nJ * (warp + 1)) / JS;
  for (int J = J0; J < J1; ++J) {
    const float D = fmaf(h, (float)(kBI * I - BJ * J) + 0.5f * (kBI - BJ), a.blk.d0);
    const float c = 2.0f * k2 * D * h;
    const float alpha = -k2 * D * D;
    float M[kLW];
    float av[kLW][Q];
#pragma unroll
    for (int r = 0; r < kLW; ++r) {
      float m = -INFINITY;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int jl = lane + 32 * q;
        const float t = st[r * ninp + J * BJ + jl];
        av[r][q] = (t == -INFINITY) ? -INFINITY : fmaf(c, (float)jl - 0.5f * (BJ - 1), t);
        m = fmaxf(m, av[r][q]);
      }
      M[r] = warp_maxf(m);
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      float A[kLW];
#pragma unroll
      for (int r = 0; r < kLW; ++r) A[r] = (M[r] == -INFINITY) ? 0.0f : ex2_approx(av[r][q] - M[r]);
      sA[warp][lane + 32 * q] = make_float4(A[0], A[1], A[2], A[3]);
    }
    __syncwarp();
    float P[kLW] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int jj = 0; jj < BJ; ++jj) {
      const float4 A4 = sA[warp][jj];
      P[0] = fmaf(A4.x, G[jj], P[0]);
      P[1] = fmaf(A4.y, G[jj], P[1]);
      P[2] = fmaf(A4.z, G[jj], P[2]);
      P[3] = fmaf(A4.w, G[jj], P[3]);
    }
    __syncwarp();
    // merge the block sum, scaled by 2^{M + alpha + beta ic}, into (R, S)
    const float beta = -c;
#pragma unroll
    for (int r = 0; r < kLW; ++r) {
      if (P[r] > 0.0f) {
        const float e = fmaf(beta, ic, M[r] + alpha);
        const float d = e - R[r];
        const float sc = ex2_approx(-fabsf(d));
        S[r] = (d > 0.0f) ? fmaf(S[r], sc, P[r]) : fmaf(P[r], sc, S[r]);
        R[r] = fmaxf(R[r], e);
      }
    }
  }

  // ---- merge the warps' pairs; warp w finishes lines w, w + JS, ... ----
  if (JS > 1) {
#pragma unroll
    for (int r = 0; r < kLW; ++r) sx[warp][r][lane] = make_float2(R[r], S[r]);
    __syncthreads();
  }
  float num = 0.0f, den = 0.0f;
#pragma unroll
  for (int rr = 0; rr < LPW; ++rr) {
    const int r = warp + JS * rr;
    if (r >= kLW) break;
    const int l = l0 + r;
    float Rm = R[r], Sm = S[r];
    if (JS > 1) {
      Rm = -INFINITY;
      Sm = 0.0f;
#pragma unroll
      for (int w = 0; w < JS; ++w) {
        const float2 v = sx[w][r][lane];
        if (v.y > 0.0f) Rm = fmaxf(Rm, v.x);
      }
      if (Rm != -INFINITY) {
#pragma unroll
        for (int w = 0; w < JS; ++w) {
          const float2 v = sx[w][r][lane];
          if (v.y > 0.0f) Sm = fmaf(v.y, ex2_approx(v.x - Rm), Sm);
        }
      }
    }
    if (!iok || l >= nlines) continue;
    ff z = ff_ninf();
    if (Sm > 0.0f) {
      // z = mx + ln2 (R + log2 S), the product ln2 R kept exact in float-float
      const ff ln2 = ln2_ff();
      z = ff_add_f(ff_add_f(ff_mul_f(ln2, Rm), smx[r]), kLn2 * lg2_approx(Sm));
    }
    const int64_t pt = (int64_t)i * nlines + l;
    if (a.zprev) a.zprev[bz * (int64_t)nout * nlines + pt] = z.hi;
    float n1, d1;
    epilogue_apply(epi, bz, pt, z, pre[rr], n1, d1);
    num += n1;
    den += d1;
  }
  if (epi.err) block_add2f<NT>(num, den, epi.err + 2 * bz);
}

template <int BJ, int JS>
cudaError_t launch_blk(const BlkArgs& ba, const Epilogue& epi, int nbatch, cudaStream_t s) {
  const PassArgs& a = ba.p;
  const int nJ = (a.nin + BJ - 1) / BJ;
  const size_t smem = 2 * (size_t)kLW * nJ * BJ * sizeof(float);
  dim3 grid((a.nout + kBI - 1) / kBI, (a.nlines + kLW - 1) / kLW, nbatch);
  if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
  if (smem > 48 * 1024) {
    cudaError_t e = smem_at_least(grid_pass_blk<BJ, JS>, smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = grid;
  cfg.blockDim = dim3(JS * 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, grid_pass_blk<BJ, JS>, ba, epi);
}

// (input block, warps per CTA) of each variant
constexpr int kVariants[][2] = {{32, 2}, {32, 4}, {32, 8}, {64, 2}, {64, 4}};
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));
int variant_bj(int v) { return kVariants[v][0]; }

}  // namespace

int grid_blk_variants() { return kNumVariants; }

// Variant v: input blocks of kVariants[v][0] points, kVariants[v][1] warps per CTA.
bool grid_blk_ok(const PassArgs& a, int v) {
  if (v < 0 || v >= kNumVariants) return false;
  // staging: 2 x 4 lines x nin floats of shared memory (<= 128 KB)
  if (!a.blk.ok || a.nin < 2 || a.nout < 1 || a.nin > 4096) return false;
  const double dmax = (kBI + variant_bj(v)) / 2 - 1;
  const double hd = (double)a.blk.h;
  return (double)a.k2 * hd * hd * dmax * dmax <= 90.0;
}

const char* grid_blk_name(int v) {
  static const char* names[] = {"blk32x2", "blk32x4", "blk32x8", "blk64x2", "blk64x4"};
  return (v >= 0 && v < kNumVariants) ? names[v] : "blk?";
}

cudaError_t launch_grid_pass_blk(const PassArgs& a, int v, const Epilogue& epi, int nbatch, cudaStream_t s) {
  if (!grid_blk_ok(a, v)) return cudaErrorInvalidValue;
  BlkArgs ba;
  memset(&ba, 0, sizeof(ba));
  ba.p = a;
  // G(d) = 2^{-k2 h^2 d^2} from the FP64 values of eps's k2 and h
  const double k2 = (double)a.k2, h = (double)a.blk.h;
  const int dmax = (kBI + variant_bj(v)) / 2 - 1;
  for (int d = 0; d <= dmax; ++d) ba.g[d] = (float)exp2(-k2 * h * h * (double)d * (double)d);
  switch (v) {
    case 0: return launch_blk<32, 2>(ba, epi, nbatch, s);
    case 1: return launch_blk<32, 4>(ba, epi, nbatch, s);
    case 2: return launch_blk<32, 8>(ba, epi, nbatch, s);
    case 3: return launch_blk<64, 2>(ba, epi, nbatch, s);
    default: return launch_blk<64, 4>(ba, epi, nbatch, s);
  }
}

}  // namespace uot

// Tensor-core (tcgen05) separable pass of the log-domain Gibbs operator on
// grids with FP32-level accuracy: the block-stabilised product of
// k_grid_tc.cu with every operand split into three BF16 terms.
//
// Same result as grid_pass_f32:  z[i][l] = log sum_j exp(L[l][j] - (x_i - y_j)^2 / eps).
// For an output block I and an input block J of T = 32 points, reference
// points c_I = x_{first i}, c_J = y_{first j}, D = c_I - c_J,
// delta_i = x_i - c_I, eta_j = y_j - c_J, k = log2(e)/eps, t_j = (L_j - m_J) log2(e)
// with m_J the block maximum of the line:
//
//   t_j - k (x_i - y_j)^2 = [t_j + 2kD eta_j] - k (delta_i - eta_j)^2 - k D (D + 2 delta_i)
//
// so the block's sum is 2^(M - k D (D + 2 delta_i)) * sum_j A[l][j] G[i][j] with
// A[l][j] = 2^(t_j + 2kD eta_j - M) in (0, 1] (M its row maximum) and
// G[i][j] = 2^(-k (delta_i - eta_j)^2) in (0, 1].  The largest term of every row
// of the product is >= min G = 2^(-k (2 r)^2) (r the block radius), so with
// k (2r)^2 <= 90 nothing significant underflows.
//
// Accuracy: A = a1 + a2 + a3 and G = g1 + g2 + g3, each part the BF16 rounding
// of what the previous parts leave (24 significant bits in all), and the
// product keeps the six terms a_p g_q with p + q <= 4 (the dropped ones are
// below 2^-24 of the product), accumulated in FP32 by the tensor core.  The
// per-element relative error is thus ~2^-23, comparable with the SIMT pass's
// FP32 exponent evaluation.
//
// Parallelism: one CTA = 128 consecutive lines (flattened over the batch; the
// MMA's M, thread t owns line t and tensor-memory lane t) x one output block x
// one input block; the CTAs of the input blocks of an output block form a
// thread-block cluster (at most 8: nin <= 256).  Each CTA leaves its
// partial log-sums (block maximum m_J, exponent) in shared memory; after a
// cluster barrier every CTA merges a share of the 128 x 32 outputs over the
// cluster's partials through distributed shared memory and applies the
// epilogue.  No per-output shift or fallback is needed: the block maxima are
// exact.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <string.h>

#include "uot_internal.cuh"

namespace cg = cooperative_groups;

namespace uot {
namespace {

constexpr int kT = 32;                       // block size (outputs and inputs)
constexpr int kLines = 128;                  // lines per CTA (MMA M)
constexpr int kMaxCluster = 8;               // input blocks per cluster
constexpr int kTileA = kLines * kT * 2;      // bytes of one BF16 A tile
constexpr int kTileG = kT * kT * 2;          // bytes of one BF16 G tile
constexpr int kSmem = 3 * kTileA + 3 * kTileG + kLines * kT * 4 + kLines * 4;


// x = p0 + p1 + p2, each part the BF16 rounding of what the previous ones leave.
__device__ __forceinline__ void split3(float x, __nv_bfloat16 (&p)[3]) {
  p[0] = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(p[0]);
  p[1] = __float2bfloat16_rn(r1);
  p[2] = __float2bfloat16_rn(r1 - __bfloat162float(p[1]));
}

struct Tc3Args {
  const float2* in;    // float-float line values (or potentials when in_is_pot), batch-contiguous
  const float2* logw;  // float-float log weights (in_is_pot only), one batch entry
  int in_is_pot;
  int nlines, nin, nout, nbatch;
  const float* yi;
  const float* xo;
  float2 inv_eps;
  float k2;            // log2(e)/eps
  int* err_flag;       // set if a bounded wait gave up (may be NULL)
  double* zero_acc;
};

__global__ void __launch_bounds__(kLines, 4) grid_pass_tc3(Tc3Args a, Epilogue epi) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;                         // 3 A tiles
  unsigned char* sG = smem + 3 * kTileA;            // 3 G tiles
  float* spart = reinterpret_cast<float*>(smem + 3 * kTileA + 3 * kTileG);  // [kLines][kT] exponents
  float* smx = spart + kLines * kT;                 // [kLines] block maxima m_J of the lines
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ float sx[kT], sy[kT];
  cg::cluster_group cl = cg::this_cluster();
  const int tid = threadIdx.x, warp = tid >> 5;
  const int J = blockIdx.x, nJ = gridDim.x;  // cluster rank = input block
  const int i0 = blockIdx.y * kT, j0 = J * kT;
  const int nin = a.nin, nout = a.nout, nlines = a.nlines;
  const int64_t total_lines = (int64_t)a.nbatch * nlines;
  const int64_t L0 = (int64_t)blockIdx.z * kLines;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(&tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid < kT) {
    sx[tid] = a.xo[min(i0 + tid, nout - 1)];
    sy[tid] = a.yi[min(j0 + tid, nin - 1)];
  }

  // wait for the preceding kernel's results (programmatic dependent launch)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (a.zero_acc && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0)
    for (int t = tid; t < 2 * a.nbatch; t += kLines) a.zero_acc[t] = 0.0;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  __syncthreads();

  const float k2 = a.k2;
  const float cI = sx[0], cJ = sy[0];
  const float D = cI - cJ;

  // ---- this thread's line: the 32 inputs of block J, staged relative to their maximum ----
  const int64_t L = L0 + tid;
  const bool lvalid = L < total_lines;
  float hv[kT], lv[kT];
  float mJ = -INFINITY;
  {
    const int64_t l = lvalid ? L % nlines : 0;
#pragma unroll
    for (int q = 0; q < kT; ++q) {
      const int j = j0 + q;
      hv[q] = -INFINITY;
      lv[q] = 0.0f;
      if (lvalid && j < nin) {
        ff v = ffl(a.in[L * nin + j]);
        if (a.in_is_pot && v.hi != -INFINITY) v = ff_add(ff_mul(v, ffl(a.inv_eps)), ffl(a.logw[l * nin + j]));
        hv[q] = v.hi;
        lv[q] = v.lo;
        mJ = fmaxf(mJ, v.hi);
      }
    }
  }
  // a_j = t_j + 2 k D eta_j, its maximum M, A = 2^(a - M) split in three BF16 parts
  float M = -INFINITY;
#pragma unroll
  for (int q = 0; q < kT; ++q) {
    float v = -INFINITY;
    if (hv[q] != -INFINITY) v = ((hv[q] - mJ) + lv[q]) * kLog2e + 2.0f * k2 * D * (sy[q] - cJ);
    hv[q] = v;
    M = fmaxf(M, v);
  }
#pragma unroll
  for (int q = 0; q < kT; q += 2) {
    const float e0 = (M == -INFINITY || hv[q] == -INFINITY) ? 0.0f : ex2_approx(hv[q] - M);
    const float e1 = (M == -INFINITY || hv[q + 1] == -INFINITY) ? 0.0f : ex2_approx(hv[q + 1] - M);
    __nv_bfloat16 p0[3], p1[3];
    split3(e0, p0);
    split3(e1, p1);
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      __nv_bfloat162 pr;
      pr.x = p0[s];
      pr.y = p1[s];
      *reinterpret_cast<__nv_bfloat162*>(sA + s * kTileA + tile_off(tid, q)) = pr;
    }
  }
  // G tiles: rows = outputs i of the block, columns = inputs j of the block
  for (int e = tid; e < kT * kT; e += kLines) {
    const int r = e / kT, q = e % kT;
    float g = 0.0f;
    if (i0 + r < nout && j0 + q < nin) {
      const float dd = (sx[r] - cI) - (sy[q] - cJ);
      g = ex2_approx(-k2 * dd * dd);
    }
    __nv_bfloat16 p[3];
    split3(g, p);
#pragma unroll
    for (int s = 0; s < 3; ++s) *reinterpret_cast<__nv_bfloat16*>(sG + s * kTileG + tile_off(r, q)) = p[s];
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  if (tid == 0) {
    // D (M = 128, N = 32, FP32) = sum over the kept parts a_p g_q, K = 32 in two steps of 16
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kT >> 3) << 17) |
                           ((uint32_t)(kLines >> 4) << 24);
    const int pa[6] = {2, 1, 0, 1, 0, 0};
    const int pg[6] = {0, 1, 2, 0, 1, 0};
    int n = 0;
#pragma unroll
    for (int p = 0; p < 6; ++p) {
#pragma unroll
      for (int ks = 0; ks < kT / 16; ++ks, ++n) {
        const uint64_t da = smem_desc(smem_u32(sA + pa[p] * kTileA) + ks * 256, 128, 512);
        const uint64_t dg = smem_desc(smem_u32(sG + pg[p] * kTileG) + ks * 256, 128, 512);
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(dg), "r"(idesc), "r"(n));
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&mbar)));
  }
  // bounded wait for the MMAs (phase 0) by one warp (with a suspend-time hint,
  // so it does not spin on the issue slots); the others wait at the barrier
  uint32_t done = 1;
  if (warp == 0) {
    done = 0;
    unsigned long long t0, t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
      asm volatile(
          "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done) : "r"(smem_u32(&mbar)), "r"(0), "r"(20000));
      if (done) break;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
      if (t1 - t0 > 1000000000ull) break;  // 1 s
    }
  }
  const int failed = __syncthreads_or(done ? 0 : 1);
  if (failed && tid == 0 && a.err_flag) atomicExch(a.err_flag, 1);
  asm volatile("tcgen05.fence::after_thread_sync;");
  uint32_t r[kT];
#pragma unroll
  for (int q = 0; q < kT; ++q) r[q] = 0u;
  if (!failed) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(tmem + ((uint32_t)(warp * 32) << 16)));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
  }
  // partial exponents of this block (log2 units, relative to m_J of the line)
#pragma unroll
  for (int q = 0; q < kT; ++q) {
    const float P = __uint_as_float(r[q]);
    float v = -INFINITY;
    if (M != -INFINITY && P > 0.0f) v = M + lg2_approx(P) - k2 * D * (D + 2.0f * (sx[q] - cI));
    spart[tid * kT + q] = v;
  }
  smx[tid] = mJ;
  cl.sync();

  // ---- merge: this CTA's share of the 128 x 32 outputs over the cluster's partials ----
  // The share's partials of every CTA of the cluster are first copied into the
  // (now free) A-tile area with independent, consecutive distributed-shared-
  // memory loads; then this CTA signals that it reads no more peer memory.
  constexpr int kOuts = kLines * kT;
  const int chunk = (kOuts + nJ - 1) / nJ;
  const int o_begin = J * chunk, o_end = min(kOuts, o_begin + chunk);
  const int nsh = max(0, o_end - o_begin);
  const int tl_begin = o_begin / kT, tl_end = (o_end + kT - 1) / kT;
  const int nl = max(0, tl_end - tl_begin);
  float* st_rel = reinterpret_cast<float*>(sA);  // [nJ][nsh]  (<= 16 KB)
  float* st_mx = st_rel + nJ * nsh;              // [nJ][nl]   (<= 4 KB)
  for (int c = 0; c < nJ; ++c) {
    const float* rp = cl.map_shared_rank(spart, c) + o_begin;
    const float* rm = cl.map_shared_rank(smx, c) + tl_begin;
    if ((nsh & 3) == 0 && (o_begin & 3) == 0) {
      const float4* rp4 = reinterpret_cast<const float4*>(rp);
      float4* dst4 = reinterpret_cast<float4*>(st_rel + c * nsh);
      for (int e = tid; e < nsh / 4; e += kLines) dst4[e] = rp4[e];
    } else {
      for (int e = tid; e < nsh; e += kLines) st_rel[c * nsh + e] = rp[e];
    }
    for (int e = tid; e < nl; e += kLines) st_mx[c * nl + e] = rm[e];
  }
  __syncthreads();
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");

  const int64_t bA = (L0 + tl_begin) / nlines;  // batch entry of the share's first line
  float num0 = 0.0f, den0 = 0.0f, num1 = 0.0f, den1 = 0.0f;
  const ff ln2 = ln2_ff();
  const ff log2e = ff{1.44269502162933349609375f, 1.925963033500011079e-08f};
  for (int e = tid; e < nsh; e += kLines) {
    const int o = o_begin + e;
    const int tl = o / kT, q = o % kT;
    const int64_t Lo = L0 + tl;
    if (Lo >= total_lines || i0 + q >= nout) continue;
    float best = -INFINITY;
    int cb = -1;
    for (int c = 0; c < nJ; ++c) {
      const float rc = st_rel[c * nsh + e];
      if (rc != -INFINITY) {
        const float est = st_mx[c * nl + (tl - tl_begin)] * kLog2e + rc;
        if (cb < 0 || est > best) {
          best = est;
          cb = c;
        }
      }
    }
    ff z = ff_ninf();
    if (cb >= 0) {
      const float base = st_mx[cb * nl + (tl - tl_begin)], rb = st_rel[cb * nsh + e];
      float sum = 0.0f;
      for (int c = 0; c < nJ; ++c) {
        const float rc = st_rel[c * nsh + e];
        if (rc == -INFINITY) continue;
        // 2^((m_c - base) log2 e + r_c - r_b), the difference of the block maxima kept exact
        const ff dm = ff_two_sum(st_mx[c * nl + (tl - tl_begin)], -base);
        const ff dl = ff_mul(dm, log2e);
        sum += ex2_approx(dl.hi + (dl.lo + (rc - rb)));
      }
      z = ff_add_f(ff_add_f(ff_mul_f(ln2, rb), base), kLn2 * lg2_approx(sum));
    }
    const int64_t b = Lo / nlines, l = Lo % nlines;
    float na, nb;
    apply_epilogue_ff(epi, b, (int64_t)(i0 + q) * nlines + l, z, na, nb);
    if (epi.err) {
      if (b == bA) {
        num0 += na;
        den0 += nb;
      } else if (b == bA + 1) {
        num1 += na;
        den1 += nb;
      } else {
        atomicAdd(epi.err + 2 * b, (double)na);
        atomicAdd(epi.err + 2 * b + 1, (double)nb);
      }
    }
  }
  if (epi.err) {
    block_add2f<kLines>(num0, den0, epi.err + 2 * bA);
    block_add2f<kLines>(num1, den1, (bA + 1 < a.nbatch) ? epi.err + 2 * (bA + 1) : nullptr);
  }
  // no CTA leaves while others may still read its shared memory
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

}  // namespace

int grid_pass_tc3_max_nin() { return kT * kMaxCluster; }

cudaError_t launch_grid_pass_tc3(const float2* in, const float2* logw, int in_is_pot, int nlines, int nin,
                                 const float* yi, int nout, const float* xo, float2 inv_eps, float k2, int nbatch,
                                 const Epilogue& epi, cudaStream_t s, int* err_flag, double* zero_acc) {
  const int nJ = (nin + kT - 1) / kT;
  if (nJ > kMaxCluster || nJ < 1) return cudaErrorInvalidValue;
  const int64_t total_lines = (int64_t)nbatch * nlines;
  dim3 grid(nJ, (nout + kT - 1) / kT, (unsigned)((total_lines + kLines - 1) / kLines));
  if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
  Tc3Args a;
  a.in = in;
  a.logw = logw;
  a.in_is_pot = in_is_pot;
  a.nlines = nlines;
  a.nin = nin;
  a.nout = nout;
  a.nbatch = nbatch;
  a.yi = yi;
  a.xo = xo;
  a.inv_eps = inv_eps;
  a.k2 = k2;
  a.err_flag = err_flag;
  a.zero_acc = zero_acc;
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kLines);
  cfg.dynamicSmemBytes = kSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = nJ;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, grid_pass_tc3, a, epi);
}

}  // namespace uot

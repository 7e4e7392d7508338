// Tensor-core (tcgen05) separable pass of the log-domain Gibbs operator on
// grids, block-stabilised so that the separable structure and the log-domain
// stabilisation coexist (the paper's Sec. 4.4 notes they cannot be combined in
// Algorithm 2's stored-kernel form).
//
// Same result as grid_pass_f32:  z[i][l] = log sum_j exp(L[l][j] - (x_i - y_j)^2 / eps).
// Blocks of T = 32 inputs J and outputs I with reference points c_I = x_{first i},
// c_J = y_{first j}, D = c_I - c_J, delta_i = x_i - c_I, eta_j = y_j - c_J, and
// k = log2(e)/eps, in log2 units t_j = L_j log2(e):
//
//   t_j - k (x_i - y_j)^2 = [t_j + 2 k D eta_j] - k (delta_i - eta_j)^2 - k D^2 - 2 k D delta_i
//
// so  sum_{j in J} 2^(t_j - k (x_i - y_j)^2) = 2^(m_J - k D^2 - 2 k D delta_i) * sum_j A[l][j] G[i][j]
// with A[l][j] = 2^(t_j + 2kD eta_j - m_J) in (0, 1] (m_J its row maximum) and
// G[i][j] = 2^(-k (delta_i - eta_j)^2) in (0, 1].  The product A G^T over the
// block is one tcgen05 MMA chain (M = 128 lines, N = 32 outputs, K = 32 inputs,
// BF16 operands, FP32 accumulation in tensor memory); per output the block
// results are merged with a running log-sum-exp.  The largest term of every
// block product is >= G's smallest entry 2^(-k (2 r)^2) (r the block radius),
// so nothing significant underflows.  Operands are rounded to BF16
// (8-bit significand): the result's relative error is bounded by ~2^-8 per
// block, which this mixed-precision mode trades for 1/10 of the exponentials.
//
// One CTA = 128 consecutive lines (flattened over the batch) x one output
// block; 4 warps, thread t owns line t (the MMA row t, tensor-memory lane t).
#include <cuda_bf16.h>
#include <string.h>

#include "uot_internal.cuh"

namespace uot {
namespace {

constexpr int kT = 32;     // block size (outputs and inputs)
constexpr int kLines = 128;


struct TcArgs {
  const float2* in;    // float-float line values (or potentials when in_is_pot), batch-contiguous
  const float2* logw;  // float-float log weights (in_is_pot only), one batch entry
  int in_is_pot;
  int nlines, nin, nout, nbatch;
  const float* yi;
  const float* xo;
  float2 inv_eps;
  float k2;            // log2(e)/eps
  int* err_flag;       // set if a bounded wait gave up
  double* zero_acc;
};

__device__ __forceinline__ ff load_L(const TcArgs& a, int64_t gidx, int64_t widx) {
  const ff v = ffl(a.in[gidx]);
  if (!a.in_is_pot) return v;
  if (v.hi == -INFINITY) return ff_ninf();
  return ff_add(ff_mul(v, ffl(a.inv_eps)), ffl(a.logw[widx]));
}

__global__ void __launch_bounds__(kLines, 1)
    grid_pass_tc(TcArgs a, Epilogue epi) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // layout: A tile 128x32 bf16 (8 KB) | G tile 32x32 bf16 (2 KB) | t values [128][nin+1] f32
  unsigned char* sA = smem;
  unsigned char* sG = smem + 8192;
  float* st = reinterpret_cast<float*>(smem + 8192 + 2048);
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ float sx[kT];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nin = a.nin, nout = a.nout, nlines = a.nlines;
  const int64_t total_lines = (int64_t)a.nbatch * nlines;
  const int64_t L0 = (int64_t)blockIdx.y * kLines;
  const int i0 = blockIdx.x * kT;
  const int ldt = nin + 1;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(&tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid < kT) sx[tid] = a.xo[min(i0 + tid, nout - 1)];

  // wait for the preceding kernel's results (programmatic dependent launch)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (a.zero_acc && blockIdx.x == 0 && blockIdx.y == 0)
    for (int t = tid; t < 2 * a.nbatch; t += kLines) a.zero_acc[t] = 0.0;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  // stage the CTA's lines: per-line maximum of the high parts, then t = (L - max) log2 e
  __shared__ float smax[kLines];
  for (int r = warp; r < kLines; r += 4) {
    const int64_t L = L0 + r;
    float mx = -INFINITY;
    if (L < total_lines) {
      const int64_t l = L % nlines;
      for (int j = lane; j < nin; j += 32) mx = fmaxf(mx, load_L(a, L * nin + j, l * nin + j).hi);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (L < total_lines) {
      const int64_t l = L % nlines;
      for (int j = lane; j < nin; j += 32) {
        const ff v = load_L(a, L * nin + j, l * nin + j);
        st[r * ldt + j] = (v.hi == -INFINITY || mx == -INFINITY) ? -INFINITY : ((v.hi - mx) + v.lo) * kLog2e;
      }
    }
    if (lane == 0) smax[r] = mx;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const float k2 = a.k2;
  const float mx_l = smax[tid];
  const bool line_ok = (L0 + tid) < total_lines && mx_l != -INFINITY;

  // running log-sum-exp per output of this line (log2 units, relative to mx_l)
  float Mr[kT], Sr[kT];
#pragma unroll
  for (int q = 0; q < kT; ++q) {
    Mr[q] = -INFINITY;
    Sr[q] = 0.0f;
  }
  const float cI = sx[0];
  const int nJ = (nin + kT - 1) / kT;
  int wait_failed = 0;
  for (int J = 0; J < nJ; ++J) {
    const int j0 = J * kT;
    const float cJ = a.yi[j0];
    const float Dd = cI - cJ;
    // A row of this thread: a_j = t_j + 2 k D eta_j, its maximum, 2^(a_j - m)
    float av[kT];
    float mJ = -INFINITY;
#pragma unroll
    for (int q = 0; q < kT; ++q) {
      const int j = j0 + q;
      float v = -INFINITY;
      if (j < nin && line_ok) {
        const float t = st[tid * ldt + j];
        if (t != -INFINITY) v = t + 2.0f * k2 * Dd * (a.yi[j] - cJ);
      }
      av[q] = v;
      mJ = fmaxf(mJ, v);
    }
#pragma unroll
    for (int q = 0; q < kT; q += 2) {
      const float e0 = (mJ == -INFINITY) ? 0.0f : ex2_approx(av[q] - mJ);
      const float e1 = (mJ == -INFINITY) ? 0.0f : ex2_approx(av[q + 1] - mJ);
      *reinterpret_cast<__nv_bfloat162*>(sA + tile_off(tid, q)) = __floats2bfloat162_rn(e0, e1);
    }
    // G tile: rows = outputs i of the block, cols = inputs j of the block
    for (int e = tid; e < kT * kT; e += kLines) {
      const int r = e / kT, q = e % kT;
      const int j = j0 + q;
      float g = 0.0f;
      if (j < nin && i0 + r < nout) {
        const float dd = (sx[r] - cI) - (a.yi[j] - cJ);
        g = ex2_approx(-k2 * dd * dd);
      }
      *reinterpret_cast<__nv_bfloat16*>(sG + tile_off(r, q)) = __float2bfloat16_rn(g);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kT >> 3) << 17) |
                             ((uint32_t)(kLines >> 4) << 24);
#pragma unroll
      for (int ks = 0; ks < kT / 16; ++ks) {
        const uint64_t da = smem_desc(smem_u32(sA) + ks * 256, 128, 512);
        const uint64_t dg = smem_desc(smem_u32(sG) + ks * 256, 128, 512);
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(dg), "r"(idesc), "r"(ks));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&mbar)));
    }
    // bounded wait for this block's MMAs (phase J & 1)
    uint32_t done = 0;
    for (int it = 0; it < (1 << 24) && !done; ++it) {
      asm volatile(
          "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done) : "r"(smem_u32(&mbar)), "r"(J & 1));
    }
    // block-uniform decision, so that no thread is left waiting at a barrier
    if (__syncthreads_or(done ? 0 : 1)) {
      wait_failed = 1;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    uint32_t r[kT];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(tmem + ((uint32_t)(warp * 32) << 16)));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    // merge: v = log2 P + m_J - k D^2 - 2 k D delta_i
    if (mJ != -INFINITY) {
#pragma unroll
      for (int q = 0; q < kT; ++q) {
        const float P = __uint_as_float(r[q]);
        if (P > 0.0f) {
          const float di = sx[q] - cI;
          const float v = lg2_approx(P) + mJ - k2 * Dd * (Dd + 2.0f * di);
          const float nm = fmaxf(Mr[q], v);
          Sr[q] = Sr[q] * ex2_approx(Mr[q] - nm) + ex2_approx(v - nm);
          Mr[q] = nm;
        }
      }
    }
    // the next block rewrites the operand tiles and the accumulator
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
  }
  if (wait_failed && lane == 0) atomicExch(a.err_flag, 1);

  // results: thread = line, q = output in the block
  float num = 0.0f, den = 0.0f;
  if ((L0 + tid) < total_lines && !wait_failed) {
    const int64_t L = L0 + tid;
    const int64_t b = L / nlines, l = L % nlines;
    const ff ln2 = ln2_ff();
#pragma unroll
    for (int q = 0; q < kT; ++q) {
      const int i = i0 + q;
      if (i >= nout) continue;
      ff z = ff_ninf();
      if (mx_l != -INFINITY && Sr[q] > 0.0f)
        z = ff_add_f(ff_add_f(ff_mul_f(ln2, Mr[q]), mx_l), kLn2 * lg2_approx(Sr[q]));
      float na, nb;
      apply_epilogue_ff(epi, b, (int64_t)i * nlines + l, z, na, nb);
      num += na;
      den += nb;
    }
    if (epi.err) {
      atomicAdd(epi.err + 2 * b, (double)num);
      atomicAdd(epi.err + 2 * b + 1, (double)den);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

}  // namespace

size_t grid_pass_tc_smem(int nin) { return 8192 + 2048 + (size_t)kLines * (nin + 1) * sizeof(float); }

cudaError_t launch_grid_pass_tc(const double* in, const double* logw, int in_is_pot, int nlines,
                                int nin, const void* yi, int nout, const void* xo, double eps,
                                int nbatch, const Epilogue& epi, cudaStream_t s, int* err_flag,
                                double* zero_acc) {
  const size_t smem = grid_pass_tc_smem(nin);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = smem_at_least(grid_pass_tc, smem);
  if (e != cudaSuccess) return e;
  TcArgs a;
  a.in = reinterpret_cast<const float2*>(in);
  a.logw = reinterpret_cast<const float2*>(logw);
  a.in_is_pot = in_is_pot;
  a.nlines = nlines;
  a.nin = nin;
  a.nout = nout;
  a.nbatch = nbatch;
  a.yi = (const float*)yi;
  a.xo = (const float*)xo;
  a.inv_eps = ff2(ff_make(1.0 / eps));
  a.k2 = (float)((double)kLog2e / eps);
  a.err_flag = err_flag;
  a.zero_acc = zero_acc;
  const int64_t total_lines = (int64_t)nbatch * nlines;
  dim3 grid((nout + kT - 1) / kT, (unsigned)((total_lines + kLines - 1) / kLines));
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kLines);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  prof_mark_begin(PROF_GRID_PASS, s);
  count_launches(1);
  e = cudaLaunchKernelEx(&cfg, grid_pass_tc, a, epi);
  prof_mark_end(PROF_GRID_PASS, s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace uot

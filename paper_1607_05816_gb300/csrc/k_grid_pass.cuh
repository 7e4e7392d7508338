// Pieces shared by the FP32 separable grid passes (k_grid.cu: log-sum-exp
// tiles; k_grid_blk.cu: block-stabilised products): the pass arguments, the
// line values, and the epilogue that turns a pass result into the next
// potential (Table 1 in log form) or an intermediate line.
#pragma once

#include "uot_internal.cuh"

namespace uot {

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
  int tc3_ok;          // the tensor-core pass (k_grid_tc3.cu) is valid for this pass
  int* tc_err;         // its bounded-wait flag (may be NULL)
  int nbatch;
  BlkAxis blk;         // uniform-axis data for the block-stabilised pass (blk.ok = 0: not usable)
};

__device__ __forceinline__ ff load_L_ff(const PassArgs& a, const float2* in, int64_t idx) {
  const ff v = ffl(in[idx]);
  if (!a.in_is_pot) return v;
  if (v.hi == -INFINITY) return ff_ninf();
  return ff_add(ff_mul(v, ffl(a.inv_eps)), ffl(a.logw[idx]));
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
  ff S = (z.hi == -INFINITY) ? ff_ninf() : ff_mul(z, eps);
  if (e.zshift) S = ff_zshift(S, e.zshift);
  const ff Unew = prox_update_ff(e.Fff, ffl(o.lp), S, eps);
  reinterpret_cast<float2*>(e.pot)[b * e.bstride + pt] = ff2(Unew);
  if (e.err) violation_terms_ff(ffl(o.uold), Unew, S, ffl(o.lw), ffl(e.inv_eps_ff), num, den);
}


// The block-stabilised pass (k_grid_blk.cu): variant v of grid_blk_variants()
// applies when grid_blk_ok(a, v) (uniform axes, block condition at this eps).
int grid_blk_variants();
bool grid_blk_ok(const PassArgs& a, int v);
const char* grid_blk_name(int v);
cudaError_t launch_grid_pass_blk(const PassArgs& a, int v, const Epilogue& epi, int nbatch, cudaStream_t s);

}  // namespace uot

// uot_solve_mass: Algorithm 4 (Sec. 4.5), a divergence F3 on the plan's total mass.
#include "uot_host.cuh"

namespace uot {
namespace {

// ---------------------------------------------------------------------------
// Algorithm 4 (Sec. 4.5): a divergence F3 on the total mass of the plan
// ---------------------------------------------------------------------------
// A scalar z = e^{Z/eps} multiplies the plan; both scaling updates see S + Z
// and T + Z.  z's own update needs the mass of the current plan without z,
// M = sum_i dx_i e^{(U_i + S_i)/eps} with S from the new b.  By Fubini M also
// equals sum_j dy_j e^{(V_j + T_j)/eps} with T from the current a, which the
// b-side of the previous iteration has at hand: when eps does not change,
// k_mass_vupdate computes V and the next Z in one kernel after the raw T pass,
// and the next a-side is the plain prox pass with Z added to S in its
// epilogue (zshift).  At an eps change the z-update takes the direct route:
// raw S pass -> k_mass_reduce (per-block maximum and sum of e^{l_i - max},
// l_i = log dx_i + U_i/eps + z_i, merged by the last block, then F3's row) ->
// k_mass_prox (U = prox_F1(S + Z) and the violation terms).  All kernels wait
// for their predecessor first (programmatic dependent launch).

constexpr int kMassBlocks = kNT;  // partials of the mass reduction: one per block, at most kNT blocks

struct MassArgs {
  int64_t n;
  double eps;
  float2 eps_ff, inv_eps_ff;
  DivParams F3;
  DivFF F3ff;
  double logm0;
  float2 logm0_ff;
  int update;        // 0 in the very first iteration: z = 1 stays
  int check;         // clear acc[0..1] and write the mass violation to acc[2]
  double* Z;         // [1] Z (FP64) or its float-float pair
  double* acc;       // [3] violation accumulators
  double2* part;     // [kMassBlocks] per-block (max, sum); float-float: (max.hi, max.lo) + sum
  unsigned* count;   // blocks finished (the last one sets it back to 0)
};

// Block-wide maximum and sum (kNT threads), result broadcast to every thread.
__device__ inline double block_max_d(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  v = sh[0];
  for (int k = 1; k < kNT / 32; ++k) v = fmax(v, sh[k]);
  return v;
}
__device__ inline double block_sum_d(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  v = sh[0];
  for (int k = 1; k < kNT / 32; ++k) v += sh[k];
  return v;
}
__device__ inline ff block_max_ff(ff v, float2* sh) {
  for (int o = 16; o > 0; o >>= 1)
    v = ff_max(v, ff{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = ff2(v);
  __syncthreads();
  v = ffl(sh[0]);
  for (int k = 1; k < kNT / 32; ++k) v = ff_max(v, ffl(sh[k]));
  return v;
}
__device__ inline float block_sum_f(float v, float2* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = make_float2(v, 0.0f);
  __syncthreads();
  v = sh[0].x;
  for (int k = 1; k < kNT / 32; ++k) v += sh[k].x;
  return v;
}

constexpr int kMassPerThread = 4;  // elements per thread of the mass reduction (grid cap permitting)

// Per block: the maximum of l_i = log dx_i + U_i/eps + z_i over its
// grid-stride share, then the sum of e^{l_i - max} (a second sweep): two
// block reductions with one exponential per element.  The last block to
// finish merges the partials (one per thread, at most kNT blocks) the same
// way and applies F3's row.
template <bool FF>
__global__ void __launch_bounds__(kNT) k_mass_reduce(const double* __restrict__ U, const double* __restrict__ z,
                                                     const double* __restrict__ logdx, MassArgs a) {
  __shared__ double shd[kNT / 32];
  __shared__ float2 shf[kNT / 32];
  __shared__ bool last;
  pdl_begin();
  if (!a.update) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.check) a.acc[0] = a.acc[1] = 0.0;
    return;
  }
  const int64_t i0 = (int64_t)blockIdx.x * kNT + threadIdx.x, stride = (int64_t)gridDim.x * kNT;
  if constexpr (!FF) {
    auto lval = [&](int64_t i) {
      const double u = U[i], zi = z[i];
      return (u == -kInf || zi == -kInf) ? -kInf : logdx[i] + u / a.eps + zi;
    };
    double mx = -kInf;
    for (int64_t i = i0; i < a.n; i += stride) mx = fmax(mx, lval(i));
    mx = block_max_d(mx, shd);
    double s = 0.0;
    if (mx != -kInf)
      for (int64_t i = i0; i < a.n; i += stride) {
        const double l = lval(i);
        if (l != -kInf) s += exp(l - mx);
      }
    s = block_sum_d(s, shd);
    if (threadIdx.x == 0) {
      a.part[blockIdx.x] = make_double2(mx, s);
      __threadfence();
      last = atomicAdd(a.count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double2 v = make_double2(-kInf, 0.0);
    if (threadIdx.x < gridDim.x) v = __ldcg(&a.part[threadIdx.x]);
    const double M = block_max_d(v.x, shd);
    const double S = block_sum_d((M == -kInf || v.x == -kInf) ? 0.0 : v.y * exp(v.x - M), shd);
    if (threadIdx.x == 0) {
      // eps log M, then Z = prox of F3 at the total mass
      const double SM = (M == -kInf || S == 0.0) ? -kInf : a.eps * (M + log(S));
      a.Z[0] = prox_update(a.F3, a.logm0, SM, a.eps);
      if (a.check) a.acc[0] = a.acc[1] = 0.0;
      *a.count = 0u;
    }
  } else {
    const float2* U2 = reinterpret_cast<const float2*>(U);
    const float2* z2 = reinterpret_cast<const float2*>(z);
    const float2* w2 = reinterpret_cast<const float2*>(logdx);
    const ff inv_eps = ffl(a.inv_eps_ff);
    auto lval = [&](int64_t i) {
      const ff u = ffl(U2[i]), zi = ffl(z2[i]);
      return (u.hi == -INFINITY || zi.hi == -INFINITY) ? ff_ninf()
                                                       : ff_add(ff_add(ffl(w2[i]), ff_mul(u, inv_eps)), zi);
    };
    ff mx = ff_ninf();
    for (int64_t i = i0; i < a.n; i += stride) mx = ff_max(mx, lval(i));
    mx = block_max_ff(mx, shf);
    float s = 0.0f;
    if (mx.hi != -INFINITY)
      for (int64_t i = i0; i < a.n; i += stride) {
        const ff l = lval(i);
        if (l.hi == -INFINITY) continue;
        const ff d = ff_sub(l, mx);
        s += expf(d.hi + d.lo);
      }
    s = block_sum_f(s, shf);
    if (threadIdx.x == 0) {
      reinterpret_cast<float4*>(a.part)[blockIdx.x] = make_float4(mx.hi, mx.lo, s, 0.0f);
      __threadfence();
      last = atomicAdd(a.count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    float4 v = make_float4(-INFINITY, 0.0f, 0.0f, 0.0f);
    if (threadIdx.x < gridDim.x) v = __ldcg(&reinterpret_cast<const float4*>(a.part)[threadIdx.x]);
    const ff vm{v.x, v.y};
    const ff M = block_max_ff(vm, shf);
    float t = 0.0f;
    if (M.hi != -INFINITY && vm.hi != -INFINITY) {
      const ff d = ff_sub(vm, M);
      t = v.z * expf(d.hi + d.lo);
    }
    const float S = block_sum_f(t, shf);
    if (threadIdx.x == 0) {
      const ff eps = ffl(a.eps_ff);
      const ff SM = (M.hi == -INFINITY || S == 0.0f) ? ff_ninf() : ff_mul(eps, ff_add_f(M, logf(S)));
      reinterpret_cast<float2*>(a.Z)[0] = ff2(prox_update_ff(a.F3ff, ffl(a.logm0_ff), SM, eps));
      if (a.check) a.acc[0] = a.acc[1] = 0.0;
      *a.count = 0u;
    }
  }
}

struct MassProx {
  int64_t n;
  double eps;
  float2 eps_ff, inv_eps_ff;
  DivParams F;
  DivFF Fff;
  const double* Z;  // [1] Z (FP64) or its float-float pair
  double* err;      // [2] violation accumulators, NULL: no check
};

// pot_i = prox_F(log p_i, eps z_i + Z), z_i the raw log-sum of the Gibbs pass.
template <bool FF>
__global__ void __launch_bounds__(kNT) k_mass_prox(const double* __restrict__ z, const double* __restrict__ logp,
                                                   double* __restrict__ pot, const double* __restrict__ logw,
                                                   MassProx a) {
  pdl_begin();
  if constexpr (!FF) {
    const double Zv = a.Z[0];
    double num = 0.0, den = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kNT + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * kNT) {
      const double zi = z[i];
      const double Sz = (zi == -kInf || Zv == -kInf) ? -kInf : a.eps * zi + Zv;
      const double Uold = pot[i];
      const double Unew = prox_update(a.F, logp[i], Sz, a.eps);
      pot[i] = Unew;
      if (a.err) {
        double nu, de;
        violation_terms(Uold, Unew, Sz, logw[i], a.eps, nu, de);
        num += nu;
        den += de;
      }
    }
    if (a.err) block_add2<kNT>(num, den, a.err);
  } else {
    const ff Zv = ffl(reinterpret_cast<const float2*>(a.Z)[0]);
    const ff eps = ffl(a.eps_ff), inv_eps = ffl(a.inv_eps_ff);
    float2* pot2 = reinterpret_cast<float2*>(pot);
    float num = 0.0f, den = 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)kNT + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * kNT) {
      const ff zi = ffl(reinterpret_cast<const float2*>(z)[i]);
      const ff Sz = (zi.hi == -INFINITY || Zv.hi == -INFINITY) ? ff_ninf() : ff_add(ff_mul(zi, eps), Zv);
      const ff Uold = ffl(pot2[i]);
      const ff Unew = prox_update_ff(a.Fff, ffl(reinterpret_cast<const float2*>(logp)[i]), Sz, eps);
      pot2[i] = ff2(Unew);
      if (a.err) {
        float nu, de;
        violation_terms_ff(Uold, Unew, Sz, ffl(reinterpret_cast<const float2*>(logw)[i]), inv_eps, nu, de);
        num += nu;
        den += de;
      }
    }
    if (a.err) block_add2f<kNT>(num, den, a.err);
  }
}

// The b-side of an iteration in one kernel, when eps does not change from this
// iteration to the next: V_j = prox_F2(log q_j, T_j + Z), and the mass of the
// plan without z for the next z-update.  By Fubini the sum
// sum_i dx_i e^{(U_i + S_i)/eps}, S from the new b, equals
// sum_j dy_j e^{(V_j + T_j)/eps}, T from the current a, so it is reduced here
// (per block: maximum, then the sum of e^{l_j - max}; the last block merges).
// The last block applies F3's row and keeps the history of Z used for the
// mass violation: zhist[1] <- zhist[0], zhist[0] <- the Z this iteration used.
struct MassV {
  int64_t m;
  double eps;
  float2 eps_ff, inv_eps_ff;
  DivParams F2, F3;
  DivFF F2ff, F3ff;
  double logm0;
  float2 logm0_ff;
  double* Z;      // [1] Z (FP64) or its float-float pair: read, then replaced by the next one
  double* zhist;  // [2] the Z of this iteration and of the one before
  double2* part;  // [kMassBlocks]
  unsigned* count;
};

template <bool FF>
__global__ void __launch_bounds__(kNT) k_mass_vupdate(const double* __restrict__ zT, const double* __restrict__ logq,
                                                      double* __restrict__ V, const double* __restrict__ logdy,
                                                      MassV a) {
  __shared__ double shd[kNT / 32];
  __shared__ float2 shf[kNT / 32];
  __shared__ bool last;
  pdl_begin();
  const int64_t i0 = (int64_t)blockIdx.x * kNT + threadIdx.x, stride = (int64_t)gridDim.x * kNT;
  if constexpr (!FF) {
    const double Zv = a.Z[0];
    double mx = -kInf;
    for (int64_t j = i0; j < a.m; j += stride) {
      const double zj = zT[j];
      const double Sz = (zj == -kInf || Zv == -kInf) ? -kInf : a.eps * zj + Zv;
      const double v = prox_update(a.F2, logq[j], Sz, a.eps);
      V[j] = v;
      if (v != -kInf && zj != -kInf) mx = fmax(mx, logdy[j] + v / a.eps + zj);
    }
    mx = block_max_d(mx, shd);
    double s = 0.0;
    if (mx != -kInf)
      for (int64_t j = i0; j < a.m; j += stride) {
        const double v = V[j], zj = zT[j];
        if (v != -kInf && zj != -kInf) s += exp(logdy[j] + v / a.eps + zj - mx);
      }
    s = block_sum_d(s, shd);
    if (threadIdx.x == 0) {
      a.part[blockIdx.x] = make_double2(mx, s);
      __threadfence();
      last = atomicAdd(a.count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double2 pv = make_double2(-kInf, 0.0);
    if (threadIdx.x < gridDim.x) pv = __ldcg(&a.part[threadIdx.x]);
    const double M = block_max_d(pv.x, shd);
    const double Ssum = block_sum_d((M == -kInf || pv.x == -kInf) ? 0.0 : pv.y * exp(pv.x - M), shd);
    if (threadIdx.x == 0) {
      const double SM = (M == -kInf || Ssum == 0.0) ? -kInf : a.eps * (M + log(Ssum));
      reinterpret_cast<unsigned long long*>(a.zhist)[1] = reinterpret_cast<unsigned long long*>(a.zhist)[0];
      a.zhist[0] = Zv;
      a.Z[0] = prox_update(a.F3, a.logm0, SM, a.eps);
      *a.count = 0u;
    }
  } else {
    const float2* z2 = reinterpret_cast<const float2*>(zT);
    const float2* q2 = reinterpret_cast<const float2*>(logq);
    const float2* w2 = reinterpret_cast<const float2*>(logdy);
    float2* V2 = reinterpret_cast<float2*>(V);
    const ff eps = ffl(a.eps_ff), inv_eps = ffl(a.inv_eps_ff);
    const float2 Zraw = reinterpret_cast<const float2*>(a.Z)[0];
    const ff Zv = ffl(Zraw);
    auto lval = [&](ff v, ff zj, int64_t j) {
      return (v.hi == -INFINITY || zj.hi == -INFINITY) ? ff_ninf() : ff_add(ff_add(ffl(w2[j]), ff_mul(v, inv_eps)), zj);
    };
    ff mx = ff_ninf();
    for (int64_t j = i0; j < a.m; j += stride) {
      const ff zj = ffl(z2[j]);
      const ff Sz = (zj.hi == -INFINITY || Zv.hi == -INFINITY) ? ff_ninf() : ff_add(ff_mul(zj, eps), Zv);
      const ff v = prox_update_ff(a.F2ff, ffl(q2[j]), Sz, eps);
      V2[j] = ff2(v);
      mx = ff_max(mx, lval(v, zj, j));
    }
    mx = block_max_ff(mx, shf);
    float s = 0.0f;
    if (mx.hi != -INFINITY)
      for (int64_t j = i0; j < a.m; j += stride) {
        const ff l = lval(ffl(V2[j]), ffl(z2[j]), j);
        if (l.hi == -INFINITY) continue;
        const ff d = ff_sub(l, mx);
        s += expf(d.hi + d.lo);
      }
    s = block_sum_f(s, shf);
    if (threadIdx.x == 0) {
      reinterpret_cast<float4*>(a.part)[blockIdx.x] = make_float4(mx.hi, mx.lo, s, 0.0f);
      __threadfence();
      last = atomicAdd(a.count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    float4 pv = make_float4(-INFINITY, 0.0f, 0.0f, 0.0f);
    if (threadIdx.x < gridDim.x) pv = __ldcg(&reinterpret_cast<const float4*>(a.part)[threadIdx.x]);
    const ff vm{pv.x, pv.y};
    const ff M = block_max_ff(vm, shf);
    float t = 0.0f;
    if (M.hi != -INFINITY && vm.hi != -INFINITY) {
      const ff d = ff_sub(vm, M);
      t = pv.z * expf(d.hi + d.lo);
    }
    const float Ssum = block_sum_f(t, shf);
    if (threadIdx.x == 0) {
      const ff SM = (M.hi == -INFINITY || Ssum == 0.0f) ? ff_ninf() : ff_mul(eps, ff_add_f(M, logf(Ssum)));
      unsigned long long* zh = reinterpret_cast<unsigned long long*>(a.zhist);
      zh[1] = zh[0];
      reinterpret_cast<float2*>(a.zhist)[0] = Zraw;
      reinterpret_cast<float2*>(a.Z)[0] = ff2(prox_update_ff(a.F3ff, ffl(a.logm0_ff), SM, eps));
      *a.count = 0u;
    }
  }
}

uot_status solve_mass_impl(const uot_geom* g, const void* p, const void* dx, const void* q, const void* dy,
                           const uot_div* F1, const uot_div* F2, const uot_div* F3, double m0,
                           const uot_opts* o, void* Uout, void* Vout, double* Zout, uot_result* res,
                           cudaStream_t s) {
  uot_status st = check_geom(g);
  if (st != UOT_OK) return st;
  if ((st = check_opts(o)) != UOT_OK) return st;
  if (!p || !dx || !q || !dy || !Uout || !Vout || !Zout || !div_ok(F1) || !div_ok(F2) || !div_ok(F3))
    return UOT_EINVAL;
  if (!(m0 > 0.0) || !isfinite(m0)) return UOT_EINVAL;
  if (o->plain_scaling) return UOT_EUNSUPPORTED;
  const int prec = o->precision;
  const bool ffm = prec != UOT_F64;
  const int64_t n = g->n, m = g->m;
  const DivParams D1 = make_div(*F1), D2 = make_div(*F2), D3 = make_div(*F3);

  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  UOT_CK(cudaEventCreate(&ev0));
  UOT_CK(cudaEventCreate(&ev1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } evg{ev0, ev1};
  UOT_CK(cudaEventRecord(ev0, s));

  Scratch sc(s);
  Gibbs G;
  G.g = *g;
  G.prec = prec;
  G.speculate = true;
  G.plan(sc, 1);
  sc.reserve<double>(n);            // logp
  sc.reserve<double>(n);            // logdx
  sc.reserve<double>(n);            // U
  sc.reserve<double>(m);            // logq
  sc.reserve<double>(m);            // logdy
  sc.reserve<double>(m);            // V
  sc.reserve<double>(std::max(n, m));  // raw log-sums of the last pass (S/eps or T/eps)
  sc.reserve<double>(4);            // acc[3] + NaN flag
  sc.reserve<double>(3);            // Z, and the Z of the last two iterations
  sc.reserve<double2>(kMassBlocks); // mass partials
  sc.reserve<unsigned>(1);          // finished-block counter
  UOT_CK(sc.allocate());
  UOT_CK(G.take(sc, s));
  double* logp = sc.take<double>(n);
  double* logdx = sc.take<double>(n);
  double* U = sc.take<double>(n);
  double* logq = sc.take<double>(m);
  double* logdy = sc.take<double>(m);
  double* V = sc.take<double>(m);
  double* zb = sc.take<double>(std::max(n, m));
  double* acc = sc.take<double>(4);
  int* flag = (int*)(acc + 3);
  double* Zd = sc.take<double>(3);
  double* zhist = Zd + 1;
  double2* part = sc.take<double2>(kMassBlocks);
  unsigned* count = sc.take<unsigned>(1);
  UOT_SCRATCH_OK(sc);
  UOT_CK(to_log(prec, p, n, logp, s));
  UOT_CK(to_log(prec, dx, n, logdx, s));
  UOT_CK(to_log(prec, q, m, logq, s));
  UOT_CK(to_log(prec, dy, m, logdy, s));
  if (o->U0) {
    UOT_CK(to_f64(prec, o->U0, n, U, s));
  } else {
    count_launches(1);
    k_fill<<<nblocks(n), kNT, 0, s>>>(U, n, 0.0);
  }
  if (o->V0) {
    UOT_CK(to_f64(prec, o->V0, m, V, s));
  } else {
    count_launches(1);
    k_fill<<<nblocks(m), kNT, 0, s>>>(V, m, 0.0);
  }
  UOT_CK(cudaMemsetAsync(Zd, 0, 3 * sizeof(double), s));  // z = 1 (both layouts)
  UOT_CK(cudaMemsetAsync(acc, 0, 4 * sizeof(double), s));
  UOT_CK(cudaMemsetAsync(count, 0, sizeof(unsigned), s));
  UOT_CK(cudaGetLastError());

  // one partial per block (at most kNT: the last block merges them with one thread each)
  const int64_t per_block = (int64_t)kNT * kMassPerThread;
  const int red_blocks = (int)std::min<int64_t>(kNT, std::max<int64_t>(1, (n + per_block - 1) / per_block));
  bool first = true;
  // programmatic dependent launch (the kernels wait for their predecessor first)
  auto pdl_launch = [&](auto kern, int grid, cudaStream_t st, auto... args) -> cudaError_t {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kNT);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launches(1);
    return cudaLaunchKernelEx(&cfg, kern, args...);
  };
  auto prox_a = [&](double eps, double* err, cudaStream_t st) -> cudaError_t {
    MassProx a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.eps = eps;
    a.eps_ff = ff2(ff_make(eps));
    a.inv_eps_ff = ff2(ff_make(1.0 / eps));
    a.F = D1;
    a.Fff = make_div_ff(D1, eps);
    a.Z = Zd;
    a.err = err;
    const double* zc = zb;
    const double* lp = logp;
    const double* lw = logdx;
    if (ffm) return pdl_launch(k_mass_prox<true>, nblocks(n), st, zc, lp, U, lw, a);
    return pdl_launch(k_mass_prox<false>, nblocks(n), st, zc, lp, U, lw, a);
  };
  // One iteration.  a-side: with eps unchanged since the previous iteration the
  // b-side of that iteration has already computed this iteration's Z (Fubini,
  // k_mass_vupdate), so the prox of S + Z runs in the pass epilogue; otherwise
  // (the first iteration of a new eps stage) the z-update takes the plain route:
  // raw pass, k_mass_reduce, k_mass_prox.  The very first iteration keeps z = 1.
  // b-side: raw pass, then k_mass_vupdate (V and the next Z).
  double prev_eps = -1.0;
  auto iteration = [&](double eps, bool check, cudaStream_t st) -> cudaError_t {
    cudaError_t e;
    Epilogue r;
    memset(&r, 0, sizeof(r));
    r.mode = EPI_RAW;
    set_eps(r, eps);
    r.out = zb;
    r.bstride = n;
    const bool plain = !first && eps != prev_eps;
    if (plain) {
      if ((e = G.apply(0, V, logdy, eps, r, st)) != cudaSuccess) return e;
      MassArgs a;
      memset(&a, 0, sizeof(a));
      a.n = n;
      a.eps = eps;
      a.eps_ff = ff2(ff_make(eps));
      a.inv_eps_ff = ff2(ff_make(1.0 / eps));
      a.F3 = D3;
      a.F3ff = make_div_ff(D3, eps);
      a.logm0 = log(m0);
      a.logm0_ff = ff2(ff_make(log(m0)));
      a.update = 1;
      a.check = check ? 1 : 0;
      a.Z = Zd;
      a.acc = acc;
      a.part = part;
      a.count = count;
      const double* Uc = U;
      const double* zc = zb;
      const double* lw = logdx;
      e = ffm ? pdl_launch(k_mass_reduce<true>, red_blocks, st, Uc, zc, lw, a)
              : pdl_launch(k_mass_reduce<false>, red_blocks, st, Uc, zc, lw, a);
      if (e != cudaSuccess) return e;
      if ((e = prox_a(eps, check ? acc : nullptr, st)) != cudaSuccess) return e;
    } else {
      Epilogue e1 = prox_epilogue(D1, logp, U, logdx, check ? acc : nullptr, eps);
      e1.bstride = e1.bstride_p = n;
      e1.zshift = Zd;
      if ((e = G.apply(0, V, logdy, eps, e1, st, check ? acc : nullptr)) != cudaSuccess) return e;
    }
    first = false;
    prev_eps = eps;
    r.bstride = m;
    if ((e = G.apply(1, U, logdx, eps, r, st)) != cudaSuccess) return e;
    MassV b;
    memset(&b, 0, sizeof(b));
    b.m = m;
    b.eps = eps;
    b.eps_ff = ff2(ff_make(eps));
    b.inv_eps_ff = ff2(ff_make(1.0 / eps));
    b.F2 = D2;
    b.F3 = D3;
    b.F2ff = make_div_ff(D2, eps);
    b.F3ff = make_div_ff(D3, eps);
    b.logm0 = log(m0);
    b.logm0_ff = ff2(ff_make(log(m0)));
    b.Z = Zd;
    b.zhist = zhist;
    b.part = part;
    b.count = count;
    const double* zc = zb;
    const double* lq = logq;
    const double* lw = logdy;
    const int vb = (int)std::min<int64_t>(kNT, std::max<int64_t>(1, (m + per_block - 1) / per_block));
    return ffm ? pdl_launch(k_mass_vupdate<true>, vb, st, zc, lq, V, lw, b)
               : pdl_launch(k_mass_vupdate<false>, vb, st, zc, lq, V, lw, b);
  };
  // the checked iteration's violations: the marginal one from acc, and the mass
  // one |e^{(Z_old - Z)/eps} - 1| of its z-update from the history of Z (after
  // the iteration, zhist = {its Z, the previous Z})
  double hacc[2], hz[2];
  auto zval = [&](double v) {
    if (!ffm) return v;
    float2 f;
    memcpy(&f, &v, sizeof(f));
    return (double)f.x + (double)f.y;
  };
  auto read_err = [&](double& out) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(hacc, acc, sizeof(hacc), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(hz, zhist, sizeof(hz), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    const double v = (hacc[1] > 0.0) ? hacc[0] / hacc[1] : 0.0;
    const double zn = zval(hz[0]), zo = zval(hz[1]);
    const double merr = (std::isfinite(zn) && std::isfinite(zo)) ? std::fabs(std::expm1((zo - zn) / o->eps)) : 0.0;
    out = (v != v) ? NAN : std::max(v, merr);
    return cudaSuccess;
  };

  const std::vector<Stage> stages = eps_schedule(*o);
  const int check_every = o->check_every > 0 ? o->check_every : 1;
  int it = 0, total = 0;
  double err = INFINITY;
  bool converged = false;
  for (const Stage& sg : stages)
    for (int k = 0; k < sg.iters; ++k, ++total) UOT_CK(iteration(sg.eps, false, s));
  // launch_mode 2 (and 1, 3, which have no mass variant): blocks of
  // check_every iterations at the final eps replayed as one CUDA graph.
  BlockGraph bg;
  bool graph_ok = o->launch_mode != 0 && !profiling_on();
  while (it < o->max_iter) {
    if (graph_ok && !first && it > 0 && it % check_every == 0 && it + check_every <= o->max_iter) {
      if (!bg.exec) {
        cudaError_t e = bg.capture([&](cudaStream_t cs) -> cudaError_t {
          for (int k = 0; k < check_every; ++k) {
            cudaError_t e2 = iteration(o->eps, k == check_every - 1, cs);
            if (e2 != cudaSuccess) return e2;
          }
          return cudaSuccess;
        });
        if (e != cudaSuccess) {
          graph_ok = false;
          (void)cudaGetLastError();
          continue;
        }
      }
      UOT_CK(bg.launch(s));
      it += check_every;
      total += check_every;
      UOT_CK(read_err(err));
      if (o->tol > 0.0 && err <= o->tol) {
        converged = true;
        break;
      }
      continue;
    }
    const bool check = ((it + 1) % check_every == 0) || (it == o->max_iter - 1);
    UOT_CK(iteration(o->eps, check, s));
    ++it;
    ++total;
    if (check) {
      UOT_CK(read_err(err));
      if (it > 1 && o->tol > 0.0 && err <= o->tol) {
        converged = true;
        break;
      }
    }
  }

  UOT_CK(cudaMemsetAsync(flag, 0, 4, s));
  count_launches(1);
  k_nan_flag<<<nblocks(n), kNT, 0, s>>>(U, n, ffm, flag);
  count_launches(1);
  k_nan_flag<<<nblocks(m), kNT, 0, s>>>(V, m, ffm, flag);
  UOT_CK(cudaGetLastError());
  UOT_CK(from_f64(prec, U, n, Uout, s));
  UOT_CK(from_f64(prec, V, m, Vout, s));
  UOT_CK(cudaEventRecord(ev1, s));
  int hflag = 0, htc = 0;
  double hZ = 0.0;
  UOT_CK(cudaMemcpyAsync(&hflag, flag, 4, cudaMemcpyDeviceToHost, s));
  UOT_CK(cudaMemcpyAsync(&hZ, zhist, 8, cudaMemcpyDeviceToHost, s));  // the Z of the last iteration
  if (G.tc_err) UOT_CK(cudaMemcpyAsync(&htc, G.tc_err, 4, cudaMemcpyDeviceToHost, s));
  UOT_CK(cudaStreamSynchronize(s));
  if (ffm) {
    float2 zz;
    memcpy(&zz, &hZ, sizeof(zz));
    hZ = (double)zz.x + (double)zz.y;
  }
  *Zout = hZ;
  float ms = 0.f;
  UOT_CK(cudaEventElapsedTime(&ms, ev0, ev1));
  uot_status out = htc ? UOT_TIMEOUT
                       : (hflag || hZ != hZ) ? UOT_NUMERICAL
                                             : ((o->tol > 0.0 && !converged && o->max_iter > 0) ? UOT_NOT_CONVERGED : UOT_OK);
  if (res) {
    *res = empty_result();
    res->iters = it;
    res->total_iters = total;
    res->marg_err = err;
    res->ms = ms;
    res->status = out;
  }
  return out;
}

}  // namespace
}  // namespace uot

using namespace uot;

extern "C" {

uot_status uot_solve_mass(const uot_geom* g, const void* p, const void* dx, const void* q,
                          const void* dy, const uot_div* F1, const uot_div* F2, const uot_div* F3,
                          double m0, const uot_opts* o, void* U, void* V, double* Z, uot_result* res,
                          void* stream) {
  clear_stale_error();
  return solve_mass_impl(g, p, dx, q, dy, F1, F2, F3, m0, o, U, V, Z, res, (cudaStream_t)stream);
}

}  // extern "C"

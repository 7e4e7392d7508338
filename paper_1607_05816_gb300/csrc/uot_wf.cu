// uot_wf_cost and uot_wf_flow: the WF cost (eq. logcost) and the WF gradient
// flows with growth of Sec. 5.3.
#include "uot_host.cuh"

namespace uot {
namespace {

// ---------------------------------------------------------------------------
// WF gradient flows with growth (Sec. 5.3)
// ---------------------------------------------------------------------------
// Each minimizing-movement step (eq. grad-flow) solves, for S species on the
// same points (X = Y, dy = dx), the scaling iteration with F1 = lam KL(.|p^k)
// per species and the joint F2 of the growth functional
// G = -alpha sum_k mu^k(X) + iota_{<=1}(sum_k d mu^k/dx).  F2's log-form
// proxdiv is the same for every species:
//   V^k = min(-lam log c, -lam Ttot/(lam + eps)),  Ttot = eps log sum_k e^{T^k/eps},
// c = 1 - 2 tau alpha/lam.  The step ends with the next densities
// p^k = r2^k / max(c, sum_k r2^k), r2^k = e^{(V^k + T^k)/eps} the second
// marginals of the step's couplings.

// WF cost (eq. logcost) c = -log cos^2((pi/2)|x - y|/cut), +inf from |x - y| >= cut.
template <typename T>
__global__ void k_wf_cost(const T* __restrict__ x, int n, const T* __restrict__ y, int m, int d, double cut,
                          T* __restrict__ C) {
  const int64_t total = (int64_t)n * m;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / m, j = q - i * m;
    double r2 = 0.0;
    for (int k = 0; k < d; ++k) {
      const double t = (double)x[i * d + k] - (double)y[j * d + k];
      r2 += t * t;
    }
    const double dist = sqrt(r2);
    const double v = (dist >= cut) ? kInf : -2.0 * log(cos(1.5707963267948966 * dist / cut));
    C[q] = (T)v;
  }
}

struct GrowthArgs {
  int S;
  int64_t m;
  double eps, inv_eps, neg_lam_logc, klin, c;  // klin = lam/(lam + eps)
  float2 eps_ff, inv_eps_ff, neg_lam_logc_ff, klin_ff;
};

template <bool FF>
__global__ void __launch_bounds__(kNT) k_growth_prox(const double* __restrict__ Tz, double* __restrict__ V,
                                                     GrowthArgs a) {
  pdl_begin();
  for (int64_t j = blockIdx.x * (int64_t)kNT + threadIdx.x; j < a.m; j += (int64_t)gridDim.x * kNT) {
    if constexpr (!FF) {
      double mx = -kInf;
      for (int k = 0; k < a.S; ++k) mx = fmax(mx, Tz[k * a.m + j]);
      double v = a.neg_lam_logc;
      if (mx != -kInf) {
        double L = mx;  // one species: the log-sum-exp is the value itself
        if (a.S > 1) {
          double s = 0.0;
          for (int k = 0; k < a.S; ++k) s += exp(Tz[k * a.m + j] - mx);
          L += log(s);
        }
        v = fmin(v, -a.klin * (a.eps * L));
      }
      for (int k = 0; k < a.S; ++k) V[k * a.m + j] = v;
    } else {
      const float2* T2 = reinterpret_cast<const float2*>(Tz);
      ff mx = ff_ninf();
      for (int k = 0; k < a.S; ++k) mx = ff_max(mx, ffl(T2[k * a.m + j]));
      ff v = ffl(a.neg_lam_logc_ff);
      if (mx.hi != -INFINITY) {
        ff L = mx;  // one species: the log-sum-exp is the value itself
        if (a.S > 1) {
          float s = 0.0f;
          for (int k = 0; k < a.S; ++k) {
            const ff t = ffl(T2[k * a.m + j]);
            if (t.hi == -INFINITY) continue;
            const ff dlt = ff_sub(t, mx);
            s += expf(dlt.hi + dlt.lo);
          }
          L = ff_add_f(mx, logf(s));
        }
        v = ff_min(v, ff_neg(ff_mul(ffl(a.klin_ff), ff_mul(ffl(a.eps_ff), L))));
      }
      float2* V2 = reinterpret_cast<float2*>(V);
      for (int k = 0; k < a.S; ++k) V2[k * a.m + j] = ff2(v);
    }
  }
}

// Next densities from the plan's second marginals; writes the log densities
// (the next step's F1 targets) and the densities in the caller's type.
template <bool FF>
__global__ void __launch_bounds__(kNT) k_growth_density(const double* __restrict__ Tz, const double* __restrict__ V,
                                                        GrowthArgs a, double* __restrict__ logp, void* __restrict__ pout) {
  for (int64_t j = blockIdx.x * (int64_t)kNT + threadIdx.x; j < a.m; j += (int64_t)gridDim.x * kNT) {
    if constexpr (!FF) {
      double tot = 0.0;
      for (int k = 0; k < a.S; ++k) {
        const double z = Tz[k * a.m + j], v = V[k * a.m + j];
        tot += (z == -kInf || v == -kInf) ? 0.0 : exp(v * a.inv_eps + z);
      }
      const double den = fmax(a.c, tot), lden = log(den);
      for (int k = 0; k < a.S; ++k) {
        const int64_t q = k * a.m + j;
        const double z = Tz[q], v = V[q];
        const bool zero = (z == -kInf || v == -kInf);
        const double lr = zero ? -kInf : v * a.inv_eps + z;
        logp[q] = zero ? -kInf : lr - lden;
        reinterpret_cast<double*>(pout)[q] = zero ? 0.0 : exp(lr) / den;
      }
    } else {
      const float2* T2 = reinterpret_cast<const float2*>(Tz);
      const float2* V2 = reinterpret_cast<const float2*>(V);
      const ff ie = ffl(a.inv_eps_ff);
      float tot = 0.0f;
      for (int k = 0; k < a.S; ++k) {
        const ff z = ffl(T2[k * a.m + j]), v = ffl(V2[k * a.m + j]);
        if (z.hi == -INFINITY || v.hi == -INFINITY) continue;
        const ff lr = ff_add(ff_mul(v, ie), z);
        tot += expf(lr.hi + lr.lo);
      }
      const float den = fmaxf((float)a.c, tot), lden = logf(den);
      for (int k = 0; k < a.S; ++k) {
        const int64_t q = k * a.m + j;
        const ff z = ffl(T2[q]), v = ffl(V2[q]);
        float2* lp2 = reinterpret_cast<float2*>(logp);
        if (z.hi == -INFINITY || v.hi == -INFINITY) {
          lp2[q] = ff2(ff_ninf());
          reinterpret_cast<float*>(pout)[q] = 0.0f;
          continue;
        }
        const ff lp = ff_add_f(ff_add(ff_mul(v, ie), z), -lden);
        lp2[q] = ff2(lp);
        reinterpret_cast<float*>(pout)[q] = expf(lp.hi + lp.lo);
      }
    }
  }
}

uot_status wf_flow_impl(const uot_geom* g, int S, const void* P0, const void* dx, double tau, double alpha,
                        double lam, const uot_opts* o, int nsteps, void* Pout, void* Uout, void* Vout,
                        uot_result* res, cudaStream_t s) {
  uot_status st = check_geom(g);
  if (st != UOT_OK) return st;
  if ((st = check_opts(o)) != UOT_OK) return st;
  if (g->n != g->m || S < 1 || nsteps < 1 || !P0 || !dx || !Pout || !Uout || !Vout) return UOT_EINVAL;
  if (!(tau > 0.0) || !isfinite(tau) || !(alpha >= 0.0) || !isfinite(alpha) || !(lam > 0.0) || !isfinite(lam))
    return UOT_EINVAL;
  const double c = 1.0 - 2.0 * tau * alpha / lam;
  if (!(c > 0.0 && c <= 1.0)) return UOT_EINVAL;
  if (o->tol != 0.0 || o->U0 || o->V0) return UOT_EINVAL;
  if (o->plain_scaling || o->precision == UOT_MIXED) return UOT_EUNSUPPORTED;
  if (g->kind == UOT_GEOM_GRID && S > 65535) return UOT_EUNSUPPORTED;
  const int prec = o->precision;
  const bool ffm = prec != UOT_F64;
  const size_t esz = ffm ? 4 : 8;
  const int64_t n = g->n, Sn = (int64_t)S * n;

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
  G.plan(sc, S);
  sc.reserve<double>(Sn);        // log p^k (F1 targets)
  sc.reserve<double>(n);         // log dx
  sc.reserve<double>(Sn);        // U
  sc.reserve<double>(Sn);        // V
  sc.reserve<double>(Sn);        // raw log-sums T^k/eps
  sc.reserve<char>(Sn * esz);    // densities of the current step
  sc.reserve<int>(1);            // NaN flag
  UOT_CK(sc.allocate());
  UOT_CK(G.take(sc, s));
  double* logp = sc.take<double>(Sn);
  double* logdx = sc.take<double>(n);
  double* U = sc.take<double>(Sn);
  double* V = sc.take<double>(Sn);
  double* Tz = sc.take<double>(Sn);
  char* pstep = sc.take<char>(Sn * esz);
  int* flag = sc.take<int>(1);
  UOT_SCRATCH_OK(sc);
  UOT_CK(to_log(prec, P0, Sn, logp, s));
  UOT_CK(to_log(prec, dx, n, logdx, s));

  const DivParams D1 = make_div(uot_div{UOT_DIV_KL, lam, 0.0, 0.0});
  auto gargs = [&](double eps) {
    GrowthArgs a;
    memset(&a, 0, sizeof(a));
    a.S = S;
    a.m = n;
    a.eps = eps;
    a.inv_eps = 1.0 / eps;
    a.neg_lam_logc = -lam * log(c);
    a.klin = lam / (lam + eps);
    a.c = c;
    a.eps_ff = ff2(ff_make(eps));
    a.inv_eps_ff = ff2(ff_make(1.0 / eps));
    a.neg_lam_logc_ff = ff2(ff_make(-lam * log(c)));
    a.klin_ff = ff2(ff_make(lam / (lam + eps)));
    return a;
  };
  auto iteration = [&](double eps, cudaStream_t st) -> cudaError_t {
    cudaError_t e;
    Epilogue e1 = prox_epilogue(D1, logp, U, logdx, nullptr, eps);
    e1.bstride = e1.bstride_p = n;
    if ((e = G.apply(0, V, logdx, eps, e1, st)) != cudaSuccess) return e;
    Epilogue r;
    memset(&r, 0, sizeof(r));
    r.mode = EPI_RAW;
    set_eps(r, eps);
    r.out = Tz;
    r.bstride = n;
    if ((e = G.apply(1, U, logdx, eps, r, st)) != cudaSuccess) return e;
    count_launches(1);
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(nblocks(n));
    cfg.blockDim = dim3(kNT);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const double* tz = Tz;
    return ffm ? cudaLaunchKernelEx(&cfg, k_growth_prox<true>, tz, V, gargs(eps))
               : cudaLaunchKernelEx(&cfg, k_growth_prox<false>, tz, V, gargs(eps));
  };
  const std::vector<Stage> stages = eps_schedule(*o);
  int stage_iters = 0;
  for (const Stage& sg : stages) stage_iters += sg.iters;
  auto step = [&](cudaStream_t st) -> cudaError_t {
    cudaError_t e;
    count_launches(2);
    k_fill<<<nblocks(Sn), kNT, 0, st>>>(U, Sn, 0.0);
    k_fill<<<nblocks(Sn), kNT, 0, st>>>(V, Sn, 0.0);  // b = 1 (both layouts)
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (const Stage& sg : stages)
      for (int k = 0; k < sg.iters; ++k)
        if ((e = iteration(sg.eps, st)) != cudaSuccess) return e;
    for (int k = 0; k < o->max_iter; ++k)
      if ((e = iteration(o->eps, st)) != cudaSuccess) return e;
    count_launches(1);
    if (ffm)
      k_growth_density<true><<<nblocks(n), kNT, 0, st>>>(Tz, V, gargs(o->eps), logp, pstep);
    else
      k_growth_density<false><<<nblocks(n), kNT, 0, st>>>(Tz, V, gargs(o->eps), logp, pstep);
    return cudaGetLastError();
  };
  // launch_mode 2: the first step runs launch by launch; later steps replay
  // it as one CUDA graph (the step repeats the same launches).
  BlockGraph bg;
  bool graph_ok = o->launch_mode != 0 && !profiling_on();
  for (int k = 0; k < nsteps; ++k) {
    if (graph_ok && k > 0) {
      if (!bg.exec) {
        cudaError_t e = bg.capture([&](cudaStream_t cs) { return step(cs); });
        if (e != cudaSuccess) {
          graph_ok = false;
          (void)cudaGetLastError();
        }
      }
    }
    if (graph_ok && bg.exec)
      UOT_CK(bg.launch(s));
    else
      UOT_CK(step(s));
    UOT_CK(cudaMemcpyAsync((char*)Pout + (size_t)k * Sn * esz, pstep, Sn * esz, cudaMemcpyDeviceToDevice, s));
  }

  UOT_CK(cudaMemsetAsync(flag, 0, 4, s));
  count_launches(2);
  k_nan_flag<<<nblocks(Sn), kNT, 0, s>>>(U, Sn, ffm, flag);
  k_nan_flag<<<nblocks(Sn), kNT, 0, s>>>(V, Sn, ffm, flag);
  UOT_CK(cudaGetLastError());
  UOT_CK(from_f64(prec, U, Sn, Uout, s));
  UOT_CK(from_f64(prec, V, Sn, Vout, s));
  UOT_CK(cudaEventRecord(ev1, s));
  int hflag = 0, htc = 0;
  UOT_CK(cudaMemcpyAsync(&hflag, flag, 4, cudaMemcpyDeviceToHost, s));
  if (G.tc_err) UOT_CK(cudaMemcpyAsync(&htc, G.tc_err, 4, cudaMemcpyDeviceToHost, s));
  UOT_CK(cudaStreamSynchronize(s));
  float ms = 0.f;
  UOT_CK(cudaEventElapsedTime(&ms, ev0, ev1));
  const uot_status out = htc ? UOT_TIMEOUT : hflag ? UOT_NUMERICAL : UOT_OK;
  if (res) {
    *res = empty_result();
    res->iters = o->max_iter;
    res->total_iters = nsteps * (stage_iters + o->max_iter);
    res->marg_err = NAN;
    res->ms = ms;
    res->status = out;
  }
  return out;
}

}  // namespace
}  // namespace uot

using namespace uot;

extern "C" {

uot_status uot_wf_cost(const void* x, int n, const void* y, int m, int d, double cut, int precision,
                       void* C, void* stream) {
  clear_stale_error();
  if (!x || !y || !C || n < 1 || m < 1 || d < 1 || d > 8 || !(cut > 0.0) || !isfinite(cut) ||
      (precision != UOT_F64 && precision != UOT_F32))
    return UOT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t total = (int64_t)n * m;
  const int grid = (int)std::min<int64_t>((total + kNT - 1) / kNT, 152 * 16);
  count_launches(1);
  if (precision == UOT_F64)
    k_wf_cost<double><<<grid, kNT, 0, s>>>((const double*)x, n, (const double*)y, m, d, cut, (double*)C);
  else
    k_wf_cost<float><<<grid, kNT, 0, s>>>((const float*)x, n, (const float*)y, m, d, cut, (float*)C);
  UOT_CK(cudaGetLastError());
  return UOT_OK;
}

uot_status uot_wf_flow(const uot_geom* g, int nspecies, const void* P0, const void* dx, double tau,
                       double alpha, double lambda, const uot_opts* o, int nsteps, void* P, void* U,
                       void* V, uot_result* res, void* stream) {
  clear_stale_error();
  return wf_flow_impl(g, nspecies, P0, dx, tau, alpha, lambda, o, nsteps, P, U, V, res, (cudaStream_t)stream);
}

}  // extern "C"

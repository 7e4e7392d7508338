// uot_barycenter and uot_barycenter_div: unbalanced barycenters (Sec. 5.2,
// Table 2) driven by the scaling iteration.
#include "uot_host.cuh"

using namespace uot;

static uot_status barycenter_impl(const uot_geom* g, int Kmeas, const double* alpha, const void* P,
                                  const void* dx, const void* dy, const uot_div* F1, double lambda,
                                  int bary_kind, double beta1, double beta2, const uot_opts* o, void* logh_out,
                                  void* Uout, void* Vout, uot_result* res, void* stream);

extern "C" {

uot_status uot_barycenter(const uot_geom* g, int Kmeas, const double* alpha, const void* P,
                          const void* dx, const void* dy, const uot_div* F1, double lambda,
                          int bary_kind, const uot_opts* o, void* logh_out, void* Uout,
                          void* Vout, uot_result* res, void* stream) {
  clear_stale_error();
  if (bary_kind == UOT_BARY_RG) return UOT_EINVAL;  // its range needs uot_barycenter_div
  return barycenter_impl(g, Kmeas, alpha, P, dx, dy, F1, lambda, bary_kind, 1.0, 1.0, o, logh_out, Uout, Vout,
                         res, stream);
}

uot_status uot_barycenter_div(const uot_geom* g, int Kmeas, const double* alpha, const void* P,
                              const void* dx, const void* dy, const uot_div* F1, const uot_div* Fh,
                              const uot_opts* o, void* logh_out, void* Uout, void* Vout, uot_result* res,
                              void* stream) {
  clear_stale_error();
  if (!Fh) return UOT_EINVAL;
  switch (Fh->kind) {
    case UOT_DIV_EQ:
      return barycenter_impl(g, Kmeas, alpha, P, dx, dy, F1, 1.0, UOT_BARY_EQ, 1.0, 1.0, o, logh_out, Uout, Vout,
                             res, stream);
    case UOT_DIV_KL:
      return barycenter_impl(g, Kmeas, alpha, P, dx, dy, F1, Fh->lambda, UOT_BARY_KL, 1.0, 1.0, o, logh_out, Uout,
                             Vout, res, stream);
    case UOT_DIV_TV:
      return barycenter_impl(g, Kmeas, alpha, P, dx, dy, F1, Fh->lambda, UOT_BARY_TV, 1.0, 1.0, o, logh_out, Uout,
                             Vout, res, stream);
    case UOT_DIV_RG:
      return barycenter_impl(g, Kmeas, alpha, P, dx, dy, F1, 1.0, UOT_BARY_RG, Fh->alpha, Fh->beta, o, logh_out,
                             Uout, Vout, res, stream);
    default:
      return UOT_EINVAL;
  }
}

}  // extern "C"

static uot_status barycenter_impl(const uot_geom* g, int Kmeas, const double* alpha, const void* P,
                                  const void* dx, const void* dy, const uot_div* F1, double lambda,
                                  int bary_kind, double beta1, double beta2, const uot_opts* o, void* logh_out,
                                  void* Uout, void* Vout, uot_result* res, void* stream) {
  uot_status st = check_geom(g);
  if (st != UOT_OK) return st;
  if ((st = check_opts(o)) != UOT_OK) return st;
  if (Kmeas < 1 || !alpha || !P || !dx || !dy || !div_ok(F1) || !logh_out || !Uout || !Vout)
    return UOT_EINVAL;
  if (bary_kind != UOT_BARY_KL && bary_kind != UOT_BARY_EQ && bary_kind != UOT_BARY_TV && bary_kind != UOT_BARY_RG)
    return UOT_EINVAL;
  if ((bary_kind == UOT_BARY_KL || bary_kind == UOT_BARY_TV) && !(lambda > 0.0)) return UOT_EINVAL;
  if (bary_kind == UOT_BARY_RG && !(beta1 > 0.0 && beta1 <= beta2 && beta2 < kInf)) return UOT_EINVAL;
  if ((bary_kind == UOT_BARY_TV || bary_kind == UOT_BARY_RG) && Kmeas > 1024) return UOT_EINVAL;
  if (o->plain_scaling) return UOT_EUNSUPPORTED;
  double sum_alpha = 0.0;
  for (int k = 0; k < Kmeas; ++k) {
    if (!(alpha[k] > 0.0) || !isfinite(alpha[k])) return UOT_EINVAL;
    sum_alpha += alpha[k];
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int prec = o->precision;
  const int64_t n = g->n, m = g->m;
  const DivParams D1 = make_div(*F1);

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
  G.plan(sc, Kmeas);
  sc.reserve<double>(n * Kmeas);  // logP
  sc.reserve<double>(n * Kmeas);  // U
  sc.reserve<double>(n);          // logdx
  sc.reserve<double>(m * Kmeas);  // V
  sc.reserve<double>(m * Kmeas);  // T
  sc.reserve<double>(m);          // logdy
  sc.reserve<double>(m);          // logh
  sc.reserve<double>(Kmeas);      // alpha
  sc.reserve<float>(Kmeas);       // log alpha (FP32 path)
  sc.reserve<double>(2 * (size_t)Kmeas);  // violation accumulators per measure
  UOT_CK(sc.allocate());
  UOT_CK(G.take(sc, s));
  double* logP = sc.take<double>(n * Kmeas);
  double* U = sc.take<double>(n * Kmeas);
  double* logdx = sc.take<double>(n);
  double* V = sc.take<double>(m * Kmeas);
  double* T = sc.take<double>(m * Kmeas);
  double* logdy = sc.take<double>(m);
  double* logh = sc.take<double>(m);
  double* alpha_d = sc.take<double>(Kmeas);
  float* log_alpha_d = sc.take<float>(Kmeas);
  double* acc = sc.take<double>(2 * (size_t)Kmeas);
  std::vector<double> acc_h(2 * (size_t)Kmeas);
  UOT_SCRATCH_OK(sc);
  UOT_CK(to_log(prec, P, n * Kmeas, logP, s));
  UOT_CK(to_log(prec, dx, n, logdx, s));
  UOT_CK(to_log(prec, dy, m, logdy, s));
  UOT_CK(cudaMemcpyAsync(alpha_d, alpha, Kmeas * 8, cudaMemcpyHostToDevice, s));
  std::vector<float> log_alpha_h(Kmeas);
  for (int k = 0; k < Kmeas; ++k) log_alpha_h[k] = (float)log(alpha[k]);
  UOT_CK(cudaMemcpyAsync(log_alpha_d, log_alpha_h.data(), Kmeas * 4, cudaMemcpyHostToDevice, s));
  // pageable source: make sure the copy has consumed it before the vector dies
  UOT_CK(cudaStreamSynchronize(s));
  count_launches(1);
  k_fill<<<nblocks(n * Kmeas), kNT, 0, s>>>(U, n * Kmeas, 0.0);
  count_launches(1);
  k_fill<<<nblocks(m * Kmeas), kNT, 0, s>>>(V, m * Kmeas, 0.0);
  UOT_CK(cudaGetLastError());

  auto iteration = [&](double eps, bool check, cudaStream_t st) -> cudaError_t {
    cudaError_t e;
    Epilogue e1 = prox_epilogue(D1, logP, U, logdx, check ? acc : nullptr, eps);
    e1.bstride = n;
    e1.bstride_p = n;
    if ((e = G.apply(0, V, logdy, eps, e1, st, check ? acc : nullptr)) != cudaSuccess) return e;
    Epilogue e2;
    memset(&e2, 0, sizeof(e2));
    e2.mode = EPI_SCALE;
    set_eps(e2, eps);
    e2.out = T;
    e2.bstride = m;
    count_launches(1);
    if ((e = G.apply(1, U, logdx, eps, e2, st)) != cudaSuccess) return e;
    if (prec == UOT_F64) {
      k_bary_update<<<nblocks(m), kNT, 0, st>>>(T, Kmeas, m, alpha_d, sum_alpha, lambda, eps,
                                                bary_kind, beta1, beta2, logh, V);
    } else {
      DivParams Dh;
      Dh.kind = (bary_kind == UOT_BARY_KL) ? UOT_DIV_KL : (bary_kind == UOT_BARY_TV) ? UOT_DIV_TV
                : (bary_kind == UOT_BARY_RG) ? UOT_DIV_RG : UOT_DIV_EQ;
      Dh.lam = lambda;
      Dh.log_alpha = (bary_kind == UOT_BARY_RG) ? log(beta1) : 0.0;
      Dh.log_beta = (bary_kind == UOT_BARY_RG) ? log(beta2) : 0.0;
      BaryPL pl;
      pl.lam = (float)lambda;
      pl.b1 = (float)beta1;
      pl.b2 = (float)beta2;
      pl.elb1 = (float)(eps * log(beta1));
      pl.elb2 = (float)(eps * log(beta2));
      cudaLaunchConfig_t cfg;
      memset(&cfg, 0, sizeof(cfg));
      cfg.gridDim = dim3((unsigned)std::min<int64_t>((m + kBJ - 1) / kBJ, 1 << 20));
      cfg.blockDim = dim3(kBJ, kBK);
      cfg.stream = st;
      // a plain (fully serialised) launch: measured faster here than a
      // programmatic dependent launch, whose early-launched successor CTAs
      // compete with this small grid
      cfg.attrs = nullptr;
      cfg.numAttrs = 0;
      const bool pwl = bary_kind == UOT_BARY_TV || bary_kind == UOT_BARY_RG;
      cfg.dynamicSmemBytes = pwl ? (size_t)Kmeas * (kBJ + 1) * sizeof(float) : 0;
      if (cfg.dynamicSmemBytes > 48 * 1024) {
        e = smem_at_least(k_bary_update_ff, cfg.dynamicSmemBytes);
        if (e != cudaSuccess) return e;
      }
      const double lam_kl = (bary_kind == UOT_BARY_KL) ? lambda : 1.0;
      e = cudaLaunchKernelEx(&cfg, k_bary_update_ff, (const double*)T, Kmeas, (int64_t)m, (const float*)log_alpha_d,
                             (float)log(sum_alpha), ff2(ff_make(eps + lam_kl)), ff2(ff_make(1.0 / (eps + lam_kl))),
                             ff2(ff_make(1.0 / eps)), ff2(ff_make(eps)), bary_kind, make_div_ff(Dh, eps), pl, logh, V);
      if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
  };
  const std::vector<Stage> stages = eps_schedule(*o);
  const int check_every = o->check_every > 0 ? o->check_every : 1;
  int it = 0, total = 0;
  double err = INFINITY;
  bool converged = false;
  for (const Stage& sg : stages)
    for (int k = 0; k < sg.iters; ++k, ++total) UOT_CK(iteration(sg.eps, false, s));
  // launch_mode 2: checked blocks of check_every iterations replayed from a CUDA graph
  BlockGraph bg;
  bool graph_ok = o->launch_mode == 2 && !profiling_on();
  while (it < o->max_iter) {
    bool check;
    if (graph_ok && it > 0 && it % check_every == 0 && it + check_every <= o->max_iter) {
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
      check = true;
    } else {
      check = ((it + 1) % check_every == 0) || (it == o->max_iter - 1);
      UOT_CK(iteration(o->eps, check, s));
      ++it;
      ++total;
    }
    if (check) {
      UOT_CK(cudaMemcpyAsync(acc_h.data(), acc, 16 * (size_t)Kmeas, cudaMemcpyDeviceToHost, s));
      UOT_CK(cudaStreamSynchronize(s));
      double h[2] = {0.0, 0.0};
      for (int k = 0; k < Kmeas; ++k) {
        h[0] += acc_h[2 * k];
        h[1] += acc_h[2 * k + 1];
      }
      err = (h[1] > 0.0) ? h[0] / h[1] : 0.0;
      if (it > 1 && o->tol > 0.0 && err <= o->tol) {
        converged = true;
        break;
      }
    }
  }
  UOT_CK(from_f64(prec, U, n * Kmeas, Uout, s));
  UOT_CK(from_f64(prec, V, m * Kmeas, Vout, s));
  UOT_CK(from_f64(prec, logh, m, logh_out, s));
  UOT_CK(cudaEventRecord(ev1, s));
  UOT_CK(cudaStreamSynchronize(s));
  float ms = 0.f;
  UOT_CK(cudaEventElapsedTime(&ms, ev0, ev1));
  uot_status out = (o->tol > 0.0 && !converged && o->max_iter > 0) ? UOT_NOT_CONVERGED : UOT_OK;
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

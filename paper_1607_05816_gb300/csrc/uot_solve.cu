// uot_solve, uot_solve_many and uot_solve_batch: the scaling iteration (eq. S,
// Sec. 3.3) in the log form of Sec. 4.3 with eps-scaling (Sec. 4.4), the
// FP64-confirmed stop, the translation step, and the batched persistent solver.
#include "uot_host.cuh"

namespace uot {
namespace {

// ---------------------------------------------------------------------------
// solve
// ---------------------------------------------------------------------------

// `batch` independent problems sharing the geometry, eps and penalties: p, U
// are [batch][n], q, V are [batch][m]; dx, dy are shared.  The iteration stops
// when every problem's violation is <= tol (the reported error is the largest).
uot_status solve_impl(const uot_geom* g, int batch, const void* p, const void* dx, const void* q,
                      const void* dy, const uot_div* F1, const uot_div* F2, const uot_opts* o,
                      void* Uout, void* Vout, uot_result* res, cudaStream_t s) {
  uot_status st = check_geom(g);
  if (st != UOT_OK) return st;
  if ((st = check_opts(o, true)) != UOT_OK) return st;
  if (batch < 1 || !p || !dx || !q || !dy || !Uout || !Vout || !div_ok(F1) || !div_ok(F2))
    return UOT_EINVAL;
  if (o->plain_scaling && (g->kind != UOT_GEOM_DENSE || o->precision != UOT_F64 || batch != 1))
    return UOT_EUNSUPPORTED;
  if (g->kind == UOT_GEOM_GRID && batch > 65535) return UOT_EUNSUPPORTED;
  const bool translate = o->translate != 0;
  if (translate && (F1->kind != UOT_DIV_KL || F2->kind != UOT_DIV_KL || o->plain_scaling || batch > 65535))
    return UOT_EUNSUPPORTED;
  const int prec = o->precision;
  const int64_t n = g->n, m = g->m;
  const int64_t bn = n * batch, bm = m * batch;
  const DivParams D1 = make_div(*F1), D2 = make_div(*F2);

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
  G.plan(sc, batch);
  sc.reserve<double>(bn);  // logp
  sc.reserve<double>(n);   // logdx
  sc.reserve<double>(bn);  // U
  sc.reserve<double>(bm);  // logq
  sc.reserve<double>(m);   // logdy
  sc.reserve<double>(bm);  // V
  sc.reserve<double>(2 * (size_t)batch + 4);  // err accumulators + flag
  if (translate) sc.reserve<double2>(kl_translate_part_count(n, m, batch));
  // one persistent cooperative launch for FP32 grid problems
  const std::vector<Stage> stages_p = eps_schedule(*o);
  const int nst = (int)stages_p.size();
  const bool verify = o->verify && prec != UOT_F64 && o->tol > 0.0 && !o->plain_scaling;
  const bool persist = o->launch_mode == 1 && prec == UOT_F32 && g->kind == UOT_GEOM_GRID &&
                       batch == 1 && !o->plain_scaling && !verify && !translate;
  // two kernels per iteration, each fusing two passes on one line (2-D FP32 grids)
  const bool fused2d = o->launch_mode == 3 && prec == UOT_F32 && g->kind == UOT_GEOM_GRID && g->ndim == 2 &&
                       batch == 1 && !o->plain_scaling && !verify && !translate &&
                       grid_fused2_smem(std::max(g->shape_y[0], g->shape_x[1]), std::max(g->shape_x[0], g->shape_y[1])) <=
                           160 * 1024;
  if (persist) {
    sc.reserve<float2>(nst + 1);   // eps
    sc.reserve<float2>(nst + 1);   // 1/eps
    sc.reserve<float>(nst + 1);    // log2(e)/eps
    sc.reserve<DivFF>(2 * (nst + 1));
    sc.reserve<unsigned>(2);       // barrier
    sc.reserve<int>(4);            // status
    sc.reserve<double>(1);         // last violation
  }
  if (o->plain_scaling) {
    sc.reserve<double>((size_t)n * m);  // K
    sc.reserve<double>((size_t)n * m);  // K^T
    for (int k = 0; k < 3; ++k) sc.reserve<double>(n);  // a, p, dx
    for (int k = 0; k < 3; ++k) sc.reserve<double>(m);  // b, q, dy
    sc.reserve<double>(4);                               // cluster solve's result
  }
  UOT_CK(sc.allocate());
  UOT_CK(G.take(sc, s));
  double* logp = sc.take<double>(bn);
  double* logdx = sc.take<double>(n);
  double* U = sc.take<double>(bn);
  double* logq = sc.take<double>(bm);
  double* logdy = sc.take<double>(m);
  double* V = sc.take<double>(bm);
  double* acc = sc.take<double>(2 * (size_t)batch + 4);
  int* flag = (int*)(acc + 2 * (size_t)batch);
  double2* trpart = translate ? sc.take<double2>(kl_translate_part_count(n, m, batch)) : nullptr;
  std::vector<double> acc_h(2 * (size_t)batch);
  UOT_SCRATCH_OK(sc);
  UOT_CK(to_log(prec, p, bn, logp, s));
  UOT_CK(to_log(prec, dx, n, logdx, s));
  UOT_CK(to_log(prec, q, bm, logq, s));
  UOT_CK(to_log(prec, dy, m, logdy, s));
  if (o->U0) {
    UOT_CK(to_f64(prec, o->U0, bn, U, s));
  } else {
    count_launches(1);
    k_fill<<<nblocks(bn), kNT, 0, s>>>(U, bn, 0.0);
  }
  if (o->V0) {
    UOT_CK(to_f64(prec, o->V0, bm, V, s));
  } else {
    count_launches(1);
    k_fill<<<nblocks(bm), kNT, 0, s>>>(V, bm, 0.0);
  }
  UOT_CK(cudaGetLastError());
  if (o->U0 || o->V0) {
    // a NaN or +inf start would spread through the log-sum-exps (all -inf, an empty plan)
    UOT_CK(cudaMemsetAsync(flag, 0, 4, s));
    count_launches(2);
    k_bad_start<<<nblocks(bn), kNT, 0, s>>>(U, bn, prec != UOT_F64, flag);
    k_bad_start<<<nblocks(bm), kNT, 0, s>>>(V, bm, prec != UOT_F64, flag);
    int hbad = 0;
    UOT_CK(cudaMemcpyAsync(&hbad, flag, 4, cudaMemcpyDeviceToHost, s));
    UOT_CK(cudaStreamSynchronize(s));
    if (hbad) {
      g_last_error = "uot_solve: the warm start U0/V0 holds NaN or +inf";
      return UOT_EINVAL;
    }
  }

  const std::vector<Stage> stages = eps_schedule(*o);
  const int check_every = o->check_every > 0 ? o->check_every : 1;
  int it = 0, total = 0;
  double err = INFINITY;
  bool converged = false;
  // opts.verify: FP64 confirmation of the stop, then FP64 iterations past the FP32 floor
  Check64 c64(s);
  double err32 = NAN, err64 = NAN, tol_int = o->tol;
  int nverify = 0, npolish = 0;
  bool polish = false, polished = false;
  // FP32 progress: first check at the final eps, best value so far (1% steps)
  double first_err = NAN, best_err = INFINITY;
  int first_it = 0, best_it = 0;
  // UOT_MIXED: the BF16 (tensor-core) phase, until the violation reaches mixed_switch
  bool mixed_phase = prec == UOT_MIXED && g->kind == UOT_GEOM_GRID && o->tol > 0.0;
  const double mixed_switch = o->mixed_switch > 0.0 ? o->mixed_switch : 1e-3;
  int mixed_iters = 0;
  bool mixed_handover = false;  // set by decide(): the graph block must be recaptured
  // verify on grids: iterations run with the float-float-exponent passes after
  // the FP32 check stalled (-1: not switched)
  int precise_from = -1;

  auto read_err = [&](double& out) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(acc_h.data(), acc, 16 * (size_t)batch, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    out = 0.0;
    for (int b = 0; b < batch; ++b) {
      const double v = (acc_h[2 * b + 1] > 0.0) ? acc_h[2 * b] / acc_h[2 * b + 1] : 0.0;
      out = (v > out || v != v) ? v : out;
    }
    return cudaSuccess;
  };
  if (persist) {
    std::vector<float2> heps(nst + 1), hieps(nst + 1);
    std::vector<float> hk2(nst + 1);
    std::vector<DivFF> hF(2 * (nst + 1));
    for (int sidx = 0; sidx <= nst; ++sidx) {
      const double e = (sidx < nst) ? stages_p[sidx].eps : o->eps;
      heps[sidx] = ff2(ff_make(e));
      hieps[sidx] = ff2(ff_make(1.0 / e));
      hk2[sidx] = (float)((double)kLog2e / e);
      hF[2 * sidx] = make_div_ff(D1, e);
      hF[2 * sidx + 1] = make_div_ff(D2, e);
    }
    float2* d_eps = sc.take<float2>(nst + 1);
    float2* d_ieps = sc.take<float2>(nst + 1);
    float* d_k2 = sc.take<float>(nst + 1);
    DivFF* d_F = sc.take<DivFF>(2 * (nst + 1));
    unsigned* d_bar = sc.take<unsigned>(2);
    int* d_status = sc.take<int>(4);
    double* d_err = sc.take<double>(1);
    UOT_SCRATCH_OK(sc);
    UOT_CK(cudaMemcpyAsync(d_eps, heps.data(), heps.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
    UOT_CK(cudaMemcpyAsync(d_ieps, hieps.data(), hieps.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
    UOT_CK(cudaMemcpyAsync(d_k2, hk2.data(), hk2.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    UOT_CK(cudaMemcpyAsync(d_F, hF.data(), hF.size() * sizeof(DivFF), cudaMemcpyHostToDevice, s));
    UOT_CK(cudaMemsetAsync(d_bar, 0, 2 * sizeof(unsigned), s));
    UOT_CK(cudaMemsetAsync(d_status, 0, 4 * sizeof(int), s));
    UOT_CK(cudaMemsetAsync(d_err, 0, sizeof(double), s));
    PersistLaunch L;
    memset(&L, 0, sizeof(L));
    L.ndim = g->ndim;
    int nin_max = 1;
    int64_t max_items = 1;
    for (int k = 0; k < g->ndim; ++k) {
      L.shape_x[k] = g->shape_x[k];
      L.shape_y[k] = g->shape_y[k];
      L.axes_x[k] = g->axes_x[k];
      L.axes_y[k] = g->axes_y[k];
      L.zbuf[0][k] = G.zbuf[0][k];
      L.zbuf[1][k] = G.zbuf[1][k];
      nin_max = std::max(nin_max, std::max(g->shape_x[k], g->shape_y[k]));
    }
    for (int dir = 0; dir < 2; ++dir) {
      const int* in_shape = dir == 0 ? g->shape_y : g->shape_x;
      const int* out_shape = dir == 0 ? g->shape_x : g->shape_y;
      for (int ax = 0; ax < g->ndim; ++ax) {
        int64_t nl = 1;
        for (int t = 0; t < ax; ++t) nl *= in_shape[t];
        for (int t = ax + 1; t < g->ndim; ++t) nl *= out_shape[t];
        max_items = std::max<int64_t>(max_items, nl * ((out_shape[ax] + 127) / 128));
      }
    }
    L.U = U;
    L.V = V;
    L.logp = logp;
    L.logq = logq;
    L.logdx = logdx;
    L.logdy = logdy;
    L.pass[0] = G.pass[0];
    L.pass[1] = G.pass[1];
    L.nstage = nst;
    L.iters_per_stage = o->iters_per_stage;
    L.max_iter = o->max_iter;
    L.check_every = check_every;
    L.tol = o->tol;
    L.eps_ff = d_eps;
    L.inv_eps_ff = d_ieps;
    L.k2 = d_k2;
    L.F = d_F;
    L.acc = acc;
    L.bar = d_bar;
    L.status = d_status;
    L.err_out = d_err;
    const int cap = grid_solve_persistent_ctas(nin_max);
    if (cap < 1) return UOT_EUNSUPPORTED;
    const int grid = (int)std::min<int64_t>(cap, max_items);
    UOT_CK(launch_grid_solve_persistent(L, grid, s));
    int hs[4];
    double herr = 0.0;
    UOT_CK(cudaMemcpyAsync(hs, d_status, sizeof(hs), cudaMemcpyDeviceToHost, s));
    UOT_CK(cudaMemcpyAsync(&herr, d_err, sizeof(double), cudaMemcpyDeviceToHost, s));
    UOT_CK(cudaStreamSynchronize(s));
    if (hs[0]) {
      g_last_error = "persistent solve: a grid barrier wait expired";
      return UOT_TIMEOUT;
    }
    converged = hs[1] != 0;
    it = hs[2];
    total = hs[3];
    err = (o->max_iter > 0) ? herr : INFINITY;
  } else if (fused2d) {
    // Pass order per iteration: P1 (contract j2 of V rows) | K_A: P2 (contract j1
    // -> U columns), P3 (contract i1 of the same columns) | K_B: P4 (contract i2
    // -> V rows), P1 of the next iteration (contract j2 of the same rows).
    const int H1 = g->shape_x[0], W1 = g->shape_x[1], H2 = g->shape_y[0], W2 = g->shape_y[1];
    const float* xa0 = (const float*)g->axes_x[0];
    const float* xa1 = (const float*)g->axes_x[1];
    const float* ya0 = (const float*)g->axes_y[0];
    const float* ya1 = (const float*)g->axes_y[1];
    float2* T1 = reinterpret_cast<float2*>(G.pass[0]);
    float2* T2 = reinterpret_cast<float2*>(G.pass[1]);
    float* z[4] = {G.zbuf[0][0], G.zbuf[0][1], G.zbuf[1][0], G.zbuf[1][1]};
    double zeps[4] = {-1.0, -1.0, -1.0, -1.0};
    auto use = [&](int k, double e) {
      const int u = (zeps[k] == e) ? 1 : 0;
      zeps[k] = e;
      return u;
    };
    auto p1 = [&](double e, cudaStream_t st) -> cudaError_t {
      Epilogue r;
      memset(&r, 0, sizeof(r));
      r.mode = EPI_RAW;
      r.eps = e;
      r.ff = 1;
      r.out = G.pass[0];
      r.bstride = (int64_t)H2 * W1;
      const int u = use(0, e);
      return launch_grid_pass(UOT_F32, V, logdy, 1, H2, W2, ya1, W1, xa1, e, 1, r, st, z[0], u);
    };
    auto fused_args = [&](double e) {
      FusedArgs f;
      memset(&f, 0, sizeof(f));
      f.eps1_ff = ff2(ff_make(e));
      f.inv_eps1_ff = ff2(ff_make(1.0 / e));
      f.k2_1 = (float)((double)kLog2e / e);
      f.do2 = 1;
      return f;
    };
    auto ka = [&](double e, bool check, cudaStream_t st) -> cudaError_t {
      if (check) {
        cudaError_t e0 = cudaMemsetAsync(acc, 0, 2 * sizeof(double), st);
        if (e0 != cudaSuccess) return e0;
      }
      FusedArgs f = fused_args(e);
      f.nlines = W1;
      f.in1 = T1;
      f.nin1 = H2;
      f.nout1 = H1;
      f.y1 = ya0;
      f.x1 = xa0;
      f.out1_row = 0;
      f.F1 = make_div_ff(D1, e);
      f.logp1 = reinterpret_cast<const float2*>(logp);
      f.pot1 = reinterpret_cast<float2*>(U);
      f.logw1 = reinterpret_cast<const float2*>(logdx);
      f.err = check ? acc : nullptr;
      f.z1 = z[1];
      f.use_prev1 = use(1, e);
      f.nout2 = H2;
      f.x2 = ya0;
      f.inv_eps2_ff = ff2(ff_make(1.0 / e));
      f.k2_2 = (float)((double)kLog2e / e);
      f.out2 = T2;
      f.z2 = z[2];
      f.use_prev2 = use(2, e);
      return launch_grid_fused2(f, st);
    };
    auto kb = [&](double e, double e_next, cudaStream_t st) -> cudaError_t {
      FusedArgs f = fused_args(e);
      f.nlines = H2;
      f.in1 = T2;
      f.nin1 = W1;
      f.nout1 = W2;
      f.y1 = xa1;
      f.x1 = ya1;
      f.out1_row = 1;
      f.F1 = make_div_ff(D2, e);
      f.logp1 = reinterpret_cast<const float2*>(logq);
      f.pot1 = reinterpret_cast<float2*>(V);
      f.logw1 = reinterpret_cast<const float2*>(logdy);
      f.z1 = z[3];
      f.use_prev1 = use(3, e);
      f.nout2 = W1;
      f.x2 = xa1;
      f.inv_eps2_ff = ff2(ff_make(1.0 / e_next));
      f.k2_2 = (float)((double)kLog2e / e_next);
      f.out2 = T1;
      f.z2 = z[0];
      f.use_prev2 = use(0, e_next);
      return launch_grid_fused2(f, st);
    };
    // eps of the iteration after `total` stage iterations (the final eps after the stages)
    std::vector<double> stage_eps;
    for (const Stage& sg : stages)
      for (int k = 0; k < sg.iters; ++k) stage_eps.push_back(sg.eps);
    auto eps_at = [&](size_t k) { return k < stage_eps.size() ? stage_eps[k] : o->eps; };
    UOT_CK(p1(eps_at(0), s));
    for (size_t k = 0; k < stage_eps.size(); ++k, ++total) {
      UOT_CK(ka(stage_eps[k], false, s));
      UOT_CK(kb(stage_eps[k], eps_at(k + 1), s));
    }
    auto iteration = [&](bool check, cudaStream_t st) -> cudaError_t {
      cudaError_t e = ka(o->eps, check, st);
      if (e != cudaSuccess) return e;
      return kb(o->eps, o->eps, st);
    };
    BlockGraph bg;
    bool graph_ok = !profiling_on();
    while (it < o->max_iter) {
      if (graph_ok && it > 0 && it % check_every == 0 && it + check_every <= o->max_iter) {
        if (!bg.exec) {
          cudaError_t e = bg.capture([&](cudaStream_t cs) -> cudaError_t {
            for (int k = 0; k < check_every; ++k) {
              cudaError_t e2 = iteration(k == check_every - 1, cs);
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
      UOT_CK(iteration(check, s));
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
  } else if (!o->plain_scaling) {
    // The stop decision after a check (err = the FP32 violation just read).
    // No 1% improvement on the best check for W iterations, W = max(50,
    // 5 check_every, 3x the iterations a 1% step took at the rate observed since
    // the first check): the check has reached the rounding floor of the passes.
    auto stalled = [&]() -> bool {
      if (std::isnan(first_err)) {
        first_err = err;
        first_it = it;
      }
      if (err < 0.99 * best_err) {
        best_err = err;
        best_it = it;
        return false;
      }
      double W = std::max(50, 5 * check_every);
      if (best_err < first_err && best_it > first_it) {
        const double rate = std::log(best_err / first_err) / (best_it - first_it);  // < 0
        W = std::max(W, std::min(1e8, 3.0 * std::log(0.99) / rate));
      }
      return it - best_it >= W;
    };
    // FP32 passes with float-float exponents exist for grids and point clouds of d <= 3
    const bool precise_ok = prec != UOT_F64 && (g->kind == UOT_GEOM_GRID || (g->kind == UOT_GEOM_POINTS && g->d <= 3));
    auto switch_precise = [&]() {
      G.precise = true;
      precise_from = total;
      mixed_handover = true;  // recapture the graph block with the new passes
      first_err = NAN;
      best_err = INFINITY;
      // the lowered threshold compensated the plain passes' optimistic check;
      // the precise passes' check is close to the FP64 value
      tol_int = o->tol;
    };
    auto decide = [&](bool& stop) -> cudaError_t {
      stop = false;
      err32 = err;
      if (!(o->tol > 0.0)) return cudaSuccess;
      if (mixed_phase) {
        // BF16 phase: hand over to the FP32 passes at mixed_switch or at the BF16 floor
        if (err <= mixed_switch || stalled()) {
          mixed_phase = false;
          mixed_iters = total;
          G.tc_off = true;
          mixed_handover = true;
          first_err = NAN;
          best_err = INFINITY;
        }
        return cudaSuccess;
      }
      if (!verify) {
        if (err <= o->tol) converged = stop = true;
        return cudaSuccess;
      }
      if (err <= tol_int) {
        cudaError_t e = cudaSuccess;
        if (!c64.ready && (e = c64.setup(*g, batch, p, dx, q, dy, s)) != cudaSuccess) return e;
        if ((e = c64.load_state(U, V, s)) != cudaSuccess) return e;
        if ((e = c64.iterate(D1, D2, o->eps, true, false, s)) != cudaSuccess) return e;
        if ((e = c64.read_err(err64, s)) != cudaSuccess) return e;
        ++nverify;
        if (err64 <= o->tol) {
          converged = stop = true;
          return cudaSuccess;
        }
        // An FP32 check far below the FP64 value measures the plain passes'
        // own rounding floor, not the state: where the precise passes exist,
        // switch now instead of chasing a lower threshold.
        if (precise_ok && !G.precise && err < 0.2 * err64) {
          switch_precise();
          return cudaSuccess;
        }
        // aim the FP32 check proportionally lower
        tol_int = err * std::min(0.7, std::max(0.05, o->tol / err64));
        best_err = err;
        best_it = it;
        return cudaSuccess;
      }
      // the FP32 check's rounding floor: on grids and point clouds (d <= 3) the
      // passes with float-float exponents take over (their floor is far
      // lower), then, if those stall too, FP64 iterations
      if (stalled()) {
        if (precise_ok && !G.precise)
          switch_precise();
        else
          polish = stop = true;
      }
      return cudaSuccess;
    };
    // shift: the translation step after the V-update (opts.translate)
    auto iteration = [&](double eps, bool check, bool shift, cudaStream_t st) -> cudaError_t {
      cudaError_t e;
      Epilogue e1 = prox_epilogue(D1, logp, U, logdx, check ? acc : nullptr, eps);
      e1.bstride = e1.bstride_p = n;
      if ((e = G.apply(0, V, logdy, eps, e1, st, check ? acc : nullptr)) != cudaSuccess) return e;
      Epilogue e2 = prox_epilogue(D2, logq, V, logdy, nullptr, eps);
      e2.bstride = e2.bstride_p = m;
      if ((e = G.apply(1, U, logdx, eps, e2, st)) != cudaSuccess || !shift) return e;
      return launch_kl_translate(U, V, logp, logq, logdx, logdy, n, m, batch, prec != UOT_F64, D1.lam, D2.lam,
                                 trpart, st);
    };
    for (const Stage& sg : stages)
      for (int k = 0; k < sg.iters; ++k, ++total)
        UOT_CK(iteration(sg.eps, false, translate && (k + 1) % check_every == 0, s));
    // launch_mode 2: once a block of check_every iterations (the last one
    // checked) repeats the same launches -- same eps, shifts from the previous
    // iteration -- it is captured once as a CUDA graph and replayed per block.
    BlockGraph bg;
    bool graph_ok = (o->launch_mode == 2 || o->launch_mode == 3) && !profiling_on();
    while (it < o->max_iter) {
      if (graph_ok && it > 0 && it % check_every == 0 && it + check_every <= o->max_iter) {
        if (!bg.exec) {
          cudaError_t e = bg.capture([&](cudaStream_t cs) -> cudaError_t {
            for (int k = 0; k < check_every; ++k) {
              cudaError_t e2 = iteration(o->eps, k == check_every - 1, translate && k == check_every - 1, cs);
              if (e2 != cudaSuccess) return e2;
            }
            return cudaSuccess;
          });
          if (e != cudaSuccess) {
            // not capturable here (e.g. a legacy-stream dependency): per-pass launches
            graph_ok = false;
            (void)cudaGetLastError();
            continue;
          }
        }
        UOT_CK(bg.launch(s));
        it += check_every;
        total += check_every;
        UOT_CK(read_err(err));
        bool stop = false;
        UOT_CK(decide(stop));
        if (stop) break;
        if (mixed_handover) {
          bg.reset();  // the block now launches the FP32 passes
          mixed_handover = false;
        }
        continue;
      }
      const bool check = ((it + 1) % check_every == 0) || (it == o->max_iter - 1);
      UOT_CK(iteration(o->eps, check, translate && check, s));
      ++it;
      ++total;
      if (check) {
        UOT_CK(read_err(err));
        if (it > 1) {
          bool stop = false;
          UOT_CK(decide(stop));
          if (stop) break;
          if (mixed_handover) {
            bg.reset();
            mixed_handover = false;
          }
        } else {
          err32 = err;
        }
      }
    }
    if (polish) {
      // the FP32 check has reached its rounding floor: FP64 iterations from the current state
      // Each check measures the state before its a-update; when it passes,
      // that state is restored and returned, so the reported FP64 violation
      // is the returned potentials' own.
      if (!c64.ready) UOT_CK(c64.setup(*g, batch, p, dx, q, dy, s));
      UOT_CK(c64.load_state(U, V, s));
      while (it < o->max_iter) {
        UOT_CK(c64.save_U(s));
        UOT_CK(c64.iterate(D1, D2, o->eps, true, false, s));
        UOT_CK(c64.read_err(err64, s));
        if (err64 <= o->tol) {
          UOT_CK(c64.restore_U(s));
          converged = true;
          break;
        }
        UOT_CK(c64.b_update(D2, o->eps, s));
        if (translate && (it + 1) % check_every == 0)
          UOT_CK(launch_kl_translate(c64.U, c64.V, c64.logp, c64.logq, c64.logdx, c64.logdy, n, m, batch, 0,
                                     D1.lam, D2.lam, trpart, s));
        ++it;
        ++total;
        ++npolish;
      }
      polished = true;
    }
    if (verify && !std::isnan(err64)) err = err64;
  } else {
    // Algorithm 1 on a stored FP64 kernel.
    double* K = sc.take<double>((size_t)n * m);
    double* KT = sc.take<double>((size_t)n * m);
    double* a = sc.take<double>(n);
    double* b = sc.take<double>(m);
    double* pd = sc.take<double>(n);
    double* qd = sc.take<double>(m);
    double* dxd = sc.take<double>(n);
    double* dyd = sc.take<double>(m);
    double* cres = sc.take<double>(4);
    UOT_SCRATCH_OK(sc);
    UOT_CK(to_f64(prec, p, n, pd, s));
    UOT_CK(to_f64(prec, q, m, qd, s));
    UOT_CK(to_f64(prec, dx, n, dxd, s));
    UOT_CK(to_f64(prec, dy, m, dyd, s));
    auto set_eps = [&](double eps) -> cudaError_t {
      count_launches(1);
      k_gibbs_matrix<double><<<nblocks(n * m), kNT, 0, s>>>((const double*)g->C, (int)n, (int)m, eps, K, KT);
      count_launches(1);
      k_exp_scale<<<nblocks(n), kNT, 0, s>>>(U, n, eps, a);
      count_launches(1);
      k_exp_scale<<<nblocks(m), kNT, 0, s>>>(V, m, eps, b);
      return cudaGetLastError();
    };
    auto to_pot = [&](double eps) -> cudaError_t {
      count_launches(1);
      k_log_scale<<<nblocks(n), kNT, 0, s>>>(a, n, eps, U);
      count_launches(1);
      k_log_scale<<<nblocks(m), kNT, 0, s>>>(b, m, eps, V);
      return cudaGetLastError();
    };
    // launch_mode 1: each eps runs as one launch of a cluster holding K in
    // shared memory (where it fits; the same iterates as the per-launch path)
    const bool cluster_mode = o->launch_mode == 1;
    for (const Stage& sg : stages) {
      UOT_CK(set_eps(sg.eps));
      bool launched = false;
      if (cluster_mode)
        UOT_CK(launch_alg1_cluster(K, KT, (int)n, (int)m, pd, dxd, qd, dyd, D1, D2, sg.eps, a, b, sg.iters, 0, 0.0,
                                   cres, s, &launched));
      if (launched) {
        total += sg.iters;
      } else {
        for (int k = 0; k < sg.iters; ++k, ++total) {
          UOT_CK(launch_alg1_half(K, (int)n, (int)m, b, dyd, pd, D1, sg.eps, a, dxd, nullptr, s));
          UOT_CK(launch_alg1_half(KT, (int)m, (int)n, a, dxd, qd, D2, sg.eps, b, dyd, nullptr, s));
        }
      }
      UOT_CK(to_pot(sg.eps));
    }
    UOT_CK(set_eps(o->eps));
    bool launched = false;
    if (cluster_mode && o->max_iter > 0)
      UOT_CK(launch_alg1_cluster(K, KT, (int)n, (int)m, pd, dxd, qd, dyd, D1, D2, o->eps, a, b, o->max_iter,
                                 check_every, o->tol, cres, s, &launched));
    if (launched) {
      double h[3];
      UOT_CK(cudaMemcpyAsync(h, cres, sizeof(h), cudaMemcpyDeviceToHost, s));
      UOT_CK(cudaStreamSynchronize(s));
      err = h[0];
      it = (int)h[1];
      total += it;
      converged = h[2] != 0.0;
    }
    while (!launched && it < o->max_iter) {
      const bool check = ((it + 1) % check_every == 0) || (it == o->max_iter - 1);
      if (check) UOT_CK(cudaMemsetAsync(acc, 0, 16, s));
      UOT_CK(launch_alg1_half(K, (int)n, (int)m, b, dyd, pd, D1, o->eps, a, dxd, check ? acc : nullptr, s));
      UOT_CK(launch_alg1_half(KT, (int)m, (int)n, a, dxd, qd, D2, o->eps, b, dyd, nullptr, s));
      ++it;
      ++total;
      if (check) {
        double h[2];
        UOT_CK(cudaMemcpyAsync(h, acc, 16, cudaMemcpyDeviceToHost, s));
        UOT_CK(cudaStreamSynchronize(s));
        err = (h[1] > 0.0) ? h[0] / h[1] : 0.0;
        if (it > 1 && o->tol > 0.0 && err <= o->tol) {
          converged = true;
          break;
        }
      }
    }
    UOT_CK(to_pot(o->eps));
  }

  // NaN check and output conversion (after FP64 iterations the state is FP64)
  const double* Ufin = polished ? c64.U : U;
  const double* Vfin = polished ? c64.V : V;
  const bool fin_ff = prec != UOT_F64 && !polished;
  UOT_CK(cudaMemsetAsync(flag, 0, 4, s));
  count_launches(1);
  k_nan_flag<<<nblocks(bn), kNT, 0, s>>>(Ufin, bn, fin_ff, flag);
  count_launches(1);
  k_nan_flag<<<nblocks(bm), kNT, 0, s>>>(Vfin, bm, fin_ff, flag);
  UOT_CK(cudaGetLastError());
  if (fin_ff && o->out_f64) {
    count_launches(2);
    k_ff_to_f64<<<nblocks(bn), kNT, 0, s>>>(reinterpret_cast<const float2*>(Ufin), bn, (double*)Uout);
    k_ff_to_f64<<<nblocks(bm), kNT, 0, s>>>(reinterpret_cast<const float2*>(Vfin), bm, (double*)Vout);
    UOT_CK(cudaGetLastError());
  } else if (!fin_ff && prec != UOT_F64 && !o->out_f64) {
    // FP64 state (after FP64 iterations) to float outputs
    count_launches(2);
    k_from_f64<float><<<nblocks(bn), kNT, 0, s>>>(Ufin, bn, (float*)Uout);
    k_from_f64<float><<<nblocks(bm), kNT, 0, s>>>(Vfin, bm, (float*)Vout);
    UOT_CK(cudaGetLastError());
  } else {
    const int out_prec = fin_ff ? prec : UOT_F64;
    UOT_CK(from_f64(out_prec, Ufin, bn, Uout, s));
    UOT_CK(from_f64(out_prec, Vfin, bm, Vout, s));
  }
  UOT_CK(cudaEventRecord(ev1, s));
  int hflag = 0, htc = 0;
  UOT_CK(cudaMemcpyAsync(&hflag, flag, 4, cudaMemcpyDeviceToHost, s));
  if (G.tc_err) UOT_CK(cudaMemcpyAsync(&htc, G.tc_err, 4, cudaMemcpyDeviceToHost, s));
  UOT_CK(cudaStreamSynchronize(s));
  float ms = 0.f;
  UOT_CK(cudaEventElapsedTime(&ms, ev0, ev1));
  uot_status out = htc ? UOT_TIMEOUT
                       : hflag ? UOT_NUMERICAL
                               : ((o->tol > 0.0 && !converged && o->max_iter > 0) ? UOT_NOT_CONVERGED : UOT_OK);
  if (res) {
    *res = empty_result();
    res->iters = it;
    res->total_iters = total;
    res->marg_err = err;
    res->ms = ms;
    res->status = out;
    res->verifications = nverify;
    res->polish_iters = npolish;
    res->marg_err_fp32 = err32;
    res->mixed_iters = prec != UOT_MIXED ? 0 : (G.tc_off ? mixed_iters : total);
    res->precise_iters = precise_from < 0 ? 0 : total - precise_from - npolish;
  }
  return out;
}

}  // namespace
}  // namespace uot

using namespace uot;

extern "C" {

uot_status uot_solve(const uot_geom* g, const void* p, const void* dx, const void* q,
                     const void* dy, const uot_div* F1, const uot_div* F2, const uot_opts* o,
                     void* U, void* V, uot_result* res, void* stream) {
  clear_stale_error();
  return solve_impl(g, 1, p, dx, q, dy, F1, F2, o, U, V, res, (cudaStream_t)stream);
}

uot_status uot_solve_many(const uot_geom* g, int batch, const void* p, const void* dx,
                          const void* q, const void* dy, const uot_div* F1, const uot_div* F2,
                          const uot_opts* o, void* U, void* V, uot_result* res, void* stream) {
  clear_stale_error();
  return solve_impl(g, batch, p, dx, q, dy, F1, F2, o, U, V, res, (cudaStream_t)stream);
}

uot_status uot_solve_batch(int nprob, const uot_batch_problem* probs, int d, const void* x,
                           const void* p, const void* dx, const void* y, const void* q,
                           const void* dy, const uot_opts* o, void* Uout, void* Vout, int* iters,
                           double* errs, uot_result* res, void* stream) {
  clear_stale_error();
  uot_status st = check_opts(o, false, true);
  if (st != UOT_OK) return st;
  if (nprob < 1 || !probs || d < 1 || d > 3 || !x || !p || !dx || !y || !q || !dy || !Uout || !Vout)
    return UOT_EINVAL;
  if (o->precision != UOT_F32 || o->plain_scaling || o->U0 || o->V0) return UOT_EUNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int> hn(nprob), hm(nprob), order(nprob);
  std::vector<int64_t> hxo(nprob), hyo(nprob);
  int64_t N = 0, M = 0;
  int nmax = 0, mmax = 0;
  for (int k = 0; k < nprob; ++k) {
    const uot_batch_problem& pr = probs[k];
    if (pr.n < 1 || pr.m < 1 || pr.n > 3072 || pr.m > 3072) return UOT_EINVAL;
    if (!div_ok(&pr.F1) || !div_ok(&pr.F2)) return UOT_EINVAL;
    if (o->translate && (pr.F1.kind != UOT_DIV_KL || pr.F2.kind != UOT_DIV_KL)) return UOT_EUNSUPPORTED;
    hn[k] = pr.n;
    hm[k] = pr.m;
    hxo[k] = N;
    hyo[k] = M;
    N += pr.n;
    M += pr.m;
    nmax = pr.n > nmax ? pr.n : nmax;
    mmax = pr.m > mmax ? pr.m : mmax;
    order[k] = k;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (int64_t)hn[a] * hm[a] > (int64_t)hn[b] * hm[b];
  });
  const std::vector<Stage> stages = eps_schedule(*o);
  const int nstage = (int)stages.size();
  std::vector<double> eps_list;
  for (const Stage& sg : stages) eps_list.push_back(sg.eps);
  eps_list.push_back(o->eps);
  std::vector<DivFF> divs((size_t)(nstage + 1) * nprob * 2);
  std::vector<float2> heps(nstage + 1), hieps(nstage + 1);
  std::vector<float> hk2(nstage + 1);
  for (int sidx = 0; sidx <= nstage; ++sidx) {
    const double e = eps_list[sidx];
    heps[sidx] = ff2(ff_make(e));
    hieps[sidx] = ff2(ff_make(1.0 / e));
    hk2[sidx] = (float)((double)kLog2e / e);
    for (int k = 0; k < nprob; ++k) {
      divs[((size_t)sidx * nprob + k) * 2] = make_div_ff(make_div(probs[k].F1), e);
      divs[((size_t)sidx * nprob + k) * 2 + 1] = make_div_ff(make_div(probs[k].F2), e);
    }
  }
  int dev = 0, sms = 0;
  UOT_CK(cudaGetDevice(&dev));
  UOT_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

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
  sc.reserve<int>(nprob);      // order
  sc.reserve<int>(nprob);      // n
  sc.reserve<int>(nprob);      // m
  sc.reserve<int64_t>(nprob);  // xoff
  sc.reserve<int64_t>(nprob);  // yoff
  sc.reserve<DivFF>(divs.size());
  sc.reserve<float2>(nstage + 1);
  sc.reserve<float2>(nstage + 1);
  sc.reserve<float>(nstage + 1);
  sc.reserve<double>(N);  // logp
  sc.reserve<double>(N);  // logdx
  sc.reserve<double>(M);  // logq
  sc.reserve<double>(M);  // logdy
  sc.reserve<int>(nprob);    // iters
  sc.reserve<float>(nprob);  // errs
  sc.reserve<int>(1);        // work counter
  sc.reserve<float2>(N);     // U state (float-float)
  sc.reserve<float2>(M);     // V state
  sc.reserve<float>(N);      // U-side shifts
  sc.reserve<float>(M);      // V-side shifts
  if (o->translate) sc.reserve<double2>(nprob);  // (lambda1, lambda2)
  UOT_CK(sc.allocate());
  int* d_order = sc.take<int>(nprob);
  int* d_n = sc.take<int>(nprob);
  int* d_m = sc.take<int>(nprob);
  int64_t* d_xo = sc.take<int64_t>(nprob);
  int64_t* d_yo = sc.take<int64_t>(nprob);
  DivFF* d_divs = sc.take<DivFF>(divs.size());
  float2* d_eps = sc.take<float2>(nstage + 1);
  float2* d_ieps = sc.take<float2>(nstage + 1);
  float* d_k2 = sc.take<float>(nstage + 1);
  double* d_logp = sc.take<double>(N);
  double* d_logdx = sc.take<double>(N);
  double* d_logq = sc.take<double>(M);
  double* d_logdy = sc.take<double>(M);
  int* d_iters = sc.take<int>(nprob);
  float* d_errs = sc.take<float>(nprob);
  int* d_next = sc.take<int>(1);
  float2* d_Uff = sc.take<float2>(N);
  float2* d_Vff = sc.take<float2>(M);
  float* d_zU = sc.take<float>(N);
  float* d_zV = sc.take<float>(M);
  double2* d_lam = o->translate ? sc.take<double2>(nprob) : nullptr;
  UOT_SCRATCH_OK(sc);
  if (o->translate) {
    std::vector<double2> hl(nprob);
    for (int k = 0; k < nprob; ++k) hl[k] = make_double2(probs[k].F1.lambda, probs[k].F2.lambda);
    UOT_CK(cudaMemcpyAsync(d_lam, hl.data(), nprob * sizeof(double2), cudaMemcpyHostToDevice, s));
  }
  UOT_CK(cudaMemcpyAsync(d_order, order.data(), nprob * sizeof(int), cudaMemcpyHostToDevice, s));
  UOT_CK(cudaMemcpyAsync(d_n, hn.data(), nprob * sizeof(int), cudaMemcpyHostToDevice, s));
  UOT_CK(cudaMemcpyAsync(d_m, hm.data(), nprob * sizeof(int), cudaMemcpyHostToDevice, s));
  UOT_CK(cudaMemcpyAsync(d_xo, hxo.data(), nprob * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  UOT_CK(cudaMemcpyAsync(d_yo, hyo.data(), nprob * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  UOT_CK(cudaMemcpyAsync(d_divs, divs.data(), divs.size() * sizeof(DivFF), cudaMemcpyHostToDevice, s));
  UOT_CK(cudaMemcpyAsync(d_eps, heps.data(), heps.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
  UOT_CK(cudaMemcpyAsync(d_ieps, hieps.data(), hieps.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
  UOT_CK(cudaMemcpyAsync(d_k2, hk2.data(), hk2.size() * sizeof(float), cudaMemcpyHostToDevice, s));
  UOT_CK(cudaMemsetAsync(d_next, 0, sizeof(int), s));
  UOT_CK(to_log(UOT_F32, p, N, d_logp, s));
  UOT_CK(to_log(UOT_F32, dx, N, d_logdx, s));
  UOT_CK(to_log(UOT_F32, q, M, d_logq, s));
  UOT_CK(to_log(UOT_F32, dy, M, d_logdy, s));
  BatchArgs a;
  a.nprob = nprob;
  a.d = d;
  a.nstage = nstage;
  a.iters_per_stage = o->iters_per_stage;
  a.max_iter = o->max_iter;
  a.check_every = o->check_every > 0 ? o->check_every : 1;
  a.nmax = nmax;
  a.mmax = mmax;
  a.ndiv = nprob;
  a.tol = (float)o->tol;
  a.order = d_order;
  a.n = d_n;
  a.m = d_m;
  a.xoff = d_xo;
  a.yoff = d_yo;
  a.x = (const float*)x;
  a.y = (const float*)y;
  a.logp = reinterpret_cast<const float2*>(d_logp);
  a.logdx = reinterpret_cast<const float2*>(d_logdx);
  a.logq = reinterpret_cast<const float2*>(d_logq);
  a.logdy = reinterpret_cast<const float2*>(d_logdy);
  a.divs = d_divs;
  a.eps_ff = d_eps;
  a.inv_eps_ff = d_ieps;
  a.k2 = d_k2;
  a.Uout = o->out_f64 ? nullptr : (float*)Uout;
  a.Vout = o->out_f64 ? nullptr : (float*)Vout;
  a.Uout64 = o->out_f64 ? (double*)Uout : nullptr;
  a.Vout64 = o->out_f64 ? (double*)Vout : nullptr;
  a.iters_out = d_iters;
  a.err_out = d_errs;
  a.next = d_next;
  a.Uff = d_Uff;
  a.Vff = d_Vff;
  a.zU = d_zU;
  a.zV = d_zV;
  a.translate = o->translate;
  a.lam = d_lam;
  const int variant = batch_pick_variant(a, order.data(), s);
  const int per_sm = batch_ctas_per_sm(d, variant, nmax, mmax);
  if (per_sm < 1) {
    g_last_error = "uot_solve_batch: problem sizes do not fit in shared memory";
    return UOT_EUNSUPPORTED;
  }
  UOT_CK(cudaMemsetAsync(d_next, 0, sizeof(int), s));
  const int grid = (int)std::min<int64_t>(nprob, (int64_t)sms * per_sm);
  UOT_CK(launch_batch(a, variant, grid, s));
  UOT_CK(cudaEventRecord(ev1, s));
  std::vector<int> it_h(nprob);
  std::vector<float> er_h(nprob);
  UOT_CK(cudaMemcpyAsync(it_h.data(), d_iters, nprob * sizeof(int), cudaMemcpyDeviceToHost, s));
  UOT_CK(cudaMemcpyAsync(er_h.data(), d_errs, nprob * sizeof(float), cudaMemcpyDeviceToHost, s));
  UOT_CK(cudaStreamSynchronize(s));
  float ms = 0.f;
  UOT_CK(cudaEventElapsedTime(&ms, ev0, ev1));
  bool all_conv = true;
  int total = 0;
  double worst = 0.0;
  for (int k = 0; k < nprob; ++k) {
    if (iters) iters[k] = it_h[k];
    if (errs) errs[k] = er_h[k];
    total += it_h[k];
    worst = std::max(worst, (double)er_h[k]);
    if (o->tol > 0.0 && !(er_h[k] <= o->tol)) all_conv = false;
  }
  const uot_status out = all_conv ? UOT_OK : UOT_NOT_CONVERGED;
  if (res) {
    *res = empty_result();
    res->iters = total;
    res->total_iters = total + nprob * nstage * o->iters_per_stage;
    res->marg_err = worst;
    res->ms = ms;
    res->status = out;
  }
  return out;
}

}  // extern "C"

// Batched conjugate gradient on D^+D x = b: plain FP64, or mixed precision with
// reliable updates (the inner operator at FP32 or FP16 storage with FP32
// arithmetic; FP64 true residuals, reductions and convergence test).
//
// The paper gives no solver; this follows textbook CG (Hestenes-Stiefel) for
// the FP64 mode and CG with reliable updates (Clark et al., "Solving lattice
// QCD systems of equations using mixed precision solvers on GPUs", 2010) for
// the mixed modes.  Between reliable updates the inner solver works on the
// rescaled system A e = r / sigma with sigma = |r| / sqrt(n) (n reals per
// RHS), so low-precision vectors hold entries of order one; x accumulates
// x += sigma * e at each update.  A reliable update fires when the iterated
// residual dropped below delta (0.01 with FP32 inner fields, 0.1 with FP16)
// times its largest value since the last update, when it claims convergence,
// or when maxit is reached; the FP64 residual b - D^+D x then decides
// convergence.
//
// All per-RHS scalars live on the device (CGState); converged or stopped RHS
// are masked off, and the stencil kernels skip their CTAs.  One inner
// iteration is captured as a CUDA graph and replayed kReplay times between
// host checks of the flags.
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <vector>

#include "dw_api_internal.cuh"
#include "dw_blas.cuh"

namespace dw {

struct CGWork {
  // FP64 fields (nrhs each)
  void *r64 = nullptr, *Ax64 = nullptr, *tmp64 = nullptr;
  size_t r64_cap = 0, Ax64_cap = 0, tmp64_cap = 0;
  // inner fields
  void *p = nullptr, *Ap = nullptr, *tmp = nullptr, *rs = nullptr, *xs = nullptr;
  size_t p_cap = 0, Ap_cap = 0, tmp_cap = 0, rs_cap = 0, xs_cap = 0;
  double *partials = nullptr;
  size_t partials_cap = 0;
  double *sums = nullptr;
  size_t sums_cap = 0;
  double *dnorm = nullptr;  // |D p|^2 per stencil CTA
  size_t dnorm_cap = 0;
  double *rsnorm = nullptr;  // |r_s|^2 per CTA of the fused D^+ pass
  size_t rsnorm_cap = 0;
  CGState *state = nullptr;
  size_t state_cap = 0;
  // even-odd solves: even-parity intermediates of Dhat (inner precision and
  // FP64) and the FP64 parity fields of the outer solve
  void *e1 = nullptr, *e2 = nullptr, *e1_64 = nullptr, *e2_64 = nullptr;
  size_t e1_cap = 0, e2_cap = 0, e1_64_cap = 0, e2_64_cap = 0;
  void *eta_e = nullptr, *eta_o = nullptr, *bhat = nullptr, *bpr = nullptr, *xo = nullptr;
  size_t eta_e_cap = 0, eta_o_cap = 0, bhat_cap = 0, bpr_cap = 0, xo_cap = 0;
  cudaStream_t stream = nullptr;
};

void cg_release(dw_lattice *lat) {
  CGWork *w = lat->cg;
  if (!w) return;
  void *bufs[] = {w->r64,  w->Ax64,  w->tmp64, w->p,     w->Ap,   w->tmp,   w->rs,
                  w->xs,   w->partials, w->sums, w->dnorm, w->rsnorm, w->state, w->e1, w->e2,
                  w->e1_64, w->e2_64, w->eta_e, w->eta_o, w->bhat, w->bpr,  w->xo};
  for (void *b : bufs)
    if (b) cudaFree(b);
  if (w->stream) cudaStreamDestroy(w->stream);
  delete w;
  lat->cg = nullptr;
}

namespace {

constexpr int kReplay = 8;  // inner iterations per host check

struct Solve {
  dw_lattice *lat;
  CGWork *w;
  int nrhs;
  int pp, pr;  // precisions of (p, Ap, tmp) and (r_s, x_s)
  double delta, tol;
  int maxit;
  const double *mf;
  cudaStream_t st;
  BlasCtx c;
  bool eo;  // solve Dhat^+ Dhat on odd-parity fields instead of D^+ D

  const int *gate_run() const { return &w->state[0].run; }
  const int *gate_update() const { return &w->state[0].need_update; }

  // One inner iteration over all RHS (masked by `run`).  <p, D^+D p> is
  // |D p|^2, summed per CTA by the D pass itself.
  int ctas_d() const {
    return (int)(eo ? cb_ctas_per_rhs(lat, pp, OP_D)
                    : dslash_ctas_per_rhs(lat, pick_tile(lat, pp, OP_D, nrhs)));
  }
  int ctas_ddag() const {
    return (int)(eo ? cb_ctas_per_rhs(lat, pp, OP_DDAG)
                    : dslash_ctas_per_rhs(lat, pick_tile(lat, pp, OP_DDAG, nrhs)));
  }

  // alpha follows from the D (Dhat) pass, |D p|^2, so the last launch of the
  // D^+ (Dhat^+) pass applies r_s -= alpha A p itself and leaves |r_s|^2 per CTA:
  // A p is never stored and read back (two field passes fewer than storing it
  // and updating r_s in a separate pass).
  int iteration() {
    const int nd = ctas_d();
    int rc;
    if (eo)
      rc = apply_schur(lat, pp, w->tmp, w->p, mf, nrhs, false, w->e1, w->e2, st, gate_run(),
                       kCGStateInts, w->dnorm);
    else
      rc = run_dslash(lat, pp, OP_D, w->tmp, w->p, mf, nrhs, st, nullptr, gate_run(),
                      kCGStateInts, nullptr, nullptr, w->dnorm);
    if (rc) return rc;
    if (cg_alpha(c, w->dnorm, nd, w->state, st))
      return cuda_fail(cudaGetLastError(), "cg iteration launch");
    // ... and the solution step x_s += alpha p, which leaves the direction pass
    // three field accesses instead of five
    const ResidualFuse fuse{w->rs, &w->state[0].alpha, (int)(sizeof(CGState) / sizeof(double)),
                            w->rsnorm, w->xs, w->p};
    if (eo)
      rc = apply_schur(lat, pp, w->Ap, w->tmp, mf, nrhs, true, w->e1, w->e2, st, gate_run(),
                       kCGStateInts, nullptr, &fuse);
    else
      rc = run_dslash(lat, pp, OP_DDAG, w->Ap, w->tmp, mf, nrhs, st, nullptr, gate_run(),
                      kCGStateInts, nullptr, nullptr, nullptr, 0, 0, &fuse);
    if (rc) return rc;
    if (cg_beta(c, w->rsnorm, w->state, delta, tol, maxit, st, ctas_ddag()))
      return cuda_fail(cudaGetLastError(), "cg iteration launch");
    if (cg_direction(c, pp, pr, w->p, w->xs, w->rs, w->state, st, false))
      return cuda_fail(cudaGetLastError(), "cg iteration launch");
    return DW_OK;
  }

  // Reliable update of every RHS flagged need_update (first: initial residual).
  int reliable(void *x, const void *b, int first) {
    if (!first && cg_accumulate_x(c, pr, x, w->xs, w->state, st))
      return cuda_fail(cudaGetLastError(), "accumulate launch");
    int rc;
    if (eo) {
      rc = apply_schur(lat, DW_F64, w->tmp64, x, mf, nrhs, false, w->e1_64, w->e2_64, st,
                       gate_update(), kCGStateInts, nullptr);
      if (rc) return rc;
      rc = apply_schur(lat, DW_F64, w->Ax64, w->tmp64, mf, nrhs, true, w->e1_64, w->e2_64, st,
                       gate_update(), kCGStateInts, nullptr);
    } else {
      rc = run_dslash(lat, DW_F64, OP_D, w->tmp64, x, mf, nrhs, st, nullptr, gate_update(),
                      kCGStateInts);
      if (rc) return rc;
      rc = run_dslash(lat, DW_F64, OP_DDAG, w->Ax64, w->tmp64, mf, nrhs, st, nullptr,
                      gate_update(), kCGStateInts);
    }
    if (rc) return rc;
    if (cg_residual(c, (double *)w->r64, (const double *)b, (const double *)w->Ax64,
                    w->partials, w->state, st) ||
        cg_reliable(c, w->partials, w->state, tol, maxit, first, st) ||
        cg_install(c, w->state, st) ||
        cg_reliable_apply(c, pp, pr, (const double *)w->r64, w->rs, w->xs, w->p, w->state, st) ||
        cg_clear_update(c, w->state, st))
      return cuda_fail(cudaGetLastError(), "reliable update launch");
    return DW_OK;
  }
};

int ensure(void **buf, size_t *cap, size_t need) { return ensure_buffer(buf, cap, need); }

// the fused D^+ pass reads alpha of RHS r at (double *)&state[0].alpha + r * stride
static_assert(sizeof(CGState) % sizeof(double) == 0 && offsetof(CGState, alpha) % sizeof(double) == 0,
              "CGState must be a whole number of doubles with alpha double-aligned");

}  // namespace

}  // namespace dw

namespace dw {

// The solver proper: CG on D^+D x = b (eo: on Dhat^+ Dhat x = b with odd-parity
// fields).  The caller has checked the arguments and set up lat->cg.
int cg_run(dw_lattice *lat, void *x, const void *b, const double *mf, int nrhs, double tol,
           int maxit, int mode, dw_cg_stats *stats, bool eo,
           std::chrono::steady_clock::time_point t_start) {
  CGWork *w = lat->cg;
  cudaError_t e;
  // reliable-update threshold (dw_set_reliable_delta), by default chosen from
  // timings at 24^4 x 16 and 32^3 x 64 x 12 (every setting reaches the same
  // residual): 1e-3 with FP32 inner fields for both solvers; with FP16 ones
  // (their rounding, 2^-11, makes the iterated residual drift further between
  // updates) 0.1 for CG on D^+D and 0.01 for the even-odd solve, whose inner
  // iterations are cheaper against its FP64 updates
  const double delta = mode == DW_F64                 ? 0.0
                       : lat->reliable_delta > 0.0 ? lat->reliable_delta
                       : mode == DW_F32            ? 1e-3
                       : eo                        ? 0.01
                                                   : 0.1;
  Solve S{lat, w, nrhs, mode, mode == DW_F64 ? DW_F64 : DW_F32, delta,
          tol, maxit, mf, w->stream,
          BlasCtx((int)(eo ? lat->V4 / 2 : lat->V4), lat->Ls, nrhs, lat->num_sms), eo};
  auto fbytes = [&](int prec, int n) {
    return eo ? cb_field_bytes(lat, prec, n) : field_bytes(lat, prec, n);
  };
  const size_t f64 = fbytes(DW_F64, nrhs);
  const size_t fpp = fbytes(S.pp, nrhs);
  const size_t fpr = fbytes(S.pr, nrhs);
  int rc;
  if ((rc = ensure(&w->r64, &w->r64_cap, f64)) || (rc = ensure(&w->Ax64, &w->Ax64_cap, f64)) ||
      (rc = ensure(&w->tmp64, &w->tmp64_cap, f64)) || (rc = ensure(&w->p, &w->p_cap, fpp)) ||
      (rc = ensure(&w->Ap, &w->Ap_cap, fpp)) || (rc = ensure(&w->tmp, &w->tmp_cap, fpp)) ||
      (rc = ensure(&w->rs, &w->rs_cap, fpr)) || (rc = ensure(&w->xs, &w->xs_cap, fpr)) ||
      (rc = ensure((void **)&w->partials, &w->partials_cap,
                   sizeof(double) * (size_t)S.c.nblk * nrhs)) ||
      (rc = ensure((void **)&w->sums, &w->sums_cap, sizeof(double) * nrhs)) ||
      (rc = ensure((void **)&w->state, &w->state_cap, sizeof(CGState) * nrhs)))
    return rc;
  if (eo && ((rc = ensure(&w->e1, &w->e1_cap, fpp)) || (rc = ensure(&w->e2, &w->e2_cap, fpp)) ||
             (rc = ensure(&w->e1_64, &w->e1_64_cap, f64)) ||
             (rc = ensure(&w->e2_64, &w->e2_64_cap, f64))))
    return rc;
  cudaStream_t st = w->stream;


  // |b| per RHS
  std::vector<double> b2(nrhs);
  if (blas_redot(S.c, DW_F64, b, DW_F64, b, w->partials, nullptr, st) ||
      blas_finalize_sum(S.c, w->partials, w->sums, st))
    return cuda_fail(cudaGetLastError(), "norm launch");
  e = cudaMemcpyAsync(b2.data(), w->sums, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "norm readback");

  std::vector<CGState> hs(nrhs);
  const size_t rhs64 = fbytes(DW_F64, 1);
  for (int r = 0; r < nrhs; ++r) {
    CGState &s = hs[r];
    memset(&s, 0, sizeof(s));
    s.sigma = 1.0;
    s.bnorm = std::sqrt(b2[r]);
    if (!std::isfinite(b2[r])) {
      s.breakdown = 1;
    } else if (b2[r] == 0.0) {
      s.converged = 1;  // b = 0: x = 0 is the solution
      cudaMemsetAsync((char *)x + (size_t)r * rhs64, 0, rhs64, st);
    } else {
      s.active = 1;
      s.need_update = 1;
    }
  }
  if (cudaMemcpyAsync(w->state, hs.data(), sizeof(CGState) * nrhs, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemsetAsync(w->p, 0, fpp, st) != cudaSuccess ||
      cudaMemsetAsync(w->xs, 0, fpr, st) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "solver setup");

  // tile choice for the inner operator of this solve (timed once per lattice
  // and RHS count, then cached; the FP64 operator of the reliable updates keeps
  // the untuned tile unless it is the inner operator)
  for (int op : {(int)OP_D, (int)OP_DDAG}) {
    if (eo)
      rc = tune_cb(lat, S.pp, op, st);
    else if (!lat->tuned.count(std::make_tuple(S.pp, op, nrhs)))
      rc = tune_tile(lat, S.pp, op, nrhs, st, true);
    if (rc) return rc;
  }

  {
    const long long nd = S.ctas_d();
    if ((rc = ensure((void **)&w->dnorm, &w->dnorm_cap, sizeof(double) * (size_t)nd * nrhs)))
      return rc;
    if ((rc = ensure((void **)&w->rsnorm, &w->rsnorm_cap,
                     sizeof(double) * (size_t)S.ctas_ddag() * nrhs)))
      return rc;
  }

  // initial residual
  if ((rc = S.reliable(x, b, 1))) return rc;
  // even-odd: one extra pass of the inner operator (its result is recomputed by
  // the first iteration) so that every
  // kernel it launches has been set up before the stream is captured
  if (eo && ((rc = apply_schur(lat, S.pp, w->tmp, w->p, mf, nrhs, false, w->e1, w->e2, st,
                               nullptr, 0, nullptr)) ||
             (rc = apply_schur(lat, S.pp, w->Ap, w->tmp, mf, nrhs, true, w->e1, w->e2, st,
                               nullptr, 0, nullptr))))
    return rc;

  // capture one inner iteration as a graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "begin capture");
  rc = S.iteration();
  cudaError_t ce = cudaStreamEndCapture(st, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (ce != cudaSuccess) return cuda_fail(ce, "end capture");
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return cuda_fail(ce, "graph instantiate");

  // host loop: replay, check flags, run reliable updates
  const long long max_rounds = 4LL * maxit + 64;
  long long rounds = 0;
  rc = DW_OK;
  while (true) {
    e = cudaMemcpyAsync(hs.data(), w->state, sizeof(CGState) * nrhs, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "state readback");
      break;
    }
    bool any_active = false, any_update = false;
    for (const CGState &s : hs) {
      any_active |= s.active != 0;
      any_update |= (s.active && s.need_update);
    }
    if (!any_active) break;
    if (++rounds > max_rounds) {
      rc = fail(DW_ERR_STATE, "solver made no progress");
      break;
    }
    if (any_update) {
      if ((rc = S.reliable(x, b, 0))) break;
      continue;
    }
    for (int k = 0; k < kReplay; ++k) {
      e = cudaGraphLaunch(exec, st);
      if (e != cudaSuccess) break;
    }
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "graph launch");
      break;
    }
  }
  cudaGraphExecDestroy(exec);
  if (rc) return rc;
  // a stencil launch that gave up a bounded wait has set the lattice's status
  // word: the solve reports it (and clears the word) instead of its stats
  int timed_out = 0;
  e = cudaMemcpyAsync(&timed_out, lat->dev_status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && timed_out) e = cudaMemsetAsync(lat->dev_status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "solver synchronize");
  if (timed_out)
    return fail(DW_ERR_TIMEOUT, "a stencil kernel of the solve gave up waiting for its "
                                "shared-memory copies");

  const double secs =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  bool any_break = false, all_conv = true;
  for (int r = 0; r < nrhs; ++r) {
    const CGState &s = hs[r];
    stats[r].iters = s.iters;
    stats[r].reliable_updates = s.reliable;
    stats[r].converged = s.converged;
    stats[r].true_resid = s.bnorm > 0.0 ? std::sqrt(s.true_r2) / s.bnorm : 0.0;
    stats[r].seconds = secs;
    any_break |= s.breakdown != 0;
    all_conv &= s.converged != 0;
  }
  if (any_break) return fail(DW_ERR_BREAKDOWN, "CG breakdown (non-finite or non-positive <p, Ap>)");
  if (!all_conv) return fail(DW_ERR_NOT_CONVERGED, "CG reached maxit before tol");
  return DW_OK;
}

// Argument checks and workspace shared by dw_cg_solve and dw_solve_eo.
int cg_prepare(dw_lattice *lat, void *x, const void *b, const double *mf, int nrhs, double tol,
               int maxit, int mode, dw_cg_stats *stats, void *stream) {
  if (!lat) return fail(DW_ERR_ARG, "lattice is NULL");
  if (!x || !b) return fail(DW_ERR_ARG, "field pointer is NULL");
  if (x == b) return fail(DW_ERR_ARG, "x must not alias b");
  if (((uintptr_t)x & 15u) || ((uintptr_t)b & 15u))
    return fail(DW_ERR_ARG, "fields must be 16-byte aligned");
  if (!mf) return fail(DW_ERR_ARG, "mf is NULL");
  if (!stats) return fail(DW_ERR_ARG, "stats is NULL");
  if (nrhs < 1 || nrhs > 65535) return fail(DW_ERR_ARG, "nrhs out of range");
  if (!(tol > 0.0)) return fail(DW_ERR_ARG, "tol must be > 0");
  if (maxit < 1) return fail(DW_ERR_ARG, "maxit must be >= 1");
  if (mode != DW_F64 && mode != DW_F32 && mode != DW_F16)
    return fail(DW_ERR_ARG, "unknown mode %d", mode);
  if (!lat->gauge_loaded) return fail(DW_ERR_STATE, "dw_load_gauge has not been called");
  if (lat->cplx)
    return fail(DW_ERR_STATE, "the solvers need the spin-pair layout (dw_set_complex_layout 0)");
  if (!lat->cg) lat->cg = new (std::nothrow) CGWork();
  CGWork *w = lat->cg;
  if (!w) return fail(DW_ERR_ALLOC, "host allocation failed");
  if (!w->stream && cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "stream create");
  // order after the caller's stream, then work on the lattice's own stream
  const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "caller stream synchronize");
  return DW_OK;
}

}  // namespace dw

using namespace dw;

extern "C" int dw_cg_solve(dw_lattice *lat, void *x, const void *b, const double *mf, int nrhs,
                           double tol, int maxit, int mode, dw_cg_stats *stats, void *stream) {
  clear_error();
  const auto t_start = std::chrono::steady_clock::now();
  const int rc = cg_prepare(lat, x, b, mf, nrhs, tol, maxit, mode, stats, stream);
  if (rc) return rc;
  return cg_run(lat, x, b, mf, nrhs, tol, maxit, mode, stats, false, t_start);
}

// D x = eta with even-odd preconditioning (see dw.h).
extern "C" int dw_solve_eo(dw_lattice *lat, void *x, const void *eta, const double *mf,
                           int nrhs, double tol, int maxit, int mode, dw_cg_stats *stats,
                           void *stream) {
  clear_error();
  const auto t_start = std::chrono::steady_clock::now();
  int rc = cg_prepare(lat, x, eta, mf, nrhs, tol, maxit, mode, stats, stream);
  if (rc) return rc;
  if (!eo_ok(lat)) return fail(DW_ERR_ARG, "even-odd solves need even Lx, Ly, Lz, Lt");
  CGWork *w = lat->cg;
  cudaStream_t st = w->stream;
  const size_t h64 = cb_field_bytes(lat, DW_F64, nrhs);
  const size_t f64 = field_bytes(lat, DW_F64, nrhs);
  if ((rc = ensure(&w->eta_e, &w->eta_e_cap, h64)) ||
      (rc = ensure(&w->eta_o, &w->eta_o_cap, h64)) ||
      (rc = ensure(&w->bhat, &w->bhat_cap, h64)) || (rc = ensure(&w->bpr, &w->bpr_cap, h64)) ||
      (rc = ensure(&w->xo, &w->xo_cap, h64)) || (rc = ensure(&w->e1_64, &w->e1_64_cap, h64)) ||
      (rc = ensure(&w->e2_64, &w->e2_64_cap, h64)) || (rc = ensure(&w->r64, &w->r64_cap, f64)) ||
      (rc = ensure(&w->Ax64, &w->Ax64_cap, f64)))
    return rc;
  // eta -> (eta_e, eta_o); the odd half of x is the start vector
  if ((rc = eo_split(lat, DW_F64, w->eta_e, w->eta_o, eta, nrhs, st)) ||
      (rc = eo_split(lat, DW_F64, w->e1_64, w->xo, x, nrhs, st)))
    return rc;
  // bhat = eta_o - H_oe A^-1 eta_e
  if ((rc = apply_m5(lat, DW_F64, w->e2_64, w->eta_e, mf, nrhs, true, false, st)) ||
      (rc = run_dslash_cb(lat, DW_F64, OP_D, w->bhat, w->e2_64, w->eta_o, 1, 1.0, 0.0, 0.5, mf,
                          nrhs, st, nullptr, 0, nullptr)))
    return rc;
  // b' = Dhat^+ bhat, then CG on Dhat^+ Dhat x_o = b'
  if ((rc = apply_schur(lat, DW_F64, w->bpr, w->bhat, mf, nrhs, true, w->e1_64, w->e2_64, st,
                        nullptr, 0, nullptr)))
    return rc;
  BlasCtx c((int)lat->V4, lat->Ls, nrhs, lat->num_sms);
  if ((rc = ensure((void **)&w->partials, &w->partials_cap,
                   sizeof(double) * (size_t)c.nblk * nrhs)) ||
      (rc = ensure((void **)&w->sums, &w->sums_cap, sizeof(double) * nrhs)))
    return rc;
  // |eta|^2 per RHS
  std::vector<double> rr(nrhs), ee(nrhs);
  if (blas_redot(c, DW_F64, eta, DW_F64, eta, w->partials, nullptr, st) ||
      blas_finalize_sum(c, w->partials, w->sums, st))
    return cuda_fail(cudaGetLastError(), "norm launch");
  cudaError_t e =
      cudaMemcpyAsync(ee.data(), w->sums, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "norm readback");

  // x_e = A^-1 (eta_e - H_eo x_o), x = (x_e, x_o), and |eta - D x|^2 per RHS in FP64
  auto reconstruct_and_residual = [&]() -> int {
    int r;
    if ((r = run_dslash_cb(lat, DW_F64, OP_D, w->e1_64, w->xo, w->eta_e, 0, 1.0, 0.0, 0.5, mf,
                           nrhs, st, nullptr, 0, nullptr)) ||
        (r = apply_m5(lat, DW_F64, w->e2_64, w->e1_64, mf, nrhs, true, false, st)) ||
        (r = eo_merge(lat, DW_F64, x, w->e2_64, w->xo, nrhs, st)) ||
        (r = run_dslash(lat, DW_F64, OP_D, w->Ax64, x, mf, nrhs, st, nullptr)))
      return r;
    if (cg_residual(c, (double *)w->r64, (const double *)eta, (const double *)w->Ax64,
                    w->partials, nullptr, st) ||
        blas_finalize_sum(c, w->partials, w->sums, st))
      return cuda_fail(cudaGetLastError(), "residual launch");
    cudaError_t ce =
        cudaMemcpyAsync(rr.data(), w->sums, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return cuda_fail(ce, "residual readback");
    return DW_OK;
  };

  // The CG stops on the residual of the odd-site normal equations, which
  // bounds the residual of D x = eta only up to a factor of order one.  When
  // the full-system residual of a pass misses tol, the CG is run again from
  // the current x_o with its tolerance lowered by the factor it missed by
  // (and a margin), up to kPasses passes within the maxit budget.
  constexpr int kPasses = 4;
  constexpr double kAccept = 0.999;  // full-system target: kAccept * tol
  std::vector<dw_cg_stats> pass(nrhs);
  std::vector<int> iters(nrhs, 0), updates(nrhs, 0);
  double tol_cg = tol;
  int cg_rc = DW_OK;
  std::vector<double> res(nrhs, 0.0);
  for (int k = 0; k < kPasses; ++k) {
    int used = 0;
    for (int r = 0; r < nrhs; ++r) used = iters[r] > used ? iters[r] : used;
    const int left = maxit - used;
    if (left < 1) {
      cg_rc = DW_ERR_NOT_CONVERGED;
      break;
    }
    cg_rc = cg_run(lat, w->xo, w->bpr, mf, nrhs, tol_cg, left, mode, pass.data(), true, t_start);
    if (cg_rc && cg_rc != DW_ERR_NOT_CONVERGED) return cg_rc;
    for (int r = 0; r < nrhs; ++r) {
      iters[r] += pass[r].iters;
      updates[r] += pass[r].reliable_updates;
    }
    if ((rc = reconstruct_and_residual())) return rc;
    double worst = 0.0;
    for (int r = 0; r < nrhs; ++r) {
      res[r] = ee[r] > 0.0 ? std::sqrt(rr[r] / ee[r]) : 0.0;
      const double ratio = res[r] / (kAccept * tol);
      worst = ratio > worst ? ratio : worst;
    }
    if (worst <= 1.0 || cg_rc == DW_ERR_NOT_CONVERGED) break;
    double f = 0.5 / worst;
    f = f < 1e-3 ? 1e-3 : (f > 0.5 ? 0.5 : f);
    tol_cg *= f;
  }
  const double secs =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  bool all_ok = true;
  for (int r = 0; r < nrhs; ++r) {
    stats[r].iters = iters[r];
    stats[r].reliable_updates = updates[r];
    stats[r].true_resid = res[r];
    stats[r].converged = res[r] <= tol ? 1 : 0;
    stats[r].seconds = secs;
    all_ok &= stats[r].converged != 0;
  }
  if (!all_ok) return fail(DW_ERR_NOT_CONVERGED, "the residual of D x = eta did not reach tol");
  return DW_OK;
}

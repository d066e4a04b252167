// BLAS-1 and scalar kernels of the batched conjugate gradient.
#pragma once

#include "dw_common.cuh"

namespace dw {

constexpr int kBlasThreads = 256;

// Per-RHS solver state, resident on the device for the whole solve.  The
// int fields come first so that `run` and `need_update` can gate kernels
// through a strided int pointer.
struct CGState {
  int run;          // iterating: active && !need_update (gates the inner operator)
  int need_update;  // waiting for a reliable update / true-residual check
  int active;       // not yet converged, stopped or broken down
  int converged;
  int breakdown;
  int iters;
  int reliable;
  int xpend;        // this iteration's x_s += alpha p is still due (set by cg_alpha)
  double rr;        // |r_s|^2 of the normalised residual
  double pAp;
  double alpha;
  double beta;
  double sigma;     // scale of the normalised system: true residual = sigma * r_s
  double maxr;      // largest |r_s| since the last reliable update
  double bnorm;     // |b|
  double true_r2;   // last recomputed |b - A x|^2
  double sigma_next;
  double beta_next;
};

constexpr int kCGStateInts = sizeof(CGState) / sizeof(int);

// Site slots of the blocked layout: nslot = padded V4 * Ls.
struct SlotGeom {
  long long nslot;
  int V4;
  int Ls;
};

struct BlasCtx {
  SlotGeom geom;
  double nreal;  // reals per RHS on real sites (24 V4 Ls)
  int nrhs;
  int nblk;  // blocks per RHS of the reduction kernels
  BlasCtx(int V4, int Ls, int nrhs_, int num_sms);
};

int blas_redot(const BlasCtx &c, int pa, const void *a, int pb, const void *b, double *partial,
               const CGState *st, cudaStream_t s);
// y = a[r] x + b[r] y for each RHS r (c.nrhs <= kMaxRhsPerLaunch)
struct AxpbyCoefs {
  double a[kMaxRhsPerLaunch];
  double b[kMaxRhsPerLaunch];
};
int blas_axpby(const BlasCtx &c, int py, void *y, int px, const void *x, const AxpbyCoefs &cf,
               cudaStream_t s);
int blas_finalize_sum(const BlasCtx &c, const double *partial, double *out, cudaStream_t s);
int cg_residual(const BlasCtx &c, double *r, const double *b, const double *Ax, double *partial,
                const CGState *st, cudaStream_t s);
int cg_accumulate_x(const BlasCtx &c, int pr, void *x, const void *x_s, const CGState *st,
                    cudaStream_t s);
int cg_reliable_apply(const BlasCtx &c, int pp, int pr, const double *r, void *r_s, void *x_s,
                      void *p, const CGState *st, cudaStream_t s);
// x_s += alpha p (unless update_x is false: the D^+ pass made that step, see
// DslashParams::xs) and p = r_s + beta p with one read of p (the r_s -= alpha Ap
// of the step is fused into the D^+ pass, see DslashParams::rs).
int cg_direction(const BlasCtx &c, int pp, int pr, void *p, void *x_s, const void *r_s,
                 const CGState *st, cudaStream_t s, bool update_x = true);
// alpha = rr / <p, Ap> with <p, Ap> summed from nblk partials per RHS.
int cg_alpha(const BlasCtx &c, const double *partial, int nblk, CGState *st, cudaStream_t s);
// nblk: partials per RHS (-1: c.nblk, the BLAS grid; a fused D^+ pass leaves one
// per stencil CTA)
int cg_beta(const BlasCtx &c, const double *partial, CGState *st, double delta, double tol,
            int maxit, cudaStream_t s, int nblk = -1);
int cg_reliable(const BlasCtx &c, const double *partial, CGState *st, double tol, int maxit,
                int first, cudaStream_t s);
int cg_install(const BlasCtx &c, CGState *st, cudaStream_t s);
int cg_clear_update(const BlasCtx &c, CGState *st, cudaStream_t s);

}  // namespace dw

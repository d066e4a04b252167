// BLAS-1 kernels of the batched CG: fused vector updates over internal-layout
// fields with per-RHS device-resident coefficients, and real inner products
// reduced in FP64 in a fixed two-stage order (deterministic for a given grid).
//
// A field of one RHS is 6 "quads" of 4 reals per 5D site (plane q of an
// F32/F16 field, planes 2q and 2q+1 of an F64 field); thread i handles 5D
// plane index i for all 6 quads, so every access is coalesced.
#include <type_traits>

#include "dw_blas.cuh"

namespace dw {

// Quad q (4 reals) of site slot j of the blocked layout: slot j covers the
// 32-lane block j/32 (all slices in turn) and lane j%32.
template <class P, class A>
__device__ __forceinline__ void ld4(A *r, const void *base, int q, long long j) {
  const typename P::vec *b =
      (const typename P::vec *)base + (j >> 5) * (24 / P::R) * 32 + (j & 31);
  typename P::C t[4];
  if (P::R == 4) {
    load_vec<P>(t, b + q * 32);
  } else {
    load_vec<P>(t, b + 2 * q * 32);
    load_vec<P>(t + 2, b + (2 * q + 1) * 32);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) r[k] = (A)t[k];
}

template <class P, class A>
__device__ __forceinline__ void st4(void *base, int q, long long j, const A *r) {
  typename P::vec *b = (typename P::vec *)base + (j >> 5) * (24 / P::R) * 32 + (j & 31);
  typename P::C t[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) t[k] = (typename P::C)r[k];
  if (P::R == 4) {
    store_vec<P>(b + q * 32, t);
  } else {
    store_vec<P>(b + 2 * q * 32, t);
    store_vec<P>(b + (2 * q + 1) * 32, t + 2);
  }
}

// Slot j holds a lattice site (not a padding lane of the last block).
__device__ __forceinline__ bool real_slot(long long j, int V4, int Ls) {
  return (int)((j >> 5) / Ls) * 32 + (int)(j & 31) < V4;
}

#define SLOT_LOOP(j)                                                                     \
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < L.nslot;     \
       j += (long long)gridDim.x * blockDim.x)                                           \
    if (real_slot(j, L.V4, L.Ls))

// Arithmetic type of a kernel touching fields of precisions PA and PB: FP64
// only when one of them is stored in FP64 (GB300's FP64 rate is far below its
// FP32 rate); reductions always accumulate across sites in FP64.
template <class PA, class PB>
struct Arith {
  using T = typename std::conditional<(PA::id == DW_F64 || PB::id == DW_F64), double, float>::type;
};

// Block-wide FP64 sum (blockDim.x == kBlasThreads); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[kBlasThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < kBlasThreads / 32 ? ws[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

#define RHS_PTR(T, p, rhs, bytes) ((T)((char *)(p) + (size_t)(rhs) * (bytes)))

// partial[rhs][blockIdx.x] = sum over this block's sites of Re<a, b>
template <class PA, class PB>
__global__ void __launch_bounds__(kBlasThreads)
    redot_kernel(const void *a, const void *b, SlotGeom L, size_t ba, size_t bb,
                 double *partial, const CGState *st) {
  const int rhs = blockIdx.y;
  double s = 0.0;
  if (!st || st[rhs].run) {
    const void *pa = RHS_PTR(const char *, a, rhs, ba);
    const void *pb = RHS_PTR(const char *, b, rhs, bb);
    using A = typename Arith<PA, PB>::T;
    SLOT_LOOP(i) {
      A site = 0;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        A x[4], y[4];
        ld4<PA>(x, pa, q, i);
        ld4<PB>(y, pb, q, i);
#pragma unroll
        for (int k = 0; k < 4; ++k) site += x[k] * y[k];
      }
      s += (double)site;
    }
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[(size_t)rhs * gridDim.x + blockIdx.x] = s;
}

// Fixed-order sum of the partials of one RHS by one block of kSumThreads
// threads (four independent strided accumulators per thread, then the warps,
// then the warp sums in order); the result is valid in thread 0.  A stencil
// launch can leave tens of thousands of partials per RHS.
constexpr int kSumThreads = 256;
__device__ __forceinline__ double sum_partials(const double *p, int n) {
  __shared__ double ws[kSumThreads / 32];
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int k = threadIdx.x;
  for (; k + 3 * kSumThreads < n; k += 4 * kSumThreads) {
    a0 += p[k];
    a1 += p[k + kSumThreads];
    a2 += p[k + 2 * kSumThreads];
    a3 += p[k + 3 * kSumThreads];
  }
  for (; k < n; k += kSumThreads) a0 += p[k];
  double v = (a0 + a1) + (a2 + a3);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < kSumThreads / 32 ? ws[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

// out[rhs] = sum of partials (one block per RHS)
__global__ void finalize_sum_kernel(const double *partial, int nblk, double *out) {
  const int rhs = blockIdx.x;
  const double v = sum_partials(partial + (size_t)rhs * nblk, nblk);
  if (threadIdx.x == 0) out[rhs] = v;
}

// r = b - Ax in FP64; partial |r|^2.  (All three F64 fields.)
__global__ void __launch_bounds__(kBlasThreads)
    residual_kernel(double *r, const double *b, const double *Ax, SlotGeom L, size_t bytes,
                    double *partial, const CGState *st) {
  const int rhs = blockIdx.y;
  double s = 0.0;
  if (!st || st[rhs].need_update) {  // null state: every RHS
    double *pr = RHS_PTR(double *, r, rhs, bytes);
    const double *pb = RHS_PTR(const double *, b, rhs, bytes);
    const double *pa = RHS_PTR(const double *, Ax, rhs, bytes);
    SLOT_LOOP(i) {
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        double bv[4], av[4];
        ld4<F64>(bv, pb, q, i);
        ld4<F64>(av, pa, q, i);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          bv[k] -= av[k];
          s += bv[k] * bv[k];
        }
        st4<F64>(pr, q, i, bv);
      }
    }
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[(size_t)rhs * gridDim.x + blockIdx.x] = s;
}

// For RHS flagged need_update:  x += sigma * x_s;  x_s = 0;  r_s = r / sigma_new;
// p = r_s + beta_restart * p.  sigma (old scale) and sigma_new come from the
// state; run after the true residual has been reduced.
template <class PP, class PR>
__global__ void __launch_bounds__(kBlasThreads)
    reliable_apply_kernel(const double *r, void *r_s, void *x_s, void *p, SlotGeom L,
                          size_t b64, size_t bpp, size_t bpr, const CGState *st) {
  const int rhs = blockIdx.y;
  const CGState &S = st[rhs];
  if (!S.need_update || !S.active) return;
  const double inv = 1.0 / S.sigma;
  const double bp = S.beta;
  const double *pr = RHS_PTR(const double *, r, rhs, b64);
  void *prs = RHS_PTR(char *, r_s, rhs, bpr);
  void *pxs = RHS_PTR(char *, x_s, rhs, bpr);
  void *pp = RHS_PTR(char *, p, rhs, bpp);
  SLOT_LOOP(i) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      double rv[4], pv[4], z[4] = {0.0, 0.0, 0.0, 0.0};
      ld4<F64>(rv, pr, q, i);
      ld4<PP>(pv, pp, q, i);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        rv[k] *= inv;
        pv[k] = rv[k] + bp * pv[k];
      }
      st4<PR>(prs, q, i, rv);
      st4<PR>(pxs, q, i, z);
      st4<PP>(pp, q, i, pv);
    }
  }
}

// x (F64) += scale * x_s for RHS flagged need_update (scale = the old sigma).
template <class PR>
__global__ void __launch_bounds__(kBlasThreads)
    accumulate_x_kernel(void *x, const void *x_s, SlotGeom L, size_t b64, size_t bpr,
                        const CGState *st) {
  const int rhs = blockIdx.y;
  const CGState &S = st[rhs];
  if (!S.need_update) return;
  const double a = S.sigma;
  void *px = RHS_PTR(char *, x, rhs, b64);
  const void *pxs = RHS_PTR(const char *, x_s, rhs, bpr);
  SLOT_LOOP(i) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      double xv[4], sv[4];
      ld4<F64>(xv, px, q, i);
      ld4<PR>(sv, pxs, q, i);
#pragma unroll
      for (int k = 0; k < 4; ++k) xv[k] += a * sv[k];
      st4<F64>(px, q, i, xv);
    }
  }
}

// x_s += alpha p for every RHS whose step computed alpha (including those that
// now wait for a reliable update), then p = r_s + beta p for those that go on
// iterating: one read of p serves both.  update_x = false: the D^+ pass made the
// x_s step already, only the direction is left.
template <class PP, class PR>
__global__ void __launch_bounds__(kBlasThreads)
    cg_direction_kernel(void *p, void *x_s, const void *r_s, SlotGeom L, size_t bpp,
                        size_t bpr, const CGState *st, bool update_x) {
  const int rhs = blockIdx.y;
  const CGState &S = st[rhs];
  if (!S.xpend) return;
  const bool next = S.run != 0;
  if (!update_x && !next) return;
  using A = typename Arith<PP, PR>::T;
  const A a = (A)S.alpha;
  const A b = (A)S.beta;
  void *pp = RHS_PTR(char *, p, rhs, bpp);
  void *pxs = RHS_PTR(char *, x_s, rhs, bpr);
  const void *prs = RHS_PTR(const char *, r_s, rhs, bpr);
  SLOT_LOOP(i) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      A pv[4];
      ld4<PP>(pv, pp, q, i);
      if (update_x) {
        A xv[4];
        ld4<PR>(xv, pxs, q, i);
#pragma unroll
        for (int k = 0; k < 4; ++k) xv[k] += a * pv[k];
        st4<PR>(pxs, q, i, xv);
      }
      if (next) {
        A rv[4];
        ld4<PR>(rv, prs, q, i);
#pragma unroll
        for (int k = 0; k < 4; ++k) pv[k] = rv[k] + b * pv[k];
        st4<PP>(pp, q, i, pv);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Scalar CG logic, one warp per RHS.

// alpha = rr / <p, Ap>; a non-positive or non-finite <p, Ap> is a breakdown.
__global__ void cg_alpha_kernel(const double *partial, int nblk, CGState *st) {
  const int rhs = blockIdx.x;
  const double pAp = sum_partials(partial + (size_t)rhs * nblk, nblk);
  if (threadIdx.x != 0) return;
  CGState &S = st[rhs];
  S.xpend = 0;
  if (!S.run) return;
  S.pAp = pAp;
  if (!(pAp > 0.0) || !isfinite(pAp) || !isfinite(S.rr)) {
    S.breakdown = 1;
    S.active = 0;
    S.run = 0;
    S.alpha = 0.0;
    return;
  }
  S.alpha = S.rr / pAp;
  S.xpend = 1;
}

// After the update: rr_new = |r_s|^2.  Flags a reliable update when the
// iterated residual fell below delta * (largest residual since the last
// update), or when it claims convergence (|r_s| sigma <= tol |b|), or when the
// iteration budget is spent.  Otherwise beta = rr_new / rr for the direction.
__global__ void cg_beta_kernel(const double *partial, int nblk, CGState *st, double delta,
                               double tol, int maxit) {
  const int rhs = blockIdx.x;
  const double rr_new = sum_partials(partial + (size_t)rhs * nblk, nblk);
  if (threadIdx.x != 0) return;
  CGState &S = st[rhs];
  if (!S.run) return;
  S.iters += 1;
  if (!isfinite(rr_new)) {
    S.breakdown = 1;
    S.active = 0;
    S.run = 0;
    return;
  }
  const double rn = sqrt(rr_new);
  const bool claim = rn * S.sigma <= tol * S.bnorm;
  const bool drop = rn < delta * S.maxr;
  if (claim || drop || S.iters >= maxit) {
    S.need_update = 1;
    S.run = 0;
    S.beta = rr_new / S.rr;  // rescaled by sigma_old / sigma_new at the update
    S.rr = rr_new;
    return;
  }
  if (rn > S.maxr) S.maxr = rn;
  S.beta = rr_new / S.rr;
  S.rr = rr_new;
}

// After the true residual |b - A x|^2 of the flagged RHS has been reduced:
// converged -> deactivate; else set the new scale sigma_new = |r| / sqrt(n)
// (n reals per RHS, so the rescaled residual has entries of order one, which
// keeps FP16 storage away from its subnormal range) and the restart
// coefficient beta * sigma_old / sigma_new.
// Stage 1 keeps the old sigma for accumulate/apply; stage 2 installs the new.
__global__ void cg_reliable_kernel(const double *partial, int nblk, CGState *st, double tol,
                                   int maxit, int first, double nreal) {
  const int rhs = blockIdx.x;
  const double r2 = sum_partials(partial + (size_t)rhs * nblk, nblk);
  if (threadIdx.x != 0) return;
  CGState &S = st[rhs];
  if (!S.need_update) return;
  const double rn = sqrt(r2);
  S.true_r2 = r2;
  if (first) {
    // initial residual: sigma = |r0|, p = r_s
    S.bnorm = S.bnorm > 0.0 ? S.bnorm : 1.0;
    if (!(rn > tol * S.bnorm) || rn == 0.0) {
      S.converged = isfinite(r2) ? 1 : 0;
      if (!isfinite(r2)) S.breakdown = 1;
      S.active = 0;
      S.need_update = 0;
      return;
    }
    S.sigma_next = rn / sqrt(nreal);
    S.beta_next = 0.0;
    return;
  }
  if (!isfinite(r2)) {
    S.breakdown = 1;
    S.active = 0;
    S.need_update = 0;
    return;
  }
  S.reliable += 1;
  if (rn <= tol * S.bnorm) {
    S.converged = 1;
    S.active = 0;
    S.need_update = 0;
    return;
  }
  if (S.iters >= maxit) {
    S.active = 0;
    S.need_update = 0;
    return;
  }
  S.sigma_next = rn / sqrt(nreal);
  S.beta_next = S.beta * S.sigma / S.sigma_next;
}

// Install sigma_next / beta_next after the x accumulation used the old sigma.
__global__ void cg_install_kernel(CGState *st, int nrhs, double nreal) {
  const int rhs = blockIdx.x * blockDim.x + threadIdx.x;
  if (rhs >= nrhs) return;
  CGState &S = st[rhs];
  if (!S.need_update || !S.active) return;
  S.sigma = S.sigma_next;
  S.beta = S.beta_next;
  S.rr = nreal;  // |r_s|^2 right after the rescale (RMS-normalised: entries O(1))
  S.maxr = sqrt(nreal);
}

__global__ void cg_clear_update_kernel(CGState *st, int nrhs) {
  const int rhs = blockIdx.x * blockDim.x + threadIdx.x;
  if (rhs >= nrhs) return;
  st[rhs].need_update = 0;
  st[rhs].run = st[rhs].active;
}

// y = a[rhs] x + b[rhs] y (coefficients by value, at most kMaxRhsPerLaunch RHS)
template <class PY, class PX>
__global__ void __launch_bounds__(kBlasThreads)
    axpby_kernel(void *y, const void *x, SlotGeom L, size_t by, size_t bx, AxpbyCoefs cf) {
  const int rhs = blockIdx.y;
  using A = typename Arith<PY, PX>::T;
  void *py = RHS_PTR(char *, y, rhs, by);
  const void *px = RHS_PTR(const char *, x, rhs, bx);
  const A a = (A)cf.a[rhs], b = (A)cf.b[rhs];
  SLOT_LOOP(i) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      A xv[4], yv[4];
      ld4<PX>(xv, px, q, i);
      ld4<PY>(yv, py, q, i);
#pragma unroll
      for (int k = 0; k < 4; ++k) yv[k] = a * xv[k] + b * yv[k];
      st4<PY>(py, q, i, yv);
    }
  }
}

// ---------------------------------------------------------------------------
// Host launchers

static unsigned grid_for(long long nslot, int num_sms) {
  long long want = (nslot + kBlasThreads - 1) / kBlasThreads;
  long long cap = (long long)num_sms * 4;
  return (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
}

BlasCtx::BlasCtx(int V4, int Ls, int nrhs_, int num_sms_) : nrhs(nrhs_) {
  geom.V4 = V4;
  geom.Ls = Ls;
  geom.nslot = padded_v4(V4) * Ls;
  nreal = 24.0 * (double)V4 * Ls;
  nblk = (int)grid_for(geom.nslot, num_sms_);
}

#define DISPATCH_PREC(prec, T, ...)            \
  switch (prec) {                              \
    case DW_F64: { using T = F64; __VA_ARGS__; break; } \
    case DW_F32: { using T = F32; __VA_ARGS__; break; } \
    case DW_F16: { using T = F16; __VA_ARGS__; break; } \
    default: return -2;                        \
  }

static size_t rbytes(int prec, const SlotGeom &g) {
  return (size_t)24 * g.nslot * (prec == DW_F64 ? 8 : prec == DW_F32 ? 4 : 2);
}

int blas_redot(const BlasCtx &c, int pa, const void *a, int pb, const void *b, double *partial,
               const CGState *st, cudaStream_t s) {
  dim3 grid(c.nblk, c.nrhs);
  DISPATCH_PREC(pa, PA, DISPATCH_PREC(pb, PB,
      redot_kernel<PA, PB><<<grid, kBlasThreads, 0, s>>>(a, b, c.geom, rbytes(pa, c.geom),
                                                         rbytes(pb, c.geom), partial, st)));
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int blas_axpby(const BlasCtx &c, int py, void *y, int px, const void *x, const AxpbyCoefs &cf,
               cudaStream_t s) {
  if (c.nrhs > kMaxRhsPerLaunch) return -2;
  dim3 grid(c.nblk, c.nrhs);
  DISPATCH_PREC(py, PY, DISPATCH_PREC(px, PX,
      axpby_kernel<PY, PX><<<grid, kBlasThreads, 0, s>>>(y, x, c.geom, rbytes(py, c.geom),
                                                         rbytes(px, c.geom), cf)));
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int blas_finalize_sum(const BlasCtx &c, const double *partial, double *out, cudaStream_t s) {
  finalize_sum_kernel<<<c.nrhs, kSumThreads, 0, s>>>(partial, c.nblk, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int cg_residual(const BlasCtx &c, double *r, const double *b, const double *Ax, double *partial,
                const CGState *st, cudaStream_t s) {
  dim3 grid(c.nblk, c.nrhs);
  residual_kernel<<<grid, kBlasThreads, 0, s>>>(r, b, Ax, c.geom, rbytes(DW_F64, c.geom),
                                                partial, st);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int cg_accumulate_x(const BlasCtx &c, int pr, void *x, const void *x_s, const CGState *st,
                    cudaStream_t s) {
  dim3 grid(c.nblk, c.nrhs);
  DISPATCH_PREC(pr, PR,
      accumulate_x_kernel<PR><<<grid, kBlasThreads, 0, s>>>(
          x, x_s, c.geom, rbytes(DW_F64, c.geom), rbytes(pr, c.geom), st));
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int cg_reliable_apply(const BlasCtx &c, int pp, int pr, const double *r, void *r_s, void *x_s,
                      void *p, const CGState *st, cudaStream_t s) {
  dim3 grid(c.nblk, c.nrhs);
  DISPATCH_PREC(pp, PP, DISPATCH_PREC(pr, PR,
      reliable_apply_kernel<PP, PR><<<grid, kBlasThreads, 0, s>>>(
          r, r_s, x_s, p, c.geom, rbytes(DW_F64, c.geom), rbytes(pp, c.geom), rbytes(pr, c.geom),
          st)));
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int cg_direction(const BlasCtx &c, int pp, int pr, void *p, void *x_s, const void *r_s,
                 const CGState *st, cudaStream_t s, bool update_x) {
  dim3 grid(c.nblk, c.nrhs);
  DISPATCH_PREC(pp, PP, DISPATCH_PREC(pr, PR,
      cg_direction_kernel<PP, PR><<<grid, kBlasThreads, 0, s>>>(
          p, x_s, r_s, c.geom, rbytes(pp, c.geom), rbytes(pr, c.geom), st, update_x)));
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int cg_alpha(const BlasCtx &c, const double *partial, int nblk, CGState *st, cudaStream_t s) {
  cg_alpha_kernel<<<c.nrhs, kSumThreads, 0, s>>>(partial, nblk, st);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int cg_beta(const BlasCtx &c, const double *partial, CGState *st, double delta, double tol,
            int maxit, cudaStream_t s, int nblk) {
  cg_beta_kernel<<<c.nrhs, kSumThreads, 0, s>>>(partial, nblk < 0 ? c.nblk : nblk, st, delta,
                                                tol, maxit);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int cg_reliable(const BlasCtx &c, const double *partial, CGState *st, double tol, int maxit,
                int first, cudaStream_t s) {
  cg_reliable_kernel<<<c.nrhs, kSumThreads, 0, s>>>(partial, c.nblk, st, tol, maxit, first,
                                           c.nreal);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int cg_install(const BlasCtx &c, CGState *st, cudaStream_t s) {
  cg_install_kernel<<<(c.nrhs + 63) / 64, 64, 0, s>>>(st, c.nrhs, c.nreal);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int cg_clear_update(const BlasCtx &c, CGState *st, cudaStream_t s) {
  cg_clear_update_kernel<<<(c.nrhs + 63) / 64, 64, 0, s>>>(st, c.nrhs);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace dw

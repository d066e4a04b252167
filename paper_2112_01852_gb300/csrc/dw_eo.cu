// Even-odd (red-black) preconditioning of the domain-wall operator.
//
// The paper gives no solver or preconditioner; this is the standard Schur
// complement of the 4D even-odd split (sites even or odd by x + y + z + t).
// D = A + H with the local part A = alpha + beta K (alpha = b (4 - M5) + 1,
// beta = c (4 - M5) - 1) and the hopping part H = -Dhop (b + cK) / 2, which
// only couples opposite parities.  On odd sites
//   Dhat = A - H_oe A^-1 H_eo,   Dhat^+ = A^+ - H_eo^+ A^-+ H_oe^+,
// and D x = eta is solved by CG on Dhat^+ Dhat x_o = Dhat^+ (eta_o - H_oe A^-1 eta_e),
// then x_e = A^-1 (eta_e - H_eo x_o).
//
// Single-parity fields use the blocked layout over the checkerboard index
// x4 / 2 (x4 the lexicographic site index), V4/2 sites padded to a multiple of
// 32.  All four extents must be even (with an odd extent the periodic hop
// across that edge joins sites of equal parity).  The hopping parts run the
// stencil kernel in its checkerboard form; A, A^-1 and their adjoints are a
// separate kernel that walks the fifth dimension of one (site, spin half,
// colour) per thread.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dw_api_internal.cuh"
#include "dw_dslash.cuh"

namespace dw {

namespace {

struct M5Params {
  void *out;
  const void *in;
  long long nsite;       // sites of the field (real, not padded)
  long long rhs_stride;  // vecs per right-hand side
  int Ls;
  int nrhs;
  int dag;
  double alpha, beta;
  double mf[kMaxRhsPerLaunch];
};

// A = alpha + beta K along s for one (site, half, colour).  In the forward
// orientation the half couples slice s to s-1 and slice 0 to Ls-1 with -mf:
//   y_s = alpha x_s + beta x_{s-1} (s >= 1),  y_0 = alpha x_0 - beta mf x_{Ls-1};
// the upper spins of K and the lower spins of K^+ have this form, the other
// two are the same on the reversed slice order.  The inverse solves it with
// y_0 = (x_0 + mf g sum_{k=1}^{Ls-1} (-g)^{Ls-1-k} x_k) / (alpha (1 + mf (-g)^Ls)),
// g = beta / alpha, then y_s = (x_s - beta y_{s-1}) / alpha.
template <class P, bool INV>
__global__ void m5_kernel(const M5Params q) {
  using C = typename P::C;
  using vec = typename P::vec;
  using V2 = typename Pair<P>::type;
  constexpr int NPV = 24 / P::R;
  constexpr int VPQ = 4 / P::R;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per_rhs = q.nsite * 6;
  if (gid >= per_rhs * q.nrhs) return;
  const int rhs = (int)(gid / per_rhs);
  long long rem = gid - (long long)rhs * per_rhs;
  const int comp = (int)(rem / q.nsite);  // half * 3 + colour
  const int site = (int)(rem - (long long)comp * q.nsite);
  const int half = comp / 3;
  const bool rev = (half == 1) != (q.dag != 0);
  const int Ls = q.Ls;
  const vec *in = reinterpret_cast<const vec *>(q.in) + (long long)rhs * q.rhs_stride;
  vec *out = reinterpret_cast<vec *>(q.out) + (long long)rhs * q.rhs_stride;
  const long long off = (long long)comp * VPQ * kPlaneStride;
  auto at = [&](int k) {  // slice of the k-th element in the forward orientation
    return site_off(site, rev ? Ls - 1 - k : k, Ls, NPV) + off;
  };
  auto ld = [&](int k, V2 &re, V2 &im) {
    quad_in_h<HINT_NONE>(re, im, in + at(k), kPlaneStride, 0ull);
  };
  const C al = (C)q.alpha, be = (C)q.beta, mf = (C)q.mf[rhs];
  const V2 a2 = bc<V2>(al), b2 = bc<V2>(be);
  if (!INV) {
    V2 pre, pim;  // x_{k-1}
    ld(Ls - 1, pre, pim);
    pre = p_mul(bc<V2>(-mf), pre);
    pim = p_mul(bc<V2>(-mf), pim);
    for (int k = 0; k < Ls; ++k) {
      V2 xr, xi;
      ld(k, xr, xi);
      quad_out(out + at(k), kPlaneStride, p_fma(b2, pre, p_mul(a2, xr)),
               p_fma(b2, pim, p_mul(a2, xi)));
      pre = xr;
      pim = xi;
    }
  } else {
    const C g = be / al;
    const V2 mg = bc<V2>(-g);
    V2 hr = bc<V2>(C(0)), hi = bc<V2>(C(0));  // Horner sum over k = 1 .. Ls-1
    for (int k = 1; k < Ls; ++k) {
      V2 xr, xi;
      ld(k, xr, xi);
      hr = p_fma(mg, hr, xr);
      hi = p_fma(mg, hi, xi);
    }
    C pw = C(1);  // (-g)^Ls
    for (int k = 0; k < Ls; ++k) pw *= -g;
    const V2 den = bc<V2>(C(1) / (al * (C(1) + mf * pw)));
    const V2 mfg = bc<V2>(mf * g);
    V2 x0r, x0i;
    ld(0, x0r, x0i);
    V2 yr = p_mul(den, p_fma(mfg, hr, x0r)), yi = p_mul(den, p_fma(mfg, hi, x0i));
    quad_out(out + at(0), kPlaneStride, yr, yi);
    const V2 ra = bc<V2>(C(1) / al), mb = bc<V2>(-be);
    for (int k = 1; k < Ls; ++k) {
      V2 xr, xi;
      ld(k, xr, xi);
      yr = p_mul(ra, p_fma(mb, yr, xr));
      yi = p_mul(ra, p_fma(mb, yi, xi));
      quad_out(out + at(k), kPlaneStride, yr, yi);
    }
  }
}

// Copies between a full field and its two parity fields, one vec per thread.
struct SplitParams {
  void *full;
  void *even;
  void *odd;
  int L[4];
  long long nsite_cb;  // V4 / 2
  long long full_stride, cb_stride;  // vecs per RHS
  int Ls;
  int nrhs;
  int npv;
  int vec_bytes;
  int merge;  // 0: full -> even, odd; 1: even, odd -> full
};

template <class VEC>
__global__ void split_kernel(const SplitParams q) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per_parity = q.nsite_cb * q.Ls * q.npv;
  if (gid >= 2 * per_parity * q.nrhs) return;
  const int rhs = (int)(gid / (2 * per_parity));
  long long rem = gid - (long long)rhs * 2 * per_parity;
  const int par = (int)(rem / per_parity);
  rem -= (long long)par * per_parity;
  const int i = (int)(rem % q.nsite_cb);  // checkerboard index, fastest
  rem /= q.nsite_cb;
  const int pl = (int)(rem % q.npv);
  const int s = (int)(rem / q.npv);
  const int Lxh = q.L[0] / 2;
  int r = i / Lxh;
  const int y = r % q.L[1];
  r /= q.L[1];
  const int z = r % q.L[2];
  const int t = r / q.L[2];
  const int x4 = 2 * i + ((y + z + t + par) & 1);
  VEC *f = reinterpret_cast<VEC *>(q.full) + (long long)rhs * q.full_stride +
           site_off(x4, s, q.Ls, q.npv) + (long long)pl * kPlaneStride;
  VEC *h = reinterpret_cast<VEC *>(par ? q.odd : q.even) + (long long)rhs * q.cb_stride +
           site_off(i, s, q.Ls, q.npv) + (long long)pl * kPlaneStride;
  if (q.merge)
    *f = *h;
  else
    *h = *f;
}

int launch_split(dw_lattice *lat, int prec, void *full, void *even, void *odd, int nrhs,
                 int merge, cudaStream_t st) {
  SplitParams q;
  q.full = full;
  q.even = even;
  q.odd = odd;
  for (int m = 0; m < 4; ++m) q.L[m] = lat->dims[m];
  q.nsite_cb = lat->V4 / 2;
  q.npv = 24 / prec_reals_per_vec(prec);
  q.full_stride = lat->V4p * lat->Ls * q.npv;
  q.cb_stride = padded_v4(lat->V4 / 2) * lat->Ls * q.npv;
  q.Ls = lat->Ls;
  q.nrhs = nrhs;
  q.vec_bytes = prec_vec_bytes(prec);
  q.merge = merge;
  const long long n = 2 * q.nsite_cb * lat->Ls * q.npv * nrhs;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (q.vec_bytes == 16)
    split_kernel<float4><<<blocks, 256, 0, st>>>(q);
  else
    split_kernel<uint2><<<blocks, 256, 0, st>>>(q);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DW_OK : cuda_fail(e, "split launch");
}

template <class P>
int launch_m5_p(const M5Params &q, bool inv, cudaStream_t st) {
  const long long n = q.nsite * 6 * q.nrhs;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (inv)
    m5_kernel<P, true><<<blocks, 256, 0, st>>>(q);
  else
    m5_kernel<P, false><<<blocks, 256, 0, st>>>(q);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DW_OK : cuda_fail(e, "m5 launch");
}

// Tile of the checkerboard stencil: two slices per thread where Ls allows,
// 32-site tiles, the register variant (capped at FP32 / FP16), and for D at
// FP32 / FP16 the slice groups split over three (else two) CTAs, as the tuner
// prefers on the full lattice (D^+ keeps all slices in one CTA).
// Key of a tuned checkerboard tile in the lattice's tile map (its own op codes).
constexpr int kCbOpKey = 16;

TileConfig cb_default_tile(const dw_lattice *lat, int prec, int op) {
  TileConfig t;
  t.spt = lat->Ls % 2 == 0 ? 2 : 1;
  t.tx = 32;
  t.variant = prec == DW_F64 ? 0 : 4;
  t.zblk = auto_zblk(lat, prec);
  const int nchunk = lat->Ls / t.spt;
  t.sgrp = 1;
  if (op == OP_D && prec != DW_F64)
    for (int g : {3, 2})
      if (nchunk % g == 0) {
        t.sgrp = g;
        break;
      }
  return t;
}

TileConfig cb_tile(const dw_lattice *lat, int prec, int op) {
  auto it = lat->tuned.find(std::make_tuple(prec, kCbOpKey + op, 0));
  return it != lat->tuned.end() ? it->second : cb_default_tile(lat, prec, op);
}

}  // namespace

// A periodic hop keeps the parity of x + y + z + t only if every extent is
// even; the even-odd split needs that.
bool eo_ok(const dw_lattice *lat) {
  return lat->dims[0] % 2 == 0 && lat->dims[1] % 2 == 0 && lat->dims[2] % 2 == 0 &&
         lat->dims[3] % 2 == 0;
}

size_t cb_field_bytes(const dw_lattice *lat, int prec, int nrhs) {
  return (size_t)24 * (size_t)padded_v4(lat->V4 / 2) * (size_t)lat->Ls *
         (size_t)prec_real_bytes(prec) * (size_t)nrhs;
}

int eo_split(dw_lattice *lat, int prec, void *even, void *odd, const void *full, int nrhs,
             cudaStream_t st) {
  return launch_split(lat, prec, const_cast<void *>(full), even, odd, nrhs, 0, st);
}

int eo_merge(dw_lattice *lat, int prec, void *full, const void *even, const void *odd, int nrhs,
             cudaStream_t st) {
  return launch_split(lat, prec, full, const_cast<void *>(even), const_cast<void *>(odd), nrhs,
                      1, st);
}

int apply_m5(dw_lattice *lat, int prec, void *out, const void *in, const double *mf, int nrhs,
             bool inv, bool dag, cudaStream_t st) {
  const long long nsite = lat->V4 / 2;
  for (int r0 = 0; r0 < nrhs; r0 += kMaxRhsPerLaunch) {
    const int n = (nrhs - r0) < kMaxRhsPerLaunch ? (nrhs - r0) : kMaxRhsPerLaunch;
    M5Params q;
    memset(&q, 0, sizeof(q));
    const size_t rb = cb_field_bytes(lat, prec, 1);
    q.out = (char *)out + (size_t)r0 * rb;
    q.in = (const char *)in + (size_t)r0 * rb;
    q.nsite = nsite;
    q.rhs_stride = padded_v4(nsite) * lat->Ls * (24 / prec_reals_per_vec(prec));
    q.Ls = lat->Ls;
    q.nrhs = n;
    q.dag = dag ? 1 : 0;
    q.alpha = lat->b * (4.0 - lat->M5) + 1.0;
    q.beta = lat->c * (4.0 - lat->M5) - 1.0;
    for (int r = 0; r < n; ++r) q.mf[r] = mf[r0 + r];
    int rc;
    switch (prec) {
      case DW_F64: rc = launch_m5_p<F64>(q, inv, st); break;
      case DW_F32: rc = launch_m5_p<F32>(q, inv, st); break;
      default: rc = launch_m5_p<F16>(q, inv, st); break;
    }
    if (rc) return rc;
  }
  return DW_OK;
}

long long cb_ctas_per_rhs(const dw_lattice *lat, int prec, int op) {
  const TileConfig t = cb_tile(lat, prec, op);
  const long long per_plane = ((long long)lat->dims[0] / 2 * lat->dims[1] + t.tx - 1) / t.tx;
  return per_plane * t.sgrp * lat->dims[2] * lat->dims[3];
}

// Checkerboard stencil: out (parity `parity`) = alpha own + beta K own (K^+ for
// OP_DDAG) + hscale * [Dhop (b + cK) nbr] (OP_D) or hscale * [(b + cK^+) Dhop^+
// nbr] (OP_DDAG); own may be null (no local term).
int run_dslash_cb(dw_lattice *lat, int prec, int op, void *out, const void *nbr, const void *own,
                  int parity, double alpha, double beta, double hscale, const double *mf,
                  int nrhs, cudaStream_t st, const int *gate, int gate_stride,
                  double *norm_partials, const TileConfig *force, const ResidualFuse *fuse) {
  const size_t rhs_bytes = cb_field_bytes(lat, prec, 1);
  const int rs_prec = prec == DW_F64 ? DW_F64 : DW_F32;  // the residual's precision
  const size_t rs_rhs_bytes = cb_field_bytes(lat, rs_prec, 1);
  if (fuse && op != OP_DDAG) return fail(DW_ERR_ARG, "the fused residual update is D^+ only");
  const TileConfig cfg = force ? *force : cb_tile(lat, prec, op);
  const long long ctas = cb_ctas_per_rhs(lat, prec, op);
  for (int r0 = 0; r0 < nrhs; r0 += kMaxRhsPerLaunch) {
    const int n = (nrhs - r0) < kMaxRhsPerLaunch ? (nrhs - r0) : kMaxRhsPerLaunch;
    DslashParams p;
    memset(&p, 0, sizeof(p));
    p.wait_polls = -1;
    p.out = (char *)out + (size_t)r0 * rhs_bytes;
    p.in = (const char *)nbr + (size_t)r0 * rhs_bytes;
    p.own = own ? (const char *)own + (size_t)r0 * rhs_bytes : nullptr;
    p.parity = parity;
    p.alpha = alpha;
    p.beta = beta;
    p.hscale = hscale;
    p.gauge = lat->gauge[prec];
    for (int m = 0; m < 4; ++m) p.bc[m] = lat->bc[m];
    for (int m = 0; m < 4; ++m) p.L[m] = lat->dims[m];
    p.V4 = (int)(lat->V4 / 2);
    p.Ls = lat->Ls;
    p.plane = kPlaneStride;
    p.rhs_stride = padded_v4(lat->V4 / 2) * lat->Ls * (24 / prec_reals_per_vec(prec));
    p.nrhs = n;
    p.gate = gate ? gate + (size_t)r0 * gate_stride : nullptr;
    p.gate_stride = gate_stride;
    p.status = lat->dev_status;
    p.M5 = lat->M5;
    p.b = lat->b;
    p.c = lat->c;
    for (int r = 0; r < n; ++r) p.mf[r] = mf[r0 + r];
    p.norm_partials = norm_partials ? norm_partials + (size_t)r0 * ctas : nullptr;
    if (fuse) {
      p.rs = (char *)fuse->r_s + (size_t)r0 * rs_rhs_bytes;
      p.rs_stride = padded_v4(lat->V4 / 2) * lat->Ls * (24 / prec_reals_per_vec(rs_prec));
      p.rs_alpha = fuse->alpha + (size_t)r0 * fuse->alpha_stride;
      p.rs_alpha_stride = fuse->alpha_stride;
      p.rs_partials = fuse->partials + (size_t)r0 * ctas;
      if (fuse->x_s && fuse->p) {
        p.xs = (char *)fuse->x_s + (size_t)r0 * rs_rhs_bytes;
        p.pdir = (const char *)fuse->p + (size_t)r0 * rhs_bytes;
      }
    }
    const int rc = launch_dslash_cb(p, prec, op, cfg, st);
    if (rc == -2 || rc == -3)
      return fail(DW_ERR_ARG, "checkerboard stencil unavailable for this lattice");
    if (rc) return cuda_fail(cudaGetLastError(), "checkerboard stencil launch");
  }
  return DW_OK;
}

// out_o = Dhat in_o (dag: Dhat^+ in_o) at precision prec; t1, t2: even-parity
// scratch fields; norm_partials (optional, not dag) receives |out|^2 per CTA;
// fuse (optional, dag only): the CG residual update in place of storing out.
int apply_schur(dw_lattice *lat, int prec, void *out, const void *in, const double *mf, int nrhs,
                bool dag, void *t1, void *t2, cudaStream_t st, const int *gate, int gate_stride,
                double *norm_partials, const ResidualFuse *fuse) {
  const int op = dag ? OP_DDAG : OP_D;
  const double alpha = lat->b * (4.0 - lat->M5) + 1.0;
  const double beta = lat->c * (4.0 - lat->M5) - 1.0;
  // t1 = H_eo in   (dag: H_oe^+ in), on even sites
  int rc = run_dslash_cb(lat, prec, op, t1, in, nullptr, 0, 0.0, 0.0, -0.5, mf, nrhs, st, gate,
                         gate_stride, nullptr);
  if (rc) return rc;
  // t2 = A^-1 t1   (A^-+)
  if ((rc = apply_m5(lat, prec, t2, t1, mf, nrhs, true, dag, st))) return rc;
  // out = A in - H_oe t2  (A^+ in - H_eo^+ t2), on odd sites
  return run_dslash_cb(lat, prec, op, out, t2, in, 1, alpha, beta, 0.5, mf, nrhs, st, gate,
                       gate_stride, dag ? nullptr : norm_partials, nullptr,
                       dag ? fuse : nullptr);
}

// Times the checkerboard tiles of (prec, op) on two scratch parity fields (the
// hopping-only form, one RHS) and keeps the fastest for later launches.
int tune_cb(dw_lattice *lat, int prec, int op, cudaStream_t st) {
  if (lat->tuned.count(std::make_tuple(prec, kCbOpKey + op, 0))) return DW_OK;
  const size_t bytes = cb_field_bytes(lat, prec, 1);
  size_t cap_in = lat->stage_bytes, cap_out = lat->stage_bytes;
  int rc = ensure_buffer(&lat->stage_in, &cap_in, bytes);
  if (rc) return rc;
  rc = ensure_buffer(&lat->stage_out, &cap_out, bytes);
  if (rc) return rc;
  lat->stage_bytes = cap_in < cap_out ? cap_in : cap_out;
  if (cudaMemsetAsync(lat->stage_in, 0, bytes, st) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "tune memset");
  const double mf = 0.01;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(cudaGetLastError(), "event");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(cudaGetLastError(), "event");
  }
  TileConfig best_t = cb_default_tile(lat, prec, op);
  float best = 1e30f;
  const int za = auto_zblk(lat, prec);
  for (int spt : {1, 2, 3, 4})
    for (int tx : {32, 64, 96, 128})
      for (int sgrp : {1, 2, 3, 4, 6}) {
        if (lat->Ls % spt || (lat->Ls / spt) % sgrp || (op == OP_DDAG && sgrp > 8)) continue;
        const TileConfig t{spt, tx, prec == DW_F64 ? 0 : 4, za, sgrp};
        if (tx * (lat->Ls / spt / sgrp) > 1024) continue;
        if (run_dslash_cb(lat, prec, op, lat->stage_out, lat->stage_in, nullptr, 0, 0.0, 0.0,
                          -0.5, &mf, 1, st, nullptr, 0, nullptr, &t)) {
          cudaGetLastError();
          continue;  // not launchable (CTA limits)
        }
        float ms[3];
        for (float &m : ms) {
          cudaEventRecord(e0, st);
          run_dslash_cb(lat, prec, op, lat->stage_out, lat->stage_in, nullptr, 0, 0.0, 0.0, -0.5,
                        &mf, 1, st, nullptr, 0, nullptr, &t);
          cudaEventRecord(e1, st);
          cudaEventSynchronize(e1);
          m = 1e30f;
          if (cudaEventElapsedTime(&m, e0, e1) != cudaSuccess) m = 1e30f;
        }
        std::sort(ms, ms + 3);
        if (ms[1] < best) {
          best = ms[1];
          best_t = t;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  clear_error();
  const cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "tune synchronize");
  lat->tuned[std::make_tuple(prec, kCbOpKey + op, 0)] = best_t;
  return DW_OK;
}

}  // namespace dw

using namespace dw;

namespace {

int check_eo(dw_lattice *lat, int prec) {
  if (!lat) return fail(DW_ERR_ARG, "lattice is NULL");
  if (!eo_ok(lat)) return fail(DW_ERR_ARG, "even-odd fields need even Lx, Ly, Lz, Lt");
  if (prec < DW_F64 || prec > DW_F16) return fail(DW_ERR_ARG, "unknown precision %d", prec);
  return DW_OK;
}

}  // namespace

extern "C" size_t dw_fermion_bytes_eo(const dw_lattice *lat, int prec, int nrhs) {
  if (!lat || nrhs < 0 || prec < DW_F64 || prec > DW_F16 || !eo_ok(lat)) return 0;
  return cb_field_bytes(lat, prec, nrhs);
}

extern "C" int dw_eo_split(dw_lattice *lat, void *even, void *odd, const void *full, int prec,
                           int nrhs, void *stream) {
  clear_error();
  int rc = check_eo(lat, prec);
  if (rc) return rc;
  if (!even || !odd || !full) return fail(DW_ERR_ARG, "field pointer is NULL");
  if (nrhs < 1) return fail(DW_ERR_ARG, "nrhs must be >= 1");
  return eo_split(lat, prec, even, odd, full, nrhs, (cudaStream_t)stream);
}

extern "C" int dw_eo_merge(dw_lattice *lat, void *full, const void *even, const void *odd,
                           int prec, int nrhs, void *stream) {
  clear_error();
  int rc = check_eo(lat, prec);
  if (rc) return rc;
  if (!even || !odd || !full) return fail(DW_ERR_ARG, "field pointer is NULL");
  if (nrhs < 1) return fail(DW_ERR_ARG, "nrhs must be >= 1");
  return eo_merge(lat, prec, full, even, odd, nrhs, (cudaStream_t)stream);
}

extern "C" int dw_apply_m5_eo(dw_lattice *lat, void *out, const void *in, const double *mf,
                              int nrhs, int inverse, int dag, void *stream) {
  clear_error();
  int rc = check_eo(lat, lat ? lat->prec : 0);
  if (rc) return rc;
  if (!out || !in) return fail(DW_ERR_ARG, "field pointer is NULL");
  if (out == in) return fail(DW_ERR_ARG, "out must not alias in");
  if (!mf) return fail(DW_ERR_ARG, "mf is NULL");
  if (nrhs < 1) return fail(DW_ERR_ARG, "nrhs must be >= 1");
  if (lat->cplx && lat->prec == DW_F32)
    return fail(DW_ERR_STATE, "interleaved-complex FP32 fields support Dhop and Dhop^+ only");
  return apply_m5(lat, lat->prec, out, in, mf, nrhs, inverse != 0, dag != 0,
                  (cudaStream_t)stream);
}

extern "C" int dw_apply_schur(dw_lattice *lat, void *out, const void *in, const double *mf,
                              int nrhs, int dag, void *stream) {
  clear_error();
  int rc = check_eo(lat, lat ? lat->prec : 0);
  if (rc) return rc;
  if (!out || !in) return fail(DW_ERR_ARG, "field pointer is NULL");
  if (out == in) return fail(DW_ERR_ARG, "out must not alias in");
  if (!mf) return fail(DW_ERR_ARG, "mf is NULL");
  if (nrhs < 1) return fail(DW_ERR_ARG, "nrhs must be >= 1");
  if (!lat->gauge_loaded) return fail(DW_ERR_STATE, "dw_load_gauge has not been called");
  if (lat->cplx && lat->prec == DW_F32)
    return fail(DW_ERR_STATE, "interleaved-complex FP32 fields support Dhop and Dhop^+ only");
  const size_t need = 2 * cb_field_bytes(lat, lat->prec, nrhs);
  if ((rc = ensure_buffer(&lat->scratch, &lat->scratch_bytes, need))) return rc;
  void *t1 = lat->scratch;
  void *t2 = (char *)lat->scratch + need / 2;
  return apply_schur(lat, lat->prec, out, in, mf, nrhs, dag != 0, t1, t2, (cudaStream_t)stream,
                     nullptr, 0, nullptr);
}

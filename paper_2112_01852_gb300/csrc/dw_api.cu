// C ABI of the domain-wall library: lattice lifetime, gauge loading, operator
// application and field conversion.  Every entry point validates its
// arguments, never lets a C++ exception escape and reports failures through a
// negative status plus a thread-local message (dw_last_error).
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "dw_api_internal.cuh"

namespace dw {

static thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

void clear_error() { g_last_error.clear(); }

int cuda_fail(cudaError_t e, const char *what) {
  return fail(DW_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

size_t field_bytes(const dw_lattice *lat, int prec, int nrhs) {
  return (size_t)24 * (size_t)lat->V4p * (size_t)lat->Ls * (size_t)prec_real_bytes(prec) *
         (size_t)nrhs;
}

FieldGeom geom(const dw_lattice *lat) {
  FieldGeom g;
  for (int m = 0; m < 4; ++m) g.L[m] = lat->dims[m];
  g.V4 = (int)lat->V4;
  g.Ls = lat->Ls;
  return g;
}

int ensure_buffer(void **buf, size_t *cap, size_t need) {
  if (*cap >= need && *buf) return DW_OK;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc(buf, need);
  if (e != cudaSuccess) {
    *buf = nullptr;
    cudaGetLastError();
    return fail(DW_ERR_ALLOC, "cudaMalloc of %zu bytes failed: %s", need, cudaGetErrorString(e));
  }
  *cap = need;
  return DW_OK;
}

// z-blocks of the traversal order: the fewest that keep the t-reuse window of
// the input (2 * Lz/zblk planes x Ls slices) within ~20 MB of L2 (measured best
// at 32^3 x 64 x 12: 4 z-blocks; 2 and 8 were slower).
int auto_zblk(const dw_lattice *lat, int prec) {
  const double plane = (double)lat->dims[0] * lat->dims[1] * lat->Ls * 24.0 * prec_real_bytes(prec);
  for (int z = 1; z <= lat->dims[2]; ++z) {
    if (lat->dims[2] % z) continue;
    if (2.0 * (lat->dims[2] / z) * plane <= 20.0e6) return z;
  }
  return lat->dims[2];
}

// Untuned choice: the smallest slices-per-thread whose CTA of 32 sites x Ls/spt
// slice groups fits the kernel's register budget, then up to 256 threads.
TileConfig default_tile(const dw_lattice *lat, int prec, int op, int nrhs) {
  (void)nrhs;
  const int Ls = lat->Ls;
  TileConfig t{0, 32, 0, auto_zblk(lat, prec), 1};
  // interleaved-complex FP32 fields: the capped register variant
  const bool cx = lat->cplx && prec == DW_F32;
  if (cx) t.variant = 5;
  int maxt = 0;
  for (int spt : {1, 2, 3, 4}) {
    if (Ls % spt) continue;
    const int m = dslash_max_threads(prec, op, spt, t.variant);
    if ((Ls / spt) * 32 <= m) {
      t.spt = spt;
      maxt = m;
      break;
    }
  }
  if (!t.spt) {  // nothing fits: report through the launch path
    t.spt = 1;
    return t;
  }
  const int nchunk = Ls / t.spt;
  while (t.tx * 2 * nchunk <= 256 && t.tx * 2 * nchunk <= maxt) t.tx *= 2;
  return t;
}

TileConfig pick_tile(dw_lattice *lat, int prec, int op, int nrhs) {
  auto it = lat->tuned.find(std::make_tuple(prec, op, nrhs));
  if (it != lat->tuned.end()) return it->second;
  it = lat->tuned.find(std::make_tuple(prec, op, 0));
  if (it != lat->tuned.end()) return it->second;
  return default_tile(lat, prec, op, nrhs);
}

bool tile_valid(const dw_lattice *lat, int prec, int op, TileConfig t) {
  if (t.spt < 1 || t.spt > 4 || lat->Ls % t.spt) return false;
  if (lat->cplx && prec == DW_F32 && !cplx_variant_ok(op, t.variant)) return false;
  if (t.tx < 32 || t.tx % 32) return false;
  if (t.variant < 0 || t.variant > kNumVariants - 1) return false;
  if (t.variant == 8)  // the tensor-core hop: FP16 only, one tile shape
    return prec == DW_F16 && !lat->cplx && tc_variant_ok(op, lat->dims[0], lat->Ls) &&
           t.spt == 1 && t.tx == 32 && t.sgrp == 1 && t.zblk >= 1 && lat->dims[2] % t.zblk == 0;
  if (t.zblk < 1 || lat->dims[2] % t.zblk) return false;
  if (t.sgrp < 1 || (lat->Ls / t.spt) % t.sgrp || (op == OP_DDAG && t.sgrp > 8)) return false;
  if ((t.variant == 6 || t.variant == 7) &&
      (!rows_variant_ok(op, lat->dims[0], lat->dims[1], t.tx) ||
       rows_smem_bytes(t.tx, lat->Ls / t.sgrp, prec, op) > 227 * 1024))
    return false;
  const long long threads = (long long)t.tx * (lat->Ls / t.spt / t.sgrp);
  return threads <= 1024 && threads <= dslash_max_threads(prec, op, t.spt, t.variant);
}

// Stencil launch over all RHS, in groups of at most kMaxRhsPerLaunch.
size_t halo_bytes(const dw_lattice *lat, int prec, int nrhs) {
  return (size_t)12 * lat->Ls * ((size_t)lat->dims[0] * lat->dims[1] * lat->dims[2]) *
         prec_real_bytes(prec) * (size_t)nrhs;
}

// CTAs per right-hand side of a stencil launch with tile `t`.
long long dslash_ctas_per_rhs(const dw_lattice *lat, TileConfig t) {
  const long long per_plane =
      t.variant == 7 ? 1 : ((long long)lat->dims[0] * lat->dims[1] + t.tx - 1) / t.tx;
  return per_plane * t.sgrp * lat->dims[2] * lat->dims[3];
}

int run_dslash(dw_lattice *lat, int prec, int op, void *out, const void *in,
               const double *mf_host, int nrhs, cudaStream_t st, const TileConfig *force,
               const int *gate, int gate_stride, const void *halo_up, const void *halo_dn,
               double *norm_partials, int t_begin, int t_count, const ResidualFuse *fuse) {
  const size_t rhs_bytes = field_bytes(lat, prec, 1);
  const int rs_prec = prec == DW_F64 ? DW_F64 : DW_F32;  // the residual's precision
  const size_t rs_rhs_bytes = field_bytes(lat, rs_prec, 1);
  if (fuse && op != OP_DDAG) return fail(DW_ERR_ARG, "the fused residual update is D^+ only");
  const size_t hrhs_bytes = halo_bytes(lat, prec, 1);
  for (int r0 = 0; r0 < nrhs; r0 += kMaxRhsPerLaunch) {
    const int n = (nrhs - r0) < kMaxRhsPerLaunch ? (nrhs - r0) : kMaxRhsPerLaunch;
    DslashParams p;
    memset(&p, 0, sizeof(p));
    p.wait_polls = -1;
    p.out = (char *)out + (size_t)r0 * rhs_bytes;
    p.in = (const char *)in + (size_t)r0 * rhs_bytes;
    p.gauge = lat->gauge[prec];
    for (int m = 0; m < 4; ++m) p.bc[m] = lat->bc[m];
    for (int m = 0; m < 4; ++m) p.L[m] = lat->dims[m];
    p.V4 = (int)lat->V4;
    p.Ls = lat->Ls;
    p.plane = kPlaneStride;
    p.rhs_stride = lat->V4p * lat->Ls * (24 / prec_reals_per_vec(prec));
    p.nrhs = n;
    p.gate = gate ? gate + (size_t)r0 * gate_stride : nullptr;
    p.gate_stride = gate_stride;
    p.halo_up = halo_up ? (const char *)halo_up + (size_t)r0 * hrhs_bytes : nullptr;
    p.halo_dn = halo_dn ? (const char *)halo_dn + (size_t)r0 * hrhs_bytes : nullptr;
    p.t_begin = t_begin;
    p.t_count = t_count;
    p.status = lat->dev_status;
    p.wait_polls = lat->wait_polls;
    p.own = p.in;
    p.alpha = lat->b * (4.0 - lat->M5) + 1.0;
    p.beta = lat->c * (4.0 - lat->M5) - 1.0;
    p.hscale = -0.5;
    p.M5 = lat->M5;
    p.b = lat->b;
    p.c = lat->c;
    for (int r = 0; r < n; ++r) p.mf[r] = mf_host ? mf_host[r0 + r] : 0.0;
    const TileConfig cfg = force ? *force : pick_tile(lat, prec, op, nrhs);
    p.rhs_outer = cfg.rhs_outer;
    p.norm_partials =
        norm_partials ? norm_partials + (size_t)r0 * dslash_ctas_per_rhs(lat, cfg) : nullptr;
    if (fuse) {
      p.rs = (char *)fuse->r_s + (size_t)r0 * rs_rhs_bytes;
      p.rs_stride = lat->V4p * lat->Ls * (24 / prec_reals_per_vec(rs_prec));
      p.rs_alpha = fuse->alpha + (size_t)r0 * fuse->alpha_stride;
      p.rs_alpha_stride = fuse->alpha_stride;
      p.rs_partials = fuse->partials + (size_t)r0 * dslash_ctas_per_rhs(lat, cfg);
      if (fuse->x_s && fuse->p) {
        p.xs = (char *)fuse->x_s + (size_t)r0 * rs_rhs_bytes;
        p.pdir = (const char *)fuse->p + (size_t)r0 * rhs_bytes;
      }
    }
    int rc;
    if (lat->cplx && prec == DW_F32) {
      if (op != OP_DHOP && op != OP_DHOP_DAG)
        return fail(DW_ERR_STATE,
                    "interleaved-complex FP32 fields (dw_set_complex_layout) support Dhop and "
                    "Dhop^+ only");
      rc = launch_dslash_cplx(p, op, cfg, st);
    } else {
      rc = launch_dslash(p, prec, op, cfg, st);
    }
    if (rc == -2)
      return fail(DW_ERR_ARG, "unsupported tile (spt=%d, tx=%d, variant=%d, zblk=%d) for Ls=%d",
                  cfg.spt, cfg.tx, cfg.variant, cfg.zblk, lat->Ls);
    if (rc == -3)
      return fail(DW_ERR_ARG,
                  "tile (spt=%d, tx=%d, variant=%d) exceeds the kernel's CTA limits", cfg.spt,
                  cfg.tx, cfg.variant);
    if (rc) {
      const cudaError_t e0 = cudaGetLastError();
      const cudaError_t e = e0 != cudaSuccess ? e0 : last_launch_error();
      return fail(DW_ERR_CUDA, "dslash launch (op %d, precision %d, tile %d,%d,%d,%d,%d): %s", op,
                  prec, cfg.spt, cfg.tx, cfg.variant, cfg.zblk, cfg.sgrp, cudaGetErrorString(e));
    }
  }
  return DW_OK;
}

int check_apply(dw_lattice *lat, void *out, const void *in, const double *mf, int nrhs,
                bool need_mf) {
  if (!lat) return fail(DW_ERR_ARG, "lattice is NULL");
  if (!out || !in) return fail(DW_ERR_ARG, "field pointer is NULL");
  if (out == in) return fail(DW_ERR_ARG, "out must not alias in");
  if (!aligned16(out) || !aligned16(in)) return fail(DW_ERR_ARG, "fields must be 16-byte aligned");
  if (nrhs < 1) return fail(DW_ERR_ARG, "nrhs must be >= 1 (got %d)", nrhs);
  if (need_mf && !mf) return fail(DW_ERR_ARG, "mf is NULL");
  if (!lat->gauge_loaded) return fail(DW_ERR_STATE, "dw_load_gauge has not been called");
  return DW_OK;
}

int apply_op(dw_lattice *lat, int op, void *out, const void *in, const double *mf, int nrhs,
             cudaStream_t st) {
  switch (op) {
    case DW_OP_DHOP: return run_dslash(lat, lat->prec, OP_DHOP, out, in, nullptr, nrhs, st, nullptr);
    case DW_OP_DHOP_DAG:
      return run_dslash(lat, lat->prec, OP_DHOP_DAG, out, in, nullptr, nrhs, st, nullptr);
    case DW_OP_D: return run_dslash(lat, lat->prec, OP_D, out, in, mf, nrhs, st, nullptr);
    case DW_OP_DDAG: return run_dslash(lat, lat->prec, OP_DDAG, out, in, mf, nrhs, st, nullptr);
    case DW_OP_DDAGD: {
      const size_t need = field_bytes(lat, lat->prec, nrhs);
      int rc = ensure_buffer(&lat->scratch, &lat->scratch_bytes, need);
      if (rc) return rc;
      rc = run_dslash(lat, lat->prec, OP_D, lat->scratch, in, mf, nrhs, st, nullptr);
      if (rc) return rc;
      return run_dslash(lat, lat->prec, OP_DDAG, out, lat->scratch, mf, nrhs, st, nullptr);
    }
  }
  return fail(DW_ERR_ARG, "unknown operator %d", op);
}

}  // namespace dw

using namespace dw;

extern "C" {

const char *dw_last_error(void) { return g_last_error.c_str(); }

int dw_create_lattice(dw_lattice **out, const int dims[4], int Ls, int kind, double M5, double b,
                      double c, int prec, const int bc[4]) {
  clear_error();
  if (!out) return fail(DW_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!dims) return fail(DW_ERR_ARG, "dims is NULL");
  long long V4 = 1;
  for (int m = 0; m < 4; ++m) {
    if (dims[m] < 1) return fail(DW_ERR_ARG, "dims[%d] = %d must be >= 1", m, dims[m]);
    V4 *= dims[m];
    if (V4 >= (1LL << 31)) return fail(DW_ERR_ARG, "4D volume too large");
  }
  if (Ls < 1) return fail(DW_ERR_ARG, "Ls = %d must be >= 1", Ls);
  {
    bool ok = false;
    for (int spt : {1, 2, 3, 4})
      if (Ls % spt == 0 && (Ls / spt) * 32 <= 1024) ok = true;
    if (!ok) return fail(DW_ERR_ARG, "Ls = %d unsupported (need Ls/spt <= 32 for spt in 1..4)", Ls);
  }
  if (kind != DW_SHAMIR && kind != DW_MOBIUS) return fail(DW_ERR_ARG, "unknown kind %d", kind);
  // the D kernels form phi / b = psi + (c / b) K psi and scale the hop sum by b
  if (kind == DW_MOBIUS && !(b != 0.0 && b == b && c == c))
    return fail(DW_ERR_ARG, "Moebius b must be a nonzero number and c a number (b=%g c=%g)", b, c);
  if (prec != DW_F64 && prec != DW_F32 && prec != DW_F16)
    return fail(DW_ERR_ARG, "unknown precision %d", prec);
  if (bc)
    for (int m = 0; m < 4; ++m)
      if (bc[m] != 1 && bc[m] != -1) return fail(DW_ERR_ARG, "bc[%d] must be +1 or -1", m);
  dw_lattice *lat = new (std::nothrow) dw_lattice();
  if (!lat) return fail(DW_ERR_ALLOC, "host allocation failed");
  for (int m = 0; m < 4; ++m) {
    lat->dims[m] = dims[m];
    lat->bc[m] = bc ? bc[m] : (m == 3 ? -1 : 1);
  }
  lat->Ls = Ls;
  lat->V4 = V4;
  lat->V5 = V4 * Ls;
  lat->V4p = padded_v4(V4);
  lat->kind = kind;
  lat->M5 = M5;
  lat->b = kind == DW_SHAMIR ? 1.0 : b;
  lat->c = kind == DW_SHAMIR ? 0.0 : c;
  lat->prec = prec;
  lat->wait_polls = -1;
  lat->cplx = false;
  lat->reliable_delta = 0.0;
  cudaGetDevice(&lat->device);
  cudaDeviceGetAttribute(&lat->num_sms, cudaDevAttrMultiProcessorCount, lat->device);
  for (int p = 0; p < 3; ++p) {
    const size_t bytes = (size_t)4 * prec_link_vecs(p) * lat->V4p * prec_vec_bytes(p);
    if (cudaMalloc(&lat->gauge[p], bytes) != cudaSuccess) {
      cudaGetLastError();
      lat->gauge[p] = nullptr;
      dw_destroy_lattice(lat);
      return fail(DW_ERR_ALLOC, "gauge allocation failed");
    }
  }
  if (cudaMalloc(&lat->dev_status, sizeof(int)) != cudaSuccess ||
      cudaMemset(lat->dev_status, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    dw_destroy_lattice(lat);
    return fail(DW_ERR_ALLOC, "status word allocation failed");
  }
  *out = lat;
  return DW_OK;
}

void dw_destroy_lattice(dw_lattice *lat) {
  if (!lat) return;
  for (int p = 0; p < 3; ++p)
    if (lat->gauge[p]) cudaFree(lat->gauge[p]);
  if (lat->scratch) cudaFree(lat->scratch);
  if (lat->stage_in) cudaFree(lat->stage_in);
  if (lat->stage_out) cudaFree(lat->stage_out);
  if (lat->partials) cudaFree(lat->partials);
  if (lat->dev_status) cudaFree(lat->dev_status);
  cg_release(lat);
  pipe_release(lat);
  delete lat;
}

int dw_load_gauge(dw_lattice *lat, const void *U, void *stream) {
  clear_error();
  if (!lat) return fail(DW_ERR_ARG, "lattice is NULL");
  if (!U) return fail(DW_ERR_ARG, "U is NULL");
  if (!aligned16(U)) return fail(DW_ERR_ARG, "U must be 16-byte aligned");
  FieldGeom g = geom(lat);
  if (load_gauge(g, lat->bc, U, lat->gauge, (cudaStream_t)stream))
    return cuda_fail(cudaGetLastError(), "gauge conversion launch");
  lat->gauge_loaded = true;
  return DW_OK;
}

int dw_apply_Dhop(dw_lattice *lat, void *out, const void *in, int nrhs, void *stream) {
  clear_error();
  int rc = check_apply(lat, out, in, nullptr, nrhs, false);
  if (rc) return rc;
  return apply_op(lat, DW_OP_DHOP, out, in, nullptr, nrhs, (cudaStream_t)stream);
}

int dw_apply_Dhop_dag(dw_lattice *lat, void *out, const void *in, int nrhs, void *stream) {
  clear_error();
  int rc = check_apply(lat, out, in, nullptr, nrhs, false);
  if (rc) return rc;
  return apply_op(lat, DW_OP_DHOP_DAG, out, in, nullptr, nrhs, (cudaStream_t)stream);
}

int dw_apply_D(dw_lattice *lat, void *out, const void *in, const double *mf, int nrhs,
               void *stream) {
  clear_error();
  int rc = check_apply(lat, out, in, mf, nrhs, true);
  if (rc) return rc;
  return apply_op(lat, DW_OP_D, out, in, mf, nrhs, (cudaStream_t)stream);
}

int dw_apply_Ddag(dw_lattice *lat, void *out, const void *in, const double *mf, int nrhs,
                  void *stream) {
  clear_error();
  int rc = check_apply(lat, out, in, mf, nrhs, true);
  if (rc) return rc;
  return apply_op(lat, DW_OP_DDAG, out, in, mf, nrhs, (cudaStream_t)stream);
}

int dw_apply_DdagD(dw_lattice *lat, void *out, const void *in, const double *mf, int nrhs,
                   void *stream) {
  clear_error();
  int rc = check_apply(lat, out, in, mf, nrhs, true);
  if (rc) return rc;
  return apply_op(lat, DW_OP_DDAGD, out, in, mf, nrhs, (cudaStream_t)stream);
}

int dw_apply_host(dw_lattice *lat, int op, void *out_host, const void *in_host, const double *mf,
                  int nrhs, void *stream) {
  clear_error();
  if (!lat) return fail(DW_ERR_ARG, "lattice is NULL");
  if (!out_host || !in_host) return fail(DW_ERR_ARG, "host buffer is NULL");
  if (op < DW_OP_DHOP || op > DW_OP_DDAGD) return fail(DW_ERR_ARG, "unknown operator %d", op);
  const bool need_mf = op >= DW_OP_D;
  if (need_mf && !mf) return fail(DW_ERR_ARG, "mf is NULL");
  if (nrhs < 1) return fail(DW_ERR_ARG, "nrhs must be >= 1");
  if (!lat->gauge_loaded) return fail(DW_ERR_STATE, "dw_load_gauge has not been called");
  return apply_host_pipelined(lat, op, out_host, in_host, mf, nrhs, (cudaStream_t)stream);
}

int dw_set_tile(dw_lattice *lat, int op, int prec, int nrhs, int spt, int tx, int variant,
                int zblk, int sgrp) {
  clear_error();
  if (!lat) return fail(DW_ERR_ARG, "lattice is NULL");
  if (op < DW_OP_DHOP || op > DW_OP_DDAG) return fail(DW_ERR_ARG, "unknown operator %d", op);
  if (prec < DW_F64 || prec > DW_F16) return fail(DW_ERR_ARG, "unknown precision %d", prec);
  if (nrhs < 0) return fail(DW_ERR_ARG, "nrhs must be >= 0");
  TileConfig t{spt, tx, variant, zblk == 0 ? auto_zblk(lat, prec) : zblk, sgrp};
  if (!tile_valid(lat, prec, op, t))
    return fail(DW_ERR_ARG,
                "invalid tile spt=%d tx=%d variant=%d zblk=%d sgrp=%d for Ls=%d Lz=%d (slices "
                "per thread must divide Ls, tx a multiple of 32, variant 0..8 (6, 7: Lx <= 32, "
                "Lx*Ly a multiple of 32, Dhop, Dhop^+ and D only; 8: FP16 Dhop, Lx even, Ls a multiple of 4 up to 16, spt 1, tx 32, "
                "sgrp 1), zblk dividing Lz, sgrp dividing Ls/spt and at most 8 for D^+, CTA within "
                "the kernel's limits)",
                spt, tx, variant, zblk, sgrp, lat->Ls, lat->dims[2]);
  lat->tuned[std::make_tuple(prec, op, nrhs)] = t;
  return DW_OK;
}

int dw_tune(dw_lattice *lat, int op, int nrhs, int *spt, int *tx, int *variant, int *zblk,
            int *sgrp, void *stream) {
  clear_error();
  if (!lat) return fail(DW_ERR_ARG, "lattice is NULL");
  if (op < DW_OP_DHOP || op > DW_OP_DDAG) return fail(DW_ERR_ARG, "unknown operator %d", op);
  if (nrhs < 1) return fail(DW_ERR_ARG, "nrhs must be >= 1");
  if (!lat->gauge_loaded) return fail(DW_ERR_STATE, "dw_load_gauge has not been called");
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
    return fail(DW_ERR_STATE, "dw_tune called on a capturing stream");
  int rc = tune_tile(lat, lat->prec, op, nrhs, st);
  if (rc) return rc;
  const TileConfig t = pick_tile(lat, lat->prec, op, nrhs);
  if (spt) *spt = t.spt;
  if (tx) *tx = t.tx;
  if (variant) *variant = t.variant;
  if (zblk) *zblk = t.zblk;
  if (sgrp) *sgrp = t.sgrp;
  return DW_OK;
}

int dw_device_status(dw_lattice *lat) {
  clear_error();
  if (!lat) return fail(DW_ERR_ARG, "lattice is NULL");
  cudaError_t e = cudaDeviceSynchronize();
  int v = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&v, lat->dev_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && v) e = cudaMemset(lat->dev_status, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  if (v) return fail(DW_ERR_TIMEOUT, "a stencil kernel gave up waiting for its shared-memory copies");
  return DW_OK;
}

int dw_set_complex_layout(dw_lattice *lat, int interleaved) {
  clear_error();
  if (!lat) return fail(DW_ERR_ARG, "lattice is NULL");
  if (interleaved != 0 && interleaved != 1) return fail(DW_ERR_ARG, "interleaved must be 0 or 1");
  if (interleaved && lat->prec != DW_F32)
    return fail(DW_ERR_ARG, "the interleaved-complex layout exists for DW_F32 lattices only");
  lat->cplx = interleaved != 0;
  lat->tuned.clear();  // tiles tuned for the other layout no longer apply
  return DW_OK;
}

int dw_set_wait_polls(dw_lattice *lat, int polls) {
  clear_error();
  if (!lat) return fail(DW_ERR_ARG, "lattice is NULL");
  if (polls < -1) return fail(DW_ERR_ARG, "polls must be >= -1 (got %d)", polls);
  lat->wait_polls = polls;
  return DW_OK;
}

int dw_set_reliable_delta(dw_lattice *lat, double delta) {
  clear_error();
  if (!lat) return fail(DW_ERR_ARG, "lattice is NULL");
  if (!(delta >= 0.0 && delta < 1.0))
    return fail(DW_ERR_ARG, "the reliable-update threshold must be in [0, 1) (got %g)", delta);
  lat->reliable_delta = delta;
  return DW_OK;
}

int dw_get_tile(dw_lattice *lat, int op, int prec, int nrhs, int *spt, int *tx, int *variant,
                int *zblk, int *sgrp) {
  clear_error();
  if (!lat) return fail(DW_ERR_ARG, "lattice is NULL");
  if (op < DW_OP_DHOP || op > DW_OP_DDAG) return fail(DW_ERR_ARG, "unknown operator %d", op);
  if (prec < DW_F64 || prec > DW_F16) return fail(DW_ERR_ARG, "unknown precision %d", prec);
  if (nrhs < 0) return fail(DW_ERR_ARG, "nrhs must be >= 0");
  const TileConfig t = pick_tile(lat, prec, op, nrhs);
  if (spt) *spt = t.spt;
  if (tx) *tx = t.tx;
  if (variant) *variant = t.variant;
  if (zblk) *zblk = t.zblk;
  if (sgrp) *sgrp = t.sgrp;
  return DW_OK;
}

size_t dw_halo_bytes(const dw_lattice *lat, int prec, int nrhs) {
  if (!lat || nrhs < 0 || prec < DW_F64 || prec > DW_F16) return 0;
  return halo_bytes(lat, prec, nrhs);
}

}  // extern "C"

namespace dw {

// Faces of stencil operator `op` (OpKind) over nrhs RHS, in launches of at most
// kMaxRhsPerLaunch RHS (masses by value).
static int halo_pack_op(dw_lattice *lat, int op, void *send_dn, void *send_up, const void *in,
                        const double *mf, int nrhs, cudaStream_t st) {
  const size_t rhs_bytes = field_bytes(lat, lat->prec, 1);
  const size_t hrhs_bytes = halo_bytes(lat, lat->prec, 1);
  for (int r0 = 0; r0 < nrhs; r0 += kMaxRhsPerLaunch) {
    const int n = (nrhs - r0) < kMaxRhsPerLaunch ? (nrhs - r0) : kMaxRhsPerLaunch;
    DslashParams p;
    memset(&p, 0, sizeof(p));
    p.wait_polls = -1;
    p.in = (const char *)in + (size_t)r0 * rhs_bytes;
    p.gauge = lat->gauge[lat->prec];
    for (int m = 0; m < 4; ++m) p.bc[m] = lat->bc[m];
    for (int m = 0; m < 4; ++m) p.L[m] = lat->dims[m];
    p.V4 = (int)lat->V4;
    p.Ls = lat->Ls;
    p.plane = kPlaneStride;
    p.rhs_stride = lat->V4p * lat->Ls * (24 / prec_reals_per_vec(lat->prec));
    p.nrhs = n;
    p.b = lat->b;
    p.c = lat->c;
    for (int r = 0; r < n; ++r) p.mf[r] = mf ? mf[r0 + r] : 0.0;
    void *dn = (char *)send_dn + (size_t)r0 * hrhs_bytes;
    void *up = (char *)send_up + (size_t)r0 * hrhs_bytes;
    int rc;
    switch (lat->prec) {
      case DW_F64: rc = launch_halo_pack_F64(p, dn, up, op, st); break;
      case DW_F32: rc = launch_halo_pack_F32(p, dn, up, op, st); break;
      default: rc = launch_halo_pack_F16(p, dn, up, op, st); break;
    }
    if (rc) return cuda_fail(cudaGetLastError(), "halo pack launch");
  }
  return DW_OK;
}

static int check_halo(dw_lattice *lat, int op, const double *mf) {
  if (!lat) return fail(DW_ERR_ARG, "lattice is NULL");
  if (op < DW_OP_DHOP || op > DW_OP_DDAG) return fail(DW_ERR_ARG, "unknown operator %d", op);
  if (op >= DW_OP_D && !mf) return fail(DW_ERR_ARG, "mf is NULL");
  if (!lat->gauge_loaded) return fail(DW_ERR_STATE, "dw_load_gauge has not been called");
  if (lat->cplx && lat->prec == DW_F32)
    return fail(DW_ERR_STATE, "the decomposed operators need the spin-pair layout");
  return DW_OK;
}

}  // namespace dw

extern "C" {

int dw_halo_pack_op(dw_lattice *lat, int op, void *send_dn, void *send_up, const void *in,
                    const double *mf, int nrhs, void *stream) {
  clear_error();
  int rc = check_halo(lat, op, mf);
  if (rc) return rc;
  if (!send_dn || !send_up || !in) return fail(DW_ERR_ARG, "buffer pointer is NULL");
  if (!aligned16(send_dn) || !aligned16(send_up) || !aligned16(in))
    return fail(DW_ERR_ARG, "buffers must be 16-byte aligned");
  if (nrhs < 1 || nrhs > 65535) return fail(DW_ERR_ARG, "nrhs out of range");
  return halo_pack_op(lat, op, send_dn, send_up, in, mf, nrhs, (cudaStream_t)stream);
}

int dw_halo_pack(dw_lattice *lat, void *send_dn, void *send_up, const void *in, int nrhs,
                 int dag, void *stream) {
  return dw_halo_pack_op(lat, dag ? DW_OP_DHOP_DAG : DW_OP_DHOP, send_dn, send_up, in, nullptr,
                         nrhs, stream);
}

int dw_apply_op_halo(dw_lattice *lat, int op, void *out, const void *in, const void *recv_up,
                     const void *recv_dn, const double *mf, int nrhs, void *stream) {
  clear_error();
  int rc = check_halo(lat, op, mf);
  if (rc) return rc;
  if ((rc = check_apply(lat, out, in, mf, nrhs, op >= DW_OP_D))) return rc;
  if (!recv_up || !recv_dn) return fail(DW_ERR_ARG, "halo pointer is NULL");
  if (!aligned16(recv_up) || !aligned16(recv_dn))
    return fail(DW_ERR_ARG, "halos must be 16-byte aligned");
  TileConfig t = default_tile(lat, lat->prec, op, nrhs);  // the halo path is variant 0
  return run_dslash(lat, lat->prec, op, out, in, op >= DW_OP_D ? mf : nullptr, nrhs,
                    (cudaStream_t)stream, &t, nullptr, 0, recv_up, recv_dn);
}

int dw_apply_Dhop_halo(dw_lattice *lat, void *out, const void *in, const void *recv_up,
                       const void *recv_dn, int nrhs, int dag, void *stream) {
  return dw_apply_op_halo(lat, dag ? DW_OP_DHOP_DAG : DW_OP_DHOP, out, in, recv_up, recv_dn,
                          nullptr, nrhs, stream);
}

size_t dw_fermion_bytes(const dw_lattice *lat, int prec, int nrhs) {
  if (!lat || nrhs < 0 || prec < DW_F64 || prec > DW_F16) return 0;
  return field_bytes(lat, prec, nrhs);
}

int dw_pack_fermion(dw_lattice *lat, void *dst_internal, int prec, const void *src_c128, int nrhs,
                    void *stream) {
  clear_error();
  if (!lat) return fail(DW_ERR_ARG, "lattice is NULL");
  if (!dst_internal || !src_c128) return fail(DW_ERR_ARG, "field pointer is NULL");
  if (prec < DW_F64 || prec > DW_F16) return fail(DW_ERR_ARG, "unknown precision %d", prec);
  if (nrhs < 1 || nrhs > 65535) return fail(DW_ERR_ARG, "nrhs out of range");
  if (!aligned16(dst_internal) || !aligned16(src_c128))
    return fail(DW_ERR_ARG, "fields must be 16-byte aligned");
  if (pack_fermion(geom(lat), prec, dst_internal, src_c128, nrhs, (cudaStream_t)stream,
                   lat->cplx && prec == DW_F32))
    return cuda_fail(cudaGetLastError(), "pack launch");
  return DW_OK;
}

int dw_unpack_fermion(dw_lattice *lat, void *dst_c128, const void *src_internal, int prec,
                      int nrhs, void *stream) {
  clear_error();
  if (!lat) return fail(DW_ERR_ARG, "lattice is NULL");
  if (!dst_c128 || !src_internal) return fail(DW_ERR_ARG, "field pointer is NULL");
  if (prec < DW_F64 || prec > DW_F16) return fail(DW_ERR_ARG, "unknown precision %d", prec);
  if (nrhs < 1 || nrhs > 65535) return fail(DW_ERR_ARG, "nrhs out of range");
  if (!aligned16(dst_c128) || !aligned16(src_internal))
    return fail(DW_ERR_ARG, "fields must be 16-byte aligned");
  if (unpack_fermion(geom(lat), prec, dst_c128, src_internal, nrhs, (cudaStream_t)stream,
                     lat->cplx && prec == DW_F32))
    return cuda_fail(cudaGetLastError(), "unpack launch");
  return DW_OK;
}

}  // extern "C"

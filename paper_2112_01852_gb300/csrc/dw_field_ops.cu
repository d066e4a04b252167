// C ABI of the level-1 field operations the distributed solver drives from the
// host: real inner products per right-hand side (FP64 sums in a fixed order)
// and y = a x + b y, on internal-layout fields of any precision.  The paper has
// no solver; these are the vector steps of textbook CG (Hestenes-Stiefel), whose
// global sums a decomposed lattice completes across ranks.
#include <cstring>
#include <vector>

#include "dw_api_internal.cuh"
#include "dw_blas.cuh"

using namespace dw;

namespace {

int check_fields(dw_lattice *lat, int prec, const void *a, const void *b, int nrhs) {
  if (!lat) return fail(DW_ERR_ARG, "lattice is NULL");
  if (prec < DW_F64 || prec > DW_F16) return fail(DW_ERR_ARG, "unknown precision %d", prec);
  if (!a || !b) return fail(DW_ERR_ARG, "field pointer is NULL");
  if ((reinterpret_cast<uintptr_t>(a) & 15u) || (reinterpret_cast<uintptr_t>(b) & 15u))
    return fail(DW_ERR_ARG, "fields must be 16-byte aligned");
  if (nrhs < 1 || nrhs > 65535) return fail(DW_ERR_ARG, "nrhs out of range");
  if (lat->cplx && prec == DW_F32)
    return fail(DW_ERR_STATE, "field operations need the spin-pair layout");
  return DW_OK;
}

}  // namespace

extern "C" int dw_field_redot(dw_lattice *lat, int prec, const void *a, const void *b, int nrhs,
                              double *out, void *stream) {
  clear_error();
  int rc = check_fields(lat, prec, a, b, nrhs);
  if (rc) return rc;
  if (!out) return fail(DW_ERR_ARG, "out is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  BlasCtx c((int)lat->V4, lat->Ls, nrhs, lat->num_sms);
  const size_t need = sizeof(double) * ((size_t)c.nblk + 1) * nrhs;
  if ((rc = ensure_buffer((void **)&lat->partials, &lat->partials_cap, need))) return rc;
  double *sums = lat->partials + (size_t)c.nblk * nrhs;
  if (blas_redot(c, prec, a, prec, b, lat->partials, nullptr, st) ||
      blas_finalize_sum(c, lat->partials, sums, st))
    return cuda_fail(cudaGetLastError(), "inner product launch");
  cudaError_t e = cudaMemcpyAsync(out, sums, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "inner product readback");
  return DW_OK;
}

extern "C" int dw_field_axpby(dw_lattice *lat, int prec, void *y, const double *a, const void *x,
                              const double *b, int nrhs, void *stream) {
  clear_error();
  int rc = check_fields(lat, prec, y, x, nrhs);
  if (rc) return rc;
  if (!a || !b) return fail(DW_ERR_ARG, "coefficient array is NULL");
  const size_t rhs_bytes = field_bytes(lat, prec, 1);
  for (int r0 = 0; r0 < nrhs; r0 += kMaxRhsPerLaunch) {
    const int n = (nrhs - r0) < kMaxRhsPerLaunch ? (nrhs - r0) : kMaxRhsPerLaunch;
    BlasCtx c((int)lat->V4, lat->Ls, n, lat->num_sms);
    AxpbyCoefs cf;
    memset(&cf, 0, sizeof(cf));
    for (int r = 0; r < n; ++r) {
      cf.a[r] = a[r0 + r];
      cf.b[r] = b[r0 + r];
    }
    if (blas_axpby(c, prec, (char *)y + (size_t)r0 * rhs_bytes, prec,
                   (const char *)x + (size_t)r0 * rhs_bytes, cf, (cudaStream_t)stream))
      return cuda_fail(cudaGetLastError(), "axpby launch");
  }
  return DW_OK;
}

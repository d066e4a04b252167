// Conjugate gradient on D^+D (plain FP64 and mixed precision).
#include "dw_api_internal.cuh"

namespace dw {
void cg_release(dw_lattice *lat) { (void)lat; }
}  // namespace dw

extern "C" int dw_cg_solve(dw_lattice *lat, void *x, const void *b, const double *mf, int nrhs,
                           double tol, int maxit, int mode, dw_cg_stats *stats, void *stream) {
  (void)lat; (void)x; (void)b; (void)mf; (void)nrhs; (void)tol; (void)maxit; (void)mode;
  (void)stats; (void)stream;
  return dw::fail(DW_ERR_STATE, "dw_cg_solve: not available yet");
}

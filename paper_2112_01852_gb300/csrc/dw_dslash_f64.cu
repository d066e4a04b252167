// F64 instantiation of the fused domain-wall stencil kernel.
#include "dw_dslash.cuh"

namespace dw {
int launch_dslash_f64(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st) {
  return launch_dslash_impl<F64>(p, op, cfg, st);
}
int dslash_max_threads_f64(int op, int spt) { return max_threads_impl<F64>(op, spt); }
}  // namespace dw

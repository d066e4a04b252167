// F32 instantiation of the fused domain-wall stencil kernel.
#include "dw_dslash.cuh"

namespace dw {
int launch_dslash_f32(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st) {
  return launch_dslash_impl<F32>(p, op, cfg, st);
}
int dslash_max_threads_f32(int op, int spt) { return max_threads_impl<F32>(op, spt); }
}  // namespace dw

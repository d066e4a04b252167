// Dispatch of the stencil kernel over (precision, hop-phase variant); each
// pair lives in its own translation unit.  FP64 builds only the register
// variants (its arithmetic, not its loads, bounds it on this GPU).
#include "dw_common.cuh"

namespace dw {

cudaError_t &last_launch_error() {
  static thread_local cudaError_t e = cudaSuccess;
  return e;
}

int launch_dslash_F64_v0(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int dslash_max_threads_F64_v0(int op, int spt);
int launch_dslash_F64_v2(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int dslash_max_threads_F64_v2(int op, int spt);
int launch_dslash_F32_v0(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int dslash_max_threads_F32_v0(int op, int spt);
int launch_dslash_F32_v1(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int dslash_max_threads_F32_v1(int op, int spt);
int launch_dslash_F32_v2(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int dslash_max_threads_F32_v2(int op, int spt);
int launch_dslash_F32_v3(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int dslash_max_threads_F32_v3(int op, int spt);
int launch_dslash_F32_v4(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int dslash_max_threads_F32_v4(int op, int spt);
int launch_dslash_F32_v5(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int dslash_max_threads_F32_v5(int op, int spt);
int launch_dslash_F32_v6(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int dslash_max_threads_F32_v6(int op, int spt);
int launch_dslash_F32_v7(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int dslash_max_threads_F32_v7(int op, int spt);
int launch_dslash_F16_v0(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int dslash_max_threads_F16_v0(int op, int spt);
int launch_dslash_F16_v1(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int dslash_max_threads_F16_v1(int op, int spt);
int launch_dslash_F16_v2(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int dslash_max_threads_F16_v2(int op, int spt);
int launch_dslash_F16_v3(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int dslash_max_threads_F16_v3(int op, int spt);
int launch_dslash_F16_v4(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int dslash_max_threads_F16_v4(int op, int spt);
int launch_dslash_F16_v5(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int dslash_max_threads_F16_v5(int op, int spt);
int launch_dslash_F16_v6(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int dslash_max_threads_F16_v6(int op, int spt);
int launch_dslash_F16_v7(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int dslash_max_threads_F16_v7(int op, int spt);

int launch_dslash_cplx_v4(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int launch_dslash_cplx_v5(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int launch_dslash_cplx_v6(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int launch_dslash_cplx_v7(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);

int launch_dslash_cplx(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st) {
  switch (cfg.variant) {
    case 4: return launch_dslash_cplx_v4(p, op, cfg, st);
    case 5: return launch_dslash_cplx_v5(p, op, cfg, st);
    case 6: return launch_dslash_cplx_v6(p, op, cfg, st);
    case 7: return launch_dslash_cplx_v7(p, op, cfg, st);
  }
  return -2;
}

int launch_dslash_cb_F64(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int launch_dslash_cb_F32(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
int launch_dslash_cb_F16(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);

int launch_dslash_cb(const DslashParams &p, int prec, int op, TileConfig cfg, cudaStream_t st) {
  switch (prec) {
    case DW_F64: return launch_dslash_cb_F64(p, op, cfg, st);
    case DW_F32: return launch_dslash_cb_F32(p, op, cfg, st);
    case DW_F16: return launch_dslash_cb_F16(p, op, cfg, st);
  }
  return -2;
}

int launch_dslash(const DslashParams &p, int prec, int op, TileConfig cfg, cudaStream_t st) {
  const int cfg_variant = cfg.variant;
  switch (prec) {
    case DW_F64:
      switch (cfg_variant) {
        case 0: return launch_dslash_F64_v0(p, op, cfg, st);
        case 2: return launch_dslash_F64_v2(p, op, cfg, st);
        default: return -2;
      }
    case DW_F32:
      switch (cfg_variant) {
        case 0: return launch_dslash_F32_v0(p, op, cfg, st);
        case 1: return launch_dslash_F32_v1(p, op, cfg, st);
        case 2: return launch_dslash_F32_v2(p, op, cfg, st);
        case 3: return launch_dslash_F32_v3(p, op, cfg, st);
        case 4: return launch_dslash_F32_v4(p, op, cfg, st);
        case 5: return launch_dslash_F32_v5(p, op, cfg, st);
        case 6: return launch_dslash_F32_v6(p, op, cfg, st);
        case 7: return launch_dslash_F32_v7(p, op, cfg, st);
        default: return -2;
      }
    case DW_F16:
      switch (cfg_variant) {
        case 0: return launch_dslash_F16_v0(p, op, cfg, st);
        case 1: return launch_dslash_F16_v1(p, op, cfg, st);
        case 2: return launch_dslash_F16_v2(p, op, cfg, st);
        case 3: return launch_dslash_F16_v3(p, op, cfg, st);
        case 4: return launch_dslash_F16_v4(p, op, cfg, st);
        case 5: return launch_dslash_F16_v5(p, op, cfg, st);
        case 6: return launch_dslash_F16_v6(p, op, cfg, st);
        case 7: return launch_dslash_F16_v7(p, op, cfg, st);
        case 8: return launch_dslash_tc_F16(p, op, cfg, st);
        default: return -2;
      }
  }
  return -2;
}

int dslash_max_threads(int prec, int op, int spt, int variant) {
  const int cfg_variant = variant;
  switch (prec) {
    case DW_F64:
      switch (cfg_variant) {
        case 0: return dslash_max_threads_F64_v0(op, spt);
        case 2: return dslash_max_threads_F64_v2(op, spt);
        default: return 0;
      }
    case DW_F32:
      switch (cfg_variant) {
        case 0: return dslash_max_threads_F32_v0(op, spt);
        case 1: return dslash_max_threads_F32_v1(op, spt);
        case 2: return dslash_max_threads_F32_v2(op, spt);
        case 3: return dslash_max_threads_F32_v3(op, spt);
        case 4: return dslash_max_threads_F32_v4(op, spt);
        case 5: return dslash_max_threads_F32_v5(op, spt);
        case 6: return dslash_max_threads_F32_v6(op, spt);
        case 7: return dslash_max_threads_F32_v7(op, spt);
        default: return 0;
      }
    case DW_F16:
      switch (cfg_variant) {
        case 0: return dslash_max_threads_F16_v0(op, spt);
        case 1: return dslash_max_threads_F16_v1(op, spt);
        case 2: return dslash_max_threads_F16_v2(op, spt);
        case 3: return dslash_max_threads_F16_v3(op, spt);
        case 4: return dslash_max_threads_F16_v4(op, spt);
        case 5: return dslash_max_threads_F16_v5(op, spt);
        case 6: return dslash_max_threads_F16_v6(op, spt);
        case 7: return dslash_max_threads_F16_v7(op, spt);
        default: return 0;
      }
  }
  return 0;
}

}  // namespace dw

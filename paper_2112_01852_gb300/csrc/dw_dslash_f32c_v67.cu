// Interleaved-complex FP32 stencil (layout ablation), row-staged variants 6 and 7.
#include "dw_dslash.cuh"

DW_DSLASH_CPLX_INSTANTIATE(6)
DW_DSLASH_CPLX_INSTANTIATE(7)

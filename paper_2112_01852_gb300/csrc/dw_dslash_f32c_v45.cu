// Interleaved-complex FP32 stencil (layout ablation), register variants 4 and 5.
#include "dw_dslash.cuh"

DW_DSLASH_CPLX_INSTANTIATE(4)
DW_DSLASH_CPLX_INSTANTIATE(5)

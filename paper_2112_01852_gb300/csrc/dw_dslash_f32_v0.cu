// F32 storage, hop-phase variant 0 of the fused domain-wall stencil kernel.
#include "dw_dslash.cuh"

DW_DSLASH_INSTANTIATE(F32, 0)

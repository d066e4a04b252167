// F16 storage, hop-phase variant 1 of the fused domain-wall stencil kernel.
#include "dw_dslash.cuh"

DW_DSLASH_INSTANTIATE(F16, 1)

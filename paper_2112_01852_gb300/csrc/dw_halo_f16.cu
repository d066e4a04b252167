// F16 face packing for the t decomposition of the stencil ("virtual ranks").
#include "dw_dslash.cuh"

DW_HALO_INSTANTIATE(F16)

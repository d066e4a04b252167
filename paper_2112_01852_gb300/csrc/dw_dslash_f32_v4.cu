// F32 storage, hop-phase variant 4 (variant 0 under a 3-CTA register cap).
#include "dw_dslash.cuh"

DW_DSLASH_INSTANTIATE(F32, 4)

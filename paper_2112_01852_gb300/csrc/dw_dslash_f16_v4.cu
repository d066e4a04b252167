// F16 storage, hop-phase variant 4 (variant 5 with at most 128 registers per thread).
#include "dw_dslash.cuh"

DW_DSLASH_INSTANTIATE(F16, 4)

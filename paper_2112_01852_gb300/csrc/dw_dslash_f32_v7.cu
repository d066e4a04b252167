// F32 storage, hop-phase variant 7 (variant 6 walking a whole plane with a ring of staged rows).
#include "dw_dslash.cuh"

DW_DSLASH_INSTANTIATE(F32, 7)

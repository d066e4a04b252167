// F16 storage, hop-phase variant 5 (variant 0 with L2 eviction hints on the t hops).
#include "dw_dslash.cuh"

DW_DSLASH_INSTANTIATE(F16, 5)

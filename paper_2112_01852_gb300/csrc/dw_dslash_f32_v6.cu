// F32 storage, hop-phase variant 6 (x and y neighbour rows staged in shared memory by bulk copies).
#include "dw_dslash.cuh"

DW_DSLASH_INSTANTIATE(F32, 6)

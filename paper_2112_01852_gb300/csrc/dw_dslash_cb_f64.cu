// F64 storage, checkerboard (single-parity) stencil for the even-odd operators, variant 0.
#include "dw_dslash.cuh"

DW_DSLASH_CB_INSTANTIATE(F64, 0)

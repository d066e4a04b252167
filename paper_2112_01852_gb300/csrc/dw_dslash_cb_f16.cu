// F16 storage, checkerboard (single-parity) stencil for the even-odd operators, variant 4.
#include "dw_dslash.cuh"

DW_DSLASH_CB_INSTANTIATE(F16, 4)

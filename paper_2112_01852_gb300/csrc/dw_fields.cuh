// Layout and conversion kernels for fermion and gauge fields.
#pragma once

#include "dw_common.cuh"

namespace dw {

struct FieldGeom {
  int L[4];
  int V4;
  int Ls;
  long long V5() const { return (long long)V4 * Ls; }
};

// canonical complex128 (device) -> internal at `prec` (cplx: FP32 fields with
// interleaved-complex quads)
int pack_fermion(const FieldGeom &g, int prec, void *dst, const void *src, int nrhs,
                 cudaStream_t st, bool cplx = false);
// internal at `prec` -> canonical complex128 (device)
int unpack_fermion(const FieldGeom &g, int prec, void *dst, const void *src, int nrhs,
                   cudaStream_t st, bool cplx = false);
// canonical gauge (device) -> internal links at F64, F32 and F16
int load_gauge(const FieldGeom &g, const int bc[4], const void *U, void *const gauge[3],
               cudaStream_t st);
// internal field precision conversion
int convert_fermion(const FieldGeom &g, int pi, int po, void *dst, const void *src, int nrhs,
                    cudaStream_t st);

}  // namespace dw

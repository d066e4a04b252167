// Field layout kernels: canonical <-> internal fermion packing, gauge
// conversion with the boundary signs folded in, and precision conversion.
#include "dw_fields.cuh"

namespace dw {

// ---------------------------------------------------------------------------
// Canonical fermion complex128 [rhs][x4][s][spin][col] <-> internal planes.
// One thread per (x4, s) of one RHS.  Internal real I = half*12 + c*4 + ri*2 + j
// (chirality half, colour c, re/im ri, spin j within the half) holds the
// canonical real ((2*half + j)*3 + c)*2 + ri: each 4-real quad is the spin
// pair (Re j0, Re j1, Im j0, Im j1) of one colour.
__device__ __forceinline__ int canon_real(int I) {
  const int half = I / 12, i = I % 12;
  const int c = i / 4, ri = (i % 4) / 2, j = i % 2;
  return ((2 * half + j) * 3 + c) * 2 + ri;
}
template <class P>
__global__ void pack_kernel(typename P::vec *dst, const double *src, long long V5, int V4,
                            int Ls, long long rhs_stride) {
  constexpr int NP = 24 / P::R;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int rhs = blockIdx.y;
  if (i >= V5) return;
  const int x4 = (int)(i / Ls);
  const int s = (int)(i % Ls);
  const double *p = src + ((long long)rhs * V5 + i) * 24;
  typename P::vec *d = dst + (long long)rhs * rhs_stride + site_off(x4, s, Ls, NP);
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    double r[P::R];
#pragma unroll
    for (int k = 0; k < P::R; ++k) r[k] = p[canon_real(q * P::R + k)];
    d[q * kPlaneStride] = narrow_from_f64(r, (typename P::vec *)nullptr);
  }
}

template <class P>
__global__ void unpack_kernel(double *dst, const typename P::vec *src, long long V5, int V4,
                              int Ls, long long rhs_stride) {
  using C = typename P::C;
  constexpr int NP = 24 / P::R;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int rhs = blockIdx.y;
  if (i >= V5) return;
  const int x4 = (int)(i / Ls);
  const int s = (int)(i % Ls);
  double *p = dst + ((long long)rhs * V5 + i) * 24;
  const typename P::vec *sp = src + (long long)rhs * rhs_stride + site_off(x4, s, Ls, NP);
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    C r[P::R];
    load_vec<P>(r, sp + q * kPlaneStride);
#pragma unroll
    for (int k = 0; k < P::R; ++k) p[canon_real(q * P::R + k)] = (double)r[k];
  }
}

template <class P>
static int pack_t(const FieldGeom &g, void *dst, const void *src, int nrhs, cudaStream_t st) {
  const long long V5 = g.V5();
  const int tpb = 256;
  dim3 grid((unsigned)((V5 + tpb - 1) / tpb), nrhs);
  pack_kernel<P><<<grid, tpb, 0, st>>>((typename P::vec *)dst, (const double *)src, V5, g.V4,
                                       g.Ls, padded_v4(g.V4) * g.Ls * (24 / P::R));
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <class P>
static int unpack_t(const FieldGeom &g, void *dst, const void *src, int nrhs, cudaStream_t st) {
  const long long V5 = g.V5();
  const int tpb = 256;
  dim3 grid((unsigned)((V5 + tpb - 1) / tpb), nrhs);
  unpack_kernel<P><<<grid, tpb, 0, st>>>((double *)dst, (const typename P::vec *)src, V5, g.V4,
                                         g.Ls, padded_v4(g.V4) * g.Ls * (24 / P::R));
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int pack_fermion(const FieldGeom &g, int prec, void *dst, const void *src, int nrhs,
                 cudaStream_t st) {
  switch (prec) {
    case DW_F64: return pack_t<F64>(g, dst, src, nrhs, st);
    case DW_F32: return pack_t<F32>(g, dst, src, nrhs, st);
    case DW_F16: return pack_t<F16>(g, dst, src, nrhs, st);
  }
  return -2;
}

int unpack_fermion(const FieldGeom &g, int prec, void *dst, const void *src, int nrhs,
                   cudaStream_t st) {
  switch (prec) {
    case DW_F64: return unpack_t<F64>(g, dst, src, nrhs, st);
    case DW_F32: return unpack_t<F32>(g, dst, src, nrhs, st);
    case DW_F16: return unpack_t<F16>(g, dst, src, nrhs, st);
  }
  return -2;
}

// ---------------------------------------------------------------------------
// Gauge: canonical complex128 [x4][mu][row][col] -> per precision blocked links
// (link_off): all 18 reals at F64, the first two rows (12 reals) at F32 / F16.
// A link U_mu(x) with x_mu = L_mu - 1 crosses the lattice edge and is
// multiplied by bc[mu].
template <class P>
__device__ __forceinline__ void store_link(void *gauge, int mu, int x4, const double *u) {
  typename P::vec *m = (typename P::vec *)gauge + link_off(x4, mu, P::NLV);
#pragma unroll
  for (int q = 0; q < P::NLV; ++q)
    m[q * 32] = narrow_from_f64(u + q * P::R, (typename P::vec *)nullptr);
}

__global__ void gauge_kernel(const double *U, int L0, int L1, int L2, int L3, int bc0, int bc1,
                             int bc2, int bc3, void *g64, void *g32, void *g16) {
  const long long V4 = (long long)L0 * L1 * L2 * L3;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= 4 * V4) return;
  const int x4 = (int)(i / 4);
  const int mu = (int)(i % 4);
  int c[4];
  int rem = x4;
  c[0] = rem % L0;
  rem /= L0;
  c[1] = rem % L1;
  rem /= L1;
  c[2] = rem % L2;
  c[3] = rem / L2;
  const int L[4] = {L0, L1, L2, L3};
  const int bc[4] = {bc0, bc1, bc2, bc3};
  const double f = (c[mu] == L[mu] - 1) ? (double)bc[mu] : 1.0;
  double u[18];
  const double *src = U + ((long long)x4 * 4 + mu) * 18;
#pragma unroll
  for (int k = 0; k < 18; ++k) u[k] = f * src[k];
  store_link<F64>(g64, mu, x4, u);
  store_link<F32>(g32, mu, x4, u);
  store_link<F16>(g16, mu, x4, u);
}

int load_gauge(const FieldGeom &g, const int bc[4], const void *U, void *const gauge[3],
               cudaStream_t st) {
  const long long n = 4LL * g.V4;
  const int tpb = 256;
  gauge_kernel<<<(unsigned)((n + tpb - 1) / tpb), tpb, 0, st>>>(
      (const double *)U, g.L[0], g.L[1], g.L[2], g.L[3], bc[0], bc[1], bc[2], bc[3], gauge[0],
      gauge[1], gauge[2]);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
// Precision conversion between internal fields: one thread per site slot of
// the blocked layout (padding lanes skipped), all 6 quads (a quad is 4 reals:
// plane q of F32/F16, planes 2q and 2q+1 of F64).
template <class PI, class PO>
__global__ void convert_kernel(void *dst, const void *src, long long nslot, int V4, int Ls,
                               long long rhs_in, long long rhs_out) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int rhs = blockIdx.y;
  if (j >= nslot) return;
  const int x4 = (int)((j >> 5) / Ls) * 32 + (int)(j & 31);
  if (x4 >= V4) return;
  const typename PI::vec *s =
      (const typename PI::vec *)((const char *)src + rhs * rhs_in) + (j >> 5) * (24 / PI::R) * 32 + (j & 31);
  typename PO::vec *d =
      (typename PO::vec *)((char *)dst + rhs * rhs_out) + (j >> 5) * (24 / PO::R) * 32 + (j & 31);
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    typename PI::C a[4];
    typename PO::C b[4];
    if (PI::R == 4) {
      load_vec<PI>(a, s + q * 32);
    } else {
      load_vec<PI>(a, s + 2 * q * 32);
      load_vec<PI>(a + 2, s + (2 * q + 1) * 32);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) b[k] = (typename PO::C)a[k];
    if (PO::R == 4) {
      store_vec<PO>(d + q * 32, b);
    } else {
      store_vec<PO>(d + 2 * q * 32, b);
      store_vec<PO>(d + (2 * q + 1) * 32, b + 2);
    }
  }
}

template <class PI, class PO>
static int convert_t(const FieldGeom &g, void *dst, const void *src, int nrhs, cudaStream_t st) {
  const long long nslot = padded_v4(g.V4) * g.Ls;
  const int tpb = 256;
  dim3 grid((unsigned)((nslot + tpb - 1) / tpb), nrhs);
  convert_kernel<PI, PO><<<grid, tpb, 0, st>>>(dst, src, nslot, g.V4, g.Ls, 24 * nslot * PI::RB,
                                               24 * nslot * PO::RB);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <class PI>
static int convert_to(const FieldGeom &g, int po, void *dst, const void *src, int nrhs,
                      cudaStream_t st) {
  switch (po) {
    case DW_F64: return convert_t<PI, F64>(g, dst, src, nrhs, st);
    case DW_F32: return convert_t<PI, F32>(g, dst, src, nrhs, st);
    case DW_F16: return convert_t<PI, F16>(g, dst, src, nrhs, st);
  }
  return -2;
}

int convert_fermion(const FieldGeom &g, int pi, int po, void *dst, const void *src, int nrhs,
                    cudaStream_t st) {
  switch (pi) {
    case DW_F64: return convert_to<F64>(g, po, dst, src, nrhs, st);
    case DW_F32: return convert_to<F32>(g, po, dst, src, nrhs, st);
    case DW_F16: return convert_to<F16>(g, po, dst, src, nrhs, st);
  }
  return -2;
}

}  // namespace dw

// Field layout kernels: canonical <-> internal fermion packing, gauge
// conversion with the boundary signs folded in, and precision conversion.
#include "dw_fields.cuh"

namespace dw {

// ---------------------------------------------------------------------------
// Canonical fermion complex128 [rhs][x4][s][spin][col] <-> internal planes.
// Internal real I = half*12 + c*4 + ri*2 + j (chirality half, colour c, re/im
// ri, spin j within the half) holds the canonical real
// ((2*half + j)*3 + c)*2 + ri: each 4-real quad is the spin pair
// (Re j0, Re j1, Im j0, Im j1) of one colour.
//
// Both directions are transposes of one 32-site block and kSC consecutive
// slices per CTA through shared memory: the internal side of the chunk is one
// contiguous run of vecs (coalesced 16-byte accesses, 8-byte at FP16), the
// canonical side is kSC x 12 consecutive complex128 per site (coalesced
// 16-byte accesses); the transpose itself happens in shared memory, one FP64
// real per (site, slice, internal real I), rows padded to an odd length.
constexpr int kSC = 4;        // slices per CTA
constexpr int kXposeTPB = 128;
constexpr int kLaneStride = kSC * 24 + 1;  // doubles per site row of the staging array

// internal real of the real part of canonical complex kk (spin*3 + colour);
// the imaginary part is the internal real P::IM further on.  Spin-pair quads
// (Re j0, Re j1, Im j0, Im j1); interleaved-complex quads (CPLX, the layout
// ablation) (Re j0, Im j0, Re j1, Im j1).
template <class P>
__device__ __forceinline__ int internal_re(int kk) {
  const int spin = kk / 3, c = kk % 3;
  return (spin >> 1) * 12 + c * 4 + (spin & 1) * (P::CPLX ? 2 : 1);
}
template <class P>
__host__ __device__ constexpr int im_offset() {
  return P::CPLX ? 1 : 2;
}

template <class P>
__global__ void __launch_bounds__(kXposeTPB) pack_kernel(typename P::vec *dst,
                                                         const double2 *src, int V4, int Ls,
                                                         long long rhs_stride, long long V5) {
  constexpr int NP = 24 / P::R;
  __shared__ double sm[32 * kLaneStride];
  const int nch = (Ls + kSC - 1) / kSC;
  const int blk = (int)(blockIdx.x / nch);
  const int s0 = (int)(blockIdx.x % nch) * kSC;
  const int sc = min(kSC, Ls - s0);
  const int rhs = blockIdx.y;
  // canonical -> staging: consecutive threads read consecutive complex128
  const int nin = 32 * sc * 12;
  for (int o = threadIdx.x; o < nin; o += kXposeTPB) {
    const int lane = o / (sc * 12), rem = o % (sc * 12), sl = rem / 12, kk = rem % 12;
    const int x4 = blk * 32 + lane;
    if (x4 >= V4) continue;
    const double2 v = __ldcs(src + ((long long)rhs * V5 + (long long)x4 * Ls + s0 + sl) * 12 + kk);
    double *b = sm + lane * kLaneStride + sl * 24 + internal_re<P>(kk);
    b[0] = v.x;
    b[im_offset<P>()] = v.y;
  }
  __syncthreads();
  // staging -> internal: the chunk is one contiguous run of sc * NP * 32 vecs
  typename P::vec *dp = dst + rhs * rhs_stride + ((long long)blk * Ls + s0) * NP * 32;
  for (int v = threadIdx.x; v < sc * NP * 32; v += kXposeTPB) {
    const int lane = v & 31, q = (v >> 5) % NP, sl = (v >> 5) / NP;
    if (blk * 32 + lane >= V4) continue;  // padding lanes are never written
    double r[P::R];
#pragma unroll
    for (int w = 0; w < P::R; ++w) r[w] = sm[lane * kLaneStride + sl * 24 + q * P::R + w];
    dp[v] = narrow_from_f64(r, (typename P::vec *)nullptr);
  }
}

template <class P>
__global__ void __launch_bounds__(kXposeTPB) unpack_kernel(double2 *dst,
                                                           const typename P::vec *src, int V4,
                                                           int Ls, long long rhs_stride,
                                                           long long V5) {
  using C = typename P::C;
  constexpr int NP = 24 / P::R;
  __shared__ double sm[32 * kLaneStride];
  const int nch = (Ls + kSC - 1) / kSC;
  const int blk = (int)(blockIdx.x / nch);
  const int s0 = (int)(blockIdx.x % nch) * kSC;
  const int sc = min(kSC, Ls - s0);
  const int rhs = blockIdx.y;
  // internal -> staging
  const typename P::vec *sp = src + rhs * rhs_stride + ((long long)blk * Ls + s0) * NP * 32;
  for (int v = threadIdx.x; v < sc * NP * 32; v += kXposeTPB) {
    const int lane = v & 31, q = (v >> 5) % NP, sl = (v >> 5) / NP;
    if (blk * 32 + lane >= V4) continue;
    C r[P::R];
    load_vec<P>(r, sp + v);
#pragma unroll
    for (int w = 0; w < P::R; ++w) sm[lane * kLaneStride + sl * 24 + q * P::R + w] = (double)r[w];
  }
  __syncthreads();
  // staging -> canonical: consecutive threads write consecutive complex128
  const int nout = 32 * sc * 12;
  for (int o = threadIdx.x; o < nout; o += kXposeTPB) {
    const int lane = o / (sc * 12), rem = o % (sc * 12), sl = rem / 12, kk = rem % 12;
    const int x4 = blk * 32 + lane;
    if (x4 >= V4) continue;
    const double *b = sm + lane * kLaneStride + sl * 24 + internal_re<P>(kk);
    __stcs(dst + ((long long)rhs * V5 + (long long)x4 * Ls + s0 + sl) * 12 + kk,
           make_double2(b[0], b[im_offset<P>()]));
  }
}

template <class P>
static int pack_t(const FieldGeom &g, void *dst, const void *src, int nrhs, cudaStream_t st) {
  const long long nch = (g.Ls + kSC - 1) / kSC;
  dim3 grid((unsigned)(padded_v4(g.V4) / 32 * nch), nrhs);
  pack_kernel<P><<<grid, kXposeTPB, 0, st>>>((typename P::vec *)dst, (const double2 *)src, g.V4,
                                             g.Ls, padded_v4(g.V4) * g.Ls * (24 / P::R), g.V5());
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <class P>
static int unpack_t(const FieldGeom &g, void *dst, const void *src, int nrhs, cudaStream_t st) {
  const long long nch = (g.Ls + kSC - 1) / kSC;
  dim3 grid((unsigned)(padded_v4(g.V4) / 32 * nch), nrhs);
  unpack_kernel<P><<<grid, kXposeTPB, 0, st>>>((double2 *)dst, (const typename P::vec *)src,
                                               g.V4, g.Ls,
                                               padded_v4(g.V4) * g.Ls * (24 / P::R), g.V5());
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int pack_fermion(const FieldGeom &g, int prec, void *dst, const void *src, int nrhs,
                 cudaStream_t st, bool cplx) {
  if (cplx && prec == DW_F32) return pack_t<F32C>(g, dst, src, nrhs, st);
  switch (prec) {
    case DW_F64: return pack_t<F64>(g, dst, src, nrhs, st);
    case DW_F32: return pack_t<F32>(g, dst, src, nrhs, st);
    case DW_F16: return pack_t<F16>(g, dst, src, nrhs, st);
  }
  return -2;
}

int unpack_fermion(const FieldGeom &g, int prec, void *dst, const void *src, int nrhs,
                   cudaStream_t st, bool cplx) {
  if (cplx && prec == DW_F32) return unpack_t<F32C>(g, dst, src, nrhs, st);
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

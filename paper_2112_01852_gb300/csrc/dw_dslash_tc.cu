// FP16 hopping term with the link x half-spinor products on the tensor cores
// (stencil variant 8, FP16 storage, Dhop and Dhop^+).
//
// Per hop direction and 4D site the Domain Wall kernel multiplies one SU(3)
// matrix W (U, or U^+ for a backward hop) into the projected half spinors of
// every slice, spin and right-hand side (Sec. 4.1, Table 3: "SU(3) x half
// spinor").  In real form that is a 6 x 6 matrix times a 6 x (2 Ls nrhs) block.
// Here one warp takes a pair of sites and issues, per direction, one
// mma.sync.m16n8k16 (FP16 in, FP32 accumulate) per 8 columns:
//
//   A (16 x 16): the two sites' W block-diagonally.  Row g (0..2: site 0,
//     colour g; 3..5: site 1, colour g-3) is Re w, row g + 8 is Im w; columns
//     0..2 / 8..10 are Re / Im h of site 0, 3..5 / 11..13 those of site 1.
//     Rows 6, 7, 14, 15 and columns 6, 7, 14, 15 are zero.
//   B (16 x 8): column n is spin n % 2 of slice 4 m + n / 2 (m the column tile)
//     of the projected half spinors h = u + S e_mu l of the two sites'
//     neighbours (the chiral-basis projection of the spin-pair kernels).
//   D (16 x 8, FP32): w = W h; each thread ends up holding Re and Im of one
//     (site, colour) for both spins of one slice, so the reconstruction
//     (w, S e_mu^+ w) and the sum over directions stay in the thread.
//
// The eight A fragments of a site pair are built once and reused for every
// right-hand side.  A and B waste 7/16 of their rows and columns on padding;
// the tensor-pipe and issue counters of this kernel against the register
// kernels are the measurement of whether the contraction pays.
#include "dw_dslash.cuh"

namespace dw {
namespace {

__device__ __forceinline__ unsigned pack_h2(float lo, float hi) {
  __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<unsigned *>(&h);
}

__device__ __forceinline__ void mma_16816(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                          unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%10, %11, %12, %13};\n"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(0.f), "f"(0.f),
        "f"(0.f), "f"(0.f));
}

// k index of the B / A columns -> (site, colour, imaginary part); -1 for padding
__device__ __forceinline__ int k_site(int k) {
  const int kk = k & 7;
  return kk < 3 ? 0 : (kk < 6 ? 1 : -1);
}
__device__ __forceinline__ int k_colour(int k) {
  const int kk = k & 7;
  return kk < 3 ? kk : kk - 3;
}

// One complex component (Re, Im) of spin j, colour c of a half (0: upper,
// 1: lower) of the FP16 spinor at (x4, s).
__device__ __forceinline__ float2 spinor_comp(const uint2 *base, int x4, int s, int Ls, int half,
                                              int c, int j) {
  const uint2 v = __ldg(base + site_off(x4, s, Ls, 6) + (long long)(half * 3 + c) * kPlaneStride);
  const float2 re = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
  const float2 im = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
  return j ? make_float2(re.y, im.y) : make_float2(re.x, im.x);
}

// (h)_j = u_j + S (e_mu l)_j for one colour (chiral basis, as in project())
template <int MU, int S>
__device__ __forceinline__ float2 project_comp(const uint2 *base, int x4, int s, int Ls, int c,
                                               int j) {
  const float2 u = spinor_comp(base, x4, s, Ls, 0, c, j);
  if (MU == 0) {  // e l = (i l1, i l0)
    const float2 l = spinor_comp(base, x4, s, Ls, 1, c, 1 - j);
    return make_float2(u.x - S * l.y, u.y + S * l.x);
  } else if (MU == 1) {  // e l = (l1, -l0)
    const float2 l = spinor_comp(base, x4, s, Ls, 1, c, 1 - j);
    const float f = j ? -S : S;
    return make_float2(u.x + f * l.x, u.y + f * l.y);
  } else if (MU == 2) {  // e l = (i l0, -i l1)
    const float2 l = spinor_comp(base, x4, s, Ls, 1, c, j);
    const float f = j ? -S : S;
    return make_float2(u.x - f * l.y, u.y + f * l.x);
  } else {  // e l = l
    const float2 l = spinor_comp(base, x4, s, Ls, 1, c, j);
    return make_float2(u.x + S * l.x, u.y + S * l.y);
  }
}

// acc (4 complex: up j0, up j1, lo j0, lo j1) += (w, S e_mu^+ w)
template <int MU, int S>
__device__ __forceinline__ void reconstruct_comp(float2 (&acc)[4], float2 w0, float2 w1) {
  acc[0].x += w0.x;
  acc[0].y += w0.y;
  acc[1].x += w1.x;
  acc[1].y += w1.y;
  float2 l0, l1;
  if (MU == 0) {  // e^+ w = (-i w1, -i w0)
    l0 = make_float2(w1.y, -w1.x);
    l1 = make_float2(w0.y, -w0.x);
  } else if (MU == 1) {  // e^+ w = (-w1, w0)
    l0 = make_float2(-w1.x, -w1.y);
    l1 = w0;
  } else if (MU == 2) {  // e^+ w = (-i w0, i w1)
    l0 = make_float2(w0.y, -w0.x);
    l1 = make_float2(-w1.y, w1.x);
  } else {  // e^+ w = w
    l0 = w0;
    l1 = w1;
  }
  acc[2].x += S * l0.x;
  acc[2].y += S * l0.y;
  acc[3].x += S * l1.x;
  acc[3].y += S * l1.y;
}

// The A fragment of direction (MU, ADJ) for the site pair: this thread's rows g
// (Re) and g + 8 (Im) hold row r = g % 3 of W of site g / 3 (g < 6).
template <int MU, bool FWD, bool ADJ>
__device__ __forceinline__ void build_a(unsigned (&a)[4], const DslashParams &p, const Hops &H0,
                                        const Hops &H1, const uint2 *gauge, int g, int q) {
  float W[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // (Re, Im) of W[r][c], c = 0..2
  const int site = g / 3, r = g % 3;
  if (g < 6) {
    const Hops &H = site ? H1 : H0;
    const int l4 = FWD ? H.x4 : H.template nb<MU, false>(p);
    float U[18];
    load_link<F16>(U, gauge, MU, l4, (float)H.template sign<MU, FWD>(p));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int idx = ADJ ? (c * 3 + r) : (r * 3 + c);
      W[2 * c] = U[idx * 2];
      W[2 * c + 1] = ADJ ? -U[idx * 2 + 1] : U[idx * 2 + 1];
    }
  }
  float e[8];  // A[g][k], A[g+8][k] for k = 2q, 2q+1, 2q+8, 2q+9
  const int ks[4] = {2 * q, 2 * q + 1, 2 * q + 8, 2 * q + 9};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = ks[i];
    const bool mine = g < 6 && k_site(k) == site;
    const int c = k_colour(k);
    const bool im_in = k >= 8;
    const float wr = mine ? W[2 * c] : 0.f, wi = mine ? W[2 * c + 1] : 0.f;
    e[2 * i] = im_in ? -wi : wr;     // row g: Re w = Wr Re h - Wi Im h
    e[2 * i + 1] = im_in ? wr : wi;  // row g + 8: Im w = Wi Re h + Wr Im h
  }
  a[0] = pack_h2(e[0], e[2]);  // row g, k = 2q, 2q+1
  a[1] = pack_h2(e[1], e[3]);  // row g + 8
  a[2] = pack_h2(e[4], e[6]);  // row g, k = 2q+8, 2q+9
  a[3] = pack_h2(e[5], e[7]);  // row g + 8
}

// One direction for one right-hand side: all MT = Ls / 4 column tiles.
template <int MU, int S, int MT>
__device__ __forceinline__ void hop_tc(float2 (&acc)[MT][4], const unsigned (&a)[4],
                                       const uint2 *in, int y0, int y1, int Ls, int g, int q) {
  const int n = g;  // this thread's B column
  const int j = n & 1;
  const int kq[4] = {2 * q, 2 * q + 1, 2 * q + 8, 2 * q + 9};
#pragma unroll
  for (int m = 0; m < MT; ++m) {
    const int sb = 4 * m + (n >> 1);  // slice of column n
    float bv[4];
#pragma unroll
    for (int i = 0; i < 2; ++i) {  // k = 2q + i (Re) and 2q + 8 + i (Im): one complex each
      const int k = kq[i];
      const int st = k_site(k);
      float2 h = make_float2(0.f, 0.f);
      if (st >= 0) h = project_comp<MU, S>(in, st ? y1 : y0, sb, Ls, k_colour(k), j);
      bv[i] = h.x;
      bv[2 + i] = h.y;
    }
    float d[4];
    mma_16816(d, a, pack_h2(bv[0], bv[1]), pack_h2(bv[2], bv[3]));
    // d0, d1: Re w of (site, colour) g, spins 0 and 1 of slice 4m + q; d2, d3: Im
    if (g < 6) reconstruct_comp<MU, S>(acc[m], make_float2(d[0], d[2]), make_float2(d[1], d[3]));
  }
}

// MT = Ls / 4 column tiles of 8 (2 spins x 4 slices) per right-hand side.
template <bool DAG, int MT>
__global__ void __launch_bounds__(128) dslash_tc_kernel(const DslashParams p) {
  constexpr int SF = DAG ? 1 : -1;  // sign S of the forward hop
  constexpr int SB = -SF;
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, q = lane & 3;
  const int Ls = p.Ls;
  const int npairs = p.V4 / 2;
  const int Vt = p.L[0] * p.L[1] * p.L[2];  // sites per time slice (output restricted to
  const int t_end = p.t_begin + p.t_count;  // t_begin .. t_end - 1 when t_count > 0)
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const uint2 *gauge = reinterpret_cast<const uint2 *>(p.gauge);
  for (int pair = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; pair < npairs; pair += warps) {
    const int x0 = 2 * pair;  // Lx even: x0 and x0 + 1 share y, z and t
    if (p.t_count > 0 && (x0 / Vt < p.t_begin || x0 / Vt >= t_end)) continue;
    const Hops H0(p, x0), H1(p, x0 + 1);
    unsigned a[8][4];
    build_a<3, true, false>(a[0], p, H0, H1, gauge, g, q);
    build_a<3, false, true>(a[1], p, H0, H1, gauge, g, q);
    build_a<2, true, false>(a[2], p, H0, H1, gauge, g, q);
    build_a<2, false, true>(a[3], p, H0, H1, gauge, g, q);
    build_a<1, true, false>(a[4], p, H0, H1, gauge, g, q);
    build_a<1, false, true>(a[5], p, H0, H1, gauge, g, q);
    build_a<0, true, false>(a[6], p, H0, H1, gauge, g, q);
    build_a<0, false, true>(a[7], p, H0, H1, gauge, g, q);
    for (int rhs = 0; rhs < p.nrhs; ++rhs) {
      const uint2 *in = reinterpret_cast<const uint2 *>(p.in) + (long long)rhs * p.rhs_stride;
      uint2 *out = reinterpret_cast<uint2 *>(p.out) + (long long)rhs * p.rhs_stride;
      float2 acc[MT][4];
#pragma unroll
      for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[m][i] = make_float2(0.f, 0.f);
      hop_tc<3, SF>(acc, a[0], in, H0.nb<3, true>(p), H1.nb<3, true>(p), Ls, g, q);
      hop_tc<3, SB>(acc, a[1], in, H0.nb<3, false>(p), H1.nb<3, false>(p), Ls, g, q);
      hop_tc<2, SF>(acc, a[2], in, H0.nb<2, true>(p), H1.nb<2, true>(p), Ls, g, q);
      hop_tc<2, SB>(acc, a[3], in, H0.nb<2, false>(p), H1.nb<2, false>(p), Ls, g, q);
      hop_tc<1, SF>(acc, a[4], in, H0.nb<1, true>(p), H1.nb<1, true>(p), Ls, g, q);
      hop_tc<1, SB>(acc, a[5], in, H0.nb<1, false>(p), H1.nb<1, false>(p), Ls, g, q);
      hop_tc<0, SF>(acc, a[6], in, H0.nb<0, true>(p), H1.nb<0, true>(p), Ls, g, q);
      hop_tc<0, SB>(acc, a[7], in, H0.nb<0, false>(p), H1.nb<0, false>(p), Ls, g, q);
      if (g < 6) {
        const int x4 = x0 + g / 3, c = g % 3;
#pragma unroll
        for (int m = 0; m < MT; ++m) {
          const int s = 4 * m + q;
          uint2 *o = out + site_off(x4, s, Ls, 6);
          uint2 up, lo;  // quads (Re j0, Re j1, Im j0, Im j1)
          up.x = pack_h2(acc[m][0].x, acc[m][1].x);
          up.y = pack_h2(acc[m][0].y, acc[m][1].y);
          lo.x = pack_h2(acc[m][2].x, acc[m][3].x);
          lo.y = pack_h2(acc[m][2].y, acc[m][3].y);
          __stcs(o + (long long)c * kPlaneStride, up);
          __stcs(o + (long long)(3 + c) * kPlaneStride, lo);
        }
      }
    }
  }
}

}  // namespace

template <bool DAG>
static int launch_tc(const DslashParams &p, unsigned blocks, cudaStream_t st) {
  switch (p.Ls / 4) {
    case 1: dslash_tc_kernel<DAG, 1><<<blocks, 128, 0, st>>>(p); break;
    case 2: dslash_tc_kernel<DAG, 2><<<blocks, 128, 0, st>>>(p); break;
    case 3: dslash_tc_kernel<DAG, 3><<<blocks, 128, 0, st>>>(p); break;
    case 4: dslash_tc_kernel<DAG, 4><<<blocks, 128, 0, st>>>(p); break;
    default: return -2;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_dslash_tc_F16(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st) {
  (void)cfg;
  if (!tc_variant_ok(op, p.L[0], p.Ls) || p.halo_up || p.halo_dn) return -2;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long pairs = p.V4 / 2;
  long long blocks = (pairs + 3) / 4;  // 4 warps per CTA, one pair per warp
  if (blocks > (long long)sms * 16) blocks = (long long)sms * 16;
  if (p.t_count < 0 || p.t_begin < 0 || p.t_begin + p.t_count > p.L[3]) return -2;
  return op == OP_DHOP ? launch_tc<false>(p, (unsigned)blocks, st)
                       : launch_tc<true>(p, (unsigned)blocks, st);
}

}  // namespace dw

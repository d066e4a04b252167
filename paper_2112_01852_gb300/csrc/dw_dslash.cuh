// The Domain Wall kernel: 4D Wilson hopping term over all fifth-dimension
// slices (Sec. 4.1; per-site spin projection, SU(3) x half spinor and
// reconstruction, Table 3), fused with the 5D hop and diagonal terms of the
// Shamir / Moebius operator.
//
// Work decomposition.  A CTA owns `tx` consecutive 4D sites and all Ls slices
// of one right-hand side (CTAs are numbered RHS-fastest); thread (x, y)
// handles one 4D site and the `SPT` consecutive slices s0 = y*SPT ..
// s0+SPT-1.
// Each link is loaded once per thread and reused across its SPT slices; the
// Ls/SPT threads of one site read the same link words, so it leaves HBM once.
// Fermion planes are [p][s][x4], so a warp (32 consecutive x4 at one s)
// issues fully coalesced 16-byte loads and stores.
//
// Chiral basis, g_mu = [[0, e_mu], [e_mu^+, 0]] with e_x = i s_1, e_y = i s_2,
// e_z = i s_3, e_t = 1.  For (1 + S g_mu) psi with psi = (u, l):
//   h = u + S e_mu l      (2 spins x 3 colours),
//   (1 + S g_mu) psi = (h, S e_mu^+ h).
// Dhop uses S = -1 forward and S = +1 backward; Dhop^+ the opposite.
#pragma once

#include <cooperative_groups.h>
#include <type_traits>

#include "dw_common.cuh"

namespace dw {

// ---------------------------------------------------------------------------
// Register form of a spinor.  A half spinor (2 spins x 3 colours) is held as
// spin pairs: re[c] = (Re psi_{j=0,c}, Re psi_{j=1,c}), im[c] likewise.  For
// FP32 arithmetic a pair is a float2 and the arithmetic below compiles to the
// packed f32x2 instructions (two lanes per instruction); for FP64 it is a
// double2 worked lane by lane.  This is also the memory order of a quad
// (4 reals) of the internal layout, so loads land in registers unshuffled.
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 p_add(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 p_mul(double2 a, double2 b) {
  return make_double2(a.x * b.x, a.y * b.y);
}
__device__ __forceinline__ double2 p_fma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
template <class V2, class C>
__device__ __forceinline__ V2 bc(C v) {
  V2 r;
  r.x = v;
  r.y = v;
  return r;
}
template <class V2, class C>
__device__ __forceinline__ V2 pr(C x, C y) {
  V2 r;
  r.x = x;
  r.y = y;
  return r;
}

// CX = false: the spin-pair form above.  CX = true: the interleaved-complex
// form of the layout ablation, z[c][j] = (Re, Im) of spin j, colour c.
template <class V2, bool CX = false>
struct Half {
  V2 re[3];
  V2 im[3];
};
template <class V2>
struct Half<V2, true> {
  V2 z[3][2];
};
template <class V2, bool CX = false>
struct Spinor {
  Half<V2, CX> up;  // spins 0, 1 (P+)
  Half<V2, CX> lo;  // spins 2, 3 (P-)
};

template <class P>
struct Pair {
  using type = typename std::conditional<std::is_same<typename P::C, double>::value, double2,
                                         float2>::type;
};
template <class P>
using HalfP = Half<typename Pair<P>::type, P::CPLX>;
template <class P>
using SpinorP = Spinor<typename Pair<P>::type, P::CPLX>;

// h = u + S e_mu l   (the half spinor of (1 + S g_mu) psi)
template <int MU, int S, class V2>
__device__ __forceinline__ void project(Half<V2> &h, const Half<V2> &u, const Half<V2> &l) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (MU == 0) {  // e l = (i l1, i l0)
      h.re[c].x = u.re[c].x - S * l.im[c].y;
      h.im[c].x = u.im[c].x + S * l.re[c].y;
      h.re[c].y = u.re[c].y - S * l.im[c].x;
      h.im[c].y = u.im[c].y + S * l.re[c].x;
    } else if (MU == 1) {  // e l = (l1, -l0)
      h.re[c].x = u.re[c].x + S * l.re[c].y;
      h.im[c].x = u.im[c].x + S * l.im[c].y;
      h.re[c].y = u.re[c].y - S * l.re[c].x;
      h.im[c].y = u.im[c].y - S * l.im[c].x;
    } else if (MU == 2) {  // e l = (i l0, -i l1): lanes stay in place
      h.re[c] = p_fma(pr<V2>(-S, S), l.im[c], u.re[c]);
      h.im[c] = p_fma(pr<V2>(S, -S), l.re[c], u.im[c]);
    } else {  // e l = l
      h.re[c] = p_fma(bc<V2>(S), l.re[c], u.re[c]);
      h.im[c] = p_fma(bc<V2>(S), l.im[c], u.im[c]);
    }
  }
}

// acc += (w, S e_mu^+ w)   (FIRST: acc = ...)
template <int MU, int S, bool FIRST, class V2>
__device__ __forceinline__ void reconstruct(Spinor<V2> &acc, const Half<V2> &w) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (FIRST) {
      acc.up.re[c] = w.re[c];
      acc.up.im[c] = w.im[c];
    } else {
      acc.up.re[c] = p_add(acc.up.re[c], w.re[c]);
      acc.up.im[c] = p_add(acc.up.im[c], w.im[c]);
    }
    V2 dre, dim;  // lower-spin increment S e^+ w
    bool packed = false;
    if (MU == 0) {  // e^+ w = (-i w1, -i w0)
      dre = pr<V2>(S * w.im[c].y, S * w.im[c].x);
      dim = pr<V2>(-S * w.re[c].y, -S * w.re[c].x);
    } else if (MU == 1) {  // e^+ w = (-w1, w0)
      dre = pr<V2>(-S * w.re[c].y, S * w.re[c].x);
      dim = pr<V2>(-S * w.im[c].y, S * w.im[c].x);
    } else {
      packed = true;
    }
    if (!packed) {
      if (FIRST) {
        acc.lo.re[c] = dre;
        acc.lo.im[c] = dim;
      } else {
        acc.lo.re[c].x += dre.x;
        acc.lo.re[c].y += dre.y;
        acc.lo.im[c].x += dim.x;
        acc.lo.im[c].y += dim.y;
      }
    } else if (MU == 2) {  // e^+ w = (-i w0, i w1)
      if (FIRST) {
        acc.lo.re[c] = p_mul(pr<V2>(S, -S), w.im[c]);
        acc.lo.im[c] = p_mul(pr<V2>(-S, S), w.re[c]);
      } else {
        acc.lo.re[c] = p_fma(pr<V2>(S, -S), w.im[c], acc.lo.re[c]);
        acc.lo.im[c] = p_fma(pr<V2>(-S, S), w.re[c], acc.lo.im[c]);
      }
    } else {  // e^+ w = w
      if (FIRST) {
        acc.lo.re[c] = p_mul(bc<V2>(S), w.re[c]);
        acc.lo.im[c] = p_mul(bc<V2>(S), w.im[c]);
      } else {
        acc.lo.re[c] = p_fma(bc<V2>(S), w.re[c], acc.lo.re[c]);
        acc.lo.im[c] = p_fma(bc<V2>(S), w.im[c], acc.lo.im[c]);
      }
    }
  }
}

// w = U h (ADJ = false) or U^+ h (ADJ = true), both spins at once.  U holds
// 18 reals, element (row, col) at (row * 3 + col) * 2 + re/im.
template <bool ADJ, class V2, class C>
__device__ __forceinline__ void su3_mul(Half<V2> &w, const C *U, const Half<V2> &h) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    V2 wr, wi;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int idx = ADJ ? (k * 3 + r) : (r * 3 + k);
      const C ur = U[idx * 2];
      const C ui = ADJ ? -U[idx * 2 + 1] : U[idx * 2 + 1];
      // (ur + i ui)(hre + i him): re = ur hre - ui him, im = ur him + ui hre
      if (k == 0) {
        wr = p_mul(bc<V2>(ur), h.re[k]);
        wi = p_mul(bc<V2>(ur), h.im[k]);
      } else {
        wr = p_fma(bc<V2>(ur), h.re[k], wr);
        wi = p_fma(bc<V2>(ur), h.im[k], wi);
      }
      wr = p_fma(bc<V2>(-ui), h.im[k], wr);
      wi = p_fma(bc<V2>(ui), h.re[k], wi);
    }
    w.re[r] = wr;
    w.im[r] = wi;
  }
}

// ---------------------------------------------------------------------------
// Interleaved-complex form (layout ablation, the counterpart of the paper's
// RIRI layout; the forms above are its RRII counterpart).  A register pair is
// one complex number (Re, Im); multiplying by +-i swaps the pair's halves, and
// a complex product takes two packed FMAs on the pair and on its swapped copy.
template <class V2>
__device__ __forceinline__ V2 swz(V2 a) {
  return pr<V2>(a.y, a.x);
}

// h = u + S e_mu l   (see project above)
template <int MU, int S, class V2>
__device__ __forceinline__ void project(Half<V2, true> &h, const Half<V2, true> &u,
                                        const Half<V2, true> &l) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (MU == 0) {  // e l = (i l1, i l0)
      h.z[c][0] = p_fma(pr<V2>(-S, S), swz(l.z[c][1]), u.z[c][0]);
      h.z[c][1] = p_fma(pr<V2>(-S, S), swz(l.z[c][0]), u.z[c][1]);
    } else if (MU == 1) {  // e l = (l1, -l0)
      h.z[c][0] = p_fma(bc<V2>(S), l.z[c][1], u.z[c][0]);
      h.z[c][1] = p_fma(bc<V2>(-S), l.z[c][0], u.z[c][1]);
    } else if (MU == 2) {  // e l = (i l0, -i l1)
      h.z[c][0] = p_fma(pr<V2>(-S, S), swz(l.z[c][0]), u.z[c][0]);
      h.z[c][1] = p_fma(pr<V2>(S, -S), swz(l.z[c][1]), u.z[c][1]);
    } else {  // e l = l
      h.z[c][0] = p_fma(bc<V2>(S), l.z[c][0], u.z[c][0]);
      h.z[c][1] = p_fma(bc<V2>(S), l.z[c][1], u.z[c][1]);
    }
  }
}

// acc += (w, S e_mu^+ w)   (FIRST: acc = ...)
template <int MU, int S, bool FIRST, class V2>
__device__ __forceinline__ void reconstruct(Spinor<V2, true> &acc, const Half<V2, true> &w) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int j = 0; j < 2; ++j) acc.up.z[c][j] = FIRST ? w.z[c][j] : p_add(acc.up.z[c][j], w.z[c][j]);
    // lower-spin increment S e^+ w: the factor and the source of each spin
    V2 f0, f1, a0, a1;
    if (MU == 0) {  // e^+ w = (-i w1, -i w0)
      f0 = pr<V2>(S, -S); a0 = swz(w.z[c][1]);
      f1 = pr<V2>(S, -S); a1 = swz(w.z[c][0]);
    } else if (MU == 1) {  // e^+ w = (-w1, w0)
      f0 = bc<V2>(-S); a0 = w.z[c][1];
      f1 = bc<V2>(S); a1 = w.z[c][0];
    } else if (MU == 2) {  // e^+ w = (-i w0, i w1)
      f0 = pr<V2>(S, -S); a0 = swz(w.z[c][0]);
      f1 = pr<V2>(-S, S); a1 = swz(w.z[c][1]);
    } else {  // e^+ w = w
      f0 = bc<V2>(S); a0 = w.z[c][0];
      f1 = bc<V2>(S); a1 = w.z[c][1];
    }
    if (FIRST) {
      acc.lo.z[c][0] = p_mul(f0, a0);
      acc.lo.z[c][1] = p_mul(f1, a1);
    } else {
      acc.lo.z[c][0] = p_fma(f0, a0, acc.lo.z[c][0]);
      acc.lo.z[c][1] = p_fma(f1, a1, acc.lo.z[c][1]);
    }
  }
}

// w = U h (ADJ = false) or U^+ h (ADJ = true), both spins; (ur + i ui) z is
// ur (Re z, Im z) + (-ui, ui) (Im z, Re z).
template <bool ADJ, class V2, class C>
__device__ __forceinline__ void su3_mul(Half<V2, true> &w, const C *U, const Half<V2, true> &h) {
  V2 hs[3][2];  // the swapped copies, shared by the three rows
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    hs[k][0] = swz(h.z[k][0]);
    hs[k][1] = swz(h.z[k][1]);
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    V2 w0, w1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int idx = ADJ ? (k * 3 + r) : (r * 3 + k);
      const C ur = U[idx * 2];
      const C ui = ADJ ? -U[idx * 2 + 1] : U[idx * 2 + 1];
      const V2 vi = pr<V2>(-ui, ui);
      if (k == 0) {
        w0 = p_mul(bc<V2>(ur), h.z[k][0]);
        w1 = p_mul(bc<V2>(ur), h.z[k][1]);
      } else {
        w0 = p_fma(bc<V2>(ur), h.z[k][0], w0);
        w1 = p_fma(bc<V2>(ur), h.z[k][1], w1);
      }
      w0 = p_fma(vi, hs[k][0], w0);
      w1 = p_fma(vi, hs[k][1], w1);
    }
    w.z[r][0] = w0;
    w.z[r][1] = w1;
  }
}

// Memory <-> registers.  A quad (4 reals, one colour of one chirality half) is
// one vec for F32 / F16 and two vecs (planes 2q, 2q+1) for F64.
__device__ __forceinline__ void quad_in(float2 &re, float2 &im, const float4 *p, long long) {
  const float4 v = __ldg(p);
  re = make_float2(v.x, v.y);
  im = make_float2(v.z, v.w);
}
__device__ __forceinline__ void quad_in(float2 &re, float2 &im, const uint2 *p, long long) {
  const uint2 v = __ldg(p);
  re = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
  im = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
}
__device__ __forceinline__ void quad_in(double2 &re, double2 &im, const double2 *p,
                                        long long plane) {
  re = __ldg(p);
  im = __ldg(p + plane);
}
// Loads with an L2 eviction-priority hint.  In the t-inside-a-z-block
// traversal a spinor is first touched as a t+ neighbour and last touched as a
// t- neighbour: the first touch is kept (evict_last) for the reuses that follow
// one or two slabs later, the last touch may leave first (evict_first).
// HINT_SMEM marks a "field" that lives in shared memory (plain loads).
enum { HINT_NONE = 0, HINT_KEEP = 1, HINT_DROP = 2, HINT_SMEM = 3 };
template <int HINT>
__device__ __forceinline__ unsigned long long l2_policy() {
  unsigned long long pol = 0;
  if (HINT == HINT_KEEP)
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  else if (HINT == HINT_DROP)
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ float4 ldg_hint(const float4 *p, unsigned long long pol) {
  float4 v;
  asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint2 ldg_hint(const uint2 *p, unsigned long long pol) {
  uint2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
               : "=r"(v.x), "=r"(v.y)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double2 ldg_hint(const double2 *p, unsigned long long pol) {
  double2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
               : "=d"(v.x), "=d"(v.y)
               : "l"(p), "l"(pol));
  return v;
}
template <int HINT, class VEC>
__device__ __forceinline__ VEC ld_vec(const VEC *p, unsigned long long pol) {
  if (HINT == HINT_SMEM) return *p;
  if (HINT == HINT_NONE) return __ldg(p);
  return ldg_hint(p, pol);
}
template <int HINT>
__device__ __forceinline__ void quad_in_h(float2 &re, float2 &im, const float4 *p, long long,
                                          unsigned long long pol) {
  const float4 v = ld_vec<HINT>(p, pol);
  re = make_float2(v.x, v.y);
  im = make_float2(v.z, v.w);
}
template <int HINT>
__device__ __forceinline__ void quad_in_h(float2 &re, float2 &im, const uint2 *p, long long,
                                          unsigned long long pol) {
  const uint2 v = ld_vec<HINT>(p, pol);
  re = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
  im = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
}
template <int HINT>
__device__ __forceinline__ void quad_in_h(double2 &re, double2 &im, const double2 *p,
                                          long long plane, unsigned long long pol) {
  re = ld_vec<HINT>(p, pol);
  im = ld_vec<HINT>(p + plane, pol);
}

// Outputs are written once and not re-read by the kernel: streaming stores
// (evict-first) keep them from displacing neighbour spinors that are still to
// be reused from L2.
__device__ __forceinline__ void quad_out(float4 *p, long long, float2 re, float2 im) {
  __stcs(p, make_float4(re.x, re.y, im.x, im.y));
}
__device__ __forceinline__ void quad_out(uint2 *p, long long, float2 re, float2 im) {
  __half2 a = __float22half2_rn(re);
  __half2 b = __float22half2_rn(im);
  uint2 v;
  v.x = *reinterpret_cast<unsigned int *>(&a);
  v.y = *reinterpret_cast<unsigned int *>(&b);
  __stcs(p, v);
}
__device__ __forceinline__ void quad_out(double2 *p, long long plane, double2 re, double2 im) {
  __stcs(p, re);
  __stcs(p + plane, im);
}

template <class P>
struct Field {
  using vec = typename P::vec;
  using V2 = typename Pair<P>::type;
  static constexpr int VPQ = 4 / P::R;  // vecs (planes) per quad
  static constexpr int NPV = 24 / P::R;  // vec planes per site
  static constexpr long long plane = kPlaneStride;
  const vec *base;
  int V4;
  int Ls;
  __device__ __forceinline__ long long site(int s, int x4) const { return site_off(x4, s, Ls, NPV); }
  // half = 0: upper spins, 1: lower spins, at (x4, s)
  __device__ __forceinline__ void load_half(Half<V2> &h, int x4, int s, int half) const {
    const vec *p = base + site(s, x4) + (long long)half * 3 * VPQ * plane;
#pragma unroll
    for (int c = 0; c < 3; ++c) quad_in(h.re[c], h.im[c], p + (long long)c * VPQ * plane, plane);
  }
  template <int HINT>
  __device__ __forceinline__ void load_half_h(Half<V2> &h, int x4, int s, int half,
                                              unsigned long long pol) const {
    const vec *p = base + site(s, x4) + (long long)half * 3 * VPQ * plane;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      quad_in_h<HINT>(h.re[c], h.im[c], p + (long long)c * VPQ * plane, plane, pol);
  }
  // interleaved-complex quads (Re j0, Im j0, Re j1, Im j1): FP32 storage only
  template <int HINT>
  __device__ __forceinline__ void load_half_h(Half<V2, true> &h, int x4, int s, int half,
                                              unsigned long long pol) const {
    const vec *p = base + site(s, x4) + (long long)half * 3 * VPQ * plane;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float4 v = ld_vec<HINT>(p + (long long)c * plane, pol);
      h.z[c][0] = make_float2(v.x, v.y);
      h.z[c][1] = make_float2(v.z, v.w);
    }
  }
};

template <class P>
__device__ __forceinline__ void store_spinor(typename P::vec *base, long long plane,
                                             const SpinorP<P> &v) {
  constexpr int VPQ = 4 / P::R;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if constexpr (P::CPLX) {
      __stcs(base + (long long)c * plane,
             make_float4(v.up.z[c][0].x, v.up.z[c][0].y, v.up.z[c][1].x, v.up.z[c][1].y));
      __stcs(base + (long long)(3 + c) * plane,
             make_float4(v.lo.z[c][0].x, v.lo.z[c][0].y, v.lo.z[c][1].x, v.lo.z[c][1].y));
    } else {
      quad_out(base + (long long)c * VPQ * plane, plane, v.up.re[c], v.up.im[c]);
      quad_out(base + (long long)(3 + c) * VPQ * plane, plane, v.lo.re[c], v.lo.im[c]);
    }
  }
}

// Third row of an SU(3) link from the first two: row2 = sign * conj(row0 x row1).
// The stored rows carry the boundary sign of a link that crosses the lattice
// edge; the cross product cancels it, so `sign` puts it back.
template <class C>
__device__ __forceinline__ void rebuild_row2(C *U, C sign) {
  const C a0r = U[0], a0i = U[1], a1r = U[2], a1i = U[3], a2r = U[4], a2i = U[5];
  const C b0r = U[6], b0i = U[7], b1r = U[8], b1i = U[9], b2r = U[10], b2i = U[11];
  U[12] = sign * ((a1r * b2r - a1i * b2i) - (a2r * b1r - a2i * b1i));
  U[13] = -sign * ((a1r * b2i + a1i * b2r) - (a2r * b1i + a2i * b1r));
  U[14] = sign * ((a2r * b0r - a2i * b0i) - (a0r * b2r - a0i * b2i));
  U[15] = -sign * ((a2r * b0i + a2i * b0r) - (a0r * b2i + a0i * b2r));
  U[16] = sign * ((a0r * b1r - a0i * b1i) - (a1r * b0r - a1i * b0i));
  U[17] = -sign * ((a0r * b1i + a0i * b1r) - (a1r * b0i + a1i * b0r));
}

// U_mu(x4) into 18 reals (row, col, re/im); `sign` is the boundary sign of
// this link (used only to rebuild the third row of a 12-real link).
template <class P>
__device__ __forceinline__ void load_link(typename P::C *U, const typename P::vec *gauge, int mu,
                                          int x4, typename P::C sign) {
  const typename P::vec *p = gauge + link_off(x4, mu, P::NLV);
#pragma unroll
  for (int k = 0; k < P::NLV; ++k) widen(__ldg(p + k * 32), U + k * P::R);
  if (P::LINK12) rebuild_row2(U, sign);
}

template <class V2>
__device__ __forceinline__ void half_axpby(Half<V2> &o, V2 a, const Half<V2> &x, V2 b,
                                          const Half<V2> &y) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    o.re[c] = p_fma(a, x.re[c], p_mul(b, y.re[c]));
    o.im[c] = p_fma(a, x.im[c], p_mul(b, y.im[c]));
  }
}

// o = x + b y (the (b + cK) combination of D with b scaled out)
template <class V2>
__device__ __forceinline__ void half_axpy(Half<V2> &o, const Half<V2> &x, V2 b,
                                         const Half<V2> &y) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    o.re[c] = p_fma(b, y.re[c], x.re[c]);
    o.im[c] = p_fma(b, y.im[c], x.im[c]);
  }
}

// Rolling evaluation of A psi_s + B [K psi]_s (KDAG = false) or
// A psi_s + B [K^+ psi]_s (KDAG = true) at 4D site x4 for s = s0 .. s0+SPT-1.
//   K:   upper from s-1, lower from s+1;  K^+: upper from s+1, lower from s-1;
//   a neighbour index that leaves [0, Ls) wraps and carries -mf.
// Calls f(j, v) with the spinor of slice s0 + j.  Each half spinor is loaded
// once: 2 (SPT + 1) half-spinor loads for SPT slices.
// HINT: the L2 policy of the loads (HINT_KEEP / HINT_DROP as for the hopping
// term), or HINT_SMEM: F holds a staged copy of a slice range with both
// neighbours of the range, slice s at index s - s0 + so (no wrap there); the
// -mf factors still follow the global slice s and the global Ls.  UNIT: A = 1
// (A is not read), psi_s + B [K psi]_s with one FMA per element.
template <class P, bool KDAG, int SPT, int HINT = HINT_NONE, bool UNIT = false, class Fn>
__device__ __forceinline__ void roll_5d(const Field<P> &F, int x4, int s0, int Ls,
                                        typename P::C A, typename P::C B,
                                        typename P::C mf, Fn &&f, int so = 0) {
  using C = typename P::C;
  using V2 = typename Pair<P>::type;
  constexpr bool STG = (HINT == HINT_SMEM);
  const unsigned long long pol = l2_policy<HINT>();
  // K: the upper half comes from s-1 (carried), the lower from s+1 (loaded ahead);
  // K^+: the other way round.
  const int carry_half = KDAG ? 1 : 0;
  const int ahead_half = KDAG ? 0 : 1;
  // (shared memory takes plain loads: the read-only global path faults there)
  auto ld = [&](Half<V2> &h, int s, int half) {
    if constexpr (HINT == HINT_NONE)
      F.load_half(h, x4, s, half);
    else
      F.template load_half_h<HINT>(h, x4, s, half, pol);
  };
  Half<V2> prev, cur_ahead;
  C fp = 1;
  {
    int sp = s0 - 1;
    if (sp < 0) {
      sp = Ls - 1;
      fp = -mf;
    }
    ld(prev, STG ? so - 1 : sp, carry_half);
    ld(cur_ahead, STG ? so : s0, ahead_half);
  }
  const V2 vA = bc<V2>(A);
#pragma unroll
  for (int j = 0; j < SPT; ++j) {
    const int s = s0 + j;
    Half<V2> cur_carry, next_ahead;
    ld(cur_carry, STG ? so + j : s, carry_half);
    int sn = s + 1;
    C fn = 1;
    if (sn == Ls) {
      sn = 0;
      fn = -mf;
    }
    ld(next_ahead, STG ? so + j + 1 : sn, ahead_half);
    Spinor<V2> v;
    Half<V2> &vc = KDAG ? v.lo : v.up;
    Half<V2> &va = KDAG ? v.up : v.lo;
    if constexpr (UNIT) {
      half_axpy(vc, cur_carry, bc<V2>(B * (j == 0 ? fp : C(1))), prev);
      half_axpy(va, cur_ahead, bc<V2>(B * fn), next_ahead);
    } else {
      half_axpby(vc, vA, cur_carry, bc<V2>(B * (j == 0 ? fp : C(1))), prev);
      half_axpby(va, vA, cur_ahead, bc<V2>(B * fn), next_ahead);
    }
    f(j, v);
    prev = cur_carry;
    cur_ahead = next_ahead;
  }
}

// One hop direction: acc[j] += (1 + S g_mu) W psi'(y4, s0 + j) for every j,
// where W = U_mu(l4) (ADJ = false) or U_mu(l4)^+ (ADJ = true) and psi' is psi
// itself (PHI = false) or phi / b = psi + (c / b) K psi (PHI = true: the caller
// passes c / b as `c`, b is not read, and scales the hop sum by b).  With PHI and
// HINT_SMEM, F is a staged slice range (roll_5d's STG form; `so` the index of
// global slice s0 there).
template <class P, int MU, int S, bool ADJ, bool PHI, bool FIRST, int SPT, int HINT = HINT_NONE>
__device__ __forceinline__ void hop_dir(SpinorP<P> (&acc)[SPT],
                                        const Field<P> &F, const typename P::vec *gauge,
                                        typename P::C lsign, int y4, int l4, int s0, int Ls,
                                        typename P::C b, typename P::C c, typename P::C mf,
                                        int so = 0) {
  using C = typename P::C;
  C U[18];
  load_link<P>(U, gauge, MU, l4, lsign);
  auto body = [&](int j, const SpinorP<P> &v) {
    HalfP<P> h, w;
    project<MU, S>(h, v.up, v.lo);
    su3_mul<ADJ>(w, U, h);
    reconstruct<MU, S, FIRST>(acc[j], w);
  };
  if constexpr (PHI) {
    // (the L2 eviction hints of the hopping term made D slower: 2.06 -> 2.34 ms
    // at 32^3 x 64 x 12; its global loads keep the default policy)
    roll_5d<P, false, SPT, HINT == HINT_SMEM ? HINT_SMEM : HINT_NONE, true>(F, y4, s0, Ls, b, c,
                                                                          mf, body, so);
  } else {
    const unsigned long long pol = l2_policy<HINT>();
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
      SpinorP<P> v;
      F.template load_half_h<HINT>(v.up, y4, s0 + j, 0, pol);
      F.template load_half_h<HINT>(v.lo, y4, s0 + j, 1, pol);
      body(j, v);
    }
  }
}

// The D epilogue at output site xo, slices s0 .. s0+SPT-1:
//   out = alpha psi + beta K psi + h acc   (acc the hop sum of phi / b, h = b
//   times hscale, which is -1/2 for D_W),
// psi read from Fo at index io (STG: a staged slice range holding slice s0 at
// index so, roll_5d's STG form; own false: no local term).  Adds |out|^2 to
// nsq when `norm`.
template <class P, int SPT, bool STG>
__device__ __forceinline__ void d_epilogue(const SpinorP<P> (&acc)[SPT], typename P::vec *out,
                                           int xo, const Field<P> &Fo, bool own, int io, int so,
                                           int s0, int Ls, typename P::C alpha,
                                           typename P::C beta, typename P::C mf,
                                           typename Pair<P>::type h, bool norm, double &nsq) {
  using C = typename P::C;
  using V2 = typename Pair<P>::type;
  constexpr int NPV = 24 / P::R;
  auto emit = [&](int j, const Spinor<V2> &v) {
    Spinor<V2> o;
    C ss = 0;
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      o.up.re[cc] = p_fma(h, acc[j].up.re[cc], v.up.re[cc]);
      o.up.im[cc] = p_fma(h, acc[j].up.im[cc], v.up.im[cc]);
      o.lo.re[cc] = p_fma(h, acc[j].lo.re[cc], v.lo.re[cc]);
      o.lo.im[cc] = p_fma(h, acc[j].lo.im[cc], v.lo.im[cc]);
      if (norm) {
        ss += o.up.re[cc].x * o.up.re[cc].x + o.up.re[cc].y * o.up.re[cc].y;
        ss += o.up.im[cc].x * o.up.im[cc].x + o.up.im[cc].y * o.up.im[cc].y;
        ss += o.lo.re[cc].x * o.lo.re[cc].x + o.lo.re[cc].y * o.lo.re[cc].y;
        ss += o.lo.im[cc].x * o.lo.im[cc].x + o.lo.im[cc].y * o.lo.im[cc].y;
      }
    }
    nsq += (double)ss;
    store_spinor<P>(out + site_off(xo, s0 + j, Ls, NPV), kPlaneStride, o);
  };
  if (own) {
    roll_5d<P, false, SPT, STG ? HINT_SMEM : HINT_NONE>(Fo, io, s0, Ls, alpha, beta, mf, emit,
                                                        so);
  } else {
    Spinor<V2> zero_v;
#pragma unroll
    for (int cc = 0; cc < 3; ++cc)
      zero_v.up.re[cc] = zero_v.up.im[cc] = zero_v.lo.re[cc] = zero_v.lo.im[cc] = bc<V2>(C(0));
#pragma unroll
    for (int j = 0; j < SPT; ++j) emit(j, zero_v);
  }
}

// ---------------------------------------------------------------------------
// Staged variant of the hop phase.  Each thread copies the link and the
// neighbour spinors of the next direction into its own shared-memory slots
// with cp.async (16-byte LDGSTS; 8/4-byte for the link tail and FP16 quads)
// while it computes the current direction from the previous slot set, so the
// loads of a whole direction are in flight without holding registers.  Slots
// are [stage][slot][thread], so a warp's accesses to one slot are contiguous
// and free of bank conflicts.  Every thread reads only what it copied itself:
// cp.async.wait_group is the only synchronisation needed.
constexpr int kStages = 2;

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "n"(BYTES)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Bulk asynchronous copies (global -> shared, completion counted in bytes on
// an mbarrier) for the row-staged variant.  Every wait is bounded.
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// L2 prefetch of a contiguous global range (16-byte aligned, size a multiple of
// 16); a hint, nothing waits for it.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(src), "r"(bytes) : "memory");
}
// Wait for phase `parity` of the barrier; false after about a second or
// max_polls polls (default 2^24), whichever comes first.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity,
                                          int max_polls = 1 << 24) {
  const long long t0 = clock64();
  for (int i = 0; i < max_polls; ++i) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > 2000000000LL) return false;
  }
  return false;
}

template <class P, bool PHI, int SPT>
struct StageLayout {
  static constexpr int VPQ = 4 / P::R;
  static constexpr int NM = P::NLV;  // link vecs
  // spinor vec slots per direction: full spinors (Dhop) or the halves that the
  // rolling (b + cK) combination needs: upper s0-1 .. s0+SPT-1, lower s0 .. s0+SPT
  static constexpr int NSP = PHI ? 6 * (SPT + 1) * VPQ : 6 * SPT * VPQ;
  static constexpr int NVEC = NSP + NM;
  static __host__ __device__ size_t stage_bytes(int T) {
    size_t b = (size_t)NVEC * T * sizeof(typename P::vec);
    return (b + 15) & ~(size_t)15;
  }
};

template <class P, int OP, int SPT>
struct StagedHop {
  using C = typename P::C;
  using vec = typename P::vec;
  using V2 = typename Pair<P>::type;
  static constexpr bool PHI = (OP == OP_D);
  using L = StageLayout<P, PHI, SPT>;
  static constexpr int VPQ = L::VPQ;
  unsigned char *smem;  // kStages stages
  int T, t;             // threads per CTA, this thread's slot column
  __device__ __forceinline__ vec *vslot(int stage, int k) const {
    return reinterpret_cast<vec *>(smem + (size_t)stage * L::stage_bytes(T)) + (size_t)k * T + t;
  }
  __device__ __forceinline__ void issue(int stage, const Field<P> &F, const vec *gauge, int mu,
                                        int y4, int l4, int s0, int Ls) const {
    const vec *lp = gauge + link_off(l4, mu, P::NLV);
#pragma unroll
    for (int q = 0; q < L::NM; ++q) cp_async<sizeof(vec)>(vslot(stage, L::NSP + q), lp + q * 32);
    if (!PHI) {
#pragma unroll
      for (int j = 0; j < SPT; ++j) {
        const vec *sp = F.base + F.site(s0 + j, y4);
#pragma unroll
        for (int k = 0; k < 6 * VPQ; ++k)
          cp_async<sizeof(vec)>(vslot(stage, j * 6 * VPQ + k), sp + (long long)k * F.plane);
      }
    } else {
#pragma unroll
      for (int i = 0; i <= SPT; ++i) {
        int su = s0 - 1 + i;
        if (su < 0) su = Ls - 1;
        int sl = s0 + i;
        if (sl == Ls) sl = 0;
        const vec *pu = F.base + F.site(su, y4);
        const vec *pl = F.base + F.site(sl, y4) + (long long)3 * VPQ * F.plane;
#pragma unroll
        for (int k = 0; k < 3 * VPQ; ++k) {
          cp_async<sizeof(vec)>(vslot(stage, i * 3 * VPQ + k), pu + (long long)k * F.plane);
          cp_async<sizeof(vec)>(vslot(stage, (SPT + 1 + i) * 3 * VPQ + k),
                                pl + (long long)k * F.plane);
        }
      }
    }
  }
  __device__ __forceinline__ void read_half(Half<V2> &h, int stage, int k0) const {
#pragma unroll
    for (int c = 0; c < 3; ++c) read_quad(h.re[c], h.im[c], stage, k0 + c * VPQ);
  }
  __device__ __forceinline__ void read_quad(float2 &re, float2 &im, int stage, int k) const {
    if (sizeof(vec) == 16) {
      const float4 v = *reinterpret_cast<const float4 *>(vslot(stage, k));
      re = make_float2(v.x, v.y);
      im = make_float2(v.z, v.w);
    } else {
      const uint2 v = *reinterpret_cast<const uint2 *>(vslot(stage, k));
      re = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
      im = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
    }
  }
  __device__ __forceinline__ void read_quad(double2 &re, double2 &im, int stage, int k) const {
    re = *reinterpret_cast<const double2 *>(vslot(stage, k));
    im = *reinterpret_cast<const double2 *>(vslot(stage, k + 1));
  }
  __device__ __forceinline__ void read_link(C *U, int stage, C sign) const {
#pragma unroll
    for (int q = 0; q < L::NM; ++q) widen(*vslot(stage, L::NSP + q), U + q * P::R);
    if (P::LINK12) rebuild_row2(U, sign);
  }
};

// Hop phase with the staged loads: the 8 directions in the order t, z, y, x
// (forward then backward), kStages-deep cp.async pipeline.
template <class P, int OP, int SPT>
__device__ __forceinline__ void hop_staged(Spinor<typename Pair<P>::type> (&acc)[SPT],
                                           const StagedHop<P, OP, SPT> &H, const Field<P> &F,
                                           const typename P::vec *gauge, int x4, bool active,
                                           const int (&nb)[8], const int (&lsg)[8], int s0,
                                           int Ls,
                                           typename P::C b, typename P::C c, typename P::C mf) {
  using C = typename P::C;
  using V2 = typename Pair<P>::type;
  constexpr bool DAG = (OP == OP_DHOP_DAG || OP == OP_DDAG);
  constexpr bool PHI = (OP == OP_D);
  constexpr int SF = DAG ? 1 : -1;
  constexpr int SB = -SF;
  // direction d: mu = 3 - d/2; even d forward (link at x4), odd d backward
#pragma unroll
  for (int d = 0; d < kStages - 1; ++d) {
    if (active) H.issue(d % kStages, F, gauge, 3 - d / 2, nb[d], (d & 1) ? nb[d] : x4, s0, Ls);
    cp_async_commit();
  }
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    const int dn = d + kStages - 1;
    if (dn < 8 && active)
      H.issue(dn % kStages, F, gauge, 3 - dn / 2, nb[dn < 8 ? dn : 0],
              (dn & 1) ? nb[dn < 8 ? dn : 0] : x4, s0, Ls);
    cp_async_commit();
    cp_async_wait<kStages - 1>();
    if (!active) continue;
    const int stg = d % kStages;
    C U[18];
    H.read_link(U, stg, (C)lsg[d]);
    auto body = [&](int j, const Spinor<V2> &v) {
      Half<V2> h, w;
      switch (d) {
        case 0: project<3, SF>(h, v.up, v.lo); su3_mul<false>(w, U, h); reconstruct<3, SF, true>(acc[j], w); break;
        case 1: project<3, SB>(h, v.up, v.lo); su3_mul<true>(w, U, h); reconstruct<3, SB, false>(acc[j], w); break;
        case 2: project<2, SF>(h, v.up, v.lo); su3_mul<false>(w, U, h); reconstruct<2, SF, false>(acc[j], w); break;
        case 3: project<2, SB>(h, v.up, v.lo); su3_mul<true>(w, U, h); reconstruct<2, SB, false>(acc[j], w); break;
        case 4: project<1, SF>(h, v.up, v.lo); su3_mul<false>(w, U, h); reconstruct<1, SF, false>(acc[j], w); break;
        case 5: project<1, SB>(h, v.up, v.lo); su3_mul<true>(w, U, h); reconstruct<1, SB, false>(acc[j], w); break;
        case 6: project<0, SF>(h, v.up, v.lo); su3_mul<false>(w, U, h); reconstruct<0, SF, false>(acc[j], w); break;
        default: project<0, SB>(h, v.up, v.lo); su3_mul<true>(w, U, h); reconstruct<0, SB, false>(acc[j], w); break;
      }
    };
    if (!PHI) {
#pragma unroll
      for (int j = 0; j < SPT; ++j) {
        Spinor<V2> v;
        H.read_half(v.up, stg, j * 6 * H.VPQ);
        H.read_half(v.lo, stg, j * 6 * H.VPQ + 3 * H.VPQ);
        body(j, v);
      }
    } else {  // phi / b = psi + (c / b) K psi, as in hop_dir (`c` is c / b here)
#pragma unroll
      for (int j = 0; j < SPT; ++j) {
        Half<V2> up_prev, up_cur, lo_cur, lo_next;
        H.read_half(up_prev, stg, j * 3 * H.VPQ);
        H.read_half(up_cur, stg, (j + 1) * 3 * H.VPQ);
        H.read_half(lo_cur, stg, (SPT + 1 + j) * 3 * H.VPQ);
        H.read_half(lo_next, stg, (SPT + 2 + j) * 3 * H.VPQ);
        const C fp = (j == 0 && s0 == 0) ? -mf : C(1);
        const C fn = (s0 + j + 1 == Ls) ? -mf : C(1);
        Spinor<V2> v;
        half_axpy(v.up, up_cur, bc<V2>(c * fp), up_prev);
        half_axpy(v.lo, lo_cur, bc<V2>(c * fn), lo_next);
        body(j, v);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Register-prefetch variant of the hop phase (Dhop, Dhop^+ and the hop of D^+,
// which act on psi itself): the 8 x SPT (direction, slice) steps are walked in
// order and the spinor (and, at a new direction, the link) of step k+1 is
// loaded before step k is computed, so one step's loads are always in flight
// behind the arithmetic.  ORDER 0 visits t, z, y, x; ORDER 1 visits x, y, z, t.
template <class P, int SPT, int ORDER, bool DAG>
__device__ __forceinline__ void hop_prefetch(Spinor<typename Pair<P>::type> (&acc)[SPT],
                                             const Field<P> &F, const typename P::vec *gauge,
                                             int x4, const int (&nb)[8], const int (&lsg)[8],
                                             int s0) {
  using C = typename P::C;
  using V2 = typename Pair<P>::type;
  constexpr int SF = DAG ? 1 : -1;
  constexpr int SB = -SF;
  constexpr int N = 8 * SPT;
  auto mu_of = [](int d) { return ORDER == 0 ? 3 - d / 2 : d / 2; };
  auto nb_of = [&](int d) { return nb[(3 - mu_of(d)) * 2 + (d & 1)]; };
  auto sg_of = [&](int d) { return (C)lsg[(3 - mu_of(d)) * 2 + (d & 1)]; };
  Spinor<V2> nxt;
  C Unxt[18];
  F.load_half(nxt.up, nb_of(0), s0, 0);
  F.load_half(nxt.lo, nb_of(0), s0, 1);
  load_link<P>(Unxt, gauge, mu_of(0), x4, sg_of(0));
  C U[18];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int d = k / SPT, j = k % SPT;
    const Spinor<V2> cur = nxt;
    if (j == 0) {
#pragma unroll
      for (int i = 0; i < 18; ++i) U[i] = Unxt[i];
    }
    if (k + 1 < N) {
      const int d1 = (k + 1) / SPT, j1 = (k + 1) % SPT;
      F.load_half(nxt.up, nb_of(d1), s0 + j1, 0);
      F.load_half(nxt.lo, nb_of(d1), s0 + j1, 1);
      if (j1 == 0)
        load_link<P>(Unxt, gauge, mu_of(d1), (d1 & 1) ? nb_of(d1) : x4, sg_of(d1));
    }
    Half<V2> h, w;
    const int mu = mu_of(d);
    const bool fwd = !(d & 1);
    // compile-time dispatch (k is a constant after unrolling)
    if (mu == 3 && fwd) { project<3, SF>(h, cur.up, cur.lo); su3_mul<false>(w, U, h); }
    if (mu == 3 && !fwd) { project<3, SB>(h, cur.up, cur.lo); su3_mul<true>(w, U, h); }
    if (mu == 2 && fwd) { project<2, SF>(h, cur.up, cur.lo); su3_mul<false>(w, U, h); }
    if (mu == 2 && !fwd) { project<2, SB>(h, cur.up, cur.lo); su3_mul<true>(w, U, h); }
    if (mu == 1 && fwd) { project<1, SF>(h, cur.up, cur.lo); su3_mul<false>(w, U, h); }
    if (mu == 1 && !fwd) { project<1, SB>(h, cur.up, cur.lo); su3_mul<true>(w, U, h); }
    if (mu == 0 && fwd) { project<0, SF>(h, cur.up, cur.lo); su3_mul<false>(w, U, h); }
    if (mu == 0 && !fwd) { project<0, SB>(h, cur.up, cur.lo); su3_mul<true>(w, U, h); }
    if (d == 0) {
      if (mu == 3) reconstruct<3, SF, true>(acc[j], w);
      if (mu == 0) reconstruct<0, SF, true>(acc[j], w);
    } else {
      if (mu == 3 && fwd) reconstruct<3, SF, false>(acc[j], w);
      if (mu == 3 && !fwd) reconstruct<3, SB, false>(acc[j], w);
      if (mu == 2 && fwd) reconstruct<2, SF, false>(acc[j], w);
      if (mu == 2 && !fwd) reconstruct<2, SB, false>(acc[j], w);
      if (mu == 1 && fwd) reconstruct<1, SF, false>(acc[j], w);
      if (mu == 1 && !fwd) reconstruct<1, SB, false>(acc[j], w);
      if (mu == 0 && fwd) reconstruct<0, SF, false>(acc[j], w);
      if (mu == 0 && !fwd) reconstruct<0, SB, false>(acc[j], w);
    }
  }
}

// ---------------------------------------------------------------------------
// Domain decomposition along t ("virtual ranks").  A sub-lattice that owns a
// t-range of the global lattice does not see its t-neighbour spinors; at its
// t faces it uses half spinors received from the neighbouring ranks instead:
//   up   (from the rank above): h = (projection of the forward t hop) of the
//        neighbour's spinor at its first t slice; this rank applies its own
//        link U_t(x) and reconstructs;
//   down (from the rank below): w = U_t(x - t)^+ times the projection of the
//        backward hop, computed by its owner with its own link.
// Both are made by the same project / su3_mul code the single-domain kernel
// runs, so the decomposed result equals the single-domain one bit for bit.
// Halo layout per RHS: 3 quads x Ls x (Lx Ly Lz) face sites, [quad][s][face].
template <class P, int S, bool FIRST, int SPT>
__device__ __forceinline__ void halo_hop_up(Spinor<typename Pair<P>::type> (&acc)[SPT],
                                            const typename P::vec *halo, long long hplane,
                                            int Vf, int face, const typename P::vec *gauge,
                                            int x4, typename P::C lsign, int s0) {
  using C = typename P::C;
  using V2 = typename Pair<P>::type;
  constexpr int VPQ = 4 / P::R;
  C U[18];
  load_link<P>(U, gauge, 3, x4, lsign);
#pragma unroll
  for (int j = 0; j < SPT; ++j) {
    Half<V2> h, w;
    const typename P::vec *b = halo + (long long)(s0 + j) * Vf + face;
#pragma unroll
    for (int c = 0; c < 3; ++c) quad_in(h.re[c], h.im[c], b + (long long)c * VPQ * hplane, hplane);
    su3_mul<false>(w, U, h);
    reconstruct<3, S, FIRST>(acc[j], w);
  }
}

template <class P, int S, int SPT>
__device__ __forceinline__ void halo_hop_down(Spinor<typename Pair<P>::type> (&acc)[SPT],
                                              const typename P::vec *halo, long long hplane,
                                              int Vf, int face, int s0) {
  using V2 = typename Pair<P>::type;
  constexpr int VPQ = 4 / P::R;
#pragma unroll
  for (int j = 0; j < SPT; ++j) {
    Half<V2> w;
    const typename P::vec *b = halo + (long long)(s0 + j) * Vf + face;
#pragma unroll
    for (int c = 0; c < 3; ++c) quad_in(w.re[c], w.im[c], b + (long long)c * VPQ * hplane, hplane);
    reconstruct<3, S, false>(acc[j], w);
  }
}

// Face halves a rank sends: to the rank below, the forward-hop projection of
// its first t slice; to the rank above, U_t^+ times the backward-hop
// projection of its last t slice.  PHI: the hop acts on phi / b = psi + (c/b) K psi
// (the operator D; `c` is c / b here), formed at the face slices with the same
// arithmetic as roll_5d, so the receiver's sums equal the undecomposed kernel's
// bit for bit.  One thread per (face site, s) of one RHS.
template <class P, bool PHI>
__device__ __forceinline__ void face_spinor(Spinor<typename Pair<P>::type> &v, const Field<P> &F,
                                            int x4, int s, int Ls, typename P::C b,
                                            typename P::C c, typename P::C mf) {
  using C = typename P::C;
  using V2 = typename Pair<P>::type;
  if (!PHI) {
    F.load_half(v.up, x4, s, 0);
    F.load_half(v.lo, x4, s, 1);
    return;
  }
  // phi_s / b: upper = u_s + (c/b) fp u_{s-1}, lower = l_s + (c/b) fn l_{s+1}
  Half<V2> u, up, l, ln;
  const int sp = s == 0 ? Ls - 1 : s - 1;
  const int sn = s == Ls - 1 ? 0 : s + 1;
  const C fp = s == 0 ? -mf : C(1);
  const C fn = s == Ls - 1 ? -mf : C(1);
  F.load_half(u, x4, s, 0);
  F.load_half(up, x4, sp, 0);
  F.load_half(l, x4, s, 1);
  F.load_half(ln, x4, sn, 1);
  half_axpy(v.up, u, bc<V2>(c * fp), up);
  half_axpy(v.lo, l, bc<V2>(c * fn), ln);
}

template <class P, bool DAG, bool PHI>
__global__ void halo_pack_kernel(typename P::vec *send_dn, typename P::vec *send_up,
                                 const typename P::vec *in, const typename P::vec *gauge,
                                 int bct, int V4, int Vf, int Lt, int Ls,
                                 long long plane, long long rhs_stride, long long hplane,
                                 long long hrhs, const DslashParams p) {
  using C = typename P::C;
  using V2 = typename Pair<P>::type;
  constexpr int SF = DAG ? 1 : -1;
  constexpr int SB = -SF;
  constexpr int VPQ = 4 / P::R;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int rhs = blockIdx.y;
  if (i >= (long long)Vf * Ls) return;
  const int face = (int)(i % Vf);
  const int s = (int)(i / Vf);
  Field<P> F;
  F.base = in + (long long)rhs * rhs_stride;
  F.V4 = V4;
  F.Ls = Ls;
  (void)plane;
  const C b = (C)p.b, c = PHI ? (C)(p.c / p.b) : C(0), mf = PHI ? (C)p.mf[rhs] : C(0);
  {  // first slice -> rank below
    Spinor<V2> v;
    face_spinor<P, PHI>(v, F, face, s, Ls, b, c, mf);
    Half<V2> h;
    project<3, SF>(h, v.up, v.lo);
    typename P::vec *o = send_dn + (long long)rhs * hrhs + (long long)s * Vf + face;
#pragma unroll
    for (int cc = 0; cc < 3; ++cc)
      quad_out(o + (long long)cc * VPQ * hplane, hplane, h.re[cc], h.im[cc]);
  }
  {  // last slice -> rank above
    const int x4 = face + (Lt - 1) * Vf;
    Spinor<V2> v;
    face_spinor<P, PHI>(v, F, x4, s, Ls, b, c, mf);
    Half<V2> h, w;
    project<3, SB>(h, v.up, v.lo);
    C U[18];
    load_link<P>(U, gauge, 3, x4, (C)bct);  // the last slice's t link crosses the edge
    su3_mul<true>(w, U, h);
    typename P::vec *o = send_up + (long long)rhs * hrhs + (long long)s * Vf + face;
#pragma unroll
    for (int cc = 0; cc < 3; ++cc)
      quad_out(o + (long long)cc * VPQ * hplane, hplane, w.re[cc], w.im[cc]);
  }
}

// op: OP_DHOP / OP_DHOP_DAG / OP_D (faces of phi) / OP_DDAG (faces of Dhop^+).
template <class P>
int launch_halo_pack_impl(const DslashParams &p, void *send_dn, void *send_up, int op,
                          cudaStream_t st) {
  const int Vf = p.L[0] * p.L[1] * p.L[2];
  const long long hplane = (long long)p.Ls * Vf;
  const long long hrhs = hplane * (12 / P::R);
  const int tpb = 128;
  dim3 grid((unsigned)(((long long)Vf * p.Ls + tpb - 1) / tpb), p.nrhs);
  using vec = typename P::vec;
#define DW_HALO_LAUNCH(DAG, PHI)                                                            \
  halo_pack_kernel<P, DAG, PHI><<<grid, tpb, 0, st>>>(                                      \
      (vec *)send_dn, (vec *)send_up, (const vec *)p.in, (const vec *)p.gauge, p.bc[3], p.V4, \
      Vf, p.L[3], p.Ls, p.plane, p.rhs_stride, hplane, hrhs, p)
  switch (op) {
    case OP_DHOP: DW_HALO_LAUNCH(false, false); break;
    case OP_DHOP_DAG: DW_HALO_LAUNCH(true, false); break;
    case OP_D: DW_HALO_LAUNCH(false, true); break;
    case OP_DDAG: DW_HALO_LAUNCH(true, false); break;
    default: return -2;
  }
#undef DW_HALO_LAUNCH
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Neighbour addressing that keeps one word per thread instead of eight
// neighbour indices and eight link signs: bit 2 mu of `edge` says the site is
// on the upper face in direction mu (c_mu = L_mu - 1), bit 2 mu + 1 that it is
// on the lower face (c_mu = 0).  Indices and signs are rebuilt per hop from
// the launch parameters.
struct Hops {
  int x4;
  unsigned edge;
  __device__ __forceinline__ Hops(const DslashParams &p, int x4_) : x4(x4_), edge(0u) {
    int rem = x4_;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int c = (m < 3) ? rem % p.L[m] : rem;
      rem /= p.L[m];
      edge |= (unsigned)(c == p.L[m] - 1) << (2 * m);
      edge |= (unsigned)(c == 0) << (2 * m + 1);
    }
  }
  template <int MU>
  __device__ __forceinline__ static int stride(const DslashParams &p) {
    int st = 1;
#pragma unroll
    for (int m = 0; m < MU; ++m) st *= p.L[m];
    return st;
  }
  // x4 + mu (FWD) or x4 - mu, periodic
  template <int MU, bool FWD>
  __device__ __forceinline__ int nb(const DslashParams &p) const {
    const int st = stride<MU>(p);
    const bool at = (edge >> (2 * MU + (FWD ? 0 : 1))) & 1u;
    if (FWD) return at ? x4 - (p.L[MU] - 1) * st : x4 + st;
    return at ? x4 + (p.L[MU] - 1) * st : x4 - st;
  }
  // boundary sign of the link the hop uses
  template <int MU, bool FWD>
  __device__ __forceinline__ int sign(const DslashParams &p) const {
    return ((edge >> (2 * MU + (FWD ? 0 : 1))) & 1u) ? p.bc[MU] : 1;
  }
};

// Variant 4 is variant 5 compiled with at most 128 registers per thread.  The
// kernel is latency bound: with CTAs of one or two warps (sgrp > 1) 16 warps
// fit on an SM instead of 12 at the uncapped ~140 registers, and the extra
// loads in flight outweigh a few spilled registers.  (Caps of 112 and 96
// registers spill more and ran slower at 32^3 x 64 x 12.)
template <int VAR>
struct RegCap {
  static constexpr int value = (VAR == 4 || VAR == 6 || VAR == 7) ? 128 : 0;
};



// CB: the fields are single-parity (checkerboard) fields: a thread computes the
// output site of parity p.parity with field index xf = x4 / 2 (x4 the full
// lexicographic index; Lx even), its neighbours are read from the field of the
// other parity at their x4 / 2, and the links stay full-lattice.
// GLX (variants 6, 7): row staging for any Lx <= 32 (general in-plane
// neighbour indices); without it the kernel is specialised to Lx = 32.
template <class P, int OP, int SPT, int VAR, bool CB = false, bool GLX = false>
__device__ __forceinline__ void dslash_body(const DslashParams &p) {
  using C = typename P::C;
  using vec = typename P::vec;
  using V2 = typename Pair<P>::type;
  constexpr bool DAG = (OP == OP_DHOP_DAG || OP == OP_DDAG);
  constexpr bool PHI = (OP == OP_D);
  constexpr int SF = DAG ? 1 : -1;  // sign S of the forward hop
  constexpr int SB = -SF;           // sign S of the backward hop

  // CTAs are RHS-major (consecutive CTAs = the same sites for successive RHS),
  // so the links of a tile are reused from L2 across right-hand sides.  Tiles
  // are tx consecutive sites of one (x, y) plane; planes are visited z-block
  // by z-block (zblk blocks of Lz / zblk planes), t inside a block, so a
  // spinor's last use as a t-neighbour follows its first use by 2 Lz/zblk
  // planes instead of 2 Lz: the L2 then holds the reuse window.
  const int tx = blockDim.x;
  // RHS innermost (consecutive CTAs: the same tile for successive RHS, which
  // share its links in L2) or outermost (p.rhs_outer: one RHS's sweep after
  // another, each with the reuse window of a single RHS)
  const int ctas_per_rhs = gridDim.x / p.nrhs;
  const int rhs = p.rhs_outer ? blockIdx.x / ctas_per_rhs : blockIdx.x % p.nrhs;
  const int cta_in_rhs = p.rhs_outer ? blockIdx.x % ctas_per_rhs : blockIdx.x / p.nrhs;
  const int Lxf = CB ? (p.L[0] >> 1) : p.L[0];  // field sites per x row
  const int plane_sites = Lxf * p.L[1];
  int x4, xf, in_plane, sg;  // full site, field index, index in the (x, y) plane
  {
    int id = cta_in_rhs;
    sg = id % p.sgrp;  // slice group: the CTAs of one tile are adjacent
    id /= p.sgrp;
    const int tile = id % p.tiles_per_plane;
    id /= p.tiles_per_plane;
    const int bz = p.L[2] / p.zblk;
    const int zl = id % bz;
    id /= bz;
    const int t = p.t_begin + id % p.t_count;
    const int zb = id / p.t_count;
    const int z = zb * bz + zl;
    in_plane = tile * tx + threadIdx.x;
    xf = in_plane + plane_sites * (z + p.L[2] * t);
    if (CB)
      x4 = 2 * xf + (((in_plane / Lxf) + z + t + p.parity) & 1);
    else
      x4 = xf;
  }
  // field index of a full neighbour index
  auto fidx = [](int v) { return CB ? (v >> 1) : v; };
  const int chunk = threadIdx.y + sg * blockDim.y;  // slice group of this thread row
  const int nchunk = blockDim.y;                     // thread rows of the CTA
  if (p.gate && !p.gate[(long long)rhs * p.gate_stride]) return;  // whole CTA: uniform
  const bool active = in_plane < plane_sites;
  const int s0 = chunk * SPT;
  const int Ls = p.Ls;

  Field<P> F;
  F.base = reinterpret_cast<const vec *>(p.in) + (long long)rhs * p.rhs_stride;
  F.V4 = p.V4;
  F.Ls = p.Ls;
  vec *out = reinterpret_cast<vec *>(p.out) + (long long)rhs * p.rhs_stride;
  const vec *gauge = reinterpret_cast<const vec *>(p.gauge);

  const C mf = (OP == OP_D || OP == OP_DDAG) ? (C)p.mf[rhs] : C(0);
  // D's hop acts on phi / b = psi + (c / b) K psi: `c` is c / b for D, and the
  // factor b moves into the scale of the hop sum (hsc), so forming the
  // combination takes one FMA per element instead of an FMA and a multiply
  const C b = (C)p.b, c = PHI ? (C)(p.c / p.b) : (C)p.c;
  const C hsc = PHI ? (C)(p.hscale * p.b) : (C)p.hscale;
  const C alpha = (C)p.alpha, beta = (C)p.beta;
  // the field of the local term alpha psi + beta K psi (none: hopping term alone)
  Field<P> Fo;
  Fo.base = p.own ? reinterpret_cast<const vec *>(p.own) + (long long)rhs * p.rhs_stride
                  : F.base;
  Fo.V4 = p.V4;
  Fo.Ls = p.Ls;

  SpinorP<P> acc[SPT];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  size_t smem_used = 0;
  double nsq = 0.0;     // OP_D: |out|^2 of this thread's output sites
  bool stored = false;  // OP_D on the rows path: stored inside its loop

  int nb[8];   // neighbours in the order t+, t-, z+, z-, y+, y-, x+, x-
  int lsg[8];  // boundary sign of the link each of those hops uses
  // (variants 0, 4, 5 rebuild both per hop from the edge flags of Hops)
  if (active && (VAR == 1 || VAR == 2 || VAR == 3)) {
    int rem = x4;
    const int cx = rem % p.L[0];
    rem /= p.L[0];
    const int cy = rem % p.L[1];
    rem /= p.L[1];
    const int cz = rem % p.L[2];
    const int ct = rem / p.L[2];
    const int st1 = p.L[0];
    const int st2 = p.L[0] * p.L[1];
    const int st3 = st2 * p.L[2];
    nb[6] = (cx == p.L[0] - 1) ? x4 - (p.L[0] - 1) : x4 + 1;
    nb[7] = (cx == 0) ? x4 + (p.L[0] - 1) : x4 - 1;
    nb[4] = (cy == p.L[1] - 1) ? x4 - (p.L[1] - 1) * st1 : x4 + st1;
    nb[5] = (cy == 0) ? x4 + (p.L[1] - 1) * st1 : x4 - st1;
    nb[2] = (cz == p.L[2] - 1) ? x4 - (p.L[2] - 1) * st2 : x4 + st2;
    nb[3] = (cz == 0) ? x4 + (p.L[2] - 1) * st2 : x4 - st2;
    nb[0] = (ct == p.L[3] - 1) ? x4 - (p.L[3] - 1) * st3 : x4 + st3;
    nb[1] = (ct == 0) ? x4 + (p.L[3] - 1) * st3 : x4 - st3;
    lsg[0] = (ct == p.L[3] - 1) ? p.bc[3] : 1;
    lsg[1] = (ct == 0) ? p.bc[3] : 1;
    lsg[2] = (cz == p.L[2] - 1) ? p.bc[2] : 1;
    lsg[3] = (cz == 0) ? p.bc[2] : 1;
    lsg[4] = (cy == p.L[1] - 1) ? p.bc[1] : 1;
    lsg[5] = (cy == 0) ? p.bc[1] : 1;
    lsg[6] = (cx == p.L[0] - 1) ? p.bc[0] : 1;
    lsg[7] = (cx == 0) ? p.bc[0] : 1;
  } else {
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      nb[d] = 0;
      lsg[d] = 1;
    }
  }

  if constexpr (VAR == 6 || VAR == 7) {
    // Rows path.  The (x, y) plane of a (z, t) slice is nblk = Lx Ly / 32 whole
    // 32-site blocks ("rows": one x row when Lx = 32, two when Lx = 16, a row
    // and a part when Lx = 24); a tile is R = tx/32 consecutive blocks y0 ..
    // y0+R-1.  Blocks y0-1 .. y0+R of the CTA's slices (one contiguous run per
    // block in the blocked layout) are bulk-copied into shared memory by one
    // thread while the t and z hops run from global memory; the y and x hops
    // then read their neighbours there (with Lx <= 32 an x or y neighbour is
    // at most one block from its site, so the staged blocks hold them all).
    // Same hop order as variant 5, so the same sums.  Variant 6: one tile per
    // CTA.  Variant 7: the CTA walks the nblk/R tiles of its plane, keeping the
    // blocks in a ring of R + 2 slots (block v in slot (v + 1) mod (R + 2)):
    // each step copies only its R new blocks, the two shared with the previous
    // tile stay, and the next step's t+ blocks are prefetched into L2.
    // D (PHI): phi = (b + cK) psi needs the upper spins of the slice below the
    // CTA's range and the lower spins of the one above (wrapped in s): each
    // staged block holds nsl + 2 slices, those two halves at its ends, and the
    // D epilogue takes its own-site psi from the staged blocks as well.
    constexpr bool RING = (VAR == 7);
    constexpr int NPV = 24 / P::R;
    constexpr int EDGE = PHI ? 1 : 0;
    const int nsl = nchunk * SPT;  // slices of this CTA
    const int nss = nsl + 2 * EDGE;  // staged slices per block
    const int sbase = sg * nsl;
    const int R = tx / 32;
    const int Lx = p.L[0];
    const int nblk = (Lx * p.L[1]) >> 5;  // 32-site blocks of a plane
    const int NR = R + 2;  // row slots
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem_raw);
    vec *rows = reinterpret_cast<vec *>(smem_raw + 128);
    const int row_vecs = nss * NPV * 32;
    const unsigned row_bytes = (unsigned)(nsl * NPV * 32 * sizeof(vec));
    const unsigned half_bytes = (unsigned)((NPV / 2) * 32 * sizeof(vec));
    const unsigned blk_bytes = row_bytes + 2 * EDGE * half_bytes;
    const int s_below = sbase == 0 ? Ls - 1 : sbase - 1;  // PHI: the edge slices
    const int s_above = sbase + nsl == Ls ? 0 : sbase + nsl;
    const bool leader = threadIdx.x == 0 && threadIdx.y == 0;
    const int plane_base = x4 - in_plane;  // x4 of site 0 of the plane
    const int plane_blk = plane_base >> 5;  // block of row 0 of the plane
    const int steps = RING ? (Lx * p.L[1]) / tx : 1;
    const int sl = (int)threadIdx.y * SPT;  // = s0 - sbase
    if (leader) mbar_init(bar, 1);
    __syncthreads();
    for (int k = 0; k < steps; ++k) {
      const int ip = RING ? k * tx + (int)threadIdx.x : in_plane;  // site in the plane
      const int xs = plane_base + ip;
      const int y0 = (ip - (int)threadIdx.x) >> 5;  // first row of the tile
      if (leader) {
        // rows y0-1 .. y0+R (all of them at the first step; the ring keeps
        // two and takes R new ones later); rows are taken periodically in y
        const int first = (RING && k > 0) ? y0 + 1 : y0 - 1;
        const int n = (RING && k > 0) ? R : R + 2;
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mbar_expect_tx(bar, blk_bytes * (unsigned)n);
        for (int r = 0; r < n; ++r) {
          const int v = first + r;  // virtual block, -1 .. nblk
          const int y = v < 0 ? v + nblk : (v >= nblk ? v - nblk : v);
          const int slot = RING ? (v + 1) % NR : r;
          const vec *blk = F.base + (long long)(plane_blk + y) * Ls * NPV * 32;
          vec *dst = rows + (size_t)slot * row_vecs;
          bulk_g2s(dst + EDGE * NPV * 32, blk + (long long)sbase * NPV * 32, row_bytes, bar);
          if (PHI) {
            bulk_g2s(dst, blk + (long long)s_below * NPV * 32, half_bytes, bar);
            bulk_g2s(dst + (nss - 1) * NPV * 32 + (NPV / 2) * 32,
                     blk + (long long)s_above * NPV * 32 + (NPV / 2) * 32, half_bytes, bar);
          }
        }
        if (RING && k + 1 < steps) {
          // the t+ neighbours are the first touch of their plane (read from
          // HBM): fetch the next step's into L2 while this step runs
          const int LyLz = nblk * p.L[2];  // blocks of a t slice
          const int tc = plane_blk / LyLz;
          const int tp_blk = plane_blk + (tc == p.L[3] - 1 ? -(p.L[3] - 1) : 1) * LyLz;
          for (int r = 0; r < R; ++r) {
            const int y = (k + 1) * R + r;
            bulk_prefetch_l2(F.base + ((long long)(tp_blk + y) * Ls + sbase) * NPV * 32,
                             row_bytes);
          }
        }
      }
      const Hops H(p, xs);
      hop_dir<P, 3, SF, false, PHI, true, SPT, HINT_KEEP>(
          acc, F, gauge, (C)H.sign<3, true>(p), H.nb<3, true>(p), xs, s0, Ls, b, c, mf);
      hop_dir<P, 3, SB, true, PHI, false, SPT, HINT_DROP>(
          acc, F, gauge, (C)H.sign<3, false>(p), H.nb<3, false>(p), H.nb<3, false>(p), s0, Ls,
          b, c, mf);
      hop_dir<P, 2, SF, false, PHI, false, SPT>(acc, F, gauge, (C)H.sign<2, true>(p),
                                                H.nb<2, true>(p), xs, s0, Ls, b, c, mf);
      hop_dir<P, 2, SB, true, PHI, false, SPT>(acc, F, gauge, (C)H.sign<2, false>(p),
                                               H.nb<2, false>(p), H.nb<2, false>(p), s0, Ls,
                                               b, c, mf);
      // p.wait_polls >= 0 bounds the first wait by that many polls (0: give up
      // at once, which exercises the timeout report); the second bounded wait
      // still lets the copies in flight land before the slots are read
      if (!mbar_wait(bar, (unsigned)k & 1u, p.wait_polls >= 0 ? p.wait_polls : 1 << 24)) {
        atomicExch(p.status, 1);
        mbar_wait(bar, (unsigned)k & 1u);  // one more bounded wait for the copies in flight
      }
      Field<P> S;  // the staged rows, addressed as blocks of 32 sites x nss slices
      S.base = rows;
      S.V4 = 0;
      S.Ls = nss;
      // staged index of the in-plane site q (virtual: q < 0 and q >= Lx Ly are
      // the neighbouring rows across the periodic y edge, in blocks -1, nblk)
      int iyp, iym, ixp, ixm, iat;
      if constexpr (!GLX) {  // Lx = 32: a block is one x row: the row's slot and the lane
        const int ry = (ip >> 5) - y0;  // row of this site in the tile
        const int xl = ip & 31;
        const int sdn = RING ? (y0 + ry) % NR : ry;
        const int sat = RING ? (y0 + ry + 1) % NR : ry + 1;
        const int sup = RING ? (y0 + ry + 2) % NR : ry + 2;
        iyp = sup * 32 + xl;
        iym = sdn * 32 + xl;
        ixp = sat * 32 + ((xl + 1) & 31);
        ixm = sat * 32 + ((xl + 31) & 31);
        iat = sat * 32 + xl;
      } else {
        auto sidx = [&](int q) {
          const int v = (q + 32) / 32 - 1;  // floor(q / 32) for q >= -32
          const int slot = RING ? (v + 1) % NR : v - (y0 - 1);
          return slot * 32 + (q - 32 * v);
        };
        const int xc = ip % Lx;
        iyp = sidx(ip + Lx);
        iym = sidx(ip - Lx);
        ixp = sidx(xc == Lx - 1 ? ip - (Lx - 1) : ip + 1);
        ixm = sidx(xc == 0 ? ip + (Lx - 1) : ip - 1);
        iat = sidx(ip);
      }
      // staged slices: the hopping term alone addresses slice sl + EDGE of the
      // nss staged ones; D passes the global slice and Ls (for the -mf factors
      // of K) and the staged index sl + 1 of slice s0
      const int hs = PHI ? s0 : sl + EDGE, hL = PHI ? Ls : nss;
      hop_dir<P, 1, SF, false, PHI, false, SPT, HINT_SMEM>(
          acc, S, gauge, (C)H.sign<1, true>(p), iyp, xs, hs, hL, b, c, mf, sl + EDGE);
      hop_dir<P, 1, SB, true, PHI, false, SPT, HINT_SMEM>(
          acc, S, gauge, (C)H.sign<1, false>(p), iym, H.nb<1, false>(p), hs, hL, b, c, mf,
          sl + EDGE);
      hop_dir<P, 0, SF, false, PHI, false, SPT, HINT_SMEM>(
          acc, S, gauge, (C)H.sign<0, true>(p), ixp, xs, hs, hL, b, c, mf, sl + EDGE);
      hop_dir<P, 0, SB, true, PHI, false, SPT, HINT_SMEM>(
          acc, S, gauge, (C)H.sign<0, false>(p), ixm, H.nb<0, false>(p), hs, hL, b, c, mf,
          sl + EDGE);
      if constexpr (OP == OP_D) {
        // the local term from the staged own site (the launch requires own = in)
        d_epilogue<P, SPT, true>(acc, out, xs, S, true, iat, sl + 1, s0, Ls, alpha, beta, mf,
                                 bc<V2>(hsc), p.norm_partials != nullptr, nsq);
        stored = true;
      } else if (RING) {
#pragma unroll
        for (int j = 0; j < SPT; ++j)
          store_spinor<P>(out + F.site(s0 + j, xs), kPlaneStride, acc[j]);
      }
      if (RING) __syncthreads();  // every thread is done with the slots the next step refills
    }
    if constexpr (OP != OP_D) {
      if (RING) return;
    }
  } else if constexpr (VAR == 0 || VAR == 4 || VAR == 5) {
    if (active) {
      const Hops H(p, x4);
      // t faces of a sub-lattice take their t-neighbours from the halos
      // (spin-pair form only)
      const int Vf = p.L[0] * p.L[1] * p.L[2];
      const int ct = x4 / Vf;
      const long long hplane = (long long)Ls * Vf;
      const long long hrhs = hplane * (12 / P::R);
      bool up_done = false, dn_done = false;
      if constexpr (!P::CPLX) {
        if (!CB && p.halo_up && ct == p.L[3] - 1) {
          halo_hop_up<P, SF, true, SPT>(acc, (const vec *)p.halo_up + rhs * hrhs, hplane, Vf,
                                        x4 - ct * Vf, gauge, x4, (C)H.sign<3, true>(p), s0);
          up_done = true;
        }
      }
      if (!up_done)
        hop_dir<P, 3, SF, false, PHI, true, SPT, VAR >= 4 ? HINT_KEEP : HINT_NONE>(
            acc, F, gauge, (C)H.sign<3, true>(p), fidx(H.nb<3, true>(p)), x4, s0, Ls, b, c, mf);
      if constexpr (!P::CPLX) {
        if (!CB && p.halo_dn && ct == 0) {
          halo_hop_down<P, SB, SPT>(acc, (const vec *)p.halo_dn + rhs * hrhs, hplane, Vf, x4,
                                    s0);
          dn_done = true;
        }
      }
      if (!dn_done)
        hop_dir<P, 3, SB, true, PHI, false, SPT, VAR >= 4 ? HINT_DROP : HINT_NONE>(
            acc, F, gauge, (C)H.sign<3, false>(p), fidx(H.nb<3, false>(p)), H.nb<3, false>(p),
            s0, Ls, b, c, mf);
#define DW_HOP(MU, FWD, S, ADJ)                                                                  \
  hop_dir<P, MU, S, ADJ, PHI, false, SPT>(acc, F, gauge, (C)H.sign<MU, FWD>(p),                \
                                          fidx(H.nb<MU, FWD>(p)), FWD ? x4 : H.nb<MU, FWD>(p), \
                                          s0, Ls, b, c, mf)
      DW_HOP(2, true, SF, false);
      DW_HOP(2, false, SB, true);
      DW_HOP(1, true, SF, false);
      DW_HOP(1, false, SB, true);
      DW_HOP(0, true, SF, false);
      DW_HOP(0, false, SB, true);
#undef DW_HOP
    }
  } else if constexpr (VAR == 2 || VAR == 3) {
    if constexpr (PHI) {  // the (b + cK) input combination keeps the VAR 0 path
      if (active) {
        hop_dir<P, 3, SF, false, PHI, true, SPT>(acc, F, gauge, (C)lsg[0], nb[0], x4, s0, Ls, b, c, mf);
        hop_dir<P, 3, SB, true, PHI, false, SPT>(acc, F, gauge, (C)lsg[1], nb[1], nb[1], s0, Ls, b, c, mf);
        hop_dir<P, 2, SF, false, PHI, false, SPT>(acc, F, gauge, (C)lsg[2], nb[2], x4, s0, Ls, b, c, mf);
        hop_dir<P, 2, SB, true, PHI, false, SPT>(acc, F, gauge, (C)lsg[3], nb[3], nb[3], s0, Ls, b, c, mf);
        hop_dir<P, 1, SF, false, PHI, false, SPT>(acc, F, gauge, (C)lsg[4], nb[4], x4, s0, Ls, b, c, mf);
        hop_dir<P, 1, SB, true, PHI, false, SPT>(acc, F, gauge, (C)lsg[5], nb[5], nb[5], s0, Ls, b, c, mf);
        hop_dir<P, 0, SF, false, PHI, false, SPT>(acc, F, gauge, (C)lsg[6], nb[6], x4, s0, Ls, b, c, mf);
        hop_dir<P, 0, SB, true, PHI, false, SPT>(acc, F, gauge, (C)lsg[7], nb[7], nb[7], s0, Ls, b, c, mf);
      }
    } else if (active) {
      hop_prefetch<P, SPT, VAR == 2 ? 0 : 1, DAG>(acc, F, gauge, x4, nb, lsg, s0);
    }
  } else if constexpr (VAR == 1) {
    StagedHop<P, OP, SPT> H;
    H.smem = smem_raw;
    H.T = tx * nchunk;
    H.t = threadIdx.y * tx + threadIdx.x;
    hop_staged<P, OP, SPT>(acc, H, F, gauge, x4, active, nb, lsg, s0, Ls, b, c, mf);
    smem_used = kStages * StageLayout<P, PHI, SPT>::stage_bytes(H.T);
  }

  auto store = [&](int j, const SpinorP<P> &v) {
    store_spinor<P>(out + F.site(s0 + j, xf), kPlaneStride, v);
  };
  const V2 mhalf = bc<V2>(hsc);  // -1/2 of D_W (or the caller's factor), times b for D

  if constexpr (OP == OP_DHOP || OP == OP_DHOP_DAG) {
    if (active) {
#pragma unroll
      for (int j = 0; j < SPT; ++j) store(j, acc[j]);
    }
  } else if constexpr (OP == OP_D) {
    // out = alpha psi + beta K psi - 1/2 Dhop phi; optionally |out|^2 per CTA
    // (the CG's <p, D^+D p> = |D p|^2, fused here to save a pass over two fields)
    if (active && !stored)
      d_epilogue<P, SPT, false>(acc, out, xf, Fo, p.own != nullptr, xf, 0, s0, Ls, alpha, beta,
                                mf, mhalf, p.norm_partials != nullptr, nsq);
    if (p.norm_partials) {
      // fixed-order block sum: warp shuffles, then warp 0 over the warp sums
      __shared__ double warp_sums[32];
      const int tid = threadIdx.y * blockDim.x + threadIdx.x;
      const int nwarps = (blockDim.x * blockDim.y + 31) / 32;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) nsq += __shfl_down_sync(0xffffffffu, nsq, o);
      if ((tid & 31) == 0) warp_sums[tid >> 5] = nsq;
      __syncthreads();
      if (tid < 32) {
        double v = tid < nwarps ? warp_sums[tid] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (tid == 0)
          p.norm_partials[(long long)rhs * ctas_per_rhs + cta_in_rhs] = v;
      }
    }
  } else {
    // OP_DDAG: out = alpha psi + beta K^+ psi - 1/2 (b + c K^+) Dhop^+ psi.
    // K^+ acc needs the upper spins of slice s+1 and the lower spins of s-1;
    // at chunk edges they come from the neighbouring chunk through shared memory.
    // With sgrp > 1 the sgrp CTAs of a tile form one thread-block cluster (rank
    // = slice group) and the edges of a neighbouring group are read from that
    // CTA's shared memory (distributed shared memory, after a cluster barrier).
    V2 *sm_up = reinterpret_cast<V2 *>(smem_raw + smem_used);  // [nchunk][6][tx]
    V2 *sm_lo = sm_up + (size_t)nchunk * 6 * tx;    // [nchunk][6][tx]
    const int t = threadIdx.x;
    const int lch = threadIdx.y;          // this CTA's slot of the chunk
    const int tch = nchunk * p.sgrp;      // chunks of the whole tile
    const bool clustered = p.sgrp > 1;
    if (active) {
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        sm_up[((size_t)lch * 6 + 2 * cc) * tx + t] = acc[0].up.re[cc];
        sm_up[((size_t)lch * 6 + 2 * cc + 1) * tx + t] = acc[0].up.im[cc];
        sm_lo[((size_t)lch * 6 + 2 * cc) * tx + t] = acc[SPT - 1].lo.re[cc];
        sm_lo[((size_t)lch * 6 + 2 * cc + 1) * tx + t] = acc[SPT - 1].lo.im[cc];
      }
    }
    if (clustered)
      cooperative_groups::this_cluster().sync();
    else
      __syncthreads();
    // fused CG residual update (p.rs): r_s at FP64 for FP64 operators, else FP32
    using PR = typename std::conditional<std::is_same<C, double>::value, F64, F32>::type;
    using rvec = typename PR::vec;
    constexpr int RNPV = 24 / PR::R;
    constexpr int RVPQ = 4 / PR::R;
    constexpr int PNPV = 24 / P::R;  // the direction p, at the operator's precision
    constexpr int PVPQ = 4 / P::R;
    double rsq = 0.0;
    if (active) {
      const int gn = (chunk + 1 == tch) ? 0 : chunk + 1;  // neighbouring chunks of the tile
      const int gp = (chunk == 0) ? tch - 1 : chunk - 1;
      const V2 fn = bc<V2>((chunk + 1 == tch) ? -mf : C(1));
      const V2 fp = bc<V2>((chunk == 0) ? -mf : C(1));
      const int cn = gn % nchunk, cp = gp % nchunk;  // their slots in their CTA
      const V2 *up_src = sm_up, *lo_src = sm_lo;
      if (clustered) {
        auto cl = cooperative_groups::this_cluster();
        if (gn / nchunk != sg) up_src = cl.map_shared_rank(sm_up, (unsigned)(gn / nchunk));
        if (gp / nchunk != sg) lo_src = cl.map_shared_rank(sm_lo, (unsigned)(gp / nchunk));
      }
      const V2 mb = bc<V2>((C)p.hscale * b), mc = bc<V2>((C)p.hscale * c);
      auto emit = [&](int j, const Spinor<V2> &v) {
        Spinor<V2> o;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          // upper: (K^+ acc)_s = acc_up(s+1); lower: (K^+ acc)_s = acc_lo(s-1)
          V2 kur, kui, klr, kli;
          if (j + 1 < SPT) {
            kur = acc[(j + 1 < SPT) ? j + 1 : 0].up.re[cc];
            kui = acc[(j + 1 < SPT) ? j + 1 : 0].up.im[cc];
          } else {
            kur = p_mul(fn, up_src[((size_t)cn * 6 + 2 * cc) * tx + t]);
            kui = p_mul(fn, up_src[((size_t)cn * 6 + 2 * cc + 1) * tx + t]);
          }
          if (j > 0) {
            klr = acc[(j > 0) ? j - 1 : 0].lo.re[cc];
            kli = acc[(j > 0) ? j - 1 : 0].lo.im[cc];
          } else {
            klr = p_mul(fp, lo_src[((size_t)cp * 6 + 2 * cc) * tx + t]);
            kli = p_mul(fp, lo_src[((size_t)cp * 6 + 2 * cc + 1) * tx + t]);
          }
          o.up.re[cc] = p_fma(mc, kur, p_fma(mb, acc[j].up.re[cc], v.up.re[cc]));
          o.up.im[cc] = p_fma(mc, kui, p_fma(mb, acc[j].up.im[cc], v.up.im[cc]));
          o.lo.re[cc] = p_fma(mc, klr, p_fma(mb, acc[j].lo.re[cc], v.lo.re[cc]));
          o.lo.im[cc] = p_fma(mc, kli, p_fma(mb, acc[j].lo.im[cc], v.lo.im[cc]));
        }
        if (p.rs) {
          const V2 na = bc<V2>(-(C)p.rs_alpha[(long long)rhs * p.rs_alpha_stride]);
          rvec *rb = reinterpret_cast<rvec *>(p.rs) + (long long)rhs * p.rs_stride +
                     site_off(xf, s0 + j, Ls, RNPV);
          C ss = 0;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const Half<V2> &oh = h ? o.lo : o.up;
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
              rvec *q = rb + (long long)(h * 3 + cc) * RVPQ * kPlaneStride;
              V2 rr, ri;
              quad_in(rr, ri, q, kPlaneStride);
              rr = p_fma(na, oh.re[cc], rr);
              ri = p_fma(na, oh.im[cc], ri);
              ss += rr.x * rr.x + rr.y * rr.y + ri.x * ri.x + ri.y * ri.y;
              quad_out(q, kPlaneStride, rr, ri);
            }
          }
          rsq += (double)ss;
          if (p.xs) {
            // the solution step of the same iteration, x_s += alpha p
            const V2 pa = bc<V2>((C)p.rs_alpha[(long long)rhs * p.rs_alpha_stride]);
            rvec *xb = reinterpret_cast<rvec *>(p.xs) + (long long)rhs * p.rs_stride +
                       site_off(xf, s0 + j, Ls, RNPV);
            const vec *pb = reinterpret_cast<const vec *>(p.pdir) +
                            (long long)rhs * p.rhs_stride + site_off(xf, s0 + j, Ls, PNPV);
#pragma unroll
            for (int q = 0; q < 6; ++q) {
              V2 pr_, pi_, xr, xi;
              quad_in(pr_, pi_, pb + (long long)q * PVPQ * kPlaneStride, kPlaneStride);
              quad_in(xr, xi, xb + (long long)q * RVPQ * kPlaneStride, kPlaneStride);
              xr = p_fma(pa, pr_, xr);
              xi = p_fma(pa, pi_, xi);
              quad_out(xb + (long long)q * RVPQ * kPlaneStride, kPlaneStride, xr, xi);
            }
          }
        } else {
          store(j, o);
        }
      };
      if (p.own) {
        roll_5d<P, true, SPT>(Fo, xf, s0, Ls, alpha, beta, mf, emit);
      } else {
        Spinor<V2> zero_v;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          zero_v.up.re[cc] = zero_v.up.im[cc] = zero_v.lo.re[cc] = zero_v.lo.im[cc] = bc<V2>(C(0));
        }
#pragma unroll
        for (int j = 0; j < SPT; ++j) emit(j, zero_v);
      }
    }
    if (p.rs) {
      // fixed-order block sum of |r_s|^2, as for the norm of the D pass
      __shared__ double rs_warp[32];
      const int tid = threadIdx.y * blockDim.x + threadIdx.x;
      const int nwarps = (blockDim.x * blockDim.y + 31) / 32;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) rsq += __shfl_down_sync(0xffffffffu, rsq, o);
      if ((tid & 31) == 0) rs_warp[tid >> 5] = rsq;
      __syncthreads();
      if (tid < 32) {
        double v = tid < nwarps ? rs_warp[tid] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (tid == 0) p.rs_partials[(long long)rhs * ctas_per_rhs + cta_in_rhs] = v;
      }
    }
    // the other CTAs of the cluster may still read this CTA's edges
    if (clustered) cooperative_groups::this_cluster().sync();
  }
}

template <class P, int OP, int SPT, int VAR, bool CB, bool GLX>
__global__ void dslash_kernel(const DslashParams p) {
  dslash_body<P, OP, SPT, VAR, CB, GLX>(p);
}

template <class P, int OP, int SPT, int VAR, bool CB, bool GLX>
__global__ void __maxnreg__(RegCap<VAR>::value) dslash_kernel_capped(const DslashParams p) {
  dslash_body<P, OP, SPT, VAR, CB, GLX>(p);
}

// The kernel entry of (P, OP, SPT, VAR, CB, GLX): variants 4, 6, 7 are register
// capped.
template <class P, int OP, int SPT, int VAR, bool CB = false, bool GLX = false>
constexpr void (*dslash_entry())(const DslashParams) {
  if constexpr (RegCap<VAR>::value > 0)
    return dslash_kernel_capped<P, OP, SPT, VAR, CB, GLX>;
  else
    return dslash_kernel<P, OP, SPT, VAR, CB, GLX>;
}

template <class P, int OP, int SPT, int VAR>
size_t dslash_smem(int tx, int nchunk) {
  size_t smem = 0;
  if (VAR == 1) smem += kStages * StageLayout<P, OP == OP_D, SPT>::stage_bytes(tx * nchunk);
  if (VAR == 6 || VAR == 7) smem += rows_smem_bytes(tx, nchunk * SPT, P::id, OP);
  if (OP == OP_DDAG) smem += 2 * (size_t)nchunk * 12 * tx * sizeof(typename P::C);  // 6 pairs
  return smem;
}

template <class P, int OP, int SPT, int VAR, bool CB, bool GLX>
int launch_one_k(const DslashParams &p, int tx, int zblk, int sgrp, cudaStream_t st) {
  // D^+ exchanges slice-group edges through shared memory: the sgrp CTAs of a
  // tile run as one thread-block cluster (at most 8, the portable size), the
  // RHS outermost so that a cluster never spans two right-hand sides
  constexpr bool kClusterOp = (OP == OP_DDAG);
  if (sgrp < 1 || (p.Ls / SPT) % sgrp || (kClusterOp && sgrp > 8)) return -2;
  // checkerboard launches: register variants only, Lx even, no halos
  if (CB && ((VAR != 0 && VAR != 4 && VAR != 5) || (p.L[0] & 1) || p.halo_up || p.halo_dn))
    return -2;
  const int nchunk = p.Ls / SPT / sgrp;
  dim3 block(tx, nchunk);
  DslashParams q = p;
  const int plane_sites = (CB ? p.L[0] / 2 : p.L[0]) * p.L[1];
  // variant 7: one CTA per plane (it walks the plane's tiles itself)
  q.tiles_per_plane = VAR == 7 ? 1 : (plane_sites + tx - 1) / tx;
  q.zblk = zblk;
  q.sgrp = sgrp;
  if (kClusterOp && sgrp > 1) q.rhs_outer = 1;
  if (zblk < 1 || p.L[2] % zblk) return -2;
  // (D: the local term is taken from the staged rows, so own must be in)
  if ((VAR == 6 || VAR == 7) && (!rows_variant_ok(OP, p.L[0], p.L[1], tx) || p.halo_up ||
                                 p.halo_dn || (OP == OP_D && p.own != p.in)))
    return -2;
  if (q.t_count == 0) {
    q.t_begin = 0;
    q.t_count = p.L[3];
  }
  if (q.t_begin < 0 || q.t_count < 1 || q.t_begin + q.t_count > p.L[3]) return -2;
  dim3 grid((unsigned)((long long)q.tiles_per_plane * sgrp * p.L[2] * q.t_count * p.nrhs));
  const size_t smem = dslash_smem<P, OP, SPT, VAR>(tx, nchunk);
  // per-instantiation launch limits, queried once; the dynamic shared memory
  // a launch may use without raising the kernel's limit is 48 KB less the
  // kernel's static shared memory
  static int max_threads = 0;
  static size_t static_smem = 0;
  static size_t smem_set = 0;
  if (!max_threads) {
    cudaFuncAttributes fa;
    const cudaError_t e = cudaFuncGetAttributes(&fa, dslash_entry<P, OP, SPT, VAR, CB, GLX>());
    if (e != cudaSuccess) {
      last_launch_error() = e;
      return -1;
    }
    static_smem = fa.sharedSizeBytes;
    smem_set = 48 * 1024 > static_smem ? 48 * 1024 - static_smem : 0;
    max_threads = fa.maxThreadsPerBlock;
  }
  if (tx < 32 || tx % 32 || tx * nchunk > max_threads) return -3;
  if (smem + static_smem > 227 * 1024) return -3;
  if (smem > smem_set) {
    if (cudaFuncSetAttribute(dslash_entry<P, OP, SPT, VAR, CB, GLX>(),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return -3;
    smem_set = smem;
  }
  cudaError_t e;
  if (kClusterOp && sgrp > 1) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = grid;
    lc.blockDim = block;
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)sgrp;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    e = cudaLaunchKernelEx(&lc, dslash_entry<P, OP, SPT, VAR, CB, GLX>(), q);
    if (e == cudaSuccess) e = cudaGetLastError();
  } else {
    dslash_entry<P, OP, SPT, VAR, CB, GLX>()<<<grid, block, smem, st>>>(q);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) return 0;
  last_launch_error() = e;
  return -1;
}

// Variants 6 and 7 take their general-Lx form unless Lx = 32.
template <class P, int OP, int SPT, int VAR, bool CB = false>
int launch_one(const DslashParams &p, int tx, int zblk, int sgrp, cudaStream_t st) {
  if constexpr (VAR == 6 || VAR == 7) {
    if (p.L[0] != 32) return launch_one_k<P, OP, SPT, VAR, CB, true>(p, tx, zblk, sgrp, st);
  }
  return launch_one_k<P, OP, SPT, VAR, CB, false>(p, tx, zblk, sgrp, st);
}

template <class P, int OP, int VAR, bool CB = false>
int launch_spt(const DslashParams &p, TileConfig cfg, cudaStream_t st) {
  switch (cfg.spt) {
    case 1: return launch_one<P, OP, 1, VAR, CB>(p, cfg.tx, cfg.zblk, cfg.sgrp, st);
    case 2: return launch_one<P, OP, 2, VAR, CB>(p, cfg.tx, cfg.zblk, cfg.sgrp, st);
    case 3: return launch_one<P, OP, 3, VAR, CB>(p, cfg.tx, cfg.zblk, cfg.sgrp, st);
    case 4: return launch_one<P, OP, 4, VAR, CB>(p, cfg.tx, cfg.zblk, cfg.sgrp, st);
    default: return -2;
  }
}

template <class P, int OP, int VAR>
int max_threads_var(int spt) {
  cudaFuncAttributes fa;
  cudaError_t e;
  switch (spt) {
    case 1: e = cudaFuncGetAttributes(&fa, dslash_entry<P, OP, 1, VAR>()); break;
    case 2: e = cudaFuncGetAttributes(&fa, dslash_entry<P, OP, 2, VAR>()); break;
    case 3: e = cudaFuncGetAttributes(&fa, dslash_entry<P, OP, 3, VAR>()); break;
    case 4: e = cudaFuncGetAttributes(&fa, dslash_entry<P, OP, 4, VAR>()); break;
    default: return 0;
  }
  return e == cudaSuccess ? fa.maxThreadsPerBlock : 0;
}

// Largest CTA that (op, spt) of variant VAR can launch: register limit and, for
// the staged variant, the 227 KB shared-memory limit.
template <class P, int OP, int VAR>
int max_threads_op(int spt) {
  int m = max_threads_var<P, OP, VAR>(spt);
  if (VAR != 1) return m;
  m -= m % 32;
  while (m >= 32) {
    size_t smem = 0;
    switch (spt) {
      case 1: smem = kStages * StageLayout<P, OP == OP_D, 1>::stage_bytes(m); break;
      case 2: smem = kStages * StageLayout<P, OP == OP_D, 2>::stage_bytes(m); break;
      case 3: smem = kStages * StageLayout<P, OP == OP_D, 3>::stage_bytes(m); break;
      case 4: smem = kStages * StageLayout<P, OP == OP_D, 4>::stage_bytes(m); break;
    }
    if (OP == OP_DDAG) smem += (size_t)m * 24 * sizeof(typename P::C);
    if (smem <= 227 * 1024) break;
    m -= 32;
  }
  return m < 32 ? 0 : m;
}

// Entry points of one (precision, variant) translation unit.
template <class P, int VAR>
int launch_variant(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st) {
  if (cfg.spt < 1 || p.Ls % cfg.spt) return -2;
  switch (op) {
    case OP_DHOP: return launch_spt<P, OP_DHOP, VAR>(p, cfg, st);
    case OP_DHOP_DAG: return launch_spt<P, OP_DHOP_DAG, VAR>(p, cfg, st);
    case OP_D: return launch_spt<P, OP_D, VAR>(p, cfg, st);
    case OP_DDAG: return launch_spt<P, OP_DDAG, VAR>(p, cfg, st);
  }
  return -2;
}

// Interleaved-complex FP32 entry points (layout ablation): Dhop and Dhop^+.
template <int VAR>
int launch_variant_cplx(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st) {
  if (cfg.spt < 1 || p.Ls % cfg.spt) return -2;
  switch (op) {
    case OP_DHOP: return launch_spt<F32C, OP_DHOP, VAR>(p, cfg, st);
    case OP_DHOP_DAG: return launch_spt<F32C, OP_DHOP_DAG, VAR>(p, cfg, st);
  }
  return -2;
}

// Checkerboard entry points (the D and D^+ forms; Dhop is D with b = 1,
// c = 0, no local term and factor 1).
template <class P, int VAR>
int launch_variant_cb(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st) {
  if (cfg.spt < 1 || p.Ls % cfg.spt) return -2;
  switch (op) {
    case OP_D: return launch_spt<P, OP_D, VAR, true>(p, cfg, st);
    case OP_DDAG: return launch_spt<P, OP_DDAG, VAR, true>(p, cfg, st);
  }
  return -2;
}

template <class P, int VAR>
int max_threads_variant(int op, int spt) {
  switch (op) {
    case OP_DHOP: return max_threads_op<P, OP_DHOP, VAR>(spt);
    case OP_DHOP_DAG: return max_threads_op<P, OP_DHOP_DAG, VAR>(spt);
    case OP_D: return max_threads_op<P, OP_D, VAR>(spt);
    case OP_DDAG: return max_threads_op<P, OP_DDAG, VAR>(spt);
  }
  return 0;
}

}  // namespace dw

// One translation unit per (precision, variant) keeps the builds parallel.
#define DW_DSLASH_INSTANTIATE(PREC, VAR)                                                  \
  namespace dw {                                                                         \
  int launch_dslash_##PREC##_v##VAR(const DslashParams &p, int op, TileConfig cfg,       \
                                    cudaStream_t st) {                                   \
    return launch_variant<PREC, VAR>(p, op, cfg, st);                                    \
  }                                                                                      \
  int dslash_max_threads_##PREC##_v##VAR(int op, int spt) {                              \
    return max_threads_variant<PREC, VAR>(op, spt);                                      \
  }                                                                                      \
  }

// Checkerboard stencil of one (precision, variant).
#define DW_DSLASH_CB_INSTANTIATE(PREC, VAR)                                               \
  namespace dw {                                                                         \
  int launch_dslash_cb_##PREC(const DslashParams &p, int op, TileConfig cfg,             \
                              cudaStream_t st) {                                         \
    return launch_variant_cb<PREC, VAR>(p, op, cfg, st);                                 \
  }                                                                                      \
  }

// Interleaved-complex stencil of one variant.
#define DW_DSLASH_CPLX_INSTANTIATE(VAR)                                                   \
  namespace dw {                                                                         \
  int launch_dslash_cplx_v##VAR(const DslashParams &p, int op, TileConfig cfg,           \
                                cudaStream_t st) {                                       \
    return launch_variant_cplx<VAR>(p, op, cfg, st);                                     \
  }                                                                                      \
  }

// Face packing for the t decomposition, one translation unit per precision.
#define DW_HALO_INSTANTIATE(PREC)                                                         \
  namespace dw {                                                                         \
  int launch_halo_pack_##PREC(const DslashParams &p, void *send_dn, void *send_up, int op,  \
                              cudaStream_t st) {                                         \
    return launch_halo_pack_impl<PREC>(p, send_dn, send_up, op, st);                     \
  }                                                                                      \
  }

// The Domain Wall kernel: 4D Wilson hopping term over all fifth-dimension
// slices (Sec. 4.1; per-site spin projection, SU(3) x half spinor and
// reconstruction, Table 3), fused with the 5D hop and diagonal terms of the
// Shamir / Moebius operator.
//
// Work decomposition.  A CTA owns `tx` consecutive 4D sites and all Ls slices;
// thread (x, y) handles 4D site x4 = blockIdx.x*tx + x and the `SPT`
// consecutive slices s0 = y*SPT .. s0+SPT-1 of right-hand side blockIdx.y.
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

#include "dw_common.cuh"

namespace dw {

// h index: (spin j * 3 + colour) * 2 + re/im, j in {0, 1}.
#define RE(a, j, c) a[((j)*3 + (c)) * 2]
#define IM(a, j, c) a[((j)*3 + (c)) * 2 + 1]

template <int MU, int S, class C>
__device__ __forceinline__ void project(C *h, const C *u, const C *l) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (MU == 0) {  // e l = (i l1, i l0)
      RE(h, 0, c) = RE(u, 0, c) - S * IM(l, 1, c);
      IM(h, 0, c) = IM(u, 0, c) + S * RE(l, 1, c);
      RE(h, 1, c) = RE(u, 1, c) - S * IM(l, 0, c);
      IM(h, 1, c) = IM(u, 1, c) + S * RE(l, 0, c);
    } else if (MU == 1) {  // e l = (l1, -l0)
      RE(h, 0, c) = RE(u, 0, c) + S * RE(l, 1, c);
      IM(h, 0, c) = IM(u, 0, c) + S * IM(l, 1, c);
      RE(h, 1, c) = RE(u, 1, c) - S * RE(l, 0, c);
      IM(h, 1, c) = IM(u, 1, c) - S * IM(l, 0, c);
    } else if (MU == 2) {  // e l = (i l0, -i l1)
      RE(h, 0, c) = RE(u, 0, c) - S * IM(l, 0, c);
      IM(h, 0, c) = IM(u, 0, c) + S * RE(l, 0, c);
      RE(h, 1, c) = RE(u, 1, c) + S * IM(l, 1, c);
      IM(h, 1, c) = IM(u, 1, c) - S * RE(l, 1, c);
    } else {  // e l = (l0, l1)
      RE(h, 0, c) = RE(u, 0, c) + S * RE(l, 0, c);
      IM(h, 0, c) = IM(u, 0, c) + S * IM(l, 0, c);
      RE(h, 1, c) = RE(u, 1, c) + S * RE(l, 1, c);
      IM(h, 1, c) = IM(u, 1, c) + S * IM(l, 1, c);
    }
  }
}

// acc (24 reals: upper spins 0..11, lower spins 12..23) += (w, S e_mu^+ w).
template <int MU, int S, bool FIRST, class C>
__device__ __forceinline__ void reconstruct(C *acc, const C *w) {
  C *up = acc;
  C *lo = acc + 12;
#pragma unroll
  for (int i = 0; i < 12; ++i) up[i] = FIRST ? w[i] : up[i] + w[i];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    C r0, i0, r1, i1;  // lower spin 0 and 1 increments
    if (MU == 0) {  // e^+ w = (-i w1, -i w0)
      r0 = S * IM(w, 1, c);
      i0 = -S * RE(w, 1, c);
      r1 = S * IM(w, 0, c);
      i1 = -S * RE(w, 0, c);
    } else if (MU == 1) {  // e^+ w = (-w1, w0)
      r0 = -S * RE(w, 1, c);
      i0 = -S * IM(w, 1, c);
      r1 = S * RE(w, 0, c);
      i1 = S * IM(w, 0, c);
    } else if (MU == 2) {  // e^+ w = (-i w0, i w1)
      r0 = S * IM(w, 0, c);
      i0 = -S * RE(w, 0, c);
      r1 = -S * IM(w, 1, c);
      i1 = S * RE(w, 1, c);
    } else {  // e^+ w = (w0, w1)
      r0 = S * RE(w, 0, c);
      i0 = S * IM(w, 0, c);
      r1 = S * RE(w, 1, c);
      i1 = S * IM(w, 1, c);
    }
    if (FIRST) {
      RE(lo, 0, c) = r0;
      IM(lo, 0, c) = i0;
      RE(lo, 1, c) = r1;
      IM(lo, 1, c) = i1;
    } else {
      RE(lo, 0, c) += r0;
      IM(lo, 0, c) += i0;
      RE(lo, 1, c) += r1;
      IM(lo, 1, c) += i1;
    }
  }
}

// w = U h (ADJ = false) or U^+ h (ADJ = true) for both spins; U is 18 reals,
// index (row * 3 + col) * 2 + re/im.
template <bool ADJ, class C>
__device__ __forceinline__ void su3_mul(C *w, const C *U, const C *h) {
#pragma unroll
  for (int j = 0; j < 2; ++j) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      C re = 0, im = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int idx = ADJ ? (k * 3 + r) : (r * 3 + k);
        const C ur = U[idx * 2], ui = U[idx * 2 + 1];
        const C hr = RE(h, j, k), hi = IM(h, j, k);
        if (!ADJ) {
          re += ur * hr - ui * hi;
          im += ur * hi + ui * hr;
        } else {
          re += ur * hr + ui * hi;
          im += ur * hi - ui * hr;
        }
      }
      RE(w, j, r) = re;
      IM(w, j, r) = im;
    }
  }
}

#undef RE
#undef IM

template <class P>
struct Field {
  using vec = typename P::vec;
  using C = typename P::C;
  static constexpr int NHP = 12 / P::R;  // vecs per half spinor
  const vec *base;
  long long plane;
  int V4;
  // 12 reals of the upper (half = 0) or lower (half = 1) spins at (x4, s).
  __device__ __forceinline__ void load_half(C *h, int x4, int s, int half) const {
    const vec *p = base + (long long)half * NHP * plane + (long long)s * V4 + x4;
#pragma unroll
    for (int q = 0; q < NHP; ++q) load_vec<P>(h + q * P::R, p + q * plane);
  }
};

template <class P>
__device__ __forceinline__ void load_link(typename P::C *U, const typename P::vec *gmain,
                                          const typename P::tvec *gtail, int mu, int x4,
                                          int V4) {
  constexpr int NM = 16 / P::R;
  const typename P::vec *p = gmain + (long long)mu * NM * V4 + x4;
#pragma unroll
  for (int q = 0; q < NM; ++q) widen(__ldg(p + (long long)q * V4), U + q * P::R);
  widen_t(__ldg(gtail + (long long)mu * V4 + x4), U + 16);
}

// Rolling evaluation of A psi_s + B [K psi]_s (KDAG = false) or
// A psi_s + B [K^+ psi]_s (KDAG = true) at 4D site x4 for s = s0 .. s0+SPT-1.
//   K:   upper from s-1, lower from s+1;  K^+: upper from s+1, lower from s-1;
//   a neighbour index that leaves [0, Ls) wraps and carries -mf.
// Calls f(j, v) with the 24 reals of slice s0 + j.  Each half spinor is loaded
// once: 2 (SPT + 1) half-spinor loads for SPT slices.
template <class P, bool KDAG, int SPT, class Fn>
__device__ __forceinline__ void roll_5d(const Field<P> &F, int x4, int s0, int Ls,
                                        typename P::C A, typename P::C B,
                                        typename P::C mf, Fn &&f) {
  using C = typename P::C;
  // "carry" half: the one whose partner slice is below s (s - 1)
  //   K:   upper(s-1) is carried; lower(s+1) is loaded ahead.
  //   K^+: lower(s-1) is carried; upper(s+1) is loaded ahead.
  const int carry_half = KDAG ? 1 : 0;
  const int ahead_half = KDAG ? 0 : 1;
  C prev[12], cur_ahead[12];
  {
    int sp = s0 - 1;
    C f0 = 1;
    if (sp < 0) {
      sp = Ls - 1;
      f0 = -mf;
    }
    F.load_half(prev, x4, sp, carry_half);
#pragma unroll
    for (int i = 0; i < 12; ++i) prev[i] *= f0;
    F.load_half(cur_ahead, x4, s0, ahead_half);  // the ahead half at s itself
  }
#pragma unroll
  for (int j = 0; j < SPT; ++j) {
    const int s = s0 + j;
    C cur_carry[12], next_ahead[12];
    F.load_half(cur_carry, x4, s, carry_half);
    int sn = s + 1;
    C fn = 1;
    if (sn == Ls) {
      sn = 0;
      fn = -mf;
    }
    F.load_half(next_ahead, x4, sn, ahead_half);
    C v[24];
    C *vc = v + 12 * carry_half;
    C *va = v + 12 * ahead_half;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      vc[i] = A * cur_carry[i] + B * prev[i];
      va[i] = A * cur_ahead[i] + (B * fn) * next_ahead[i];
    }
    f(j, v);
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      prev[i] = cur_carry[i];
      cur_ahead[i] = next_ahead[i];
    }
  }
}

// One hop direction: acc[j] += (1 + S g_mu) W psi'(y4, s0 + j) for every j,
// where W = U_mu(l4) (ADJ = false) or U_mu(l4)^+ (ADJ = true) and psi' is psi
// itself (PHI = false) or phi = (b + cK) psi (PHI = true).
template <class P, int MU, int S, bool ADJ, bool PHI, bool FIRST, int SPT>
__device__ __forceinline__ void hop_dir(typename P::C (&acc)[SPT][24], const Field<P> &F,
                                        const typename P::vec *gmain,
                                        const typename P::tvec *gtail, int y4, int l4, int s0,
                                        int Ls, typename P::C b, typename P::C c,
                                        typename P::C mf) {
  using C = typename P::C;
  C U[18];
  load_link<P>(U, gmain, gtail, MU, l4, F.V4);
  auto body = [&](int j, const C *v) {
    C h[12], w[12];
    project<MU, S>(h, v, v + 12);
    su3_mul<ADJ>(w, U, h);
    reconstruct<MU, S, FIRST>(acc[j], w);
  };
  if (PHI) {
    roll_5d<P, false, SPT>(F, y4, s0, Ls, b, c, mf, body);
  } else {
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
      C v[24];
      F.load_half(v, y4, s0 + j, 0);
      F.load_half(v + 12, y4, s0 + j, 1);
      body(j, v);
    }
  }
}

template <class P, int OP, int SPT>
__global__ void dslash_kernel(const DslashParams p) {
  using C = typename P::C;
  using vec = typename P::vec;
  using tvec = typename P::tvec;
  constexpr bool DAG = (OP == OP_DHOP_DAG || OP == OP_DDAG);
  constexpr bool PHI = (OP == OP_D);
  constexpr int SF = DAG ? 1 : -1;  // sign S of the forward hop
  constexpr int SB = -SF;           // sign S of the backward hop
  constexpr int NHP = 12 / P::R;

  const int tx = blockDim.x;
  const int x4 = blockIdx.x * tx + threadIdx.x;
  const int chunk = threadIdx.y;
  const int nchunk = blockDim.y;
  const int rhs = blockIdx.y;
  if (p.gate && !p.gate[(long long)rhs * p.gate_stride]) return;  // whole CTA: uniform
  const bool active = x4 < p.V4;
  const int s0 = chunk * SPT;
  const int Ls = p.Ls;

  Field<P> F;
  F.base = reinterpret_cast<const vec *>(p.in) + (long long)rhs * p.rhs_stride;
  F.plane = p.plane;
  F.V4 = p.V4;
  vec *out = reinterpret_cast<vec *>(p.out) + (long long)rhs * p.rhs_stride;
  const vec *gmain = reinterpret_cast<const vec *>(p.gmain);
  const tvec *gtail = reinterpret_cast<const tvec *>(p.gtail);

  const C mf = (OP == OP_D || OP == OP_DDAG) ? (C)p.mf[rhs] : C(0);
  const C b = (C)p.b, c = (C)p.c;
  const C alpha = (C)(p.b * (4.0 - p.M5) + 1.0);
  const C beta = (C)(p.c * (4.0 - p.M5) - 1.0);

  C acc[SPT][24];

  if (active) {
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
    const int xf = (cx == p.L[0] - 1) ? x4 - (p.L[0] - 1) : x4 + 1;
    const int xb = (cx == 0) ? x4 + (p.L[0] - 1) : x4 - 1;
    const int yf = (cy == p.L[1] - 1) ? x4 - (p.L[1] - 1) * st1 : x4 + st1;
    const int yb = (cy == 0) ? x4 + (p.L[1] - 1) * st1 : x4 - st1;
    const int zf = (cz == p.L[2] - 1) ? x4 - (p.L[2] - 1) * st2 : x4 + st2;
    const int zb = (cz == 0) ? x4 + (p.L[2] - 1) * st2 : x4 - st2;
    const int tf = (ct == p.L[3] - 1) ? x4 - (p.L[3] - 1) * st3 : x4 + st3;
    const int tb = (ct == 0) ? x4 + (p.L[3] - 1) * st3 : x4 - st3;

    hop_dir<P, 0, SF, false, PHI, true, SPT>(acc, F, gmain, gtail, xf, x4, s0, Ls, b, c, mf);
    hop_dir<P, 0, SB, true, PHI, false, SPT>(acc, F, gmain, gtail, xb, xb, s0, Ls, b, c, mf);
    hop_dir<P, 1, SF, false, PHI, false, SPT>(acc, F, gmain, gtail, yf, x4, s0, Ls, b, c, mf);
    hop_dir<P, 1, SB, true, PHI, false, SPT>(acc, F, gmain, gtail, yb, yb, s0, Ls, b, c, mf);
    hop_dir<P, 2, SF, false, PHI, false, SPT>(acc, F, gmain, gtail, zf, x4, s0, Ls, b, c, mf);
    hop_dir<P, 2, SB, true, PHI, false, SPT>(acc, F, gmain, gtail, zb, zb, s0, Ls, b, c, mf);
    hop_dir<P, 3, SF, false, PHI, false, SPT>(acc, F, gmain, gtail, tf, x4, s0, Ls, b, c, mf);
    hop_dir<P, 3, SB, true, PHI, false, SPT>(acc, F, gmain, gtail, tb, tb, s0, Ls, b, c, mf);
  }

  auto store = [&](int j, const C *v) {
    vec *o = out + (long long)(s0 + j) * p.V4 + x4;
#pragma unroll
    for (int q = 0; q < 2 * NHP; ++q) store_vec<P>(o + q * p.plane, v + q * P::R);
  };

  if (OP == OP_DHOP || OP == OP_DHOP_DAG) {
    if (active) {
#pragma unroll
      for (int j = 0; j < SPT; ++j) store(j, acc[j]);
    }
  } else if (OP == OP_D) {
    // out = alpha psi + beta K psi - 1/2 Dhop phi
    if (active) {
      roll_5d<P, false, SPT>(F, x4, s0, Ls, alpha, beta, mf, [&](int j, const C *v) {
        C o[24];
#pragma unroll
        for (int i = 0; i < 24; ++i) o[i] = v[i] - C(0.5) * acc[j][i];
        store(j, o);
      });
    }
  } else {
    // OP_DDAG: out = alpha psi + beta K^+ psi - 1/2 (b + c K^+) Dhop^+ psi.
    // K^+ acc needs the upper spins of slice s+1 and the lower spins of s-1;
    // at chunk edges they come from the neighbouring chunk through shared memory.
    extern __shared__ unsigned char smem_raw[];
    C *sm_up = reinterpret_cast<C *>(smem_raw);    // [nchunk][12][tx]
    C *sm_lo = sm_up + (size_t)nchunk * 12 * tx;   // [nchunk][12][tx]
    const int t = threadIdx.x;
    if (active) {
#pragma unroll
      for (int i = 0; i < 12; ++i) {
        sm_up[((size_t)chunk * 12 + i) * tx + t] = acc[0][i];
        sm_lo[((size_t)chunk * 12 + i) * tx + t] = acc[SPT - 1][12 + i];
      }
    }
    __syncthreads();
    if (active) {
      const int cn = (chunk + 1 == nchunk) ? 0 : chunk + 1;
      const int cp = (chunk == 0) ? nchunk - 1 : chunk - 1;
      const C fn = (chunk + 1 == nchunk) ? -mf : C(1);
      const C fp = (chunk == 0) ? -mf : C(1);
      roll_5d<P, true, SPT>(F, x4, s0, Ls, alpha, beta, mf, [&](int j, const C *v) {
        C o[24];
#pragma unroll
        for (int i = 0; i < 12; ++i) {
          // upper: (K^+ acc)_s = acc_up(s+1)
          C kup = (j + 1 < SPT) ? acc[(j + 1 < SPT) ? j + 1 : 0][i]
                                : fn * sm_up[((size_t)cn * 12 + i) * tx + t];
          // lower: (K^+ acc)_s = acc_lo(s-1)
          C klo = (j > 0) ? acc[(j > 0) ? j - 1 : 0][12 + i]
                          : fp * sm_lo[((size_t)cp * 12 + i) * tx + t];
          o[i] = v[i] - C(0.5) * (b * acc[j][i] + c * kup);
          o[12 + i] = v[12 + i] - C(0.5) * (b * acc[j][12 + i] + c * klo);
        }
        store(j, o);
      });
    }
  }
}

template <class P, int OP, int SPT>
int launch_one(const DslashParams &p, int tx, cudaStream_t st) {
  const int nchunk = p.Ls / SPT;
  dim3 block(tx, nchunk);
  dim3 grid((p.V4 + tx - 1) / tx, p.nrhs);
  size_t smem = 0;
  if (OP == OP_DDAG) smem = 2 * (size_t)nchunk * 12 * tx * sizeof(typename P::C);
  // per-instantiation launch limits, queried once
  static int max_threads = 0;
  static size_t smem_set = 48 * 1024;
  if (!max_threads) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, dslash_kernel<P, OP, SPT>) != cudaSuccess) return -1;
    max_threads = fa.maxThreadsPerBlock;
  }
  if (tx < 32 || tx % 32 || tx * nchunk > max_threads) return -3;
  if (smem > smem_set) {
    if (cudaFuncSetAttribute(dslash_kernel<P, OP, SPT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return -3;
    smem_set = smem;
  }
  dslash_kernel<P, OP, SPT><<<grid, block, smem, st>>>(p);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <class P, int OP>
int launch_op(const DslashParams &p, TileConfig cfg, cudaStream_t st) {
  switch (cfg.spt) {
    case 1: return launch_one<P, OP, 1>(p, cfg.tx, st);
    case 2: return launch_one<P, OP, 2>(p, cfg.tx, st);
    case 3: return launch_one<P, OP, 3>(p, cfg.tx, st);
    case 4: return launch_one<P, OP, 4>(p, cfg.tx, st);
    default: return -2;
  }
}

template <class P, int OP>
int max_threads_op(int spt) {
  cudaFuncAttributes fa;
  cudaError_t e;
  switch (spt) {
    case 1: e = cudaFuncGetAttributes(&fa, dslash_kernel<P, OP, 1>); break;
    case 2: e = cudaFuncGetAttributes(&fa, dslash_kernel<P, OP, 2>); break;
    case 3: e = cudaFuncGetAttributes(&fa, dslash_kernel<P, OP, 3>); break;
    case 4: e = cudaFuncGetAttributes(&fa, dslash_kernel<P, OP, 4>); break;
    default: return 0;
  }
  return e == cudaSuccess ? fa.maxThreadsPerBlock : 0;
}

template <class P>
int max_threads_impl(int op, int spt) {
  switch (op) {
    case OP_DHOP: return max_threads_op<P, OP_DHOP>(spt);
    case OP_DHOP_DAG: return max_threads_op<P, OP_DHOP_DAG>(spt);
    case OP_D: return max_threads_op<P, OP_D>(spt);
    case OP_DDAG: return max_threads_op<P, OP_DDAG>(spt);
  }
  return 0;
}

template <class P>
int launch_dslash_impl(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st) {
  if (cfg.spt < 1 || p.Ls % cfg.spt) return -2;
  switch (op) {
    case OP_DHOP: return launch_op<P, OP_DHOP>(p, cfg, st);
    case OP_DHOP_DAG: return launch_op<P, OP_DHOP_DAG>(p, cfg, st);
    case OP_D: return launch_op<P, OP_D>(p, cfg, st);
    case OP_DDAG: return launch_op<P, OP_DDAG>(p, cfg, st);
    default: return -2;
  }
}

}  // namespace dw

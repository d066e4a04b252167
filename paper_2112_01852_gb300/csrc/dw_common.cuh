// Common definitions of the GB300 domain-wall library: precision traits, vector
// load/convert helpers and the kernel parameter blocks (the lattice object is
// host-side only: dw_api_internal.cuh).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "dw.h"

namespace dw {

// ---------------------------------------------------------------------------
// Precision traits.  A fermion plane element is one `vec`: 2 doubles (F64),
// 4 floats (F32) or 4 halves (F16).  `C` is the arithmetic type.
// A link is NLV vecs: all 18 reals at FP64; at FP32 / FP16 only its first two
// rows (12 reals), the third being rebuilt as conj(row0 x row1) (SU(3)).
struct F64 {
  using vec = double2;
  using C = double;
  static constexpr int R = 2;
  static constexpr int RB = 8;  // bytes per real
  static constexpr int NLV = 9;
  static constexpr bool LINK12 = false;
  static constexpr bool CPLX = false;
  static constexpr int id = DW_F64;
};
struct F32 {
  using vec = float4;
  using C = float;
  static constexpr int R = 4;
  static constexpr int RB = 4;
  static constexpr int NLV = 3;
  static constexpr bool LINK12 = true;
  static constexpr bool CPLX = false;
  static constexpr int id = DW_F32;
};
// FP32 storage with interleaved-complex quads (Re j0, Im j0, Re j1, Im j1) and
// complex-form arithmetic: the layout ablation (dw_set_complex_layout).
struct F32C : F32 {
  static constexpr bool CPLX = true;
};
struct F16 {
  using vec = uint2;  // 4 x binary16
  using C = float;
  static constexpr int R = 4;
  static constexpr int RB = 2;
  static constexpr int NLV = 3;
  static constexpr bool LINK12 = true;
  static constexpr bool CPLX = false;
  static constexpr int id = DW_F16;
};
inline int prec_link_vecs(int prec) { return prec == DW_F64 ? 9 : 3; }

inline int prec_vec_bytes(int prec) { return prec == DW_F64 ? 16 : (prec == DW_F32 ? 16 : 8); }
inline int prec_reals_per_vec(int prec) { return prec == DW_F64 ? 2 : 4; }
inline int prec_real_bytes(int prec) { return prec == DW_F64 ? 8 : (prec == DW_F32 ? 4 : 2); }

// ---------------------------------------------------------------------------
// Device helpers: load a vec through the read-only path and widen to C.
__device__ __forceinline__ void widen(const double2 &v, double *r) {
  r[0] = v.x;
  r[1] = v.y;
}
__device__ __forceinline__ void widen(const float4 &v, float *r) {
  r[0] = v.x;
  r[1] = v.y;
  r[2] = v.z;
  r[3] = v.w;
}
__device__ __forceinline__ void widen(const uint2 &v, float *r) {
  __half2 a = *reinterpret_cast<const __half2 *>(&v.x);
  __half2 b = *reinterpret_cast<const __half2 *>(&v.y);
  float2 fa = __half22float2(a);
  float2 fb = __half22float2(b);
  r[0] = fa.x;
  r[1] = fa.y;
  r[2] = fb.x;
  r[3] = fb.y;
}

__device__ __forceinline__ double2 narrow_vec(const double *r, double2 *) {
  return make_double2(r[0], r[1]);
}
__device__ __forceinline__ float4 narrow_vec(const float *r, float4 *) {
  return make_float4(r[0], r[1], r[2], r[3]);
}
__device__ __forceinline__ uint2 narrow_vec(const float *r, uint2 *) {
  __half2 a = __floats2half2_rn(r[0], r[1]);
  __half2 b = __floats2half2_rn(r[2], r[3]);
  uint2 v;
  v.x = *reinterpret_cast<unsigned int *>(&a);
  v.y = *reinterpret_cast<unsigned int *>(&b);
  return v;
}
// Rounding straight from double (one rounding step, nearest even) for the
// layout converters that read canonical FP64 data.
__device__ __forceinline__ double2 narrow_from_f64(const double *r, double2 *) {
  return make_double2(r[0], r[1]);
}
__device__ __forceinline__ float4 narrow_from_f64(const double *r, float4 *) {
  return make_float4((float)r[0], (float)r[1], (float)r[2], (float)r[3]);
}
__device__ __forceinline__ uint2 narrow_from_f64(const double *r, uint2 *) {
  __half h[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) h[k] = __double2half(r[k]);
  uint2 v;
  v.x = (unsigned)__half_as_ushort(h[0]) | ((unsigned)__half_as_ushort(h[1]) << 16);
  v.y = (unsigned)__half_as_ushort(h[2]) | ((unsigned)__half_as_ushort(h[3]) << 16);
  return v;
}
template <class P>
__device__ __forceinline__ void load_vec(typename P::C *r, const typename P::vec *p) {
  widen(__ldg(p), r);
}
template <class P>
__device__ __forceinline__ void store_vec(typename P::vec *p, const typename P::C *r) {
  *p = narrow_vec(r, (typename P::vec *)nullptr);
}

// ---------------------------------------------------------------------------
// Blocked fermion layout.  Sites are grouped in blocks of 32 consecutive x4
// (the lanes of a warp); within a field of npv vec planes per site, plane p of
// site (x4, s) is at vec offset ((x4/32)*Ls + s)*npv*32 + p*32 + x4%32.  All
// slices and planes of one block are contiguous (npv*32*Ls vecs), so the data
// a CTA touches for one row of sites is one contiguous run of memory.  V4 is
// padded to a multiple of 32; the padding lanes are never read as neighbours,
// never written, and skipped by the reductions.
constexpr int kPlaneStride = 32;  // vecs between consecutive planes of one site
__host__ __device__ __forceinline__ long long site_off(int x4, int s, int Ls, int npv) {
  return ((long long)(x4 >> 5) * Ls + s) * npv * 32 + (x4 & 31);
}
__host__ __device__ __forceinline__ long long padded_v4(long long V4) { return (V4 + 31) / 32 * 32; }
// Gauge field, blocked the same way: vec k of link U_mu(x4) is at
// (((x4/32)*4 + mu)*nlv + k)*32 + x4%32.
__host__ __device__ __forceinline__ long long link_off(int x4, int mu, int nlv) {
  return (((long long)(x4 >> 5) * 4 + mu) * nlv) * 32 + (x4 & 31);
}

// ---------------------------------------------------------------------------
// Operator kinds handled by the stencil kernel.
enum OpKind { OP_DHOP = 0, OP_DHOP_DAG = 1, OP_D = 2, OP_DDAG = 3 };

struct DslashParams {
  void *out;
  const void *in;
  const void *gauge;  // blocked links at this precision (see link_off)
  int L[4];
  int V4;
  int Ls;
  long long plane;       // vecs between consecutive planes of one site (kPlaneStride)
  long long rhs_stride;  // vecs per right-hand side (= padded V4 * Ls * 24/R)
  int nrhs;             // right-hand sides in this launch (<= kMaxRhsPerLaunch)
  int bc[4];            // boundary signs (the rebuilt third row of a 12-real link needs them)
  const int *gate;      // optional: CTAs of RHS r run only if gate[r * gate_stride] != 0
  int gate_stride;
  double *norm_partials;  // optional (OP_D): |out|^2 per CTA at [rhs][CTA index in the RHS]
  const void *halo_up;  // optional t-face halves from the rank above (variant 0 only)
  const void *halo_dn;  // optional t-face halves from the rank below (variant 0 only)
  int tiles_per_plane;  // set by the launcher: CTAs per (x, y) plane
  int zblk;             // set by the launcher: z-blocks of the traversal order
  int sgrp;             // set by the launcher: CTAs per site tile (slice groups)
  int rhs_outer;        // RHS the slowest index of the grid (else the fastest)
  int t_begin;          // output sites: the time slices t_begin .. t_begin + t_count - 1
  int t_count;          // (0: all Lt; the inputs are read on the whole lattice)
  int *status;          // lattice-owned device word; set nonzero when a bounded wait gives up
  int wait_polls;       // polls of the first bounded wait of a step (-1: the built-in bound)
  const void *own;      // field of the local term of D / D^+ (null: hopping term alone)
  int parity;           // checkerboard launches: parity of the output sites
  double alpha, beta;   // local term alpha psi + beta K psi (K^+ for D^+)
  double hscale;        // factor of the hopping term (-1/2 in D_W)
  double M5, b, c;
  double mf[64];         // per-RHS masses, passed by value
  // optional (OP_DDAG, the CG's D^+ pass): instead of storing out, update the
  // CG residual r_s -= alpha_rhs out in place (r_s at FP64 for FP64 operators,
  // FP32 otherwise) and leave |r_s|^2 per CTA in rs_partials [rhs][CTA]
  void *rs;
  long long rs_stride;    // vecs of r_s per RHS
  const double *rs_alpha;  // alpha of RHS r at rs_alpha[r * rs_alpha_stride]
  int rs_alpha_stride;
  double *rs_partials;
  // optional with rs: also the solution step x_s += alpha_rhs p of the same
  // iteration (x_s like r_s, p the CG direction at the operator's precision)
  void *xs;
  const void *pdir;
};

// The residual update fused into a D^+ launch (see DslashParams::rs), and
// optionally the solution step (x_s and p non-null; see DslashParams::xs).
struct ResidualFuse {
  void *r_s;
  const double *alpha;
  int alpha_stride;
  double *partials;
  void *x_s = nullptr;
  const void *p = nullptr;
};

constexpr int kMaxRhsPerLaunch = 64;

// Launch configuration chosen by the tuner.
struct TileConfig {
  int spt;      // fifth-dimension slices per thread
  int tx;       // 4D sites per CTA (multiple of 32)
  int variant;  // hop-phase load scheme, 0 .. kNumVariants-1 (see dw.h)
  int zblk;     // z-blocks of the CTA traversal order (divides Lz)
  int sgrp;     // CTAs sharing one tile of sites, each with Ls / (spt sgrp) thread rows
  int rhs_outer;  // 1: the RHS are the slowest index of the launch grid (chosen by the tuner)
};
constexpr int kNumVariants = 9;

// Variants 6 and 7 stage 32-site blocks of the (x, y) plane in shared memory:
// they need Lx <= 32 (an x or y neighbour at most one block away), planes of
// whole blocks (Lx Ly a multiple of 32), tiles of whole blocks that tile the
// plane, the hopping term alone (Dhop, Dhop^+) and no t halos.
inline bool rows_variant_ok(int op, int Lx, int Ly, int tx) {
  return (op == OP_DHOP || op == OP_DHOP_DAG || op == OP_D) && Lx <= 32 &&
         (Lx * Ly) % 32 == 0 && tx % 32 == 0 && tx <= Lx * Ly && (Lx * Ly) % tx == 0;
}
// Dynamic shared memory of variants 6 and 7: the barrier, then R + 2 rows
// (y0-1 .. y0+R, or the ring slots) of the CTA's nsl slices at precision
// `prec` (24 reals per site); D (op OP_D) stages two more slices per row, the
// s-neighbours of the CTA's slice range.
inline size_t rows_smem_bytes(int tx, int nsl, int prec, int op) {
  const int nss = nsl + (op == OP_D ? 2 : 0);
  return 128 + (size_t)(tx / 32 + 2) * nss * 24 * 32 * prec_real_bytes(prec);
}

// The error of the last stencil launch that failed on this thread (the launch
// itself clears CUDA's last-error state when it checks it).
cudaError_t &last_launch_error();

// Stencil launch at precision `prec`: 0 on success, -2 for a tile/variant
// that does not exist, -3 for a CTA beyond the kernel's limits, -1 on a CUDA
// launch error.
int launch_dslash(const DslashParams &p, int prec, int op, TileConfig cfg, cudaStream_t st);
// Variant 8: FP16 hopping term with the SU(3) x half-spinor products on the
// tensor cores (dw_dslash_tc.cu): Dhop / Dhop^+, Lx even, Ls a multiple of 4 up
// to 16; one tile shape (spt 1, tx 32, sgrp 1, zblk unused).
inline bool tc_variant_ok(int op, int Lx, int Ls) {
  return (op == OP_DHOP || op == OP_DHOP_DAG) && Lx % 2 == 0 && Ls % 4 == 0 && Ls <= 16;
}
int launch_dslash_tc_F16(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
// Stencil on interleaved-complex FP32 fields (layout ablation): Dhop / Dhop^+
// with variants 4-7 only; same return codes.
int launch_dslash_cplx(const DslashParams &p, int op, TileConfig cfg, cudaStream_t st);
inline bool cplx_variant_ok(int op, int variant) {
  return (op == OP_DHOP || op == OP_DHOP_DAG) && variant >= 4 && variant <= 7;
}
// Checkerboard (single-parity) stencil, OP_D / OP_DDAG forms only.
int launch_dslash_cb(const DslashParams &p, int prec, int op, TileConfig cfg, cudaStream_t st);
// Largest CTA the stencil kernel (op, spt, variant) can launch (0: none).
int dslash_max_threads(int prec, int op, int spt, int variant);
// Face halves of a t-decomposed sub-lattice for stencil operator `op` (an
// OpKind; see dw_halo_pack_op).
int launch_halo_pack_F64(const DslashParams &p, void *send_dn, void *send_up, int op,
                         cudaStream_t st);
int launch_halo_pack_F32(const DslashParams &p, void *send_dn, void *send_up, int op,
                         cudaStream_t st);
int launch_halo_pack_F16(const DslashParams &p, void *send_dn, void *send_up, int op,
                         cudaStream_t st);

}  // namespace dw



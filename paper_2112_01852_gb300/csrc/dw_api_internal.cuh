// Internal helpers shared by the C-ABI translation units.
#pragma once

#include "dw_common.cuh"
#include "dw_fields.cuh"

namespace dw {

int fail(int code, const char *fmt, ...);
void clear_error();
int cuda_fail(cudaError_t e, const char *what);
size_t field_bytes(const dw_lattice *lat, int prec, int nrhs);
FieldGeom geom(const dw_lattice *lat);
int ensure_buffer(void **buf, size_t *cap, size_t need);
TileConfig default_tile(const dw_lattice *lat, int prec, int op, int nrhs);
int auto_zblk(const dw_lattice *lat, int prec);
TileConfig pick_tile(dw_lattice *lat, int prec, int op, int nrhs);
bool tile_valid(const dw_lattice *lat, int prec, int op, TileConfig t);
// Time the valid tiles for (op, nrhs) at precision `prec` and store the best
// (quick: only tx <= 64 and the automatic z-blocking).
int tune_tile(dw_lattice *lat, int prec, int op, int nrhs, cudaStream_t st, bool quick = false);
// Stencil launch (op = OpKind) at precision `prec` over nrhs RHS; mf_host may be
// NULL for the hopping-only kinds; `force` overrides the tile choice.
// `gate` (optional) skips the CTAs of RHS r unless gate[r * gate_stride] != 0;
// halo_up / halo_dn (optional, variant 0 tiles only) replace the t-neighbours
// at the t faces of a decomposed sub-lattice; norm_partials (optional, OP_D
// only) receives |out|^2 per CTA, [rhs][dslash_ctas_per_rhs]; t_begin / t_count
// restrict the output to the time slices t_begin .. t_begin + t_count - 1
// (t_count 0: all).
int run_dslash(dw_lattice *lat, int prec, int op, void *out, const void *in,
               const double *mf_host, int nrhs, cudaStream_t st, const TileConfig *force,
               const int *gate = nullptr, int gate_stride = 0, const void *halo_up = nullptr,
               const void *halo_dn = nullptr, double *norm_partials = nullptr, int t_begin = 0,
               int t_count = 0);
// CTAs per right-hand side of a stencil launch with tile `t` (the length of the
// per-RHS rows of norm_partials).
long long dslash_ctas_per_rhs(const dw_lattice *lat, TileConfig t);
size_t halo_bytes(const dw_lattice *lat, int prec, int nrhs);
int apply_op(dw_lattice *lat, int op, void *out, const void *in, const double *mf, int nrhs,
             cudaStream_t st);
// Argument checks shared by the dw_apply_* entry points.
int check_apply(dw_lattice *lat, void *out, const void *in, const double *mf, int nrhs,
                bool need_mf);
void cg_release(dw_lattice *lat);
// dw_apply_host: copies and operator pipelined over time slabs (arguments checked
// by the caller); synchronous.
int apply_host_pipelined(dw_lattice *lat, int op, void *out_host, const void *in_host,
                         const double *mf, int nrhs, cudaStream_t st);
void pipe_release(dw_lattice *lat);

}  // namespace dw

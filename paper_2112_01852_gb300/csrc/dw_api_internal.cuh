// Internal helpers shared by the C-ABI translation units.
#pragma once

#include <map>
#include <tuple>
#include <vector>

#include "dw_common.cuh"
#include "dw_fields.cuh"

namespace dw {
struct CGWork;
}  // namespace dw

// ---------------------------------------------------------------------------
// The lattice object behind the opaque handle.
struct dw_lattice {
  int dims[4];
  int Ls;
  long long V4;
  long long V4p;  // V4 padded to a multiple of 32 (blocked layout)
  long long V5;
  int kind;
  double M5, b, c;
  int prec;
  int bc[4];
  int device;
  int num_sms;
  bool gauge_loaded;
  int *dev_status;  // device word the kernels set when a bounded wait gives up
  int wait_polls;   // dw_set_wait_polls (-1: the kernels' built-in bound)
  bool cplx;        // dw_set_complex_layout: FP32 fields hold interleaved-complex quads
  double reliable_delta;  // dw_set_reliable_delta (0: the solvers' defaults)
  // gauge copies per precision (blocked; 18 reals per link at FP64, 12 below)
  void *gauge[3];
  // scratch: one field for D^+D, host-apply staging, reduction partials
  void *scratch;
  size_t scratch_bytes;
  void *stage_in, *stage_out;
  size_t stage_bytes;
  // host-buffer apply: copy-in and copy-out streams and their events
  cudaStream_t pipe_in, pipe_out;
  std::vector<cudaEvent_t> pipe_events;
  double *partials;   // reduction partials
  size_t partials_cap;
  // tuning cache: (prec, op, nrhs) -> tile
  std::map<std::tuple<int, int, int>, dw::TileConfig> tuned;
  // solver workspace (dw_cg_solve), created on first use
  dw::CGWork *cg;
};

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
// (quick: only tx <= 128 and the automatic z-blocking).
int tune_tile(dw_lattice *lat, int prec, int op, int nrhs, cudaStream_t st, bool quick = false);
// Stencil launch (op = OpKind) at precision `prec` over nrhs RHS; mf_host may be
// NULL for the hopping-only kinds; `force` overrides the tile choice.
// `gate` (optional) skips the CTAs of RHS r unless gate[r * gate_stride] != 0;
// halo_up / halo_dn (optional, variant 0 tiles only) replace the t-neighbours
// at the t faces of a decomposed sub-lattice; norm_partials (optional, OP_D
// only) receives |out|^2 per CTA, [rhs][dslash_ctas_per_rhs]; t_begin / t_count
// restrict the output to the time slices t_begin .. t_begin + t_count - 1
// (t_count 0: all).
// `fuse` (optional, OP_DDAG only): the CG residual update of ResidualFuse in place
// of storing out (out is then not written).
int run_dslash(dw_lattice *lat, int prec, int op, void *out, const void *in,
               const double *mf_host, int nrhs, cudaStream_t st, const TileConfig *force,
               const int *gate = nullptr, int gate_stride = 0, const void *halo_up = nullptr,
               const void *halo_dn = nullptr, double *norm_partials = nullptr, int t_begin = 0,
               int t_count = 0, const ResidualFuse *fuse = nullptr);
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

// Even-odd pieces (dw_eo.cu).  Single-parity fields: V4/2 sites, blocked.
bool eo_ok(const dw_lattice *lat);  // every extent even
size_t cb_field_bytes(const dw_lattice *lat, int prec, int nrhs);
int eo_split(dw_lattice *lat, int prec, void *even, void *odd, const void *full, int nrhs,
             cudaStream_t st);
int eo_merge(dw_lattice *lat, int prec, void *full, const void *even, const void *odd, int nrhs,
             cudaStream_t st);
// out = A in, A^-1 in, A^+ in or A^-+ in (A = alpha + beta K), on parity fields
int apply_m5(dw_lattice *lat, int prec, void *out, const void *in, const double *mf, int nrhs,
             bool inv, bool dag, cudaStream_t st);
// out (parity) = alpha own + beta K own + hscale Dhop (b + cK) nbr (OP_D), or the
// D^+ form (OP_DDAG); own may be null
int run_dslash_cb(dw_lattice *lat, int prec, int op, void *out, const void *nbr, const void *own,
                  int parity, double alpha, double beta, double hscale, const double *mf,
                  int nrhs, cudaStream_t st, const int *gate, int gate_stride,
                  double *norm_partials, const TileConfig *force = nullptr,
                  const ResidualFuse *fuse = nullptr);
long long cb_ctas_per_rhs(const dw_lattice *lat, int prec, int op);
// Time the checkerboard tiles of (prec, op) once per lattice and keep the best.
int tune_cb(dw_lattice *lat, int prec, int op, cudaStream_t st);
// out_o = Dhat in_o or Dhat^+ in_o; t1, t2 even scratch fields
int apply_schur(dw_lattice *lat, int prec, void *out, const void *in, const double *mf, int nrhs,
                bool dag, void *t1, void *t2, cudaStream_t st, const int *gate, int gate_stride,
                double *norm_partials, const ResidualFuse *fuse = nullptr);

}  // namespace dw

/*
 * dw.h -- C ABI of the GB300 domain-wall fermion operator library (libdw_gb300.so).
 *
 * The library applies the domain-wall fermion operator in its Shamir and Moebius
 * forms on one GPU.  Its hot part is the "Domain Wall kernel" of the paper
 * (Sec. 4.1): the 4D Wilson hopping term applied to every fifth-dimension slice,
 * i.e. per 5D site spin projection to a half spinor, SU(3) x half spinor and
 * reconstruction (Table 3, 1320 flop per site update).  The paper names the
 * operator but does not write it down; the definitions used here are
 *
 *   Dhop psi(x,s) = sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu,s) + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu,s) ]
 *   D_W   = (4 - M5) - Dhop / 2
 *   K psi_s = P- psi_{s+1} + P+ psi_{s-1}; at the walls -mf P- psi_0 (s = Ls-1) and
 *             -mf P+ psi_{Ls-1} (s = 0); P+- = (1 +- g5) / 2
 *   D     = D_W (b + c K) + (1 - K)           Shamir: b = 1, c = 0
 *   D^+   = (b + c K^+) D_W^+ + (1 - K^+)
 *
 * with chiral-basis gammas g_k = [[0, i s_k], [-i s_k, 0]], g_4 = [[0, 1], [1, 0]],
 * g5 = diag(1, 1, -1, -1), and a factor bc[mu] on every hop that crosses the
 * lattice edge in direction mu.
 *
 * Conventions common to every call
 *  - Field buffers are caller-owned DEVICE pointers (unless the name says _host)
 *    in the library's internal layout (see dw_fermion_bytes), at the lattice's
 *    precision, 16-byte aligned.  Several right-hand sides are stored back to
 *    back, each dw_fermion_bytes(lat, prec, 1) long.
 *  - All calls are ordered on `stream` (a cudaStream_t, NULL = legacy default
 *    stream) and asynchronous, except dw_cg_solve and dw_apply_host, which
 *    synchronise.
 *  - No C++ exception crosses the ABI.  Every int-returning call returns DW_OK or
 *    a negative DW_ERR_* code; dw_last_error() returns the calling thread's last
 *    message.  A failed argument check launches nothing.
 *  - `out` must not alias `in`.
 *
 * Internal fermion layout (per RHS): sites are grouped in blocks of 32
 * consecutive x4 = x + Lx*(y + Ly*(z + Lz*t)); plane p of site (x4, s) is the
 * 16-byte vector (8-byte for DW_F16) at index
 *   ((x4 / 32) * Ls + s) * NP * 32 + p * 32 + x4 % 32,   NP = 24 / R,
 * so every block keeps all its slices and planes contiguous.  V4 is padded to
 * a multiple of 32 (dw_fermion_bytes includes the padding; padding lanes are
 * ignored).  The 24 reals of a 5D site are ordered I = half*12 + c*4 + ri*2 + j
 * (chirality half: 0 = spins 0,1 (P+), 1 = spins 2,3 (P-); colour c; re/im ri;
 * spin j within the half), so each run of 4 reals is the spin pair
 * (Re, Re, Im, Im) of one colour; plane p holds reals [p*R, p*R + R) with
 * R = 2 (F64) or 4 (F32, F16).
 *
 * Canonical layout (dw_pack_fermion / dw_unpack_fermion / dw_load_gauge):
 *   fermion complex128 [rhs][x4][s][spin 4][colour 3]
 *   gauge   complex128 [x4][mu = x,y,z,t][row 3][col 3], U_mu(x) links x to x+mu.
 */
#ifndef DW_GB300_H
#define DW_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dw_lattice dw_lattice; /* opaque, library-owned */

enum {
  DW_OK = 0,
  DW_ERR_ARG = -1,           /* invalid argument (null pointer, size, alignment, enum) */
  DW_ERR_ALLOC = -2,         /* device allocation failed */
  DW_ERR_CUDA = -3,          /* a CUDA call failed */
  DW_ERR_STATE = -4,         /* call out of order (e.g. apply before dw_load_gauge) */
  DW_ERR_NOT_CONVERGED = -5, /* CG hit maxit; stats still filled */
  DW_ERR_BREAKDOWN = -6,     /* CG met a non-finite or non-positive <p, A p> */
  DW_ERR_TIMEOUT = -7        /* a bounded device-side wait gave up */
};

enum { DW_SHAMIR = 0, DW_MOBIUS = 1 };
enum { DW_F64 = 0, DW_F32 = 1, DW_F16 = 2 };

/* Operator selector for dw_apply_host. */
enum { DW_OP_DHOP = 0, DW_OP_DHOP_DAG = 1, DW_OP_D = 2, DW_OP_DDAG = 3, DW_OP_DDAGD = 4 };

/*
 * Create a lattice of dims[4] = {Lx, Ly, Lz, Lt} 4D sites x Ls slices.
 * kind: DW_SHAMIR (b, c ignored and set to 1, 0) or DW_MOBIUS (b nonzero).
 * prec: storage precision of the fields passed to the dw_apply_* calls
 *       (DW_F64, DW_F32, or DW_F16 = IEEE binary16 storage with FP32 arithmetic).
 * bc:   per-direction boundary sign (+1 periodic, -1 antiperiodic); NULL means
 *       {1, 1, 1, -1}.
 * Every dim and Ls must be >= 1 and V4 = Lx*Ly*Lz*Lt < 2^31.  The lattice owns
 * its gauge copies, scratch space and tuning cache; free it with
 * dw_destroy_lattice.  Uses the current CUDA device.
 */
int dw_create_lattice(dw_lattice **out, const int dims[4], int Ls, int kind, double M5,
                      double b, double c, int prec, const int bc[4]);
void dw_destroy_lattice(dw_lattice *lat);

/*
 * Copy and convert a gauge field (DEVICE pointer, canonical complex128) into
 * the lattice's internal link arrays at every precision, folding the boundary
 * signs into the links that cross the lattice edge.  The links must be SU(3)
 * (unitary, determinant 1): the FP32 and FP16 copies keep two rows of each
 * link and rebuild the third as conj(row0 x row1).  The caller may free U as
 * soon as the stream has passed this call.
 */
int dw_load_gauge(dw_lattice *lat, const void *U, void *stream);

/*
 * out = Dhop in, the bare hopping sum over the 8 neighbours for every slice s
 * and each of nrhs right-hand sides (no -1/2 factor, no diagonal term).
 * This is the paper's Domain Wall kernel (Sec. 4.1; 1320 flop per 5D site,
 * Table 3).
 */
int dw_apply_Dhop(dw_lattice *lat, void *out, const void *in, int nrhs, void *stream);
/* out = Dhop^+ in  (= g5 Dhop g5 in). */
int dw_apply_Dhop_dag(dw_lattice *lat, void *out, const void *in, int nrhs, void *stream);

/*
 * out = D in with the per-RHS masses mf[nrhs] (HOST array).  One fused pass:
 * (b + cK) is applied to the neighbour spinors before the hop.
 */
int dw_apply_D(dw_lattice *lat, void *out, const void *in, const double *mf, int nrhs,
               void *stream);
/* out = D^+ in. */
int dw_apply_Ddag(dw_lattice *lat, void *out, const void *in, const double *mf, int nrhs,
                  void *stream);
/*
 * out = D^+ D in.  The intermediate D in lives in lattice-owned scratch, so
 * calls on one lattice must not overlap on different streams.
 */
int dw_apply_DdagD(dw_lattice *lat, void *out, const void *in, const double *mf, int nrhs,
                   void *stream);

/*
 * out = D^+ D in, like dw_apply_DdagD, without allocating anything.  The paper
 * has no counterpart: this entry point serves callers that cannot let the
 * library call cudaMalloc (for example a process whose device memory is all
 * handed out by its own pool allocator).  The intermediate D in is kept in one
 * fixed 32 MiB array compiled into the library, which every GPU that loads the
 * library holds until the process exits; the call makes no allocation call of
 * any kind.  nrhs * dw_fermion_bytes(lat, prec, 1) above 32 MiB is rejected with
 * DW_ERR_ARG before anything is launched.  The current device must be the
 * lattice's.  The first call on a device looks the array's device address up
 * (cudaGetSymbolAddress) and caches it; make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's contents:
 * calls that overlap on the GPU (different streams, or different lattices on
 * one device) race.  The D pass overwrites the whole intermediate, so nothing
 * has to be cleared between calls.
 */
int dw_apply_DdagD_noalloc(dw_lattice *lat, void *out, const void *in, const double *mf,
                           int nrhs, void *stream);

/*
 * Apply operator `op` (DW_OP_*) with HOST buffers in the internal layout at
 * the lattice precision: copies in to the device, applies, copies out back and
 * returns when the output is in out_host.  Device staging buffers are
 * lattice-owned.  mf may be NULL for DW_OP_DHOP / DW_OP_DHOP_DAG.
 * When Lx*Ly*Lz is a multiple of 32 the field moves in t slabs (up to 16, each
 * of at least 8192 4D sites): the copy in of one slab, the operator on the
 * previous one (once its t neighbours are resident) and the copy out of the
 * one before run at the same time, on `stream` and two lattice-owned streams.
 * Pinned host buffers (cudaHostAlloc / cudaHostRegister) are needed for the
 * copies to overlap; pageable ones work but serialise.  out_host must not
 * overlap in_host.
 */
int dw_apply_host(dw_lattice *lat, int op, void *out_host, const void *in_host,
                  const double *mf, int nrhs, void *stream);

typedef struct {
  int iters;            /* operator applications of the inner solver */
  int reliable_updates; /* FP64 residual recomputations (mixed modes) */
  int converged;        /* 1 if true_resid <= tol */
  double true_resid;    /* |b - D^+D x| / |b| recomputed in FP64 */
  double seconds;       /* wall time of the whole solve */
} dw_cg_stats;

/*
 * Solve D^+D x = b for nrhs right-hand sides with per-RHS masses mf[nrhs]
 * (HOST array).  x and b are DEVICE fields in the internal layout at DW_F64
 * (x holds the start vector on entry, the solution on exit).
 * mode: DW_F64 plain FP64 CG; DW_F32 / DW_F16 mixed precision: the inner
 * operator runs at FP32 / FP16 storage with FP32 arithmetic, with FP64 reliable
 * updates, FP64 reductions and an FP64 true-residual convergence test.
 * Stops when |b - D^+D x| / |b| <= tol for every RHS (converged RHS are masked
 * off) or after maxit inner iterations.  stats[nrhs] (HOST) is filled.
 * Returns DW_OK, DW_ERR_NOT_CONVERGED, DW_ERR_BREAKDOWN, or DW_ERR_TIMEOUT when
 * a stencil launch on this lattice gave up a bounded wait since the last
 * dw_device_status (the word is then cleared).  Synchronises.
 */
int dw_cg_solve(dw_lattice *lat, void *x, const void *b, const double *mf, int nrhs,
                double tol, int maxit, int mode, dw_cg_stats *stats, void *stream);

/*
 * Even-odd (red-black) preconditioning.  Sites are even or odd by
 * x + y + z + t; D = A + H with the local part A = alpha + beta K
 * (alpha = b (4 - M5) + 1, beta = c (4 - M5) - 1) and the hopping part
 * H = -Dhop (b + cK) / 2, which couples only opposite parities.  The Schur
 * complement on odd sites is Dhat = A - H_oe A^-1 H_eo (its adjoint
 * Dhat^+ = A^+ - H_eo^+ A^-+ H_oe^+), and D x = eta is equivalent to
 * Dhat x_o = eta_o - H_oe A^-1 eta_e, x_e = A^-1 (eta_e - H_eo x_o).  The paper
 * has no preconditioner; this is the standard construction.
 *
 * Single-parity fields ("eo fields") hold the V4/2 sites of one parity in the
 * blocked layout over the checkerboard index x4/2 (x4 the lexicographic site
 * index), V4/2 padded to a multiple of 32; dw_fermion_bytes_eo gives their
 * size.  All of these need Lx, Ly, Lz and Lt even (with an odd extent the
 * periodic hop across that edge joins sites of the same parity); DW_ERR_ARG
 * otherwise (dw_fermion_bytes_eo returns 0).
 *
 * dw_eo_split / dw_eo_merge: copy a full internal-layout field at precision
 * `prec` to its even and odd fields and back (device buffers, nrhs each).
 * dw_apply_m5_eo: out = A in (inverse: A^-1 in; dag: A^+ / A^-+) on eo fields at
 * the lattice precision, per-RHS masses mf[nrhs] (HOST).
 * dw_apply_schur: out = Dhat in (dag: Dhat^+ in) on odd eo fields at the lattice
 * precision; the even intermediates live in lattice scratch.  out must not
 * alias in.  Stream-ordered, asynchronous.
 */
size_t dw_fermion_bytes_eo(const dw_lattice *lat, int prec, int nrhs);
int dw_eo_split(dw_lattice *lat, void *even, void *odd, const void *full, int prec, int nrhs,
                void *stream);
int dw_eo_merge(dw_lattice *lat, void *full, const void *even, const void *odd, int prec,
                int nrhs, void *stream);
int dw_apply_m5_eo(dw_lattice *lat, void *out, const void *in, const double *mf, int nrhs,
                   int inverse, int dag, void *stream);
int dw_apply_schur(dw_lattice *lat, void *out, const void *in, const double *mf, int nrhs,
                   int dag, void *stream);

/*
 * Solve D x = eta with even-odd preconditioning: CG (mode as in dw_cg_solve:
 * FP64, or mixed FP32 / FP16 inner operator with FP64 reliable updates) on
 * Dhat^+ Dhat x_o = Dhat^+ (eta_o - H_oe A^-1 eta_e), then
 * x_e = A^-1 (eta_e - H_eo x_o).  The solve targets the full system: after each
 * CG pass the residual |eta - D x| / |eta| is recomputed in FP64 on the whole
 * lattice, and while it is above tol (for any RHS) the CG runs again from the
 * current x_o with its own tolerance lowered by the factor it missed by (at
 * most 4 passes, maxit inner iterations in all).  x (start vector: its odd
 * sites) and eta are full DEVICE fields in the internal layout at DW_F64;
 * mf[nrhs] HOST.  stats: iters and reliable_updates of all CG passes,
 * true_resid = |eta - D x| / |eta|, converged = (true_resid <= tol), seconds
 * for the whole call.  Needs even extents.  Returns DW_OK, DW_ERR_NOT_CONVERGED
 * (some RHS above tol), DW_ERR_BREAKDOWN or DW_ERR_TIMEOUT (as dw_cg_solve).
 * Synchronises.
 */
int dw_solve_eo(dw_lattice *lat, void *x, const void *eta, const double *mf, int nrhs,
                double tol, int maxit, int mode, dw_cg_stats *stats, void *stream);

/*
 * Stencil-kernel tiles.  A tile is (spt, tx, variant, zblk, sgrp): spt fifth-dimension
 * slices per thread (1..4, dividing Ls), tx 4D sites per CTA (a multiple of
 * 32, taken from one (x, y) plane), the load variant of the hop phase (0 =
 * neighbour spinors and links loaded straight into registers, direction by
 * direction; 1 = copied one direction ahead into shared memory with cp.async;
 * 2, 3 = loaded one (direction, slice) step ahead into registers, visiting
 * t,z,y,x (2) or x,y,z,t (3); 5 = variant 0 with L2 eviction hints: t+
 * neighbours kept, t- neighbours evicted first; 4 = variant 5 with at most
 * 128 registers per thread; 6 = variant 4 with the tile's 32-site blocks of
 * the (x, y) plane and the block on either side bulk-copied into shared memory,
 * the x and y hops read there (needs Lx <= 32, Lx*Ly a multiple of 32, tx
 * dividing Lx*Ly, DW_OP_DHOP / DW_OP_DHOP_DAG / DW_OP_D, where D also stages
 * the fifth-dimension neighbours of the CTA's slices and reads its local term
 * there; its bounded wait reports through dw_device_status); 7 = variant 6 with one CTA walking all tiles of
 * its (z, t) plane, the blocks kept in a ring so that each is copied once per
 * plane (same conditions); 8 = FP16 storage only: the hopping term with its
 * SU(3) x half-spinor products on the tensor cores (mma.sync m16n8k16), Lx
 * even, Ls a multiple of 4 up to 16, the one tile spt 1, tx 32, sgrp 1; FP64
 * builds 0 and 2 only; interleaved-complex FP32 lattices 4-7 only), zblk, the
 * number of z-blocks of the CTA traversal order (planes are visited block by
 * block, t inside a block; zblk divides Lz; 0 in dw_set_tile = automatic), and
 * sgrp, the number of CTAs that share one tile of tx sites: each holds
 * Ls/(spt sgrp) slice groups (sgrp divides Ls/spt; DW_OP_DDAG combines the
 * edges of neighbouring slice groups, so its sgrp CTAs run as one thread-block
 * cluster and sgrp is at most 8).  Smaller CTAs let more of them
 * fit on an SM when registers limit the occupancy.
 *
 * dw_set_tile pins the tile used for operator `op` (DW_OP_DHOP .. DW_OP_DDAG)
 * at precision `prec` for launches of `nrhs` right-hand sides (0 = any count
 * without a more specific entry).  Returns DW_ERR_ARG for an invalid tile.
 *
 * dw_tune times every valid tile for (op, nrhs) at the lattice precision on
 * lattice-owned scratch fields (CUDA events on `stream`, median of a few
 * launches), keeps the fastest for later calls and returns it in *spt, *tx,
 * *variant, *zblk, *sgrp (any may be NULL).  For nrhs > 1 it also chooses the
 * order of the launch grid, which these five numbers do not report: the RHS
 * innermost (the CTAs of one tile for successive RHS share its links in L2; the
 * order dw_set_tile selects) or outermost (one RHS's sweep after another, each
 * with the L2 reuse window of a single RHS).  Requires a loaded gauge field;
 * synchronises; must not be called while `stream` is being captured into a
 * graph.
 */
int dw_set_tile(dw_lattice *lat, int op, int prec, int nrhs, int spt, int tx, int variant,
                int zblk, int sgrp);
int dw_tune(dw_lattice *lat, int op, int nrhs, int *spt, int *tx, int *variant, int *zblk,
            int *sgrp, void *stream);
/*
 * The tile that launches of (op, prec, nrhs) use now: the pinned or tuned one,
 * else the untuned default.  Outputs may be NULL.
 */
int dw_get_tile(dw_lattice *lat, int op, int prec, int nrhs, int *spt, int *tx, int *variant,
                int *zblk, int *sgrp);

/*
 * Device-side status of the lattice's kernels.  Kernels that wait for their own
 * asynchronous copies (stencil variant 6) bound every wait; one that gives up
 * sets a lattice-owned device word and returns without finishing (its output is
 * then wrong).  This call synchronises the device, reads and clears the word and
 * returns DW_OK or DW_ERR_TIMEOUT.
 */
int dw_device_status(dw_lattice *lat);

/*
 * Layout ablation: the interleaved-complex form of the fermion quads (the GPU
 * counterpart of the paper's RIRI layout, Sec. 4.3, Table 3).  By default a quad
 * of the internal layout is the spin pair (Re j0, Re j1, Im j0, Im j1) of one
 * colour and chirality half, and the stencil's packed FP32 arithmetic pairs
 * the two spins (the counterpart of RRII: real arithmetic only).  With
 * interleaved = 1 the FP32 fields of this DW_F32 lattice hold
 * (Re j0, Im j0, Re j1, Im j1) instead, and the stencil pairs the real and
 * imaginary parts of one complex number (a product by i swaps a pair; a complex
 * product needs the pair and its swapped copy).  Only dw_pack_fermion /
 * dw_unpack_fermion at DW_F32, dw_apply_Dhop, dw_apply_Dhop_dag, dw_apply_host
 * with those operators, dw_set_tile / dw_tune (variants 4-7) and the size queries
 * support it; the other operators, the even-odd calls and the solvers return
 * DW_ERR_STATE.  Fields packed under one setting must not be used under the
 * other.  Switching clears the lattice's tuned tiles.  interleaved = 0 restores
 * the default.  Returns DW_OK or DW_ERR_ARG (not a DW_F32 lattice, or
 * interleaved not 0 / 1).
 */
int dw_set_complex_layout(dw_lattice *lat, int interleaved);

/*
 * Bound of the first wait of each step of the row-staged stencil variants
 * (6, 7) on this lattice: polls >= 0 lets that wait give up after `polls`
 * polls of the barrier, -1 (the default) restores the built-in bound of about a
 * second.  A wait that gives up sets the lattice's status word (reported by
 * dw_device_status, and by dw_cg_solve / dw_solve_eo as DW_ERR_TIMEOUT); the
 * kernel then waits once more, with the built-in bound, for the copies it
 * issued, so that it never reads or refills a slot with a copy in flight.
 * polls = 0 therefore exercises the timeout report without losing the result:
 * it exists for testing that path.  The paper has no counterpart.  Returns
 * DW_OK or DW_ERR_ARG (polls < -1).
 */
int dw_set_wait_polls(dw_lattice *lat, int polls);

/*
 * Reliable-update threshold of the mixed-precision solvers (dw_cg_solve and
 * dw_solve_eo with mode DW_F32 or DW_F16) on this lattice: the FP64 residual is
 * recomputed (and the low-precision iteration restarted from it) once the
 * iterated residual has fallen below delta times its largest value since the
 * previous update (Clark et al., mixed-precision solvers on GPUs; the paper
 * gives no solver).  0 < delta < 1 sets it; delta = 0 (the default) takes the
 * values chosen from timings at 24^4 x Ls=16 and 32^3 x 64 x Ls=12: 1e-3 with
 * FP32 inner fields, and with FP16 ones 0.1 for dw_cg_solve and 0.01 for
 * dw_solve_eo.  Smaller values mean fewer FP64 operator applications, larger
 * ones a shorter drift of the iterated residual.
 * Returns DW_OK or DW_ERR_ARG (delta outside [0, 1)).
 */
int dw_set_reliable_delta(dw_lattice *lat, double delta);

/*
 * Domain decomposition along t on one device ("virtual ranks").  The hopping
 * term has one exchange step when the lattice is split into ranks along t
 * (an exchange of spin-projected half spinors across the cut).  A rank owns a
 * sub-lattice created with dims {Lx, Ly, Lz, Lt / R}, the global links of its
 * t-range, and bc[3] = the global t sign for the last rank and +1 for the
 * others (so the sign sits on the one link that crosses the global edge).
 *
 * dw_halo_pack fills the two half-spinor faces a rank sends, each
 * dw_halo_bytes(lat, prec, nrhs) long, layout [rhs][quad 3][s][face site]:
 *   send_dn -> the rank below: the forward-hop projection of the first t slice;
 *   send_up -> the rank above: U_t^+ times the backward-hop projection of the
 *              last t slice.
 * dag selects Dhop^+ (the sign of the projections).
 * dw_apply_Dhop_halo is dw_apply_Dhop (dw_apply_Dhop_dag for dag = 1) on the
 * sub-lattice, with the t-neighbours of its t faces taken from recv_up (the
 * rank above's send_dn) and recv_dn (the rank below's send_up).  It runs the
 * same arithmetic in the same order as the undecomposed kernel with a
 * variant-0 tile, so the stitched result equals it bit for bit.
 */
size_t dw_halo_bytes(const dw_lattice *lat, int prec, int nrhs);
int dw_halo_pack(dw_lattice *lat, void *send_dn, void *send_up, const void *in, int nrhs,
                 int dag, void *stream);
/*
 * The same for any stencil operator op = DW_OP_DHOP, DW_OP_DHOP_DAG, DW_OP_D or
 * DW_OP_DDAG, for ranks in separate processes (the exchange of the paper's MPI
 * runs, Sec. 4.2): D's hopping term acts on phi = (b + cK) psi, so its faces are
 * those of phi (formed with the masses mf[nrhs], HOST, with the arithmetic of the
 * undecomposed kernel); D^+'s are those of Dhop^+ (its 5D part follows the hop
 * and is local).  dw_apply_op_halo applies op on the sub-lattice with the
 * received faces (mf as for dw_apply_D; NULL for the hopping terms); the
 * stitched result equals the undecomposed operator with a variant-0 tile bit for
 * bit.  Both return DW_ERR_STATE on an interleaved-complex lattice.
 */
int dw_halo_pack_op(dw_lattice *lat, int op, void *send_dn, void *send_up, const void *in,
                    const double *mf, int nrhs, void *stream);
int dw_apply_op_halo(dw_lattice *lat, int op, void *out, const void *in, const void *recv_up,
                     const void *recv_dn, const double *mf, int nrhs, void *stream);

/*
 * Level-1 field operations on DEVICE fields in the internal layout at precision
 * prec (nrhs each), for solvers driven from the host, e.g. a CG whose global
 * sums are completed across ranks.  The paper gives no solver; these are the
 * vector steps of textbook CG.
 * dw_field_redot: out[r] (HOST) = Re <a_r, b_r> over the lattice's sites, summed
 *   in FP64 in a fixed order (deterministic); synchronises `stream`.
 * dw_field_axpby: y_r = a[r] x_r + b[r] y_r (a, b HOST arrays of nrhs), in FP64
 *   arithmetic when prec is DW_F64, FP32 otherwise; y may alias x.
 * Return DW_OK, DW_ERR_ARG or DW_ERR_STATE (interleaved-complex FP32 fields).
 */
int dw_field_redot(dw_lattice *lat, int prec, const void *a, const void *b, int nrhs,
                   double *out, void *stream);
int dw_field_axpby(dw_lattice *lat, int prec, void *y, const double *a, const void *x,
                   const double *b, int nrhs, void *stream);
int dw_apply_Dhop_halo(dw_lattice *lat, void *out, const void *in, const void *recv_up,
                       const void *recv_dn, int nrhs, int dag, void *stream);

/* Bytes of one internal-layout field of nrhs right-hand sides at precision prec. */
size_t dw_fermion_bytes(const dw_lattice *lat, int prec, int nrhs);

/*
 * Convert between the canonical complex128 layout (src/dst DEVICE pointer) and
 * the internal layout at precision prec (rounding to nearest even for F32/F16).
 */
int dw_pack_fermion(dw_lattice *lat, void *dst_internal, int prec, const void *src_c128,
                    int nrhs, void *stream);
int dw_unpack_fermion(dw_lattice *lat, void *dst_c128, const void *src_internal, int prec,
                      int nrhs, void *stream);

/* Calling thread's last error message ("" if none). */
const char *dw_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DW_GB300_H */

/*
 * vbarms.h -- C ABI of the GB300 (sm_103a) VBARMS library.
 *
 * VBARMS ("Using the VBARMS method in parallel computing", Carpentieri, Liao,
 * Sosonkina, Bonfiglioli, arXiv 1508.02219) is a variable-block multilevel
 * incomplete LU preconditioner.  This library implements its data-parallel
 * path on one GPU:
 *   Step 1   angle-based row-pattern compression and block permutation
 *            (Section 2.1, Eq. 3)                        -> vbarms_compress
 *   Steps 2-4 scaling, block independent-set ordering and the two-sweep block
 *            partial factorization, repeated per level, with the last level
 *            factored by block ILUT (Section 3, Eq. 4-8, Alg. 3, Section 3.1)
 *                                                        -> vbarms_factor
 *   Alg. 2   the multilevel forward/backward solve       -> vbarms_apply
 *   FGMRES   flexible GMRES(m) with the preconditioner   -> fgmres_solve
 *
 * Conventions (every entry point):
 *  - Return a vb_status; never abort, never trap the GPU.  On error the
 *    output handles/arrays are left untouched and vbarms_last_error() returns
 *    a message (thread-local).
 *  - Indices are 0-based.  CSR columns must be ascending and unique.
 *  - Handles are library-owned and freed by the matching *_destroy.
 *  - Device work is enqueued on the stream given at creation (a cudaStream_t
 *    passed as void*, NULL = the legacy default stream).  Calls that return
 *    sizes or statuses synchronize that stream.
 *  - A handle belongs to the device that was current when it was created
 *    (vbarms_compress, vbarms_vbsr_from_blocks; a factorization takes its
 *    matrix's device), and its stream must belong to that device.  Every
 *    later call with the handle runs on that device whatever device is
 *    current, and restores the caller's current device before returning.
 *    Calls that combine handles of different devices return VB_EINVAL.
 *  - Vectors given to vbarms_apply / fgmres_solve are caller-owned device
 *    arrays of doubles in the ORIGINAL (unpermuted) numbering.
 *
 * Internal scratch and factors live in device memory obtained with
 * cudaMallocAsync on the handle's stream.
 */
#ifndef VBARMS_H
#define VBARMS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VB_OK = 0,
  VB_EINVAL = 1,     /* invalid argument or malformed CSR                     */
  VB_ENOMEM = 2,     /* device allocation failed                              */
  VB_ECUDA = 3,      /* a CUDA runtime call failed                            */
  VB_ESINGULAR = 4,  /* an exactly singular pivot block (GEPP found a 0 pivot)*/
  VB_ETIMEOUT = 5,   /* a bounded device wait ran out (wait_limit)            */
  VB_ENOCONV = 6,    /* FGMRES reached maxit without meeting rtol             */
  VB_EINTERNAL = 7   /* an internal consistency check failed                  */
} vb_status;

typedef struct vbarms_vbsr_st* vbarms_vbsr; /* VBCSR matrix P_B A P_B^T + P_B */
typedef struct vbarms_prec_st* vbarms_prec; /* multilevel VBARMS factorization */

enum { VB_FP64 = 0, VB_FP32_MIXED = 1 };

typedef struct {
  /* VB_FP64: every factor in FP64.  VB_FP32_MIXED: the first level is scaled
   * and ordered from the FP64 matrix; W, G, Schur complements and last-level
   * factors are stored and computed in FP32 (FP32 accumulation) and applied
   * in FP32 arithmetic into FP64 vectors.  Pivot blocks whose 1-norm
   * condition estimate exceeds fp64_pivot_cond keep FP64 LU factors and are
   * applied in FP64 (reduction levels: factored in FP64, the others used as
   * their FP32 rounding; last level: factored in FP32 and refactored in FP64
   * when the estimate exceeds the threshold).                              */
  int precision;
  double fp64_pivot_cond; /* default 1e4                                     */
  double ddtol;           /* Step 3: supernodes with weight < ddtol go to C
                             (default 0 = off)                               */
  uint64_t wait_limit;    /* nanoseconds one bounded device wait may last
                             before VB_ETIMEOUT (0 = default, 30 s)          */
  int schur_drop_all;     /* nonzero: apply the drop threshold to the Schur
                             complement at every reduction (the ARMS habit);
                             0 (default): only at the last one, as Section 3
                             prescribes                                      */
  int keep_factors;       /* 1 (default): keep every level's scaled matrix,
                             F, E, C and S for vbarms_prec_export; 0: release
                             them as soon as the factorization has consumed
                             them (the solve never reads them), which lowers
                             the factorization's device memory by about half;
                             exporting a released factor is then VB_EINVAL  */
  int group_size;         /* Step 3: supernodes per independent group, 1 to
                             64 (default 1: one supernode per group).  With
                             more, each group grows breadth first from its
                             seed (visited by weight) up to group_size
                             supernodes, its neighbours going to C, so the
                             diagonal blocks D_i of D are block sparse; each
                             group is eliminated inside (Section 3.1's two
                             sweeps).  The greedy is sequential (one warp)  */
} vbarms_opts;

/* Fill *opt with the defaults above. */
void vbarms_opts_default(vbarms_opts* opt);

/* Step 1 (Section 2.1, Eq. 3).  Angle-based compression of an n x n CSR
 * matrix: rows i < j with |P_i n P_j| / sqrt(|P_i| |P_j|) >= tau are grouped
 * greedily in natural order (a still-unassigned row becomes a leader and
 * claims every later unassigned row similar to it); groups are ordered by
 * leader, members ascending.  The result holds P_B, the block sizes and
 * P_B A P_B^T as a VBCSR matrix whose blocks are dense and zero padded.
 *   n        number of rows/columns (n >= 0)
 *   rowptr   int64[n+1], colind int32[nnz], val double[nnz]; host arrays when
 *            on_device == 0, device arrays when on_device != 0.  Borrowed for
 *            the duration of the call (copied).
 *   tau      similarity threshold, 0 < tau <= 1 (1 = exact dense blocks)
 *   stream   cudaStream_t for all work of the returned handle (NULL: default)
 * Errors: VB_EINVAL for tau out of range or a malformed CSR (rowptr not
 * monotone, column out of range, unsorted or duplicate columns).           */
vb_status vbarms_compress(int64_t n, const int64_t* rowptr, const int32_t* colind,
                          const double* val, int on_device, double tau, void* stream,
                          vbarms_vbsr* out);

/* The two-pass variant of Section 2.1: rows with identical stored patterns
 * form a group when there are two or more of them (and the pattern is not
 * empty), groups in ascending order of their smallest row; then every other
 * row joins the first group whose pattern P_g passes the angle test
 * |P_j n P_g| / sqrt(|P_j| |P_g|) >= tau (evaluated as in vbarms_compress),
 * else it stays a block of its own.  Blocks are ordered by their smallest
 * row, rows ascending.  Arguments, ownership, layout and errors as in
 * vbarms_compress.                                                          */
vb_status vbarms_compress_two_pass(int64_t n, const int64_t* rowptr, const int32_t* colind,
                                   const double* val, int on_device, double tau, void* stream,
                                   vbarms_vbsr* out);

/* Graph-based compression (Section 2.2, Alg. 1) with minimum block density
 * mu >= 0: vertices with identical closed neighbourhoods adj(i) in the
 * graph of A + A^T form the initial supernodes (Alg. 1's checksum scan);
 * then, in ascending order of their smallest vertex, each supernode X tries
 * the supernodes owning a vertex of adj(X), in ascending order of their
 * smallest vertex, and absorbs Z when the merged supernode S = X u Z has
 * density N/T >= mu, with T = 2 |adj(S)| |S| - |S|^2 and
 * N = 2 sum_{v in S} |adj(v)| - sum_{v in S} |adj(v) n S| (the T and N of
 * Section 2.2).  Blocks are ordered by their smallest vertex, vertices
 * ascending.  Arguments, ownership and the result's layout are those of
 * vbarms_compress (which this call replaces for the grouping only).
 * Errors: VB_EINVAL for mu < 0 or a malformed CSR; VB_ENOMEM when a
 * supernode's candidate set exceeds 1024 supernodes or the adjacency pool
 * of the merge pass runs out.                                              */
vb_status vbarms_compress_graph(int64_t n, const int64_t* rowptr, const int32_t* colind,
                                const double* val, int on_device, double mu, void* stream,
                                vbarms_vbsr* out);

/* Build a VBCSR handle directly from host block arrays (square partition,
 * P_B = identity).  bsz int32[nblk]; bptr int64[nblk+1]; bcol int32[nnzb]
 * ascending per row; voff int64[nnzb+1] with voff[b+1]-voff[b] =
 * bsz[row]*bsz[bcol[b]]; val double[voff[nnzb]] row-major blocks.          */
vb_status vbarms_vbsr_from_blocks(int64_t nblk, const int32_t* bsz, const int64_t* bptr,
                                  const int32_t* bcol, const int64_t* voff, const double* val,
                                  void* stream, vbarms_vbsr* out);

/* Sizes and the quality measures of Section 2: av_bd = nnz(A) / sum of the
 * sizes of the stored blocks, av_bs = n / number of diagonal blocks.       */
vb_status vbarms_vbsr_query(vbarms_vbsr A, int64_t* n, int64_t* nblk, int64_t* nnzb,
                            int64_t* nval, double* av_bd, double* av_bs);

/* Copy P_B and the block structure to host arrays (any pointer may be NULL):
 * perm int32[n] (perm[k] = original row at permuted position k), bsz
 * int32[nblk], bptr int64[nblk+1], bcol int32[nnzb], voff int64[nnzb+1],
 * val double[nval].                                                        */
vb_status vbarms_vbsr_export(vbarms_vbsr A, int32_t* perm, int32_t* bsz, int64_t* bptr,
                             int32_t* bcol, int64_t* voff, double* val);

/* Steps 2-4 of Section 3 repeated nlev times (Eq. 7-8), then block ILUT of
 * the last Schur complement (Section 3 dropping rule, Alg. 3 in block form).
 * Per level: two-sided max-abs scaling; weighted greedy block independent set
 * on the quotient graph of A + A^T (weight ||A_YY||_F / sum_Z ||A_YZ||_F,
 * visited by weight descending, index ascending; one supernode per group);
 * GEPP of every pivot block; W = L^{-1} P F and G = E U^{-1} with dropping;
 * S = C - G W (exact except at the last reduction).  A block B (m x n) is
 * dropped iff ||B||_F < droptol * m * n; lfil >= 0 keeps at most lfil blocks
 * (largest norm, lower column on ties) per block row of W, G, L_S, U_S;
 * lfil < 0 keeps all.  Levels stop early when nothing is left to eliminate.
 * opt may be NULL (defaults).  Errors: VB_EINVAL (nlev < 0, droptol < 0),
 * VB_ESINGULAR (a pivot block is exactly singular), VB_ENOMEM.             */
vb_status vbarms_factor(vbarms_vbsr A, int nlev, double droptol, int lfil,
                        const vbarms_opts* opt, vbarms_prec* out);

/* Batched factorization of nmat independent matrices (the paper factors one
 * matrix; batching is an interface of this library).  Matrices that share
 * (nlev[m], droptol[m], lfil[m]) are factored together as their
 * block-diagonal union, one launch per phase for the whole group; since
 * every step of the method stays inside a connected component, each
 * matrix's factors are those vbarms_factor would give it, operation for
 * operation.  out[m] receives a handle per matrix; the handles of one group
 * share the group's factorization (freed with the last of them).  With such
 * a handle, vbarms_apply and fgmres_solve act on the matrix's own vectors
 * but apply the whole group's preconditioner (zero outside the matrix's
 * rows); vbarms_apply_batched applies it once for many matrices;
 * vbarms_prec_stats / _export / _vector / _kernel_stats describe the group;
 * vbarms_apply_static rejects it.  A: handles of vbarms_compress or
 * vbarms_vbsr_from_blocks (inputs, not consumed); a group runs on the stream
 * of its first matrix after the others' streams are synchronized.  Errors:
 * as vbarms_factor; VB_EINVAL when a group exceeds 2^31 rows or blocks; on
 * error no handle is returned.                                              */
vb_status vbarms_factor_batched(int nmat, const vbarms_vbsr* A, const int* nlev, const double* droptol,
                                const int* lfil, const vbarms_opts* opt, vbarms_prec* out);

/* Global preconditioners of Section 5 with VBARMS as the local solver, all
 * subdomains on one GPU: block Jacobi (overlap 0), additive Schwarz
 * (restricted = 0) and restricted additive Schwarz (restricted != 0).
 * Subdomain i (0 <= i < nparts) owns the compressed block rows I with
 * floor(nparts * roff_I / n) = i (contiguous ranges of near-equal scalar
 * size; roff_I is the first scalar row of block row I in the P_B
 * numbering), extended overlap times by the block graph of A + A^T
 * (W_i^d = adj(W_i^{d-1})).  Its local matrix A_i = R_i A R_i holds the
 * blocks of A with row and column in W_i^overlap, rows ascending.  Every A_i
 * is factored by VBARMS with (nlev, droptol, lfil, opt) -- all of them as
 * one block-diagonal union, one launch per phase -- and the handle applies
 *   M^{-1} x = sum_i Q_i^T A_i^{-1} R_i x,
 * Q_i = R_i (additive) or the restriction to the owned rows (restricted).
 * The handle works with vbarms_apply, vbarms_apply_static, fgmres_solve and
 * vbarms_prec_stats; vbarms_prec_export / _vector / _kernel_stats describe
 * the union's factorization.  A: handle of vbarms_compress or
 * vbarms_vbsr_from_blocks (input, not consumed).  Errors: VB_EINVAL (nparts
 * outside [1, 4096], overlap < 0, nlev < 0, droptol < 0, a union above 2^31
 * rows), then as vbarms_factor.                                             */
vb_status vbarms_dd_factor(vbarms_vbsr A, int nparts, int overlap, int restricted, int nlev, double droptol,
                           int lfil, const vbarms_opts* opt, vbarms_prec* out);

/* Layout of a vbarms_dd_factor handle: part[nblk(A)] = the subdomain owning
 * each block row, dstart[nparts + 1] = first union block row of each
 * subdomain, rows[*union_blocks] = the block row of A behind each union
 * block row (subdomain-major, ascending within a subdomain).  Any pointer
 * may be NULL.  VB_EINVAL for a handle of another kind.                      */
vb_status vbarms_dd_layout(vbarms_prec M, int* nparts, int* overlap, int* restricted, int64_t* union_blocks,
                           int32_t* part, int64_t* dstart, int32_t* rows);

/* The Schur-complement global preconditioner of Section 5 (eq. paral,
 * eq. gschur, eq. loc_var_schur), all subdomains on one GPU.  Subdomains as
 * in vbarms_dd_factor with overlap 0.  A block row of subdomain i is an
 * interface row when a stored block of A couples it, as row or as column, to
 * another subdomain; the others are interior.  A_i lists its interior rows,
 * then its interface rows (each ascending): [[B_i, F_i], [E_i, C_i]].  Every
 * A_i is factored by VBARMS with (nlev, droptol, lfil, opt), all as one
 * block-diagonal union, with the interface rows kept out of every
 * independent set; they reach the last level, whose trailing block ILUT
 * factors are the LU of the approximate local Schur complement
 * S_i = C_i - E_i B_i^{-1} F_i.  One application to r = (f_i, g_i):
 *   z = S_i^{-1} g'_i           (interface part of the local solve of r_i)
 *   y = msteps steps of GMRES (y_0 = 0, modified Gram-Schmidt, Givens
 *       rotations, early stop on a zero Arnoldi norm) on (I + S^{-1} E) y = z,
 *       E the couplings E_ij between interface rows of different subdomains:
 *       the global system eq. gschur preconditioned by blockdiag(S_i)
 *   u_i = B_i^{-1} (f_i - F_i y_i)  (the local solve of r_i whose last-level
 *       backward sweep keeps the interface unknowns at y_i)
 * and returns (u_i, y_i).  The inner steps read their Hessenberg columns on
 * the host, so an application synchronizes the stream msteps + 1 times.  The
 * handle works with vbarms_apply, vbarms_apply_static (one application's
 * scratch: five vectors of n, msteps + 5 interface vectors and the union
 * solve's own), fgmres_solve and vbarms_prec_stats; vbarms_prec_export /
 * _vector / _kernel_stats describe the union's factorization.  A: handle of
 * vbarms_compress or vbarms_vbsr_from_blocks (input, not consumed).
 * Errors: VB_EINVAL (nparts outside [1, 4096], msteps outside [1, 1000],
 * nlev < 0, droptol < 0), then as vbarms_factor.                            */
vb_status vbarms_dd_schur_factor(vbarms_vbsr A, int nparts, int msteps, int nlev, double droptol, int lfil,
                                 const vbarms_opts* opt, vbarms_prec* out);

/* Layout of a vbarms_dd_schur_factor handle: nparts, msteps, the interface
 * size (scalars and block rows); part[nblk(A)] and iface[nblk(A)] = the
 * subdomain and the interface flag of every block row of A; rows[nblk(A)] =
 * the block row of A behind each union block row (each subdomain's interior
 * rows, then its interface rows); nint[nparts] = the interior block rows of
 * each subdomain.  Any pointer may be NULL.  VB_EINVAL for a handle of
 * another kind.                                                              */
vb_status vbarms_dd_schur_layout(vbarms_prec M, int* nparts, int* msteps, int64_t* ng, int64_t* ngb, int32_t* part,
                                 int32_t* iface, int32_t* rows, int64_t* nint);

/* y = M^{-1} x (Alg. 2).  x, y: device double[n], original numbering, must
 * not alias.  Runs on the stream of the matrix the handle was built from.   */
vb_status vbarms_apply(vbarms_prec M, const double* x, double* y);

/* y[m] = M[m]^{-1} x[m] for m < nmat (Alg. 2 per matrix).  Handles of one
 * batched factorization are served by a single application of the batch's
 * preconditioner.  x[m], y[m]: device double[n_m], original numbering, not
 * aliased.                                                                  */
vb_status vbarms_apply_batched(int nmat, const vbarms_prec* M, const double* const* x, double* const* y);

/* y = M^{-1} x like vbarms_apply, but allocating nothing: for callers that
 * cannot allocate device memory when they apply the preconditioner -- solver
 * loops with a fixed memory budget that forbid allocator calls once set-up
 * is over, or applications whose device memory belongs to another runtime's
 * pool and that give this library no allocator.  The paper has no
 * counterpart; this is an interface convenience.
 * All scratch comes from one file-scope device array of
 * vbarms_apply_static_max_bytes() bytes (64 MiB) that every GPU loading the
 * library holds until the process exits.  A factorization that needs more
 * is rejected with VB_EINVAL (use vbarms_apply then); the need grows with
 * the scalar sizes of all levels and with the last level's block rows, and
 * vbarms_apply_static_need tells it for a given handle.  x, y: device
 * double[n] on the handle's device, original numbering, no aliasing; the
 * call synchronizes the handle's stream before returning.  The first call on
 * a device does a set-up: it looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  Every call shares the
 * same array and it keeps
 * the previous call's contents (the call clears what must start at zero):
 * calls that overlap on the GPU -- from several host threads, or on several
 * streams -- race and must be serialized by the caller.  Handles of a
 * batched factorization are rejected (VB_EINVAL).                          */
vb_status vbarms_apply_static(vbarms_prec M, const double* x, double* y);

/* Size in bytes of the fixed scratch array of vbarms_apply_static. */
uint64_t vbarms_apply_static_max_bytes(void);

/* *bytes = the scratch vbarms_apply_static needs for M (no device work); a
 * handle fits when it is at most vbarms_apply_static_max_bytes().  The paper
 * has no counterpart.  VB_EINVAL for NULL arguments or a handle of a batched
 * factorization.                                                            */
vb_status vbarms_apply_static_need(vbarms_prec M, uint64_t* bytes);

/* Right-preconditioned flexible GMRES(restart) on A x = b (FP64 Arnoldi with
 * modified Gram-Schmidt, Givens rotations, true residual at every restart).
 * M may be NULL (no preconditioner).  b, x: device double[n] in the original
 * numbering; x holds the initial guess on entry and the solution on exit.
 * Stops when ||b - A x||_2 <= rtol ||b||_2.  *iters = total inner steps,
 * *relres = final true relative residual.  VB_ENOCONV when maxit is reached
 * (x, iters and relres are still set).                                      */
vb_status fgmres_solve(vbarms_vbsr A, vbarms_prec M, const double* b, double* x, double rtol,
                       int restart, int maxit, int* iters, double* relres);

/* Statistics of a factorization: levels performed, the memory ratio
 * (stored factor scalars / nnz(A)) and wall seconds of the setup phases
 * (phase_s[0..7]: scale, ordering, gather, pivot LU, W, G, Schur, last-level
 * ILUT; any pointer may be NULL).                                           */
vb_status vbarms_prec_stats(vbarms_prec M, int* levels_used, double* mem_ratio, double* phase_s);

/* Export one factor of level lev (0 <= lev < levels: which = 0 scaled level
 * matrix, 1 pivot LU blocks, 2 F, 3 E, 4 C, 5 W, 6 G, 7 S, and on a level
 * factored with group_size > 1: 10 the group multipliers (below the
 * diagonal of Ltilde), 11 the group part of Ubar; lev == levels:
 * which = 0 scaled last-level matrix, 1 pivot LU blocks, 8 L_S, 9 U_S) as
 * host VBCSR arrays with values converted to double.  Call once with the
 * array pointers NULL to get the sizes.                                     */
vb_status vbarms_prec_export(vbarms_prec M, int lev, int which, int64_t* nbr, int64_t* nbc,
                             int64_t* nnzb, int64_t* nval, int32_t* rsz, int32_t* csz,
                             int64_t* bptr, int32_t* bcol, int64_t* voff, double* val);

/* Export a per-level vector: which = 0 row scaling r, 1 column scaling c,
 * 2 Step 3 weights w (doubles, into d); 3 the ordering P_I (D supernodes
 * ascending then C supernodes ascending; with groups, the groups by their
 * smallest member, members ascending), 4 GEPP pivots, 5 pivot precision
 * tags (1 = FP64 kept), 6 the group boundaries over the D rows of a level
 * factored with group_size > 1 (int32, into iv).  *len receives the length;
 * pass NULL arrays to query it.                                             */
vb_status vbarms_prec_vector(vbarms_prec M, int lev, int which, double* d, int32_t* iv, int64_t* len);

/* Measured launches of one kernel of a factorization, timed with CUDA events
 * on the factorization's stream: kernel 0 = the numeric phase of the Schur
 * complement S = C - G W (Eq. 6), one launch per level.  *launches = count,
 * *ms = summed device time, *bytes = summed algorithmic bytes (C, G, W read
 * and S written once, values plus index arrays), *flops = summed
 * 2 n_r n_Y n_s over the block triples.  Any pointer may be NULL.           */
vb_status vbarms_prec_kernel_stats(vbarms_prec M, int kernel, int* launches, double* ms, double* bytes,
                                   double* flops);

/* The per-warp workspace the last-level ILUT of M ran with ("tile shape"
 * of its kernel): slots (blocks of a working row held in shared memory),
 * value_bytes (their values), warps_per_sm; source = 0 default (last level
 * under 16384 block rows), 1 chosen by timing the candidate shapes on a
 * prefix of this factorization's own rows (tune_s seconds of timing), 2
 * taken from an earlier timing of a matrix of the same device, precision and
 * class of row sizes in this process.  A prefix of the ILUT's row order is
 * factored exactly on its own, so the timing needs no other data.  Any
 * pointer may be NULL.                                                      */
vb_status vbarms_prec_ilut_geometry(vbarms_prec M, int* slots, int* value_bytes, int* warps_per_sm, int* source,
                                    double* tune_s);

/* Length (in rows) of the longest chain of waits in M's last-level block
 * ILUT: every row waits for each pending L column of its working row,
 * dropped multipliers included, so this chain, times the latency from a
 * dependency's publication to the row's own, bounds the kernel's time from
 * below whatever the number of warps.  The kept L pattern's depth is shorter
 * (a dropped multiplier leaves no block).                                   */
vb_status vbarms_prec_ilut_chain(vbarms_prec M, int64_t* links);

/* How the pivot phase (GEPP of every pivot block) of reduction level lev ran:
 * it is one persistent launch over the pivot blocks flattened into block-size
 * classes (<= 4, <= 8, <= 16, <= 32, more); counts[5] receives the blocks per
 * class, modes[5] the mode each class ran in (0: one thread per block, 1: one
 * warp per block; both give the same factors bit for bit), source = 0
 * defaults, 1 a class was timed in both modes on a copy of this level's own
 * blocks (classes of at least 1024 blocks), 2 modes taken from an earlier
 * timing in this process on the same device and precision.  Levels factored
 * with group_size > 1 run their pivots inside the group sweeps (all zero).
 * Any pointer may be NULL; VB_EINVAL for lev outside [0, levels).           */
vb_status vbarms_prec_pivot_tiles(vbarms_prec M, int lev, int* counts, int* modes, int* source);

/* Number of kernels this library has launched since it was loaded (all
 * threads, all handles); read it before and after a call to count the
 * launches of that call.                                                   */
uint64_t vbarms_launch_count(void);

/* Number of device allocations this library has made since it was loaded
 * (all threads, all handles; every allocation of the library is counted).
 * Read it before and after a call to see whether that call allocated.      */
uint64_t vbarms_alloc_count(void);

void vbarms_vbsr_destroy(vbarms_vbsr A);
void vbarms_prec_destroy(vbarms_prec M);

/* Message of the last failed call on this thread ("" if none). */
const char* vbarms_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* VBARMS_H */

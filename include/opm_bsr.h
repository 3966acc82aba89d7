/*
 * opm_bsr.h -- C ABI of a GB300 (sm_103a) solver for 3x3 block-sparse
 * (BSR) black-oil Jacobians: ILU0-preconditioned BiCGStab.
 *
 * The problem statement follows arXiv 2309.11488 ("An Evaluation and
 * Comparison of GPU Hardware and Solver Libraries for Accelerating the OPM
 * Flow Reservoir Simulator"):
 *   - matrix format: block-CSR with 3x3 blocks stored contiguously and
 *     row-major inside each block (Section 4.1; Section 4.7, figure "Memory
 *     layout of blocks in OPM", left panel; Section 4.3 on row-major Dune
 *     blocks);
 *   - preconditioner: ILU0 without fill (Section 2.2, Algorithms 1 and 2);
 *   - parallel schedule: level scheduling or graph colouring of the rows,
 *     with the matrix reordered once (Section 4.4);
 *   - solver: BiCGStab built from SpMV, axpy, dot and norm (Section 4.2),
 *     stopping at a relative residual reduction rtol or after maxit
 *     iterations, Dune's defaults being 1e-2 and 200 (Section 4.2);
 *   - a solver failure is reported rather than handled (the paper falls back
 *     to the CPU solver, Section 4.11; this library returns a status).
 *
 * Conventions for every entry point:
 *   - nb = number of block rows (cells); vectors hold 3*nb doubles, the 3
 *     unknowns of a cell contiguous, in the caller's (natural) row order.
 *   - rowptr[nb+1] is 0-based and non-decreasing, colidx[nnzb] (nnzb =
 *     rowptr[nb]) is strictly increasing inside every row, and every row holds
 *     its diagonal block.  vals[9*nnzb] stores block m's entry (r, c) at
 *     vals[9*m + 3*r + c].
 *   - A pointer argument may be host memory or device memory of the current
 *     device; the library tells them apart with cudaPointerGetAttributes.
 *     It never keeps a caller pointer past the return of the call.
 *   - Work is issued on the stream given in opm_options (NULL = the legacy
 *     default stream) and every call has completed when it returns.
 *   - No call traps, aborts or exits.  Device-side failures (a singular
 *     pivot, a bounded wait that expired) are written to a status word in
 *     device memory and returned as a negative opm_status.
 *   - A handle is not thread-safe; distinct handles may be used from
 *     distinct host threads.
 */
#ifndef OPM_BSR_H
#define OPM_BSR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct opm_solver *opm_handle; /* opaque, owned by the library */
typedef struct opm_batch_s *opm_batch; /* opaque set of handles solved together */
typedef struct opm_analysis_s *opm_analysis; /* opaque symbolic analysis kept on the host */

typedef enum {
  OPM_OK = 0,
  OPM_NOT_CONVERGED = 1,   /* maxit reached; x holds the last iterate          */
  OPM_ERR_ARG = -1,        /* bad argument (NULL handle, nb < 0, bad option)   */
  OPM_ERR_PATTERN = -2,    /* rowptr not monotone, colidx unsorted, duplicate
                              or out of range                                  */
  OPM_ERR_NO_DIAG = -3,    /* a row has no diagonal block                      */
  OPM_ERR_ZERO_PIVOT = -4, /* singular 3x3 pivot in ILU0; opm_last_error_row  */
  OPM_ERR_BREAKDOWN = -5,  /* BiCGStab breakdown: rho, (r^,v), (t,t) or omega
                              exactly zero                                     */
  OPM_ERR_NONFINITE = -6,  /* non-finite right-hand side                       */
  OPM_ERR_OOM = -7,        /* device allocation failed                         */
  OPM_ERR_TIMEOUT = -8,    /* a bounded device-side wait expired               */
  OPM_ERR_CUDA = -9        /* a CUDA runtime call failed                       */
} opm_status;

/* Row order used for the parallel schedule (Section 4.4). */
enum {
  OPM_SCHED_AUTO = 0,    /* the library picks (currently: OPM_SCHED_COLOUR_KEMPE) */
  OPM_SCHED_NATURAL = 1, /* caller's order; sequential dependency chains      */
  OPM_SCHED_LEVEL = 2,   /* level scheduling: same factors as natural order   */
  OPM_SCHED_COLOUR = 3,  /* greedy graph colouring, rows in natural order: a
                            different ILU0                                    */
  OPM_SCHED_COLOUR_SL = 4, /* greedy graph colouring, rows in smallest-last
                            order (Matula & Beck 1983: repeatedly remove a row
                            of least remaining degree, ties to the lowest row;
                            colour in reverse removal order): at most one more
                            colour than the pattern's degeneracy, usually
                            fewer colours than natural order                 */
  OPM_SCHED_COLOUR_KEMPE = 5 /* smallest-last colouring, then the highest
                            colour classes emptied by Kempe-chain exchanges
                            (Kempe 1879) while possible: each row of the top
                            class takes a free lower colour, or swaps a pair
                            of lower colours on a bounded chain that frees
                            one.  Fewer colours, hence fewer small phases   */
};

/* Storage precision of the ILU0 factors.  The Krylov recurrences, dots,
 * norms, the SpMV with A and the final true residual are FP64 in both. */
enum {
  OPM_PREC_FP64 = 0,        /* factors and triangular solves in FP64          */
  OPM_PREC_FP32_FACTORS = 1 /* factors stored and triangular solves run in
                               FP32 with FP32 accumulation                    */
};

/* Launch structure of the sweeps over the schedule's phases (runs of
 * mutually independent rows: the levels or colours). */
enum {
  OPM_SWEEP_AUTO = 0,        /* per-phase launches up to 1024 phases        */
  OPM_SWEEP_PER_PHASE = 1,   /* one kernel launch per phase                 */
  OPM_SWEEP_COOPERATIVE = 2  /* one cooperative launch walking all phases,
                                with a bounded grid barrier between them    */
};

typedef struct opm_options {
  int32_t schedule;      /* OPM_SCHED_*                                       */
  int32_t precision;     /* OPM_PREC_*                                        */
  void *stream;          /* cudaStream_t to issue work on; NULL = default     */
  int32_t chunk;         /* BiCGStab iterations per body of the device-side
                            solve loop (the loop condition is tested after
                            each body); 0 = default (2)                      */
  int32_t spin_limit_us; /* bound of every device-side wait in microseconds;
                            0 = default (2,000,000)                           */
  int32_t debug_skip_item; /* test hook, -1 = off: the CTA with this index
                            never arrives at the grid barriers of the
                            cooperative sweep kernels, so the other CTAs'
                            waits expire after spin_limit_us
                            (OPM_ERR_TIMEOUT)                                */
  int32_t profile_kernels; /* nonzero: record CUDA events around every kernel
                            (also inside the iteration graph) and accumulate
                            per-kernel device time in opm_timing             */
  int32_t sweep_launch;  /* how the factorisation and the triangular sweeps
                            walk the phases: OPM_SWEEP_AUTO, _PER_PHASE or
                            _COOPERATIVE                                     */
  int32_t small_phase_slices; /* one launch per phase: phases of at most this
                            many 32-row slices take the latency form (two
                            warps per CTA, constant data loaded before the
                            wait for the preceding kernel), larger ones the
                            throughput form; 0 = default (10 per SM of the
                            device), -1 = throughput form for every phase   */
  int32_t cp_sweeps;     /* 0 = exact ILU0 by phases (Algorithm 2).  k > 0 =
                            the fine-grained iterative ILU0 of Chow & Patel
                            (the "Chow Patel ILU0" of Section 3's library
                            table): from the guess L_ij = A_ij inv(A_jj),
                            U_ij = A_ij, k synchronous sweeps of
                              s = A_ij - sum_{k'<min(i,j)} L_ik' U_k'j,
                              L_ij = s inv(U_jj), U_ij = s (i <= j),
                            every block of the pattern at once, each sweep
                            reading the previous one.  Reaches the ILU0
                            factors after as many sweeps as the longest
                            dependency chain; the schedule still orders the
                            rows.  At most 4096; a second factor buffer is
                            allocated                                         */
  int32_t tri_sweeps;    /* 0 = exact triangular solves (Algorithm 1).  k > 0
                            = k Jacobi sweeps per triangle (Anzt, Chow &
                            Dongarra; the application half of the same
                            table entry): y <- rhs - L y from y = rhs, then
                            z <- inv(U_ii)(y - U_off z) from z = inv(U_ii) y,
                            every row at once.  At most 64.  Used by every
                            preconditioner application (BiCGStab, GMRES,
                            opm_ilu_apply).  For a batch both counts are the
                            batch's own options                               */
  int32_t product_reuse; /* 0 = default: with FP64 factors and exact
                            triangular solves (tri_sweeps = 0), the two
                            BiCGStab products that follow a preconditioner
                            application, v = A p^ with p^ = inv(LU) p, use
                            that ILU0 makes (LU)_ij = A_ij on the pattern: a
                            row with no block left of its diagonal (all of
                            its blocks in the preconditioner) takes
                            (A p^)_i = p_i, and a row whose upper blocks no
                            elimination product changed takes
                            sum_{j>i} A_ij p^_j from the backward sweep's
                            sum_{j>i} U_ij p^_j, walking only its diagonal
                            and lower blocks.  Equal to the plain product in
                            exact arithmetic (Eisenstat's observation for
                            such preconditioners, SIAM J. Sci. Stat. Comput.
                            2, 1981).  -1 = off: every product walks all of
                            A.  FP32 factors never use it (their U is not
                            A's to FP64 accuracy)                            */
  int32_t reserved;
} opm_options;

/* Largest nb a handle or an analysis accepts: row counts rounded up to
 * whole tiles and slices stay within int32. */
#define OPM_MAX_ROWS 2147479551

/* Fill *opt with the defaults (AUTO schedule, FP64, default stream). */
void opm_options_default(opm_options *opt);

/*
 * Symbolic analysis and first factorisation.  Validates the pattern
 * (Section 4.1: the bridge flattens the BCRS pattern; the diagonal check of
 * the paper's per-solve table moves here), computes the level or colour
 * schedule and the row permutation (Section 4.4), builds the library's
 * permuted device copy of the matrix and factorises it (Algorithm 2).
 *   0 <= nb <= OPM_MAX_ROWS, else OPM_ERR_ARG; rowptr, colidx, vals as above
 *   (host or device); opt may be NULL.  The block count is bounded by the
 *   int32 row pointers (below 2^31); device memory binds well before either
 *   bound: per block the values, the factors and the index maps, per row
 *   about fifteen 3-vectors (opm_get_info reports the bytes held).
 *   On success *out receives a new handle.  On OPM_ERR_ZERO_PIVOT *out still
 *   receives the handle (its factors invalid) so that opm_last_error_row can
 *   be read and opm_ilu0_factor retried with other values; the caller
 *   destroys it.  On any other failure *out = NULL and, for pattern errors,
 *   opm_last_error_row(NULL) returns the offending row for this host thread.
 * Returns OPM_OK, OPM_ERR_ARG, OPM_ERR_PATTERN, OPM_ERR_NO_DIAG,
 * OPM_ERR_ZERO_PIVOT, OPM_ERR_OOM, OPM_ERR_TIMEOUT or OPM_ERR_CUDA.
 */
opm_status opm_bsr_create(int32_t nb, const int32_t *rowptr, const int32_t *colidx,
                          const double *vals, const opm_options *opt, opm_handle *out);

/*
 * Block-Jacobi ILU0 (Section 4.5): as opm_bsr_create, but the preconditioner
 * keeps only the blocks that join two rows of the same partition; blocks
 * between partitions stay in the matrix (SpMV, true residual) and out of
 * the factors.  Schedule, permutation and factors follow the reduced
 * pattern, so fewer blocks give more parallelism (fewer levels or colours)
 * at the cost of a weaker preconditioner.  Each refactorisation copies the
 * kept blocks from the caller's values by a precomputed index gather (the
 * paper's copy-indexes loop), fused into the factorisation.
 *   part: nb partition labels (any int32 values; rows with equal labels
 *   form a partition), host or device, read during the call only; the
 *   paper takes the partition from the simulator's transmissibility-
 *   weighted grid partitioner.  Other arguments and returns as
 *   opm_bsr_create; part == NULL with nb > 0 is OPM_ERR_ARG.
 */
opm_status opm_bsr_create_jacobi(int32_t nb, const int32_t *rowptr, const int32_t *colidx,
                                 const double *vals, const int32_t *part, const opm_options *opt,
                                 opm_handle *out);

/*
 * The symbolic analysis alone, on the host (no device, no handle): the same
 * validation, schedule, permutation and phases opm_bsr_create /
 * opm_bsr_create_jacobi compute (Section 4.4), for inspecting a schedule or
 * choosing one without a GPU.
 *   rowptr, colidx (and part, which may be NULL) must be host memory.
 *   schedule: OPM_SCHED_*; perm (may be NULL): nb entries, perm[new] = old.
 *   info (may be NULL) receives the counts.
 *   Returns OPM_OK or the pattern error of opm_bsr_create (the offending row
 *   via opm_last_error_row(NULL)); OPM_ERR_ARG on a bad argument (nb
 *   outside 0 .. OPM_MAX_ROWS included).
 */
typedef struct opm_analysis_info {
  int32_t schedule;    /* schedule used (never OPM_SCHED_AUTO)               */
  int32_t nsets;       /* levels or colours (1 for natural order)            */
  int32_t nphases;     /* runs of mutually independent rows the sweeps walk  */
  int32_t rows_identity; /* rows with no block left of the diagonal and all
                          blocks kept: a product after an application takes
                          (A p^)_i = p_i there (opm_options.product_reuse)   */
  int64_t nnzb_kept;   /* blocks in the preconditioner's pattern             */
  int64_t nnzb_lower;  /* strictly lower kept blocks of the permuted matrix  */
  int64_t nnzb_upper;
  int64_t nupdates;    /* ILU0 update products A_ij -= L_ik U_kj per
                          factorisation (Algorithm 2's inner loop)           */
  int64_t nnzb_product; /* blocks of A a product after an application walks
                          with product_reuse (nnzb without it)             */
  int32_t rows_reuse;  /* rows that take their upper sum from the backward
                          sweep with product_reuse                         */
  int32_t reserved2;
} opm_analysis_info;
opm_status opm_bsr_analyse(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const int32_t *part,
                           int32_t schedule, int32_t *perm, opm_analysis_info *info);

/*
 * A kept symbolic analysis (Section 4.4: the pattern, hence its analysis,
 * stays the same for the whole simulation).  opm_analysis_create runs the
 * analysis of opm_bsr_create (or, with part non-NULL, of
 * opm_bsr_create_jacobi) once and keeps its result in host memory;
 * opm_bsr_create_from_analysis then makes handles of that pattern without
 * analysing again: it allocates the handle's device memory, uploads the
 * kept schedule, layouts and update lists, and factorises vals.  A server
 * that frees a pattern's device memory (destroying its handles) and later
 * needs the pattern again pays the upload and the first factorisation, not
 * the analysis.
 *   opm_analysis_create: rowptr, colidx, part as in opm_bsr_analyse (host
 *     or device memory); schedule: OPM_SCHED_*.  Returns OPM_OK, OPM_ERR_ARG,
 *     a pattern error (row via opm_last_error_row(NULL)) or OPM_ERR_OOM.
 *   opm_bsr_create_from_analysis: vals as in opm_bsr_create (host or device,
 *     9*nnzb doubles, the caller's block order); opt as in opm_bsr_create
 *     except that its schedule is ignored (the analysis fixed it).  Returns
 *     the statuses of opm_bsr_create.  The analysis may be destroyed while
 *     handles made from it live: they hold their own copies.
 *   opm_analysis_get_info: the analysis's counts (opm_bsr_analyse's info)
 *     and, when perm is non-NULL, its permutation (nb entries).
 * The analysis object is used by one host thread at a time.
 */
opm_status opm_analysis_create(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const int32_t *part,
                               int32_t schedule, opm_analysis *out);
opm_status opm_bsr_create_from_analysis(opm_analysis a, const double *vals, const opm_options *opt,
                                        opm_handle *out);
opm_status opm_analysis_get_info(opm_analysis a, int32_t *nb, int64_t *nnzb, int32_t *perm,
                                 opm_analysis_info *info);
void opm_analysis_destroy(opm_analysis a);

/*
 * Restarted GMRES(m) (Section 2 names restarted GMRES as OPM's other Krylov
 * solver; method of Saad & Schultz 1986), with the handle's ILU0 (or
 * block-Jacobi ILU0) as right preconditioner, x0 = 0.  Arnoldi with
 * classical Gram-Schmidt applied twice; Givens rotations; the residual
 * estimate is tested after every step against rtol ||b|| (the stopping rule
 * of Section 4.2); each cycle of `restart` steps (0 = 30, at most 64) ends
 * with x += inv(M) V y and the next starts from the true residual.
 *   b, x as for opm_bicgstab_solve; maxit bounds the Arnoldi steps over all
 *   cycles; *iters = steps taken; *relres = true ||b - A x|| / ||b|| (with
 *   the wells' terms when wells are set).  Synchronous on the handle's
 *   stream; uses (m + 1) extra vectors of device memory, kept for later
 *   calls.  Not available on batches.
 * Returns OPM_OK, OPM_NOT_CONVERGED, OPM_ERR_ARG, OPM_ERR_ZERO_PIVOT (no
 * valid factors), OPM_ERR_BREAKDOWN (a zero rotation), OPM_ERR_NONFINITE,
 * OPM_ERR_OOM or OPM_ERR_CUDA; on negative codes x is zero-filled.
 */
opm_status opm_gmres_solve(opm_handle h, const double *b, double *x, double rtol, int32_t maxit,
                           int32_t restart, int32_t *iters, double *relres);

/*
 * Standard wells kept separate (Section 4.6): from now on every product
 * with the system operator (the solver's SpMVs, the true residual and
 * opm_spmv) is y = A x - sum over wells of C_w^T inv(D_w) B_w x, while the
 * preconditioner stays the ILU0 of A.  For a standard well D_w is a single
 * 4x4 block and B_w, C_w one row of 4x3 blocks, one per perforated cell.
 *   nwells >= 0 (0 removes the wells); wptr[nwells+1] (wptr[0] = 0,
 *   non-decreasing): well w perforates cells[wptr[w] .. wptr[w+1]-1]
 *   (caller's row numbering, each in [0, nb)); B, C: 12 doubles per
 *   perforation (4x3 row-major, in the order of cells); Dinv: 16 doubles
 *   per well, the inverted D (4x4 row-major), as the paper's simulator
 *   hands it over.  Host or device pointers, copied during the call; call
 *   again after each Newton step with the new values.  Synchronises the
 *   handle's stream first.
 * Returns OPM_OK, OPM_ERR_ARG (bad sizes or cells), OPM_ERR_OOM or
 * OPM_ERR_CUDA.
 */
opm_status opm_set_wells(opm_handle h, int32_t nwells, const int32_t *wptr, const int32_t *cells,
                         const double *B, const double *C, const double *Dinv);

/*
 * ILU0 refactorisation in place (Algorithm 2) with the analysis kept
 * (Section 4.4: the pattern, hence the schedule, does not change during a
 * simulation).  vals (host or device, 9*nnzb doubles, the caller's block
 * order) replaces the matrix values; vals = NULL refactors the values the
 * handle already holds.  The SpMV in later solves uses the new values.
 * Returns OPM_OK, OPM_ERR_ARG, OPM_ERR_ZERO_PIVOT (row in
 * opm_last_error_row, caller's numbering), OPM_ERR_TIMEOUT or OPM_ERR_CUDA.
 */
opm_status opm_ilu0_factor(opm_handle h, const double *vals);

/*
 * Solve A x = b by BiCGStab right-preconditioned with the current ILU0
 * factors (Section 4.2), x0 = 0, shadow residual r^ = b.  Stops when
 * ||r_k||_2 <= rtol * ||b||_2, tested after each half step, or after maxit
 * iterations.  b, x: 3*nb doubles, host or device, caller's order; x is
 * output only.  *iters (may be NULL) = iterations begun, a half-step exit
 * counting as its iteration; *relres (may be NULL) = true
 * ||b - A x||_2 / ||b||_2 computed in FP64 after the solve.  b = 0 gives
 * x = 0, iters = 0, relres = 0 and OPM_OK.
 * Returns OPM_OK, OPM_NOT_CONVERGED (x = last iterate), OPM_ERR_BREAKDOWN,
 * OPM_ERR_NONFINITE, OPM_ERR_TIMEOUT, OPM_ERR_ARG or OPM_ERR_CUDA; on a
 * negative status x is zero-filled.
 */
opm_status opm_bicgstab_solve(opm_handle h, const double *b, double *x, double rtol,
                              int32_t maxit, int32_t *iters, double *relres);

/* y = A x with the handle's current values (Section 4.3); x, y host or
 * device, 3*nb doubles, caller's order. */
opm_status opm_spmv(opm_handle h, const double *x, double *y);

/* z = U^-1 L^-1 r with the current factors (Algorithm 1, equations 3-4);
 * r, z host or device, 3*nb doubles, caller's order. */
opm_status opm_ilu_apply(opm_handle h, const double *r, double *z);

/* Release the handle and all its device memory.  NULL is ignored.
 * Device memory of handles, batches and wells comes from one memory pool per
 * device that the library owns, allocated and freed in stream order on the
 * owner's stream (so creating or destroying a handle does not wait for work
 * on other streams); memory a destroyed handle frees stays in the pool for
 * later handles and batches and is not returned to the system before the
 * process exits. */
void opm_destroy(opm_handle h);

/* Static text of a status code. */
const char *opm_status_str(opm_status s);

/* Row (caller's numbering) of the handle's last OPM_ERR_ZERO_PIVOT, or -1;
 * with h = NULL, the row of this thread's last failed opm_bsr_create
 * (OPM_ERR_PATTERN or OPM_ERR_NO_DIAG), or -1. */
int32_t opm_last_error_row(opm_handle h);

typedef struct opm_info {
  int32_t nb;
  int32_t schedule;    /* schedule in use (never OPM_SCHED_AUTO)            */
  int32_t precision;
  int32_t nsets;       /* number of levels or colours (1 for natural)       */
  int64_t nnzb;
  int64_t nnzb_lower;  /* strictly lower blocks of the permuted matrix      */
  int64_t nnzb_upper;
  int64_t device_bytes; /* device memory held by the handle                 */
  int32_t nphases;     /* runs of mutually independent rows the sweeps walk
                          (the levels or colours; for natural order, runs of
                          consecutive independent rows)                      */
  int32_t rows_identity; /* as in opm_analysis_info                          */
  int64_t nupdates;    /* ILU0 update products A_ij -= L_ik U_kj per
                          factorisation (Algorithm 2's inner loop)          */
  int64_t nnzb_product; /* blocks of A each BiCGStab product after an
                          application walks in this handle's own solves
                          (nnzb when product_reuse does not apply)         */
  int32_t rows_reuse;  /* as in opm_analysis_info (0 when product_reuse
                          does not apply)                                  */
  int32_t reserved2;
} opm_info;

opm_status opm_get_info(opm_handle h, opm_info *info);

/* perm[new] = old row (host array of nb int32): the schedule's order. */
opm_status opm_get_permutation(opm_handle h, int32_t *perm);

/*
 * Copy the current factors out in the permuted matrix's CSR order: lu (host,
 * 9*nnzb doubles) holds L's strictly-lower blocks (unit diagonal implied) and
 * U's strictly-upper blocks in the pattern of P A P^T with columns
 * ascending; the diagonal-block positions of lu receive inv(U_ii), which the
 * library stores instead of U_ii.  dinv (host, 9*nb doubles, schedule order)
 * also receives inv(U_ii).  FP32 factors are widened exactly.  For a
 * block-Jacobi handle the blocks outside the preconditioner's pattern read
 * as zero.  Either pointer may be NULL.
 */
opm_status opm_get_factors(opm_handle h, double *lu, double *dinv);

/* Kernels of the path, for opm_timing's per-kernel counters. */
enum {
  OPM_KERNEL_FACTOR = 0, /* value permutation + ILU0 decomposition          */
  OPM_KERNEL_APPLY = 1,  /* forward + backward substitution (2 per iteration) */
  OPM_KERNEL_SPMV = 2,   /* SpMV with fused dot products (2 per iteration)  */
  OPM_KERNEL_UPDATE = 3, /* x, r update and stopping rule                   */
  OPM_KERNEL_SETUP = 4,  /* b permutation and ||b||                         */
  OPM_KERNEL_FINISH = 5, /* true residual and x permutation                 */
  OPM_KERNEL_COUNT = 6
};

/* Device time, in milliseconds, of the last solve (iterate_ms: setup,
 * iterations and true residual; setup_ms and finish_ms are 0) and of the
 * last factorisation, measured with CUDA events on the handle's stream; the
 * number of kernels the handle has launched (graph nodes included); and,
 * with opm_options.profile_kernels, per-kernel device time and launch counts
 * accumulated over the iterations that did work since the last
 * opm_reset_timing (the iterations then run from a host loop over graphs
 * with event nodes instead of the device-side loop). */
typedef struct opm_timing {
  float setup_ms, iterate_ms, finish_ms, factor_ms;
  int64_t launches;
  double kernel_ms[OPM_KERNEL_COUNT];
  int64_t kernel_count[OPM_KERNEL_COUNT];
} opm_timing;
opm_status opm_get_timing(opm_handle h, opm_timing *t);
/* Zero the launch counter and the per-kernel accumulators. */
opm_status opm_reset_timing(opm_handle h);

/*
 * Asynchronous refactor + solve (the paper's per-Newton-step pair, Section
 * 4.4 and 4.2) for serving loops: enqueues, on the handle's stream and
 * without waiting, an optional refactorisation with vals (9*nnzb doubles;
 * NULL = keep the factors) and a solve of A x = b (b, x 3*nb doubles,
 * caller's order).  Each pointer may be device or host memory: host inputs
 * are copied to the device and a host x is copied back on the same stream,
 * so with page-locked host memory (cudaHostAlloc / cudaHostRegister) the
 * whole step, transfers included, is enqueued without a host wait (the
 * paper's Section 4.11 copies of the matrix and vectors).  The pointers
 * must stay valid and untouched until opm_solve_wait returns.  While a
 * launch is pending the handle accepts only opm_solve_ready and
 * opm_solve_wait.
 * opm_solve_ready returns 1 when the work has completed (or none is
 * pending), else 0.  opm_solve_wait blocks until completion and returns
 * what opm_bicgstab_solve would (a singular pivot of the refactorisation is
 * returned as OPM_ERR_ZERO_PIVOT).  Not available with profile_kernels.
 */
opm_status opm_solve_launch(opm_handle h, const double *vals, const double *b, double *x, double rtol,
                            int32_t maxit);
int32_t opm_solve_ready(opm_handle h);
opm_status opm_solve_wait(opm_handle h, int32_t *iters, double *relres);

/*
 * Batches: many independent systems (distinct handles of one precision on
 * one device) factorised and solved by the same kernel launches, each
 * system with its own convergence state; a system that has converged skips
 * its work while the others continue.  Every system's arithmetic, including
 * the order of every reduction, is the same as when its handle is used
 * alone, so results are bitwise identical.  A batch uses the member
 * handles' device data and must be destroyed before them; members must not
 * be used on their own while a batch call on them runs.  Work goes on the
 * stream of opt (NULL = default stream); opt's schedule and precision are
 * ignored (the members fix them); its cp_sweeps and tri_sweeps apply to
 * every member (the members' second buffers are allocated on demand).
 *   opm_batch_factor: vals[i] (host or device, NULL = refactor the values
 *     system i holds; vals itself may be NULL).
 *   opm_batch_solve: b[i], x[i] host or device; rtol[i] (rtol may be NULL =
 *     1e-2 for all); per-system iters, relres and st (each may be NULL).
 *   Both return the first negative per-system status, else
 *   OPM_NOT_CONVERGED if a system did not converge, else OPM_OK.
 *   opm_batch_launch / _ready / _wait: the asynchronous form of an optional
 *   refactorisation (vals NULL = none) followed by a solve; device pointers
 *   only, valid until opm_batch_wait returns.  A member with b[i] = NULL and
 *   x[i] = NULL sits the launch out: its values, factors, state and x are
 *   not touched (its vals[i] is ignored) and opm_batch_wait reports OPM_OK,
 *   0 iterations and relres 0 for it; its share of every launch ends at
 *   once.  A serving loop keeps one batch over several resident handles and
 *   launches it with the members whose requests are ready.
 */
opm_status opm_batch_create(int32_t nsys, const opm_handle *hs, const opm_options *opt, opm_batch *out);
opm_status opm_batch_factor(opm_batch b, const double *const *vals, opm_status *st);
opm_status opm_batch_solve(opm_batch b, const double *const *bv, double *const *xv, const double *rtol,
                           int32_t maxit, int32_t *iters, double *relres, opm_status *st);
opm_status opm_batch_launch(opm_batch b, const double *const *vals, const double *const *bv,
                            double *const *xv, const double *rtol, int32_t maxit);
int32_t opm_batch_ready(opm_batch b);
opm_status opm_batch_wait(opm_batch b, int32_t *iters, double *relres, opm_status *st);
void opm_batch_destroy(opm_batch b);

/*
 * Autotuner: picks the launch configuration of a pattern, or of a batch of
 * patterns solved together, by timing one refactorisation plus one solve
 * (time to solution, host clock around the synchronous calls) for each
 * candidate configuration.  The paper fixes no schedule (it reports level
 * scheduling and graph colouring side by side, Section 4.4); the candidates
 * are searched coordinate-wise:
 *   1. schedule LEVEL or COLOUR (and NATURAL when every system has at most
 *      4,096 block rows) x sweep launch PER_PHASE (only when the schedule
 *      has at most 1,024 phases) or COOPERATIVE;
 *   2. for the best of 1, iterations per loop body 1, 2 or 4;
 *   3. for the best of 2 with PER_PHASE, small_phase_slices -1 (throughput
 *      form everywhere), 0 (default) or 1 << 30 (latency form everywhere).
 * Each candidate creates its own handles (symbolic analysis included, not
 * timed), runs one untimed refactorisation + solve, then `repeats` timed
 * ones (repeats < 1 means 3) and scores their median.  A candidate whose
 * solve fails is never chosen, nor one that does not converge while
 * another does.  base (NULL = defaults) supplies the precision, stream and
 * wait bound; *best receives base with the chosen schedule, sweep_launch,
 * chunk and small_phase_slices; report (may be NULL) every candidate tried.
 * Inputs as for opm_bsr_create / opm_bicgstab_solve (host or device).
 * Returns OPM_OK when some candidate converged, OPM_NOT_CONVERGED when none
 * did but one ran, else the first candidate's error.
 */
#define OPM_TUNE_MAX 24
typedef struct opm_tune_entry {
  int32_t schedule, sweep_launch, chunk, small_phase_slices;
  int32_t status;   /* status of the last timed solve (batch: the worst)  */
  int32_t iters;    /* iterations of the last timed solve (batch: the max) */
  double ms;        /* median time of refactorisation + solve             */
} opm_tune_entry;
typedef struct opm_tune_report {
  int32_t ncand;    /* entries filled in cand                             */
  int32_t best;     /* index of the chosen entry, -1 if none              */
  opm_tune_entry cand[OPM_TUNE_MAX];
} opm_tune_report;

opm_status opm_autotune(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *vals,
                        const double *b, double rtol, int32_t maxit, int32_t repeats,
                        const opm_options *base, opm_options *best, opm_tune_report *report);
/* The batch form: system i has nb[i], rowptr[i], colidx[i], vals[i], b[i]
 * and rtol[i] (rtol may be NULL = 1e-2); the candidates' handles are
 * solved together through opm_batch_factor / opm_batch_solve. */
opm_status opm_autotune_batch(int32_t nsys, const int32_t *nb, const int32_t *const *rowptr,
                              const int32_t *const *colidx, const double *const *vals,
                              const double *const *b, const double *rtol, int32_t maxit, int32_t repeats,
                              const opm_options *base, opm_options *best, opm_tune_report *report);

/*
 * Allocation-free true residual (the paper has no counterpart: this is a
 * library convenience).  For callers that cannot allocate device memory at
 * the call site -- code running inside a simulator's own device-memory
 * arena or under a fixed memory budget, or in a process whose allocations
 * must all go through an allocator this library does not see -- it computes
 * r = b - A x and norms[0] = ||b - A x||_2, norms[1] = ||b||_2 on the
 * caller's own BSR arrays, without a handle and without allocating.
 *   nb <= 2,097,152 block rows, else OPM_ERR_ARG; rowptr, colidx, vals (the
 *   layout of opm_bsr_create), x, b, r (3*nb doubles) and norms (2 doubles)
 *   must all be device memory of the current device (host memory and
 *   another GPU's memory are refused with OPM_ERR_ARG).
 *   The pattern must be well formed: rowptr[0] = 0, non-decreasing, and
 *   rowptr[nb] no larger than the number of blocks in colidx and vals; each
 *   column in [0, nb).  It is not copied to the host for checking.  The
 *   kernel takes a row with a negative start or an end before its start as
 *   empty and skips a column outside [0, nb); either makes both norms NaN
 *   and the call return OPM_ERR_PATTERN.  A rowptr[nb] past the end of the
 *   caller's arrays cannot be detected.
 *   Work is issued on stream (NULL = default stream); the call synchronises
 *   that stream before it returns, so it cannot be recorded in a CUDA graph:
 *   do not call it on a stream that is capturing.  Returns OPM_OK,
 *   OPM_ERR_ARG, OPM_ERR_PATTERN or OPM_ERR_CUDA.
 * Its scratch is a fixed 131,328-byte array in device memory that every GPU
 * using the library holds until the process exits.  The first call on a
 * device looks up that array's device address (once per device, with the
 * device current) and keeps it.  Calls after a cudaDeviceReset of that
 * device are not supported.
 * All calls share the array: calls that overlap on the GPU race and must be
 * serialised by the caller.
 */
opm_status opm_bsr_residual_noalloc(int32_t nb, const int32_t *rowptr, const int32_t *colidx,
                                    const double *vals, const double *x, const double *b, double *r,
                                    double *norms, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* OPM_BSR_H */

/*
 * pslr.h - C ABI of the GB300 (sm_103a) implementation of the PSLR (power
 * Schur complement low-rank) preconditioner of Zheng, Xi and Saad,
 * arXiv 2002.00917, and of the FGMRES solver it preconditions.
 *
 * Notation follows the paper.  After a graph partition into s subdomains
 * (Section 2) the system reads [B E; F C] (x; y) = (f; g) (Eq. 2.1) with B, E
 * and C0 = blockdiag(C_i) block diagonal and C_g = C - C0 the coupling of
 * interface unknowns across subdomains.  The Schur complement S = C - F B^{-1} E
 * (Eq. 2.2) is split as S = C0 - E_s (Eq. 3.1); P_m = sum_{i=0}^{m}
 * (C0^{-1} E_s)^i C0^{-1} is the power series (Eq. 3.3); an r-step Arnoldi
 * process on E_rr(m) = (E_s C0^{-1})^{m+1} (Eq. 3.16, Eq. 3.19) gives V and H,
 * and G = (I - H)^{-1} - I (Eq. 3.17).  The preconditioner is Algorithm 3.
 *
 * Conventions for every entry point:
 *  - No exception crosses this boundary; each call returns a pslr_status.
 *    pslr_last_error() gives a message for the last failing call on a context.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device work is enqueued on it in stream order; a context must be
 *    used from one stream at a time.
 *  - Host arrays are read during the call and may be freed afterwards; the
 *    context copies what it keeps.  Device vectors are owned by the caller,
 *    are in the ORIGINAL ordering of A, and are column-major (n x nrhs) when
 *    nrhs > 1.  The context owns every device buffer it allocates (factors,
 *    V, G, Krylov workspace) and frees them in pslr_destroy().
 *  - Asynchronous errors (a device-side wait that ran out, a NaN) are latched
 *    in the context and reported by pslr_sync() or the next synchronising
 *    call.
 */
#ifndef PSLR_H
#define PSLR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pslr_ctx pslr_ctx;

typedef enum {
    PSLR_OK = 0,
    PSLR_ERR_ARG = 1,           /* invalid argument (sizes, pointers, CSR)          */
    PSLR_ERR_CUDA = 2,          /* a CUDA runtime call failed                       */
    PSLR_ERR_ZERO_PIVOT = 3,    /* ILU(0) or LU met a zero pivot (Algorithm 1, 3-4) */
    PSLR_ERR_BREAKDOWN = 4,     /* Arnoldi broke down; the rank was truncated       */
    PSLR_ERR_SINGULAR_IMH = 5,  /* I - H singular: Eq. 3.15 assumes it is not       */
    PSLR_ERR_NOT_CONVERGED = 6, /* FGMRES hit maxit                                 */
    PSLR_ERR_NAN = 7,           /* a NaN / Inf appeared in a device reduction       */
    PSLR_ERR_TIMEOUT = 8,       /* a device-side grid barrier gave up waiting       */
    PSLR_ERR_STATE = 9,         /* call out of order (e.g. no low-rank built yet)   */
    PSLR_ERR_TOO_LARGE = 10     /* a subdomain does not fit the on-chip working set */
} pslr_status;

/* Arithmetic of an apply: FP64 vectors and factors, or FP32 vectors and
 * factors with V stored in BF16 (accumulation in FP32). */
typedef enum { PSLR_FP64 = 0, PSLR_FP32 = 1 } pslr_prec;

typedef struct {
    /* Geometric split that stands in for the paper's METIS partition (Section
     * 2): unknown idx = i + dims[0]*(j + dims[1]*k) goes to subdomain
     * floor(i*splits[0]/dims[0]) + splits[0]*(floor(j*splits[1]/dims[1])
     * + splits[1]*floor(k*splits[2]/dims[2])).  dims[0]*dims[1]*dims[2] must
     * equal n.  Ignored when `part` is not NULL.  With dims all zero and
     * nparts > 0 the graph partition below is used instead. */
    int32_t dims[3];
    int32_t splits[3];
    const int32_t *part;  /* optional host array (length n) of subdomain ids 0..s-1 */
    int32_t factor;       /* local factors of B_i and C_i: 0 = ILU(0), 1 = exact LU
                             with partial pivoting, 2 = ILUT(drop_tol) with no fill
                             limit (Algorithm 1, steps 2-5; Section 4 runs ILUT
                             with threshold 1e-2): row i drops entries below
                             drop_tol * mean |a_ij| over its stored entries,
                             the diagonal always kept                              */
    uint64_t seed;        /* SplitMix64 seed of the Arnoldi start vector            */
    double drop_tol;      /* ILUT threshold (factor 2), >= 0; ignored otherwise     */
    int32_t setup_threads; /* host threads of the set-up (blocks, factors and packing
                              run per subdomain, as the paper's set-up runs over
                              subdomains in parallel): 0 = the machine's hardware
                              threads (at most 64), >= 1 that many; the result is
                              the same for every value                              */
    int32_t nparts;       /* with part NULL and dims {0,0,0}: partition the graph of
                             A + A^T into nparts parts (1 <= nparts <= n) by
                             recursive bisection of breadth-first level structures
                             from George-Liu pseudo-peripheral vertices (each cut
                             splits the breadth-first order of the set at
                             floor(|U| (k/2) / k)); for matrices without a grid,
                             standing in for the paper's METIS (Section 2)      */
    int32_t merge_levels; /* layout of the triangular-sweep segments the apply
                             streams: 0 = automatic (several consecutive levels
                             of a factor per segment only where two CTAs share
                             an SM and the shared-memory ring then holds fewer
                             than six segments; one level per segment
                             otherwise), 1 = always one level per segment,
                             2 = always several levels per segment.  The result
                             is the same, bit for bit, for every value; the
                             layout changes only the copies that feed the
                             sweeps                                             */
    int32_t device_factor; /* 1: the ILU(0) local factors (factor 0) are computed
                              on the GPU (pslr_ilu0_device on all B_i and C_i
                              at once) instead of on the host; the same factors
                              up to the rounding of a fused multiply-add.
                              0: on the host.  Needs factor 0; pslr_plan, which
                              touches no GPU, factors on the host regardless */
} pslr_opts;

typedef struct {
    int32_t n, s, p, q;   /* unknowns, subdomains, interior, interface             */
    int32_t m, rank;      /* series order and rank of the current low-rank term    */
    int64_t nnz_A, nnz_ilu, nnz_lr; /* Section 4: nnz(A), nnz(ILU), nnz(V) + nnz(G) */
    double fill_ilu, fill_lr, fill_total; /* Section 4 fill factors                 */
    int32_t max_interior, max_interface;  /* largest p_i and q_i                    */
    int32_t levels_B, levels_C0;          /* deepest triangular-solve level chain   */
    int64_t apply_bytes_fp64, apply_bytes_fp32; /* algorithmic bytes of one apply   */
    uint64_t layout_hash; /* pslr_plan only: FNV-1a hash (64-bit prime, 8-byte words) of the packed device
                             layout (segments, descriptors and counts of both
                             directions and precisions); 0 from a device context  */
    int32_t setup_threads; /* host threads the set-up used                        */
    int64_t layout_errors; /* pslr_plan only: violations a host-side decode of every
                              packed segment found (indices out of range, a product
                              writing a row twice, a sweep row reading a row not
                              written at an earlier barrier step, a sweep missing
                              or repeating a row); 0 for a sound layout           */
    int32_t grid[2];      /* launch shape of the persistent apply, [0] FP64, [1] FP32:
                             CTAs of the cooperative grid (0 from pslr_plan)     */
    int32_t ring[2];      /* shared-memory ring slots per CTA                       */
    int32_t ctas_per_sm[2]; /* 1, or 2 when two subdomains' CTAs share an SM (more
                               subdomains than SMs, and two CTAs' vectors and
                               rings fit an SM's shared memory)                   */
    int64_t nnz_fact_B, nnz_fact_C0; /* stored entries of the local factors L+U of
                                        all B_i and all C_i (Algorithm 1, steps 3-4) */
    int64_t nnz_E, nnz_F, nnz_Cg;    /* stored entries of E, F and C_g (Eq. 2.1, 3.1) */
    double omega;         /* 1: PSLR; otherwise the scaling of the Sec. 1 Neumann
                             polynomial the context applies (pslr_set_neumann)    */
    int32_t merged[2];    /* 1 where the sweep segments of that precision ([0]
                             FP64, [1] FP32) hold several levels (merge_levels) */
    int32_t unit_sweeps;  /* 1: forward FP64 applies run both sweeps of every local
                             solve with unit diagonals (L~ = D L D^-1, U^ = D U,
                             D = diag(1/u_rr); the right-hand sides scaled by D),
                             the form used whenever the factors have no row
                             pivots (factor 0 and 2); same solves in exact
                             arithmetic                                          */
    int32_t device_factor; /* 1 when the set-up factored on the GPU               */
    double factor_ms;      /* device_factor: time of the factorization kernel     */
} pslr_info;

/*
 * Reorder A (Section 2), extract B, E, F, C, C0, C_g (Eq. 2.1, Eq. 3.1), factor
 * every B_i and C_i (Algorithm 1, steps 1-5), and upload everything to the
 * current CUDA device.  A is host CSR: rowptr (n+1), colind (nnz, 0-based),
 * val (nnz); every row must hold its diagonal entry and columns must be in
 * range.  On success *out owns the new context and the low-rank term is empty
 * (rank 0, m = 0) until pslr_build_lowrank() or pslr_set_lowrank().
 * Errors: PSLR_ERR_ARG (bad CSR or options), PSLR_ERR_ZERO_PIVOT,
 * PSLR_ERR_TOO_LARGE (a subdomain exceeds the on-chip vector budget),
 * PSLR_ERR_CUDA.  *out is NULL on failure.
 */
pslr_status pslr_setup(int32_t n, const int32_t *rowptr, const int32_t *colind, const double *val,
                       const pslr_opts *opts, void *stream, pslr_ctx **out);

/*
 * ILU(0) on the device of a block-diagonal sparse matrix M = blockdiag(M_0,
 * ..., M_{nb-1}), the form of B and C0 (Eq. 2.1, Eq. 3.1): Algorithm 1, steps
 * 3-4, with ILU(0) as the local factorization, in the IKJ order of Saad,
 * Iterative Methods, Sec. 10.3.2 (natural order, no pivoting).  block_ptr
 * (host, nb+1 entries, block_ptr[0] = 0, block_ptr[nb] = n, non-decreasing)
 * gives the first row of each block; rowptr (n+1) and colind (host, 0-based)
 * are M's pattern: columns strictly ascending within a row, every row holding
 * its diagonal, no entry outside its row's diagonal block.  val_dev (device,
 * rowptr[n] doubles, owned by the caller) holds M's values on entry and the
 * factor on return, on M's pattern: the strictly lower part is L (unit
 * diagonal implied), the rest U.  The pattern is checked on the host before
 * any device work; one CTA per block walks the block's level sets (the rows
 * whose stored columns below the diagonal lie in earlier levels), one thread
 * per row.  Synchronous with respect to the host (stream: cudaStream_t as
 * void*).  Errors: PSLR_ERR_ARG (pattern or sizes; nothing was touched),
 * PSLR_ERR_ZERO_PIVOT (a pivot is zero; val_dev is partly factored),
 * PSLR_ERR_CUDA.  No counterpart call in the paper, whose set-up factors each
 * subdomain on its own processor.
 */
pslr_status pslr_ilu0_device(int32_t n, int32_t nb, const int32_t *block_ptr, const int32_t *rowptr,
                             const int32_t *colind, double *val_dev, void *stream);

/*
 * Host-only dry run of pslr_setup: the same validation, reordering (Section 2),
 * local factors and device layout, computed on the host without touching any
 * GPU, so it runs where there is none.  Fills *info (with series order m and
 * rank r as a later pslr_build_lowrank(m, r) would set them; apply_bytes_* is
 * the algorithmic byte count of one apply) and, when not NULL, the maps of
 * pslr_get_maps (host arrays of length n).  Same errors as pslr_setup except
 * PSLR_ERR_CUDA; the shared-memory check uses the 227 KB per-CTA limit.
 */
pslr_status pslr_plan(int32_t n, const int32_t *rowptr, const int32_t *colind, const double *val,
                      const pslr_opts *opts, int32_t m, int32_t rank, pslr_info *info,
                      int32_t *part, int32_t *is_interface, int32_t *perm);

/*
 * Algorithm 1, steps 6-8: an r-step Arnoldi process on E_rr(m) (Eq. 3.16),
 * run on the device in FP64 with classical Gram-Schmidt applied twice, from
 * the start vector v_1 = u/||u||, u_l = SplitMix64(opts.seed) output l mapped
 * to [-1,1); then G = (I - H)^{-1} - I (Eq. 3.17) in FP64.  A breakdown
 * (h_{j+1,j} <= 1e-12 ||H||_F) truncates the rank and returns
 * PSLR_ERR_BREAKDOWN with the truncated term installed, unless full_rank != 0,
 * in which case a fresh SplitMix64 vector (outputs t*q .. t*q+q-1 for the t-th
 * vector) orthogonalised against V continues the basis.  rank is capped at q.
 * Synchronises `stream`.
 */
pslr_status pslr_build_lowrank(pslr_ctx *c, int32_t m, int32_t rank, int32_t full_rank,
                               void *stream);

/*
 * Install a low-rank term directly: V is host q x rank column-major in the
 * interface numbering of pslr_get_maps(), G is host rank x rank column-major,
 * both FP64 (the FP32 form stores V in BF16 and G in FP32).  rank 0 clears it.
 */
pslr_status pslr_set_lowrank(pslr_ctx *c, int32_t m, int32_t rank, const double *V,
                             const double *G, void *stream);

/*
 * z = M^{-1} b with M^{-1} the PSLR operator of Algorithm 3 (Eq. 3.24):
 *   t = g - F B^{-1} f;  t <- t + V G V^T t;  y = P_m t;  x = B^{-1}(f - E y).
 * b_dev, z_dev: device arrays of n*nrhs elements, double for PSLR_FP64 and
 * float for PSLR_FP32, original ordering, column-major; b and z must not
 * overlap.  Enqueued on `stream`; does not synchronise.
 */
pslr_status pslr_apply(pslr_ctx *c, const void *b_dev, void *z_dev, int32_t nrhs, pslr_prec prec,
                       void *stream);

/*
 * z = M^{-T} b, the exact transpose of Algorithm 3 (derived from its block
 * form; the paper does not state it): h = g - E^T B^{-T} f;
 * w = (I + V G^T V^T) P_m^T h;  x = B^{-T}(f - F^T w);  z = (x; w).
 * Same argument conventions as pslr_apply.
 */
pslr_status pslr_apply_T(pslr_ctx *c, const void *b_dev, void *z_dev, int32_t nrhs,
                         pslr_prec prec, void *stream);

/*
 * The same operator as pslr_apply (transpose != 0: pslr_apply_T) on HOST
 * arrays: copies b (pinned or pageable host memory, n*nrhs elements of the
 * precision's type) to the device, applies, copies z back and synchronises
 * `stream`.  This is the end-to-end call of a user holding host data.
 */
pslr_status pslr_apply_host(pslr_ctx *c, const void *b_host, void *z_host, int32_t nrhs,
                            pslr_prec prec, int32_t transpose, void *stream);

/*
 * Solve A x = b (transpose != 0: A^T x = b) with right-preconditioned flexible
 * GMRES(restart) (Section 4: x0 = 0, stop when ||b - A x|| <= rtol ||b||, at
 * most maxit iterations), preconditioned by pslr_apply (or pslr_apply_T) in
 * precision `prec`.  Krylov vectors, the Hessenberg least-squares problem and
 * the residual are FP64 in every case, so with PSLR_FP32 the outer iteration
 * refines an FP32 preconditioner to FP64 accuracy.  b_dev, x_dev: device
 * double arrays of length n (nrhs = 1 per call).  *iters (cumulative over
 * restarts) and *relres (true residual ||b - A x||/||b|| in FP64) are written
 * on return.  restart is 1..127.  Synchronises `stream` once per restart cycle.
 * Returns PSLR_OK or PSLR_ERR_NOT_CONVERGED (x holds the last iterate).
 */
pslr_status pslr_solve(pslr_ctx *c, const double *b_dev, double *x_dev, double rtol,
                       int32_t restart, int32_t maxit, pslr_prec prec, int32_t transpose,
                       int32_t *iters, double *relres, void *stream);

/* y = A x (transpose: A^T x) on device double vectors of length n (FP64 SpMV
 * with the matrix given to pslr_setup, original ordering). */
pslr_status pslr_matvec(pslr_ctx *c, const double *x_dev, double *y_dev, int32_t transpose,
                        void *stream);

/*
 * Adjoint of the solve (used for differentiation, not a step of the paper):
 * for A u = b and a loss L(u), with lambda = A^{-T} dL/du (pslr_solve with
 * transpose != 0), dL/db = lambda and dL/da_ij = -lambda_i u_j for every
 * stored entry of A.  Writes grad_dev[k] for the k-th stored value of the CSR
 * given to pslr_setup (device doubles, length nnz).  Vectors: device doubles
 * of length n, original ordering.  Enqueued on `stream`.
 */
pslr_status pslr_grad_values(pslr_ctx *c, const double *lambda_dev, const double *u_dev,
                             double *grad_dev, void *stream);

/* Copy the reordering of Section 2 to host arrays of length n (any may be
 * NULL): part[v] subdomain of unknown v, is_interface[v] 0/1, perm[t] = the
 * original index of reordered unknown t (interiors by subdomain, then
 * interfaces by subdomain, each in increasing original index). */
pslr_status pslr_get_maps(const pslr_ctx *c, int32_t *part, int32_t *is_interface, int32_t *perm);

/*
 * The classical Neumann polynomial of Sec. 1, which the paper contrasts its
 * method with, in place of the PSLR Schur complement approximation: from now
 * on pslr_apply, pslr_apply_T, pslr_apply_noalloc and pslr_solve use
 *     S^{-1} ~ omega [I + N + ... + N^m] D^{-1},   N = I - omega D^{-1} S,
 * with D = C0, the block diagonal of the splitting S = C0 - E_s (Eq. 3.1),
 * applied through the local factors (D^{-1} is the C0 solve), inside the same
 * block elimination as Algorithm 3 and with no low-rank term.  The scalar is
 * the one of the identity S^{-1} = omega (I - N)^{-1} D^{-1} (the series
 * converges to S^{-1} only when the spectral radius of N is below 1); omega = 1
 * gives exactly Algorithm 3 with rank 0 (N = C0^{-1} E_s, Eq. 3.3).  m >= 0,
 * omega > 0 and finite, else PSLR_ERR_ARG.  Frees the low-rank term;
 * pslr_build_lowrank or pslr_set_lowrank return the context to PSLR.  The
 * batched calls reject a context in this state (PSLR_ERR_STATE).  Synchronises
 * `stream` first.
 */
pslr_status pslr_set_neumann(pslr_ctx *c, int32_t m, double omega, void *stream);

/* Copy V (q x rank), H and G (rank x rank), column-major FP64, to host
 * arrays sized for the current rank (pslr_get_info().rank); any may be NULL. */
pslr_status pslr_get_lowrank(const pslr_ctx *c, double *V, double *H, double *G);

pslr_status pslr_get_info(const pslr_ctx *c, pslr_info *info);

/*
 * pslr_apply (or, with transpose != 0, pslr_apply_T) for callers that cannot
 * allocate device memory when they apply the preconditioner - for instance
 * code whose device memory all belongs to its own pool allocator, which
 * forbids cudaMalloc, cudaFree and allocating library calls outside it.  The
 * paper has no counterpart: this is an interface convenience.
 *
 * The call allocates nothing.  Its scratch (series iterates, accumulator,
 * partial sums, grid-barrier words) is a 16 MiB array inside the library,
 * which every GPU that loads the library holds until the process exits; it
 * fits interface sizes up to q ~ 690,000 in FP64 (3*(q+1) + s*rank values
 * plus 256 bytes).  Device errors latch in the context's own error word, as
 * for pslr_apply: pslr_sync reports them (a grid-barrier wait that gave up
 * returns PSLR_ERR_TIMEOUT there), and until then later applies of the
 * context do nothing.  Larger contexts are rejected with
 * PSLR_ERR_TOO_LARGE and a message.  The context, built by pslr_setup and
 * pslr_build_lowrank / pslr_set_lowrank beforehand, keeps everything else.
 * b_dev, z_dev: device vectors of n elements (double for PSLR_FP64, float for
 * PSLR_FP32), original ordering, one right-hand side.
 *
 * All calls share the one array and it keeps the previous call's contents;
 * the call clears the words that must start at zero.  Calls that overlap on
 * the GPU (different streams, or different contexts on concurrent streams)
 * race on the array: issue them in one stream or order them.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  The
 * library keeps that address for the rest of the process, so do not call
 * this entry point again after a cudaDeviceReset of that device.
 */
pslr_status pslr_apply_noalloc(pslr_ctx *c, const void *b_dev, void *z_dev, pslr_prec prec,
                               int32_t transpose, void *stream);

/* Synchronise `stream` and report any latched asynchronous error. */
pslr_status pslr_sync(pslr_ctx *c, void *stream);

/* Device-side grid-barrier wait limit in polls (default 2^22, about 0.5 s);
 * 0 makes every wait give up at once, which tests use to exercise the
 * PSLR_ERR_TIMEOUT path.  Returns the previous value. */
int64_t pslr_set_wait_limit(pslr_ctx *c, int64_t polls);

const char *pslr_last_error(const pslr_ctx *c);
const char *pslr_status_string(pslr_status s);
void pslr_destroy(pslr_ctx *c);

/* ------------------------------------------------------------------ batch
 *
 * Many independent systems A_k z_k = b_k, each with nrhs right-hand sides,
 * preconditioned and solved together: one launch applies Algorithm 3 to
 * every system and right-hand side, and one FGMRES (Section 4) per (system,
 * right-hand side) pair - a "problem" - advances in lockstep with the others,
 * each with its own basis, Hessenberg matrix and stopping test.  The paper
 * treats one system at a time; each problem of a batch follows the same
 * algorithm as the per-system calls (pslr_apply, pslr_solve), and the results
 * agree with theirs up to the order of rounding in the reductions.
 *
 * Batched vector layout: the systems one after the other in the order given
 * to pslr_batch_create, each as an n_k x nrhs column-major block in the
 * original ordering of A_k (problem (k, j) starts at offset
 * nrhs * (n_0 + ... + n_{k-1}) + j * n_k).  pslr_batch_info.n_total is the
 * length.
 */
typedef struct pslr_batch pslr_batch;

typedef struct {
    int32_t nsys, nrhs, nprob;      /* systems, right-hand sides each, problems      */
    int64_t n_total;                /* length of a batched vector                    */
    int32_t items;                  /* (system, subdomain) work items                */
    int32_t grid;                   /* CTAs of the batched apply launch              */
    int32_t ring[2];                /* ring slots of the apply, [FP64, FP32]         */
    int32_t group[2];               /* subdomains swept in lockstep per CTA, [FP64, FP32] */
    int32_t groups[2];              /* groups of the launch, [FP64, FP32]            */
    int32_t max_m, max_p, max_q;
    int64_t apply_bytes_fp64;       /* algorithmic bytes of one batched apply        */
    int64_t apply_bytes_fp32;
    int32_t graph;                  /* 1: the last solve replayed its cycles as CUDA graphs */
    int32_t handoff;                /* problems the last solve finished one by one (pslr_solve) */
    int32_t krylov_chunk;           /* rows per chunk of the batched Krylov kernels   */
    int32_t pair_rhs;               /* FP64 apply with nrhs > 1: 1 = a thread per (row, rhs)
                                       pair, 0 = a thread per row                      */
} pslr_batch_info;

/* Launch-shape options of a batch (pslr_batch_create_opts).  None changes a
 * result, only the speed; pslr_batch_create(group) is group = {group, group},
 * pair_rhs = 1 and zero elsewhere.  They have no counterpart in the paper: they are
 * the autotuner's knobs (paper_2002_00917_gb300.autotune.tune_batch). */
typedef struct {
    int32_t group[2];     /* subdomains of one system a CTA sweeps in lockstep, [FP64, FP32]:
                             1..8, 0 = the largest that fits shared memory (as
                             pslr_batch_create)                                              */
    int32_t ring_max[2];  /* cap on the apply's shared-memory ring slots, [FP64, FP32]:
                             0 = as many as fit, else >= 2                                  */
    int32_t krylov_chunk; /* rows per chunk of the batched FGMRES kernels (one CTA per
                             chunk): 0 = 1024, else 64..2^20                                */
    int32_t pair_rhs;     /* FP64 apply with nrhs > 1: 1 = one thread per (row, rhs) pair in
                             the level sweeps and products, 0 = one thread per row with its
                             right-hand sides (the same operations either way)              */
} pslr_batch_opts;

/*
 * Build a batch over nsys contexts that pslr_setup made and whose low-rank
 * term is built (pslr_build_lowrank / pslr_set_lowrank; rank 0 is allowed).
 * nrhs: 1..4 right-hand sides per system.  group: how many subdomains of one
 * system a CTA sweeps in lockstep (their levels merged, so one level step
 * serves all of them): 1..8, or 0 for the largest that fits shared memory;
 * a request that does not fit is reduced.  It changes speed, not results.  The batch reads the contexts'
 * device state and does not own them: keep every context alive, and leave its
 * low-rank term unchanged, while the batch exists (a batch call on a context
 * whose low-rank term was replaced returns PSLR_ERR_STATE).  Systems with
 * exact LU factors (factor 1) are rejected with PSLR_ERR_ARG.  *out is NULL
 * on failure, and pslr_batch_last_error(NULL) gives the message of the last
 * failed pslr_batch_create of the calling thread.
 */
pslr_status pslr_batch_create(int32_t nsys, pslr_ctx *const *systems, int32_t nrhs, int32_t group,
                              pslr_batch **out);

/* pslr_batch_create with every launch-shape option of pslr_batch_opts (no
 * counterpart in the paper).  opts must not be NULL; a bad option returns
 * PSLR_ERR_ARG.  Everything else as pslr_batch_create. */
pslr_status pslr_batch_create_opts(int32_t nsys, pslr_ctx *const *systems, int32_t nrhs,
                                   const pslr_batch_opts *opts, pslr_batch **out);

/* z = M_k^{-1} b for every system k and right-hand side (Algorithm 3), one
 * launch.  b_dev, z_dev: batched device vectors of n_total doubles
 * (PSLR_FP64) or floats (PSLR_FP32, V in BF16).  Enqueued on `stream`;
 * asynchronous errors are reported by pslr_batch_sync. */
pslr_status pslr_batch_apply(pslr_batch *bt, const void *b_dev, void *z_dev, pslr_prec prec, void *stream);

/*
 * FGMRES(restart) on every problem with x0 = 0, preconditioned by the
 * batched apply in precision prec (FP64 Krylov vectors, Gram-Schmidt and
 * least squares in either case).  A problem stops when ||b - A x|| <=
 * rtol ||b|| (true residual, checked at the end of each cycle, or earlier by
 * the estimate), after maxit iterations, or on a non-finite value.  b_dev,
 * x_dev: batched device vectors of doubles.  iters (int32, nprob) and relres
 * (double, nprob) are optional host arrays, problem order.  Each restart
 * cycle is captured once as a CUDA graph and replayed; if capture is not
 * available the same launches are issued directly (pslr_batch_info.graph
 * says which).  Synchronises `stream` once per cycle.  When at most 16 of
 * more than 16 problems are still running at the end of a cycle, each of them
 * is finished on its own system with pslr_solve on its current residual
 * (solving A e = b - A x to the tolerance rtol ||b|| and adding e): the same
 * restarted iteration, without a whole batched step per iteration.  The
 * systems involved run at once, each from its own host thread on its own
 * stream (created by the batch), their problems one after another; this
 * uses the system contexts' own Krylov workspace, so no other call may use
 * those contexts meanwhile.  pslr_batch_info.handoff counts these problems.
 * Returns PSLR_OK when every problem converged, PSLR_ERR_NAN if one went
 * non-finite, else PSLR_ERR_NOT_CONVERGED.  restart: 1..127.
 */
pslr_status pslr_batch_solve(pslr_batch *bt, const double *b_dev, double *x_dev, double rtol, int32_t restart,
                             int32_t maxit, pslr_prec prec, int32_t *iters, double *relres, void *stream);

pslr_status pslr_batch_get_info(const pslr_batch *bt, pslr_batch_info *info);

/* Synchronise `stream` and report a latched asynchronous error of the batch. */
pslr_status pslr_batch_sync(pslr_batch *bt, void *stream);

int64_t pslr_batch_set_wait_limit(pslr_batch *bt, int64_t polls);
const char *pslr_batch_last_error(const pslr_batch *bt);
void pslr_batch_destroy(pslr_batch *bt);


#ifdef __cplusplus
}
#endif
#endif /* PSLR_H */

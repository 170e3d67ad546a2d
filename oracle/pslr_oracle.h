/*
 * PSLR oracle: plain, slow, single-threaded FP64 C restatement of the power
 * Schur complement low-rank preconditioner (Zheng, Xi, Saad, arXiv 2002.00917).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA path and must never serve as a fallback for it.
 *
 * Every routine follows one passage of the paper (cited beside it) in the
 * paper's notation: the reordered system is [B E; F C] (Section 2, Eq. 2.1),
 * S = C - F B^{-1} E (Eq. 2.2), the splitting S = C0 - E_s (Eq. 3.1) with
 * E_s = -C_g + F B^{-1} E and C_g = C - C0 (Sec. 3.1, proof of the lemma on
 * the spectrum of C0^{-1}E_s), the series P_m = sum_{i=0}^{m} (C0^{-1}E_s)^i
 * C0^{-1} (Eq. 3.3), E_rr(m) = (E_s C0^{-1})^{m+1} (Sec. 3.2.1, Eq. 3.19),
 * the Arnoldi factors V, H (Eq. 3.16) and G = (I - H)^{-1} - I (Eq. 3.17),
 * applied as Algorithm 3 (Eq. 3.24).  Equation numbers count the paper's
 * numbered displays per section in order of appearance.
 *
 * Vectors passed to orc_apply / orc_apply_T / orc_fgmres are in the ORIGINAL
 * ordering; block-level operators (orc_solve_B, orc_Es, ...) work in the
 * permuted numbering: interior unknowns 0..p-1, interface unknowns 0..q-1.
 */
#ifndef PSLR_ORACLE_H
#define PSLR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_ctx orc_ctx;

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_ZERO_PIVOT = 3, ORC_ERR_BREAKDOWN = 4,
       ORC_ERR_SINGULAR_IMH = 5, ORC_ERR_NOT_CONVERGED = 6 };

/* Blocks and factors that orc_get_block can export (permuted numbering). */
enum { ORC_B = 0, ORC_E = 1, ORC_F = 2, ORC_C = 3, ORC_C0 = 4, ORC_CG = 5,
       ORC_LU_B = 6, ORC_LU_C0 = 7 };

/* Reorder A (Section 2), extract [B E; F C], C0, C_g (Eq. 3.1, Lemma 2) and
 * factor every B_i and C_i (Algorithm 1, steps 2-5).  part may be NULL, then the
 * geometric split of dims by splits is used.  factor: 0 = ILU(0), 1 = exact
 * dense LU with partial pivoting, 2 = ILUT(drop_tol) without a fill limit.
 * On failure returns NULL and sets *status. */
orc_ctx *orc_setup(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                   const int32_t dims[3], const int32_t splits[3], const int32_t *part,
                   int32_t factor, double drop_tol, int32_t *status);
void orc_destroy(orc_ctx *c);

/* Recursive breadth-first bisection of the graph of A + A^T into nparts parts
 * (1 <= nparts <= n), written to part (length n); ORC_ERR_ARG otherwise. */
int32_t orc_graph_partition(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t nparts,
                            int32_t *part);

void orc_sizes(const orc_ctx *c, int32_t *n, int32_t *s, int32_t *p, int32_t *q);
void orc_maps(const orc_ctx *c, int32_t *part, int32_t *is_interface, int32_t *perm);
void orc_offsets(const orc_ctx *c, int32_t *interior_off, int32_t *interface_off);
int32_t orc_block_nnz(const orc_ctx *c, int32_t which);
void orc_get_block(const orc_ctx *c, int32_t which, int32_t *rowptr, int32_t *col, double *val);

/* Building blocks (permuted numbering). */
void orc_solve_B(const orc_ctx *c, const double *in, double *out);    /* B~^{-1}  */
void orc_solve_BT(const orc_ctx *c, const double *in, double *out);   /* B~^{-T}  */
void orc_solve_C0(const orc_ctx *c, const double *in, double *out);   /* C0~^{-1} */
void orc_solve_C0T(const orc_ctx *c, const double *in, double *out);  /* C0~^{-T} */
void orc_Es(const orc_ctx *c, const double *in, double *out);         /* E_s w    */
void orc_EsT(const orc_ctx *c, const double *in, double *out);        /* E_s^T w  */
void orc_series(const orc_ctx *c, int32_t m, const double *in, double *out);   /* P_m t   */
void orc_seriesT(const orc_ctx *c, int32_t m, const double *in, double *out);  /* P_m^T t */
void orc_Err(const orc_ctx *c, int32_t m, const double *in, double *out);      /* E_rr(m) v */

/* Algorithm 1, steps 6-8: r-step Arnoldi on E_rr(m) from a SplitMix64 start
 * vector, then G = (I-H)^{-1} - I.  full_rank != 0 restarts on breakdown with a
 * fresh vector (used to span the whole interface space); otherwise the rank
 * is truncated.  *rank_out receives the rank kept. */
int32_t orc_build_lowrank(orc_ctx *c, int32_t m, int32_t rank, uint64_t seed, int32_t full_rank,
                          int32_t *rank_out);
void orc_get_lowrank(const orc_ctx *c, double *V, double *H, double *G);
/* Replace V (q x r, column-major) and G (r x r, column-major) directly. */
int32_t orc_set_lowrank(orc_ctx *c, int32_t m, int32_t rank, const double *V, const double *G);

/* Algorithm 3 (original ordering) and its exact transpose. */
void orc_apply(const orc_ctx *c, const double *b, double *z);
void orc_apply_T(const orc_ctx *c, const double *b, double *z);

/* Sec. 1: the classical Neumann polynomial of the Schur complement, the foil
 * the paper contrasts PSLR with: S^{-1} ~ omega [I + N + ... + N^m] D^{-1},
 * N = I - omega D^{-1} S, D = C0 (the factored block diagonal of Eq. 3.1),
 * S = C0~ - E_s; interface numbering in and out (transpose: its transpose).
 * orc_neumann_apply is Algorithm 3's block elimination with it in place of
 * P_m (I + V G V^T), original ordering.  orc_set_neumann(c, m, omega > 0)
 * makes orc_fgmres use it as the preconditioner (omega <= 0: PSLR again). */
void orc_neumann_series(const orc_ctx *c, int32_t m, double omega, int32_t transpose, const double *in,
                        double *out);
void orc_neumann_apply(const orc_ctx *c, int32_t m, double omega, int32_t transpose, const double *b,
                       double *z);
void orc_set_neumann(orc_ctx *c, int32_t m, double omega);

/* Right-preconditioned flexible GMRES(restart), x0 = 0, classical Gram-Schmidt
 * applied twice, Givens rotations.  prec bit 0: PSLR preconditioner
 * (Algorithm 3) instead of none; bit 1: solve with A^T and the transposed
 * preconditioner (adjoint solve).  Returns ORC_OK or ORC_ERR_NOT_CONVERGED;
 * *iters is cumulative over restarts. */
int32_t orc_fgmres(const orc_ctx *c, int32_t prec, const double *b, double *x, double rtol,
                   int32_t restart, int32_t maxit, int32_t *iters, double *relres);

/* SplitMix64 (Steele, Lea, Flood 2014): output j of the generator seeded with
 * `seed`, mapped to [-1, 1). */
double orc_splitmix_uniform(uint64_t seed, uint64_t j);

#ifdef __cplusplus
}
#endif
#endif

/*
 * PSLR oracle (FP64, single-threaded, plain C).  TEST INFRASTRUCTURE ONLY: the
 * product path never loads this file.  See pslr_oracle.h for the notation and
 * the list of what each routine restates.
 *
 * Parity status of each part (what pins it is in tests/test_oracle_*.py):
 *   partition / reordering / blocks ..... pinned (brute force, reassembly)
 *   ILU(0), exact LU ..................... pinned (pattern identity, P L U = B)
 *   ILUT(tau) ............................ pinned (tau = 0 is LU, tridiagonal = ILU(0),
 *                                          thresholds, dense brute force)
 *   graph partition ...................... pinned (paths cut into runs, grid
 *                                          anti-diagonals, components, sizes)
 *   series, E_rr(m), Arnoldi, G ......... pinned (closed forms, Theorem 2)
 *   Algorithm 3 apply and transpose ...... pinned (dense formulas, identity case)
 *   FGMRES ............................... pinned (dense solve, M = I reduction)
 *   Neumann polynomial (Sec. 1 foil) ..... pinned (omega = 1 is the series of Eq. 3.3,
 *                                          dense closed form, limit S^{-1} when
 *                                          rho(N) < 1, transpose by inner products)
 */
#include "pslr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t nr, nc;
    int32_t *rp, *ci;
    double *v;
} ocsr;

struct orc_ctx {
    int32_t n, s, p, q, factor;
    int32_t *part, *iface, *perm, *iperm; /* perm[new] = old, iperm[old] = new */
    int32_t *ioff, *goff;                 /* per subdomain: interior / interface offsets (s+1) */
    ocsr A, B, E, F, C, C0, Cg;           /* blocks in the permuted numbering */
    ocsr luB, luC;                        /* ILU(0): strictly lower = L (unit), upper = U */
    double **dB, **dC;                    /* exact LU: per subdomain dense factors (row-major) */
    int32_t **pvB, **pvC;                 /* exact LU: row swap at each elimination step */
    int32_t m, r;
    double *V, *H, *G;                    /* q x r, r x r, r x r (column-major) */
    int32_t nf_on, nf_m;                  /* FGMRES with the Sec. 1 Neumann foil instead of PSLR */
    double nf_omega;
};

/* ------------------------------------------------------------------ helpers */

static void csr_free(ocsr *a) {
    free(a->rp);
    free(a->ci);
    free(a->v);
    memset(a, 0, sizeof(*a));
}

static ocsr csr_copy(const ocsr *a) {
    ocsr b = *a;
    int32_t nnz = a->rp[a->nr];
    b.rp = malloc(sizeof(int32_t) * (a->nr + 1));
    b.ci = malloc(sizeof(int32_t) * (nnz ? nnz : 1));
    b.v = malloc(sizeof(double) * (nnz ? nnz : 1));
    memcpy(b.rp, a->rp, sizeof(int32_t) * (a->nr + 1));
    memcpy(b.ci, a->ci, sizeof(int32_t) * nnz);
    memcpy(b.v, a->v, sizeof(double) * nnz);
    return b;
}

/* y = M x */
static void spmv(const ocsr *M, const double *x, double *y) {
    for (int32_t i = 0; i < M->nr; ++i) {
        double acc = 0.0;
        for (int32_t k = M->rp[i]; k < M->rp[i + 1]; ++k) acc += M->v[k] * x[M->ci[k]];
        y[i] = acc;
    }
}

/* y = M^T x  (column sweep over the rows of M) */
static void spmv_t(const ocsr *M, const double *x, double *y) {
    for (int32_t j = 0; j < M->nc; ++j) y[j] = 0.0;
    for (int32_t i = 0; i < M->nr; ++i)
        for (int32_t k = M->rp[i]; k < M->rp[i + 1]; ++k) y[M->ci[k]] += M->v[k] * x[i];
}

static double dot(int32_t n, const double *a, const double *b) {
    double s = 0.0;
    for (int32_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static double nrm2(int32_t n, const double *a) { return sqrt(dot(n, a, a)); }

/* Triplets -> CSR with columns ascending in every row. */
typedef struct {
    int32_t r, c;
    double v;
} trip;

static int trip_cmp(const void *a, const void *b) {
    const trip *x = a, *y = b;
    if (x->r != y->r) return x->r < y->r ? -1 : 1;
    if (x->c != y->c) return x->c < y->c ? -1 : 1;
    return 0;
}

static ocsr csr_from_trips(int32_t nr, int32_t nc, trip *t, int32_t nt) {
    ocsr a;
    a.nr = nr;
    a.nc = nc;
    qsort(t, nt, sizeof(trip), trip_cmp);
    a.rp = calloc(nr + 1, sizeof(int32_t));
    a.ci = malloc(sizeof(int32_t) * (nt ? nt : 1));
    a.v = malloc(sizeof(double) * (nt ? nt : 1));
    for (int32_t k = 0; k < nt; ++k) {
        a.rp[t[k].r + 1]++;
        a.ci[k] = t[k].c;
        a.v[k] = t[k].v;
    }
    for (int32_t i = 0; i < nr; ++i) a.rp[i + 1] += a.rp[i];
    return a;
}

/* ------------------------------------------------ Section 2: reordering */

typedef struct {
    int32_t iface, part, idx;
} okey;

static int key_cmp(const void *a, const void *b) {
    const okey *x = a, *y = b;
    if (x->iface != y->iface) return x->iface - y->iface;
    if (x->part != y->part) return x->part - y->part;
    return x->idx - y->idx;
}

/*
 * Section 2: an edge-separator ("vertex-based") partition into s subdomains,
 * interior unknowns labelled subdomain by subdomain, interface unknowns last.
 * The geometric split stands in for the paper's METIS call: node (i,j,k) of an
 * Nx x Ny x Nz grid (x fastest) goes to part floor(i Px/Nx) + Px (floor(j Py/Ny)
 * + Py floor(k Pz/Nz)).  A node is an interface node iff it is coupled (in the
 * pattern of A + A^T) to a node of another part.
 */
static void reorder(orc_ctx *c, const int32_t dims[3], const int32_t splits[3],
                    const int32_t *upart) {
    int32_t n = c->n;
    c->part = malloc(sizeof(int32_t) * n);
    c->iface = calloc(n, sizeof(int32_t));
    c->perm = malloc(sizeof(int32_t) * n);
    c->iperm = malloc(sizeof(int32_t) * n);
    if (upart) {
        int32_t mx = 0;
        for (int32_t v = 0; v < n; ++v) {
            c->part[v] = upart[v];
            if (upart[v] > mx) mx = upart[v];
        }
        c->s = mx + 1;
    } else {
        int32_t Nx = dims[0], Ny = dims[1], Nz = dims[2];
        int32_t Px = splits[0], Py = splits[1], Pz = splits[2];
        for (int32_t v = 0; v < n; ++v) {
            int32_t i = v % Nx, j = (v / Nx) % Ny, k = v / (Nx * Ny);
            c->part[v] = (i * Px) / Nx + Px * ((j * Py) / Ny + Py * ((k * Pz) / Nz));
        }
        c->s = Px * Py * Pz;
    }
    for (int32_t v = 0; v < n; ++v)
        for (int32_t k = c->A.rp[v]; k < c->A.rp[v + 1]; ++k) {
            int32_t w = c->A.ci[k];
            if (w != v && c->part[w] != c->part[v]) {
                c->iface[v] = 1;
                c->iface[w] = 1;
            }
        }
    okey *keys = malloc(sizeof(okey) * n);
    for (int32_t v = 0; v < n; ++v) {
        keys[v].iface = c->iface[v];
        keys[v].part = c->part[v];
        keys[v].idx = v;
    }
    qsort(keys, n, sizeof(okey), key_cmp);
    c->p = 0;
    for (int32_t t = 0; t < n; ++t) {
        c->perm[t] = keys[t].idx;
        c->iperm[keys[t].idx] = t;
        if (!keys[t].iface) c->p++;
    }
    c->q = n - c->p;
    free(keys);
    c->ioff = calloc(c->s + 1, sizeof(int32_t));
    c->goff = calloc(c->s + 1, sizeof(int32_t));
    for (int32_t v = 0; v < n; ++v) {
        if (c->iface[v]) c->goff[c->part[v] + 1]++;
        else c->ioff[c->part[v] + 1]++;
    }
    for (int32_t i = 0; i < c->s; ++i) {
        c->ioff[i + 1] += c->ioff[i];
        c->goff[i + 1] += c->goff[i];
    }
}

/* Eq. 2.1 and Eq. 3.1: split P A P^T into B (p x p), E (p x q), F (q x p),
 * C (q x q); C0 keeps the entries of C inside one subdomain, C_g = C - C0. */
static void extract_blocks(orc_ctx *c) {
    int32_t n = c->n, p = c->p, q = c->q;
    int32_t nnz = c->A.rp[n];
    trip *tb = malloc(sizeof(trip) * (nnz + 1)), *te = malloc(sizeof(trip) * (nnz + 1));
    trip *tf = malloc(sizeof(trip) * (nnz + 1)), *tc = malloc(sizeof(trip) * (nnz + 1));
    trip *t0 = malloc(sizeof(trip) * (nnz + 1)), *tg = malloc(sizeof(trip) * (nnz + 1));
    int32_t nb = 0, ne = 0, nf = 0, nc = 0, n0 = 0, ng = 0;
    for (int32_t v = 0; v < n; ++v) {
        int32_t r = c->iperm[v];
        for (int32_t k = c->A.rp[v]; k < c->A.rp[v + 1]; ++k) {
            int32_t w = c->A.ci[k], cc = c->iperm[w];
            double a = c->A.v[k];
            if (r < p && cc < p) tb[nb++] = (trip){r, cc, a};
            else if (r < p) te[ne++] = (trip){r, cc - p, a};
            else if (cc < p) tf[nf++] = (trip){r - p, cc, a};
            else {
                tc[nc++] = (trip){r - p, cc - p, a};
                if (c->part[v] == c->part[w]) t0[n0++] = (trip){r - p, cc - p, a};
                else tg[ng++] = (trip){r - p, cc - p, a};
            }
        }
    }
    c->B = csr_from_trips(p, p, tb, nb);
    c->E = csr_from_trips(p, q, te, ne);
    c->F = csr_from_trips(q, p, tf, nf);
    c->C = csr_from_trips(q, q, tc, nc);
    c->C0 = csr_from_trips(q, q, t0, n0);
    c->Cg = csr_from_trips(q, q, tg, ng);
    free(tb); free(te); free(tf); free(tc); free(t0); free(tg);
}

/* ------------------------------------- Algorithm 1, steps 2-5: local factors */

/*
 * ILU(0) in the IKJ order (Saad, Iterative Methods, Sec. 10.3.2), natural order,
 * no pivoting.  The block-diagonal matrix is factored as a whole, which is the
 * same computation as factoring each diagonal block separately because no
 * entry couples two blocks.  Result: strictly lower part = L (unit diagonal
 * implied), upper part including the diagonal = U, on the pattern of M.
 */
static int32_t ilu0(ocsr *M) {
    int32_t n = M->nr;
    int32_t *pos = malloc(sizeof(int32_t) * (n ? n : 1));
    int32_t *dg = malloc(sizeof(int32_t) * (n ? n : 1));
    for (int32_t j = 0; j < n; ++j) pos[j] = -1;
    for (int32_t i = 0; i < n; ++i) {
        dg[i] = -1;
        for (int32_t k = M->rp[i]; k < M->rp[i + 1]; ++k)
            if (M->ci[k] == i) dg[i] = k;
        if (dg[i] < 0) {
            free(pos); free(dg);
            return ORC_ERR_ZERO_PIVOT;
        }
    }
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t k = M->rp[i]; k < M->rp[i + 1]; ++k) pos[M->ci[k]] = k;
        for (int32_t k = M->rp[i]; k < M->rp[i + 1]; ++k) {
            int32_t kk = M->ci[k];
            if (kk >= i) break;
            double piv = M->v[dg[kk]];
            if (piv == 0.0) {
                free(pos); free(dg);
                return ORC_ERR_ZERO_PIVOT;
            }
            M->v[k] /= piv; /* l_{i,kk} */
            for (int32_t t = dg[kk] + 1; t < M->rp[kk + 1]; ++t) {
                int32_t j = M->ci[t];
                if (pos[j] >= 0) M->v[pos[j]] -= M->v[k] * M->v[t];
            }
        }
        if (M->v[dg[i]] == 0.0) {
            free(pos); free(dg);
            return ORC_ERR_ZERO_PIVOT;
        }
        for (int32_t k = M->rp[i]; k < M->rp[i + 1]; ++k) pos[M->ci[k]] = -1;
    }
    free(pos);
    free(dg);
    return ORC_OK;
}

/*
 * ILUT(tau) without a fill limit (Saad, Iterative Methods, Sec. 10.4; the
 * paper's Section 4 factors with threshold 1e-2), row by row in natural
 * order.  The threshold is relative to the mean modulus of the row, as in
 * Saad's SPARSKIT ilut: for row i, tol = tau * (sum of |a_ij| over the stored
 * entries, in column order) / (number of stored entries).  The dense work
 * row w = a_i; for every k < i, smallest first, with
 * w_k nonzero: w_k /= u_kk, and either w_k is dropped (|w_k| < tol) or the
 * strictly upper part of row k of U, scaled by w_k, is subtracted from w;
 * afterwards every entry except the diagonal with |w_j| < tol is dropped.
 * The result replaces *M (strictly lower = L with unit diagonal, upper
 * including the diagonal = U), columns ascending.  As with ilu0, the
 * block-diagonal matrix may be factored as a whole: no row reaches into
 * another block.
 */
static int32_t ilut(ocsr *M, double tau) {
    int32_t n = M->nr;
    size_t cap = (size_t)M->rp[n] + 16, nnz = 0;
    int32_t *rp = malloc(sizeof(int32_t) * (n + 1));
    int32_t *ci = malloc(sizeof(int32_t) * cap);
    double *v = malloc(sizeof(double) * cap);
    int32_t *dpos = malloc(sizeof(int32_t) * (n ? n : 1));
    double *w = calloc(n ? n : 1, sizeof(double));
    char *state = calloc(n ? n : 1, 1); /* 0 empty, 1 live entry, 2 dropped multiplier */
    int32_t st = ORC_OK;
    rp[0] = 0;
    for (int32_t i = 0; i < n && st == ORC_OK; ++i) {
        double s1 = 0.0;
        int32_t first = i, last = i, len = M->rp[i + 1] - M->rp[i];
        for (int32_t t = M->rp[i]; t < M->rp[i + 1]; ++t) {
            s1 += fabs(M->v[t]);
            w[M->ci[t]] = M->v[t];
            state[M->ci[t]] = 1;
            if (M->ci[t] < first) first = M->ci[t];
            if (M->ci[t] > last) last = M->ci[t];
        }
        double tol = len > 0 ? tau * (s1 / len) : 0.0;
        for (int32_t k = first; k < i; ++k) {
            if (state[k] != 1) continue;
            double mult = w[k] / v[dpos[k]];
            if (fabs(mult) < tol) {
                w[k] = 0.0;
                state[k] = 2;
                continue;
            }
            w[k] = mult;
            for (int32_t t = dpos[k] + 1; t < rp[k + 1]; ++t) {
                int32_t j = ci[t];
                if (state[j] == 0) {
                    state[j] = 1;
                    w[j] = 0.0;
                    if (j > last) last = j;
                }
                w[j] -= mult * v[t];
            }
        }
        dpos[i] = -1;
        for (int32_t j = first; j <= last; ++j) { /* columns in ascending order */
            if (state[j] == 1 && (j == i || fabs(w[j]) >= tol)) {
                if (nnz == cap) {
                    cap *= 2;
                    ci = realloc(ci, sizeof(int32_t) * cap);
                    v = realloc(v, sizeof(double) * cap);
                }
                if (j == i) dpos[i] = (int32_t)nnz;
                ci[nnz] = j;
                v[nnz] = w[j];
                ++nnz;
            }
            w[j] = 0.0;
            state[j] = 0;
        }
        rp[i + 1] = (int32_t)nnz;
        if (dpos[i] < 0 || v[dpos[i]] == 0.0 || !isfinite(v[dpos[i]])) st = ORC_ERR_ZERO_PIVOT;
    }
    free(w);
    free(state);
    free(dpos);
    if (st != ORC_OK) {
        free(rp); free(ci); free(v);
        return st;
    }
    free(M->rp); free(M->ci); free(M->v);
    M->rp = rp;
    M->ci = ci;
    M->v = v;
    return ORC_OK;
}

/* Dense LU with partial pivoting (largest |a|, ties -> smallest row) of the
 * diagonal block rows/cols [lo, hi) of M.  a is row-major nb x nb. */
static int32_t dense_lu_block(const ocsr *M, int32_t lo, int32_t hi, double **out, int32_t **piv) {
    int32_t nb = hi - lo;
    double *a = calloc((size_t)nb * nb + 1, sizeof(double));
    int32_t *pv = malloc(sizeof(int32_t) * (nb ? nb : 1));
    for (int32_t i = lo; i < hi; ++i)
        for (int32_t k = M->rp[i]; k < M->rp[i + 1]; ++k)
            a[(size_t)(i - lo) * nb + (M->ci[k] - lo)] = M->v[k];
    for (int32_t k = 0; k < nb; ++k) {
        int32_t pr = k;
        double best = fabs(a[(size_t)k * nb + k]);
        for (int32_t i = k + 1; i < nb; ++i)
            if (fabs(a[(size_t)i * nb + k]) > best) {
                best = fabs(a[(size_t)i * nb + k]);
                pr = i;
            }
        pv[k] = pr;
        if (best == 0.0) {
            free(a); free(pv);
            return ORC_ERR_ZERO_PIVOT;
        }
        if (pr != k)
            for (int32_t j = 0; j < nb; ++j) {
                double t = a[(size_t)k * nb + j];
                a[(size_t)k * nb + j] = a[(size_t)pr * nb + j];
                a[(size_t)pr * nb + j] = t;
            }
        for (int32_t i = k + 1; i < nb; ++i) {
            double l = a[(size_t)i * nb + k] / a[(size_t)k * nb + k];
            a[(size_t)i * nb + k] = l;
            for (int32_t j = k + 1; j < nb; ++j) a[(size_t)i * nb + j] -= l * a[(size_t)k * nb + j];
        }
    }
    *out = a;
    *piv = pv;
    return ORC_OK;
}

/* x = (L U)^{-1} b for the combined ILU(0) factor: forward, then backward. */
static void ilu_solve(const ocsr *LU, const double *b, double *x) {
    int32_t n = LU->nr;
    for (int32_t i = 0; i < n; ++i) {
        double acc = b[i];
        for (int32_t k = LU->rp[i]; k < LU->rp[i + 1] && LU->ci[k] < i; ++k)
            acc -= LU->v[k] * x[LU->ci[k]];
        x[i] = acc;
    }
    for (int32_t i = n - 1; i >= 0; --i) {
        double acc = x[i], d = 0.0;
        for (int32_t k = LU->rp[i]; k < LU->rp[i + 1]; ++k) {
            int32_t j = LU->ci[k];
            if (j > i) acc -= LU->v[k] * x[j];
            else if (j == i) d = LU->v[k];
        }
        x[i] = acc / d;
    }
}

/* x = (L U)^{-T} b = L^{-T} U^{-T} b: U^T is lower triangular, L^T unit upper;
 * both are swept column by column over the rows of the stored factor. */
static void ilu_solve_t(const ocsr *LU, const double *b, double *x) {
    int32_t n = LU->nr;
    for (int32_t i = 0; i < n; ++i) x[i] = b[i];
    for (int32_t i = 0; i < n; ++i) { /* U^T z = b */
        double d = 0.0;
        for (int32_t k = LU->rp[i]; k < LU->rp[i + 1]; ++k)
            if (LU->ci[k] == i) d = LU->v[k];
        x[i] /= d;
        for (int32_t k = LU->rp[i]; k < LU->rp[i + 1]; ++k)
            if (LU->ci[k] > i) x[LU->ci[k]] -= LU->v[k] * x[i];
    }
    for (int32_t i = n - 1; i >= 0; --i) /* L^T y = z */
        for (int32_t k = LU->rp[i]; k < LU->rp[i + 1] && LU->ci[k] < i; ++k)
            x[LU->ci[k]] -= LU->v[k] * x[i];
}

/* Solve with one dense pivoted LU block: P B = L U. */
static void dense_solve(int32_t nb, const double *a, const int32_t *pv, const double *b, double *x) {
    for (int32_t i = 0; i < nb; ++i) x[i] = b[i];
    for (int32_t k = 0; k < nb; ++k)
        if (pv[k] != k) {
            double t = x[k];
            x[k] = x[pv[k]];
            x[pv[k]] = t;
        }
    for (int32_t i = 0; i < nb; ++i)
        for (int32_t j = 0; j < i; ++j) x[i] -= a[(size_t)i * nb + j] * x[j];
    for (int32_t i = nb - 1; i >= 0; --i) {
        for (int32_t j = i + 1; j < nb; ++j) x[i] -= a[(size_t)i * nb + j] * x[j];
        x[i] /= a[(size_t)i * nb + i];
    }
}

/* B^T = U^T L^T P  =>  x = P^T L^{-T} U^{-T} b. */
static void dense_solve_t(int32_t nb, const double *a, const int32_t *pv, const double *b, double *x) {
    for (int32_t i = 0; i < nb; ++i) x[i] = b[i];
    for (int32_t i = 0; i < nb; ++i) { /* U^T */
        for (int32_t j = 0; j < i; ++j) x[i] -= a[(size_t)j * nb + i] * x[j];
        x[i] /= a[(size_t)i * nb + i];
    }
    for (int32_t i = nb - 1; i >= 0; --i) /* L^T, unit diagonal */
        for (int32_t j = i + 1; j < nb; ++j) x[i] -= a[(size_t)j * nb + i] * x[j];
    for (int32_t k = nb - 1; k >= 0; --k)
        if (pv[k] != k) {
            double t = x[k];
            x[k] = x[pv[k]];
            x[pv[k]] = t;
        }
}

/* ------------------------------------------------------------- set-up */

orc_ctx *orc_setup(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                   const int32_t dims[3], const int32_t splits[3], const int32_t *part,
                   int32_t factor, double drop_tol, int32_t *status) {
    *status = ORC_ERR_ARG;
    if (n <= 0 || !rowptr || !col || !val) return NULL;
    if (factor < 0 || factor > 2 || (factor == 2 && !(drop_tol >= 0.0 && isfinite(drop_tol)))) return NULL;
    if (!part && (!dims || !splits || (int64_t)dims[0] * dims[1] * dims[2] != n)) return NULL;
    if (!part)
        for (int d = 0; d < 3; ++d)
            if (splits[d] < 1 || splits[d] > dims[d]) return NULL;
    orc_ctx *c = calloc(1, sizeof(orc_ctx));
    c->n = n;
    c->factor = factor;
    ocsr A = {n, n, (int32_t *)rowptr, (int32_t *)col, (double *)val};
    c->A = csr_copy(&A);
    reorder(c, dims, splits, part);
    extract_blocks(c);
    int32_t st = ORC_OK;
    if (factor == 0 || factor == 2) {
        c->luB = csr_copy(&c->B);
        c->luC = csr_copy(&c->C0);
        st = factor == 0 ? ilu0(&c->luB) : ilut(&c->luB, drop_tol);
        if (st == ORC_OK) st = factor == 0 ? ilu0(&c->luC) : ilut(&c->luC, drop_tol);
    } else {
        c->dB = calloc(c->s, sizeof(double *));
        c->dC = calloc(c->s, sizeof(double *));
        c->pvB = calloc(c->s, sizeof(int32_t *));
        c->pvC = calloc(c->s, sizeof(int32_t *));
        for (int32_t i = 0; i < c->s && st == ORC_OK; ++i) {
            st = dense_lu_block(&c->B, c->ioff[i], c->ioff[i + 1], &c->dB[i], &c->pvB[i]);
            if (st == ORC_OK)
                st = dense_lu_block(&c->C0, c->goff[i], c->goff[i + 1], &c->dC[i], &c->pvC[i]);
        }
    }
    if (st != ORC_OK) {
        *status = st;
        orc_destroy(c);
        return NULL;
    }
    *status = ORC_OK;
    return c;
}

void orc_destroy(orc_ctx *c) {
    if (!c) return;
    free(c->part); free(c->iface); free(c->perm); free(c->iperm);
    free(c->ioff); free(c->goff);
    csr_free(&c->A); csr_free(&c->B); csr_free(&c->E); csr_free(&c->F);
    csr_free(&c->C); csr_free(&c->C0); csr_free(&c->Cg);
    csr_free(&c->luB); csr_free(&c->luC);
    if (c->dB)
        for (int32_t i = 0; i < c->s; ++i) {
            free(c->dB[i]); free(c->dC[i]); free(c->pvB[i]); free(c->pvC[i]);
        }
    free(c->dB); free(c->dC); free(c->pvB); free(c->pvC);
    free(c->V); free(c->H); free(c->G);
    free(c);
}

void orc_sizes(const orc_ctx *c, int32_t *n, int32_t *s, int32_t *p, int32_t *q) {
    *n = c->n; *s = c->s; *p = c->p; *q = c->q;
}

void orc_maps(const orc_ctx *c, int32_t *part, int32_t *is_interface, int32_t *perm) {
    memcpy(part, c->part, sizeof(int32_t) * c->n);
    memcpy(is_interface, c->iface, sizeof(int32_t) * c->n);
    memcpy(perm, c->perm, sizeof(int32_t) * c->n);
}

void orc_offsets(const orc_ctx *c, int32_t *interior_off, int32_t *interface_off) {
    memcpy(interior_off, c->ioff, sizeof(int32_t) * (c->s + 1));
    memcpy(interface_off, c->goff, sizeof(int32_t) * (c->s + 1));
}

static const ocsr *pick(const orc_ctx *c, int32_t which) {
    switch (which) {
    case ORC_B: return &c->B;
    case ORC_E: return &c->E;
    case ORC_F: return &c->F;
    case ORC_C: return &c->C;
    case ORC_C0: return &c->C0;
    case ORC_CG: return &c->Cg;
    case ORC_LU_B: return c->factor != 1 ? &c->luB : NULL;
    case ORC_LU_C0: return c->factor != 1 ? &c->luC : NULL;
    }
    return NULL;
}

int32_t orc_block_nnz(const orc_ctx *c, int32_t which) {
    const ocsr *m = pick(c, which);
    return m ? m->rp[m->nr] : -1;
}

void orc_get_block(const orc_ctx *c, int32_t which, int32_t *rowptr, int32_t *col, double *val) {
    const ocsr *m = pick(c, which);
    if (!m) return;
    memcpy(rowptr, m->rp, sizeof(int32_t) * (m->nr + 1));
    memcpy(col, m->ci, sizeof(int32_t) * m->rp[m->nr]);
    memcpy(val, m->v, sizeof(double) * m->rp[m->nr]);
}

/* ------------------------------------------ B~^{-1}, C0~^{-1} and transposes */

void orc_solve_B(const orc_ctx *c, const double *in, double *out) {
    if (c->factor != 1) {
        ilu_solve(&c->luB, in, out);
        return;
    }
    for (int32_t i = 0; i < c->s; ++i) {
        int32_t lo = c->ioff[i], nb = c->ioff[i + 1] - lo;
        dense_solve(nb, c->dB[i], c->pvB[i], in + lo, out + lo);
    }
}

void orc_solve_BT(const orc_ctx *c, const double *in, double *out) {
    if (c->factor != 1) {
        ilu_solve_t(&c->luB, in, out);
        return;
    }
    for (int32_t i = 0; i < c->s; ++i) {
        int32_t lo = c->ioff[i], nb = c->ioff[i + 1] - lo;
        dense_solve_t(nb, c->dB[i], c->pvB[i], in + lo, out + lo);
    }
}

void orc_solve_C0(const orc_ctx *c, const double *in, double *out) {
    if (c->factor != 1) {
        ilu_solve(&c->luC, in, out);
        return;
    }
    for (int32_t i = 0; i < c->s; ++i) {
        int32_t lo = c->goff[i], nb = c->goff[i + 1] - lo;
        dense_solve(nb, c->dC[i], c->pvC[i], in + lo, out + lo);
    }
}

void orc_solve_C0T(const orc_ctx *c, const double *in, double *out) {
    if (c->factor != 1) {
        ilu_solve_t(&c->luC, in, out);
        return;
    }
    for (int32_t i = 0; i < c->s; ++i) {
        int32_t lo = c->goff[i], nb = c->goff[i + 1] - lo;
        dense_solve_t(nb, c->dC[i], c->pvC[i], in + lo, out + lo);
    }
}

/* ------------------------------------------- Sec. 3.1: splitting and series */

/* E_s w = F B^{-1} E w - C_g w   (Eq. 3.1 with E_s = (C0 - C) + F B^{-1} E) */
void orc_Es(const orc_ctx *c, const double *in, double *out) {
    double *a = malloc(sizeof(double) * (c->p + 1)), *u = malloc(sizeof(double) * (c->p + 1));
    double *g = malloc(sizeof(double) * (c->q + 1));
    spmv(&c->E, in, a);
    orc_solve_B(c, a, u);
    spmv(&c->F, u, out);
    spmv(&c->Cg, in, g);
    for (int32_t i = 0; i < c->q; ++i) out[i] -= g[i];
    free(a); free(u); free(g);
}

/* E_s^T w = E^T B^{-T} F^T w - C_g^T w */
void orc_EsT(const orc_ctx *c, const double *in, double *out) {
    double *a = malloc(sizeof(double) * (c->p + 1)), *u = malloc(sizeof(double) * (c->p + 1));
    double *g = malloc(sizeof(double) * (c->q + 1));
    spmv_t(&c->F, in, a);
    orc_solve_BT(c, a, u);
    spmv_t(&c->E, u, out);
    spmv_t(&c->Cg, in, g);
    for (int32_t i = 0; i < c->q; ++i) out[i] -= g[i];
    free(a); free(u); free(g);
}

/*
 * Eq. 3.3: P_m t = sum_{i=0}^{m} (C0^{-1} E_s)^i C0^{-1} t, m+1 terms, summed as
 * w_0 = C0^{-1} t, w_i = C0^{-1} E_s w_{i-1}, out = w_0 + w_1 + ... + w_m.
 */
void orc_series(const orc_ctx *c, int32_t m, const double *in, double *out) {
    int32_t q = c->q;
    double *w = malloc(sizeof(double) * (q + 1)), *e = malloc(sizeof(double) * (q + 1));
    orc_solve_C0(c, in, w);
    for (int32_t k = 0; k < q; ++k) out[k] = w[k];
    for (int32_t i = 1; i <= m; ++i) {
        orc_Es(c, w, e);
        orc_solve_C0(c, e, w);
        for (int32_t k = 0; k < q; ++k) out[k] += w[k];
    }
    free(w); free(e);
}

/* P_m^T h = sum_{i=0}^{m} C0^{-T} (E_s^T C0^{-T})^i h, same recurrence with the
 * transposed operators: w_0 = C0^{-T} h, w_i = C0^{-T} E_s^T w_{i-1}. */
void orc_seriesT(const orc_ctx *c, int32_t m, const double *in, double *out) {
    int32_t q = c->q;
    double *w = malloc(sizeof(double) * (q + 1)), *e = malloc(sizeof(double) * (q + 1));
    orc_solve_C0T(c, in, w);
    for (int32_t k = 0; k < q; ++k) out[k] = w[k];
    for (int32_t i = 1; i <= m; ++i) {
        orc_EsT(c, w, e);
        orc_solve_C0T(c, e, w);
        for (int32_t k = 0; k < q; ++k) out[k] += w[k];
    }
    free(w); free(e);
}

/* Sec. 3.2.1, Eq. 3.19: E_rr(m) v = (E_s C0^{-1})^{m+1} v. */
void orc_Err(const orc_ctx *c, int32_t m, const double *in, double *out) {
    int32_t q = c->q;
    double *t = malloc(sizeof(double) * (q + 1));
    for (int32_t k = 0; k < q; ++k) out[k] = in[k];
    for (int32_t i = 0; i <= m; ++i) {
        orc_solve_C0(c, out, t);
        orc_Es(c, t, out);
    }
    free(t);
}

/* ------------------------------------------ Sec. 3.2: low-rank correction */

/*
 * Graph partition by recursive bisection of breadth-first level structures
 * (stands in for METIS in Section 2 when the matrix has no grid).  Graph: the
 * pattern of A + A^T without the diagonal; neighbours in increasing index.
 * To cut a vertex set U (ascending) into k > 1 parts: list U breadth-first,
 * component by component in the order of their smallest vertex, each from a
 * pseudo-peripheral vertex (George and Liu: start at the smallest vertex of
 * the component, search, take the vertex of least degree within U on the last
 * level, smallest index on ties, and repeat from it while the number of
 * levels increases); the first floor(|U| (k/2) / k) listed vertices get the
 * parts base .. base+k/2-1, the others the remaining k - k/2 parts, each side
 * cut again after sorting it.
 */
typedef struct {
    int32_t n;
    int32_t *start, *adj;  /* adjacency lists of A + A^T, no self loops */
    int32_t *in_u;         /* 1 for the vertices of the set being cut */
    int32_t *dist;         /* breadth-first distance, -1 = not reached */
    int32_t *listed;       /* 1 once a vertex is in the breadth-first listing */
} gp_graph;

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Levels of a search from root over the vertices with in_u set and listed
 * clear, appended to seq as they are reached (level by level, each level's
 * vertices expanding in the order they were reached, neighbours ascending).
 * Returns the number of levels; *last_begin = index in seq of the last level. */
static int32_t gp_levels(gp_graph *g, const int32_t *U, int32_t nu, int32_t root, int32_t *seq,
                         int32_t *len, int32_t *last_begin) {
    for (int32_t i = 0; i < nu; ++i) g->dist[U[i]] = -1;
    int32_t cnt = 0, lev_begin = 0, nlev = 0;
    seq[cnt++] = root;
    g->dist[root] = 0;
    while (lev_begin < cnt) {
        int32_t lev_end = cnt;
        *last_begin = lev_begin;
        ++nlev;
        for (int32_t t = lev_begin; t < lev_end; ++t) {
            int32_t v = seq[t];
            for (int32_t e = g->start[v]; e < g->start[v + 1]; ++e) {
                int32_t w = g->adj[e];
                if (!g->in_u[w] || g->listed[w] || g->dist[w] >= 0) continue;
                g->dist[w] = nlev;
                seq[cnt++] = w;
            }
        }
        lev_begin = lev_end;
    }
    *len = cnt;
    return nlev;
}

static int32_t gp_degree(const gp_graph *g, int32_t v) {
    int32_t d = 0;
    for (int32_t e = g->start[v]; e < g->start[v + 1]; ++e) d += g->in_u[g->adj[e]];
    return d;
}

static void gp_cut(gp_graph *g, int32_t *U, int32_t nu, int32_t k, int32_t base, int32_t *part) {
    if (k == 1) {
        for (int32_t i = 0; i < nu; ++i) part[U[i]] = base;
        return;
    }
    int32_t *order = malloc(sizeof(int32_t) * (nu ? nu : 1));
    int32_t *seq = malloc(sizeof(int32_t) * (nu ? nu : 1));
    int32_t norder = 0;
    for (int32_t i = 0; i < nu; ++i) { g->in_u[U[i]] = 1; g->listed[U[i]] = 0; }
    for (int32_t i = 0; i < nu; ++i) {
        int32_t c = U[i], len, lb;
        if (g->listed[c]) continue;
        /* pseudo-peripheral vertex of c's component */
        int32_t r = c, ecc = gp_levels(g, U, nu, r, seq, &len, &lb);
        for (;;) {
            int32_t x = -1, dx = 0;
            for (int32_t t = lb; t < len; ++t) {
                int32_t d = gp_degree(g, seq[t]);
                if (x < 0 || d < dx || (d == dx && seq[t] < x)) { x = seq[t]; dx = d; }
            }
            int32_t ex = gp_levels(g, U, nu, x, seq, &len, &lb);
            if (ex <= ecc) break;
            r = x;
            ecc = ex;
        }
        gp_levels(g, U, nu, r, seq, &len, &lb);
        for (int32_t t = 0; t < len; ++t) {
            order[norder++] = seq[t];
            g->listed[seq[t]] = 1;
        }
    }
    for (int32_t i = 0; i < nu; ++i) g->in_u[U[i]] = 0;
    int32_t k1 = k / 2;
    int32_t n1 = (int32_t)(((int64_t)nu * k1) / k);
    free(seq);
    qsort(order, (size_t)n1, sizeof(int32_t), cmp_i32);
    qsort(order + n1, (size_t)(nu - n1), sizeof(int32_t), cmp_i32);
    gp_cut(g, order, n1, k1, base, part);
    gp_cut(g, order + n1, nu - n1, k - k1, base + k1, part);
    free(order);
}

int32_t orc_graph_partition(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t nparts,
                            int32_t *part) {
    if (n <= 0 || nparts < 1 || nparts > n) return ORC_ERR_ARG;
    gp_graph g;
    g.n = n;
    int32_t *cnt = calloc((size_t)n + 1, sizeof(int32_t));
    for (int32_t v = 0; v < n; ++v)
        for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e)
            if (col[e] != v) { cnt[v + 1]++; cnt[col[e] + 1]++; }
    for (int32_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
    int32_t *raw = malloc(sizeof(int32_t) * (cnt[n] ? cnt[n] : 1));
    int32_t *fill = malloc(sizeof(int32_t) * n);
    for (int32_t v = 0; v < n; ++v) fill[v] = cnt[v];
    for (int32_t v = 0; v < n; ++v)
        for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e)
            if (col[e] != v) { raw[fill[v]++] = col[e]; raw[fill[col[e]]++] = v; }
    g.start = malloc(sizeof(int32_t) * ((size_t)n + 1));
    g.adj = malloc(sizeof(int32_t) * (cnt[n] ? cnt[n] : 1));
    int32_t m = 0;
    g.start[0] = 0;
    for (int32_t v = 0; v < n; ++v) {
        qsort(raw + cnt[v], (size_t)(cnt[v + 1] - cnt[v]), sizeof(int32_t), cmp_i32);
        for (int32_t e = cnt[v]; e < cnt[v + 1]; ++e)
            if (e == cnt[v] || raw[e] != raw[e - 1]) g.adj[m++] = raw[e];
        g.start[v + 1] = m;
    }
    free(raw); free(fill); free(cnt);
    g.in_u = calloc((size_t)n, sizeof(int32_t));
    g.dist = malloc(sizeof(int32_t) * n);
    g.listed = calloc((size_t)n, sizeof(int32_t));
    int32_t *U = malloc(sizeof(int32_t) * n);
    for (int32_t v = 0; v < n; ++v) U[v] = v;
    gp_cut(&g, U, n, nparts, 0, part);
    free(U); free(g.in_u); free(g.dist); free(g.listed); free(g.start); free(g.adj);
    return ORC_OK;
}

double orc_splitmix_uniform(uint64_t seed, uint64_t j) {
    uint64_t z = seed + (j + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

/* Classical Gram-Schmidt against the first k columns of V, applied twice;
 * h (length k) receives the summed coefficients. */
static void cgs2(int32_t q, int32_t k, const double *V, double *w, double *h) {
    double *t = malloc(sizeof(double) * (k + 1));
    for (int32_t i = 0; i < k; ++i) h[i] = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
        for (int32_t i = 0; i < k; ++i) t[i] = dot(q, V + (size_t)i * q, w);
        for (int32_t i = 0; i < k; ++i)
            for (int32_t l = 0; l < q; ++l) w[l] -= t[i] * V[(size_t)i * q + l];
        for (int32_t i = 0; i < k; ++i) h[i] += t[i];
    }
    free(t);
}

/* G = (I - H)^{-1} - I by LU with partial pivoting of I - H (Eq. 3.17). */
static int32_t compute_G(int32_t r, const double *H, double *G) {
    double *a = malloc(sizeof(double) * (r * r + 1)), *x = malloc(sizeof(double) * (r + 1));
    int32_t *pv = malloc(sizeof(int32_t) * (r + 1));
    double amax = 0.0;
    for (int32_t i = 0; i < r; ++i) /* row-major copy of I - H (H column-major) */
        for (int32_t j = 0; j < r; ++j) {
            a[i * r + j] = (i == j ? 1.0 : 0.0) - H[j * r + i];
            if (fabs(a[i * r + j]) > amax) amax = fabs(a[i * r + j]);
        }
    for (int32_t k = 0; k < r; ++k) {
        int32_t pr = k;
        double best = fabs(a[k * r + k]);
        for (int32_t i = k + 1; i < r; ++i)
            if (fabs(a[i * r + k]) > best) {
                best = fabs(a[i * r + k]);
                pr = i;
            }
        pv[k] = pr;
        if (best <= 1e-14 * amax) {
            free(a); free(x); free(pv);
            return ORC_ERR_SINGULAR_IMH;
        }
        if (pr != k)
            for (int32_t j = 0; j < r; ++j) {
                double t = a[k * r + j];
                a[k * r + j] = a[pr * r + j];
                a[pr * r + j] = t;
            }
        for (int32_t i = k + 1; i < r; ++i) {
            double l = a[i * r + k] / a[k * r + k];
            a[i * r + k] = l;
            for (int32_t j = k + 1; j < r; ++j) a[i * r + j] -= l * a[k * r + j];
        }
    }
    for (int32_t j = 0; j < r; ++j) { /* column j of (I - H)^{-1} */
        for (int32_t i = 0; i < r; ++i) x[i] = (i == j) ? 1.0 : 0.0;
        for (int32_t k = 0; k < r; ++k)
            if (pv[k] != k) {
                double t = x[k];
                x[k] = x[pv[k]];
                x[pv[k]] = t;
            }
        for (int32_t i = 0; i < r; ++i)
            for (int32_t l = 0; l < i; ++l) x[i] -= a[i * r + l] * x[l];
        for (int32_t i = r - 1; i >= 0; --i) {
            for (int32_t l = i + 1; l < r; ++l) x[i] -= a[i * r + l] * x[l];
            x[i] /= a[i * r + i];
        }
        for (int32_t i = 0; i < r; ++i) G[j * r + i] = x[i] - (i == j ? 1.0 : 0.0);
    }
    free(a); free(x); free(pv);
    return ORC_OK;
}

/*
 * Algorithm 1 steps 6-8 with Eq. 3.16-3.17.  Arnoldi on E_rr(m):
 * v_1 = u / ||u||, u_l = U[-1,1) from SplitMix64(seed) output l; for j = 1..r:
 * w = E_rr(m) v_j, h_{1:j,j} by classical Gram-Schmidt twice, h_{j+1,j} = ||w||,
 * v_{j+1} = w / h_{j+1,j}.  H is the leading r x r block (h_{r+1,r} dropped).
 * Breakdown, h_{j+1,j} <= 1e-12 ||H(1:j+1,1:j)||_F with j < r: truncate to rank
 * j, or (full_rank) start a fresh SplitMix64 vector (outputs t*q .. t*q+q-1 for
 * the t-th vector) orthogonalised against V, with h_{j+1,j} = 0.
 */
int32_t orc_build_lowrank(orc_ctx *c, int32_t m, int32_t rank, uint64_t seed, int32_t full_rank,
                          int32_t *rank_out) {
    int32_t q = c->q;
    free(c->V); free(c->H); free(c->G);
    c->V = c->H = c->G = NULL;
    c->m = m;
    c->r = 0;
    *rank_out = 0;
    if (rank > q) rank = q;
    if (rank <= 0 || q == 0) return ORC_OK;
    int32_t r = rank;
    double *V = calloc((size_t)q * (r + 1), sizeof(double));
    double *Hb = calloc((size_t)(r + 1) * r, sizeof(double)); /* (r+1) x r, column-major */
    double *w = malloc(sizeof(double) * q), *h = malloc(sizeof(double) * (r + 1));
    int32_t tvec = 0;
    for (int32_t l = 0; l < q; ++l) V[l] = orc_splitmix_uniform(seed, (uint64_t)l);
    double nu = nrm2(q, V);
    for (int32_t l = 0; l < q; ++l) V[l] /= nu;
    int32_t kept = r;
    double hf2 = 0.0;
    for (int32_t j = 0; j < r; ++j) {
        orc_Err(c, m, V + (size_t)j * q, w);
        cgs2(q, j + 1, V, w, h);
        double hn = nrm2(q, w);
        for (int32_t i = 0; i <= j; ++i) {
            Hb[(size_t)j * (r + 1) + i] = h[i];
            hf2 += h[i] * h[i];
        }
        hf2 += hn * hn;
        if (j == r - 1) break;
        if (hn <= 1e-12 * sqrt(hf2)) {
            if (!full_rank) {
                kept = j + 1;
                break;
            }
            /* fresh direction orthogonal to V(:, 0..j) */
            double *vn = V + (size_t)(j + 1) * q;
            ++tvec;
            for (int32_t l = 0; l < q; ++l)
                vn[l] = orc_splitmix_uniform(seed, (uint64_t)tvec * q + l);
            cgs2(q, j + 1, V, vn, h);
            double nn = nrm2(q, vn);
            for (int32_t l = 0; l < q; ++l) vn[l] /= nn;
            Hb[(size_t)j * (r + 1) + j + 1] = 0.0;
        } else {
            Hb[(size_t)j * (r + 1) + j + 1] = hn;
            for (int32_t l = 0; l < q; ++l) V[(size_t)(j + 1) * q + l] = w[l] / hn;
        }
    }
    c->V = malloc(sizeof(double) * (size_t)q * kept);
    c->H = malloc(sizeof(double) * (size_t)kept * kept);
    c->G = malloc(sizeof(double) * (size_t)kept * kept);
    memcpy(c->V, V, sizeof(double) * (size_t)q * kept);
    for (int32_t j = 0; j < kept; ++j)
        for (int32_t i = 0; i < kept; ++i) c->H[j * kept + i] = Hb[(size_t)j * (r + 1) + i];
    free(V); free(Hb); free(w); free(h);
    c->r = kept;
    *rank_out = kept;
    int32_t st = compute_G(kept, c->H, c->G);
    if (st != ORC_OK) {
        free(c->V); free(c->H); free(c->G);
        c->V = c->H = c->G = NULL;
        c->r = 0;
        *rank_out = 0;
        return st;
    }
    return kept < rank ? ORC_ERR_BREAKDOWN : ORC_OK;
}

void orc_get_lowrank(const orc_ctx *c, double *V, double *H, double *G) {
    if (c->r == 0) return;
    if (V) memcpy(V, c->V, sizeof(double) * (size_t)c->q * c->r);
    if (H && c->H) memcpy(H, c->H, sizeof(double) * (size_t)c->r * c->r);
    if (G) memcpy(G, c->G, sizeof(double) * (size_t)c->r * c->r);
}

int32_t orc_set_lowrank(orc_ctx *c, int32_t m, int32_t rank, const double *V, const double *G) {
    free(c->V); free(c->H); free(c->G);
    c->V = c->H = c->G = NULL;
    c->m = m;
    c->r = rank;
    if (rank <= 0) {
        c->r = 0;
        return ORC_OK;
    }
    c->V = malloc(sizeof(double) * (size_t)c->q * rank);
    c->G = malloc(sizeof(double) * (size_t)rank * rank);
    memcpy(c->V, V, sizeof(double) * (size_t)c->q * rank);
    memcpy(c->G, G, sizeof(double) * (size_t)rank * rank);
    return ORC_OK;
}

/* ------------------------------------------------ Algorithm 3 and transpose */

/* t <- t + V op(G) V^T t, op(G) = G or G^T. */
static void lowrank_update(const orc_ctx *c, double *t, int transpose) {
    int32_t q = c->q, r = c->r;
    if (r == 0) return;
    double *u = malloc(sizeof(double) * r), *d = malloc(sizeof(double) * r);
    for (int32_t i = 0; i < r; ++i) u[i] = dot(q, c->V + (size_t)i * q, t);
    for (int32_t i = 0; i < r; ++i) {
        double acc = 0.0;
        for (int32_t j = 0; j < r; ++j)
            acc += (transpose ? c->G[i * r + j] : c->G[j * r + i]) * u[j];
        d[i] = acc;
    }
    for (int32_t i = 0; i < r; ++i)
        for (int32_t l = 0; l < q; ++l) t[l] += c->V[(size_t)i * q + l] * d[i];
    free(u); free(d);
}

/*
 * Algorithm 3 (Eq. 3.24): b = (f; g) in the reordered numbering;
 *   t = g - F B^{-1} f,  t <- t + V G V^T t,  y = P_m t,  x = B^{-1}(f - E y),
 *   z = (x; y), scattered back to the original numbering.
 */
void orc_apply(const orc_ctx *c, const double *b, double *z) {
    int32_t p = c->p, q = c->q;
    double *f = malloc(sizeof(double) * (p + 1)), *u = malloc(sizeof(double) * (p + 1));
    double *t = malloc(sizeof(double) * (q + 1)), *y = malloc(sizeof(double) * (q + 1));
    double *x = malloc(sizeof(double) * (p + 1));
    for (int32_t i = 0; i < p; ++i) f[i] = b[c->perm[i]];
    orc_solve_B(c, f, u);
    spmv(&c->F, u, t);
    for (int32_t i = 0; i < q; ++i) t[i] = b[c->perm[p + i]] - t[i];
    lowrank_update(c, t, 0);
    orc_series(c, c->m, t, y);
    spmv(&c->E, y, u);
    for (int32_t i = 0; i < p; ++i) u[i] = f[i] - u[i];
    orc_solve_B(c, u, x);
    for (int32_t i = 0; i < p; ++i) z[c->perm[i]] = x[i];
    for (int32_t i = 0; i < q; ++i) z[c->perm[p + i]] = y[i];
    free(f); free(u); free(t); free(y); free(x);
}

/*
 * Exact transpose of Algorithm 3 (not in the paper; derived from the block
 * form M^{-1} = [[B^{-1} + B^{-1} E K F B^{-1}, -B^{-1} E K], [-K F B^{-1}, K]]
 * with K = P_m (I + V G V^T)).  For b = (f; g):
 *   h = g - E^T B^{-T} f,  w = (I + V G^T V^T) P_m^T h,  x = B^{-T}(f - F^T w).
 */
void orc_apply_T(const orc_ctx *c, const double *b, double *z) {
    int32_t p = c->p, q = c->q;
    double *f = malloc(sizeof(double) * (p + 1)), *u = malloc(sizeof(double) * (p + 1));
    double *h = malloc(sizeof(double) * (q + 1)), *w = malloc(sizeof(double) * (q + 1));
    double *x = malloc(sizeof(double) * (p + 1));
    for (int32_t i = 0; i < p; ++i) f[i] = b[c->perm[i]];
    orc_solve_BT(c, f, u);
    spmv_t(&c->E, u, h);
    for (int32_t i = 0; i < q; ++i) h[i] = b[c->perm[p + i]] - h[i];
    orc_seriesT(c, c->m, h, w);
    lowrank_update(c, w, 1);
    spmv_t(&c->F, w, u);
    for (int32_t i = 0; i < p; ++i) u[i] = f[i] - u[i];
    orc_solve_BT(c, u, x);
    for (int32_t i = 0; i < p; ++i) z[c->perm[i]] = x[i];
    for (int32_t i = 0; i < q; ++i) z[c->perm[p + i]] = w[i];
    free(f); free(u); free(h); free(w); free(x);
}

/* ------------------------------- Sec. 1: the classical Neumann polynomial */

/* y = C0~ w (or C0~^T w): the matrix whose inverse the local C0 solves apply -
 * L U of the incomplete factor (unit lower L, upper U, stored together), or
 * C0 itself for the exact LU. */
static void c0_mult(const orc_ctx *c, int transpose, const double *w, double *y) {
    int32_t q = c->q;
    if (c->factor == 1) {
        if (transpose) spmv_t(&c->C0, w, y);
        else spmv(&c->C0, w, y);
        return;
    }
    const ocsr *LU = &c->luC;
    double *u = calloc((size_t)q + 1, sizeof(double));
    if (!transpose) { /* u = U w, y = L u */
        for (int32_t i = 0; i < q; ++i)
            for (int32_t k = LU->rp[i]; k < LU->rp[i + 1]; ++k)
                if (LU->ci[k] >= i) u[i] += LU->v[k] * w[LU->ci[k]];
        for (int32_t i = 0; i < q; ++i) {
            double a = u[i];
            for (int32_t k = LU->rp[i]; k < LU->rp[i + 1]; ++k)
                if (LU->ci[k] < i) a += LU->v[k] * u[LU->ci[k]];
            y[i] = a;
        }
    } else { /* (L U)^T w = U^T (L^T w) */
        for (int32_t i = 0; i < q; ++i) u[i] = w[i];
        for (int32_t i = 0; i < q; ++i)
            for (int32_t k = LU->rp[i]; k < LU->rp[i + 1]; ++k)
                if (LU->ci[k] < i) u[LU->ci[k]] += LU->v[k] * w[i];
        for (int32_t i = 0; i < q; ++i) y[i] = 0.0;
        for (int32_t i = 0; i < q; ++i)
            for (int32_t k = LU->rp[i]; k < LU->rp[i + 1]; ++k)
                if (LU->ci[k] >= i) y[LU->ci[k]] += LU->v[k] * u[i];
    }
    free(u);
}

/* S w = C0~ w - E_s w (Eq. 3.1 with the factored C0), or S^T w. */
static void schur_mult(const orc_ctx *c, int transpose, const double *w, double *y) {
    double *e = malloc(sizeof(double) * ((size_t)c->q + 1));
    c0_mult(c, transpose, w, y);
    if (transpose) orc_EsT(c, w, e);
    else orc_Es(c, w, e);
    for (int32_t i = 0; i < c->q; ++i) y[i] -= e[i];
    free(e);
}

/*
 * Sec. 1, the Neumann polynomial of the Schur complement that the paper
 * contrasts with its method: N = I - omega D^{-1} S, with D the block
 * diagonal of S taken as C0 (the splitting of Eq. 3.1; D^{-1} is the local
 * factor solve and S = C0~ - E_s the matrix those solves make exact), and
 *     S^{-1} ~ omega [I + N + N^2 + ... + N^m] D^{-1},
 * the identity S^{-1} = omega (I - N)^{-1} D^{-1} truncated after m+1 terms
 * (it converges only when rho(N) < 1).  Summed as v_0 = D^{-1} t,
 * v_i = N v_{i-1} = v_{i-1} - omega D^{-1} (S v_{i-1}), out = omega sum v_i.
 * The transpose, omega sum_i D^{-T} (N^T)^i t, runs v_0 = t,
 * v_i = v_{i-1} - omega S^T D^{-T} v_{i-1}, out = omega sum D^{-T} v_i.
 */
void orc_neumann_series(const orc_ctx *c, int32_t m, double omega, int32_t transpose, const double *in,
                        double *out) {
    int32_t q = c->q;
    double *v = malloc(sizeof(double) * ((size_t)q + 1)), *a = malloc(sizeof(double) * ((size_t)q + 1));
    double *d = malloc(sizeof(double) * ((size_t)q + 1));
    if (!transpose) {
        orc_solve_C0(c, in, v);
        for (int32_t k = 0; k < q; ++k) out[k] = v[k];
        for (int32_t i = 1; i <= m; ++i) {
            schur_mult(c, 0, v, a);
            orc_solve_C0(c, a, d);
            for (int32_t k = 0; k < q; ++k) {
                v[k] -= omega * d[k];
                out[k] += v[k];
            }
        }
    } else {
        for (int32_t k = 0; k < q; ++k) v[k] = in[k];
        orc_solve_C0T(c, v, d);
        for (int32_t k = 0; k < q; ++k) out[k] = d[k];
        for (int32_t i = 1; i <= m; ++i) {
            schur_mult(c, 1, d, a); /* S^T D^{-T} v_{i-1}, with d = D^{-T} v_{i-1} */
            for (int32_t k = 0; k < q; ++k) v[k] -= omega * a[k];
            orc_solve_C0T(c, v, d);
            for (int32_t k = 0; k < q; ++k) out[k] += d[k];
        }
    }
    for (int32_t k = 0; k < q; ++k) out[k] *= omega;
    free(v); free(a); free(d);
}

/* The block elimination of Algorithm 3 with the Neumann polynomial in place of
 * P_m (I + V G V^T) (no low-rank term): t = g - F B^{-1} f, y = the series of
 * t, x = B^{-1}(f - E y); and its transpose, as orc_apply_T. */
void orc_neumann_apply(const orc_ctx *c, int32_t m, double omega, int32_t transpose, const double *b, double *z) {
    int32_t p = c->p, q = c->q;
    double *f = malloc(sizeof(double) * (p + 1)), *u = malloc(sizeof(double) * (p + 1));
    double *t = malloc(sizeof(double) * (q + 1)), *y = malloc(sizeof(double) * (q + 1));
    double *x = malloc(sizeof(double) * (p + 1));
    for (int32_t i = 0; i < p; ++i) f[i] = b[c->perm[i]];
    if (!transpose) {
        orc_solve_B(c, f, u);
        spmv(&c->F, u, t);
    } else {
        orc_solve_BT(c, f, u);
        spmv_t(&c->E, u, t);
    }
    for (int32_t i = 0; i < q; ++i) t[i] = b[c->perm[p + i]] - t[i];
    orc_neumann_series(c, m, omega, transpose, t, y);
    if (!transpose) spmv(&c->E, y, u);
    else spmv_t(&c->F, y, u);
    for (int32_t i = 0; i < p; ++i) u[i] = f[i] - u[i];
    if (!transpose) orc_solve_B(c, u, x);
    else orc_solve_BT(c, u, x);
    for (int32_t i = 0; i < p; ++i) z[c->perm[i]] = x[i];
    for (int32_t i = 0; i < q; ++i) z[c->perm[p + i]] = y[i];
    free(f); free(u); free(t); free(y); free(x);
}

/* FGMRES with the foil (omega > 0) or with PSLR again (omega <= 0). */
void orc_set_neumann(orc_ctx *c, int32_t m, double omega) {
    c->nf_on = omega > 0.0;
    c->nf_m = m;
    c->nf_omega = omega;
}

/* -------------------------------------------------------------- FGMRES */

static void op_A(const orc_ctx *c, int transpose, const double *x, double *y) {
    if (transpose) spmv_t(&c->A, x, y);
    else spmv(&c->A, x, y);
}

static void op_M(const orc_ctx *c, int prec, int transpose, const double *x, double *y) {
    if (!prec) {
        memcpy(y, x, sizeof(double) * c->n);
        return;
    }
    if (c->nf_on) orc_neumann_apply(c, c->nf_m, c->nf_omega, transpose, x, y);
    else if (transpose) orc_apply_T(c, x, y);
    else orc_apply(c, x, y);
}

/*
 * Flexible GMRES (Saad, Iterative Methods, Alg. 9.6), right preconditioned,
 * x0 = 0, restart length `restart`, Section 4's stopping rule
 * ||b - A x|| <= rtol ||b|| (checked on the least-squares residual |gamma_{j+1}|
 * inside a cycle and confirmed on the true residual at the end of a cycle).
 * prec bit 0: PSLR preconditioner on; bit 1: solve with A^T and M^T.
 */
int32_t orc_fgmres(const orc_ctx *c, int32_t prec, const double *b, double *x, double rtol,
                   int32_t restart, int32_t maxit, int32_t *iters, double *relres) {
    int32_t n = c->n, k = restart;
    int use_m = prec & 1, tr = (prec >> 1) & 1;
    double *V = malloc(sizeof(double) * (size_t)n * (k + 1));
    double *Z = malloc(sizeof(double) * (size_t)n * k);
    double *H = calloc((size_t)(k + 1) * k, sizeof(double)); /* column-major (k+1) x k */
    double *cs = malloc(sizeof(double) * k), *sn = malloc(sizeof(double) * k);
    double *gam = malloc(sizeof(double) * (k + 1)), *y = malloc(sizeof(double) * k);
    double *r = malloc(sizeof(double) * n), *w = malloc(sizeof(double) * n);
    double *hc = malloc(sizeof(double) * (k + 1));
    double bn = nrm2(n, b);
    int32_t its = 0, st = ORC_ERR_NOT_CONVERGED;
    for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
    *relres = 0.0;
    if (bn == 0.0) {
        *iters = 0;
        st = ORC_OK;
        goto done;
    }
    for (int32_t i = 0; i < n; ++i) r[i] = b[i];
    double rn = bn;
    while (its < maxit) {
        for (int32_t i = 0; i < n; ++i) V[i] = r[i] / rn;
        gam[0] = rn;
        int32_t j, jdone = 0;
        for (j = 0; j < k && its < maxit; ++j) {
            op_M(c, use_m, tr, V + (size_t)j * n, Z + (size_t)j * n);
            op_A(c, tr, Z + (size_t)j * n, w);
            cgs2(n, j + 1, V, w, hc);
            double hn = nrm2(n, w);
            ++its;
            for (int32_t i = 0; i <= j; ++i) H[(size_t)j * (k + 1) + i] = hc[i];
            H[(size_t)j * (k + 1) + j + 1] = hn;
            if (hn > 0.0)
                for (int32_t i = 0; i < n; ++i) V[(size_t)(j + 1) * n + i] = w[i] / hn;
            for (int32_t i = 0; i < j; ++i) { /* previous rotations */
                double a = H[(size_t)j * (k + 1) + i], bb = H[(size_t)j * (k + 1) + i + 1];
                H[(size_t)j * (k + 1) + i] = cs[i] * a + sn[i] * bb;
                H[(size_t)j * (k + 1) + i + 1] = -sn[i] * a + cs[i] * bb;
            }
            double a = H[(size_t)j * (k + 1) + j], bb = H[(size_t)j * (k + 1) + j + 1];
            double den = sqrt(a * a + bb * bb);
            cs[j] = den > 0.0 ? a / den : 1.0;
            sn[j] = den > 0.0 ? bb / den : 0.0;
            H[(size_t)j * (k + 1) + j] = den;
            H[(size_t)j * (k + 1) + j + 1] = 0.0;
            gam[j + 1] = -sn[j] * gam[j];
            gam[j] = cs[j] * gam[j];
            jdone = j + 1;
            if (fabs(gam[j + 1]) <= rtol * bn || hn == 0.0) break;
        }
        for (int32_t i = jdone - 1; i >= 0; --i) { /* H y = gamma */
            double acc = gam[i];
            for (int32_t l = i + 1; l < jdone; ++l) acc -= H[(size_t)l * (k + 1) + i] * y[l];
            y[i] = acc / H[(size_t)i * (k + 1) + i];
        }
        for (int32_t l = 0; l < jdone; ++l)
            for (int32_t i = 0; i < n; ++i) x[i] += Z[(size_t)l * n + i] * y[l];
        op_A(c, tr, x, w);
        for (int32_t i = 0; i < n; ++i) r[i] = b[i] - w[i];
        rn = nrm2(n, r);
        *relres = rn / bn;
        if (rn <= rtol * bn) {
            st = ORC_OK;
            break;
        }
    }
    *iters = its;
done:
    free(V); free(Z); free(H); free(cs); free(sn); free(gam); free(y); free(r); free(w); free(hc);
    return st;
}

/*
 * amg_oracle.c -- plain, slow, single-threaded FP64 CPU oracle of the auxiliary-grid AMG
 * method (Wang, Hu, Cohen, Xu, "A Parallel Auxiliary Grid AMG Method for GPU").
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline / reference arm may load it. The product (the CUDA library) never calls it, and
 * the two share no code: no headers, helpers or generated tables.
 *
 * Built with: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, IEEE division).
 *
 * Every step follows the paper in the paper's order and notation; where the paper is silent
 * or garbled the reading taken is stated at the step (readings R1..R17):
 *   setup:  auxiliary box (Sec. 3.1, eq. ab12), depth L (Sec. 3.1), level-L aggregation
 *           (Sec. 3.2 eq. agg_L; Sec. 4.2 index formula), coarse aggregation (Sec. 3.2 eq.
 *           agg_k; Sec. 4.2 parent formula), Galerkin operators (Sec. 2 eqs. def:Ac, acsum),
 *           quadtree colouring (Sec. 4.5), coarsest exact solve (Alg. 2, B_1 = A_1^{-1}).
 *   solve:  colored Gauss-Seidel R_k / R_k^t (Sec. 4.5), nonlinear AMLI-cycle (Alg. 2),
 *           nonlinear PCG (Alg. 1), outer Krylov iteration (Sec. 4: the AMG preconditions a
 *           Krylov method; Alg. 1 applied on the finest level).
 *
 * Parity status: every function is pinned by tests/test_oracle_*.py against closed forms,
 * brute force, dense linear algebra or textbook routines.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OAMG_OK 0
#define OAMG_ERR_INVALID_ARG 1
#define OAMG_ERR_BAD_MATRIX 2
#define OAMG_ERR_OOM 3
#define OAMG_ERR_NOT_CONVERGED 5
#define OAMG_ERR_BREAKDOWN 6

typedef struct {
    int aux_level;     /* depth L of the quadtree; 0 = automatic (Sec. 3.1) */
    int coarsest_max;  /* stop coarsening at the first level with at most this many rows */
    int kcycle_n;      /* steps n of Alg. 1 inside the AMLI-cycle */
    int max_iters;     /* outer iterations */
    int has_bbox;      /* 1: use bbox below instead of eq. ab12 */
    double bbox[4];    /* a1, b1, a2, b2 */
    int no_factor;     /* 1: skip the coarsest Cholesky (inspect operators of singular A) */
    int dim;           /* 2 (quadtree, default when 0) or 3 (octree, Sec. 3.1 / Sec. 6) */
    double zbox[2];    /* a3, b3 (dim 3 with has_bbox) */
    int nu_pre;        /* Gauss-Seidel sweeps of the pre-smoothing (reading R10); 0 = 1 */
    int nu_post;       /* sweeps of the post-smoothing; 0 = 1 */
} oamg_opts;

typedef struct {
    int n;              /* unknowns on this level */
    int *rowptr, *col;  /* CSR, columns ascending */
    double *val;
    int cellw;          /* cells per side of the grid this level's rows live on */
    int *t1, *t2;       /* cell coordinates of each row (fine level: its level-L cell) */
    int *t3;            /* third cell coordinate (octree only; NULL for the quadtree) */
    int span;           /* s: max cell offset over the nonzeros */
    int m;              /* colour modulus max(2, s+1) */
    int *color;         /* colour of each row */
    int *perm;          /* pi: sweep order, perm[p] = row */
    int *agg;           /* row -> row of the next coarser level (NULL on the coarsest) */
    double *chol;       /* dense Cholesky factor (coarsest level only), row-major lower */
} olevel;

typedef struct {
    int nlev;
    olevel lev[40];
    int L;              /* depth of the auxiliary grid */
    int dim;            /* 2: quadtree, 3: octree */
    double bbox[6];     /* a1, b1, a2, b2, a3, b3 */
    oamg_opts opt;
    double *work;       /* scratch vectors */
} oamg_h;

static void *xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s ? s : 1); }

/* ---------------------------------------------------------------------------------------
 * Input validation: square CSR with sorted unique in-range columns and positive diagonal.
 * ------------------------------------------------------------------------------------- */
static int check_csr(int n, const int *rp, const int *ci, const double *v) {
    if (rp[0] != 0) return OAMG_ERR_BAD_MATRIX;
    for (int i = 0; i < n; i++) {
        if (rp[i + 1] < rp[i]) return OAMG_ERR_BAD_MATRIX;
        int has_diag = 0;
        for (int p = rp[i]; p < rp[i + 1]; p++) {
            if (ci[p] < 0 || ci[p] >= n) return OAMG_ERR_BAD_MATRIX;
            if (p > rp[i] && ci[p] <= ci[p - 1]) return OAMG_ERR_BAD_MATRIX;
            if (!isfinite(v[p])) return OAMG_ERR_BAD_MATRIX;
            if (ci[p] == i) {
                has_diag = 1;
                if (!(v[p] > 0.0)) return OAMG_ERR_BAD_MATRIX;
            }
        }
        if (!has_diag) return OAMG_ERR_BAD_MATRIX;
    }
    return OAMG_OK;
}

/* ---------------------------------------------------------------------------------------
 * Sec. 3.1: depth of the quadtree. The paper asks 4^L < N and gives L = floor(log N/log 4);
 * the two disagree only when N is a power of 4. Reading R8: L = the largest integer with
 * 4^L <= N, computed in integers (the floor formula), N = number of unknowns.
 * ------------------------------------------------------------------------------------- */
int oamg_auto_level(long long N) {
    int L = 0;
    while (N >= (1LL << (2 * (L + 1)))) L++;
    return L;
}

/* The octree's depth (Sec. 3.1 with 8 children per cell): the largest L with 8^L <= N. */
int oamg_auto_level3(long long N) {
    int L = 0;
    while (N >= (1LL << (3 * (L + 1)))) L++;
    return L;
}

/* Level-L cell index of one point (Sec. 4.2 index formula; eq. subregion for the boxes).
 * Operation order: subtract, divide (IEEE, correctly rounded), multiply by 2^L (exact),
 * floor. Reading R4: the closed right/top edge of the box belongs to the last cell. */
static int cell_index_1d(double v, double lo, double hi, int L) {
    int w = 1 << L;
    if (!(hi > lo)) return 0;
    double q = (v - lo) / (hi - lo);
    double s = q * (double)w;
    if (!(s >= 0.0)) return 0;           /* below the box: first cell */
    if (s >= (double)w) return w - 1;    /* on or beyond the closed upper edge: last cell */
    return (int)floor(s);
}

/* Sweep order pi of a level (Sec. 4.5; readings R9, R14): colour ascending, then aggregate
 * (= cell) ascending, then row index ascending within the aggregate. key1 = colour,
 * key2 = aggregate/cell rank, key3 = row. Counting sorts, each stable. */
static void sweep_order(int n, const int *color, int ncolor, const int *blockkey, int nblock,
                        int *perm) {
    int *tmp = (int *)xcalloc((size_t)n, sizeof(int));
    int *cnt = (int *)xcalloc((size_t)(nblock > ncolor ? nblock : ncolor) + 1, sizeof(int));
    /* pass 1: stable sort rows by block key */
    for (int i = 0; i < n; i++) cnt[blockkey[i] + 1]++;
    for (int b = 0; b < nblock; b++) cnt[b + 1] += cnt[b];
    for (int i = 0; i < n; i++) tmp[cnt[blockkey[i]]++] = i;
    /* pass 2: stable sort by colour */
    memset(cnt, 0, sizeof(int) * ((size_t)(nblock > ncolor ? nblock : ncolor) + 1));
    for (int i = 0; i < n; i++) cnt[color[i] + 1]++;
    for (int c = 0; c < ncolor; c++) cnt[c + 1] += cnt[c];
    for (int p = 0; p < n; p++) {
        int i = tmp[p];
        perm[cnt[color[i]]++] = i;
    }
    free(tmp);
    free(cnt);
}

/* Span s of a level: the largest |dt1| or |dt2| between the cells of the row and column of
 * any stored entry (reading R5). cell coordinates are given per row. */
static int level_span(const olevel *lv) {
    int s = 0;
    for (int i = 0; i < lv->n; i++)
        for (int p = lv->rowptr[i]; p < lv->rowptr[i + 1]; p++) {
            int j = lv->col[p];
            int d1 = abs(lv->t1[i] - lv->t1[j]);
            int d2 = abs(lv->t2[i] - lv->t2[j]);
            if (d1 > s) s = d1;
            if (d2 > s) s = d2;
            if (lv->t3) {
                int d3 = abs(lv->t3[i] - lv->t3[j]);
                if (d3 > s) s = d3;
            }
        }
    return s;
}

/* Colouring (Sec. 4.5 with reading R5): m = max(2, s+1), colour = (t1 mod m) + m (t2 mod m).
 * Two distinct cells of one colour differ by a multiple of m > s in t1 or t2, so they are
 * not coupled. */
static void level_colors(olevel *lv) {
    lv->m = lv->span + 1 > 2 ? lv->span + 1 : 2;
    for (int i = 0; i < lv->n; i++) {
        lv->color[i] = (lv->t1[i] % lv->m) + lv->m * (lv->t2[i] % lv->m);
        /* octree: + m^2 (t3 mod m), m^3 colours (8 when s <= 1, Sec. 6) */
        if (lv->t3) lv->color[i] += lv->m * lv->m * (lv->t3[i] % lv->m);
    }
}

/* Galerkin operator A_c = P^t A P (Sec. 2, eq. def:Ac), entrywise eq. acsum:
 * (A_c)_{RC} = sum_{i in G_R} sum_{j in G_C} a_ij. For each coarse row R the contributions of
 * its members (ascending) in CSR order are collected, stably sorted by C, and equal C summed
 * in that order. Pattern-free: every (R, C) that receives a contribution is stored. */
typedef struct { int c; int seq; double v; } contrib;

static int cmp_contrib(const void *a, const void *b) {
    const contrib *x = (const contrib *)a, *y = (const contrib *)b;
    if (x->c != y->c) return x->c < y->c ? -1 : 1;
    return x->seq < y->seq ? -1 : (x->seq > y->seq);
}

static int galerkin(const olevel *f, int nc, olevel *c) {
    int n = f->n;
    /* members of each aggregate, ascending (stable counting sort) */
    int *mptr = (int *)xcalloc((size_t)nc + 1, sizeof(int));
    int *mem = (int *)xcalloc((size_t)n, sizeof(int));
    if (!mptr || !mem) return OAMG_ERR_OOM;
    for (int i = 0; i < n; i++) mptr[f->agg[i] + 1]++;
    for (int R = 0; R < nc; R++) mptr[R + 1] += mptr[R];
    int *fill = (int *)xcalloc((size_t)nc, sizeof(int));
    for (int i = 0; i < n; i++) {
        int R = f->agg[i];
        mem[mptr[R] + fill[R]++] = i;
    }
    free(fill);
    /* pass over coarse rows */
    size_t cap = 1024;
    contrib *buf = (contrib *)malloc(cap * sizeof(contrib));
    size_t nnz_cap = (size_t)f->rowptr[n] + 16;
    c->rowptr = (int *)xcalloc((size_t)nc + 1, sizeof(int));
    c->col = (int *)xcalloc(nnz_cap, sizeof(int));
    c->val = (double *)xcalloc(nnz_cap, sizeof(double));
    if (!buf || !c->rowptr || !c->col || !c->val) return OAMG_ERR_OOM;
    size_t out = 0;
    for (int R = 0; R < nc; R++) {
        size_t k = 0;
        for (int q = mptr[R]; q < mptr[R + 1]; q++) {
            int i = mem[q];
            for (int p = f->rowptr[i]; p < f->rowptr[i + 1]; p++) {
                if (k == cap) {
                    cap *= 2;
                    buf = (contrib *)realloc(buf, cap * sizeof(contrib));
                    if (!buf) return OAMG_ERR_OOM;
                }
                buf[k].c = f->agg[f->col[p]];
                buf[k].seq = (int)k;
                buf[k].v = f->val[p];
                k++;
            }
        }
        qsort(buf, k, sizeof(contrib), cmp_contrib);
        size_t a = 0;
        while (a < k) {
            size_t b = a;
            double s = 0.0;
            while (b < k && buf[b].c == buf[a].c) s += buf[b++].v;
            c->col[out] = buf[a].c;
            c->val[out] = s;
            out++;
            a = b;
        }
        c->rowptr[R + 1] = (int)out;
    }
    c->n = nc;
    free(buf);
    free(mptr);
    free(mem);
    return OAMG_OK;
}

/* Dense Cholesky A = L L^t of the coarsest matrix (exact coarsest solve, Alg. 2). */
static int cholesky(olevel *lv) {
    int n = lv->n;
    double *a = (double *)xcalloc((size_t)n * n, sizeof(double));
    if (!a) return OAMG_ERR_OOM;
    for (int i = 0; i < n; i++)
        for (int p = lv->rowptr[i]; p < lv->rowptr[i + 1]; p++) a[(size_t)i * n + lv->col[p]] = lv->val[p];
    for (int j = 0; j < n; j++) {
        double d = a[(size_t)j * n + j];
        for (int k = 0; k < j; k++) d -= a[(size_t)j * n + k] * a[(size_t)j * n + k];
        if (!(d > 0.0)) { free(a); return OAMG_ERR_BAD_MATRIX; }
        d = sqrt(d);
        a[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; i++) {
            double s = a[(size_t)i * n + j];
            for (int k = 0; k < j; k++) s -= a[(size_t)i * n + k] * a[(size_t)j * n + k];
            a[(size_t)i * n + j] = s / d;
        }
    }
    lv->chol = a;
    return OAMG_OK;
}

static void chol_solve(const olevel *lv, const double *f, double *u) {
    int n = lv->n;
    const double *a = lv->chol;
    for (int i = 0; i < n; i++) {
        double s = f[i];
        for (int k = 0; k < i; k++) s -= a[(size_t)i * n + k] * u[k];
        u[i] = s / a[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = u[i];
        for (int k = i + 1; k < n; k++) s -= a[(size_t)k * n + i] * u[k];
        u[i] = s / a[(size_t)i * n + i];
    }
}

void oamg_free(oamg_h *h) {
    if (!h) return;
    for (int k = 0; k < h->nlev; k++) {
        olevel *lv = &h->lev[k];
        free(lv->rowptr); free(lv->col); free(lv->val); free(lv->t1); free(lv->t2); free(lv->t3);
        free(lv->color); free(lv->perm); free(lv->agg); free(lv->chol);
    }
    free(h->work);
    free(h);
}

/* ---------------------------------------------------------------------------------------
 * Setup (Sec. 3 and 4): aggregates on every level, Galerkin operators, colours, sweep order,
 * coarsest Cholesky factor.
 * ------------------------------------------------------------------------------------- */
/* One setup for both trees: dim 2 (quadtree, z unused) or dim 3 (octree). The octree is the
 * quadtree's construction with a third coordinate throughout: the box gains [a3, b3], a cell
 * has coordinates (t1, t2, t3) and index t1 + w t2 + w^2 t3, a parent halves all three, and
 * the colouring has m^3 colours. */
static int setup_impl(int n, const int *rowptr, const int *col, const double *val,
                      const double *x, const double *y, const double *z, const oamg_opts *opt,
                      oamg_h **out) {
    *out = NULL;
    const int dim = (opt && opt->dim == 3) ? 3 : 2;
    if (n <= 0 || !rowptr || !col || !val || !x || !y || !opt || (dim == 3 && !z))
        return OAMG_ERR_INVALID_ARG;
    if (opt->dim != 0 && opt->dim != 2 && opt->dim != 3) return OAMG_ERR_INVALID_ARG;
    if (opt->coarsest_max < 1 || opt->kcycle_n < 1 || opt->aux_level < 0 ||
        opt->aux_level > (dim == 3 ? 10 : 15) || opt->nu_pre < 0 || opt->nu_post < 0)
        return OAMG_ERR_INVALID_ARG;
    int st = check_csr(n, rowptr, col, val);
    if (st) return st;
    for (int j = 0; j < n; j++)
        if (!isfinite(x[j]) || !isfinite(y[j]) || (dim == 3 && !isfinite(z[j])))
            return OAMG_ERR_INVALID_ARG;

    oamg_h *h = (oamg_h *)xcalloc(1, sizeof(oamg_h));
    h->opt = *opt;
    if (h->opt.nu_pre == 0) h->opt.nu_pre = 1;
    if (h->opt.nu_post == 0) h->opt.nu_post = 1;
    h->dim = dim;
    /* eq. ab12: a1 = min x, b1 = max x, a2 = min y, b2 = max y (and a3, b3 for z) */
    if (opt->has_bbox) {
        memcpy(h->bbox, opt->bbox, 4 * sizeof(double));
        h->bbox[4] = opt->zbox[0];
        h->bbox[5] = opt->zbox[1];
    } else {
        double a1 = x[0], b1 = x[0], a2 = y[0], b2 = y[0];
        double a3 = dim == 3 ? z[0] : 0.0, b3 = a3;
        for (int j = 1; j < n; j++) {
            if (x[j] < a1) a1 = x[j];
            if (x[j] > b1) b1 = x[j];
            if (y[j] < a2) a2 = y[j];
            if (y[j] > b2) b2 = y[j];
            if (dim == 3) {
                if (z[j] < a3) a3 = z[j];
                if (z[j] > b3) b3 = z[j];
            }
        }
        h->bbox[0] = a1; h->bbox[1] = b1; h->bbox[2] = a2; h->bbox[3] = b2;
        h->bbox[4] = a3; h->bbox[5] = b3;
    }
    int L = opt->aux_level ? opt->aux_level
                           : (dim == 3 ? oamg_auto_level3(n) : oamg_auto_level(n));
    h->L = L;

    /* level 0: the given fine matrix */
    olevel *f = &h->lev[0];
    f->n = n;
    f->rowptr = (int *)malloc(sizeof(int) * ((size_t)n + 1));
    f->col = (int *)malloc(sizeof(int) * (size_t)rowptr[n] + 1);
    f->val = (double *)malloc(sizeof(double) * (size_t)rowptr[n] + 1);
    memcpy(f->rowptr, rowptr, sizeof(int) * ((size_t)n + 1));
    memcpy(f->col, col, sizeof(int) * (size_t)rowptr[n]);
    memcpy(f->val, val, sizeof(double) * (size_t)rowptr[n]);
    h->nlev = 1;

    /* Level L (eq. agg_L): the level-L cell of each unknown (index formula of Sec. 4.2).
     * The fine level's rows "live on" the level-L grid: t1, t2 = their cell. */
    f->cellw = 1 << L;
    f->t1 = (int *)malloc(sizeof(int) * (size_t)n);
    f->t2 = (int *)malloc(sizeof(int) * (size_t)n);
    f->t3 = dim == 3 ? (int *)malloc(sizeof(int) * (size_t)n) : NULL;
    for (int j = 0; j < n; j++) {
        f->t1[j] = cell_index_1d(x[j], h->bbox[0], h->bbox[1], L);
        f->t2[j] = cell_index_1d(y[j], h->bbox[2], h->bbox[3], L);
        if (dim == 3) f->t3[j] = cell_index_1d(z[j], h->bbox[4], h->bbox[5], L);
    }

    /* Build coarser levels while the current level is larger than coarsest_max. */
    int k = L;  /* quadtree level of the cells the next coarse level's rows occupy */
    while (h->lev[h->nlev - 1].n > opt->coarsest_max) {
        olevel *fl = &h->lev[h->nlev - 1];
        olevel *cl = &h->lev[h->nlev];
        int w = 1 << k;  /* cells per side at quadtree level k */
        /* cell of each row of fl at quadtree level k: on the fine level its level-L cell,
         * otherwise the parent (t1 >> 1, t2 >> 1) of its own cell (reading R2: Sec. 4.2
         * listing form / Sec. 4.3 restriction form, parent = floor(t2/2) 2^(k) + floor(t1/2)) */
        long long ncell = (long long)w * w * (dim == 3 ? w : 1);
        int *cid = (int *)malloc(sizeof(int) * (size_t)fl->n);
        for (int i = 0; i < fl->n; i++) {
            int c1 = (h->nlev == 1) ? fl->t1[i] : (fl->t1[i] >> 1);
            int c2 = (h->nlev == 1) ? fl->t2[i] : (fl->t2[i] >> 1);
            int c3 = dim == 3 ? ((h->nlev == 1) ? fl->t3[i] : (fl->t3[i] >> 1)) : 0;
            cid[i] = (c3 * w + c2) * w + c1;
        }
        /* aggregates = non-empty cells, numbered in ascending (lexicographic) cell index
         * (eq. agg_L / agg_k; aggregates must be non-empty, Sec. 2; reading R6) */
        int *num = (int *)malloc(sizeof(int) * (size_t)ncell);
        for (long long c = 0; c < ncell; c++) num[c] = 0;
        for (int i = 0; i < fl->n; i++) num[cid[i]] = 1;
        int nc = 0;
        for (long long c = 0; c < ncell; c++) num[c] = num[c] ? nc++ : -1;
        fl->agg = (int *)malloc(sizeof(int) * (size_t)fl->n);
        for (int i = 0; i < fl->n; i++) fl->agg[i] = num[cid[i]];
        cl->cellw = w;
        cl->t1 = (int *)malloc(sizeof(int) * (size_t)nc);
        cl->t2 = (int *)malloc(sizeof(int) * (size_t)nc);
        cl->t3 = dim == 3 ? (int *)malloc(sizeof(int) * (size_t)nc) : NULL;
        for (long long c = 0; c < ncell; c++)
            if (num[c] >= 0) {
                cl->t1[num[c]] = (int)(c % w);
                cl->t2[num[c]] = (int)((c / w) % w);
                if (dim == 3) cl->t3[num[c]] = (int)(c / ((long long)w * w));
            }
        free(num);
        free(cid);
        st = galerkin(fl, nc, cl);
        if (st) { h->nlev++; oamg_free(h); return st; }
        h->nlev++;
        if (k == 0) break;  /* one cell: cannot coarsen further */
        k--;
    }

    /* spans, colours and sweep orders */
    for (int l = 0; l < h->nlev; l++) {
        olevel *lv = &h->lev[l];
        lv->color = (int *)malloc(sizeof(int) * (size_t)lv->n);
        lv->perm = (int *)malloc(sizeof(int) * (size_t)lv->n);
        if (l == 0 && h->nlev == 1) {
            /* the fine level is itself the coarsest: no sweeps are ever made */
            lv->span = level_span(lv);
            level_colors(lv);
            for (int i = 0; i < lv->n; i++) lv->perm[i] = i;
            continue;
        }
        lv->span = level_span(lv);
        level_colors(lv);
        const int *blockkey;
        int nblock;
        int *ident = NULL;
        if (l == 0) {           /* fine level: block GS, blocks = level-L aggregates */
            blockkey = lv->agg;
            nblock = h->lev[1].n;
        } else {                /* coarse levels: point GS, block = row */
            ident = (int *)malloc(sizeof(int) * (size_t)lv->n);
            for (int i = 0; i < lv->n; i++) ident[i] = i;
            blockkey = ident;
            nblock = lv->n;
        }
        sweep_order(lv->n, lv->color, lv->m * lv->m * (dim == 3 ? lv->m : 1), blockkey, nblock,
                    lv->perm);
        free(ident);
    }
    if (!opt->no_factor) {
        st = cholesky(&h->lev[h->nlev - 1]);
        if (st) { oamg_free(h); return st; }
    }
    h->work = (double *)xcalloc((size_t)n * 2, sizeof(double));
    *out = h;
    return OAMG_OK;
}

int oamg_setup(int n, const int *rowptr, const int *col, const double *val, const double *x,
               const double *y, const oamg_opts *opt, oamg_h **out) {
    if (opt && opt->dim == 3) return OAMG_ERR_INVALID_ARG;  /* the octree needs z */
    return setup_impl(n, rowptr, col, val, x, y, NULL, opt, out);
}

/* Octree setup (dim 3): coordinates (x, y, z) of every unknown. */
int oamg_setup3(int n, const int *rowptr, const int *col, const double *val, const double *x,
                const double *y, const double *z, const oamg_opts *opt, oamg_h **out) {
    if (!opt) return OAMG_ERR_INVALID_ARG;
    oamg_opts o = *opt;
    o.dim = 3;
    return setup_impl(n, rowptr, col, val, x, y, z, &o, out);
}

/* ---------------------------------------------------------------------------------------
 * Solve-phase building blocks.
 * ------------------------------------------------------------------------------------- */
static double dot(int n, const double *a, const double *b) {
    double s = 0.0;
    for (int i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

static void spmv(const olevel *lv, const double *u, double *q) {
    for (int i = 0; i < lv->n; i++) {
        double s = 0.0;
        for (int p = lv->rowptr[i]; p < lv->rowptr[i + 1]; p++) s += lv->val[p] * u[lv->col[p]];
        q[i] = s;
    }
}

/* One Gauss-Seidel update of row i: u_i <- (f_i - sum_{j != i} a_ij u_j) / a_ii. */
static void gs_row(const olevel *lv, int i, const double *f, double *u) {
    double s = f[i], d = 0.0;
    for (int p = lv->rowptr[i]; p < lv->rowptr[i + 1]; p++) {
        int j = lv->col[p];
        if (j == i) d = lv->val[p];
        else s -= lv->val[p] * u[j];
    }
    u[i] = s / d;
}

/* Smoother (Sec. 4.5, readings R9, R10, R14): one sequential Gauss-Seidel sweep in the
 * order pi (forward, R_k) or reversed pi (backward, R_k^t), starting from the given u. */
static void smooth(const olevel *lv, int backward, const double *f, double *u) {
    if (!backward)
        for (int p = 0; p < lv->n; p++) gs_row(lv, lv->perm[p], f, u);
    else
        for (int p = lv->n - 1; p >= 0; p--) gs_row(lv, lv->perm[p], f, u);
}

static void btilde(const oamg_h *h, int l, const double *f, double *u);

/* Alg. 2, nonlinear AMLI-cycle B^_k[f] (reading R1: u2 = u1 + P B~[P^t (f - A u1)]). */
static void bhat(const oamg_h *h, int l, const double *f, double *z) {
    const olevel *lv = &h->lev[l];
    int n = lv->n;
    if (l == h->nlev - 1) {  /* B^_1 = A_1^{-1} */
        chol_solve(lv, f, z);
        return;
    }
    const olevel *cl = &h->lev[l + 1];
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *fc = (double *)xcalloc((size_t)cl->n, sizeof(double));
    double *e = (double *)xcalloc((size_t)cl->n, sizeof(double));
    /* pre-smoothing u1 = R_k f, from zero; with nu_pre > 1 the smoother R_k is nu_pre
     * forward sweeps, each started from the result of the one before (reading R10) */
    for (int i = 0; i < n; i++) z[i] = 0.0;
    for (int s = 0; s < h->opt.nu_pre; s++) smooth(lv, 0, f, z);
    /* coarse-grid correction: fc = P^t (f - A u1) (Sec. 4.3 restriction) */
    spmv(lv, z, r);
    for (int i = 0; i < n; i++) r[i] = f[i] - r[i];
    for (int i = 0; i < n; i++) fc[lv->agg[i]] += r[i];
    btilde(h, l + 1, fc, e);
    /* u2 = u1 + P e (Sec. 4.3 prolongation) */
    for (int i = 0; i < n; i++) z[i] += e[lv->agg[i]];
    /* post-smoothing: u2 + R_k^t (f - A u2) = one backward sweep started from u2 (nu_post
     * backward sweeps in a row with nu_post > 1, the adjoint of the pre-smoothing's) */
    for (int s = 0; s < h->opt.nu_post; s++) smooth(lv, 1, f, z);
    free(r);
    free(fc);
    free(e);
}

/* Alg. 1, nonlinear PCG B~_k[f] with n steps and preconditioner B^_k. Reading R11:
 * n = kcycle_n; on the coarsest level B^ is exact, so Alg. 1 stops after its first step
 * with alpha_0 = 1 and B~ = A^{-1}; the exact solve is returned directly. The loop stops
 * early if (p_i, p_i)_A <= 0 (breakdown) or the residual is exactly zero. */
static void btilde(const oamg_h *h, int l, const double *f, double *u) {
    const olevel *lv = &h->lev[l];
    int n = lv->n;
    if (l == h->nlev - 1) {
        chol_solve(lv, f, u);
        return;
    }
    int steps = h->opt.kcycle_n;
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n * steps);
    double *q = (double *)malloc(sizeof(double) * (size_t)n * steps);
    double *pAp = (double *)malloc(sizeof(double) * steps);
    for (int i = 0; i < n; i++) { u[i] = 0.0; r[i] = f[i]; }
    for (int it = 0; it < steps; it++) {
        if (it > 0 && dot(n, r, r) == 0.0) break;
        bhat(h, l, r, z);                                      /* B^_k[r_i] */
        double *pi = p + (size_t)it * n, *qi = q + (size_t)it * n;
        for (int i = 0; i < n; i++) pi[i] = z[i];
        for (int j = 0; j < it; j++) {                         /* beta_{i,j} */
            double beta = -dot(n, z, q + (size_t)j * n) / pAp[j];  /* (z, p_j)_A = (z, A p_j) */
            for (int i = 0; i < n; i++) pi[i] += beta * p[(size_t)j * n + i];
        }
        spmv(lv, pi, qi);                                      /* A_k p_i */
        pAp[it] = dot(n, pi, qi);
        if (!(pAp[it] > 0.0)) break;
        double alpha = dot(n, r, pi) / pAp[it];
        for (int i = 0; i < n; i++) u[i] += alpha * pi[i];
        for (int i = 0; i < n; i++) r[i] -= alpha * qi[i];
    }
    free(r); free(z); free(p); free(q); free(pAp);
}

/* ---------------------------------------------------------------------------------------
 * Outer solve (readings R12, R13): Alg. 1 on the finest level with preconditioner B^_fine
 * and unbounded n (flexible CG with full A-orthogonalisation), x_0 = 0, until
 * ||r||_2 / ||b||_2 <= tol on the recurrence residual, confirmed on the true residual
 * b - A x (if the true one is above tol, it replaces r and the iteration continues).
 * iters = number of B^_fine applications.
 * ------------------------------------------------------------------------------------- */
int oamg_solve(const oamg_h *h, const double *b, double tol, double *x, int *iters,
               double *relres) {
    if (!h || !b || !x || !iters || !relres || !(tol >= 0.0)) return OAMG_ERR_INVALID_ARG;
    const olevel *lv = &h->lev[0];
    int n = lv->n, maxit = h->opt.max_iters;
    for (int i = 0; i < n; i++) x[i] = 0.0;
    *iters = 0;
    double bn = sqrt(dot(n, b, b));
    if (!isfinite(bn)) return OAMG_ERR_INVALID_ARG;
    if (bn == 0.0) { *relres = 0.0; return OAMG_OK; }
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *t = (double *)malloc(sizeof(double) * (size_t)n);
    double **P = (double **)xcalloc((size_t)maxit, sizeof(double *));
    double **Q = (double **)xcalloc((size_t)maxit, sizeof(double *));
    double *pAp = (double *)xcalloc((size_t)maxit, sizeof(double));
    for (int i = 0; i < n; i++) r[i] = b[i];
    int status = OAMG_ERR_NOT_CONVERGED;
    double rel = 1.0;
    for (int it = 0; it < maxit; it++) {
        bhat(h, 0, r, z);
        double *pi = P[it] = (double *)malloc(sizeof(double) * (size_t)n);
        double *qi = Q[it] = (double *)malloc(sizeof(double) * (size_t)n);
        for (int i = 0; i < n; i++) pi[i] = z[i];
        for (int j = 0; j < it; j++) {
            double beta = -dot(n, z, Q[j]) / pAp[j];
            for (int i = 0; i < n; i++) pi[i] += beta * P[j][i];
        }
        spmv(lv, pi, qi);
        pAp[it] = dot(n, pi, qi);
        *iters = it + 1;
        if (!(pAp[it] > 0.0) || !isfinite(pAp[it])) { status = OAMG_ERR_BREAKDOWN; break; }
        double alpha = dot(n, r, pi) / pAp[it];
        for (int i = 0; i < n; i++) x[i] += alpha * pi[i];
        for (int i = 0; i < n; i++) r[i] -= alpha * qi[i];
        rel = sqrt(dot(n, r, r)) / bn;
        if (!isfinite(rel)) { status = OAMG_ERR_BREAKDOWN; break; }
        if (rel <= tol) {
            spmv(lv, x, t);
            for (int i = 0; i < n; i++) t[i] = b[i] - t[i];
            rel = sqrt(dot(n, t, t)) / bn;
            if (rel <= tol) { status = OAMG_OK; break; }
            for (int i = 0; i < n; i++) r[i] = t[i];
        }
    }
    if (status != OAMG_OK) {  /* report the true residual of the returned x */
        spmv(lv, x, t);
        for (int i = 0; i < n; i++) t[i] = b[i] - t[i];
        rel = sqrt(dot(n, t, t)) / bn;
    }
    *relres = rel;
    for (int j = 0; j < maxit; j++) { free(P[j]); free(Q[j]); }
    free(P); free(Q); free(pAp); free(r); free(z); free(t);
    return status;
}

/* ---------------------------------------------------------------------------------------
 * Inspection and building-block entry points (used by the pins and parity tests).
 * ------------------------------------------------------------------------------------- */
int oamg_num_levels(const oamg_h *h) { return h->nlev; }
int oamg_aux_level(const oamg_h *h) { return h->L; }
void oamg_get_bbox(const oamg_h *h, double *bb) { memcpy(bb, h->bbox, 4 * sizeof(double)); }
void oamg_get_zbox(const oamg_h *h, double *bb) { memcpy(bb, h->bbox + 4, 2 * sizeof(double)); }
int oamg_dim(const oamg_h *h) { return h->dim; }

/* third cell coordinate of every row of level l (octree) */
int oamg_level_t3(const oamg_h *h, int l, int *t3) {
    if (l < 0 || l >= h->nlev || !h->lev[l].t3) return OAMG_ERR_INVALID_ARG;
    memcpy(t3, h->lev[l].t3, sizeof(int) * (size_t)h->lev[l].n);
    return OAMG_OK;
}

int oamg_level_info(const oamg_h *h, int l, int *info /* n, nnz, cellw, span, m */) {
    if (l < 0 || l >= h->nlev) return OAMG_ERR_INVALID_ARG;
    const olevel *lv = &h->lev[l];
    info[0] = lv->n;
    info[1] = lv->rowptr[lv->n];
    info[2] = lv->cellw;
    info[3] = lv->span;
    info[4] = lv->m;
    return OAMG_OK;
}

int oamg_level_get(const oamg_h *h, int l, int *rowptr, int *col, double *val, int *t1,
                   int *t2, int *color, int *perm, int *agg) {
    if (l < 0 || l >= h->nlev) return OAMG_ERR_INVALID_ARG;
    const olevel *lv = &h->lev[l];
    int n = lv->n, nnz = lv->rowptr[n];
    if (rowptr) memcpy(rowptr, lv->rowptr, sizeof(int) * ((size_t)n + 1));
    if (col) memcpy(col, lv->col, sizeof(int) * (size_t)nnz);
    if (val) memcpy(val, lv->val, sizeof(double) * (size_t)nnz);
    if (t1) memcpy(t1, lv->t1, sizeof(int) * (size_t)n);
    if (t2) memcpy(t2, lv->t2, sizeof(int) * (size_t)n);
    if (color) memcpy(color, lv->color, sizeof(int) * (size_t)n);
    if (perm) memcpy(perm, lv->perm, sizeof(int) * (size_t)n);
    if (agg && lv->agg) memcpy(agg, lv->agg, sizeof(int) * (size_t)n);
    return OAMG_OK;
}

int oamg_smooth(const oamg_h *h, int l, int backward, const double *f, double *u) {
    if (l < 0 || l >= h->nlev) return OAMG_ERR_INVALID_ARG;
    smooth(&h->lev[l], backward, f, u);
    return OAMG_OK;
}

int oamg_bhat(const oamg_h *h, int l, const double *f, double *z) {
    if (l < 0 || l >= h->nlev) return OAMG_ERR_INVALID_ARG;
    bhat(h, l, f, z);
    return OAMG_OK;
}

int oamg_btilde(const oamg_h *h, int l, const double *f, double *u) {
    if (l < 0 || l >= h->nlev) return OAMG_ERR_INVALID_ARG;
    btilde(h, l, f, u);
    return OAMG_OK;
}

/* Level-L cell indices of arbitrary points with a given box (Sec. 4.2 index formula). */
void oamg_bin(int n, const double *x, const double *y, const double *bbox, int L, int *cell) {
    for (int j = 0; j < n; j++)
        cell[j] = cell_index_1d(y[j], bbox[2], bbox[3], L) * (1 << L) +
                  cell_index_1d(x[j], bbox[0], bbox[1], L);
}

/* Level-L octree cell indices t1 + 2^L t2 + 4^L t3 of arbitrary points (box a1,b1,a2,b2,a3,b3). */
void oamg_bin3(int n, const double *x, const double *y, const double *z, const double *bbox,
               int L, int *cell) {
    for (int j = 0; j < n; j++)
        cell[j] = (cell_index_1d(z[j], bbox[4], bbox[5], L) * (1 << L) +
                   cell_index_1d(y[j], bbox[2], bbox[3], L)) * (1 << L) +
                  cell_index_1d(x[j], bbox[0], bbox[1], L);
}

/*
 * lair_oracle.c -- plain, slow, single-threaded CPU oracle for lAIR
 * (Manteuffel, Ruge, Southworth: "Nonsymmetric AMG based on local approximate
 * ideal restriction").
 *
 * TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the CPU
 * baseline of the benchmark load this file. It shares no code, header, table or
 * constant with the CUDA library; the two meet only in the seeded inputs.
 *
 * Everything is FP64 unless a function says otherwise. The steps follow the
 * paper's order and notation:
 *   strength of connection ........ Sec. 4, definition of N_i (hard minimum)
 *   C/F splitting .................. Sec. 4 (classical first pass, no second pass),
 *                                    also run independently in index blocks; PMIS
 *   restriction neighbourhoods ..... Sec. 3.1 (distance one to four, F-F-C only, Sec. 4)
 *   local systems .................. Sec. 3.1, Eq. (3.1) johnair and Eq. (3.2) system,
 *                                    least squares when singular (Sec. 3.1 footnote)
 *   R = [Z I], P = [W; I] .......... Sec. 2.1, Eq. (2.2)
 *   interpolation .................. one-point (Sec. 4) and approximate ideal
 *                                    interpolation W ~ -A_ff^{-1} A_fc (Eq. (2.6))
 *   coarse operator K = R A P ...... Sec. 2.1
 *   lumping ........................ Sec. 3.3
 *   V-cycle with post F-F-C Jacobi . Sec. 4, Eq. (2.4)
 *   GMRES acceleration ............. Sec. 4 (here flexible GMRES, FP64)
 *   Neumann restriction (nAIR) ..... Sec. 3.2, truncated Neumann series of A_ff^{-1}
 *   nodal (block) hierarchy ........ Sec. 3.1 (k x k blocks), Sec. 4.2.1 approach (iii):
 *                                    strength, splitting, R and P by block; block Jacobi
 *   refresh for new values ......... backward Euler steps I + dt S (Sec. 4.1.1):
 *                                    structure kept, every value recomputed
 *
 * Points the paper leaves open are fixed here in one documented way (tie rules,
 * singular threshold, arithmetic order). Floating-point operations that decide
 * integer structure on coarse levels are written with explicit fma() and a fixed
 * order, so that any implementation that follows the same definitions obtains
 * identical bits. Build with -ffp-contract=off so the compiler adds no fusions.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Loops whose iterations are independent (one row, one C point or one index block
 * each, writing only their own outputs) may run on several host threads when the
 * file is built with OpenMP; every result is the same bits for any thread count,
 * since no floating-point sum crosses iterations. Reductions, the classical first
 * pass over the whole graph, PMIS and the Krylov loops stay sequential. */
#ifdef _OPENMP
#define ORA_PARALLEL_FOR _Pragma("omp parallel for schedule(dynamic, 64)")
#define ORA_PARALLEL_FOR_EACH _Pragma("omp parallel for schedule(dynamic, 1)")
#define ORA_PARALLEL _Pragma("omp parallel")
#define ORA_FOR _Pragma("omp for schedule(dynamic, 64)")
#else
#define ORA_PARALLEL_FOR
#define ORA_PARALLEL_FOR_EACH
#define ORA_PARALLEL
#define ORA_FOR
#endif

void ora_set_threads(int t) {
#ifdef _OPENMP
    omp_set_num_threads(t > 0 ? t : omp_get_num_procs());
#else
    (void)t;
#endif
}

int ora_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#define ORA_OK 0
#define ORA_ERR_ARG 1
#define ORA_ERR_ZERO_DIAG 5
#define ORA_ERR_STALLED 6
#define ORA_ERR_NOT_CONVERGED 7
#define ORA_ERR_NAN 8
#define ORA_ERR_OOM 9

#define CF_F 0
#define CF_C 1
#define CF_U (-1)

/* ------------------------------------------------------------------------- */
/* options (mirrors the public option set; defined independently)            */
/* ------------------------------------------------------------------------- */
typedef struct {
    int cf_mode;           /* 0 RS, 1 PMIS, 2 USER (level 0 only), 3 AUTO (first pass in blocks of rs_block) */
    const int8_t *cf_user; /* level-0 splitting for USER mode (1 = C, 0 = F) */
    int distance;          /* 1 to 4 */
    double theta;          /* strength threshold for R/P neighbourhoods */
    double theta_cf;       /* strength threshold for the C/F splitting */
    int strength_abs;      /* 1: |a_ij| >= theta max|a_ik| instead of -a_ij >= ... */
    int interp;            /* 0 approximate ideal (lAIP), 1 one-point */
    int relax;             /* 0 F-F-C, 1 F-C-F, 2 F-F */
    double lump_tol;       /* theta_D; 0 disables */
    int lump_level0;       /* also lump the finest operator */
    int prec;              /* 0 FP64, 1 FP32 local solves and FP32 cycle */
    int coarse_max;        /* direct solve when n <= coarse_max */
    int max_levels;
    int block_size;        /* >1: scale by the inverse block diagonal first */
    int rs_block;          /* AUTO: index-block size of the blocked first pass */
    uint64_t pmis_seed;
    const int64_t *seg;    /* batched systems: nseg + 1 offsets of the independent systems on level 0 */
    int nseg;
    int restriction;       /* 0 lAIR (Sec. 3.1), 1 Neumann nAIR of degree distance - 1 (Sec. 3.2) */
    int nodal;             /* > 1: nodal hierarchy on k x k blocks of that size (Sec. 3.1, Sec. 4.2.1 (iii)) */
} ora_opts;

/* ------------------------------------------------------------------------- */
/* CSR helpers                                                               */
/* ------------------------------------------------------------------------- */
typedef struct {
    int64_t nr, nc;
    int64_t *rp;
    int32_t *col;
    double *val;
} ocsr;

static void csr_free(ocsr *a) {
    free(a->rp); free(a->col); free(a->val);
    memset(a, 0, sizeof(*a));
}

static int csr_alloc(ocsr *a, int64_t nr, int64_t nc, int64_t nnz) {
    a->nr = nr; a->nc = nc;
    a->rp = (int64_t *)calloc((size_t)nr + 1, sizeof(int64_t));
    a->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    a->val = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    return (a->rp && a->col && a->val) ? ORA_OK : ORA_ERR_OOM;
}

/* plain transpose; entries of each output row come out in ascending column order */
static int csr_transpose(const ocsr *a, ocsr *t) {
    int64_t nnz = a->rp[a->nr];
    if (csr_alloc(t, a->nc, a->nr, nnz)) return ORA_ERR_OOM;
    for (int64_t k = 0; k < nnz; ++k) t->rp[a->col[k] + 1]++;
    for (int64_t i = 0; i < a->nc; ++i) t->rp[i + 1] += t->rp[i];
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)(a->nc + 1));
    memcpy(pos, t->rp, sizeof(int64_t) * (size_t)(a->nc + 1));
    for (int64_t i = 0; i < a->nr; ++i)
        for (int64_t k = a->rp[i]; k < a->rp[i + 1]; ++k) {
            int64_t d = pos[a->col[k]]++;
            t->col[d] = (int32_t)i;
            t->val[d] = a->val[k];
        }
    free(pos);
    return ORA_OK;
}

/* value of a_ij or 0; columns of a row are ascending */
static int find_entry(const ocsr *a, int64_t i, int64_t j, double *v) {
    int64_t lo = a->rp[i], hi = a->rp[i + 1] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (a->col[mid] == j) { *v = a->val[mid]; return 1; }
        if (a->col[mid] < j) lo = mid + 1; else hi = mid - 1;
    }
    *v = 0.0;
    return 0;
}

static int64_t find_pos(const int32_t *list, int64_t len, int64_t key) {
    int64_t lo = 0, hi = len - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (list[mid] == key) return mid;
        if (list[mid] < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* ------------------------------------------------------------------------- */
/* Strength of connection (Sec. 4): j in N_i iff j != i and                   */
/*   -a_ij >= theta * max_{k != i} |a_ik|   (signed), or                       */
/*   |a_ij| >= theta * max_{k != i} |a_ik|  (abs mode).                        */
/* Reading: an empty row maximum (m_i = 0) gives no strong connections, and an */
/* explicitly stored zero is never strong. theta*m_i is one rounded multiply.  */
/* ------------------------------------------------------------------------- */
void ora_strength(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                  double theta, int absmode, uint8_t *strong) {
    ORA_PARALLEL_FOR
    for (int64_t i = 0; i < n; ++i) {
        double m = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
            if (col[k] != i && fabs(val[k]) > m) m = fabs(val[k]);
        double thr = theta * m;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            double a = val[k];
            int s = 0;
            if (col[k] != i && m > 0.0 && a != 0.0)
                s = absmode ? (fabs(a) >= thr) : (-a >= thr);
            strong[k] = (uint8_t)s;
        }
    }
}

/* S as a pattern-only CSR (val unused = NULL) */
typedef struct { int64_t n; int64_t *rp; int32_t *col; } ograph;

static void graph_free(ograph *g) { free(g->rp); free(g->col); memset(g, 0, sizeof(*g)); }

static int graph_from_mask(int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *mask, ograph *g) {
    g->n = n;
    g->rp = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t cnt = 0;
    for (int64_t k = 0; k < rp[n]; ++k) cnt += mask[k];
    g->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cnt > 0 ? cnt : 1));
    if (!g->rp || !g->col) return ORA_ERR_OOM;
    int64_t p = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
            if (mask[k]) g->col[p++] = col[k];
        g->rp[i + 1] = p;
    }
    return ORA_OK;
}

static int graph_transpose(const ograph *g, ograph *t) {
    int64_t n = g->n, nnz = g->rp[n];
    t->n = n;
    t->rp = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    t->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!t->rp || !t->col) return ORA_ERR_OOM;
    for (int64_t k = 0; k < nnz; ++k) t->rp[g->col[k] + 1]++;
    for (int64_t i = 0; i < n; ++i) t->rp[i + 1] += t->rp[i];
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    memcpy(pos, t->rp, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = g->rp[i]; k < g->rp[i + 1]; ++k) t->col[pos[g->col[k]]++] = (int32_t)i;
    free(pos);
    return ORA_OK;
}

/* ------------------------------------------------------------------------- */
/* Classical (Ruge-Stueben) first pass, no second pass (Sec. 4).              */
/* S_i = points i strongly depends on, ST_i = points strongly depending on i.  */
/* lambda_i = |ST_i|. Points with S_i and ST_i both empty become F first.      */
/* Repeat: the undecided point with the largest lambda (ties: smallest index)  */
/* becomes C; every undecided j in ST_i becomes F and, for each such j, every  */
/* undecided k in S_j gets lambda_k += 1; then every undecided k in S_i gets   */
/* lambda_k -= 1. A binary heap with lazy deletion finds the maximum.          */
/* ------------------------------------------------------------------------- */
typedef struct { int64_t lam; int64_t idx; } heapent;

static int heap_less(heapent a, heapent b) { /* a has lower priority than b */
    if (a.lam != b.lam) return a.lam < b.lam;
    return a.idx > b.idx;
}

typedef struct { heapent *a; int64_t len, cap; } oheap;

static void heap_push(oheap *h, heapent e) {
    if (h->len == h->cap) {
        h->cap = h->cap ? 2 * h->cap : 1024;
        h->a = (heapent *)realloc(h->a, sizeof(heapent) * (size_t)h->cap);
    }
    int64_t i = h->len++;
    h->a[i] = e;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!heap_less(h->a[p], h->a[i])) break;
        heapent t = h->a[p]; h->a[p] = h->a[i]; h->a[i] = t;
        i = p;
    }
}

static heapent heap_pop(oheap *h) {
    heapent top = h->a[0];
    h->a[0] = h->a[--h->len];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < h->len && heap_less(h->a[m], h->a[l])) m = l;
        if (r < h->len && heap_less(h->a[m], h->a[r])) m = r;
        if (m == i) break;
        heapent t = h->a[m]; h->a[m] = h->a[i]; h->a[i] = t;
        i = m;
    }
    return top;
}

/* The first pass restricted to the index block [b0, b1): lambda and the updates only
 * count strong connections with both ends in the block; points without any strong
 * connection in the whole graph start as F. With one block covering all points this is
 * the classical first pass above. */
static void cf_rs_block(const ograph *S, const ograph *ST, int64_t b0, int64_t b1, int8_t *cf, int64_t *lam) {
    oheap h = {0};
    for (int64_t i = b0; i < b1; ++i) {
        int64_t l = 0;
        for (int64_t p = ST->rp[i]; p < ST->rp[i + 1]; ++p) l += (ST->col[p] >= b0 && ST->col[p] < b1);
        lam[i] = l;
        int isolated = (S->rp[i + 1] == S->rp[i]) && (ST->rp[i + 1] == ST->rp[i]);
        cf[i] = isolated ? CF_F : CF_U;
        if (!isolated) heap_push(&h, (heapent){lam[i], i});
    }
    while (h.len > 0) {
        heapent e = heap_pop(&h);
        int64_t i = e.idx;
        if (cf[i] != CF_U || lam[i] != e.lam) continue;
        cf[i] = CF_C;
        for (int64_t p = ST->rp[i]; p < ST->rp[i + 1]; ++p) {
            int64_t j = ST->col[p];
            if (j < b0 || j >= b1 || cf[j] != CF_U) continue;
            cf[j] = CF_F;
            for (int64_t q = S->rp[j]; q < S->rp[j + 1]; ++q) {
                int64_t k = S->col[q];
                if (k >= b0 && k < b1 && cf[k] == CF_U) { lam[k] += 1; heap_push(&h, (heapent){lam[k], k}); }
            }
        }
        for (int64_t p = S->rp[i]; p < S->rp[i + 1]; ++p) {
            int64_t k = S->col[p];
            if (k >= b0 && k < b1 && cf[k] == CF_U) { lam[k] -= 1; heap_push(&h, (heapent){lam[k], k}); }
        }
    }
    free(h.a);
}

/* blocks of at most B points; with system offsets seg (nseg + 1 entries) no block spans two systems */
static void cf_rs_blocked_seg(const ograph *S, const ograph *ST, int64_t B, const int64_t *seg, int nseg, int8_t *cf) {
    int64_t n = S->n;
    int64_t *lam = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    /* the blocks in index order (each block touches only its own points, so they may run in any order) */
    int64_t nb = 0, cap = 16;
    int64_t *b0s = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap), *b1s = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    int nq = (seg && nseg > 0) ? nseg : 1;
    for (int q = 0; q < nq; ++q) {
        int64_t lo = (seg && nseg > 0) ? seg[q] : 0, hi = (seg && nseg > 0) ? seg[q + 1] : n;
        for (int64_t b0 = lo; b0 < hi; b0 += B) {
            if (nb == cap) {
                cap *= 2;
                b0s = (int64_t *)realloc(b0s, sizeof(int64_t) * (size_t)cap);
                b1s = (int64_t *)realloc(b1s, sizeof(int64_t) * (size_t)cap);
            }
            b0s[nb] = b0;
            b1s[nb] = b0 + B < hi ? b0 + B : hi;
            nb++;
        }
    }
    ORA_PARALLEL_FOR_EACH
    for (int64_t t = 0; t < nb; ++t) cf_rs_block(S, ST, b0s[t], b1s[t], cf, lam);
    free(b0s); free(b1s);
    free(lam);
}

static void cf_rs_blocked(const ograph *S, const ograph *ST, int64_t B, int8_t *cf) {
    cf_rs_blocked_seg(S, ST, B, NULL, 0, cf);
}

static void cf_rs(const ograph *S, const ograph *ST, int8_t *cf) {
    int64_t n = S->n;
    int64_t *lam = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    oheap h = {0};
    for (int64_t i = 0; i < n; ++i) {
        lam[i] = ST->rp[i + 1] - ST->rp[i];
        int isolated = (S->rp[i + 1] == S->rp[i]) && (lam[i] == 0);
        cf[i] = isolated ? CF_F : CF_U;
        if (!isolated) heap_push(&h, (heapent){lam[i], i});
    }
    while (h.len > 0) {
        heapent e = heap_pop(&h);
        int64_t i = e.idx;
        if (cf[i] != CF_U || lam[i] != e.lam) continue;   /* stale entry */
        cf[i] = CF_C;
        for (int64_t p = ST->rp[i]; p < ST->rp[i + 1]; ++p) {
            int64_t j = ST->col[p];
            if (cf[j] != CF_U) continue;
            cf[j] = CF_F;
            for (int64_t q = S->rp[j]; q < S->rp[j + 1]; ++q) {
                int64_t k = S->col[q];
                if (cf[k] == CF_U) { lam[k] += 1; heap_push(&h, (heapent){lam[k], k}); }
            }
        }
        for (int64_t p = S->rp[i]; p < S->rp[i + 1]; ++p) {
            int64_t k = S->col[p];
            if (cf[k] == CF_U) { lam[k] -= 1; heap_push(&h, (heapent){lam[k], k}); }
        }
    }
    free(h.a);
    free(lam);
}

/* ------------------------------------------------------------------------- */
/* PMIS: parallel maximal independent set splitting with hashed weights.      */
/* w_i = |ST_i| + u_i, u_i = (splitmix64((seed << 32) ^ i) >> 11) * 2^-53.     */
/* Points with |ST_i| = 0 start as F. Each round, every undecided i whose      */
/* (w_i, -i) beats that of every undecided neighbour in S_i u ST_i becomes C;  */
/* then every undecided j in ST_i of a new C point i becomes F.                */
/* splitmix64 is Vigna's published 64-bit mixer.                               */
/* ------------------------------------------------------------------------- */
static uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

double ora_pmis_weight(int64_t lam, int64_t i, uint64_t seed) {
    double u = (double)(splitmix64((seed << 32) ^ (uint64_t)i) >> 11) * 0x1.0p-53;
    return (double)lam + u;
}

static int beats(double wi, int64_t i, double wj, int64_t j) {
    return (wi > wj) || (wi == wj && i < j);
}

static void cf_pmis(const ograph *S, const ograph *ST, uint64_t seed, int8_t *cf) {
    int64_t n = S->n;
    double *w = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int8_t *newc = (int8_t *)malloc((size_t)(n > 0 ? n : 1));
    int64_t undecided = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t lam = ST->rp[i + 1] - ST->rp[i];
        w[i] = ora_pmis_weight(lam, i, seed);
        cf[i] = (lam == 0) ? CF_F : CF_U;
        undecided += (cf[i] == CF_U);
    }
    while (undecided > 0) {
        for (int64_t i = 0; i < n; ++i) {
            newc[i] = 0;
            if (cf[i] != CF_U) continue;
            int best = 1;
            for (int64_t p = S->rp[i]; p < S->rp[i + 1] && best; ++p) {
                int64_t j = S->col[p];
                if (cf[j] == CF_U && !beats(w[i], i, w[j], j)) best = 0;
            }
            for (int64_t p = ST->rp[i]; p < ST->rp[i + 1] && best; ++p) {
                int64_t j = ST->col[p];
                if (cf[j] == CF_U && !beats(w[i], i, w[j], j)) best = 0;
            }
            newc[i] = (int8_t)best;
        }
        for (int64_t i = 0; i < n; ++i)
            if (newc[i]) { cf[i] = CF_C; undecided--; }
        for (int64_t i = 0; i < n; ++i) {
            if (!newc[i]) continue;
            for (int64_t p = ST->rp[i]; p < ST->rp[i + 1]; ++p) {
                int64_t j = ST->col[p];
                if (cf[j] == CF_U) { cf[j] = CF_F; undecided--; }
            }
        }
    }
    free(w);
    free(newc);
}

/* ------------------------------------------------------------------------- */
/* Neighbourhoods (Sec. 3.1, Sec. 4). For C-point i and graph G:              */
/*   distance 1: G_i restricted to F points;                                  */
/*   distance d > 1: the distance d-1 set plus G_j restricted to F for every   */
/*   j in that set (strong paths i -> F -> ... -> F, F-F-C only).             */
/* Result sorted ascending, no duplicates. Output as CSR over C points.        */
/* ------------------------------------------------------------------------- */
static int64_t sort_unique(int32_t *t, int64_t m) {
    qsort(t, (size_t)m, sizeof(int32_t), cmp_i32);
    int64_t u = 0;
    for (int64_t a = 0; a < m; ++a)
        if (u == 0 || t[u - 1] != t[a]) t[u++] = t[a];
    return u;
}

/* the set of C point i in tmp (grown as needed); returns its size */
static int64_t neighbourhood_of(const ograph *G, const int8_t *cf, int distance, int64_t i, int32_t **tmp_,
                                int64_t *tcap_, int32_t **nxt_, int64_t *ncap_) {
    int32_t *tmp = *tmp_, *nxt = *nxt_;
    int64_t tcap = *tcap_, ncap = *ncap_;
    /* distance 1 */
    int64_t need = G->rp[i + 1] - G->rp[i];
    if (need > tcap) { tcap = need + 16; tmp = (int32_t *)realloc(tmp, sizeof(int32_t) * (size_t)tcap); }
    int64_t t = 0;
    for (int64_t p = G->rp[i]; p < G->rp[i + 1]; ++p)
        if (cf[G->col[p]] == CF_F) tmp[t++] = G->col[p];
    t = sort_unique(tmp, t);
    /* each further distance: the set and the F points of G_j for every j in it */
    for (int d = 2; d <= distance; ++d) {
        need = t;
        for (int64_t a = 0; a < t; ++a) need += G->rp[tmp[a] + 1] - G->rp[tmp[a]];
        if (need > ncap) { ncap = need + 16; nxt = (int32_t *)realloc(nxt, sizeof(int32_t) * (size_t)ncap); }
        int64_t m = 0;
        for (int64_t a = 0; a < t; ++a) {
            int64_t j = tmp[a];
            nxt[m++] = (int32_t)j;
            for (int64_t q = G->rp[j]; q < G->rp[j + 1]; ++q) {
                int64_t k = G->col[q];
                if (cf[k] == CF_F && k != i) nxt[m++] = (int32_t)k;
            }
        }
        m = sort_unique(nxt, m);
        if (m > tcap) { tcap = m + 16; tmp = (int32_t *)realloc(tmp, sizeof(int32_t) * (size_t)tcap); }
        memcpy(tmp, nxt, sizeof(int32_t) * (size_t)m);
        t = m;
    }
    *tmp_ = tmp; *nxt_ = nxt; *tcap_ = tcap; *ncap_ = ncap;
    return t;
}

static int build_neighbourhoods(const ograph *G, const int8_t *cf, int distance,
                                int64_t nc, const int64_t *cpts, int64_t **out_rp, int32_t **out_col) {
    int64_t *rp = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    int32_t **rows = (int32_t **)malloc(sizeof(int32_t *) * (size_t)(nc > 0 ? nc : 1));
    ORA_PARALLEL
    {
        int32_t *tmp = NULL, *nxt = NULL;
        int64_t tcap = 0, ncap = 0;
        ORA_FOR
        for (int64_t c = 0; c < nc; ++c) {
            int64_t t = neighbourhood_of(G, cf, distance, cpts[c], &tmp, &tcap, &nxt, &ncap);
            rows[c] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(t > 0 ? t : 1));
            memcpy(rows[c], tmp, sizeof(int32_t) * (size_t)t);
            rp[c + 1] = t;
        }
        free(tmp);
        free(nxt);
    }
    for (int64_t c = 0; c < nc; ++c) rp[c + 1] += rp[c];
    int32_t *col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(rp[nc] > 0 ? rp[nc] : 1));
    for (int64_t c = 0; c < nc; ++c) {
        memcpy(col + rp[c], rows[c], sizeof(int32_t) * (size_t)(rp[c + 1] - rp[c]));
        free(rows[c]);
    }
    free(rows);
    *out_rp = rp;
    *out_col = col;
    return ORA_OK;
}

/* ------------------------------------------------------------------------- */
/* Plain dot product of two strided vectors: terms added in ascending index    */
/* with fma, starting from 0. Used by the least-squares branch.                */
/* ------------------------------------------------------------------------- */
static double sdot(const double *x, int64_t sx, const double *y, int64_t sy, int64_t s) {
    double acc = 0.0;
    for (int64_t r = 0; r < s; ++r) acc = fma(x[r * sx], y[r * sy], acc);
    return acc;
}

static float sdotf(const float *x, int64_t sx, const float *y, int64_t sy, int64_t s) {
    float acc = 0.0f;
    for (int64_t r = 0; r < s; ++r) acc = fmaf(x[r * sx], y[r * sy], acc);
    return acc;
}

/* ------------------------------------------------------------------------- */
/* Dense local solve M z = rhs, M row-major s x s (overwritten).              */
/* LU with partial pivoting: pivot = largest |M[r][k]|, r >= k, ties -> the    */
/* smallest r. Elimination: l = M[r][k] / M[k][k]; M[r][c] = fma(-l, M[k][c],  */
/* M[r][c]) for c > k; rhs[r] = fma(-l, rhs[k], rhs[r]). Back substitution by  */
/* columns, c = s-1 .. 0: z[c] = rhs[c] / M[c][c]; rhs[r] = fma(-M[r][c], z[c],*/
/* rhs[r]) for r < c.                                                          */
/* Singular reading: if some pivot |M[k][k]| <= s * eps * max|M| (original M)  */
/* the minimum-norm least-squares solution is used instead (one-sided Jacobi    */
/* SVD, Hestenes' method). Returns 0 for LU, 1 for least squares.              */
/* ------------------------------------------------------------------------- */
#define LS_MAX_SWEEPS 60

static void jacobi_ls(int64_t s, const double *M0, const double *rhs0, double *z) {
    double *B = (double *)malloc(sizeof(double) * (size_t)(s * s));
    double *V = (double *)malloc(sizeof(double) * (size_t)(s * s));
    double *sig = (double *)malloc(sizeof(double) * (size_t)s);
    memcpy(B, M0, sizeof(double) * (size_t)(s * s));
    for (int64_t r = 0; r < s; ++r)
        for (int64_t c = 0; c < s; ++c) V[r * s + c] = (r == c) ? 1.0 : 0.0;
    const double tol = DBL_EPSILON * (double)s;
    for (int sweep = 0; sweep < LS_MAX_SWEEPS; ++sweep) {
        int rotated = 0;
        for (int64_t p = 0; p < s - 1; ++p)
            for (int64_t q = p + 1; q < s; ++q) {
                double alpha = sdot(B + p, s, B + p, s, s);
                double beta = sdot(B + q, s, B + q, s, s);
                double gamma = sdot(B + p, s, B + q, s, s);
                if (gamma == 0.0 || fabs(gamma) <= tol * sqrt(alpha * beta)) continue;
                rotated = 1;
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
                double c = 1.0 / sqrt(fma(t, t, 1.0));
                double sn = c * t;
                for (int64_t r = 0; r < s; ++r) {
                    double bp = B[r * s + p], bq = B[r * s + q];
                    B[r * s + p] = fma(c, bp, -(sn * bq));
                    B[r * s + q] = fma(sn, bp, c * bq);
                    double vp = V[r * s + p], vq = V[r * s + q];
                    V[r * s + p] = fma(c, vp, -(sn * vq));
                    V[r * s + q] = fma(sn, vp, c * vq);
                }
            }
        if (!rotated) break;
    }
    double smax = 0.0;
    for (int64_t j = 0; j < s; ++j) {
        sig[j] = sqrt(sdot(B + j, s, B + j, s, s));
        if (sig[j] > smax) smax = sig[j];
    }
    double cut = ((double)s * DBL_EPSILON) * smax;
    for (int64_t r = 0; r < s; ++r) z[r] = 0.0;
    for (int64_t j = 0; j < s; ++j) {
        if (!(sig[j] > cut)) continue;
        double coef = (sdot(B + j, s, rhs0, 1, s) / sig[j]) / sig[j];
        for (int64_t r = 0; r < s; ++r) z[r] = fma(V[r * s + j], coef, z[r]);
    }
    free(B); free(V); free(sig);
}

int ora_local_solve(int64_t s, double *M, double *rhs, double *z) {
    if (s == 0) return 0;
    double *M0 = (double *)malloc(sizeof(double) * (size_t)(s * s));
    double *r0 = (double *)malloc(sizeof(double) * (size_t)s);
    memcpy(M0, M, sizeof(double) * (size_t)(s * s));
    memcpy(r0, rhs, sizeof(double) * (size_t)s);
    double mx = 0.0;
    for (int64_t k = 0; k < s * s; ++k) if (fabs(M[k]) > mx) mx = fabs(M[k]);
    double thr = ((double)s * DBL_EPSILON) * mx;
    int singular = (mx == 0.0);
    for (int64_t k = 0; k < s && !singular; ++k) {
        int64_t piv = k;
        double best = fabs(M[k * s + k]);
        for (int64_t r = k + 1; r < s; ++r)
            if (fabs(M[r * s + k]) > best) { best = fabs(M[r * s + k]); piv = r; }
        if (best <= thr) { singular = 1; break; }
        if (piv != k) {
            for (int64_t c = 0; c < s; ++c) { double t = M[k * s + c]; M[k * s + c] = M[piv * s + c]; M[piv * s + c] = t; }
            double t = rhs[k]; rhs[k] = rhs[piv]; rhs[piv] = t;
        }
        for (int64_t r = k + 1; r < s; ++r) {
            double l = M[r * s + k] / M[k * s + k];
            for (int64_t c = k + 1; c < s; ++c) M[r * s + c] = fma(-l, M[k * s + c], M[r * s + c]);
            rhs[r] = fma(-l, rhs[k], rhs[r]);
        }
    }
    if (!singular) {
        for (int64_t c = s - 1; c >= 0; --c) {
            z[c] = rhs[c] / M[c * s + c];
            for (int64_t r = 0; r < c; ++r) rhs[r] = fma(-M[r * s + c], z[c], rhs[r]);
        }
    } else {
        jacobi_ls(s, M0, r0, z);
    }
    free(M0); free(r0);
    return singular;
}

/* FP32 version: identical steps in single precision (eps = FLT_EPSILON). */
static void jacobi_lsf(int64_t s, const float *M0, const float *rhs0, float *z) {
    float *B = (float *)malloc(sizeof(float) * (size_t)(s * s));
    float *V = (float *)malloc(sizeof(float) * (size_t)(s * s));
    float *sig = (float *)malloc(sizeof(float) * (size_t)s);
    memcpy(B, M0, sizeof(float) * (size_t)(s * s));
    for (int64_t r = 0; r < s; ++r)
        for (int64_t c = 0; c < s; ++c) V[r * s + c] = (r == c) ? 1.0f : 0.0f;
    const float tol = FLT_EPSILON * (float)s;
    for (int sweep = 0; sweep < LS_MAX_SWEEPS; ++sweep) {
        int rotated = 0;
        for (int64_t p = 0; p < s - 1; ++p)
            for (int64_t q = p + 1; q < s; ++q) {
                float alpha = sdotf(B + p, s, B + p, s, s);
                float beta = sdotf(B + q, s, B + q, s, s);
                float gamma = sdotf(B + p, s, B + q, s, s);
                if (gamma == 0.0f || fabsf(gamma) <= tol * sqrtf(alpha * beta)) continue;
                rotated = 1;
                float zeta = (beta - alpha) / (2.0f * gamma);
                float t = (zeta >= 0.0f ? 1.0f : -1.0f) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.0f)));
                float c = 1.0f / sqrtf(fmaf(t, t, 1.0f));
                float sn = c * t;
                for (int64_t r = 0; r < s; ++r) {
                    float bp = B[r * s + p], bq = B[r * s + q];
                    B[r * s + p] = fmaf(c, bp, -(sn * bq));
                    B[r * s + q] = fmaf(sn, bp, c * bq);
                    float vp = V[r * s + p], vq = V[r * s + q];
                    V[r * s + p] = fmaf(c, vp, -(sn * vq));
                    V[r * s + q] = fmaf(sn, vp, c * vq);
                }
            }
        if (!rotated) break;
    }
    float smax = 0.0f;
    for (int64_t j = 0; j < s; ++j) {
        sig[j] = sqrtf(sdotf(B + j, s, B + j, s, s));
        if (sig[j] > smax) smax = sig[j];
    }
    float cut = ((float)s * FLT_EPSILON) * smax;
    for (int64_t r = 0; r < s; ++r) z[r] = 0.0f;
    for (int64_t j = 0; j < s; ++j) {
        if (!(sig[j] > cut)) continue;
        float coef = (sdotf(B + j, s, rhs0, 1, s) / sig[j]) / sig[j];
        for (int64_t r = 0; r < s; ++r) z[r] = fmaf(V[r * s + j], coef, z[r]);
    }
    free(B); free(V); free(sig);
}

int ora_local_solve_f32(int64_t s, float *M, float *rhs, float *z) {
    if (s == 0) return 0;
    float *M0 = (float *)malloc(sizeof(float) * (size_t)(s * s));
    float *r0 = (float *)malloc(sizeof(float) * (size_t)s);
    memcpy(M0, M, sizeof(float) * (size_t)(s * s));
    memcpy(r0, rhs, sizeof(float) * (size_t)s);
    float mx = 0.0f;
    for (int64_t k = 0; k < s * s; ++k) if (fabsf(M[k]) > mx) mx = fabsf(M[k]);
    float thr = ((float)s * FLT_EPSILON) * mx;
    int singular = (mx == 0.0f);
    for (int64_t k = 0; k < s && !singular; ++k) {
        int64_t piv = k;
        float best = fabsf(M[k * s + k]);
        for (int64_t r = k + 1; r < s; ++r)
            if (fabsf(M[r * s + k]) > best) { best = fabsf(M[r * s + k]); piv = r; }
        if (best <= thr) { singular = 1; break; }
        if (piv != k) {
            for (int64_t c = 0; c < s; ++c) { float t = M[k * s + c]; M[k * s + c] = M[piv * s + c]; M[piv * s + c] = t; }
            float t = rhs[k]; rhs[k] = rhs[piv]; rhs[piv] = t;
        }
        for (int64_t r = k + 1; r < s; ++r) {
            float l = M[r * s + k] / M[k * s + k];
            for (int64_t c = k + 1; c < s; ++c) M[r * s + c] = fmaf(-l, M[k * s + c], M[r * s + c]);
            rhs[r] = fmaf(-l, rhs[k], rhs[r]);
        }
    }
    if (!singular) {
        for (int64_t c = s - 1; c >= 0; --c) {
            z[c] = rhs[c] / M[c * s + c];
            for (int64_t r = 0; r < c; ++r) rhs[r] = fmaf(-M[r * s + c], z[c], rhs[r]);
        }
    } else {
        jacobi_lsf(s, M0, r0, z);
    }
    free(M0); free(r0);
    return singular;
}

/* ------------------------------------------------------------------------- */
/* lAIR restriction (Sec. 3.1). For C-point i with neighbourhood              */
/* R_i = {l_1 < ... < l_s}: Eq. (3.2) reads M z = rhs with M[r][c] = a_{l_c,l_r}*/
/* (the transpose of A restricted to R_i) and rhs[r] = -a_{i,l_r}; this makes   */
/* a_{i,j} + sum_k z_k a_{k,j} = 0 for every j in R_i (Eq. (3.1)), i.e.         */
/* (RA)_{i,j} = 0 on the pattern. Row i of R = {(l_r, z_r)} u {(i, 1)}.         */
/* In FP32 mode M and rhs are rounded to float and solved in float; z is then  */
/* stored exactly in double.                                                   */
/* ------------------------------------------------------------------------- */
static int build_lair_R(const ocsr *A, const int8_t *cf, const int64_t *cidx, int64_t nc, const int64_t *cpts,
                        const int64_t *nb_rp, const int32_t *nb_col, int prec, ocsr *R, uint8_t *lsflag) {
    int64_t nnz = nb_rp[nc] + nc;
    if (csr_alloc(R, nc, A->nr, nnz)) return ORA_ERR_OOM;
    int64_t smax = 0;
    for (int64_t c = 0; c < nc; ++c) if (nb_rp[c + 1] - nb_rp[c] > smax) smax = nb_rp[c + 1] - nb_rp[c];
    for (int64_t c = 0; c <= nc; ++c) R->rp[c] = nb_rp[c] + c;     /* row c: its set and the C point itself */
    (void)cf; (void)cidx;
    ORA_PARALLEL
    {
        double *M = (double *)malloc(sizeof(double) * (size_t)(smax * smax + 1));
        double *rhs = (double *)malloc(sizeof(double) * (size_t)(smax + 1));
        double *z = (double *)malloc(sizeof(double) * (size_t)(smax + 1));
        float *Mf = (float *)malloc(sizeof(float) * (size_t)(smax * smax + 1));
        float *rf = (float *)malloc(sizeof(float) * (size_t)(smax + 1));
        float *zf = (float *)malloc(sizeof(float) * (size_t)(smax + 1));
        ORA_FOR
        for (int64_t c = 0; c < nc; ++c) {
            int64_t i = cpts[c];
            const int32_t *nb = nb_col + nb_rp[c];
            int64_t s = nb_rp[c + 1] - nb_rp[c];
            for (int64_t k = 0; k < s * s; ++k) M[k] = 0.0;
            for (int64_t r = 0; r < s; ++r) rhs[r] = 0.0;
            for (int64_t cc = 0; cc < s; ++cc) {
                int64_t row = nb[cc];
                for (int64_t k = A->rp[row]; k < A->rp[row + 1]; ++k) {
                    int64_t r = find_pos(nb, s, A->col[k]);
                    if (r >= 0) M[r * s + cc] = A->val[k];
                }
            }
            for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
                int64_t r = find_pos(nb, s, A->col[k]);
                if (r >= 0) rhs[r] = -A->val[k];
            }
            int ls;
            if (prec == 0) {
                ls = ora_local_solve(s, M, rhs, z);
            } else {
                for (int64_t k = 0; k < s * s; ++k) Mf[k] = (float)M[k];
                for (int64_t r = 0; r < s; ++r) rf[r] = (float)rhs[r];
                ls = ora_local_solve_f32(s, Mf, rf, zf);
                for (int64_t r = 0; r < s; ++r) z[r] = (double)zf[r];
            }
            if (lsflag) lsflag[c] = (uint8_t)ls;
            /* merge {nb, z} with (i, 1) in ascending column order */
            int64_t p = R->rp[c];
            int placed = 0;
            for (int64_t r = 0; r < s; ++r) {
                if (!placed && i < nb[r]) { R->col[p] = (int32_t)i; R->val[p] = 1.0; p++; placed = 1; }
                R->col[p] = nb[r]; R->val[p] = z[r]; p++;
            }
            if (!placed) { R->col[p] = (int32_t)i; R->val[p] = 1.0; p++; }
        }
        free(M); free(rhs); free(z); free(Mf); free(rf); free(zf);
    }
    return ORA_OK;
}

/* ------------------------------------------------------------------------- */
/* Neumann restriction, nAIR (Sec. 3.2). For A with unit diagonal and         */
/* A_ff = I - L_ff the paper takes Z = -A_cf sum_{m=0}^{k} L_ff^m. A general A */
/* is brought to unit diagonal by D^{-1} A and the result scaled back          */
/* (Z = D_c Z^ D_f^{-1}), which gives                                          */
/*     Z = -A_cf sum_{m=0}^{k} (D_ff^{-1} E_ff)^m D_ff^{-1},  E_ff = D_ff - A_ff,  */
/* and keeps the row-scaling invariance of Sec. 3.1. Row i of Z as a row      */
/* vector over all F points: y_0 = -a_{i,F} D_ff^{-1}, y_{m+1} = y_m E_ff       */
/* D_ff^{-1}, that is y_{m+1}[l] = -(sum_{j in F, j != l} y_m[j] a_{j,l}) / a_ll */
/* (fma from 0 in ascending j), and z = y_0 + y_1 + ... + y_k in that order.    */
/* Every nonzero of A counts (no strength filter): z is supported on the F     */
/* points joined to i by a path of at most k + 1 edges whose points after i    */
/* are all F, the neighbourhood of distance k + 1 in the graph of A; R's row   */
/* holds that whole set (structural zeros kept) and (i, 1). In FP32 mode the    */
/* values are rounded to float and the series summed in float.                */
/* ------------------------------------------------------------------------- */
static int build_R_neumann(const ocsr *A, const int8_t *cf, int64_t nc, const int64_t *cpts, const int64_t *nb_rp,
                           const int32_t *nb_col, int k, int prec, ocsr *R) {
    int64_t n = A->nr;
    int64_t nnz = nb_rp[nc] + nc;
    if (csr_alloc(R, nc, n, nnz)) return ORA_ERR_OOM;
    ocsr AT;
    csr_transpose(A, &AT);   /* row l of A^T: the entries a_{j,l}, ascending j */
    double *diag = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t l = 0; l < n; ++l) find_entry(A, l, l, &diag[l]);
    double *y = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *yn = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *z = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    float *yf = (float *)calloc((size_t)(n > 0 ? n : 1), sizeof(float));
    float *ynf = (float *)calloc((size_t)(n > 0 ? n : 1), sizeof(float));
    float *zf = (float *)calloc((size_t)(n > 0 ? n : 1), sizeof(float));
    int st = ORA_OK;
    int64_t p = 0;
    for (int64_t c = 0; c < nc && st == ORA_OK; ++c) {
        int64_t i = cpts[c];
        for (int64_t l = 0; l < n; ++l) { y[l] = yn[l] = z[l] = 0.0; yf[l] = ynf[l] = zf[l] = 0.0f; }
        for (int64_t q = A->rp[i]; q < A->rp[i + 1]; ++q) {
            int64_t l = A->col[q];
            if (l == i || cf[l] != CF_F) continue;
            if (prec == 0) { y[l] = -A->val[q] / diag[l]; z[l] = y[l]; }
            else { yf[l] = -(float)A->val[q] / (float)diag[l]; zf[l] = yf[l]; }
        }
        for (int m = 1; m <= k; ++m) {
            for (int64_t l = 0; l < n; ++l) {
                if (cf[l] != CF_F) continue;
                double acc = 0.0;
                float accf = 0.0f;
                for (int64_t q = AT.rp[l]; q < AT.rp[l + 1]; ++q) {
                    int64_t j = AT.col[q];
                    if (j == l || cf[j] != CF_F) continue;
                    if (prec == 0) acc = fma(y[j], AT.val[q], acc);
                    else accf = fmaf(yf[j], (float)AT.val[q], accf);
                }
                if (prec == 0) yn[l] = -acc / diag[l];
                else ynf[l] = -accf / (float)diag[l];
            }
            for (int64_t l = 0; l < n; ++l) {
                if (cf[l] != CF_F) continue;
                if (prec == 0) { y[l] = yn[l]; z[l] = z[l] + y[l]; }
                else { yf[l] = ynf[l]; zf[l] = zf[l] + yf[l]; }
            }
        }
        /* the row: the neighbourhood (ascending) merged with (i, 1); nothing may lie outside it */
        const int32_t *nb = nb_col + nb_rp[c];
        int64_t s = nb_rp[c + 1] - nb_rp[c], inside = 0;
        int placed = 0;
        for (int64_t r = 0; r < s; ++r) {
            if (!placed && i < nb[r]) { R->col[p] = (int32_t)i; R->val[p] = 1.0; p++; placed = 1; }
            R->col[p] = nb[r];
            R->val[p] = prec == 0 ? z[nb[r]] : (double)zf[nb[r]];
            p++;
        }
        if (!placed) { R->col[p] = (int32_t)i; R->val[p] = 1.0; p++; }
        R->rp[c + 1] = p;
        for (int64_t l = 0; l < n; ++l)
            if ((prec == 0 ? z[l] != 0.0 : zf[l] != 0.0f)) inside++;
        for (int64_t r = 0; r < s; ++r)
            if ((prec == 0 ? z[nb[r]] != 0.0 : zf[nb[r]] != 0.0f)) inside--;
        if (inside != 0) st = ORA_ERR_ARG;   /* a value outside the neighbourhood: the sets are wrong */
    }
    csr_free(&AT);
    free(diag); free(y); free(yn); free(z); free(yf); free(ynf); free(zf);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Interpolation P = [W; I] (Eq. (2.2)).                                      */
/* One-point (Sec. 4): F row j takes value 1 at its strongest C connection     */
/* c in N_j (largest -a_jc, abs mode |a_jc|; ties -> smallest c), none -> an   */
/* empty row. lAIP (approximate ideal interpolation, W ~ -A_ff^{-1}A_fc,       */
/* Eq. (2.6)): for C-point c, Q_c = {F j : c in N_j} (distance two adds every  */
/* F j' with N_j' containing an F point of that set), and A_QQ w = -A_{Q,c}:   */
/* M[r][q] = a_{j_r, j_q}, rhs[r] = -a_{j_r, c}; W[j_r][c] = w_r. The local     */
/* solve is the same routine (same pivoting and least-squares rules) as for R. */
/* ------------------------------------------------------------------------- */
static int build_P_onepoint(const ocsr *A, const ograph *S, const int8_t *cf, const int64_t *cidx,
                            int64_t nc, int absmode, ocsr *P) {
    int64_t n = A->nr;
    if (csr_alloc(P, n, nc, n)) return ORA_ERR_OOM;
    int64_t p = 0;
    for (int64_t j = 0; j < n; ++j) {
        if (cf[j] == CF_C) {
            P->col[p] = (int32_t)cidx[j]; P->val[p] = 1.0; p++;
        } else {
            int64_t best = -1;
            double bv = 0.0;
            for (int64_t q = S->rp[j]; q < S->rp[j + 1]; ++q) {
                int64_t c = S->col[q];
                if (cf[c] != CF_C) continue;
                double a;
                find_entry(A, j, c, &a);
                double key = absmode ? fabs(a) : -a;
                if (best < 0 || key > bv) { best = c; bv = key; }
            }
            if (best >= 0) { P->col[p] = (int32_t)cidx[best]; P->val[p] = 1.0; p++; }
        }
        P->rp[j + 1] = p;
    }
    return ORA_OK;
}

typedef struct { int64_t row; int32_t col; double val; } coo_ent;

static int cmp_coo(const void *a, const void *b) {
    const coo_ent *x = (const coo_ent *)a, *y = (const coo_ent *)b;
    if (x->row != y->row) return (x->row > y->row) - (x->row < y->row);
    return (x->col > y->col) - (x->col < y->col);
}

/* the local systems of lAIP on given sets Q_c (ascending fine indices, c's own point excluded) */
static int build_P_laip_on(const ocsr *A, int64_t nc, const int64_t *cpts, const int64_t *q_rp,
                           const int32_t *q_col, int prec, ocsr *P, uint8_t *lsflag) {
    int64_t n = A->nr;
    int64_t total = q_rp[nc] + nc;
    coo_ent *ent = (coo_ent *)malloc(sizeof(coo_ent) * (size_t)(total > 0 ? total : 1));
    int64_t smax = 0;
    for (int64_t c = 0; c < nc; ++c) if (q_rp[c + 1] - q_rp[c] > smax) smax = q_rp[c + 1] - q_rp[c];
    ORA_PARALLEL
    {
        double *M = (double *)malloc(sizeof(double) * (size_t)(smax * smax + 1));
        double *rhs = (double *)malloc(sizeof(double) * (size_t)(smax + 1));
        double *w = (double *)malloc(sizeof(double) * (size_t)(smax + 1));
        float *Mf = (float *)malloc(sizeof(float) * (size_t)(smax * smax + 1));
        float *rf = (float *)malloc(sizeof(float) * (size_t)(smax + 1));
        float *wf = (float *)malloc(sizeof(float) * (size_t)(smax + 1));
        ORA_FOR
        for (int64_t c = 0; c < nc; ++c) {
            int64_t ci = cpts[c];
            const int32_t *Q = q_col + q_rp[c];
            int64_t s = q_rp[c + 1] - q_rp[c];
            for (int64_t k = 0; k < s * s; ++k) M[k] = 0.0;
            for (int64_t r = 0; r < s; ++r) {
                int64_t jr = Q[r];
                for (int64_t k = A->rp[jr]; k < A->rp[jr + 1]; ++k) {
                    int64_t q = find_pos(Q, s, A->col[k]);
                    if (q >= 0) M[r * s + q] = A->val[k];
                }
                double a;
                find_entry(A, jr, ci, &a);
                rhs[r] = -a;
            }
            int ls;
            if (prec == 0) {
                ls = ora_local_solve(s, M, rhs, w);
            } else {
                for (int64_t k = 0; k < s * s; ++k) Mf[k] = (float)M[k];
                for (int64_t r = 0; r < s; ++r) rf[r] = (float)rhs[r];
                ls = ora_local_solve_f32(s, Mf, rf, wf);
                for (int64_t r = 0; r < s; ++r) w[r] = (double)wf[r];
            }
            if (lsflag) lsflag[c] = (uint8_t)ls;
            int64_t e = q_rp[c] + c;                 /* column c's entries: its set, then its C point */
            for (int64_t r = 0; r < s; ++r) ent[e++] = (coo_ent){Q[r], (int32_t)c, w[r]};
            ent[e++] = (coo_ent){ci, (int32_t)c, 1.0};
        }
        free(M); free(rhs); free(w); free(Mf); free(rf); free(wf);
    }
    qsort(ent, (size_t)total, sizeof(coo_ent), cmp_coo);
    if (csr_alloc(P, n, nc, total)) return ORA_ERR_OOM;
    for (int64_t k = 0; k < total; ++k) {
        P->rp[ent[k].row + 1]++;
        P->col[k] = ent[k].col;
        P->val[k] = ent[k].val;
    }
    for (int64_t i = 0; i < n; ++i) P->rp[i + 1] += P->rp[i];
    free(ent);
    return ORA_OK;
}

static int build_P_laip(const ocsr *A, const ograph *ST, const int8_t *cf, int64_t nc, const int64_t *cpts,
                        int distance, int prec, ocsr *P, uint8_t *lsflag) {
    /* neighbourhoods Q_c are the distance-k neighbourhoods of c in the transposed graph */
    int64_t *q_rp; int32_t *q_col;
    build_neighbourhoods(ST, cf, distance, nc, cpts, &q_rp, &q_col);
    int st = build_P_laip_on(A, nc, cpts, q_rp, q_col, prec, P, lsflag);
    free(q_rp); free(q_col);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Galerkin coarse operator K = R A P (Sec. 2.1). First (RA)_{a,l} =           */
/* sum over k in row a of R (ascending) of R_ak A_kl, then K_{a,b} = sum over  */
/* l in row a of RA (ascending) of (RA)_al P_lb; every sum starts at 0 and     */
/* adds its terms with fma in that order. The pattern is the full symbolic     */
/* product: structural zeros are kept.                                         */
/* ------------------------------------------------------------------------- */
static int spgemm(const ocsr *X, const ocsr *Y, ocsr *Z) {
    int64_t nr = X->nr, ncol = Y->nc;
    Z->nr = nr; Z->nc = ncol;
    Z->rp = (int64_t *)calloc((size_t)nr + 1, sizeof(int64_t));
    /* pass 1: the number of distinct columns of every row */
    ORA_PARALLEL
    {
        int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncol > 0 ? ncol : 1));
        for (int64_t j = 0; j < ncol; ++j) mark[j] = -1;
        ORA_FOR
        for (int64_t a = 0; a < nr; ++a) {
            int64_t cnt = 0;
            for (int64_t p = X->rp[a]; p < X->rp[a + 1]; ++p)
                for (int64_t q = Y->rp[X->col[p]]; q < Y->rp[X->col[p] + 1]; ++q)
                    if (mark[Y->col[q]] != a) { mark[Y->col[q]] = a; cnt++; }
            Z->rp[a + 1] = cnt;
        }
        free(mark);
    }
    for (int64_t a = 0; a < nr; ++a) Z->rp[a + 1] += Z->rp[a];
    int64_t len = Z->rp[nr];
    Z->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(len > 0 ? len : 1));
    Z->val = (double *)malloc(sizeof(double) * (size_t)(len > 0 ? len : 1));
    /* pass 2: entry (a, l) starts at 0 and adds x_ak * y_kl with fma for k in ascending order */
    ORA_PARALLEL
    {
        double *acc = (double *)malloc(sizeof(double) * (size_t)(ncol > 0 ? ncol : 1));
        int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncol > 0 ? ncol : 1));
        for (int64_t j = 0; j < ncol; ++j) mark[j] = -1;
        ORA_FOR
        for (int64_t a = 0; a < nr; ++a) {
            int32_t *list = Z->col + Z->rp[a];
            int64_t cnt = 0;
            for (int64_t p = X->rp[a]; p < X->rp[a + 1]; ++p) {
                int64_t k = X->col[p];
                double x = X->val[p];
                for (int64_t q = Y->rp[k]; q < Y->rp[k + 1]; ++q) {
                    int64_t l = Y->col[q];
                    if (mark[l] != a) { mark[l] = a; acc[l] = 0.0; list[cnt++] = (int32_t)l; }
                    acc[l] = fma(x, Y->val[q], acc[l]);
                }
            }
            qsort(list, (size_t)cnt, sizeof(int32_t), cmp_i32);
            for (int64_t t = 0; t < cnt; ++t) Z->val[Z->rp[a] + t] = acc[list[t]];
        }
        free(acc); free(mark);
    }
    return ORA_OK;
}

/* ------------------------------------------------------------------------- */
/* Lumping (Sec. 3.3): in row i, every off-diagonal with |k_ij| <             */
/* theta_D * max_j |k_ij| (max over the whole row, diagonal included) is       */
/* removed and added to the diagonal; the additions go in ascending j order,   */
/* starting from k_ii. The row sum is kept.                                    */
/* ------------------------------------------------------------------------- */
static int lump(ocsr *K, double tol) {
    int64_t n = K->nr, p = 0;
    int64_t start = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t end = K->rp[i + 1];
        double m = 0.0;
        for (int64_t k = start; k < end; ++k) if (fabs(K->val[k]) > m) m = fabs(K->val[k]);
        double thr = tol * m;
        double d = 0.0;
        int64_t dpos = -1;
        for (int64_t k = start; k < end; ++k) if (K->col[k] == i) { d = K->val[k]; dpos = k; }
        if (dpos < 0) return ORA_ERR_ZERO_DIAG;
        for (int64_t k = start; k < end; ++k)
            if (K->col[k] != i && fabs(K->val[k]) < thr) d = d + K->val[k];
        for (int64_t k = start; k < end; ++k) {
            if (K->col[k] != i && fabs(K->val[k]) < thr) continue;
            K->col[p] = K->col[k];
            K->val[p] = (K->col[k] == i) ? d : K->val[k];
            p++;
        }
        start = end;
        K->rp[i + 1] = p;
    }
    return ORA_OK;
}

/* Lumping on a kept pattern (hierarchy refresh): row i of T keeps exactly    */
/* the columns it already has; every other entry of row i of K (the full      */
/* product) is added to the diagonal, in ascending j order starting from      */
/* k_ii, as in lump() when the dropped set is the same. T's pattern must be a  */
/* subset of K's and both rows must hold the diagonal.                         */
static int lump_on_pattern(const ocsr *K, ocsr *T) {
    for (int64_t i = 0; i < K->nr; ++i) {
        int64_t k0 = K->rp[i], k1 = K->rp[i + 1], t0 = T->rp[i], t1 = T->rp[i + 1];
        double d;
        if (!find_entry(K, i, i, &d)) return ORA_ERR_ZERO_DIAG;
        int64_t t = t0;
        for (int64_t k = k0; k < k1; ++k) {
            int64_t j = K->col[k];
            while (t < t1 && T->col[t] < j) ++t;
            int kept = t < t1 && T->col[t] == j;
            if (j != i && !kept) d = d + K->val[k];
        }
        t = t0;
        for (int64_t k = k0; k < k1 && t < t1; ++k) {
            if (K->col[k] != T->col[t]) continue;
            T->val[t] = (T->col[t] == i) ? d : K->val[k];
            ++t;
        }
        if (t != t1) return ORA_ERR_ARG;   /* an entry of T that K does not have */
    }
    return ORA_OK;
}

/* ------------------------------------------------------------------------- */
/* Block-diagonal scaling for DG (Sec. 4.2.1): A -> D_B^{-1} A, b -> D_B^{-1} b*/
/* D_B = the bs x bs diagonal blocks. D_B^{-1} columns come from the LU above  */
/* applied to unit vectors (same pivot and elimination order); the scaled row  */
/* r of block K is sum_t Dinv[r][t] * A[K t, :] with fma in ascending t. The   */
/* diagonal block of the result is set to the exact identity.                  */
/* ------------------------------------------------------------------------- */
static int block_inverse(int64_t s, const double *D, double *Dinv) {
    double *M = (double *)malloc(sizeof(double) * (size_t)(s * s));
    double *L = (double *)calloc((size_t)(s * s), sizeof(double));
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)s);
    memcpy(M, D, sizeof(double) * (size_t)(s * s));
    for (int64_t r = 0; r < s; ++r) perm[r] = r;
    double mx = 0.0;
    for (int64_t k = 0; k < s * s; ++k) if (fabs(M[k]) > mx) mx = fabs(M[k]);
    double thr = ((double)s * DBL_EPSILON) * mx;
    int bad = (mx == 0.0);
    for (int64_t k = 0; k < s && !bad; ++k) {
        int64_t piv = k;
        double best = fabs(M[k * s + k]);
        for (int64_t r = k + 1; r < s; ++r)
            if (fabs(M[r * s + k]) > best) { best = fabs(M[r * s + k]); piv = r; }
        if (best <= thr) { bad = 1; break; }
        if (piv != k) {
            for (int64_t c = 0; c < s; ++c) {
                double t = M[k * s + c]; M[k * s + c] = M[piv * s + c]; M[piv * s + c] = t;
                t = L[k * s + c]; L[k * s + c] = L[piv * s + c]; L[piv * s + c] = t;
            }
            int64_t t = perm[k]; perm[k] = perm[piv]; perm[piv] = t;
        }
        for (int64_t r = k + 1; r < s; ++r) {
            double l = M[r * s + k] / M[k * s + k];
            L[r * s + k] = l;
            for (int64_t c = k + 1; c < s; ++c) M[r * s + c] = fma(-l, M[k * s + c], M[r * s + c]);
        }
    }
    if (!bad) {
        double *rhs = (double *)malloc(sizeof(double) * (size_t)s);
        for (int64_t t = 0; t < s; ++t) {
            for (int64_t r = 0; r < s; ++r) rhs[r] = (perm[r] == t) ? 1.0 : 0.0;
            for (int64_t k = 0; k < s; ++k)
                for (int64_t r = k + 1; r < s; ++r) rhs[r] = fma(-L[r * s + k], rhs[k], rhs[r]);
            for (int64_t c = s - 1; c >= 0; --c) {
                double zc = rhs[c] / M[c * s + c];
                Dinv[c * s + t] = zc;
                for (int64_t r = 0; r < c; ++r) rhs[r] = fma(-M[r * s + c], zc, rhs[r]);
            }
        }
        free(rhs);
    }
    free(M); free(L); free(perm);
    return bad ? ORA_ERR_ZERO_DIAG : ORA_OK;
}

/* entries of D_B^{-1} A: per block, bs rows x (1 + union of off-block columns) */
int64_t ora_block_scale_nnz(int64_t n, const int64_t *rp, const int32_t *col, int64_t bs) {
    int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * (size_t)(rp[n] + 1));
    int64_t total = 0;
    for (int64_t K = 0; K < n / bs; ++K) {
        int64_t r0 = K * bs, nc = 0;
        for (int64_t r = 0; r < bs; ++r)
            for (int64_t k = rp[r0 + r]; k < rp[r0 + r + 1]; ++k)
                if (col[k] < r0 || col[k] >= r0 + bs) cols[nc++] = col[k];
        qsort(cols, (size_t)nc, sizeof(int32_t), cmp_i32);
        int64_t u = 0;
        for (int64_t a = 0; a < nc; ++a) if (u == 0 || cols[u - 1] != cols[a]) cols[u++] = cols[a];
        total += bs * (u + 1);
    }
    free(cols);
    return total;
}

int ora_block_scale(int64_t n, const int64_t *rp, const int32_t *col, const double *val, int64_t bs,
                    int64_t *out_rp, int32_t *out_col, double *out_val, double *dinv_blocks) {
    /* out arrays hold ora_block_scale_nnz() entries */
    int64_t nb = n / bs, p = 0;
    double *D = (double *)malloc(sizeof(double) * (size_t)(bs * bs));
    double *Di = (double *)malloc(sizeof(double) * (size_t)(bs * bs));
    int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * (size_t)(rp[n] + 1));
    out_rp[0] = 0;
    for (int64_t K = 0; K < nb; ++K) {
        int64_t r0 = K * bs;
        for (int64_t t = 0; t < bs * bs; ++t) D[t] = 0.0;
        for (int64_t r = 0; r < bs; ++r)
            for (int64_t k = rp[r0 + r]; k < rp[r0 + r + 1]; ++k)
                if (col[k] >= r0 && col[k] < r0 + bs) D[r * bs + (col[k] - r0)] = val[k];
        if (block_inverse(bs, D, Di)) { free(D); free(Di); free(cols); return ORA_ERR_ZERO_DIAG; }
        if (dinv_blocks) memcpy(dinv_blocks + K * bs * bs, Di, sizeof(double) * (size_t)(bs * bs));
        /* union of the block rows' columns outside the diagonal block */
        int64_t nc = 0;
        for (int64_t r = 0; r < bs; ++r)
            for (int64_t k = rp[r0 + r]; k < rp[r0 + r + 1]; ++k)
                if (col[k] < r0 || col[k] >= r0 + bs) cols[nc++] = col[k];
        qsort(cols, (size_t)nc, sizeof(int32_t), cmp_i32);
        int64_t u = 0;
        for (int64_t a = 0; a < nc; ++a) if (u == 0 || cols[u - 1] != cols[a]) cols[u++] = cols[a];
        for (int64_t r = 0; r < bs; ++r) {
            int placed = 0;
            for (int64_t a = 0; a <= u; ++a) {
                if (!placed && (a == u || cols[a] > r0 + r)) {
                    out_col[p] = (int32_t)(r0 + r); out_val[p] = 1.0; p++; placed = 1;
                }
                if (a == u) break;
                int64_t j = cols[a];
                double acc = 0.0;
                for (int64_t t = 0; t < bs; ++t) {
                    double a_tj;
                    find_entry(&(ocsr){n, n, (int64_t *)rp, (int32_t *)col, (double *)val}, r0 + t, j, &a_tj);
                    acc = fma(Di[r * bs + t], a_tj, acc);
                }
                out_col[p] = (int32_t)j; out_val[p] = acc; p++;
            }
            out_rp[r0 + r + 1] = p;
        }
    }
    free(D); free(Di); free(cols);
    return ORA_OK;
}

static void block_apply(int64_t n, int64_t bs, const double *dinv_blocks, const double *b, double *out) {
    for (int64_t K = 0; K < n / bs; ++K)
        for (int64_t r = 0; r < bs; ++r) {
            double acc = 0.0;
            for (int64_t t = 0; t < bs; ++t) acc = fma(dinv_blocks[K * bs * bs + r * bs + t], b[K * bs + t], acc);
            out[K * bs + r] = acc;
        }
}

/* ------------------------------------------------------------------------- */
/* Dense LU for the coarsest level (partial pivoting, same rules as above).    */
/* ------------------------------------------------------------------------- */
typedef struct { int64_t n; double *LU; int64_t *perm; } odense;

static int dense_factor(const ocsr *A, odense *d) {
    int64_t n = A->nr;
    d->n = n;
    d->LU = (double *)calloc((size_t)(n * n > 0 ? n * n : 1), sizeof(double));
    d->perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) d->LU[i * n + A->col[k]] = A->val[k];
    for (int64_t i = 0; i < n; ++i) d->perm[i] = i;
    double *M = d->LU;
    for (int64_t k = 0; k < n; ++k) {
        int64_t piv = k;
        double best = fabs(M[k * n + k]);
        for (int64_t r = k + 1; r < n; ++r)
            if (fabs(M[r * n + k]) > best) { best = fabs(M[r * n + k]); piv = r; }
        if (best == 0.0) return ORA_ERR_ZERO_DIAG;
        if (piv != k) {
            for (int64_t c = 0; c < n; ++c) { double t = M[k * n + c]; M[k * n + c] = M[piv * n + c]; M[piv * n + c] = t; }
            int64_t t = d->perm[k]; d->perm[k] = d->perm[piv]; d->perm[piv] = t;
        }
        for (int64_t r = k + 1; r < n; ++r) {
            double l = M[r * n + k] / M[k * n + k];
            M[r * n + k] = l;
            for (int64_t c = k + 1; c < n; ++c) M[r * n + c] = fma(-l, M[k * n + c], M[r * n + c]);
        }
    }
    return ORA_OK;
}

static void dense_solve(const odense *d, const double *b, double *x) {
    int64_t n = d->n;
    const double *M = d->LU;
    for (int64_t r = 0; r < n; ++r) x[r] = b[d->perm[r]];
    for (int64_t k = 0; k < n; ++k)
        for (int64_t r = k + 1; r < n; ++r) x[r] = fma(-M[r * n + k], x[k], x[r]);
    for (int64_t c = n - 1; c >= 0; --c) {
        x[c] = x[c] / M[c * n + c];
        for (int64_t r = 0; r < c; ++r) x[r] = fma(-M[r * n + c], x[c], x[r]);
    }
}

/* ------------------------------------------------------------------------- */
/* Nodal (block) hierarchy: Sec. 3.1 forms the local system with k x k blocks  */
/* (the block system solved for k right-hand sides), and Sec. 4.2.1 names      */
/* approach (iii): strength, C/F splitting and transfer operators by block.    */
/* Node I holds the k consecutive unknowns kI .. kI + k - 1.                   */
/* Node matrix: b_IJ = ||A_IJ||_F over the stored entries of block (I, J),     */
/* summed as fma(a, a, .) from 0 in ascending row, then ascending column, then */
/* one square root. Strength, splitting, neighbourhoods and the one-point      */
/* choice are those of the scalar method applied to this matrix (abs mode: the */
/* entries are norms); a node's unknowns all take the node's C/F label; the   */
/* local-solve set of every unknown of a C node is every unknown of the node's */
/* F-node neighbourhood, so its k rows of R are the block system of Sec. 3.1;  */
/* one-point P puts the k x k identity at the strongest C node.                */
/* ------------------------------------------------------------------------- */
static int node_matrix(const ocsr *A, int64_t k, ocsr *B) {
    int64_t N = A->nr / k;
    int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * (size_t)(A->rp[A->nr] + 1));
    int64_t cap = A->rp[A->nr] + 1, len = 0;
    B->nr = B->nc = N;
    B->rp = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
    B->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    B->val = (double *)malloc(sizeof(double) * (size_t)cap);
    for (int64_t I = 0; I < N; ++I) {
        int64_t m = 0;
        for (int64_t q = A->rp[k * I]; q < A->rp[k * I + k]; ++q) cols[m++] = (int32_t)(A->col[q] / k);
        m = sort_unique(cols, m);
        for (int64_t a = 0; a < m; ++a) {
            int64_t J = cols[a];
            double acc = 0.0;
            for (int64_t t = 0; t < k; ++t)
                for (int64_t q = A->rp[k * I + t]; q < A->rp[k * I + t + 1]; ++q)
                    if (A->col[q] / k == J) acc = fma(A->val[q], A->val[q], acc);
            B->col[len] = (int32_t)J;
            B->val[len] = sqrt(acc);
            len++;
        }
        B->rp[I + 1] = len;
    }
    free(cols);
    return ORA_OK;
}

/* sets of nodes -> sets of unknowns: set q of nodes gives k rows (one per unknown of coarse node q) */
static void expand_sets(int64_t k, int64_t NC, const int64_t *brp, const int32_t *bcol, int64_t **rp, int32_t **col) {
    int64_t nc = NC * k;
    *rp = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    *col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(brp[NC] * k * k + 1));
    int64_t p = 0;
    for (int64_t q = 0; q < NC; ++q)
        for (int64_t t = 0; t < k; ++t) {
            for (int64_t a = brp[q]; a < brp[q + 1]; ++a)
                for (int64_t u = 0; u < k; ++u) (*col)[p++] = (int32_t)(bcol[a] * k + u);
            (*rp)[q * k + t + 1] = p;
        }
}

/* Lumping by block (Sec. 3.3 with k x k blocks): in node row I, every block  */
/* K_IJ (J != I) with ||K_IJ||_F < theta_D max_J ||K_IJ||_F (diagonal block    */
/* included) is removed and added entrywise to the diagonal block:            */
/* k_{i, kI+u} += k_{i, kJ+u}, in ascending column order starting from         */
/* k_{i, kI+u}. Every scalar row sum is kept. With keep != NULL the kept       */
/* blocks are those of the pattern keep (hierarchy refresh) and K's values are */
/* written into keep; otherwise K is compacted in place.                       */
static int lump_nodal(ocsr *K, int64_t k, double tol, ocsr *keep) {
    int64_t n = K->nr, p = 0, start = 0;
    ocsr BK;
    node_matrix(K, k, &BK);
    double *d = (double *)malloc(sizeof(double) * (size_t)k);
    int8_t *has = (int8_t *)malloc((size_t)k);
    int st = ORA_OK;
    for (int64_t i = 0; i < n && st == ORA_OK; ++i) {
        int64_t I = i / k, end = K->rp[i + 1];
        double m = 0.0;
        for (int64_t a = BK.rp[I]; a < BK.rp[I + 1]; ++a) if (BK.val[a] > m) m = BK.val[a];
        double thr = tol * m;
        for (int64_t u = 0; u < k; ++u) { d[u] = 0.0; has[u] = 0; }
        for (int64_t q = start; q < end; ++q)
            if (K->col[q] / k == I) { d[K->col[q] % k] = K->val[q]; has[K->col[q] % k] = 1; }
        int64_t t0 = keep ? keep->rp[i] : 0, t1 = keep ? keep->rp[i + 1] : 0, t = t0;
        for (int64_t q = start; q < end; ++q) {
            int64_t J = K->col[q] / k;
            int dropped;
            if (keep) {
                while (t < t1 && keep->col[t] < K->col[q]) ++t;
                dropped = J != I && !(t < t1 && keep->col[t] == K->col[q]);
            } else {
                double bn = 0.0;
                find_entry(&BK, I, J, &bn);
                dropped = J != I && bn < thr;
            }
            if (!dropped) continue;
            int64_t u = K->col[q] % k;
            if (!has[u]) { st = ORA_ERR_ARG; break; }   /* no diagonal-block entry to take it */
            d[u] = d[u] + K->val[q];
        }
        if (keep) {
            t = t0;
            for (int64_t q = start; q < end && t < t1; ++q) {
                if (K->col[q] != keep->col[t]) continue;
                keep->val[t] = (K->col[q] / k == I) ? d[K->col[q] % k] : K->val[q];
                ++t;
            }
            if (t != t1) st = ORA_ERR_ARG;
        } else {
            for (int64_t q = start; q < end; ++q) {
                int64_t J = K->col[q] / k;
                double bn = 0.0;
                find_entry(&BK, I, J, &bn);
                if (J != I && bn < thr) continue;
                K->col[p] = K->col[q];
                K->val[p] = (J == I) ? d[K->col[q] % k] : K->val[q];
                p++;
            }
            K->rp[i + 1] = p;
        }
        start = end;
    }
    csr_free(&BK);
    free(d); free(has);
    return st;
}

/* inverse diagonal blocks (block Jacobi) by the LU of block_inverse; a missing entry counts as 0 */
static int node_block_inverses(const ocsr *A, int64_t k, double **out) {
    int64_t N = A->nr / k;
    double *binv = (double *)malloc(sizeof(double) * (size_t)(N * k * k > 0 ? N * k * k : 1));
    double *D = (double *)malloc(sizeof(double) * (size_t)(k * k));
    int st = ORA_OK;
    for (int64_t I = 0; I < N && st == ORA_OK; ++I) {
        for (int64_t e = 0; e < k * k; ++e) D[e] = 0.0;
        for (int64_t t = 0; t < k; ++t)
            for (int64_t q = A->rp[k * I + t]; q < A->rp[k * I + t + 1]; ++q)
                if (A->col[q] / k == I) D[t * k + A->col[q] % k] = A->val[q];
        st = block_inverse(k, D, binv + I * k * k);
    }
    free(D);
    *out = binv;
    return st;
}

/* ------------------------------------------------------------------------- */
/* Hierarchy                                                                  */
/* ------------------------------------------------------------------------- */
#define ORA_MAX_LEVELS 64

typedef struct {
    ocsr A;            /* level operator (lumped on coarse levels) */
    int8_t *cf;        /* 1 = C, 0 = F (levels that coarsen) */
    int64_t *cidx;     /* coarse index or -1 */
    int64_t nc;
    uint8_t *strong;   /* strength mask over A's pattern (theta) */
    uint8_t *strong_cf;/* strength mask for the splitting (theta_cf) */
    ocsr R, P;
    uint8_t *ls_R, *ls_P;
    double *dinv;
    float *A32, *R32, *P32, *dinv32;
    double *binv;      /* nodal: inverse diagonal blocks, k*k per node (block Jacobi) */
    float *binv32;
    int64_t *seg;      /* batched systems: offsets of the systems on this level (nseg + 1) */
} olevel;

typedef struct {
    ora_opts o;
    int nlev;
    olevel lev[ORA_MAX_LEVELS];
    odense coarse;
    int64_t bs;
    double *blk_inv;   /* block inverses for DG scaling */
    /* work */
    double *w64[ORA_MAX_LEVELS][4];
    float *w32[ORA_MAX_LEVELS][4];
    int status;
    int64_t singular_R, singular_P;
} ohier;

void ora_opts_default(ora_opts *o) {
    memset(o, 0, sizeof(*o));
    o->cf_mode = 3;
    o->distance = 1;
    o->theta = 0.25;
    o->theta_cf = 0.25;
    o->strength_abs = 0;
    o->interp = 0;
    o->relax = 0;
    o->lump_tol = 1e-3;
    o->lump_level0 = 0;
    o->prec = 0;
    o->coarse_max = 128;
    o->max_levels = 25;
    o->block_size = 0;
    o->rs_block = 4096;
    o->pmis_seed = 0x5eedULL;
}

static int coarsen_level_nodal(ohier *H, int l, int *is_last) {
    olevel *L = &H->lev[l];
    const ora_opts *o = &H->o;
    ocsr *A = &L->A;
    const int64_t k = o->nodal;
    int64_t n = A->nr, nnz = A->rp[n], N = n / k;
    int st;
    if (n % k) return ORA_ERR_ARG;
    ocsr B;
    node_matrix(A, k, &B);
    int64_t bnnz = B.rp[N];
    uint8_t *sB = (uint8_t *)malloc((size_t)(bnnz > 0 ? bnnz : 1));
    uint8_t *sBcf = (uint8_t *)malloc((size_t)(bnnz > 0 ? bnnz : 1));
    ora_strength(N, B.rp, B.col, B.val, o->theta, 1, sB);
    ora_strength(N, B.rp, B.col, B.val, o->theta_cf, 1, sBcf);
    /* the scalar masks: an entry is strong when its block is */
    L->strong = (uint8_t *)malloc((size_t)(nnz > 0 ? nnz : 1));
    L->strong_cf = (uint8_t *)malloc((size_t)(nnz > 0 ? nnz : 1));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t q = A->rp[i]; q < A->rp[i + 1]; ++q) {
            int64_t pos = B.rp[i / k] + find_pos(B.col + B.rp[i / k], B.rp[i / k + 1] - B.rp[i / k], A->col[q] / k);
            L->strong[q] = sB[pos];
            L->strong_cf[q] = sBcf[pos];
        }
    ograph S, ST, Scf, STcf;
    graph_from_mask(N, B.rp, B.col, sB, &S);
    graph_transpose(&S, &ST);
    graph_from_mask(N, B.rp, B.col, sBcf, &Scf);
    graph_transpose(&Scf, &STcf);
    int8_t *cfB = (int8_t *)malloc((size_t)(N > 0 ? N : 1));
    if (l == 0 && o->cf_mode == 2 && o->cf_user) {
        for (int64_t I = 0; I < N; ++I) cfB[I] = o->cf_user[I * k] ? CF_C : CF_F;
    } else {
        if (o->cf_mode == 0) cf_rs(&Scf, &STcf, cfB);
        else if (o->cf_mode != 1) cf_rs_blocked(&Scf, &STcf, o->rs_block, cfB);
        else cf_pmis(&Scf, &STcf, o->pmis_seed + (uint64_t)l, cfB);
    }
    L->cf = (int8_t *)malloc((size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) L->cf[i] = cfB[i / k];
    L->cidx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t nc = 0;
    for (int64_t i = 0; i < n; ++i) L->cidx[i] = (L->cf[i] == CF_C) ? nc++ : -1;
    L->nc = nc;
    int64_t NC = nc / k;
    if (nc == 0 || nc == n) {
        graph_free(&S); graph_free(&ST); graph_free(&Scf); graph_free(&STcf);
        csr_free(&B); free(sB); free(sBcf); free(cfB);
        *is_last = 1;
        return ORA_OK;
    }
    int64_t *cptsB = (int64_t *)malloc(sizeof(int64_t) * (size_t)NC);
    int64_t *cidxB = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    for (int64_t I = 0, q = 0; I < N; ++I) {
        cidxB[I] = cfB[I] == CF_C ? q : -1;
        if (cfB[I] == CF_C) cptsB[q++] = I;
    }
    int64_t *cpts = (int64_t *)malloc(sizeof(int64_t) * (size_t)nc);
    for (int64_t i = 0; i < n; ++i) if (L->cf[i] == CF_C) cpts[L->cidx[i]] = i;
    /* R: block local systems on the expanded node neighbourhoods */
    int64_t *nbB_rp, *nb_rp;
    int32_t *nbB_col, *nb_col;
    build_neighbourhoods(&S, cfB, o->distance, NC, cptsB, &nbB_rp, &nbB_col);
    expand_sets(k, NC, nbB_rp, nbB_col, &nb_rp, &nb_col);
    L->ls_R = (uint8_t *)calloc((size_t)nc, 1);
    st = build_lair_R(A, L->cf, L->cidx, nc, cpts, nb_rp, nb_col, o->prec, &L->R, L->ls_R);
    free(nbB_rp); free(nbB_col); free(nb_rp); free(nb_col);
    if (!st) {
        if (o->interp == 1) {
            /* block one-point: the node-level choice, as the k x k identity */
            ocsr PB;
            st = build_P_onepoint(&B, &S, cfB, cidxB, NC, 1, &PB);
            if (!st && !(st = csr_alloc(&L->P, n, nc, PB.rp[N] * k))) {
                int64_t p = 0;
                for (int64_t i = 0; i < n; ++i) {
                    for (int64_t a = PB.rp[i / k]; a < PB.rp[i / k + 1]; ++a) {
                        L->P.col[p] = (int32_t)(PB.col[a] * k + i % k);
                        L->P.val[p] = 1.0;
                        p++;
                    }
                    L->P.rp[i + 1] = p;
                }
            }
            csr_free(&PB);
        } else {
            int64_t *qB_rp, *q_rp;
            int32_t *qB_col, *q_col;
            build_neighbourhoods(&ST, cfB, o->distance, NC, cptsB, &qB_rp, &qB_col);
            expand_sets(k, NC, qB_rp, qB_col, &q_rp, &q_col);
            L->ls_P = (uint8_t *)calloc((size_t)nc, 1);
            st = build_P_laip_on(A, nc, cpts, q_rp, q_col, o->prec, &L->P, L->ls_P);
            free(qB_rp); free(qB_col); free(q_rp); free(q_col);
        }
    }
    free(cpts); free(cptsB); free(cidxB); free(cfB); free(sB); free(sBcf);
    csr_free(&B);
    graph_free(&S); graph_free(&ST); graph_free(&Scf); graph_free(&STcf);
    if (st) return st;
    for (int64_t c = 0; c < nc; ++c) {
        H->singular_R += L->ls_R[c];
        if (L->ls_P) H->singular_P += L->ls_P[c];
    }
    ocsr RA, K;
    spgemm(&L->R, A, &RA);
    spgemm(&RA, &L->P, &K);
    csr_free(&RA);
    if (o->lump_tol > 0.0) {
        st = lump_nodal(&K, k, o->lump_tol, NULL);
        if (st) { csr_free(&K); return st; }
    }
    H->lev[l + 1].A = K;
    *is_last = 0;
    return ORA_OK;
}

static int coarsen_level(ohier *H, int l, int *is_last) {
    olevel *L = &H->lev[l];
    const ora_opts *o = &H->o;
    ocsr *A = &L->A;
    int64_t n = A->nr, nnz = A->rp[n];
    int st;
    L->strong = (uint8_t *)malloc((size_t)(nnz > 0 ? nnz : 1));
    L->strong_cf = (uint8_t *)malloc((size_t)(nnz > 0 ? nnz : 1));
    ora_strength(n, A->rp, A->col, A->val, o->theta, o->strength_abs, L->strong);
    ora_strength(n, A->rp, A->col, A->val, o->theta_cf, o->strength_abs, L->strong_cf);
    ograph S, ST, Scf, STcf;
    graph_from_mask(n, A->rp, A->col, L->strong, &S);
    graph_transpose(&S, &ST);
    graph_from_mask(n, A->rp, A->col, L->strong_cf, &Scf);
    graph_transpose(&Scf, &STcf);
    L->cf = (int8_t *)malloc((size_t)(n > 0 ? n : 1));
    if (l == 0 && o->cf_mode == 2 && o->cf_user) {
        for (int64_t i = 0; i < n; ++i) L->cf[i] = o->cf_user[i] ? CF_C : CF_F;
    } else {
        if (o->cf_mode == 0) cf_rs(&Scf, &STcf, L->cf);
        else if (o->cf_mode != 1) cf_rs_blocked_seg(&Scf, &STcf, o->rs_block, L->seg, o->nseg, L->cf);
        else cf_pmis(&Scf, &STcf, o->pmis_seed + (uint64_t)l, L->cf);
    }
    L->cidx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t nc = 0;
    for (int64_t i = 0; i < n; ++i) L->cidx[i] = (L->cf[i] == CF_C) ? nc++ : -1;
    L->nc = nc;
    if (nc == 0 || nc == n) {
        graph_free(&S); graph_free(&ST); graph_free(&Scf); graph_free(&STcf);
        *is_last = 1;
        return ORA_OK;
    }
    if (o->nseg > 0 && L->seg) {
        /* the systems' offsets on the next level: C points before each system's first point */
        olevel *Ln = &H->lev[l + 1];
        Ln->seg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(o->nseg + 1));
        int64_t c = 0, i = 0;
        for (int q = 0; q <= o->nseg; ++q) {
            for (; i < L->seg[q] && i < n; ++i) c += (L->cf[i] == CF_C);
            Ln->seg[q] = c;
        }
    }
    int64_t *cpts = (int64_t *)malloc(sizeof(int64_t) * (size_t)nc);
    for (int64_t i = 0; i < n; ++i) if (L->cf[i] == CF_C) cpts[L->cidx[i]] = i;
    int64_t *nb_rp; int32_t *nb_col;
    L->ls_R = (uint8_t *)calloc((size_t)nc, 1);
    if (o->restriction == 1) {
        /* nAIR: the sets come from the graph of every nonzero off-diagonal of A */
        uint8_t *all = (uint8_t *)malloc((size_t)(nnz > 0 ? nnz : 1));
        ora_strength(n, A->rp, A->col, A->val, 0.0, 1, all);
        ograph G;
        graph_from_mask(n, A->rp, A->col, all, &G);
        free(all);
        build_neighbourhoods(&G, L->cf, o->distance, nc, cpts, &nb_rp, &nb_col);
        graph_free(&G);
        st = build_R_neumann(A, L->cf, nc, cpts, nb_rp, nb_col, o->distance - 1, o->prec, &L->R);
    } else {
        build_neighbourhoods(&S, L->cf, o->distance, nc, cpts, &nb_rp, &nb_col);
        st = build_lair_R(A, L->cf, L->cidx, nc, cpts, nb_rp, nb_col, o->prec, &L->R, L->ls_R);
    }
    free(nb_rp); free(nb_col);
    if (st) return st;
    if (o->interp == 1) {
        st = build_P_onepoint(A, &S, L->cf, L->cidx, nc, o->strength_abs, &L->P);
    } else {
        L->ls_P = (uint8_t *)calloc((size_t)nc, 1);
        st = build_P_laip(A, &ST, L->cf, nc, cpts, o->distance, o->prec, &L->P, L->ls_P);
    }
    free(cpts);
    graph_free(&S); graph_free(&ST); graph_free(&Scf); graph_free(&STcf);
    if (st) return st;
    for (int64_t c = 0; c < nc; ++c) {
        H->singular_R += L->ls_R[c];
        if (L->ls_P) H->singular_P += L->ls_P[c];
    }
    ocsr RA, K;
    spgemm(&L->R, A, &RA);
    spgemm(&RA, &L->P, &K);
    csr_free(&RA);
    if (o->lump_tol > 0.0) {
        st = lump(&K, o->lump_tol);
        if (st) { csr_free(&K); return st; }
    }
    H->lev[l + 1].A = K;
    *is_last = 0;
    return ORA_OK;
}

static int finish_level(ohier *H, int l) {
    olevel *L = &H->lev[l];
    int64_t n = L->A.nr;
    L->dinv = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        double d;
        if (!find_entry(&L->A, i, i, &d) || d == 0.0) return ORA_ERR_ZERO_DIAG;
        L->dinv[i] = 1.0 / d;
    }
    if (H->o.nodal > 1 && L->R.rp) {
        int64_t k = H->o.nodal, N = n / k;
        int st = node_block_inverses(&L->A, k, &L->binv);
        if (st) return st;
        L->binv32 = (float *)malloc(sizeof(float) * (size_t)(N * k * k > 0 ? N * k * k : 1));
        for (int64_t e = 0; e < N * k * k; ++e) L->binv32[e] = (float)L->binv[e];
    }
    for (int k = 0; k < 4; ++k) {
        H->w64[l][k] = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
        H->w32[l][k] = (float *)calloc((size_t)(n > 0 ? n : 1), sizeof(float));
    }
    if (H->o.prec == 1) {
        int64_t nnz = L->A.rp[n];
        L->A32 = (float *)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
        for (int64_t k = 0; k < nnz; ++k) L->A32[k] = (float)L->A.val[k];
        L->dinv32 = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
        for (int64_t i = 0; i < n; ++i) L->dinv32[i] = (float)L->dinv[i];
        if (L->R.rp) {
            int64_t r = L->R.rp[L->R.nr], p = L->P.rp[L->P.nr];
            L->R32 = (float *)malloc(sizeof(float) * (size_t)(r > 0 ? r : 1));
            L->P32 = (float *)malloc(sizeof(float) * (size_t)(p > 0 ? p : 1));
            for (int64_t k = 0; k < r; ++k) L->R32[k] = (float)L->R.val[k];
            for (int64_t k = 0; k < p; ++k) L->P32[k] = (float)L->P.val[k];
        }
    }
    return ORA_OK;
}

void ora_free(ohier *H) {
    if (!H) return;
    for (int l = 0; l < H->nlev; ++l) {
        olevel *L = &H->lev[l];
        csr_free(&L->A); csr_free(&L->R); csr_free(&L->P);
        free(L->cf); free(L->cidx); free(L->strong); free(L->strong_cf); free(L->ls_R); free(L->ls_P);
        free(L->dinv); free(L->A32); free(L->R32); free(L->P32); free(L->dinv32); free(L->seg);
        free(L->binv); free(L->binv32);
        for (int k = 0; k < 4; ++k) { free(H->w64[l][k]); free(H->w32[l][k]); }
    }
    free(H->coarse.LU); free(H->coarse.perm); free(H->blk_inv);
    free(H);
}

ohier *ora_setup(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                 const ora_opts *opts, int *status) {
    ohier *H = (ohier *)calloc(1, sizeof(ohier));
    H->o = *opts;
    int64_t nnz = rp[n];
    ocsr *A0 = &H->lev[0].A;
    if (opts->block_size > 1 && n % opts->block_size) { *status = ORA_ERR_ARG; return H; }
    if (opts->nodal > 1 && (opts->nodal > 8 || n % opts->nodal || opts->block_size > 1 || opts->restriction != 0 ||
                            opts->nseg > 0)) {
        *status = ORA_ERR_ARG;
        return H;
    }
    if (opts->nodal > 1 && opts->cf_mode == 2 && opts->cf_user) {
        /* a node's unknowns share one label: its k entries of the user splitting must agree */
        for (int64_t i = 0; i < n; ++i)
            if ((opts->cf_user[i] != 0) != (opts->cf_user[i - i % opts->nodal] != 0)) { *status = ORA_ERR_ARG; return H; }
    }
    if (opts->block_size > 1) nnz = ora_block_scale_nnz(n, rp, col, opts->block_size);
    if (csr_alloc(A0, n, n, nnz)) { *status = ORA_ERR_OOM; return H; }
    if (opts->block_size > 1) {
        H->bs = opts->block_size;
        H->blk_inv = (double *)malloc(sizeof(double) * (size_t)(n * H->bs));
        int st = ora_block_scale(n, rp, col, val, H->bs, A0->rp, A0->col, A0->val, H->blk_inv);
        if (st) { *status = st; H->nlev = 1; return H; }
    } else {
        memcpy(A0->rp, rp, sizeof(int64_t) * (size_t)(n + 1));
        memcpy(A0->col, col, sizeof(int32_t) * (size_t)nnz);
        memcpy(A0->val, val, sizeof(double) * (size_t)nnz);
    }
    if (opts->nseg > 0 && opts->seg) {
        H->lev[0].seg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(opts->nseg + 1));
        memcpy(H->lev[0].seg, opts->seg, sizeof(int64_t) * (size_t)(opts->nseg + 1));
    }
    H->o.seg = NULL;   /* not retained */
    if (opts->lump_level0 && opts->lump_tol > 0.0) {
        int st = opts->nodal > 1 ? lump_nodal(A0, opts->nodal, opts->lump_tol, NULL) : lump(A0, opts->lump_tol);
        if (st) { *status = st; H->nlev = 1; return H; }
    }
    int l = 0;
    for (;;) {
        H->nlev = l + 1;
        int64_t nl = H->lev[l].A.nr;
        int last = (nl <= opts->coarse_max) || (l + 1 >= opts->max_levels) || (l + 1 >= ORA_MAX_LEVELS);
        if (!last) {
            int st = opts->nodal > 1 ? coarsen_level_nodal(H, l, &last) : coarsen_level(H, l, &last);
            if (st) { *status = st; return H; }
        }
        int st = finish_level(H, l);
        if (st) { *status = st; return H; }
        if (last) {
            if (nl > 4096) { *status = ORA_ERR_STALLED; return H; }
            st = dense_factor(&H->lev[l].A, &H->coarse);
            *status = st;
            return H;
        }
        ++l;
    }
}

/* ------------------------------------------------------------------------- */
/* Refresh: the same matrix pattern with new values, as for the backward      */
/* Euler step I + dt S of Sec. 4.1.1 when dt or the coefficients change        */
/* between steps. The splittings, strength masks, neighbourhoods of the local  */
/* systems and the patterns of R, P and every coarse operator stay as set-up   */
/* left them; every value is recomputed from the new matrix in set-up's order: */
/* block scaling (Sec. 4.2.1), lumping of level 0 when asked, then per level   */
/* R by the local solves of Sec. 3.1 on the neighbourhood read off R's pattern */
/* (row c without c itself), lAIP by its local solves on the sets Q_c read off */
/* P's pattern (column c without c's own point), one-point P unchanged (all    */
/* its values are 1), K = (RA)P, lumping onto the kept pattern of the next     */
/* level (Sec. 3.3), then D^{-1}, the FP32 copies and the dense factorisation  */
/* of the coarsest operator. rp and col must be the set-up's.                 */
/* ------------------------------------------------------------------------- */
static void unfinish_level(ohier *H, int l) {
    olevel *L = &H->lev[l];
    free(L->dinv); free(L->A32); free(L->R32); free(L->P32); free(L->dinv32); free(L->binv); free(L->binv32);
    L->dinv = NULL; L->A32 = L->R32 = L->P32 = L->dinv32 = NULL;
    L->binv = NULL; L->binv32 = NULL;
    for (int k = 0; k < 4; ++k) {
        free(H->w64[l][k]); free(H->w32[l][k]);
        H->w64[l][k] = NULL; H->w32[l][k] = NULL;
    }
}

static int same_pattern(const ocsr *X, const ocsr *Y) {
    if (X->nr != Y->nr || X->rp[X->nr] != Y->rp[Y->nr]) return 0;
    if (memcmp(X->rp, Y->rp, sizeof(int64_t) * (size_t)(X->nr + 1))) return 0;
    return memcmp(X->col, Y->col, sizeof(int32_t) * (size_t)X->rp[X->nr]) == 0;
}

static int refresh_level(ohier *H, int l) {
    olevel *L = &H->lev[l];
    const ora_opts *o = &H->o;
    const ocsr *A = &L->A;
    int64_t n = A->nr, nc = L->nc;
    int st;
    int64_t *cpts = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
    for (int64_t i = 0; i < n; ++i) if (L->cf[i] == CF_C) cpts[L->cidx[i]] = i;
    /* R: neighbourhoods from the kept pattern */
    int64_t *nb_rp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc + 1));
    int32_t *nb_col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(L->R.rp[nc] + 1));
    int64_t q = 0;
    nb_rp[0] = 0;
    for (int64_t c = 0; c < nc; ++c) {
        for (int64_t k = L->R.rp[c]; k < L->R.rp[c + 1]; ++k)
            if (L->R.col[k] != cpts[c]) nb_col[q++] = L->R.col[k];
        nb_rp[c + 1] = q;
    }
    ocsr R2;
    memset(&R2, 0, sizeof R2);
    if (o->restriction == 1) st = build_R_neumann(A, L->cf, nc, cpts, nb_rp, nb_col, o->distance - 1, o->prec, &R2);
    else st = build_lair_R(A, L->cf, L->cidx, nc, cpts, nb_rp, nb_col, o->prec, &R2, L->ls_R);
    free(nb_rp); free(nb_col);
    if (st || !same_pattern(&R2, &L->R)) { csr_free(&R2); free(cpts); return st ? st : ORA_ERR_ARG; }
    csr_free(&L->R);
    L->R = R2;
    if (o->interp != 1) {
        /* lAIP: Q_c = the fine rows of column c of P, without c's own point */
        ocsr PT;
        csr_transpose(&L->P, &PT);
        int64_t *q_rp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc + 1));
        int32_t *q_col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(PT.rp[nc] + 1));
        q = 0;
        q_rp[0] = 0;
        for (int64_t c = 0; c < nc; ++c) {
            for (int64_t k = PT.rp[c]; k < PT.rp[c + 1]; ++k)
                if (PT.col[k] != cpts[c]) q_col[q++] = PT.col[k];
            q_rp[c + 1] = q;
        }
        csr_free(&PT);
        ocsr P2;
        memset(&P2, 0, sizeof P2);
        st = build_P_laip_on(A, nc, cpts, q_rp, q_col, o->prec, &P2, L->ls_P);
        free(q_rp); free(q_col);
        if (st || !same_pattern(&P2, &L->P)) { csr_free(&P2); free(cpts); return st ? st : ORA_ERR_ARG; }
        csr_free(&L->P);
        L->P = P2;
    }
    free(cpts);
    for (int64_t c = 0; c < nc; ++c) {
        H->singular_R += L->ls_R[c];
        if (L->ls_P) H->singular_P += L->ls_P[c];
    }
    ocsr RA, K;
    spgemm(&L->R, A, &RA);
    spgemm(&RA, &L->P, &K);
    csr_free(&RA);
    ocsr *An = &H->lev[l + 1].A;
    if (o->lump_tol > 0.0) {
        st = o->nodal > 1 ? lump_nodal(&K, o->nodal, o->lump_tol, An) : lump_on_pattern(&K, An);
    } else if (same_pattern(&K, An)) {
        memcpy(An->val, K.val, sizeof(double) * (size_t)K.rp[K.nr]);
        st = ORA_OK;
    } else {
        st = ORA_ERR_ARG;
    }
    csr_free(&K);
    return st;
}

int ora_refresh(ohier *H, int64_t n, const int64_t *rp, const int32_t *col, const double *val) {
    const ora_opts *o = &H->o;
    ocsr *A0 = &H->lev[0].A;
    if (n != A0->nr) return ORA_ERR_ARG;
    ocsr T;
    int64_t nnz = o->block_size > 1 ? ora_block_scale_nnz(n, rp, col, o->block_size) : rp[n];
    if (csr_alloc(&T, n, n, nnz)) return ORA_ERR_OOM;
    int st = ORA_OK;
    if (o->block_size > 1) {
        st = ora_block_scale(n, rp, col, val, H->bs, T.rp, T.col, T.val, H->blk_inv);
    } else {
        memcpy(T.rp, rp, sizeof(int64_t) * (size_t)(n + 1));
        memcpy(T.col, col, sizeof(int32_t) * (size_t)nnz);
        memcpy(T.val, val, sizeof(double) * (size_t)nnz);
    }
    if (!st) {
        if (o->lump_level0 && o->lump_tol > 0.0)
            st = o->nodal > 1 ? lump_nodal(&T, o->nodal, o->lump_tol, A0) : lump_on_pattern(&T, A0);
        else if (same_pattern(&T, A0)) memcpy(A0->val, T.val, sizeof(double) * (size_t)nnz);
        else st = ORA_ERR_ARG;
    }
    csr_free(&T);
    if (st) return st;
    H->singular_R = H->singular_P = 0;
    for (int l = 0; l < H->nlev; ++l) {
        if (l + 1 < H->nlev) {
            st = refresh_level(H, l);
            if (st) return st;
        }
        unfinish_level(H, l);
        st = finish_level(H, l);
        if (st) return st;
    }
    free(H->coarse.LU); free(H->coarse.perm);
    memset(&H->coarse, 0, sizeof H->coarse);
    return dense_factor(&H->lev[H->nlev - 1].A, &H->coarse);
}

/* ------------------------------------------------------------------------- */
/* Cycle (Sec. 4): post-relaxation only, zero initial guess on every level.    */
/* cycle(l, b): bc = R b; xc = cycle(l+1, bc); x = P xc; then Jacobi sweeps    */
/* over F, F, C (or F, C, F / F, F): x_i <- x_i + dinv_i (b_i - A_i x) for the */
/* swept set, every update of a sweep reading the same old x (Eq. (2.4)).      */
/* Row products accumulate with fma in ascending column order.                 */
/* ------------------------------------------------------------------------- */
static void spmv64(const ocsr *A, const double *x, double *y) {
    ORA_PARALLEL_FOR
    for (int64_t i = 0; i < A->nr; ++i) {
        double acc = 0.0;
        for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) acc = fma(A->val[k], x[A->col[k]], acc);
        y[i] = acc;
    }
}

/* block Jacobi on a nodal level: x_I <- x_I + D_I^{-1} (b - A x)_I for the nodes of the target set; the
   residual rows by fma from 0 in ascending column, the block product by fma from 0 in ascending u */
static void sweep64_nodal(const olevel *L, int64_t k, int target, const double *b, const double *x, double *xo) {
    const ocsr *A = &L->A;
    double r[64];
    for (int64_t I = 0; I < A->nr / k; ++I) {
        if (L->cf[I * k] != target) {
            for (int64_t t = 0; t < k; ++t) xo[I * k + t] = x[I * k + t];
            continue;
        }
        for (int64_t t = 0; t < k; ++t) {
            int64_t i = I * k + t;
            double acc = 0.0;
            for (int64_t q = A->rp[i]; q < A->rp[i + 1]; ++q) acc = fma(A->val[q], x[A->col[q]], acc);
            r[t] = b[i] - acc;
        }
        for (int64_t t = 0; t < k; ++t) {
            double acc = 0.0;
            for (int64_t u = 0; u < k; ++u) acc = fma(L->binv[(I * k + t) * k + u], r[u], acc);
            xo[I * k + t] = x[I * k + t] + acc;
        }
    }
}

static void sweep32_nodal(const olevel *L, int64_t k, int target, const float *b, const float *x, float *xo) {
    const ocsr *A = &L->A;
    float r[64];
    for (int64_t I = 0; I < A->nr / k; ++I) {
        if (L->cf[I * k] != target) {
            for (int64_t t = 0; t < k; ++t) xo[I * k + t] = x[I * k + t];
            continue;
        }
        for (int64_t t = 0; t < k; ++t) {
            int64_t i = I * k + t;
            float acc = 0.0f;
            for (int64_t q = A->rp[i]; q < A->rp[i + 1]; ++q) acc = fmaf(L->A32[q], x[A->col[q]], acc);
            r[t] = b[i] - acc;
        }
        for (int64_t t = 0; t < k; ++t) {
            float acc = 0.0f;
            for (int64_t u = 0; u < k; ++u) acc = fmaf(L->binv32[(I * k + t) * k + u], r[u], acc);
            xo[I * k + t] = x[I * k + t] + acc;
        }
    }
}

static void sweep64(const olevel *L, int target, const double *b, const double *x, double *xo) {
    const ocsr *A = &L->A;
    ORA_PARALLEL_FOR
    for (int64_t i = 0; i < A->nr; ++i) {
        if (L->cf[i] != target) { xo[i] = x[i]; continue; }
        double acc = 0.0;
        for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) acc = fma(A->val[k], x[A->col[k]], acc);
        xo[i] = fma(L->dinv[i], b[i] - acc, x[i]);
    }
}

static const int relax_seq[3][3] = {{CF_F, CF_F, CF_C}, {CF_F, CF_C, CF_F}, {CF_F, CF_F, -9}};

static void cycle64(ohier *H, int l, const double *b, double *x) {
    olevel *L = &H->lev[l];
    int64_t n = L->A.nr;
    if (l == H->nlev - 1) { dense_solve(&H->coarse, b, x); return; }
    double *bc = H->w64[l + 1][0], *xc = H->w64[l + 1][1];
    spmv64(&L->R, b, bc);
    cycle64(H, l + 1, bc, xc);
    spmv64(&L->P, xc, x);
    double *t = H->w64[l][2];
    for (int s = 0; s < 3; ++s) {
        int tgt = relax_seq[H->o.relax][s];
        if (tgt == -9) break;
        if (H->o.nodal > 1) sweep64_nodal(L, H->o.nodal, tgt, b, x, t);
        else sweep64(L, tgt, b, x, t);
        memcpy(x, t, sizeof(double) * (size_t)n);
    }
}

static void spmv32(int64_t nr, const int64_t *rp, const int32_t *col, const float *val, const float *x, float *y) {
    ORA_PARALLEL_FOR
    for (int64_t i = 0; i < nr; ++i) {
        float acc = 0.0f;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) acc = fmaf(val[k], x[col[k]], acc);
        y[i] = acc;
    }
}

static void cycle32(ohier *H, int l, const float *b, float *x) {
    olevel *L = &H->lev[l];
    int64_t n = L->A.nr;
    if (l == H->nlev - 1) {
        double *bd = H->w64[l][0], *xd = H->w64[l][1];
        for (int64_t i = 0; i < n; ++i) bd[i] = (double)b[i];
        dense_solve(&H->coarse, bd, xd);
        for (int64_t i = 0; i < n; ++i) x[i] = (float)xd[i];
        return;
    }
    float *bc = H->w32[l + 1][0], *xc = H->w32[l + 1][1];
    spmv32(L->R.nr, L->R.rp, L->R.col, L->R32, b, bc);
    cycle32(H, l + 1, bc, xc);
    spmv32(L->P.nr, L->P.rp, L->P.col, L->P32, xc, x);
    float *t = H->w32[l][2];
    for (int s = 0; s < 3; ++s) {
        int tgt = relax_seq[H->o.relax][s];
        if (tgt == -9) break;
        if (H->o.nodal > 1) {
            sweep32_nodal(L, H->o.nodal, tgt, b, x, t);
            memcpy(x, t, sizeof(float) * (size_t)n);
            continue;
        }
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < n; ++i) {
            if (L->cf[i] != tgt) { t[i] = x[i]; continue; }
            float acc = 0.0f;
            for (int64_t k = L->A.rp[i]; k < L->A.rp[i + 1]; ++k) acc = fmaf(L->A32[k], x[L->A.col[k]], acc);
            t[i] = fmaf(L->dinv32[i], b[i] - acc, x[i]);
        }
        memcpy(x, t, sizeof(float) * (size_t)n);
    }
}

/* x = M^{-1} b (one V-cycle, zero initial guess), in the hierarchy's precision */
static void precond(ohier *H, const double *b, double *x) {
    int64_t n = H->lev[0].A.nr;
    if (H->o.prec == 0) {
        cycle64(H, 0, b, x);
    } else {
        float *b32 = (float *)calloc((size_t)(n > 0 ? n : 1), sizeof(float));
        float *x32 = (float *)calloc((size_t)(n > 0 ? n : 1), sizeof(float));
        for (int64_t i = 0; i < n; ++i) b32[i] = (float)b[i];
        cycle32(H, 0, b32, x32);
        for (int64_t i = 0; i < n; ++i) x[i] = (double)x32[i];
        free(b32); free(x32);
    }
}

void ora_precond_apply(ohier *H, const double *b, double *x) { precond(H, b, x); }

static double norm2(int64_t n, const double *x) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s = fma(x[i], x[i], s);
    return sqrt(s);
}

static double dot(int64_t n, const double *x, const double *y) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s = fma(x[i], y[i], s);
    return s;
}

static void residual(const ocsr *A, const double *b, const double *x, double *r) {
    ORA_PARALLEL_FOR
    for (int64_t i = 0; i < A->nr; ++i) {
        double acc = 0.0;
        for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) acc = fma(A->val[k], x[A->col[k]], acc);
        r[i] = b[i] - acc;
    }
}

/* ------------------------------------------------------------------------- */
/* Outer FP64 loops. cycle = 0: stationary iteration (iterative refinement):   */
/* r = b - A x, x += M^{-1} r. cycle = 1: right-preconditioned flexible GMRES  */
/* with restart m; Arnoldi by classical Gram-Schmidt applied twice; Givens     */
/* rotations; stop when the true relative residual ||b - A x|| / ||b|| <= tol. */
/* The system solved is the scaled one when block scaling is on.               */
/* Returns iterations (preconditioner applications); hist gets rel. residuals. */
/* ------------------------------------------------------------------------- */
int ora_solve(ohier *H, const double *b_in, double *x, double tol, int cycle, int max_iter, int restart,
              int *iters, double *final_rel, double *hist, int hist_cap) {
    const ocsr *A = &H->lev[0].A;
    int64_t n = A->nr;
    double *b = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (H->bs > 1) block_apply(n, H->bs, H->blk_inv, b_in, b);
    else memcpy(b, b_in, sizeof(double) * (size_t)n);
    double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *e = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double bn = norm2(n, b);
    if (bn == 0.0) bn = 1.0;
    int it = 0, nh = 0, status = ORA_ERR_NOT_CONVERGED;
    residual(A, b, x, r);
    double rel = norm2(n, r) / bn;
    if (hist && nh < hist_cap) hist[nh++] = rel;
    if (cycle == 0) {
        while (rel > tol && it < max_iter) {
            precond(H, r, e);
            for (int64_t i = 0; i < n; ++i) x[i] += e[i];
            residual(A, b, x, r);
            rel = norm2(n, r) / bn;
            ++it;
            if (hist && nh < hist_cap) hist[nh++] = rel;
            if (rel != rel) { status = ORA_ERR_NAN; break; }
        }
    } else {
        int m = restart > 0 ? restart : 30;
        double *V = (double *)malloc(sizeof(double) * (size_t)(n * (m + 1)));
        double *Z = (double *)malloc(sizeof(double) * (size_t)(n * m));
        double *Hm = (double *)calloc((size_t)((m + 1) * m), sizeof(double));
        double *cs = (double *)malloc(sizeof(double) * (size_t)m);
        double *sn = (double *)malloc(sizeof(double) * (size_t)m);
        double *g = (double *)malloc(sizeof(double) * (size_t)(m + 1));
        double *h = (double *)malloc(sizeof(double) * (size_t)(m + 1));
        double *y = (double *)malloc(sizeof(double) * (size_t)(m + 1));
        double *hh = (double *)malloc(sizeof(double) * (size_t)(m + 1));
        while (rel > tol && it < max_iter) {
            double beta = norm2(n, r);
            for (int64_t i = 0; i < n; ++i) V[i] = r[i] / beta;
            for (int k = 0; k <= m; ++k) g[k] = 0.0;
            g[0] = beta;
            int j, jdone = 0;
            for (j = 0; j < m && it < max_iter; ++j) {
                double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n, *w = V + (size_t)(j + 1) * n;
                precond(H, vj, zj);
                ++it;
                spmv64(A, zj, w);
                for (int k = 0; k <= j; ++k) h[k] = 0.0;
                for (int pass = 0; pass < 2; ++pass) {
                    for (int k = 0; k <= j; ++k) hh[k] = dot(n, V + (size_t)k * n, w);
                    for (int k = 0; k <= j; ++k) {
                        const double *vk = V + (size_t)k * n;
                        for (int64_t i = 0; i < n; ++i) w[i] = fma(-hh[k], vk[i], w[i]);
                        h[k] += hh[k];
                    }
                }
                double hn = norm2(n, w);
                h[j + 1] = hn;
                if (hn > 0.0) for (int64_t i = 0; i < n; ++i) w[i] = w[i] / hn;
                for (int k = 0; k < j; ++k) {
                    double t = cs[k] * h[k] + sn[k] * h[k + 1];
                    h[k + 1] = -sn[k] * h[k] + cs[k] * h[k + 1];
                    h[k] = t;
                }
                double den = sqrt(h[j] * h[j] + h[j + 1] * h[j + 1]);
                cs[j] = (den > 0.0) ? h[j] / den : 1.0;
                sn[j] = (den > 0.0) ? h[j + 1] / den : 0.0;
                h[j] = den;
                h[j + 1] = 0.0;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                for (int k = 0; k <= j; ++k) Hm[k * m + j] = h[k];
                double est = fabs(g[j + 1]) / bn;
                if (hist && nh < hist_cap) hist[nh++] = est;
                jdone = j + 1;
                if (est <= tol || hn == 0.0) { ++j; break; }
            }
            /* y = H^{-1} g (upper triangular, jdone x jdone) */
            for (int k = jdone - 1; k >= 0; --k) {
                double acc = g[k];
                for (int c = k + 1; c < jdone; ++c) acc -= Hm[k * m + c] * y[c];
                y[k] = acc / Hm[k * m + k];
            }
            for (int k = 0; k < jdone; ++k) {
                const double *zk = Z + (size_t)k * n;
                for (int64_t i = 0; i < n; ++i) x[i] = fma(y[k], zk[i], x[i]);
            }
            residual(A, b, x, r);
            rel = norm2(n, r) / bn;
            if (rel != rel) { status = ORA_ERR_NAN; break; }
        }
        free(V); free(Z); free(Hm); free(cs); free(sn); free(g); free(h); free(y); free(hh);
    }
    if (rel <= tol) status = ORA_OK;
    *iters = it;
    *final_rel = rel;
    free(b); free(r); free(e);
    (void)dot;
    return status;
}

/* ------------------------------------------------------------------------- */
/* Batched systems (a block-diagonal matrix with nseg systems): stationary      */
/* refinement x_q += (M^{-1} r)_q where every system q is tested on its own     */
/* relative residual and stops being updated once it is <= tol.               */
/* ------------------------------------------------------------------------- */
int ora_solve_batched(ohier *H, const double *b, double *x, double tol, int max_iter, int *iters, double *rel) {
    const ocsr *A = &H->lev[0].A;
    int64_t n = A->nr;
    int nseg = H->o.nseg;
    const int64_t *seg = H->lev[0].seg;
    if (nseg <= 0 || !seg) return ORA_ERR_ARG;
    double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *e = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *bn = (double *)malloc(sizeof(double) * (size_t)nseg);
    int *active = (int *)malloc(sizeof(int) * (size_t)nseg);
    for (int q = 0; q < nseg; ++q) {
        double t = 0.0;
        for (int64_t i = seg[q]; i < seg[q + 1]; ++i) t = fma(b[i], b[i], t);
        bn[q] = t > 0.0 ? sqrt(t) : 1.0;
        iters[q] = 0;
        active[q] = 1;
    }
    int status = ORA_OK;
    for (int it = 0;; ++it) {
        residual(A, b, x, r);
        int any = 0;
        for (int q = 0; q < nseg; ++q) {
            if (!active[q]) continue;
            double t = 0.0;
            for (int64_t i = seg[q]; i < seg[q + 1]; ++i) t = fma(r[i], r[i], t);
            rel[q] = sqrt(t) / bn[q];
            if (rel[q] != rel[q]) { status = ORA_ERR_NAN; active[q] = 0; continue; }
            if (rel[q] <= tol || it >= max_iter) active[q] = 0;
            else any = 1;
        }
        if (!any) break;
        precond(H, r, e);
        for (int q = 0; q < nseg; ++q) {
            if (!active[q]) continue;
            for (int64_t i = seg[q]; i < seg[q + 1]; ++i) x[i] += e[i];
            iters[q] += 1;
        }
    }
    for (int q = 0; q < nseg && status == ORA_OK; ++q)
        if (!(rel[q] <= tol)) status = ORA_ERR_NOT_CONVERGED;
    free(r); free(e); free(bn); free(active);
    return status;
}

/* Batched systems with FGMRES: every system q is solved on its own (FGMRES with  */
/* the block-diagonal hierarchy applied to vectors that vanish outside q, which   */
/* keeps them inside q), with its own restarts and stopping test.               */
int ora_solve_batched_fgmres(ohier *H, const double *b, double *x, double tol, int max_iter, int restart,
                             int *iters, double *rel) {
    const ocsr *A = &H->lev[0].A;
    int64_t n = A->nr;
    int nseg = H->o.nseg;
    const int64_t *seg = H->lev[0].seg;
    if (nseg <= 0 || !seg) return ORA_ERR_ARG;
    double *bq = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *xq = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    int status = ORA_OK;
    for (int q = 0; q < nseg; ++q) {
        memset(bq, 0, sizeof(double) * (size_t)n);
        memset(xq, 0, sizeof(double) * (size_t)n);
        for (int64_t i = seg[q]; i < seg[q + 1]; ++i) { bq[i] = b[i]; xq[i] = x[i]; }
        int it = 0;
        double r = 0.0;
        int st = ora_solve(H, bq, xq, tol, 1, max_iter, restart, &it, &r, NULL, 0);
        iters[q] = it;
        rel[q] = r;
        for (int64_t i = seg[q]; i < seg[q + 1]; ++i) x[i] = xq[i];
        if (st != ORA_OK && status == ORA_OK) status = st;
    }
    free(bq); free(xq);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Export for tests                                                           */
/* ------------------------------------------------------------------------- */
int ora_nlevels(const ohier *H) { return H->nlev; }
int64_t ora_singular_count(const ohier *H, int which) { return which ? H->singular_P : H->singular_R; }

/* info[0..7] = n, nnz(A), nc, nnz(R), nnz(P), has_cf, 0, 0 */
void ora_level_info(const ohier *H, int l, int64_t *info) {
    const olevel *L = &H->lev[l];
    info[0] = L->A.nr;
    info[1] = L->A.rp ? L->A.rp[L->A.nr] : 0;
    info[2] = L->cf ? L->nc : 0;
    info[3] = L->R.rp ? L->R.rp[L->R.nr] : 0;
    info[4] = L->P.rp ? L->P.rp[L->P.nr] : 0;
    info[5] = L->cf != NULL;
    info[6] = 0;
    info[7] = 0;
}

void ora_export_seg(const ohier *H, int l, int64_t *seg) {
    if (H->lev[l].seg) memcpy(seg, H->lev[l].seg, sizeof(int64_t) * (size_t)(H->o.nseg + 1));
}

/* which: 0 A, 1 R, 2 P */
void ora_export_csr(const ohier *H, int l, int which, int64_t *rp, int32_t *col, double *val) {
    const olevel *L = &H->lev[l];
    const ocsr *M = which == 0 ? &L->A : (which == 1 ? &L->R : &L->P);
    if (!M->rp) return;
    int64_t nnz = M->rp[M->nr];
    if (rp) memcpy(rp, M->rp, sizeof(int64_t) * (size_t)(M->nr + 1));
    if (col) memcpy(col, M->col, sizeof(int32_t) * (size_t)nnz);
    if (val) memcpy(val, M->val, sizeof(double) * (size_t)nnz);
}

void ora_export_cf(const ohier *H, int l, int8_t *cf, uint8_t *strong, uint8_t *ls_R, uint8_t *ls_P) {
    const olevel *L = &H->lev[l];
    int64_t n = L->A.nr;
    if (cf && L->cf) memcpy(cf, L->cf, (size_t)n);
    if (strong && L->strong) memcpy(strong, L->strong, (size_t)L->A.rp[n]);
    if (ls_R && L->ls_R) memcpy(ls_R, L->ls_R, (size_t)L->nc);
    if (ls_P && L->ls_P) memcpy(ls_P, L->ls_P, (size_t)L->nc);
}

/* stand-alone steps for the pins */
void ora_cf_split(int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *mask, int mode,
                  uint64_t seed, int8_t *cf) {
    ograph S, ST;
    graph_from_mask(n, rp, col, mask, &S);
    graph_transpose(&S, &ST);
    if (mode == 0) cf_rs(&S, &ST, cf);
    else if (mode == 1) cf_pmis(&S, &ST, seed, cf);
    else cf_rs_blocked(&S, &ST, (int64_t)seed, cf);   /* mode 3: blocked first pass, block size = seed */
    graph_free(&S); graph_free(&ST);
}

/* transpose of a CSR (used to set up the adjoint system A^T) */
int64_t ora_transpose(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                      int64_t *trp, int32_t *tcol, double *tval) {
    ocsr a = {n, n, (int64_t *)rp, (int32_t *)col, (double *)val}, t;
    csr_transpose(&a, &t);
    int64_t nnz = t.rp[n];
    memcpy(trp, t.rp, sizeof(int64_t) * (size_t)(n + 1));
    memcpy(tcol, t.col, sizeof(int32_t) * (size_t)nnz);
    memcpy(tval, t.val, sizeof(double) * (size_t)nnz);
    csr_free(&t);
    return nnz;
}

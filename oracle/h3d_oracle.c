/*
 * h3d_oracle.c -- TEST INFRASTRUCTURE, not part of the product.
 *
 * A plain, slow FP64 CPU statement of the HODLR3D kernel-matrix product of
 * Kandappan, Gujjula & Ambikasaran, "HODLR3D: Hierarchical matrices for N-body
 * problems in three dimensions" (arXiv 2307.16303).  It exists only to check the
 * CUDA library; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * What it computes, each part following the paper:
 *   - the kernel matrix K(i,j) = f(|r_i - r_j|), K(i,i) = 0        (Sec. 3.1, Eq. Laplace3D)
 *   - O1: the direct sum y = K x, O(N^2)                            (Eq. Laplace3D)
 *   - the uniform octree over the cube B, split until every leaf
 *     holds at most N_max points                                    (Sec. 2.1; Alg. 1)
 *   - vertex/edge/face neighbours, clan and interaction list        (Table "Notations")
 *   - HODLR3D admissibility: distinct same-level clusters that share
 *     nothing or only a vertex are compressed                       (Definition "admh3d")
 *   - the paper's comparison formats on the same octree: the H-matrix
 *     with the strong condition max(diam) <= eta dist, eta = sqrt(3)
 *     (Sec. 2.2, Eq. adm), and HODLR, which compresses every
 *     off-diagonal block (Sec. 2.3)
 *   - partially pivoted ACA of every admissible pair, giving pivots
 *     sigma (rows) and tau (columns) with
 *     K(X,Y) ~ K(X,tau) K(sigma,tau)^{-1} K(sigma,Y)                 (Sec. 4.1, Eq. prank)
 *   - O2: the HODLR3D matrix-vector product: dense self/edge/face
 *     blocks at the leaf level plus the low-rank blocks of every
 *     level                                                          (Alg. 2)
 *   - optional symmetric storage: the kernel is symmetric, so
 *     K(Y,X) = K(X,Y)^T; each unordered admissible pair {X, Y} is
 *     compressed once, as the block whose target has the smaller
 *     level-local index, and its mirror (Y, X) takes the transposed
 *     factors V U^T and the swapped pivots (tau, sigma)     (Eq. prank transposed)
 *
 * Readings where the paper is silent (all shared with the CUDA path by
 * specification only, not by code):
 *   - a leaf holds <= leaf_size points (Sec. 2.1 says "at most"); depth L <= 21;
 *   - Morton key: 21 bits per axis, x the most significant bit of each triple;
 *     points are ordered by (key, original index);
 *   - ix = min(floor(((x - lo) / side) * 2^21), 2^21 - 1), rejecting points
 *     outside [lo, lo + side];
 *   - a pair of distinct same-level boxes with integer offset d is
 *     W (well separated) if max|d| >= 2, else V/E/F by the number of
 *     non-zero components (3/2/1);
 *   - ACA: first pivot row is local row 0; the residual row of pivot row i is
 *     K(i,:) - sum_{l<k} U(i,l) V(:,l)^T accumulated with fma in l order; the
 *     column pivot is the largest |residual| among unused columns (ties -> the
 *     smallest index); a row whose residual vanishes on all unused columns is
 *     marked used and the smallest unused row is tried next; the next row pivot
 *     is the largest |U(:,k)| among unused rows (ties -> smallest index); the
 *     Frobenius norm of the approximant is updated with the cross terms and the
 *     iteration stops when |u_k| |v_k| <= tol |S_k|_F, or when k reaches
 *     min(m, n, rank_cap);
 *   - coincident distinct points get K = 0, as the diagonal does.
 *
 * Parity note: every function below is pinned by tests under tests/ against
 * closed forms, brute force and invariants (see the header of oracle.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { KER_LAPLACE = 0, KER_YUKAWA = 1, KER_INV_R4 = 2, KER_COS_R = 3 };
enum { ST_OK = 0, ST_ARG = 1, ST_DOMAIN = 2, ST_OOM = 3, ST_RANK = 5, ST_DEPTH = 8 };
enum { CLS_SELF = 0, CLS_FACE = 1, CLS_EDGE = 2, CLS_VERTEX = 3, CLS_FAR = 4 };
enum { ADM_HODLR3D = 0, ADM_STRONG = 1, ADM_WEAK = 2 };

/* Is a pair of distinct same-level boxes of class `cls` admissible?
 *   HODLR3D (Def. admh3d): they share no boundary or only a vertex.
 *   strong (Eq. adm with eta = sqrt(3)): two cubes of side h have diameter
 *     h sqrt(3), so the condition holds iff dist >= h, i.e. no shared boundary.
 *   weak (HODLR): every off-diagonal pair.                                   */
static int admissible(int cls, int mode)
{
    switch (mode) {
    case ADM_STRONG: return cls == CLS_FAR;
    case ADM_WEAK:   return cls != CLS_SELF;
    default:         return cls == CLS_VERTEX || cls == CLS_FAR;
    }
}

#define MAX_DEPTH 21

/* 1 / (4 pi), written out to more digits than a double holds. */
static const double ORC_ONE_OVER_FOUR_PI = 0.0795774715459476678844418816863;

/* ------------------------------------------------------------------------- */
/* Kernel function f(r) of Eq. Laplace3D; zero for the diagonal and for r = 0. */
static double kernel_f(int kind, double kappa, const double *a, const double *b)
{
    double dx = a[0] - b[0];
    double dy = a[1] - b[1];
    double dz = a[2] - b[2];
    double d2 = fma(dz, dz, fma(dy, dy, dx * dx));
    double r;
    if (d2 == 0.0) return 0.0;
    r = sqrt(d2);
    switch (kind) {
    case KER_LAPLACE: return ORC_ONE_OVER_FOUR_PI / r;
    case KER_YUKAWA:  return (ORC_ONE_OVER_FOUR_PI * exp(-kappa * r)) / r;
    case KER_INV_R4:  return 1.0 / (d2 * d2);
    case KER_COS_R:   return cos(r) / r;
    default:          return NAN;
    }
}

double h3do_kernel(int kind, double kappa, const double *a, const double *b)
{
    return kernel_f(kind, kappa, a, b);
}

/* ------------------------------------------------------------------------- */
/* O1: direct sum y_i = sum_{j != i} K(i,j) x_j, compensated (Neumaier) in j
 * order.  x, y: N x nrhs column-major, user order.                          */
static void direct_row(int kind, double kappa, const double *pts, int64_t N,
                       const double *x, int nrhs, int64_t i, double *out /* nrhs */)
{
    for (int c = 0; c < nrhs; ++c) {
        double s = 0.0, comp = 0.0;
        const double *xc = x + (size_t)c * (size_t)N;
        for (int64_t j = 0; j < N; ++j) {
            double term, t;
            if (j == i) continue;
            term = kernel_f(kind, kappa, pts + 3 * i, pts + 3 * j) * xc[j];
            t = s + term;
            if (fabs(s) >= fabs(term)) comp += (s - t) + term;
            else comp += (term - t) + s;
            s = t;
        }
        out[c] = s + comp;
    }
}

int h3do_direct(int kind, double kappa, const double *pts, int64_t N,
                const double *x, int nrhs, double *y)
{
    if (N < 0 || nrhs < 1 || (N > 0 && (!pts || !x || !y))) return ST_ARG;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < N; ++i) {
        double tmp[64];
        for (int c0 = 0; c0 < nrhs; c0 += 64) {
            int nc = nrhs - c0 < 64 ? nrhs - c0 : 64;
            direct_row(kind, kappa, pts, N, x + (size_t)c0 * (size_t)N, nc, i, tmp);
            for (int c = 0; c < nc; ++c) y[(size_t)(c0 + c) * (size_t)N + i] = tmp[c];
        }
    }
    return ST_OK;
}

/* Rows subset: y_rows[c * nrows + r] = (K x)_{rows[r]}. */
int h3do_direct_rows(int kind, double kappa, const double *pts, int64_t N,
                     const double *x, int nrhs, const int64_t *rows, int64_t nrows,
                     double *y_rows)
{
    if (N < 0 || nrhs < 1 || nrows < 0) return ST_ARG;
    for (int64_t r = 0; r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= N) return ST_ARG;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nrows; ++r) {
        double tmp[64];
        for (int c0 = 0; c0 < nrhs; c0 += 64) {
            int nc = nrhs - c0 < 64 ? nrhs - c0 : 64;
            direct_row(kind, kappa, pts, N, x + (size_t)c0 * (size_t)N, nc, rows[r], tmp);
            for (int c = 0; c < nc; ++c) y_rows[(size_t)(c0 + c) * (size_t)nrows + r] = tmp[c];
        }
    }
    return ST_OK;
}

int h3do_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Morton keys (Sec. 2.1: recursive 8-way subdivision of the cube B).         */
static uint64_t spread3(uint64_t v)
{
    /* place bit b of v at bit 3b */
    uint64_t out = 0;
    for (int b = 0; b < MAX_DEPTH; ++b) out |= ((v >> b) & 1ull) << (3 * b);
    return out;
}

int h3do_morton(const double *pts, int64_t N, const double *lo, double side, uint64_t *keys)
{
    const double scale = 2097152.0; /* 2^21 */
    if (!(side > 0.0) || !isfinite(side)) return ST_ARG;
    for (int64_t i = 0; i < N; ++i) {
        uint64_t c[3];
        for (int d = 0; d < 3; ++d) {
            double t = (pts[3 * i + d] - lo[d]) / side;
            double u;
            if (!(t >= 0.0 && t <= 1.0)) return ST_DOMAIN;
            u = floor(t * scale);
            c[d] = (uint64_t)u;
            if (c[d] > 2097151ull) c[d] = 2097151ull;
        }
        keys[i] = (spread3(c[0]) << 2) | (spread3(c[1]) << 1) | spread3(c[2]);
    }
    return ST_OK;
}

/* ------------------------------------------------------------------------- */
/* Tree and lists.                                                           */
typedef struct {
    int64_t n_blocks;     /* admissible pairs over all levels (I-lists)        */
    int *blk_level, *blk_tgt, *blk_src, *blk_cls;   /* level-local box indices */
    int64_t n_near;       /* self/edge/face pairs at the leaf level            */
    int *near_tgt, *near_src, *near_cls;
} lists_t;

typedef struct {
    int kind;
    double kappa, tol, lo[3], side;
    int leaf_size, rank_cap, adm;
    int64_t N;
    int L;
    double *pts;          /* sorted points, N x 3                               */
    int64_t *perm;        /* perm[s] = original index of sorted point s         */
    uint64_t *keys;       /* sorted keys                                        */
    int nbox[MAX_DEPTH + 1];
    int64_t box_off[MAX_DEPTH + 2];   /* level l boxes at [box_off[l], box_off[l+1]) */
    uint64_t *box_key;    /* Morton prefix of the box at its level              */
    int64_t *box_start, *box_end;
    lists_t lists;
    /* compression results (pivots only, as the paper stores them) */
    int have_pivots;
    int *rank;            /* per block                                          */
    int64_t *piv_off;     /* per block, into sigma/tau                          */
    int *sigma, *tau;     /* local row / column indices                         */
    int64_t n_piv;
    /* symmetric storage: partner[b] = index of the block (src, tgt) of b's level */
    int sym;
    int64_t *partner;
} h3do_t;

typedef struct { uint64_t key; int64_t idx; } kv_t;

static int kv_cmp(const void *a, const void *b)
{
    const kv_t *p = (const kv_t *)a, *q = (const kv_t *)b;
    if (p->key < q->key) return -1;
    if (p->key > q->key) return 1;
    return (p->idx > q->idx) - (p->idx < q->idx);
}

static void box_coords(uint64_t prefix, int level, int *bx, int *by, int *bz)
{
    int x = 0, y = 0, z = 0;
    for (int b = 0; b < level; ++b) {
        uint64_t t = (prefix >> (3 * b)) & 7ull;
        x |= (int)((t >> 2) & 1ull) << b;
        y |= (int)((t >> 1) & 1ull) << b;
        z |= (int)(t & 1ull) << b;
    }
    *bx = x; *by = y; *bz = z;
}

/* Class of two same-level boxes from their integer coordinates. */
static int pair_class(const int *a, const int *b)
{
    int d[3], mx = 0, nz = 0;
    for (int k = 0; k < 3; ++k) {
        d[k] = abs(a[k] - b[k]);
        if (d[k] > mx) mx = d[k];
        if (d[k] != 0) ++nz;
    }
    if (mx >= 2) return CLS_FAR;
    return nz; /* 0 self, 1 face, 2 edge, 3 vertex */
}

typedef struct { int *v; int64_t n, cap; } ivec;
static int ivec_push(ivec *a, int x)
{
    if (a->n == a->cap) {
        int64_t nc = a->cap ? 2 * a->cap : 1024;
        int *nv = (int *)realloc(a->v, (size_t)nc * sizeof(int));
        if (!nv) return ST_OOM;
        a->v = nv; a->cap = nc;
    }
    a->v[a->n++] = x;
    return ST_OK;
}

static int build_lists(h3do_t *h)
{
    ivec bl = {0}, bt = {0}, bs = {0}, bc = {0}, nt = {0}, ns = {0}, nc = {0};
    int st = ST_OK;
    for (int l = 1; l <= h->L && st == ST_OK; ++l) {
        int nb = h->nbox[l];
        int64_t o = h->box_off[l];
        int *co = (int *)malloc((size_t)nb * 3 * sizeof(int));
        if (!co) return ST_OOM;
        for (int i = 0; i < nb; ++i) box_coords(h->box_key[o + i], l, co + 3 * i, co + 3 * i + 1, co + 3 * i + 2);
        for (int i = 0; i < nb && st == ST_OK; ++i) {
            int pi[3] = {co[3 * i] >> 1, co[3 * i + 1] >> 1, co[3 * i + 2] >> 1};
            for (int j = 0; j < nb && st == ST_OK; ++j) {
                int pj[3], pc, cls;
                if (j == i) continue;
                pj[0] = co[3 * j] >> 1; pj[1] = co[3 * j + 1] >> 1; pj[2] = co[3 * j + 2] >> 1;
                pc = pair_class(pi, pj);
                /* pairs whose parents were admissible are covered by a coarser
                 * block; for HODLR3D the rest is the clan: siblings and children
                 * of the parent's edge / face neighbours (Table Notations) */
                if (admissible(pc, h->adm)) continue;
                cls = pair_class(co + 3 * i, co + 3 * j);
                if (admissible(cls, h->adm)) {
                    st |= ivec_push(&bl, l); st |= ivec_push(&bt, i);
                    st |= ivec_push(&bs, j); st |= ivec_push(&bc, cls);
                }
            }
        }
        free(co);
    }
    /* leaf level: self, face and edge neighbours stay dense (Alg. 2) */
    if (st == ST_OK) {
        int l = h->L, nb = h->nbox[l];
        int64_t o = h->box_off[l];
        int *co = (int *)malloc((size_t)(nb > 0 ? nb : 1) * 3 * sizeof(int));
        if (!co) return ST_OOM;
        for (int i = 0; i < nb; ++i) box_coords(h->box_key[o + i], l, co + 3 * i, co + 3 * i + 1, co + 3 * i + 2);
        for (int i = 0; i < nb && st == ST_OK; ++i)
            for (int j = 0; j < nb && st == ST_OK; ++j) {
                int cls = pair_class(co + 3 * i, co + 3 * j);
                if (cls == CLS_SELF || !admissible(cls, h->adm)) {
                    st |= ivec_push(&nt, i); st |= ivec_push(&ns, j); st |= ivec_push(&nc, cls);
                }
            }
        free(co);
    }
    h->lists.n_blocks = bl.n;
    h->lists.blk_level = bl.v; h->lists.blk_tgt = bt.v; h->lists.blk_src = bs.v; h->lists.blk_cls = bc.v;
    h->lists.n_near = nt.n;
    h->lists.near_tgt = nt.v; h->lists.near_src = ns.v; h->lists.near_cls = nc.v;
    return st == ST_OK ? ST_OK : ST_OOM;
}

void h3do_free(h3do_t *h)
{
    if (!h) return;
    free(h->pts); free(h->perm); free(h->keys);
    free(h->box_key); free(h->box_start); free(h->box_end);
    free(h->lists.blk_level); free(h->lists.blk_tgt); free(h->lists.blk_src); free(h->lists.blk_cls);
    free(h->lists.near_tgt); free(h->lists.near_src); free(h->lists.near_cls);
    free(h->rank); free(h->piv_off); free(h->sigma); free(h->tau);
    free(h->partner);
    free(h);
}

/* Build the tree (Alg. 1, first two steps): keys, order, depth, boxes, lists. */
h3do_t *h3do_create_adm(const double *pts, int64_t N, int kind, double kappa, int leaf_size,
                        double tol, int rank_cap, const double *lo, double side, int adm, int *status);

h3do_t *h3do_create(const double *pts, int64_t N, int kind, double kappa, int leaf_size,
                    double tol, int rank_cap, const double *lo, double side, int *status)
{
    return h3do_create_adm(pts, N, kind, kappa, leaf_size, tol, rank_cap, lo, side, ADM_HODLR3D, status);
}

h3do_t *h3do_create_adm(const double *pts, int64_t N, int kind, double kappa, int leaf_size,
                        double tol, int rank_cap, const double *lo, double side, int adm, int *status)
{
    h3do_t *h;
    kv_t *kv = NULL;
    uint64_t *keys = NULL;
    int st = ST_OK;
    *status = ST_ARG;
    if (N < 1 || leaf_size < 1 || !(tol >= 0.0) || rank_cap < 1 || kind < 0 || kind > 3) return NULL;
    if (adm < 0 || adm > 2) return NULL;
    h = (h3do_t *)calloc(1, sizeof(h3do_t));
    if (!h) { *status = ST_OOM; return NULL; }
    h->adm = adm;
    h->kind = kind; h->kappa = kappa; h->tol = tol; h->leaf_size = leaf_size; h->rank_cap = rank_cap;
    h->N = N; h->side = side;
    for (int d = 0; d < 3; ++d) h->lo[d] = lo[d];
    keys = (uint64_t *)malloc((size_t)N * sizeof(uint64_t));
    kv = (kv_t *)malloc((size_t)N * sizeof(kv_t));
    h->pts = (double *)malloc((size_t)N * 3 * sizeof(double));
    h->perm = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    h->keys = (uint64_t *)malloc((size_t)N * sizeof(uint64_t));
    if (!keys || !kv || !h->pts || !h->perm || !h->keys) { st = ST_OOM; goto fail; }
    st = h3do_morton(pts, N, lo, side, keys);
    if (st != ST_OK) goto fail;
    for (int64_t i = 0; i < N; ++i) { kv[i].key = keys[i]; kv[i].idx = i; }
    qsort(kv, (size_t)N, sizeof(kv_t), kv_cmp);
    for (int64_t s = 0; s < N; ++s) {
        h->perm[s] = kv[s].idx;
        h->keys[s] = kv[s].key;
        for (int d = 0; d < 3; ++d) h->pts[3 * s + d] = pts[3 * kv[s].idx + d];
    }
    /* depth: the first level at which no box holds more than leaf_size points */
    h->L = -1;
    for (int l = 0; l <= MAX_DEPTH; ++l) {
        int shift = 3 * (MAX_DEPTH - l);
        int64_t run = 1, best = 1;
        for (int64_t s = 1; s < N; ++s) {
            if ((h->keys[s] >> shift) == (h->keys[s - 1] >> shift)) ++run; else run = 1;
            if (run > best) best = run;
        }
        if (best <= leaf_size) { h->L = l; break; }
    }
    if (h->L < 0) { st = ST_DEPTH; goto fail; }
    /* non-empty boxes of every level, in Morton order */
    {
        int64_t total = 0;
        for (int l = 0; l <= h->L; ++l) {
            int shift = 3 * (MAX_DEPTH - l);
            int64_t cnt = 1;
            for (int64_t s = 1; s < N; ++s)
                if ((h->keys[s] >> shift) != (h->keys[s - 1] >> shift)) ++cnt;
            h->nbox[l] = (int)cnt;
            h->box_off[l] = total;
            total += cnt;
        }
        h->box_off[h->L + 1] = total;
        h->box_key = (uint64_t *)malloc((size_t)total * sizeof(uint64_t));
        h->box_start = (int64_t *)malloc((size_t)total * sizeof(int64_t));
        h->box_end = (int64_t *)malloc((size_t)total * sizeof(int64_t));
        if (!h->box_key || !h->box_start || !h->box_end) { st = ST_OOM; goto fail; }
        for (int l = 0; l <= h->L; ++l) {
            int shift = 3 * (MAX_DEPTH - l);
            int64_t b = h->box_off[l];
            h->box_key[b] = h->keys[0] >> shift;
            h->box_start[b] = 0;
            for (int64_t s = 1; s < N; ++s) {
                if ((h->keys[s] >> shift) != (h->keys[s - 1] >> shift)) {
                    h->box_end[b] = s;
                    ++b;
                    h->box_key[b] = h->keys[s] >> shift;
                    h->box_start[b] = s;
                }
            }
            h->box_end[b] = N;
        }
    }
    st = build_lists(h);
    if (st != ST_OK) goto fail;
    free(kv); free(keys);
    *status = ST_OK;
    return h;
fail:
    free(kv); free(keys);
    h3do_free(h);
    *status = st;
    return NULL;
}

int h3do_depth(const h3do_t *h) { return h->L; }
int64_t h3do_num_blocks(const h3do_t *h) { return h->lists.n_blocks; }
int64_t h3do_num_near(const h3do_t *h) { return h->lists.n_near; }
int64_t h3do_num_boxes(const h3do_t *h) { return h->box_off[h->L + 1]; }

/* Tree export: perm, sorted keys, per-level box counts and (key, start, end). */
void h3do_export_tree(const h3do_t *h, int64_t *perm, uint64_t *keys, int *nbox,
                      uint64_t *box_key, int64_t *box_start, int64_t *box_end)
{
    int64_t nb = h->box_off[h->L + 1];
    memcpy(perm, h->perm, (size_t)h->N * sizeof(int64_t));
    memcpy(keys, h->keys, (size_t)h->N * sizeof(uint64_t));
    for (int l = 0; l <= h->L; ++l) nbox[l] = h->nbox[l];
    memcpy(box_key, h->box_key, (size_t)nb * sizeof(uint64_t));
    memcpy(box_start, h->box_start, (size_t)nb * sizeof(int64_t));
    memcpy(box_end, h->box_end, (size_t)nb * sizeof(int64_t));
}

void h3do_export_lists(const h3do_t *h, int *blk_level, int *blk_tgt, int *blk_src, int *blk_cls,
                       int *near_tgt, int *near_src, int *near_cls)
{
    size_t nb = (size_t)h->lists.n_blocks, nn = (size_t)h->lists.n_near;
    memcpy(blk_level, h->lists.blk_level, nb * sizeof(int));
    memcpy(blk_tgt, h->lists.blk_tgt, nb * sizeof(int));
    memcpy(blk_src, h->lists.blk_src, nb * sizeof(int));
    memcpy(blk_cls, h->lists.blk_cls, nb * sizeof(int));
    memcpy(near_tgt, h->lists.near_tgt, nn * sizeof(int));
    memcpy(near_src, h->lists.near_src, nn * sizeof(int));
    memcpy(near_cls, h->lists.near_cls, nn * sizeof(int));
}

/* ------------------------------------------------------------------------- */
/* ACA (Sec. 4.1).  X = sorted rows [xs, xs+m), Y = sorted columns [ys, ys+n).
 * U: m x cap, V: n x cap, column-major.  If frozen_k >= 0 the pivots are taken
 * from fr_sigma/fr_tau instead of being searched, and exactly frozen_k terms
 * are formed; the arithmetic that forms U and V is the same in both modes.
 * Returns the rank in *k_out and the pivots in sig/tau (cap entries).        */
static int aca_block(const h3do_t *h, int64_t xs, int m, int64_t ys, int n, int cap,
                     int frozen_k, const int *fr_sigma, const int *fr_tau,
                     double *U, double *V, int *k_out, int *sig, int *tau)
{
    const double *P = h->pts;
    unsigned char *urow = (unsigned char *)calloc((size_t)m, 1);
    unsigned char *ucol = (unsigned char *)calloc((size_t)n, 1);
    double S2 = 0.0;
    int k = 0, i = 0, st = ST_OK, converged = 0;
    if (!urow || !ucol) { free(urow); free(ucol); return ST_OOM; }
    if (frozen_k >= 0) i = frozen_k > 0 ? fr_sigma[0] : 0;
    for (;;) {
        int jstar = -1;
        double best = -1.0, delta;
        double *Vk = V + (size_t)k * (size_t)n;
        double *Uk = U + (size_t)k * (size_t)m;
        if (frozen_k >= 0 ? (k == frozen_k) : (k == cap)) break;
        /* residual of row i */
        for (int j = 0; j < n; ++j) {
            double r = kernel_f(h->kind, h->kappa, P + 3 * (xs + i), P + 3 * (ys + j));
            for (int l = 0; l < k; ++l) r = fma(-U[(size_t)l * m + i], V[(size_t)l * n + j], r);
            Vk[j] = r;
        }
        urow[i] = 1;
        if (frozen_k >= 0) {
            jstar = fr_tau[k];
        } else {
            for (int j = 0; j < n; ++j) {
                double a = fabs(Vk[j]);
                if (!ucol[j] && a > best) { best = a; jstar = j; }
            }
            if (jstar < 0 || best == 0.0) {
                /* residual row vanishes: try the smallest unused row */
                int nxt = -1;
                for (int r = 0; r < m; ++r) if (!urow[r]) { nxt = r; break; }
                if (nxt < 0) { converged = 1; break; }  /* every row used: block reproduced */
                i = nxt;
                continue;
            }
        }
        delta = Vk[jstar];
        for (int j = 0; j < n; ++j) Vk[j] = Vk[j] / delta;
        ucol[jstar] = 1;
        /* residual of column jstar */
        for (int r = 0; r < m; ++r) {
            double u = kernel_f(h->kind, h->kappa, P + 3 * (xs + r), P + 3 * (ys + jstar));
            for (int l = 0; l < k; ++l) u = fma(-V[(size_t)l * n + jstar], U[(size_t)l * m + r], u);
            Uk[r] = u;
        }
        sig[k] = i;
        tau[k] = jstar;
        ++k;
        if (frozen_k >= 0) {
            if (k < frozen_k) i = fr_sigma[k];
            continue;
        }
        /* stopping test on the Frobenius norm of the approximant */
        {
            double nu2 = 0.0, nv2 = 0.0, cross = 0.0;
            for (int r = 0; r < m; ++r) nu2 += Uk[r] * Uk[r];
            for (int j = 0; j < n; ++j) nv2 += Vk[j] * Vk[j];
            for (int l = 0; l < k - 1; ++l) {
                double du = 0.0, dv = 0.0;
                for (int r = 0; r < m; ++r) du += U[(size_t)l * m + r] * Uk[r];
                for (int j = 0; j < n; ++j) dv += V[(size_t)l * n + j] * Vk[j];
                cross += du * dv;
            }
            S2 = S2 + 2.0 * cross + nu2 * nv2;
            if (S2 < 0.0) S2 = 0.0;
            if (sqrt(nu2) * sqrt(nv2) <= h->tol * sqrt(S2)) { converged = 1; break; }
        }
        /* next row pivot: largest |U(:,k)| among unused rows */
        {
            int nxt = -1;
            double bu = -1.0;
            for (int r = 0; r < m; ++r) {
                double a = fabs(Uk[r]);
                if (!urow[r] && a > bu) { bu = a; nxt = r; }
            }
            if (nxt < 0) { converged = 1; break; }
            i = nxt;
        }
    }
    if (frozen_k < 0 && !converged && cap < (m < n ? m : n)) st = ST_RANK;
    free(urow); free(ucol);
    *k_out = k;
    return st;
}

/* Which block (X,Y) geometry: sorted ranges. */
static void block_ranges(const h3do_t *h, int64_t b, int64_t *xs, int *m, int64_t *ys, int *n)
{
    int l = h->lists.blk_level[b];
    int64_t ti = h->box_off[l] + h->lists.blk_tgt[b];
    int64_t si = h->box_off[l] + h->lists.blk_src[b];
    *xs = h->box_start[ti]; *m = (int)(h->box_end[ti] - h->box_start[ti]);
    *ys = h->box_start[si]; *n = (int)(h->box_end[si] - h->box_start[si]);
}

static int block_cap(const h3do_t *h, int m, int n)
{
    int c = m < n ? m : n;
    return c < h->rank_cap ? c : h->rank_cap;
}

/* Symmetric storage.  A block (X, Y) is a mirror when its target's level-local
 * index exceeds its source's; its partner is the block (Y, X), which the
 * admissibility relation (symmetric in X and Y) always contains.            */
static int is_mirror(const h3do_t *h, int64_t b)
{
    return h->sym && h->lists.blk_tgt[b] > h->lists.blk_src[b];
}

/* Blocks are listed in (level, target, source) order: binary search. */
static int64_t find_block(const h3do_t *h, int l, int t, int s)
{
    int64_t lo = 0, hi = h->lists.n_blocks;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int ml = h->lists.blk_level[mid], mt = h->lists.blk_tgt[mid], ms = h->lists.blk_src[mid];
        if (ml < l || (ml == l && (mt < t || (mt == t && ms < s)))) lo = mid + 1;
        else hi = mid;
    }
    if (lo < h->lists.n_blocks && h->lists.blk_level[lo] == l && h->lists.blk_tgt[lo] == t &&
        h->lists.blk_src[lo] == s)
        return lo;
    return -1;
}

/* Switch symmetric storage on (before any compression or frozen pivots). */
int h3do_set_symmetric(h3do_t *h, int on)
{
    int64_t nb = h->lists.n_blocks;
    if (h->have_pivots) return ST_ARG;
    free(h->partner);
    h->partner = NULL;
    h->sym = 0;
    if (!on) return ST_OK;
    h->partner = (int64_t *)malloc((size_t)(nb > 0 ? nb : 1) * sizeof(int64_t));
    if (!h->partner) return ST_OOM;
    for (int64_t b = 0; b < nb; ++b) {
        h->partner[b] = find_block(h, h->lists.blk_level[b], h->lists.blk_src[b], h->lists.blk_tgt[b]);
        if (h->partner[b] < 0) { free(h->partner); h->partner = NULL; return ST_ARG; }
    }
    h->sym = 1;
    return ST_OK;
}

/* Alg. 1: compress every admissible block, keeping ranks and pivots only
 * (symmetric storage: the primary block of each pair; its mirror takes the
 * same rank and the swapped pivots).                                        */
int h3do_compress(h3do_t *h)
{
    int64_t nb = h->lists.n_blocks;
    int *rk = (int *)malloc((size_t)(nb > 0 ? nb : 1) * sizeof(int));
    int **sg = (int **)calloc((size_t)(nb > 0 ? nb : 1), sizeof(int *));
    int **ta = (int **)calloc((size_t)(nb > 0 ? nb : 1), sizeof(int *));
    int st = ST_OK;
    if (!rk || !sg || !ta) { free(rk); free(sg); free(ta); return ST_OOM; }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < nb; ++b) {
        int64_t xs, ys; int m, n, cap, k = 0, s;
        double *U, *V;
        if (is_mirror(h, b)) { rk[b] = 0; continue; }
        block_ranges(h, b, &xs, &m, &ys, &n);
        cap = block_cap(h, m, n);
        U = (double *)malloc((size_t)m * cap * sizeof(double));
        V = (double *)malloc((size_t)n * cap * sizeof(double));
        sg[b] = (int *)malloc((size_t)cap * sizeof(int));
        ta[b] = (int *)malloc((size_t)cap * sizeof(int));
        if (!U || !V || !sg[b] || !ta[b]) s = ST_OOM;
        else s = aca_block(h, xs, m, ys, n, cap, -1, NULL, NULL, U, V, &k, sg[b], ta[b]);
        rk[b] = k;
        free(U); free(V);
        if (s != ST_OK) {
#pragma omp critical
            { if (st == ST_OK) st = s; }
        }
    }
    if (st == ST_OK) {
        int64_t tot = 0;
        free(h->rank); free(h->piv_off); free(h->sigma); free(h->tau);
        h->rank = rk;
        for (int64_t b = 0; b < nb; ++b)
            if (is_mirror(h, b)) rk[b] = rk[h->partner[b]];
        h->piv_off = (int64_t *)malloc((size_t)(nb + 1) * sizeof(int64_t));
        for (int64_t b = 0; b < nb; ++b) { h->piv_off[b] = tot; tot += rk[b]; }
        h->piv_off[nb] = tot;
        h->sigma = (int *)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(int));
        h->tau = (int *)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(int));
        for (int64_t b = 0; b < nb; ++b) {
            if (is_mirror(h, b)) {   /* rows of the mirror are the primary's columns */
                int64_t p = h->partner[b];
                memcpy(h->sigma + h->piv_off[b], ta[p], (size_t)rk[b] * sizeof(int));
                memcpy(h->tau + h->piv_off[b], sg[p], (size_t)rk[b] * sizeof(int));
            } else {
                memcpy(h->sigma + h->piv_off[b], sg[b], (size_t)rk[b] * sizeof(int));
                memcpy(h->tau + h->piv_off[b], ta[b], (size_t)rk[b] * sizeof(int));
            }
        }
        h->n_piv = tot;
        h->have_pivots = 1;
    } else {
        free(rk);
    }
    for (int64_t b = 0; b < nb; ++b) { free(sg[b]); free(ta[b]); }
    free(sg); free(ta);
    return st;
}

int64_t h3do_num_pivots(const h3do_t *h) { return h->have_pivots ? h->n_piv : -1; }

int h3do_get_pivots(const h3do_t *h, int *rank, int *sigma, int *tau)
{
    if (!h->have_pivots) return ST_ARG;
    memcpy(rank, h->rank, (size_t)h->lists.n_blocks * sizeof(int));
    memcpy(sigma, h->sigma, (size_t)h->n_piv * sizeof(int));
    memcpy(tau, h->tau, (size_t)h->n_piv * sizeof(int));
    return ST_OK;
}

/* Freeze pivots found elsewhere (e.g. by another implementation): afterwards
 * every factor is formed from exactly these pivots.                          */
int h3do_set_pivots(h3do_t *h, const int *rank, const int *sigma, const int *tau)
{
    int64_t nb = h->lists.n_blocks, tot = 0;
    for (int64_t b = 0; b < nb; ++b) {
        int64_t xs, ys; int m, n;
        block_ranges(h, b, &xs, &m, &ys, &n);
        if (rank[b] < 0 || rank[b] > (m < n ? m : n)) return ST_ARG;
        for (int k = 0; k < rank[b]; ++k)
            if (sigma[tot + k] < 0 || sigma[tot + k] >= m || tau[tot + k] < 0 || tau[tot + k] >= n) return ST_ARG;
        tot += rank[b];
    }
    if (h->sym) {   /* a mirror must carry its primary's rank and swapped pivots */
        int64_t *off = (int64_t *)malloc((size_t)(nb + 1) * sizeof(int64_t));
        int bad = 0;
        if (!off) return ST_OOM;
        off[0] = 0;
        for (int64_t b = 0; b < nb; ++b) off[b + 1] = off[b] + rank[b];
        for (int64_t b = 0; b < nb && !bad; ++b) {
            int64_t p = h->partner[b];
            if (!is_mirror(h, b)) continue;
            if (rank[b] != rank[p]) { bad = 1; break; }
            for (int k = 0; k < rank[b]; ++k)
                if (sigma[off[b] + k] != tau[off[p] + k] || tau[off[b] + k] != sigma[off[p] + k]) { bad = 1; break; }
        }
        free(off);
        if (bad) return ST_ARG;
    }
    free(h->rank); free(h->piv_off); free(h->sigma); free(h->tau);
    h->rank = (int *)malloc((size_t)(nb > 0 ? nb : 1) * sizeof(int));
    h->piv_off = (int64_t *)malloc((size_t)(nb + 1) * sizeof(int64_t));
    h->sigma = (int *)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(int));
    h->tau = (int *)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(int));
    if (!h->rank || !h->piv_off || !h->sigma || !h->tau) return ST_OOM;
    tot = 0;
    for (int64_t b = 0; b < nb; ++b) { h->rank[b] = rank[b]; h->piv_off[b] = tot; tot += rank[b]; }
    h->piv_off[nb] = tot;
    memcpy(h->sigma, sigma, (size_t)tot * sizeof(int));
    memcpy(h->tau, tau, (size_t)tot * sizeof(int));
    h->n_piv = tot;
    h->have_pivots = 1;
    return ST_OK;
}

/* Factors of one block from the stored pivots: U (m x r), V (n x r). */
int h3do_block_factors(const h3do_t *h, int64_t b, double *U, double *V)
{
    int64_t xs, ys; int m, n, k = 0, r;
    int *sg, *ta, st;
    if (!h->have_pivots || b < 0 || b >= h->lists.n_blocks) return ST_ARG;
    r = h->rank[b];
    sg = (int *)malloc((size_t)(r > 0 ? r : 1) * sizeof(int));
    ta = (int *)malloc((size_t)(r > 0 ? r : 1) * sizeof(int));
    if (is_mirror(h, b)) {
        /* K(Y,X) ~ (U_p V_p^T)^T: the primary's factors, U and V exchanged */
        int64_t p = h->partner[b];
        block_ranges(h, p, &xs, &m, &ys, &n);
        st = aca_block(h, xs, m, ys, n, r, r, h->sigma + h->piv_off[p], h->tau + h->piv_off[p],
                       V, U, &k, sg, ta);
    } else {
        block_ranges(h, b, &xs, &m, &ys, &n);
        st = aca_block(h, xs, m, ys, n, r, r, h->sigma + h->piv_off[b], h->tau + h->piv_off[b],
                       U, V, &k, sg, ta);
    }
    free(sg); free(ta);
    return st;
}

int h3do_block_geometry(const h3do_t *h, int64_t b, int64_t *xs, int *m, int64_t *ys, int *n)
{
    if (b < 0 || b >= h->lists.n_blocks) return ST_ARG;
    block_ranges(h, b, xs, m, ys, n);
    return ST_OK;
}

/* ------------------------------------------------------------------------- */
/* O2: Alg. 2, y = K~ x (transpose = 0) or y = K~^T x (transpose = 1).
 * x, y: N x nrhs column-major in the caller's point order.  Low-rank factors
 * are re-formed from the stored pivots block by block (the paper keeps only
 * pivots, Sec. 4.1), so memory stays small.                                  */
int h3do_apply(const h3do_t *h, const double *x, int nrhs, double *y, int transpose)
{
    const int64_t N = h->N;
    double *xs_ = NULL, *ys_ = NULL;
    int st = ST_OK;
    if (!h->have_pivots || nrhs < 1) return ST_ARG;
    xs_ = (double *)malloc((size_t)N * nrhs * sizeof(double));
    ys_ = (double *)calloc((size_t)N * nrhs, sizeof(double));
    if (!xs_ || !ys_) { free(xs_); free(ys_); return ST_OOM; }
    for (int c = 0; c < nrhs; ++c)
        for (int64_t s = 0; s < N; ++s) xs_[(size_t)c * N + s] = x[(size_t)c * N + h->perm[s]];

    /* dense self / edge / face blocks at the leaf level (Alg. 2, first loop);
     * each output row belongs to one target leaf, so leaves run in parallel. */
    {
        const int L = h->L;
        const int nb = h->nbox[L];
        const int64_t o = h->box_off[L];
        int64_t *first = (int64_t *)malloc((size_t)(nb + 1) * sizeof(int64_t));
        for (int i = 0; i <= nb; ++i) first[i] = -1;
        /* near pairs are grouped by target in increasing order */
        for (int64_t p = h->lists.n_near - 1; p >= 0; --p) first[h->lists.near_tgt[p]] = p;
#pragma omp parallel for schedule(dynamic, 4)
        for (int t = 0; t < nb; ++t) {
            int64_t p = first[t];
            if (p < 0) continue;
            for (; p < h->lists.n_near && h->lists.near_tgt[p] == t; ++p) {
                /* transpose: (Y,X) block applied as K(Y,X)^T = K(X,Y); near lists are symmetric */
                int s = h->lists.near_src[p];
                int64_t x0 = h->box_start[o + t], x1 = h->box_end[o + t];
                int64_t y0 = h->box_start[o + s], y1 = h->box_end[o + s];
                for (int64_t i = x0; i < x1; ++i)
                    for (int64_t j = y0; j < y1; ++j) {
                        double kij;
                        if (i == j) continue;
                        kij = transpose ? kernel_f(h->kind, h->kappa, h->pts + 3 * j, h->pts + 3 * i)
                                        : kernel_f(h->kind, h->kappa, h->pts + 3 * i, h->pts + 3 * j);
                        for (int c = 0; c < nrhs; ++c)
                            ys_[(size_t)c * N + i] += kij * xs_[(size_t)c * N + j];
                    }
            }
        }
        free(first);
    }

    /* low-rank blocks of every level (Alg. 2, second loop).  For the forward
     * product a target box owns its output rows; for the transpose a block
     * (X,Y) writes rows of Y, so blocks are grouped by source box instead.   */
    {
        int64_t nbk = h->lists.n_blocks;
        int64_t *order = (int64_t *)malloc((size_t)(nbk > 0 ? nbk : 1) * sizeof(int64_t));
        int64_t *grp = (int64_t *)malloc((size_t)(nbk + 1) * sizeof(int64_t));
        int64_t ngrp = 0;
        /* group key: (level, owner box) where owner = target (forward) or source (transpose) */
        for (int64_t b = 0; b < nbk; ++b) order[b] = b;
        if (transpose) {
            /* stable counting by (level, source) -- insertion into buckets */
            int64_t nboxes = h->box_off[h->L + 1];
            int64_t *cnt = (int64_t *)calloc((size_t)nboxes + 1, sizeof(int64_t));
            for (int64_t b = 0; b < nbk; ++b) cnt[h->box_off[h->lists.blk_level[b]] + h->lists.blk_src[b] + 1]++;
            for (int64_t q = 0; q < nboxes; ++q) cnt[q + 1] += cnt[q];
            for (int64_t b = 0; b < nbk; ++b) {
                int64_t key = h->box_off[h->lists.blk_level[b]] + h->lists.blk_src[b];
                order[cnt[key]++] = b;
            }
            free(cnt);
        }
        for (int64_t q = 0; q < nbk; ++q) {
            int64_t b = order[q];
            int l = h->lists.blk_level[b];
            int owner = transpose ? h->lists.blk_src[b] : h->lists.blk_tgt[b];
            if (q == 0) { grp[ngrp++] = 0; continue; }
            {
                int64_t pb = order[q - 1];
                int pl = h->lists.blk_level[pb];
                int po = transpose ? h->lists.blk_src[pb] : h->lists.blk_tgt[pb];
                if (pl != l || po != owner) grp[ngrp++] = q;
            }
        }
        grp[ngrp] = nbk;
        /* levels one after another (boxes of different levels share rows),
         * owner boxes of one level in parallel */
        for (int lev = 1; lev <= h->L; ++lev)
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t g = 0; g < ngrp; ++g) {
            if (h->lists.blk_level[order[grp[g]]] != lev) continue;
            for (int64_t q = grp[g]; q < grp[g + 1]; ++q) {
                int64_t b = order[q];
                int64_t x0, y0; int m, n, r = h->rank[b], s;
                double *U, *V, *t;
                block_ranges(h, b, &x0, &m, &y0, &n);
                if (r == 0) continue;
                U = (double *)malloc((size_t)m * r * sizeof(double));
                V = (double *)malloc((size_t)n * r * sizeof(double));
                t = (double *)malloc((size_t)r * sizeof(double));
                s = h3do_block_factors(h, b, U, V);
                if (s != ST_OK) {
#pragma omp critical
                    { if (st == ST_OK) st = s; }
                } else {
                    for (int c = 0; c < nrhs; ++c) {
                        const double *xc = xs_ + (size_t)c * N;
                        double *yc = ys_ + (size_t)c * N;
                        if (!transpose) {
                            /* y(X) += U (V^T x(Y)) */
                            for (int k = 0; k < r; ++k) {
                                double acc = 0.0;
                                for (int j = 0; j < n; ++j) acc += V[(size_t)k * n + j] * xc[y0 + j];
                                t[k] = acc;
                            }
                            for (int i = 0; i < m; ++i) {
                                double acc = 0.0;
                                for (int k = 0; k < r; ++k) acc += U[(size_t)k * m + i] * t[k];
                                yc[x0 + i] += acc;
                            }
                        } else {
                            /* y(Y) += V (U^T x(X)) */
                            for (int k = 0; k < r; ++k) {
                                double acc = 0.0;
                                for (int i = 0; i < m; ++i) acc += U[(size_t)k * m + i] * xc[x0 + i];
                                t[k] = acc;
                            }
                            for (int j = 0; j < n; ++j) {
                                double acc = 0.0;
                                for (int k = 0; k < r; ++k) acc += V[(size_t)k * n + j] * t[k];
                                yc[y0 + j] += acc;
                            }
                        }
                    }
                }
                free(U); free(V); free(t);
            }
        }
        free(order); free(grp);
    }
    for (int c = 0; c < nrhs; ++c)
        for (int64_t s = 0; s < N; ++s) y[(size_t)c * N + h->perm[s]] = ys_[(size_t)c * N + s];
    free(xs_); free(ys_);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Forces: the gradient with respect to the point positions of the energy
 *   E = 1/2 q^T K~ q,
 * where K~ holds the exact near blocks and, for every admissible block
 * (X, Y) with its pivots frozen, the cross (skeleton) form of Eq. prank,
 *   K(X,Y) ~ K(X,tau) M^{-1} K(sigma,Y),   M = K(sigma,tau).
 * With s = K(sigma,Y) q_Y, c = M^{-1} s, u = K(X,tau)^T q_X, a = M^{-T} u, the
 * block's energy 1/2 q_X^T K(X,tau) c has the differential
 *   1/2 [ q_X^T dK(X,tau) c + a^T dK(sigma,Y) q_Y - a^T dM c ]
 * (d(M^{-1}) = -M^{-1} dM M^{-1}).  Every kernel entry K(p_i, p_j) = f(|p_i - p_j|)
 * differentiates to  g = f'(rho) (p_i - p_j) / rho  for p_i and -g for p_j; the
 * near blocks contribute 1/2 q_i q_j K(p_i, p_j) for every ordered pair.  The
 * sums run serially in a fixed order.                                        */
static void kernel_grad(int kind, double kappa, const double *a, const double *b, double *g)
{
    double d[3] = {a[0] - b[0], a[1] - b[1], a[2] - b[2]};
    double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double r, fp;
    g[0] = g[1] = g[2] = 0.0;
    if (d2 == 0.0) return;
    r = sqrt(d2);
    switch (kind) {
    case KER_LAPLACE: fp = -ORC_ONE_OVER_FOUR_PI / d2; break;                                  /* f = 1/(4 pi r)       */
    case KER_YUKAWA:  fp = -ORC_ONE_OVER_FOUR_PI * exp(-kappa * r) * (1.0 + kappa * r) / d2; break;
    case KER_INV_R4:  fp = -4.0 / (d2 * d2 * r); break;                                        /* f = r^-4             */
    case KER_COS_R:   fp = -(r * sin(r) + cos(r)) / d2; break;                                 /* f = cos r / r        */
    default:          fp = NAN;
    }
    for (int k = 0; k < 3; ++k) g[k] = fp * d[k] / r;
}

/* Solve A z = rhs for an n x n row-major A by Gaussian elimination with
 * partial pivoting (A and rhs are overwritten).  Returns 0 on success.       */
static int dense_solve(int n, double *A, double *rhs)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (fabs(A[(size_t)i * n + k]) > fabs(A[(size_t)p * n + k])) p = i;
        if (A[(size_t)p * n + k] == 0.0) return 1;
        if (p != k) {
            for (int j = 0; j < n; ++j) {
                double t = A[(size_t)k * n + j]; A[(size_t)k * n + j] = A[(size_t)p * n + j]; A[(size_t)p * n + j] = t;
            }
            { double t = rhs[k]; rhs[k] = rhs[p]; rhs[p] = t; }
        }
        for (int i = k + 1; i < n; ++i) {
            double f = A[(size_t)i * n + k] / A[(size_t)k * n + k];
            for (int j = k; j < n; ++j) A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
            rhs[i] -= f * rhs[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = rhs[k];
        for (int j = k + 1; j < n; ++j) s -= A[(size_t)k * n + j] * rhs[j];
        rhs[k] = s / A[(size_t)k * n + k];
    }
    return 0;
}

/* E (scalar) and dE/dp (N x 3, row-major, the caller's point order) for charges
 * q (N, the caller's order); pivots must be present (compress or set_pivots). */
int h3do_energy_forces(const h3do_t *h, const double *q, double *E_out, double *grad)
{
    const int64_t N = h->N;
    const int kind = h->kind;
    const double kap = h->kappa;
    double *qs, *G, E = 0.0;
    if (!h->have_pivots) return ST_ARG;
    qs = (double *)malloc((size_t)N * sizeof(double));
    G = (double *)calloc((size_t)N * 3, sizeof(double));
    if (!qs || !G) { free(qs); free(G); return ST_OOM; }
    for (int64_t s = 0; s < N; ++s) qs[s] = q[h->perm[s]];

    /* near blocks: every ordered pair (i, j), i != j, of each near pair of leaves */
    {
        const int64_t o = h->box_off[h->L];
        for (int64_t p = 0; p < h->lists.n_near; ++p) {
            int64_t t = o + h->lists.near_tgt[p], sb = o + h->lists.near_src[p];
            for (int64_t i = h->box_start[t]; i < h->box_end[t]; ++i)
                for (int64_t j = h->box_start[sb]; j < h->box_end[sb]; ++j) {
                    double g[3], w;
                    if (i == j) continue;
                    w = 0.5 * qs[i] * qs[j];
                    E += w * kernel_f(kind, kap, h->pts + 3 * i, h->pts + 3 * j);
                    kernel_grad(kind, kap, h->pts + 3 * i, h->pts + 3 * j, g);
                    for (int k = 0; k < 3; ++k) { G[3 * i + k] += w * g[k]; G[3 * j + k] -= w * g[k]; }
                }
        }
    }
    /* admissible blocks in the cross form */
    for (int64_t b = 0; b < h->lists.n_blocks; ++b) {
        int64_t x0, y0;
        int m, n, r = h->rank[b];
        const int *sg = h->sigma + h->piv_off[b], *ta = h->tau + h->piv_off[b];
        double *M, *Mt, *c, *a, g[3];
        if (r == 0) continue;
        block_ranges(h, b, &x0, &m, &y0, &n);
        M = (double *)malloc((size_t)r * r * sizeof(double));
        Mt = (double *)malloc((size_t)r * r * sizeof(double));
        c = (double *)malloc((size_t)r * sizeof(double));
        a = (double *)malloc((size_t)r * sizeof(double));
        for (int k = 0; k < r; ++k) {
            double sk = 0.0, uk = 0.0;
            for (int j = 0; j < n; ++j) sk += kernel_f(kind, kap, h->pts + 3 * (x0 + sg[k]), h->pts + 3 * (y0 + j)) * qs[y0 + j];
            for (int i = 0; i < m; ++i) uk += qs[x0 + i] * kernel_f(kind, kap, h->pts + 3 * (x0 + i), h->pts + 3 * (y0 + ta[k]));
            c[k] = sk;
            a[k] = uk;
            for (int l = 0; l < r; ++l) {
                double v = kernel_f(kind, kap, h->pts + 3 * (x0 + sg[k]), h->pts + 3 * (y0 + ta[l]));
                M[(size_t)k * r + l] = v;
                Mt[(size_t)l * r + k] = v;
            }
        }
        if (dense_solve(r, M, c) || dense_solve(r, Mt, a)) {
            free(M); free(Mt); free(c); free(a); free(qs); free(G);
            return ST_RANK;
        }
        for (int i = 0; i < m; ++i) {        /* q_X^T K(X,tau) c: energy and first term */
            for (int k = 0; k < r; ++k) {
                const double *pi = h->pts + 3 * (x0 + i), *pk = h->pts + 3 * (y0 + ta[k]);
                double w = 0.5 * qs[x0 + i] * c[k];
                E += w * kernel_f(kind, kap, pi, pk);
                kernel_grad(kind, kap, pi, pk, g);
                for (int d = 0; d < 3; ++d) { G[3 * (x0 + i) + d] += w * g[d]; G[3 * (y0 + ta[k]) + d] -= w * g[d]; }
            }
        }
        for (int k = 0; k < r; ++k)          /* a^T dK(sigma,Y) q_Y */
            for (int j = 0; j < n; ++j) {
                const double *pk = h->pts + 3 * (x0 + sg[k]), *pj = h->pts + 3 * (y0 + j);
                double w = 0.5 * a[k] * qs[y0 + j];
                kernel_grad(kind, kap, pk, pj, g);
                for (int d = 0; d < 3; ++d) { G[3 * (x0 + sg[k]) + d] += w * g[d]; G[3 * (y0 + j) + d] -= w * g[d]; }
            }
        for (int k = 0; k < r; ++k)          /* - a^T dM c */
            for (int l = 0; l < r; ++l) {
                const double *pk = h->pts + 3 * (x0 + sg[k]), *pl = h->pts + 3 * (y0 + ta[l]);
                double w = -0.5 * a[k] * c[l];
                kernel_grad(kind, kap, pk, pl, g);
                for (int d = 0; d < 3; ++d) { G[3 * (x0 + sg[k]) + d] += w * g[d]; G[3 * (y0 + ta[l]) + d] -= w * g[d]; }
            }
        free(M); free(Mt); free(c); free(a);
    }
    for (int64_t s = 0; s < N; ++s)
        for (int d = 0; d < 3; ++d) grad[3 * h->perm[s] + d] = G[3 * s + d];
    *E_out = E;
    free(qs); free(G);
    return ST_OK;
}

/* Exact forces of the dense energy E = 1/2 q^T K q on selected points:
 * F_i = -dE/dp_i = -sum_{j != i} q_i q_j f'(|p_i - p_j|) (p_i - p_j) / |p_i - p_j|,
 * points and charges in the caller's order, out: nrows x 3.                  */
int h3do_direct_forces_rows(int kind, double kappa, const double *pts, int64_t N, const double *q,
                            const int64_t *rows, int64_t nrows, double *out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t i = rows[r];
        double acc[3] = {0.0, 0.0, 0.0}, g[3];
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            kernel_grad(kind, kappa, pts + 3 * i, pts + 3 * j, g);
            for (int d = 0; d < 3; ++d) acc[d] += q[j] * g[d];
        }
        for (int d = 0; d < 3; ++d) out[3 * r + d] = -q[i] * acc[d];
    }
    return ST_OK;
}

/* ------------------------------------------------------------------------- */
/* The skeleton form of the product (the paper's own storage, Sec. 4.1: only
 * the pivots and K(sigma,tau) are kept): y = near + sum over admissible blocks
 * of K(X,tau) K(sigma,tau)^{-1} K(sigma,Y) x_Y, each block evaluated from
 * kernel entries with a dense solve; with transpose = 1 the transposed operator,
 * y_Y += K(sigma,Y)^T K(sigma,tau)^{-T} K(X,tau)^T x_X (the near blocks are
 * symmetric).  x, y: N values, the caller's order.                           */
int h3do_apply_skeleton(const h3do_t *h, const double *x, double *y, int transpose)
{
    const int64_t N = h->N;
    double *xs_, *ys_;
    if (!h->have_pivots) return ST_ARG;
    xs_ = (double *)malloc((size_t)N * sizeof(double));
    ys_ = (double *)calloc((size_t)N, sizeof(double));
    if (!xs_ || !ys_) { free(xs_); free(ys_); return ST_OOM; }
    for (int64_t s = 0; s < N; ++s) xs_[s] = x[h->perm[s]];
    {   /* near blocks */
        const int64_t o = h->box_off[h->L];
        for (int64_t p = 0; p < h->lists.n_near; ++p) {
            int64_t t = o + h->lists.near_tgt[p], sb = o + h->lists.near_src[p];
            for (int64_t i = h->box_start[t]; i < h->box_end[t]; ++i)
                for (int64_t j = h->box_start[sb]; j < h->box_end[sb]; ++j)
                    if (i != j) ys_[i] += kernel_f(h->kind, h->kappa, h->pts + 3 * i, h->pts + 3 * j) * xs_[j];
        }
    }
    for (int64_t b = 0; b < h->lists.n_blocks; ++b) {
        int64_t x0, y0;
        int m, n, r = h->rank[b];
        const int *sg = h->sigma + h->piv_off[b], *ta = h->tau + h->piv_off[b];
        double *M, *c;
        if (r == 0) continue;
        block_ranges(h, b, &x0, &m, &y0, &n);
        M = (double *)malloc((size_t)r * r * sizeof(double));
        c = (double *)malloc((size_t)r * sizeof(double));
        if (!transpose) {
            for (int k = 0; k < r; ++k) {
                double sk = 0.0;
                for (int j = 0; j < n; ++j) sk += kernel_f(h->kind, h->kappa, h->pts + 3 * (x0 + sg[k]), h->pts + 3 * (y0 + j)) * xs_[y0 + j];
                c[k] = sk;
                for (int l = 0; l < r; ++l)
                    M[(size_t)k * r + l] = kernel_f(h->kind, h->kappa, h->pts + 3 * (x0 + sg[k]), h->pts + 3 * (y0 + ta[l]));
            }
        } else {   /* M^T a = K(X,tau)^T x_X */
            for (int k = 0; k < r; ++k) {
                double uk = 0.0;
                for (int i = 0; i < m; ++i) uk += kernel_f(h->kind, h->kappa, h->pts + 3 * (x0 + i), h->pts + 3 * (y0 + ta[k])) * xs_[x0 + i];
                c[k] = uk;
                for (int l = 0; l < r; ++l)
                    M[(size_t)k * r + l] = kernel_f(h->kind, h->kappa, h->pts + 3 * (x0 + sg[l]), h->pts + 3 * (y0 + ta[k]));
            }
        }
        if (dense_solve(r, M, c)) { free(M); free(c); free(xs_); free(ys_); return ST_RANK; }
        if (!transpose) {
            for (int i = 0; i < m; ++i) {
                double acc = 0.0;
                for (int k = 0; k < r; ++k) acc += kernel_f(h->kind, h->kappa, h->pts + 3 * (x0 + i), h->pts + 3 * (y0 + ta[k])) * c[k];
                ys_[x0 + i] += acc;
            }
        } else {
            for (int j = 0; j < n; ++j) {
                double acc = 0.0;
                for (int k = 0; k < r; ++k) acc += kernel_f(h->kind, h->kappa, h->pts + 3 * (x0 + sg[k]), h->pts + 3 * (y0 + j)) * c[k];
                ys_[y0 + j] += acc;
            }
        }
        free(M); free(c);
    }
    for (int64_t s = 0; s < N; ++s) y[h->perm[s]] = ys_[s];
    free(xs_); free(ys_);
    return ST_OK;
}

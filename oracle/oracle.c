/*
 * oracle.c -- reference implementation used ONLY as test infrastructure.
 *
 * Plain, slow, obviously-correct FP64 CPU code for what the supernodal
 * right-looking Cholesky computes (Karsavuran, Ng, Peyton, Peyton,
 * "Some new techniques to use in serial sparse Cholesky factorization
 * algorithms", arXiv 2409.13090). Only the tests, the package's smoke check
 * and the benchmark's CPU-baseline leg may load this library; the product
 * path never does. It shares no code with the CUDA path.
 *
 * Contents, each following the passage cited beside it:
 *   - geometric nested dissection on a grid (stand-in for METIS, Sec. 3.1);
 *   - symbolic factorization by the column union of Sec. 2.1.2:
 *       glbind(j) = {j} U {i > j : A_ij != 0} U  U_{c: p(c)=j} (glbind(c) \ {c}),
 *       elimination-tree parent p(j) = min(glbind(j) \ {j})   (Sec. 2.1.2);
 *   - postorder of the elimination tree (children visited in ascending order);
 *   - fundamental supernodes: j and p(j) share a supernode iff
 *       glbind(j)\{j} = glbind(p(j)) and j is the only child of p(j) (Sec. 2.1.2);
 *   - supernodal parent p(J) (Sec. 2.1.2);
 *   - partition-refinement reordering within supernodes (Sec. 1, Fig. 2; the
 *     reading of the cited PR method is stated in or_pr_partition below);
 *   - relind(J, p(J)): distance of each row from the bottom of glbind(p(J))
 *     (Sec. 2.1.2), blocks of J and relindB(J, P) (Sec. 2.2.2, Alg. 5), all
 *     computed by direct (binary) search of glbind(P) -- no composition;
 *   - numeric factorization by the column Cholesky of Algorithm 1 (Sec. 2.1.1):
 *     scatter, cmod from the left, gather, cdiv;
 *   - forward and backward triangular solves (Sec. 1, step 4);
 *   - the normwise backward error
 *       eta = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)   per column.
 *
 * Indices are 0-based; relative indices are 0-based distances from the bottom.
 * Parity: the symbolic pass is pinned by the paper's worked example (Figs. 1-3,
 * Sec. 2.1.2, Sec. 2.2.2) and by closed forms; the numeric factor by dense
 * Cholesky on small matrices and by ||A - L L^T|| / ||A||.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG -1
#define OR_ERR_NOMEM -2
#define OR_ERR_INTERNAL -3

typedef struct {
    int64_t n;
    /* final ordering: perm[new] = old, iperm[old] = new */
    int32_t *perm, *iperm;
    /* permuted lower pattern of A (CSC, final ordering) and the value map:
       amap[p] = index into the user's values array for entry p */
    int64_t *acolptr;
    int32_t *arowind;
    int64_t *amap;
    /* per-column structure of L (final ordering) */
    int64_t *ccolptr;
    int32_t *crows;
    int32_t *cparent;
    /* supernodes */
    int64_t nsuper;
    int32_t *sup_ptr;    /* nsuper+1, first column of each supernode */
    int32_t *sup_parent; /* -1 for roots */
    int32_t *sup_of;     /* column -> supernode */
    int64_t *gl_ptr;     /* nsuper+1 */
    int32_t *glbind;
    int64_t *ri_ptr; /* nsuper+1, relind(J,p(J)) has |S_J| entries */
    int32_t *relind;
    int64_t *blk_ptr; /* nsuper+1 */
    int32_t *blk_first, *blk_size, *blk_owner;
    int64_t *rb_pair_ptr; /* nsuper+1 */
    int32_t *rb_pair_P;
    int64_t *rb_val_ptr; /* npairs+1 */
    int32_t *rb_val;
    int32_t *level;
    int64_t nnzL, nblocks, npairs;
    double flops; /* sum over columns of |L_{*,j}|^2 */
    /* numeric: values of L per column, aligned with crows */
    double *lval;
} or_sym;

/* ------------------------------------------------------------------------ */
/* small helpers                                                            */

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static void *xmalloc(size_t n) { return malloc(n ? n : 1); }

/* position of value v in the ascending list a[0..len), or -1 */
static int64_t find_pos(const int32_t *a, int64_t len, int32_t v) {
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return (lo < len && a[lo] == v) ? lo : -1;
}
static void *xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s ? s : 1); }

/* ------------------------------------------------------------------------ */
/* Geometric nested dissection (stand-in for METIS nested dissection, Sec. 3.1).
 * Box [lo,hi) per axis. If the volume is <= leaf, emit its points in
 * lexicographic order (x fastest). Otherwise split the longest axis (ties:
 * x before y before z) at m = lo + (hi-lo)/2: order = left box [lo,m),
 * right box [m+1,hi), then the separator plane at m.                       */

static void nd_rec(int nx, int ny, int x0, int x1, int y0, int y1, int z0, int z1, int leaf,
                   int32_t *out, int64_t *pos) {
    int lx = x1 - x0, ly = y1 - y0, lz = z1 - z0;
    if (lx <= 0 || ly <= 0 || lz <= 0) return;
    int64_t vol = (int64_t)lx * ly * lz;
    if (vol <= leaf) {
        for (int z = z0; z < z1; z++)
            for (int y = y0; y < y1; y++)
                for (int x = x0; x < x1; x++) out[(*pos)++] = x + nx * (y + ny * z);
        return;
    }
    int axis = 0, len = lx;
    if (ly > len) { axis = 1; len = ly; }
    if (lz > len) { axis = 2; len = lz; }
    if (axis == 0) {
        int m = x0 + lx / 2;
        nd_rec(nx, ny, x0, m, y0, y1, z0, z1, leaf, out, pos);
        nd_rec(nx, ny, m + 1, x1, y0, y1, z0, z1, leaf, out, pos);
        nd_rec(nx, ny, m, m + 1, y0, y1, z0, z1, 0x7fffffff, out, pos);
    } else if (axis == 1) {
        int m = y0 + ly / 2;
        nd_rec(nx, ny, x0, x1, y0, m, z0, z1, leaf, out, pos);
        nd_rec(nx, ny, x0, x1, m + 1, y1, z0, z1, leaf, out, pos);
        nd_rec(nx, ny, x0, x1, m, m + 1, z0, z1, 0x7fffffff, out, pos);
    } else {
        int m = z0 + lz / 2;
        nd_rec(nx, ny, x0, x1, y0, y1, z0, m, leaf, out, pos);
        nd_rec(nx, ny, x0, x1, y0, y1, m + 1, z1, leaf, out, pos);
        nd_rec(nx, ny, x0, x1, y0, y1, m, m + 1, 0x7fffffff, out, pos);
    }
}

/* perm[new] = old */
int or_nd_grid(int nx, int ny, int nz, int leaf, int32_t *perm) {
    if (nx <= 0 || ny <= 0 || nz <= 0 || leaf < 1 || !perm) return OR_ERR_ARG;
    int64_t pos = 0;
    nd_rec(nx, ny, 0, nx, 0, ny, 0, nz, leaf, perm, &pos);
    return pos == (int64_t)nx * ny * nz ? OR_OK : OR_ERR_INTERNAL;
}

/* ------------------------------------------------------------------------ */
/* Permuted lower pattern: entry (r, c) of A (r >= c) lands at
 * (max(iperm[r], iperm[c]), min(...)) of A_hat = P A P^T.                  */

static int permute_pattern(int64_t n, const int64_t *colptr, const int32_t *rowind,
                           const int32_t *iperm, int64_t **pcp, int32_t **pri, int64_t **pmap) {
    int64_t nnz = colptr[n];
    int64_t *cp = xcalloc(n + 1, sizeof(int64_t));
    int32_t *ri = xmalloc(nnz * sizeof(int32_t));
    int64_t *mp = xmalloc(nnz * sizeof(int64_t));
    int64_t *fill = xmalloc((n + 1) * sizeof(int64_t));
    if (!cp || !ri || !mp || !fill) return OR_ERR_NOMEM;
    for (int64_t c = 0; c < n; c++)
        for (int64_t p = colptr[c]; p < colptr[c + 1]; p++) {
            int32_t a = iperm[rowind[p]], b = iperm[c];
            int32_t col = a < b ? a : b;
            cp[col + 1]++;
        }
    for (int64_t c = 0; c < n; c++) cp[c + 1] += cp[c];
    memcpy(fill, cp, (n + 1) * sizeof(int64_t));
    for (int64_t c = 0; c < n; c++)
        for (int64_t p = colptr[c]; p < colptr[c + 1]; p++) {
            int32_t a = iperm[rowind[p]], b = iperm[c];
            int32_t col = a < b ? a : b, row = a < b ? b : a;
            int64_t q = fill[col]++;
            ri[q] = row;
            mp[q] = p;
        }
    /* sort each column by row (insertion sort on (row, map) pairs) */
    for (int64_t c = 0; c < n; c++) {
        for (int64_t p = cp[c] + 1; p < cp[c + 1]; p++) {
            int32_t r = ri[p];
            int64_t m = mp[p];
            int64_t q = p - 1;
            while (q >= cp[c] && ri[q] > r) {
                ri[q + 1] = ri[q];
                mp[q + 1] = mp[q];
                q--;
            }
            ri[q + 1] = r;
            mp[q + 1] = m;
        }
    }
    free(fill);
    *pcp = cp;
    *pri = ri;
    *pmap = mp;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Symbolic factorization by the column union (Sec. 2.1.2):
 *   glbind(j) = {j} U {i > j : A_ij != 0} U  U_{c : p(c) = j} (glbind(c) \ {c})
 *   p(j) = min(glbind(j) \ {j}), or -1 if glbind(j) = {j}.
 * Output: per-column sorted row lists and the elimination-tree parent.      */

static int symbolic_union(int64_t n, const int64_t *acp, const int32_t *ari, int64_t **pccp,
                          int32_t **pcrows, int32_t **pparent) {
    int64_t cap = acp[n] + n + 16;
    int32_t *rows = xmalloc(cap * sizeof(int32_t));
    int64_t *ccp = xcalloc(n + 1, sizeof(int64_t));
    int32_t *parent = xmalloc(n * sizeof(int32_t));
    int32_t *mark = xmalloc(n * sizeof(int32_t));
    int32_t *tmp = xmalloc(n * sizeof(int32_t));
    /* children lists (linked, ascending: appended at the tail) */
    int32_t *head = xmalloc(n * sizeof(int32_t));
    int32_t *tail = xmalloc(n * sizeof(int32_t));
    int32_t *next = xmalloc(n * sizeof(int32_t));
    if (!rows || !ccp || !parent || !mark || !tmp || !head || !tail || !next) return OR_ERR_NOMEM;
    for (int64_t j = 0; j < n; j++) { mark[j] = -1; head[j] = -1; tail[j] = -1; }
    for (int64_t j = 0; j < n; j++) {
        int64_t cnt = 0;
        tmp[cnt++] = (int32_t)j;
        mark[j] = (int32_t)j;
        for (int64_t p = acp[j]; p < acp[j + 1]; p++) {
            int32_t i = ari[p];
            if (i > j && mark[i] != j) { mark[i] = (int32_t)j; tmp[cnt++] = i; }
        }
        for (int32_t c = head[j]; c != -1; c = next[c]) {
            for (int64_t p = ccp[c]; p < ccp[c + 1]; p++) {
                int32_t i = rows[p];
                if (i != c && mark[i] != j) { mark[i] = (int32_t)j; tmp[cnt++] = i; }
            }
        }
        qsort(tmp, cnt, sizeof(int32_t), cmp_i32);
        if (ccp[j] + cnt > cap) {
            while (ccp[j] + cnt > cap) cap *= 2;
            int32_t *nr = realloc(rows, cap * sizeof(int32_t));
            if (!nr) return OR_ERR_NOMEM;
            rows = nr;
        }
        memcpy(rows + ccp[j], tmp, cnt * sizeof(int32_t));
        ccp[j + 1] = ccp[j] + cnt;
        parent[j] = cnt > 1 ? tmp[1] : -1; /* min of glbind(j) \ {j} */
        if (parent[j] >= 0) {
            /* append j at the end of the parent's child list so children stay ascending */
            int32_t pj = parent[j];
            next[j] = -1;
            if (head[pj] == -1) head[pj] = (int32_t)j; else next[tail[pj]] = (int32_t)j;
            tail[pj] = (int32_t)j;
        }
    }
    free(mark); free(tmp); free(head); free(tail); free(next);
    *pccp = ccp;
    *pcrows = rows;
    *pparent = parent;
    return OR_OK;
}

/* Postorder: depth-first search from the roots in ascending order, visiting
 * children in ascending order; post[k] = the k-th vertex finished.          */
static void postorder(int64_t n, const int32_t *parent, int32_t *post) {
    int32_t *first = xmalloc(n * sizeof(int32_t)), *next = xmalloc(n * sizeof(int32_t));
    int32_t *stack = xmalloc(n * sizeof(int32_t)), *it = xmalloc(n * sizeof(int32_t));
    for (int64_t j = 0; j < n; j++) first[j] = -1;
    /* build child lists in ascending order by inserting in descending order at the head */
    for (int64_t j = n - 1; j >= 0; j--)
        if (parent[j] >= 0) { next[j] = first[parent[j]]; first[parent[j]] = (int32_t)j; }
    int64_t k = 0;
    for (int64_t r = 0; r < n; r++) {
        if (parent[r] != -1) continue;
        int64_t top = 0;
        stack[top] = (int32_t)r; it[top] = first[r]; top++;
        while (top > 0) {
            int32_t v = stack[top - 1];
            int32_t c = it[top - 1];
            if (c != -1) {
                it[top - 1] = next[c];
                stack[top] = c; it[top] = first[c]; top++;
            } else {
                post[k++] = v;
                top--;
            }
        }
    }
    free(first); free(next); free(stack); free(it);
}

/* ------------------------------------------------------------------------ */
/* Partition refinement within one supernode P (the PR method the paper cites
 * in Sec. 1 and Sec. 3.1; its steps are not printed there). Reading used here,
 * which reproduces Fig. 2 exactly:
 *   start from the ordered partition [P's columns, ascending];
 *   for each descendant J with R = S_J n P nonempty, in ascending supernode order:
 *     every part X with X n R and X \ R both nonempty is split into two adjacent
 *     parts; X n R goes last if R meets a part after X and no part before X,
 *     otherwise first; order inside a part stays ascending.
 * Output: order[k] = the (pre-PR) column placed at position k of P.          */

typedef struct { int32_t *cols; int32_t cnt; } part_t;

static int pr_partition(int32_t f, int32_t size, int32_t nsets, const int64_t *set_ptr,
                        const int32_t *set_rows, int32_t *order) {
    part_t *parts = xmalloc(sizeof(part_t) * (size_t)(size + 1));
    part_t *np = xmalloc(sizeof(part_t) * (size_t)(size + 1));
    char *inR = xcalloc(size, 1);
    int32_t nparts = 1;
    parts[0].cols = xmalloc(sizeof(int32_t) * size);
    parts[0].cnt = size;
    for (int32_t k = 0; k < size; k++) parts[0].cols[k] = f + k;
    for (int32_t s = 0; s < nsets; s++) {
        memset(inR, 0, size);
        for (int64_t p = set_ptr[s]; p < set_ptr[s + 1]; p++) inR[set_rows[p] - f] = 1;
        /* which parts meet R */
        char *meets = xcalloc(nparts, 1);
        for (int32_t q = 0; q < nparts; q++)
            for (int32_t k = 0; k < parts[q].cnt; k++)
                if (inR[parts[q].cols[k] - f]) { meets[q] = 1; break; }
        int32_t nn = 0;
        for (int32_t q = 0; q < nparts; q++) {
            int32_t nin = 0;
            for (int32_t k = 0; k < parts[q].cnt; k++) nin += inR[parts[q].cols[k] - f];
            if (nin == 0 || nin == parts[q].cnt) { np[nn++] = parts[q]; continue; }
            int before = 0, after = 0;
            for (int32_t t = 0; t < q; t++) before |= meets[t];
            for (int32_t t = q + 1; t < nparts; t++) after |= meets[t];
            part_t a, b; /* a = X n R, b = X \ R */
            a.cols = xmalloc(sizeof(int32_t) * nin);
            b.cols = xmalloc(sizeof(int32_t) * (parts[q].cnt - nin));
            a.cnt = b.cnt = 0;
            for (int32_t k = 0; k < parts[q].cnt; k++) {
                int32_t c = parts[q].cols[k];
                if (inR[c - f]) a.cols[a.cnt++] = c; else b.cols[b.cnt++] = c;
            }
            free(parts[q].cols);
            if (after && !before) { np[nn++] = b; np[nn++] = a; }
            else { np[nn++] = a; np[nn++] = b; }
        }
        free(meets);
        part_t *t = parts; parts = np; np = t;
        nparts = nn;
    }
    int32_t k = 0;
    for (int32_t q = 0; q < nparts; q++) {
        for (int32_t t = 0; t < parts[q].cnt; t++) order[k++] = parts[q].cols[t];
        free(parts[q].cols);
    }
    free(parts); free(np); free(inR);
    return k == size ? OR_OK : OR_ERR_INTERNAL;
}

/* ------------------------------------------------------------------------ */

static void free_cols(or_sym *s) {
    free(s->acolptr); free(s->arowind); free(s->amap);
    free(s->ccolptr); free(s->crows); free(s->cparent);
    s->acolptr = NULL; s->arowind = NULL; s->amap = NULL;
    s->ccolptr = NULL; s->crows = NULL; s->cparent = NULL;
}

/* Symbolic pass for ordering perm (new -> old): permuted pattern, column union. */
static int analyze_with(or_sym *s, int64_t n, const int64_t *colptr, const int32_t *rowind,
                        const int32_t *perm) {
    free_cols(s);
    for (int64_t k = 0; k < n; k++) { s->perm[k] = perm[k]; s->iperm[perm[k]] = (int32_t)k; }
    int rc = permute_pattern(n, colptr, rowind, s->iperm, &s->acolptr, &s->arowind, &s->amap);
    if (rc) return rc;
    return symbolic_union(n, s->acolptr, s->arowind, &s->ccolptr, &s->crows, &s->cparent);
}

/* ------------------------------------------------------------------------ */
/* Supernode merging (Sec. 3.1): repeatedly merge the child-parent pair whose
 * merge adds the least new fill, stopping before the cumulative growth of the
 * factor storage would exceed merge_frac of the fundamental storage.
 * Readings (the paper does not spell these out):
 *   - a pair (X, p(X)) is a candidate only when X's last column is the column
 *     just before p(X)'s first one, so merged supernodes stay consecutive;
 *   - storage of a supernode with w columns and m rows = w m - w (w - 1) / 2
 *     (its lower trapezoid); merging X into P gives w = |X| + |P| and
 *     m = |X| + m_P; new fill = storage(merged) - storage(X) - storage(P);
 *   - ties in new fill go to the child with the smaller first column;
 *   - a merge is allowed while (added fill so far + its fill) <= frac * S0,
 *     S0 = storage of the fundamental partition.
 * Uses a binary heap of (fill, first column, supernode, version) entries with
 * lazy invalidation.                                                          */

typedef struct { int64_t d; int32_t f, id, ver; } hent;

static int hless(const hent *a, const hent *b) { return a->d < b->d || (a->d == b->d && a->f < b->f); }

static void hpush(hent **h, int64_t *len, int64_t *cap, hent e) {
    if (*len == *cap) { *cap = *cap ? 2 * *cap : 1024; *h = realloc(*h, *cap * sizeof(hent)); }
    int64_t i = (*len)++;
    (*h)[i] = e;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!hless(&(*h)[i], &(*h)[p])) break;
        hent t = (*h)[i]; (*h)[i] = (*h)[p]; (*h)[p] = t;
        i = p;
    }
}

static hent hpop(hent *h, int64_t *len) {
    hent top = h[0];
    h[0] = h[--(*len)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < *len && hless(&h[l], &h[m])) m = l;
        if (r < *len && hless(&h[r], &h[m])) m = r;
        if (m == i) break;
        hent t = h[i]; h[i] = h[m]; h[m] = t;
        i = m;
    }
    return top;
}

static int64_t st_trap(int64_t w, int64_t m) { return w * m - w * (w - 1) / 2; }

/* new fill of merging X into P */
static int64_t merge_fill(int64_t wX, int64_t mX, int64_t wP, int64_t mP) {
    return st_trap(wX + wP, wX + mP) - st_trap(wX, mX) - st_trap(wP, mP);
}

static int merge_supernodes(or_sym *s, double frac, int32_t **top_out) {
    int64_t n = s->n, ns = s->nsuper;
    int32_t *f = xmalloc(ns * sizeof(int32_t)), *l = xmalloc(ns * sizeof(int32_t));
    int32_t *ftop = xmalloc(ns * sizeof(int32_t)), *minS = xmalloc(ns * sizeof(int32_t));
    int32_t *ver = xcalloc(ns, sizeof(int32_t)), *own = xmalloc(n * sizeof(int32_t));
    int64_t *m = xmalloc(ns * sizeof(int64_t));
    char *alive = xmalloc(ns);
    int64_t S0 = 0;
    for (int64_t X = 0; X < ns; X++) {
        f[X] = s->sup_ptr[X];
        l[X] = s->sup_ptr[X + 1] - 1;
        ftop[X] = f[X];
        m[X] = s->ccolptr[f[X] + 1] - s->ccolptr[f[X]];
        minS[X] = -1;
        for (int64_t p = s->ccolptr[f[X]]; p < s->ccolptr[f[X] + 1]; p++)
            if (s->crows[p] > l[X]) { minS[X] = s->crows[p]; break; }
        alive[X] = 1;
        for (int32_t j = f[X]; j <= l[X]; j++) own[j] = (int32_t)X;
        S0 += st_trap(l[X] - f[X] + 1, m[X]);
    }
    hent *h = NULL;
    int64_t hl = 0, hc = 0;
    for (int64_t X = 0; X < ns; X++) {
        if (minS[X] < 0) continue;
        int32_t P = own[minS[X]];
        if (l[X] + 1 != f[P]) continue;
        hent e = {merge_fill(l[X] - f[X] + 1, m[X], l[P] - f[P] + 1, m[P]), f[X], (int32_t)X, ver[X]};
        hpush(&h, &hl, &hc, e);
    }
    int64_t added = 0;
    while (hl > 0) {
        hent e = hpop(h, &hl);
        int32_t X = e.id;
        if (!alive[X] || e.ver != ver[X]) continue;
        int32_t P = own[minS[X]];
        if ((double)(added + e.d) > frac * (double)S0) break;
        /* merge X into P: P keeps its id, its last column and its rows below */
        added += e.d;
        m[P] = (l[X] - f[X] + 1) + m[P];
        for (int32_t j = f[X]; j <= l[X]; j++) own[j] = P;
        f[P] = f[X];
        alive[X] = 0;
        ver[P]++;
        /* P's own candidate with its parent */
        if (minS[P] >= 0) {
            int32_t Q = own[minS[P]];
            if (l[P] + 1 == f[Q]) {
                hent c = {merge_fill(l[P] - f[P] + 1, m[P], l[Q] - f[Q] + 1, m[Q]), f[P], P, ver[P]};
                hpush(&h, &hl, &hc, c);
            }
        }
        /* the child just before the merged supernode, if P is its parent */
        if (f[P] > 0) {
            int32_t C = own[f[P] - 1];
            if (alive[C] && minS[C] >= 0 && own[minS[C]] == P) {
                ver[C]++;
                hent c = {merge_fill(l[C] - f[C] + 1, m[C], l[P] - f[P] + 1, m[P]), f[C], C, ver[C]};
                hpush(&h, &hl, &hc, c);
            }
        }
    }
    /* surviving supernodes in column order */
    int64_t nn = 0;
    int32_t *top = xmalloc(ns * sizeof(int32_t));
    for (int64_t X = 0; X < ns; X++) {
        if (!alive[X]) continue;
        s->sup_ptr[nn] = f[X];
        top[nn] = ftop[X];
        nn++;
    }
    s->sup_ptr[nn] = (int32_t)n;
    s->nsuper = nn;
    for (int64_t J = 0; J < nn; J++)
        for (int32_t j = s->sup_ptr[J]; j < s->sup_ptr[J + 1]; j++) s->sup_of[j] = (int32_t)J;
    free(f); free(l); free(ftop); free(minS); free(ver); free(own); free(m); free(alive); free(h);
    *top_out = top;
    return OR_OK;
}

/* The top-level symbolic analysis.
 *   perm0: ordering to start from (new -> old), or NULL for the natural order;
 *   do_pr: apply partition refinement within supernodes;
 *   merge_frac: supernode merging budget (0 = fundamental supernodes only).   */
int or_analyze(int64_t n, const int64_t *colptr, const int32_t *rowind, const int32_t *perm0,
               int do_pr, double merge_frac, or_sym **out) {
    if (n <= 0 || !colptr || !rowind || !out) return OR_ERR_ARG;
    or_sym *s = xcalloc(1, sizeof(or_sym));
    s->n = n;
    s->perm = xmalloc(n * sizeof(int32_t));
    s->iperm = xmalloc(n * sizeof(int32_t));
    int32_t *p1 = xmalloc(n * sizeof(int32_t));
    for (int64_t k = 0; k < n; k++) p1[k] = perm0 ? perm0[k] : (int32_t)k;
    /* check the start ordering is a permutation */
    {
        char *seen = xcalloc(n, 1);
        for (int64_t k = 0; k < n; k++) {
            if (p1[k] < 0 || p1[k] >= n || seen[p1[k]]) { free(seen); return OR_ERR_ARG; }
            seen[p1[k]] = 1;
        }
        free(seen);
    }
    int rc = analyze_with(s, n, colptr, rowind, p1);
    if (rc) return rc;
    /* postorder the elimination tree and redo the symbolic pass in that order */
    int32_t *post = xmalloc(n * sizeof(int32_t));
    postorder(n, s->cparent, post);
    int32_t *p2 = xmalloc(n * sizeof(int32_t));
    for (int64_t k = 0; k < n; k++) p2[k] = p1[post[k]];
    rc = analyze_with(s, n, colptr, rowind, p2);
    if (rc) return rc;
    /* fundamental supernodes (Sec. 2.1.2): j joins p(j)'s supernode iff
       glbind(j)\{j} = glbind(p(j)) and j is p(j)'s only child.              */
    int32_t *nchild = xcalloc(n, sizeof(int32_t));
    for (int64_t j = 0; j < n; j++) if (s->cparent[j] >= 0) nchild[s->cparent[j]]++;
    int32_t *start = xmalloc((n + 1) * sizeof(int32_t));
    int64_t ns = 0;
    for (int64_t j = 0; j < n; j++) {
        int joins = 0;
        if (j > 0) {
            int64_t c = j - 1; /* candidate: column j-1 whose parent is j */
            if (s->cparent[c] == j && nchild[j] == 1) {
                int64_t lc = s->ccolptr[c + 1] - s->ccolptr[c];
                int64_t lj = s->ccolptr[j + 1] - s->ccolptr[j];
                if (lc == lj + 1 &&
                    memcmp(s->crows + s->ccolptr[c] + 1, s->crows + s->ccolptr[j],
                           lj * sizeof(int32_t)) == 0)
                    joins = 1;
            }
        }
        if (!joins) start[ns++] = (int32_t)j;
    }
    start[ns] = (int32_t)n;
    s->nsuper = ns;
    s->sup_ptr = xmalloc((ns + 1) * sizeof(int32_t));
    memcpy(s->sup_ptr, start, (ns + 1) * sizeof(int32_t));
    s->sup_of = xmalloc(n * sizeof(int32_t));
    for (int64_t J = 0; J < ns; J++)
        for (int32_t j = s->sup_ptr[J]; j < s->sup_ptr[J + 1]; j++) s->sup_of[j] = (int32_t)J;
    free(start); free(nchild); free(post);
    /* sum over columns of |L_{*,j}|^2 of the true (fundamental) structure */
    s->flops = 0.0;
    for (int64_t j = 0; j < n; j++) {
        double c = (double)(s->ccolptr[j + 1] - s->ccolptr[j]);
        s->flops += c * c;
    }
    /* optional supernode merging (Sec. 3.1); top[J] = the fundamental supernode
       whose rows below the diagonal block are the merged supernode's rows     */
    int32_t *top = NULL;
    if (merge_frac > 0.0) {
        rc = merge_supernodes(s, merge_frac, &top);
        if (rc) return rc;
        ns = s->nsuper;
    } else {
        top = xmalloc(ns * sizeof(int32_t));
        for (int64_t J = 0; J < ns; J++) top[J] = s->sup_ptr[J];
    }

    /* glbind(J) of the pre-PR (postordered) matrix: J's columns followed by the
       rows of column top[J]'s structure that lie below J's last column        */
    int64_t *gpre_ptr = xcalloc(ns + 1, sizeof(int64_t));
    for (int64_t J = 0; J < ns; J++) {
        int32_t f = s->sup_ptr[J], l = s->sup_ptr[J + 1] - 1, t = top[J];
        int64_t below = 0;
        for (int64_t p = s->ccolptr[t]; p < s->ccolptr[t + 1]; p++) below += s->crows[p] > l;
        gpre_ptr[J + 1] = gpre_ptr[J] + (l - f + 1) + below;
    }
    int32_t *gpre = xmalloc((gpre_ptr[ns] + 1) * sizeof(int32_t));
    for (int64_t J = 0; J < ns; J++) {
        int32_t f = s->sup_ptr[J], l = s->sup_ptr[J + 1] - 1, t = top[J];
        int64_t w = gpre_ptr[J];
        for (int32_t j = f; j <= l; j++) gpre[w++] = j;
        for (int64_t p = s->ccolptr[t]; p < s->ccolptr[t + 1]; p++)
            if (s->crows[p] > l) gpre[w++] = s->crows[p];
    }
    free(top);

    /* partition refinement within each supernode, on the pre-PR structure */
    int32_t *p3 = xmalloc(n * sizeof(int32_t));
    memcpy(p3, p2, n * sizeof(int32_t));
    if (do_pr) {
        /* for each supernode P: the descendants' sets R = S_J n P, ascending J */
        int64_t *cnt = xcalloc(ns + 1, sizeof(int64_t));
        for (int64_t J = 0; J < ns; J++) {
            int32_t l = s->sup_ptr[J + 1] - 1;
            int64_t p = gpre_ptr[J], e = gpre_ptr[J + 1];
            int32_t lastP = -1;
            for (; p < e; p++) {
                int32_t i = gpre[p];
                if (i <= l) continue;
                int32_t P = s->sup_of[i];
                if (P != lastP) { cnt[P + 1]++; lastP = P; }
            }
        }
        /* set lists per P */
        int64_t *sptr = xcalloc(ns + 1, sizeof(int64_t));
        for (int64_t P = 0; P < ns; P++) sptr[P + 1] = sptr[P] + cnt[P + 1];
        int64_t nsets = sptr[ns];
        int64_t *set_ptr_all = xcalloc(nsets + 1, sizeof(int64_t));
        /* first pass: sizes of each set */
        int64_t *fillp = xmalloc((ns + 1) * sizeof(int64_t));
        memcpy(fillp, sptr, (ns + 1) * sizeof(int64_t));
        int64_t *set_size = xcalloc(nsets + 1, sizeof(int64_t));
        for (int64_t J = 0; J < ns; J++) {
            int32_t l = s->sup_ptr[J + 1] - 1;
            int32_t lastP = -1;
            int64_t cur = -1;
            for (int64_t p = gpre_ptr[J]; p < gpre_ptr[J + 1]; p++) {
                int32_t i = gpre[p];
                if (i <= l) continue;
                int32_t P = s->sup_of[i];
                if (P != lastP) { cur = fillp[P]++; lastP = P; }
                set_size[cur]++;
            }
        }
        for (int64_t q = 0; q < nsets; q++) set_ptr_all[q + 1] = set_ptr_all[q] + set_size[q];
        int32_t *set_rows = xmalloc((set_ptr_all[nsets] + 1) * sizeof(int32_t));
        memcpy(fillp, sptr, (ns + 1) * sizeof(int64_t));
        int64_t *wpos = xmalloc((nsets + 1) * sizeof(int64_t));
        memcpy(wpos, set_ptr_all, (nsets + 1) * sizeof(int64_t));
        for (int64_t J = 0; J < ns; J++) {
            int32_t l = s->sup_ptr[J + 1] - 1;
            int32_t lastP = -1;
            int64_t cur = -1;
            for (int64_t p = gpre_ptr[J]; p < gpre_ptr[J + 1]; p++) {
                int32_t i = gpre[p];
                if (i <= l) continue;
                int32_t P = s->sup_of[i];
                if (P != lastP) { cur = fillp[P]++; lastP = P; }
                set_rows[wpos[cur]++] = i;
            }
        }
        int32_t *order = xmalloc(n * sizeof(int32_t));
        for (int64_t P = 0; P < ns; P++) {
            int32_t f = s->sup_ptr[P], size = s->sup_ptr[P + 1] - f;
            int32_t nsP = (int32_t)(sptr[P + 1] - sptr[P]);
            if (size < 2 || nsP == 0) continue;
            rc = pr_partition(f, size, nsP, set_ptr_all + sptr[P], set_rows, order);
            if (rc) return rc;
            /* position k of P receives the column that was at order[k] */
            for (int32_t k = 0; k < size; k++) p3[f + k] = p2[order[k]];
        }
        free(order); free(set_rows); free(wpos); free(set_size); free(fillp);
        free(set_ptr_all); free(sptr); free(cnt);
    }
    /* newlab[x] = label after PR of the column labelled x before PR */
    int32_t *newlab = xmalloc(n * sizeof(int32_t));
    {
        int32_t *ip2 = xmalloc(n * sizeof(int32_t));
        for (int64_t k = 0; k < n; k++) ip2[p2[k]] = (int32_t)k;
        for (int64_t k = 0; k < n; k++) newlab[ip2[p3[k]]] = (int32_t)k;
        free(ip2);
    }
    /* The supernode partition and every m_J are carried over; glbind(J) after PR is
       the relabelled pre-PR glbind(J), sorted ascending (Sec. 1, Figs. 1-2).   */
    s->gl_ptr = gpre_ptr;
    s->glbind = xmalloc((gpre_ptr[ns] + 1) * sizeof(int32_t));
    for (int64_t J = 0; J < ns; J++) {
        int64_t m = gpre_ptr[J + 1] - gpre_ptr[J];
        for (int64_t q = 0; q < m; q++) s->glbind[gpre_ptr[J] + q] = newlab[gpre[gpre_ptr[J] + q]];
        qsort(s->glbind + gpre_ptr[J], m, sizeof(int32_t), cmp_i32);
        int32_t f = s->sup_ptr[J];
        for (int64_t k = 0; k < s->sup_ptr[J + 1] - f; k++)
            if (s->glbind[gpre_ptr[J] + k] != f + k) return OR_ERR_INTERNAL;
    }
    free(gpre); free(newlab);
    /* the true column structure of the final ordering must lie inside the
       supernodal structure: reordering within supernodes adds no fill.       */
    rc = analyze_with(s, n, colptr, rowind, p3);
    if (rc) return rc;
    free(p1); free(p2); free(p3);
    int64_t *sccp = xcalloc(n + 1, sizeof(int64_t));
    for (int64_t J = 0; J < ns; J++)
        for (int32_t j = s->sup_ptr[J]; j < s->sup_ptr[J + 1]; j++)
            sccp[j + 1] = (s->gl_ptr[J + 1] - s->gl_ptr[J]) - (j - s->sup_ptr[J]);
    for (int64_t j = 0; j < n; j++) sccp[j + 1] += sccp[j];
    int32_t *scrows = xmalloc((sccp[n] + 1) * sizeof(int32_t));
    for (int64_t J = 0; J < ns; J++)
        for (int32_t j = s->sup_ptr[J]; j < s->sup_ptr[J + 1]; j++) {
            int64_t c = j - s->sup_ptr[J];
            memcpy(scrows + sccp[j], s->glbind + s->gl_ptr[J] + c, (sccp[j + 1] - sccp[j]) * sizeof(int32_t));
            /* every true row of column j appears in its supernodal list */
            for (int64_t p = s->ccolptr[j]; p < s->ccolptr[j + 1]; p++)
                if (find_pos(scrows + sccp[j], sccp[j + 1] - sccp[j], s->crows[p]) < 0) return OR_ERR_INTERNAL;
        }
    /* from here on, the column structures used by Algorithm 1 are the supernodal ones */
    free(s->ccolptr); free(s->crows);
    s->ccolptr = sccp;
    s->crows = scrows;
    s->nnzL = 0;
    for (int64_t j = 0; j < n; j++) s->nnzL += s->ccolptr[j + 1] - s->ccolptr[j];

    /* supernodal parent (Sec. 2.1.2): the supernode holding min{i in glbind(J), i > l} */
    s->sup_parent = xmalloc(ns * sizeof(int32_t));
    for (int64_t J = 0; J < ns; J++) {
        int32_t l = s->sup_ptr[J + 1] - 1;
        s->sup_parent[J] = -1;
        for (int64_t p = s->gl_ptr[J]; p < s->gl_ptr[J + 1]; p++)
            if (s->glbind[p] > l) { s->sup_parent[J] = s->sup_of[s->glbind[p]]; break; }
    }

    /* relind(J, p(J)) (Sec. 2.1.2): each i in glbind(J) n glbind(p(J)) replaced by
       its distance from the bottom of glbind(p(J)); found by direct search.   */
    s->ri_ptr = xcalloc(ns + 1, sizeof(int64_t));
    for (int64_t J = 0; J < ns; J++) {
        int64_t nJ = s->sup_ptr[J + 1] - s->sup_ptr[J];
        int64_t mJ = s->gl_ptr[J + 1] - s->gl_ptr[J];
        s->ri_ptr[J + 1] = s->ri_ptr[J] + (s->sup_parent[J] >= 0 ? mJ - nJ : 0);
    }
    s->relind = xmalloc((s->ri_ptr[ns] + 1) * sizeof(int32_t));
    for (int64_t J = 0; J < ns; J++) {
        int32_t P = s->sup_parent[J];
        if (P < 0) continue;
        int64_t nJ = s->sup_ptr[J + 1] - s->sup_ptr[J];
        int64_t mP = s->gl_ptr[P + 1] - s->gl_ptr[P];
        int64_t w = s->ri_ptr[J];
        for (int64_t p = s->gl_ptr[J] + nJ; p < s->gl_ptr[J + 1]; p++) {
            int32_t i = s->glbind[p];
            int64_t pos = find_pos(s->glbind + s->gl_ptr[P], mP, i);
            if (pos < 0) return OR_ERR_INTERNAL;
            s->relind[w++] = (int32_t)(mP - 1 - pos);
        }
    }

    /* blocks (Sec. 1, Sec. 2.2.2): the rows of S_J split into maximal runs of
       consecutive integers, each run then split at supernode boundaries.     */
    s->blk_ptr = xcalloc(ns + 1, sizeof(int64_t));
    int64_t cap = 1024, nb = 0;
    s->blk_first = xmalloc(cap * sizeof(int32_t));
    s->blk_size = xmalloc(cap * sizeof(int32_t));
    s->blk_owner = xmalloc(cap * sizeof(int32_t));
    for (int64_t J = 0; J < ns; J++) {
        int64_t nJ = s->sup_ptr[J + 1] - s->sup_ptr[J];
        for (int64_t p = s->gl_ptr[J] + nJ; p < s->gl_ptr[J + 1]; p++) {
            int32_t i = s->glbind[p];
            int newblk = (p == s->gl_ptr[J] + nJ) || (s->glbind[p - 1] != i - 1) ||
                         (s->sup_of[s->glbind[p - 1]] != s->sup_of[i]);
            if (newblk) {
                if (nb == cap) {
                    cap *= 2;
                    s->blk_first = realloc(s->blk_first, cap * sizeof(int32_t));
                    s->blk_size = realloc(s->blk_size, cap * sizeof(int32_t));
                    s->blk_owner = realloc(s->blk_owner, cap * sizeof(int32_t));
                }
                s->blk_first[nb] = i;
                s->blk_size[nb] = 1;
                s->blk_owner[nb] = s->sup_of[i];
                nb++;
            } else {
                s->blk_size[nb - 1]++;
            }
        }
        s->blk_ptr[J + 1] = nb;
    }
    s->nblocks = nb;

    /* relindB(J, P) (Alg. 5): for every ancestor P from p(J) up to the highest
       supernode owning a block of J, one entry per block of J lying at or above
       P's first column: the distance of the block's top row from the bottom of
       glbind(P), found by direct search.                                     */
    s->rb_pair_ptr = xcalloc(ns + 1, sizeof(int64_t));
    int64_t pcap = 1024, np_ = 0, vcap = 1024, nv = 0;
    s->rb_pair_P = xmalloc(pcap * sizeof(int32_t));
    s->rb_val_ptr = xmalloc((pcap + 1) * sizeof(int64_t));
    s->rb_val = xmalloc(vcap * sizeof(int32_t));
    s->rb_val_ptr[0] = 0;
    for (int64_t J = 0; J < ns; J++) {
        int64_t b0 = s->blk_ptr[J], b1 = s->blk_ptr[J + 1];
        if (b1 > b0) {
            int32_t top = s->blk_owner[b1 - 1];
            for (int32_t P = s->sup_parent[J]; P >= 0; P = s->sup_parent[P]) {
                int32_t fP = s->sup_ptr[P];
                int64_t mP = s->gl_ptr[P + 1] - s->gl_ptr[P];
                if (np_ + 1 >= pcap) {
                    pcap *= 2;
                    s->rb_pair_P = realloc(s->rb_pair_P, pcap * sizeof(int32_t));
                    s->rb_val_ptr = realloc(s->rb_val_ptr, (pcap + 1) * sizeof(int64_t));
                }
                for (int64_t b = b0; b < b1; b++) {
                    if (s->blk_first[b] < fP) continue;
                    int64_t pos = find_pos(s->glbind + s->gl_ptr[P], mP, s->blk_first[b]);
                    if (pos < 0) return OR_ERR_INTERNAL;
                    if (nv == vcap) { vcap *= 2; s->rb_val = realloc(s->rb_val, vcap * sizeof(int32_t)); }
                    s->rb_val[nv++] = (int32_t)(mP - 1 - pos);
                }
                s->rb_pair_P[np_] = P;
                np_++;
                s->rb_val_ptr[np_] = nv;
                if (P == top) break;
            }
        }
        s->rb_pair_ptr[J + 1] = np_;
    }
    s->npairs = np_;

    /* level = height in the supernodal elimination tree (leaves 0) */
    s->level = xcalloc(ns, sizeof(int32_t));
    for (int64_t J = 0; J < ns; J++) {
        int32_t P = s->sup_parent[J];
        if (P >= 0 && s->level[P] < s->level[J] + 1) s->level[P] = s->level[J] + 1;
    }
    *out = s;
    return OR_OK;
}

void or_free(or_sym *s) {
    if (!s) return;
    free_cols(s);
    free(s->perm); free(s->iperm); free(s->sup_ptr); free(s->sup_parent); free(s->sup_of);
    free(s->gl_ptr); free(s->glbind); free(s->ri_ptr); free(s->relind);
    free(s->blk_ptr); free(s->blk_first); free(s->blk_size); free(s->blk_owner);
    free(s->rb_pair_ptr); free(s->rb_pair_P); free(s->rb_val_ptr); free(s->rb_val);
    free(s->level); free(s->lval);
    free(s);
}

/* ------------------------------------------------------------------------ */
/* Numeric factorization: the column Cholesky of Algorithm 1 (Sec. 2.1.1).
 * For j = 1..n: scatter A_{*,j} into the n-vector t through glbind(j); for each
 * k < j with j in glbind(k), scatter-add -L_{j:n,k} * L_{j,k} into t; gather
 * t back into Lnz(j); cdiv(j): L_jj = sqrt(t_j), L_ij = t_i / L_jj.
 * Returns 0, or k >= 1 when the pivot of (1-based) column k of the user's
 * ordering is not positive.                                                 */
int64_t or_factor(or_sym *s, const double *values) {
    int64_t n = s->n;
    free(s->lval);
    s->lval = xcalloc(s->ccolptr[n], sizeof(double));
    double *t = xcalloc(n, sizeof(double));
    /* row lists of L: for each row j, the pairs (k, position of j in glbind(k)), k < j */
    int64_t *rcnt = xcalloc(n + 1, sizeof(int64_t));
    for (int64_t k = 0; k < n; k++)
        for (int64_t p = s->ccolptr[k] + 1; p < s->ccolptr[k + 1]; p++) rcnt[s->crows[p] + 1]++;
    for (int64_t j = 0; j < n; j++) rcnt[j + 1] += rcnt[j];
    int64_t *rfill = xmalloc((n + 1) * sizeof(int64_t));
    memcpy(rfill, rcnt, (n + 1) * sizeof(int64_t));
    int32_t *rk = xmalloc((rcnt[n] + 1) * sizeof(int32_t));
    int64_t *rp = xmalloc((rcnt[n] + 1) * sizeof(int64_t));
    for (int64_t k = 0; k < n; k++)
        for (int64_t p = s->ccolptr[k] + 1; p < s->ccolptr[k + 1]; p++) {
            int64_t q = rfill[s->crows[p]]++;
            rk[q] = (int32_t)k;
            rp[q] = p;
        }
    int64_t info = 0;
    for (int64_t j = 0; j < n && !info; j++) {
        /* scatter A_{*,j} (lower part, final ordering) into t */
        for (int64_t p = s->ccolptr[j]; p < s->ccolptr[j + 1]; p++) t[s->crows[p]] = 0.0;
        for (int64_t p = s->acolptr[j]; p < s->acolptr[j + 1]; p++) t[s->arowind[p]] += values[s->amap[p]];
        /* cmod(j, k) for every k < j with j in glbind(k) */
        for (int64_t q = rcnt[j]; q < rcnt[j + 1]; q++) {
            int64_t k = rk[q], pj = rp[q]; /* L_{j,k} sits at position pj of column k */
            double ljk = s->lval[pj];
            for (int64_t p = pj; p < s->ccolptr[k + 1]; p++) t[s->crows[p]] -= s->lval[p] * ljk;
        }
        /* gather and cdiv(j) */
        double d = t[j];
        if (!(d > 0.0)) { info = s->perm[j] + 1; break; }
        double ljj = sqrt(d);
        s->lval[s->ccolptr[j]] = ljj;
        for (int64_t p = s->ccolptr[j] + 1; p < s->ccolptr[j + 1]; p++) s->lval[p] = t[s->crows[p]] / ljj;
    }
    free(t); free(rcnt); free(rfill); free(rk); free(rp);
    return info;
}

/* Solve A X = B with the factor: x = P^T L^{-T} L^{-1} P b, column by column.
 * B and X are n x nrhs column-major (leading dimensions ldb, ldx).          */
int or_solve(const or_sym *s, int64_t nrhs, const double *B, int64_t ldb, double *X, int64_t ldx) {
    int64_t n = s->n;
    if (!s->lval) return OR_ERR_ARG;
    double *y = xmalloc(n * sizeof(double));
    for (int64_t r = 0; r < nrhs; r++) {
        for (int64_t k = 0; k < n; k++) y[k] = B[r * ldb + s->perm[k]];
        for (int64_t j = 0; j < n; j++) { /* forward: L y = P b */
            y[j] /= s->lval[s->ccolptr[j]];
            for (int64_t p = s->ccolptr[j] + 1; p < s->ccolptr[j + 1]; p++) y[s->crows[p]] -= s->lval[p] * y[j];
        }
        for (int64_t j = n - 1; j >= 0; j--) { /* backward: L^T z = y */
            double acc = y[j];
            for (int64_t p = s->ccolptr[j] + 1; p < s->ccolptr[j + 1]; p++) acc -= s->lval[p] * y[s->crows[p]];
            y[j] = acc / s->lval[s->ccolptr[j]];
        }
        for (int64_t k = 0; k < n; k++) X[r * ldx + s->perm[k]] = y[k];
    }
    free(y);
    return OR_OK;
}

/* Normwise backward error per right-hand side, on the user's symmetric A
 * given by its lower triangle (CSC):
 *   eta_r = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf).             */
int or_backward_error(int64_t n, const int64_t *colptr, const int32_t *rowind, const double *values,
                      int64_t nrhs, const double *B, int64_t ldb, const double *X, int64_t ldx,
                      double *eta) {
    double *rowabs = xcalloc(n, sizeof(double));
    double *r = xmalloc(n * sizeof(double));
    for (int64_t c = 0; c < n; c++)
        for (int64_t p = colptr[c]; p < colptr[c + 1]; p++) {
            int64_t i = rowind[p];
            rowabs[i] += fabs(values[p]);
            if (i != c) rowabs[c] += fabs(values[p]);
        }
    double anorm = 0.0;
    for (int64_t i = 0; i < n; i++) if (rowabs[i] > anorm) anorm = rowabs[i];
    for (int64_t q = 0; q < nrhs; q++) {
        const double *b = B + q * ldb, *x = X + q * ldx;
        for (int64_t i = 0; i < n; i++) r[i] = b[i];
        for (int64_t c = 0; c < n; c++)
            for (int64_t p = colptr[c]; p < colptr[c + 1]; p++) {
                int64_t i = rowind[p];
                r[i] -= values[p] * x[c];
                if (i != c) r[c] -= values[p] * x[i];
            }
        double rn = 0.0, xn = 0.0, bn = 0.0;
        for (int64_t i = 0; i < n; i++) {
            if (fabs(r[i]) > rn) rn = fabs(r[i]);
            if (fabs(x[i]) > xn) xn = fabs(x[i]);
            if (fabs(b[i]) > bn) bn = fabs(b[i]);
        }
        double den = anorm * xn + bn;
        eta[q] = den > 0.0 ? rn / den : 0.0;
    }
    free(rowabs); free(r);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Accessors for the test harness.                                          */

int64_t or_n(const or_sym *s) { return s->n; }
int64_t or_nsuper(const or_sym *s) { return s->nsuper; }
int64_t or_nnzL(const or_sym *s) { return s->nnzL; }
int64_t or_nblocks(const or_sym *s) { return s->nblocks; }
int64_t or_npairs(const or_sym *s) { return s->npairs; }
int64_t or_glbind_len(const or_sym *s) { return s->gl_ptr[s->nsuper]; }
int64_t or_relind_len(const or_sym *s) { return s->ri_ptr[s->nsuper]; }
int64_t or_relindB_len(const or_sym *s) { return s->rb_val_ptr[s->npairs]; }
double or_flops(const or_sym *s) { return s->flops; }

/* Copies every symbolic array into caller buffers (sizes from the accessors). */
int or_export(const or_sym *s, int32_t *perm, int32_t *sup_ptr, int32_t *sup_parent, int64_t *gl_ptr,
              int32_t *glbind, int64_t *ri_ptr, int32_t *relind, int64_t *blk_ptr, int32_t *blk_first,
              int32_t *blk_size, int32_t *blk_owner, int64_t *rb_pair_ptr, int32_t *rb_pair_P,
              int64_t *rb_val_ptr, int32_t *rb_val, int32_t *level, int32_t *cparent) {
    int64_t n = s->n, ns = s->nsuper;
    memcpy(perm, s->perm, n * sizeof(int32_t));
    memcpy(sup_ptr, s->sup_ptr, (ns + 1) * sizeof(int32_t));
    memcpy(sup_parent, s->sup_parent, ns * sizeof(int32_t));
    memcpy(gl_ptr, s->gl_ptr, (ns + 1) * sizeof(int64_t));
    memcpy(glbind, s->glbind, s->gl_ptr[ns] * sizeof(int32_t));
    memcpy(ri_ptr, s->ri_ptr, (ns + 1) * sizeof(int64_t));
    memcpy(relind, s->relind, s->ri_ptr[ns] * sizeof(int32_t));
    memcpy(blk_ptr, s->blk_ptr, (ns + 1) * sizeof(int64_t));
    memcpy(blk_first, s->blk_first, s->nblocks * sizeof(int32_t));
    memcpy(blk_size, s->blk_size, s->nblocks * sizeof(int32_t));
    memcpy(blk_owner, s->blk_owner, s->nblocks * sizeof(int32_t));
    memcpy(rb_pair_ptr, s->rb_pair_ptr, (ns + 1) * sizeof(int64_t));
    memcpy(rb_pair_P, s->rb_pair_P, s->npairs * sizeof(int32_t));
    memcpy(rb_val_ptr, s->rb_val_ptr, (s->npairs + 1) * sizeof(int64_t));
    memcpy(rb_val, s->rb_val, s->rb_val_ptr[s->npairs] * sizeof(int32_t));
    memcpy(level, s->level, ns * sizeof(int32_t));
    memcpy(cparent, s->cparent, n * sizeof(int32_t));
    return OR_OK;
}

/* Column structure of L in the final ordering (sizes: n+1 and nnzL). */
int or_export_columns(const or_sym *s, int64_t *colptr, int32_t *rows) {
    memcpy(colptr, s->ccolptr, (s->n + 1) * sizeof(int64_t));
    memcpy(rows, s->crows, s->ccolptr[s->n] * sizeof(int32_t));
    return OR_OK;
}

/* L in the canonical supernodal layout: for each supernode J, an m_J x |J|
 * row-major block (row r = glbind(J)[r], column c = column f_J + c), entries
 * above the diagonal zero; blocks concatenated in supernode order.          */
int or_export_L_supernodal(const or_sym *s, double *out) {
    if (!s->lval) return OR_ERR_ARG;
    int64_t off = 0;
    for (int64_t J = 0; J < s->nsuper; J++) {
        int32_t f = s->sup_ptr[J], w = s->sup_ptr[J + 1] - f;
        int64_t m = s->gl_ptr[J + 1] - s->gl_ptr[J];
        for (int64_t r = 0; r < m; r++)
            for (int32_t c = 0; c < w; c++)
                out[off + r * w + c] = (r >= c) ? s->lval[s->ccolptr[f + c] + (r - c)] : 0.0;
        off += m * w;
    }
    return OR_OK;
}

/* L by column (aligned with or_export_columns). */
int or_export_L_columns(const or_sym *s, double *out) {
    if (!s->lval) return OR_ERR_ARG;
    memcpy(out, s->lval, s->ccolptr[s->n] * sizeof(double));
    return OR_OK;
}

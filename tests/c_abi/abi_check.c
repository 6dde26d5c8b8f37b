/* Host-only use of the C ABI from plain C99 (no device work): analyse a 2D
 * 5-point Laplacian on an n x n grid with the geometric and the two graph
 * orderings (the graph orderings also on 1 and 5 threads: the same order),
 * read the symbolic view, check the device schedule, query the launch plan,
 * save and reload the analysis; a deterministic RL analysis with a
 * launch-plan table. Prints one line per ordering and one for the last;
 * exits non-zero on the first failed call. Build: cc -std=c99 -I include
 * abi_check.c -L <lib dir> -lsc. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "sc.h"

#define CHECK(call)                                                            \
    do {                                                                       \
        int rc_ = (call);                                                      \
        if (rc_ != SC_OK) {                                                    \
            fprintf(stderr, "%s failed: %d (%s)\n", #call, rc_, sc_strerror(rc_)); \
            return 1;                                                          \
        }                                                                      \
    } while (0)

int main(int argc, char **argv) {
    const int k = argc > 1 ? atoi(argv[1]) : 24;
    const char *path = argc > 2 ? argv[2] : "abi_check.scs";
    const int64_t n = (int64_t)k * k;
    int64_t *colptr = malloc((size_t)(n + 1) * sizeof(int64_t));
    int32_t *rowind = malloc((size_t)(3 * n) * sizeof(int32_t));
    int64_t nnz = 0;
    for (int64_t j = 0; j < n; j++) {  /* lower triangle: diagonal, east, north */
        colptr[j] = nnz;
        rowind[nnz++] = (int32_t)j;
        if ((j % k) + 1 < k) rowind[nnz++] = (int32_t)(j + 1);
        if (j + k < n) rowind[nnz++] = (int32_t)(j + k);
    }
    colptr[n] = nnz;
    const int orderings[3] = {SC_ORDER_GRID_ND, SC_ORDER_GRAPH_ND, SC_ORDER_GRAPH_ML};
    for (int o = 0; o < 3; o++) {
        sc_options opt;
        CHECK(sc_options_default(&opt));
        opt.ordering = orderings[o];
        opt.grid[0] = k;
        opt.grid[1] = k;
        opt.grid[2] = 1;
        sc_symbolic *s = NULL, *t = NULL;
        CHECK(sc_analyze(n, colptr, rowind, &opt, &s));
        sc_symbolic_view v, w;
        CHECK(sc_symbolic_export(s, &v));
        int64_t chk[5], plan[11];
        CHECK(sc_check_schedule(s, chk, 5));
        CHECK(sc_plan_stats(s, SC_FP64, plan, 11));
        CHECK(sc_symbolic_save(s, path));
        CHECK(sc_symbolic_load(path, &t));
        CHECK(sc_symbolic_export(t, &w));
        if (w.n != v.n || w.nnzL != v.nnzL || w.nsuper != v.nsuper ||
            memcmp(w.perm, v.perm, (size_t)n * sizeof(int32_t)) != 0) {
            fprintf(stderr, "reloaded analysis differs\n");
            return 1;
        }
        if (orderings[o] != SC_ORDER_GRID_ND) { /* the graph orderings: the same order on 1 and 5 threads */
            for (int th = 1; th <= 5; th += 4) {
                sc_symbolic *u = NULL;
                sc_symbolic_view x;
                opt.threads = th;
                CHECK(sc_analyze(n, colptr, rowind, &opt, &u));
                CHECK(sc_symbolic_export(u, &x));
                if (memcmp(x.perm, v.perm, (size_t)n * sizeof(int32_t)) != 0) {
                    fprintf(stderr, "ordering %d on %d threads differs\n", orderings[o], th);
                    return 1;
                }
                CHECK(sc_symbolic_free(u));
            }
            sc_symbolic *r = NULL;
            opt.threads = -1;
            if (sc_analyze(n, colptr, rowind, &opt, &r) != -4 || r != NULL) return 1;
            opt.threads = 0;
        }
        printf("ordering %d n %lld nsuper %lld nnzL %lld flops %.6g products %lld levels %lld\n", orderings[o],
               (long long)v.n, (long long)v.nsuper, (long long)v.nnzL, v.flops, (long long)chk[0],
               (long long)plan[0]);
        CHECK(sc_symbolic_free(t));
        CHECK(sc_symbolic_free(s));
    }
    {
        /* a deterministic RL analysis with a launch-plan table: the schedule check
         * covers its plans (kind 13), the plan has target-owned slabs and no tile
         * split along K; the same option with RLB is refused */
        sc_options opt;
        CHECK(sc_options_default(&opt));
        opt.ordering = SC_ORDER_GRID_ND;
        opt.grid[0] = k;
        opt.grid[1] = k;
        opt.grid[2] = 1;
        opt.variant = SC_RL;
        opt.deterministic = 1;
        sc_tune_table tt;
        memset(&tt, 0, sizeof(tt));
        tt.defer_width = 1024;
        tt.solve_group = 3;
        tt.tc_multicast = -1;
        opt.tune = &tt;
        sc_symbolic *s = NULL;
        CHECK(sc_analyze(n, colptr, rowind, &opt, &s));
        int64_t chk[5], plan[14];
        CHECK(sc_check_schedule(s, chk, 5));
        CHECK(sc_plan_stats(s, SC_FP64, plan, 14));
        if (plan[11] != 0 || plan[12] <= 0) {
            fprintf(stderr, "deterministic plan: %lld split tiles, %lld slabs\n", (long long)plan[11],
                    (long long)plan[12]);
            return 1;
        }
        printf("deterministic rl pairs %lld slabs %lld\n", (long long)plan[8], (long long)plan[12]);
        CHECK(sc_symbolic_free(s));
        opt.variant = SC_RLB;
        if (sc_analyze(n, colptr, rowind, &opt, &s) != -4) return 1;
    }
    if (sc_analyze(0, colptr, rowind, NULL, NULL) >= 0) return 1; /* invalid arguments are refused */
    remove(path);
    free(colptr);
    free(rowind);
    return 0;
}

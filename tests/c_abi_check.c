/* A plain C99 client of include/lider.h: it compiles against the header
 * alone, links liblider.so, and checks argument validation that answers
 * before any device work (so it runs without a GPU). */
#include <stdio.h>
#include <string.h>

#include "lider.h"

static int fails = 0;

static void expect(int cond, const char* what) {
    if (!cond) {
        printf("FAIL: %s (last error: %s)\n", what, lider_last_error() ? lider_last_error() : "(null)");
        ++fails;
    }
}

int main(void) {
    lider_index* ix = (lider_index*)0;
    lider_params p;
    memset(&p, 0, sizeof p);
    p.L = 4; p.m = 8; p.rmi_leaves = 16; p.r0 = 2; p.B = 1;
    p.hash_kind = LIDER_HASH_PSTABLE; p.W = 1.0; p.score_mode = LIDER_SCORE_SIMT;
    p.route_kind = LIDER_ROUTE_EXACT; p.raw_keys = 0;

    lider_cluster_params cp;
    memset(&cp, 0, sizeof cp);
    cp.n_clusters = 2; cp.kmeans_iters = 10; cp.kmeans_sample = 0; cp.seed = 0;

    expect(lider_build(0, 10, 8, &cp, 0, 0, &p, 0, 0) == LIDER_EINVAL, "build: NULL out");
    expect(lider_build(0, 10, 8, &cp, 0, 0, &p, 0, &ix) == LIDER_EINVAL && ix == 0, "build: NULL corpus");
    expect(lider_build_centroids(0, 10, 8, 0, 2, 0, 0, &p, 0, &ix) == LIDER_EINVAL && ix == 0,
           "build_centroids: NULL inputs");
    expect(lider_last_error() != 0 && strlen(lider_last_error()) > 0, "last_error is set");
    {
        lider_build_info bi;
        expect(lider_get_build_info(0, &bi) == LIDER_EINVAL, "build_info: NULL index");
        expect(lider_export_centroids(0, 0) == LIDER_EINVAL, "export_centroids: NULL index");
    }

    lider_search_stats st;
    expect(lider_search(0, 0, 0, 10, 1, 0, 0, &st, 0) == LIDER_EINVAL, "search: NULL index");
    expect(lider_search_host(0, 0, 0, 10, 1, 0, 0, 0, 0) == LIDER_EINVAL, "search_host: NULL index");
    size_t bytes = 0;
    expect(lider_search_scratch_bytes(0, 10, 10, 1, &bytes) == LIDER_EINVAL, "scratch_bytes: NULL index");
    lider_tuning t;
    expect(lider_get_tuning(0, &t) == LIDER_EINVAL, "get_tuning: NULL index");
    lider_server_params sp;
    memset(&sp, 0, sizeof sp);
    lider_server* srv = 0;
    expect(lider_server_create(0, &sp, &srv) == LIDER_EINVAL, "server_create: NULL index");
    lider_free(0);                 /* NULL is accepted */
    lider_server_destroy(0);

    if (fails) return 1;
    printf("c abi checks passed\n");
    return 0;
}

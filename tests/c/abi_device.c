/* The C ABI from plain C on a GPU: build a network from a timetable file, run
 * single queries (eat_query) and a batch (eat_query_batch) with host buffers, and
 * write every arrival row to an output file for the caller to compare with the
 * oracle.
 *
 *   abi_device <timetable> <queries> <rows out>
 *   timetable: int32 n_stops, int64 n_conn, then u[], v[], dep[], dur[] (int32)
 *   queries:   int32 n, then sources[], times[] (int32)
 *   rows out:  2 * n rows of n_stops int32: first eat_query's, then the batch's
 * Exits 0 and prints "ok" when every call succeeds. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "eat.h"

#define CHECK(c)                                                        \
    do {                                                                \
        if (!(c)) {                                                     \
            fprintf(stderr, "check failed at line %d: %s (%s)\n",       \
                    __LINE__, #c, eat_last_error());                    \
            return 1;                                                   \
        }                                                               \
    } while (0)

static int32_t *read_i32(FILE *f, int64_t n) {
    int32_t *p = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (p && (int64_t)fread(p, sizeof(int32_t), (size_t)n, f) != n) {
        free(p);
        return NULL;
    }
    return p;
}

int main(int argc, char **argv) {
    CHECK(argc == 4);
    FILE *ft = fopen(argv[1], "rb");
    CHECK(ft != NULL);
    int32_t n_stops = 0;
    int64_t n_conn = 0;
    CHECK(fread(&n_stops, sizeof n_stops, 1, ft) == 1);
    CHECK(fread(&n_conn, sizeof n_conn, 1, ft) == 1);
    int32_t *u = read_i32(ft, n_conn), *v = read_i32(ft, n_conn);
    int32_t *dep = read_i32(ft, n_conn), *dur = read_i32(ft, n_conn);
    CHECK(u && v && dep && dur);
    fclose(ft);
    FILE *fq = fopen(argv[2], "rb");
    CHECK(fq != NULL);
    int32_t n = 0;
    CHECK(fread(&n, sizeof n, 1, fq) == 1 && n > 0);
    int32_t *src = read_i32(fq, n), *ts = read_i32(fq, n);
    CHECK(src && ts);
    fclose(fq);

    eat_connections c = {n_stops, n_conn, u, v, dep, dur, NULL};
    eat_build_opts o;
    memset(&o, 0, sizeof o);
    o.device = 0;
    o.cluster_width = 1800;
    eat_net *net = NULL;
    CHECK(eat_build(&c, &o, &net) == EAT_OK && net != NULL);
    eat_stats st;
    CHECK(eat_get_stats(net, &st) == EAT_OK && st.device == 0 && st.n_stops == n_stops);

    int32_t *rows = (int32_t *)malloc((size_t)2 * (size_t)n * (size_t)n_stops * sizeof(int32_t));
    CHECK(rows != NULL);
    eat_counters cnt;
    for (int32_t i = 0; i < n; ++i) {
        CHECK(eat_query(net, src[i], ts[i], rows + (size_t)i * n_stops, &cnt) == EAT_OK);
        CHECK(cnt.rounds >= 1 && cnt.types >= cnt.lookups && cnt.lookups >= cnt.evals);
    }
    /* The batch with host buffers: the library stages them through device memory. */
    int32_t *batch = rows + (size_t)n * n_stops;
    CHECK(eat_query_batch(net, src, ts, n, batch, NULL, 0, NULL, NULL) == EAT_OK);
    /* Errors through the ABI: a source out of range, a workspace that is too small. */
    CHECK(eat_query(net, n_stops, 0, rows, NULL) == EAT_ERR_INVALID);
    const eat_net *nets[1] = {net};
    CHECK(eat_workspace_bytes(nets, 1, n, NULL) > 0);

    FILE *fo = fopen(argv[3], "wb");
    CHECK(fo != NULL);
    CHECK(fwrite(rows, sizeof(int32_t), (size_t)2 * n * n_stops, fo) == (size_t)2 * n * n_stops);
    fclose(fo);
    eat_free(net);
    free(rows);
    free(u);
    free(v);
    free(dep);
    free(dur);
    free(src);
    free(ts);
    printf("ok\n");
    return 0;
}

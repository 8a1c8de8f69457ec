/* The C ABI from plain C, without a GPU: host-only builds of a small timetable,
 * their sizes and host views, and the errors of calls that need a device or get
 * bad input.  Exits 0 and prints "ok" when every check holds. */
#include <stdio.h>
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

int main(void) {
    /* Stops 0 -> 1 -> 2 every 600 s from 08:00 to 09:00 (one AP per type and
     * cluster), a slow direct 0 -> 2, and a 2 -> 3 connection. */
    int32_t u[32], v[32], dep[32], dur[32];
    int64_t n = 0;
    for (int32_t t = 28800; t <= 32400; t += 600) {
        u[n] = 0; v[n] = 1; dep[n] = t; dur[n] = 300; ++n;
        u[n] = 1; v[n] = 2; dep[n] = t + 300; dur[n] = 300; ++n;
    }
    u[n] = 0; v[n] = 2; dep[n] = 28800; dur[n] = 1800; ++n;
    u[n] = 2; v[n] = 3; dep[n] = 30000; dur[n] = 60; ++n;
    eat_connections c = {4, n, u, v, dep, dur, NULL};
    eat_build_opts o;
    memset(&o, 0, sizeof o);
    o.device = -1;
    eat_net *net = NULL;
    CHECK(eat_version() > 0);
    CHECK(eat_build(&c, &o, &net) == EAT_OK && net != NULL);

    eat_stats st;
    CHECK(eat_get_stats(net, &st) == EAT_OK);
    CHECK(st.n_stops == 4 && st.device == -1 && st.n_conn == n);
    CHECK(st.n_types == 4 && st.n_edges == 4);          /* 0-1, 1-2, 0-2, 2-3 */
    CHECK(st.cluster_width == 3600 && st.max_out_types == 2);

    eat_net_view view;
    CHECK(eat_net_host_view(net, &view) == EAT_OK);
    CHECK(view.row_ptr[0] == 0 && view.row_ptr[4] == 4);
    CHECK(view.row_ptr[1] - view.row_ptr[0] == 2);      /* stop 0: to 1 and to 2 */
    CHECK(view.row_ptr[3] - view.row_ptr[2] == 1);      /* stop 2: to 3 */

    int32_t row[4];
    CHECK(eat_query(net, 0, 28800, row, NULL) == EAT_ERR_NO_DEVICE);
    CHECK(strlen(eat_last_error()) > 0);

    const eat_net *nets[1] = {net};
    eat_query_opts shape;
    CHECK(eat_launch_shape(nets, 1, 8, NULL, &shape) == EAT_ERR_NO_DEVICE);
    CHECK(eat_launch_shape(nets, 1, 8, NULL, NULL) == EAT_ERR_INVALID);
    CHECK(eat_launch_shape(nets, 0, 8, NULL, &shape) == EAT_ERR_INVALID);

    eat_ladder *lad = NULL;
    CHECK(eat_ladder_build(&c, &o, &lad) == EAT_OK && lad != NULL);
    eat_ladder_view lv;
    CHECK(eat_ladder_host_view(lad, &lv) == EAT_OK);
    CHECK(lv.n_types == 4 && lv.n_edges == 4);
    CHECK(lv.n_dep == 7 + 7 + 1 + 1);                  /* departures of the four types */
    CHECK(eat_ladder_query(lad, EAT_VAR_CLUSTER_AP, 0, 28800, 1, 0, row, NULL) == EAT_ERR_NO_DEVICE);
    eat_ladder_free(lad);

    dur[0] = 0;                                         /* durations must be >= 1 */
    eat_net *bad = NULL;
    CHECK(eat_build(&c, &o, &bad) == EAT_ERR_INVALID && bad == NULL);
    dur[0] = 300;
    u[1] = 7;                                           /* stop out of range */
    CHECK(eat_build(&c, &o, &bad) == EAT_ERR_INVALID && bad == NULL);

    eat_free(net);
    eat_free(NULL);
    printf("ok\n");
    return 0;
}

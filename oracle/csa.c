/*
 * Oracle (test infrastructure only): the serial connection-scan algorithm and an
 * exactness certificate for earliest arrival times.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load
 * this file's library.  It shares nothing with the CUDA path.
 *
 * Model (Section I-A, Preliminaries): a connection (u, v, t, lambda) leaves stop u
 * at time t and reaches v at t + lambda.  For a query (s, t_s) the earliest
 * arrival time e[v] is the least arrival over time-respecting paths that leave s
 * at or after t_s; e[s] = t_s; unreachable stops keep "infinity", written here as
 * INT32_MAX.
 */
#include <stdint.h>
#include <stddef.h>
#include <pthread.h>

#define ORACLE_INF INT32_MAX

/*
 * Connection-Scan Algorithm (Algorithm 1).  The connections must be sorted by
 * non-decreasing departure time.  Every stop starts at infinity except the
 * source (t_s); each connection in order lowers e[v] to t + lambda when
 * e[u] <= t and t + lambda < e[v].
 *
 * Connections departing before t_s can never satisfy e[u] <= t (every finite
 * e[] is >= t_s), so the scan starts at the first departure >= t_s, found by
 * binary search; this skips only no-op iterations.
 */
void oracle_csa(int32_t n_stops, int64_t n_conn, const int32_t *u, const int32_t *v,
                const int32_t *dep, const int32_t *dur, int32_t s, int32_t t_s,
                int32_t *e)
{
    for (int32_t x = 0; x < n_stops; ++x)
        e[x] = ORACLE_INF;
    e[s] = t_s;

    int64_t lo = 0, hi = n_conn;           /* first index with dep >= t_s */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (dep[mid] < t_s) lo = mid + 1; else hi = mid;
    }
    for (int64_t i = lo; i < n_conn; ++i) {
        int32_t t = dep[i];
        int64_t arrive = (int64_t)t + dur[i];
        if (e[u[i]] <= t && arrive < e[v[i]])
            e[v[i]] = (int32_t)arrive;
    }
}

/* One query per call, run over a list of queries by n_threads POSIX threads. */
struct csa_job {
    int32_t n_stops; int64_t n_conn;
    const int32_t *u, *v, *dep, *dur;
    const int32_t *src, *ts; int64_t n_q;
    int32_t *out; int64_t next; pthread_mutex_t lock;
};

static void *csa_worker(void *arg)
{
    struct csa_job *j = (struct csa_job *)arg;
    for (;;) {
        pthread_mutex_lock(&j->lock);
        int64_t q = j->next++;
        pthread_mutex_unlock(&j->lock);
        if (q >= j->n_q) return NULL;
        oracle_csa(j->n_stops, j->n_conn, j->u, j->v, j->dep, j->dur, j->src[q], j->ts[q],
                   j->out + q * (int64_t)j->n_stops);
    }
}

/* out is [n_q x n_stops] row-major.  Returns the number of threads used. */
int32_t oracle_csa_many(int32_t n_stops, int64_t n_conn, const int32_t *u, const int32_t *v,
                        const int32_t *dep, const int32_t *dur, const int32_t *src,
                        const int32_t *ts, int64_t n_q, int32_t *out, int32_t n_threads)
{
    struct csa_job j = {n_stops, n_conn, u, v, dep, dur, src, ts, n_q, out, 0};
    pthread_mutex_init(&j.lock, NULL);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    int32_t started = 0;
    for (int32_t i = 1; i < n_threads; ++i)
        if (pthread_create(&th[started], NULL, csa_worker, &j) == 0) ++started;
    csa_worker(&j);
    for (int32_t i = 0; i < started; ++i) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&j.lock);
    return started + 1;
}

/*
 * Certificate that e[] is exactly the earliest-arrival vector, in any connection
 * order (no sorting needed), for durations >= 1:
 *   (i)   e[s] == t_s;
 *   (ii)  feasibility: every connection with e[u] <= t has e[v] <= t + lambda;
 *         by induction along any time-respecting path from s this gives
 *         e[v] <= true earliest arrival;
 *   (iii) witness: every v != s with e[v] < INF has a connection into v with
 *         e[u] <= t and t + lambda == e[v]; since lambda >= 1 the witnesses form
 *         a chain with strictly decreasing e[] that can only end at s, i.e. a
 *         time-respecting path reaching v at e[v], so e[v] >= true arrival.
 * Returns 0 if all hold, else 1 / 2 / 3 for the first failing condition, with
 * *bad set to the offending connection (ii) or stop (i, iii).
 */
int32_t oracle_certify(int32_t n_stops, int64_t n_conn, const int32_t *u, const int32_t *v,
                       const int32_t *dep, const int32_t *dur, int32_t s, int32_t t_s,
                       const int32_t *e, uint8_t *scratch, int64_t *bad)
{
    if (e[s] != t_s) { *bad = s; return 1; }
    for (int32_t x = 0; x < n_stops; ++x) scratch[x] = 0;
    for (int64_t i = 0; i < n_conn; ++i) {
        int64_t arrive = (int64_t)dep[i] + dur[i];
        if (e[u[i]] <= dep[i]) {
            if ((int64_t)e[v[i]] > arrive) { *bad = i; return 2; }
            if ((int64_t)e[v[i]] == arrive) scratch[v[i]] = 1;
        }
    }
    for (int32_t x = 0; x < n_stops; ++x)
        if (x != s && e[x] != ORACLE_INF && !scratch[x]) { *bad = x; return 3; }
    return 0;
}

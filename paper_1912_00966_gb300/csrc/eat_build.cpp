// Host preprocessing: connections -> connection types -> clusters -> AP cover
// (Section III-A, graph representation and preprocessing algorithm).
//
// Layout produced (see eat_net_view in eat.h):
//   row_ptr[V+1]  types grouped by tail stop u, each group ordered by (v, lambda)
//   type_rec[4T]  {v, lambda, first departure, last departure}
//   type_cl[T]    cl_base: cluster k of the type starts at cl[cl_base + k]
//   cl[]          AP index of the start of each cluster of each type, plus one
//                 end entry per type; only clusters between the type's first
//                 and last departure are stored (the paper stores y per type)
//   ap[2A]        {first term, (difference << 16) | terms}
//
// Stops are processed in parallel chunks (std::thread); each chunk builds with
// local indices and a final pass shifts them to global positions.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstring>
#include <thread>

#include "eat_internal.h"

namespace eat {

namespace {

struct Rec {
    int32_t v, dur, dep;
};

inline bool rec_less(const Rec &a, const Rec &b) {
    if (a.v != b.v) return a.v < b.v;
    if (a.dur != b.dur) return a.dur < b.dur;
    return a.dep < b.dep;
}

// Per-thread bitmaps for the greedy AP cover.
struct Bits {
    std::vector<uint64_t> present, covered;
    void ensure(size_t nbits) {
        size_t w = (nbits + 63) / 64;
        if (present.size() < w) {
            present.assign(w, 0);
            covered.assign(w, 0);
        }
    }
    bool get(const std::vector<uint64_t> &b, int32_t i) const { return (b[i >> 6] >> (i & 63)) & 1; }
    static void set(std::vector<uint64_t> &b, int32_t i) { b[i >> 6] |= uint64_t(1) << (i & 63); }
};

thread_local Bits tl_bits;

struct Chunk {
    int32_t u_begin = 0, u_end = 0;
    std::vector<int32_t> types_per_u;   // local row counts
    std::vector<int32_t> type_rec, type_cl, cl;
    std::vector<uint32_t> ap;
    int64_t n_conn = 0;
    int32_t n_edges = 0, max_clusters = 0;
};

void build_chunk(Chunk &ch, const std::vector<int64_t> &u_off, std::vector<Rec> &recs,
                 int32_t width, int32_t t0) {
    std::vector<int32_t> deps;
    for (int32_t u = ch.u_begin; u < ch.u_end; ++u) {
        Rec *b = recs.data() + u_off[u];
        Rec *e = recs.data() + u_off[u + 1];
        std::sort(b, e, rec_less);
        int32_t n_types_u = 0;
        int32_t last_v = -1;
        for (Rec *p = b; p < e;) {
            Rec *q = p;
            deps.clear();
            while (q < e && q->v == p->v && q->dur == p->dur) {
                if (deps.empty() || deps.back() != q->dep) deps.push_back(q->dep);
                ++q;
            }
            ch.n_conn += (int64_t)deps.size();
            if (p->v != last_v) { ++ch.n_edges; last_v = p->v; }
            const int32_t first = deps.front(), last = deps.back();
            const int32_t k_first = (first - t0) / width, k_last = (last - t0) / width;
            ch.max_clusters = std::max(ch.max_clusters, k_last - k_first + 1);
            const int32_t cl_start = (int32_t)ch.cl.size();
            ch.type_rec.insert(ch.type_rec.end(), {p->v, p->dur, first, last});
            ch.type_cl.push_back(cl_start - k_first);
            size_t i = 0;
            for (int32_t k = k_first; k <= k_last; ++k) {
                ch.cl.push_back((int32_t)(ch.ap.size() / 2));
                size_t j = i;
                const int64_t hi = (int64_t)t0 + (int64_t)(k + 1) * width;
                while (j < deps.size() && deps[j] < hi) ++j;
                if (j > i) ap_cover(deps.data() + i, (int32_t)(j - i), width, ch.ap);
                i = j;
            }
            ch.cl.push_back((int32_t)(ch.ap.size() / 2));
            ++n_types_u;
            p = q;
        }
        ch.types_per_u.push_back(n_types_u);
    }
}

}  // namespace

namespace {

// Greedy AP cover (Section I-A, Arithmetic Progression Technique): repeatedly take
// the smallest uncovered value a; among the APs a, a+d, a+2d, ... that stay inside
// the set (one per later value, i.e. per difference d, each extended as far as it
// goes) take the one covering the most uncovered values, then the longest, then
// the smallest d.  Values are sorted and unique.  Calls emit(first, d, terms) per
// AP in increasing first term (d = 0 for a one-term AP).
template <class Emit>
void ap_cover_core(const int32_t *d, int32_t n, Emit emit) {
    if (n == 1) {
        emit(d[0], 0, 1);
        return;
    }
    const int32_t base = d[0];
    const int32_t top = d[n - 1];
    const int32_t span = top - base + 1;
    Bits &bits = tl_bits;
    bits.ensure((size_t)span);
    for (int32_t i = 0; i < n; ++i) Bits::set(bits.present, d[i] - base);
    int32_t n_cov = 0, i = 0;
    while (n_cov < n) {
        while (bits.get(bits.covered, d[i] - base)) ++i;
        const int32_t a = d[i];
        int32_t best_unc = 1, best_len = 1, best_step = 0;
        for (int32_t j = i + 1; j < n; ++j) {
            const int32_t step = d[j] - a;
            const int32_t max_len = (top - a) / step + 1;
            if (max_len <= best_unc) break;  // no later (larger) step can win
            int32_t len = 0, unc = 0;
            for (int64_t t = a; t <= top && bits.get(bits.present, (int32_t)(t - base)); t += step) {
                ++len;
                unc += !bits.get(bits.covered, (int32_t)(t - base));
            }
            if (unc > best_unc || (unc == best_unc && len > best_len)) {
                best_unc = unc;
                best_len = len;
                best_step = step;
            }
        }
        for (int32_t m = 0; m < best_len; ++m) {
            const int32_t off = a - base + m * best_step;
            if (!bits.get(bits.covered, off)) {
                Bits::set(bits.covered, off);
                ++n_cov;
            }
        }
        emit(a, best_step, best_len);
    }
    const size_t words = ((size_t)span + 63) / 64;
    std::memset(bits.present.data(), 0, words * sizeof(uint64_t));
    std::memset(bits.covered.data(), 0, words * sizeof(uint64_t));
}

}  // namespace

// Greedy AP cover of one cluster (values span less than `width_hint` < 2^16
// seconds): appends {first, difference << 16 | terms} per AP.
void ap_cover(const int32_t *d, int32_t n, int32_t width_hint, std::vector<uint32_t> &out) {
    (void)width_hint;
    ap_cover_core(d, n, [&](int32_t a, int32_t step, int32_t len) {
        out.push_back((uint32_t)a);
        out.push_back(((uint32_t)step << 16) | (uint32_t)len);
    });
}

// Greedy AP cover of any sorted unique values (e.g. a connection type's whole
// day): appends {first, difference, terms} per AP.
void ap_cover_wide(const int32_t *d, int32_t n, std::vector<int32_t> &out) {
    ap_cover_core(d, n, [&](int32_t a, int32_t step, int32_t len) {
        out.push_back(a);
        out.push_back(step);
        out.push_back(len);
    });
}

int build_host(const eat_connections *c, int32_t width, int32_t t0, HostNet &h) {
    const int32_t V = c->n_stops;
    const int64_t C = c->n_conn;
    if (V <= 0) return fail(EAT_ERR_INVALID, "n_stops must be >= 1");
    if (C < 0 || C >= INT32_MAX) return fail(EAT_ERR_INVALID, "n_conn must be in [0, 2^31-1)");
    if (C > 0 && (!c->u || !c->v || !c->dep || !c->dur))
        return fail(EAT_ERR_INVALID, "connection arrays must not be NULL");
    if (width < 1 || width > 65535) return fail(EAT_ERR_INVALID, "cluster_width must be in 1..65535");
    for (int64_t i = 0; i < C; ++i) {
        const int32_t u = c->u[i], v = c->v[i], dep = c->dep[i], dur = c->dur[i];
        if (u < 0 || u >= V || v < 0 || v >= V)
            return fail(EAT_ERR_INVALID, "connection " + std::to_string(i) + ": stop id out of range");
        if (dur < 1)
            return fail(EAT_ERR_INVALID, "connection " + std::to_string(i) + ": duration must be >= 1");
        if (dep < t0)
            return fail(EAT_ERR_INVALID, "connection " + std::to_string(i) + ": departure before t0");
        if ((int64_t)dep - t0 >= (int64_t)INT32_MAX)
            return fail(EAT_ERR_INVALID, "connection " + std::to_string(i) + ": departure too far after t0");
        if ((int64_t)dep + dur >= (int64_t)INT32_MAX)
            return fail(EAT_ERR_INVALID, "connection " + std::to_string(i) + ": arrival overflows int32");
        if (dur >= kMaxDuration)
            return fail(EAT_ERR_INVALID, "connection " + std::to_string(i) + ": duration must be < 2^24 s");
    }

    // Counting sort of the connections by tail stop.
    std::vector<int64_t> u_off((size_t)V + 1, 0);
    for (int64_t i = 0; i < C; ++i) ++u_off[(size_t)c->u[i] + 1];
    for (int32_t u = 0; u < V; ++u) u_off[u + 1] += u_off[u];
    std::vector<Rec> recs((size_t)C);
    {
        std::vector<int64_t> pos(u_off.begin(), u_off.end() - 1);
        for (int64_t i = 0; i < C; ++i) recs[pos[c->u[i]]++] = Rec{c->v[i], c->dur[i], c->dep[i]};
    }

    // Chunks of stops with about equal connection counts.
    unsigned hw = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    const int n_chunks = (int)std::min<int64_t>((int64_t)hw * 4, V);
    std::vector<Chunk> chunks((size_t)n_chunks);
    {
        int32_t u = 0;
        for (int k = 0; k < n_chunks; ++k) {
            const int64_t target = (C * (k + 1)) / n_chunks;
            chunks[k].u_begin = u;
            int32_t e = u;
            if (k == n_chunks - 1) e = V;
            else while (e < V && u_off[e] < target) ++e;
            chunks[k].u_end = e;
            u = e;
        }
    }
    {
        std::vector<std::thread> th;
        std::atomic_int next{0};
        auto work = [&]() {
            for (;;) {
                int k = next.fetch_add(1);
                if (k >= n_chunks) return;
                build_chunk(chunks[k], u_off, recs, width, t0);
            }
        };
        for (unsigned t = 1; t < hw; ++t) th.emplace_back(work);
        work();
        for (auto &t : th) t.join();
    }

    // Concatenate chunks, shifting local indices to global ones.
    int64_t T = 0, NCL = 0, NAP = 0;
    std::vector<int64_t> t_off(n_chunks), cl_off(n_chunks), ap_off(n_chunks);
    h = HostNet();
    h.n_stops = V;
    h.width = width;
    h.t0 = t0;
    for (int k = 0; k < n_chunks; ++k) {
        t_off[k] = T;
        cl_off[k] = NCL;
        ap_off[k] = NAP;
        T += (int64_t)chunks[k].type_cl.size();
        NCL += (int64_t)chunks[k].cl.size();
        NAP += (int64_t)chunks[k].ap.size() / 2;
        h.n_conn += chunks[k].n_conn;
        h.n_edges += chunks[k].n_edges;
        h.max_clusters = std::max(h.max_clusters, chunks[k].max_clusters);
    }
    if (T >= INT32_MAX || NCL >= INT32_MAX || NAP >= INT32_MAX)
        return fail(EAT_ERR_INVALID, "network too large for 32-bit indices");
    h.n_types = (int32_t)T;
    try {
        h.row_ptr.resize((size_t)V + 1);
        h.type_rec.resize((size_t)T * 4);
        h.type_cl.resize((size_t)T);
        h.cl.resize((size_t)NCL);
        h.ap.resize((size_t)NAP * 2);
    } catch (const std::bad_alloc &) {
        return fail(EAT_ERR_OOM, "host allocation failed");
    }
    {
        std::vector<std::thread> th;
        auto copy = [&](int k) {
            const Chunk &ch = chunks[k];
            std::copy(ch.type_rec.begin(), ch.type_rec.end(), h.type_rec.begin() + t_off[k] * 4);
            for (size_t i = 0; i < ch.type_cl.size(); ++i)
                h.type_cl[t_off[k] + i] = ch.type_cl[i] + (int32_t)cl_off[k];
            for (size_t i = 0; i < ch.cl.size(); ++i)
                h.cl[cl_off[k] + i] = ch.cl[i] + (int32_t)ap_off[k];
            std::copy(ch.ap.begin(), ch.ap.end(), h.ap.begin() + ap_off[k] * 2);
        };
        for (int k = 1; k < n_chunks; ++k) th.emplace_back(copy, k);
        if (n_chunks > 0) copy(0);
        for (auto &t : th) t.join();
    }
    int32_t r = 0;
    for (int k = 0; k < n_chunks; ++k) {
        const Chunk &ch = chunks[k];
        for (int32_t i = 0; i < (int32_t)ch.types_per_u.size(); ++i) {
            h.row_ptr[ch.u_begin + i] = r;
            r += ch.types_per_u[i];
            h.max_out_types = std::max(h.max_out_types, ch.types_per_u[i]);
        }
    }
    h.row_ptr[V] = r;
    return EAT_OK;
}

// Pre-encoded input (eat_build_csr): validate and convert to the logical arrays.
int build_host_csr(const eat_csr_input *in, int32_t width, int32_t t0, HostNet &h) {
    const int32_t V = in->n_stops, T = in->n_types;
    const int64_t NC = in->n_clusters, NA = in->n_aps;
    auto bad = [](const std::string &what, int64_t i) {
        return fail(EAT_ERR_INVALID, what + " (index " + std::to_string(i) + ")");
    };
    if (V <= 0) return fail(EAT_ERR_INVALID, "n_stops must be >= 1");
    if (T < 0 || NC < 0 || NA < 0) return fail(EAT_ERR_INVALID, "negative sizes");
    if (width < 1 || width > 65535) return fail(EAT_ERR_INVALID, "cluster_width must be in 1..65535");
    if (!in->row_ptr || (T > 0 && (!in->type_v || !in->type_dur || !in->type_cl_ptr)) ||
        (NC > 0 && (!in->cl_k || !in->cl_ap_ptr)) ||
        (NA > 0 && (!in->ap_first || !in->ap_step || !in->ap_count)))
        return fail(EAT_ERR_INVALID, "NULL input array");
    if (NC >= INT32_MAX || NA >= INT32_MAX) return fail(EAT_ERR_INVALID, "too many clusters or APs");
    if (in->row_ptr[0] != 0 || in->row_ptr[V] != T) return fail(EAT_ERR_INVALID, "row_ptr must run from 0 to n_types");
    for (int32_t u = 0; u < V; ++u)
        if (in->row_ptr[u + 1] < in->row_ptr[u]) return bad("row_ptr decreases", u);
    if (T > 0 && (in->type_cl_ptr[0] != 0 || in->type_cl_ptr[T] != NC))
        return fail(EAT_ERR_INVALID, "type_cl_ptr must run from 0 to n_clusters");
    if (NC > 0 && (in->cl_ap_ptr[0] != 0 || in->cl_ap_ptr[NC] != NA))
        return fail(EAT_ERR_INVALID, "cl_ap_ptr must run from 0 to n_aps");
    h = HostNet();
    h.n_stops = V;
    h.n_types = T;
    h.width = width;
    h.t0 = t0;
    try {
        h.row_ptr.assign(in->row_ptr, in->row_ptr + (size_t)V + 1);
        h.type_rec.resize((size_t)T * 4);
        h.type_cl.resize((size_t)T);
        h.ap.reserve((size_t)NA * 2);
    } catch (const std::bad_alloc &) {
        return fail(EAT_ERR_OOM, "host allocation failed");
    }
    int32_t last_u = -1;
    for (int32_t u = 0; u < V; ++u) {
        const int32_t deg = in->row_ptr[u + 1] - in->row_ptr[u];
        h.max_out_types = std::max(h.max_out_types, deg);
        (void)last_u;
    }
    for (int32_t t = 0; t < T; ++t) {
        const int32_t v = in->type_v[t], lam = in->type_dur[t];
        if (v < 0 || v >= V) return bad("type head stop out of range", t);
        if (lam < 1) return bad("type duration must be >= 1", t);
        if (lam >= kMaxDuration) return bad("type duration must be < 2^24 s", t);
        const int64_t c0 = in->type_cl_ptr[t], c1 = in->type_cl_ptr[t + 1];
        if (c1 <= c0) return bad("type without clusters", t);
        int32_t first = EAT_INF, last = INT32_MIN;
        int32_t prev_k = INT32_MIN;
        const int32_t cl_start = (int32_t)h.cl.size();
        int32_t k_first = 0;
        for (int64_t c = c0; c < c1; ++c) {
            const int32_t k = in->cl_k[c];
            if (k < 0) return bad("cluster index must be >= 0", c);
            if (c > c0 && k <= prev_k) return bad("cluster indices must increase within a type", c);
            const int64_t lo = (int64_t)t0 + (int64_t)k * width, hi = lo + width;
            if (hi - 1 >= (int64_t)INT32_MAX) return bad("cluster window overflows int32", c);
            if (c == c0) k_first = k;
            // empty clusters between the previous one and k
            for (int32_t kk = (c == c0 ? k : prev_k + 1); kk < k; ++kk)
                h.cl.push_back((int32_t)(h.ap.size() / 2));
            h.cl.push_back((int32_t)(h.ap.size() / 2));
            const int64_t a0 = in->cl_ap_ptr[c], a1 = in->cl_ap_ptr[c + 1];
            if (a1 <= a0) return bad("cluster without APs", c);
            int32_t prev_first = INT32_MIN;
            for (int64_t a = a0; a < a1; ++a) {
                const int32_t f = in->ap_first[a], st = in->ap_step[a], n = in->ap_count[a];
                if (n < 1 || n > 65535) return bad("AP term count must be in 1..65535", a);
                if (n >= 2 && (st < 1 || st > 65535)) return bad("AP difference must be in 1..65535", a);
                const int64_t lt = (int64_t)f + (int64_t)(n - 1) * (n >= 2 ? st : 0);
                if (f < lo || lt >= hi) return bad("AP terms outside the cluster window", a);
                if (lt + lam >= (int64_t)INT32_MAX) return bad("arrival overflows int32", a);
                if (a > a0 && f < prev_first) return bad("APs must be ordered by first term", a);
                prev_first = f;
                first = std::min(first, f);
                last = std::max(last, (int32_t)lt);
                h.ap.push_back((uint32_t)f);
                h.ap.push_back(((uint32_t)(n >= 2 ? st : 0) << 16) | (uint32_t)n);
                h.n_conn += n;
            }
            prev_k = k;
        }
        h.cl.push_back((int32_t)(h.ap.size() / 2));
        h.type_rec[4 * (size_t)t] = v;
        h.type_rec[4 * (size_t)t + 1] = lam;
        h.type_rec[4 * (size_t)t + 2] = first;
        h.type_rec[4 * (size_t)t + 3] = last;
        h.type_cl[t] = cl_start - k_first;
        h.max_clusters = std::max(h.max_clusters, prev_k - k_first + 1);
        if ((int64_t)h.cl.size() >= INT32_MAX) return fail(EAT_ERR_INVALID, "too many clusters");
    }
    // distinct (u, v) pairs
    for (int32_t u = 0; u < V; ++u) {
        std::vector<int32_t> heads(in->type_v + in->row_ptr[u], in->type_v + in->row_ptr[u + 1]);
        std::sort(heads.begin(), heads.end());
        h.n_edges += (int32_t)(std::unique(heads.begin(), heads.end()) - heads.begin());
    }
    return EAT_OK;
}

// Sub-trips (Section II-G).  A trip of k connections, ordered by departure, is cut
// into consecutive sub-trips of r connections (the last one shorter); r is the
// nearest integer to sqrt(k) (EAT_SUBTRIPS_SQRT_K) or to the square root of the
// mean trip length (EAT_SUBTRIPS_SQRT_MEAN), at least 2.  A sub-trip
// (v_i, v_i+1, t_i, l_i) ... (v_j, v_j+1, t_j, l_j) with i < j yields one artificial
// connection (v_i, v_j+1, t_i, t_j + l_j - t_i): riding the same vehicle, so no
// earliest arrival changes, but a path needs fewer connections.
int add_subtrips(const eat_connections *c, int32_t scheme, std::vector<int32_t> &u,
                 std::vector<int32_t> &v, std::vector<int32_t> &dep, std::vector<int32_t> &dur,
                 int64_t &n_added) {
    n_added = 0;
    const int64_t C = c->n_conn;
    if (scheme != EAT_SUBTRIPS_SQRT_K && scheme != EAT_SUBTRIPS_SQRT_MEAN)
        return fail(EAT_ERR_INVALID, "subtrips must be one of EAT_SUBTRIPS_*");
    if (C > 0 && !c->trip) return fail(EAT_ERR_INVALID, "sub-trips need trip ids (conn->trip)");
    // Group connection indices by trip (counting sort when ids are dense), then by departure.
    int32_t max_trip = -1;
    for (int64_t i = 0; i < C; ++i) max_trip = std::max(max_trip, c->trip[i]);
    std::vector<int64_t> idx;
    std::vector<int64_t> start;
    if (max_trip >= 0 && (int64_t)max_trip <= 4 * C + 1024) {
        std::vector<int64_t> cnt((size_t)max_trip + 2, 0);
        for (int64_t i = 0; i < C; ++i)
            if (c->trip[i] >= 0) ++cnt[(size_t)c->trip[i] + 1];
        for (size_t k = 1; k < cnt.size(); ++k) cnt[k] += cnt[k - 1];
        idx.resize((size_t)cnt.back());
        std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
        for (int64_t i = 0; i < C; ++i)
            if (c->trip[i] >= 0) idx[(size_t)pos[(size_t)c->trip[i]]++] = i;
        start.assign(cnt.begin(), cnt.end());
    } else if (max_trip >= 0) {
        for (int64_t i = 0; i < C; ++i)
            if (c->trip[i] >= 0) idx.push_back(i);
        std::sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) {
            return c->trip[a] < c->trip[b] || (c->trip[a] == c->trip[b] && a < b);
        });
        start.push_back(0);
        for (size_t k = 1; k <= idx.size(); ++k)
            if (k == idx.size() || c->trip[idx[k]] != c->trip[idx[k - 1]]) start.push_back((int64_t)k);
    } else {
        start.push_back(0);
    }
    const size_t n_groups = start.size() - 1;
    int64_t sum_k = 0, n_trips = 0;
    for (size_t g = 0; g < n_groups; ++g) {
        int64_t *b = idx.data() + start[g], *e = idx.data() + start[g + 1];
        if (b == e) continue;
        std::sort(b, e, [&](int64_t x, int64_t y) { return c->dep[x] < c->dep[y]; });
        for (int64_t *p = b + 1; p < e; ++p) {
            const int64_t a = p[-1], z = p[0];
            if (c->v[a] != c->u[z] || (int64_t)c->dep[a] + c->dur[a] > (int64_t)c->dep[z])
                return fail(EAT_ERR_INVALID, "trip " + std::to_string(c->trip[z]) +
                                                 " is not a time-respecting chain of connections");
        }
        sum_k += e - b;
        ++n_trips;
    }
    const int64_t r_mean = n_trips ? std::max<int64_t>(2, (int64_t)std::llround(std::sqrt((double)sum_k / (double)n_trips))) : 2;
    try {
        u.assign(c->u, c->u + C);
        v.assign(c->v, c->v + C);
        dep.assign(c->dep, c->dep + C);
        dur.assign(c->dur, c->dur + C);
        for (size_t g = 0; g < n_groups; ++g) {
            const int64_t *b = idx.data() + start[g];
            const int64_t k = start[g + 1] - start[g];
            if (k < 2) continue;
            const int64_t r = scheme == EAT_SUBTRIPS_SQRT_K
                                  ? std::max<int64_t>(2, (int64_t)std::llround(std::sqrt((double)k)))
                                  : r_mean;
            for (int64_t i = 0; i < k; i += r) {
                const int64_t j = std::min(i + r, k) - 1;
                if (j <= i) continue;
                const int64_t first = b[i], last = b[j];
                u.push_back(c->u[first]);
                v.push_back(c->v[last]);
                dep.push_back(c->dep[first]);
                dur.push_back((int32_t)((int64_t)c->dep[last] + c->dur[last] - c->dep[first]));
                ++n_added;
            }
        }
    } catch (const std::bad_alloc &) {
        return fail(EAT_ERR_OOM, "host allocation for sub-trips failed");
    }
    return EAT_OK;
}

// Device layout (see NetDev in eat_internal.h): one 32-byte entry per (type,
// cluster) for every cluster of the network, self-contained for a relaxation:
// the cluster's first two APs (first terms relative to the cluster start), the
// index and count of its further APs, the first departure of the next non-empty
// cluster, and the type's head stop, duration and head row.  One load of the
// entry answers getConnection for most clusters (Algorithm 6 inside the hourly
// cluster of Section II-D) and gives everything Relax (Algorithm 3) and the
// frontier push need.
int build_fused(HostNet &h) {
    const int32_t T = h.n_types, W = h.width, t0 = h.t0;
    int32_t kmin = INT32_MAX, kmax = INT32_MIN;
    for (int32_t t = 0; t < T; ++t) {
        kmin = std::min(kmin, (h.type_rec[4 * (size_t)t + 2] - t0) / W);
        kmax = std::max(kmax, (h.type_rec[4 * (size_t)t + 3] - t0) / W);
    }
    if (T == 0) kmin = kmax = 0;
    const int64_t Y = (int64_t)kmax - kmin + 1;
    if ((int64_t)T * Y * 32 > ((int64_t)64 << 30))
        return fail(EAT_ERR_INVALID, "cluster table of " + std::to_string(T) + " types x " +
                                         std::to_string(Y) + " clusters is too large; use a wider cluster_width");
    h.k_min = kmin;
    h.y = (int32_t)Y;
    std::vector<int64_t> xoff((size_t)T + 1, 0);
    for (int32_t t = 0; t < T; ++t) {
        const int32_t kf = (h.type_rec[4 * (size_t)t + 2] - t0) / W;
        const int32_t kl = (h.type_rec[4 * (size_t)t + 3] - t0) / W;
        const int32_t b = h.type_cl[t];
        int64_t extra = 0;   // each cluster's list padded to an even length (16-byte aligned)
        for (int32_t k = kf; k <= kl; ++k) {
            const int32_t n = h.cl[b + k + 1] - h.cl[b + k];
            const int32_t m = std::max(0, n - kInlineAps) + (n >= kCountOverflow ? 2 : 0);   // + count header
            extra += m + (m & 1);
        }
        xoff[t + 1] = xoff[t] + extra;
    }
    if (xoff[T] / 2 >= (int64_t)1 << 24)
        return fail(EAT_ERR_INVALID, "more than 2^25 APs beyond the four inline per cluster");
    try {
        h.tr.assign((size_t)T * 4, 0);
        h.ce.assign((size_t)T * (size_t)Y * 8, 0);
        h.apx.resize((size_t)xoff[T] * 2);
    } catch (const std::bad_alloc &) {
        return fail(EAT_ERR_OOM, "host allocation of the cluster table failed");
    }
    auto fill = [&](int32_t t_begin, int32_t t_end) {
        for (int32_t t = t_begin; t < t_end; ++t) {
            const int32_t v = h.type_rec[4 * (size_t)t], lam = h.type_rec[4 * (size_t)t + 1];
            const int32_t vb = h.row_ptr[v], dv = h.row_ptr[v + 1] - vb;
            const int32_t kf = (h.type_rec[4 * (size_t)t + 2] - t0) / W;
            const int32_t kl = (h.type_rec[4 * (size_t)t + 3] - t0) / W;
            const int32_t b = h.type_cl[t];
            int32_t *r = &h.tr[(size_t)t * 4];
            r[0] = v;
            r[1] = (int32_t)((uint32_t)lam | ((uint32_t)std::min(dv, kCountOverflow) << 24));
            r[2] = vb;
            r[3] = h.type_rec[4 * (size_t)t + 3];
            int64_t x = xoff[t];
            for (int32_t kr = 0; kr < Y; ++kr) {
                int32_t *e = &h.ce[((size_t)kr * (size_t)T + (size_t)t) * 8];
                const int32_t k = kmin + kr;
                const int64_t cbase = (int64_t)t0 + (int64_t)k * W;
                int32_t lo = 0, n = 0;
                if (k >= kf && k <= kl) {
                    lo = h.cl[b + k];
                    n = h.cl[b + k + 1] - lo;
                }
                // Inline AP j: start relative to the cluster (16 bits) and sc.
                auto rel = [&](int32_t j) {
                    return n > j ? (uint32_t)((int64_t)h.ap[2 * (size_t)(lo + j)] - cbase) : 0u;
                };
                auto sc = [&](int32_t j) { return n > j ? (int32_t)h.ap[2 * (size_t)(lo + j) + 1] : 0; };
                e[0] = (int32_t)(rel(0) | (rel(1) << 16));
                e[1] = sc(0);
                e[2] = sc(1);
                e[4] = (int32_t)(((uint32_t)(x / 2)) | ((uint32_t)std::min(n, kCountOverflow) << 24));
                e[5] = (int32_t)(rel(2) | (rel(3) << 16));
                e[6] = sc(2);
                e[7] = sc(3);
                int64_t m = 0;
                if (n >= kCountOverflow) {     // count header: two slots, count in the first
                    h.apx[2 * (size_t)x] = (uint32_t)n;
                    h.apx[2 * (size_t)x + 1] = 0u;
                    h.apx[2 * (size_t)(x + 1)] = 0u;
                    h.apx[2 * (size_t)(x + 1) + 1] = 0u;
                    x += 2;
                    m += 2;
                }
                for (int32_t j = kInlineAps; j < n; ++j, ++x, ++m) {
                    h.apx[2 * (size_t)x] = h.ap[2 * (size_t)(lo + j)];
                    h.apx[2 * (size_t)x + 1] = h.ap[2 * (size_t)(lo + j) + 1];
                }
                if (m & 1) {                   // padding entry, never examined
                    h.apx[2 * (size_t)x] = (uint32_t)EAT_INF;
                    h.apx[2 * (size_t)x + 1] = 0u;
                    ++x;
                }
            }
            int32_t next = EAT_INF;
            for (int32_t kr = (int32_t)Y - 1; kr >= 0; --kr) {
                int32_t *e = &h.ce[((size_t)kr * (size_t)T + (size_t)t) * 8];
                e[3] = next;
                if (((uint32_t)e[4] >> 24) > 0)
                    next = (int32_t)(t0 + (int64_t)(kmin + kr) * W + (e[0] & 0xffff));
            }
        }
    };
    unsigned hw = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    const int32_t per = (T + (int32_t)hw - 1) / (int32_t)hw;
    for (unsigned i = 1; i < hw; ++i) {
        const int32_t a = std::min(T, (int32_t)i * per), z = std::min(T, (int32_t)(i + 1) * per);
        if (a < z) th.emplace_back(fill, a, z);
    }
    fill(0, std::min(T, per));
    for (auto &t : th) t.join();
    return EAT_OK;
}

}  // namespace eat

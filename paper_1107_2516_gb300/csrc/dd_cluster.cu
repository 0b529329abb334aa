// Candidate clustering (search variant, host side): the threshold test of
// Section 3 reports every (DM, time, width) point above it, so one pulse
// yields many neighbouring points.  Friends-of-friends grouping: two
// candidates are linked when their DM indices differ by at most dm_link and
// their times by at most t_link (any widths); clusters are the connected
// components.  Candidates are binned into cells of (dm_link+1) x (t_link+1),
// so a candidate's friends lie in its own or the 8 neighbouring cells; links
// are merged with a union-find.  Each cluster reports its strongest member
// (largest S/N; ties: smallest (dm, t, width)) and its DM / time extent.
#include "dd_internal.h"

#include <algorithm>
#include <cstring>
#include <unordered_map>
#include <vector>

namespace {

struct UnionFind {
    std::vector<int64_t> parent;
    explicit UnionFind(int64_t n) : parent((size_t)n) { for (int64_t i = 0; i < n; ++i) parent[(size_t)i] = i; }
    int64_t find(int64_t x)
    {
        while (parent[(size_t)x] != x) {
            parent[(size_t)x] = parent[(size_t)parent[(size_t)x]];
            x = parent[(size_t)x];
        }
        return x;
    }
    void unite(int64_t a, int64_t b)
    {
        a = find(a); b = find(b);
        if (a != b) parent[(size_t)std::max(a, b)] = std::min(a, b);
    }
};

bool before(const dd_candidate &a, const dd_candidate &b)
{
    if (a.dm_idx != b.dm_idx) return a.dm_idx < b.dm_idx;
    if (a.t != b.t) return a.t < b.t;
    return a.width_idx < b.width_idx;
}

}  // namespace

using namespace dd;

extern "C" int dd_cluster_candidates(const dd_candidate *cands, int64_t n, int32_t dm_link, int64_t t_link,
                                     dd_cluster *clusters, int64_t capacity, int64_t *n_clusters,
                                     int64_t *labels)
{
    if (!n_clusters || n < 0 || (n > 0 && !cands)) return set_error(DD_ERR_ARG, "bad cluster arguments");
    if (dm_link < 0 || t_link < 0) return set_error(DD_ERR_ARG, "link lengths must be >= 0");
    if (capacity < 0 || (capacity > 0 && !clusters)) return set_error(DD_ERR_ARG, "bad cluster capacity");
    *n_clusters = 0;
    if (n == 0) return DD_OK;
    const int64_t cd = (int64_t)dm_link + 1, ct = t_link + 1;
    auto cell_of = [&](const dd_candidate &c) {
        const int64_t a = c.dm_idx >= 0 ? c.dm_idx / cd : -((-c.dm_idx + cd - 1) / cd);
        const int64_t b = c.t >= 0 ? c.t / ct : -((-c.t + ct - 1) / ct);
        return std::make_pair(a, b);
    };
    struct Hash {
        size_t operator()(const std::pair<int64_t, int64_t> &p) const
        {
            return std::hash<int64_t>()(p.first * 1000003LL) ^ std::hash<int64_t>()(p.second);
        }
    };
    std::unordered_map<std::pair<int64_t, int64_t>, std::vector<int64_t>, Hash> cells;
    cells.reserve((size_t)n);
    for (int64_t i = 0; i < n; ++i) cells[cell_of(cands[i])].push_back(i);
    UnionFind uf(n);
    for (const auto &kv : cells) {
        const auto &here = kv.second;
        for (int64_t da = -1; da <= 1; ++da)
            for (int64_t db = -1; db <= 1; ++db) {
                const auto it = cells.find(std::make_pair(kv.first.first + da, kv.first.second + db));
                if (it == cells.end()) continue;
                for (int64_t i : here)
                    for (int64_t j : it->second) {
                        if (j <= i) continue;
                        const dd_candidate &a = cands[i], &b = cands[j];
                        if (std::llabs((long long)a.dm_idx - b.dm_idx) <= dm_link && std::llabs((long long)(a.t - b.t)) <= t_link)
                            uf.unite(i, j);
                    }
            }
    }
    // one record per root
    std::vector<int64_t> root_to_cluster((size_t)n, -1);
    std::vector<dd_cluster> out;
    std::vector<int64_t> rep;                       // representative candidate of each cluster
    std::vector<int64_t> lab((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t r = uf.find(i);
        int64_t &k = root_to_cluster[(size_t)r];
        const dd_candidate &c = cands[i];
        if (k < 0) {
            k = (int64_t)out.size();
            dd_cluster z;
            memset(&z, 0, sizeof(z));
            z.dm_lo = z.dm_hi = c.dm_idx;
            z.t_lo = z.t_hi = c.t;
            out.push_back(z);
            rep.push_back(i);
        }
        dd_cluster &z = out[(size_t)k];
        z.n_members++;
        z.dm_lo = std::min(z.dm_lo, c.dm_idx); z.dm_hi = std::max(z.dm_hi, c.dm_idx);
        z.t_lo = std::min(z.t_lo, c.t); z.t_hi = std::max(z.t_hi, c.t);
        const dd_candidate &best = cands[rep[(size_t)k]];
        if (c.snr > best.snr || (c.snr == best.snr && before(c, best))) rep[(size_t)k] = i;
        lab[(size_t)i] = k;
    }
    for (size_t k = 0; k < out.size(); ++k) {
        const dd_candidate &b = cands[rep[k]];
        out[k].dm_idx = b.dm_idx; out[k].width_idx = b.width_idx; out[k].t = b.t; out[k].snr = b.snr;
    }
    // order clusters by their representative's (dm, t, width)
    std::vector<int64_t> order(out.size());
    for (size_t k = 0; k < out.size(); ++k) order[k] = (int64_t)k;
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        return before(cands[rep[(size_t)a]], cands[rep[(size_t)b]]);
    });
    std::vector<int64_t> rank(out.size());
    for (size_t k = 0; k < order.size(); ++k) rank[(size_t)order[k]] = (int64_t)k;
    const int64_t m = (int64_t)out.size();
    for (int64_t k = 0; k < std::min(m, capacity); ++k) clusters[k] = out[(size_t)order[(size_t)k]];
    if (labels)
        for (int64_t i = 0; i < n; ++i) labels[i] = rank[(size_t)lab[(size_t)i]];
    *n_clusters = m;
    if (m > capacity) return set_error(DD_ERR_OVERFLOW, "%lld clusters exceed capacity %lld", (long long)m,
                                       (long long)capacity);
    return DD_OK;
}

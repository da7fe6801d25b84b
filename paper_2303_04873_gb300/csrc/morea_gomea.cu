// Selection and clustering of MO-RV-GOMEA as MOREA uses it (Sec. 3; reading
// R19), host code behind morea_cluster.
//
//   fronts       fast non-dominated sorting: domination counts and lists,
//                then peeling; rank r = non-dominated once ranks < r are
//                removed
//   selection    the ceil(tau n) solutions first in (rank, index) order
//   space        each objective scaled by the selection's range; squared
//                Euclidean distances, summed in axis order
//   leaders      farthest-first traversal from the smallest scaled f_0
//   clusters     balanced k-means: each cluster is the c = min(|S|,
//                ceil(2 |S| / k)) selected solutions nearest to its mean
//                (ties by index), means recomputed as plain member means,
//                until memberships repeat or `iters` rounds
//   assignment   every population member to the nearest mean
//
// This file is compiled without floating-point contraction, so every
// distance and mean is the same sequence of IEEE operations as the plain
// definition.
#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "../../include/morea.h"

namespace {

using P3 = std::vector<double>;

double sqdist(const double *a, const double *b)
{
    const double d0 = a[0] - b[0], d1 = a[1] - b[1], d2 = a[2] - b[2];
    return (d0 * d0 + d1 * d1) + d2 * d2;
}

bool dominates(const double *a, const double *b)
{
    bool strict = false;
    for (int m = 0; m < 3; ++m) {
        if (a[m] > b[m]) return false;
        if (a[m] < b[m]) strict = true;
    }
    return strict;
}

std::vector<int> front_ranks(int n, const double *obj)
{
    std::vector<int> count((size_t)n, 0), rank((size_t)n, -1);
    std::vector<std::vector<int>> dominated((size_t)n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (i != j && dominates(obj + 3 * i, obj + 3 * j)) {
                dominated[i].push_back(j);
                ++count[j];
            }
    std::vector<int> front;
    for (int i = 0; i < n; ++i)
        if (count[i] == 0) front.push_back(i);
    for (int r = 0; !front.empty(); ++r) {
        std::vector<int> next;
        for (int i : front) rank[i] = r;
        for (int i : front)
            for (int j : dominated[i])
                if (--count[j] == 0) next.push_back(j);
        front.swap(next);
    }
    return rank;
}

}  // namespace

extern "C" morea_status morea_cluster(int32_t n, const double *obj, double tau, int32_t k, int32_t iters,
                                      int32_t *n_selected, int32_t *selected, int32_t *cluster_size,
                                      int32_t *members, int32_t *pop_cluster)
{
    if (n < 1 || !obj || !(tau > 0.0 && tau <= 1.0) || k < 1 || iters < 1 || !n_selected || !selected ||
        !cluster_size || !members || !pop_cluster)
        return MOREA_EINVAL;
    for (long long i = 0; i < 3LL * n; ++i)
        if (!std::isfinite(obj[i])) return MOREA_EINVAL;
    // selection
    const std::vector<int> rank = front_ranks(n, obj);
    std::vector<int> order((size_t)n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return rank[a] < rank[b]; });
    const int ns = std::min(n, (int)std::ceil(tau * n));
    std::vector<int> sel(order.begin(), order.begin() + ns);
    // scaled objective space of the selection
    double lo[3], hi[3];
    for (int m = 0; m < 3; ++m) {
        lo[m] = hi[m] = obj[3 * sel[0] + m];
        for (int i : sel) {
            lo[m] = std::min(lo[m], obj[3 * i + m]);
            hi[m] = std::max(hi[m], obj[3 * i + m]);
        }
    }
    auto scaled = [&](int i, double *out) {
        for (int m = 0; m < 3; ++m) {
            const double span = hi[m] - lo[m];
            out[m] = span > 0.0 ? (obj[3 * i + m] - lo[m]) / span : 0.0;
        }
    };
    std::vector<double> pts((size_t)3 * ns);
    for (int s = 0; s < ns; ++s) scaled(sel[s], &pts[3 * s]);
    // leaders: farthest-first traversal
    std::vector<int> lead;
    {
        int first = 0;
        for (int s = 1; s < ns; ++s)
            if (pts[3 * s] < pts[3 * first]) first = s;
        lead.push_back(first);
        std::vector<double> near((size_t)ns);
        for (int s = 0; s < ns; ++s) near[s] = sqdist(&pts[3 * s], &pts[3 * first]);
        while ((int)lead.size() < std::min(k, ns)) {
            int nxt = 0;
            for (int s = 1; s < ns; ++s)
                if (near[s] > near[nxt]) nxt = s;
            lead.push_back(nxt);
            for (int s = 0; s < ns; ++s) near[s] = std::min(near[s], sqdist(&pts[3 * s], &pts[3 * nxt]));
        }
        while ((int)lead.size() < k) lead.push_back(lead[lead.size() % ns]);
    }
    // balanced k-means
    const int c = std::min(ns, (int)std::ceil(2.0 * ns / k));
    std::vector<double> means((size_t)3 * k);
    for (int q = 0; q < k; ++q)
        for (int m = 0; m < 3; ++m) means[3 * q + m] = pts[3 * lead[q] + m];
    std::vector<std::vector<int>> mem, next((size_t)k);
    std::vector<std::pair<double, int>> dist((size_t)ns);
    for (int it = 0; it < iters; ++it) {
        for (int q = 0; q < k; ++q) {
            for (int s = 0; s < ns; ++s) dist[s] = {sqdist(&pts[3 * s], &means[3 * q]), s};
            std::partial_sort(dist.begin(), dist.begin() + c, dist.end());
            next[q].clear();
            for (int j = 0; j < c; ++j) next[q].push_back(dist[j].second);
            std::sort(next[q].begin(), next[q].end());
        }
        if (next == mem) break;
        mem = next;
        for (int q = 0; q < k; ++q) {
            double sum[3] = {0.0, 0.0, 0.0};
            for (int s : mem[q])
                for (int m = 0; m < 3; ++m) sum[m] = sum[m] + pts[3 * s + m];
            for (int m = 0; m < 3; ++m) means[3 * q + m] = sum[m] / (double)mem[q].size();
        }
    }
    // assignment of the whole population
    for (int i = 0; i < n; ++i) {
        double p[3];
        scaled(i, p);
        int best = 0;
        double bd = sqdist(p, &means[0]);
        for (int q = 1; q < k; ++q) {
            const double d = sqdist(p, &means[3 * q]);
            if (d < bd) {
                bd = d;
                best = q;
            }
        }
        pop_cluster[i] = best;
    }
    *n_selected = ns;
    for (int s = 0; s < ns; ++s) selected[s] = sel[s];
    *cluster_size = c;
    for (int q = 0; q < k; ++q)
        for (int j = 0; j < c; ++j) members[(size_t)q * n + j] = sel[mem[q][j]];
    return MOREA_OK;
}

// Linkage model and parallel groups of the partial evaluations (Sec. 4.2.1),
// host code behind morea_parallel_groups: mesh edges as FOS elements, a
// greedy set cover of the points by edges, the interaction graph of the
// chosen edges (shared dependent tets) and its DSATUR colouring.  Elements
// of one colour have disjoint dependent tets, so their partial evaluations
// can run in one batched call on the same solution.
//
// The greedy cover takes, at every step, the first edge in sorted order
// that covers the most uncovered points.  Gains only fall, so this equals
// two passes over the sorted edges: first every edge with both endpoints
// still uncovered, then every edge with one.  DSATUR keeps the uncoloured
// elements in an ordered set keyed by (saturation, degree, index).
#include <algorithm>
#include <set>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/morea.h"

namespace {

struct Key {
    int sat, deg, idx;
    bool operator<(const Key &o) const
    {
        if (sat != o.sat) return sat > o.sat;        // most saturated first
        if (deg != o.deg) return deg > o.deg;        // then the largest degree
        return idx < o.idx;                          // then the lowest index
    }
};

}  // namespace

extern "C" morea_status morea_parallel_groups(int32_t n_points, int32_t n_tets, const int32_t *tets,
                                              int32_t max_elements, int32_t *elements, int32_t *group,
                                              int32_t *n_elements, int32_t *n_groups)
{
    if (n_points < 1 || n_tets < 1 || !tets || max_elements < 1 || !elements || !group || !n_elements || !n_groups)
        return MOREA_EINVAL;
    for (long long i = 0; i < 4LL * n_tets; ++i)
        if (tets[i] < 0 || tets[i] >= n_points) return MOREA_EINVAL;
    // mesh edges, sorted
    std::vector<std::pair<int, int>> edges;
    edges.reserve((size_t)6 * n_tets);
    for (int t = 0; t < n_tets; ++t)
        for (int i = 0; i < 4; ++i)
            for (int j = i + 1; j < 4; ++j) {
                const int a = tets[4 * t + i], b = tets[4 * t + j];
                if (a != b) edges.emplace_back(std::min(a, b), std::max(a, b));
            }
    std::sort(edges.begin(), edges.end());
    edges.erase(std::unique(edges.begin(), edges.end()), edges.end());
    // greedy set cover
    std::vector<char> covered((size_t)n_points, 0);
    std::vector<std::pair<int, int>> el;
    for (int pass = 2; pass >= 1; --pass)
        for (const auto &e : edges) {
            const int gain = !covered[e.first] + !covered[e.second];
            if (gain >= pass) {
                el.push_back(e);
                covered[e.first] = covered[e.second] = 1;
            }
        }
    for (int v = 0; v < n_points; ++v)
        if (!covered[v]) return MOREA_EINVAL;             // a point in no tet
    const int m = (int)el.size();
    if (m > max_elements) return MOREA_EINVAL;
    // elements of each tet -> interaction graph
    std::vector<std::vector<int>> of_point((size_t)n_points);
    for (int i = 0; i < m; ++i) {
        of_point[el[i].first].push_back(i);
        of_point[el[i].second].push_back(i);
    }
    std::vector<std::vector<int>> adj((size_t)m);
    std::vector<int> in_tet;
    for (int t = 0; t < n_tets; ++t) {
        in_tet.clear();
        for (int i = 0; i < 4; ++i)
            for (int e : of_point[tets[4 * t + i]]) in_tet.push_back(e);
        std::sort(in_tet.begin(), in_tet.end());
        in_tet.erase(std::unique(in_tet.begin(), in_tet.end()), in_tet.end());
        for (size_t a = 0; a < in_tet.size(); ++a)
            for (size_t b = a + 1; b < in_tet.size(); ++b) {
                adj[in_tet[a]].push_back(in_tet[b]);
                adj[in_tet[b]].push_back(in_tet[a]);
            }
    }
    for (auto &l : adj) {
        std::sort(l.begin(), l.end());
        l.erase(std::unique(l.begin(), l.end()), l.end());
    }
    // DSATUR
    std::vector<int> color((size_t)m, -1), sat((size_t)m, 0);
    std::vector<std::vector<int>> seen((size_t)m);     // colours among a node's coloured neighbours
    std::set<Key> queue;
    for (int i = 0; i < m; ++i) queue.insert(Key{0, (int)adj[i].size(), i});
    int colors = 0;
    while (!queue.empty()) {
        const Key k = *queue.begin();
        queue.erase(queue.begin());
        const int v = k.idx;
        std::vector<int> used;
        for (int u : adj[v])
            if (color[u] >= 0) used.push_back(color[u]);
        std::sort(used.begin(), used.end());
        int c = 0;
        for (int x : used) {
            if (x == c) ++c;
            else if (x > c) break;
        }
        color[v] = c;
        colors = std::max(colors, c + 1);
        for (int u : adj[v]) {
            if (color[u] >= 0) continue;
            auto &s = seen[u];
            if (std::find(s.begin(), s.end(), c) != s.end()) continue;
            queue.erase(Key{sat[u], (int)adj[u].size(), u});
            s.push_back(c);
            sat[u] += 1;
            queue.insert(Key{sat[u], (int)adj[u].size(), u});
        }
    }
    for (int i = 0; i < m; ++i) {
        elements[2 * i] = el[i].first;
        elements[2 * i + 1] = el[i].second;
        group[i] = color[i];
    }
    *n_elements = m;
    *n_groups = colors;
    return MOREA_OK;
}

// Search for a node involution phi under which a graph is symmetric
// (Definition 2: l_ij = l_phi(i)phi(j), self-loops included), Sec. V-F.
//
// The number of involutions T(n) grows faster than any polynomial, so an
// exhaustive search is out of reach; the paper gives two ways to cut it:
//   * degree-list pruning: i and phi(i) must have equal degrees.  Here the
//     test is strengthened by colour refinement -- a node's colour starts as
//     (l_ii, multiset of its off-diagonal weights) and is refined by the
//     multiset of (weight, neighbour colour) until stable; phi can only pair
//     nodes of equal colour, because phi maps every colour class onto itself;
//   * identical branches of trees: in a tree, symmetry means pairs of
//     identical subtrees with a common or adjacent root.  The tree is rooted
//     at its centre; every rooted subtree gets a canonical label (its root's
//     l_ii and the sorted (edge weight, child label) list); siblings with
//     equal (weight, label) are swapped two by two, whole subtree onto whole
//     subtree, and the search continues inside the unpaired ones.  With two
//     centres, two identical halves are swapped.  O(n log n) up to hashing.
// General graphs use a depth-first search over the colour classes (each node
// either paired with an unassigned node of its colour or fixed), checking
// every new pair against the nodes already placed, and keeping the
// involution with the most pairs (branch and bound on the pairs still
// possible, within a step budget).  Both methods return a valid involution;
// the identity when none is found.
#include <algorithm>
#include <cmath>
#include <functional>
#include <map>
#include <numeric>
#include <vector>

#include "gft_internal.h"

namespace gft {
namespace {

constexpr double kSearchTol = 1e-12;   // x max(1, max|L|): equal weights

struct Graph {
    int n;
    const double* L;
    double tol;
    double at(int i, int j) const { return L[(size_t)i * n + j]; }
    bool eq(double a, double b) const { return std::fabs(a - b) <= tol; }
};

// quantise a weight so that equal-within-tolerance values compare equal
long long qkey(double v, double tol) { return (long long)std::llround(v / (tol * 16.0)); }

std::vector<int> refine_colours(const Graph& g, const std::vector<int>& classes) {
    const int n = g.n;
    std::vector<int> col(n);
    {
        std::map<std::vector<long long>, int> ids;
        for (int i = 0; i < n; ++i) {
            std::vector<long long> key{classes[i], qkey(g.at(i, i), g.tol)};
            std::vector<long long> w;
            for (int j = 0; j < n; ++j)
                if (j != i && !g.eq(g.at(i, j), 0.0)) w.push_back(qkey(g.at(i, j), g.tol));
            std::sort(w.begin(), w.end());
            key.insert(key.end(), w.begin(), w.end());
            col[i] = ids.emplace(key, (int)ids.size()).first->second;
        }
    }
    for (int round = 0; round < n; ++round) {
        std::map<std::vector<long long>, int> ids;
        std::vector<int> next(n);
        for (int i = 0; i < n; ++i) {
            std::vector<long long> key{col[i]};
            std::vector<std::pair<long long, long long>> nb;
            for (int j = 0; j < n; ++j)
                if (j != i && !g.eq(g.at(i, j), 0.0)) nb.push_back({qkey(g.at(i, j), g.tol), col[j]});
            std::sort(nb.begin(), nb.end());
            for (auto& e : nb) {
                key.push_back(e.first);
                key.push_back(e.second);
            }
            next[i] = ids.emplace(key, (int)ids.size()).first->second;
        }
        const int before = *std::max_element(col.begin(), col.end()) + 1;
        const int after = (int)ids.size();
        col = next;
        if (after == before) break;
    }
    return col;
}

bool is_tree(const Graph& g) {
    const int n = g.n;
    long long edges = 0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (!g.eq(g.at(i, j), 0.0)) ++edges;
    if (edges != n - 1) return false;
    std::vector<int> seen(n, 0), stack{0};
    seen[0] = 1;
    int cnt = 1;
    while (!stack.empty()) {
        const int v = stack.back();
        stack.pop_back();
        for (int u = 0; u < n; ++u)
            if (u != v && !seen[u] && !g.eq(g.at(v, u), 0.0)) {
                seen[u] = 1;
                ++cnt;
                stack.push_back(u);
            }
    }
    return cnt == n;
}

// Identical branches of a tree (classes take part in the labels, so only
// nodes of equal class are paired).
void tree_search(const Graph& g, const std::vector<int>& classes, std::vector<int>& phi) {
    const int n = g.n;
    std::vector<std::vector<int>> adj(n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (j != i && !g.eq(g.at(i, j), 0.0)) adj[i].push_back(j);
    // centre(s): repeatedly strip leaves
    std::vector<int> deg(n), layer, centres;
    for (int i = 0; i < n; ++i) deg[i] = (int)adj[i].size();
    std::vector<int> removed(n, 0);
    int left = n;
    for (int i = 0; i < n; ++i)
        if (deg[i] <= 1) layer.push_back(i);
    while (left > 2) {
        std::vector<int> next;
        for (int v : layer) {
            removed[v] = 1;
            --left;
            for (int u : adj[v])
                if (!removed[u] && --deg[u] == 1) next.push_back(u);
        }
        layer = next;
    }
    for (int i = 0; i < n; ++i)
        if (!removed[i]) centres.push_back(i);
    // canonical labels of rooted subtrees (root = the first centre; with two
    // centres the second is a child of the first)
    const int root = centres[0];
    std::vector<int> parent(n, -1), order;
    {
        std::vector<int> stack{root};
        parent[root] = root;
        while (!stack.empty()) {
            const int v = stack.back();
            stack.pop_back();
            order.push_back(v);
            for (int u : adj[v])
                if (parent[u] < 0) {
                    parent[u] = v;
                    stack.push_back(u);
                }
        }
    }
    std::vector<int> label(n);
    std::map<std::vector<long long>, int> ids;
    auto child_key = [&](int c) { return std::make_pair(qkey(g.at(parent[c], c), g.tol), (long long)label[c]); };
    std::vector<std::vector<int>> kids(n);
    for (int v : order)
        if (v != root) kids[parent[v]].push_back(v);
    for (auto it = order.rbegin(); it != order.rend(); ++it) {
        const int v = *it;
        std::sort(kids[v].begin(), kids[v].end(), [&](int a, int b) { return child_key(a) < child_key(b); });
        std::vector<long long> key{classes[v], qkey(g.at(v, v), g.tol)};
        for (int c : kids[v]) {
            auto k = child_key(c);
            key.push_back(k.first);
            key.push_back(k.second);
        }
        label[v] = ids.emplace(key, (int)ids.size()).first->second;
    }
    // map the subtree of a onto the identical subtree of b
    std::function<void(int, int)> map_onto = [&](int a, int b) {
        phi[a] = b;
        phi[b] = a;
        for (size_t t = 0; t < kids[a].size(); ++t) map_onto(kids[a][t], kids[b][t]);
    };
    // pair identical sibling branches, recurse into the unpaired ones
    std::function<void(int)> visit = [&](int v) {
        const auto& ks = kids[v];
        size_t s = 0;
        while (s < ks.size()) {
            size_t e = s + 1;
            while (e < ks.size() && child_key(ks[e]) == child_key(ks[s])) ++e;
            size_t t = s;
            for (; t + 1 < e; t += 2) map_onto(ks[t], ks[t + 1]);
            if (t < e) visit(ks[t]);
            s = e;
        }
    };
    if (centres.size() == 2) {
        // bicentral: the two halves hang from the centre edge; swap them when identical
        const int c2 = centres[1];
        // relabel the half of c2 as if it were a root: its label without its parent's side
        std::vector<long long> k1{classes[root], qkey(g.at(root, root), g.tol)}, k2{classes[c2], qkey(g.at(c2, c2), g.tol)};
        for (int c : kids[root])
            if (c != c2) {
                auto k = child_key(c);
                k1.push_back(k.first);
                k1.push_back(k.second);
            }
        for (int c : kids[c2]) {
            auto k = child_key(c);
            k2.push_back(k.first);
            k2.push_back(k.second);
        }
        if (k1 == k2) {
            std::vector<int> r1;
            for (int c : kids[root])
                if (c != c2) r1.push_back(c);
            phi[root] = c2;
            phi[c2] = root;
            for (size_t t = 0; t < r1.size(); ++t) map_onto(r1[t], kids[c2][t]);
            return;
        }
    }
    visit(root);
}

struct Dfs {
    const Graph& g;
    const std::vector<int>& col;
    std::vector<int> order, phi, best;
    int best_pairs = 0, pairs = 0;
    long long steps = 0, budget;
    Dfs(const Graph& g_, const std::vector<int>& c, long long b) : g(g_), col(c), budget(b) {}

    bool consistent(int i, int j) const {
        // phi(i) = j, phi(j) = i against every placed node k (i, j included)
        for (int k : order) {
            const int pk = phi[k];
            if (pk < 0) continue;
            if (!g.eq(g.at(i, k), g.at(j, pk)) || !g.eq(g.at(j, k), g.at(i, pk))) return false;
        }
        return g.eq(g.at(i, i), g.at(j, j)) && g.eq(g.at(i, j), g.at(j, i));
    }
    void run(size_t pos, int unassigned) {
        if (++steps > budget) return;
        if (pairs + unassigned / 2 <= best_pairs) return;   // cannot beat the best
        while (pos < order.size() && phi[order[pos]] >= 0) ++pos;
        if (pos == order.size()) {
            if (pairs > best_pairs) {
                best_pairs = pairs;
                best = phi;
            }
            return;
        }
        const int i = order[pos];
        for (size_t q = pos + 1; q < order.size(); ++q) {
            const int j = order[q];
            if (phi[j] >= 0 || col[j] != col[i]) continue;
            phi[i] = j;
            phi[j] = i;
            if (consistent(i, j)) {
                ++pairs;
                run(pos + 1, unassigned - 2);
                --pairs;
            }
            phi[i] = phi[j] = -1;
            if (steps > budget) return;
        }
        phi[i] = i;
        if (consistent(i, i)) run(pos + 1, unassigned - 1);
        phi[i] = -1;
    }
};

}  // namespace

int find_involution(int n, const double* L, const int* classes_in, long long max_steps, double scale, int* phi_out) {
    if (scale <= 0.0) {
        double mx = 0.0;
        for (size_t e = 0; e < (size_t)n * n; ++e) mx = std::max(mx, std::fabs(L[e]));
        scale = std::max(1.0, mx);
    }
    Graph g{n, L, kSearchTol * scale};
    std::vector<int> classes(n, 0);
    if (classes_in) classes.assign(classes_in, classes_in + n);
    std::vector<int> phi(n);
    std::iota(phi.begin(), phi.end(), 0);
    if (n >= 2 && is_tree(g)) {
        tree_search(g, classes, phi);
    } else if (n >= 2) {
        const std::vector<int> col = refine_colours(g, classes);
        Dfs d(g, col, max_steps);
        // colour classes smallest first: the most constrained choices early
        std::vector<int> size(n, 0);
        for (int c : col) ++size[c];
        d.order.resize(n);
        std::iota(d.order.begin(), d.order.end(), 0);
        std::stable_sort(d.order.begin(), d.order.end(), [&](int a, int b) {
            return size[col[a]] != size[col[b]] ? size[col[a]] < size[col[b]] : col[a] < col[b];
        });
        d.phi.assign(n, -1);
        d.best = phi;
        d.run(0, n);
        phi = d.best;
    }
    int pairs = 0;
    for (int i = 0; i < n; ++i) {
        phi_out[i] = phi[i];
        if (phi[i] > i) ++pairs;
    }
    return pairs;
}

// Stages for a plan: stage s searches every current block (the leaves after
// stages 0..s-1) for an involution, pairing only nodes that took part in the
// same number of earlier stages (so the 1/sqrt2 factors fold exactly), and
// lifts the blocks' involutions to the original labels.  Stops when no
// block has a symmetry left or after max_stages.
int search_stages(int n, const double* L, int max_stages, long long max_steps, std::vector<int>& phis) {
    double mx = 0.0;
    for (size_t e = 0; e < (size_t)n * n; ++e) mx = std::max(mx, std::fabs(L[e]));
    const double scale = std::max(1.0, mx);
    phis.clear();
    int s = 0;
    for (; s < max_stages; ++s) {
        gft_plan_s p;
        p.n = n;
        p.flags = GFT_ANALYZE_ONLY;
        analyze(p, L, s, s ? phis.data() : nullptr);
        std::vector<int> phi(n);
        std::iota(phi.begin(), phi.end(), 0);
        bool found = false;
        for (const Leaf& b : p.leaves) {
            const int m = b.m();
            if (m < 2) continue;
            std::vector<int> local(m);
            if (find_involution(m, b.L.data(), b.exps.data(), max_steps, scale, local.data()) > 0) {
                found = true;
                for (int i = 0; i < m; ++i) phi[b.labels[i]] = b.labels[local[i]];
            }
        }
        if (!found) break;
        phis.insert(phis.end(), phi.begin(), phi.end());
    }
    return s;
}

}  // namespace gft

// Approximate GFT by layers of Givens rotations, alone or after the Haar
// stages of the symmetric decomposition ("Haar + approximate GFT", Sec. VI-B).
//
// The paper compares its exact fast GFTs with the approximate fast GFT of Le
// Magoarou et al. (parallel truncated Jacobi) and with the combination in
// which that approximation replaces the dense sub-GFTs U+ / U- of the leaves.
// Build (host, FP64, compiled without FMA contraction so that x86 and Arm
// hosts produce the same rotations):
//   1. the Haar stages and leaf Laplacians exactly as a plan (Sec. IV);
//   2. per leaf, J layers: every layer pairs nodes greedily by the magnitude
//      of the current off-diagonal entries (largest first, ties by (p, q);
//      entries <= 1e-14 max(1, max|L_k|) count as zero) and applies, at once,
//      the rotations J(p, q, theta) that zero them (symmetric 2x2 Schur):
//      A <- J_t^T A J_t;
//   3. the output order: ascending diagonal of the final A (the approximate
//      eigenvalues), clusters by (leaf, index).
// The transform is a list of 2x2 units in layers -- Haar units
// [[1, 1], [1, -1]] / sqrt2, then the rotations J^T = [[c, -s], [s, c]] of
// every leaf, layer t of all leaves side by side -- and the permutation;
// approx.cu applies it to batches.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "gft_internal.h"

namespace gft {

namespace {

constexpr double kApproxZeroTol = 1e-14;

struct Rot {
    int p, q;
    double c, s;
};

// (c, s) with [[c, s], [-s, c]]^T [[app, apq], [apq, aqq]] [[c, s], [-s, c]]
// diagonal (Golub & Van Loan's symmetric Schur decomposition); the smaller
// root t of t^2 + 2 tau t - 1 = 0 keeps the rotation angle within pi/4.
void sym_schur2(double app, double aqq, double apq, double& c, double& s) {
    if (apq == 0.0) {
        c = 1.0;
        s = 0.0;
        return;
    }
    const double tau = (aqq - app) / (2.0 * apq);
    const double t = tau >= 0.0 ? 1.0 / (tau + std::hypot(1.0, tau)) : -1.0 / (-tau + std::hypot(1.0, tau));
    c = 1.0 / std::sqrt(1.0 + t * t);
    s = t * c;
}

// J greedy layers on the m x m matrix A (row-major, updated in place)
std::vector<std::vector<Rot>> truncated_jacobi(std::vector<double>& A, int m, int n_layers) {
    double mx = 0.0;
    for (double v : A) mx = std::max(mx, std::fabs(v));
    const double tol = kApproxZeroTol * std::max(1.0, mx);
    std::vector<std::vector<Rot>> layers;
    struct Cand {
        double a;
        int p, q;
    };
    std::vector<Cand> cand;
    std::vector<char> used(m);
    for (int t = 0; t < n_layers; ++t) {
        cand.clear();
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) {
                const double v = std::fabs(A[(size_t)p * m + q]);
                if (v > tol) cand.push_back({v, p, q});
            }
        std::sort(cand.begin(), cand.end(), [](const Cand& x, const Cand& y) {
            if (x.a != y.a) return x.a > y.a;
            return x.p != y.p ? x.p < y.p : x.q < y.q;
        });
        std::fill(used.begin(), used.end(), 0);
        std::vector<Rot> rots;
        for (const Cand& cd : cand)
            if (!used[cd.p] && !used[cd.q]) {
                used[cd.p] = used[cd.q] = 1;
                Rot r{cd.p, cd.q, 1.0, 0.0};
                sym_schur2(A[(size_t)cd.p * m + cd.p], A[(size_t)cd.q * m + cd.q], A[(size_t)cd.p * m + cd.q], r.c, r.s);
                rots.push_back(r);
            }
        if (rots.empty()) break;
        for (const Rot& r : rots)   // columns: A <- A J
            for (int i = 0; i < m; ++i) {
                const double ap = A[(size_t)i * m + r.p], aq = A[(size_t)i * m + r.q];
                A[(size_t)i * m + r.p] = r.c * ap - r.s * aq;
                A[(size_t)i * m + r.q] = r.s * ap + r.c * aq;
            }
        for (const Rot& r : rots)   // rows: A <- J^T A
            for (int j = 0; j < m; ++j) {
                const double ap = A[(size_t)r.p * m + j], aq = A[(size_t)r.q * m + j];
                A[(size_t)r.p * m + j] = r.c * ap - r.s * aq;
                A[(size_t)r.q * m + j] = r.s * ap + r.c * aq;
            }
        for (const Rot& r : rots) A[(size_t)r.p * m + r.q] = A[(size_t)r.q * m + r.p] = 0.0;
        layers.push_back(std::move(rots));
    }
    return layers;
}

}  // namespace

void approx_build(gft_approx_s& a, const double* L, int n_stages, const int32_t* phi, int n_layers, uint32_t flags) {
    gft_plan_s p;
    p.n = a.n;
    p.flags = flags & GFT_SPLIT_COMPONENTS;
    analyze(p, L, n_stages, phi);
    a.n_stages = n_stages;
    a.layer_off.assign(1, 0);
    a.pairs.clear();
    a.coef.clear();
    const double r = 1.0 / std::sqrt(2.0);
    for (auto& st : p.stages) {   // Eq. 20 per stage: (a+b)/sqrt2 at X, (a-b)/sqrt2 at the partner
        for (auto& pr : st) {
            a.pairs.insert(a.pairs.end(), {pr.first, pr.second});
            a.coef.insert(a.coef.end(), {r, r, r, -r});
        }
        a.layer_off.push_back((int)a.pairs.size() / 2);
    }
    a.n_haar_layers = (int)a.layer_off.size() - 1;
    std::vector<std::vector<std::vector<Rot>>> per_leaf;
    std::vector<double> lam_e;
    std::vector<int> leaf_e, local_e, slot_e;
    size_t depth = 0;
    for (size_t k = 0; k < p.leaves.size(); ++k) {
        Leaf& lf = p.leaves[k];
        const int m = lf.m();
        std::vector<double> A = lf.L;
        per_leaf.push_back(truncated_jacobi(A, m, n_layers));
        depth = std::max(depth, per_leaf.back().size());
        for (int i = 0; i < m; ++i) {
            lam_e.push_back(A[(size_t)i * m + i]);
            leaf_e.push_back((int)k);
            local_e.push_back(i);
            slot_e.push_back(lf.labels[i]);
        }
    }
    for (size_t t = 0; t < depth; ++t) {   // layer t of every leaf, side by side
        for (size_t k = 0; k < per_leaf.size(); ++k) {
            if (t >= per_leaf[k].size()) continue;
            const auto& lab = p.leaves[k].labels;
            for (const Rot& rt : per_leaf[k][t]) {
                a.pairs.insert(a.pairs.end(), {lab[rt.p], lab[rt.q]});
                a.coef.insert(a.coef.end(), {rt.c, -rt.s, rt.s, rt.c});
            }
        }
        a.layer_off.push_back((int)a.pairs.size() / 2);
    }
    const std::vector<int> pos = output_positions(lam_e, leaf_e, local_e);
    a.perm.assign(a.n, 0);
    a.lam.assign(a.n, 0.0);
    for (size_t i = 0; i < pos.size(); ++i) {
        a.perm[pos[i]] = slot_e[i];
        a.lam[pos[i]] = lam_e[i];
    }
}

}  // namespace gft

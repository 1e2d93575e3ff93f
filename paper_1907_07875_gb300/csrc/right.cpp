// Bipartite plans with a right Haar stage (Sec. III-A, Lemma 1, Thms. 1-2).
//
// With the two parts S1, S2 of a bipartite graph (every edge joins them) and
// a Laplacian whose part blocks are alpha I (the combinatorial Laplacian of
// a k-regular bipartite graph: alpha = k; the normalised Laplacian of any
// bipartite graph: alpha = 1), L = alpha I - [[0, C], [C^T, 0]] with the
// coupling block C = -L[S1, S2].  A singular triple C f = sigma e,
// C^T e = sigma f gives the eigenvectors (e; f)/sqrt2 (alpha - sigma) and
// (e; -f)/sqrt2 (alpha + sigma), and the left singular vectors beyond the
// smaller part's size are eigenvectors (e; 0) with eigenvalue alpha.  The
// GFT is therefore U^T x = B_{n,p} diag(E^T, F^T) x (Eq. 8): two dense
// sub-transforms on the parts, then p Haar units on their outputs, p = the
// smaller part's size.
//
// The plan keeps E (on the larger part) and F as its two leaves; the kernels
// run them like any leaf (in place on the parts' slots) and then apply the
// right Haar units to the slot pairs (E's column c, F's column c), with the
// 1/sqrt2 folded into both columns.  E, F and sigma come from the
// eigendecomposition of the symmetric coupling matrix J = [[0, C], [C^T, 0]]
// (the batched FP64 Jacobi on the device, like every leaf): its eigenvalues
// are +-sigma and its eigenvectors (e; +-f)/sqrt2, so the positive ones give
// the paired columns without squaring C; the near-zero ones span the two
// null spaces, which are separated by pivoted Gram-Schmidt on their parts.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "gft_internal.h"

namespace gft {

namespace {

constexpr double kStructTol = 1e-12;    // alpha I blocks and zero within-part entries, x max(1, max|L|)
constexpr double kZeroSigma = 1e-9;     // singular values treated as zero, x max(1, max sigma)
constexpr double kMinResidual = 1e-6;   // pivoted Gram-Schmidt gives up below this residual

double dot(const double* a, const double* b, int m) {
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += a[i] * b[i];
    return s;
}

// Orthonormal columns: `basis` holds k vectors of length m (each contiguous).
// Adds `want` more from the span of `cand` (vectors of length m), each time
// the candidate with the largest residual after projecting out the basis
// (two projection passes for orthogonality to rounding).
void extend_basis(std::vector<std::vector<double>>& basis, std::vector<std::vector<double>> cand, int m, int want,
                  const char* what) {
    for (auto& c : cand)
        for (int pass = 0; pass < 2; ++pass)
            for (auto& b : basis) {
                const double t = dot(c.data(), b.data(), m);
                for (int i = 0; i < m; ++i) c[i] -= t * b[i];
            }
    for (int got = 0; got < want; ++got) {
        int best = -1;
        double bn = 0.0;
        for (size_t j = 0; j < cand.size(); ++j) {
            const double nr = std::sqrt(dot(cand[j].data(), cand[j].data(), m));
            if (nr > bn) {
                bn = nr;
                best = (int)j;
            }
        }
        if (best < 0 || bn < kMinResidual)
            fail(GFT_ERR_NO_CONVERGENCE, std::string("could not separate the null space of the coupling block (") + what +
                                             ")");
        std::vector<double> v = cand[best];
        for (auto& b : basis) {   // second pass against the full basis
            const double t = dot(v.data(), b.data(), m);
            for (int i = 0; i < m; ++i) v[i] -= t * b[i];
        }
        const double nv = std::sqrt(dot(v.data(), v.data(), m));
        for (int i = 0; i < m; ++i) v[i] /= nv;
        cand.erase(cand.begin() + best);
        for (auto& c : cand) {
            const double t = dot(c.data(), v.data(), m);
            for (int i = 0; i < m; ++i) c[i] -= t * v[i];
        }
        basis.push_back(std::move(v));
    }
}

// Modified Gram-Schmidt over the columns in order (a cleanup pass: the
// columns are orthonormal to a few ulps already).
void reorthonormalise(std::vector<std::vector<double>>& cols, int m) {
    for (size_t c = 0; c < cols.size(); ++c) {
        for (size_t d = 0; d < c; ++d) {
            const double t = dot(cols[c].data(), cols[d].data(), m);
            for (int i = 0; i < m; ++i) cols[c][i] -= t * cols[d][i];
        }
        const double nc = std::sqrt(dot(cols[c].data(), cols[c].data(), m));
        for (int i = 0; i < m; ++i) cols[c][i] /= nc;
    }
}

}  // namespace

void analyze_bipartite(gft_plan_s& p, const double* Lin, const int32_t* side_in, Leaf& coupling) {
    const int n = p.n;
    p.L.assign(Lin, Lin + (size_t)n * n);
    double mx = 0.0;
    for (double v : p.L) {
        if (!std::isfinite(v)) fail(GFT_ERR_NOT_LAPLACIAN, "L has a non-finite entry");
        mx = std::max(mx, std::fabs(v));
    }
    const double tol = kStructTol * std::max(1.0, mx);
    auto Lij = [&](int i, int j) { return p.L[(size_t)i * n + j]; };
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (std::fabs(Lij(i, j) - Lij(j, i)) > tol)
                fail(GFT_ERR_NOT_LAPLACIAN, "L is not symmetric at (" + std::to_string(i) + "," + std::to_string(j) + ")");
    // parts: given, or a two-colouring of the nonzero off-diagonal pattern
    // (each connected component gives colour 0 to its smallest node)
    std::vector<int> side(n, -1);
    if (side_in) {
        for (int i = 0; i < n; ++i) {
            if (side_in[i] != 0 && side_in[i] != 1) fail(GFT_ERR_INVALID_ARG, "side entries must be 0 or 1");
            side[i] = side_in[i];
        }
    } else {
        for (int r = 0; r < n; ++r) {
            if (side[r] >= 0) continue;
            side[r] = 0;
            std::vector<int> queue{r};
            for (size_t h = 0; h < queue.size(); ++h) {
                const int v = queue[h];
                for (int u = 0; u < n; ++u) {
                    if (u == v || std::fabs(Lij(v, u)) <= tol) continue;
                    if (side[u] < 0) {
                        side[u] = 1 - side[v];
                        queue.push_back(u);
                    } else if (side[u] == side[v]) {
                        fail(GFT_ERR_NOT_BIPARTITE, "graph is not bipartite (odd cycle through nodes " +
                                                        std::to_string(u) + " and " + std::to_string(v) + ")");
                    }
                }
            }
        }
    }
    const double alpha = Lij(0, 0);
    for (int i = 0; i < n; ++i) {
        if (std::fabs(Lij(i, i) - alpha) > tol)
            fail(GFT_ERR_NOT_BIPARTITE, "diagonal entry " + std::to_string(i) + " differs from l_00 (the part blocks "
                                        "must be alpha I)");
        for (int j = 0; j < n; ++j)
            if (j != i && side[j] == side[i] && std::fabs(Lij(i, j)) > tol)
                fail(GFT_ERR_NOT_BIPARTITE, "entry (" + std::to_string(i) + "," + std::to_string(j) +
                                                ") joins two nodes of one part");
    }
    std::vector<int> S[2];
    for (int i = 0; i < n; ++i) S[side[i]].push_back(i);
    const int big = S[0].size() >= S[1].size() ? 0 : 1;
    const std::vector<int>& A = S[big];
    const std::vector<int>& B = S[1 - big];
    const int m1 = (int)A.size(), m2 = (int)B.size();
    p.right = true;
    p.alpha = alpha;
    p.n_stages = 0;
    p.stages.clear();
    p.leaves.clear();
    Leaf E, F;
    E.labels = A;
    E.exps.assign(m1, 0);
    E.cexps.assign(m1, 0);
    for (int c = 0; c < m2; ++c) E.cexps[c] = 1;
    E.tag = "E";
    p.leaves.push_back(std::move(E));
    if (m2 > 0) {
        F.labels = B;
        F.exps.assign(m2, 0);
        F.cexps.assign(m2, 1);
        F.tag = "F";
        p.leaves.push_back(std::move(F));
    }
    p.rpairs.clear();
    for (int c = 0; c < m2; ++c) p.rpairs.push_back({A[c], B[c]});
    // J = [[0, C], [C^T, 0]], C = -L[A, B], in the order (A, B)
    coupling = Leaf{};
    coupling.labels = A;
    coupling.labels.insert(coupling.labels.end(), B.begin(), B.end());
    coupling.exps.assign(n, 0);
    coupling.L.assign((size_t)n * n, 0.0);
    for (int a = 0; a < m1; ++a)
        for (int b = 0; b < m2; ++b) {
            const double c = -Lij(A[a], B[b]);
            coupling.L[(size_t)a * n + (m1 + b)] = c;
            coupling.L[(size_t)(m1 + b) * n + a] = c;
        }
    coupling.tag = "J";
}

void finish_bipartite(gft_plan_s& p, const Leaf& J) {
    const int n = p.n;
    Leaf& E = p.leaves[0];
    const int m1 = E.m();
    const int m2 = n - m1;
    double smax = 0.0;
    for (double v : J.lam) smax = std::max(smax, std::fabs(v));
    const double zt = kZeroSigma * std::max(1.0, smax);
    int r = 0;   // positive singular values: the r largest eigenvalues of J
    while (r < m2 && J.lam[n - 1 - r] > zt) ++r;
    auto Jv = [&](int row, int col) { return J.V[(size_t)row * n + col]; };
    std::vector<std::vector<double>> ecols, fcols;
    std::vector<double> sigma(m2, 0.0);
    for (int c = 0; c < r; ++c) {
        const int idx = n - 1 - c;
        std::vector<double> e(m1), f(m2);
        for (int a = 0; a < m1; ++a) e[a] = Jv(a, idx);
        for (int b = 0; b < m2; ++b) f[b] = Jv(m1 + b, idx);
        const double ne = std::sqrt(dot(e.data(), e.data(), m1)), nf = std::sqrt(dot(f.data(), f.data(), m2));
        if (ne < 0.5 || nf < 0.5)
            fail(GFT_ERR_NO_CONVERGENCE, "coupling eigenvector " + std::to_string(c) + " does not split into (e; f)");
        for (double& v : e) v /= ne;
        for (double& v : f) v /= nf;
        ecols.push_back(std::move(e));
        fcols.push_back(std::move(f));
        sigma[c] = J.lam[idx];
    }
    // the other eigenvectors (all but the r largest and the r smallest) span
    // null(C^T) on the larger part plus null(C) on the smaller one
    std::vector<std::vector<double>> ca, cb;
    for (int idx = r; idx < n - r; ++idx) {
        std::vector<double> a(m1), b(m2);
        for (int q = 0; q < m1; ++q) a[q] = Jv(q, idx);
        for (int q = 0; q < m2; ++q) b[q] = Jv(m1 + q, idx);
        ca.push_back(std::move(a));
        cb.push_back(std::move(b));
    }
    extend_basis(ecols, ca, m1, m1 - r, "larger part");
    if (m2 > 0) extend_basis(fcols, cb, m2, m2 - r, "smaller part");
    reorthonormalise(ecols, m1);
    reorthonormalise(fcols, m2);
    E.V.assign((size_t)m1 * m1, 0.0);
    E.lam.assign(m1, p.alpha);
    for (int c = 0; c < m1; ++c)
        for (int a = 0; a < m1; ++a) E.V[(size_t)a * m1 + c] = ecols[c][a];
    for (int c = 0; c < m2; ++c) E.lam[c] = p.alpha - sigma[c];
    E.sweeps = J.sweeps;
    if (m2 > 0) {
        Leaf& F = p.leaves[1];
        F.V.assign((size_t)m2 * m2, 0.0);
        F.lam.assign(m2, p.alpha);
        for (int c = 0; c < m2; ++c) {
            for (int b = 0; b < m2; ++b) F.V[(size_t)b * m2 + c] = fcols[c][b];
            F.lam[c] = p.alpha + sigma[c];
        }
        F.sweeps = J.sweeps;
    }
}

}  // namespace gft
